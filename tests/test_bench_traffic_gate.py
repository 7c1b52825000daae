"""bench.py reports the committed full-size DRAM traffic of the dominant
kernel only while that kernel's source is the one the capture measured
(its sha256 prefix is recorded beside the figure)."""

import hashlib

import bench


def _summary(path, digest, traffic="123456"):
    path.write_text("# capture\n\nkernel_source: csrc/k.cu sha256[:16] = " + digest + "\n"
                    + ("traffic_bytes_per_launch: " + traffic + "\n" if traffic is not None else ""))


def test_traffic_while_source_unchanged(tmp_path):
    src = tmp_path / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    summ = tmp_path / "t.md"
    _summary(summ, hashlib.sha256(src.read_bytes()).hexdigest()[:16])
    assert bench._recorded_traffic(str(src), str(summ)) == 123456
    src.write_bytes(b"__global__ void k() { }\n")  # any edit invalidates the figure
    assert bench._recorded_traffic(str(src), str(summ)) is None


def test_traffic_missing_or_malformed(tmp_path):
    src = tmp_path / "k.cu"
    src.write_bytes(b"x")
    digest = hashlib.sha256(b"x").hexdigest()[:16]
    summ = tmp_path / "t.md"
    _summary(summ, digest, traffic=None)
    assert bench._recorded_traffic(str(src), str(summ)) is None
    _summary(summ, digest, traffic="n/a")
    assert bench._recorded_traffic(str(src), str(summ)) is None
    assert bench._recorded_traffic(str(src), str(tmp_path / "absent.md")) is None


def test_committed_summary_is_readable():
    # the committed summary parses; it gives a figure exactly when the
    # committed kernel source is the captured one
    v = bench._recorded_traffic()
    assert v is None or v > 0
