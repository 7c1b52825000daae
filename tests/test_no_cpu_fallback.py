"""The product path has no CPU fallback: without the built library, or
without a GPU, every call raises instead of computing anything on the
host."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _py(code):
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)


def test_missing_library_raises():
    r = _py("from paper_1212_4779_gb300 import sg\n"
            "sg._LIB_PATH = '/nonexistent/libsg.so'\n"
            "try:\n"
            "    sg.lib()\n"
            "    print('LOADED')\n"
            "except sg.SGError as e:\n"
            "    print('RAISED', e.status, 'not built' in str(e))\n")
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["RAISED", "3", "True"]


def test_no_gpu_raises():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible; this checks the host without one")
    r = _py("import numpy as np\n"
            "from paper_1212_4779_gb300 import sg\n"
            "try:\n"
            "    sg.Graph.from_coo(3, np.array([0, 1], dtype=np.int32), np.array([1, 2], dtype=np.int32))\n"
            "    print('COMPUTED')\n"
            "except sg.SGError as e:\n"
            "    print('RAISED', e.status)\n")
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["RAISED", "3"]
