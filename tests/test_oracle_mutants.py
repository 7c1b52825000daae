"""The oracle pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a wrong
shift, a transposed operand, a dropped term, a flipped comparison), builds
that copy on the CPU, and runs the pin suite against it in a subprocess;
the suite must fail.  Nothing here touches a GPU."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sg_oracle.c")

MUTANTS = {
    "mix_shift": ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;",
                  "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;"),
    "snapshot_shift": ("uint64_t x = seed ^ ((uint64_t)r << 40) ^ e;",
                       "uint64_t x = seed ^ ((uint64_t)r << 32) ^ e;"),
    "coin_direction": ("return hi < thr;", "return hi > thr;"),
    "uic_scale": ("uint64_t t = (uint64_t)floor(p * 4294967296.0);",
                  "uint64_t t = (uint64_t)floor(p * 2147483648.0);"),
    "wic_outdegree": ("for (int64_t e = 0; e < m; e++) thr[e] = (1ULL << 32) / (uint64_t)indeg[col[e]];",
                      "for (int64_t u = 0; u < n; u++) for (int64_t e = rp[u]; e < rp[u + 1]; e++)"
                      " thr[e] = (1ULL << 32) / (uint64_t)(rp[u + 1] - rp[u]);"),
    "tie_highest_id": ("if (best < 0 || s[v] > s[best]) best = (int32_t)v;",
                       "if (best < 0 || s[v] >= s[best]) best = (int32_t)v;"),
    "no_self_count": ("                    acc += reach_count(S, r, rp, 1, &vv, NULL, &w, &edges);",
                      "                    acc += reach_count(S, r, rp, 1, &vv, NULL, &w, &edges) - 1;"),
    "du_no_decrement": ("                        s[u] -= 1;\n", "\n"),
    "du_reverse_uses_out_lists": ("const int64_t *irp = S->in_rp[r];\n                const int32_t *icol = S->in_col[r];",
                                  "const int64_t *irp = S->out_rp[r];\n                const int32_t *icol = S->out_col[r];"),
    "keep_duplicates": ("if (i == 0 || key[i] != key[i - 1]) key[m++] = key[i];", "key[m++] = key[i];"),
    "gain_literal_no_base": ("gains[i] = (mode == OR_LITERAL) ? s[vs] - f_S : s[vs];", "gains[i] = s[vs];"),
    "fwd_counter_indeg": ("c_fwd += (uint64_t)(rp[u + 1] - rp[u]);", "c_fwd += (uint64_t)indeg[u];"),
    "celf_accepts_stale_bound": ("if (stamp == i) { s[v] = b; vs = v; break; }",
                                 "if (stamp <= i) { s[v] = b; vs = v; break; }"),
    "coupled_higher_arc_id": ("cid[e] = e < lo ? e : lo;", "cid[e] = e > lo ? e : lo;"),
    "masks_last_word_unmasked": ("if (r < R && arc_live(seed, (uint32_t)r, e, thr, cid, lo)) word |= 1ULL << b;",
                                 "if (arc_live(seed, (uint32_t)r, e, thr, cid, lo)) word |= 1ULL << b;"),
    "masks_bit_reversed": ("if (r < R && arc_live(seed, (uint32_t)r, e, thr, cid, lo)) word |= 1ULL << b;",
                           "if (r < R && arc_live(seed, (uint32_t)r, e, thr, cid, lo)) word |= 1ULL << (63 - b);"),
    "lt_hashes_source": ("            key[e] = v;\n", "            key[e] = u;\n"),
    "lt_overlapping_intervals": ("hi[e] = (uint64_t)(j + 1) * w;", "hi[e] = (uint64_t)(j + 2) * w;"),
    "celf_ties_to_highest_id": ("return h->b[x] > h->b[y] || (h->b[x] == h->b[y] && h->v[x] < h->v[y]);",
                                "return h->b[x] > h->b[y] || (h->b[x] == h->b[y] && h->v[x] > h->v[y]);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut_c = tmp_path / "mut.c"
    mut_c.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", str(so), str(mut_c), "-lm"],
                   check=True)
    env = dict(os.environ, SG_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
