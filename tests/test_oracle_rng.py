"""Pins of the oracle's counter-based random numbers (Philox4x32-10, Box-Muller).

The method draws its Wiener increments per particle and step (Sec. 2.1: Ito
SDEs integrated forward in time); the build reads this as one Philox4x32-10
call per particle-step (Salmon et al. 2011) keyed by (seed, set) with counter
(step, particle id, tag, 0).
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert O.philox(ctr, key) == out


def test_philox_matches_triton_interpreter():
    """Triton's own Philox4x32-10 (run by its CPU interpreter) is an independent implementation."""
    pytest.importorskip("triton")
    import subprocess
    import sys
    code = r"""
import os
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out_ptr, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    a, b, c, d = tl.randint4x(seed, offs, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)
out = torch.zeros(64, dtype=torch.int32)
k[(1,)](out, 987654321, 16)
print(" ".join(str(int(x) & 0xFFFFFFFF) for x in out.tolist()))
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-200:])
    got = [int(t) for t in r.stdout.split()]
    for i in range(16):
        # triton: counter (offset, 0, 0, 0), key (seed low 32 bits, seed high 32 bits)
        assert O.philox([i, 0, 0, 0], [987654321, 0]) == got[4 * i:4 * i + 4]


def test_uniforms_open_interval_and_exact():
    u = O.uniforms(0, 0, 0, 0, 0)
    x = O.philox([0, 0, 0, 0], [0, 0])
    for ui, xi in zip(u, x):
        assert ui == ((xi >> 8) + 0.5) / 2 ** 24
        assert 0.0 < ui < 1.0


def test_counter_layout_step_id_tag():
    # step n, particle id, tag and set enter the counter / key as documented
    assert O.uniforms(7, 3, 11, 5, 0) == [((x >> 8) + 0.5) / 2 ** 24
                                          for x in O.philox([11, 5, 0, 0], [7, 3])]
    assert O.uniforms(7, 3, 0, 5, 1) == [((x >> 8) + 0.5) / 2 ** 24
                                         for x in O.philox([0, 5, 1, 0], [7, 3])]


def test_box_muller_definition():
    u = O.uniforms(1, 0, 42, 9, 0)
    z = O.normals(1, 0, 42, 9)
    a = math.sqrt(-2 * math.log(u[0]))
    assert z[0] == pytest.approx(a * math.cos(2 * math.pi * u[1]), rel=1e-15)
    assert z[1] == pytest.approx(a * math.sin(2 * math.pi * u[1]), rel=1e-15)
    assert z[2] == pytest.approx(math.sqrt(-2 * math.log(u[2])) * math.cos(2 * math.pi * u[3]),
                                 rel=1e-15)


def test_normals_are_standard_normal():
    zs = np.array([O.normals(0, 0, n, i) for n in range(40) for i in range(500)])
    for k in range(3):
        s = zs[:, k]
        assert abs(s.mean()) < 4 / math.sqrt(len(s))
        assert abs(s.var() - 1) < 5 * math.sqrt(2 / len(s))
        assert stats.kstest(s, "norm").pvalue > 1e-3
    # the three normals of one draw are uncorrelated
    c = np.corrcoef(zs.T)
    assert np.all(np.abs(c - np.eye(3)) < 4 / math.sqrt(len(zs)))
