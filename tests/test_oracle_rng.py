"""Pins of the oracle's Philox4x32-10 and Box-Muller normals.

Philox is checked against PyTorch's header-only engine (an implementation that
shares nothing with ours), compiled here with g++, on counters that exercise
every word and the carry-free high bits.  The normals are checked against the
standard normal law (moments and a Kolmogorov-Smirnov test) and at the edges of
the uniform mapping.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.stats as st

from oracle import philox as ph

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def torch_ref(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    exe = str(tmp_path_factory.mktemp("tpr") / "tpr")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I" + inc,
                    os.path.join(HERE, "helpers", "torch_philox_ref.cpp"), "-o", exe],
                   check=True, capture_output=True)
    return exe


def test_philox_matches_independent_engine(torch_ref):
    rng = np.random.default_rng(7)
    rows = []
    for _ in range(300):
        seed = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        c = [int(x) for x in rng.integers(0, 2 ** 32, size=4)]
        rows.append((seed, *c))
    rows += [(0, 0, 0, 0, 0), (2 ** 64 - 1, 2 ** 32 - 1, 2 ** 32 - 1, 2 ** 32 - 1, 2 ** 32 - 1),
             (1, 5, 3, 7, 1), (12345, 0, 1999, 15, 0)]
    inp = "\n".join(" ".join(str(v) for v in r) for r in rows) + "\n"
    out = subprocess.run([torch_ref], input=inp, capture_output=True, text=True, check=True)
    ref = np.array([[int(v) for v in line.split()] for line in out.stdout.strip().splitlines()],
                   dtype=np.uint64)
    for r, want in zip(rows, ref):
        got = ph.philox4x32_10(r[1], r[2], r[3], r[4], r[0])
        assert [int(g) for g in got] == [int(w) for w in want], r


def test_philox_vectorised_equals_scalar():
    idx = np.arange(50, dtype=np.uint64)
    vec = ph.philox4x32_10(idx, 3, 9, 1, 42)
    for i in range(50):
        sc = ph.philox4x32_10(i, 3, 9, 1, 42)
        assert all(int(vec[q][i]) == int(sc[q]) for q in range(4))


def test_uniform_mapping_edges():
    u = ph.uniform_open0(np.array([0, 2 ** 32 - 1], dtype=np.uint64))
    assert u[0] == 2.0 ** -33
    assert u[1] == 1.0 - 2.0 ** -33
    assert np.float32(u[1]) == np.float32(1.0)


def test_box_muller_is_standard_normal():
    idx = np.arange(1 << 19, dtype=np.uint64)
    z = np.concatenate(ph.normals4(idx, 0, 0, 1, 2024))
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2.0 / n)
    assert abs(st.skew(z)) < 5 * np.sqrt(6.0 / n)
    assert abs(st.kurtosis(z)) < 5 * np.sqrt(24.0 / n)
    assert st.kstest(z, "norm").pvalue > 1e-4


def test_box_muller_pairs_are_independent():
    idx = np.arange(1 << 18, dtype=np.uint64)
    z0, z1, z2, z3 = ph.normals4(idx, 1, 2, 0, 99)
    n = z0.size
    for a, b in ((z0, z1), (z0, z2), (z1, z3), (z2, z3)):
        assert abs(np.mean(a * b)) < 5 / np.sqrt(n)
    # the radius is shared by a pair: z0^2 + z1^2 ~ chi^2_2 (exponential, mean 2)
    assert st.kstest(z0 ** 2 + z1 ** 2, "chi2", args=(2,)).pvalue > 1e-4
