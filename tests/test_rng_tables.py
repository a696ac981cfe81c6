"""The tables of the FP64 Box-Muller path (paper_1402_1763_gb300/csrc/
mg_rng_tables.h) against Python's math library, which shares nothing with the
decimal arithmetic that made them, and the header against its generator.

* hi(ln F) + lo(ln F) = ln(1 + j/128) and 1/F within an ulp; hi(ln F) and
  ln2_hi on the 2^-44 grid the exact first sum relies on.
* sin and cos of 2 pi j/256 within an ulp (absolute, of 1).
* ln2_hi + ln2_lo = ln 2 and 2 pi 2^-33 exactly as math's 2 pi scaled.
* Re-running the generator reproduces the header byte for byte.
"""
import math
import os
import re
import shutil
import subprocess
import sys

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1402_1763_gb300", "csrc")


def tables():
    src = open(os.path.join(CSRC, "mg_rng_tables.h")).read()
    body = lambda name: src.split(name)[1].split("};")[0]
    pairs = lambda txt: [(float.fromhex(a), float.fromhex(b))
                         for a, b in re.findall(r"\{(-?0x[0-9a-fp.+-]+), (-?0x[0-9a-fp.+-]+)\}", txt)]
    ln = pairs(body("kLnTab128[128] = {"))
    lo = [float.fromhex(x.strip().rstrip(",")) for x in body("kLnLo128[128] = {").strip().splitlines()]
    sc = pairs(body("kSinCos256[256] = {"))
    const = {k: float.fromhex(v) for k, v in re.findall(r"constexpr double (\w+) = (\S+);", src)}
    return ln, lo, sc, const


def test_log_table():
    ln, lo, _, const = tables()
    assert len(ln) == 128 and len(lo) == 128
    for j, ((hi, inv), l) in enumerate(zip(ln, lo)):
        F = 1.0 + j / 128.0
        assert abs((hi + l) - math.log(F)) <= math.ulp(math.log(F)) if j else hi == 0.0 and l == 0.0
        assert abs(inv - 1.0 / F) <= 0.5 * math.ulp(1.0 / F)
        assert hi * 2.0 ** 44 == round(hi * 2.0 ** 44) and abs(l) <= 2.0 ** -45
    assert const["kLn2Hi"] * 2.0 ** 44 == round(const["kLn2Hi"] * 2.0 ** 44)
    assert abs(const["kLn2Hi"] + const["kLn2Lo"] - math.log(2.0)) <= math.ulp(math.log(2.0))


def sincos_ref(j):
    """sin, cos of 2 pi j/256 from math's sin and cos at pi i/128 <= pi/4
    (quadrant and octant symmetries taken in integers, so the argument math
    sees is off by at most half an ulp)."""
    q, r = divmod(j, 64)
    if r <= 32:
        a = math.pi * r / 128.0
        s0, c0 = math.sin(a), math.cos(a)
    else:
        a = math.pi * (64 - r) / 128.0
        s0, c0 = math.cos(a), math.sin(a)
    return [(s0, c0), (c0, -s0), (-s0, -c0), (-c0, s0)][q]


def test_sincos_table_and_angle_scale():
    _, _, sc, const = tables()
    assert len(sc) == 256
    for j, (s, c) in enumerate(sc):
        rs, rc = sincos_ref(j)
        assert abs(s - rs) <= 2.0 ** -53 and abs(c - rc) <= 2.0 ** -53, j
    assert sc[0] == (0.0, 1.0) and abs(sc[64][1]) < 1e-30
    assert const["kTwoPi2m33"] == 2.0 * math.pi * 2.0 ** -33


def test_header_matches_generator(tmp_path):
    shutil.copy(os.path.join(CSRC, "gen_rng_tables.py"), tmp_path)
    subprocess.run([sys.executable, "gen_rng_tables.py"], cwd=tmp_path, check=True)
    assert (tmp_path / "mg_rng_tables.h").read_text() == open(os.path.join(CSRC, "mg_rng_tables.h")).read()
