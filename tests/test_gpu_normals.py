"""The unit normals the kernels make from Philox words (mg_normals) against
references in 40-digit decimal arithmetic: z0 = sqrt(-2 ln U_a) cos(2 pi U_b),
z1 = sqrt(-2 ln U_a) sin(2 pi U_b) and -2 ln U_a with U(w) = (2w + 1) 2^-33
(Box & Muller 1958).

* FP64 (the table-driven logarithm, sine and cosine): -2 ln U within 2 ulp,
  z0, z1 within 4 ulp of max(r, 1) absolute (r the pair's radius).
* FP32 (the special-function unit on U rounded to FP32), within the bounds of
  that construction: U carries a relative error up to 2^-23 (w rounded to 24
  bits, then the fused scale-and-offset), so -2 ln U is off by up to
  B = 2^-21 (1 + r^2) (with the hardware logarithm's relative error); the
  radius r by min(sqrt(B), B / (2r)) (sqrt is 1/2-Hoelder) plus its own
  rounding; the angle by 2 pi 2^-23 plus the hardware sine's 2^-21.4.
Words: random, plus the smallest and largest, powers of two and their
neighbours (the logarithm's octaves and table points) and multiples of 2^24
(the angle table's points).
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu

getcontext().prec = 40
PI = Decimal("3.141592653589793238462643383279502884197")


def sin_cos(a: Decimal):
    a = a - 2 * PI if a > PI else a
    s, c, term, k = Decimal(0), Decimal(0), Decimal(1), 0
    while abs(term) > Decimal(10) ** -42:
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        k += 1
        term = term * a / k
    return s, c


def reference(wa, wb):
    out = np.empty((len(wa), 3))
    for i, (a, b) in enumerate(zip(wa, wb)):
        ua = Decimal(2 * int(a) + 1) / Decimal(2) ** 33
        ub = Decimal(2 * int(b) + 1) / Decimal(2) ** 33
        r2 = -2 * ua.ln()
        r = r2.sqrt()
        s, c = sin_cos(2 * PI * ub)
        out[i] = [float(r * c), float(r * s), float(r2)]
    return out


def words():
    rng = np.random.default_rng(12)
    edge = [0, 1, 2, 3, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1]
    edge += [2 ** k for k in range(32)] + [2 ** k - 1 for k in range(1, 33)] + [2 ** k + 1 for k in range(1, 32)]
    edge += [(j << 24) for j in range(256)] + [(j << 24) - 1 for j in range(1, 256)]
    edge += [2 ** 32 - 1 - int(x) for x in rng.integers(0, 2 ** 14, 200)]
    wa = np.array(edge + [int(x) for x in rng.integers(0, 2 ** 32, 3000)], dtype=np.uint64)
    wb = np.concatenate([rng.integers(0, 2 ** 32, len(edge)), rng.integers(0, 2 ** 32, 3000)]).astype(np.uint64)
    # every edge word also as the angle word
    wa = np.concatenate([wa, rng.integers(0, 2 ** 32, len(edge)).astype(np.uint64)])
    wb = np.concatenate([wb, np.array(edge, dtype=np.uint64)])
    return wa.astype(np.uint32), wb.astype(np.uint32)


def gpu_normals(precision, wa, wb):
    import torch
    from paper_1402_1763_gb300 import mg_normals
    w = torch.from_numpy(np.stack([wa, wb], axis=1).reshape(-1).view(np.int32).copy()).cuda()
    out = torch.empty(3 * len(wa), dtype=torch.float64 if precision == 64 else torch.float32, device="cuda")
    mg_normals(precision, w.data_ptr(), len(wa), out.data_ptr())
    return out.cpu().numpy().astype(np.float64).reshape(-1, 3)


def test_fp64_normals_within_a_few_ulp():
    need_gpu()
    wa, wb = words()
    got = gpu_normals(64, wa, wb)
    ref = reference(wa, wb)
    r = np.sqrt(ref[:, 2])
    ulp = np.spacing(np.maximum(r, 1.0))
    assert np.all(np.abs(got[:, 0] - ref[:, 0]) <= 4 * ulp)
    assert np.all(np.abs(got[:, 1] - ref[:, 1]) <= 4 * ulp)
    assert np.all(np.abs(got[:, 2] - ref[:, 2]) <= 2 * np.spacing(ref[:, 2]))


def test_fp32_normals_within_their_construction():
    need_gpu()
    wa, wb = words()
    got = gpu_normals(32, wa, wb)
    ref = reference(wa, wb)
    r2 = ref[:, 2]
    r = np.sqrt(r2)
    B = 2.0 ** -21 * (1.0 + r2)
    assert np.all(np.abs(got[:, 2] - r2) <= B)
    dr = np.minimum(np.sqrt(B), B / (2.0 * np.maximum(r, 1e-300))) + 2.0 ** -22 * r
    dang = 2.0 * np.pi * 2.0 ** -23 + 2.0 ** -21.4
    bound = dr + r * dang + 1e-7
    assert np.all(np.abs(got[:, 0] - ref[:, 0]) <= bound)
    assert np.all(np.abs(got[:, 1] - ref[:, 1]) <= bound)
    # away from U_a = 1 that is a few 1e-6 absolute
    far = r > 0.1
    assert np.all(np.abs(got[far, :2] - ref[far, :2]) <= 2e-5)


def test_invalid_arguments():
    need_gpu()
    from paper_1402_1763_gb300 import MG_EINVAL, MgError, mg_normals
    for args in ((16, 1, 1, 1), (64, 0, 4, 1), (64, 1, -1, 1)):
        with pytest.raises(MgError) as e:
            mg_normals(*args)
        assert e.value.status == MG_EINVAL
    mg_normals(64, 0, 0, 0)  # nothing to do
