"""mg_shell_sums_noalloc: the shell sums of a spectrum for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI:
  * against the oracle's shell table (oracle.bins: shell ids, dof weights and
    full-grid mode counts) with a plain numpy sum of w |s_hat|^2, on two calls
    in a row, at a grid the sampler runs (32^3, 16 shells), at grids it does not
    (20^3 and 200^3) and at the largest shell count the scratch holds (254);
  * against the shell sums the sampler's own sweep reports (mg_read_stats)
    for the unitary transform of the chain's current field;
  * two calls on the same input give the same bits, and a warmed call leaves
    the device's free memory unchanged.
The sums are FP64 on both sides (FP32 inputs convert exactly), so every
comparison uses the FP64 parity bar 1e-12.  This file is collected last and
also passes on its own.
"""
import numpy as np
import pytest

import mockgen
from oracle.bins import make_bins

from gpu_helpers import TOL, gpu_sampler, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def oracle_shell_sums(s_hat, n, nb):
    """sigma_b = sum over shell b of w |s_hat|^2 and n_b, from the oracle's table."""
    bins = make_bins((n, n, n), (1000.0,) * 3, nb)
    keep = bins.bin_of >= 0
    a2 = (s_hat.real.astype(np.float64) ** 2 + s_hat.imag.astype(np.float64) ** 2)
    sig = np.bincount(bins.bin_of[keep], weights=(bins.weight * a2)[keep], minlength=nb + 1)
    return sig, bins.n_b.astype(np.float64)


@pytest.mark.parametrize("n,nb,precision,with_nmodes", [(32, 16, 64, True), (32, 16, 32, True),
                                                         (20, 254, 64, False), (200, 254, 32, False)])
def test_noalloc_matches_the_oracle_shell_table(n, nb, precision, with_nmodes):
    torch = need_gpu()
    from paper_1402_1763_gb300 import mg_shell_sums_noalloc
    rng = np.random.default_rng(1000 + n + nb)
    shape = (n, n, n // 2 + 1)
    ctype = np.complex128 if precision == 64 else np.complex64
    s_hat = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(ctype)
    ref_sig, ref_nb = oracle_shell_sums(s_hat, n, nb)
    dev = torch.from_numpy(s_hat).cuda()
    sigma = torch.empty(nb + 1, dtype=torch.float64, device="cuda")
    nmodes = torch.empty(nb + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    got = []
    for _ in range(2):
        sigma.fill_(-1.0)
        nmodes.fill_(-1.0)
        mg_shell_sums_noalloc(dev.data_ptr(), precision, n, nb, sigma.data_ptr(),
                              nmodes.data_ptr() if with_nmodes else 0, stream)
        torch.cuda.synchronize()
        got.append(sigma.cpu().numpy().copy())
        assert rel_l2(got[-1], ref_sig) <= TOL[64]
        if with_nmodes:
            np.testing.assert_array_equal(nmodes.cpu().numpy(), ref_nb)
        else:
            assert np.all(nmodes.cpu().numpy() == -1.0)  # NULL: left untouched
    np.testing.assert_array_equal(got[0], got[1])  # same bits on a repeat


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_shell_sums_match_the_sweep(precision):
    torch = need_gpu()
    from paper_1402_1763_gb300 import mg_shell_sums_noalloc
    n, nb = 32, 16
    m = mockgen.make_mock(n, seed=17, n_bins=nb)
    ctype = torch.complex128 if precision == 64 else torch.complex64
    rtype = torch.float64 if precision == 64 else torch.float32
    sigma = torch.empty(nb + 1, dtype=torch.float64, device="cuda")
    nmodes = torch.empty(nb + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with gpu_sampler(m, nb, 17, precision) as g:
        for _ in range(2):
            g.sweep(1)
            st = g.read_stats(0)
            s = torch.tensor(g.read_s(0), dtype=rtype, device="cuda")
            s_hat = (torch.fft.rfftn(s) / np.sqrt(n ** 3)).to(ctype).contiguous()
            sigma.fill_(-1.0)
            mg_shell_sums_noalloc(s_hat.data_ptr(), precision, n, nb, sigma.data_ptr(), nmodes.data_ptr(), stream)
            torch.cuda.synchronize()
            assert rel_l2(sigma.cpu().numpy(), st["sigma_b"]) <= TOL[precision]
            np.testing.assert_array_equal(nmodes.cpu().numpy(), st["n_b"].astype(np.float64))


def test_noalloc_allocates_nothing_and_rejects_oversized_requests():
    torch = need_gpu()
    from paper_1402_1763_gb300 import MG_EINVAL, MgError, mg_shell_sums_noalloc
    n, nb = 64, 32
    s_hat = torch.randn(n, n, n // 2 + 1, dtype=torch.complex64, device="cuda")
    sigma = torch.empty(nb + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    mg_shell_sums_noalloc(s_hat.data_ptr(), 32, n, nb, sigma.data_ptr(), 0, stream)  # warm
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    mg_shell_sums_noalloc(s_hat.data_ptr(), 32, n, nb, sigma.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    with pytest.raises(MgError) as e:
        mg_shell_sums_noalloc(s_hat.data_ptr(), 32, n, 255, sigma.data_ptr(), 0, stream)
    assert e.value.status == MG_EINVAL and "255 shells" in str(e.value)
    with pytest.raises(MgError) as e:
        mg_shell_sums_noalloc(s_hat.data_ptr(), 32, 4098, 8, sigma.data_ptr(), 0, stream)
    assert e.value.status == MG_EINVAL and "4096" in str(e.value)
