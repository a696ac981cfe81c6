"""mg_shell_sums_noalloc: the shell sums of a spectrum for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the shell sums the sampler's own sweep
reports (mg_read_stats, sigma_b and n_b), on two calls in a row: the spectrum
passed in is the unitary transform of the chain's current field (mg_read_s),
which is the sample whose shell sums the sweep just formed.  Tolerances are
the parity bars of the other GPU tests (relative L2 1e-12 in FP64, 2e-5 in
FP32).  This file is collected last and also passes on its own.
"""
import numpy as np
import pytest

import mockgen

from gpu_helpers import TOL, gpu_sampler, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_shell_sums_match_the_sweep(precision):
    torch = need_gpu()
    from paper_1402_1763_gb300 import MG_EINVAL, MgError, mg_shell_sums_noalloc
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
    with pytest.raises(MgError) as e:
        mg_shell_sums_noalloc(s_hat.data_ptr(), precision, n, 255, sigma.data_ptr(), 0, stream)
    assert e.value.status == MG_EINVAL and "255 shells" in str(e.value)
