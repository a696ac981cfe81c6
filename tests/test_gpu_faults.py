"""Failure paths of the library on the GPU, made without a GPU fault.

* A numeric fault: a shell whose power is set (mg_set_pk) so large that its
  draw coefficient sd = sqrt(S tau / (S + tau)) overflows gives that shell a
  non-finite sum in the next sweep.  The shell draw keeps the shell's P and
  sets the numeric status bit; the host reports MG_ENUMERIC, which stays
  sticky, and every other shell and chain holds a valid P.
* A failing CUDA call, faked on the host (mg_inject_cuda_error): the library
  call that meets it returns MG_ECUDA, sticky on that context only.
"""
import ctypes

import numpy as np
import pytest

import mockgen

from gpu_helpers import gpu_sampler, need_gpu

pytestmark = pytest.mark.gpu


def _raw_read_pk(g, chain, B1):
    from paper_1402_1763_gb300 import library
    buf = np.full(B1, np.nan)
    st = library().mg_read_pk(g.ctx, chain, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, buf


@pytest.mark.parametrize("precision", [64, 32])
def test_numeric_fault_holds_the_shell_and_is_sticky(precision):
    need_gpu()
    from paper_1402_1763_gb300 import MG_ENUMERIC, MgError, Sampler, library
    n, nb = 16, 8
    L = float(n)          # M / V = 1: S_hat = P
    rng = np.random.default_rng(5)
    R = np.ones((n, n, n))
    N = np.full((n, n, n), 4.0)  # tau = 4, so S_hat tau overflows for S_hat > 4.5e307
    d = rng.standard_normal((n, n, n))
    with Sampler.single(n, L, N, R, d, nb, 5, precision=precision, n_chains=2) as g:
        g.sweep(3)
        P1 = g.read_pk(1)
        bad = g.read_pk(0)
        bad[3] = 1e308
        g.set_pk(0, bad)           # finite, accepted; its coefficients overflow
        g.sweep(1)                  # shell 3 of chain 0 meets a non-finite sum
        st, P0 = _raw_read_pk(g, 0, nb + 1)
        assert st == MG_ENUMERIC
        assert P0[3] == 1e308       # the faulty shell kept its P
        others = np.delete(P0, 3)
        assert np.all(np.isfinite(others)) and np.all(others > 0)
        assert np.any(others != np.delete(bad, 3))  # the healthy shells were drawn
        st1, Pc1 = _raw_read_pk(g, 1, nb + 1)
        assert st1 == MG_ENUMERIC   # sticky on the context
        assert np.all(np.isfinite(Pc1)) and np.all(Pc1 > 0) and np.any(Pc1 != P1)
        assert library().mg_sweep(g.ctx, 1) == MG_ENUMERIC  # nothing more runs
        st2, P0b = _raw_read_pk(g, 0, nb + 1)
        assert st2 == MG_ENUMERIC
        np.testing.assert_array_equal(P0b, P0)
        with pytest.raises(MgError) as e:
            g.sync()
        assert e.value.status == MG_ENUMERIC and "non-finite" in str(e.value)


@pytest.mark.parametrize("after", [1, 3])
def test_injected_cuda_error_is_sticky_on_its_context_only(after):
    need_gpu()
    from paper_1402_1763_gb300 import MG_ECUDA, MgError, library, mg_inject_cuda_error
    n, nb = 32, 16
    m = mockgen.make_mock(n, seed=1, n_bins=nb)
    with gpu_sampler(m, nb, 1, 32, n_chains=2) as g, gpu_sampler(m, nb, 1, 32, n_chains=2) as h:
        g.sweep(2)
        h.sweep(2)
        ref = h.read_pk(0)
        mg_inject_cuda_error(g.ctx, after)
        statuses = []
        for _ in range(after + 1):  # read_pk makes at least two checked calls
            st, _ = _raw_read_pk(g, 0, nb + 1)
            statuses.append(st)
            if st != 0:
                break
        assert statuses[-1] == MG_ECUDA
        assert "injected" in library().mg_last_error(g.ctx).decode()
        assert library().mg_sweep(g.ctx, 1) == MG_ECUDA
        with pytest.raises(MgError) as e:
            g.read_s(0)
        assert e.value.status == MG_ECUDA
        # the other context is unaffected
        np.testing.assert_array_equal(h.read_pk(0), ref)
        h.sweep(1)
        assert np.all(np.isfinite(h.read_pk(0)))
