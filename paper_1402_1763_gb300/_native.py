"""ctypes binding of include/mg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ETIMEOUT, MG_ENUMERIC, MG_ESTATE, MG_EUNSUPPORTED, MG_EBOUNDS = range(9)
_NAMES = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ETIMEOUT",
          5: "MG_ENUMERIC", 6: "MG_ESTATE", 7: "MG_EUNSUPPORTED", 8: "MG_EBOUNDS"}
MG_BUILD_CHECKED = 1

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    """The main library, or its bounds-checked build when MG_CHECKED=1."""
    name = "libmg_checked.so" if os.environ.get("MG_CHECKED") == "1" else "libmg.so"
    return os.path.join(_HERE, "_lib", name)


class MgGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("L", C.c_double * 3)]


class MgOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_chains", C.c_int32), ("chain_id0", C.c_int32),
                ("tau_scale", C.c_double), ("P0", C.POINTER(C.c_double)),
                ("record_every", C.c_int32), ("fix_P", C.c_int32),
                ("timeout_cycles", C.c_int64), ("cuda_stream", C.c_void_p),
                ("yz_cluster", C.c_int32), ("persistent", C.c_int32), ("autotune", C.c_int32),
                ("mixing", C.c_int32), ("start_dispersion", C.c_double)]


class MgStats(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("records", C.c_int64), ("tau", C.c_double),
                ("n_bins", C.c_int32), ("n_b", C.POINTER(C.c_int64)),
                ("sigma_b", C.POINTER(C.c_double)), ("chi_b", C.POINTER(C.c_double)),
                ("mean", C.POINTER(C.c_double)), ("var", C.POINTER(C.c_double))]


class MgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def library():
    """Load libmg.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_1402_1763_gb300.build)")
    lib = C.CDLL(path)
    sig = {
        "mg_options_init": (None, [C.POINTER(MgOptions)]),
        "mg_init": (C.c_int, [C.POINTER(_P), C.POINTER(MgGrid), _D, _D, _D, _D, C.c_int32, C.c_uint64,
                              C.POINTER(MgOptions)]),
        "mg_init_batch": (C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(MgGrid), C.POINTER(_D),
                                    C.POINTER(_D), C.POINTER(_D), C.POINTER(_D), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_uint64), C.POINTER(MgOptions)]),
        "mg_sweep": (C.c_int, [_P, C.c_int64]),
        "mg_sweep_timed": (C.c_int, [_P, C.c_int64, _D]),
        "mg_read_s": (C.c_int, [_P, C.c_int32, _P, C.c_int32]),
        "mg_read_pk": (C.c_int, [_P, C.c_int32, _D]),
        "mg_read_stats": (C.c_int, [_P, C.c_int32, C.POINTER(MgStats)]),
        "mg_set_s": (C.c_int, [_P, C.c_int32, _P, C.c_int32]),
        "mg_set_pk": (C.c_int, [_P, C.c_int32, _D]),
        "mg_set_data": (C.c_int, [_P, C.c_int32, _D]),
        "mg_tune": (C.c_int, [_P, C.c_int32]),
        "mg_schedule": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32)]),
        "mg_adjoint": (C.c_int, [_P, C.c_int32, C.c_int32, _D, _D, _D, _D, _D]),
        "mg_get_sweep_count": (C.c_int, [_P, C.POINTER(C.c_int64)]),
        "mg_set_sweep_count": (C.c_int, [_P, C.c_int64]),
        "mg_chain_info": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32)]),
        "mg_sync": (C.c_int, [_P]),
        "mg_last_error": (C.c_char_p, [_P]),
        "mg_destroy": (None, [_P]),
        "mg_philox": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64,
                                _P, _P]),
        "mg_normals": (C.c_int, [C.c_int32, _P, C.c_int64, _P, _P]),
        "mg_shell_sums_noalloc": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P]),
        "mg_read_pk_trace": (C.c_int, [_P, C.c_int32, _D, C.c_int64, C.POINTER(C.c_int64)]),
        "mg_pk_acf": (C.c_int, [_P, C.c_int32, C.c_int32, _D, C.POINTER(C.c_int32)]),
        "mg_pk_quantiles": (C.c_int, [_P, C.c_int32, C.c_int32, _D, _D]),
        "mg_pk_rhat": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int64, _D]),
        "mg_read_pk_all": (C.c_int, [_P, _D]),
        "mg_inject_cuda_error": (C.c_int, [_P, C.c_int32]),
        "mg_build_flags": (C.c_int32, []),
        "mg_fp64_fma_peak": (C.c_int, [_D, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != MG_OK:
        msg = library().mg_last_error(ctx).decode()
        raise MgError(status, msg or "call failed")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, M=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if M is not None and a.size != M:
        raise ValueError(f"expected {M} values, got {a.size}")
    return a


def mg_options_init() -> MgOptions:
    o = MgOptions()
    library().mg_options_init(C.byref(o))
    return o


def _grid(n: int, L: float) -> MgGrid:
    g = MgGrid()
    g.nx = g.ny = g.nz = int(n)
    for i in range(3):
        g.L[i] = float(L)
    return g


def mg_init(n: int, L: float, N, R, d, n_bins: int, seed: int, opt: MgOptions, k_edges=None):
    """Returns the context handle (c_void_p)."""
    M = int(n) ** 3
    Na, Ra, da = _f64(N, M), _f64(R, M), _f64(d, M)
    ea = None if k_edges is None else _f64(k_edges, n_bins + 1)
    ctx = _P()
    g = _grid(n, L)
    st = library().mg_init(C.byref(ctx), C.byref(g), _dptr(Na), _dptr(Ra), _dptr(da),
                           _dptr(ea) if ea is not None else None, int(n_bins), C.c_uint64(seed),
                           C.byref(opt))
    _check(st)
    return ctx


def mg_init_batch(ns: Sequence[int], Ls: Sequence[float], Ns, Rs, ds, n_bins: Sequence[int],
                  seeds: Sequence[int], opt: MgOptions, k_edges=None):
    G = len(ns)
    grids = (MgGrid * G)(*[_grid(n, L) for n, L in zip(ns, Ls)])
    keep = []
    arrs = []
    for lst in (Ns, Rs, ds):
        ptrs = (_D * G)()
        for i in range(G):
            a = _f64(lst[i], int(ns[i]) ** 3)
            keep.append(a)
            ptrs[i] = _dptr(a)
        arrs.append(ptrs)
    eptr = None
    if k_edges is not None:
        eptr = (_D * G)()
        for i in range(G):
            if k_edges[i] is not None:
                a = _f64(k_edges[i], n_bins[i] + 1)
                keep.append(a)
                eptr[i] = _dptr(a)
    nb = (C.c_int32 * G)(*[int(b) for b in n_bins])
    sd = (C.c_uint64 * G)(*[int(s) for s in seeds])
    ctx = _P()
    st = library().mg_init_batch(C.byref(ctx), G, grids, arrs[0], arrs[1], arrs[2], eptr, nb, sd,
                                 C.byref(opt))
    _check(st)
    return ctx


def mg_sweep(ctx, n: int):
    _check(library().mg_sweep(ctx, int(n)), ctx)


def mg_sweep_timed(ctx, n: int) -> np.ndarray:
    """Milliseconds spent in (pass YZ, pass X, shell draw) over n sweeps."""
    ms = np.zeros(3)
    _check(library().mg_sweep_timed(ctx, int(n), _dptr(ms)), ctx)
    return ms


def mg_read_s(ctx, chain: int, out_ptr: int, out_is_device: bool):
    _check(library().mg_read_s(ctx, int(chain), C.c_void_p(out_ptr), int(bool(out_is_device))), ctx)


def mg_read_pk(ctx, chain: int, out: np.ndarray):
    _check(library().mg_read_pk(ctx, int(chain), _dptr(out)), ctx)


def mg_read_pk_trace(ctx, chain: int, out, max_records: int) -> int:
    """Fill out (max_records x (n_bins+1) doubles) with the recorded P(k)
    trace; returns the number of records."""
    n = C.c_int64(0)
    _check(library().mg_read_pk_trace(ctx, int(chain), _dptr(out) if out is not None else None,
                                      int(max_records), C.byref(n)), ctx)
    return int(n.value)


def mg_pk_acf(ctx, chain: int, max_lag: int, acf: np.ndarray, n_c: np.ndarray):
    _check(library().mg_pk_acf(ctx, int(chain), int(max_lag), _dptr(acf),
                               n_c.ctypes.data_as(C.POINTER(C.c_int32))), ctx)


def mg_pk_quantiles(ctx, chain: int, q: np.ndarray, out: np.ndarray):
    _check(library().mg_pk_quantiles(ctx, int(chain), int(q.size), _dptr(q), _dptr(out)), ctx)


def mg_pk_rhat(ctx, first_chain: int, n_chains: int, burn: int, out: np.ndarray):
    _check(library().mg_pk_rhat(ctx, int(first_chain), int(n_chains), int(burn), _dptr(out)), ctx)


def mg_read_pk_all(ctx, out: np.ndarray):
    """out: (n_chains, B_max+1) float64, C-contiguous (pinned host memory for speed)."""
    _check(library().mg_read_pk_all(ctx, _dptr(out)), ctx)


def mg_read_stats(ctx, chain: int, stats: MgStats):
    _check(library().mg_read_stats(ctx, int(chain), C.byref(stats)), ctx)


def mg_set_s(ctx, chain: int, ptr: int, is_device: bool):
    _check(library().mg_set_s(ctx, int(chain), C.c_void_p(ptr), int(bool(is_device))), ctx)


def mg_set_pk(ctx, chain: int, P: np.ndarray):
    _check(library().mg_set_pk(ctx, int(chain), _dptr(P)), ctx)


def mg_set_data(ctx, group: int, d):
    _check(library().mg_set_data(ctx, int(group), _dptr(_f64(d))), ctx)


def mg_adjoint(ctx, chain: int, K: int, logP, w):
    """(L, dL/dlogP, dL/dd) of K fixed-P sweeps; see include/mg.h."""
    lp = _f64(logP)
    wa = _f64(w)
    n = mg_chain_info(ctx, chain)[0]
    if wa.size != n * n * (n // 2 + 1):
        raise ValueError("w must hold n*n*(n/2+1) stored-mode weights")
    L = np.zeros(1)
    gl = np.empty(lp.size)
    gd = np.empty(n ** 3)
    _check(library().mg_adjoint(ctx, int(chain), int(K), _dptr(lp), _dptr(wa), _dptr(L), _dptr(gl),
                                _dptr(gd)), ctx)
    return float(L[0]), gl, gd.reshape(n, n, n)


def mg_tune(ctx, reps: int = 5):
    _check(library().mg_tune(ctx, int(reps)), ctx)


def mg_schedule(ctx) -> dict:
    ns, pers = C.c_int32(), C.c_int32()
    n = (C.c_int32 * 8)()
    cl = (C.c_int32 * 8)()
    _check(library().mg_schedule(ctx, C.byref(ns), n, cl, C.byref(pers)), ctx)
    return {"sizes": [n[i] for i in range(ns.value)], "yz_cluster": [cl[i] for i in range(ns.value)],
            "persistent": bool(pers.value)}


def mg_get_sweep_count(ctx) -> int:
    v = C.c_int64()
    _check(library().mg_get_sweep_count(ctx, C.byref(v)), ctx)
    return int(v.value)


def mg_set_sweep_count(ctx, n: int):
    _check(library().mg_set_sweep_count(ctx, int(n)), ctx)


def mg_chain_info(ctx, chain: int):
    n, nb, nc = C.c_int32(), C.c_int32(), C.c_int32()
    _check(library().mg_chain_info(ctx, int(chain), C.byref(n), C.byref(nb), C.byref(nc)), ctx)
    return n.value, nb.value, nc.value


def mg_sync(ctx):
    _check(library().mg_sync(ctx), ctx)


def mg_last_error(ctx) -> str:
    return library().mg_last_error(ctx).decode()


def mg_destroy(ctx):
    library().mg_destroy(ctx)


def mg_normals(precision: int, words_ptr: int, n_pairs: int, out_ptr: int, stream: int = 0):
    """(z0, z1, -2 ln U(wa)) per word pair, as the kernels make them; device pointers."""
    _check(library().mg_normals(int(precision), C.c_void_p(words_ptr), int(n_pairs), C.c_void_p(out_ptr),
                                C.c_void_p(stream or None)))


def mg_philox(seed: int, ctr0: int, ctr1: int, ctr2: int, ctr3: int, n_calls: int, out_ptr: int,
              stream: int = 0):
    _check(library().mg_philox(C.c_uint64(seed), ctr0 & 0xffffffff, ctr1 & 0xffffffff,
                               ctr2 & 0xffffffff, ctr3 & 0xffffffff, int(n_calls),
                               C.c_void_p(out_ptr), C.c_void_p(stream or None)))


class Sampler:
    """One context: a data set (or a batch of them) and its chains.

    ``Sampler.single(n, L, N, R, d, n_bins, seed, precision=64, n_chains=1, ...)``
    or ``Sampler.batch(ns, Ls, Ns, Rs, ds, n_bins, seeds, ...)``.  Device work is
    enqueued on ``stream`` (an int cudaStream_t, e.g. a torch stream's
    ``cuda_stream``) or on the library's own stream.
    """

    def __init__(self, ctx, precision: int):
        self.ctx = ctx
        self.precision = precision
        self.n_chains = mg_chain_info(ctx, 0)[2]

    @staticmethod
    def _opts(precision, n_chains, chain_id0, tau_scale, P0, record_every, fix_P, stream,
              yz_cluster=0, persistent=False, autotune=False, timeout_cycles=0, mixing=False,
              start_dispersion=0.0):
        o = mg_options_init()
        o.precision = int(precision)
        o.n_chains = int(n_chains)
        o.chain_id0 = int(chain_id0)
        o.tau_scale = float(tau_scale)
        keep = None
        if P0 is not None:
            keep = _f64(P0)
            o.P0 = _dptr(keep)
        o.record_every = int(record_every)
        o.fix_P = int(bool(fix_P))
        o.cuda_stream = stream or None
        o.yz_cluster = int(yz_cluster)
        o.persistent = int(bool(persistent))
        o.autotune = int(bool(autotune))
        o.timeout_cycles = int(timeout_cycles)
        o.mixing = int(mixing)  # False/True, or 2 to alternate plain and mixing sweeps
        o.start_dispersion = float(start_dispersion)
        return o, keep

    @classmethod
    def single(cls, n, L, N, R, d, n_bins, seed, precision=64, n_chains=1, chain_id0=0,
               tau_scale=1.0, P0=None, record_every=0, fix_P=False, k_edges=None, stream=0,
               yz_cluster=0, persistent=False, autotune=False, timeout_cycles=0, mixing=False,
               start_dispersion=0.0):
        o, keep = cls._opts(precision, n_chains, chain_id0, tau_scale, P0, record_every, fix_P, stream,
                            yz_cluster, persistent, autotune, timeout_cycles, mixing, start_dispersion)
        ctx = mg_init(n, L, N, R, d, n_bins, seed, o, k_edges)
        del keep
        return cls(ctx, precision)

    @classmethod
    def batch(cls, ns, Ls, Ns, Rs, ds, n_bins, seeds, precision=32, n_chains=1, chain_id0=0,
              tau_scale=1.0, P0=None, record_every=0, fix_P=False, k_edges=None, stream=0,
              yz_cluster=0, persistent=False, autotune=False, timeout_cycles=0, mixing=False,
              start_dispersion=0.0):
        o, keep = cls._opts(precision, n_chains, chain_id0, tau_scale, P0, record_every, fix_P, stream,
                            yz_cluster, persistent, autotune, timeout_cycles, mixing, start_dispersion)
        ctx = mg_init_batch(ns, Ls, Ns, Rs, ds, n_bins, seeds, o, k_edges)
        del keep
        return cls(ctx, precision)

    def info(self, chain=0):
        return mg_chain_info(self.ctx, chain)

    def sweep(self, n=1):
        mg_sweep(self.ctx, n)
        return self

    def sweep_timed(self, n=1) -> np.ndarray:
        return mg_sweep_timed(self.ctx, n)

    def pk_trace(self, chain=0) -> np.ndarray:
        """The recorded P(k) of one chain, shape (records, n_bins+1)."""
        nb = self.info(chain)[1] + 1
        R = mg_read_pk_trace(self.ctx, chain, None, 0)
        out = np.empty((R, nb))
        if R:
            mg_read_pk_trace(self.ctx, chain, out, R)
        return out

    def pk_acf(self, max_lag, chain=0):
        """(acf (n_bins+1, max_lag+1), n_c (n_bins+1)) from the recorded trace."""
        nb = self.info(chain)[1] + 1
        acf = np.empty((nb, int(max_lag) + 1))
        nc = np.empty(nb, dtype=np.int32)
        mg_pk_acf(self.ctx, chain, max_lag, acf, nc)
        return acf, nc

    def pk_rhat(self, first_chain=0, n_chains=None, burn=0) -> np.ndarray:
        """Gelman-Rubin R-hat per shell over chains first_chain .. +n_chains-1
        (default: all chains of the context) from their recorded traces."""
        if n_chains is None:
            n_chains = self.info(0)[2] - first_chain
        out = np.empty(self.info(first_chain)[1] + 1)
        mg_pk_rhat(self.ctx, first_chain, n_chains, burn, out)
        return out

    def pk_quantiles(self, q, chain=0) -> np.ndarray:
        """Quantiles of each shell's recorded P, shape (n_bins+1, len(q))."""
        q = _f64(q)
        nb = self.info(chain)[1] + 1
        out = np.empty((nb, q.size))
        mg_pk_quantiles(self.ctx, chain, q, out)
        return out

    def sync(self):
        mg_sync(self.ctx)

    def read_s(self, chain=0) -> np.ndarray:
        n = self.info(chain)[0]
        out = np.empty(n ** 3, dtype=np.float32 if self.precision == 32 else np.float64)
        mg_read_s(self.ctx, chain, out.ctypes.data, False)
        return out.reshape(n, n, n)

    def read_s_device(self, chain, out_ptr: int):
        mg_read_s(self.ctx, chain, out_ptr, True)

    def read_pk(self, chain=0) -> np.ndarray:
        nb = self.info(chain)[1]
        out = np.empty(nb + 1)
        mg_read_pk(self.ctx, chain, out)
        return out

    def read_pk_all(self, out=None) -> np.ndarray:
        """Every chain's P(k) in one transfer, shape (n_chains, max n_bins + 1);
        a chain with fewer shells is padded with zeros."""
        if out is None:
            B1 = max(self.info(c)[1] for c in range(self.n_chains)) + 1
            out = np.empty((self.n_chains, B1))
        mg_read_pk_all(self.ctx, out)
        return out

    def read_stats(self, chain=0, fields=True, maps=False) -> dict:
        n, nb, _ = self.info(chain)
        st = MgStats()
        res = {}
        if fields:
            res["n_b"] = np.empty(nb + 1, dtype=np.int64)
            res["sigma_b"] = np.empty(nb + 1)
            res["chi_b"] = np.empty(nb + 1)
            st.n_b = res["n_b"].ctypes.data_as(C.POINTER(C.c_int64))
            st.sigma_b = _dptr(res["sigma_b"])
            st.chi_b = _dptr(res["chi_b"])
        if maps:
            res["mean"] = np.empty(n ** 3)
            res["var"] = np.empty(n ** 3)
            st.mean = _dptr(res["mean"])
            st.var = _dptr(res["var"])
        mg_read_stats(self.ctx, chain, st)
        res.update(sweeps=st.sweeps, records=st.records, tau=st.tau, n_bins=st.n_bins)
        return res

    def set_s(self, chain, s):
        a = np.ascontiguousarray(np.asarray(s, dtype=np.float32 if self.precision == 32 else np.float64))
        mg_set_s(self.ctx, chain, a.ctypes.data, False)

    def set_pk(self, chain, P):
        mg_set_pk(self.ctx, chain, _f64(P))

    def tune(self, reps=5):
        mg_tune(self.ctx, reps)

    def schedule(self) -> dict:
        return mg_schedule(self.ctx)

    def set_data(self, group, d):
        mg_set_data(self.ctx, group, d)

    def adjoint(self, chain, K, logP, w):
        return mg_adjoint(self.ctx, chain, K, logP, w)

    @property
    def sweep_count(self) -> int:
        return mg_get_sweep_count(self.ctx)

    @sweep_count.setter
    def sweep_count(self, v: int):
        mg_set_sweep_count(self.ctx, v)

    def close(self):
        if self.ctx:
            mg_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_shell_sums_noalloc(s_hat_ptr: int, precision: int, n: int, n_bins: int, sigma_ptr: int,
                          nmodes_ptr: int = 0, stream: int = 0):
    """Shell sums of a device half-complex spectrum into device buffers, with
    no device allocation (see include/mg.h)."""
    _check(library().mg_shell_sums_noalloc(C.c_void_p(s_hat_ptr), int(precision), int(n), int(n_bins),
                                           C.c_void_p(sigma_ptr), C.c_void_p(nmodes_ptr or None),
                                           C.c_void_p(stream or None)))


def mg_inject_cuda_error(ctx, after_calls: int):
    """Fake the failure of the after_calls-th checked CUDA call of ctx (see include/mg.h)."""
    _check(library().mg_inject_cuda_error(ctx, int(after_calls)), ctx)


def mg_build_flags() -> int:
    return int(library().mg_build_flags())


def mg_fp64_fma_peak(stream: int = 0) -> float:
    """Measured FP64 FMA throughput of the current device, GFLOP/s (see include/mg.h)."""
    out = C.c_double(0.0)
    _check(library().mg_fp64_fma_peak(C.byref(out), C.c_void_p(stream or None)))
    return out.value
