"""GB300 messenger Gibbs sampler (Jasche & Lavaux 2014) — Python binding.

Every step of the sweep runs in the CUDA library ``_lib/libmg.so`` (built by
``paper_1402_1763_gb300.build``); this package only marshals arguments to the C
ABI of ``include/mg.h``, whose function names it mirrors, plus a small
``Sampler`` convenience class.  There is no CPU fallback: if the library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

from ._native import (  # noqa: F401
    MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ETIMEOUT, MG_ENUMERIC, MG_ESTATE, MG_EUNSUPPORTED, MG_EBOUNDS,
    MG_BUILD_CHECKED,
    MgError, MgGrid, MgOptions, MgStats, library, library_path,
    mg_options_init, mg_init, mg_init_batch, mg_sweep, mg_sweep_timed, mg_read_s, mg_read_pk, mg_read_stats,
    mg_set_s, mg_set_pk, mg_set_data, mg_adjoint, mg_tune, mg_schedule, mg_get_sweep_count, mg_set_sweep_count, mg_chain_info, mg_sync,
    mg_last_error, mg_destroy, mg_philox, mg_normals, mg_shell_sums_noalloc, mg_read_pk_trace, mg_pk_acf, mg_pk_quantiles, mg_pk_rhat, mg_read_pk_all,
    mg_inject_cuda_error, mg_build_flags, mg_fp64_fma_peak,
    Sampler,
)
