"""Run by tests/test_gpu_checked.py in a fresh process with MG_CHECKED=1, so the
binding loads the bounds-checked library: plain sweeps at 8^3 and 16^3 (FP64
and FP32), mixing sweeps and one persistent batch against the oracle, draw for
draw.  Prints one JSON line with the worst errors; any library error (an
MG_EBOUNDS from a check that fired included) propagates as an exception."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import mockgen  # noqa: E402
from gpu_helpers import compare_run, oracle_chains, rel_l2  # noqa: E402


def main():
    import torch
    assert torch.cuda.is_available()
    from paper_1402_1763_gb300 import MG_BUILD_CHECKED, Sampler, library_path, mg_build_flags
    assert library_path().endswith("libmg_checked.so")
    assert mg_build_flags() & MG_BUILD_CHECKED
    out = {"library": os.path.basename(library_path())}
    for n, nb in ((8, 4), (16, 8)):
        m = mockgen.make_mock(n, seed=40 + n, n_bins=nb)
        for prec in (64, 32):
            res = compare_run(m, nb, 7, prec, [1, 4], n_chains=2)
            out[f"plain_{n}_{prec}"] = max(max(es, ep) for _, es, ep in res)
    # mixing sweeps (Sec. 3.3) at 16^3, FP64
    from oracle import mixing as mx, sampler
    m = mockgen.make_mock(16, seed=56, n_bins=8)
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, 8)
    orc = mx.MixingChains(prob, seed=9, chain_ids=[0, 1])
    with Sampler.single(16, m.L, m.N, m.R, m.d, 8, 9, precision=64, n_chains=2, mixing=1) as g:
        orc.sweep(3)
        g.sweep(3)
        out["mixing_16_64"] = max(max(rel_l2(g.read_s(c), orc.s[c]), rel_l2(g.read_pk(c), orc.P[c]))
                                  for c in range(2))
    # one persistent launch per sweep over a batch of 16^3 and 24^3 grids, FP32
    mocks = [mockgen.make_mock(16, seed=61, n_bins=4), mockgen.make_mock(24, seed=62, n_bins=6)]
    seeds = [31, 32]
    with Sampler.batch([x.n for x in mocks], [x.L for x in mocks], [x.N for x in mocks], [x.R for x in mocks],
                       [x.d for x in mocks], [x.n_bins for x in mocks], seeds, precision=32, n_chains=1,
                       persistent=True) as g:
        assert g.schedule()["persistent"]
        g.sweep(3)
        worst = 0.0
        for gi, x in enumerate(mocks):
            o = oracle_chains(x, x.n_bins, seeds[gi], [0])
            o.sweep(3)
            worst = max(worst, rel_l2(g.read_s(gi), o.s[0]), rel_l2(g.read_pk(gi), o.P[0]))
        out["persistent_16_24_32"] = worst
    print(json.dumps(out))


if __name__ == "__main__":
    main()
