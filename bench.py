#!/usr/bin/env python3
"""Throughput of the messenger Gibbs sweep on GB300.

Workload (default): the 256^3 batched-FP32 configuration — one Gaussian mock
data set (L = 1000, P(k) = A k/(1+(k/0.02)^2)^2, radial selection, N = 0.1/R),
64 linear k-shells, 16 independent chains swept together.  A step is one full
sweep of all 16 chains: pass YZ (inverse y/z FFTs, messenger draw, forward z/y
FFTs), pass X (forward x FFT, signal draw, shell sums, inverse x FFT) and the
shell draw of P.  The chain state (1.08 GB) is larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (under torchrun) each rank sweeps its own 16 chains (disjoint
chain ids: replicas, no data-path collective); the time is the max over ranks.
--impl reference times the FP64 CPU oracle on this host on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mockgen  # noqa: E402
from paper_1402_1763_gb300 import replicas  # noqa: E402

METRIC = "Gibbs sweeps/s and voxel-updates/s at 256^3 (batched FP32 vs plain FP64); HBM %"
UNIT = "voxel-updates/s"
N_GRID = 256
N_CHAINS = 16
N_BINS = 64
SEED = 3
WORKLOAD = "gaussian-mock-256^3-fp32-16chains-64shells"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(n: int, chains: int, esz: int, n_observed: int):
    """Bytes one launch of each pass must move.

    State per chain: n*n*(n/2) + n*n complex values, each pass reads and writes
    it once.  The messenger constants (b, c) are one complex value per observed
    voxel (unobserved voxels have b = 1, c = 0 and need none), read once per
    pass-YZ launch and shared by every chain of the data set.
    """
    cplx = 2 * esz
    state = (n * n * (n // 2) + n * n) * cplx
    yz = chains * 2 * state + n_observed * cplx
    x = chains * 2 * state
    return yz, x


# the sources the two sweep pass kernels are compiled from (the ncu counters in
# profiles/ stand for these; host code and the other kernels do not change them)
PASS_KERNEL_SOURCES = ["mg_device.cuh", "mg_fft.cuh", "mg_rng.cuh", "mg_launch.h", "mg_pass_x.cuh", "mg_pass_x.cu",
                       "mg_pass_yz.cuh", "mg_pass_yz_launch.cuh", "mg_pass_yz_f32.cu", "mg_pass_yz_f64.cu"]


def kernel_source_hash() -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_1402_1763_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in PASS_KERNEL_SOURCES]
    h = hashlib.sha256()
    for fn in files:
        with open(fn, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _oracle_worker(conn, chain_id):
    """One process of the CPU baseline: one oracle chain of the 256^3 workload
    (its own chain id), one sweep per request; replies with the sweep's wall time."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import sampler
    m = mockgen.make_mock(N_GRID, seed=SEED, n_bins=N_BINS)
    prob = sampler.make_problem(m.shape, m.L, m.N, m.R, m.d, N_BINS)
    ch = sampler.Chains(prob, seed=SEED, chain_ids=[chain_id])
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg != "sweep":
            break
        t0 = time.perf_counter()
        ch.sweep(1)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OraclePool:
    """The FP64 oracle on every host core: one independent chain per process
    (the paper's independent-chains strategy, Sec. 3.4), each single-threaded.
    Processes are started with spawn (safe after CUDA is initialised)."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.cores = cores
        self.conns, self.procs = [], []
        env_threads = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env_threads:
            os.environ[k] = "1"
        try:
            for c in range(cores):
                a, b = ctx.Pipe()
                p = ctx.Process(target=_oracle_worker, args=(b, c), daemon=True)
                p.start()
                self.conns.append(a)
                self.procs.append(p)
        finally:
            for k, v in env_threads.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for cn in self.conns:
            assert cn.recv() == "ready"

    def step(self) -> float:
        """One sweep of every chain, all processes at once; wall seconds."""
        t0 = time.perf_counter()
        for cn in self.conns:
            cn.send("sweep")
        for cn in self.conns:
            cn.recv()
        return time.perf_counter() - t0

    def close(self):
        for cn in self.conns:
            try:
                cn.send("stop")
            except (BrokenPipeError, OSError):
                pass
        for p in self.procs:
            p.join(timeout=30)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, rank):
    """FP64 CPU oracle on this host's cores: each step is one sweep of one
    chain per core of the same 256^3 workload (independent chains, a bounded
    sample of the 16-chain step)."""
    if rank != 0:
        return 0
    cores = host_cores()
    pool = OraclePool(cores)
    try:
        for _ in range(args.warmup):
            pool.step()
        t = 0.0
        for _ in range(args.steps):
            t += pool.step()
    finally:
        pool.close()
    dt = t / args.steps
    v = cores * N_GRID ** 3 / dt
    sample = (f"{cores} independent chains x 1 sweep of the 256^3 workload per step, one single-threaded "
              "numpy FP64 process per core")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "grid": N_GRID, "shells": N_BINS},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(sweeps=2):
    """The oracle as it stands on every host core: one independent chain per
    core, `sweeps` sweeps each (a bounded sample of the workload)."""
    cores = host_cores()
    pool = OraclePool(cores)
    try:
        t = sum(pool.step() for _ in range(sweeps))
    finally:
        pool.close()
    dt = t / sweeps
    return {"value": cores * N_GRID ** 3 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent chains (one single-threaded numpy FP64 process per core) x {sweeps} "
                      "sweeps of the 256^3 workload"}


def tau_int(x) -> float:
    """Integrated autocorrelation time of a trace (Sokal's automatic window:
    sum the normalised autocorrelation up to the first lag k >= 5 tau)."""
    x = np.asarray(x, dtype=np.float64) - np.mean(x)
    n = len(x)
    f = np.fft.rfft(x, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    acf /= acf[0]
    t = 1.0
    for k in range(1, n // 2):
        t += 2.0 * acf[k]
        if k >= 5.0 * t:
            break
    return float(t)


def run_other_workload(args):
    """Secondary workloads (not the headline line): the batching workload in
    one persistent launch per sweep, the adjoint of 8 sweeps at 128^3 FP32, the
    plain FP64 sampler on the 128^3 grid with holes (alone, and against 16 FP32
    chains on the same data), the 256^3 sweeps with every sweep recorded (mean
    and variance maps, P(k) trace), mixing sweeps (Sec. 3.3)
    on the 256^3 workload, and the P(k) autocorrelation of plain, mixing and
    alternating sweeps."""
    import torch
    from paper_1402_1763_gb300 import Sampler
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    if args.workload == "batch-48chains":
        w = mockgen.workload(4)
        g = Sampler.batch([m.n for m in w.mocks], [m.L for m in w.mocks], [m.N for m in w.mocks],
                          [m.R for m in w.mocks], [m.d for m in w.mocks], [m.n_bins for m in w.mocks], w.seeds,
                          precision=32, autotune=True, stream=stream.cuda_stream)
        units = sum(m.n ** 3 for m in w.mocks)
        g.sweep(args.warmup)
        g.sync()
        ev[0].record(stream)
        g.sweep(args.steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        line.update(value=units / (ms * 1e-3), ms_per_step=ms, dtype="f32",
                    config={"workload": w.name, "schedule": g.schedule(), "chains": len(w.mocks)})
    elif args.workload == "adjoint-128":
        w = mockgen.workload(5)
        m = w.mocks[0]
        g = Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 5, precision=32, stream=stream.cuda_stream)
        wts = mockgen.mode_weights(m.n, 5)
        logP = np.log(np.full(m.n_bins + 1, m.L ** 3 / m.n ** 3))
        for _ in range(args.warmup):
            g.adjoint(0, 8, logP, wts)
        t0 = time.perf_counter()
        reps = max(1, args.steps // 20)
        for _ in range(reps):
            g.adjoint(0, 8, logP, wts)
        dt = (time.perf_counter() - t0) / reps
        line.update(metric="adjoint of K = 8 fixed-P sweeps (loss + dL/dlogP + dL/dd), wall time",
                    value=dt * 1e3, unit="ms per call", higher_is_better=False, ms_per_step=dt * 1e3,
                    dtype="f32", config={"workload": w.name, "K": 8,
                                         "note": "host buffers in and out (weights, dL/dd); work buffers kept between calls"})
    elif args.workload == "fp32-vs-fp64-128":
        # the batched-FP32 / plain-FP64 ratio at 128^3 (the 128^3 data set
        # with holes, 32 shells): 16 FP32 chains against 1 FP64 chain
        w = mockgen.workload(2)
        m = w.mocks[0]
        res = {}
        for prec, nc in ((32, 16), (64, 1)):
            g = Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 2, precision=prec, n_chains=nc,
                               stream=stream.cuda_stream)
            g.sweep(args.warmup)
            g.sync()
            ev[0].record(stream)
            g.sweep(args.steps)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / args.steps
            res[prec] = (nc * m.n ** 3 / (ms * 1e-3), ms)
            g.close()
        line.update(value=res[32][0], ms_per_step=res[32][1], dtype="f32",
                    config={"workload": w.name.replace("fp64-1chain", "fp32-16chains-vs-fp64-1chain"),
                            "chains": 16},
                    fp64_single_chain={"value": res[64][0], "unit": UNIT, "ms_per_sweep": res[64][1]},
                    batched_fp32_over_fp64=res[32][0] / res[64][0])
    elif args.workload == "record-256":
        # full-rate posterior summaries: the 256^3 workload (16 FP32 chains)
        # with every sweep recorded (the sums behind the mean and variance maps of s
        # and the P(k) trace of every chain), against the same sweeps unrecorded
        w = mockgen.workload(3)
        m = w.mocks[0]
        res = {}
        nc = args.chains
        for rec in (1, 0):
            g = Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 3, precision=32, n_chains=nc,
                               record_every=rec, stream=stream.cuda_stream)
            g.sweep(args.warmup)
            g.sync()
            ev[0].record(stream)
            g.sweep(args.steps)
            ev[1].record(stream)
            torch.cuda.synchronize()
            res[rec] = ev[0].elapsed_time(ev[1]) / args.steps
            g.close()
        line.update(value=nc * m.n ** 3 / (res[1] * 1e-3), ms_per_step=res[1], dtype="f32",
                    config={"workload": w.name.replace("16chains", f"{nc}chains") + "-record-every-sweep",
                            "chains": nc},
                    ms_per_step_unrecorded=res[0])
    elif args.workload == "fp64-128holes":
        w = mockgen.workload(2)
        m = w.mocks[0]
        g = Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 2, precision=64, stream=stream.cuda_stream)
        g.sweep(args.warmup)
        g.sync()
        ev[0].record(stream)
        g.sweep(args.steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        line.update(value=m.n ** 3 / (ms * 1e-3), ms_per_step=ms, dtype="f64",
                    config={"workload": w.name, "removed_fraction": m.removed_fraction})
    elif args.workload == "fp64-256":
        # the plain FP64 sampler, one chain of the 256^3 data (the headline
        # line times it too; standalone for its FP64 counters)
        w = mockgen.workload(3)
        m = w.mocks[0]
        g = Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 3, precision=64, stream=stream.cuda_stream)
        g.sweep(args.warmup)
        g.sync()
        ev[0].record(stream)
        g.sweep(args.steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        line.update(value=m.n ** 3 / (ms * 1e-3), ms_per_step=ms, dtype="f64",
                    config={"workload": w.name.replace("fp32-16chains", "fp64-1chain")})
    elif args.workload == "precision-256":
        # The precision form's accuracy as the 256^3 configuration states it:
        # 16 FP32 chains over 2000 sweeps against the FP64 path (which matches
        # the oracle to 1e-12) on the same seeds, chains 0 and 15, every 10th
        # sweep: relative L2 of the mean s and mean P(k) over sweeps 21..2000
        # and the worst single sweep.
        w = mockgen.workload(3)
        m = w.mocks[0]
        S = 2000
        mk = lambda prec, nc, c0: Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 3, precision=prec,
                                                 n_chains=nc, chain_id0=c0, stream=stream.cuda_stream)
        g32, g0, g15 = mk(32, 16, 0), mk(64, 1, 0), mk(64, 1, 15)
        acc = {c: [0.0, 0.0, 0.0, 0.0] for c in (0, 15)}
        worst_s = worst_p = 0.0
        t0 = time.perf_counter()
        for sw in range(1, S + 1):
            g32.sweep(1)
            g0.sweep(1)
            g15.sweep(1)
            if sw % 10:
                continue
            for c, g64 in ((0, g0), (15, g15)):
                s32, s64 = g32.read_s(c).astype(np.float64), g64.read_s(0)
                p32, p64 = g32.read_pk(c), g64.read_pk(0)
                worst_s = max(worst_s, float(np.linalg.norm(s32 - s64) / np.linalg.norm(s64)))
                worst_p = max(worst_p, float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64)))
                if sw > 20:
                    a = acc[c]
                    a[0], a[1], a[2], a[3] = a[0] + s32, a[1] + s64, a[2] + p32, a[3] + p64
        dt = time.perf_counter() - t0
        rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
        errs = {f"chain{c}_mean_s_rel_l2": rel(acc[c][0], acc[c][1]) for c in (0, 15)}
        errs.update({f"chain{c}_mean_P_rel_l2": rel(acc[c][2], acc[c][3]) for c in (0, 15)})
        g0.close()
        g15.close()
        g = g32
        line.update(metric="FP32 precision form against the FP64 path, 2000 sweeps at 256^3: worst relative L2 "
                           "of the mean s and mean P(k)",
                    value=max(errs.values()), unit="relative L2", higher_is_better=False,
                    ms_per_step=dt * 1e3 / S, dtype="f32",
                    config={"workload": w.name + "-2000-sweeps", "chains_compared": [0, 15],
                            "sampling": "every 10th sweep; means over sweeps 21..2000"},
                    errors=errs, worst_sample_s_rel_l2=worst_s, worst_sample_P_rel_l2=worst_p)
    elif args.workload == "mixing-256":
        w = mockgen.workload(3)
        m = w.mocks[0]
        g = Sampler.single(m.n, m.L, m.N, m.R, m.d, m.n_bins, 3, precision=32, n_chains=16, mixing=1,
                           stream=stream.cuda_stream)
        g.sweep(args.warmup)
        g.sync()
        ev[0].record(stream)
        g.sweep(args.steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        per = g.sweep_timed(5) / 5
        acc = np.mean([g.read_stats(c)["chi_b"][1:-1].mean() for c in range(16)])
        line.update(value=16 * m.n ** 3 / (ms * 1e-3), ms_per_step=ms, dtype="f32",
                    config={"workload": w.name + "-mixing-sweeps", "chains_per_gpu": 16,
                            "l2": "inputs larger than L2 (1.08 GB chain state)"},
                    per_pass_ms={"pass_yz": per[0], "pass_x_mixing": per[1], "sweep_counter": per[2]},
                    acceptance_rate=float(acc))
    elif args.workload == "mixing-acf":
        # Fully observed 64^3 grid, constant noise N = 1 (R = 1): the shells
        # run from S/N ~ 80 to ~0.2.  Integrated autocorrelation time of
        # log P_b over 3000 sweeps after 300, for plain, mixing and
        # alternating sweeps (the statistical efficiency claim of Sec. 3.3).
        n, L, Nn = 64, 1000.0, 1.0
        s_true = mockgen.gaussian_field(n, L, 9)
        rng = np.random.default_rng(4)
        N = np.full((n, n, n), Nn)
        R = np.ones((n, n, n))
        d = s_true + np.sqrt(Nn) * rng.standard_normal((n, n, n))
        K, burn = 3000, 300
        taus, snr = {}, None
        t0 = time.perf_counter()
        for kind, mix in (("plain", 0), ("mixing", 1), ("alternating", 2)):
            g = Sampler.single(n, L, N, R, d, n // 4, 5, precision=32, mixing=mix, stream=stream.cuda_stream)
            g.sweep(burn)
            tr = np.empty((K, n // 4 + 1))
            for k in range(K):
                g.sweep(1)
                tr[k] = g.read_pk(0)
            nb = g.read_stats(0)["n_b"]
            taus[kind] = [round(tau_int(np.log(tr[:, b])), 1) if nb[b] else 0.0 for b in range(tr.shape[1])]
            if kind == "plain":
                snr = (tr.mean(0) * n ** 3 / L ** 3 / Nn).round(3).tolist()
            g.close()
        g = None
        low = [b for b in range(len(snr)) if snr[b] < 1.0]
        line.update(metric="worst integrated autocorrelation time of log P_b over shells with S/N < 1 "
                           "(alternating plain/mixing sweeps)",
                    value=max(taus["alternating"][b] for b in low), unit="sweeps", higher_is_better=False,
                    ms_per_step=(time.perf_counter() - t0) * 1e3 / (3 * (K + burn)), dtype="f32",
                    config={"workload": "fully observed 64^3, N = 1, 16 shells", "sweeps": K, "burn_in": burn},
                    s_over_n=snr, tau_plain=taus["plain"], tau_mixing=taus["mixing"],
                    tau_alternating=taus["alternating"],
                    worst_low_snr={k: max(v[b] for b in low) for k, v in taus.items()})
    if g is not None:
        g.close()
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chains", type=int, default=16, help="chains of the record-256 workload")
    ap.add_argument("--workload", default="256-fp32-16chains",
                    choices=["256-fp32-16chains", "batch-48chains", "adjoint-128", "fp64-128holes",
                             "fp32-vs-fp64-128", "record-256", "mixing-256", "mixing-acf", "precision-256",
                             "fp64-256"])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local_rank = replicas.rank_world()

    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload != "256-fp32-16chains":
        return run_other_workload(args)

    import torch
    import torch.distributed as dist
    from paper_1402_1763_gb300 import Sampler
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl")
    dd = dist if world > 1 else None
    stream = torch.cuda.Stream()  # a real stream: the library enqueues on it, the events time it
    torch.cuda.set_stream(stream)

    m = mockgen.make_mock(N_GRID, seed=SEED, n_bins=N_BINS)
    M = N_GRID ** 3
    t_init = time.perf_counter()
    smp = Sampler.single(N_GRID, m.L, m.N, m.R, m.d, N_BINS, SEED, precision=32, n_chains=N_CHAINS,
                         chain_id0=replicas.chain_id_base(rank, N_CHAINS), stream=stream.cuda_stream)
    init_s = time.perf_counter() - t_init

    smp.sweep(args.warmup)
    smp.sync()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    replicas.barrier(dd)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    smp.sweep(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier(dd)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = replicas.max_over_ranks(ms, dd)
    units_per_step = world * N_CHAINS * M
    value = units_per_step / (ms * 1e-3)

    # per-pass breakdown over the same number of sweeps (CUDA events per pass)
    per = smp.sweep_timed(args.steps) / args.steps
    yz_bytes, x_bytes = algorithmic_bytes(N_GRID, N_CHAINS, 4, int((m.R > 0).sum()))
    peak, peak_kind = measured_peaks()
    kern = {"pass_yz": (per[0], yz_bytes), "pass_x": (per[1], x_bytes)}
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_bytes = kern[dom]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    sweep_bytes = yz_bytes + x_bytes
    traffic = None
    inst = None
    prof = os.path.join(ROOT, "profiles", "pass_traffic_256cubed_fp32_16chains.json")
    if os.path.exists(prof):
        with open(prof) as f:
            tr = json.load(f)
        # counters only count for the kernel build they were taken on
        if tr.get("source_hash") == kernel_source_hash():
            traffic = tr["per_launch_bytes"].get(dom)
            inst = tr.get("warp_instructions_per_launch")
    # instruction issue, the limit both passes actually meet: the ncu warp
    # instruction count of a launch (same kernel build) over the live launch
    # time, against 4 schedulers x 152 SMs issuing one warp instruction per
    # cycle at the maximum SM clock
    issue = None
    if inst:
        sm_mhz = 2070.0  # GB300 maximum SM clock
        pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pp):
            with open(pp) as f:
                sm_mhz = float(json.load(f).get("sm_max_mhz", sm_mhz))
        issue_peak = 4 * 152 * sm_mhz * 1e6 / 1e9  # G warp instructions / s
        issue = {}
        for name, (kms, _) in kern.items():
            if name in inst:
                ach = inst[name] / (kms * 1e-3) / 1e9
                issue[name] = {"warp_instructions": inst[name], "achieved_ginst_s": ach, "peak_ginst_s": issue_peak,
                               "frac": ach / issue_peak}

    # end to end through the public API with host buffers: each step sweeps
    # all chains and reads every chain's P(k) back to pinned host memory
    from paper_1402_1763_gb300 import mg_read_pk_all
    pk = torch.empty((N_CHAINS, N_BINS + 1), dtype=torch.float64, pin_memory=True).numpy()
    smp.sync()
    replicas.barrier(dd)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.sweep(1)
        mg_read_pk_all(smp.ctx, pk)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = replicas.max_over_ranks(e2e_s, dd)
    smp.close()

    # end to end including set-up: the context made from the host arrays (N, R,
    # d in FP64 uploaded, constants and shell table built), 200 sweeps, every
    # chain's P(k) read back after each.  One such run is half a second of
    # host wall time, so it is taken three times and the median reported.
    e2e_init_sweeps = 200
    e2e_init_runs = []
    e2e_setup_s = []
    for _ in range(3):
        replicas.barrier(dd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        smp2 = Sampler.single(N_GRID, m.L, m.N, m.R, m.d, N_BINS, SEED, precision=32, n_chains=N_CHAINS,
                              chain_id0=replicas.chain_id_base(rank, N_CHAINS), stream=stream.cuda_stream)
        e2e_setup_s.append(time.perf_counter() - t0)
        for _ in range(e2e_init_sweeps):
            smp2.sweep(1)
            mg_read_pk_all(smp2.ctx, pk)
        e2e_init_runs.append(replicas.max_over_ranks(time.perf_counter() - t0, dd))
        smp2.close()
    e2e_init_s = sorted(e2e_init_runs)[1]

    # the plain FP64 single-chain sampler on the same data, same GPU
    fp64 = None
    if rank == 0:
        s64 = Sampler.single(N_GRID, m.L, m.N, m.R, m.d, N_BINS, SEED, precision=64, n_chains=1,
                             stream=stream.cuda_stream)
        s64.sweep(3)
        s64.sync()
        k64 = 10
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        s64.sweep(k64)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1) / k64
        s64.close()
        fp64 = {"value": M / (ms64 * 1e-3), "unit": UNIT, "ms_per_sweep": ms64,
                "config": "plain FP64, 1 chain, same 256^3 data"}
        # The FP64 sweep is bound by the FP64 pipe: its roofline is the FP64
        # flops of one sweep (2 per DFMA, 1 per DADD / DMUL, counted by ncu on
        # the same kernel build) over the sweep time, against the DFMA
        # throughput measured live on this GPU.
        from paper_1402_1763_gb300 import mg_fp64_fma_peak
        peak64 = mg_fp64_fma_peak(stream.cuda_stream)
        fp64["fp64_peak_gflops"] = peak64
        fp64["fp64_peak_kind"] = "measured (DFMA microkernel, mg_fp64_fma_peak)"
        flops64 = inst64 = None
        fp = os.path.join(ROOT, "profiles", "fp64_flops_256cubed_1chain.json")
        if os.path.exists(fp):
            with open(fp) as f:
                fj = json.load(f)
            if fj.get("source_hash") == kernel_source_hash():
                flops64 = fj["fp64_flops_per_sweep"]
                inst64 = fj["fp64_thread_instructions_per_sweep"]
        fp64["fp64_flops_per_sweep"] = flops64
        fp64["fp64_frac"] = (flops64 / (ms64 * 1e-3) / 1e9 / peak64) if flops64 else None
        # DADD and DMUL occupy the FP64 pipe like a DFMA: its occupancy is the
        # FP64 instruction rate against the DFMA rate (peak flops / 2)
        fp64["fp64_pipe_frac"] = (inst64 / (ms64 * 1e-3) / 1e9 / (peak64 / 2)) if inst64 else None

    # comparison only: the library transforms (cuFFT via torch.fft) of one
    # sweep's work, one forward R2C and one inverse C2R 3D FFT per chain, with
    # none of the sweep's draws, shell sums or messenger constants
    cufft = None
    if rank == 0:
        x = torch.randn(N_CHAINS, N_GRID, N_GRID, N_GRID, device="cuda")
        for _ in range(3):
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=x.shape[1:], dim=(1, 2, 3))
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        kc = 10
        c0.record()
        for _ in range(kc):
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=x.shape[1:], dim=(1, 2, 3))
        c1.record()
        torch.cuda.synchronize()
        cufft = {"ms_fwd_inv_16chains": c0.elapsed_time(c1) / kc,
                 "note": "torch.fft (cuFFT) rfftn + irfftn of 16 x 256^3 FP32 fields: the transforms alone of "
                         "one sweep, timed for comparison only (not used by the sampler)"}
        del x, y

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None if args.no_cpu_baseline else cpu_baseline()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": N_GRID, "chains_per_gpu": N_CHAINS, "shells": N_BINS,
                   "precision": "FP32 FFTs and draws, FP64 shell sums and inverse-gamma parameters",
                   "l2": "inputs larger than L2 (1.08 GB chain state per GPU)",
                   "parallelism": f"replicas x{world}"},
        "sweeps_per_s": 1e3 / ms,
        "chain_sweeps_per_s": world * N_CHAINS * 1e3 / ms,
        "fp64_single_chain": fp64,
        "cufft_comparison": cufft,
        "batched_fp32_over_fp64": (value / world) / fp64["value"] if fp64 else None,
        "per_pass_ms": {"pass_yz": per[0], "pass_x": per[1], "shell_draw": per[2]},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": dom_bytes},
        "issue_roofline": issue,
        "sweep_roofline": {"algorithmic_bytes_per_step": sweep_bytes,
                           "achieved_gbs": sweep_bytes / (ms * 1e-3) / 1e9,
                           "frac": sweep_bytes / (ms * 1e-3) / 1e9 / peak},
        "e2e": {"value": units_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": N_CHAINS * (N_BINS + 1) * 8},
        "e2e_with_setup": {"value": units_per_step * e2e_init_sweeps / e2e_init_s, "unit": UNIT,
                           "sweeps": e2e_init_sweeps, "seconds": e2e_init_s,
                           "runs_seconds": e2e_init_runs, "setup_seconds": e2e_setup_s,
                           "h2d_bytes": 3 * M * 8, "d2h_bytes": e2e_init_sweeps * N_CHAINS * (N_BINS + 1) * 8,
                           "note": "context made from host arrays (N, R, d in FP64) inside the timed region, "
                                   "then the sweeps, every chain's P(k) read back after each; median of "
                                   "three runs"},
        "init_seconds": init_s,
        "gpu_launches": args.steps * 3,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
