#!/usr/bin/env python3
"""Throughput benchmark: learned DBP (fused CUDA kernel) vs plain FFT DBP on GB300.

Workload (per GPU): 256 waveforms x 65536 complex64 samples = 32768 16-QAM
symbols at 10 GBd, 2 samples/symbol, RRC roll-off 0.1, launched at 2 dBm over
25 x 80 km SSMF.  The received waveforms are made on the GPU by the library's
own transmitter and split-step channel (100 symmetric steps/span, EDFA ASE at
NF 5 dB).  LDBP has M = 25 steps (one per span).

Set-up (untimed):
  * LDBP is trained on the GPU (library kernels only) in the stated training
    configuration: batches of 64 frames of 16384 symbols made by the channel
    (100 StPS, ASE) with launch powers from {-4, ..., 6} dBm, filters starting
    at T = 31 and pruned by magnitude to T = 7 (40000 Adam iterations, cosine
    learning rate 3e-4 -> 3e-5, a pool of 64 channel batches made once).
    T = 7 is the shortest uniform length whose trained model passed the
    0.1 dB gate in the pruning study (`--workload train_prune`).
  * The gate: the model's effective SNR on the bench waveforms within 0.1 dB
    of 1-step-per-span frequency-domain DBP (or better); reported either way.
  * LS-initialised models with T in {3, 5, 9, 15} are timed for reference.

One bench step = one LDBP pass over the whole 256 x 65536 batch.  Metric:
complex samples * steps / s, whole job (all ranks).  Plain FFT DBP (the
fused cluster kernel and cuFFT) is timed on the same waveforms.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload with the same T, one waveform per host core per step, in worker
processes on every core (the paper has no implementation to run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LDBP vs plain FFT DBP complex samples·steps/s on 1 GB300 at ΔSNR≤0.1 dB; % roofline"
UNIT = "samples·steps/s"
B, N_SAMP, M_STEPS = 256, 65536, 25
NSYM = N_SAMP // 2
SPAN_KM = 80.0
FS = 20e9
POWER_DBM = 2.0
CHANNEL_STEPS = 100
E2E_CHUNKS = 12
HEAD_T = 7  # filter length of the headline model (trained, pruned from 31)

# FP32 pipe of GB300: 152 SMs x 128 FP32 lanes per clock x 2.07 GHz maximum
# SM clock, one fused multiply-add = 2 floating-point operations.
SMS, FP32_LANES, SM_MAX_HZ = 152, 128, 2.07e9
FP32_PEAK_FLOPS = 2 * SMS * FP32_LANES * SM_MAX_HZ


# plain FD DBP: two n-point FFTs (5 n log2 n flops each), the spectral multiply
# (6) and the Kerr step (10) per sample and step
DBP_FLOPS_PER_SAMPLE_STEP = 2 * 5 * int(np.log2(N_SAMP)) + 6 + 10


def ldbp_flops_per_sample_step(T: int) -> int:
    """Algorithmic FP32 work of one LDBP step per complex sample (direct form).

    FIR: T complex multiply-adds = 8T flops (the folded form of Fig. 3 does
    fewer, which counts in the kernel's favour); Kerr: |x|^2 (3) and the
    rotation x e^{j phi} (6), with c folded into the phase polynomial and
    sin/cos counted as one special function of the phase (Sec. V-B assumes
    a look-up table for it).
    """
    return 8 * T + 9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--taps", type=int, default=0, help="skip training and time LS-initialised filters of this length")
    ap.add_argument("--train-iters", type=int, default=40000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=B, help="waveforms per GPU (profiling runs use fewer)")
    ap.add_argument("--profile", default="", choices=["", "ldbp", "dbp", "dbp_cufft", "ldbp_bwd", "channel",
                                                      "resample", "analog_channel", "train_channel", "long_channel",
                                                      "essm", "essm_bwd"],
                    help="run only this kernel (warmup + steps launches) on random input, for ncu captures")
    ap.add_argument("--workload", default="ldbp",
                    choices=["ldbp", "channel", "ragged", "train", "train_prune", "sym32", "essm", "analog"],
                    help="ldbp: the headline; channel / ragged / train: the other workloads, reported separately")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def ls_model(T: int, M: int = M_STEPS):
    """LS-initialised taps (host FP64) and Kerr coefficients of 1-StPS LDBP."""
    from paper_2010_14258_gb300 import init as pinit
    return pinit.ldbp_init([T] * M, span_km=SPAN_KM, fs=FS, steps_per_span=1)


def pack_taps(taps, M=M_STEPS):
    import torch
    arr = np.zeros((M, max(len(h) for h in taps)), np.complex64)
    for i, h in enumerate(taps):
        arr[i, : len(h)] = h
    return torch.from_numpy(arr).cuda()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [t.strip() for t in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_fn(fn, reps, warmup=1):
    """Mean CUDA-event milliseconds of fn() on the current stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ldbp_fwd_traffic.txt")
FWD_SOURCES = ("ldbp_fwd.cu", "ldbp_fwd.cuh", "ldbp_tile.cuh", "common.cuh")


def fwd_source_sha256() -> str:
    h = hashlib.sha256()
    for f in FWD_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2010_14258_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def traffic_from_profiles(kernel: str, T: int):
    """DRAM bytes per launch from the committed ncu summary (a JSON object in a
    text file), if it was taken on the current source of the kernel (else None)."""
    try:
        rec = json.load(open(TRAFFIC_FILE)).get(kernel)
        sha = fwd_source_sha256()
    except (OSError, ValueError, AttributeError):
        return None
    if not rec or rec.get("src_sha256") != sha or rec.get("T") != T:
        return None
    return rec.get("bytes_per_launch")


def job_throughput(ms_local: float, units_per_rank: int, steps: int, world: int, device: str = "cpu"):
    """Whole-job throughput of a weak-scaling replica run: the slowest rank's
    time (max over ranks) and the units of all ranks per second."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank * steps / (ms / 1e3)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_waveform(job):
    """One waveform of the workload through the FP64 oracle (worker process).
    The waveform is drawn in the worker from its seed; returns the seconds spent."""
    seed, taps, c = job
    from oracle import ldbp as oldbp
    import synth
    x = synth.gaussian_waveform(1, N_SAMP, seed, 1e-3)
    t = time.perf_counter()
    oldbp.forward(x, taps, c)
    return time.perf_counter() - t


class OraclePool:
    """Worker processes (spawned: safe after CUDA is initialised) on every host core."""

    def __init__(self, T: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.cores = host_cores()
        self.ex = cf.ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"))
        taps, c = ls_model(T)
        self.taps = [np.asarray(h, np.complex128) for h in taps]
        self.c = [float(v) for v in c]
        list(self.ex.map(_oracle_waveform, [(1, self.taps[:1], self.c[:1])] * self.cores))  # start the workers

    def run(self, waves: int, seed0: int):
        """Wall time of `waves` oracle waveforms spread over the workers."""
        t = time.perf_counter()
        list(self.ex.map(_oracle_waveform, [(seed0 + w, self.taps, self.c) for w in range(waves)]))
        return time.perf_counter() - t

    def close(self):
        self.ex.shutdown()


def cpu_baseline_ldbp(T: int):
    """The FP64 oracle (numpy) on every host core, one waveform per worker at a time,
    over a bounded sample of the workload (two rounds of one waveform per core)."""
    pool = OraclePool(T)
    try:
        waves = min(B, 2 * pool.cores)
        dt = pool.run(waves, 124)
    finally:
        pool.close()
    return {"value": waves * N_SAMP * M_STEPS / dt, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{waves} of {B} waveforms x {N_SAMP} samples x {M_STEPS} steps, T={T}, numpy FP64, "
                      f"one worker process per core", "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    T = args.taps or HEAD_T
    pool = OraclePool(T)
    try:
        for i in range(args.warmup):
            pool.run(pool.cores, 1000 + i)
        tot = 0.0
        for i in range(args.steps):
            tot += pool.run(pool.cores, 2000 + i * pool.cores)
    finally:
        pool.close()
    units = pool.cores * N_SAMP * M_STEPS
    value = args.steps * units / tot
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": f"ldbp_infer_{B}x{N_SAMP}_M{M_STEPS}", "T": T,
                                           "sample": f"{pool.cores} of {B} waveforms per step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                            "sample": f"{pool.cores} waveforms x {N_SAMP} samples x {M_STEPS} steps per step "
                                      f"(one per core), numpy FP64"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def profile_only(args, api):
    """Launch one kernel (warmup + steps times) on random resident input; prints its mean time."""
    import torch
    import synth
    T = args.taps or 3
    B = args.batch
    # two resident inputs, alternated as in the timed region (2 x 134 MB > L2)
    xs = [torch.randn(B, N_SAMP, device="cuda", dtype=torch.complex64) * (1e-3 ** 0.5) for _ in range(2)]
    x = xs[0]
    y = torch.empty_like(x)
    it = [0]

    def nxt():
        it[0] += 1
        return xs[it[0] % 2]
    fib, link = synth.Fiber(), synth.Link(M_STEPS, SPAN_KM, 1, False, False)
    taps_np, c = ls_model(T)
    taps = pack_taps(taps_np)
    units = B * N_SAMP * M_STEPS
    n_wave = N_SAMP
    if args.profile == "ldbp":
        fn = lambda: api.ldbp_apply(taps, [T] * M_STEPS, c, nxt(), out=y)  # noqa: E731
    elif args.profile == "ldbp_bwd":
        ck = torch.empty((M_STEPS, B, N_SAMP), dtype=torch.complex64, device="cuda")
        api.ldbp_apply(taps, [T] * M_STEPS, c, x, ckpt=ck, out=y)
        fn = lambda: api.ldbp_backward(taps, [T] * M_STEPS, c, ck, x, want_gx=True)  # noqa: E731
    elif args.profile == "dbp":
        fn = lambda: api.dbp_apply(fib, link, FS, x, steps_per_span=1, symmetric=False, out=y)  # noqa: E731
    elif args.profile == "channel":
        ch = synth.Link(M_STEPS, SPAN_KM, 4, True, True)
        units = B * N_SAMP * M_STEPS * 4
        fn = lambda: api.ssm_forward(fib, ch, FS, x, out=y)  # noqa: E731
    elif args.profile == "train_channel":
        # the training channel's shape: --batch frames of 32768 samples, 25 x 80 km,
        # 4 symmetric StPS with ASE (the cluster kernel with 8-block clusters)
        xt = torch.randn(B, 32768, device="cuda", dtype=torch.complex64) * (1e-3 ** 0.5)
        yt = torch.empty_like(xt)
        ch = synth.Link(M_STEPS, SPAN_KM, 4, True, True)
        units = B * 32768 * M_STEPS * 4
        n_wave = 32768
        fn = lambda: api.ssm_forward(fib, ch, FS, xt, out=yt)  # noqa: E731
    elif args.profile in ("essm", "essm_bwd"):
        # the learned enhanced SSM on --batch waveforms: T = --taps (default 9), a
        # unit (2 kappa + 1)-tap filter with kappa = 20 in every step
        kap = 20
        T = args.taps or 9
        taps_np, c = ls_model(T)
        taps = pack_taps(taps_np)
        e = np.zeros((M_STEPS, 2 * kap + 1), np.float32)
        e[:, kap] = 1.0
        ed = torch.from_numpy(e).cuda()
        ks = [kap] * M_STEPS
        if args.profile == "essm":
            fn = lambda: api.ldbp_essm_apply(taps, [T] * M_STEPS, c, ed, ks, nxt(), out=y)  # noqa: E731
        else:
            ck = torch.empty((M_STEPS, B, N_SAMP), dtype=torch.complex64, device="cuda")
            api.ldbp_essm_apply(taps, [T] * M_STEPS, c, ed, ks, x, ckpt=ck, out=y)
            fn = lambda: api.ldbp_essm_backward(taps, [T] * M_STEPS, c, ed, ks, ck, x)  # noqa: E731
    elif args.profile == "long_channel":
        # the data-generation channel's shape: --batch frames of 131072 samples,
        # 10 x 100 km, 200 symmetric StPS with ASE (the L2-resident path from 8 frames)
        xt = torch.randn(B, 131072, device="cuda", dtype=torch.complex64) * (1e-3 ** 0.5)
        yt = torch.empty_like(xt)
        ch = synth.Link(10, 100.0, 200, True, True, 5.0, 1.946e14, seed=4, counter=0)
        units = B * 131072 * 10 * 200
        n_wave = 131072
        fn = lambda: api.ssm_forward(fib, ch, 128e9, xt, out=yt)  # noqa: E731
    elif args.profile in ("resample", "analog_channel"):
        # the analog-rate workload's grids: frames of 1024 symbols at rho_a = 6
        # (n = 6144) and rho_d = 2 (n = 2048); --batch frames, two inputs alternated
        n_a, n_d = 6144, 2048
        xa = [torch.randn(B, n_a, device="cuda", dtype=torch.complex64) for _ in range(2)]
        r = torch.empty((B, n_d), dtype=torch.complex64, device="cuda")
        def nxt_a():
            it[0] += 1
            return xa[it[0] % 2]
        if args.profile == "resample":
            units = B * n_a
            fn = lambda: api.resample(nxt_a(), n_d, out=r)  # noqa: E731
        else:
            ch = synth.Link(M_STEPS, SPAN_KM, 4, True, True)
            ya = torch.empty_like(xa[0])
            units = B * n_a * M_STEPS * 4
            fn = lambda: api.ssm_forward(fib, ch, FS * 3, xa[0], out=ya)  # noqa: E731
    else:
        fn = lambda: api.ssm_cufft(fib, link, FS, x, dbp_steps_per_span=1, dbp_symmetric=False, out=y)  # noqa: E731
    ms = time_fn(fn, args.steps, args.warmup)
    print(json.dumps({"profile": args.profile, "batch": B, "n": n_wave, "T": T, "ms": ms,
                      "samples_steps_per_s": units / (ms / 1e3)}))


def workload_channel(args, api):
    """Channel data generation at scale: 128 x 2^17 samples, 32 GBd 16-QAM at 4 samples/symbol,
    10 x 100 km, 200 symmetric steps/span, ASE; fused kernel vs cuFFT; FP32 error vs the FP64
    oracle on sampled waveforms (one span, to bound the oracle's time)."""
    import torch
    import synth
    from oracle import nlse
    Bc, nsym, sps, fs = 128, 32768, 4, 128e9
    fib = synth.Fiber()
    link = synth.Link(10, 100.0, 200, True, True, 5.0, 1.946e14, seed=4, counter=0)
    s = torch.from_numpy(synth.qam16_symbols(Bc, nsym, 4).astype(np.complex64)).cuda()
    pw = torch.full((Bc,), 1e-3, dtype=torch.float32, device="cuda")
    x = api.tx(s, pw, sps=sps)
    y = torch.empty_like(x)
    units = Bc * nsym * sps * 10 * 200
    fused = time_fn(lambda: api.ssm_forward(fib, link, fs, x, out=y), 2)
    cufft = time_fn(lambda: api.ssm_cufft(fib, link, fs, x, out=y), 2)
    # FP32 vs FP64 on two sampled waveforms over one span (200 steps, no ASE), bounding the oracle's time
    one_span = synth.Link(1, 100.0, 200, True, False)
    errs = []
    for b in (0, 64):
        xb = x[b: b + 1].contiguous()
        ref = nlse.channel(xb.cpu().numpy().astype(np.complex128), fib, one_span, fs)
        yb = api.ssm_forward(fib, one_span, fs, xb)
        errs.append(float(np.linalg.norm(yb.cpu().numpy() - ref) / np.linalg.norm(ref)))
    print(json.dumps({"workload": "channel_128x131072_10x100km_200stps", "unit": UNIT,
                      "fused_samples_steps_per_s": units / (fused / 1e3), "fused_ms": fused,
                      "cufft_samples_steps_per_s": units / (cufft / 1e3), "cufft_ms": cufft,
                      "speedup_vs_cufft": cufft / fused,
                      "fp32_rel_l2_vs_fp64_per_waveform_1span_200steps": errs}))


def workload_ragged(args, api):
    """1000 LDBP waveforms, n log-uniform 2^12..2^18, 5..40 spans (1 step each), T in {3,5,9,15,31}:
    one persistent launch (autotuned, graph-replayed) vs one ldbp_apply launch per waveform."""
    import torch
    import synth
    from paper_2010_14258_gb300 import init as pinit
    count = 1000
    n = [int(v) for v in synth.ragged_lengths(count, 5)]
    spans = [int(v) for v in synth.ragged_spans(count, 5)]
    tt = [int(v) for v in synth.ragged_taps(count, 5)]
    stride = 16
    models = {T: pinit.ldbp_init([T], span_km=SPAN_KM, fs=FS) for T in set(tt)}
    rows = sum(spans)
    tarr = np.zeros((rows, stride), np.complex64)
    carr = np.zeros(rows, np.float32)
    r = 0
    for w in range(count):
        h, c = models[tt[w]]
        tarr[r: r + spans[w], : len(h[0])] = h[0]
        carr[r: r + spans[w]] = c[0]
        r += spans[w]
    taps, cd = torch.from_numpy(tarr).cuda(), torch.from_numpy(carr).cuda()
    x = torch.randn(sum(n), device="cuda", dtype=torch.complex64) * (1e-3 ** 0.5)
    y = torch.empty_like(x)
    plan = api.RaggedPlan(n, [[tt[w]] * spans[w] for w in range(count)], stride)
    plan.autotune(taps, cd, x, y)
    plan.capture(taps, cd, x, y)
    units = sum(n[w] * spans[w] for w in range(count))
    graph_ms = time_fn(plan.replay, 10, 2)
    done = torch.zeros(count, dtype=torch.int64, device="cuda")
    start = torch.full((1,), 2 ** 63 - 1, dtype=torch.int64, device="cuda")
    plan.apply(taps, cd, x, y, done_ns=done, start_ns=start)
    torch.cuda.synchronize()
    lat = (done - start).double().cpu().numpy() / 1e6
    # per-waveform launches
    off = np.cumsum([0] + n[:-1])
    rs = np.cumsum([0] + spans[:-1])
    per = []
    for w in range(count):
        Ts = [tt[w]] * spans[w]
        per.append((taps[rs[w]: rs[w] + spans[w]], Ts, carr[rs[w]: rs[w] + spans[w]].tolist(),
                    x[off[w]: off[w] + n[w]].view(1, -1), y[off[w]: off[w] + n[w]].view(1, -1)))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(count + 1)]

    def per_wave():
        evs[0].record()
        for w, (tp, Ts, cl, xw, yw) in enumerate(per):
            api.ldbp_apply(tp, Ts, cl, xw, out=yw)
            evs[w + 1].record()

    per_wave()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_wave()
    torch.cuda.synchronize()
    per_ms = evs[0].elapsed_time(evs[-1])
    plat = np.array([evs[0].elapsed_time(evs[w + 1]) for w in range(count)])
    info = plan.info()
    print(json.dumps({"workload": "ragged_1000_lengths_2^12-2^18_spans_5-40_T_3-31", "unit": UNIT,
                      "persistent_graph_samples_steps_per_s": units / (graph_ms / 1e3), "persistent_ms": graph_ms,
                      "persistent_latency_ms_p50": float(np.percentile(lat, 50)),
                      "persistent_latency_ms_p99": float(np.percentile(lat, 99)),
                      "per_waveform_samples_steps_per_s": units / (per_ms / 1e3), "per_waveform_ms": per_ms,
                      "per_waveform_latency_ms_p50": float(np.percentile(plat, 50)),
                      "per_waveform_latency_ms_p99": float(np.percentile(plat, 99)),
                      "host_enqueue_s": time.perf_counter() - t0, "plan": info, "samples_steps": units}))
    plan.close()


def workload_train(args, api):
    """One LDBP training iteration at 64 x 32768 samples: GPU channel (25 x 80 km, 100 steps/span, ASE),
    M = 25, T = 31, forward with checkpoints, receiver loss, adjoint, Adam."""
    import torch
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    cfg = TrainConfig(batch=64, nsym=16384, n_spans=25, channel_steps=100, t_start=31, t_end=3, iters=1000,
                      lr=1e-3, seed=3)
    tr = Trainer(cfg)
    it_ms = time_fn(lambda: tr.train_step(tr.step_count), 5, 2)
    sd, pw, yw = tr.frames(0)
    ch_ms = time_fn(lambda: tr.frames(0), 5, 1)
    fw_ms = time_fn(lambda: api.ldbp_apply(tr.taps, tr.T, tr.c, yw, ckpt=tr.ckpt, out=tr.out), 5, 1)
    st, _, g = api.rx(tr.out, sd, pw, grad=True)
    bw_ms = time_fn(lambda: api.ldbp_backward(tr.taps, tr.T, tr.c, tr.ckpt, g, want_gx=False), 5, 1)
    print(json.dumps({"workload": "train_64x32768_M25_T31", "ms_per_iteration": it_ms, "channel_ms": ch_ms,
                      "ldbp_forward_ckpt_ms": fw_ms, "ldbp_backward_ms": bw_ms,
                      "taps_after": int(sum(tr.T))}))


def workload_train_prune(args, api):
    """The training configuration as stated (Sec. IV-B/IV-C, Table I): batches of 64
    frames of 16384 16-QAM symbols (n = 32768) made on the GPU by the channel (25 x 80
    km, 100 symmetric StPS, ASE), launch powers drawn from {-4, ..., 6} dBm per frame,
    M = 25 filters starting at T = 31 (LS initialisation) and pruned by magnitude to
    the target lengths on a front-loaded schedule over the first half of the run,
    Adam with a cosine learning rate 3e-4 -> 3e-5.  The channel makes a pool of 64
    batches (4096 frames) once, cycled through by the iterations.  Targets: 3, the
    alternating 5/3 of Sec. V-B (77 total taps), 5 and 7.  Each pruned model is
    evaluated at 2 dBm on 64 frames of the inference link against 1-StPS FD DBP on
    the same waveforms, and timed on the 256 x 65536 inference batch."""
    import torch
    import synth
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    fib = synth.Fiber()
    iters = args.train_iters
    Be = 64
    sym = torch.from_numpy(synth.qam16_symbols(Be, NSYM, 2000).astype(np.complex64)).cuda()
    pw = torch.full((Be,), 1e-3 * 10 ** (POWER_DBM / 10), dtype=torch.float32, device="cuda")
    y = api.ssm_forward(fib, synth.Link(M_STEPS, SPAN_KM, CHANNEL_STEPS, True, True, 5.0, 1.946e14, seed=77,
                                        counter=0), FS, api.tx(sym, pw))
    z = torch.empty_like(y)
    dbp_link = synth.Link(M_STEPS, SPAN_KM, 1, False, False)

    def snr_of(out):
        st, _, _ = api.rx(out, sym, pw)
        return api.snr_db(st)
    api.dbp_apply(fib, dbp_link, FS, y, steps_per_span=1, symmetric=False, out=z)
    snr_dbp = snr_of(z)
    xb = torch.randn(256, N_SAMP, device="cuda", dtype=torch.complex64) * (1e-3 ** 0.5)
    zb = torch.empty_like(xb)
    units = 256 * N_SAMP * M_STEPS
    res = {}
    for name, t_end, t_odd in (("3", 3, 0), ("5/3", 5, 3), ("5", 5, 0), ("7", 7, 0)):
        cfg = TrainConfig(batch=64, nsym=16384, n_spans=M_STEPS, span_km=SPAN_KM, channel_steps=100, ase=True,
                          powers_dbm=tuple(range(-4, 7)), t_start=31, t_end=t_end, t_end_odd=t_odd, iters=iters,
                          lr=3e-4, lr_final=3e-5, prune_frac=0.5, seed=5, data_pool=64)
        t0 = time.perf_counter()
        tr = Trainer(cfg)
        torch.cuda.synchronize()
        pool_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        trace = []
        for it in range(iters):
            tr.train_step(it)
            if (it + 1) % max(1, iters // 16) == 0:
                trace.append([it + 1, float(np.mean(tr.history[-50:])), int(sum(tr.T))])
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        api.ldbp_apply(tr.taps, tr.T, tr.c, y, out=z)
        snr = snr_of(z)
        ms = time_fn(lambda: api.ldbp_apply(tr.taps, tr.T, tr.c, xb, out=zb), 20, 3)
        flops = sum(ldbp_flops_per_sample_step(T) for T in tr.T) * 256 * N_SAMP
        res[name] = {"T": list(tr.T), "total_taps": int(sum(T - 1 for T in tr.T) + 1), "snr_db": snr,
                     "delta_vs_dbp_db": snr - snr_dbp, "within_0p1_db": bool(snr >= snr_dbp - 0.1),
                     "pool_s": pool_s, "train_s": train_s, "ms_per_iteration": train_s / iters * 1e3,
                     "loss_trace_iter_loss_sumT": trace,
                     "final_loss": float(np.mean(tr.history[-50:])),
                     "ldbp_ms_256x65536": ms, "samples_steps_per_s": units / (ms / 1e3),
                     "frac_fp32": flops / (ms / 1e3) / FP32_PEAK_FLOPS}
        print(json.dumps({"target": name, **res[name]}), flush=True)
    print(json.dumps({"workload": f"train_prune_64x32768_M{M_STEPS}_T31", "iters": iters, "unit": UNIT,
                      "eval": f"{Be} x {N_SAMP} at {POWER_DBM} dBm, 25 x 80 km, 100 StPS, ASE",
                      "dbp_1stps_snr_db": snr_dbp, "models": res}))


def workload_sym32(args, api):
    """Symmetric-SSM-based LDBP with logarithmic step sizes (Sec. IV-C) at 32 GBd, T = 31 (2 StPS) and 21 (4 StPS):
    256 x 65536 samples (2 samples/symbol, fs = 64 GHz), 10 x 100 km at 4 dBm, data from
    the GPU channel (50 symmetric steps/span, ASE).  LS-initialised LDBP with 2 StPS
    (l = 21 layers) and 4 StPS (l = 41), against symmetric FD DBP with 2 and 4 uniform StPS
    and linear compensation (gamma = 0), all on the same waveforms."""
    import torch
    import synth
    from paper_2010_14258_gb300 import init
    Bw, nsym, fs, nsp, lsp, pdbm = args.batch, 32768, 64e9, 10, 100.0, 4.0
    n = 2 * nsym
    fib = synth.Fiber()
    sym = torch.from_numpy(synth.qam16_symbols(Bw, nsym, 3000).astype(np.complex64)).cuda()
    pw = torch.full((Bw,), 1e-3 * 10 ** (pdbm / 10), dtype=torch.float32, device="cuda")
    x = api.tx(sym, pw)
    y = api.ssm_forward(fib, synth.Link(nsp, lsp, 50, True, True, 5.0, 1.946e14, seed=91, counter=0), fs, x, out=x)
    z = torch.empty_like(y)

    def snr_of(out):
        st, _, _ = api.rx(out, sym, pw)
        return api.snr_db(st)

    res = {}
    lin = synth.Fiber(fib.alpha_db_per_km, fib.beta2_ps2_per_km, 0.0)
    api.dbp_apply(lin, synth.Link(nsp, lsp, 1, True, False), fs, y, steps_per_span=1, symmetric=True, out=z)
    res["linear_cd_snr_db"] = snr_of(z)
    for stps, T in ((2, 31), (4, 21)):
        link = synth.Link(nsp, lsp, stps, True, False)
        dms = time_fn(lambda: api.dbp_apply(fib, link, fs, y, steps_per_span=stps, symmetric=True, out=z), 5, 1)
        res[f"fd_dbp_{stps}stps"] = {"snr_db": snr_of(z), "ms": dms}
        taps, c = init.ldbp_init_symmetric(T, nsp, lsp, fs, steps_per_span=stps)
        tp = pack_taps(taps, M=len(taps))
        Ts, cs = [T] * len(taps), [float(v) for v in c]
        ms = time_fn(lambda: api.ldbp_apply(tp, Ts, cs, y, out=z), 20, 3)
        units = Bw * n * len(Ts)
        res[f"ldbp_{stps}stps_T{T}"] = {
            "layers": len(Ts), "snr_db": snr_of(z), "ms": ms, "samples_steps_per_s": units / (ms / 1e3),
            "frac_fp32": ldbp_flops_per_sample_step(T) * units / (ms / 1e3) / FP32_PEAK_FLOPS,
            "speedup_vs_fd_dbp_same_stps": dms / ms}
    print(json.dumps({"workload": f"ldbp_symmetric_logsteps_32gbd_{Bw}x{n}_10x100km", "unit": UNIT,
                      "model": "LS-initialised (untrained)", **res}))


def measured_hbm_gbs():
    """HBM copy bandwidth of this GPU model (measured copy), else the fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback"


def workload_analog(args, api):
    """Analog-rate system model of Sec. IV-A with the paper's frames (Table I:
    N_sym = 1024, rho_a = 6, rho_d = 2): 2048 frames of 1024 16-QAM symbols at 10 GBd
    simulated at rho_a = 6 samples/symbol (n = 6144) over 25 x 80 km (100 symmetric
    steps/span, ASE) on the fused cluster kernel (clusters of 3 blocks), timed against
    the library-FFT evaluation of the same program; then brick-wall low-pass
    (Delta B = f_s) and sampling at rho_d = 2 by the single-pass front end, reported
    against HBM (algorithmic bytes: one read of the input grid, one write of the
    output grid; two input batches alternated, 201 MB > L2); and the effective SNR
    of 1-StPS DBP on the received samples compared with the same link simulated at
    rho_d."""
    import torch
    import synth
    Bw, nsym, rho_a, rho_d, Rs = 2048, 1024, 6, 2, FS / 2
    n_a, n_d = nsym * rho_a, nsym * rho_d
    steps = M_STEPS * 100
    fib = synth.Fiber()
    link = synth.Link(M_STEPS, SPAN_KM, 100, True, True, 5.0, 1.946e14, seed=78, counter=0)
    sym = torch.from_numpy(synth.qam16_symbols(Bw, nsym, 3000).astype(np.complex64)).cuda()
    pw = torch.full((Bw,), 1e-3 * 10 ** (POWER_DBM / 10), dtype=torch.float32, device="cuda")
    xd = api.tx(sym, pw, sps=rho_d)
    xa = api.resample(xd, n_a)
    ya = torch.empty_like(xa)
    ya2 = torch.empty_like(xa)
    r = torch.empty_like(xd)
    ch_ms = time_fn(lambda: api.ssm_forward(fib, link, rho_a * Rs, xa, out=ya), 2, 1)
    ch_cufft_ms = time_fn(lambda: api.ssm_cufft(fib, link, rho_a * Rs, xa, out=ya2), 1, 1)
    api.ssm_forward(fib, link, rho_a * Rs, xa, out=ya)
    ya2.copy_(ya)
    bufs = [ya, ya2]
    k = [0]

    def down():
        k[0] ^= 1
        api.resample(bufs[k[0]], n_d, out=r)
    down_ms = time_fn(down, 20, 3)
    xa2 = torch.empty_like(xa)
    outs = [xa, xa2]

    def up():
        k[0] ^= 1
        api.resample(xd, n_a, out=outs[k[0]])
    up_ms = time_fn(up, 20, 3)
    api.resample(ya, n_d, out=r)
    peak, kind = measured_hbm_gbs()
    alg = (n_a + n_d) * 8 * Bw
    dbp_a = api.dbp_apply(fib, link, FS, r, 1, False)
    st_a, _, _ = api.rx(dbp_a, sym, pw)
    yd = api.ssm_forward(fib, link, FS, xd)
    dbp_d = api.dbp_apply(fib, link, FS, yd, 1, False)
    st_d, _, _ = api.rx(dbp_d, sym, pw)
    print(json.dumps({"workload": f"analog_rate_{Bw}x{nsym}sym_rho6_to_rho2_25x80km_100stps", "unit": UNIT,
                      "channel_ms": ch_ms, "channel_cufft_ms": ch_cufft_ms,
                      "channel_samples_steps_per_s": Bw * n_a * steps / (ch_ms / 1e3),
                      "channel_speedup_vs_cufft": ch_cufft_ms / ch_ms,
                      "front_end_down_ms": down_ms, "front_end_up_ms": up_ms,
                      "front_end_input_samples_per_s": Bw * n_a / (down_ms / 1e3),
                      "front_end_roofline": {"bound": "hbm", "achieved": alg / (down_ms / 1e3) / 1e9, "peak": peak,
                                             "unit": "GB/s", "frac": alg / (down_ms / 1e3) / 1e9 / peak,
                                             "peak_kind": kind,
                                             "algorithmic_bytes": "8 (n_in + n_out) per waveform"},
                      "front_end_up_roofline_frac": alg / (up_ms / 1e3) / 1e9 / peak,
                      "dbp_1stps_snr_db_rho_a6": api.snr_db(st_a), "dbp_1stps_snr_db_rho_d2": api.snr_db(st_d)}))


def workload_essm(args, api):
    """Learned enhanced SSM (filtered nonlinear steps, Sec. III-C): the LDBP inference
    workload (256 x 65536, 25 x 80 km at 2 dBm, GPU channel data) with a (2 kappa + 1)-tap
    real filter on |v|^2 in every nonlinear step; T = 9, kappa in {0, 8, 20}, unit-filter
    and low-pass initialisations; throughput, FP32 fraction of the direct-form work
    (8T + 9 + 2(2 kappa + 1) flops per sample-step) and effective SNR."""
    import torch
    import synth
    fib = synth.Fiber()
    Bw = args.batch
    sym = torch.from_numpy(synth.qam16_symbols(Bw, NSYM, 2000).astype(np.complex64)).cuda()
    pw = torch.full((Bw,), 1e-3 * 10 ** (POWER_DBM / 10), dtype=torch.float32, device="cuda")
    x = api.tx(sym, pw)
    y = api.ssm_forward(fib, synth.Link(M_STEPS, SPAN_KM, CHANNEL_STEPS, True, True, 5.0, 1.946e14, seed=77,
                                        counter=0), FS, x, out=x)
    z = torch.empty_like(y)
    T = 9
    taps_np, c = ls_model(T)
    tp = pack_taps(taps_np)
    res = {}
    for kappa in (0, 8, 20):
        for init_kind in (("unit",) if kappa == 0 else ("unit", "lowpass")):
            e = np.zeros((M_STEPS, 2 * kappa + 1), np.float32)
            if init_kind == "unit":
                e[:, kappa] = 1.0
            else:
                t = np.arange(-kappa, kappa + 1)
                g = np.exp(-0.5 * (t / (kappa / 4.0)) ** 2)
                e[:] = g / g.sum()
            ed = torch.from_numpy(e).cuda()
            ks = [kappa] * M_STEPS
            ms = time_fn(lambda: api.ldbp_essm_apply(tp, [T] * M_STEPS, c, ed, ks, y, out=z), 20, 3)
            st, _, _ = api.rx(z, sym, pw)
            units = Bw * N_SAMP * M_STEPS
            flops = (8 * T + 9 + 2 * (2 * kappa + 1)) * units
            res[f"kappa{kappa}_{init_kind}"] = {"ms": ms, "samples_steps_per_s": units / (ms / 1e3),
                                                "frac_fp32": flops / (ms / 1e3) / FP32_PEAK_FLOPS,
                                                "snr_db": api.snr_db(st)}
    print(json.dumps({"workload": f"ldbp_essm_{Bw}x{N_SAMP}_M{M_STEPS}_T{T}", "unit": UNIT,
                      "model": "LS-initialised FIR steps (untrained)", **res}))


def train_model(T: int, iters: int, rank: int):
    """Train LDBP on the GPU in the stated training configuration, pruning from T = 31 to T."""
    from paper_2010_14258_gb300.train import Trainer, TrainConfig
    cfg = TrainConfig(batch=64, nsym=16384, n_spans=M_STEPS, span_km=SPAN_KM, channel_steps=CHANNEL_STEPS, ase=True,
                      powers_dbm=tuple(range(-4, 7)), t_start=31, t_end=T, iters=iters, lr=3e-4, lr_final=3e-5,
                      prune_frac=0.5, seed=5 + rank, data_pool=64)
    tr = Trainer(cfg)
    tr.fit()
    out = tr.taps.clone(), list(tr.T), list(tr.c)
    del tr
    return out


def main():
    global B
    args = parse()
    B = args.batch
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2010_14258_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2010_14258_gb300 import api
    import synth

    if args.profile:
        return profile_only(args, api)
    if args.workload == "channel":
        return workload_channel(args, api)
    if args.workload == "ragged":
        return workload_ragged(args, api)
    if args.workload == "train":
        return workload_train(args, api)
    if args.workload == "train_prune":
        return workload_train_prune(args, api)
    if args.workload == "sym32":
        return workload_sym32(args, api)
    if args.workload == "essm":
        return workload_essm(args, api)
    if args.workload == "analog":
        return workload_analog(args, api)

    fib = synth.Fiber()
    t_setup = time.perf_counter()
    # ---- synthetic received waveforms, made on the GPU by the library ----
    s = synth.qam16_symbols(B, NSYM, 2000 + rank).astype(np.complex64)
    sym = torch.from_numpy(s).cuda()
    pw = torch.full((B,), 1e-3 * 10 ** (POWER_DBM / 10), dtype=torch.float32, device="cuda")
    x = api.tx(sym, pw)
    chan = synth.Link(M_STEPS, SPAN_KM, CHANNEL_STEPS, True, True, 5.0, 1.946e14, seed=77 + rank, counter=0)
    y = api.ssm_forward(fib, chan, FS, x, out=x)
    y2 = y.clone()  # a second resident batch: inputs alternate (268 MB > 129 MB L2)
    dbp_link = synth.Link(M_STEPS, SPAN_KM, 1, False, False)
    z = torch.empty_like(y)

    def snr_of(out):
        st, _, _ = api.rx(out, sym, pw)
        return api.snr_db(st)

    api.dbp_apply(fib, dbp_link, FS, y, steps_per_span=1, symmetric=False, out=z)
    snr_dbp = snr_of(z)

    # ---- model: trained T = 7 (pruned from 31), or LS-initialised with --taps ----
    T_head = args.taps or HEAD_T
    if args.taps:
        tl, cl = ls_model(T_head)
        taps, Ts, cs, kind = pack_taps(tl), [T_head] * M_STEPS, cl, "ls_init"
    else:
        tp, Ts, cs = train_model(T_head, args.train_iters, rank)
        taps, kind = tp, "trained"
    api.ldbp_apply(taps, Ts, cs, y, out=z)
    snrs = {T_head: snr_of(z)}
    setup_s = time.perf_counter() - t_setup

    # ---- timed region: K LDBP passes over the resident batch ----
    st = torch.cuda.current_stream()
    xs = [y, y2]

    def step(i):
        api.ldbp_apply(taps, Ts, cs, xs[i % 2], out=z)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as cs_:
        torch.cuda.nvtx.range_push("timed")
        e0.record(st)
        for i in range(args.steps):
            step(i)
        e1.record(st)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    clocks = cs_.summary()
    units = B * N_SAMP * M_STEPS
    ms, value = job_throughput(ms, units, args.steps, world, device="cuda")
    per_launch_s = ms / 1e3 / args.steps
    flops = sum(ldbp_flops_per_sample_step(T) for T in Ts) * B * N_SAMP
    achieved = flops / per_launch_s / 1e12

    # ---- comparisons on the same waveforms (not part of the headline) ----
    reps = max(3, args.steps // 4)
    dbp_ms = time_fn(lambda: api.dbp_apply(fib, dbp_link, FS, y, steps_per_span=1, symmetric=False, out=z), reps)
    cufft_ms = time_fn(lambda: api.ssm_cufft(fib, dbp_link, FS, y, dbp_steps_per_span=1, dbp_symmetric=False,
                                             out=z), reps)
    ls_sweep = {}
    for T in (3, 5, 9, 15):
        tl, cl = ls_model(T)
        tp = pack_taps(tl)
        tms = time_fn(lambda: api.ldbp_apply(tp, [T] * M_STEPS, cl, y, out=z), reps)
        api.ldbp_apply(tp, [T] * M_STEPS, cl, y, out=z)
        ls_sweep[str(T)] = {"samples_steps_per_s": units / (tms / 1e3), "ms": tms, "snr_db": snr_of(z),
                            "frac_fp32": ldbp_flops_per_sample_step(T) * units / (tms / 1e3) / FP32_PEAK_FLOPS}

    # ---- end to end through the C-ABI host-buffer call (pinned host memory) ----
    xh = y.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    ws = torch.empty(api.ldbp_apply_host_workspace(N_SAMP, B), dtype=torch.uint8, device="cuda")
    e2e_ms = time_fn(lambda: api.ldbp_apply_host(taps, Ts, cs, xh, yh, chunks=E2E_CHUNKS, workspace=ws),
                     max(3, args.steps // 4))
    nbytes = xh.numel() * 8

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"ldbp_infer_{B}x{N_SAMP}_M{M_STEPS}", "batch_per_gpu": B, "n": N_SAMP,
                      "M": M_STEPS, "T": T_head, "model": kind, "power_dbm": POWER_DBM,
                      "parallelism": f"replicas{world}",
                      "l2": "two resident input batches alternated (268 MB > 129 MB L2), no flush"},
           "snr": {"ldbp_db": snrs[T_head], "dbp_1stps_db": snr_dbp, "delta_db": snrs[T_head] - snr_dbp,
                   "gate_met": bool(snrs[T_head] >= snr_dbp - 0.1),
                   "training": "64 x 32768 frames, P in -4..6 dBm, 100 StPS + ASE, T 31 -> 7 pruned, "
                               f"{args.train_iters} Adam iterations" if kind == "trained" else "none"},
           "dbp": {"fused_samples_steps_per_s": units / (dbp_ms / 1e3), "fused_ms": dbp_ms,
                   "fused_frac_fp32": DBP_FLOPS_PER_SAMPLE_STEP * units / (dbp_ms / 1e3) / FP32_PEAK_FLOPS,
                   "fused_work": "2*5*log2(n) + 6 + 10 flops per sample-step (two FFTs, spectral multiply, Kerr)",
                   "cufft_samples_steps_per_s": units / (cufft_ms / 1e3), "cufft_ms": cufft_ms,
                   "ldbp_speedup_vs_fused_dbp": dbp_ms / (ms / args.steps),
                   "ldbp_speedup_vs_cufft_dbp": cufft_ms / (ms / args.steps)},
           "ls_init_sweep": ls_sweep,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                        "frac": achieved * 1e12 / FP32_PEAK_FLOPS,
                        "traffic": traffic_from_profiles("ldbp_fwd_kernel", T_head),
                        "kernel": "ldbp_fwd_kernel",
                        "work": "8T+9 flops per sample-step (direct-form FIR + Kerr), T per step",
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz x 2 (FMA = 2 flops); "
                                       "ldbp_ubench measures 3.9e13 FMA/s = 78 TFLOP/s"},
           "clocks": clocks,
           "e2e": {"value": world * units / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes, "call": f"ldbp_apply_host, {E2E_CHUNKS} chunks, pinned host buffers"},
           "gpu_launches": args.steps,
           "setup_s": setup_s}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline_ldbp(T_head)
        cb.pop("seconds", None)
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
