"""Benchmark of the uPDI hot path on GB300.

One step = the whole path over one ensemble: vessel membership -> advection
-> RF synthesis -> rf2iq -> DAS compounding -> SVD clutter filter -> power
Doppler.  The default workload is the 3D volumetric one (32x32 matrix
array, 9 plane-wave tilts, 1536 samples, 500k scatterers in a vessel tree,
100 frames, 128^3 voxels, RF and channel IQ stored in BF16 with FP32
arithmetic); `--workload c2` runs the 2D compounded one (128-element linear
array, 5 plane waves, 2048 samples, 100k scatterers, 200 frames, 256x256
pixels, FP32).

Prints one JSON line.  `value` is channel-samples/s of the whole step
(F * A * M * Ns / step time), summed over ranks; `e2e` is the same metric
through the public API with the scatterer inputs copied from pinned host
memory and the power Doppler image copied back inside the timed region.
`roofline` covers the dominant kernel (RF synthesis, FP32-ALU bound) and
`roofline_das` the DAS kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c3|c2|...]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "channel-samples/s + DAS voxel-angle/s per GB300, % roofline, err vs FP64"
UNIT = "channel-samples/s"
# FP32 work of the model per (scatterer, element, transmit) pair, counted
# from its plain definition: 17 for geometry and amplitude (22 for matrix
# arrays, whose directivity has a second sinc factor), 10 per pulse tap,
# n_cycles * fs / f0 taps on average.
GEOM_FLOP_PER_PAIR = 17.0
GEOM_FLOP_MATRIX_EXTRA = 5.0
FLOP_PER_TAP = 10.0
# FP32 work of DAS per active (voxel, transmit, element) triple: 14 per
# frame (linear interpolation 6, phase rotation 6, accumulation 2) and 20
# for the delay and phase shared by all frames (differences, squares, root,
# transmit path, scale to samples, floor, phase, sine and cosine).
DAS_FLOP_PER_FRAME = 14.0
DAS_FLOP_PER_TRIPLE = 20.0
# DRAM bytes (read + write) of one full-size RF launch per workload, from
# ncu captures of rf_synth_quad_kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); a workload is absent (traffic null) once the
# kernel changes until it is captured again.
RF_TRAFFIC_BYTES = {
    # 3D volumetric, 100 frames, BF16 RF, all 9 transmits per CTA:
    # 689,863,936 read + 2,824,233,472 written
    "c3": 689_863_936 + 2_824_233_472,
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flop per FMA x clock.  The packed f32x2
    # FMA (two lanes per instruction) does not raise this: `--workload
    # alupeak` measures 76.9 TFLOP/s with scalar FFMA and 79.3 with f32x2 at
    # 2070 MHz, i.e. a packed instruction occupies the FMA pipe for two
    # cycles; it saves issue slots, not pipe time.
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------ workloads --
# single-ensemble workloads: storage of the RF, the channel IQ and the
# Casorati matrix (arithmetic is FP32 throughout)
STEP_WORKLOADS = {
    "c3": {"rf": "bfloat16", "ch": "bfloat16", "iq": "float32", "dtype": "bf16"},
    "c2": {"rf": "float32", "ch": "float32", "iq": "float32", "dtype": "f32"},
}


def make_workload(name, seed_offset=0, n_frames=0):
    from paper_2509_05464_gb300 import workload as W
    if name == "c3":
        return W.config3(seed=3 + seed_offset, n_frames=n_frames or 100)
    return W.config2(seed=2 + seed_offset, n_frames=n_frames or 200)


def reduced_workload(name, w):
    """A seeded subset of the workload that the oracle runs through the whole
    path in seconds (for the error of each storage variant)."""
    from paper_2509_05464_gb300 import workload as W
    if name == "c3":
        return W.shrink(W.config3(seed=3, n_frames=16), max_scat=20_000, grid_div=4)
    import dataclasses
    return dataclasses.replace(w, n_frames=6, k_cut=min(w.k_cut, 5))


def das_active_triples(w) -> int:
    """(voxel, transmit, element) triples inside the receive aperture, decided
    as the kernels decide it (binary32 |x_p - x_m| <= z_p / (2 f#), and in y
    for matrix arrays); delays outside the record are not excluded."""
    p, g = w.probe, w.grid
    ex = ((np.arange(p.nx) - 0.5 * (p.nx - 1)) * p.pitch_x).astype(np.float32)
    ey = ((np.arange(p.ny) - 0.5 * (p.ny - 1)) * p.pitch_y).astype(np.float32)
    xs = (g.x0 + np.arange(g.nx) * g.dx).astype(np.float32)
    ys = (g.y0 + np.arange(g.ny) * g.dy).astype(np.float32)
    zs = (g.z0 + np.arange(g.nz) * g.dz).astype(np.float32)
    half = zs * np.float32(0.5 / g.fnumber)
    cx = (np.abs(xs[None, :, None] - ex[None, None, :]) <= half[:, None, None]).sum(-1).astype(np.int64)
    if p.ny > 1:
        cy = (np.abs(ys[None, :, None] - ey[None, None, :]) <= half[:, None, None]).sum(-1).astype(np.int64)
    else:
        cy = np.ones((g.nz, g.ny), np.int64)
    return int(w.A * (cx.sum(1) * cy.sum(1)).sum())


def rf_flop(w) -> float:
    p = w.probe
    geom = GEOM_FLOP_PER_PAIR + (GEOM_FLOP_MATRIX_EXTRA if p.ny > 1 else 0.0)
    return float(w.n_frames) * w.A * w.M * w.S * (geom + FLOP_PER_TAP * p.n_cycles * p.fs / p.f0)


def das_flop(w, triples) -> float:
    return float(triples) * (DAS_FLOP_PER_FRAME * w.n_frames + DAS_FLOP_PER_TRIPLE)


# ---------------------------------------------------------------- oracle --
def oracle_run(w, n_frames):
    """The oracle through the whole path on the first n_frames frames:
    (seconds, results)."""
    import oracle
    from paper_2509_05464_gb300 import workload as W
    st, mt = W.segment_table(w), W.motion_table(w.motion)
    t0 = time.perf_counter()
    r = oracle.pipeline(w, st, mt, n_frames=n_frames, k_cut=min(w.k_cut, n_frames - 1))
    return time.perf_counter() - t0, r


def oracle_sample_3d(w, n_lines=64, block=32, p_svd=16384):
    """The oracle on bounded subsets of a 3D ensemble, each stage timed and
    extrapolated linearly by its exact work count to the whole step:
    membership once; advection of one frame (x F); RF of n_lines (transmit,
    element) lines of frame 0 with every scatterer (x A M F / n_lines);
    rf2iq of those lines; DAS of a block^3 voxel sub-grid at 1 and 9 frames
    (cost a + b F fitted, x P / block^3); the SVD filter of a p_svd x F
    stand-in Casorati matrix (x P / p_svd).  Returns (seconds per step,
    description)."""
    import oracle
    from paper_2509_05464_gb300 import workload as W
    st, mt = W.segment_table(w), W.motion_table(w.motion)
    F, A, M, Ns, P = w.n_frames, w.A, w.M, w.Ns, w.P
    t = {}
    t_start = time.perf_counter()
    c = time.perf_counter()
    _, amp = oracle.classify(w.p0, w.seg, st, len(w.segments), w.amp)
    t["classify"] = time.perf_counter() - c
    c = time.perf_counter()
    pos = oracle.advect(w.p0, w.seg, w.flow, st, mt, 0.0)
    t["advect"] = (time.perf_counter() - c) * F
    a_mid = A // 2
    lines = a_mid * M + np.arange(n_lines)
    c = time.perf_counter()
    rf = oracle.simulate_rf_lines(w.probe, w.tilt_x, w.tilt_y, lines, pos, amp).astype(np.float32)
    t["rf"] = (time.perf_counter() - c) * A * M * F / n_lines
    c = time.perf_counter()
    iq = oracle.rf2iq(w.probe, rf)
    t["rf2iq"] = (time.perf_counter() - c) * A * M * F / n_lines
    g = w.grid
    off = [(n - block) // 2 for n in (g.nx, g.ny, g.nz)]
    sub = W.Grid(block, block if g.ny > 1 else 1, block, g.x0 + off[0] * g.dx, g.y0 + off[1] * g.dy,
                 g.z0 + off[2] * g.dz, g.dx, g.dy, g.dz, g.fnumber)
    ch = np.resize(iq, (A * M, Ns))  # the computed lines stand in for every channel (timing only)
    dt = []
    for nf in (1, 9):
        chf = np.broadcast_to(ch.reshape(1, A, M, Ns), (nf, A, M, Ns)).copy()
        c = time.perf_counter()
        oracle.das(w.probe, w.tilt_x, w.tilt_y, chf, sub)
        dt.append(time.perf_counter() - c)
    b = max(dt[1] - dt[0], 0.0) / 8
    a0 = max(dt[0] - b, 0.0)
    t["das"] = (a0 + b * F) * P / sub.n_pixels
    rng = np.random.default_rng(0)
    S = rng.standard_normal((p_svd, F)) + 1j * rng.standard_normal((p_svd, F))
    c = time.perf_counter()
    oracle.svd_filter(S, w.k_cut, w.energy_thresh)
    t["svd_pd"] = (time.perf_counter() - c) * P / p_svd
    measured = time.perf_counter() - t_start
    total = sum(t.values())
    desc = (f"FP64 oracle on bounded subsets, each stage extrapolated linearly by its work count: membership "
            f"of all {w.S} scatterers, advection of 1 of {F} frames, RF of {n_lines} of {A * M} (transmit, "
            f"element) lines of frame 0 with every scatterer, rf2iq of those lines, DAS of a {block}^3 voxel "
            f"block at 1 and 9 frames (a + b F fit), the SVD filter of a {p_svd} x {F} random stand-in; "
            f"{measured:.1f} s measured; extrapolated stage seconds "
            + json.dumps({k: round(v, 1) for k, v in t.items()}))
    return total, desc


def cpu_baseline(name, w):
    """The oracle as it stands on the host cores: (cpu_baseline dict, oracle
    results of the reduced workload or None)."""
    import oracle
    if name == "c3":
        sec, desc = oracle_sample_3d(w)
        cs = w.n_frames * w.A * w.M * w.Ns
        return {"value": cs / sec, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                "sample": desc}
    n_frames = 6
    dt, _ = oracle_run(w, n_frames)
    cs = n_frames * w.A * w.M * w.Ns
    return {"value": cs / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"whole path (advect, membership, RF, rf2iq, DAS, SVD filter, PD) on the first {n_frames} "
                      f"of {w.n_frames} frames of the same workload, FP64, {dt:.1f} s"}


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# Storage variants of the path: (name, RF, channel IQ, Casorati, Gram)
VARIANTS = [("f32", "float32", "float32", "float32", "f32"),
            ("f16", "float16", "float16", "float32", "f32"),
            ("bf16", "bfloat16", "bfloat16", "float32", "f32"),
            ("f32+tf32_gram", "float32", "float32", "float32", "tf32"),
            ("bf16_all", "bfloat16", "bfloat16", "bfloat16", "bf16")]


def variant_kwargs(rf_t, ch_t, iq_t, gm):
    import torch
    from paper_2509_05464_gb300 import fq
    gmode = {"f32": fq.FQ_GRAM_F32, "tf32": fq.FQ_GRAM_TF32, "bf16": fq.FQ_GRAM_BF16}
    return dict(rf_dtype=getattr(torch, rf_t), ch_dtype=getattr(torch, ch_t), iq_dtype=getattr(torch, iq_t),
                gram_mode=gmode[gm])


STAGES = ("classify", "advect", "simulate", "rf2iq", "das", "clutter")


def time_steps(pl, steps, flush=None):
    """Device time of `steps` whole steps on the current stream, with events
    between the stages: (mean ms per step, mean ms per stage)."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)] for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        if flush is not None:
            flush.zero_()  # L2 flush outside the timed events
        ev[i][0].record(stream)
        for j, name in enumerate(STAGES):
            getattr(pl, name)()
            ev[i][j + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[-1]) for e in ev]
    stage_ms = {name: sum(e[j].elapsed_time(e[j + 1]) for e in ev) / steps for j, name in enumerate(STAGES)}
    return sum(step_ms) / steps, stage_ms


def variant_errors(w_small, ref, kw):
    """Errors of one storage variant against the FP64 oracle on the reduced
    workload: RF, Casorati IQ and PD relative L2."""
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300.pipeline import Pipeline
    ps = Pipeline(w_small, **kw)
    ps.upload()
    ps.step()
    fq.fq_clutter_status(ps.ws_svd)
    pd = ps.download().numpy().copy()
    rf = ps.rf.float().cpu().numpy()
    iq = ps.iq.float().cpu().numpy()
    del ps
    S_ref = ref["S"]
    return {"rf_rel_l2": rel_l2(rf, ref["rf"]),
            "iq_rel_l2": rel_l2(np.stack([iq[..., 0], iq[..., 1]]), np.stack([S_ref.real, S_ref.imag])),
            "pd_rel_l2": rel_l2(pd, ref["pd"])}


def precision_variants(w, w_small, ref, steps, warmup):
    """Each storage variant on the full workload (device-timed steps) and its
    error against the FP64 oracle on the reduced workload."""
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300.pipeline import Pipeline
    out = []
    for name, rf_t, ch_t, iq_t, gm in VARIANTS:
        kw = variant_kwargs(rf_t, ch_t, iq_t, gm)
        pl = Pipeline(w, **kw)
        pl.upload()
        for _ in range(warmup):
            pl.step()
        ms, stage = time_steps(pl, steps)
        fq.fq_clutter_status(pl.ws_svd)
        del pl
        torch.cuda.empty_cache()
        err = variant_errors(w_small, ref, kw) if ref is not None else None
        out.append({"variant": name, "rf": rf_t, "channel_iq": ch_t, "casorati": iq_t, "gram": gm,
                    "steps": steps, "ms_per_step": ms, "stage_ms": stage, "err_vs_fp64": err})
        torch.cuda.empty_cache()
    return out


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, each step a bounded sample of the
    workload extrapolated to the whole step (3D) or the whole path on the
    first 2 frames (2D)."""
    import oracle
    if rank != 0:
        return
    name = args.workload if args.workload in STEP_WORKLOADS else "c3"
    w = make_workload(name, 0, args.frames)
    if name == "c3":
        def one():
            return oracle_sample_3d(w, n_lines=32, block=24, p_svd=8192)
        cs = w.n_frames * w.A * w.M * w.Ns
    else:
        nf = 2

        def one():
            return oracle_run(w, nf)[0], f"each step: the whole path on the first {nf} of {w.n_frames} frames"
        cs = nf * w.A * w.M * w.Ns
    for _ in range(args.warmup):
        one()
    res = [one() for _ in range(args.steps)]
    t = sum(r[0] for r in res) / len(res)
    v = cs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": oracle.num_threads(),
                             "sample": res[-1][1]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours --
def run_ours(args, rank, world, local):
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300.pipeline import Pipeline

    torch.cuda.set_device(local)
    fq.lib()
    name = args.workload
    spec = STEP_WORKLOADS[name]
    w = make_workload(name, rank, args.frames)  # an independent ensemble per rank (weak scaling)
    if args.scatterers or args.grid_div:  # reduced cases for profiler captures only
        from paper_2509_05464_gb300 import workload as W
        w = W.shrink(w, max_scat=args.scatterers or None, grid_div=args.grid_div or None)
    gram = args.gram or "f32"
    kw = variant_kwargs(spec["rf"], spec["ch"], spec["iq"], gram)
    pl = Pipeline(w, **kw)
    pl.upload()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        pl.step()
    torch.cuda.synchronize()
    fq.fq_clutter_status(pl.ws_svd)

    clk = ClockSampler(local)
    clk.start()
    barrier()
    ms_local, stage_ms = time_steps(pl, args.steps, flush)
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(ms_local)

    # end to end through the public API (pinned host in, PD out)
    e2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        e2[i][0].record(stream)
        pl.step_e2e()
        e2[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2) / args.steps)
    fq.fq_clutter_status(pl.ws_svd)

    n_launches, h2d_bytes, d2h_bytes = pl.n_launches, pl.h2d_bytes, pl.d2h_bytes
    total_cs = sum_over_ranks(float(pl.channel_samples))
    total_va = sum_over_ranks(float(pl.voxel_angles))
    if rank != 0:
        return
    pk, src = peaks()
    sm_for_peak = float(pk.get("sm_max_mhz", 2070.0))
    peak = fp32_alu_peak_tflops(sm_for_peak)
    peak_src = (f"152 SMs x 128 FP32 lanes x 2 (FMA) x {sm_for_peak:.0f} MHz "
                f"({src} max clock)")
    p = w.probe
    taps = p.n_cycles * p.fs / p.f0
    pairs = float(w.n_frames) * w.A * w.M * w.S
    flop = rf_flop(w)
    rf_ms = stage_ms["simulate"]
    achieved = flop / (rf_ms * 1e-3) / 1e12
    triples = das_active_triples(w)
    dflop = das_flop(w, triples)
    das_ms = stage_ms["das"]
    d_ach = dflop / (das_ms * 1e-3) / 1e12
    full = args.frames == 0 and not (args.scatterers or args.grid_div)
    traffic = RF_TRAFFIC_BYTES.get(name) if full else None
    cpu = None
    if args.cpu_baseline:
        cpu = cpu_baseline(name, w)
    variants, err = None, None
    if args.variants:
        import oracle
        from paper_2509_05464_gb300 import workload as W
        w_small = reduced_workload(name, w)
        st, mt = W.segment_table(w_small), W.motion_table(w_small.motion)
        t0 = time.perf_counter()
        ref = oracle.pipeline(w_small, st, mt)
        ref_s = time.perf_counter() - t0
        del pl, flush
        torch.cuda.empty_cache()
        vsteps = args.variant_steps or (4 if name == "c3" else 20)
        variants = precision_variants(w, w_small, ref, steps=vsteps, warmup=2)
        err = next(v["err_vs_fp64"] for v in variants
                   if (v["rf"], v["channel_iq"], v["casorati"], v["gram"]) == (spec["rf"], spec["ch"], spec["iq"], gram))
        err = dict(err, reduced_workload=w_small.name, oracle_s=round(ref_s, 1))
    stor = f"RF {spec['rf']}, channel IQ {spec['ch']}, Casorati {spec['iq']}, Gram {gram}, FP32 arithmetic"
    line = {
        "metric": METRIC, "value": total_cs / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": spec["dtype"], "data": "synthetic",
        "config": {"workload": w.name, "frames": w.n_frames, "angles": w.A, "elements": w.M, "samples": w.Ns,
                   "scatterers": w.S, "voxels": w.P, "storage": stor,
                   "parallelism": f"independent ensemble per GPU x{world}",
                   "l2": "256 MiB buffer rewritten between timed steps, outside the timed events"},
        "das_voxel_angle_per_s": total_va / (ms * 1e-3),
        "das_voxel_angle_per_s_das_kernel": total_va / (das_ms * 1e-3),
        "stage_ms": stage_ms,
        "roofline": {"bound": "alu", "kernel": "rf_synth_quad_kernel", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_src,
                     "work": f"{flop / pairs:.2f} FLOP per (scatterer, element, transmit, frame) pair "
                             f"({taps:.3f} taps), {pairs:.3e} pairs"},
        "roofline_das": {"bound": "alu",
                         "kernel": "das_kernel" if kw["ch_dtype"] == torch.float32 else "das_w_kernel",
                         "achieved": d_ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": d_ach / peak, "traffic": None, "peak_source": peak_src,
                         "work": f"{DAS_FLOP_PER_FRAME:.0f} FLOP per frame + {DAS_FLOP_PER_TRIPLE:.0f} per active "
                                 f"(voxel, transmit, element) triple, {triples:.4e} triples x {w.n_frames} frames",
                         "hbm_gbs_algorithmic": (w.A * w.M * w.Ns * fq.frame_pad(w.n_frames) * 2
                                                 * torch.empty((), dtype=kw["ch_dtype"]).element_size()
                                                 + w.P * w.n_frames * 2
                                                 * torch.empty((), dtype=kw["iq_dtype"]).element_size())
                                                / (das_ms * 1e-3) / 1e9},
        "cpu_baseline": cpu,
        "e2e": {"value": total_cs / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": d2h_bytes, "ms_per_step": e2e_ms},
        "err_vs_fp64": err,
        "precision_variants": variants,
        "gpu_launches": n_launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------- batched (uneven C4) --
def run_batched(args, rank, world, local):
    """The 64-ensemble uneven batch through the persistent per-stage kernels
    under a captured CUDA graph, tiles from the autotuner."""
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300 import workload as W
    from paper_2509_05464_gb300.pipeline import Pipeline

    torch.cuda.set_device(local)
    fq.lib()
    ms = W.config4(seed=1000 + 64 * rank)  # an independent batch per rank (weak scaling)
    b = fq.Batch(ms, max_arena_bytes=args.arena_gb << 30)
    cost = [w.n_frames * w.A * w.M * w.S for w in ms]
    big = int(np.argmax(cost))
    tiles = {}
    for op, name in ((fq.FQ_OP_RF, "rf_resident_warps_per_sm"), (fq.FQ_OP_DAS, "das_threads")):
        c = fq.fq_autotune(op, b, big)
        b.set_tile(c)
        tiles[name] = {"choice": c.choice, "tried": list(c.tried[:c.n_tried]),
                       "tried_ms": [round(x, 3) for x in c.tried_ms[:c.n_tried]]}
    torch.cuda.empty_cache()
    n_waves, items = b.info()
    b.launch()
    b.status()
    evs = b.launch_profiled()
    torch.cuda.synchronize()
    b.status()
    stage_ms = {st: 0.0 for st in fq.STAGES}
    for wv in range(n_waves):
        for j, st in enumerate(fq.STAGES):
            stage_ms[st] += evs[wv * 9 + j].elapsed_time(evs[wv * 9 + j + 1])
    b.capture()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.graph_launch()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        b.graph_launch()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    b.status()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps)

    # end to end: pinned host inputs copied in, PD images copied out, every step
    h_in = [[t.cpu().pin_memory() for t in ins] for ins in b.inputs]
    h_pd = [p.cpu().pin_memory() for p in b.pd]
    h2d = sum(t.numel() * t.element_size() for ins in h_in for t in ins)
    d2h = sum(t.numel() * t.element_size() for t in h_pd)
    e2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e2[0].record(stream)
    for _ in range(args.steps):
        for hs, ds in zip(h_in, b.inputs):
            for h, d in zip(hs, ds):
                d.copy_(h, non_blocking=True)
        b.graph_launch()
        for h, d in zip(h_pd, b.pd):
            h.copy_(d, non_blocking=True)
        stream.synchronize()
    e2[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e2[0].elapsed_time(e2[1]) / args.steps)

    # the same ensembles one by one through the single-ensemble calls
    seq_ms = 0.0
    if args.sequential:
        b.close()
        del b
        torch.cuda.empty_cache()
        for w in ms:
            pl = Pipeline(w)
            pl.upload()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pl.step()
            z.record(stream)
            torch.cuda.synchronize()
            seq_ms += a.elapsed_time(z)
            del pl
            torch.cuda.empty_cache()
    cs = float(sum(w.n_frames * w.A * w.M * w.Ns for w in ms))
    total_cs = sum_over_ranks(cs)
    if rank != 0:
        return
    pk, src = peaks()
    sm_for_peak = float(pk.get("sm_max_mhz", 2070.0))
    peak = fp32_alu_peak_tflops(sm_for_peak)
    pairs = float(sum(w.n_frames * w.A * w.M * w.S for w in ms))
    taps = sum(w.n_frames * w.A * w.M * w.S * w.probe.n_cycles * w.probe.fs / w.probe.f0 for w in ms) / pairs
    flop = pairs * (GEOM_FLOP_PER_PAIR + FLOP_PER_TAP * taps)
    achieved = flop / (stage_ms["rf"] * 1e-3) / 1e12
    launches = sum(1 for st in fq.STAGES if items[st] > 0) * n_waves
    line = {
        "metric": METRIC, "value": total_cs / (ms_step * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "C4 uneven batch: 64 ensembles, S 10k-300k log-uniform, F 50-400, "
                               "grids 128^2..96^3, C1/C2 probes",
                   "ensembles": len(ms), "waves": n_waves, "arena_gb": round(b_arena_gb(ms, args), 1),
                   "graph": True, "tiles": tiles, "items": items,
                   "parallelism": f"independent batch per GPU x{world}",
                   "l2": "no flush: every stage's working set is several GB, far above L2"},
        "stage_ms": stage_ms,
        "sequential_ms": seq_ms if args.sequential else None,
        "batched_speedup_vs_sequential": (seq_ms / ms_step) if args.sequential else None,
        "roofline": {"bound": "alu", "kernel": "rf_quad_batched_kernel", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 (FMA) x {sm_for_peak:.0f} MHz "
                                    f"({src} max clock)",
                     "work": f"{GEOM_FLOP_PER_PAIR:.0f} + {FLOP_PER_TAP:.0f} x {taps:.3f} taps FLOP per pair, "
                             f"{pairs:.3e} pairs"},
        "cpu_baseline": None,
        "e2e": {"value": total_cs / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------ learned clutter filter (C5) --
def run_cnn(args, rank, world, local):
    """Training throughput and held-out PD quality of the learned filter on
    GPU-simulated C1-like ensembles, and inference on a 200-frame 256x256
    ensemble of the benchmark workload."""
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300 import learned
    from paper_2509_05464_gb300 import workload as W
    from paper_2509_05464_gb300.pipeline import Pipeline

    torch.cuda.set_device(local)
    fq.lib()
    n_ens = args.cnn_ensembles
    n_test = max(2, n_ens // 8)
    seeds = list(range(10000 + rank * 100000, 10000 + rank * 100000 + n_ens))
    t0 = time.perf_counter()
    vol, tgt, scales, pd_gt, pd_svd = learned.ensembles(seeds, target_gain=args.cnn_gain)
    gen_s = time.perf_counter() - t0
    n_tr = n_ens - n_test
    F, Z, X = vol.shape[1:4]
    batch = 4
    learned.train(fq.CNN(0), vol[:n_tr], tgt[:n_tr], steps=max(1, args.warmup), batch=batch, lr=args.cnn_lr, seed=1)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    net, init, hist, tries = learned.fit(vol[:n_tr], tgt[:n_tr], steps=args.cnn_train_steps, batch=batch,
                                         lr=args.cnn_lr, seed=2, log_every=max(1, args.cnn_train_steps // 10))
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / (args.cnn_train_steps * len(tries))
    held = slice(n_tr, n_ens)
    pd_cnn = learned.predict_pd(net, vol[held], scales[n_tr:], args.cnn_gain)
    inv = torch.tensor([1.0 / (s * s) for s in scales[n_tr:]], device=vol.device)[:, None]
    raw = (vol[held, ..., :2].float() ** 2).sum(-1).mean(1).reshape(n_test, -1) * inv  # after mean removal
    quality = {"pd_rel_l2_cnn": learned.rel_l2(pd_cnn, pd_gt[held]),
               "pd_rel_l2_svd_k2": learned.rel_l2(pd_svd[held], pd_gt[held]),
               "pd_rel_l2_unfiltered": learned.rel_l2(raw, pd_gt[held]),
               "held_out_ensembles": n_test}

    # inference on the benchmark ensemble (200 frames, 256 x 256 pixels)
    w = W.config2(n_frames=args.cnn_infer_frames)
    pl = Pipeline(w)
    pl.upload()
    pl.step()
    Fi, Zi, Xi = w.n_frames, w.grid.nz, w.grid.nx
    vin = torch.empty((1, Fi, Zi, Xi, 32), dtype=torch.bfloat16, device="cuda")
    _, _, sc = fq.fq_cnn_from_casorati(pl.iq, Fi, Zi, Xi, True, vol=vin[0])
    scale = float(sc.item()) * args.cnn_gain
    del pl
    torch.cuda.empty_cache()
    acts = fq.cnn_act_workspace(1, Fi, Zi, Xi)
    for _ in range(max(1, args.warmup)):
        fq.fq_cnn_forward(net, vin, acts)
    clk = ClockSampler(local)
    clk.start()
    e0.record(stream)
    for _ in range(args.steps):
        fq.fq_cnn_forward(net, vin, acts)
        pd = fq.fq_cnn_power_doppler(fq.cnn_output(acts, 1, Fi, Zi, Xi)[0], scale)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    assert int(net.status.item()) == 0, "a bounded wait in a convolution ran out"
    inf_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    V = Fi * Zi * Xi
    mac_true = sum(45 * a * b for a, b in zip(fq.CNN_CHANNELS[:-1], fq.CNN_CHANNELS[1:]))
    mac_exec = 4 * 45 * 32 * 32
    pk, src = peaks()
    peak = float(pk.get("bf16_tflops", 1900.0))
    ach = 2.0 * mac_true * V / (inf_ms * 1e-3) / 1e12
    total_v = sum_over_ranks(float(V))
    if rank != 0:
        return
    line = {
        "metric": "CNN clutter-filter inference voxel-frames/s (4 x 3D conv, 5x3x3, 32 ch, BF16/FP32)",
        "value": total_v / (inf_ms * 1e-3), "unit": "voxel-frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": inf_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"C5 learned filter: inference on {Fi} x {Zi} x {Xi} (C2 ensemble); training on "
                               f"{n_tr} C1-like 64 x 32 x 32 ensembles, batch {batch}",
                   "train_ms_per_step": train_ms, "train_voxels_per_s": batch * F * Z * X / (train_ms * 1e-3),
                   "train_loss": hist, "train_attempts": [{"init": t[0], "first_loss": t[1], "last_loss": t[2]}
                                                           for t in tries],
                   "data_generation_s": gen_s,
                   "l2": "inference working set (activations 0.84 GB per layer) far above L2"},
        "quality": quality,
        "roofline": {"bound": "tensor", "kernel": "conv_ring_kernel", "achieved": ach, "peak": peak,
                     "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                     "peak_source": f"bf16_tflops of {src} peaks (cuBLAS burst)",
                     "work": f"2 x {mac_true} MAC per voxel (the 2-32-32-32-2 network); the kernels execute "
                             f"{mac_exec} (2-channel ends padded to 32)"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": 5 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------- gridded-field advection (Sec. 2.2.2) --
# FP32 operations of one RK4 step as defined: four trilinear evaluations
# (grid coordinates 3 x 2, seven lerps per component 7 x 3 x 2 = 42), the
# three stage points (3 x 3 x 2 = 18) and the weighted sum (3 x 7 = 21)
FIELD_FLOP_PER_STEP = 4 * (6 + 42) + 18 + 21


def run_field(args, rank, world, local):
    """Trajectories of the C2 medium in a gridded steady velocity field
    (RK4, lumen confinement of the blood) for a 200-frame ensemble."""
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300 import workload as W

    torch.cuda.set_device(local)
    fq.lib()
    fw = W.field_c2(seed=2 + rank, n_frames=args.frames or 200)
    h_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (fw.p0, fw.seg, fw.v)]
    p0, seg, v = (t.to("cuda") for t in h_in)
    pos = torch.empty((fw.n_frames, 3, fw.S), dtype=torch.float32, device="cuda")
    h_pos = torch.empty(pos.shape, dtype=torch.float32).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        fq.fq_advect_field(p0, seg, fw.segments, fw.origin, fw.spacing, v, fw.dt, fw.n_sub, fw.n_frames,
                           pos_out=pos)

    for _ in range(args.warmup):
        step()
    clk = ClockSampler(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / args.steps)
    # end to end: inputs from pinned host memory, every position back
    e2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in e2:
        flush.zero_()
        a.record(stream)
        for d, hsrc in zip((p0, seg, v), h_in):
            d.copy_(hsrc, non_blocking=True)
        step()
        h_pos.copy_(pos, non_blocking=True)
        b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2) / args.steps)
    got = pos.cpu().numpy()
    units = float(fw.n_frames * fw.S)
    total = sum_over_ranks(units)
    if rank != 0:
        return
    # parity on a sample of scatterers (every 97th) against the oracle
    import oracle
    idx = np.arange(0, fw.S, 97)
    want = oracle.advect_field(np.ascontiguousarray(fw.p0[:, idx]), np.ascontiguousarray(fw.seg[idx]),
                               W.segment_table(fw), len(fw.segments), fw.v, fw.origin, fw.spacing, fw.dt,
                               fw.n_sub, fw.n_frames)
    d = np.abs(got[:, :, idx].astype(np.float64) - want.astype(np.float64))
    ulps = d / float(np.spacing(np.float32(np.abs(want).max())))  # in ulps of the largest coordinate
    cpu = None
    if args.cpu_baseline:
        t0 = time.perf_counter()
        oracle.advect_field(fw.p0, fw.seg, W.segment_table(fw), len(fw.segments), fw.v, fw.origin, fw.spacing,
                            fw.dt, fw.n_sub, fw.n_frames)
        dt_cpu = time.perf_counter() - t0
        cpu = {"value": units / dt_cpu, "unit": "positions/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"the whole workload ({fw.S} scatterers x {fw.n_frames} frames, FP64), {dt_cpu:.1f} s"}
    steps = (fw.n_frames - 1) * fw.n_sub * fw.S  # RK4 steps (frame 0 is p0)
    pk, src = peaks()
    sm_for_peak = float(pk.get("sm_max_mhz", 2070.0))
    peak = fp32_alu_peak_tflops(sm_for_peak)
    ach = steps * FIELD_FLOP_PER_STEP / (ms * 1e-3) / 1e12
    line = {
        "metric": "scatterer positions/s (steady gridded velocity field, RK4, lumen confinement)",
        "value": total / (ms * 1e-3), "unit": "positions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": fw.name, "scatterers": fw.S, "frames": fw.n_frames, "rk4_steps_per_frame": fw.n_sub,
                   "field_samples": int(np.prod(fw.v.shape[:3])),
                   "parallelism": f"independent ensemble per GPU x{world}",
                   "l2": "256 MiB buffer rewritten between timed steps, outside the timed events"},
        "parity": {"sampled_scatterers": int(idx.size), "max_abs_m": float(d.max()),
                   "max_ulps_of_largest_coordinate": float(ulps.max()),
                   "frac_over_2_ulps": float((ulps > 2).any(axis=(0, 1)).mean())},
        "roofline": {"bound": "alu", "kernel": "advect_field_kernel", "achieved": ach, "peak": peak,
                     "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 (FMA) x {sm_for_peak:.0f} MHz "
                                    f"({src} max clock)",
                     "work": f"{FIELD_FLOP_PER_STEP} FLOP per RK4 step, {steps:.3e} steps"},
        "cpu_baseline": cpu,
        "e2e": {"value": total / (e2e_ms * 1e-3), "unit": "positions/s",
                "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in h_in)),
                "d2h_bytes_per_step": int(h_pos.numel() * 4), "ms_per_step": e2e_ms},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------ display and quality (Sec. 5.2-5.3) --
def run_post(args, rank, world, local):
    """B-mode and uPDI display of the C2 ensemble, MIPs of a 128^3 volume
    and the quality metrics of the uPDI image against the blood-only
    ground truth."""
    import copy
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300 import workload as W
    from paper_2509_05464_gb300.pipeline import Pipeline

    torch.cuda.set_device(local)
    fq.lib()
    w = W.config2(seed=2 + rank, n_frames=args.frames or 200)
    pl = Pipeline(w)
    pl.upload()
    pl.step()
    pd = pl.pd.clone()
    iq = pl.iq
    wb = copy.deepcopy(w)
    wb.amp = wb.amp.copy()
    wb.amp[wb.seg < 0] = 0.0
    pb = Pipeline(wb, keep_iq_f=False)
    pb.upload()
    pb.step()
    b = pb.iq.double()
    pd_gt = ((b[..., 0] ** 2 + b[..., 1] ** 2).mean(dim=1)).float()
    del pb
    torch.cuda.empty_cache()
    H, Wd = w.grid.nz, w.grid.nx
    rng = np.random.default_rng(7)
    vol = torch.from_numpy(rng.lognormal(0.0, 1.5, (128, 128, 128)).astype(np.float32)).cuda()
    ws = fq.post_workspace(H, Wd)
    bm = torch.empty(w.P, dtype=torch.float32, device="cuda")
    disp = torch.empty_like(bm)
    disp_gt = torch.empty_like(bm)
    mips = [torch.empty(s, dtype=torch.float32, device="cuda") for s in ((128, 128),) * 3]
    q = torch.empty(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        fq.fq_bmode(iq, 0, 75.0, out=bm, ws=ws)
        fq.fq_log_compress(pd, 60.0, power=True, out=disp, ws=ws)
        fq.fq_log_compress(pd_gt, 60.0, power=True, out=disp_gt, ws=ws)
        for a in range(3):
            fq.fq_mip(vol, a, out=mips[a])
        fq.fq_image_quality(disp.view(H, Wd), disp_gt.view(H, Wd), out=q, ws=ws)

    for _ in range(max(args.warmup, 1)):
        step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clk = ClockSampler(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for a, bb in ev:
        flush.zero_()
        a.record(stream)
        step()
        bb.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(sum(a.elapsed_time(bb) for a, bb in ev) / args.steps)
    # bytes each step reads and writes (algorithmic): B-mode reads one frame
    # of S (8 B per pixel, strided) twice (max, compress) and writes 4 B;
    # each display reads 4 B twice and writes 4 B; the MIPs read the volume
    # three times and write three planes; the metrics read both images twice
    P, V = w.P, 128 ** 3
    nbytes = P * (8 * 2 + 4) + 2 * P * (4 * 2 + 4) + 3 * (V * 4) + 3 * 128 * 128 * 4 + 2 * P * 4 * 2
    pixels = sum_over_ranks(float(3 * P + V))
    if rank != 0:
        return
    qh = q.cpu().numpy()
    # parity: the metrics against the oracle on the same display images
    from oracle import post as opost
    dh, gh = disp.cpu().numpy().reshape(H, Wd), disp_gt.cpu().numpy().reshape(H, Wd)
    want = (opost.mse(dh, gh), opost.psnr(dh, gh), opost.ssim(dh, gh))
    pk, src = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))
    ach = nbytes / (ms * 1e-3) / 1e9
    line = {
        "metric": "display + quality pixels/s (B-mode, uPDI 60 dB, 3 MIPs of 128^3, MSE/PSNR/SSIM)",
        "value": pixels / (ms * 1e-3), "unit": "pixels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"C2 ensemble ({H} x {Wd} px, {w.n_frames} frames): B-mode of frame 0 (75 dB), "
                               f"uPDI display (60 dB) of the SVD PD and the blood-only PD, their MSE/PSNR/SSIM; "
                               f"MIPs along x, y, z of a 128^3 lognormal volume",
                   "l2": "256 MiB buffer rewritten between timed steps, outside the timed events"},
        "quality_vs_blood_only": {"mse": float(qh[0]), "psnr_db": float(qh[1]), "ssim": float(qh[2]),
                                  "oracle": {"mse": want[0], "psnr_db": want[1], "ssim": want[2]}},
        "roofline": {"bound": "hbm", "kernel": "all display / quality kernels of the step", "achieved": ach,
                     "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                     "peak_source": f"hbm_gbs of {src} peaks",
                     "work": f"{nbytes / 1e6:.1f} MB algorithmic per step (11 launches: launch-bound at these sizes)"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": 11 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------ the paper's DAS-matrix route (Alg. 3) --
def run_das_matrix(args, rank, world, local):
    """Explicit per-transmit DAS matrices (build once, apply to all frames)
    against the fused DAS kernel on the C2 ensemble."""
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300 import workload as W
    from paper_2509_05464_gb300.pipeline import Pipeline

    torch.cuda.set_device(local)
    fq.lib()
    w = W.config2(seed=2 + rank, n_frames=args.frames or 200)
    pl = Pipeline(w)
    pl.upload()
    pl.classify()
    pl.advect()
    pl.simulate()
    F, A, M = w.n_frames, w.A, w.M
    ch = fq.fq_rf2iq(w.probe, A * M, F, pl.rf)
    del pl
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    t0 = time.perf_counter()
    dm = fq.DasMatrix(w.probe, w.tilt_x, w.tilt_y, w.grid)
    torch.cuda.synchronize()
    build_wall_ms = (time.perf_counter() - t0) * 1e3
    build_ms = timed(lambda: fq.DasMatrix(w.probe, w.tilt_x, w.tilt_y, w.grid), 2)
    iq_m = torch.empty((w.P, F, 2), dtype=torch.float32, device="cuda")
    iq_f = torch.empty_like(iq_m)
    clk = ClockSampler(local)
    clk.start()
    apply_ms = max_over_ranks(timed(lambda: dm.apply(ch, F, iq=iq_m), args.steps))
    fused_ms = max_over_ranks(timed(lambda: fq.fq_das(w.probe, w.tilt_x, w.tilt_y, ch, F, w.grid, iq=iq_f),
                                    args.steps))
    clocks = clk.stop()
    diff = float(torch.linalg.norm(iq_m - iq_f) / torch.linalg.norm(iq_f))
    va = float(F * A * w.P)
    total = sum_over_ranks(va)
    if rank != 0:
        return
    pk, src = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))
    # algorithmic bytes of one apply: the matrices once (12 B per entry +
    # offsets) and the channel IQ once (the rows the entries touch), the
    # Casorati written
    nbytes = dm.nbytes + ch.numel() * 4 + w.P * F * 8
    ach = nbytes / (apply_ms * 1e-3) / 1e9
    line = {
        "metric": "DAS voxel-angle/s, explicit DAS matrices (Alg. 3) vs the fused kernel",
        "value": total / (apply_ms * 1e-3), "unit": "voxel-angles/s", "n_gpus": world, "steps": args.steps,
        "warmup": 1, "ms_per_step": apply_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{w.name}: {A} transmits x {M} elements x {w.P} pixels x {F} frames",
                   "nnz": dm.nnz, "matrix_bytes": dm.nbytes, "build_ms": build_ms,
                   "first_build_wall_ms": build_wall_ms,
                   "l2": "inputs (channel IQ 2.2 GB) far above L2"},
        "fused_das": {"ms": fused_ms, "value": total / (fused_ms * 1e-3),
                      "matrix_vs_fused_rel_l2": diff,
                      "break_even_ensembles": build_ms / max(fused_ms - apply_ms, 1e-9) if fused_ms > apply_ms
                      else None},
        "roofline": {"bound": "hbm", "kernel": "apply_kernel", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "traffic": None, "peak_source": f"hbm_gbs of {src} peaks",
                     "work": f"{nbytes / 1e9:.2f} GB algorithmic per apply (matrices + channel IQ + Casorati)"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------ frequency-domain RF (Alg. 2) --
def run_rf_freq(args, rank, world, local):
    """Eq. 1 per frequency (the paper's frequency loop) against the
    time-domain kernel on the C2 ensemble, a few frames."""
    import torch
    from paper_2509_05464_gb300 import fq
    from paper_2509_05464_gb300 import workload as W
    from paper_2509_05464_gb300.pipeline import Pipeline

    torch.cuda.set_device(local)
    fq.lib()
    F = args.frames or 2
    w = W.config2(seed=2 + rank, n_frames=F)
    pl = Pipeline(w)
    pl.upload()
    pl.classify()
    pl.advect()
    pop = pl.pops[0]
    pos, amp = pop.pos, pop.amp_eff
    stream = torch.cuda.current_stream()
    rf_t = torch.empty((F, w.A, w.M, w.Ns), dtype=torch.float32, device="cuda")
    rf_f = torch.empty_like(rf_t)
    n_fft = 2 * w.Ns

    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    clk = ClockSampler(local)
    clk.start()
    freq_ms = max_over_ranks(timed(lambda: fq.fq_simulate_rf_freq(w.probe, w.tilt_x, w.tilt_y, pos, amp, F,
                                                                  n_fft=n_fft, rf=rf_f), args.steps))
    time_ms = max_over_ranks(timed(lambda: fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos, amp, F, rf=rf_t),
                                   args.steps))
    clocks = clk.stop()
    cs = float(F * w.A * w.M * w.Ns)
    total = sum_over_ranks(cs)
    if rank != 0:
        return
    # parity against the oracle on a sample: the first 2000 scatterers of
    # frame 0, transmit 2, every element (the oracle's cost is S x M x bins)
    import oracle
    ns_s = 2000
    p1 = np.ascontiguousarray(pos[0, :, :ns_s].cpu().numpy())
    a1 = np.ascontiguousarray(amp[:ns_s].cpu().numpy())
    sub = fq.fq_simulate_rf_freq(w.probe, w.tilt_x[2:3], w.tilt_y[2:3],
                                 torch.from_numpy(p1[None]).cuda(), torch.from_numpy(a1).cuda(), 1, n_fft=n_fft)
    t0 = time.perf_counter()
    want = oracle.simulate_rf_freq(w.probe, w.tilt_x[2:3], w.tilt_y[2:3], p1, a1, n_fft=n_fft)
    oracle_s = time.perf_counter() - t0
    got = sub[0].cpu().numpy()
    err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    td_vs_fd = float(torch.linalg.norm(rf_f - rf_t) / torch.linalg.norm(rf_t))
    # Eq. 1's transmit sum over all 128 elements and Eq. 2's sub-elements
    # (2 per element), on the first 10000 scatterers of frame 0, every
    # transmit; parity against the oracle on 200 of them, transmit 2
    n_tx = 10_000
    ptx = torch.from_numpy(np.ascontiguousarray(pos[0, :, :n_tx].cpu().numpy())[None]).cuda()
    atx = torch.from_numpy(np.ascontiguousarray(amp[:n_tx].cpu().numpy())).cuda()
    rf_p = torch.empty((1, w.A, w.M, w.Ns), dtype=torch.float32, device="cuda")
    pf_ms = timed(lambda: fq.fq_simulate_rf_pfield(w.probe, w.tilt_x, w.tilt_y, ptx, atx, 1, n_sub=2, n_fft=n_fft,
                                                   rf=rf_p), 1)
    n_ps = 200
    sub_p = fq.fq_simulate_rf_pfield(w.probe, w.tilt_x[2:3], w.tilt_y[2:3], ptx[:, :, :n_ps].contiguous(),
                                     atx[:n_ps].contiguous(), 1, n_sub=2, n_fft=n_fft)
    t0 = time.perf_counter()
    want_p = oracle.simulate_rf_pfield(w.probe, w.tilt_x[2:3], w.tilt_y[2:3], np.ones(w.M),
                                       ptx[0, :, :n_ps].cpu().numpy(), atx[:n_ps].cpu().numpy(), n_sub=2,
                                       n_fft=n_fft)
    oracle_p_s = time.perf_counter() - t0
    err_p = float(np.linalg.norm(sub_p[0].cpu().numpy() - want_p) / np.linalg.norm(want_p))
    pk, src = peaks()
    peak = fp32_alu_peak_tflops(float(pk.get("sm_max_mhz", 2070.0)))
    terms = F * w.A * w.M * w.S * (n_fft // 2)
    ach = terms * 22 / (freq_ms * 1e-3) / 1e12
    line = {
        "metric": "channel-samples/s, RF synthesis in the frequency domain (Eq. 1 per frequency) vs time domain",
        "value": total / (freq_ms * 1e-3), "unit": "channel-samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": 1, "ms_per_step": freq_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{w.name} ({F} frames)", "n_fft": n_fft, "bins": n_fft // 2,
                   "l2": "no flush: positions 2.4 MB per frame, spectra 42 MB per frame"},
        "time_domain": {"ms": time_ms, "value": total / (time_ms * 1e-3), "freq_over_time": freq_ms / time_ms,
                        "rel_l2_freq_vs_time": td_vs_fd},
        "parity": {"sample": f"first {ns_s} scatterers of frame 0, transmit 2, every element",
                   "rel_l2_vs_oracle": err, "oracle_s": oracle_s},
        "transmit_sum": {"what": "Eq. 1 transmit sum over all 128 elements (uniform weights, steering delays) and "
                                 "2 sub-elements per element (Eq. 2)",
                         "sample": f"first {n_tx} scatterers of frame 0, every transmit and element",
                         "ms": pf_ms, "channel_samples_per_s": w.A * w.M * w.Ns / (pf_ms * 1e-3),
                         "parity": {"sample": f"first {n_ps} scatterers, transmit 2", "rel_l2_vs_oracle": err_p,
                                    "oracle_s": oracle_p_s}},
        "roofline": {"bound": "alu", "kernel": "spectrum_kernel", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak, "traffic": None,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 (FMA) x max clock ({src})",
                     "work": f"22 FLOP per (scatterer, element, transmit, frame, bin) term, {terms:.3e} terms"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------- tensor-core Gram at scale --
def run_gram(args, rank, world, local):
    """The Casorati Gram S^H S on the tensor cores (BF16 and TF32 operands,
    FP32 accumulation) at the largest batched ensemble shape (96^3 voxels x
    400 frames), where it is compute-bound, beside the FP32 CUDA-core Gram."""
    import torch
    from paper_2509_05464_gb300 import fq

    torch.cuda.set_device(local)
    fq.lib()
    P, F = 96 ** 3, args.frames or 400
    g = torch.Generator(device="cuda").manual_seed(5 + rank)
    S = torch.randn((P, F, 2), generator=g, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    clk = ClockSampler(local)
    clk.start()
    for name, mode in (("bf16", fq.FQ_GRAM_BF16), ("tf32", fq.FQ_GRAM_TF32), ("f32", fq.FQ_GRAM_F32)):
        ws = fq.workspace(fq.fq_gram_workspace_size(P, F, mode))
        G = torch.empty((F, F, 2), dtype=torch.float32, device="cuda")
        for _ in range(max(args.warmup, 1)):
            fq.fq_casorati_gram(S, mode, G=G, ws=ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            fq.fq_casorati_gram(S, mode, G=G, ws=ws)
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = max_over_ranks(a.elapsed_time(b) / args.steps)
        del ws, G
        torch.cuda.empty_cache()
    clocks = clk.stop()
    if rank != 0:
        return
    pk, src = peaks()
    peak = float(pk.get("bf16_tflops", 1900.0))
    flop = 8.0 * P * F * F  # the complex Gram as defined; the kernels compute the upper tiles only
    ach = {k: flop / (v * 1e-3) / 1e12 for k, v in out.items()}
    line = {
        "metric": "Casorati Gram TFLOP/s (8 P F^2) on tcgen05, BF16 operands",
        "value": ach["bf16"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": out["bf16"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"Gram of a {P} x {F} complex Casorati matrix (96^3 voxels, {F} frames)",
                   "ms": out, "tflops": ach,
                   "l2": "input 2.8 GB FP32, far above L2"},
        "roofline": {"bound": "tensor", "kernel": "gram_tc_kernel (with its transpose and reduce)",
                     "achieved": ach["bf16"], "peak": peak, "unit": "TFLOP/s", "frac": ach["bf16"] / peak,
                     "traffic": None, "peak_source": f"bf16_tflops of {src} peaks (cuBLAS burst)",
                     "work": f"8 P F^2 = {flop:.3e} FLOP; the upper-triangular tiles execute about half plus the diagonal tiles"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ FP32 ALU probe --
def run_alu_probe(args, rank, world, local):
    """Measured FP32 throughput, scalar FFMA and packed f32x2 FMA: the
    evidence behind the ALU roof (152 SMs x 128 lanes x 2 FLOP x clock)
    that the RF and DAS lines divide by."""
    import torch
    from paper_2509_05464_gb300 import fq
    torch.cuda.set_device(local)
    fq.lib()
    sink = torch.zeros(256, device="cuda")
    stream = torch.cuda.current_stream()
    blocks, iters = 152 * 8 * 8, 4096
    out = {}
    clk = ClockSampler(local)
    clk.start()
    for packed in (0, 1):
        for _ in range(max(1, args.warmup)):
            fq.fq_alu_probe(packed, blocks, iters, sink)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            fq.fq_alu_probe(packed, blocks, iters, sink)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        flop = blocks * 256.0 * iters * 8 * 2 * (2 if packed else 1)
        out["f32x2" if packed else "scalar"] = {"ms": ms, "tflops": flop / (ms * 1e-3) / 1e12}
    clocks = clk.stop()
    if rank != 0:
        return
    pk, src = peaks()
    smax = float(pk.get("sm_max_mhz", 2070.0))
    line = {"metric": "FP32 FMA throughput (TFLOP/s), scalar and packed f32x2", "value": out["f32x2"]["tflops"],
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["f32x2"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{blocks} CTAs x 256 threads x {iters} rounds x 8 independent FMA chains"},
            "probe": out,
            "derived_peak_tflops": {"unit_count": fp32_alu_peak_tflops(smax),
                                    "clock_mhz": smax, "clock_source": src},
            "cpu_baseline": None, "e2e": None, "gpu_launches": 2 * (args.steps + max(1, args.warmup)),
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def b_arena_gb(ms, args):
    from paper_2509_05464_gb300 import fq
    b = fq.Batch(ms, plan_only=True, max_arena_bytes=args.arena_gb << 30)
    n = b.arena_bytes / 1e9
    b.close()
    return n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the precision variants (each is checked against the oracle)")
    ap.add_argument("--frames", type=int, default=0,
                    help="ensemble length (0 = the workload's own: 100 for c3, 200 for c2)")
    ap.add_argument("--variant-steps", type=int, default=0,
                    help="timed steps per storage variant (0 = 4 for c3, 20 for c2)")
    ap.add_argument("--scatterers", type=int, default=0, help="profiling only: keep this many scatterers")
    ap.add_argument("--grid-div", type=int, default=0, help="profiling only: divide the pixel grid per axis")
    ap.add_argument("--workload", choices=["c3", "c2", "c4", "c5", "field", "post", "dasmatrix", "rffreq", "gram",
                                           "alupeak"],
                    default="c3",
                    help="c3: one 100-frame 3D volumetric ensemble (default); c2: one 200-frame 2D ensemble; "
                         "c4: the 64-ensemble uneven batch; "
                         "c5: the learned clutter filter; field: advection in a gridded velocity field; "
                         "post: display compression, MIPs and image quality; dasmatrix: the paper's "
                         "explicit DAS matrices against the fused DAS; rffreq: RF synthesis in the frequency "
                         "domain against the time-domain kernel (2 frames unless --frames); gram: the tensor-core "
                         "Gram at 96^3 voxels x 400 frames")
    ap.add_argument("--cnn-ensembles", type=int, default=256, help="c5: simulated training + held-out ensembles")
    ap.add_argument("--cnn-train-steps", type=int, default=6000, help="c5: timed training steps (cosine schedule)")
    ap.add_argument("--cnn-infer-frames", type=int, default=200, help="c5: frames of the inference ensemble")
    ap.add_argument("--cnn-gain", type=float, default=8.0, help="c5: target gain of the training pairs")
    ap.add_argument("--cnn-lr", type=float, default=1e-3, help="c5: Adam peak learning rate")
    ap.add_argument("--arena-gb", type=int, default=64, help="c4: arena budget in GiB (waves beyond it)")
    ap.add_argument("--no-sequential", dest="sequential", action="store_false",
                    help="c4: skip the one-by-one comparison run")
    ap.add_argument("--gram", choices=["f32", "tf32", "bf16"], default="",
                    help="Casorati Gram arithmetic: FP32 CUDA cores or TF32 / BF16 tensor cores")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "c4":
        run_batched(args, rank, world, local)
    elif args.workload == "c5":
        run_cnn(args, rank, world, local)
    elif args.workload == "field":
        run_field(args, rank, world, local)
    elif args.workload == "post":
        run_post(args, rank, world, local)
    elif args.workload == "dasmatrix":
        run_das_matrix(args, rank, world, local)
    elif args.workload == "rffreq":
        run_rf_freq(args, rank, world, local)
    elif args.workload == "gram":
        run_gram(args, rank, world, local)
    elif args.workload == "alupeak":
        run_alu_probe(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
