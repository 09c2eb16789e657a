"""Throughput of the SMS-MUSSELS reconstruction on GB300 (one JSON line on stdout).

A step is one complete reconstruction of one slice group (every row of the
hot path: A^H y, then K outer iterations of Gram -> Jacobi eigen-decomposition
-> weights -> filters -> J CG steps of (A^H A + lambda P_W)) through the C ABI.
The default workload is the plain FP32 configuration: MB=2 slices, 4
interleaved shots, 32 coils, 128x128, FOV/2 CAIPI shift, filter 6x6, 20 outer
x 15 CG iterations, seeded synthetic data (ellipse phantom, polynomial +
band-limited shot phase, ring coil maps, SNR 30); ``--workload precision`` is
MB=3, 256x256, FOV/3 (with ``--precision bf16-split`` for the BF16 hi+lo
split Gram).  The FP64 oracle's full reconstruction of direction 0 runs on
the host cores meanwhile: its time is the CPU baseline and its result checks
the accuracy (per-slice NRMSE) of direction 0 of the timed batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload plain|precision] [--precision fp32|bf16-split]

Multi-GPU: slice groups are independent, so every rank reconstructs its own
groups (replicas, weak scaling); the host only gathers the timings.
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

from paper_1901_01893_gb300 import synth  # noqa: E402

METRIC = "slice-group recons/sec at NRMSE≤1e-3 vs FP64 oracle: learned+BF16+batched vs plain"
UNIT = "slice-groups/s"
LAM = 1e-2
ACCURACY_BAR = 1e-3  # per-slice NRMSE vs the FP64 oracle at which the metric is quoted
# CAIPI FOV shift per workload: FOV/2 for the two-slice workloads, FOV/3 for MB 3
LDIV = {"tiny": 2, "plain": 2, "precision": 3}


def workload_desc(c, D=1, name="plain"):
    return (f"{name} workload: MB={c['L']} slices, {c['Ns']} interleaved shots, {c['Nc']} coils, "
            f"{c['N']}x{c['N']}, FOV/{LDIV[name]} CAIPI shift, filter {c['r']}x{c['r']}, {c['K']} outer x {c['J']} CG; "
            f"{D} diffusion directions of one slice group per step (shared coil maps, independent shot phase)")


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def seed_for_rank(base_seed: int, rank: int) -> int:
    """Replicas reconstruct different slice groups: rank r draws its inputs from base + 1000 r."""
    return base_seed + 1000 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (timings: the job is as slow as its slowest replica)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def item_costs(geos, directions: int):
    """Estimated cost of every (group, direction) item of the batched job, N^2 Nc MB (the
    work of the per-coil stages); items are numbered group-major."""
    return [c["N"] ** 2 * c["Nc"] * c["L"] for c in geos for _ in range(directions)]


def partition_items(costs, world: int):
    """The items each rank takes: sorted by estimated cost (largest first, ties by index) and
    dealt round-robin, so every item goes to exactly one rank and the ranks' loads differ by
    at most one item's cost."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    return [sorted(order[r::world]) for r in range(world)]


def throughput(world: int, batch: int, ms_per_step: float) -> float:
    """Whole-job slice groups per second: every rank finishes `batch` groups per step."""
    return world * batch * 1000.0 / ms_per_step


# ---------------------------------------------------------------------------
# The FP64 oracle: the CPU baseline, the reference arm and the accuracy check.
# Only these functions touch oracle/; they run in a spawned worker process or
# after every GPU measurement, never on the GPU path.
# ---------------------------------------------------------------------------

def oracle_data(cfg, seed, Ldiv):
    """Direction 0's slice group and its data y = A x_true + noise (SNR 30),
    normalised to RMS |y| = 1, synthesised on the host by the oracle."""
    import oracle as O

    g = make_host_inputs(cfg, seed)
    _, y = O.make_data(g, cfg["snr"], Ldiv=Ldiv)
    return g, y / np.sqrt(np.mean(np.abs(y) ** 2))


def oracle_full_solve(cfg, y, sens, Ldiv):
    """One complete oracle reconstruction (K outer x J CG); returns (x, wall seconds,
    threads).  Run in a spawned worker while the GPU is measured."""
    import oracle as O

    t0 = time.perf_counter()
    x = O.reconstruct(y, sens, cfg["r"], dict(K=cfg["K"], J=cfg["J"], lam=LAM), Ldiv=Ldiv)
    return x, time.perf_counter() - t0, cpu_threads()


def oracle_step(cfg, y, sens, Ldiv):
    """The reference arm's step: A^H y and the first outer iteration of the oracle's
    reconstruction (Gram, eigen-decomposition and weights on the real eps schedule,
    J CG steps).  Returns its wall seconds."""
    import oracle as O

    t0 = time.perf_counter()
    O.reconstruct(y, sens, cfg["r"], dict(K=1, J=cfg["J"], lam=LAM), Ldiv=Ldiv)
    return time.perf_counter() - t0


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info

        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(max(n, os.cpu_count() or 1))
    except Exception:
        return os.cpu_count() or 1


def make_host_inputs(cfg, seed):
    g = synth.make_group(seed=seed, **{k: cfg[k] for k in ("L", "Ns", "Nc", "N", "field")})
    return g


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    name = args.workload
    cfg = dict(synth.CONFIGS[name])
    g, y = oracle_data(cfg, cfg["seed"], LDIV[name])
    for _ in range(args.warmup):
        oracle_step(cfg, y, g["sens"], LDIV[name])
    per = [oracle_step(cfg, y, g["sens"], LDIV[name]) for _ in range(args.steps)]
    t = statistics.mean(per)
    v = 1.0 / (cfg["K"] * t)
    sample = (f"each step: A^H y and the first of the {cfg['K']} outer iterations (Gram + eigh + W on the "
              f"oracle's eps schedule, {cfg['J']} CG steps) of one direction's FP64 oracle reconstruction, "
              f"{t:.2f} s; value = 1 / ({cfg['K']} x step time), the outer iterations extrapolated")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(cfg, 1, name), "form": "FP64 CPU oracle",
                   "step": "one outer iteration of one direction (see cpu_baseline.sample)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        try:
            with open(self.f.name) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

# DRAM bytes (read + write) per direction of one launch of a kernel class, measured
# by ncu on the current kernels ({workload: {class: bytes}}; a launch covering d
# directions moves d times this).  A class whose kernel changed since its capture is
# left out, so its roofline line carries traffic = null.
TRAFFIC_PER_DIRECTION: dict = {}


def stage_work(cfg, D, sweeps):
    """Algorithmic work of one launch (bracket) of each kernel class, over a batch of D problems.

    Returns {stage: (bound, amount)} with bound "alu" (FP32 flops) or "hbm" (bytes)."""
    L, Ns, Nc, N, r = cfg["L"], cfg["Ns"], cfg["Nc"], cfg["N"], cfg["r"]
    B, NN, M, C = L * Ns, N * N, N // Ns, Ns * r * r
    Cp = C + (C & 1)
    half = Cp // 2
    P = (N - r + 1) ** 2
    R2 = 2 * r - 1
    nband = NN - (N - 2 * (r - 1)) ** 2
    lg = np.log2
    # column stage, per image column: the B lines' inverse and forward N-point FFTs
    # (5 N log2 N each), the A^H A class products (8 L Ns flops per pixel and line) and
    # the Ns x Ns Hermitian periodic multiplier (8 Ns per pixel and line)
    col = N * (B * 2 * 5 * N * lg(N) + B * N * 8 * (L * Ns + Ns))
    return {
        "column": ("alu", D * col),
        "band": ("alu", D * 8 * L * nband * Ns * Ns * R2 * R2),
        "gram": ("alu", D * 8 * L * P * C * (C + 1) / 2),
        # every round: the 2x2 blocks of G (96 flops each) and the rotated column pairs of V
        # (18 flops per row and pair); plus the warm start's two C x C complex products
        "eig": ("alu", D * L * (sweeps * (Cp - 1) * ((half * (half + 1) / 2) * 96 + half * C * 18)
                                + 2 * 8 * C ** 3)),
        # the Newton-Schulz step (two C x C complex products)
        "vapply": ("alu", D * L * 2 * 8 * C ** 3),
        "rowfft_inv": ("hbm", D * 2 * 8 * B * NN),
        "rowfft_fwd": ("hbm", D * 2 * 8 * B * NN),
        "cg": ("hbm", D * 9 * 8 * B * NN),
        "weights": ("alu", D * L * 8 * C * C * C),
        # class taps, plus the periodic multiplier's Ns(Ns+1)/2 Hermitian planes by two small DFTs
        "filters": ("alu", D * L * (R2 * R2 + 1) * Ns * Ns * R2 * R2 * r * r * 2
                    + D * L * (Ns * (Ns + 1) // 2) * NN * R2 * 8),
        "adjoint": ("hbm", D * 8 * (L * Nc * NN + 2 * Ns * Nc * M * N + 2 * B * NN)),
    }


def run_ours(args):
    import torch

    rank, world, local = env_rank()
    name = args.workload
    cfg = dict(synth.CONFIGS[name])
    Ldiv = LDIV[name]
    L, Ns, Nc, N, r = cfg["L"], cfg["Ns"], cfg["Nc"], cfg["N"], cfg["r"]
    seed = seed_for_rank(cfg["seed"], rank)
    D = args.batch

    # CPU baseline and accuracy check (rank 0 at N = 1): direction 0's data is made on the
    # host by the oracle, and its full oracle reconstruction runs in a spawned worker on the
    # host cores while the GPU is measured.
    oracle_leg = world == 1 and not args.no_cpu_baseline
    pool = fut = None
    if oracle_leg:
        import concurrent.futures as cf
        import multiprocessing as mp

        g0h, y0h = oracle_data(cfg, seed, Ldiv)
        pool = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
        fut = pool.submit(oracle_full_solve, cfg, y0h, g0h["sens"], Ldiv)

    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1901_01893_gb300 import _build

    _build.build()
    from paper_1901_01893_gb300 import smsm

    c64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(dev)  # noqa: E731
    combined = args.form == "combined"
    precision = "bf16-split" if combined else args.precision
    prec = smsm.SMSM_PRECISION_BF16_SPLIT if precision == "bf16-split" else smsm.SMSM_PRECISION_FP32
    plan = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D, precision=prec)
    one = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv)  # synthesis, one direction at a time
    ys = []
    for d in range(D):
        g = make_host_inputs(cfg, seed + d)  # same coil maps for every seed; own phantom, phase, noise
        if d == 0:
            sens0 = g["sens"]
            plan.set_sens(c64(sens0))
            one.set_sens(c64(sens0))
            g0 = g
        if d == 0 and oracle_leg:
            ys.append(c64(y0h))
            continue
        # synthesis on the GPU: x_rho = F_c(rho); y = A(x_rho; phi) + noise at SNR 30; RMS(y) = 1
        xr = one.fft2c(c64(g0["rho"][:, None]))  # one object, imaged along every direction
        yc = one.forward(xr, phase=c64(g["phase"]))
        nz = c64(g["noise"])
        yd = yc + nz * (torch.linalg.vector_norm(yc) / (cfg["snr"] * torch.linalg.vector_norm(nz)))
        ys.append(yd / torch.sqrt(torch.mean(torch.abs(yd) ** 2)))
    y = (torch.stack(ys) if D > 1 else ys[0]).contiguous()
    x = torch.empty(plan.x_shape, dtype=torch.complex64, device=dev)

    allmask = (1 << len(smsm.STAGES)) - 1
    prm = smsm.default_params(lam=LAM, outer_iters=cfg["K"], cg_iters=cfg["J"])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tuned = None
    if combined:  # the batched form's autotuner: Gram split-K blocks and lanes for this shape
        tr = plan.autotune(y, params=prm)
        tuned = {"gram_nG": tr.gram_nG, "lanes": tr.lanes,
                 "gram_ms": {int(c): round(float(m), 4) for c, m in zip(list(tr.gram_candidates)[:tr.n_gram],
                                                                      list(tr.gram_ms)[:tr.n_gram])},
                 "lane_ms": [round(float(m), 3) for m in tr.lane_ms]}

    # warm-up; the first one runs the batch as one lane and times every kernel class
    # (the per-stage breakdown of the serial schedule) to find the dominant one
    prm.timing = allmask
    prm.lanes = 1
    _, rep = plan.reconstruct(y, x=x, params=prm)
    stages_all = {smsm.STAGES[k]: rep.stage_ms[k] for k in range(len(smsm.STAGES))}
    dominant = max(stages_all, key=stages_all.get)
    prm.timing = 1 << smsm.STAGE[dominant]
    prm.lanes = args.lanes
    for _ in range(max(0, args.warmup - 1)):
        plan.reconstruct(y, x=x, params=prm)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dom_ms, dom_n, launches, status = 0.0, 0, 0, 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        # an NVTX range around the timed steps, so that a profiler can take exactly their
        # kernels (ncu --nvtx --nvtx-include timed_steps/); no effect without one
        torch.cuda.nvtx.range_push("timed_steps")
        for k in range(args.steps):
            flush.zero_()  # L2 (129 MB) flushed before every step, outside the step's events
            ev[k][0].record()
            _, rep = plan.reconstruct(y, x=x, params=prm)
            ev[k][1].record()
            dom_ms += rep.stage_ms[smsm.STAGE[dominant]]
            dom_n += rep.stage_launches[smsm.STAGE[dominant]]
            launches += rep.graph_kernels
            status = status or rep.status
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if status not in (0, smsm.SMSM_ERR_EIG_UNCONVERGED):
        raise RuntimeError(f"solve reported status {status}")
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    clocks = clk.summary()
    ms = max_over_ranks(ms, dev)
    value = throughput(world, D, ms)
    x_dir0 = (x[0] if D > 1 else x).cpu().numpy()

    # end to end through the public API: pinned host y -> device, solve, x -> pinned host
    y_host = y.cpu().pin_memory()
    x_host = torch.empty(plan.x_shape, dtype=torch.complex64).pin_memory()
    prm.timing = 0
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    y_dev = torch.empty_like(y)
    for k in range(args.steps):
        flush.zero_()
        e2e_ev[k][0].record()
        y_dev.copy_(y_host, non_blocking=True)
        plan.reconstruct(y_dev, x=x, params=prm, report=False)
        x_host.copy_(x, non_blocking=True)
        e2e_ev[k][1].record()
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dev)

    forms = None
    if combined:
        # the plain form on the same data: FP32 Gram, default lanes, no autotuning
        pplan = smsm.Plan(L, Ns, Nc, N, r, caipi_div=Ldiv, batch=D)
        pplan.set_sens(c64(sens0))
        pp = smsm.default_params(lam=LAM, outer_iters=cfg["K"], cg_iters=cfg["J"])
        xp_ = torch.empty(pplan.x_shape, dtype=torch.complex64, device=dev)
        for _ in range(args.warmup):
            pplan.reconstruct(y, x=xp_, params=pp, report=False)
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            pev[k][0].record()
            pplan.reconstruct(y, x=xp_, params=pp, report=False)
            pev[k][1].record()
        torch.cuda.synchronize()
        p_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in pev) / args.steps, dev)
        forms = {
            "plain": {"value": throughput(world, D, p_ms), "ms_per_step": p_ms,
                      "form": "FP32-form Gram (three BF16 pieces), default lanes, no autotuning, start A^H y"},
            "combined": {"value": value, "ms_per_step": ms,
                         "form": "BF16 hi+lo split Gram, batch of directions in autotuned lanes with autotuned "
                                 "Gram split-K, start A^H y", "autotuned": tuned,
                         "learned_start": "not applied: the trained network saves no outer iterations on this "
                                          "workload (its residual learns nothing beyond the identity), so the "
                                          "combined form runs the plain iteration count"},
            "ratio_combined_over_plain": value / throughput(world, D, p_ms),
        }
        pplan.close()

    if rank != 0:
        torch.distributed.destroy_process_group()
        return

    # roofline of the dominant kernel class
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    sweeps = float(np.mean([rep.sweeps[k] for k in range(cfg["K"])]))
    # timed brackets cover the launches of lane 0, each over its sub-batch of directions
    d_launch = rep.lane0_batch if rep.lanes > 1 else D
    bound, amount = stage_work(cfg, d_launch, sweeps)[dominant]
    tpd = TRAFFIC_PER_DIRECTION.get(name, {}).get(dominant)
    traffic = tpd * d_launch if tpd is not None else None
    per_launch_ms = dom_ms / max(dom_n, 1)
    sm_mhz = clocks.get("sm_mhz") or 1455.0
    if bound == "alu":
        # FP32 ALU bound: 152 SMs x 128 FP32 lanes x 2 flops x the SM clock sampled under load
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        achieved = amount / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dominant, "launch_ms": per_launch_ms,
                "peak_note": f"FP32 FMA peak (152 SMs x 128 lanes x 2) at the sampled median SM clock {sm_mhz:.0f} MHz"}
    else:
        achieved = amount / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic, "kernel": dominant, "launch_ms": per_launch_ms, "peak_note": peak_src}

    # CPU baseline and accuracy: the oracle's full reconstruction of direction 0
    cpu, acc, acc_ok = None, None, True
    if fut is not None:
        import oracle as O

        ref, t_or, thr = fut.result()
        pool.shutdown()
        e = O.nrmse(x_dir0, ref, axis=(1, 2, 3))
        acc_ok = bool(np.max(e) <= ACCURACY_BAR)
        acc = {"per_slice": [float(v) for v in e], "max": float(np.max(e)), "bar": ACCURACY_BAR,
               "direction": 0, "K": cfg["K"], "J": cfg["J"],
               "what": "direction 0 of the timed batch against the FP64 oracle's reconstruction of the same data "
                       "(same K, J, lambda and eps schedule), per slice"}
        cpu = {"value": 1.0 / t_or, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": (f"one complete FP64 oracle reconstruction (NumPy, explicit Hankel; {cfg['K']} outer x "
                          f"{cfg['J']} CG) of direction 0, {t_or:.1f} s wall on the host cores, run while the GPU "
                          f"was measured; not extrapolated")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f32+bf16-split",
        "data": "synthetic",
        "forms": forms,
        "config": {"workload": workload_desc(cfg, D, name),
                   "form": ("plain FP32 (FP64 reductions)" if precision == "fp32" else
                            "BF16 hi+lo split Hankel Gram, FP32 elsewhere (FP64 reductions)"
                            + (", autotuned lanes and Gram split-K" if combined else "")),
                   "directions_per_step": D, "lanes": rep.lanes,
                   "l2": "flushed before every step (512 MB write)", "parallelism": f"replicas x{world}",
                   "lambda": LAM, "stages_ms_first_warmup": stages_all,
                   "jacobi_sweeps_per_outer": [rep.sweeps[k] for k in range(cfg["K"])],
                   "eig_status": int(status)},
        "nrmse_vs_oracle": acc,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": throughput(world, D, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(y.numel() * 8),
                "d2h_bytes_per_step": int(x.numel() * 8)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    if not acc_ok:
        sys.exit(f"accuracy check failed: direction 0 per-slice NRMSE vs the FP64 oracle {acc['per_slice']} "
                 f"above {ACCURACY_BAR}")


# ---------------------------------------------------------------------------
# the batched form: many slice groups of uneven geometry, every direction of each
# ---------------------------------------------------------------------------

BATCHED_GROUPS, BATCHED_DIRECTIONS = 20, 60
FILTER_FOR_SHOTS = {2: 4, 4: 6, 8: 6}  # the paper's 4x4 (2 shots) and 6x6 (4 shots); 8 shots keep 6x6


def batched_geometries(seed=4, n=BATCHED_GROUPS):
    """Slice groups of uneven size drawn from MB {2,3}, shots {2,4,8}, coils {16,32},
    matrices {128, 192, 256}^2 (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.choice([2, 3]))
        Ns = int(rng.choice([2, 4, 8]))
        Nc = int(rng.choice([16, 32]))
        N = int(rng.choice([128, 192, 256]))
        out.append(dict(L=L, Ns=Ns, Nc=Nc, N=N, r=FILTER_FOR_SHOTS[Ns], K=20, J=15, seed=4000 + 100 * k,
                        field=True, snr=30.0))
    return out


def run_batched(args):
    """All directions of every group through smsm_reconstruct_groups (one plan per group with its
    directions as the batch, each plan autotuned once per shape; all groups in one graph launch),
    1200 reconstructions per step."""
    import torch

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1901_01893_gb300 import _build

    _build.build()
    from paper_1901_01893_gb300 import smsm

    # one fixed job (every rank draws the same groups); its (group, direction) items are
    # partitioned over the ranks by estimated cost, so the job scales strongly
    geos_all = batched_geometries(seed=4)
    Dd = args.directions
    mine = partition_items(item_costs(geos_all, Dd), world)[rank]
    dirs_of = [[] for _ in geos_all]
    for i in mine:
        dirs_of[i // Dd].append(i % Dd)
    gidx = [k for k in range(len(geos_all)) if dirs_of[k]]  # the groups this rank holds
    geos = [geos_all[k] for k in gidx]
    dirs = [dirs_of[k] for k in gidx]
    # the oracle leg (rank 0, N = 1): the smallest group's direction 0, made on the host
    small = min(range(len(geos)), key=lambda k: geos[k]["N"] ** 2 * geos[k]["Nc"] * geos[k]["L"] * geos[k]["Ns"])
    oracle_leg = world == 1 and not args.no_cpu_baseline and dirs[small][0] == 0
    pool = fut = None
    if oracle_leg:
        import concurrent.futures as cf
        import multiprocessing as mp

        cs = geos[small]
        gsh, ysh = oracle_data(cs, cs["seed"], cs["L"])
        pool = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
        fut = pool.submit(oracle_full_solve, cs, ysh, gsh["sens"], cs["L"])
    c64 = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).to(dev)  # noqa: E731
    prec = smsm.SMSM_PRECISION_BF16_SPLIT if args.precision == "bf16-split" else smsm.SMSM_PRECISION_FP32
    prm = smsm.default_params(lam=LAM, outer_iters=20, cg_iters=15)
    plans, ys, tune = [], [], []
    t_syn = time.perf_counter()
    for k, c in enumerate(geos):
        g = synth.make_group(c["L"], c["Ns"], c["Nc"], c["N"], c["seed"], field=True)
        one = smsm.Plan(c["L"], c["Ns"], c["Nc"], c["N"], c["r"])
        one.set_sens(c64(g["sens"]))
        xr = one.fft2c(c64(g["rho"][:, None]))  # the group's object, imaged along every direction
        gen = torch.Generator(device=dev)
        yk = []
        for d in dirs[k]:
            gen.manual_seed(c["seed"] * 1000 + d)  # the item's noise, whichever rank draws it
            if d == 0 and k == small and oracle_leg:
                yk.append(c64(ysh))
                continue
            if d == 0:
                ph = c64(g["phase"])
            else:
                co = synth.draw_phase_coeffs(np.random.default_rng((c["seed"], d)), c["L"], c["Ns"], True)
                ph = synth.phase_from_coeffs(co, c["N"], xp=torch, device=dev).to(torch.complex64).contiguous()
            yc = one.forward(xr, phase=ph)
            nz = torch.randn(yc.shape, dtype=torch.complex64, device=dev, generator=gen)
            yd = yc + nz * (torch.linalg.vector_norm(yc) / (c["snr"] * torch.linalg.vector_norm(nz)))
            yk.append(yd / torch.sqrt(torch.mean(torch.abs(yd) ** 2)))
        y = torch.stack(yk).contiguous()
        p = smsm.Plan(c["L"], c["Ns"], c["Nc"], c["N"], c["r"], batch=len(dirs[k]), precision=prec)
        p.set_sens(c64(g["sens"]))
        tr = p.autotune(y, params=prm)
        tune.append({"gram_nG": tr.gram_nG, "lanes": tr.lanes})
        plans.append(p)
        ys.append(y)
        one.close()
    torch.cuda.synchronize()
    t_syn = time.perf_counter() - t_syn
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the largest group alone, every kernel class timed: the per-stage breakdown and the roofline
    big = max(range(len(geos)), key=lambda k: geos[k]["N"] ** 2 * geos[k]["Nc"] * geos[k]["L"] * geos[k]["Ns"])
    pt = smsm.default_params(lam=LAM, outer_iters=20, cg_iters=15)
    pt.timing = (1 << len(smsm.STAGES)) - 1
    pt.lanes = 1
    _, rep = plans[big].reconstruct(ys[big], params=pt)
    stages_big = {smsm.STAGES[k]: rep.stage_ms[k] for k in range(len(smsm.STAGES))}
    dominant = max(stages_big, key=stages_big.get)
    dom_ms = rep.stage_ms[smsm.STAGE[dominant]] / max(rep.stage_launches[smsm.STAGE[dominant]], 1)
    xs = [torch.empty(p.x_shape, dtype=torch.complex64, device=dev) for p in plans]
    for _ in range(args.warmup):  # the first call builds the one graph of all groups
        smsm.reconstruct_groups(plans, ys, params=prm, report=False, xs=xs)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    status = 0
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            xs, reps = smsm.reconstruct_groups(plans, ys, params=prm, xs=xs)
            ev[k][1].record()
            for r_ in reps:
                status = status or r_.status
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if status not in (0, smsm.SMSM_ERR_EIG_UNCONVERGED):
        raise RuntimeError(f"a solve reported status {status}")
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / args.steps, dev)
    clocks = clk.summary()
    n_rec = sum(len(d_) for d_ in dirs)  # this rank's items
    n_job = len(geos_all) * Dd           # the whole job's
    value = n_job * 1000.0 / ms
    x_small0 = xs[small][0].cpu().numpy()
    launches = sum(r_.graph_kernels for r_ in reps)
    # end to end: every group's y from pinned host memory, every x back
    yh = [y.cpu().pin_memory() for y in ys]
    xh = [torch.empty(p.x_shape, dtype=torch.complex64).pin_memory() for p in plans]
    yd = [torch.empty_like(y) for y in ys]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record()
    for a, b in zip(yd, yh):
        a.copy_(b, non_blocking=True)
    xo, _ = smsm.reconstruct_groups(plans, yd, params=prm, report=False, xs=xs)
    for a, b in zip(xh, xo):
        a.copy_(b, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dev)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    cb = geos[big]
    bound, amount = stage_work(cb, len(dirs[big]), float(np.mean([rep.sweeps[k] for k in range(20)])))[dominant]
    sm_mhz = clocks.get("sm_mhz") or 1455.0
    if bound == "alu":
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        achieved = amount / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dominant, "launch_ms": dom_ms,
                "peak_note": f"FP32 FMA peak at the sampled median SM clock {sm_mhz:.0f} MHz; the largest group "
                             f"({cb['L']}x{cb['Ns']}x{cb['Nc']}x{cb['N']}^2) solved alone as one lane"}
    else:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = amount / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": dominant, "launch_ms": dom_ms,
                "peak_note": "of measured" if "hbm_gbs" in peaks else "of fallback"}
    cpu, acc, acc_ok = None, None, True
    if fut is not None:
        import oracle as O

        ref, t_or, thr = fut.result()
        pool.shutdown()
        e = O.nrmse(x_small0, ref, axis=(1, 2, 3))
        acc_ok = bool(np.max(e) <= ACCURACY_BAR)
        acc = {"per_slice": [float(v) for v in e], "max": float(np.max(e)), "bar": ACCURACY_BAR, "group": small,
               "direction": 0, "K": 20, "J": 15,
               "what": "the smallest group's direction 0 of the timed step against the FP64 oracle's reconstruction"}
        cs = geos[small]
        cpu = {"value": 1.0 / t_or, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": (f"one complete FP64 oracle reconstruction (20 x 15) of the smallest group "
                          f"(MB {cs['L']}, {cs['Ns']} shots, {cs['Nc']} coils, {cs['N']}^2), {t_or:.1f} s on the host "
                          f"cores while the GPU was measured; the other groups are larger, so this overstates the "
                          f"oracle's rate on the whole workload")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f32+bf16-split", "data": "synthetic",
        "config": {"workload": (f"batched form: {len(geos_all)} slice groups x {Dd} diffusion directions, uneven "
                                f"geometry (MB 2-3, 2/4/8 shots, 16/32 coils, 128^2-256^2, FOV/MB, filters "
                                f"4x4/6x6/6x6 for 2/4/8 shots), 20 outer x 15 CG, all groups per step"),
                   "groups": [dict(L=c["L"], Ns=c["Ns"], Nc=c["Nc"], N=c["N"], r=c["r"]) for c in geos_all],
                   "reconstructions_per_step": n_job, "reconstructions_rank0": n_rec, "autotuned": tune,
                   "l2": "flushed before every step (512 MB write)",
                   "parallelism": (f"dp{world}: the job's (group, direction) items dealt to the ranks by "
                                   f"estimated cost N^2 Nc MB, no collective on the data path"),
                   "synthesis_s": t_syn, "stages_ms_largest_group": stages_big},
        "nrmse_vs_oracle": acc, "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": n_job * 1000.0 / e2e_ms, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(y.numel() * 8 for y in ys)),
                "d2h_bytes_per_step": int(sum(p_.D * p_.L * p_.Ns * p_.N * p_.N * 8 for p_ in plans))},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    if not acc_ok:
        sys.exit(f"accuracy check failed: {acc['per_slice']} above {ACCURACY_BAR}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle leg (CPU baseline and the accuracy check of direction 0)")
    ap.add_argument("--directions", type=int, default=BATCHED_DIRECTIONS,
                    help="batched workload: diffusion directions of every slice group")
    ap.add_argument("--workload", default="plain", choices=["plain", "precision", "batched"],
                    help="plain: MB 2, 4 shots, 32 coils, 128^2, FOV/2; precision: MB 3, 4 shots, 32 coils, "
                         "256^2, FOV/3 (both filter 6x6, 20 outer x 15 CG)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16-split"],
                    help="Hankel Gram form with --form plain: FP32-exact BF16 pieces or the BF16 hi+lo split")
    ap.add_argument("--form", default="combined", choices=["combined", "plain"],
                    help="combined: the BF16 split + autotuned batched form, timed beside the plain form on the "
                         "same data (value = combined); plain: only the form --precision selects")
    ap.add_argument("--lanes", type=int, default=0,
                    help="concurrent sub-batches of the solve (0: the library's automatic choice)")
    ap.add_argument("--batch", type=int, default=26,
                    help="diffusion directions of one slice group per step (the paper acquires 25 + b0)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
