"""Benchmark: TA-SC-IVR power spectrum, trajectory-steps/s and spectra/s.

One step = one pass of the whole hot path over one batch: Husimi sampling
of n_traj initial conditions, propagation of (p, q, S, M, prefactor phase,
amplitudes) over n_steps, and the time -> energy transform with the weighted
|.|^2 reduction into I(E).  Default workload: F = 9 (methane-sized) Morse +
156 cubic + 486 quartic couplings, 65536 trajectories, 5000 steps of 10 au,
4000 energies; mixed-precision propagation (FP32 monodromy and potential,
FP64 positions, momenta, action and prefactor phase) and the tensor-core
Fourier step with two BF16 digits per operand and FP32 accumulation
(--precision fp64 --ft fp64 --workload f6 gives the plain FP64 F = 6 form).

  python bench.py [--gpus N --steps K --warmup W] [--workload f6|f3|f9|batch|f9mlp|speedup]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)

Multi-GPU (torchrun): weak scaling, every rank runs its own batch (seed
base + rank); the per-rank spectra combine through one all-reduce of
n_E + 1 numbers.  Prints one JSON line on rank 0.
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

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from paper_1312_4698_gb300 import workloads as wl  # noqa: E402

METRIC = "trajectory-steps/s and spectra/s at ≤1 cm⁻¹ peak error vs FP64 oracle"
FT_MODES = {"fp64": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3, "czt64": 4}
PRECISIONS = {"fp64": 0, "mixed": 1}
MIXED_STAB_TOL = 1e-6 * 2.0 ** 29     # the FP64 threshold scaled by eps32 / eps64
L2_FLUSH_BYTES = 512 << 20
FP64_PEAK_GFLOPS = 1250.0      # GB300 dense FP64 (nominal, CUDA cores and tensor cores alike)
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07   # 80.5 TFLOP/s: SMs x FP32 lanes x 2 x max SM clock
FP64_PEAK_NOTE = ("GB300 nominal dense FP64 1.25 TFLOP/s (profiling recipe table); an FMA-chain "
                  "probe on this pool measured 1.252 TFLOP/s")
# dram read+write bytes per launch from ncu captures (profiles/), keyed by (kernel, workload);
# scaled to the full launch where the capture used fewer trajectories
TRAFFIC = {("k_ft_fp64", "f6"): 29.92e9, ("k_ft_tc2", "f6"): 7.98e9,
           ("k_mlp_fused", "f9mlp"): 0.914e6 * 8,
           # per trajectory-step (the bench multiplies by trajectories x steps), by amplitude
           # storage: one launch of 65536 trajectories x 400 steps with complex-double rows
           # read 17.06 MB and wrote 364.34 MB
           ("k_propagate_lg_mixed", "f9", "f64"): (17.06e6 + 364.34e6) / (65536 * 400),
           # complex-float rows (the default mixed line): 14.58 MB read, 153.33 MB written
           ("k_propagate_lg_mixed", "f9", "f32"): (14.58e6 + 153.33e6) / (65536 * 400)}


# trajectories of the oracle's timed sample per workload (10-30 s of host work on 16 cores),
# and of each step of the reference arm (whose --steps K --warmup W run must end in minutes)
CPU_SAMPLE = {"f3": 1024, "f6": 768, "f9": 256}
REFERENCE_SAMPLE = {"f3": 1024, "f6": 768, "f9": 64}


def workload(name: str, seed: int):
    if name == "f3":
        return wl.config_f3(seed=seed)
    if name == "f6":
        return wl.config_f6(seed=seed)
    if name == "f9":
        return wl.config_f9(seed=seed)
    raise SystemExit(f"unknown workload {name}")


def sized(w8, args):
    kw = {}
    if getattr(args, "n_traj", None):
        kw["n_traj"] = args.n_traj
    if getattr(args, "n_steps", None):
        kw["n_steps"] = args.n_steps
    if getattr(args, "n_E", None):
        kw["n_E"] = args.n_E
    return w8.with_(**kw) if kw else w8


def describe(w8, precision="fp64", ft="fp64", amplitude="ta"):
    spec = ("plain Herman-Kluk spectrum (survival amplitude, one-sided transform)" if amplitude == "hk"
            else f"time-averaged spectrum, Fourier step {ft}")
    return (f"{w8.name}: F={w8.F}, {w8.n_traj} trajectories, {w8.n_steps} steps of {w8.dt} au, "
            f"{w8.n_E} energies, propagation {precision}, {spec}")


def propagate_flops_per_traj_step(F: int, n3: int, n4: int, mixed: bool = False) -> float:
    """Algorithmic flops of one trajectory step (multiply-add = 2 flops).

    3 kicks: potential (pair products P, cubic Hessian P*F and quartic
    Hessian P*P multiply-adds, gradient and energy 2P each, Morse diagonal ~6F)
    and the monodromy kick M_p -= tau H M_q (2F * F * F multiply-adds);
    4 drifts: q and M_q (F + 2F*F multiply-adds) and the kinetic action (F);
    det M by LU of 2F x 2F ((2/3)(2F)^3 flops; the mixed path does it every
    16 steps, the FP64 path every step), det A by complex LU of F x F
    (8/3 F^3 real flops) plus building A (6 F^2), phase (~30) and the
    amplitude per reference state (~10 F + 30)."""
    fp32, fp64 = propagate_flops_split(F, n3, n4, mixed)
    return fp32 + fp64


DET_M_EVERY_MIXED = 16   # stability-test cadence of the mixed path (steps)


def propagate_flops_split(F: int, n3: int, n4: int, mixed: bool = False):
    """(bulk, fp64-kept) split of propagate_flops_per_traj_step.  Mixed path:
    everything runs on the FP32 pipe -- in FP32 the potential, monodromy, det M,
    building A, the overlap and the kinetic action increments; in double-FP32
    pairs the elimination that gives det A and the p, q and action updates,
    counted here at their algorithmic flops (the FP32 instructions that emulate
    FP64-class arithmetic show up as lost efficiency) -- except the
    continuous-phase scan and the phase sum with its reduction modulo 2 pi
    (~11 flops), which stay FP64.  FP64 path: all of it is FP64 (the split is
    then only informative)."""
    P = F * (F + 1) // 2
    pes = 2 * (P + (P * F if n3 else 0) + (P * P if n4 else 0) + 4 * P) + 6 * F
    det_m = (2.0 / 3.0) * (2 * F) ** 3 / (DET_M_EVERY_MIXED if mixed else 1)
    total = (3 * (pes + 2 * (2 * F * F * F)) + 4 * (2 * 2 * F * F) + det_m + 6 * F * F
             + (8.0 / 3.0) * F ** 3 + 3 * (2 * F + 2) + 4 * (2 * F + 2 * F) + 30 + 10 * F + 30)
    kept = 11.0 if mixed else 14.0 * F + 11.0
    return total - kept, kept


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_selector(local: int) -> str:
    """nvidia-smi -i argument for torch device `local` (UUID when available)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[local].strip()
    return str(local)


def fma_peaks(stream=None):
    """Attainable FP32 and FP64 FMA rates (TFLOP/s) of this GPU, measured live by the
    library's probe (independent FMA chains on every SM, about 30 ms per launch, best of
    three after one warm-up) -- the propagation kernels' roofline denominators."""
    import torch
    from paper_1312_4698_gb300 import scivr
    out = {}
    for name, prec, iters in (("fp32", 1, 225000), ("fp64", 0, 3750)):
        best = 0.0
        for rep in range(4):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = scivr.scivr_fma_probe(prec, iters, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        out[name] = best
    return out


def measured_peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def run_cpu_oracle(w8, n_sample: int, threads: int, amplitude: str = "ta"):
    """Time the oracle (as it stands) on the first n_sample trajectories of the workload
    (amplitude "ta": time-averaged spectrum; "hk": plain Herman-Kluk spectrum)."""
    import oracle
    oracle.build()
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, n_sample, w8.seed)
    hk = amplitude == "hk"
    t0 = time.perf_counter()
    amp, good = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                                 w8.stab_tol, threads, amplitude=oracle.AMP_HK if hk else oracle.AMP_TA)
    t1 = time.perf_counter()
    if hk:
        oracle.spectrum_hk(amp[0], good, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    else:
        oracle.spectrum(amp[0], w, good, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, threads)
    t2 = time.perf_counter()
    used = threads if threads > 0 else oracle.max_threads()
    return dict(seconds=t2 - t0, prop_s=t1 - t0, spec_s=t2 - t1, cores=used,
                value=n_sample * w8.n_steps / (t2 - t0))


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload in ("batch", "speedup"):
        print(json.dumps({"impl": "reference", "unavailable": f"the {args.workload} workload has no single oracle "
                          "configuration (its line carries the oracle's own rates); time --workload "
                          "f3/f6/f9/f9mlp instead"}))
        return 0
    n_sample = min(args.cpu_sample, REFERENCE_SAMPLE.get(args.workload, args.cpu_sample))
    if args.workload == "f9mlp":
        # the oracle on the same surface type: Morse diagonal + a network of the same shape
        base = sized(wl.config_f9(seed=0), args)
        w8 = base.with_(pes=wl.PesDesc(base.F, base.pes.diag_kind, base.pes.omega, base.pes.D, base.pes.a,
                                       np.zeros((0, 3)), np.zeros(0), np.zeros((0, 4)), np.zeros(0),
                                       wl.init_mlp(base.F, 256, 0, s_in=np.sqrt(base.pes.omega), s_out=3e-6)))
        n_sample = min(n_sample, 16)
    else:
        w8 = sized(workload(args.workload, 0), args)
    times = []
    for i in range(args.warmup + args.steps):
        r = run_cpu_oracle(w8, n_sample, 0, args.amplitude)
        if i >= args.warmup:
            times.append(r)
    sec = sum(t["seconds"] for t in times) / len(times)
    value = n_sample * w8.n_steps / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "trajectory-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(w8, amplitude=args.amplitude),
                   "sample": f"{n_sample} of {w8.n_traj} trajectories",
                   "l2": "n/a (host)"},
        "spectra_per_s": value / (w8.n_traj * w8.n_steps),
        "cpu_baseline": {"value": value, "unit": "trajectory-steps/s", "cores": times[0]["cores"],
                         "kind": "oracle",
                         "sample": f"first {n_sample} of {w8.n_traj} trajectories, all {w8.n_steps} "
                                   f"steps and {w8.n_E} energies; rate is linear in trajectories"},
        "e2e": {"value": value, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def batch_arm(args):
    """48 molecules (F cycling over the recipe's classes 3, 6, 9, 12, 15, 24; n_traj
    log-uniform in [512, 32768]; steps uniform in [2000, 8000]) sampled, propagated in one
    persistent launch per F-class and transformed, all captured in one CUDA graph.  One
    batch takes tens of seconds on a GB300: time it with --steps 2."""
    import torch
    from paper_1312_4698_gb300 import scivr
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    mols = wl.batch_molecules(args.n_mol, seed=1000 * rank, Fs=(3, 6, 9, 12, 15, 24))
    prec = PRECISIONS[args.precision]
    ftm = FT_MODES[args.ft]
    entries = []
    for w8 in mols:
        pes = scivr.scivr_create_pes(w8.pes)
        bufs = scivr.alloc_buffers(w8)
        entries.append(dict(pes=pes, wl=w8, bufs=bufs, precision=prec,
                            stab_tol=MIXED_STAB_TOL if prec == 1 else w8.stab_tol))
    plan = scivr.scivr_batch_create(entries, ft_mode=ftm)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())

    def enqueue(stream):
        for e in entries:
            w8, b = e["wl"], e["bufs"]
            scivr.scivr_sample_initial(e["pes"], w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, w8.seed,
                                       b.p0, b.q0, b.w, stream)
        scivr.scivr_batch_launch(plan, stream)

    scivr.launch_count(reset=True)
    with torch.cuda.stream(side):
        enqueue(side)                      # eager run (warms the tuner's choices and caches)
    torch.cuda.synchronize()
    launches_per_step = scivr.launch_count(reset=True)   # kernels one graph replay contains
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        enqueue(side)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    scivr.launch_count(reset=True)
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_selector(local)) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            graph.replay()
        t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    if rank != 0:
        return 0
    traj_steps = sum(w8.n_traj * w8.n_steps for w8 in mols)
    flops = 0.0
    t_bound = 0.0
    probe = fma_peaks()
    for w8 in mols:
        bulk, kept = propagate_flops_split(w8.F, w8.pes.c3.size, w8.pes.c4.size, mixed=(prec != 0))
        flops += (bulk + kept) * w8.n_traj * w8.n_steps
        t_bound += (bulk * w8.n_traj * w8.n_steps) / (probe["fp32"] * 1e12) + \
                   (kept * w8.n_traj * w8.n_steps) / (probe["fp64"] * 1e12)
    achieved = flops / (ms * 1e-3) / 1e12
    eff_peak = flops / t_bound / 1e12
    groups = plan.groups()
    line = {
        "metric": METRIC, "value": world * traj_steps / (ms * 1e-3), "unit": "trajectory-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64"}[args.precision] + ("" if ftm == 0 else f" + {args.ft} tensor FT"),
        "data": "synthetic",
        "config": {"workload": f"batch of {len(mols)} molecules, F cycling over 3/6/9/12/15/24, n_traj log-uniform "
                               f"[512, 32768], steps uniform [2000, 8000], 4000 energies; sampling, "
                               f"propagation (persistent launches, see schedule) and spectra in one CUDA graph",
                   "global_batch": world * sum(w8.n_traj for w8 in mols),
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": f"replicas x{world}",
                   "autotuned_warps_per_cta": {f"F{F}": w for F, _, w in groups},
                   "schedule": ("one persistent launch over all F classes" if plan.one_launch()
                                else "one persistent launch per F class") + " (chosen by a timed probe of the plan)"},
        "spectra_per_s": world * len(mols) / (ms * 1e-3),
        "roofline": {"kernel": "k_propagate_lg_batch<float> (scivr_batch_launch)", "bound": "alu",
                     "achieved": achieved, "peak": eff_peak, "unit": "TFLOP/s", "frac": achieved / eff_peak,
                     "traffic": None, "peak_source": f"two-pipe bound summed over molecules (FP32 bulk at "
                                                     f"{probe['fp32']:.1f} + FP64-kept at {probe['fp64']:.3f} "
                                                     f"TFLOP/s, measured live by scivr_fma_probe)"},
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def mlp_flops_per_point(F: int, H: int = 256) -> float:
    """Algorithmic flops of one value + gradient + Hessian evaluation of the
    learned residual (multiply-add = 2 flops): layer 1 for the point and its F
    tangent directions, the two 256 x 256 forward layers on 1 + F rows, the two
    reverse layers on the point row, the output layer, and the Hessian terms
    J_l^T diag(c_l) J_l of the three layers (F(F+1)/2 pairs over H units each)."""
    R = F + 1
    fwd = 2 * (F * H + F * H) + 2 * 2 * R * H * H + 2 * H
    rev = 2 * 2 * H * H + 2 * F * H
    hess = 3 * 2 * (F * (F + 1) // 2) * H
    return float(fwd + rev + hess)


def surrogate_arm(args):
    """Learned-residual surface (F = 9 recipe): the network learns the coupling
    polynomial from 2^21 points of FP64 trajectories of the analytic surface
    (training untimed, reported), then each step samples, propagates on
    diagonal + network (one fused tensor-core evaluation per force stage) and
    takes the spectrum."""
    import torch
    import torch.distributed as dist
    from paper_1312_4698_gb300 import scivr, shards, surrogate as su

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w8 = sized(wl.config_f9(seed=rank), args)
    n, K = w8.n_traj, w8.n_steps + 1
    ftm = FT_MODES[args.ft]

    # ---- training set and training (untimed)
    full = scivr.scivr_create_pes(w8.pes)
    t0 = time.perf_counter()
    q = su.trajectory_points(full, w8, n_traj=65536, n_seg=32, seg_steps=20, seed=1000 + rank)
    V, g = su.coupling_targets(full, q)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = su.initial_network(w8, V, seed=rank)
    pes = scivr.scivr_create_pes(su.surrogate_pes(w8, net))
    res = su.train(pes, q, V, g, epochs=args.train_epochs, batch=16384, lr=3e-3)
    qh = su.trajectory_points(full, w8, n_traj=2048, n_seg=2, seg_steps=50, seed=2000 + rank)
    Vh, gh = su.coupling_targets(full, qh)
    Vn = torch.empty(qh.shape[0], device=dev)
    gn = torch.empty(qh.shape[0], w8.F, device=dev)
    scivr.scivr_mlp_eval(pes, qh.shape[0], qh.float().contiguous(), Vn, gn, None)
    held = {"V": float(torch.linalg.norm(Vn.double() - Vh) / torch.linalg.norm(Vh)),
            "grad": float(torch.linalg.norm(gn.double() - gh) / torch.linalg.norm(gh))}

    # ---- accuracy on a trajectory subset: surrogate vs the FP64 path (parity-tested
    # against the FP64 oracle) and vs the same run without the network
    n_chk = min(n, args.check_traj)
    wc = w8.with_(n_traj=n_chk)

    def spectrum_of(p_, precision, tol):
        b = scivr.alloc_buffers(wc, device=dev)
        scivr.scivr_sample_initial(p_, wc.gamma, wc.p_eq[0], wc.q_eq[0], n_chk, 77, b.p0, b.q0, b.w)
        scivr.scivr_propagate(p_, wc.dt, wc.n_steps, wc.gamma, wc.p_eq, wc.q_eq, n_chk, b.p0, b.q0, b.amp, K,
                              b.good, precision=precision, stab_tol=tol)
        scivr.scivr_spectrum(b.amp[0], K, b.w, b.good, n_chk, wc.n_steps, wc.dt, wc.E_min, wc.E_max, wc.n_E,
                             b.I[0], b.n_good)
        return b.I[0].cpu().numpy()

    I_ref = spectrum_of(full, PRECISIONS["fp64"], w8.stab_tol)
    I_sur = spectrum_of(pes, PRECISIONS["mixed"], MIXED_STAB_TOL)
    I_dia = spectrum_of(scivr.scivr_create_pes(su.diagonal_part(w8.pes)), PRECISIONS["fp64"], w8.stab_tol)
    E = wc.energies()
    pk_ref = wl.spectrum_peaks(E, I_ref)
    accuracy = {
        "trajectories": n_chk, "reference": "FP64 GPU path on the analytic surface (parity-tested "
                                            "against the FP64 oracle to 1e-9)",
        "peaks": int(pk_ref.size),
        "max_peak_shift_cm1": float(wl.to_cm1(wl.peak_shift(pk_ref, wl.spectrum_peaks(E, I_sur)))),
        "max_norm_error": float(np.max(np.abs(I_sur - I_ref)) / np.max(np.abs(I_ref))),
        "without_network_max_norm_error": float(np.max(np.abs(I_dia - I_ref)) / np.max(np.abs(I_ref))),
        "without_network_max_peak_shift_cm1": float(wl.to_cm1(wl.peak_shift(pk_ref, wl.spectrum_peaks(E, I_dia)))),
    }

    # ---- timed steps
    bufs = scivr.alloc_buffers(w8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = {k: [] for k in ("prop0", "prop1", "spec1")}

    def one_step(record):
        scivr.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], n, w8.seed, bufs.p0, bufs.q0, bufs.w,
                                   stream)
        if record:
            e0 = torch.cuda.Event(enable_timing=True); e0.record(stream); ev["prop0"].append(e0)
        scivr.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0, bufs.q0, bufs.amp,
                              K, bufs.good, precision=PRECISIONS["mixed"], stab_tol=MIXED_STAB_TOL, stream=stream)
        if record:
            e1 = torch.cuda.Event(enable_timing=True); e1.record(stream); ev["prop1"].append(e1)
        scivr.scivr_spectrum(bufs.amp[0], K, bufs.w, bufs.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E,
                             bufs.I[0], bufs.n_good, ft_mode=ftm, stream=stream)
        if record:
            e2 = torch.cuda.Event(enable_timing=True); e2.record(stream); ev["spec1"].append(e2)
        if world > 1:
            shards.combine_spectra_async(bufs.I[0], bufs.n_good)

    for _ in range(args.warmup):
        flush.zero_()
        one_step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    scivr.launch_count(reset=True)
    ts = torch.cuda.Event(enable_timing=True)
    te = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_selector(local)) as clk:
        ts.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            one_step(True)
        te.record(stream)
        torch.cuda.synchronize()
    launches = scivr.launch_count(reset=True)
    if world > 1:
        dist.barrier()
    t = torch.tensor([ts.elapsed_time(te)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / args.steps
    prop_avg = float(np.mean([a.elapsed_time(b) for a, b in zip(ev["prop0"], ev["prop1"])]))
    spec_avg = float(np.mean([a.elapsed_time(b) for a, b in zip(ev["prop1"], ev["spec1"])]))
    n_good = int(bufs.n_good.item())

    # ---- the dominant kernel (fused network evaluation), timed by itself at the same batch
    qe = (torch.randn(n, w8.F, device=dev, dtype=torch.float64) /
          torch.sqrt(torch.as_tensor(w8.pes.omega, device=dev))).float().contiguous()
    Ve = torch.empty(n, device=dev)
    ge = torch.empty(n, w8.F, device=dev)
    He = torch.empty(n, w8.F, w8.F, device=dev)
    for _ in range(3):
        scivr.scivr_mlp_eval(pes, n, qe, Ve, ge, He, stream)
    reps = 20
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        scivr.scivr_mlp_eval(pes, n, qe, Ve, ge, He, stream)
    k1.record(stream)
    torch.cuda.synchronize()
    eval_ms = k0.elapsed_time(k1) / reps

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hp0 = bufs.p0.cpu().pin_memory()
        hq0 = bufs.q0.cpu().pin_memory()
        hw = bufs.w.cpu().pin_memory()
        hI = torch.empty(w8.n_E, dtype=torch.float64).pin_memory()
        hng = torch.empty(1, dtype=torch.int64).pin_memory()
        h2d = (hp0.numel() + hq0.numel() + hw.numel()) * 8
        d2h = hI.numel() * 8 + 8
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            bufs.p0.copy_(hp0, non_blocking=True)
            bufs.q0.copy_(hq0, non_blocking=True)
            bufs.w.copy_(hw, non_blocking=True)
            scivr.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0, bufs.q0,
                                  bufs.amp, K, bufs.good, precision=PRECISIONS["mixed"], stab_tol=MIXED_STAB_TOL,
                                  stream=stream)
            scivr.scivr_spectrum(bufs.amp[0], K, bufs.w, bufs.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max,
                                 w8.n_E, bufs.I[0], bufs.n_good, ft_mode=ftm, stream=stream)
            hI.copy_(bufs.I[0], non_blocking=True)
            hng.copy_(bufs.n_good, non_blocking=True)
        a1.record(stream)
        torch.cuda.synchronize()
        tt = torch.tensor([a0.elapsed_time(a1)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item()) / args.steps
        e2e = {"value": world * n * w8.n_steps / (e2e_ms * 1e-3), "unit": "trajectory-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    peaks = measured_peaks()
    pk = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    achieved = mlp_flops_per_point(w8.F) * n / (eval_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        wcpu = w8.with_(pes=su.surrogate_pes(w8, wl.init_mlp(w8.F, 256, 0, s_in=np.sqrt(w8.pes.omega),
                                                               s_out=net.s_out)))
        ns = min(args.cpu_sample, 16)   # about 1 s of one core per trajectory-thousand-steps
        p0, q0, w = oracle.sample_initial(wcpu.gamma, wcpu.p_eq, wcpu.q_eq, ns, wcpu.seed)
        c0 = time.perf_counter()
        amp, good = oracle.propagate(wcpu.pes, wcpu.gamma, wcpu.p_eq, wcpu.q_eq, wcpu.dt, wcpu.n_steps, p0, q0,
                                     wcpu.stab_tol, 0)
        oracle.spectrum(amp[0], w, good, wcpu.n_steps, wcpu.dt, wcpu.E_min, wcpu.E_max, wcpu.n_E, 0)
        c1 = time.perf_counter()
        cpu = {"value": ns * wcpu.n_steps / (c1 - c0), "unit": "trajectory-steps/s",
               "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"{ns} of {n} trajectories on the same surface type (Morse diagonal + a 9-256-256-256-1 "
                         f"network of the same shape), all {w8.n_steps} steps and {w8.n_E} energies "
                         f"({c1 - c0:.1f} s); rate is linear in trajectories"}
    value = world * n * w8.n_steps / (ms_per_step * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "trajectory-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 x bf16 -> f32 network + f32/f64 propagation" + ("" if ftm == 0 else f" + {args.ft} tensor FT"),
        "data": "synthetic",
        "config": {"workload": f"{w8.name} with a learned coupling residual: Morse diagonal + 9-256-256-256-1 "
                               f"SiLU network (BF16 weights, FP32 accumulate), {n} trajectories, {w8.n_steps} "
                               f"steps of {w8.dt} au, {w8.n_E} energies, Fourier step {args.ft}",
                   "global_batch": world * n, "seed": "base 0 + rank",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write); amplitudes "
                         f"({n * K * 16 / 1e9:.2f} GB) exceed L2",
                   "parallelism": f"replicas x{world}",
                   "training": {"points": int(q.shape[0]), "source": "FP64 trajectories of the analytic "
                                "surface, every 20 steps, |sqrt(omega) q| <= 6", "data_s": t_data,
                                "steps": res.steps, "batch": 16384, "train_s": res.seconds,
                                "loss_first": res.losses[0], "loss_last": res.losses[-1],
                                "held_out_rel_error": held},
                   "accuracy": accuracy},
        "spectra_per_s": world / (ms_per_step * 1e-3),
        "propagate_ms": prop_avg, "spectrum_ms": spec_avg, "n_good": n_good,
        "network_eval_ms": eval_ms,
        "roofline": {"kernel": "k_mlp_fused<9> (scivr_mlp_eval at the propagation batch; 3 launches per step)",
                     "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                     "traffic": TRAFFIC[("k_mlp_fused", "f9mlp")] if n == 65536 else None,
                     "traffic_note": "ncu capture at 8192 points scaled by 8; outputs stay in L2",
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained of measured"
                                    if "bf16_tflops_sustained" in peaks else "fallback 1700 TFLOP/s sustained",
                     "note": f"{mlp_flops_per_point(w8.F):.3g} algorithmic flop per point (value, gradient, "
                             f"Hessian); tile padding and the 128-row reverse GEMMs are not counted"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def speedup_arm(args):
    """F uncoupled Morse oscillators (the speed-up-versus-F comparison of Sec. IV):
    GPU trajectory-steps/s of the FP64 propagation (F = 1..9, where it is built) and of
    the mixed propagation (F = 1..24), each with its Fourier step, against the oracle on
    one host core and on all host cores."""
    import torch
    from paper_1312_4698_gb300 import scivr
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    oracle.build()
    all_threads = oracle.max_threads()     # read before any single-thread run changes it
    n = args.n_traj or 16384
    steps = args.n_steps or 300
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    scivr.launch_count(reset=True)
    with ClockSampler(gpu_selector(0)) as clk:
        for F in range(1, 25):
            w8 = wl.uncoupled_morse(F, n_traj=n, n_steps=steps, n_E=2000)
            pes = scivr.scivr_create_pes(w8.pes)
            bufs = scivr.alloc_buffers(w8)
            scivr.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], n, 0, bufs.p0, bufs.q0, bufs.w)
            K = steps + 1
            row = {"F": F}
            paths = (("gpu_fp64", 0, 0, w8.stab_tol), ("gpu_mixed", 1, 2, MIXED_STAB_TOL))
            for name, prec, ftm, tol in paths:
                if prec == 0 and F > 9:
                    row[name] = None            # the FP64 schedules are built for F <= 9
                    continue
                def run():
                    scivr.scivr_propagate(pes, w8.dt, steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0, bufs.q0,
                                          bufs.amp, K, bufs.good, precision=prec, stab_tol=tol, stream=stream)
                    scivr.scivr_spectrum(bufs.amp[0], K, bufs.w, bufs.good, n, steps, w8.dt, w8.E_min, w8.E_max,
                                         w8.n_E, bufs.I[0], bufs.n_good, ft_mode=ftm, stream=stream)
                for _ in range(args.warmup):
                    flush.zero_()
                    run()
                torch.cuda.synchronize()
                ms = 0.0
                for _ in range(args.steps):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    run()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                row[name] = n * steps / (ms / args.steps * 1e-3)
            # the oracle on a bounded sample (about a second per F and thread setting)
            for name, threads in (("cpu_1core", 1), ("cpu_all", all_threads)):
                ns = max(16, int(2e6 / (steps * (F + 1) ** 2))) * threads
                p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, ns, 0)
                c0 = time.perf_counter()
                amp, good = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, steps, p0, q0,
                                             w8.stab_tol, threads)
                oracle.spectrum(amp[0], w, good, steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, threads)
                row[name] = ns * steps / (time.perf_counter() - c0)
            row["speedup_fp64_vs_1core"] = row["gpu_fp64"] / row["cpu_1core"] if row["gpu_fp64"] else None
            row["speedup_mixed_vs_1core"] = row["gpu_mixed"] / row["cpu_1core"]
            row["speedup_fp64_vs_all_cores"] = row["gpu_fp64"] / row["cpu_all"] if row["gpu_fp64"] else None
            rows.append(row)
    line = {
        "metric": METRIC, "value": rows[-1]["gpu_mixed"], "unit": "trajectory-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": n * steps / rows[-1]["gpu_mixed"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 and f32+f64", "data": "synthetic",
        "config": {"workload": f"uncoupled Morse oscillators F = 1..24 (omega ~ U[1100, 3000] cm^-1, D ~ U[0.15, "
                               f"0.25]), {n} trajectories, {steps} steps, 2000 energies; FP64 GPU path F <= 9; "
                               f"value = mixed path at F = 24",
                   "l2": f"flushed between runs ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "cpu_cores": all_threads},
        "sweep": rows,
        "gpu_launches": scivr.launch_count(reset=True),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="f9", choices=["f3", "f6", "f9", "batch", "f9mlp", "speedup"])
    ap.add_argument("--train-epochs", type=int, default=40, help="training epochs of --workload f9mlp")
    ap.add_argument("--check-traj", type=int, default=2048,
                    help="trajectories of the --workload f9mlp accuracy check")
    ap.add_argument("--n-mol", type=int, default=48, help="molecules in --workload batch")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="trajectories of the oracle timing (default: 1024 at F = 3, 768 at F = 6, 256 at F = 9)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the untimed comparison of the spectrum with the FP64 GPU path")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="propagation arithmetic (mixed: FP32 monodromy, potential and determinants; FP64 p, q, S, phase)")
    ap.add_argument("--ft", default="bf16x3", choices=list(FT_MODES),
                    help="Fourier step: fp64 CUDA cores or tensor-core BF16 digit splits")
    ap.add_argument("--amp-storage", default="auto", choices=["auto", "fp32", "fp64"],
                    help="amplitude rows: auto = complex float for mixed time-averaged runs, else double")
    ap.add_argument("--n-traj", type=int, default=None, help="override the workload's trajectory count")
    ap.add_argument("--n-steps", type=int, default=None, help="override the workload's step count")
    ap.add_argument("--n-E", type=int, default=None, help="override the workload's energy count")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="under torchrun: weak = one batch per rank (seed base + rank); strong = one batch "
                         "split into contiguous trajectory shards, spectra combined by one all-reduce")
    ap.add_argument("--amplitude", default="ta", choices=["ta", "hk"],
                    help="ta: time-averaged spectrum (Eq. I(E)_discreto); hk: plain Herman-Kluk SC-IVR "
                         "spectrum (Eq. I(E)_SCIVR)")
    args = ap.parse_args(argv)
    if args.cpu_sample is None:
        args.cpu_sample = CPU_SAMPLE.get(args.workload, 768)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch":
        return batch_arm(args)
    if args.workload == "f9mlp":
        return surrogate_arm(args)
    if args.workload == "speedup":
        return speedup_arm(args)

    import torch
    import torch.distributed as dist
    from paper_1312_4698_gb300 import scivr, shards

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # weak scaling: one batch per rank (seed base + rank); strong scaling: one batch (seed 0)
    # whose trajectories are split into contiguous shards, one per rank
    strong = args.scaling == "strong" and world > 1
    w8 = sized(workload(args.workload, seed=0 if strong else rank), args)
    n_job = w8.n_traj
    lo, hi = shards.shard_range(n_job, rank, world) if strong else (0, n_job)
    n = hi - lo                                  # this rank's trajectories
    pes = scivr.scivr_create_pes(w8.pes)
    # amplitude rows: complex float for the mixed path's time-averaged amplitudes (it forms
    # them in FP32), complex double otherwise
    amp_f32 = (args.amp_storage == "fp32" or
               (args.amp_storage == "auto" and args.precision == "mixed" and args.amplitude == "ta"))
    bufs = scivr.alloc_buffers(w8, device=dev, n_traj=n, amp_f32=amp_f32)
    full = scivr.alloc_buffers(w8.with_(n_steps=1, n_E=2), device=dev) if strong else None   # the job's samples
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    K = w8.n_steps + 1

    prec = PRECISIONS[args.precision]
    hk = args.amplitude == "hk"
    ftm = 0 if hk else FT_MODES[args.ft]
    amp_mode = scivr.SCIVR_AMP_HK if hk else scivr.SCIVR_AMP_TA
    tol = MIXED_STAB_TOL if prec == 1 else w8.stab_tol

    def spectrum_call():
        if hk:
            scivr.scivr_spectrum_hk(bufs.amp[0], K, bufs.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E,
                                    bufs.I[0], None, bufs.n_good, stream=stream)
        else:
            scivr.scivr_spectrum(bufs.amp[0], K, bufs.w, bufs.good, n, w8.n_steps, w8.dt, w8.E_min,
                                 w8.E_max, w8.n_E, bufs.I[0], bufs.n_good, ft_mode=ftm, stream=stream)
    ev = {k: [] for k in ("prop0", "prop1", "spec1")}
    combined = [None]

    def one_step(record):
        if strong:
            # the whole job's Husimi samples (the same Philox stream on every rank), then this
            # rank's contiguous shard
            scivr.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], n_job, w8.seed, full.p0,
                                       full.q0, full.w, stream)
            bufs.p0.copy_(full.p0[:, lo:hi])
            bufs.q0.copy_(full.q0[:, lo:hi])
            bufs.w.copy_(full.w[lo:hi])
        else:
            scivr.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], n, w8.seed, bufs.p0,
                                       bufs.q0, bufs.w, stream)
        if record:
            e0 = torch.cuda.Event(enable_timing=True); e0.record(stream); ev["prop0"].append(e0)
        scivr.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0, bufs.q0,
                              bufs.amp, K, bufs.good, precision=prec, stab_tol=tol, stream=stream,
                              amplitude=amp_mode)
        if record:
            e1 = torch.cuda.Event(enable_timing=True); e1.record(stream); ev["prop1"].append(e1)
        spectrum_call()
        if record:
            e2 = torch.cuda.Event(enable_timing=True); e2.record(stream); ev["spec1"].append(e2)
        if world > 1:
            # combine spectra across ranks: one all-reduce of n_good * I and n_good
            combined[0] = shards.combine_spectra_async(bufs.I[0], bufs.n_good)

    for _ in range(args.warmup):
        flush.zero_()
        one_step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    scivr.launch_count(reset=True)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_selector(local)) as clk:
        t_start.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            one_step(True)
        t_end.record(stream)
        torch.cuda.synchronize()
    launches = scivr.launch_count(reset=True)
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    prop_ms = [a.elapsed_time(b) for a, b in zip(ev["prop0"], ev["prop1"])]
    spec_ms = [a.elapsed_time(b) for a, b in zip(ev["prop1"], ev["spec1"])]
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / args.steps
    n_good = int(bufs.n_good.item())

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e:
        hp0 = bufs.p0.cpu().pin_memory()
        hq0 = bufs.q0.cpu().pin_memory()
        hw = bufs.w.cpu().pin_memory()
        hI = torch.empty(w8.n_E, dtype=torch.float64).pin_memory()
        hng = torch.empty(1, dtype=torch.int64).pin_memory()
        h2d = hp0.numel() * 8 + hq0.numel() * 8 + hw.numel() * 8
        d2h = hI.numel() * 8 + 8
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            flush.zero_()
            bufs.p0.copy_(hp0, non_blocking=True)
            bufs.q0.copy_(hq0, non_blocking=True)
            bufs.w.copy_(hw, non_blocking=True)
            scivr.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0,
                                  bufs.q0, bufs.amp, K, bufs.good, precision=prec, stab_tol=tol,
                                  stream=stream, amplitude=amp_mode)
            spectrum_call()
            hI.copy_(bufs.I[0], non_blocking=True)
            hng.copy_(bufs.n_good, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        te = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e_ms = float(te.item()) / args.steps
        e2e = {"value": (n_job if strong else world * n) * w8.n_steps / (e2e_ms * 1e-3),
               "unit": "trajectory-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_ms}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- accuracy of the timed configuration (untimed): the same initial conditions through
    # the FP64 GPU path, itself parity-tested against the FP64 oracle to 1e-9 relative
    accuracy = None
    if not args.no_accuracy and (prec != 0 or ftm != 0):
        ref = scivr.alloc_buffers(w8, device=dev)
        ref.p0.copy_(bufs.p0)
        ref.q0.copy_(bufs.q0)
        ref.w.copy_(bufs.w)
        scivr.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, ref.p0, ref.q0, ref.amp, K,
                              ref.good, precision=0, stab_tol=w8.stab_tol, stream=stream, amplitude=amp_mode)
        if hk:
            scivr.scivr_spectrum_hk(ref.amp[0], K, ref.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E,
                                    ref.I[0], None, ref.n_good, stream=stream)
        else:
            scivr.scivr_spectrum(ref.amp[0], K, ref.w, ref.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max,
                                 w8.n_E, ref.I[0], ref.n_good, stream=stream)
        torch.cuda.synchronize()
        E = w8.energies()
        I_ref = ref.I[0].cpu().numpy()
        I_got = bufs.I[0].cpu().numpy()
        pk_ref = wl.spectrum_peaks(E, I_ref)
        accuracy = {
            "reference": "FP64 GPU propagation and FP64 Fourier step on the same initial conditions "
                         "(parity-tested against the FP64 oracle to 1e-9 relative)",
            "n_peaks": int(pk_ref.size),
            "max_peak_shift_cm1": float(wl.to_cm1(wl.peak_shift(pk_ref, wl.spectrum_peaks(E, I_got)))),
            "max_rel_error": float(np.max(np.abs(I_got - I_ref)) / np.max(np.abs(I_ref))),
            "n_good": int(bufs.n_good.item()), "n_good_fp64": int(ref.n_good.item()),
        }
        del ref

    value = (n_job if strong else world * n) * w8.n_steps / (ms_per_step * 1e-3)
    prop_avg = float(np.mean(prop_ms))
    spec_avg = float(np.mean(spec_ms))
    # time-averaged: 8 N K N_E (complex multiply-add per trajectory, sample and energy);
    # plain HK: the column sum (2 N K) and the transform of the mean (8 K N_E)
    ft_flops = (2.0 * n * K + 8.0 * K * w8.n_E) if hk else 8.0 * n * K * w8.n_E
    bulk, kept = propagate_flops_split(w8.F, w8.pes.c3.size, w8.pes.c4.size, mixed=(prec != 0))
    pr_flops = (bulk + kept) * n * w8.n_steps
    ft_tf = ft_flops / (spec_avg * 1e-3) / 1e12
    pr_tf = pr_flops / (prop_avg * 1e-3) / 1e12
    peaks = measured_peaks()
    probe = fma_peaks(stream)                 # untimed: the FP32 / FP64 pipes' attainable rates
    fp64_peak = probe["fp64"]
    fp32_peak = probe["fp32"]
    probe_note = (f"measured live by scivr_fma_probe (independent FMA chains on every SM): FP32 "
                  f"{fp32_peak:.1f}, FP64 {fp64_peak:.3f} TFLOP/s of measured")
    full = args.n_traj is None and args.n_steps is None and args.n_E is None
    if spec_avg >= prop_avg:
        if ftm == 4:
            # chirp-z: per good trajectory and energy block two length-L FFTs (5 L log2 L flops each
            # for complex radix-2) and three complex products per point (input chirp, spectrum of
            # the chirp, |y|^2)
            L_czt = 8192
            nb = L_czt - K + 1
            n_blk = -(-w8.n_E // nb)
            czt_flops = n_good * n_blk * (2 * 5 * L_czt * 13 + 3 * 6 * L_czt)
            a = czt_flops / (spec_avg * 1e-3) / 1e12
            roof = {"kernel": "k_czt (scivr_spectrum, FP64 chirp-z)", "bound": "alu", "achieved": a,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": a / fp64_peak, "traffic": None,
                    "peak_source": probe_note,
                    "note": "achieved counts the transform's own FFT flops (10 L log2 L + 18 L per good "
                            "trajectory and energy block, L = 8192), not the direct sum's 8 N K N_E"}
        elif ftm == 0:
            roof = {"kernel": "k_ft_fp64 (scivr_spectrum)", "bound": "alu", "achieved": ft_tf,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": ft_tf / fp64_peak,
                    "traffic": TRAFFIC.get(("k_ft_fp64", args.workload)) if full else None,
                    "peak_source": probe_note}
        else:
            pk = float(peaks.get("bf16_tflops", 1900.0))
            roof = {"kernel": f"k_ft_tc<{ftm}> (scivr_spectrum, {args.ft})", "bound": "tensor",
                    "achieved": ft_tf, "peak": pk, "unit": "TFLOP/s", "frac": ft_tf / pk,
                    "traffic": TRAFFIC.get((f"k_ft_tc{ftm}", args.workload)) if full else None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst) of measured"
                                   if "bf16_tflops" in peaks else "fallback 1900 TFLOP/s",
                    "note": "achieved counts the 8 N K N_E algorithmic flops; the digit "
                            "products multiply the executed tensor flops"}
    else:
        if prec == 0:
            roof = {"kernel": "k_propagate (scivr_propagate, fp64)", "bound": "alu", "achieved": pr_tf,
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": pr_tf / fp64_peak, "traffic": None,
                    "peak_source": probe_note}
        else:
            # two pipes: the FP32 bulk at the FP32 peak plus the FP64-kept part at the FP64 peak
            t_bound = (bulk * n * w8.n_steps) / (fp32_peak * 1e12) + \
                      (kept * n * w8.n_steps) / (fp64_peak * 1e12)
            eff_peak = pr_flops / t_bound / 1e12
            tr = TRAFFIC.get(("k_propagate_lg_mixed", args.workload, "f32" if amp_f32 else "f64"))
            roof = {"kernel": "k_propagate_lg<float> (scivr_propagate, mixed)", "bound": "alu",
                    "achieved": pr_tf, "peak": eff_peak, "unit": "TFLOP/s", "frac": pr_tf / eff_peak,
                    "traffic": tr * n * w8.n_steps if (tr is not None and full) else None,
                    "peak_source": (f"two-pipe bound: FP32 bulk {bulk:.0f} flop/step at {fp32_peak:.1f} "
                                    f"TFLOP/s + FP64-kept {kept:.0f} flop/step at {fp64_peak:.3f} TFLOP/s, "
                                    f"both {probe_note.split(': ', 1)[0]}"),
                    "nominal_fp32_peak": FP32_PEAK_GFLOPS / 1e3}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        r = run_cpu_oracle(w8, args.cpu_sample, 0, args.amplitude)
        cpu = {"value": r["value"], "unit": "trajectory-steps/s", "cores": r["cores"],
               "kind": "oracle",
               "sample": f"first {args.cpu_sample} of {n} trajectories, all {w8.n_steps} steps and "
                         f"{w8.n_E} energies ({r['seconds']:.1f} s); rate is linear in trajectories"}

    line = {
        "metric": METRIC, "value": value, "unit": "trajectory-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "strong" if strong else "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f32+f64"}[args.precision] + ("" if ftm == 0 else f" + {args.ft} FT"),
        "data": "synthetic",
        "config": {"workload": describe(w8, args.precision, args.ft, args.amplitude),
                   "global_batch": n_job if strong else world * n,
                   "seed": "0, one batch split into trajectory shards" if strong else "base 0 + rank",
                   "amplitude_storage": "complex float (8 B a sample)" if amp_f32 else "complex double (16 B)",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write); amplitudes "
                         f"({n * K * (8 if amp_f32 else 16) / 1e9:.2f} GB) exceed L2",
                   "parallelism": (f"trajectory shards x{world} (one all-reduce of n_E + 1 numbers)" if strong
                                   else f"replicas x{world}")},
        "spectra_per_s": world / (ms_per_step * 1e-3),
        "propagate_ms": prop_avg, "spectrum_ms": spec_avg, "n_good": n_good,
        "propagate_tflops": pr_tf, "spectrum_tflops": ft_tf,
        "roofline": roof,
        "fma_probe_tflops": probe,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "accuracy": accuracy,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
