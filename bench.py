"""Benchmark: tree-force particle updates per second on one GB300 per rank.

A step is one kick-drift-kick step of the periodic treecode (keys, sort,
tree, moments, group walk with P2P/M2P, image field, both kicks and the
drift) on the 128^3 Zel'dovich + 64 NFW halo workload (L = 250 Mpc/h,
theta = 0.6, hexadecapole, eps = spacing/30), inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun every rank runs an independent realisation (seed + rank) on
its own GPU (weak scaling, no data-path collective); rank 0 prints one JSON
line.  --impl reference times the FP64 CPU oracle tree on a bounded sample
of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tree-force particle updates/s at median force err ≤1e-3; adjoint/forward ratio"
UNIT = "particle updates/s"
H0 = math.sqrt(8.0 * math.pi / 3.0)
NG = 128
A_START = 0.02
DLNA = 0.1
THETA = 0.6
ORDER = 4
EWALD_GRID = 5       # groups never straddle a level-4 cell (measured accuracy setting)
N_DIRECT = 8         # accepted cells with <= 8 particles summed directly (fastest of 4/8/12/16 measured)
FP32_FLOPS_P2P = 19  # dx,dy,dz (3 FADD), r^2+eps^2 (3 FMA), rsqrt, 3 FMUL, 3 FMA
# DRAM traffic of one walk (per force evaluation) from the ncu captures
# summarised in profiles/ (96^3, packed variant with 8 warps x 2 blocks),
# scaled by the particle count to 2^21 particles (x 2.370): in the dual form
# the walk kernel, the cell-group expansion kernel and their evaluation
# (143.4 + 233.8 + 160.8 MB); in the M2P form the walk kernel (44.4 MB,
# captured on earlier sources).  Reported only while the walk's sources are
# the ones captured (hash of walk.cu, walk_common.cuh, m2p_gen.cuh,
# common.cuh).
WALK_TRAFFIC = {"dual": {"bytes": 1.275e9, "source_sha": "70ff0906ff041c4c"},
                "m2p": {"bytes": 105e6, "source_sha": "4124360064afd5ea"}}
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2  # GB300's nominal FP64 rate (1.25 TFLOP/s) over 152 SMs at 2070 MHz
SM_MAX_MHZ = 2070.0
# accuracy of the timed settings against the FP64 direct Ewald sum, from the
# oracle tree (same discrete decisions as the GPU; per-particle |da|/|a|):
# the metric counts a setting at median <= 1e-3; the 99th percentile is
# reported beside it (p99_le_1e-2).  The benchmark workload's figures are on
# its configuration's seeded subset of 4096 particles (ics.random_targets(n,
# 4096, 2024)); tests/test_gpu_fullsize.py asserts them on the GPU.
# p99_abs_over_rms: the 99th percentile of |da| over the rms acceleration
# (the paper's own tolerance is absolute errors of 0.1 % of the rms)
ERR_BENCH = {"median": 7.2e-4, "p99": 1.20e-2, "targets": 4096, "p99_abs_over_rms": 3.0e-4}
# the same workload with the dual (cell-group) form, NBODY_FLAG_DUAL
ERR_BENCH_DUAL = {"median": 8.3e-4, "p99": 1.34e-2, "targets": 4096, "p99_abs_over_rms": 3.1e-4}
ERR_CONFIG3 = {"median": 3.7e-4, "p99": 1.6e-3, "targets": 256}
FORMS = {"m2p": "M2P: every accepted cell expanded at every sink",
         "dual": "dual: far cells through one local expansion per group (cell-group M2L, L2P)"}


def workload(seed: int, ng: int = NG):
    """Positions (n,3) and momenta (n,3) at a = A_START, plus eps.  ng < 128
    scales the halo counts with the particle number (profiling runs)."""
    from paper_1407_2600_gb300 import ics
    q, psi = ics.zeldovich_particles(ng, -2.0, 0.6, seed)
    x = np.mod(q + psi, 1.0)
    # growing-mode momentum of the displacement psi at a: p = H0 a^(1/2) psi
    p = H0 * math.sqrt(A_START) * psi
    f = (ng / NG) ** 3
    x, members, _ = ics.add_nfw_haloes(x, 64, max(2, int(2000 * f)), max(3, int(50000 * f)), 5.0, 15.0,
                                       seed + 1000)
    p[members] = 0.0  # halo particles start at rest (their centre's velocity is not modelled)
    return x, p, 1.0 / (30.0 * ng)


def m2p_flops(order: int) -> int:
    """Flops per M2P of the generated kernel (FMA = 2, rsqrt = 1)."""
    sys.path.insert(0, os.path.join(ROOT, "paper_1407_2600_gb300", "csrc"))
    import gen_m2p
    return gen_m2p.flop_count(order)


def bg_flops(order: int) -> int:
    """Extra flops per M2P of the uniform-background term at this order."""
    sys.path.insert(0, os.path.join(ROOT, "paper_1407_2600_gb300", "csrc"))
    import gen_m2p
    return gen_m2p.bg_flop_count(gen_m2p.bg_order(order))


def walk_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("walk.cu", "walk_common.cuh", "m2p_gen.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1407_2600_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def hbm_peak():
    """(GB/s, source) of the HBM copy bandwidth the phases are measured against."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def phase_bytes(n, ncell, ngroup, order, nbox=1):
    """Algorithmic DRAM bytes of one build's sort, build and upward phases and
    of one evaluation's image-field phase: every array their kernels read or
    write, counted once, per particle / cell / group:
      sort     box ids 2, keys 36, histograms 8, 24 per digit pass, sbox 8, gather 58
      build    152 per particle + 194 per cell + 168 per group
      upward   28 per particle + (91 + 16 nmom + 4 nbs) per cell (the image-field
               source moments are the tree's level-3 moments, copied)
      periodic 64 per particle (image-field L2P and the scatter to caller order)"""
    npass = 8 + (0 if nbox == 1 else (1 if nbox <= 256 else 2))
    nm = (order + 1) * (order + 2) * (order + 3) // 6
    nbs = {0: 4, 1: 4, 2: 12, 3: 24, 4: 48}[order]
    return {"ms_sort": n * (112 + 24 * npass), "ms_build": n * 152 + ncell * 194 + ngroup * 168,
            "ms_upward": n * 28 + ncell * (91 + 16 * nm + 4 * nbs), "ms_periodic": n * 64}


def upward_flops(n, ncell, order, nbox=1) -> float:
    """FP64 flops of one upward pass: P2M per particle, one M2M shift per
    non-root cell, scaling and reduction per cell (generated code's counts)."""
    sys.path.insert(0, os.path.join(ROOT, "paper_1407_2600_gb300", "csrc"))
    import gen_m2p
    fl = gen_m2p.upward_flop_counts(order)
    return n * fl["p2m_per_particle"] + (ncell - nbox) * fl["m2m_per_daughter"] + ncell * fl["per_cell"]


def fp64_peak_tflops(mhz: float, sms: int) -> float:
    """FP64 peak: GB300's nominal 1.25 TFLOP/s is two FP64 FMA per SM per
    clock at 2070 MHz over 152 SMs (1.26 TFLOP/s); SMs x 2 x 2 flop x clock."""
    return sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12


def phase_roofline(n, ncell, ngroup, order, phases, nbox=1, sms=152):
    peak, src = hbm_peak()
    by = phase_bytes(n, ncell, ngroup, order, nbox)
    bound = {"ms_sort": "hbm", "ms_build": "latency (prefix searches)", "ms_upward": "fp64 pipe",
             "ms_periodic": "hbm"}
    out = {}
    for k, b in by.items():
        gbs = b / (phases[k] * 1e-3) / 1e9
        out[k[3:]] = {"bytes": b, "achieved_gbs": gbs, "frac": gbs / peak, "bound": bound[k]}
    # the upward pass against the FP64 pipe it is bound by
    fl = upward_flops(n, ncell, order, nbox)
    p64 = fp64_peak_tflops(SM_MAX_MHZ, sms)
    t64 = fl / (phases["ms_upward"] * 1e-3) / 1e12
    out["upward"].update({"fp64_flops": fl, "fp64_tflops": t64, "fp64_peak_tflops": p64, "fp64_frac": t64 / p64})
    out["peak_gbs"] = peak
    out["peak_source"] = src
    return out


def sm_count(dev) -> int:
    """Streaming multiprocessors of the device (cudaDeviceProp.multiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def fp32_peak_tflops(mhz: float, sms: int) -> float:
    """FP32 non-tensor peak: SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def meets_bar(err) -> bool:
    """The metric's accuracy bar: median relative force error <= 1e-3."""
    return err is not None and err["median"] <= 1e-3


def with_bar(err) -> dict:
    """An accuracy record with the metric's bar and the 99th-percentile check."""
    return dict(err, meets_accuracy_bar=meets_bar(err), **{"p99_le_1e-2": err["p99"] <= 1e-2})


def detail_path(args) -> str:
    """Where the full per-leg records go (the printed line keeps the summary):
    --detail-file, relative to the repository root unless absolute."""
    return os.path.join(ROOT, args.detail_file)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return summarise_clocks(self.lines)


def summarise_clocks(lines):
    """Median SM clock, maximum clock and the throttle reasons seen, from
    nvidia-smi lines in ClockSampler.FIELDS order (csv, no header, no units);
    lines that do not parse are skipped; None without any sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [t.strip() for t in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if f[5 + k].lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
            "samples": len(sm)}


def cpu_reference(x, eps, sample: int, seed: int):
    """Time the FP64 CPU oracle tree on a bounded sample: one tree build of
    all particles plus the walk of the groups that hold `sample` random
    targets (every sink of those groups is evaluated).  Returns the sample's
    own rate (sinks evaluated / wall time of the call), the rate of a whole
    evaluation extrapolated from it, and details."""
    import oracle
    from paper_1407_2600_gb300 import ics
    n = len(x)
    prm = oracle.tree_params(eps, THETA, ORDER, n_direct=N_DIRECT, ewald=4, ew_grid=EWALD_GRID)
    oracle.phitilde_lattice(EWALD_GRID, 5)  # build the oracle's table outside the timing
    t0 = time.perf_counter()
    oracle.tree_forces(x, None, prm, targets=np.array([0], dtype=np.int64))
    t_build = time.perf_counter() - t0
    tg = ics.random_targets(n, sample, seed)
    t0 = time.perf_counter()
    _, st = oracle.tree_forces(x, None, prm, targets=tg, return_stats=True)
    t_call = time.perf_counter() - t0
    sinks = int(st["sinks"])
    t_walk = max(t_call - t_build, 1e-9)
    t_eval = t_build + t_walk / sinks * n
    return {"sample_rate": sinks / t_call, "extrapolated_rate": n / t_eval, "t_call_s": t_call,
            "t_build_s": t_build, "sinks": sinks, "targets": len(tg)}


def run_reference(args, rank, world):
    """The CPU oracle tree as the reference arm: every step is one bounded
    sample (tree build of all particles + the walk of the groups of 256
    random targets); `value` is the sample's own rate (sinks evaluated per
    second of the step's wall time) and `ms_per_step` that wall time."""
    if rank != 0:
        return 0
    x, _, eps = workload(1)
    n = len(x)
    res = []
    for it in range(args.warmup + args.steps):
        r = cpu_reference(x, eps, 256, 100 + it)
        if it >= args.warmup:
            res.append(r)
    value = float(np.median([r["sample_rate"] for r in res]))
    ms = 1e3 * float(np.median([r["t_call_s"] for r in res]))
    sinks = int(np.median([r["sinks"] for r in res]))
    cores = os.cpu_count()
    sample = ("per step: FP64 CPU oracle tree, one build of all %d particles plus the walk of the groups of "
              "256 random targets (%d sinks evaluated); value = sinks / step wall time" % (n, sinks))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "128^3 Zel'dovich (P~k^-2, rms 0.6 spacing) + 64 NFW haloes, theta=0.6, p=4",
                   "n": n, "theta": THETA, "order": ORDER},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "extrapolated_full_evaluation_updates_per_s": float(np.median([r["extrapolated_rate"] for r in res])),
    }
    print(json.dumps(_sig(line)), flush=True)
    return 0


def reduce_over_ranks(ms: float, n_local: int, steps: int, world: int, device):
    """Whole-job throughput of independent per-rank boxes: the slowest rank's
    timed region (max over ranks) and the particles of all ranks (sum).
    Returns (t_max in ms, total particles, particle updates/s)."""
    import torch
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        m = torch.tensor([n_local], dtype=torch.int64, device=device)
        torch.distributed.all_reduce(m, op=torch.distributed.ReduceOp.SUM)
        ms, n_all = float(t.item()), int(m.item())
    else:
        n_all = n_local
    return ms, n_all, n_all * steps / (ms * 1e-3)


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nb.lib()
    x, p, eps = workload(1 + rank, args.ng)
    n = len(x)
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)
    mom = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float32, device=dev)
    dual_main = args.form == "dual"
    fl = nb.NBODY_FLAG_ASYNC | (nb.NBODY_FLAG_DUAL if dual_main else 0)
    if args.walk_variant is not None:  # a fixed launch variant instead of the autotuner's pick (profiling)
        fl |= nb.NBODY_FLAG_WALK_VARIANT(args.walk_variant)
    prm = nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=args.n_direct, ewald_grid=args.ewald_grid,
                    flags=fl)
    tree = nb.Tree(prm, pos)
    acc = tree.forces()
    a = A_START
    for _ in range(args.warmup):
        a1 = a * math.exp(DLNA)
        tree.kdk_step(mom, acc, a, a1)
        a = a1
    torch.cuda.synchronize()
    tree.timing(reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        a1 = a * math.exp(DLNA)
        tree.kdk_step(mom, acc, a, a1)
        a = a1
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ck = clocks.stop()
    rc = nb.nbody_check(tree.handle, nb._stream())
    if rc != nb.NBODY_OK:
        raise nb.NbodyError(rc, "timed KDK steps")
    if world > 1:
        torch.distributed.barrier()
    tm = tree.timing(reset=True)
    t_max, n_all, value = reduce_over_ranks(ms, n, args.steps, world, dev)

    # roofline of the dominant kernel (the walk), from the timed region
    evals = max(tm["evaluations"], 1)
    walk_ms = tm["ms_walk"] / evals
    flops = (tm["p2p"] * FP32_FLOPS_P2P + tm["m2p"] * m2p_flops(ORDER)) / evals
    if dual_main:  # per (cell, group) expansion its M2L, per sink the L2P
        flops += tm["m2l_dual"] * m2l_dual_flops(ORDER) / evals + n * l2p_flops(ORDER)
    sms = sm_count(dev)
    peak = fp32_peak_tflops(SM_MAX_MHZ, sms)
    achieved = flops / (walk_ms * 1e-3) / 1e12
    phases = {k: tm[k] / max(tm["builds"] if k in ("ms_sort", "ms_build", "ms_upward") else evals, 1)
              for k in ("ms_sort", "ms_build", "ms_upward", "ms_walk", "ms_periodic")}
    phase_rf = phase_roofline(n, nb.nbody_tree_count(tree.handle, nb.EXPORT["cell_keys"]),
                              nb.nbody_tree_count(tree.handle, nb.EXPORT["groups"]), ORDER, phases, sms=sms)

    # force evaluation alone (no kicks/drift, tree rebuilt each time)
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe0.record(stream)
    for _ in range(args.steps):
        tree.rebuild()
        tree.forces(acc)
    fe1.record(stream)
    torch.cuda.synchronize()
    force_ms = fe0.elapsed_time(fe1) / args.steps
    tree.timing(reset=True)

    # the same force evaluation with the dual (cell-group) form: accepted
    # cells far enough from a group enter one local expansion of the group
    other = run_form(dev, pos, eps, args, force_ms, sms, not dual_main) if args.other_form else None

    # end to end through the C ABI with host buffers: H2D of the state, the
    # step, D2H of the updated state, every step
    e2e = None
    if not args.no_e2e:
        hpos = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        hmom = torch.empty((3, n), dtype=torch.float32, pin_memory=True)
        hacc = torch.empty((3, n), dtype=torch.float32, pin_memory=True)
        hpos.copy_(pos)
        hmom.copy_(mom)
        hacc.copy_(acc)
        torch.cuda.synchronize()
        k2 = max(2, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(k2):
            pos.copy_(hpos, non_blocking=True)
            mom.copy_(hmom, non_blocking=True)
            acc.copy_(hacc, non_blocking=True)
            a1 = a * math.exp(DLNA)
            tree.kdk_step(mom, acc, a, a1)
            a = a1
            hpos.copy_(pos, non_blocking=True)
            hmom.copy_(mom, non_blocking=True)
            hacc.copy_(acc, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        t_e2e = time.perf_counter() - t0
        _, _, e2e_rate = reduce_over_ranks(t_e2e * 1e3, n, k2, world, dev)
        e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": 48 * n,
               "d2h_bytes_per_step": 48 * n}

    # reverse mode: a checkpointed trajectory of S steps (checkpoints every 4)
    # forward, then its reverse sweep (states recomputed from the checkpoints,
    # steps reversed by chained nbody_kdk_adjoint_acc calls), as the
    # differentiable-trajectory wrapper runs them
    adj = None
    if not args.no_adjoint:
        from paper_1407_2600_gb300.autograd import forward_steps, reverse_steps
        S = args.adjoint_steps
        a_list = [a * math.exp(DLNA * k) for k in range(S + 1)]
        g = torch.Generator(device=dev)
        g.manual_seed(17 + rank)
        lx = torch.randn((3, n), dtype=torch.float64, device=dev, generator=g)
        lp = torch.randn((3, n), dtype=torch.float32, device=dev, generator=g)
        # the reverse mode is written for the M2P form: with the dual form as
        # the headline its trajectory runs on a tree of its own
        atree, aacc = tree, acc
        if dual_main:
            atree = nb.Tree(nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=args.n_direct,
                                      ewald_grid=args.ewald_grid, flags=nb.NBODY_FLAG_ASYNC), pos)
            aacc = atree.forces()
        # warm-up: one reverse step (runs the reverse walk's autotuner)
        atree.kdk_adjoint(pos.clone(), mom.clone(), a_list[0], a_list[1], lx, lp, acc0=aacc.clone())
        torch.cuda.synchronize()
        atree.timing(reset=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        ckpt = forward_steps(atree, pos, mom, aacc, a_list, 4)
        ev[1].record(stream)
        ev[2].record(stream)
        lx0, lp0 = reverse_steps(atree, ckpt, a_list, lx, lp)
        ev[3].record(stream)
        torch.cuda.synchronize()
        rc = nb.nbody_check(atree.handle, nb._stream())
        if rc != nb.NBODY_OK:
            raise nb.NbodyError(rc, "timed reverse sweep")
        ta = atree.timing(reset=True)
        if atree is not tree:
            atree.close()
        t_fwd = ev[0].elapsed_time(ev[1]) / S
        t_bwd = ev[2].elapsed_time(ev[3]) / S
        adj = {"backward_ms_per_step": t_bwd, "forward_ms_per_step": t_fwd, "ratio": t_bwd / t_fwd,
               "steps": S, "checkpoint_every": 4, "adjoint_calls": ta["adjoint_steps"],
               "adjoint_calls_reusing": ta["adjoint_reused"],
               "finite": bool(torch.isfinite(lx0).all().item() and torch.isfinite(lp0).all().item()),
               "form": "m2p",
               "note": "backward = reverse sweep incl. the recompute of every state from its checkpoint; "
                       "forward = the same trajectory's KDK steps with checkpoint copies (M2P form)"}
        a = a_list[-1]

    # the same force evaluation with FP64 interactions (same tree, theta and
    # order: the force error is the tree's, as in mixed precision)
    fp64 = None
    if args.fp64:
        prm64 = nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=args.n_direct, ewald_grid=args.ewald_grid,
                          precision=1, flags=nb.NBODY_FLAG_ASYNC)
        t64 = nb.Tree(prm64, pos)
        a64 = t64.forces()
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        t64.rebuild()
        t64.forces(a64)
        d1.record(stream)
        torch.cuda.synchronize()
        rc = nb.nbody_check(t64.handle, nb._stream())
        if rc != nb.NBODY_OK:
            raise nb.NbodyError(rc, "FP64 force evaluation")
        ms64 = d0.elapsed_time(d1)
        t64.timing(reset=True)
        # the mixed-precision result of the same method (the FP64 walk has the M2P form)
        t32 = nb.Tree(nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=args.n_direct,
                                ewald_grid=args.ewald_grid, flags=nb.NBODY_FLAG_ASYNC), pos)
        a32 = t32.forces()
        torch.cuda.synchronize()
        t32.close()
        dif = torch.linalg.norm(a32 - a64, dim=0) / torch.linalg.norm(a64, dim=0)
        fp64 = {"force_eval_ms": ms64, "updates_per_s": n / (ms64 * 1e-3),
                "mixed_over_fp64_speed": ms64 / force_ms,
                "mixed_vs_fp64_rel_diff": {"median": float(dif.median()), "p99": float(torch.quantile(dif[:1 << 20], 0.99))},
                "note": "precision=1: FP64 interactions and coefficients, M2P form (FP32 output); the speed "
                        "ratio is against the headline form's force evaluation, the difference against the "
                        "M2P form in mixed precision"}
        t64.close()

    batched = None
    if args.batched:
        batched = run_batched(dev, max(2, args.steps // 2))
    block = run_block_steps(dev, x, p, eps, args) if args.block_steps else None
    config3 = run_config3(dev, sms) if args.config3 else None

    base = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            det = cpu_reference(x, eps, 128, 7)
            base = {"value": det["extrapolated_rate"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                    "sample": "FP64 CPU oracle tree: build of all %d particles + walk of the groups of %d "
                              "random targets (%d sinks, %.1f s), scaled to one evaluation"
                              % (n, det["targets"], det["sinks"], det["t_call_s"])}
        except Exception as exc:  # the oracle is optional on a box without a compiler
            base = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                    "sample": "failed: %s" % exc}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("%d^3" % args.ng) + " Zel'dovich (P~k^-2, rms 0.6 spacing, a=0.02) + 64 NFW haloes "
                                   "(2k-50k particles, c 5-15), L=250 Mpc/h, eps=spacing/30; KDK steps "
                                   "of dln a = 0.1",
                       "n": n, "theta": THETA, "order": ORDER, "n_group": 32, "n_leaf": 16,
                       "n_direct": args.n_direct, "form": FORMS[args.form],
                       "ewald_order": 4, "ewald_grid": args.ewald_grid, "precision": "FP32 interactions, "
                       "FP64 positions/moments",
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "dp%d (independent realisations)" % world},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": (WALK_TRAFFIC[args.form]["bytes"] if args.ng == NG and
                                     walk_source_sha() == WALK_TRAFFIC[args.form]["source_sha"] else None),
                         "kernel": ("walk_kernel + dual_m2l_kernel + dual_l2p_kernel" if dual_main else "walk_kernel"), "flops_per_launch": flops, "sm_count": sms,
                         "peak_note": "FP32 non-tensor: %d SMs x 128 lanes x 2 x 2070 MHz" % sms},
            "cpu_baseline": base,
            "e2e": e2e,
            "gpu_launches": tm["launches"] // 1,
            "clocks": ck,
            # measured by the oracle on the benchmark workload only (other sizes profile)
            "force_error_oracle": (with_bar(ERR_BENCH_DUAL if dual_main else ERR_BENCH) if args.ng == NG
                                   else None),
            "phases_ms": {k[3:]: round(v, 4) for k, v in phases.items()},
            "phase_roofline": dict({k: round(v["frac"], 4) for k, v in phase_rf.items() if isinstance(v, dict)},
                                   upward_fp64=round(phase_rf["upward"]["fp64_frac"], 4)),
            "force_updates_per_s": n / (force_ms * 1e-3),
            "interactions_per_particle": {"p2p": tm["p2p"] / evals / n, "m2p": tm["m2p"] / evals / n},
            "adjoint_forward_ratio": adj["ratio"] if adj else None,
            "other_form": _summary(other, ("form", "force_updates_per_s", "walk_frac",
                                           "meets_accuracy_bar")),
            "fp64_tree": None if fp64 is None else {"force_eval_ms": fp64["force_eval_ms"],
                                                    "mixed_over_fp64_speed": fp64["mixed_over_fp64_speed"],
                                                    "rel_diff": fp64["mixed_vs_fp64_rel_diff"]},
            "batched": _summary(batched, ("updates_per_s", "meets_accuracy_bar",
                                          "graph_state_equals_uncaptured", "tuned_force_updates_per_s")),
            "block_steps": _summary(block, ("speedup_vs_all_finest", "force_updates_per_s")),
            "config3": _summary(config3, ("updates_per_s", "ms_per_kdk_step", "phases_ms", "walk_frac",
                                          "meets_accuracy_bar")),
            "detail_file": os.path.relpath(detail_path(args), ROOT),
        }
        detail = {"phase_roofline": phase_rf, "walk_autotune": {
                      "variant": tm["walk_variant"], "tuning_ms": tm["walk_tune_ms"][:4],
                      "variants": (["scalar, 8 warps x 2 blocks/SM", "packed FP32x2, 4 x 3", "packed FP32x2, 8 x 2",
                                    "packed FP32x2, 4 x 4"] if dual_main else
                                   ["scalar M2P, 8 warps x 2 blocks/SM", "scalar M2P, 4 x 4",
                                    "packed FP32x2 M2P, 8 x 2", "packed FP32x2 M2P, 4 x 4"])},
                  "walk_traffic_last_capture": {"bytes": WALK_TRAFFIC[args.form]["bytes"],
                                                "source_sha": WALK_TRAFFIC[args.form]["source_sha"],
                                                "current_sha": walk_source_sha()},
                  "adjoint": adj, "fp64_tree": fp64, "other_form": other, "batched": batched, "block_steps": block,
                  "config3": config3}
        try:
            with open(detail_path(args), "w") as f:
                json.dump(detail, f, indent=1)
        except OSError:
            line["detail_file"] = None
        head = {k: line[k] for k in ("value", "ms_per_step")}
        print(json.dumps(dict(_sig(line), **head)), flush=True)
    tree.close()
    return 0


def run_form(dev, pos, eps, args, force_ms, sms, dual):
    """One rebuild + force evaluation of the benchmark workload in the other
    walk form than the headline's (median of 5, after a warm-up that runs its
    walk autotuner), its interaction counts and walk flops: with the dual form
    per (cell, group) expansion the generated M2L's flops plus the derivative
    tensor's, per sink the L2P."""
    try:
        import torch
        import paper_1407_2600_gb300.nbody as nb
        prm = nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=args.n_direct, ewald_grid=args.ewald_grid,
                        flags=nb.NBODY_FLAG_ASYNC | (nb.NBODY_FLAG_DUAL if dual else 0))
        tree = nb.Tree(prm, pos)
        acc = tree.forces()
        torch.cuda.synchronize()
        tree.check()
        tree.timing(reset=True)
        stream = torch.cuda.current_stream()
        ms = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree.rebuild()
            tree.forces(acc)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        tree.check()
        tm = tree.timing(reset=True)
        ngroup = nb.nbody_tree_count(tree.handle, nb.EXPORT["groups"])
        tree.close()
        n = pos.shape[1]
        ev = max(tm["evaluations"], 1)
        t = float(np.median(ms))
        walk_ms = tm["ms_walk"] / ev
        flops = (tm["p2p"] * FP32_FLOPS_P2P + tm["m2p"] * m2p_flops(ORDER)) / ev
        if dual:
            flops += tm["m2l_dual"] * m2l_dual_flops(ORDER) / ev + n * l2p_flops(ORDER)
        err = (ERR_BENCH_DUAL if dual else ERR_BENCH) if args.ng == NG else None  # oracle-measured at 128^3
        return {"form": "dual" if dual else "m2p", "force_eval_ms": t, "force_updates_per_s": n / (t * 1e-3),
                "speed_vs_headline_form": force_ms / t,
                "walk_ms": walk_ms, "walk_tflops": flops / (walk_ms * 1e-3) / 1e12,
                "walk_frac": flops / (walk_ms * 1e-3) / 1e12 / fp32_peak_tflops(SM_MAX_MHZ, sms),
                "interactions_per_particle": {"p2p": tm["p2p"] / ev / n, "m2p": tm["m2p"] / ev / n},
                "cell_group_expansions_per_group": tm["m2l_dual"] / ev / max(1, ngroup),
                "force_error_oracle": with_bar(err) if err else None,
                "meets_accuracy_bar": meets_bar(err) if err else None,
                "walk_variant": tm["walk_variant"]}
    except Exception as exc:  # a side measurement: a failure is reported in the line, not raised
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def m2l_dual_flops(order: int) -> int:
    sys.path.insert(0, os.path.join(ROOT, "paper_1407_2600_gb300", "csrc"))
    import gen_m2p
    return gen_m2p.m2l_dual_flop_count(order)


def l2p_flops(order: int) -> int:
    sys.path.insert(0, os.path.join(ROOT, "paper_1407_2600_gb300", "csrc"))
    import gen_m2p
    return gen_m2p.l2p_flop_count(order)


def _sig(o, digits: int = 5):
    """The line's floats to `digits` significant digits (keeps the line short
    enough for log tails; the detail file keeps full precision)."""
    if isinstance(o, float):
        return o if o == 0.0 or not math.isfinite(o) else float("%.*g" % (digits, o))
    if isinstance(o, dict):
        return {k: _sig(v, digits) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_sig(v, digits) for v in o]
    return o


def _summary(rec, keys):
    """The keys of a side record that go into the printed line (None if the
    leg did not run; its error if it failed)."""
    if rec is None:
        return None
    if "error" in rec and len(rec) == 1:
        return rec
    return {k: rec.get(k) for k in keys}


def run_block_steps(dev, x, p, eps, args, eta: float = 1.0, rmax: int = 3):
    """Block steps (hierarchical KDK) on the benchmark workload: rungs from
    the accelerations at a = A_START (the smallest r <= rmax with
    4^r >= |g| dlna^2 / (eta^2 H0^2 eps)), then one global step of dlna =
    DLNA in 2^rmax ticks: every tick drifts all particles and rebuilds the
    tree, and the walk evaluates only the groups holding a particle whose
    step ends.  Timed against the 2^rmax global KDK steps that would give
    every particle the finest rung's step, from the same state.  Returns a
    dict, or {"error": ...} (this is a side measurement: it must not cost the
    benchmark line)."""
    try:
        import torch
        import paper_1407_2600_gb300.nbody as nb
        pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)
        mom = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float32, device=dev)
        prm = nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=args.n_direct, ewald_grid=args.ewald_grid,
                        flags=nb.NBODY_FLAG_ASYNC)
        tree = nb.Tree(prm, pos)
        acc = tree.forces()
        a0, a1 = A_START, A_START * math.exp(DLNA)
        rung = tree.assign_rungs(acc, eta, DLNA, rmax)
        counts = torch.bincount(rung.long(), minlength=rmax + 1).cpu().tolist()
        n = len(x)
        evals = sum(c << r for r, c in enumerate(counts))  # force evaluations per global step
        x0, p0, g0 = pos.clone(), mom.clone(), acc.clone()

        def restore():
            pos.copy_(x0)
            mom.copy_(p0)
            acc.copy_(g0)
            torch.cuda.synchronize()

        stream = torch.cuda.current_stream()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        tree.kdk_multistep(mom, acc, rung, a0, a1, rmax)  # warm-up
        torch.cuda.synchronize()
        tree.check()
        ms_block = []
        for _ in range(3):
            restore()
            e[0].record(stream)
            tree.kdk_multistep(mom, acc, rung, a0, a1, rmax)
            e[1].record(stream)
            torch.cuda.synchronize()
            tree.check()
            ms_block.append(e[0].elapsed_time(e[1]))
        restore()
        T = 1 << rmax
        a_list = [a0 * math.exp(DLNA * k / T) for k in range(T + 1)]
        e[2].record(stream)
        for k in range(T):
            tree.kdk_step(mom, acc, a_list[k], a_list[k + 1])
        e[3].record(stream)
        torch.cuda.synchronize()
        tree.check()
        ms_fine = e[2].elapsed_time(e[3])
        tree.close()
        ms = float(np.median(ms_block))
        return {"workload": "benchmark workload at a=%.2f, one global step dln a = %.2f in %d ticks" % (a0, DLNA, T),
                "eta": eta, "rmax": rmax, "rung_counts": counts,
                "force_evals_per_global_step": evals, "force_evals_all_finest": n * T,
                "ms_block_step": ms, "ms_all_finest_steps": ms_fine,
                "speedup_vs_all_finest": ms_fine / ms,
                "force_updates_per_s": evals / (ms * 1e-3),
                "note": "every tick rebuilds the whole tree; only groups with an ending step are walked"}
    except Exception as exc:  # a side measurement never costs the benchmark line
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def run_config3(dev, sms: int, ng: int = 512):
    """Throughput at scale: ng^3 (default 512^3 = 134,217,728) particles, a
    Zel'dovich box with P(k) ~ k^-1.5 (rms displacement 0.25 spacing at
    a = 0.02, generated on the device), theta 0.7 with the opening distance
    measured from the cell faces and the uniform-background terms,
    hexadecapole, eps = spacing/30; ten KDK steps from a = 0.02 to 0.05
    (dln a = ln 2.5 / 10).  Reports particle updates/s per step and the phase
    times.  On this near-uniform box at theta 0.7 the oracle gives a median
    force error against the direct Ewald sum of 4.7e-2 with the centre
    distance, 1.05e-3 with the face distance and 3.7e-4 with the face
    distance and the background terms (256 targets at 512^3)."""
    try:
        return _run_config3(dev, sms, ng)
    except Exception as exc:  # a side measurement: a failure is reported in the line, not raised
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def _run_config3(dev, sms: int, ng: int):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    from paper_1407_2600_gb300 import ics
    pos, mom = ics.zeldovich_device(ng, -1.5, 0.25, 3, 0.02, dev)
    n = pos.shape[1]
    torch.cuda.synchronize()
    prm = nb.params(eps=1.0 / (30.0 * ng), theta=0.7, order=4, n_direct=N_DIRECT, ewald_grid=EWALD_GRID,
                    flags=nb.NBODY_FLAG_ASYNC | nb.NBODY_FLAG_MAC_EDGE | nb.NBODY_FLAG_BACKGROUND)
    tree = nb.Tree(prm, pos)
    acc = tree.forces()
    dlna = math.log(2.5) / 10
    a = 0.02
    torch.cuda.synchronize()
    tree.timing(reset=True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        a1 = a * math.exp(dlna)
        tree.kdk_step(mom, acc, a, a1)
        a = a1
    e1.record(stream)
    torch.cuda.synchronize()
    rc = nb.nbody_check(tree.handle, nb._stream())
    if rc != nb.NBODY_OK:
        raise nb.NbodyError(rc, "config-3 steps")
    tm = tree.timing(reset=True)
    ms = e0.elapsed_time(e1) / 10
    ev = max(tm["evaluations"], 1)
    walk_ms = tm["ms_walk"] / ev
    flops = (tm["p2p"] * FP32_FLOPS_P2P + tm["m2p"] * (m2p_flops(4) + bg_flops(4))) / ev
    out = {"workload": "%d^3 Zel'dovich (P~k^-1.5, rms 0.25 spacing at a=0.02, device-generated), L=1 Gpc/h, "
                       "theta 0.7 (opening distance from the cell faces, uniform-background terms), p=4, "
                       "eps=spacing/30; 10 KDK steps "
                       "a=0.02->0.05" % ng,
           "n": int(n), "ms_per_kdk_step": ms, "updates_per_s": n / (ms * 1e-3), "a_end": a,
           "phases_ms": {k[3:]: round(tm[k] / max(tm["builds"] if k in ("ms_sort", "ms_build", "ms_upward")
                                                   else ev, 1), 3)
                         for k in ("ms_sort", "ms_build", "ms_upward", "ms_walk", "ms_periodic")},
           "interactions_per_particle": {"p2p": tm["p2p"] / ev / n, "m2p": tm["m2p"] / ev / n},
           "walk_frac": flops / (walk_ms * 1e-3) / 1e12 / fp32_peak_tflops(SM_MAX_MHZ, sms),
           "walk_tflops": flops / (walk_ms * 1e-3) / 1e12,
           "force_error_oracle": ERR_CONFIG3, "meets_accuracy_bar": meets_bar(ERR_CONFIG3),
           "device_mem_gb": torch.cuda.max_memory_allocated(dev) / 1e9}
    phases = {k: tm[k] / max(tm["builds"] if k in ("ms_sort", "ms_build", "ms_upward") else ev, 1)
              for k in ("ms_sort", "ms_build", "ms_upward", "ms_walk", "ms_periodic")}
    rf = phase_roofline(n, nb.nbody_tree_count(tree.handle, nb.EXPORT["cell_keys"]),
                        nb.nbody_tree_count(tree.handle, nb.EXPORT["groups"]), 4, phases, sms=sms)
    out["phase_roofline"] = dict({k: round(v["frac"], 4) for k, v in rf.items() if isinstance(v, dict)},
                                 upward_fp64=round(rf["upward"]["fp64_frac"], 4))
    tree.close()
    return out


# the batched boxes' setting that meets the accuracy bar at theta 0.5 and
# quadrupole order: face distance, uniform-background terms, accepted cells of
# <= 16 particles summed directly.  Oracle tree against the direct Ewald sum
# (256 targets per box, 13 boxes of the three sizes): medians 0.59-0.74e-3
# (48^3), 0.62-0.85e-3 (64^3), 0.83-0.92e-3 (80^3), 99th percentiles <= 6.0e-3.
BATCHED_N_DIRECT = 16
ERR_BATCHED = {"median": 0.92e-3, "p99": 6.0e-3}
# the autotuned setting without the background terms (direct-sum threshold
# 2): medians 1.10e-3 / 1.36e-3 / 2.55e-3 (one box of each size)
ERR_BATCHED_TUNED = {"median": 2.55e-3, "p99": 1.7e-2}


def run_batched(dev, steps: int):
    """Many independent small boxes in one tree build and one walk launch:
    32 boxes of 48^3, 32 of 64^3 and 32 of 80^3 particles (28,311,552), each
    its own periodic unit box with Zel'dovich initial conditions; theta 0.5,
    quadrupole, at the setting that meets the accuracy bar.  Times `steps`
    KDK steps (rebuild + forces + kicks + drift) of the whole batch and one
    force evaluation (rebuild + forces), both as calls made one by one (each
    build reads its counts back) and as CUDA graphs replayed on reserved
    capacities (no host round trip at all); then one force evaluation at the
    walk tiles the autotuner picks without the background terms (faster, but
    above the accuracy bar on these boxes)."""
    try:
        return _run_batched(dev, steps)
    except Exception as exc:  # a side measurement: a failure is reported in the line, not raised
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def _run_batched(dev, steps: int):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    from paper_1407_2600_gb300 import ics
    x, p, off, eps = ics.config_batched(1)
    n = len(x)
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)
    mom = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float32, device=dev)
    del x, p
    flags = nb.NBODY_FLAG_ASYNC | nb.NBODY_FLAG_MAC_EDGE
    prm = nb.params(eps=eps[0], theta=0.5, order=2, n_direct=BATCHED_N_DIRECT, n_group=32, ewald_grid=4,
                    flags=flags | nb.NBODY_FLAG_BACKGROUND)
    tree = nb.Tree(prm, pos, offsets=off.tolist(), eps=eps)
    acc = tree.forces()
    a = A_START
    for _ in range(2):
        a1 = a * math.exp(DLNA)
        tree.kdk_step(mom, acc, a, a1)
        a = a1
    torch.cuda.synchronize()
    tree.check()
    tree.timing(reset=True)
    # the timed steps start from this state, once called one by one and once replayed
    x0, p0, g0 = pos.clone(), mom.clone(), acc.clone()
    a_list = [a * math.exp(DLNA * k) for k in range(steps + 1)]

    def restore():
        pos.copy_(x0)
        mom.copy_(p0)
        acc.copy_(g0)
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    for k in range(steps):
        tree.kdk_step(mom, acc, a_list[k], a_list[k + 1])
    e[1].record(stream)
    torch.cuda.synchronize()
    tree.check()
    x_e, p_e, g_e = pos.clone(), mom.clone(), acc.clone()
    e[2].record(stream)
    tree.rebuild()
    tree.forces(acc)
    e[3].record(stream)
    torch.cuda.synchronize()
    tree.check()
    tm = tree.timing(reset=True)
    ms = e[0].elapsed_time(e[1]) / steps
    fms = e[2].elapsed_time(e[3])
    ev = max(tm["evaluations"], 1)
    # the same steps captured on capacities fixed at 1.1x the counts of the
    # starting state (an overflow would be reported by tree.check)
    restore()
    tree.rebuild()
    caps = tree.reserve(0.1)
    tree.forces(acc)
    g_steps, g_force = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_steps):
        for k in range(steps):
            tree.kdk_step(mom, acc, a_list[k], a_list[k + 1])
    with torch.cuda.graph(g_force):
        tree.rebuild()
        tree.forces(acc)
    restore()
    g_steps.replay()  # warm-up replay
    g_force.replay()
    torch.cuda.synchronize()
    tree.check()
    restore()
    e[0].record(stream)
    g_steps.replay()
    e[1].record(stream)
    torch.cuda.synchronize()
    tree.check()
    same = bool(torch.equal(pos, x_e) and torch.equal(mom, p_e) and torch.equal(acc, g_e))
    e[2].record(stream)
    g_force.replay()
    e[3].record(stream)
    torch.cuda.synchronize()
    tree.check()
    gms = e[0].elapsed_time(e[1]) / steps
    gfms = e[2].elapsed_time(e[3])
    del g_steps, g_force
    # the autotuned walk tiles without the background terms: context only
    tuned = None
    try:
        tree.reserve(-1)
        tree.params.flags = flags
        tree.params.n_direct = 2
        restore()
        tree.rebuild()
        tune = tree.autotune()
        tree.forces(acc)
        torch.cuda.synchronize()
        e[2].record(stream)
        tree.rebuild()
        tree.forces(acc)
        e[3].record(stream)
        torch.cuda.synchronize()
        tree.check()
        tms = e[2].elapsed_time(e[3])
        tuned = {"force_eval_ms": tms, "force_updates_per_s": n / (tms * 1e-3), "n_group": tune["n_group"],
                 "n_direct": tune["n_direct"], "candidates": tune["candidates"],
                 "force_error_oracle": ERR_BATCHED_TUNED, "meets_accuracy_bar": meets_bar(ERR_BATCHED_TUNED)}
    except Exception as exc:
        tuned = {"error": "%s: %s" % (type(exc).__name__, exc)}
    out = {"workload": "96 periodic boxes: 32 x 48^3 + 32 x 64^3 + 32 x 80^3 Zel'dovich (P~k^-2, rms 0.25 "
                       "spacing, a=0.02), eps = spacing/30 per box; theta 0.5 (opening distance from the cell faces), "
                       "quadrupole with the uniform-background terms, accepted cells of <= %d particles summed "
                       "directly, groups within level-3 cells (ewald_grid 4); one tree build and one walk launch "
                       "for all boxes" % BATCHED_N_DIRECT,
           "n": int(n), "nbox": 96, "steps": steps,
           "force_error_oracle": ERR_BATCHED, "meets_accuracy_bar": meets_bar(ERR_BATCHED),
           "graph_captured": True, "graph_state_equals_uncaptured": same,
           "ms_per_kdk_step": gms, "updates_per_s": n / (gms * 1e-3),
           "force_eval_ms": gfms, "force_updates_per_s": n / (gfms * 1e-3),
           "reserved_capacity": {"cells": caps[0], "groups": caps[1]},
           "uncaptured": {"ms_per_kdk_step": ms, "updates_per_s": n / (ms * 1e-3), "force_eval_ms": fms},
           "phases_ms": {k[3:]: round(tm[k] / max(tm["builds"] if k in ("ms_sort", "ms_build", "ms_upward")
                                                   else ev, 1), 3)
                         for k in ("ms_sort", "ms_build", "ms_upward", "ms_walk", "ms_periodic")},
           "interactions_per_particle": {"p2p": tm["p2p"] / ev / n, "m2p": tm["m2p"] / ev / n},
           "walk_variant": tm["walk_variant"],
           "tuned_setting": tuned,
           "tuned_force_updates_per_s": None if not tuned or "error" in tuned else tuned["force_updates_per_s"]}
    tree.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--fp64", action=argparse.BooleanOptionalAction, default=True,
                    help="also time one all-FP64 force evaluation of the same workload")
    ap.add_argument("--config3", action=argparse.BooleanOptionalAction, default=True,
                    help="also time ten KDK steps of the 512^3 scale workload (about half a minute)")
    ap.add_argument("--detail-file", default="bench_detail.json",
                    help="where the full per-leg records are written (JSON)")
    ap.add_argument("--form", default="dual", choices=sorted(FORMS),
                    help="walk form of the timed steps: m2p (every accepted cell expanded at every sink) or dual "
                         "(far cells through one local expansion per group)")
    ap.add_argument("--other-form", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the benchmark workload's force evaluation in the other walk form")
    ap.add_argument("--batched", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the 96-box batched workload")
    ap.add_argument("--block-steps", action=argparse.BooleanOptionalAction, default=True,
                    help="also time one global step of block (hierarchical) steps on the benchmark workload")
    ap.add_argument("--adjoint-steps", type=int, default=8, help="trajectory length of the reverse-mode timing")
    ap.add_argument("--ng", type=int, default=NG, help="particles per axis (128 = the benchmark workload)")
    ap.add_argument("--walk-variant", type=int, default=None, choices=[0, 1, 2, 3],
                    help="fixed walk launch variant for the timed steps (default: the autotuner's)")
    ap.add_argument("--n-direct", type=int, default=N_DIRECT,
                    help="accepted cells with at most this many particles are summed directly")
    ap.add_argument("--ewald-grid", type=int, default=EWALD_GRID,
                    help="groups never straddle a cell of level ewald_grid - 1")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
