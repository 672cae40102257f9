#!/usr/bin/env python3
"""Benchmark of the TTN sweep hot path on GB300.

Workload: compact lattice QED on a 4x4x4 open lattice (64 dressed sites),
t = m = 1, g^2 = 1 (ge2 = 1, plaquette cB = 1/2, penalty nu = 10), zero net
charge, U(1)-symmetric binary TTN with bond dimension 64, tensors from
SplitMix64 seed 1, Lanczos tolerance 1e-6 (relative residual), Krylov 64.
One step = one full sweep (63 node updates: centre moves with QR and
operator updates, Lanczos with H_eff products, tensor updates).

value = algorithmic H_eff x flops of every product in the timed sweeps /
timed wall time (TFLOP/s); the same sweeps' seconds are in ms_per_step.
Precision (default tf32x3): bottom-node products on tcgen05 with TF32
hi/lo operand splitting and FP32 accumulation, upper nodes in FP32; Lanczos
vectors, QR, operator updates and the final energy of each update in FP64.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (H_eff x at bottom node 0 with synthetic environment operators of
the right shapes) and reports it in the same unit.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "TTN sweep s & H_eff·ψ TFLOP/s, mixed vs FP64 at |ΔE|/|E|≤1e-6, 4³ χ=64"
L = (4, 4, 4)
CHI = 64
SEED = 1
G2 = 1.0
Q = 0
TOL = 1e-6
KRYLOV = 64


def workload_name(prec):
    return (f"4x4x4 open-boundary lattice QED (64 dressed sites, d=267), t=m=1, g2=1 (ge2=1, cB=0.5, nu=10), "
            f"Q=0, TTN chi=64 U(1) blocks, seed 1, Lanczos tol 1e-6, Krylov 64, precision {prec}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_from_profile(kernel_src):
    """DRAM bytes per launch of the tensor-core kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "tc_heff_4x4x4_chi64_traffic.txt")
    try:
        digest = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        vals = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != digest:
            return None
        return float(vals["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


# ---------------------------------------------------------------- oracle sample
def oracle_sample(n_matvecs=None, budget_s=20.0):
    """Time the FP64 oracle's H_eff x at bottom node 0 of the workload.
    Environment operators are random matrices of the right shapes (the
    oracle's cost depends on shapes only).  Returns (seconds per matvec,
    matvecs timed, cores)."""
    import numpy as np
    from oracle import model as omodel
    from oracle import ttn as ottn
    c = workloads.qed_couplings(G2)
    p = omodel.Params(*L, Q=Q, **c)
    ref = ottn.TTN(p, CHI, SEED, build_ops=False)
    node = 0
    rng = np.random.default_rng(0)
    dim = ref.T[node].shape[2]
    env = {}
    for k, tm in enumerate(ref.terms):
        if ref._crosses(tm, ref.region[node]):
            env[k] = rng.standard_normal((dim, dim))
    H = rng.standard_normal((dim, dim))
    env["H"] = H + H.T
    ref.down[node] = env
    terms = ref.heff_terms(node)
    X = ref.T[node]
    ref.heff_apply(node, X, terms)   # warm
    times = []
    t_start = time.time()
    while True:
        t0 = time.time()
        ref.heff_apply(node, X, terms)
        times.append(time.time() - t0)
        if n_matvecs is not None and len(times) >= n_matvecs:
            break
        if n_matvecs is None and time.time() - t_start > budget_s:
            break
    try:
        import numpy as _np
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    return float(sum(times) / len(times)), len(times), cores


def node0_flops():
    """Algorithmic flops of one H_eff x at bottom node 0 (the same count the
    native profiler reports), from a short native run."""
    import paper_2011_10658_gb300 as q
    c = workloads.qed_couplings(G2)
    s = q.TTN(q.Model(*L, Q=Q, **c), CHI, seed=SEED, precision="tf32x3")
    s.move_center(0)
    s.set_profiling(True)
    s.reset_timing()
    import numpy as np
    s.apply_heff(np.ones(s.node_size(0)))
    t = s.kernel_timing("tc_heff")
    s.close()
    return t["flops_alg"] / max(1, t["launches"])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    flops = None
    try:
        import torch
        if torch.cuda.is_available():
            flops = node0_flops()
    except Exception:
        flops = None
    for i in range(args.warmup + args.steps):
        t, n, cores = oracle_sample(n_matvecs=2)
        if i >= args.warmup:
            per_step.append(t * n)
    sec_per_mv = sum(per_step) / (2 * len(per_step))
    value = (flops / sec_per_mv / 1e12) if flops else None
    sample = (f"FP64 NumPy/SciPy oracle, H_eff x at bottom node 0 of the 4x4x4 chi=64 workload (environment "
              f"operators random, same shapes), 2 products per step, {sec_per_mv:.3f} s per product")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per_step) / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name("fp64 CPU oracle")},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- native arm
def replica_seed(rank):
    """Seed of the independent problem rank `rank` runs (replicas only)."""
    return SEED + rank


def reduce_over_ranks(elapsed_ms, flops, device):
    """Whole-job timing of independent replicas: the slowest rank's time and
    the flops of all ranks (one all-reduce each, no data-path collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms, flops], device=device, dtype=torch.float64)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item()


def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2011_10658_gb300 as q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    c = workloads.qed_couplings(G2)
    model = q.Model(*L, Q=Q, **c)
    # replicas only: rank r runs an independent problem from seed SEED + r
    s = q.TTN(model, CHI, seed=replica_seed(rank), precision=args.precision, stream=stream.cuda_stream)
    s.set_profiling(True)
    energies = []

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        st = s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
        energies.append(st["energy"])
    s.reset_timing()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = q.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        st = s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
        stats.append(st)
        energies.append(st["energy"])
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = q.launch_count() - launches0
    clocks = sampler.stop()
    kt = {k: s.kernel_timing(k) for k in ("tc_heff", "heff_simt_bottom", "heff_simt_upper", "move", "lanczos", "move_qr", "move_ops")}
    flops = sum(kt[k]["flops_alg"] for k in ("tc_heff", "heff_simt_bottom", "heff_simt_upper"))
    if world > 1:
        elapsed_ms, flops = reduce_over_ranks(elapsed_ms, flops, "cuda")
    value = flops / (elapsed_ms * 1e-3) / 1e12

    # dominant kernel roofline (kernel classes only, not whole phases)
    dom = max(("tc_heff", "heff_simt_bottom", "heff_simt_upper"), key=lambda k: kt[k]["ms"])
    d = kt[dom]
    pk, src = peaks()
    per_launch_ms = d["ms"] / max(1, d["launches"])
    achieved = d["flops_alg"] / max(1, d["launches"]) / (per_launch_ms * 1e-3) / 1e12
    if dom == "tc_heff":
        # TF32 tensor rate = BF16 rate x nominal ratio (1.1 / 2.25 PFLOP/s dense); kernel timed inside a long step
        peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25)
        bound, peak_note = "tensor", f"TF32 dense = {src} sustained BF16 {pk['bf16_tflops_sustained']} x 1.1/2.25"
        traffic = traffic_from_profile(os.path.join(ROOT, "paper_2011_10658_gb300", "csrc", "kernels_tc.cu"))
    elif dom == "heff_simt_bottom" or args.precision == "fp64":
        # FP64 products: GB300's FP64 rate (nominal 1.25 TFLOP/s)
        peak, bound, peak_note, traffic = 1.25, "alu", "FP64 SIMT, nominal 1.25 TFLOP/s", None
    else:
        # FP32 SIMT: 152 SMs x 128 lanes x 2 flops x max SM clock
        peak = 152 * 128 * 2 * (pk.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
        bound, peak_note, traffic = "alu", "FP32 SIMT 152 x 128 x 2 x 2070 MHz", None
    # every product class and the FP64 operator updates against their own peaks
    # (context for the dominant-class roofline above; FP64 SIMT peak from the
    # nominal 1.25 TFLOP/s of this part, FP32 SIMT 152 x 128 x 2 x max clock)
    fp64_peak = 1.25
    fp32_peak = 152 * 128 * 2 * (pk.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
    tf32_peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25)
    class_rates = {}
    for k, pkv, unit_note in (("tc_heff", tf32_peak, "TF32 tensor (measured BF16 sustained x 1.1/2.25)"),
                              ("heff_simt_bottom", fp64_peak, "FP64 SIMT (nominal)"),
                              ("heff_simt_upper", fp64_peak if args.precision == "fp64" else fp32_peak,
                               "FP64 SIMT (nominal)" if args.precision == "fp64" else "FP32 SIMT (mostly)"),
                              ("move_ops", fp64_peak, "FP64 SIMT (nominal)")):
        v = kt[k]
        if v["ms"] > 0 and v["flops_alg"] > 0:
            r = v["flops_alg"] / (v["ms"] * 1e-3) / 1e12
            class_rates[k] = {"tflops": r, "peak": pkv, "frac": r / pkv, "peak_source": unit_note,
                              "ms": v["ms"], "launches": v["launches"]}
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_note,
                "launches": d["launches"], "ms_per_launch": per_launch_ms,
                "algorithmic_flops_per_launch": d["flops_alg"] / max(1, d["launches"]),
                "executed_flops_per_launch": d["flops_exec"] / max(1, d["launches"]),
                "share_of_step": d["ms"] / elapsed_ms}

    # end to end through the public API with host buffers: tensors in from
    # pinned host memory, sweep, tensors and energy back to the host
    nn = s.info()["n_nodes"]
    host = [torch.empty(s.node_size(i), dtype=torch.float64, pin_memory=True) for i in range(nn)]
    for i in range(nn):
        host[i].numpy()[:] = s.node_export(i)
    h2d = sum(h.numel() * 8 for h in host)
    e2e_flops = 0.0
    s.reset_timing()
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(args.steps):
        s.load_tensors([(h.data_ptr(), h.numel()) for h in host])
        st = s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
        for i in range(nn):
            host[i].numpy()[:] = s.node_export(i)
        e_back = st["energy"]
    torch.cuda.synchronize()
    e2e_s = time.time() - t0
    kt2 = {k: s.kernel_timing(k) for k in ("tc_heff", "heff_simt_bottom", "heff_simt_upper")}
    e2e_flops = sum(v["flops_alg"] for v in kt2.values())
    e2e = {"value": e2e_flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d + 8, "seconds_per_step": e2e_s / args.steps}

    # per-update |dE|/|E| on identical H_eff: the same node update from the
    # same state, once with FP64 products and once in the state's precision
    per_update = None
    if args.precision != "fp64" and rank == 0:
        rows = []
        for node in (0, 1, 16, 31, 32, 48, 56, 62):
            s.move_center(node)
            t0 = s.node_export(node)
            s.set_precision("fp64")
            e64 = s.optimize_node(node, tol=TOL, max_krylov=KRYLOV)
            s.node_import(node, t0)
            s.set_precision(args.precision)
            em = s.optimize_node(node, tol=TOL, max_krylov=KRYLOV)
            rows.append({"node": node, "e_fp64": e64, "e_mixed": em, "rel_dE": abs(em - e64) / abs(e64)})
        per_update = {"nodes": rows, "max_rel_dE": max(r["rel_dE"] for r in rows)}

    # FP64 GPU path on the same workload and sweeps for |dE|/|E|
    compare = None
    if args.compare_fp64 and args.precision != "fp64" and rank == 0:
        r = q.TTN(model, CHI, seed=replica_seed(rank), precision="fp64", stream=stream.cuda_stream)
        e64, t64 = [], []
        for _ in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.time()
            e64.append(r.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)["energy"])
            torch.cuda.synchronize()
            t64.append(time.time() - t0)
        rel = [abs(a - b) / abs(b) for a, b in zip(energies, e64)]
        # the same sweeps as the timed mixed ones (after the warm-up sweeps)
        fp64_timed = sum(t64[args.warmup:]) / max(1, args.steps)
        compare = {"energies_mixed": energies, "energies_fp64": e64, "max_rel_dE": max(rel),
                   "fp64_seconds_per_sweep_each": t64, "fp64_seconds_per_timed_sweep": fp64_timed,
                   "speedup_same_sweeps": fp64_timed / (elapsed_ms / args.steps / 1e3)}
        r.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_mv, n_mv, cores = oracle_sample(budget_s=args.cpu_seconds)
        f0 = node0_flops()
        cpu = {"value": f0 / t_mv / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": (f"FP64 NumPy/SciPy oracle: {n_mv} H_eff x products at bottom node 0 of this workload "
                          f"(random environment operators of the same shapes), {t_mv:.3f} s each; "
                          f"{f0 / 1e9:.2f} GFLOP algorithmic per product")}

    if rank == 0:
        total_mv = sum(st["matvecs"] for st in stats)
        mixed_mv = sum(st["matvecs_mixed"] for st in stats)
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": workload_name(args.precision), "l2": "inputs larger than L2 (working set > 1 GB)",
                       "parallelism": f"replicas x{world} (independent seeds)"},
            "sweep_s": elapsed_ms / args.steps / 1e3,
            "energy": energies[-1],
            "matvecs_per_sweep": total_mv / args.steps, "mixed_matvecs_per_sweep": mixed_mv / args.steps,
            "roofline": roofline, "class_rates": class_rates, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "kernels": kt, "per_update_vs_fp64": per_update,
            "fp64_trajectory_comparison": compare,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_heff_only(args):
    """Profiling aid: the workload state with its centre at --node, --warmup
    untimed H_eff x products on device buffers (the tile-shape tuner settles),
    --steps products timed with CUDA events, then one product between
    cudaProfilerStart and cudaProfilerStop (for ncu --profile-from-start off)."""
    import torch
    import paper_2011_10658_gb300 as q
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    c = workloads.qed_couplings(G2)
    s = q.TTN(q.Model(*L, Q=Q, **c), CHI, seed=SEED, precision=args.precision, stream=stream.cuda_stream)
    s.move_center(args.node)
    n = s.node_size(args.node)
    x = torch.randn(n, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / max(1, args.steps)
    torch.cuda.profiler.start()
    s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"mode": "heff", "node": args.node, "size": n, "precision": args.precision,
                      "ms_per_product": ms, "products_timed": args.steps,
                      "norm": float(y.norm().item())}), flush=True)
    s.close()


def batch_problems(n):
    """Independent problems of the batching workload (4x4x4, chi = 48): problem
    i has charge q = 2 (i mod 9), g^2 = (0.5, 2)[(i // 9) mod 2], m = (0.5, 1)[(i // 18)
    mod 2], seed (2 << 32) + i."""
    out = []
    for i in range(n):
        g2 = (0.5, 2.0)[(i // 9) % 2]
        mass = (0.5, 1.0)[(i // 18) % 2]
        c = workloads.qed_couplings(g2, t=1.0, m=mass)
        out.append((dict(c, Q=2 * (i % 9)), (2 << 32) + i))
    return out


def run_batch(args):
    """Batched sweeps (one grouped product launch per lockstep Lanczos step,
    CUDA graphs) against the same problems swept one after another."""
    import torch
    import paper_2011_10658_gb300 as q
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    probs = batch_problems(args.problems)

    def make():
        return [q.TTN(q.Model(4, 4, 4, **kw), 48, seed=seed, precision=args.precision, stream=stream.cuda_stream)
                for kw, seed in probs]

    seq, bat = make(), make()
    for s in seq:
        s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
    q.batch_sweep(bat, 1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
    torch.cuda.synchronize()
    t0 = time.time()
    e_seq = [s.sweep(args.steps, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)["energy"] for s in seq]
    torch.cuda.synchronize()
    t_seq = time.time() - t0
    l0 = q.launch_count()
    t0 = time.time()
    st = q.batch_sweep(bat, args.steps, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
    torch.cuda.synchronize()
    t_bat = time.time() - t0
    launches = q.launch_count() - l0
    e_bat = [x["energy"] for x in st]
    rel = max(abs(a - b) / abs(b) for a, b in zip(e_bat, e_seq))
    units = args.problems * args.steps
    print(json.dumps({
        "metric": "batched TTN sweeps (problem-sweeps/s)", "value": units / t_bat, "unit": "problem-sweeps/s",
        "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True, "dtype": args.precision,
        "data": "synthetic", "config": {"workload": f"{args.problems} independent 4x4x4 chi=48 problems "
                                                    "(q = 0..16, g^2 in {0.5, 2}, m in {0.5, 1})"},
        "sequential_value": units / t_seq, "speedup_vs_sequential": t_seq / t_bat,
        "max_rel_dE_batch_vs_sequential": rel, "gpu_launches": launches}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--compare-fp64", dest="compare_fp64", action="store_true", default=True)
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="sweep", choices=["sweep", "heff", "batch"],
                    help="heff: only H_eff x products at --node (profiling aid); batch: batched "
                         "independent problems against sequential sweeps")
    ap.add_argument("--problems", type=int, default=8, help="batch mode: number of problems")
    ap.add_argument("--node", type=int, default=0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "heff":
        run_heff_only(args)
    elif args.mode == "batch":
        run_batch(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
