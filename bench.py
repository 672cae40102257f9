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
Precision (default tf32x3): H_eff x products on tcgen05 with split-TF32
operands and FP32 accumulation, then the FP64 residual correction; Lanczos
vectors, QR and the final energy of each update in FP64.

Extra keys (rank 0, one GPU): per-class kernel times with each class's rate
against its own measured peak; the dominant class's roofline; in-run peak
probes (cuBLAS FP64 / FP32 / TF32 / BF16 GEMMs); node updates repeated from
identical states in FP64 and in the mixed precision (energy difference and
speed-up at matched accuracy); the TF32 and BF16 arms and the g^2 scan
{0.5, 2, 4} of the precision configuration; the FP64 path's sweeps and the
time each path needs to reach a common energy.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (H_eff x at bottom node 0 with synthetic environment operators of
the right shapes; algorithmic flops counted by the oracle itself).

Other configurations (--mode): batch (independent 4x4x4 chi=48 problems
swept together against one after another), scale (8x8x8 chi=128 Q=32, two
sweeps per g^2), physics (finite-density, periodic zero-charge and
capacitor workloads with the driven penalty), heff and profile (profiling
aids: products at one node, or one product / move / product inside a
profiler window).
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
PRODUCT_CLASSES = ("tc_heff", "heff_simt_bottom", "heff_simt_upper")
ALL_CLASSES = ("tc_heff", "heff_simt_bottom", "heff_simt_upper", "move", "lanczos", "move_qr", "move_ops",
               "move_ops_bottom")


def workload_name(prec, g2=G2):
    c = workloads.qed_couplings(g2)
    return (f"4x4x4 open-boundary lattice QED (64 dressed sites, d=267), t=m=1, g2={g2:g} (ge2={c['ge2']:g}, "
            f"cB={c['cB']:g}, nu={c['nu']:g}), Q=0, TTN chi=64 U(1) blocks, seed 1, Lanczos tol 1e-6, Krylov 64, "
            f"precision {prec}")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


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


# ---------------------------------------------------------------- peaks
def probe_peaks(device):
    """Dense GEMM rates of this GPU measured now (cuBLAS through torch):
    FP64, FP32 with TF32 off (SIMT), TF32 and BF16, best of 3 after a
    warm-up, CUDA events; the denominators of the per-class fractions."""
    import torch
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dtype, n, tf32 in (("fp64", torch.float64, 4096, False), ("fp32_simt", torch.float32, 8192, False),
                                     ("tf32", torch.float32, 8192, True), ("bf16", torch.bfloat16, 8192, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device=device, dtype=dtype)
            b = torch.randn(n, n, device=device, dtype=dtype)
            c = a @ b
            best = 1e30
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                c = a @ b
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- oracle sample
def _oracle_tree():
    from oracle import model as omodel
    from oracle import ttn as ottn
    c = workloads.qed_couplings(G2)
    return ottn.TTN(omodel.Params(*L, Q=Q, **c), CHI, SEED, build_ops=False)


def _oracle_with_random_env(node):
    """Oracle TTN of the workload with synthetic environment operators of
    the right shapes at `node` (the oracle's cost depends on shapes only)."""
    import numpy as np
    ref = _oracle_tree()
    _set_random_env(ref, node, np.random.default_rng(0))
    return ref


def _set_random_env(ref, node, rng):
    """Random environment and child operators of the right shapes at node."""
    dim = ref.T[node].shape[2]
    env = {}
    for k, tm in enumerate(ref.terms):
        if ref._crosses(tm, ref.region[node]):
            env[k] = rng.standard_normal((dim, dim))
    H = rng.standard_normal((dim, dim))
    env["H"] = H + H.T
    ref.down[node] = env
    if ref.nodes[node].children[0][0] == "node":
        for kind, cid in ref.nodes[node].children:
            d = ref.T[cid].shape[2]
            ops = {k: rng.standard_normal((d, d)) for k, tm in enumerate(ref.terms)
                   if ref._crosses(tm, ref.region[cid])}
            Hc = rng.standard_normal((d, d))
            ops["H"] = Hc + Hc.T
            ref.up[cid] = ops


def oracle_upper_sample():
    """Seconds of one FP64 oracle H_eff x at the first node of every upper
    layer of the workload's tree (random environments of the right shapes,
    one oracle tree for all), with the number of nodes in each layer."""
    import numpy as np
    ref = _oracle_tree()
    rng = np.random.default_rng(1)
    out = []
    for layer in sorted({nd.layer for nd in ref.nodes if nd.layer > 0}):
        ids = [nd.index for nd in ref.nodes if nd.layer == layer]
        node = ids[0]
        _set_random_env(ref, node, rng)
        terms = ref.heff_terms(node)
        X = ref.T[node]
        ref.heff_apply(node, X, terms)
        t0 = time.time()
        ref.heff_apply(node, X, terms)
        out.append((node, len(ids), time.time() - t0))
    return out


def extrapolated_oracle_sweep(kt, steps, t_bottom, upper):
    """Oracle seconds for the products of one sweep: the sweep's bottom-node
    products (tensor-core and residual-correction) at the timed bottom-node
    rate, its upper-node products at the node-weighted mean of the timed
    upper layers.  Operator updates and the eigensolver's own work are not
    included."""
    n_bottom = (kt["tc_heff"]["launches"] + kt["heff_simt_bottom"]["launches"]) / steps
    n_upper = kt["heff_simt_upper"]["launches"] / steps
    t_upper = sum(n * t for (_, n, t) in upper) / max(1, sum(n for (_, n, _) in upper))
    return n_bottom * t_bottom + n_upper * t_upper, n_bottom, n_upper, t_upper


def oracle_sample(n_matvecs=None, budget_s=20.0, node=0):
    """Time the FP64 oracle's H_eff x at `node` of the workload.  Returns
    (seconds per product, products timed, threads, flops per product); the
    flops are the oracle's own count (bottom nodes only, else None)."""
    from oracle import ttn as ottn
    ref = _oracle_with_random_env(node)
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
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    flops = ottn.bottom_heff_flops(ref, node) if ref.nodes[node].children[0][0] == "site" else None
    return float(sum(times) / len(times)), len(times), threads, flops


def oracle_single_thread(n_matvecs=2):
    """The same sample with one BLAS thread, in a child process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; t, n, th, f = bench.oracle_sample(n_matvecs=%d); "
            "print(json.dumps({'t': t, 'n': n, 'flops': f}))" % n_matvecs)
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=900)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as exc:
        return {"error": str(exc)[:200]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    flops = None
    threads = None
    for i in range(args.warmup + args.steps):
        t, n, threads, flops = oracle_sample(n_matvecs=2)
        if i >= args.warmup:
            per_step.append(t * n)
    sec_per_mv = sum(per_step) / (2 * len(per_step))
    value = flops / sec_per_mv / 1e12
    sample = (f"FP64 NumPy/SciPy oracle, H_eff x at bottom node 0 of the 4x4x4 chi=64 workload (environment "
              f"operators random, same shapes), 2 products per step, {sec_per_mv:.3f} s per product, "
              f"{flops / 1e9:.3f} GFLOP algorithmic per product (oracle's own count); CPU {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(per_step) / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name("fp64 CPU oracle")},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
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


def class_table(kt, elapsed_ms, peaks, precision):
    """Disjoint kernel classes of the timed sweeps with their share of the
    step and their rate against their own peak and the peak the hot-path
    table assigns (tensor cores for every contraction)."""
    lanczos_vec = kt["lanczos"]["ms"] - sum(kt[k]["ms"] for k in PRODUCT_CLASSES)
    rows = {}
    own = {"tc_heff": ("bf16" if precision == "bf16" else "tf32"),
           "heff_simt_bottom": "fp64",
           "heff_simt_upper": ("fp64" if precision == "fp64" else "fp32_simt"),
           "move_ops": "fp64",
           "move_ops_bottom": ("fp64" if precision == "fp64" else "bf16")}
    for k in ("tc_heff", "heff_simt_bottom", "heff_simt_upper", "move_ops", "move_ops_bottom", "move_qr"):
        v = kt[k]
        r = {"ms": v["ms"], "launches": v["launches"], "share_of_step": v["ms"] / elapsed_ms}
        if v["flops_alg"] > 0 and v["ms"] > 0:
            rate = v["flops_alg"] / (v["ms"] * 1e-3) / 1e12
            r["tflops_alg"] = rate
            if k in own:
                r["own_peak"] = {"dtype": own[k], "tflops": peaks[own[k]], "frac": rate / peaks[own[k]]}
                tp = "bf16" if precision == "bf16" else "tf32"
                r["tensor_peak"] = {"dtype": tp, "tflops": peaks[tp], "frac": rate / peaks[tp]}
        rows[k] = r
    rows["lanczos_vectors"] = {"ms": lanczos_vec, "share_of_step": lanczos_vec / elapsed_ms,
                               "note": "Lanczos time minus its products: FP64 dots, reorthogonalisation, "
                                       "tridiagonal solve, host checks"}
    return rows


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
    props = torch.cuda.get_device_properties(local)
    c = workloads.qed_couplings(G2)
    model = q.Model(*L, Q=Q, **c)
    # replicas only: rank r runs an independent problem from seed SEED + r
    s = q.TTN(model, CHI, seed=replica_seed(rank), precision=args.precision, stream=stream.cuda_stream)
    s.set_profiling(True)
    energies, warm_s = [], []

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        torch.cuda.synchronize()
        t0 = time.time()
        st = s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
        torch.cuda.synchronize()
        warm_s.append(time.time() - t0)
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
    kt = {k: s.kernel_timing(k) for k in ALL_CLASSES}
    flops = sum(kt[k]["flops_alg"] for k in PRODUCT_CLASSES)
    if world > 1:
        elapsed_ms, flops = reduce_over_ranks(elapsed_ms, flops, "cuda")
    value = flops / (elapsed_ms * 1e-3) / 1e12

    pk, src = measured_peaks()
    peaks = {"bf16": pk["bf16_tflops_sustained"]}
    probed = None
    if rank == 0 and not args.no_probe:
        probed = probe_peaks("cuda")
        peaks.update({k: v for k, v in probed.items() if k != "bf16"})
    else:
        # nominal ratios to the measured BF16 rate when the probes are skipped
        peaks.update({"tf32": peaks["bf16"] * 1.1 / 2.25, "fp64": 1.25,
                      "fp32_simt": props.multi_processor_count * 128 * 2 * pk.get("sm_max_mhz", 2070.0) / 1e6})
    classes = class_table(kt, elapsed_ms, peaks, args.precision)

    # roofline of the class with the most kernel time among the flop-counted
    # contraction classes (products and operator updates)
    dom = max(("tc_heff", "heff_simt_bottom", "heff_simt_upper", "move_ops", "move_ops_bottom"),
              key=lambda k: kt[k]["ms"])
    d = kt[dom]
    per_launch_ms = d["ms"] / max(1, d["launches"])
    achieved = d["flops_alg"] / max(1, d["launches"]) / (per_launch_ms * 1e-3) / 1e12
    tensor_dtype = "bf16" if args.precision == "bf16" else "tf32"
    peak = peaks[tensor_dtype]
    traffic = None
    if dom == "tc_heff":
        traffic = traffic_from_profile(os.path.join(ROOT, "paper_2011_10658_gb300", "csrc", "kernels_tc.cu"))
    roofline = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": (f"{tensor_dtype} dense GEMM measured in this run (cuBLAS)" if probed else
                                f"{src} BF16 sustained x nominal ratio"),
                "own_dtype_frac": classes.get(dom, {}).get("own_peak"),
                "launches": d["launches"], "ms_per_launch": per_launch_ms,
                "algorithmic_flops_per_launch": d["flops_alg"] / max(1, d["launches"]),
                "executed_flops_per_launch": d["flops_exec"] / max(1, d["launches"]),
                "share_of_step": d["ms"] / elapsed_ms}
    # the same fraction against the measured BF16 peak of the pool times the
    # nominal dense ratio of this dtype (1.1/2.25 for TF32)
    nominal = pk["bf16_tflops_sustained"] * (1.0 if tensor_dtype == "bf16" else 1.1 / 2.25)
    roofline["peak_from_measured_bf16"] = {"tflops": nominal, "frac": achieved / nominal, "source": src}
    largest = max(classes, key=lambda k: classes[k]["ms"])

    # end to end through the public API with host buffers: tensors in from
    # pinned host memory, sweep, tensors and energy back to the host
    nn = s.info()["n_nodes"]
    host = [torch.empty(s.node_size(i), dtype=torch.float64, pin_memory=True) for i in range(nn)]
    for i in range(nn):
        host[i].numpy()[:] = s.node_export(i)
    h2d = sum(h.numel() * 8 for h in host)
    s.reset_timing()
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(args.steps):
        s.load_tensors([(h.data_ptr(), h.numel()) for h in host])
        st = s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
        for i in range(nn):
            host[i].numpy()[:] = s.node_export(i)
    torch.cuda.synchronize()
    e2e_s = time.time() - t0
    kt2 = {k: s.kernel_timing(k) for k in PRODUCT_CLASSES}
    e2e_flops = sum(v["flops_alg"] for v in kt2.values())
    e2e = {"value": e2e_flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d + 8, "seconds_per_step": e2e_s / args.steps}

    extra = {}
    if rank == 0 and world == 1:
        extra = run_extras(args, q, model, s, stream, energies, warm_s, elapsed_ms / args.steps / 1e3)
    s.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_mv, n_mv, threads, f0 = oracle_sample(budget_s=args.cpu_seconds)
        one = oracle_single_thread()
        sample = (f"FP64 NumPy/SciPy oracle: {n_mv} H_eff x products at bottom node 0 of this workload "
                  f"(random environment operators of the same shapes), {t_mv:.3f} s each with {threads} threads; "
                  f"{f0 / 1e9:.3f} GFLOP algorithmic per product (oracle's own count); CPU {cpu_model()}")
        cpu = {"value": f0 / t_mv / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle", "sample": sample,
               "single_thread": ({"seconds_per_product": one["t"], "tflops": f0 / one["t"] / 1e12}
                                 if "t" in one else one)}
        # products of one sweep at the oracle's speed (a lower bound of an
        # oracle sweep: operator updates and the eigensolver's own work not
        # included), extrapolated from timed bottom- and upper-node products
        upper = oracle_upper_sample()
        sweep_s, n_b, n_u, t_u = extrapolated_oracle_sweep(kt, args.steps, t_mv, upper)
        cpu["sweep_seconds_extrapolated"] = sweep_s
        cpu["extrapolation"] = (f"{n_b:.0f} bottom-node products per sweep x {t_mv:.3f} s + {n_u:.0f} upper-node "
                                f"products x {t_u:.4f} s (one node per upper layer timed, weighted by the layer's "
                                f"node count: " + ", ".join(f"node {nd} {t:.4f} s" for (nd, _, t) in upper) + ")")

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
            "not_converged": sum(st["not_converged"] for st in stats),
            "node_updates": sum(st["node_updates"] for st in stats),
            "max_rel_residual": max(st["max_rel_residual"] for st in stats),
            "roofline": roofline, "largest_class": largest, "classes": classes, "peaks_tflops": peaks,
            "sm_count": props.multi_processor_count,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "launches_per_sweep": launches / args.steps, "kernels": kt,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed_update(q, s, node, precision, t0, stream):
    """One node update from tensor t0 in `precision`, CUDA-event timed."""
    import torch
    s.set_precision(precision)
    s.node_import(node, t0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e = s.optimize_node(node, tol=TOL, max_krylov=KRYLOV)
    e1.record(stream)
    torch.cuda.synchronize()
    return e, e0.elapsed_time(e1), s.last_update()


def run_extras(args, q, model, s, stream, energies, warm_s, sweep_s):
    """Matched-accuracy comparison with the FP64 path and the precision
    arms of the precision configuration (rank 0, one GPU)."""
    import torch
    out = {}
    # per-update: identical state and H_eff, FP64 vs mixed, both to TOL
    rows = []
    if args.precision != "fp64":
        for node in (0, 1, 16, 31, 32, 48, 56, 62):
            s.move_center(node)
            t0 = s.node_export(node)
            e64, ms64, lu64 = _timed_update(q, s, node, "fp64", t0, stream)
            em, msm, lum = _timed_update(q, s, node, args.precision, t0, stream)
            rows.append({"node": node, "e_fp64": e64, "e_mixed": em, "rel_dE": abs(em - e64) / abs(e64),
                         "ritz_low_precision": lum["ritz_mixed"],
                         "rel_dE_low_precision": abs(lum["ritz_mixed"] - e64) / abs(e64),
                         "ms_fp64": ms64, "ms_mixed": msm, "iters_fp64": lu64["iters_fp64"],
                         "iters_mixed": lum["iters_mixed"], "iters_correction": lum["iters_fp64"]})
        s.set_precision(args.precision)
        out["per_update_vs_fp64"] = {
            "nodes": rows, "max_rel_dE": max(r["rel_dE"] for r in rows),
            "speedup_matched_accuracy": sum(r["ms_fp64"] for r in rows) / sum(r["ms_mixed"] for r in rows),
            "note": "the same node updates from identical states, both to relative residual 1e-6"}
    if args.arms:
        arms = {}
        for prec, g2 in (("tf32", 1.0), ("bf16", 1.0), ("tf32x3", 0.5), ("tf32x3", 2.0), ("tf32x3", 4.0)):
            r = q.TTN(q.Model(*L, Q=Q, **workloads.qed_couplings(g2)), CHI, seed=SEED, precision=prec,
                      stream=stream.cuda_stream)
            r.set_profiling(True)
            for _ in range(3):
                r.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
            r.reset_timing()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = r.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            f = sum(r.kernel_timing(k)["flops_alg"] for k in PRODUCT_CLASSES)
            arms[f"{prec}_g2={g2:g}"] = {"sweep_s": ms / 1e3, "tflops": f / (ms * 1e-3) / 1e12,
                                         "energy_after_4_sweeps": st["energy"], "not_converged": st["not_converged"],
                                         "max_rel_residual": st["max_rel_residual"]}
            r.close()
        out["precision_arms"] = arms
    if args.compare_fp64 and args.precision != "fp64":
        # the FP64 path from the same seed: energies after every sweep and the
        # time each path needs to reach a common energy (the higher of the two
        # final energies)
        r = q.TTN(model, CHI, seed=SEED, precision="fp64", stream=stream.cuda_stream)
        e64, t64 = [], []
        for _ in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.time()
            e64.append(r.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)["energy"])
            torch.cuda.synchronize()
            t64.append(time.time() - t0)
        r.close()
        tm = list(warm_s) + [sweep_s] * (len(energies) - len(warm_s))
        target = max(e64[-1], energies[-1])

        def time_to(es, ts):
            acc = 0.0
            for e, t in zip(es, ts):
                acc += t
                if e <= target + 1e-12 * abs(target):
                    return acc
            return None

        t_m, t_f = time_to(energies, tm), time_to(e64, t64)
        out["fp64_trajectory_comparison"] = {
            "energies_mixed": energies, "energies_fp64": e64, "seconds_mixed_each": tm, "seconds_fp64_each": t64,
            "end_rel_dE": abs(energies[-1] - e64[-1]) / abs(e64[-1]), "common_target_energy": target,
            "seconds_to_target_mixed": t_m, "seconds_to_target_fp64": t_f,
            "speedup_to_common_energy": (t_f / t_m) if (t_m and t_f) else None}
    return out


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
    s.set_profiling(True)
    s.reset_timing()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / max(1, args.steps)
    kt = {k: s.kernel_timing(k) for k in PRODUCT_CLASSES}
    s.set_profiling(False)
    torch.cuda.profiler.start()
    s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    flops = sum(v["flops_alg"] for v in kt.values()) / max(1, args.steps)
    print(json.dumps({"mode": "heff", "node": args.node, "size": n, "precision": args.precision,
                      "ms_per_product": ms, "products_timed": args.steps, "flops_alg_per_product": flops,
                      "tflops": flops / (ms * 1e-3) / 1e12, "kernels": kt,
                      "norm": float(y.norm().item())}), flush=True)
    s.close()


def run_profile_window(args):
    """Profiling aid: the workload state; --warmup rounds of (centre to
    bottom node 0, H_eff x at node 0, centre to its parent 32, H_eff x at
    node 32), then one such round between cudaProfilerStart and
    cudaProfilerStop (for ncu --profile-from-start off) after the centre is
    back at node 0: the tensor-core bottom-node product, the QR and
    digit-plane operator update of the bond above node 0, and the
    tensor-core leg contractions of the upper-node product."""
    import torch
    import paper_2011_10658_gb300 as q
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    c = workloads.qed_couplings(G2)
    s = q.TTN(q.Model(*L, Q=Q, **c), CHI, seed=SEED, precision=args.precision, stream=stream.cuda_stream)
    gen = torch.Generator("cuda").manual_seed(0)
    bufs = {}
    for node in (0, 32):
        n = s.node_size(node)
        bufs[node] = (torch.randn(n, dtype=torch.float64, device="cuda", generator=gen),
                      torch.empty(n, dtype=torch.float64, device="cuda"), n)

    def one_round():
        s.move_center(0)
        x, y, n = bufs[0]
        s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
        s.move_center(32)
        x, y, n = bufs[32]
        s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)

    for _ in range(args.warmup):
        one_round()
    s.move_center(0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    ev0.record(stream)
    x, y, n = bufs[0]
    s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    s.move_center(32)
    x, y, n = bufs[32]
    s.apply_heff_device(x.data_ptr(), y.data_ptr(), n)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"mode": "profile", "ms_window": ev0.elapsed_time(ev1), "precision": args.precision,
                      "sizes": {k: v[2] for k, v in bufs.items()}}), flush=True)
    s.close()


def _links(L, periodic):
    """(x, mu) of every link in the library's order (sites, then mu)."""
    Lx, Ly, Lz = L
    dims = (Lx, Ly, Lz)
    out = []
    for s in range(Lx * Ly * Lz):
        c = [s % Lx, (s // Lx) % Ly, s // (Lx * Ly)]
        for mu in range(3):
            d = list(c)
            d[mu] += 1
            if periodic and dims[mu] > 1:
                d[mu] %= dims[mu]
            if d[mu] < dims[mu]:
                out.append((s, mu))
    return out


def run_physics(args):
    """The paper's physics workloads on the same engine (driven penalty,
    then the observables), one JSON line each:
      finite density: 4x4x4 open, Q = 16, g2 = 1: sigma(l) by surface layer
        (Results, "Finite density");
      zero charge, periodic: 4x4x4, Q = 0, g2 = 2 (ge2/2 = t = 1), cB = 0
        and cB = 1/(2 g2), m in {-1, 0.5, 2}: rho (Results, "Transition at
        zero charge");
      quantum capacitor: 4x4x4 open, Q = 0, chemical potentials -/+ mu0 on
        the faces x = 0 and x = 3, m in {-1, 1}: q_c(d) and E_c(d) along x
        (Results, "Quantum capacitor").
    Bond dimension --physics-chi (default 32), seed 7; the driven schedule
    of the library with nu_max = 10 max(|t|, |m|, ge2/2, cB)."""
    import numpy as np
    import torch
    import paper_2011_10658_gb300 as q
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    chi = args.physics_chi
    L4 = (4, 4, 4)
    N = 64

    def drive(model, nu_max):
        s = q.TTN(model, chi, seed=7, precision=args.precision, stream=stream.cuda_stream)
        t0 = time.time()
        recs, conv = s.drive(allow_noconv=True, nu_start=0.5, nu_step=2.0, quad_coef=0.25, nu_max=nu_max,
                             tol_start=1e-4, tol_factor=0.3, tol_final=1e-8, conv_rel=1e-7, rise_rel=1e-9,
                             min_final_sweeps=2, max_sweeps=args.physics_sweeps, max_krylov=KRYLOV)
        torch.cuda.synchronize()
        return s, recs, conv, time.time() - t0

    def base_line(name, recs, conv, secs, extra):
        last = recs[-1]
        line = {"mode": "physics", "workload": name, "chi": chi, "precision": args.precision, "seed": 7,
                "sweeps": len(recs), "converged": conv, "seconds": secs, "energy": last["energy"],
                "energy_without_penalty": last["energy_without_penalty"], "delta_L": last["delta_L"],
                "nu_schedule": [r["nu"] for r in recs], "stages": [r["stage"] for r in recs],
                "delta_L_per_sweep": [r["delta_L"] for r in recs],
                "energy_per_sweep": [r["energy"] for r in recs]}
        line.update(extra)
        print(json.dumps(line), flush=True)

    # finite density
    c = workloads.qed_couplings(1.0)
    nu_max = c["nu"]
    s, recs, conv, secs = drive(q.Model(*L4, Q=16, **dict(c, nu=0.5)), nu_max)
    sc = s.measure("scalars")
    base_line("finite density 4x4x4 open Q=16 g2=1", recs, conv, secs,
              {"sigma_l": [float(v) for v in s.measure("sigma")], "rho": float(sc[0]), "total_charge": float(sc[2])})
    s.close()

    # zero charge, periodic
    for cb_on in (False, True):
        for mass in (-1.0, 0.5, 2.0):
            c = dict(t=1.0, m=mass, ge2=2.0, cB=(0.25 if cb_on else 0.0), nu=0.5)
            nu_max = 10.0 * max(1.0, abs(mass), 1.0, c["cB"])
            s, recs, conv, secs = drive(q.Model(*L4, Q=0, boundary=1, **c), nu_max)
            sc = s.measure("scalars")
            base_line(f"zero charge 4x4x4 periodic g2=2 cB={c['cB']:g} m={mass:g}", recs, conv, secs,
                      {"rho": float(sc[0]), "total_charge": float(sc[2])})
            s.close()

    # quantum capacitor
    mu0 = args.capacitor_mu
    mu = [(-mu0 if s_ % 4 == 0 else (mu0 if s_ % 4 == 3 else 0.0)) for s_ in range(N)]
    parity = np.array([1 if (s_ % 4 + (s_ // 4) % 4 + s_ // 16) % 2 == 0 else -1 for s_ in range(N)])
    links = _links(L4, False)
    for mass in (-1.0, 1.0):
        c = dict(t=1.0, m=mass, ge2=2.0, cB=0.25, nu=0.5)
        nu_max = 10.0 * max(1.0, abs(mass), 1.0)
        s, recs, conv, secs = drive(q.Model(*L4, Q=0, mu=mu, **c), nu_max)
        phi = np.array(s.measure("phi"))
        el = np.array(s.measure("elink"))
        qc = [float(2.0 / 16 * sum(parity[x] * phi[x] for x in range(N) if x % 4 == d)) for d in range(4)]
        ec = [float(2.0 / 16 * sum(el[i] for i, (x, mu_) in enumerate(links) if mu_ == 0 and x % 4 == d))
              for d in range(3)]
        base_line(f"capacitor 4x4x4 open plates mu=-/+{mu0:g} on x=0/3, g2=2 cB=0.25 m={mass:g}", recs, conv,
                  secs, {"q_c": qc, "E_c": ec, "rho": float(s.measure("scalars")[0])})
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


def run_scale(args):
    """The scale configuration: 8x8x8 open lattice (512 dressed sites), t =
    m = 1, g^2 in {0.5, 3}, charge excess Q = 32, chi = 128, seed 4, two
    full sweeps from the seeded isometric start in the mixed precision.
    One JSON line per g^2 with the sweep times, the H_eff x throughput and
    the dominant class's roofline fraction, and the device memory the state
    holds."""
    import torch
    import paper_2011_10658_gb300 as q
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    pk, src = measured_peaks()
    peaks = {"bf16": pk["bf16_tflops_sustained"]}
    if not args.no_probe:
        peaks.update({k: v for k, v in probe_peaks("cuda").items() if k != "bf16"})
    else:
        peaks.update({"tf32": peaks["bf16"] * 1.1 / 2.25, "fp64": 1.25, "fp32_simt": 64.0})
    for g2 in args.scale_g2:
        torch.cuda.synchronize()
        free0, total = torch.cuda.mem_get_info()
        c = workloads.qed_couplings(g2)
        model = q.Model(8, 8, 8, Q=32, **c)
        t0 = time.time()
        s = q.TTN(model, 128, seed=4, precision=args.precision, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        create_s = time.time() - t0
        free1, _ = torch.cuda.mem_get_info()
        s.set_profiling(True)
        sampler = ClockSampler(0)
        sampler.start()
        l0 = q.launch_count()
        sweeps = []
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = s.sweep(1, tol=TOL, max_krylov=KRYLOV, allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            st["ms"] = e0.elapsed_time(e1)
            sweeps.append(st)
        ev1.record(stream)
        torch.cuda.synchronize()
        elapsed_ms = ev0.elapsed_time(ev1)
        launches = q.launch_count() - l0
        clocks = sampler.stop()
        free2, _ = torch.cuda.mem_get_info()
        kt = {k: s.kernel_timing(k) for k in ALL_CLASSES}
        flops = sum(kt[k]["flops_alg"] for k in PRODUCT_CLASSES)
        classes = class_table(kt, elapsed_ms, peaks, args.precision)
        dom = max(("tc_heff", "heff_simt_bottom", "heff_simt_upper", "move_ops", "move_ops_bottom"),
                  key=lambda k: kt[k]["ms"])
        d = kt[dom]
        achieved = d["flops_alg"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
        tp = "bf16" if args.precision == "bf16" else "tf32"
        info = s.info()
        e_tot, e_nopen, e_cls = s.energy()
        line = {
            "metric": "scale: TTN sweeps of the 8x8x8 chi=128 lattice (H_eff x TFLOP/s)",
            "value": flops / (elapsed_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 0, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": (f"8x8x8 open-boundary lattice QED (512 dressed sites), t=m=1, g2={g2:g}, Q=32, "
                                    f"TTN chi=128 U(1) blocks, seed 4, {args.steps} sweeps from the seeded start, "
                                    f"Lanczos tol {TOL:g}, Krylov {KRYLOV}, precision {args.precision}")},
            "create_s": create_s,
            "sweeps": [{k: v for k, v in st.items() if k != "seconds"} for st in sweeps],
            "energy": e_tot, "energy_without_penalty": e_nopen, "class_energies": e_cls,
            "n_nodes": info["n_nodes"], "max_node_size": info["max_node_size"],
            "device_bytes": {"after_create": free0 - free1, "after_sweeps": free0 - free2, "gpu_total": total},
            "roofline": {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peaks[tp], "unit": "TFLOP/s",
                         "frac": achieved / peaks[tp], "own_dtype_frac": classes.get(dom, {}).get("own_peak"),
                         "share_of_step": d["ms"] / elapsed_ms},
            "classes": classes, "peaks_tflops": peaks, "clocks": clocks, "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
        s.close()
        del s, model
        torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--compare-fp64", dest="compare_fp64", action="store_true", default=True)
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--arms", dest="arms", action="store_true", default=True,
                    help="TF32 and BF16 arms and the g^2 scan {0.5, 2, 4} (one timed sweep each after three)")
    ap.add_argument("--no-arms", dest="arms", action="store_false")
    ap.add_argument("--no-probe", action="store_true", help="skip the in-run GEMM peak probes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="sweep", choices=["sweep", "heff", "batch", "scale", "profile", "physics"],
                    help="heff: only H_eff x products at --node (profiling aid); batch: batched "
                         "independent problems against sequential sweeps; scale: the 8x8x8 chi=128 Q=32 "
                         "lattice, --steps sweeps from the seeded start per g^2 of --scale-g2; profile: one "
                         "bottom product, move and upper product inside a profiler window; physics: the "
                         "finite-density, periodic zero-charge and capacitor workloads (driven sweeps)")
    ap.add_argument("--physics-chi", type=int, default=32)
    ap.add_argument("--physics-sweeps", type=int, default=14)
    ap.add_argument("--capacitor-mu", type=float, default=4.0)
    ap.add_argument("--scale-g2", type=float, nargs="+", default=[0.5, 3.0])
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
    elif args.mode == "scale":
        run_scale(args)
    elif args.mode == "profile":
        run_profile_window(args)
    elif args.mode == "physics":
        run_physics(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
