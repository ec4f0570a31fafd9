"""Benchmark: full eigendecomposition of a symmetric tridiagonal matrix on GB300.

Headline workload: Toeplitz(2, 1) of order N = 16384 (Sec. 5, Example 3), all
eigenvalues and eigenvectors, accelerated DC (ADC2: randomized HSS update,
split-precision tensor-core products for Algorithm 3) against plain dense DC on
the same GPU (FP64 products and split products), orthogonality / residual
required <= 1e-10.

One step = one full eigendecomposition through the C ABI (tdeig_solve) with
inputs and outputs resident in HBM.  Between timed steps the L2 is flushed by
writing a 256 MiB buffer outside the timed events.  The timed steps run with
per-kernel CUDA events inside the library (TDEIG_FLAG_PROFILE); the roofline
of the dominant kernel is computed from them.  Under torchrun every rank solves
its own copy (independent replicas; no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batched    # 4096 uneven matrices, one batched call per step
  python bench.py --workload seed       # learned rank seed vs the rank estimate, N=32768
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "full eigendecomp time at N=16384: ADC vs plain DC on GB300, orth/resid ≤1e-10"
# arithmetic the timed path computes in, per precision flag
DTYPES = {"fp64": "f64",
          "split": "split-42/56 (BF16 7-bit digit slices: eigenvector products 42 bits, ADC2 "
                   "sampling 56 bits; exact FP32 tensor-core sums, FP64 recombination); FP64 "
                   "elsewhere",
          "bf16x2": "split-16 (BF16 hi+lo slices) products; FP64 elsewhere",
          "fp16x2": "split-22 (FP16 hi+lo slices) products; FP64 elsewhere"}
N_SMS = 152
SM_MHZ = 2070.0
FP64_FMA_PER_SM_CLK = 2          # measured: FP64 FMA chain throughput 1.19-1.20 TFLOP/s


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="single",
                   choices=["single", "batched", "seed", "families", "example2"])
    p.add_argument("--sizes", default="5000,10000,15000,20000,25000",
                   help="matrix orders of --workload families")
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--matrix", default="toeplitz", choices=["toeplitz", "random"])
    p.add_argument("--mode", default="adc2", choices=["adc1", "adc2", "dense"])
    p.add_argument("--prec", default="split", choices=["fp64", "split", "bf16x2", "fp16x2"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-dense-compare", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-profile", action="store_true")
    p.add_argument("--stats-out", default=None)
    p.add_argument("--graph", action="store_true",
                   help="--workload batched: replay the solve as a captured CUDA graph")
    return p.parse_args()


def matrix(args, rank=0):
    from paper_1510_04591_gb300 import inputs
    if args.matrix == "toeplitz":
        return inputs.toeplitz(args.n, 2.0, 1.0)
    return inputs.uniform(args.n, seed=1 + rank, lo_b=0.5, hi_b=1.0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def workload_name(args):
    if args.workload == "seed":
        return ("random (a~U[-1,1], b~U[0.5,1], held-out seed 1001) N=32768 full "
                "eigendecomposition, ADC2 update from K > 256, FP64 products: learned rank seed "
                "vs the rank estimate")
    if args.workload == "batched":
        return ("4096 tridiagonals, N uniform on [64, 2048] (seed 3), even members U[-1,1], odd "
                "members glued Wilkinson W21 (coupling 1e-8); %s update, %s products"
                % (args.mode.upper(), args.prec))
    m = "Toeplitz(2,1)" if args.matrix == "toeplitz" else "random (a~U[-1,1], b~U[0.5,1], seed 1)"
    return "%s N=%d full eigendecomposition, %s update, %s products" % (
        m, args.n, args.mode.upper(), args.prec)


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.path = os.path.join("/tmp", "tdeig_clocks_%d_%d.csv" % (os.getpid(), dev))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# roofline of the dominant kernel, from the library's per-kernel events
# --------------------------------------------------------------------------
def dense_update_flops(st):
    """Algorithmic flops of the block-structured dense update: per merge
    2 (n1 (K1 + Km) + n2 (K - K1)) K."""
    fl = 0.0
    for L in st.get("levels", []):
        if "update" not in L["ms"]:
            continue
        for n, n1, K, K1, Km in L["merges"]:
            fl += 2.0 * (n1 * (K1 + Km) + (n - n1) * (K - K1)) * K
    return fl


def grouped_flops(st):
    """FP64 flops of the grouped products (dense fallbacks, FP64 sampling, HSS
    construction, and Algorithm 3 when it is not split)."""
    fl = 0.0
    split = st.get("split_tensor_flops", 0.0) > 0.0
    for h in st.get("hss", []):
        f = h.get("flops")
        if f:
            fl += f["build"] + f["sample"]   # "sample" counts FP64 sampling only
            if not split:
                fl += f["dense"] + f["mult"]
    return fl


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel of the
# default workload (Toeplitz N=16384, ADC2, split), from an ncu capture of its timed solve
# (1-pass metrics over all 73 launches); to be removed when the kernel changes
DRAM_BYTES_PER_LAUNCH = {"k_split_umma": 4.1407e8}

# FP64 issue slots per FP64 secular term (2 subtractions, reciprocal by approximation and two
# Newton steps, multiply, add, FMA): 10 instructions, measured by an ncu capture of the
# kernel at about 14 slots of the FP64 pipe
FP64_SLOTS_PER_SECULAR_TERM = 14
# FP32 instructions per double-float secular term (two TwoSums for d_j - d_org - tau, the
# reciprocal with its correction, the term product, the TwoSum accumulation, the derivative)
FP32_INSTR_PER_DF_TERM = 37


def kernel_work(name, stats_list, pk):
    """Algorithmic work of one kernel over the profiled solves: (amount, peak,
    bound, unit, note), or None."""
    fp64_peak = N_SMS * SM_MHZ * 1e6 * 2 * FP64_FMA_PER_SM_CLK / 1e12
    if name == "k_gemm_f64":
        return (sum(dense_update_flops(s) for s in stats_list) / 1e12, fp64_peak, "alu", "TFLOP/s",
                "FP64 FMA issue: 152 SMs x 2070 MHz x 2 FMA/clk/SM (measured FMA-chain probe "
                "1.20 TFLOP/s; cuBLAS DGEMM 1.10)")
    if name == "k_gemm_grouped":
        fl = sum(grouped_flops(s) - s.get("small_gemm_flops", 0.0) for s in stats_list)
        return (fl / 1e12, fp64_peak, "alu", "TFLOP/s", "FP64 FMA issue peak, as for k_gemm_f64")
    if name == "k_gemm_small":
        return (sum(s.get("small_gemm_flops", 0.0) for s in stats_list) / 1e12, fp64_peak, "alu",
                "TFLOP/s", "FP64 FMA issue peak, as for k_gemm_f64 (HSS construction products, "
                "16 x 16 tiles)")
    if name == "k_split_umma":
        peak = pk.get("bf16_tflops", 1900.0)
        return (sum(s.get("split_tensor_flops", 0.0) for s in stats_list) / 1e12, peak, "tensor",
                "TFLOP/s", "tensor work issued (2 M N K per slice pair) against the measured bf16 "
                "peak (cuBLAS burst) %.0f TFLOP/s" % peak)
    if name in ("k_slice", "k_slice_exp", "k_slice_fused"):
        key = {"k_slice": "split_slice_bytes", "k_slice_exp": "split_exp_bytes",
               "k_slice_fused": "split_fused_bytes"}[name]
        peak = pk.get("hbm_gbs", 6800.0)
        what = {"k_slice": "reads each operand element once (8 B) and writes its s 16-bit slices "
                           "(2 s B per element, k padded to 32)",
                "k_slice_exp": "reads each operand element once (8 B) for the row exponents",
                "k_slice_fused": "one pass for operands with short rows (k <= 256): reads each "
                                 "element once (8 B), writes its s 16-bit slices (2 s B per "
                                 "element, k padded to 32) and the row exponents"}[name]
        return (sum(s.get(key, 0.0) for s in stats_list) / 1e9, peak, "hbm", "GB/s",
                "algorithmic bytes: %s; masked sampling entries counted as read; against the "
                "measured HBM copy bandwidth %.0f GB/s" % (what, peak))
    if name == "k_secular":
        # ALU roofline of two pipes working in parallel: FP64 terms on the FP64 pipe
        # (2 lanes/clk/SM), double-float terms on the FP32 pipe (128 lanes/clk/SM); the
        # kernel's bound is the larger time, reported as FP64 issue (it dominates)
        terms = sum(s.get("secular_terms", 0) for s in stats_list)
        dft = sum(s.get("secular_df_terms", 0) for s in stats_list)
        peak = N_SMS * SM_MHZ * 1e6 * 2 / 1e12   # FP64 lanes: 2/clk/SM
        t64 = terms * FP64_SLOTS_PER_SECULAR_TERM / (peak * 1e12)
        t32 = dft * FP32_INSTR_PER_DF_TERM / (N_SMS * SM_MHZ * 1e6 * 128)
        eq = max(t64, t32) * peak   # FP64-slot equivalent of the bound
        return (eq, peak, "alu", "Tinstr/s",
                "FP64 pipe issue, 152 SMs x 2070 MHz x 2 lanes/clk/SM; %d FP64 slots per FP64 "
                "secular term (ncu) and %d FP32 instructions per double-float term (on the "
                "64x faster FP32 pipe, in parallel); terms counted on the device: %.3g FP64, "
                "%.3g double-float" % (FP64_SLOTS_PER_SECULAR_TERM, FP32_INSTR_PER_DF_TERM,
                                       terms, dft))
    return None


def roofline(stats_list, pk):
    kern = {}
    for st in stats_list:
        for k, v in st.get("kernels", {}).items():
            a = kern.setdefault(k, [0.0, 0])
            a[0] += v["ms"]
            a[1] += v["launches"]
    if not kern:
        return None
    total = sum(v[0] for v in kern.values())
    order = sorted(kern, key=lambda k: -kern[k][0])
    dom = order[0]
    ms, launches = kern[dom]
    res = {"kernel": dom, "share": ms / total, "launches": launches,
           "avg_launch_ms": ms / max(launches, 1),
           "kernel_share": {k: round(kern[k][0] / total, 4) for k in order},
           "traffic": None}
    per = []
    for k in order:
        w = kernel_work(k, stats_list, pk)
        if not w or not w[0]:
            continue
        amount, peak, bound, unit, note = w
        ach = amount / (kern[k][0] / 1e3)
        ent = {"kernel": k, "share": round(kern[k][0] / total, 4), "bound": bound,
               "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
               "peak_note": note + " (of measured)"}
        per.append(ent)
        if k == dom:
            res.update({kk: ent[kk] for kk in ("bound", "achieved", "peak", "unit", "frac",
                                               "peak_note")})
    res["kernels"] = per
    return res


def flush_l2(buf):
    buf.add_(1.0)


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import dc
    mode = {"dense": dc.MODE_DENSE, "adc1": dc.MODE_ADC1, "adc2": dc.MODE_ADC2}[args.mode]
    small = argparse.Namespace(**vars(args))
    small.n = 1024
    a0, b0 = matrix(small)
    for _ in range(args.warmup):
        dc.solve(a0, b0, dc.Options(mode=mode))
    a, b = matrix(args)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        dc.solve(a, b, dc.Options(mode=mode))
        times.append(time.perf_counter() - t)
    v = float(np.mean(times))
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(args) + " (CPU oracle, FP64)", "n": args.n,
                       "matrix": args.matrix, "mode": args.mode, "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": "full N=%d solve per step (warm-up steps at N=1024)"
                                       % args.n},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig

    stream = torch.cuda.Stream(device=dev)
    solver = tdeig.Solver(stream=stream.cuda_stream)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)   # 256 MiB
    mode = tdeig.mode_code(args.mode, args.prec)
    prof = 0 if args.no_profile else (1 << 13)

    if args.workload == "batched":
        return run_batched(args, torch, dist, world, rank, local, dev, stream, solver, flush,
                           tdeig, mode, prof)
    if args.workload == "seed":
        solver.close()
        return run_seed(args, torch, dist, world, rank, local, dev, stream, flush, tdeig)
    if args.workload == "families":
        return run_families(args, torch, dist, world, rank, dev, stream, solver, flush, tdeig)
    if args.workload == "example2":
        solver.close()
        return run_example2(args, torch, dist, world, rank, dev, stream, flush, tdeig)

    a, b = matrix(args, rank)
    N = args.n
    d_d = torch.from_numpy(a).to(dev)
    e_d = torch.from_numpy(b).to(dev)
    lam = torch.empty(N, dtype=torch.float64, device=dev)
    Qt = torch.empty((N, N), dtype=torch.float64, device=dev)   # holds Q^T (column-major Q)

    def one(m):
        st = solver.solve_raw(d_d.data_ptr(), e_d.data_ptr(), N, lam.data_ptr(), Qt.data_ptr(), m)
        if st != 0:
            raise tdeig.TdeigError(st, "tdeig_solve")
        return json.loads(solver.stats())

    def timed(m, steps, warmup):
        for _ in range(warmup):
            one(m)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        stats, ms = [], []
        clocks = Clocks(local)
        clocks.start()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(one(m))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        ck = clocks.stop()
        if world > 1:
            dist.barrier()
        tot = torch.tensor([sum(ms)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        return float(tot.item()) / steps, stats, ck

    ms_step, stats, clocks = timed(mode | prof, args.steps, args.warmup)
    launches = sum(int(s.get("launches", 0)) for s in stats)
    acc = accuracy(a, b, lam, Qt, dev, sample=None)   # every column of the timed result

    out = {"metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPES[args.prec], "data": "synthetic",
           "orth": acc["orth"], "resid": acc["resid"],
           "config": {"workload": workload_name(args), "n": N, "matrix": args.matrix,
                      "mode": args.mode, "precision": args.prec, "leaf": 32,
                      "hss_threshold": 2000, "hss_leaf": 128, "tol": 1e-12, "oversample": 10,
                      "l2": "flushed between timed steps (256 MiB write outside the events)",
                      "timing": "CUDA events on the solve's stream; per-kernel events inside "
                                "the library during the timed steps",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "accuracy": acc, "stage_ms": stats[-1]["stage_ms"], "clocks": clocks,
           "gpu_launches": launches}

    if not args.no_dense_compare and args.mode != "dense":
        out["plain_dc"] = {}
        for pr in ("fp64", "split"):
            ms_d, st_d, _ = timed(tdeig.mode_code("dense", pr), 1, 1)
            out["plain_dc"][pr] = {"value": ms_d / 1e3, "unit": "s",
                                   "accuracy": accuracy(a, b, lam, Qt, dev),
                                   "stage_ms": st_d[-1]["stage_ms"]}
        out["speedup_vs_plain_dc"] = {pr: out["plain_dc"][pr]["value"] / (ms_step / 1e3)
                                      for pr in ("fp64", "split")}
    if not args.no_dense_compare and args.prec != "fp64":
        # the same ADC variant with FP64 products (the paper's precision), timed the
        # same way: 3 steps after 1 warm-up
        ms_f, st_f, ck_f = timed(tdeig.mode_code(args.mode, "fp64") | prof, 3, 1)
        out["adc_fp64"] = {"value": ms_f / 1e3, "unit": "s", "steps": 3, "warmup": 1,
                           "mode": args.mode, "precision": "fp64",
                           "accuracy": accuracy(a, b, lam, Qt, dev),
                           "stage_ms": st_f[-1]["stage_ms"], "clocks": ck_f,
                           "roofline": roofline(st_f, peaks())}
    out["roofline"] = roofline(stats, peaks())
    rl = out["roofline"]
    if (rl and args.n == 16384 and args.matrix == "toeplitz" and args.mode == "adc2"
            and args.prec == "split" and rl["kernel"] in DRAM_BYTES_PER_LAUNCH):
        rl["traffic"] = DRAM_BYTES_PER_LAUNCH[rl["kernel"]]
        rl["traffic_note"] = ("DRAM bytes read + written per launch, mean over the launches of "
                              "one timed solve of this workload in an ncu capture "
                              "(profiles/k_split_umma_toeplitz4096_full.md)")

    if not args.no_e2e:
        out["e2e"] = e2e(args, a, b, solver, mode)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, a, b)
    if args.stats_out and rank == 0:
        with open(args.stats_out, "w") as f:
            json.dump(stats, f)
    solver.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args, torch, dist, world, rank, local, dev, stream, solver, flush, tdeig, mode,
                prof):
    """configs: 4096 independent uneven tridiagonals in one tdeig_solve_batched call per step."""
    import ctypes
    from paper_1510_04591_gb300 import inputs
    ms_list = inputs.batch(4096, 3, 64, 2048)
    sizes = [len(x) for x, _ in ms_list]
    d = torch.from_numpy(np.concatenate([x for x, _ in ms_list])).to(dev)
    e = torch.from_numpy(np.concatenate([y for _, y in ms_list])).to(dev)
    lam = torch.empty(sum(sizes), dtype=torch.float64, device=dev)
    Q = torch.empty(sum(n * n for n in sizes), dtype=torch.float64, device=dev)
    Ns = (ctypes.c_int64 * len(sizes))(*sizes)
    L = tdeig.lib()

    def one(m):
        st = L.tdeig_solve_batched(solver.h, len(sizes), Ns, d.data_ptr(), e.data_ptr(),
                                   lam.data_ptr(), Q.data_ptr(), m)
        if st != 0:
            raise tdeig.TdeigError(st, "tdeig_solve_batched")
        return json.loads(solver.stats())

    if args.graph:
        mode |= tdeig.FLAG_GRAPH
    for _ in range(args.warmup):
        one(mode)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one(mode)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ck = clocks.stop()
    v = float(np.mean(ms)) / 1e3
    stats = None
    if prof:
        stats = one((mode & ~tdeig.FLAG_GRAPH) | prof)   # one extra, untimed profiled solve
        if args.stats_out and rank == 0:
            with open(args.stats_out, "w") as f:
                json.dump(stats, f)
    out = {"metric": "batched eigendecomposition time, 4096 uneven tridiagonals", "value": v,
           "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPES[args.prec], "data": "synthetic",
           "config": {"workload": workload_name(args), "members": len(sizes),
                      "rows": int(sum(sizes)), "q_entries": int(sum(n * n for n in sizes)),
                      "graph": bool(args.graph)},
           "clocks": ck, "matrices_per_s": len(sizes) / v}
    if stats is not None:
        ch = stats.get("chunks", [stats])
        kern = {}
        for c in ch:
            for k, kv in c.get("kernels", {}).items():
                kern[k] = kern.get(k, 0.0) + kv["ms"]
        tot = sum(kern.values()) or 1.0
        out["kernel_share_untimed_solve"] = {k: round(t / tot, 4) for k, t in
                                             sorted(kern.items(), key=lambda x: -x[1])[:10]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    solver.close()
    return 0


def run_seed(args, torch, dist, world, rank, local, dev, stream, flush, tdeig):
    """Learned sampling-rank seed against the rank estimate of eq. (bounds) on the
    few-deflation random class at N = 32768 (deflation leaves K of a few hundred
    per merge, so HSS runs from K > 256).  value: model-seeded solve time."""
    from paper_1510_04591_gb300 import inputs, rank_model
    N = 32768
    a, b = inputs.uniform(N, 1001 + rank, lo_b=0.5, hi_b=1.0)
    d_d = torch.from_numpy(a).to(dev)
    e_d = torch.from_numpy(b).to(dev)
    lam = torch.empty(N, dtype=torch.float64, device=dev)
    Qt = torch.empty((N, N), dtype=torch.float64, device=dev)
    solver = tdeig.Solver(stream=stream.cuda_stream, hss_threshold=256)
    solver.set_rank_model(*rank_model.load())
    base = tdeig.mode_code("adc2", "fp64")
    res = {}
    ck = None
    for name, fl in (("estimate", 0), ("model", tdeig.FLAG_MLP_SEED)):
        m = base | fl
        for _ in range(args.warmup):
            solver.solve_raw(d_d.data_ptr(), e_d.data_ptr(), N, lam.data_ptr(), Qt.data_ptr(), m)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = Clocks(local)
        clocks.start()
        ms = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solver.solve_raw(d_d.data_ptr(), e_d.data_ptr(), N, lam.data_ptr(),
                                  Qt.data_ptr(), m)
            e1.record(stream)
            e1.synchronize()
            if st != 0:
                raise tdeig.TdeigError(st, "tdeig_solve")
            ms.append(e0.elapsed_time(e1))
        c = clocks.stop()
        ck = ck or c
        stt = json.loads(solver.stats())
        hm = [h for h in stt.get("hss", []) if "K" in h]
        res[name] = {"value": float(np.mean(ms)) / 1e3, "unit": "s",
                     "accuracy": accuracy(a, b, lam, Qt, dev),
                     "hss_merges": len(hm),
                     "sampled_columns_sum_K_s": int(sum(h["K"] * h["s"] for h in hm)),
                     "mean_sample_size": float(np.mean([h["s"] for h in hm])) if hm else 0.0,
                     "ids_at_sample_size": int(sum(h["kmax"] >= h["s"] for h in hm)),
                     "fallbacks": stt.get("mlp_fallbacks", 0),
                     "stage_ms": {k: round(v, 3) for k, v in stt.get("stage_ms", {}).items()}}
    solver.close()
    v = res["model"]["value"]
    t_max = torch.tensor([v], device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    out = {"metric": "learned rank seed: ADC2 eigendecomposition time, N=32768 random",
           "value": float(t_max.item()), "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": float(t_max.item()) * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": workload_name(args), "n": N, "hss_threshold": 256,
                      "hss_leaf": 128, "oversample": 10,
                      "l2": "flushed between timed steps (256 MiB write outside the events)"},
           "clocks": ck, "estimate": res["estimate"], "model": res["model"],
           "speedup_vs_estimate": res["estimate"]["value"] / res["model"]["value"]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# Sec. 5, Example 3: ADC1 / ADC2 speedups over multithreaded MKL dstevd printed in Tables 5
# and 6 at N = 25000 (16 Xeon E5-2670 threads; context only: the comparator here is this
# library's own dense DC on the same GPU).
PAPER_SPEEDUP_25K = {"toeplitz": (6.05, 5.79), "clement": (5.03, 5.12), "legendre": (4.81, 4.72),
                     "laguerre": (5.00, 4.68), "hermite": (5.08, 5.04)}


def run_families(args, torch, dist, world, rank, dev, stream, solver, flush, tdeig):
    """The few-deflation families of Sec. 5, Example 3 (Tables 5 and 6): Toeplitz(2, 1),
    Clement, Legendre-, Laguerre- and Hermite-type matrices at N = 5000 ... 25000, each
    solved by dense DC, ADC1 and ADC2 (HSS when K > 2000, split-precision products) on
    the same GPU: one warm-up and one timed solve per case (L2 flushed before it),
    orthogonality and residual on 256 sampled columns.  value: the summed ADC2 time."""
    from paper_1510_04591_gb300 import inputs
    sizes = [int(x) for x in args.sizes.split(",") if x]
    fams = ["toeplitz", "clement", "legendre", "laguerre", "hermite"]
    rows = []
    total = 0.0
    ck = None
    for n in sizes:
        Qt = torch.empty((n, n), dtype=torch.float64, device=dev)
        lam = torch.empty(n, dtype=torch.float64, device=dev)
        for fam in fams:
            a, b = getattr(inputs, fam)(n)
            d_d = torch.from_numpy(a).to(dev)
            e_d = torch.from_numpy(b).to(dev)
            ent = {"family": fam, "n": n}
            for mode in ("dense", "adc1", "adc2"):
                m = tdeig.mode_code(mode, args.prec)
                solver.solve_raw(d_d.data_ptr(), e_d.data_ptr(), n, lam.data_ptr(), Qt.data_ptr(), m)
                torch.cuda.synchronize()
                with torch.cuda.stream(stream):
                    flush_l2(flush)
                clocks = Clocks(int(dev.index or 0))
                clocks.start()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = solver.solve_raw(d_d.data_ptr(), e_d.data_ptr(), n, lam.data_ptr(),
                                      Qt.data_ptr(), m)
                e1.record(stream)
                e1.synchronize()
                c = clocks.stop()
                ck = ck or c
                if st != 0:
                    raise tdeig.TdeigError(st, "tdeig_solve")
                t = e0.elapsed_time(e1) / 1e3
                acc = accuracy(a, b, lam, Qt, dev, sample=256)
                hm = [h for h in json.loads(solver.stats()).get("hss", []) if "K" in h]
                ent[mode] = {"s": t, "orth": acc["orth"], "resid": acc["resid"],
                             "hss_merges": len(hm)}
                if mode == "adc2":
                    total += t
            ent["speedup_adc1"] = ent["dense"]["s"] / ent["adc1"]["s"]
            ent["speedup_adc2"] = ent["dense"]["s"] / ent["adc2"]["s"]
            if n == 25000:
                ent["paper_speedup_vs_mkl_16threads"] = PAPER_SPEEDUP_25K[fam]
            rows.append(ent)
        del Qt
        torch.cuda.empty_cache()
    out = {"metric": "few-deflation families (Sec. 5 Example 3): summed ADC2 eigendecomposition "
                     "time, dense DC / ADC1 / ADC2 per case", "value": total, "unit": "s",
           "n_gpus": world, "steps": 1, "warmup": 1, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.prec], "data": "synthetic",
           "config": {"workload": "Toeplitz(2,1), Clement, Legendre, Laguerre, Hermite at N = %s; "
                                  "dense DC, ADC1, ADC2 with %s products, HSS threshold 2000, "
                                  "HSS leaves 128" % (args.sizes, args.prec),
                      "l2": "flushed before each timed solve (256 MiB write outside the events)"},
           "clocks": ck, "cases": rows}
    if rank == 0:
        print(json.dumps(out), flush=True)
    solver.close()
    return 0


# Sec. 5, Example 2 (Table 3): seconds on 16 Xeon E5-2670 threads (context only).
PAPER_TABLE3_16T = {"srrsc_construction": 0.31, "srrsc_multiply": 0.85, "rshss_sampling": 0.16,
                    "rshss_construction": 0.42, "rshss_multiply": 0.95, "srrsc_hss_rank": 57,
                    "rshss_rank_estimate": 79}


def run_example2(args, torch, dist, world, rank, dev, stream, flush, tdeig):
    """Sec. 5, Example 2 (Table 3): the Cauchy-like matrix of Example 1 (d_i = 8 i / N,
    random unit u, rho = 1) at N = 10000, HSS leaves of about 200 rows (2^6 leaves of
    156), built by SRRSC (ADC1) and by randomized sampling (ADC2) and multiplied from the
    right into a 10000 x 10000 Gaussian X (Algorithm 3), through tdeig_hss_apply; the
    generators come from the library's secular and Loewner stages.  Per variant: one
    warm-up, then `steps` timed calls (L2 flushed before each); sub-stage device times
    from the library's events; error against the dense product X Qhat."""
    from paper_1510_04591_gb300 import inputs
    N = 10000
    d, u = inputs.example1(N, 2)
    solver = tdeig.Solver(stream=stream.cuda_stream, hss_leaf=200)
    dd = torch.from_numpy(d).to(dev)
    uu = torch.from_numpy(u).to(dev)
    lam, gam, mu = solver.secular(dd, uu, 1.0)
    uh, v, Qh = solver.lowner_cauchy(dd, gam, mu, uu, 1.0, qhat=True)
    g = torch.Generator(device=dev).manual_seed(7)
    X = torch.randn((N, N), dtype=torch.float64, device=dev, generator=g).t()   # column-major
    ref = X @ Qh
    rn = float(torch.linalg.norm(ref))
    del Qh
    res = {}
    ck = None
    for mode in ("adc1", "adc2"):
        for prec in ("fp64", "split"):
            out = solver.hss_apply(dd, gam, mu, uh, X, mode, prec)   # warm-up
            torch.cuda.synchronize()
            clocks = Clocks(int(dev.index or 0))
            clocks.start()
            ms, stages = [], []
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush_l2(flush)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = solver.hss_apply(dd, gam, mu, uh, X, mode, prec)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                stages.append(json.loads(solver.stats()))
            c = clocks.stop()
            ck = ck or c
            st = stages[-1]
            rec = [h for h in st.get("hss", []) if "K" in h][0]
            sm = {k: float(np.mean([x["stage_ms"].get(k, 0.0) for x in stages])) / 1e3
                  for k in st["stage_ms"]}
            ent = {"total_s": float(np.mean(ms)) / 1e3,
                   "construction_s": sm.get("hss_build", 0.0) + (sm.get("hss_sample", 0.0)
                                                                if mode == "adc2" else 0.0),
                   "multiply_s": sm.get("hss_mult", 0.0),
                   "stage_s": sm,
                   "rel_error_vs_dense": float(torch.linalg.norm(out - ref)) / rn,
                   "hss_rank_max": rec["kmax"], "hss_rank_mean": rec["kmean"]}
            if mode == "adc2":
                ent["sampling_s"] = sm.get("hss_sample", 0.0)
                ent["rank_estimate"] = rec["r"]
                ent["sample_size"] = rec["s"]
            res["%s_%s" % (mode, prec)] = ent
    v2 = res["adc2_fp64"]["construction_s"] + res["adc2_fp64"]["multiply_s"]
    out = {"metric": "Example 2 HSS microbenchmark (Sec. 5, Table 3): randomized HSS construction "
                     "+ multiplication time, N=10000", "value": v2, "unit": "s",
           "n_gpus": world, "steps": args.steps, "warmup": 1, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (adc*_fp64 entries), "
           + DTYPES["split"] + " (adc*_split entries)", "data": "synthetic",
           "config": {"workload": "Example 1 Cauchy-like matrix N=10000 (d_i = 8i/N, random unit u, "
                                  "rho=1, seed 2), HSS leaves ~200 (2^6 leaves), tol 1e-12, p=10, "
                                  "X 10000x10000 Gaussian; ADC1 (SRRSC) and ADC2 (RSHSS)",
                      "l2": "flushed before each timed call (256 MiB write outside the events)"},
           "clocks": ck, "variants": res, "paper_table3_16_threads_context": PAPER_TABLE3_16T}
    solver.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def accuracy(a, b, lam, Qt, dev, sample=1024):
    """Orthogonality ||Q^T Q - I||_F / N (sample=None: all columns; else sampled
    columns, scaled) and residual ||T Q - Q Lambda||_F / (N ||T||_2) (all
    columns), closed-form eigenvalue error for Toeplitz(2,1)."""
    import torch
    N = lam.shape[0]
    Q = Qt.t()
    if sample is None or sample >= N:
        G = Q.t() @ Q
        G.diagonal().sub_(1.0)
        orth = float(torch.linalg.norm(G)) / N
        idx = torch.arange(N)
    else:
        g = torch.Generator(device="cpu").manual_seed(0)
        idx = torch.randperm(N, generator=g)[:min(sample, N)].to(dev)
        G = Q.t() @ Q[:, idx]
        G[idx, torch.arange(len(idx), device=dev)] -= 1.0
        orth = float(torch.linalg.norm(G)) * math.sqrt(N / len(idx)) / N
    ad = torch.from_numpy(a).to(dev)
    bd = torch.from_numpy(b).to(dev)
    TQ = ad[:, None] * Q
    TQ[:-1] += bd[:, None] * Q[1:]
    TQ[1:] += bd[:, None] * Q[:-1]
    TQ -= Q * lam[None, :]
    tn = float(lam.abs().max())
    res = float(torch.linalg.norm(TQ)) / (N * tn)
    out = {"orth": orth, "resid": res,
           "orth_note": "all %d columns" % N if len(idx) == N else "%d sampled columns" % len(idx)}
    if np.all(a == 2.0) and np.all(b == 1.0):
        k = np.arange(1, N + 1)
        ex = np.sort(2 + 2 * np.cos(k * np.pi / (N + 1)))
        lh = lam.cpu().numpy()
        out["eig_err_closed_form"] = float(np.max(np.abs(lh - ex)) / np.max(np.abs(ex)))
    del G, TQ
    return out


def e2e(args, a, b, solver, mode, steps=2):
    """Same metric through the public API with host (pinned) buffers: the
    library copies inputs to the device and results back inside the call."""
    import torch
    N = args.n
    d_h = torch.from_numpy(a).pin_memory()
    e_h = torch.from_numpy(b).pin_memory()
    lam_h = torch.empty(N, dtype=torch.float64).pin_memory()
    Q_h = torch.empty((N, N), dtype=torch.float64).pin_memory()
    ts = []
    for i in range(steps + 1):
        t = time.perf_counter()
        st = solver.solve_raw(d_h.data_ptr(), e_h.data_ptr(), N, lam_h.data_ptr(), Q_h.data_ptr(),
                              mode)
        dt = time.perf_counter() - t
        if st != 0:
            return {"error": st}
        if i > 0:
            ts.append(dt)
    return {"value": float(np.mean(ts)), "unit": "s", "h2d_bytes_per_step": 8 * (2 * N - 1),
            "d2h_bytes_per_step": 8 * (N + N * N), "steps": steps}


_CPU_JOB = r'''
import json, os, sys, time
threads = int(sys.argv[6])
if threads == 1:
    os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    os.cpu_count = lambda: 1          # the oracle sizes its root-parallel loop by this
sys.path.insert(0, sys.argv[1])
import numpy as np
kind, n, mode, matrix = sys.argv[2], int(sys.argv[3]), sys.argv[4], sys.argv[5]
from paper_1510_04591_gb300 import inputs
if matrix == "toeplitz":
    a, b = inputs.toeplitz(n, 2.0, 1.0)
else:
    a, b = inputs.uniform(n, seed=1, lo_b=0.5, hi_b=1.0)
t = time.perf_counter()
if kind == "oracle":
    from oracle import dc
    dc.solve(a, b, dc.Options(mode={"dense": 0, "adc1": 1, "adc2": 2}[mode]))
else:
    import scipy.linalg.lapack as lapack
    w, v, info = lapack.dstevd(a, b, compute_v=1)
    assert info == 0
print(json.dumps({"s": time.perf_counter() - t}))
'''


def _cpu_job(kind, n, mode, matrix, threads, timeout=600):
    """One timed CPU solve in a fresh process whose thread pools (OpenMP,
    BLAS) are limited to `threads`; returns seconds or None."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    try:
        r = subprocess.run([sys.executable, "-c", _CPU_JOB, ROOT, kind, str(n), mode, matrix,
                            str(threads)], capture_output=True, text=True, timeout=timeout,
                           env=env)
        return json.loads(r.stdout.strip().splitlines()[-1])["s"]
    except Exception:
        return None


def cpu_baseline(args, a, b):
    """The oracle on the host: one full solve of the workload on all host threads
    (the reported value), one bounded single-thread sample, and LAPACK dstevd
    (divide and conquer, scipy) on all threads as the stand-in for the paper's
    multithreaded MKL comparator (its ratios are context only)."""
    from oracle import dc
    mode = {"dense": dc.MODE_DENSE, "adc1": dc.MODE_ADC1, "adc2": dc.MODE_ADC2}[args.mode]
    t = time.perf_counter()
    dc.solve(a, b, dc.Options(mode=mode))
    v = time.perf_counter() - t
    cores = os.cpu_count()
    n1 = min(args.n, 4096)
    st = _cpu_job("oracle", n1, args.mode, args.matrix, 1)
    lp = _cpu_job("lapack", args.n, args.mode, args.matrix, cores)
    return {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": "one full N=%d solve in %s mode, FP64 (C routines with OpenMP over "
                      "roots, numpy BLAS products, all host threads)" % (args.n, args.mode),
            "single_thread": {"value": st, "unit": "s", "cores": 1, "kind": "oracle",
                              "sample": "one full N=%d solve (same matrix family and mode), "
                                        "one thread pinned to one core" % n1},
            "lapack_dstevd": {"value": lp, "unit": "s", "cores": cores, "kind": "library",
                              "sample": "scipy LAPACK dstevd (divide and conquer, all "
                                        "eigenvectors), full N=%d, %d BLAS threads"
                                        % (args.n, cores)}}


if __name__ == "__main__":
    sys.exit(main())
