"""Benchmark: full eigendecomposition of a symmetric tridiagonal matrix on GB300.

Headline workload: Toeplitz(2, 1) of order N = 16384 (Sec. 5, Example 3), all
eigenvalues and eigenvectors, accelerated DC (HSS update) against plain dense
DC on the same GPU, orthogonality / residual required <= 1e-10.

One step = one full eigendecomposition through the C ABI (tdeig_solve) with
inputs and outputs resident in HBM.  Between timed steps the L2 is flushed by
writing a 256 MiB buffer outside the timed events.  Under torchrun every rank
solves its own copy (independent replicas; no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

METRIC ="full eigendecomp time at N=16384: ADC vs plain DC on GB300, orth/resid ≤1e-10"
FP64_FMA_PER_SM_CLK = 2          # measured: FP64 FMA chain throughput 1.19-1.20 TFLOP/s
N_SMS = 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--matrix", default="toeplitz", choices=["toeplitz", "random"])
    p.add_argument("--mode", default="adc2", choices=["adc1", "adc2", "dense"])
    p.add_argument("--prec", default="fp64", choices=["fp64", "split"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-dense-compare", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--stats-out", default=None)
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
# roofline of the dominant kernel, from the library's per-stage events
# --------------------------------------------------------------------------
def stage_work(stats):
    """Algorithmic work per stage launch (per level): flops of the dense update
    product 2 (n1 (K1 + Km) + n2 (K - K1)) K per merge."""
    out = {}
    for L in stats["levels"]:
        fl = 0.0
        for n, n1, K, K1, Km in L["merges"]:
            fl += 2.0 * (n1 * (K1 + Km) + (n - n1) * (K - K1)) * K
        out[L["height"]] = {"update_flops": fl}
    return out


def roofline(stats_list):
    """Dominant stage over the timed steps and its achieved rate."""
    tot = {}
    for st in stats_list:
        for k, v in st["stage_ms"].items():
            tot[k] = tot.get(k, 0.0) + v
    dom = max(tot, key=tot.get)
    fp64_peak = N_SMS * 2070e6 * 2 * FP64_FMA_PER_SM_CLK / 1e12
    res = {"kernel": dom, "share": tot[dom] / sum(tot.values()),
           "stage_share": {k: v / sum(tot.values()) for k, v in tot.items()}}
    fl = ms = 0.0
    n_launch = 0
    if dom == "update":
        for st in stats_list:
            work = stage_work(st)
            for L in st["levels"]:
                if "update" in L["ms"]:
                    fl += work[L["height"]]["update_flops"]
                    ms += L["ms"]["update"]
                    n_launch += 1
        res["kernel"] = "k_gemm_f64 (dense update)"
    elif dom in ("hss_mult", "hss_sample", "hss_build"):
        key = dom[4:]
        for st in stats_list:
            fl += sum(h["flops"][key] for h in st.get("hss", []) if "flops" in h)
            for L in st["levels"]:
                if dom in L["ms"]:
                    ms += L["ms"][dom]
                    n_launch += 1
        res["kernel"] = "k_gemm_grouped (%s)" % {"mult": "Algorithm 3 HSS x matrix",
                                                  "sample": "sampling Y, Z",
                                                  "build": "Algorithm 2 products"}[key]
    if fl > 0 and ms > 0:
        ach = fl / (ms / 1e3) / 1e12
        res.update({"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak, "traffic": None, "stage_launches": n_launch,
                    "peak_note": "FP64 FMA issue: 152 SMs x 2070 MHz x 2 FMA/clk/SM (measured "
                                 "FMA-chain probe 1.20 TFLOP/s; cuBLAS DGEMM 1.10)"})
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
            "config": {"workload": workload_name(args), "n": args.n, "matrix": args.matrix,
                       "mode": args.mode, "precision": "fp64"},
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
    a, b = matrix(args, rank)
    N = args.n
    d_d = torch.from_numpy(a).to(dev)
    e_d = torch.from_numpy(b).to(dev)
    lam = torch.empty(N, dtype=torch.float64, device=dev)
    Qt = torch.empty((N, N), dtype=torch.float64, device=dev)   # holds Q^T (column-major Q)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)   # 256 MiB
    mode = tdeig.mode_code(args.mode, args.prec)

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

    ms_step, stats, clocks = timed(mode, args.steps, args.warmup)
    launches = sum(int(s.get("launches", 0)) for s in stats)

    # accuracy of the timed result (Q and lambda of the last step)
    acc = accuracy(a, b, lam, Qt, dev)

    out = {"metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": workload_name(args), "n": N, "matrix": args.matrix,
                      "mode": args.mode, "precision": args.prec, "leaf": 32,
                      "hss_threshold": 2000, "hss_leaf": 128, "tol": 1e-12, "oversample": 10,
                      "l2": "flushed between timed steps (256 MiB write outside the events)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "accuracy": acc, "stage_ms": stats[-1]["stage_ms"], "clocks": clocks,
           "gpu_launches": launches}

    if not args.no_dense_compare and args.mode != "dense":
        ms_d, st_d, _ = timed(tdeig.mode_code("dense", "fp64"), 1, 1)
        acc_d = accuracy(a, b, lam, Qt, dev)
        out["plain_dc"] = {"value": ms_d / 1e3, "unit": "s", "accuracy": acc_d,
                           "stage_ms": st_d[-1]["stage_ms"]}
        out["speedup_vs_plain_dc"] = ms_d / ms_step
    out["roofline"] = roofline(stats)

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


def accuracy(a, b, lam, Qt, dev, sample=1024):
    """Orthogonality ||Q^T Q - I||_F / N (sampled columns, scaled) and residual
    ||T Q - Q Lambda||_F / (N ||T||_2) (all columns), closed-form eigenvalue error
    for Toeplitz(2,1)."""
    import torch
    N = lam.shape[0]
    Q = Qt.t()
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
    out = {"orth": orth, "orth_note": "%d sampled columns" % len(idx), "resid": res}
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


def cpu_baseline(args, a, b):
    from oracle import dc
    mode = {"dense": dc.MODE_DENSE, "adc1": dc.MODE_ADC1, "adc2": dc.MODE_ADC2}[args.mode]
    t = time.perf_counter()
    dc.solve(a, b, dc.Options(mode=mode))
    v = time.perf_counter() - t
    return {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "one full N=%d solve (C routines with OpenMP over roots, numpy BLAS "
                      "products, all host threads)" % args.n}


if __name__ == "__main__":
    sys.exit(main())
