"""Learned sampling-rank seed for ADC2: data collection, GPU training, storage.

The rank estimate of eq. (bounds) (Sec. 4.1) is a bound that holds for every
distribution of the poles; on a given matrix class it can be loose (sampling
more columns than the blocks need) or, once the boundary moves run out, tight
enough that IDs stop at the sample size.  The library can instead seed each
ADC2 merge's sample size from a 7-64-64-1 network over per-node features
(TDEIG_FLAG_MLP_SEED), keeping the estimate as the fallback.

This module
  * records (features, ln(rank + 1)) of every HSS node from ADC2 solves made
    with TDEIG_FLAG_RECORD (ranks found by the interpolative decompositions at
    the solve's tolerance, with a generous oversampling so that few IDs stop
    at the sample size),
  * trains the network with the library's own forward/backward/Adam kernels
    (tdeig_mlp_train), and
  * stores it as JSON (rank_model.json beside this file) and loads it.

    python -m paper_1510_04591_gb300.rank_model [--out PATH] [--quick]

Inputs are seeded synthetic tridiagonals from ``inputs``: the few-deflation
random class (diagonal U[-1, 1], off-diagonal U[0.5, 1]) at N = 4096..32768,
Toeplitz(2, 1), and the Legendre, Laguerre, Hermite and Clement matrices.
"""
import argparse
import json
import os
import time

import numpy as np

from . import inputs
from .tdeig import FLAG_RECORD, MLP_IN, MLP_PARAMS, Solver

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PATH = os.path.join(_HERE, "rank_model.json")

# Options of the recording solves: HSS from K > 256 on (the random class
# deflates to K of a few hundred), rank cap 80 with 30 oversampling columns
# (the sample of the largest merges still fits one ID kernel's shared memory).
RECORD_OPTIONS = dict(hss_threshold=256, rank_cap=80, oversample=30)


def matrix(kind, n, seed=0):
    if kind == "random":
        return inputs.uniform(n, seed, lo_b=0.5, hi_b=1.0)
    if kind == "uniform":
        return inputs.uniform(n, seed)
    if kind == "toeplitz":
        return inputs.toeplitz(n, 2.0, 1.0)
    if kind == "legendre":
        return inputs.legendre(n)
    if kind == "laguerre":
        return inputs.laguerre(n)
    if kind == "hermite":
        return inputs.hermite(n)
    if kind == "clement":
        return inputs.clement(n)
    raise ValueError(kind)


def training_specs(quick=False):
    """(kind, n, seed, hss_leaf) of the recording solves (about 50k nodes)."""
    specs = []
    if quick:
        return [("random", 4096, 1, 128), ("random", 8192, 2, 64), ("toeplitz", 4096, 0, 128),
                ("legendre", 8192, 0, 128)]
    for n, count in ((4096, 6), (8192, 6), (16384, 6), (32768, 14)):
        for s in range(count):
            specs.append(("random", n, 1 + s, 128 if s % 2 == 0 else 64))
    for kind in ("toeplitz", "legendre", "laguerre", "hermite", "clement"):
        for n in (4096, 8192, 16384, 32768):
            for leaf in (64, 128, 160):
                if n == 32768 and leaf == 64:
                    continue
                specs.append((kind, n, 0, leaf))
    return specs


def collect(specs, options=None, log=None):
    """Records of ADC2 solves: X (m x 7), t (m,) float32, per-solve summaries."""
    import torch
    Xs, ts, info = [], [], []
    solvers = {}
    try:
        for kind, n, seed, leaf in specs:
            if leaf not in solvers:
                opts = dict(RECORD_OPTIONS, hss_leaf=leaf)
                if options:
                    opts.update(options)
                solvers[leaf] = Solver(**opts)
            S = solvers[leaf]
            a, b = matrix(kind, n, seed)
            d = torch.from_numpy(a).cuda()
            e = torch.from_numpy(b).cuda()
            t0 = time.time()
            S.solve(d, e, mode="adc2", flags=FLAG_RECORD, vectors=True)
            torch.cuda.synchronize()
            X, t = S.rank_records()
            Xs.append(X)
            ts.append(t)
            info.append(dict(kind=kind, n=n, seed=seed, hss_leaf=leaf, records=int(X.shape[0]),
                             seconds=round(time.time() - t0, 3)))
            if log:
                log(info[-1])
            del d, e
            torch.cuda.empty_cache()
    finally:
        for S in solvers.values():
            S.close()
    return np.concatenate(Xs), np.concatenate(ts), info


def init_params(seed):
    """He-normal weights, zero biases (output bias = 3, about ln(20))."""
    rng = np.random.default_rng(seed)
    H = 64
    p = np.zeros(MLP_PARAMS, dtype=np.float32)
    o = 0
    for fan_in, fan_out in ((MLP_IN, H), (H, H)):
        p[o:o + fan_in * fan_out] = rng.standard_normal(fan_in * fan_out) * np.sqrt(2.0 / fan_in)
        o += fan_in * fan_out + fan_out
    p[o:o + H] = rng.standard_normal(H) * np.sqrt(1.0 / H)
    p[o + H] = 3.0
    return p


def standardiser(X):
    mean = X.mean(axis=0).astype(np.float32)
    std = np.maximum(X.std(axis=0), 1e-3).astype(np.float32)
    return mean, std


def train(X, t, epochs=300, batch=256, lr=2e-3, seed=7, solver=None):
    """Trains on the GPU; returns (params, mean, std, final loss)."""
    mean, std = standardiser(X)
    p0 = init_params(seed)
    own = solver is None
    S = solver or Solver()
    try:
        p, loss = S.mlp_train(p0, mean, std, X, t, epochs=epochs, batch=batch, lr=lr, seed=seed)
    finally:
        if own:
            S.close()
    return p, mean, std, loss


def save(path, params, mean, std, meta=None):
    doc = {"format": "tdeig rank model: 7-64-64-1 ReLU, BF16 weights, target ln(rank + 1)",
           "mean": [float(x) for x in mean], "std": [float(x) for x in std],
           "params": [float(x) for x in params], "meta": meta or {}}
    with open(path, "w") as f:
        json.dump(doc, f, separators=(",", ":"))


def load(path=DEFAULT_PATH):
    with open(path) as f:
        doc = json.load(f)
    p = np.asarray(doc["params"], dtype=np.float32)
    if p.shape != (MLP_PARAMS,):
        raise ValueError("rank model has %d parameters, expected %d" % (p.shape[0], MLP_PARAMS))
    return p, np.asarray(doc["mean"], np.float32), np.asarray(doc["std"], np.float32)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--quick", action="store_true", help="small collection (tests)")
    ap.add_argument("--epochs", type=int, default=300)
    args = ap.parse_args(argv)
    t0 = time.time()
    X, t, info = collect(training_specs(args.quick), log=lambda r: print(json.dumps(r), flush=True))
    t1 = time.time()
    # 10 % of the records (a seeded random choice) are held out for validation
    perm = np.random.default_rng(12345).permutation(X.shape[0])
    nval = X.shape[0] // 10
    val, tr = perm[:nval], perm[nval:]
    with Solver() as S:
        p, mean, std, loss = train(X[tr], t[tr], epochs=args.epochs, solver=S)
        t2 = time.time()
        val_loss, _ = S.mlp_grad(p, mean, std, X[val], t[val])
        yv = S.mlp_forward(p, mean, std, X[val])
    rank = np.exp(t) - 1
    rel = np.abs(np.expm1(yv) - np.expm1(t[val])) / np.maximum(np.expm1(t[val]), 1.0)
    meta = dict(records=int(X.shape[0]), train_records=int(tr.shape[0]),
                solves=info, collect_s=round(t1 - t0, 1),
                train_s=round(t2 - t1, 1), final_loss=loss, val_loss=val_loss,
                val_rank_rel_err={"median": float(np.median(rel)),
                                  "p90": float(np.quantile(rel, 0.9))},
                epochs=args.epochs, record_options=RECORD_OPTIONS,
                rank_quantiles=[float(np.quantile(rank, q)) for q in (0.0, 0.5, 0.9, 1.0)])
    save(args.out, p, mean, std, meta)
    print(json.dumps({k: v for k, v in meta.items() if k != "solves"}))


if __name__ == "__main__":
    main()
