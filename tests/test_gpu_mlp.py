"""GPU tests of the learned ADC2 rank seed.

* the model's forward pass and gradient (library kernels) against the CPU
  oracle (oracle/mlp.py, which emulates the BF16 rounding of weights and
  activations and sums in FP64);
* GPU training reduces the loss, and the oracle's loss at the trained
  parameters matches the loss the library reports;
* node features against the oracle's definitions on a real merge;
* recording, seeding and the saturation fallback inside ADC2 solves;
* the gain of the committed model over the rank estimate of eq. (bounds) on
  the few-deflation random class (diagonal U[-1, 1], off-diagonal U[0.5, 1])
  at N = 32768, and on Toeplitz(2, 1).

Tolerances: a BF16 activation whose FP32 and FP64 pre-activations straddle a
rounding boundary flips by one BF16 unit (2^-8 relative); with weights of
order 0.3 this moves an output by about 1e-3, so outputs are compared to
1e-2 (1 + |y|) each and to 1e-4 in the median, gradients to 1e-2 in relative
2-norm.
"""
import json
import math

import numpy as np
import pytest

from oracle import dc, metrics
from oracle import mlp as omlp
from paper_1510_04591_gb300 import inputs

pytestmark = pytest.mark.gpu


def tdeig():
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig as t
    return t


def rank_model():
    tdeig()
    from paper_1510_04591_gb300 import rank_model as rm
    return rm


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(omlp.NPARAM) * scale
    p[omlp.OFF_B3] = 3.0
    return p.astype(np.float32)


def features_like(n, seed):
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(4, 8, n), rng.uniform(-12, -3, n), rng.uniform(-6, -2, n),
                         rng.uniform(-8, 0, n), rng.uniform(-6, 0, n), rng.uniform(0, 0.5, n),
                         rng.uniform(10, 15, n)])
    return X.astype(np.float32)


def stdz(X):
    return X.mean(axis=0).astype(np.float32), X.std(axis=0).astype(np.float32)


def test_forward_matches_oracle():
    t = tdeig()
    X = features_like(3000, 1)          # several CTAs and a ragged tail
    mean, std = stdz(X)
    p = random_params(2)
    with t.Solver() as S:
        y = S.mlp_forward(p, mean, std, X)
    yo, _ = omlp.forward(p, mean, std, X, bf16=True)
    err = np.abs(y - yo)
    assert np.all(err <= 1e-2 * (1 + np.abs(yo))), err.max()
    assert np.median(err) <= 1e-4


def test_forward_empty_and_single():
    t = tdeig()
    p = random_params(3)
    mean, std = np.zeros(7, np.float32), np.ones(7, np.float32)
    with t.Solver() as S:
        assert S.mlp_forward(p, mean, std, np.zeros((0, 7), np.float32)).shape == (0,)
        X = features_like(1, 4)
        y = S.mlp_forward(p, mean, std, X)
    yo, _ = omlp.forward(p, mean, std, X)
    assert abs(y[0] - yo[0]) <= 1e-2 * (1 + abs(yo[0]))


@pytest.mark.parametrize("n", [1, 127, 1000])
def test_gradient_matches_oracle(n):
    t = tdeig()
    X = features_like(n, 5 + n)
    mean, std = stdz(X) if n > 1 else (np.zeros(7, np.float32), np.ones(7, np.float32))
    p = random_params(6)
    rng = np.random.default_rng(7)
    tt = rng.uniform(2, 4.5, n).astype(np.float32)
    with t.Solver() as S:
        loss, g = S.mlp_grad(p, mean, std, X, tt)
    lo, go = omlp.loss_grad(p, mean, std, X, tt, bf16=True)
    assert abs(loss - lo) <= 1e-3 * lo + 1e-7
    assert np.linalg.norm(g - go) <= 1e-2 * np.linalg.norm(go)
    # every block of the parameter vector is exercised
    for a, b in ((0, omlp.OFF_B1), (omlp.OFF_W2, omlp.OFF_B2), (omlp.OFF_W3, omlp.OFF_B3)):
        assert np.linalg.norm(g[a:b] - go[a:b]) <= 2e-2 * np.linalg.norm(go[a:b]) + 1e-9


def test_training_reduces_loss():
    t = tdeig()
    X = features_like(4096, 8)
    mean, std = stdz(X)
    xs = (X - mean) / std
    tt = (3.0 + 0.4 * np.abs(xs[:, 0]) - 0.3 * xs[:, 3] + 0.2 * xs[:, 1] * xs[:, 4]).astype(np.float32)
    rm = rank_model()
    p0 = rm.init_params(1)
    l0 = omlp.loss_grad(p0, mean, std, X, tt)[0]
    with t.Solver() as S:
        p1, loss = S.mlp_train(p0, mean, std, X, tt, epochs=40, batch=256, lr=2e-3, seed=3)
    lo = omlp.loss_grad(p1, mean, std, X, tt)[0]
    assert loss < 0.05 * l0, (loss, l0)
    assert abs(loss - lo) <= 2e-2 * lo + 1e-6


def test_node_features_match_oracle():
    t = tdeig()
    K, n = 1500, 1600
    d, z = inputs.example1(K, 11)
    rho = 1.0
    lam, gam, mu, _ = dc.secular(d, z, rho)
    uh = dc.lowner(d, gam, mu, rho, z)
    ranges = [(q * 100, min((q + 1) * 100, K)) for q in range(15)]
    ranges += [(0, 700), (700, K), (0, K), (1499, 1500), (0, 1)]
    with t.Solver() as S:
        F = S.node_features(d, gam, mu, uh, n, ranges)
    for (s0, s1), f in zip(ranges, F):
        fo = omlp.node_features(d, gam, mu, uh, n, s0, s1)
        for j in (0, 1, 3, 4, 5, 6):
            assert abs(f[j] - fo[j]) <= 1e-5 * (1 + abs(fo[j])), (s0, s1, j, f[j], fo[j])
        assert abs(f[2] - fo[2]) <= 0.0125 + 1e-5, (s0, s1, f[2], fo[2])   # half a bin


def test_node_features_reject_bad_ranges():
    t = tdeig()
    d = np.arange(4.0)
    g = np.full(4, 0.5)
    with t.Solver() as S:
        for bad in ([(0, 0)], [(2, 1)], [(0, 5)], [(-1, 2)]):
            with pytest.raises(t.TdeigError) as e:
                S.node_features(d, g, g, g, 4, bad)
            assert e.value.status == t.EINVAL


def _solve(S, a, b, flags=0, mode="adc2"):
    import torch
    lam, Q = S.solve(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), mode, flags=flags)
    torch.cuda.synchronize()
    return lam, Q, json.loads(S.stats())


def _merges(st):
    return [h for h in st.get("hss", []) if "K" in h]


def test_record_mode():
    t = tdeig()
    N = 4096
    a, b = inputs.toeplitz(N)
    with t.Solver(hss_threshold=1000, oversample=30, rank_cap=80) as S:
        _, _, st = _solve(S, a, b, flags=t.FLAG_RECORD)
        X, tt = S.rank_records()
        # a solve without the flag leaves no records
        _solve(S, a, b)
        X2, _ = S.rank_records()
    hm = _merges(st)
    assert hm and X2.shape[0] == 0
    nodes = sum((2 << h["L"]) - 2 for h in hm)
    assert 0 < X.shape[0] <= nodes
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(tt))
    smax = max(h["s"] for h in hm)
    assert np.all(tt >= 0) and np.all(np.exp(tt) - 1 <= smax + 1e-3)
    # features 5 and 6 identify the merge each node came from
    keys = np.array([((h["n"] - h["K"]) / h["n"], math.log2(h["K"])) for h in hm])
    for f in X:
        assert np.any((np.abs(keys[:, 0] - f[5]) <= 1e-6) & (np.abs(keys[:, 1] - f[6]) <= 1e-5))
    # leaf nodes have about K / 2^L rows
    assert np.all(X[:, 0] <= np.log2(max(h["K"] for h in hm)) + 1e-6)


def test_seed_requires_model():
    t = tdeig()
    a, b = inputs.toeplitz(512)
    with t.Solver() as S:
        with pytest.raises(t.TdeigError) as e:
            _solve(S, a, b, flags=t.FLAG_MLP_SEED)
        assert e.value.status == t.EINVAL


def _const_model(value):
    """A model whose output is the constant ln(value + 1) (rounded to BF16)."""
    p = np.zeros(omlp.NPARAM, np.float32)
    p[omlp.OFF_B3] = math.log(value + 1.0)
    return p, np.zeros(7, np.float32), np.ones(7, np.float32)


def test_fallback_reproduces_estimate():
    """A model that asks for rank 1 saturates every ID; each merge is then
    rebuilt with the rank estimate, bit for bit the estimator's solve."""
    t = tdeig()
    a, b = inputs.toeplitz(4096)
    with t.Solver(hss_threshold=1000) as S:
        lam0, Q0, st0 = _solve(S, a, b)
        S.set_rank_model(*_const_model(1.0))
        lam1, Q1, st1 = _solve(S, a, b, flags=t.FLAG_MLP_SEED)
    h0, h1 = _merges(st0), _merges(st1)
    assert len(h0) == len(h1) > 0
    assert all(h["seed"] == 2 for h in h1)
    assert st1["mlp_fallbacks"] == len(h1)
    assert [h["s"] for h in h0] == [h["s"] for h in h1]
    assert np.array_equal(lam0.cpu().numpy(), lam1.cpu().numpy())
    assert np.array_equal(Q0.cpu().numpy(), Q1.cpu().numpy())


def test_seed_above_estimate_is_kept():
    t = tdeig()
    N = 4096
    a, b = inputs.toeplitz(N)
    with t.Solver(hss_threshold=1000) as S:
        S.set_rank_model(*_const_model(90.0))
        lam, Q, st = _solve(S, a, b, flags=t.FLAG_MLP_SEED)
    hm = _merges(st)
    assert hm and all(h["seed"] == 1 and h["r"] == 90 for h in hm)
    lam, Q = lam.cpu().numpy(), Q.cpu().numpy()
    k = np.arange(1, N + 1)
    assert metrics.eig_error(lam, np.sort(2 + 2 * np.cos(k * np.pi / (N + 1)))) <= 1e-12
    assert metrics.orthogonality(Q) <= 1e-10
    assert metrics.residual(a, b, lam, Q) <= 1e-10


def _sampled_accuracy(a, b, lam, Q, k=1024, seed=0):
    """Orthogonality ||C^T C - I||_F / k and residual ||T C - C L||_F / (k ||T||)
    of k random columns C of Q (device arithmetic, FP64)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = Q.shape[1]
    idx = torch.randperm(N, generator=g)[:k].to(Q.device)
    C = Q[:, idx]
    I = torch.eye(C.shape[1], dtype=C.dtype, device=C.device)
    orth = ((C.T @ C - I).norm() / C.shape[1]).item()
    at = torch.from_numpy(a).to(Q.device)
    bt = torch.from_numpy(b).to(Q.device)
    TC = at[:, None] * C
    TC[:-1] += bt[:, None] * C[1:]
    TC[1:] += bt[:, None] * C[:-1]
    tn = max(np.abs(a).max() + 2 * np.abs(b).max(), 1e-300)
    res = ((TC - C * lam[idx][None, :]).norm() / (C.shape[1] * tn)).item()
    return orth, res


def _compare(S, a, b):
    """Estimate-seeded and model-seeded solves of one matrix."""
    import time
    import torch
    out = {}
    for name, fl in (("est", 0), ("mlp", tdeig().FLAG_MLP_SEED)):
        _solve(S, a, b, flags=fl)                          # warm
        t0 = time.time()
        lam, Q, st = _solve(S, a, b, flags=fl)
        dt = time.time() - t0
        hm = _merges(st)
        out[name] = dict(t=dt, lam=lam.cpu().numpy(), acc=_sampled_accuracy(a, b, lam, Q),
                         cols=sum(h["K"] * h["s"] for h in hm),
                         sat=sum(h["kmax"] >= h["s"] for h in hm), merges=len(hm),
                         fallbacks=st["mlp_fallbacks"], seeds=[h["seed"] for h in hm])
        del Q
        torch.cuda.empty_cache()
    return out["est"], out["mlp"]


def test_gain_random_class_n32768():
    """Few-deflation random tridiagonal, N = 32768 (held-out seed): deflation
    leaves K of a few hundred per merge, so HSS is enabled from K > 256.  The
    model samples far fewer columns than the estimate at the same accuracy."""
    t = tdeig()
    rm = rank_model()
    a, b = inputs.uniform(32768, 1001, lo_b=0.5, hi_b=1.0)
    with t.Solver(hss_threshold=256) as S:
        S.set_rank_model(*rm.load())
        est, mlp = _compare(S, a, b)
    print("random N=32768", {k: v for k, v in est.items() if k not in ("lam", "seeds")},
          {k: v for k, v in mlp.items() if k not in ("lam", "seeds")})
    assert est["merges"] == mlp["merges"] > 50
    assert all(s == 1 for s in mlp["seeds"]) and mlp["fallbacks"] == 0
    assert mlp["cols"] <= 0.7 * est["cols"]
    # eigenvalues depend on the update only through the z vectors of later merges
    assert metrics.eig_error(mlp["lam"], est["lam"]) <= 1e-12
    for acc in (est["acc"], mlp["acc"]):
        assert acc[0] <= 1e-10 and acc[1] <= 1e-10


def test_gain_toeplitz_saturation():
    """Toeplitz(2, 1), N = 16384, default options: the estimate lets IDs stop
    at the sample size on the largest merges; the model does not."""
    t = tdeig()
    rm = rank_model()
    a, b = inputs.toeplitz(16384)
    with t.Solver() as S:
        S.set_rank_model(*rm.load())
        est, mlp = _compare(S, a, b)
    print("toeplitz N=16384", {k: v for k, v in est.items() if k not in ("lam", "seeds")},
          {k: v for k, v in mlp.items() if k not in ("lam", "seeds")})
    assert mlp["sat"] <= est["sat"]
    k = np.arange(1, 16385)
    exact = np.sort(2 + 2 * np.cos(k * np.pi / 16385))
    assert metrics.eig_error(est["lam"], exact) <= 1e-12
    assert metrics.eig_error(mlp["lam"], exact) <= 1e-12
    for acc in (est["acc"], mlp["acc"]):
        assert acc[0] <= 1e-10 and acc[1] <= 1e-10
