"""Plain FP64 divide and conquer for T = tridiag(b, a, b) (Sec. 2, Algorithm 1).

Test infrastructure only (see the package docstring).

Steps, in the paper's order, for one merge (eq. T2, eq. T3):
  1. split T = diag(T1, T2) + b_k v v^T with T1 of size k = floor(n/2);
  2. solve T1, T2 recursively (QR below the leaf size);
  3. u = [last row of Q1, s * first row of Q2], M = D + rho u u^T;
  4. sort D1, D2 into d (stable, D1 first on ties) and deflate;
  5. secular roots lambda, gamma, mu (Theorem 1, Remark 1);
  6. Loewner recomputation of u (eq. ev_z);
  7. Cauchy-like eigenvector matrix (eq. Ev-Q) and the update
     diag(Q1, Q2) P Qhat, either dense (plain DC) or through an HSS
     approximation of Qhat (ADC1 / ADC2, Algorithms 2 and 3);
  8. merge the new and deflated eigenvalues ascending.

Readings of silent passages (all listed in the design notes as well):
  * split sign: rho = |b_k|, s = sign(b_k) (+1 for 0), a_k -= rho, a_{k+1} -= rho,
    v = e_k + s e_{k+1};
  * the whole problem is scaled by max(|a|, |b|) first and eigenvalues are
    scaled back at the end;
  * final order: stable sort of [new eigenvalues, deflated eigenvalues], so
    on ties the non-deflated come first.

Parity status: pinned (closed forms for Toeplitz and Clement matrices, brute
force Jacobi on small sizes, LAPACK via numpy, interlacing, orthogonality and
residual bounds; see tests/test_oracle_pins.py).
"""
import numpy as np

from .clib import lib, dptr, iptr

MODE_DENSE, MODE_ADC1, MODE_ADC2 = 0, 1, 2


def leaf_qr(a, b):
    n = len(a)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b if n > 1 else np.zeros(1), dtype=np.float64)
    lam = np.empty(n)
    Q = np.empty((n, n), order="F")
    rc = lib().orc_leaf_qr(n, dptr(a), dptr(b), dptr(lam), dptr(Q))
    if rc != 0:
        raise RuntimeError("oracle leaf QR did not converge (rc=%d)" % rc)
    return lam, Q


def deflate(d, z, rho, W, rotations=False):
    """In-place deflation (Sec. 4.3 reading in tdeig_oracle.c); returns the keep
    mask (bool), and with rotations=True also the rotation list in sweep order
    (j, i, c, s arrays).  W is Fortran-ordered."""
    n = len(d)
    keep = np.zeros(n, dtype=np.int32)
    assert W.flags["F_CONTIGUOUS"]
    rj = np.zeros(max(n, 1), dtype=np.int32)
    ri = np.zeros(max(n, 1), dtype=np.int32)
    rc = np.zeros(max(n, 1))
    rs = np.zeros(max(n, 1))
    nr = np.zeros(1, dtype=np.int32)
    K = lib().orc_deflate(n, dptr(d), dptr(z), float(rho), dptr(W), W.shape[0], W.shape[0],
                          iptr(keep), iptr(rj), iptr(ri), dptr(rc), dptr(rs), iptr(nr))
    assert K == int(keep.sum())
    if rotations:
        m = int(nr[0])
        return keep.astype(bool), (rj[:m].copy(), ri[:m].copy(), rc[:m].copy(), rs[:m].copy())
    return keep.astype(bool)


def sum_squares(z):
    """sum_i z_i^2 correctly rounded: each square split exactly into p + e
    (Dekker's product with Veltkamp's split), then math.fsum of all the parts.
    The norm that normalises u is then a function of u alone, whatever the
    summation order of an implementation."""
    import math
    z = np.asarray(z, dtype=np.float64)
    p = z * z
    sp = 134217729.0 * z                  # 2^27 + 1
    zh = sp - (sp - z)
    zl = z - zh
    e = ((zh * zh - p) + 2.0 * zh * zl) + zl * zl
    return math.fsum(np.concatenate([p, e]).tolist())


def merge_prep(lam1, Q1, lam2, Q2, beta, rotations=False):
    """Steps 3-4 of a merge (eq. T3, then the sort and the deflation of Sec. 4.3).

    Q1, Q2 may be full eigenvector matrices or just the rows the merge uses
    (Q1's last row and Q2's first row, given as 1 x n arrays); W is then built
    from identity blocks.  Returns a dict with perm (sorted position -> index
    into [lam1, lam2]), d and z after deflation, rho, keep (bool), W (the
    sorted, rotated diag(Q1, Q2)) and, with rotations=True, the rotation list.
    """
    n1, n2 = len(lam1), len(lam2)
    n = n1 + n2
    rho = abs(beta)
    s = -1.0 if beta < 0 else 1.0
    z = np.concatenate([Q1[-1, :], s * Q2[0, :]])
    dcat = np.concatenate([lam1, lam2])
    perm = np.argsort(dcat, kind="stable")
    d = np.ascontiguousarray(dcat[perm])
    z = np.ascontiguousarray(z[perm])
    W = np.zeros((n, n), order="F")
    W[:n1, :n1] = Q1 if Q1.shape[0] == n1 else np.eye(n1)
    W[n1:, n1:] = Q2 if Q2.shape[0] == n2 else np.eye(n2)
    W = np.asfortranarray(W[:, perm])
    nrm = np.sqrt(sum_squares(z))
    if nrm > 0:
        z /= nrm
        rho *= nrm * nrm
    out = {"perm": perm, "rho": rho, "W": W}
    if rotations:
        keep, rot = deflate(d, z, rho, W, rotations=True)
        out["rot"] = rot
    else:
        keep = deflate(d, z, rho, W)
    out.update(d=d, z=z, keep=keep)
    return out


def secular(d, z, rho, nthreads=None):
    import os
    K = len(d)
    d = np.ascontiguousarray(d, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    lam = np.empty(K); gam = np.empty(K); mu = np.empty(K)
    iters = np.empty(K, dtype=np.int32)
    nt = nthreads or (os.cpu_count() or 1)
    work = np.empty(2 * K * nt + 2)
    bad = lib().orc_secular_all(K, dptr(d), dptr(z), float(rho), dptr(lam), dptr(gam), dptr(mu),
                                iptr(iters), dptr(work), nt)
    if bad:
        raise RuntimeError("oracle secular solver hit its iteration cap on %d roots" % bad)
    return lam, gam, mu, iters


def lowner(d, gam, mu, rho, z):
    K = len(d)
    uhat = np.empty(K)
    lib().orc_lowner(K, dptr(d), dptr(gam), dptr(mu), float(rho), dptr(np.ascontiguousarray(z)),
                     dptr(uhat))
    return uhat


def cauchy(d, gam, mu, uhat):
    K = len(d)
    Qh = np.empty((K, K), order="F")
    v = np.empty(K)
    lib().orc_cauchy(K, dptr(d), dptr(gam), dptr(mu), dptr(uhat), dptr(v), dptr(Qh))
    return Qh, v


def cauchy_entries(rows, cols, gen):
    """Entries of the Cauchy-like matrix at global rows x cols (generators gen)."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty((len(rows), len(cols)), order="F")
    if len(rows) and len(cols):
        lib().orc_cauchy_entries(len(rows), iptr(rows), len(cols), iptr(cols), dptr(gen["d"]),
                                 dptr(gen["gamma"]), dptr(gen["mu"]), dptr(gen["uhat"]),
                                 dptr(gen["v"]), dptr(out))
    return out


def dminus_entries(rows, cols, gen):
    """d[rows] - lambda[cols] by Remark 1 (eq. d-lambda)."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty((len(rows), len(cols)), order="F")
    if len(rows) and len(cols):
        lib().orc_dminus_entries(len(rows), iptr(rows), len(cols), iptr(cols), dptr(gen["d"]),
                                 dptr(gen["gamma"]), dptr(gen["mu"]), dptr(out))
    return out


class Options:
    def __init__(self, leaf=32, mode=MODE_DENSE, hss_threshold=2000, hss_leaf=128, tol=1e-12,
                 oversample=10, rank_eps=1e-16, rank_cap=100, boundary_shift=5, seed=0):
        self.leaf = leaf
        self.mode = mode
        self.hss_threshold = hss_threshold
        self.hss_leaf = hss_leaf
        self.tol = tol
        self.oversample = oversample
        self.rank_eps = rank_eps
        self.rank_cap = rank_cap
        self.boundary_shift = boundary_shift
        self.seed = seed


def merge(lam1, Q1, lam2, Q2, beta, opt, merge_id=0, stats=None):
    """One merge of Algorithm 1: returns (lam, Q) of the n x n subproblem."""
    n = len(lam1) + len(lam2)
    pr = merge_prep(lam1, Q1, lam2, Q2, beta)
    d, z, rho, keep, W = pr["d"], pr["z"], pr["rho"], pr["keep"], pr["W"]
    K = int(keep.sum())
    rec = {"n": n, "K": K, "hss": False, "rank": 0, "node": merge_id}
    if K == 0:
        lam_new = np.empty(0)
        Qk = np.empty((n, 0), order="F")
    else:
        dk = np.ascontiguousarray(d[keep])
        zk = np.ascontiguousarray(z[keep])
        lam_new, gam, mu, _ = secular(dk, zk, rho)
        uhat = lowner(dk, gam, mu, rho, zk)
        X = np.asfortranarray(W[:, keep])
        if opt.mode in (MODE_ADC1, MODE_ADC2) and K > opt.hss_threshold:
            from . import hss
            gen = hss.generators(dk, gam, mu, uhat)
            H, info = hss.build(gen, opt, merge_id)
            Qk = hss.matmul_right(X, H)
            rec.update(hss=True, rank=info["rank"], max_block_rank=info["max_block_rank"],
                       bounds=info["bounds"], node_ranks=info["node_ranks"])
        else:
            Qh, _ = cauchy(dk, gam, mu, uhat)
            Qk = X @ Qh
    vals = np.concatenate([lam_new, d[~keep]])
    cols = np.concatenate([Qk, W[:, ~keep]], axis=1)
    order = np.argsort(vals, kind="stable")
    if stats is not None:
        stats.append(rec)
    return vals[order], np.asfortranarray(cols[:, order])


def _dc(a, b, opt, node_id, stats):
    n = len(a)
    if n <= opt.leaf:
        return leaf_qr(a, b)
    k = n // 2
    beta = b[k - 1]
    rho = abs(beta)
    a1 = a[:k].copy(); a1[k - 1] -= rho
    a2 = a[k:].copy(); a2[0] -= rho
    lam1, Q1 = _dc(a1, b[:k - 1], opt, 2 * node_id + 1, stats)
    lam2, Q2 = _dc(a2, b[k:], opt, 2 * node_id + 2, stats)
    return merge(lam1, Q1, lam2, Q2, beta, opt, merge_id=node_id, stats=stats)


def solve(a, b, opt=None, stats=None):
    """Eigendecomposition of the symmetric tridiagonal (a: diagonal, b: off-diagonal).

    Returns (lam ascending, Q column-major n x n with Q[:, j] the eigenvector of lam[j]).
    """
    opt = opt or Options()
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = len(a)
    if n == 0:
        return np.empty(0), np.empty((0, 0), order="F")
    if not (np.all(np.isfinite(a)) and np.all(np.isfinite(b))):
        raise ValueError("non-finite input")
    scale = max(np.max(np.abs(a)), np.max(np.abs(b)) if n > 1 else 0.0)
    if scale == 0.0:
        return np.zeros(n), np.asfortranarray(np.eye(n))
    lam, Q = _dc(a / scale, b / scale, opt, 0, stats)
    return lam * scale, Q
