"""HSS pieces of the ADC eigensolver, plain FP64 numpy.

Test infrastructure only (see the package docstring).

  rank_formula      eq. (bounds): r = ceil(ln(16/eps) ln(8R) / pi^2)      [pinned: worked example]
  rank_estimate     Sec. 4.1: max over neighbouring leaf segments, boundary
                    moves of <= 5 rows when dist < 1e-10, cap 100         [pinned: worked example,
                                                                           Table 1 trend]
  philox_gaussian   Gaussian test matrix Omega (Sec. 3) from Philox4x32-10
                    (Salmon et al., SC'11) + Box-Muller                    [pinned: published
                                                                           known-answer vectors]
  interp_decomp     ID by column-pivoted QR of Phi^T (Sec. 3)             [pinned: exact on
                                                                           low-rank matrices]
  rshss             Algorithm 2 (random HSS construction, Cauchy-like)   [pinned: densify vs Qhat]
  srrsc             ADC1 compression (structured rank-revealing Schur
                    complements on the Cauchy generators)                 [pinned: densify vs Qhat,
                                                                           ranks <= RSHSS ranks]
  matmul_right      Algorithm 3 (X * H)                                   [pinned: X * densify(H)]
  densify           eq. (new-hss) recursively                             [pinned: block identities]

Readings of garbled or silent passages:
  * eq. (dist_xy): dist(I_s, I_{s+1}) is taken over d in the left segment and
    lambda in the right segment only (the printed assumption d_i < lambda_j);
    it is lambda_b - d_{b-1} = (d_b - d_{b-1}) + gamma_b at boundary b.  With
    Example 1 (spacing 0.004) this gives the printed 4.3e-3 at m = 300.
  * logarithms in eq. (bounds) are natural (the worked example needs it).
  * a boundary with dist < 1e-10 moves by up to +-5 rows to the position of
    largest dist; the moved boundary defines the HSS leaf partition.
  * ID truncation is relative: k = first index with |R_kk| <= tol |R_00|.
  * Algorithm 3 downsweep: [F_i1, F_i2] = F_i V_i^T is a horizontal split (by
    the children's column ranks); leaves also add their sibling term G_j B_j.
  * SRRSC (not specified in the paper): Gaussian elimination with complete
    pivoting on the generator form of each HSS block row (and column), where
    every Schur complement is again Cauchy-like with updated generators;
    stop when |pivot| <= tol |first pivot|; the pivot rows are the skeleton
    and U = C[:, piv_cols] C[piv_rows, piv_cols]^{-1}; parents compress the
    stacked skeleton rows of their children (nested bases).
"""
import math

import numpy as np
import scipy.linalg as sla

from .dc import cauchy_entries, cauchy, dminus_entries

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


# ----------------------------------------------------------------------------
# Off-diagonal rank estimate (Sec. 2.1 eq. bounds; Sec. 4.1 rules (1), (2))
# ----------------------------------------------------------------------------
def rank_formula(R, eps):
    """r = ceil(ln(16/eps) * ln(8 R) / pi^2), eq. (bounds)."""
    return int(math.ceil(math.log(16.0 / eps) * math.log(8.0 * R) / (math.pi ** 2)))


def leaf_bounds(K, m):
    """Equal split of [0, K) into 2^L leaves, L = max(1, round(log2(K/m)))."""
    L = max(1, int(round(math.log2(max(K, 1) / m)))) if K >= 2 * m else (1 if K >= 2 else 0)
    nl = 1 << L
    return np.array([(p * K) // nl for p in range(nl + 1)], dtype=np.int64), L


def boundary_dist(gen, b):
    d, gam = gen["d"], gen["gamma"]
    return (d[b] - d[b - 1]) + gam[b]


def rank_estimate(gen, bounds, eps=1e-16, cap=100, shift=5, small=1e-10):
    """Returns (r, bounds') following Sec. 4.1."""
    d, lam = gen["d"], gen["lam"]
    bounds = bounds.copy()
    span = lam[-1] - d[0]
    r = 1
    for s in range(1, len(bounds) - 1):
        b = int(bounds[s])
        dist = boundary_dist(gen, b)
        if dist < small:
            best_b, best = b, dist
            lo = int(bounds[s - 1]) + 1
            hi = int(bounds[s + 1]) - 1
            for t in range(1, shift + 1):
                for cand in (b - t, b + t):
                    if lo <= cand <= hi:
                        dc_ = boundary_dist(gen, cand)
                        if dc_ > best:
                            best_b, best = cand, dc_
            bounds[s] = best_b
            dist = best
        R = span / dist if dist > 0 else float("inf")
        rb = cap if not np.isfinite(R) else rank_formula(R, eps)
        r = max(r, rb)
    return min(r, cap), bounds


# ----------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Gaussian matrix.
# ----------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """ctr: (..., 4) uint64 array holding 32-bit words; key: (k0, k1)."""
    c = [ctr[..., i].astype(np.uint64) & _MASK for i in range(4)]
    k0 = np.uint64(key[0] & _MASK)
    k1 = np.uint64(key[1] & _MASK)
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c = [(hi1 ^ c[1] ^ k0) & np.uint64(_MASK), lo1, (hi0 ^ c[3] ^ k1) & np.uint64(_MASK), lo0]
        k0 = (k0 + np.uint64(PHILOX_W0)) & np.uint64(_MASK)
        k1 = (k1 + np.uint64(PHILOX_W1)) & np.uint64(_MASK)
    return np.stack(c, axis=-1)


def philox_gaussian(nrow, ncol, seed, stream):
    """Omega[i, j] ~ N(0, 1): counter (i, j, stream, 0), key (seed lo, seed hi);
    Box-Muller on the first two words, u = (x + 0.5) 2^-32."""
    i = np.arange(nrow, dtype=np.uint64)[:, None] * np.ones((1, ncol), dtype=np.uint64)
    j = np.ones((nrow, 1), dtype=np.uint64) * np.arange(ncol, dtype=np.uint64)[None, :]
    ctr = np.stack([i, j, np.full_like(i, stream & _MASK), np.zeros_like(i)], axis=-1)
    out = philox4x32_10(ctr, (seed & _MASK, (seed >> 32) & _MASK))
    u1 = (out[..., 0].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (out[..., 1].astype(np.float64) + 0.5) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------
# Generators and the HSS container
# ----------------------------------------------------------------------------
def generators(d, gamma, mu, uhat):
    """Cauchy-like generators (eq. cauchylike): d, lambda (as d + gamma), uhat, v."""
    K = len(d)
    Qh, v = cauchy(d, gamma, mu, uhat)
    return {"d": d, "gamma": gamma, "mu": mu, "uhat": uhat, "v": v, "lam": d + gamma, "K": K,
            "_dense": Qh}


class HSS:
    """Full binary HSS tree with leaves at level L, nodes (level, pos)."""

    def __init__(self, bounds, L):
        self.bounds = np.asarray(bounds, dtype=np.int64)
        self.L = L
        self.D, self.U, self.V, self.B = {}, {}, {}, {}
        self.I, self.J = {}, {}

    def span(self, l, p):
        w = 1 << (self.L - l)
        return int(self.bounds[p * w]), int(self.bounds[(p + 1) * w])

    def ranks(self):
        return [u.shape[1] for u in self.U.values()] + [v.shape[1] for v in self.V.values()]


def interp_decomp(Phi, tol):
    """Row ID Phi ~= U Phi[I, :] with U[I] = identity (Sec. 3, ID by pivoted QR of Phi^T)."""
    m = Phi.shape[0]
    if m == 0 or Phi.shape[1] == 0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    _, R, P = sla.qr(Phi.T, mode="economic", pivoting=True)
    dg = np.abs(np.diag(R))
    if dg[0] == 0.0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    k = len(dg)
    for t in range(len(dg)):
        if dg[t] <= tol * dg[0]:
            k = t
            break
    T = sla.solve_triangular(R[:k, :k], R[:k, k:]) if k < m else np.zeros((k, 0))
    U = np.zeros((m, k))
    U[P[:k], :] = np.eye(k)
    U[P[k:], :] = T.T
    return U, P[:k].astype(np.int64)


def rshss(gen, bounds, L, r, p, Omega, tol):
    """Algorithm 2 with Omega(1) = Omega(2) = Omega (K x (r+p))."""
    A = gen["_dense"]
    Y = A @ Omega
    Z = A.T @ Omega
    H = HSS(bounds, L)
    Phi, Theta, Yh, Zh = {}, {}, {}, {}
    for l in range(L, 0, -1):
        for q in range(1 << l):
            if l == L:
                s, e = H.span(l, q)
                idx = np.arange(s, e)
                Dq = cauchy_entries(idx, idx, gen)
                H.D[q] = Dq
                Ph = Y[s:e] - Dq @ Omega[s:e]
                Th = Z[s:e] - Dq.T @ Omega[s:e]
                U, Iloc = interp_decomp(Ph, tol)
                V, Jloc = interp_decomp(Th, tol)
                H.I[(l, q)] = idx[Iloc]
                H.J[(l, q)] = idx[Jloc]
                Phi[(l, q)] = Ph[Iloc]
                Theta[(l, q)] = Th[Jloc]
                Yh[(l, q)] = V.T @ Omega[s:e]
                Zh[(l, q)] = U.T @ Omega[s:e]
            else:
                c1, c2 = (l + 1, 2 * q), (l + 1, 2 * q + 1)
                B1 = cauchy_entries(H.I[c1], H.J[c2], gen)
                B2 = cauchy_entries(H.I[c2], H.J[c1], gen)
                H.B[c1], H.B[c2] = B1, B2
                Ph = np.vstack([Phi[c1] - B1 @ Yh[c2], Phi[c2] - B2 @ Yh[c1]])
                Th = np.vstack([Theta[c1] - B2.T @ Zh[c2], Theta[c2] - B1.T @ Zh[c1]])
                rows = np.concatenate([H.I[c1], H.I[c2]])
                cols = np.concatenate([H.J[c1], H.J[c2]])
                U, Iloc = interp_decomp(Ph, tol)
                V, Jloc = interp_decomp(Th, tol)
                H.I[(l, q)] = rows[Iloc]
                H.J[(l, q)] = cols[Jloc]
                Phi[(l, q)] = Ph[Iloc]
                Theta[(l, q)] = Th[Jloc]
                Yh[(l, q)] = V.T @ np.vstack([Yh[c1], Yh[c2]])
                Zh[(l, q)] = U.T @ np.vstack([Zh[c1], Zh[c2]])
            H.U[(l, q)] = U
            H.V[(l, q)] = V
    # root: couple its two children
    c1, c2 = (1, 0), (1, 1)
    H.B[c1] = cauchy_entries(H.I[c1], H.J[c2], gen)
    H.B[c2] = cauchy_entries(H.I[c2], H.J[c1], gen)
    return H


def _skeleton_rows(rows, cols, gen, tol, transpose=False):
    """Complete-pivoting GE on the generator form of C = A[rows, cols] (or of
    A[cols, rows]^T when transpose): returns (U, local pivot rows) with
    C ~= U C[piv, :], U = C[:, pc] C[piv, pc]^{-1}."""
    if transpose:
        # C[a, b] = A[cols[b], rows[a]] = v[rows[a]] uhat[cols[b]] / (d[cols[b]] - lam[rows[a]])
        C = cauchy_entries(cols, rows, gen).T
        g = gen["v"][rows].copy()
        h = gen["uhat"][cols].copy()
        DIFF = dminus_entries(cols, rows, gen).T
    else:
        C = cauchy_entries(rows, cols, gen)
        g = gen["uhat"][rows].copy()
        h = gen["v"][cols].copy()
        DIFF = dminus_entries(rows, cols, gen)
    m, n = C.shape
    ar = np.ones(m, dtype=bool)
    ac = np.ones(n, dtype=bool)
    pr, pc = [], []
    first = None
    for _ in range(min(m, n)):
        S = (g[:, None] * h[None, :]) / DIFF
        S[~ar, :] = 0.0
        S[:, ~ac] = 0.0
        flat = int(np.argmax(np.abs(S)))
        a, b = divmod(flat, n)
        piv = S[a, b]
        if first is None:
            first = abs(piv)
            if first == 0.0:
                break
        if abs(piv) <= tol * first:
            break
        col = S[:, b].copy()
        row = S[a, :].copy()
        ga, hb = g[a], h[b]
        g = g - col * (ga / piv)
        h = h - row * (hb / piv)
        ar[a] = False
        ac[b] = False
        pr.append(a)
        pc.append(b)
    k = len(pr)
    if k == 0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    pr = np.array(pr)
    pc = np.array(pc)
    U = np.linalg.solve(C[np.ix_(pr, pc)].T, C[:, pc].T).T
    U[pr, :] = np.eye(k)
    return U, pr.astype(np.int64)


def srrsc(gen, bounds, L, tol):
    """ADC1 HSS construction by structured rank-revealing Schur complements."""
    K = gen["K"]
    H = HSS(bounds, L)
    allidx = np.arange(K)
    for l in range(L, 0, -1):
        for q in range(1 << l):
            s, e = H.span(l, q)
            outside = np.concatenate([allidx[:s], allidx[e:]])
            if l == L:
                idx = np.arange(s, e)
                H.D[q] = cauchy_entries(idx, idx, gen)
                rows, cols = idx, idx
            else:
                c1, c2 = (l + 1, 2 * q), (l + 1, 2 * q + 1)
                rows = np.concatenate([H.I[c1], H.I[c2]])
                cols = np.concatenate([H.J[c1], H.J[c2]])
                H.B[c1] = cauchy_entries(H.I[c1], H.J[c2], gen)
                H.B[c2] = cauchy_entries(H.I[c2], H.J[c1], gen)
            U, Iloc = _skeleton_rows(rows, outside, gen, tol)
            V, Jloc = _skeleton_rows(cols, outside, gen, tol, transpose=True)
            H.U[(l, q)] = U
            H.V[(l, q)] = V
            H.I[(l, q)] = rows[Iloc]
            H.J[(l, q)] = cols[Jloc]
    c1, c2 = (1, 0), (1, 1)
    H.B[c1] = cauchy_entries(H.I[c1], H.J[c2], gen)
    H.B[c2] = cauchy_entries(H.I[c2], H.J[c1], gen)
    return H


def build(gen, opt, merge_id):
    """HSS approximation of the Cauchy-like matrix for one merge (Algorithm 1, else-branch)."""
    K = gen["K"]
    bounds, L = leaf_bounds(K, opt.hss_leaf)
    info = {}
    if opt.mode == 2:
        r, bounds = rank_estimate(gen, bounds, opt.rank_eps, opt.rank_cap, opt.boundary_shift)
        Omega = philox_gaussian(K, r + opt.oversample, opt.seed, merge_id)
        H = rshss(gen, bounds, L, r, opt.oversample, Omega, opt.tol)
        info["rank"] = r
    else:
        H = srrsc(gen, bounds, L, opt.tol)
        info["rank"] = max(H.ranks()) if H.ranks() else 0
    info["max_block_rank"] = max(H.ranks()) if H.ranks() else 0
    # the (possibly moved) leaf boundaries and every node's (row, column) ID
    # ranks, levels 1..L, left to right
    info["bounds"] = [int(x) for x in H.bounds]
    info["node_ranks"] = [(H.U[(l, q)].shape[1], H.V[(l, q)].shape[1])
                          for l in range(1, H.L + 1) for q in range(1 << l)]
    return H, info


# ----------------------------------------------------------------------------
# Algorithm 3 and densification
# ----------------------------------------------------------------------------
def matmul_right(X, H):
    """X (P x K) times the HSS matrix H, Algorithm 3."""
    L = H.L
    out = np.empty_like(X)
    if L == 0:
        return X @ H.D[0]
    G = {}
    for q in range(1 << L):
        s, e = H.span(L, q)
        G[(L, q)] = X[:, s:e] @ H.U[(L, q)]
    for l in range(L - 1, 0, -1):
        for q in range(1 << l):
            G[(l, q)] = np.hstack([G[(l + 1, 2 * q)], G[(l + 1, 2 * q + 1)]]) @ H.U[(l, q)]
    Fin = {}
    for l in range(1, L + 1):
        for q in range(1 << l):
            sib = (l, q ^ 1)
            F = G[sib] @ H.B[sib]
            if l > 1:
                F = F + Fin[(l, q)]
            if l < L:
                FV = F @ H.V[(l, q)].T
                k1 = H.V[(l + 1, 2 * q)].shape[1]
                Fin[(l + 1, 2 * q)] = FV[:, :k1]
                Fin[(l + 1, 2 * q + 1)] = FV[:, k1:]
            else:
                s, e = H.span(L, q)
                out[:, s:e] = X[:, s:e] @ H.D[q] + F @ H.V[(L, q)].T
    return out


def densify(H):
    """Dense matrix of H by eq. (new-hss)."""
    L = H.L
    K = int(H.bounds[-1])
    if L == 0:
        return H.D[0].copy()
    Uh, Vh, Dh = {}, {}, {}
    for q in range(1 << L):
        Uh[(L, q)] = H.U[(L, q)]
        Vh[(L, q)] = H.V[(L, q)]
        Dh[(L, q)] = H.D[q]
    for l in range(L - 1, -1, -1):
        for q in range(1 << l):
            c1, c2 = (l + 1, 2 * q), (l + 1, 2 * q + 1)
            top = np.hstack([Dh[c1], Uh[c1] @ H.B[c1] @ Vh[c2].T])
            bot = np.hstack([Uh[c2] @ H.B[c2] @ Vh[c1].T, Dh[c2]])
            Dh[(l, q)] = np.vstack([top, bot])
            if l > 0:
                Uh[(l, q)] = sla.block_diag(Uh[c1], Uh[c2]) @ H.U[(l, q)]
                Vh[(l, q)] = sla.block_diag(Vh[c1], Vh[c2]) @ H.V[(l, q)]
    A = Dh[(0, 0)]
    assert A.shape == (K, K)
    return A
