"""Accuracy measures of Sec. 5, Example 3, in the forms used by the tests.

Test infrastructure only (see the package docstring).

  orthogonality  ||Q^T Q - I||_F / N
  residual       ||T Q - Q Lambda||_F / (N ||T||_2),  ||T||_2 = max |lambda|
  eigenvalue     max_i |lam_i - ref_i| / max(|ref_i|, ||T||_2)  (normwise for tiny lambda)

These are plain definitions; a library matmul is the only step used.
"""
import numpy as np


def tridiag_apply(a, b, Q):
    """T @ Q for T = tridiag(b, a, b) without forming T."""
    out = a[:, None] * Q
    if len(a) > 1:
        out[:-1] += b[:, None] * Q[1:]
        out[1:] += b[:, None] * Q[:-1]
    return out


def orthogonality(Q):
    n = Q.shape[0]
    if n == 0:
        return 0.0
    G = Q.T @ Q
    G[np.diag_indices(n)] -= 1.0
    return float(np.linalg.norm(G) / n)


def residual(a, b, lam, Q):
    n = len(a)
    if n == 0:
        return 0.0
    R = tridiag_apply(np.asarray(a), np.asarray(b), Q) - Q * lam[None, :]
    tn = max(float(np.max(np.abs(lam))), 1e-300)
    return float(np.linalg.norm(R) / (n * tn))


def eig_error(lam, ref):
    if len(ref) == 0:
        return 0.0
    tn = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(lam - ref) / np.maximum(np.abs(ref), tn)))


def vectors_match(Q, Qref, lam_ref, gap_rel=1e-8):
    """Max column difference up to sign, over eigenvalues with a relative gap >= gap_rel.

    Columns of clustered eigenvalues are not unique; they are skipped (the
    orthogonality and residual checks cover them)."""
    n = len(lam_ref)
    if n == 0:
        return 0.0, 0
    tn = max(float(np.max(np.abs(lam_ref))), 1e-300)
    gaps = np.full(n, np.inf)
    if n > 1:
        dl = np.diff(lam_ref)
        gaps[:-1] = np.minimum(gaps[:-1], dl)
        gaps[1:] = np.minimum(gaps[1:], dl)
    sel = np.nonzero(gaps >= gap_rel * tn)[0]
    if len(sel) == 0:
        return 0.0, 0
    A = Q[:, sel]
    B = Qref[:, sel]
    idx = np.argmax(np.abs(B), axis=0)
    sg = np.sign(A[idx, np.arange(len(sel))] * B[idx, np.arange(len(sel))])
    sg[sg == 0] = 1.0
    return float(np.max(np.abs(A * sg[None, :] - B))), len(sel)
