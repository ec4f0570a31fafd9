"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form, a
brute-force algorithm written in this file, a library routine the oracle does
not call, an invariant, or a number printed in the paper (tests/golden).
"""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import dc, hss, metrics
from paper_1510_04591_gb300 import inputs


def dense_T(a, b):
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def jacobi_eig(A, sweeps=60):
    """Cyclic Jacobi (brute force, for n <= 16): independent of the oracle."""
    A = A.copy()
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= 1e-300:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                th = (A[q, q] - A[p, p]) / (2 * A[p, q])
                t = np.sign(th) / (abs(th) + math.sqrt(th * th + 1)) if th != 0 else 1.0
                c = 1 / math.sqrt(t * t + 1)
                s = t * c
                J = np.eye(n)
                J[p, p] = J[q, q] = c
                J[p, q] = s
                J[q, p] = -s
                A = J.T @ A @ J
                V = V @ J
    w = np.diag(A)
    o = np.argsort(w)
    return w[o], V[:, o]


# --------------------------------------------------------------------------
# Whole solver
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 7, 32, 33, 100, 513, 1024])
def test_toeplitz_closed_form(N):
    """Sec. 5 Toeplitz(2,1): lambda_k = 2 + 2 cos(k pi/(N+1)), q_jk = sqrt(2/(N+1)) sin(jk pi/(N+1))."""
    a, b = inputs.toeplitz(N, 2.0, 1.0)
    lam, Q = dc.solve(a, b)
    k = np.arange(1, N + 1)
    ex = 2 + 2 * np.cos(k * np.pi / (N + 1))
    o = np.argsort(ex)
    ex = ex[o]
    V = np.sqrt(2.0 / (N + 1)) * np.sin(np.outer(k, k) * np.pi / (N + 1))[:, o]
    assert metrics.eig_error(lam, ex) <= 1e-13
    err, cnt = metrics.vectors_match(Q, V, ex, gap_rel=0.0)
    assert cnt == N and err <= 1e-9
    assert metrics.orthogonality(Q) <= 1e-13
    assert metrics.residual(a, b, lam, Q) <= 1e-13


@pytest.mark.parametrize("n1", [2, 5, 40, 101])
def test_clement_closed_form(n1):
    """Clement matrix of dimension n+1 (eq. Clement-Tri): eigenvalues -n, -n+2, ..., n."""
    a, b = inputs.clement(n1)
    n = n1 - 1
    lam, Q = dc.solve(a, b, dc.Options(leaf=8))
    ex = np.arange(-n, n + 1, 2, dtype=np.float64)
    assert metrics.eig_error(lam, ex) <= 1e-13
    assert metrics.orthogonality(Q) <= 1e-13


@pytest.mark.parametrize("N,seed", [(4, 0), (9, 1), (16, 2)])
def test_jacobi_brute_force(N, seed):
    a, b = inputs.uniform(N, seed)
    w, V = jacobi_eig(dense_T(a, b))
    lam, Q = dc.solve(a, b, dc.Options(leaf=2))
    assert metrics.eig_error(lam, w) <= 1e-13
    err, _ = metrics.vectors_match(Q, V, w)
    assert err <= 1e-10


@pytest.mark.parametrize("N,seed,leaf", [(200, 3, 8), (1000, 4, 32), (777, 5, 25)])
def test_lapack_cross_check(N, seed, leaf):
    """numpy.linalg.eigh (LAPACK) on the dense matrix; the oracle never calls it."""
    a, b = inputs.uniform(N, seed)
    w, V = np.linalg.eigh(dense_T(a, b))
    lam, Q = dc.solve(a, b, dc.Options(leaf=leaf))
    assert metrics.eig_error(lam, w) <= 1e-13
    assert metrics.orthogonality(Q) <= 1e-13
    assert metrics.residual(a, b, lam, Q) <= 1e-13
    err, cnt = metrics.vectors_match(Q, V, w, gap_rel=1e-6)
    assert cnt > N // 2 and err <= 1e-8


def test_heavy_deflation_glued_wilkinson():
    a, b = inputs.glued_wilkinson(300)
    st = []
    lam, Q = dc.solve(a, b, dc.Options(leaf=16), st)
    w = np.linalg.eigvalsh(dense_T(a, b))
    assert metrics.eig_error(lam, w) <= 1e-13
    assert metrics.orthogonality(Q) <= 1e-13
    assert metrics.residual(a, b, lam, Q) <= 1e-13
    assert any(s["K"] < s["n"] for s in st)


def test_zero_offdiagonal_and_scaling():
    a = np.array([3.0, -1.0, 2.0, 2.0, 0.5] * 10)
    b = np.zeros(len(a) - 1)
    lam, Q = dc.solve(a, b, dc.Options(leaf=4))
    assert np.allclose(lam, np.sort(a), atol=0, rtol=0)
    assert metrics.orthogonality(Q) <= 1e-15
    a, b = inputs.uniform(120, 9)
    lam1, _ = dc.solve(a * 1e200, b * 1e200, dc.Options(leaf=8))
    lam2, _ = dc.solve(a, b, dc.Options(leaf=8))
    assert np.max(np.abs(lam1 / 1e200 - lam2)) <= 1e-14


# --------------------------------------------------------------------------
# Secular equation, Loewner, Cauchy-like matrix
# --------------------------------------------------------------------------
def rank_one_problem(K, seed, rho=1.0):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(-1, 1, K))
    z = rng.standard_normal(K)
    z /= np.linalg.norm(z)
    return d, z, rho


@pytest.mark.parametrize("K,seed,rho", [(2, 0, 1.0), (3, 1, 0.3), (50, 2, 2.0), (400, 3, 1.0)])
def test_secular_interlacing_and_residual(K, seed, rho):
    """Theorem 1: d_i < lambda_i < d_{i+1}; gamma, mu > 0; lambda matches LAPACK on D + rho z z^T."""
    d, z, rho = rank_one_problem(K, seed, rho)
    lam, gam, mu, it = dc.secular(d, z, rho)
    assert np.all(gam > 0)
    assert np.all(mu[:-1] > 0)
    assert np.all(lam[:-1] > d[:-1]) and np.all(lam[:-1] < d[1:]) and lam[-1] > d[-1]
    assert np.allclose(lam - d, gam, rtol=1e-12, atol=1e-15)
    assert np.allclose(d[1:] - lam[:-1], mu[:-1], rtol=1e-12, atol=1e-15)
    w = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(z, z))
    assert np.max(np.abs(w - lam)) <= 1e-14 * max(1.0, rho)
    assert lam[-1] <= d[-1] + rho * np.dot(z, z) * (1 + 1e-15)


def test_secular_closed_forms():
    # K = 1: lambda = d + rho z^2
    lam, gam, mu, _ = dc.secular(np.array([0.25]), np.array([1.0]), 0.5)
    assert lam[0] == 0.75 and gam[0] == 0.5
    # K = 2: roots of (d1 - x)(d2 - x) + rho z1^2 (d2 - x) + rho z2^2 (d1 - x) = 0
    d = np.array([-0.5, 0.25]); z = np.array([0.6, 0.8]); rho = 1.3
    lam, gam, mu, _ = dc.secular(d, z, rho)
    B = -(d[0] + d[1] + rho * (z[0] ** 2 + z[1] ** 2))
    C = d[0] * d[1] + rho * z[0] ** 2 * d[1] + rho * z[1] ** 2 * d[0]
    r = np.sort(np.roots([1.0, B, C]).real)
    assert np.max(np.abs(lam - r)) <= 4e-16


def test_secular_tiny_weight_and_clustered_poles():
    d = np.array([0.0, 1e-9, 2e-9, 0.5, 0.5 + 1e-12, 1.0])
    z = np.array([1e-7, 0.5, 0.5, 0.5, 0.4, 1e-6])
    z /= np.linalg.norm(z)
    lam, gam, mu, it = dc.secular(d, z, 1.0)
    assert np.all(gam > 0) and np.all(mu[:-1] > 0)
    w = np.linalg.eigvalsh(np.diag(d) + np.outer(z, z))
    assert np.max(np.abs(w - lam)) <= 1e-15
    assert it.max() < 60


@pytest.mark.parametrize("K,seed", [(10, 4), (300, 5)])
def test_lowner_and_cauchy(K, seed):
    """eq. ev_z: lambda are exact eigenvalues of D + rho uhat uhat^T and uhat ~ z;
    eq. Ev-Q: Qhat is orthogonal and diagonalises D + rho uhat uhat^T."""
    d, z, rho = rank_one_problem(K, seed, 1.7)
    lam, gam, mu, _ = dc.secular(d, z, rho)
    uh = dc.lowner(d, gam, mu, rho, z)
    assert np.max(np.abs(uh - z)) <= 1e-13
    assert np.all(np.sign(uh) == np.sign(z))
    M = np.diag(d) + rho * np.outer(uh, uh)
    assert np.max(np.abs(np.linalg.eigvalsh(M) - lam)) <= 1e-14
    Qh, v = dc.cauchy(d, gam, mu, uh)
    assert metrics.orthogonality(Qh) <= 1e-15
    R = M @ Qh - Qh * lam[None, :]
    assert np.max(np.abs(R)) <= 1e-13
    # displacement D Qhat - Qhat Lambda = uhat v^T (eq. cauchylike), with lambda = d + gamma
    disp = d[:, None] * Qh - Qh * lam[None, :]
    assert np.max(np.abs(disp - np.outer(uh, v))) <= 1e-13


def test_deflation_types():
    """Both deflation types: tiny z_i and (near-)equal d; deflated pairs are eigenpairs."""
    n = 12
    rng = np.random.default_rng(7)
    d = np.sort(rng.uniform(-1, 1, n))
    d[5] = d[4]            # exact tie -> rotation
    d[9] = d[8] + 1e-17    # near tie
    z = rng.standard_normal(n)
    z[2] = 1e-20           # tiny weight
    z /= np.linalg.norm(z)
    rho = 1.0
    M = np.diag(d) + rho * np.outer(z, z)
    W = np.asfortranarray(np.eye(n))
    dd, zz = d.copy(), z.copy()
    keep = dc.deflate(dd, zz, rho, W)
    assert not keep[2] and not keep[4] and not keep[8]
    for i in np.nonzero(~keep)[0]:
        q = W[:, i]
        assert np.linalg.norm(M @ q - dd[i] * q) <= 1e-14
    assert metrics.orthogonality(W) <= 1e-15
    assert np.all(np.diff(dd[keep]) > 0)


def test_sum_squares_is_correctly_rounded():
    """The norm of the merge vector: sum z_i^2 correctly rounded (exact rational
    sum, then one rounding), whatever the order of the terms."""
    from fractions import Fraction
    rng = np.random.default_rng(12)
    for n in (1, 2, 7, 1000):
        z = rng.standard_normal(n) * np.exp(rng.uniform(-20, 5, n))
        exact = float(sum(Fraction(float(x)) ** 2 for x in z))
        assert dc.sum_squares(z) == exact
        assert dc.sum_squares(z[::-1]) == exact


def test_deflation_rotation_record():
    """The recorded rotation list (sweep order) reproduces the rotated columns:
    applying each (j, i, c, s) to the identity in order gives W; i ascends, j < i,
    and every rotated j ends deflated with z_j = 0 (Sec. 4.3 reading)."""
    n = 40
    rng = np.random.default_rng(11)
    d = np.sort(rng.uniform(-1, 1, n))
    for k in (3, 10, 11, 25):
        d[k + 1] = d[k]          # exact ties: rotations, one of them chained (10, 11, 12)
    z = rng.standard_normal(n)
    z[30] = 1e-19                # tiny weight: deflates without a rotation
    z /= np.linalg.norm(z)
    W = np.asfortranarray(np.eye(n))
    dd, zz = d.copy(), z.copy()
    keep, (rj, ri, rc, rs) = dc.deflate(dd, zz, 1.3, W, rotations=True)
    assert len(rj) >= 4 and not keep[30]
    assert np.all(rj < ri) and np.all(np.diff(ri) > 0)
    assert any(rj[t + 1] == ri[t] for t in range(len(rj) - 1))   # a chain
    V = np.eye(n)
    for j, i, c, s in zip(rj, ri, rc, rs):
        qj, qi = V[:, j].copy(), V[:, i].copy()
        V[:, j] = c * qj - s * qi
        V[:, i] = s * qj + c * qi
        assert np.isclose(c * c + s * s, 1.0, rtol=0, atol=4e-16)
    assert np.array_equal(V, W)
    assert np.all(zz[rj] == 0.0) and not np.any(keep[rj])
    pr = dc.merge_prep(d[:20], np.eye(20), d[20:], np.eye(20), -0.5, rotations=True)
    assert np.array_equal(pr["perm"], np.argsort(d, kind="stable"))
    assert abs(pr["rho"] - 1.0) <= 4e-16   # |b| times |u|^2 = 2 (two unit rows)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (17, 2), (32, 3)])
def test_leaf_qr(n, seed):
    a, b = inputs.uniform(n, seed)
    lam, Q = dc.leaf_qr(a, b)
    w = np.linalg.eigvalsh(dense_T(a, b))
    assert np.max(np.abs(lam - w)) <= 1e-14
    assert metrics.orthogonality(Q) <= 1e-15
    assert metrics.residual(a, b, lam, Q) <= 1e-15


# --------------------------------------------------------------------------
# Rank estimate, Example 1 ranks, Philox Gaussian, ID, HSS
# --------------------------------------------------------------------------
def test_rank_worked_example():
    span, dist, eps, r = map(float, golden("rank_worked_example.txt")[0])
    assert hss.rank_formula(span / dist, eps) == int(r)
    # the printed, rounded R = 2.0e3 would give one more
    assert hss.rank_formula(2000.0, eps) == int(r) + 1


def example1_problem(N=2000, seed=11):
    d, u = inputs.example1(N, seed)
    lam, gam, mu, _ = dc.secular(d, u, 1.0)
    uh = dc.lowner(d, gam, mu, 1.0, u)
    return hss.generators(d, gam, mu, uh)


def test_table1_ranks():
    """Table 1: off-diagonal ranks at tolerance 1e-13, within +-3 (random u)."""
    gen = example1_problem()
    Qh = gen["_dense"]
    for m, r in golden("table1_ranks.txt"):
        m, r = int(m), int(r)
        s = np.linalg.svd(Qh[:m, m:], compute_uv=False)
        assert abs(int(np.sum(s > 1e-13)) - r) <= 3
    # the worked example's distance at m = 300 (printed 4.3e-3) is spacing + gamma
    dist = hss.boundary_dist(gen, 300)
    assert 4.0e-3 < dist < 8.0e-3


def test_rank_estimate_bounds_svd_rank():
    gen = example1_problem(1024, 3)
    bounds, L = hss.leaf_bounds(1024, 128)
    r, b2 = hss.rank_estimate(gen, bounds, eps=1e-13)
    Qh = gen["_dense"]
    for s in b2[1:-1]:
        sv = np.linalg.svd(Qh[:s, s:], compute_uv=False)
        assert int(np.sum(sv > 1e-13 * sv[0])) <= r


def test_rank_estimate_boundary_move_and_cap():
    K = 64
    d = np.arange(K, dtype=np.float64)
    gam = np.full(K, 0.5)
    gam[32] = 1e-300       # lambda_32 ~ d_32
    d[32] = d[31] + 1e-12  # boundary 32 nearly touches
    mu = np.r_[d[1:] - d[:-1] - gam[:-1], 0.0]
    gen = {"d": d, "gamma": gam, "mu": mu, "lam": d + gam}
    bounds = np.array([0, 16, 32, 48, 64])
    r, b2 = hss.rank_estimate(gen, bounds, eps=1e-16, cap=100)
    assert b2[2] != 32 and abs(int(b2[2]) - 32) <= 5
    r2, _ = hss.rank_estimate(gen, np.array([0, 32, 64]), eps=1e-16, cap=100, shift=0)
    assert r2 == 100


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the published known-answer vectors (golden file):
    a wrong multiplier, Weyl constant, round count or word shuffle fails here."""
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr = np.array([v[0:4]], dtype=np.uint64)
        out = hss.philox4x32_10(ctr, (v[4], v[5]))
        assert [int(x) for x in out[0]] == v[6:10]


def test_philox_gaussian_uses_the_counter_layout():
    """Omega[i, j] is Box-Muller on the first two words of Philox at counter
    (i, j, stream, 0) with key (seed lo, seed hi), u = (x + 0.5) 2^-32."""
    seed = 0x1234567890ABCDEF
    Om = hss.philox_gaussian(5, 3, seed, 9)
    for i, j in [(0, 0), (4, 2), (3, 1)]:
        w = hss.philox4x32_10(np.array([[i, j, 9, 0]], dtype=np.uint64),
                              (seed & 0xFFFFFFFF, seed >> 32))[0]
        u1 = (float(w[0]) + 0.5) / 2.0 ** 32
        u2 = (float(w[1]) + 0.5) / 2.0 ** 32
        assert Om[i, j] == np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def test_philox_gaussian_moments():
    Om = hss.philox_gaussian(4000, 50, seed=123, stream=5)
    assert abs(Om.mean()) < 0.01 and abs(Om.std() - 1) < 0.01
    from scipy import stats
    assert stats.kstest(Om.ravel()[:50000], "norm").pvalue > 1e-3
    Om2 = hss.philox_gaussian(4000, 50, seed=123, stream=6)
    assert abs(np.corrcoef(Om.ravel(), Om2.ravel())[0, 1]) < 0.01


def test_interp_decomp_exact_low_rank():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((60, 7)) @ rng.standard_normal((7, 25))
    U, I = hss.interp_decomp(A, 1e-12)
    assert U.shape == (60, 7)
    assert np.allclose(U[I], np.eye(7))
    assert np.linalg.norm(A - U @ A[I]) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("builder", ["rshss", "srrsc"])
def test_hss_construction_and_multiply(builder):
    gen = example1_problem(1500, 21)
    Qh = gen["_dense"]
    bounds, L = hss.leaf_bounds(1500, 128)
    r, b2 = hss.rank_estimate(gen, bounds)
    if builder == "rshss":
        Om = hss.philox_gaussian(1500, r + 10, 0, 1)
        H = hss.rshss(gen, b2, L, r, 10, Om, 1e-12)
    else:
        H = hss.srrsc(gen, b2, L, 1e-12)
    A = hss.densify(H)
    # leaves are exact
    for q in range(1 << L):
        s, e = H.span(L, q)
        assert np.array_equal(A[s:e, s:e], Qh[s:e, s:e])
    assert np.linalg.norm(A - Qh) <= 10 * 1e-12 * np.linalg.norm(Qh) * 10
    assert max(H.ranks()) <= r + 10
    X = np.random.default_rng(0).standard_normal((77, 1500))
    Y = hss.matmul_right(X, H)
    assert np.linalg.norm(Y - X @ A) <= 1e-14 * np.linalg.norm(X @ A) * 10


def test_srrsc_ranks_not_above_rshss():
    gen = example1_problem(1024, 8)
    bounds, L = hss.leaf_bounds(1024, 128)
    r, b2 = hss.rank_estimate(gen, bounds)
    H2 = hss.rshss(gen, b2, L, r, 10, hss.philox_gaussian(1024, r + 10, 0, 2), 1e-12)
    H1 = hss.srrsc(gen, b2, L, 1e-12)
    assert max(H1.ranks()) <= max(H2.ranks()) + 2
    ex = {k: float(v) for k, v in golden("example2_ranks.txt")}
    assert max(H1.ranks()) <= ex["srrsc_hss_rank"] + 10
    assert 0.5 * ex["typical_block_rank"] <= np.median(H2.ranks()) <= 1.5 * ex["typical_block_rank"]


@pytest.mark.parametrize("mode", [dc.MODE_ADC1, dc.MODE_ADC2])
def test_adc_end_to_end_toeplitz(mode):
    """Algorithm 1 with the HSS branch taken: still within 1e-10 of the closed form."""
    N = 2050
    a, b = inputs.toeplitz(N)
    st = []
    lam, Q = dc.solve(a, b, dc.Options(mode=mode, hss_threshold=500), st)
    assert any(s["hss"] for s in st)
    k = np.arange(1, N + 1)
    ex = np.sort(2 + 2 * np.cos(k * np.pi / (N + 1)))
    assert metrics.eig_error(lam, ex) <= 1e-12
    assert metrics.orthogonality(Q) <= 1e-10
    assert metrics.residual(a, b, lam, Q) <= 1e-10
