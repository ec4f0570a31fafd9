"""The split-precision tensor-core product in isolation (tdeig_split_gemm).

Reference: the same product in np.longdouble (IEEE quad on aarch64, 64-bit
significand on x86), far more precise than the bounds tested.  Errors are
measured entrywise relative to (|op(A)| |op(B)|)_ij, the natural scale of a
dot product.  With s slices of beta bits per operand row/column the bound is
about K 2^(-beta s) times the ratio of the row / column maxima to the entries;
the tests use random entries of one order of magnitude and check
  40 bits: <= 2^-36,  56 bits: <= 2^-50 and within 8x of an FP64 GEMM,
  BF16 hi+lo (16 bits): <= 2^-13,  FP16 hi+lo (22 bits): <= 2^-18.
"""
import numpy as np
import pytest

from oracle import dc
from paper_1510_04591_gb300 import inputs

pytestmark = pytest.mark.gpu


def solver():
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig
    return tdeig.Solver()


def rel_err(C, A, B, transA=False, transB=False):
    oA = A.T if transA else A
    oB = B.T if transB else B
    ref = oA.astype(np.longdouble) @ oB.astype(np.longdouble)
    scale = np.abs(oA) @ np.abs(oB)
    return float(np.max(np.abs(C.astype(np.longdouble) - ref) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("M,N,K,tA,tB", [(300, 70, 200, False, False), (129, 64, 33, True, False),
                                         (256, 17, 700, False, True), (1, 1, 1, False, False),
                                         (513, 130, 1030, True, True)])
def test_split_40_bits(M, N, K, tA, tB):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((K, M) if tA else (M, K))
    B = rng.standard_normal((N, K) if tB else (K, N))
    with solver() as s:
        C = s.split_gemm(A, B, "split", 40, tA, tB)
    e = rel_err(C, A, B, tA, tB)
    print("40 bits", (M, N, K), e)
    assert e <= 2.0 ** -36


@pytest.mark.parametrize("K", [256, 2000, 4096])
def test_split_56_bits_matches_fp64(K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((384, K))
    B = rng.standard_normal((K, 64))
    with solver() as s:
        C = s.split_gemm(A, B, "split", 56)
    e = rel_err(C, A, B)
    e64 = rel_err(A @ B, A, B)
    print("56 bits K=%d split %.3e fp64 %.3e" % (K, e, e64))
    assert e <= 2.0 ** -50
    assert e <= 8 * e64 + 2.0 ** -52


def test_sampling_shaped_product():
    """Y = Qhat Omega with Qhat a Cauchy-like eigenvector matrix and Omega
    Gaussian, as in ADC2 sampling.  The split product's error is bounded by the
    digit grid of each operand row / column, i.e. relative to the row maximum of
    Qhat times the column maximum of Omega (not to |Qhat| |Omega|): entries with
    a small |Qhat| |Omega| -- the off-diagonal part that Phi = Y - D Omega keeps
    -- can carry errors far above an FP64 product's.  This is why the solver
    samples the off-diagonal part of Qhat (leaf blocks masked) instead."""
    K = 2048
    d, z = inputs.example1(K, 7)
    lam, gam, mu, _ = dc.secular(d, z, 1.0)
    uh = dc.lowner(d, gam, mu, 1.0, z)
    Qh, _ = dc.cauchy(d, gam, mu, uh)
    Om = np.random.default_rng(1).standard_normal((K, 64))
    with solver() as s:
        Y = s.split_gemm(Qh, Om, "split", 56)
        Z = s.split_gemm(Qh, Om, "split", 56, transA=True)
    for C, A in ((Y, Qh), (Z, Qh.T)):
        ref = A.astype(np.longdouble) @ Om.astype(np.longdouble)
        grid = (np.ldexp(1.0, np.frexp(np.max(np.abs(A), axis=1))[1])[:, None] *
                np.ldexp(1.0, np.frexp(np.max(np.abs(Om), axis=0))[1])[None, :] * K)
        e = float(np.max(np.abs(C - ref) / grid))
        print("sampling-shaped: error / (2^(e_i + f_j) K) = %.3e" % e)
        assert e <= 2.0 ** -55


@pytest.mark.parametrize("prec,bound", [("bf16x2", 2.0 ** -13), ("fp16x2", 2.0 ** -18)])
def test_two_slice_products(prec, bound):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 300))
    B = rng.standard_normal((300, 50))
    with solver() as s:
        C = s.split_gemm(A, B, prec)
    e = rel_err(C, A, B)
    print(prec, e)
    assert e <= bound


def test_split_gemm_rejects_bad_arguments():
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig
    A = np.ones((4, 4))
    with tdeig.Solver() as s:
        for kw in (dict(prec="split", bits=60), dict(prec="split", bits=4)):
            with pytest.raises(tdeig.TdeigError) as e:
                s.split_gemm(A, A, **kw)
            assert e.value.status == tdeig.EINVAL


def test_zero_rows_and_columns():
    """Rows of op(A) and columns of op(B) with no nonzero entry (their exponent
    bound keeps its initial value) give exact zeros; the other entries keep the
    40-bit bound."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((150, 90))
    B = rng.standard_normal((90, 40))
    A[[0, 77, 149], :] = 0.0
    B[:, [5, 39]] = 0.0
    with solver() as s:
        C = s.split_gemm(A, B, "split", 40)
    assert np.all(C[[0, 77, 149], :] == 0.0)
    assert np.all(C[:, [5, 39]] == 0.0)
    rows = np.setdiff1d(np.arange(150), [0, 77, 149])
    cols = np.setdiff1d(np.arange(40), [5, 39])
    e = rel_err(C[np.ix_(rows, cols)], A[rows], B[:, cols])
    print("zero rows/cols", e)
    assert e <= 2.0 ** -36


@pytest.mark.parametrize("M,N,K,tA,tB", [(1000, 70, 256, False, False), (777, 45, 200, True, True),
                                         (300, 300, 96, False, True)])
def test_one_pass_and_two_pass_slicing_agree(M, N, K, tA, tB):
    """Operands with k <= 256 are sliced in one pass (exponents and digits by
    one CTA that holds whole rows); longer ones by the exponent and slicing
    kernels.  Padding k with zero columns past 256 moves the same product to the
    two-pass path without changing any exponent bound or digit, and the level
    sums stay within one drain (k <= 384), so the two results are bit-identical."""
    rng = np.random.default_rng(M + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-20, 20, (1, N)))
    Kz = 320
    Az = np.zeros((M, Kz)); Az[:, :K] = A
    Bz = np.zeros((Kz, N)); Bz[:K, :] = B
    opA = lambda X: np.ascontiguousarray(X.T) if tA else X
    opB = lambda X: np.ascontiguousarray(X.T) if tB else X
    with solver() as s:
        C1 = s.split_gemm(opA(A), opB(B), "split", 40, tA, tB)
        C2 = s.split_gemm(opA(Az), opB(Bz), "split", 40, tA, tB)
    assert np.array_equal(C1, C2)
    assert rel_err(C1, A, B) <= 2.0 ** -36
