"""Thin ctypes binding of libtdeig.so (include/tdeig.h).

Argument marshalling only: every step of the eigensolver runs in the library's
CUDA kernels.  If the library is missing or cannot be loaded this module raises;
there is no CPU fallback.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays (host).  Host inputs
are copied to the device by the library inside the call; results come back in
the same kind of memory as the inputs.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdeig.so")

MODE_DENSE, MODE_ADC1, MODE_ADC2 = 0, 1, 2
PREC_FP64, PREC_SPLIT, PREC_BF16X2, PREC_FP16X2 = 0 << 8, 1 << 8, 2 << 8, 3 << 8
FLAG_GRAPH = 1 << 12
FLAG_PROFILE = 1 << 13
FLAG_RECORD = 1 << 14
FLAG_MLP_SEED = 1 << 15
MLP_IN, MLP_HIDDEN = 7, 64
MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1
_MODES = {"dense": MODE_DENSE, "adc1": MODE_ADC1, "adc2": MODE_ADC2}
_PRECS = {"fp64": PREC_FP64, "split": PREC_SPLIT, "bf16x2": PREC_BF16X2, "fp16x2": PREC_FP16X2}

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT, ENOTIMPL = 0, -1, -2, -3, -4, -5, -6


class TdeigError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, strerror(status), status))


class Options(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("hss_threshold", ctypes.c_int),
                ("hss_leaf", ctypes.c_int), ("tol", ctypes.c_double),
                ("oversample", ctypes.c_int), ("rank_eps", ctypes.c_double),
                ("rank_cap", ctypes.c_int), ("boundary_shift", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib():
    """Load libtdeig.so (raises OSError when it is missing: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libtdeig.so not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.tdeig_default_options.argtypes = [ctypes.POINTER(Options)]
        L.tdeig_default_options.restype = None
        L.tdeig_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Options)]
        L.tdeig_create.restype = ctypes.c_int
        L.tdeig_destroy.argtypes = [_vp]
        L.tdeig_destroy.restype = ctypes.c_int
        L.tdeig_strerror.argtypes = [ctypes.c_int]
        L.tdeig_strerror.restype = ctypes.c_char_p
        L.tdeig_solve.argtypes = [_vp, _vp, _vp, _i64, _vp, _vp, ctypes.c_int]
        L.tdeig_solve.restype = ctypes.c_int
        L.tdeig_solve_batched.argtypes = [_vp, _i64, ctypes.POINTER(_i64), _vp, _vp, _vp, _vp,
                                          ctypes.c_int]
        L.tdeig_solve_batched.restype = ctypes.c_int
        L.tdeig_last_stats.argtypes = [_vp, ctypes.c_char_p, ctypes.c_size_t]
        L.tdeig_last_stats.restype = ctypes.c_int
        L.tdeig_secular.argtypes = [_vp, _i64, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]
        L.tdeig_secular.restype = ctypes.c_int
        L.tdeig_lowner_cauchy.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp,
                                          _vp]
        L.tdeig_lowner_cauchy.restype = ctypes.c_int
        L.tdeig_lowner_cauchy_split.argtypes = L.tdeig_lowner_cauchy.argtypes
        L.tdeig_lowner_cauchy_split.restype = ctypes.c_int
        L.tdeig_secular_noalloc.argtypes = [_i64, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp]
        L.tdeig_secular_noalloc.restype = ctypes.c_int
        L.tdeig_mlp_forward.argtypes = [_vp, _vp, _vp, _vp, _vp, _i64, _vp]
        L.tdeig_mlp_forward.restype = ctypes.c_int
        L.tdeig_mlp_grad.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]
        L.tdeig_mlp_grad.restype = ctypes.c_int
        L.tdeig_mlp_train.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_float, ctypes.c_uint64, _vp]
        L.tdeig_mlp_train.restype = ctypes.c_int
        L.tdeig_set_rank_model.argtypes = [_vp, _vp, _vp, _vp]
        L.tdeig_set_rank_model.restype = ctypes.c_int
        L.tdeig_rank_records.argtypes = [_vp, _vp, _i64]
        L.tdeig_rank_records.restype = ctypes.c_int
        L.tdeig_node_features.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp]
        L.tdeig_node_features.restype = ctypes.c_int
        L.tdeig_split_gemm.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64, ctypes.c_int, _vp, _i64,
                                       ctypes.c_int, _vp, _i64, ctypes.c_int, ctypes.c_int]
        L.tdeig_split_gemm.restype = ctypes.c_int
        L.tdeig_merge_deflate.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, ctypes.c_double,
                                          _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.tdeig_merge_deflate.restype = ctypes.c_int
        L.tdeig_rank_estimate.argtypes = [_vp, _i64, _vp, _vp, _i64, _vp, _vp]
        L.tdeig_rank_estimate.restype = ctypes.c_int
        L.tdeig_interp_decomp.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp]
        L.tdeig_interp_decomp.restype = ctypes.c_int
        L.tdeig_philox4x32_10.argtypes = [_vp, _i64, _vp, _vp, _vp]
        L.tdeig_philox4x32_10.restype = ctypes.c_int
        L.tdeig_gaussian.argtypes = [_vp, _i64, _i64, ctypes.c_uint64, ctypes.c_uint32, _vp]
        L.tdeig_gaussian.restype = ctypes.c_int
        L.tdeig_hss_apply.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, ctypes.c_int]
        L.tdeig_hss_apply.restype = ctypes.c_int
        L.tdeig_binary_arch.argtypes = [_vp]
        L.tdeig_binary_arch.restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(status):
    return lib().tdeig_strerror(int(status)).decode()


def default_options():
    o = Options()
    lib().tdeig_default_options(ctypes.byref(o))
    return o


def mode_code(mode="dense", prec="fp64", graph=False):
    if isinstance(mode, int):
        return mode | (FLAG_GRAPH if graph else 0)
    return _MODES[mode] | _PRECS[prec] | (FLAG_GRAPH if graph else 0)


# --------------------------------------------------------------------------
# array helpers
# --------------------------------------------------------------------------
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous() or x.t().is_contiguous()
        return x.data_ptr()
    return x.ctypes.data


def _as_f64(x):
    if _is_torch(x):
        import torch
        return x.to(torch.float64).contiguous()
    return np.ascontiguousarray(x, dtype=np.float64)


def _empty_like_kind(ref, shape, fortran=False):
    """An output array in the same kind of memory as ref."""
    if _is_torch(ref):
        import torch
        if fortran and len(shape) == 2:
            # column-major n x n buffer: allocate (n, n) row-major, hand out its transpose
            return torch.empty((shape[1], shape[0]), dtype=torch.float64, device=ref.device).t()
        return torch.empty(shape, dtype=torch.float64, device=ref.device)
    return np.empty(shape, dtype=np.float64, order="F" if fortran else "C")


class Solver:
    """A tdeig handle (one per host thread)."""

    def __init__(self, stream=None, **opts):
        o = default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %s" % k)
            setattr(o, k, v)
        if stream is not None:
            o.cuda_stream = stream
        self._keep_stream = stream
        h = _vp()
        st = lib().tdeig_create(ctypes.byref(h), ctypes.byref(o))
        if st != OK:
            raise TdeigError(st, "tdeig_create")
        self.h = h
        self.options = o

    def close(self):
        if getattr(self, "h", None):
            lib().tdeig_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self):
        n = lib().tdeig_last_stats(self.h, None, 0)
        buf = ctypes.create_string_buffer(max(n, 0) + 1)
        lib().tdeig_last_stats(self.h, buf, len(buf))
        return buf.value.decode()

    def solve_raw(self, d_ptr, e_ptr, N, lam_ptr, q_ptr, mode):
        """The C call itself on raw pointers; returns the status."""
        return lib().tdeig_solve(self.h, d_ptr, e_ptr, int(N), lam_ptr, q_ptr, int(mode))

    def solve(self, d, e, mode="dense", prec="fp64", vectors=True, out=None, check=True,
              graph=False, flags=0):
        """Eigendecomposition of tridiag(e, d, e): returns (lam, Q), Q[:, j] <-> lam[j]."""
        d = _as_f64(d)
        e = _as_f64(e)
        N = d.shape[0]
        if out is None:
            lam = _empty_like_kind(d, (N,))
            Q = _empty_like_kind(d, (N, N), fortran=True) if vectors else None
        else:
            lam, Q = out
        st = lib().tdeig_solve(self.h, _ptr(d), _ptr(e) if N > 1 else None, N, _ptr(lam), _ptr(Q),
                               mode_code(mode, prec, graph) | flags)
        if check and st != OK:
            raise TdeigError(st, "tdeig_solve")
        return lam, Q

    def solve_batched(self, ds, es, mode="dense", prec="fp64", graph=False, out=None, flags=0):
        """Independent matrices (lists of numpy arrays / CPU or CUDA tensors)."""
        sizes = [int(x.shape[0]) for x in ds]
        if _is_torch(ds[0]):
            import torch
            dcat = torch.cat([_as_f64(x) for x in ds])
            ecat = torch.cat([_as_f64(x) for x in es]) if sum(sizes) > len(sizes) else None
            lam = torch.empty(sum(sizes), dtype=torch.float64, device=dcat.device)
            Qc = torch.empty(sum(n * n for n in sizes), dtype=torch.float64, device=dcat.device)
        else:
            dcat = np.concatenate([_as_f64(x) for x in ds])
            ecat = np.concatenate([_as_f64(x) for x in es]) if sum(sizes) > len(sizes) else None
            lam = np.empty(sum(sizes))
            Qc = np.empty(sum(n * n for n in sizes))
        Ns = (_i64 * len(sizes))(*sizes)
        st = lib().tdeig_solve_batched(self.h, len(sizes), Ns, _ptr(dcat), _ptr(ecat), _ptr(lam),
                                       _ptr(Qc), mode_code(mode, prec, graph) | flags)
        if st != OK:
            raise TdeigError(st, "tdeig_solve_batched")
        outs = []
        r = q = 0
        for n in sizes:
            blk = Qc[q:q + n * n]
            Qb = blk.reshape(n, n).t() if _is_torch(blk) else blk.reshape((n, n), order="F")
            outs.append((lam[r:r + n], Qb))
            r += n
            q += n * n
        return outs

    def secular(self, d, z, rho):
        d = _as_f64(d)
        z = _as_f64(z)
        K = d.shape[0]
        lam, gam, mu = (_empty_like_kind(d, (K,)) for _ in range(3))
        st = lib().tdeig_secular(self.h, K, _ptr(d), _ptr(z), float(rho), _ptr(lam), _ptr(gam),
                                 _ptr(mu))
        if st != OK:
            raise TdeigError(st, "tdeig_secular")
        return lam, gam, mu

    def lowner_cauchy(self, d, gamma, mu, z, rho, qhat=True, split=False):
        """split=True: v and Qhat as split-precision solves form them (double-float)."""
        d, gamma, mu, z = (_as_f64(x) for x in (d, gamma, mu, z))
        K = d.shape[0]
        uh = _empty_like_kind(d, (K,))
        v = _empty_like_kind(d, (K,))
        Qh = _empty_like_kind(d, (K, K), fortran=True) if qhat else None
        name = "tdeig_lowner_cauchy_split" if split else "tdeig_lowner_cauchy"
        st = getattr(lib(), name)(self.h, K, _ptr(d), _ptr(gamma), _ptr(mu), _ptr(z),
                                  float(rho), _ptr(uh), _ptr(v), _ptr(Qh))
        if st != OK:
            raise TdeigError(st, name)
        return uh, v, Qh

    # ----------------------------------------------------------------------
    # learned rank seed (float32 host arrays; the model runs in the library)
    # ----------------------------------------------------------------------
    def mlp_forward(self, params, mean, std, X):
        params, mean, std, X = (_as_f32(a) for a in (params, mean, std, X))
        n = X.shape[0]
        y = np.empty(n, dtype=np.float32)
        st = lib().tdeig_mlp_forward(self.h, _ptr(params), _ptr(mean), _ptr(std), _ptr(X), n,
                                     _ptr(y))
        if st != OK:
            raise TdeigError(st, "tdeig_mlp_forward")
        return y

    def mlp_grad(self, params, mean, std, X, t):
        params, mean, std, X, t = (_as_f32(a) for a in (params, mean, std, X, t))
        loss = np.zeros(1, dtype=np.float32)
        grad = np.empty(MLP_PARAMS, dtype=np.float32)
        st = lib().tdeig_mlp_grad(self.h, _ptr(params), _ptr(mean), _ptr(std), _ptr(X), _ptr(t),
                                  X.shape[0], _ptr(loss), _ptr(grad))
        if st != OK:
            raise TdeigError(st, "tdeig_mlp_grad")
        return float(loss[0]), grad

    def mlp_train(self, params, mean, std, X, t, epochs=100, batch=256, lr=1e-3, seed=1):
        """Adam on the GPU; returns (trained params, final loss)."""
        p = _as_f32(params).copy()
        mean, std, X, t = (_as_f32(a) for a in (mean, std, X, t))
        loss = np.zeros(1, dtype=np.float32)
        st = lib().tdeig_mlp_train(self.h, _ptr(p), _ptr(mean), _ptr(std), _ptr(X), _ptr(t),
                                   X.shape[0], int(epochs), int(batch), float(lr), int(seed),
                                   _ptr(loss))
        if st != OK:
            raise TdeigError(st, "tdeig_mlp_train")
        return p, float(loss[0])

    def set_rank_model(self, params=None, mean=None, std=None):
        if params is None:
            st = lib().tdeig_set_rank_model(self.h, None, None, None)
        else:
            params, mean, std = (_as_f32(a) for a in (params, mean, std))
            self._model = (params, mean, std)
            st = lib().tdeig_set_rank_model(self.h, _ptr(params), _ptr(mean), _ptr(std))
        if st != OK:
            raise TdeigError(st, "tdeig_set_rank_model")

    def node_features(self, d, gamma, mu, uhat, n, ranges):
        """Features (len(ranges) x 7, float32) of the nodes [s0, s1) of one merge."""
        d, gamma, mu, uhat = (np.ascontiguousarray(_as_f64(a)) if not _is_torch(a) else _as_f64(a)
                              for a in (d, gamma, mu, uhat))
        rg = np.ascontiguousarray(np.asarray(ranges, dtype=np.int32).reshape(-1, 2))
        out = np.empty((rg.shape[0], MLP_IN), dtype=np.float32)
        st = lib().tdeig_node_features(self.h, d.shape[0], int(n), _ptr(d), _ptr(gamma), _ptr(mu),
                                       _ptr(uhat), rg.shape[0], _ptr(rg), _ptr(out))
        if st != OK:
            raise TdeigError(st, "tdeig_node_features")
        return out

    def split_gemm(self, A, B, prec="split", bits=40, transA=False, transB=False):
        """op(A) op(B) through the split-precision tensor-core product (FP64 in and out)."""
        A = np.asfortranarray(np.asarray(A, dtype=np.float64))
        B = np.asfortranarray(np.asarray(B, dtype=np.float64))
        M = A.shape[1] if transA else A.shape[0]
        K = A.shape[0] if transA else A.shape[1]
        N = B.shape[0] if transB else B.shape[1]
        C = np.empty((M, N), dtype=np.float64, order="F")
        st = lib().tdeig_split_gemm(self.h, M, N, K, A.ctypes.data, max(A.shape[0], 1),
                                    int(transA), B.ctypes.data, max(B.shape[0], 1), int(transB),
                                    C.ctypes.data, max(M, 1), _PRECS[prec], int(bits))
        if st != OK:
            raise TdeigError(st, "tdeig_split_gemm")
        return C

    # ----------------------------------------------------------------------
    # stage entry points of the integer decisions (host numpy arrays)
    # ----------------------------------------------------------------------
    def merge_deflate(self, lam1, lam2, z1, z2, beta):
        """Sort and deflation of one merge; returns a dict (perm, d, z, keep, rho, K,
        rotations (j, i, c, s))."""
        lam1, lam2, z1, z2 = (np.ascontiguousarray(x, dtype=np.float64) for x in (lam1, lam2, z1, z2))
        n1, n2 = len(lam1), len(lam2)
        n = n1 + n2
        perm = np.empty(n, dtype=np.int32)
        keep = np.empty(n, dtype=np.int32)
        d = np.empty(n)
        z = np.empty(n)
        rj = np.empty(n, dtype=np.int32)
        ri = np.empty(n, dtype=np.int32)
        rc = np.empty(n)
        rs = np.empty(n)
        rho = np.zeros(1)
        cnt = np.zeros(2, dtype=np.int64)
        st = lib().tdeig_merge_deflate(self.h, n1, n2, _ptr(lam1), _ptr(lam2), _ptr(z1), _ptr(z2),
                                       float(beta), _ptr(perm), _ptr(d), _ptr(z), _ptr(keep),
                                       _ptr(rho), _ptr(cnt), _ptr(rj), _ptr(ri), _ptr(rc), _ptr(rs))
        if st != OK:
            raise TdeigError(st, "tdeig_merge_deflate")
        m = int(cnt[1])
        return {"perm": perm, "d": d, "z": z, "keep": keep, "rho": float(rho[0]), "K": int(cnt[0]),
                "rot": (rj[:m], ri[:m], rc[:m], rs[:m])}

    def rank_estimate(self, d, gamma, bounds):
        """(r, moved bounds) of eq. (bounds) with the handle's options."""
        d, gamma = (np.ascontiguousarray(x, dtype=np.float64) for x in (d, gamma))
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.int32)).copy()
        r = np.zeros(1, dtype=np.int32)
        st = lib().tdeig_rank_estimate(self.h, len(d), _ptr(d), _ptr(gamma), len(b) - 1, _ptr(b),
                                       _ptr(r))
        if st != OK:
            raise TdeigError(st, "tdeig_rank_estimate")
        return int(r[0]), b

    def interp_decomp(self, Phi):
        """Row ID Phi ~= U Phi[piv]: returns (U m x rank, piv)."""
        Phi = np.asfortranarray(np.asarray(Phi, dtype=np.float64))
        m, s = Phi.shape
        k = min(m, s)
        U = np.zeros((m, k), order="F")
        piv = np.zeros(k, dtype=np.int32)
        rk = np.zeros(1, dtype=np.int32)
        st = lib().tdeig_interp_decomp(self.h, m, s, Phi.ctypes.data, m, U.ctypes.data, m,
                                       _ptr(piv), _ptr(rk))
        if st != OK:
            raise TdeigError(st, "tdeig_interp_decomp")
        r = int(rk[0])
        return U[:, :r].copy(), piv[:r].copy()

    def philox(self, ctr, key):
        """Philox4x32-10 words for counters ctr (n x 4) and keys key (n x 2), uint32."""
        ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
        key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
        out = np.empty_like(ctr)
        st = lib().tdeig_philox4x32_10(self.h, ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out))
        if st != OK:
            raise TdeigError(st, "tdeig_philox4x32_10")
        return out

    def gaussian(self, nrow, ncol, seed, stream_id):
        """The sampling matrix Omega (nrow x ncol) as the solver draws it."""
        out = np.empty((nrow, ncol), order="F")
        st = lib().tdeig_gaussian(self.h, nrow, ncol, int(seed), int(stream_id), out.ctypes.data)
        if st != OK:
            raise TdeigError(st, "tdeig_gaussian")
        return out

    def hss_apply(self, d, gamma, mu, uhat, X, mode="adc2", prec="fp64"):
        """out = X H with H the HSS approximation (ADC1 / ADC2) of the Cauchy-like
        matrix of the generators; X: P x K (torch CUDA or numpy, column-major)."""
        d, gamma, mu, uhat = (_as_f64(x) for x in (d, gamma, mu, uhat))
        K = d.shape[0]
        if _is_torch(X):
            import torch
            Xc = X.t().contiguous().t() if not X.t().is_contiguous() else X
            out = torch.empty((X.shape[1], X.shape[0]), dtype=torch.float64, device=X.device).t()
        else:
            Xc = np.asfortranarray(np.asarray(X, dtype=np.float64))
            out = np.empty(Xc.shape, order="F")
        st = lib().tdeig_hss_apply(self.h, K, _ptr(d), _ptr(gamma), _ptr(mu), _ptr(uhat),
                                   Xc.shape[0], _ptr(Xc), _ptr(out), mode_code(mode, prec))
        if st != OK:
            raise TdeigError(st, "tdeig_hss_apply")
        return out

    def rank_records(self):
        """(features n x 7, ln(rank + 1) n) recorded by the last TDEIG_FLAG_RECORD solve."""
        n = lib().tdeig_rank_records(self.h, None, 0)
        if n < 0:
            raise TdeigError(n, "tdeig_rank_records")
        buf = np.empty((n, MLP_IN + 1), dtype=np.float32)
        if n:
            lib().tdeig_rank_records(self.h, _ptr(buf), n)
        return buf[:, :MLP_IN].copy(), buf[:, MLP_IN].copy()


def _as_f32(x):
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=np.float32)
