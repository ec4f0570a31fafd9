"""tdeig_secular_noalloc: secular roots whose scratch is a fixed device array.

The entry point serves callers that cannot allocate device memory when they
need the roots (a process whose free device memory belongs to its own pool
allocator, or a latency-bound path that cannot take cudaMalloc's implicit
synchronisation).  Here the test itself allocates the inputs and outputs with
torch and calls the entry point through the C ABI several times in a row (a
larger K, then smaller ones, so stale scratch from an earlier call would
show).  Each result must equal the allocating entry point tdeig_secular bit
for bit (same kernel arithmetic) and match the CPU oracle within the tolerance
of the secular parity tests (Theorem 1, Remark 1), including the closed-form
cases K = 1 and K = 2.  This file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import dc

pytestmark = pytest.mark.gpu


def rank_one(K, seed, rho):
    rng = np.random.default_rng(seed)
    d = np.sort(rng.uniform(-1, 1, K))
    z = rng.standard_normal(K)
    z /= np.linalg.norm(z)
    return d, z, rho


def test_noalloc_matches_allocating_entry_point_and_oracle():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig

    L = tdeig.lib()
    stream = torch.cuda.current_stream().cuda_stream
    with tdeig.Solver() as s:
        for K, seed, rho in [(4096, 11, 0.7), (777, 12, 1.9), (2, 13, 0.4), (1, 14, 1.1)]:
            d, z, rho = rank_one(K, seed, rho)
            dd = torch.from_numpy(d).cuda()
            zd = torch.from_numpy(z).cuda()
            lam, gam, mu = (torch.empty(K, dtype=torch.float64, device="cuda") for _ in range(3))
            torch.cuda.synchronize()
            st = L.tdeig_secular_noalloc(K, dd.data_ptr(), zd.data_ptr(), rho, lam.data_ptr(),
                                         gam.data_ptr(), mu.data_ptr(), stream)
            assert st == tdeig.OK, tdeig.strerror(st)
            lam_g, gam_g, mu_g = s.secular(dd, zd, rho)
            assert torch.equal(lam, lam_g) and torch.equal(gam, gam_g) and torch.equal(mu, mu_g)
            lam_r, gam_r, mu_r, _ = dc.secular(d, z, rho)
            lh, gh, mh = lam.cpu().numpy(), gam.cpu().numpy(), mu.cpu().numpy()
            scale = max(1.0, rho)
            assert np.max(np.abs(lh - lam_r)) <= 4e-15 * scale
            assert np.max(np.abs(gh - gam_r)) <= 4e-15 * scale
            assert np.all(gh > 0)
            if K > 1:
                assert np.max(np.abs(mh[:-1] - mu_r[:-1])) <= 4e-15 * scale
                assert np.all(mh[:-1] > 0)
            if K == 1:   # closed form: lambda = d + rho z^2
                assert lh[0] == d[0] + rho * z[0] * z[0]


def test_noalloc_rejects_oversize_and_host_memory():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig

    L = tdeig.lib()
    K = 65537
    buf = torch.zeros(K, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert L.tdeig_secular_noalloc(K, p, p, 1.0, p, p, p, None) == tdeig.EINVAL
    h = np.zeros(8)
    hp = h.ctypes.data
    assert L.tdeig_secular_noalloc(8, hp, hp, 1.0, hp, hp, hp, None) == tdeig.EINVAL
