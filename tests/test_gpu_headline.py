"""GPU parity at the headline configuration: Toeplitz(2, 1), N = 16384, ADC2
with split-precision tensor-core products, default options (HSS threshold
2000, HSS leaves of 128, tolerance 1e-12, oversampling 10).

Checked against what the mathematics and the oracle fix (Sec. 5, Example 3
measures): eigenvalues against the closed form 2 + 2 cos(k pi / (N + 1)) and
against the FP64 oracle's ADC2 eigenvalues (max error / ||T||_2 <= 1e-12);
full orthogonality ||Q^T Q - I||_F / N and residual ||T Q - Q Lambda||_F /
(N ||T||_2) over all 16384 columns, both <= 1e-10 (the HSS bound); 64 sampled
eigenvectors against the closed form sqrt(2/(N+1)) sin(j k pi / (N+1)) up to
sign.
"""
import json
import math

import numpy as np
import pytest

from oracle import dc
from paper_1510_04591_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_headline_adc2_split_n16384():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig

    N = 16384
    a, b = inputs.toeplitz(N)
    with tdeig.Solver() as s:
        lam, Q = s.solve(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), "adc2", "split")
        torch.cuda.synchronize()
        st = json.loads(s.stats())
    hm = [h for h in st.get("hss", []) if "K" in h]
    assert len(hm) >= 7 and max(h["K"] for h in hm) >= 8192
    k = np.arange(1, N + 1)
    ex = np.sort(2.0 + 2.0 * np.cos(k * np.pi / (N + 1)))
    lh = lam.cpu().numpy()
    tn = np.max(np.abs(ex))
    assert np.max(np.abs(lh - ex)) / tn <= 1e-12
    # orthogonality and residual over all columns, on the GPU in FP64
    G = Q.t() @ Q
    G.diagonal().sub_(1.0)
    orth = float(torch.linalg.norm(G)) / N
    del G
    ad = torch.from_numpy(a).cuda()
    bd = torch.from_numpy(b).cuda()
    R = ad[:, None] * Q
    R[:-1] += bd[:, None] * Q[1:]
    R[1:] += bd[:, None] * Q[:-1]
    R -= Q * lam[None, :]
    resid = float(torch.linalg.norm(R)) / (N * float(lam.abs().max()))
    del R
    assert orth <= 1e-10 and resid <= 1e-10, (orth, resid)
    # sampled eigenvectors against the closed form, up to sign
    idx = np.random.default_rng(3).choice(N, 64, replace=False)
    order = np.argsort(2.0 + 2.0 * np.cos(k * np.pi / (N + 1)))
    V = math.sqrt(2.0 / (N + 1)) * np.sin(np.outer(k, k[order[idx]]) * np.pi / (N + 1))
    Qs = Q[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    sg = np.sign(np.sum(Qs * V, axis=0))
    assert np.max(np.abs(Qs * sg - V)) <= 1e-8
    del Q
    torch.cuda.empty_cache()
    # the FP64 oracle's ADC2 eigenvalues (host, all cores)
    lam_o, _ = dc.solve(a, b, dc.Options(mode=dc.MODE_ADC2))
    assert np.max(np.abs(lh - lam_o)) / tn <= 1e-12
