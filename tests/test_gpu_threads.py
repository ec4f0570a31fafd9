"""Two handles on two host threads: each handle keeps its own launch count,
split-product work counters and per-kernel timing (the header's "one handle
per host thread" contract).  Solves run concurrently on two streams; every
solve's statistics must equal those of the same solve run alone."""
import json
import threading

import numpy as np
import pytest

from paper_1510_04591_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_two_handles_two_threads_keep_their_own_stats():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1510_04591_gb300 import tdeig

    prof = tdeig.FLAG_PROFILE
    jobs = [(inputs.toeplitz(3000), "adc2", "split", 500), (inputs.uniform(2500, 4), "dense", "split", 2000)]

    def run(job, reps, out, key):
        (a, b), mode, prec, thr = job
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        with tdeig.Solver(stream=st.cuda_stream, hss_threshold=thr) as s:
            d = torch.from_numpy(a).cuda()
            e = torch.from_numpy(b).cuda()
            res = []
            for _ in range(reps):
                lam, Q = s.solve(d, e, mode, prec, flags=prof)
                js = json.loads(s.stats())
                res.append((js["launches"], js["split_tensor_flops"],
                            sum(v["launches"] for v in js["kernels"].values()),
                            lam.cpu().numpy()))
            out[key] = res

    solo = {}
    for i, job in enumerate(jobs):
        run(job, 1, solo, i)
    both = {}
    ts = [threading.Thread(target=run, args=(job, 4, both, i)) for i, job in enumerate(jobs)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for i in range(len(jobs)):
        l0, f0, k0, lam0 = solo[i][0]
        assert l0 > 0 and f0 > 0 and k0 == l0
        for l, f, k, lam in both[i]:
            assert (l, f, k) == (l0, f0, k0)
            assert np.array_equal(lam, lam0)
