"""Serving with continuous batching: requests submitted while others run are
admitted as workers and budget free up, and every answer is bitwise the one
that system gets when solved alone (and the oracle's)."""
import time

import numpy as np
import pytest

from gpu_common import cuda_device, same_array
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


def _pool(rbs, dev, count, seed):
    import torch
    pool = []
    for A, v in gen.serving_pool(count, seed, n_side_max=24):
        Ad = rbs.to_device(A, dev)
        b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
        alone = rbs.rbs_solve(Ad, b, tol=1e-8, maxit=800, variant=v)
        pool.append((A, Ad, b, v, alone))
    return pool


@pytest.mark.parametrize("workers,max_batch,budget,solo_n", [(3, 3, 8 << 30, 100000), (2, 4, 1, 100000),
                                                             (4, 2, 8 << 30, 5000)])
def test_mixed_stream_matches_solo_solves(orc, workers, max_batch, budget, solo_n):
    import torch
    dev = cuda_device()
    import paper_2302_04180_gb300 as rbs
    pool = _pool(rbs, dev, 8, seed=1)
    picks = (gen.splitmix64(77, 36) % np.uint64(len(pool))).astype(int)
    with rbs.RbsServer(workers=workers, max_batch=max_batch, budget_bytes=budget, solo_n=solo_n) as srv:
        tickets = []
        for k, p in enumerate(picks):
            A, Ad, b, v, _ = pool[p]
            sd = {"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                  "tol": 1e-8, "maxit": 800, "variant": v}
            tickets.append((srv.submit(sd), p))
            if k % 5 == 4:
                time.sleep(0.002)  # later requests arrive while earlier ones run
        results = [(srv.wait(t), p) for t, p in tickets]
    for r, p in results:
        alone = pool[p][4]
        assert r["status"] == alone["status"] == 0, r.get("error")
        assert r["iters"] == alone["iters"]
        assert same_array(r["x"].cpu().numpy(), alone["x"].cpu().numpy())
        assert r["latency_s"] >= r["queue_s"] >= 0.0
    # and the solo solves are the oracle's
    A, _, _, v, alone = pool[int(picks[0])]
    o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-8, maxit=800, variant=v)
    assert alone["iters"] == o["iters"] and same_array(alone["x"].cpu().numpy(), o["x"])
