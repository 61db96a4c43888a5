"""Serving with per-iteration continuous batching: requests submitted while
others iterate join them at the next engine step, and every answer is bitwise
the one that system gets when solved alone, and the CPU oracle's (Fig. 2,
Fig. 4), whatever else shares the steps."""
import time

import numpy as np
import pytest

from gpu_common import cuda_device, same_array
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


@pytest.fixture(scope="module")
def rbs(dev):
    import paper_2302_04180_gb300 as m
    return m


def _system(rbs, dev, A):
    import torch
    Ad = rbs.to_device(A, dev)
    b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    return Ad, b


@pytest.fixture(scope="module")
def pool(rbs, dev, orc):
    """Ten small systems of the serving mix (3D upwind convection-diffusion and
    3D Poisson), each solved alone on the GPU and by the oracle."""
    out = []
    for A, v in gen.serving_pool(10, 1, n_side_max=24):
        Ad, b = _system(rbs, dev, A)
        alone = rbs.rbs_solve(Ad, b, tol=1e-8, maxit=800, variant=v)
        o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-8, maxit=800, variant=v)
        assert alone["iters"] == o["iters"] and same_array(alone["hist"], o["hist"])
        assert same_array(alone["x"].cpu().numpy(), o["x"])
        out.append((A, Ad, b, v, alone))
    return out


def _check(r, alone):
    assert r["status"] == alone["status"] == 0, r.get("error")
    assert r["iters"] == alone["iters"] and r["converged"] == 1
    assert same_array(r["x"].cpu().numpy(), alone["x"].cpu().numpy())
    assert r["latency_s"] >= r["queue_s"] >= 0.0


@pytest.mark.parametrize("engines,max_active,budget,rows", [(1, 64, 8 << 30, 0), (2, 4, 1, 1024),
                                                            (1, 8, 8 << 30, 256)])
def test_mixed_stream_matches_solo_and_oracle(rbs, dev, pool, engines, max_active, budget, rows):
    """Every distinct system of the stream (all ten) is served and matches its
    solo solve, which matches the oracle (checked in the fixture)."""
    import torch
    picks = list(range(len(pool))) + list((gen.splitmix64(77, 30) % np.uint64(len(pool))).astype(int))
    with rbs.RbsServer(engines=engines, max_active=max_active, budget_bytes=budget, rows_per_block=rows) as srv:
        tickets = []
        for k, p in enumerate(picks):
            A, Ad, b, v, _ = pool[p]
            sd = {"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                  "tol": 1e-8, "maxit": 800, "variant": v}
            tickets.append((srv.submit(sd), p))
            if k % 5 == 4:
                time.sleep(0.002)  # later requests arrive while earlier ones iterate
        results = [(srv.wait(t), p) for t, p in tickets]
        st = srv.stats()
    for r, p in results:
        _check(r, pool[p][4])
    assert st["completed"] == len(picks) and st["pending"] == 0 and st["budget_in_use"] == 0
    if budget == 1:
        assert st["peak_active"] == 1  # one system at a time
    else:
        assert st["peak_active"] > 1


def test_request_admitted_mid_flight_matches_solo_and_oracle(rbs, dev, orc, pool):
    """A long solve is iterating; a second request submitted then joins it at a
    later step, with the first still in flight; both answers are bitwise their
    solo solves and the oracle's."""
    import torch
    A1 = gen.poisson3d(40)
    Ad1, b1 = _system(rbs, dev, A1)
    alone1 = rbs.rbs_solve(Ad1, b1, tol=1e-13, maxit=2000, variant=0)
    A2, Ad2, b2, v2, alone2 = pool[3]
    with rbs.RbsServer(engines=1, max_active=8) as srv:
        x1 = torch.empty(A1.n, dtype=torch.float64, device=dev)
        t1 = srv.submit({"A": Ad1, "b": b1, "x": x1, "tol": 1e-13, "maxit": 2000, "variant": 0})
        t0 = time.time()
        while srv.stats()["steps"] < 20 and time.time() - t0 < 30:
            time.sleep(0.0005)
        x2 = torch.empty(A2.n, dtype=torch.float64, device=dev)
        t2 = srv.submit({"A": Ad2, "b": b2, "x": x2, "tol": 1e-8, "maxit": 800, "variant": v2})
        r2 = srv.wait(t2)
        r1 = srv.wait(t1)
        s1, s2 = srv.request_stats(t1), srv.request_stats(t2)
    assert s2["admit_step"] > s1["admit_step"] + 10
    assert s2["active_at_admit"] >= 1
    assert s1["finish_step"] > s2["admit_step"]  # the first was still iterating when the second joined
    _check(r1, alone1)
    _check(r2, alone2)
    o1 = orc.solve(A1, orc.spmv(A1, np.ones(A1.n)), tol=1e-13, maxit=2000, variant=0)
    assert alone1["iters"] == o1["iters"] and same_array(alone1["x"].cpu().numpy(), o1["x"])


def test_invalid_system_and_maxit_in_the_mix(rbs, dev, pool):
    """A request whose CSR fails the device-side check ends with RBS_EINVAL and
    an iteration cap ends a request unconverged after maxit iterations (as
    rbs_solve does); the others in the same steps are unaffected."""
    import torch
    A, Ad, b, v, alone = pool[0]
    bad = gen.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[5] = A.n + 7
    Bd = rbs.to_device(bad, dev)
    capped = rbs.rbs_solve(Ad, b, tol=1e-8, maxit=3, variant=v)
    with rbs.RbsServer(engines=1, max_active=16) as srv:
        ta = srv.submit({"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                         "tol": 1e-8, "maxit": 800, "variant": v})
        tb = srv.submit({"A": Bd, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                         "tol": 1e-8, "maxit": 800, "variant": v})
        tc = srv.submit({"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                         "tol": 1e-8, "maxit": 3, "variant": v})
        ra, rb_, rc = srv.wait(ta), srv.wait(tb), srv.wait(tc)
    _check(ra, alone)
    assert rb_["status"] == rbs.RBS_EINVAL and "check" in rb_["error"]
    assert rc["status"] == 0 and rc["iters"] == 3 and rc["converged"] == 0
    assert same_array(rc["x"].cpu().numpy(), capped["x"].cpu().numpy())
