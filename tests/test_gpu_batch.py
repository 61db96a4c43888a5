"""GPU parity of the batched solver (many independent systems: one persistent
cluster launch, or the stepped schedule that advances all systems together
one iteration per step): every system's whole history, iteration count and x
are bitwise the CPU oracle's for that system alone, for a mix of 2D/3D
convection-diffusion systems, classic and pipelined, with and without x0 and a
given diagonal, with per-system iteration caps; invalid systems are reported
and skipped without affecting the rest."""

# the default persistent schedule, the stepped one, and the stepped one on
# small blocks (every system on several blocks)
SCHEDULES = (None, {"cluster": 0, "split": 0}, {"cluster": 0, "split": 256})
import numpy as np
import pytest

from gpu_common import cuda_device, same_array
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


def _device_system(rbs, dev, A, variant, tol, maxit, b=None, x0=None, diag=None):
    import torch
    Ad = rbs.to_device(A, dev)
    if b is None:
        bd = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    else:
        bd = torch.from_numpy(b).to(dev)
    sd = {"A": Ad, "b": bd, "x": torch.empty(A.n, dtype=torch.float64, device=dev), "tol": tol,
          "maxit": maxit, "variant": variant}
    if x0 is not None:
        sd["x0"] = torch.from_numpy(x0).to(dev)
    if diag is not None:
        sd["jacobi_diag"] = torch.from_numpy(diag).to(dev)
    return sd


def _check(g, o):
    assert g["status"] == o["status"]
    assert g["iters"] == o["iters"]
    assert g["converged"] == o["converged"]
    assert same_array(g["hist"], o["hist"])
    assert same_array(g["x"].cpu().numpy(), o["x"])


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_batch_matches_oracle_per_system(dev, orc, schedule):
    import paper_2302_04180_gb300 as rbs
    work = gen.batch_workload(14, seed=3, n_min=200, n_max=9000)
    systems, refs = [], []
    for k, (A, variant) in enumerate(work):
        b = orc.spmv(A, np.ones(A.n))
        x0 = gen.random_vector(A.n, 50 + k) if k % 4 == 1 else None
        diag = gen.random_vector(A.n, 70 + k, lo=6.0, hi=9.0) if k % 5 == 2 else None
        maxit = 5 + k if k % 6 == 3 else 600  # some systems stop at their cap, unconverged
        systems.append(_device_system(rbs, dev, A, variant, 1e-8, maxit, b=b, x0=x0, diag=diag))
        refs.append(orc.solve(A, b, x0=x0, diag=diag, tol=1e-8, maxit=maxit, variant=variant))
    res = rbs.rbs_solve_batched(systems, schedule=schedule)
    assert sorted({v for _, v in work}) == [0, 1]
    assert any(o["converged"] == 0 for o in refs) and any(o["converged"] == 1 for o in refs)
    for g, o in zip(res, refs):
        _check(g, o)


def test_batch_equals_single_solves_and_is_repeatable(dev):
    import paper_2302_04180_gb300 as rbs
    work = gen.batch_workload(40, seed=7, n_min=1000, n_max=60000)
    systems = [_device_system(rbs, dev, A, v, 1e-8, 2000) for A, v in work]
    res1 = rbs.rbs_solve_batched(systems)
    x1 = [r["x"].clone() for r in res1]
    res2 = rbs.rbs_solve_batched(systems)
    for k, (sd, (A, v)) in enumerate(zip(systems, work)):
        single = rbs.rbs_solve(sd["A"], sd["b"], tol=1e-8, maxit=2000, variant=v)
        for r, x in ((res1[k], x1[k]), (res2[k], res2[k]["x"])):
            assert r["iters"] == single["iters"] and r["status"] == single["status"]
            assert same_array(r["hist"], single["hist"])
            assert same_array(x.cpu().numpy(), single["x"].cpu().numpy())


@pytest.mark.parametrize("schedule", SCHEDULES[:2])
def test_batch_reports_invalid_systems(dev, orc, schedule):
    import torch
    import paper_2302_04180_gb300 as rbs
    good = gen.convdiff2d(30, 20.0, (0.6, 0.8))
    bad = gen.poisson3d(6)
    systems = [_device_system(rbs, dev, good, 0, 1e-8, 500),
               _device_system(rbs, dev, bad, 1, 1e-8, 500,
                              diag=np.zeros(bad.n)),  # zero diagonal
               _device_system(rbs, dev, good, 1, 1e-8, 500)]
    systems.append(dict(systems[0], maxit=0,
                        x=torch.empty(good.n, dtype=torch.float64, device=dev)))
    systems.append(_device_system(rbs, dev, good, 0, 1e-8, 500, b=np.zeros(good.n)))
    res = rbs.rbs_solve_batched(systems, schedule=schedule)
    assert res[1]["status"] == rbs.RBS_EINVAL
    b = orc.spmv(good, np.ones(good.n))
    _check(res[0], orc.solve(good, b, tol=1e-8, maxit=500, variant=0))
    _check(res[2], orc.solve(good, b, tol=1e-8, maxit=500, variant=1))
    assert res[3]["iters"] == 0 and res[3]["converged"] == 0
    assert res[4]["iters"] == 0 and res[4]["converged"] == 1
    assert (res[4]["x"] == 0).all()


def _ref_solves(rbs, systems, work, maxit):
    return [rbs.rbs_solve(sd["A"], sd["b"], tol=1e-8, maxit=maxit, variant=v) for sd, (A, v) in
            zip(systems, work)]


def _same_as(res, refs):
    for r, s in zip(res, refs):
        assert r["iters"] == s["iters"] and r["status"] == s["status"]
        assert same_array(r["hist"], s["hist"])
        assert same_array(r["x"].cpu().numpy(), s["x"].cpu().numpy())


def test_batch_results_do_not_depend_on_the_schedule(dev):
    import paper_2302_04180_gb300 as rbs
    work = gen.batch_workload(24, seed=11, n_min=300, n_max=30000)
    systems = [_device_system(rbs, dev, A, v, 1e-8, 1500) for A, v in work]
    refs = _ref_solves(rbs, systems, work, 1500)
    med = int(sorted(A.n for A, _ in work)[len(work) // 2])
    for cluster, split in ((1, 0), (2, 0), (4, med), (8, 0), (8, med), (8, 1 << 40), (16, med), (0, 0), (0, 1024),
                           (0, 64)):
        try:
            res = rbs.rbs_solve_batched(systems, schedule={"cluster": cluster, "split": split})
        except rbs.RbsError as e:
            # a 16-CTA cluster needs the device's non-portable cluster size
            assert cluster == 16 and e.code == rbs.RBS_EINVAL
            continue
        _same_as(res, refs)


def test_batch_rejects_bad_schedule(dev):
    import paper_2302_04180_gb300 as rbs
    A, v = gen.batch_workload(1, seed=1, n_min=500, n_max=600)[0]
    sd = _device_system(rbs, dev, A, v, 1e-8, 200)
    with pytest.raises(rbs.RbsError) as e:
        rbs.rbs_solve_batched([sd], schedule={"cluster": 3, "split": 0})
    assert e.value.code == rbs.RBS_EINVAL


def test_batch_tuner_picks_a_schedule_and_leaves_results_unchanged(dev):
    import torch
    import paper_2302_04180_gb300 as rbs
    work = gen.batch_workload(32, seed=5, n_min=500, n_max=40000)
    systems = [_device_system(rbs, dev, A, v, 1e-8, 2000) for A, v in work]
    refs = _ref_solves(rbs, systems, work, 2000)
    first = rbs.rbs_solve_batched(systems, history=False)
    for sd in systems:
        sd["x"].fill_(-7.0)
    best = rbs.rbs_batch_tune(systems, prev=first, proxy_iters=16)
    print("tuned schedule", best)
    assert best["cluster"] in (0, 1, 2, 4, 8, 16) and best["split"] >= 0 and best["ms"] > 0.0
    for sd in systems:  # proxy solves write scratch, not the callers' x
        assert bool((sd["x"] == -7.0).all())
    res = rbs.rbs_solve_batched(systems)  # now under the tuned schedule
    _same_as(res, refs)
    torch.cuda.synchronize()


def test_batch_graph_replay_sees_new_data(dev):
    """The same system set three times with new right-hand sides written into
    the same buffers: a plain launch, then the captured graph, then its replay;
    every call matches per-system solves of the data it saw."""
    import torch
    import paper_2302_04180_gb300 as rbs
    work = gen.batch_workload(12, seed=21, n_min=500, n_max=20000)
    systems = [_device_system(rbs, dev, A, v, 1e-8, 1500) for A, v in work]
    for rnd in range(3):
        for k, sd in enumerate(systems):
            n = sd["b"].numel()
            sd["b"].copy_(torch.from_numpy(gen.random_vector(n, 100 * rnd + k, lo=-1.0, hi=1.0)))
        res = rbs.rbs_solve_batched(systems)
        _same_as(res, _ref_solves(rbs, systems, work, 1500))


@pytest.fixture(scope="module")
def large_batch(orc):
    """Three systems of 195k-287k unknowns (classic and pipelined; one stops at
    its iteration cap of 400) with their oracle solves (the oracle threaded,
    which is bitwise its one-thread result)."""
    import os
    work = gen.batch_workload(3, seed=21, n_min=100000, n_max=300000)
    keep = orc.get_threads()
    orc.set_threads(min(16, os.cpu_count() or 1))
    try:
        out = []
        for A, variant in work:
            b = orc.spmv(A, np.ones(A.n))
            out.append((A, variant, b, orc.solve(A, b, tol=1e-8, maxit=400, variant=variant)))
    finally:
        orc.set_threads(keep)
    assert sorted({v for _, v, _, _ in out}) == [0, 1]
    assert any(o["converged"] == 0 for *_, o in out) and any(o["converged"] == 1 for *_, o in out)
    return out


@pytest.mark.parametrize("schedule", [None, {"cluster": 8, "split": 150000}, {"cluster": 0, "split": 0}])
def test_batch_large_systems_match_oracle(dev, large_batch, schedule):
    """Large systems under the persistent default (every CTA alone), the
    persistent schedule with a cluster per system above the split, and the
    stepped schedule: every history, iteration count and x bitwise the
    oracle's."""
    import paper_2302_04180_gb300 as rbs
    systems = [_device_system(rbs, dev, A, v, 1e-8, 400, b=b) for A, v, b, _ in large_batch]
    res = rbs.rbs_solve_batched(systems, schedule=schedule)
    for g, (*_, o) in zip(res, large_batch):
        _check(g, o)
