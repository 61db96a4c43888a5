"""GPU parity of the reproducible classic (Fig. 2) and pipelined (Fig. 4)
PBiCGStab against the CPU oracle: the whole history of scalars, the iteration
count and the final x, bit for bit, across launch shapes and repeats; plus the
full-size workloads for their first iterations, error and breakdown paths, and
the plain (non-reproducible) comparator."""
import numpy as np
import pytest

from gpu_common import bits, cuda_device, same_array
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


@pytest.fixture(scope="module")
def rbs(dev):
    import paper_2302_04180_gb300 as m
    carve = m.rbs_get_param("smem.carveout")
    yield m
    for k in ("vec.grid", "vec.block", "spmv.block", "spmv.mode", "solve.check_every"):
        m.rbs_set_param(k, 0)
    m.rbs_set_param("smem.carveout", carve)


def _gpu_solve(rbs, dev, A, tol, maxit, variant, b=None, **kw):
    import torch
    Ad = rbs.to_device(A, dev)
    if b is None:
        bd = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    else:
        bd = torch.from_numpy(b).to(dev)
    r = rbs.rbs_solve(Ad, bd, tol=tol, maxit=maxit, variant=variant, **kw)
    r["x"] = r["x"].cpu().numpy()
    return r, bd.cpu().numpy()


def _assert_same_run(g, o):
    assert g["status"] == o["status"]
    assert g["iters"] == o["iters"]
    assert g["converged"] == o["converged"]
    assert same_array([g["tau0"], g["tau_max"]], [o["tau0"], o["tau_max"]])
    assert same_array(g["hist"], o["hist"])
    assert same_array(g["x"], o["x"])


@pytest.mark.parametrize("variant", [0, 1])
def test_c1_poisson16_whole_history(rbs, dev, orc, variant):
    """Poisson 7-point 16^3, b = A*1, x0 = 0, tol 1e-8, maxit 1000."""
    A = gen.poisson3d(16)
    g, b = _gpu_solve(rbs, dev, A, 1e-8, 1000, variant)
    assert same_array(b, orc.spmv(A, np.ones(A.n)))
    o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-8, maxit=1000, variant=variant)
    assert o["converged"] == 1 and o["iters"] > 10
    _assert_same_run(g, o)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("make", [lambda: gen.convdiff3d(12, 10.0),
                                  lambda: gen.convdiff2d(40, 45.0, (0.3, -0.9)),
                                  lambda: gen.random_csr(3001, 9, 5, diag_dominant=True)])
def test_nonsymmetric_systems(rbs, dev, orc, make, variant):
    A = make()
    g, b = _gpu_solve(rbs, dev, A, 1e-10, 500, variant)
    o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-10, maxit=500, variant=variant)
    _assert_same_run(g, o)


@pytest.mark.parametrize("variant", [0, 1])
def test_x0_and_given_diagonal(rbs, dev, orc, variant):
    import torch
    A = gen.convdiff3d(10, 20.0, (1.0, -0.3, 0.5))
    b = gen.random_vector(A.n, 4)
    x0 = gen.random_vector(A.n, 5)
    d = gen.random_vector(A.n, 6, lo=4.0, hi=9.0)
    Ad = rbs.to_device(A, dev)
    g = rbs.rbs_solve(Ad, torch.from_numpy(b).to(dev), x0=torch.from_numpy(x0).to(dev),
                      jacobi_diag=torch.from_numpy(d).to(dev), tol=1e-9, maxit=400, variant=variant)
    g["x"] = g["x"].cpu().numpy()
    o = orc.solve(A, b, x0=x0, diag=d, tol=1e-9, maxit=400, variant=variant)
    _assert_same_run(g, o)


def test_launch_shape_and_chunk_independence(rbs, dev, orc):
    A = gen.convdiff3d(14, 10.0)
    o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-10, maxit=500, variant=0)
    carve = rbs.rbs_get_param("smem.carveout")
    for vg, vb, sb, ce, lm, sm, co in ((0, 0, 0, 0, 0, 0, 75), (0, 0, 0, 0, 1, 1, -1), (1, 32, 32, 1, 1, 0, 100),
                                       (7, 128, 64, 3, 0, 1, 50), (500, 256, 256, 50, 1, 2, 0),
                                       (152, 64, 128, 0, 0, 3, 75), (0, 0, 0, 5, 1, 3, 100)):
        rbs.rbs_set_param("spmv.mode", sm)
        rbs.rbs_set_param("smem.carveout", co)
        rbs.rbs_set_param("vec.grid", vg)
        rbs.rbs_set_param("vec.block", vb)
        rbs.rbs_set_param("spmv.block", sb)
        for variant in (0, 1):
            g, _ = _gpu_solve(rbs, dev, A, 1e-10, 500, variant, check_every=ce, loop_mode=lm)
            ov = o if variant == 0 else orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-10, maxit=500,
                                                  variant=1)
            _assert_same_run(g, ov)
    for k in ("vec.grid", "vec.block", "spmv.block", "spmv.mode"):
        rbs.rbs_set_param(k, 0)
    rbs.rbs_set_param("smem.carveout", carve)


def test_run_to_run_bitwise(rbs, dev):
    A = gen.poisson3d(24)
    runs = [_gpu_solve(rbs, dev, A, 1e-10, 1000, v % 2, loop_mode=(v // 2) % 2)[0] for v in range(8)]
    runs = runs[0::2]  # classic runs, graph and host loops alternating
    for r in runs[1:]:
        assert r["iters"] == runs[0]["iters"]
        assert same_array(r["hist"], runs[0]["hist"]) and same_array(r["x"], runs[0]["x"])


def test_host_pointer_path_matches(rbs, dev, orc):
    A = gen.convdiff3d(9, 10.0)
    b = orc.spmv(A, np.ones(A.n))
    g = rbs.rbs_solve(A, b, tol=1e-10, maxit=300, variant=1)  # numpy: host buffers, staged
    o = orc.solve(A, b, tol=1e-10, maxit=300, variant=1)
    _assert_same_run(g, o)


@pytest.mark.parametrize("variant", [0, 1])
def test_edge_cases(rbs, dev, orc, variant):
    import torch
    A = gen.poisson3d(5)
    Ad = rbs.to_device(A, dev)
    zero = rbs.rbs_solve(Ad, torch.zeros(A.n, dtype=torch.float64, device=dev), variant=variant)
    assert zero["status"] == 0 and zero["iters"] == 0 and zero["converged"] == 1
    assert (bits(zero["x"].cpu().numpy()) == 0).all()
    b = orc.spmv(A, np.ones(A.n))
    bd = torch.from_numpy(b).to(dev)
    m0 = rbs.rbs_solve(Ad, bd, maxit=0, variant=variant)
    assert m0["iters"] == 0 and m0["converged"] == 0
    m3 = rbs.rbs_solve(Ad, bd, tol=1e-15, maxit=3, variant=variant)
    o3 = orc.solve(A, b, tol=1e-15, maxit=3, variant=variant)
    m3["x"] = m3["x"].cpu().numpy()
    _assert_same_run(m3, o3)
    bn = b.copy()
    bn[7] = np.nan
    r = rbs.rbs_solve(Ad, torch.from_numpy(bn).to(dev), variant=variant)
    assert r["status"] == rbs.RBS_ENAN == orc.solve(A, bn, variant=variant)["status"]
    with pytest.raises(rbs.RbsError) as e:
        rbs.rbs_solve(Ad, bd, jacobi_diag=torch.zeros(A.n, dtype=torch.float64, device=dev))
    assert e.value.code == rbs.RBS_EINVAL


@pytest.mark.parametrize("variant", [0, 1])
def test_breakdown(rbs, dev, orc, variant):
    A = gen.CSR(2, np.array([0, 1, 3], np.int64), np.array([0, 0, 1], np.int32),
                np.array([1.0, -2.0, 1.0]))
    b = np.array([1.0, 1.0])
    g, _ = _gpu_solve(rbs, dev, A, 1e-8, 10, variant, b=b)
    o = orc.solve(A, b, tol=1e-8, maxit=10, variant=variant)
    assert g["status"] == o["status"] == rbs.RBS_EBREAKDOWN
    assert g["iters"] == o["iters"] == 0


def test_diagonal_converges_in_one_step(rbs, dev, orc):
    n = 1000
    d = 2.0 ** (np.arange(n) % 20 - 10.0)
    A = gen.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d)
    b = gen.random_vector(n, 3)
    for variant in (0, 1):
        g, _ = _gpu_solve(rbs, dev, A, 1e-14, 20, variant, b=b)
        assert g["iters"] == 1 and g["converged"] == 1
        assert (g["x"] == b / d).all()


def test_plain_comparator_runs(rbs, dev, orc):
    A = gen.convdiff3d(20, 10.0)
    g, _ = _gpu_solve(rbs, dev, A, 1e-10, 1000, 0, dot_mode=rbs.RBS_DOT_PLAIN)
    o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-10, maxit=1000, variant=0)
    assert g["converged"] == 1 and abs(g["iters"] - o["iters"]) <= max(3, o["iters"] // 10)
    assert np.max(np.abs(g["x"] - 1.0)) < 1e-6


@pytest.mark.parametrize("variant,iters", [(0, 3), (1, 2)])
def test_full_size_poisson256_first_iterations(rbs, dev, orc, variant, iters):
    """The benchmark workload (Poisson 7-point 256^3, tol 1e-10) for its first
    iterations, every scalar bit for bit against the oracle."""
    A = gen.poisson3d(256)
    assert A.n == 16777216 and A.nnz == 117047296
    g, b = _gpu_solve(rbs, dev, A, 1e-10, iters, variant)
    o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-10, maxit=iters, variant=variant)
    _assert_same_run(g, o)


def test_full_size_convdiff192_first_iterations(rbs, dev, orc):
    A = gen.convdiff3d(192, 10.0)
    assert A.n == 7077888 and A.nnz == 49324032
    for variant in (0, 1):
        g, _ = _gpu_solve(rbs, dev, A, 1e-10, 2, variant)
        o = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-10, maxit=2, variant=variant)
        _assert_same_run(g, o)
