"""The paper's scalability workloads (Sec. 5.2) as synthetic stand-ins: the
27-point e-type unsymmetric stencil and band matrices. CPU checks of the
generators and the oracle; GPU parity of SpMV and both solvers."""
import numpy as np
import pytest

from gpu_common import cuda_device, same_array
from paper_2302_04180_gb300 import gen


def test_stencil27_structure(orc):
    N = 5
    A = gen.stencil27(N)
    assert A.n == N ** 3
    assert A.nnz == (3 * N - 2) ** 3  # 27-point: (3N-2)^3 nonzeros with Dirichlet edges
    # row of an interior point: 27 entries, 13 perturbed below the diagonal
    i = 2 + 2 * N + 2 * N * N
    vals = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    cols = A.col[A.rowptr[i]:A.rowptr[i + 1]]
    assert vals.size == 27 and (np.diff(cols) > 0).all()
    assert (vals[cols < i] == -0.9999).all() and (vals[cols > i] == -1.0).all()
    assert vals[cols == i][0] == 26.0
    # e-type is unsymmetric
    dense = np.zeros((A.n, A.n))
    for r in range(A.n):
        dense[r, A.col[A.rowptr[r]:A.rowptr[r + 1]]] = A.val[A.rowptr[r]:A.rowptr[r + 1]]
    assert not np.array_equal(dense, dense.T)


def test_banded_structure():
    A = gen.banded(50, 4)
    assert A.nnz == 50 * 9 - 2 * (4 * 5 // 2)
    row = A.val[A.rowptr[20]:A.rowptr[21]]
    assert row.size == 9 and row[4] == 9.0


@pytest.mark.parametrize("variant", [0, 1])
def test_oracle_solves_e_type(orc, variant):
    A = gen.stencil27(8)
    b = orc.spmv(A, np.ones(A.n))
    o = orc.solve(A, b, tol=1e-10, maxit=500, variant=variant)
    assert o["converged"] == 1 and np.max(np.abs(o["x"] - 1.0)) < 1e-8


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [0, 1])
def test_gpu_e_type_and_banded_parity(orc, variant):
    import torch
    dev = cuda_device()
    import paper_2302_04180_gb300 as rbs
    # spmv.mode 0 picks the long-span staging for these rows (27 and 121
    # nonzeros); 2 forces the short spans (every chunk then takes the per-lane
    # path), 1 one thread per row
    try:
        for A in (gen.stencil27(20), gen.banded(20000, 60), gen.banded(20001, 13)):
            Ad = rbs.to_device(A, dev)
            x = gen.random_vector(A.n, 4)
            b = orc.spmv(A, np.ones(A.n))
            o = orc.solve(A, b, tol=1e-10, maxit=400, variant=variant)
            for mode in (0, 1, 2):
                rbs.rbs_set_param("spmv.mode", mode)
                assert same_array(rbs.rbs_spmv_csr(Ad, torch.from_numpy(x).to(dev)).cpu().numpy(),
                                  orc.spmv(A, x)), mode
                g = rbs.rbs_solve(Ad, torch.from_numpy(b).to(dev), tol=1e-10, maxit=400, variant=variant)
                assert g["iters"] == o["iters"] and g["status"] == o["status"]
                assert same_array(g["hist"], o["hist"])
                assert same_array(g["x"].cpu().numpy(), o["x"])
    finally:
        rbs.rbs_set_param("spmv.mode", 0)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [0, 1])
def test_gpu_e_type_63_whole_history(orc, variant):
    """The 27-point e-type matrix at 63^3 (n = 250,047: 7,814 chunks of 32 rows
    and a tail of 31; edge rows of 8 to 18 nonzeros among interior rows of 27)
    through the long-row kernels -- the fused K1/K3 of the classic loop, the
    pipelined loop's SpMV -- to tol 1e-10: every history record, the iteration
    count and x bitwise the oracle's."""
    import torch
    dev = cuda_device()
    import paper_2302_04180_gb300 as rbs
    A = gen.stencil27(63)
    Ad = rbs.to_device(A, dev)
    b = orc.spmv(A, np.ones(A.n))
    o = orc.solve(A, b, tol=1e-10, maxit=800, variant=variant)
    g = rbs.rbs_solve(Ad, torch.from_numpy(b).to(dev), tol=1e-10, maxit=800, variant=variant)
    assert g["iters"] == o["iters"] > 50 and g["status"] == o["status"] == 0
    assert same_array(g["hist"], o["hist"])
    assert same_array(g["x"].cpu().numpy(), o["x"])
