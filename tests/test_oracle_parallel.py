"""The threaded oracle (the bench's all-cores CPU baseline) is the sequential
oracle split across threads: SpMV rows and element-wise steps are divided
among threads, and each exact dot sums per-thread integer accumulators
(orc_exdot_limbs) before its single rounding -- the rank-split reduction of
Sec. 3.2, pinned in test_oracle_exact.py. Every result must be bitwise the
one-thread result, for any thread count."""
import numpy as np
import pytest

from paper_2302_04180_gb300 import gen


def _bits(a):
    a = np.asarray(a, dtype=np.float64)
    b = a.view(np.uint64).copy()
    b[np.isnan(a)] = 0x7FF8000000000000
    return b


@pytest.fixture
def threads(orc):
    yield orc
    orc.set_threads(1)


@pytest.mark.parametrize("T", [2, 3, 8])
def test_exact_dot_over_threads_is_the_one_thread_dot(threads, T):
    orc = threads
    for n, cond, seed in ((1000, 1e32, 0), (65537, 1e16, 1), (7, 1e48, 2), (1, 1.0, 3)):
        x, y, exact = gen.ill_conditioned_dot(n, cond, seed)
        orc.set_threads(1)
        one = orc.exdot(x, y)
        orc.set_threads(T)
        assert orc.get_threads() == T
        assert _bits(orc.exdot(x, y)) == _bits(one)
        if exact is not None:
            assert one == exact


@pytest.mark.parametrize("T", [2, 5])
@pytest.mark.parametrize("variant", [0, 1])
def test_threaded_solve_is_the_sequential_solve(threads, T, variant):
    orc = threads
    systems = [gen.poisson3d(12), gen.convdiff3d(10, 20.0, (1.0, -0.5, 0.25)),
               gen.random_csr(3000, 9, 4, diag_dominant=True)]
    for A in systems:
        b = orc.spmv(A, np.ones(A.n))
        orc.set_threads(1)
        o1 = orc.solve(A, b, tol=1e-10, maxit=300, variant=variant)
        orc.set_threads(T)
        oT = orc.solve(A, b, tol=1e-10, maxit=300, variant=variant)
        assert o1["status"] == 0 and o1["iters"] > 5
        assert oT["iters"] == o1["iters"] and oT["status"] == o1["status"]
        assert (_bits(oT["hist"]) == _bits(o1["hist"])).all()
        assert (_bits(oT["x"]) == _bits(o1["x"])).all()
        assert (_bits(orc.spmv(A, oT["x"])) == _bits(orc.spmv(A, o1["x"]))).all()
