"""The lightweight FPE-8 dot (Sec. 3.2): expansions of eight binary64 terms
built with TwoProd and TwoSum, early exit, and a fallback to the exact dot
when the expansions cannot hold every bit. Its value is always the correctly
rounded dot: bitwise the oracle's."""
import numpy as np
import pytest

from gpu_common import cuda_device, same
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    cuda_device()
    import paper_2302_04180_gb300 as m
    return m


def test_well_conditioned_takes_the_fpe_path(rbs, orc):
    import torch
    dev = torch.device("cuda:0")
    for n in (1, 1000, 1 << 20, (1 << 20) + 7):
        x = gen.random_vector(n, 5, 1)
        y = gen.random_vector(n, 5, 2)
        v, fb = rbs.rbs_fpe_dot(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
        assert not fb, n
        assert same(v, orc.exdot(x, y)), n
    x, y, _ = gen.ill_conditioned_dot(1 << 18, 1e16, 1)
    v, fb = rbs.rbs_fpe_dot(x, y)  # host pointers
    assert same(v, orc.exdot(x, y))


def test_wide_range_falls_back_and_stays_exact(rbs, orc):
    import torch
    dev = torch.device("cuda:0")
    # 128 products over ~2^+-600 per thread need more than 8 expansion terms
    n = 4096
    x = gen.random_vector(n, 9, 1) * 2.0 ** np.round(gen.random_vector(n, 9, 2, -300, 300))
    y = gen.random_vector(n, 9, 3) * 2.0 ** np.round(gen.random_vector(n, 9, 4, -300, 300))
    rbs.rbs_set_param("exdot.grid", 1)
    rbs.rbs_set_param("exdot.block", 32)
    try:
        v, fb = rbs.rbs_fpe_dot(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
    finally:
        rbs.rbs_set_param("exdot.grid", 0)
        rbs.rbs_set_param("exdot.block", 0)
    assert fb
    assert same(v, orc.exdot(x, y))
    # subnormal products: TwoProd may be inexact -> fallback, exact value
    xs = np.array([2.0 ** -1000, 3.0, 2.0 ** -60])
    ys = np.array([2.0 ** -70, 1.0, 2.0 ** -1000])
    v, fb = rbs.rbs_fpe_dot(torch.from_numpy(xs).to(dev), torch.from_numpy(ys).to(dev))
    assert fb and same(v, orc.exdot(xs, ys))
    xn = np.array([1.0, np.inf])
    v, fb = rbs.rbs_fpe_dot(torch.from_numpy(xn).to(dev), torch.from_numpy(np.array([0.0, 0.0])).to(dev))
    assert fb and np.isnan(v)


@pytest.mark.parametrize("cond", [1e16, 1e32, 1e48])
def test_ill_conditioned_exact_either_way(rbs, orc, cond):
    x, y, exact = gen.ill_conditioned_dot(1 << 16, cond, 2)
    v, fb = rbs.rbs_fpe_dot(x, y)
    assert same(v, float(exact))
