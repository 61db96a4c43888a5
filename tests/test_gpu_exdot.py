"""GPU parity of the exact dot (Sec. 2 exdot, Sec. 3.2) against the CPU oracle:
bit for bit on every input, at every length (empty, tiny, ragged tails, several
tiles, full 2^24 and 2^27 sizes), under every launch shape and window size,
run after run, through device and host pointers."""
import math
import os
import random

import numpy as np
import pytest

from gpu_common import bits, cuda_device, same
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


@pytest.fixture(scope="module")
def rbs(dev):
    import paper_2302_04180_gb300 as m
    yield m
    for k in ("exdot.grid", "exdot.block", "exdot.window"):
        m.rbs_set_param(k, 0)


def _gpu(rbs, dev, x, y):
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    yt = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    return rbs.rbs_exdot(xt, yt).item()


def _adversarial(rng, k):
    out = []
    for _ in range(k):
        kind = rng.randrange(6)
        if kind == 0:
            v = rng.uniform(-1, 1)
        elif kind == 1:
            v = math.ldexp(rng.uniform(1, 2), rng.randrange(-1070, 1020))
        elif kind == 2:
            v = math.ldexp(rng.randrange(1, 1 << 52), -1074)
        elif kind == 3:
            v = float(rng.randrange(-1000, 1000))
        elif kind == 4:
            v = math.ldexp(1.0, rng.randrange(-1074, 1023))
        else:
            v = math.ldexp(rng.uniform(1, 2), rng.randrange(-60, 60))
        out.append(-v if rng.random() < 0.5 else v)
    return np.array(out, dtype=np.float64)


def _golden(name):
    cases = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        xs, ys, e, cite = [t.strip() for t in line.split(";", 3)]
        conv = lambda t: float.fromhex(t) if "0x" in t else float(t)  # noqa: E731
        cases.append(([conv(t) for t in xs.split()], [conv(t) for t in ys.split()], conv(e), cite))
    return cases


@pytest.mark.parametrize("name", ["exdot_binary64_edges.txt", "exdot_nonfinite.txt"])
def test_golden(rbs, dev, orc, name):
    for x, y, e, cite in _golden(name):
        got = _gpu(rbs, dev, np.array(x), np.array(y))
        assert same(got, e), (x, y, got, e, cite)


def test_adversarial_small_vs_oracle(rbs, dev, orc):
    rng = random.Random(11)
    for trial in range(200):
        n = rng.randrange(0, 70)
        x, y = _adversarial(rng, n), _adversarial(rng, n)
        assert same(_gpu(rbs, dev, x, y), orc.exdot(x, y)), trial


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 32, 33, 255, 256, 257, 511, 513, 4095, 4097,
                               65537, (1 << 20) + 3])
def test_lengths_and_ragged_tails(rbs, dev, orc, n):
    x = gen.random_vector(n, 1, 1) * 10.0 ** gen.random_vector(n, 1, 2, -20, 20)
    y = gen.random_vector(n, 1, 3) * 10.0 ** gen.random_vector(n, 1, 4, -20, 20)
    assert same(_gpu(rbs, dev, x, y), orc.exdot(x, y))


@pytest.mark.parametrize("cond", [1e0, 1e16, 1e32, 1e48])
@pytest.mark.parametrize("n", [1 << 16, 1 << 20])
def test_ill_conditioned_vs_oracle_and_exact(rbs, dev, orc, n, cond):
    for seed in range(3):
        x, y, exact = gen.ill_conditioned_dot(n, cond, seed)
        got = _gpu(rbs, dev, x, y)
        assert same(got, orc.exdot(x, y)), (n, cond, seed)
        if exact is not None:
            assert same(got, float(exact)), (n, cond, seed)


def test_full_size_2_24_vs_oracle(rbs, dev, orc):
    x, y, exact = gen.ill_conditioned_dot(1 << 24, 1e32, 1)
    got = _gpu(rbs, dev, x, y)
    assert same(got, orc.exdot(x, y)) and same(got, float(exact))
    u, v, _ = gen.ill_conditioned_dot(1 << 24, 1e0, 1)
    assert same(_gpu(rbs, dev, u, v), orc.exdot(u, v))


def test_full_size_2_27_known_exact(rbs, dev):
    # 2 x 1 GiB operands; the exact value is known from the construction
    x, y, exact = gen.ill_conditioned_dot(1 << 27, 1e48, 2)
    assert same(_gpu(rbs, dev, x, y), float(exact))


def test_launch_shape_and_window_independence(rbs, dev, orc):
    x, y, _ = gen.ill_conditioned_dot(300007, 1e40, 4)
    ref = orc.exdot(x, y)
    import torch
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    seen = set()
    for window in (1, 2, 4):
        for block in (32, 96, 256):
            for grid in (1, 3, 152, 1217):
                rbs.rbs_set_param("exdot.window", window)
                rbs.rbs_set_param("exdot.block", block)
                rbs.rbs_set_param("exdot.grid", grid)
                seen.add(int(bits(rbs.rbs_exdot(xt, yt).item())))
    for k in ("exdot.grid", "exdot.block", "exdot.window"):
        rbs.rbs_set_param(k, 0)
    assert seen == {int(bits(ref))}


def test_long_dot_any_launch_shape(rbs, dev, orc):
    """Long dots (the shared-memory windows, n >= 2^23) under any launch shape:
    one block, a few blocks, whole waves and more blocks than fit at once, two
    block sizes; n odd. Every result is the oracle's, bit for bit."""
    import torch
    n = (1 << 23) + 13
    x, y, _ = gen.ill_conditioned_dot(n, 1e32, 11)
    ref = int(bits(orc.exdot(x, y)))
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    try:
        for block in (64, 256):
            for grid in (1, 5, 608, 1500):
                rbs.rbs_set_param("exdot.block", block)
                rbs.rbs_set_param("exdot.grid", grid)
                assert int(bits(rbs.rbs_exdot(xt, yt).item())) == ref, (block, grid)
    finally:
        rbs.rbs_set_param("exdot.grid", 0)
        rbs.rbs_set_param("exdot.block", 0)
    assert int(bits(rbs.rbs_exdot(xt, yt).item())) == ref


def test_run_to_run(rbs, dev, orc):
    import torch
    x, y, _ = gen.ill_conditioned_dot(1 << 21, 1e32, 7)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    vals = {int(bits(rbs.rbs_exdot(xt, yt).item())) for _ in range(25)}
    assert vals == {int(bits(orc.exdot(x, y)))}


def test_unaligned_views_and_host_pointers(rbs, dev, orc):
    import torch
    x, y, _ = gen.ill_conditioned_dot(100001, 1e20, 3)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    got = rbs.rbs_exdot(xt[1:], yt[1:]).item()  # 8-byte offset: scalar load path
    assert same(got, orc.exdot(x[1:], y[1:]))
    assert same(rbs.rbs_exdot(x, y), orc.exdot(x, y))  # numpy: host pointers, staged
    assert same(rbs.rbs_exdot(x, yt).item(), orc.exdot(x, y))  # mixed


def test_multi_output_with_shared_operands(rbs, dev, orc):
    import torch
    n = 200003
    vs = [gen.random_vector(n, 9, t) * 10.0 ** gen.random_vector(n, 9, t + 50, -30, 30) for t in range(5)]
    ts = [torch.from_numpy(v).to(dev) for v in vs]
    for k in range(1, 7):
        pairs = [(j % 5, (j * 3 + 1) % 5) for j in range(k)]
        out = rbs.rbs_exdot_multi([ts[a] for a, _ in pairs], [ts[b] for _, b in pairs]).cpu().numpy()
        for j, (a, b) in enumerate(pairs):
            assert same(out[j], orc.exdot(vs[a], vs[b])), (k, j)


def test_partial_limbs_integer_sum_then_round(rbs, dev, orc):
    """Row-block ranks (Sec. 3.2) emulated on one GPU: each block's limbs are
    summed as plain integers, in any order, and rounded once."""
    import torch
    x, y, exact = gen.ill_conditioned_dot(400009, 1e44, 6)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    cuts = [0, 1, 77777, 200000, 333333, 400009]
    total = torch.zeros(136, dtype=torch.int64, device=dev)
    fl = 0
    for a, b in reversed(list(zip(cuts[:-1], cuts[1:]))):
        limbs, flags = rbs.rbs_exdot_partial(xt[a:b].contiguous(), yt[a:b].contiguous())
        total += limbs
        fl |= int(flags.item())
        # each rank's limbs alone round to that rank's exact dot
        assert same(rbs.rbs_round_limbs(limbs, flags).item(), orc.exdot(x[a:b], y[a:b]))
    ft = torch.tensor([fl], dtype=torch.int32, device=dev)
    got = rbs.rbs_round_limbs(total, ft).item()
    assert same(got, orc.exdot(x, y)) and same(got, float(exact))


def test_nonfinite_inside_long_vectors(rbs, dev, orc):
    x = gen.random_vector(10001, 2, 1)
    y = gen.random_vector(10001, 2, 2)
    for pos, xv, yv in ((5000, np.inf, 0.0), (17, np.nan, 1.0), (9999, np.inf, -2.0)):
        xx, yy = x.copy(), y.copy()
        xx[pos], yy[pos] = xv, yv
        assert same(_gpu(rbs, dev, xx, yy), orc.exdot(xx, yy))


def test_long_dots_take_the_shared_window_path(rbs, dev, orc):
    """Dots of at least 2^23 elements keep one or two outputs' windows in
    shared memory: single, two-output and limb-export results against the
    oracle, with a ragged tail, a wide exponent spread and non-finite values."""
    import torch
    n = (1 << 23) + 3
    x, y, exact = gen.ill_conditioned_dot(n, 1e40, 11)
    w = gen.random_vector(n, 12, 3) * 10.0 ** gen.random_vector(n, 12, 4, -150, 150)
    xt, yt, wt = (torch.from_numpy(v).to(dev) for v in (x, y, w))
    assert same(rbs.rbs_exdot(xt, yt).item(), float(exact))
    two = rbs.rbs_exdot_multi([xt, wt], [yt, wt]).cpu().numpy()
    assert same(two[0], float(exact)) and same(two[1], orc.exdot(w, w))
    limbs, flags = rbs.rbs_exdot_partial(wt, yt)
    assert same(rbs.rbs_round_limbs(limbs, flags).item(), orc.exdot(w, y))
    ww = w.copy()
    ww[n // 2] = np.inf
    assert same(rbs.rbs_exdot(torch.from_numpy(ww).to(dev), yt).item(), orc.exdot(ww, y))
