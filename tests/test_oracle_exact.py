"""Pins for the oracle's error-free transformations and exact dot.

Each check ties the oracle to something other than itself: exact rationals
(fractions.Fraction), the correctly rounded library sum math.fsum, closed-form
cases (unit vectors, small integers, constructed cancellation), invariants
(permutation, sign flip, rank splitting) and the hand-derived binary64 edge
cases of tests/golden (Table 1 and the IEEE rounding definition).
"""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from paper_2302_04180_gb300 import gen
from oracle import fraction_ref as fr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bits(v: float) -> int:
    return int(np.float64(v).view(np.uint64))


def _same(a: float, b: float) -> bool:
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return _bits(a) == _bits(b)


def _load_golden(name):
    cases = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            xs, ys, exp, cite = [t.strip() for t in line.split(";", 3)]
            x = [float.fromhex(t) if "0x" in t else float(t) for t in xs.split()]
            y = [float.fromhex(t) if "0x" in t else float(t) for t in ys.split()]
            e = float.fromhex(exp) if "0x" in exp else float(exp)
            cases.append((x, y, e, cite))
    return cases


def _rn_fraction(q: Fraction) -> float:
    if q == 0:
        return 0.0
    try:
        v = float(q)
    except OverflowError:
        return math.inf if q > 0 else -math.inf
    if v == 0.0:
        return -0.0 if q < 0 else 0.0
    return v


def _adversarial_doubles(rng: random.Random, k: int):
    out = []
    for _ in range(k):
        kind = rng.randrange(6)
        if kind == 0:
            v = rng.uniform(-1, 1)
        elif kind == 1:
            v = math.ldexp(rng.uniform(1, 2), rng.randrange(-1070, 1020))
        elif kind == 2:  # subnormal
            v = math.ldexp(rng.randrange(1, 1 << 52), -1074)
        elif kind == 3:
            v = float(rng.randrange(-1000, 1000))
        elif kind == 4:
            v = math.ldexp(1.0, rng.randrange(-1074, 1023))
        else:
            v = math.ldexp(rng.uniform(1, 2), rng.randrange(-60, 60))
        out.append(-v if rng.random() < 0.5 else v)
    return out


# ---- Alg. 1 / Alg. 2 ---------------------------------------------------------

def test_twosum_twoprod_are_error_free(orc):
    rng = random.Random(1)
    for _ in range(4000):
        a = math.ldexp(rng.uniform(-2, 2), rng.randrange(-200, 200))
        b = math.ldexp(rng.uniform(-2, 2), rng.randrange(-200, 200))
        r, s = orc.twosum(a, b)
        assert r == a + b  # r is the rounded sum
        assert Fraction(r) + Fraction(s) == Fraction(a) + Fraction(b)
        r, s = orc.twoprod(a, b)
        assert r == a * b
        assert Fraction(r) + Fraction(s) == Fraction(a) * Fraction(b)


def test_build_does_not_contract(orc):
    # (1+2^-30)(1-2^-30) = 1 - 2^-60 rounds to 1; a contracted fma would give -2^-60
    assert orc.mul_add_unfused(1 + 2**-30, 1 - 2**-30, -1.0) == 0.0
    r, s = orc.twoprod(1 + 2**-30, 1 - 2**-30)
    assert s == -(2.0 ** -60)


# ---- exdot pins --------------------------------------------------------------

@pytest.mark.parametrize("name", ["exdot_binary64_edges.txt", "exdot_nonfinite.txt"])
def test_golden_edges(orc, name):
    cases = _load_golden(name)
    assert len(cases) >= 6
    for x, y, e, cite in cases:
        got = orc.exdot(np.array(x), np.array(y))
        assert _same(got, e), (x, y, got, e, cite)


def test_exdot_matches_fraction_bruteforce(orc):
    rng = random.Random(7)
    for trial in range(300):
        n = rng.randrange(0, 40)
        x = _adversarial_doubles(rng, n)
        y = _adversarial_doubles(rng, n)
        exact = sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0))
        got = orc.exdot(np.array(x, dtype=np.float64), np.array(y, dtype=np.float64))
        assert _same(got, _rn_fraction(exact)), (trial, x, y)
        assert _same(fr.exdot(x, y), got)


def test_exdot_against_fsum_of_exact_product_splits(orc):
    # math.fsum is correctly rounded; r_i + s_i = x_i y_i exactly (s_i computed
    # as an exact rational, products kept away from underflow)
    x = gen.random_vector(1 << 14, seed=3, tag=1, lo=-1e3, hi=1e3)
    y = gen.random_vector(1 << 14, seed=3, tag=2, lo=-1e-3, hi=1e-3)
    parts = []
    for a, b in zip(x.tolist(), y.tolist()):
        r = a * b
        s = float(Fraction(a) * Fraction(b) - Fraction(r))
        assert Fraction(r) + Fraction(s) == Fraction(a) * Fraction(b)
        parts += [r, s]
    assert _same(orc.exdot(x, y), math.fsum(parts))


def test_exdot_ones_is_correctly_rounded_sum(orc):
    for seed in range(4):
        x = gen.random_vector(5000, seed=seed, tag=3) * 10.0 ** gen.random_vector(5000, seed, 4, -8, 8)
        assert _same(orc.exdot(x, np.ones_like(x)), math.fsum(x.tolist()))
        assert _same(orc.exsum(x), math.fsum(x.tolist()))


def test_exdot_unit_vector_and_integers(orc):
    x = gen.random_vector(257, seed=5, tag=1) * 1e200
    for k in (0, 1, 100, 256):
        e = np.zeros(257)
        e[k] = 1.0
        assert _same(orc.exdot(x, e), x[k])
    a = (gen.splitmix64(11, 3000) % np.uint64(2001)).astype(np.int64) - 1000
    b = (gen.splitmix64(12, 3000) % np.uint64(2001)).astype(np.int64) - 1000
    assert orc.exdot(a.astype(np.float64), b.astype(np.float64)) == float(int(np.dot(a, b)))


def test_exdot_permutation_and_sign_invariance(orc):
    x, y, _ = gen.ill_conditioned_dot(999, 1e20, seed=2)
    ref = orc.exdot(x, y)
    for seed in range(5):
        perm = np.argsort(gen.splitmix64(50 + seed, x.size), kind="stable")
        assert _same(orc.exdot(x[perm], y[perm]), ref)
    neg = orc.exdot(-x, y)
    assert _same(neg, -ref) or (ref == 0.0 and neg == 0.0)
    assert _same(orc.exdot(y, x), ref)


@pytest.mark.parametrize("cond", [1e16, 1e32, 1e48])
@pytest.mark.parametrize("n", [2, 3, 10, 1001, 1 << 16])
def test_exdot_ill_conditioned_known_exact(orc, cond, n):
    for seed in range(3):
        x, y, exact = gen.ill_conditioned_dot(n, cond, seed)
        assert x.size == n
        got = orc.exdot(x, y)
        assert _same(got, _rn_fraction(exact)), (n, cond, seed)
        # the naive float sum is visibly wrong at these conditions
        if n >= 1001 and cond >= 1e32:
            assert float(np.dot(x, y)) != got


def test_ill_conditioned_generator_reaches_condition(orc):
    for cond in (1e16, 1e32, 1e48):
        x, y, exact = gen.ill_conditioned_dot(4000, cond, 0)
        absum = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(x.tolist(), y.tolist()))
        c = float(2 * absum / abs(exact))
        assert cond / 16 < c < cond * 16, (cond, c)


def test_rank_split_integer_reduction_equals_single(orc):
    """Sec. 3.2: ranks reduce long accumulators as plain integer arrays (any
    order, any split), normalise once and round once: bitwise the 1-rank result."""
    x, y, exact = gen.ill_conditioned_dot(5000, 1e32, 1)
    ref = orc.exdot(x, y)
    rng = random.Random(3)
    for K in (1, 2, 3, 4, 7, 16, 28):
        cuts = sorted(rng.sample(range(1, x.size), K - 1)) if K > 1 else []
        bounds = [0] + cuts + [x.size]
        parts = [orc.exdot_limbs(x[a:b], y[a:b]) for a, b in zip(bounds[:-1], bounds[1:])]
        rng.shuffle(parts)
        total = np.zeros_like(parts[0][0])
        flags = 0
        for limbs, fl in parts:
            total += limbs
            flags |= fl
        assert _same(orc.round_limbs(total, flags), ref)
    assert _same(ref, _rn_fraction(exact))


def test_exdot_empty_and_zero(orc):
    assert _same(orc.exdot(np.zeros(0), np.zeros(0)), 0.0)
    assert _same(orc.exdot(np.array([-0.0, 0.0]), np.array([1.0, -1.0])), 0.0)


def test_fma_vec_is_one_rounding(orc):
    """orc_fma_vec: fma(a, x_i, y_i) is the exact a*x_i + y_i rounded once
    (checked against exact rationals, including cases where the unfused
    a*x + y rounds differently)."""
    rng = random.Random(11)
    xs, ys, avals = [], [], []
    for _ in range(400):
        a = rng.uniform(-3, 3)
        x = rng.uniform(-1, 1) * 2.0 ** rng.randrange(-30, 30)
        y = -float(Fraction(a) * Fraction(x)) * (1 + rng.choice((0.0, 2.0 ** -52, -2.0 ** -53)))
        xs.append(x), ys.append(y), avals.append(a)
    differs = 0
    for a, x, y in zip(avals, xs, ys):
        got = orc.fma_vec(a, np.array([x]), np.array([y]))[0]
        want = _rn_fraction(Fraction(a) * Fraction(x) + Fraction(y))
        assert np.float64(got).view(np.uint64) == np.float64(want).view(np.uint64)
        differs += orc.mul_add_unfused(a, x, y) != got
    assert differs > 50
