"""The seeded input generators, pinned to their definitions (CPU only).

Both the GPU parity tests and the oracle's tests draw their inputs from
``gen``, so these checks pin it to things other than itself:
- the published SplitMix64 output sequence;
- brute-force stencil constructions;
- closed-form nonzero counts;
- the exact rational sum for the ill-conditioned dots.
"""
import numpy as np
import pytest

from paper_2302_04180_gb300 import gen

# SplitMix64 (Steele, Lea & Flood 2014) from seed 0: the first outputs of the
# reference generator, as published with Vigna's splitmix64.c.
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                    0x1B39896A51A8749B]


def test_splitmix64_matches_the_published_sequence():
    assert [int(v) for v in gen.splitmix64(0, 5)] == SPLITMIX64_SEED0


def test_splitmix64_is_counter_based():
    long = gen.splitmix64(7, 1000)
    assert np.array_equal(gen.splitmix64(7, 100, start=450), long[450:550])
    # stream s is the seed-0 sequence from word s * 2^32 on
    assert np.array_equal(gen.splitmix64(3, 4, start=10), gen.splitmix64(0, 4, start=(3 << 32) + 10))
    assert not np.array_equal(gen.splitmix64(1, 16), gen.splitmix64(2, 16))


def test_uniform_has_53_bits_in_unit_interval():
    u = gen.uniform(5, 4096)
    assert u.dtype == np.float64 and np.all(u >= 0.0) and np.all(u < 1.0)
    assert np.all(np.ldexp(u, 53) == np.floor(np.ldexp(u, 53)))
    assert abs(u.mean() - 0.5) < 0.02


def _dense(A):
    D = np.zeros((A.n, A.n))
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            D[i, A.col[k]] += A.val[k]
    return D


def _ascending(A):
    for i in range(A.n):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        if np.any(np.diff(c) <= 0):
            return False
    return True


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_poisson3d_is_the_7_point_laplacian(N):
    A = gen.poisson3d(N)
    n = N ** 3
    assert A.n == n and A.nnz == n + 6 * (N - 1) * N * N
    ref = np.zeros((n, n))
    for k in range(N):
        for j in range(N):
            for i in range(N):
                r = i + N * j + N * N * k
                ref[r, r] = 6.0
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    a, b, c = i + di, j + dj, k + dk
                    if 0 <= a < N and 0 <= b < N and 0 <= c < N:
                        ref[r, a + N * b + N * N * c] = -1.0
    assert np.array_equal(_dense(A), ref)
    assert _ascending(A)


def test_convdiff3d_upwinding():
    N, Pe = 5, 20.0
    A = gen.convdiff3d(N, Pe, direction=(1.0, -2.0, 0.5))
    D = _dense(A)
    assert _ascending(A)
    assert not np.array_equal(D, D.T)  # convection makes it unsymmetric
    centre = 2 + N * 2 + N * N * 2  # an interior point: diffusion + upwind sum to a zero row
    assert abs(D[centre].sum()) < 1e-12
    d = np.array([1.0, -2.0, 0.5]) / np.sqrt(5.25)
    h = 1.0 / (N + 1)
    for m, stride in enumerate((1, N, N * N)):
        P = Pe * h * abs(d[m])
        up, down = (centre - stride, centre + stride) if d[m] > 0 else (centre + stride, centre - stride)
        assert D[centre, up] == -(1.0 + P) and D[centre, down] == -1.0
    assert np.all(np.diag(D) > 0)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_stencil27_counts_and_values(N):
    A = gen.stencil27(N, perturb=1e-4)
    assert A.n == N ** 3 and A.nnz == (3 * N - 2) ** 3
    assert _ascending(A)
    D = _dense(A)
    assert np.all(np.diag(D) == 26.0)
    lower = D[np.tril_indices(A.n, -1)]
    upper = D[np.triu_indices(A.n, 1)]
    assert set(np.unique(lower)) <= {0.0, -(1.0 - 1e-4)}
    assert set(np.unique(upper)) <= {0.0, -1.0}
    if N >= 3:  # an interior point has all 26 neighbours
        c = 1 + N + N * N
        assert A.rowptr[c + 1] - A.rowptr[c] == 27


@pytest.mark.parametrize("n,band", [(1, 0), (10, 3), (50, 7), (7, 10)])
def test_banded_counts_and_values(n, band):
    A = gen.banded(n, band)
    b = min(band, n - 1)
    assert A.nnz == (2 * b + 1) * n - b * (b + 1)
    assert _ascending(A)
    D = _dense(A)
    for i in range(n):
        for j in range(n):
            if i == j:
                assert D[i, j] == 2 * band + 1
            elif abs(i - j) <= band:
                assert D[i, j] == (-(1.0 - 1e-4) if j < i else -1.0)
            else:
                assert D[i, j] == 0.0


@pytest.mark.parametrize("cond", [1e16, 1e32, 1e48])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 10, 301])
def test_ill_conditioned_dot_exact_value_is_the_rational_sum(cond, n):
    from fractions import Fraction
    for seed in range(3):
        x, y, exact = gen.ill_conditioned_dot(n, cond, seed)
        assert x.size == n and y.size == n and np.all(np.isfinite(x)) and np.all(np.isfinite(y))
        assert sum(Fraction(a) * Fraction(b) for a, b in zip(x.tolist(), y.tolist())) == exact
        assert exact != 0


def test_full_size_digests_are_complete():
    """The stored oracle digests of the full-size solves (written by
    tests/golden/make_c3_digests.py) list every iteration's tau and converge."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_c3_digests as D
    for name in D.WORKLOADS:
        d = D.read(name)
        it = int(d["iters"])
        assert it > 100 and int(d["status"]) == 0 and int(d["converged"]) == 1
        assert sorted(d["tau"]) == list(range(it))
        assert len(d["history_sha256"]) == 64 and len(d["x_sha256"]) == 64
        # tau falls below tau_max exactly at the last iteration (the stop test)
        tau = [np.array([int(d["tau"][j], 16)], dtype=np.uint64).view(np.float64)[0] for j in range(it)]
        tmax = np.array([int(d["tau_max"], 16)], dtype=np.uint64).view(np.float64)[0]
        assert tau[-1] <= tmax and all(t > tmax for t in tau[:-1])
