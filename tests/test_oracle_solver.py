"""Pins for the oracle's SpMV, Jacobi and PBiCGStab loops (Fig. 2, Fig. 4).

The C oracle is checked against the independent pure-Python Fraction oracle
(bitwise whole histories), against exact-rational runs of both figures
(classic and pipelined produce identical alpha/omega/beta in exact arithmetic),
and against closed forms: manufactured solutions, a diagonal system that
converges in one step, constructed breakdowns and input errors.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2302_04180_gb300 import gen
from oracle import fraction_ref as fr


def _bits(a):
    return np.asarray(a, dtype=np.float64).view(np.uint64)


def _csr_from_dense(M):
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    rowptr = [0]
    col, val = [], []
    for i in range(n):
        for j in range(n):
            if M[i, j] != 0.0:
                col.append(j)
                val.append(M[i, j])
        rowptr.append(len(col))
    return gen.CSR(n, np.array(rowptr, dtype=np.int64), np.array(col, dtype=np.int32),
                   np.array(val, dtype=np.float64), "dense")


# ---- SpMV / Jacobi -----------------------------------------------------------

def test_spmv_matches_fraction_fma_chain(orc):
    for seed, (n, mr) in enumerate([(1, 1), (17, 5), (64, 9), (200, 3)]):
        A = gen.random_csr(n, mr, seed, empty_frac=0.2, dup_frac=0.3)
        x = gen.random_vector(n, seed, tag=9) * 10.0 ** gen.random_vector(n, seed, 10, -5, 5)
        x[::7] = -0.0
        got = orc.spmv(A, x)
        ref = fr.spmv(A.n, A.rowptr, A.col, A.val, x.tolist())
        assert (_bits(got) == _bits(ref)).all()


def test_spmv_empty_row_is_plus_zero(orc):
    A = gen.CSR(3, np.array([0, 0, 1, 1], dtype=np.int64), np.array([0], dtype=np.int32),
                np.array([-1.0]), "t")
    y = orc.spmv(A, np.array([0.0, 1.0, 2.0]))
    assert (_bits(y) == _bits([0.0, -0.0 * 0 + 0.0, 0.0])).all()  # -1*0 + (+0) = +0
    assert not np.signbit(y).any()


def test_poisson_rowsums_are_exact_integers(orc):
    N = 6
    A = gen.poisson3d(N)
    assert A.nnz == N ** 3 + 6 * (N - 1) * N * N
    b = orc.spmv(A, np.ones(A.n))
    idx = np.arange(A.n)
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    nb = (i > 0).astype(int) + (i < N - 1) + (j > 0) + (j < N - 1) + (k > 0) + (k < N - 1)
    assert (b == 6.0 - nb).all()


def test_jacobi_is_reciprocal_then_multiply(orc):
    A = gen.convdiff3d(5, 10.0)
    invd = orc.jacobi_invd(A)
    d = np.array([A.val[A.rowptr[i]:A.rowptr[i + 1]][A.col[A.rowptr[i]:A.rowptr[i + 1]] == i][0]
                  for i in range(A.n)])
    assert (_bits(invd) == _bits(1.0 / d)).all()
    p = gen.random_vector(A.n, 1)
    assert (_bits(orc.jacobi_apply(invd, p)) == _bits(p * invd)).all()
    with pytest.raises(ValueError):
        orc.jacobi_invd(A, diag=np.zeros(A.n))


# ---- solvers: C oracle == Fraction oracle --------------------------------------

SYSTEMS = [
    ("poisson4", lambda: gen.poisson3d(4)),
    ("convdiff4", lambda: gen.convdiff3d(4, 10.0)),
    ("convdiff2d6", lambda: gen.convdiff2d(6, 30.0, (0.3, -1.0))),
    ("random30", lambda: gen.random_csr(30, 6, 4, diag_dominant=True)),
]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("name,make", SYSTEMS)
def test_c_oracle_matches_fraction_oracle(orc, name, make, variant):
    A = make()
    b = orc.spmv(A, np.ones(A.n))
    assert (_bits(b) == _bits(fr.spmv(A.n, A.rowptr, A.col, A.val, [1.0] * A.n))).all()
    tol = 1e-10
    c = orc.solve(A, b, tol=tol, maxit=200, variant=variant)
    p = fr.solve(A, b, tol, 200, variant)
    assert c["status"] == p["status"] == 0
    assert c["iters"] == p["iters"] > 0
    assert c["converged"] == p["converged"] == 1
    assert _bits(c["tau0"]) == _bits(p["tau0"])
    assert (_bits(c["hist"]) == _bits(np.array(p["hist"]))).all()
    assert (_bits(c["x"]) == _bits(p["x"])).all()


@pytest.mark.parametrize("variant", [0, 1])
def test_c_oracle_matches_fraction_oracle_with_x0(orc, variant):
    A = gen.convdiff3d(4, 25.0, (1.0, -0.5, 0.25))
    b = gen.random_vector(A.n, 8)
    x0 = gen.random_vector(A.n, 9)
    c = orc.solve(A, b, x0=x0, tol=1e-9, maxit=100, variant=variant)
    p = fr.solve(A, b, 1e-9, 100, variant, x0=x0.tolist())
    assert c["iters"] == p["iters"] and c["status"] == p["status"]
    assert (_bits(c["hist"]) == _bits(np.array(p["hist"]))).all()
    assert (_bits(c["x"]) == _bits(p["x"])).all()


# ---- exact-rational equivalence of Fig. 2 and Fig. 4 --------------------------

def _exact_runs(M, b, iters):
    """Run both figures in exact rational arithmetic, no rounding anywhere."""
    n = len(b)
    A = [[Fraction(v) for v in row] for row in M]
    dinv = [1 / A[i][i] for i in range(n)]
    mv = lambda v: [sum(A[i][j] * v[j] for j in range(n)) for i in range(n)]  # noqa
    jac = lambda v: [v[i] * dinv[i] for i in range(n)]  # noqa
    dot = lambda u, v: sum(a * c for a, c in zip(u, v))  # noqa
    b = [Fraction(t) for t in b]
    # classic
    r = list(b); r0 = list(r); p = list(r); x = [Fraction(0)] * n
    rho = dot(r0, r)
    cls = []
    for _ in range(iters):
        ph = jac(p); s = mv(ph); alpha = rho / dot(r0, s)
        q = [r[i] - alpha * s[i] for i in range(n)]
        qh = jac(q); y = mv(qh); omega = dot(q, y) / dot(y, y)
        x = [x[i] + alpha * ph[i] + omega * qh[i] for i in range(n)]
        r = [q[i] - omega * y[i] for i in range(n)]
        rho1 = dot(r0, r); beta = (rho1 / rho) * (alpha / omega)
        p = [r[i] + beta * (p[i] - omega * s[i]) for i in range(n)]
        cls.append((alpha, omega, beta)); rho = rho1
    # pipelined
    r = list(b); r0 = list(r); x = [Fraction(0)] * n
    rh = jac(r); w = mv(rh); wh = jac(w); t = mv(wh)
    rho = dot(r0, r); alpha = rho / dot(r0, w); beta = Fraction(0); omega = Fraction(0)
    ph = s = sh = z = zh = v = [Fraction(0)] * n
    pip = []
    for _ in range(iters):
        ph = [rh[i] + beta * (ph[i] - omega * sh[i]) for i in range(n)]
        s_new = [w[i] + beta * (s[i] - omega * z[i]) for i in range(n)]
        sh = [wh[i] + beta * (sh[i] - omega * zh[i]) for i in range(n)]
        z = [t[i] + beta * (z[i] - omega * v[i]) for i in range(n)]
        s = s_new
        q = [r[i] - alpha * s[i] for i in range(n)]
        qh = [rh[i] - alpha * sh[i] for i in range(n)]
        y = [w[i] - alpha * z[i] for i in range(n)]
        zh = jac(z); v = mv(zh)
        omega = dot(q, y) / dot(y, y)
        x = [x[i] + alpha * ph[i] + omega * qh[i] for i in range(n)]
        r = [q[i] - omega * y[i] for i in range(n)]
        rh = [qh[i] - omega * (wh[i] - alpha * zh[i]) for i in range(n)]
        w = [y[i] - omega * (t[i] - alpha * v[i]) for i in range(n)]
        rho1 = dot(r0, r); a = dot(r0, w); c = dot(r0, s); e = dot(r0, z)
        wh = jac(w); t = mv(wh)
        beta_new = (rho1 / rho) * (alpha / omega)
        pip.append((alpha, omega, beta_new))
        alpha = rho1 / (a + beta_new * c - beta_new * omega * e)
        beta = beta_new; rho = rho1
    return cls, pip


def test_fig2_and_fig4_agree_in_exact_arithmetic():
    M = [[4, -1, 0, 0.5, 0, 0], [-2, 5, -1, 0, 0, 0], [0, -1, 6, -2, 0, 1],
         [1, 0, -1, 4, -1, 0], [0, 0, 0, -3, 5, -1], [0, 0.5, 0, 0, -1, 3]]
    b = [1, 2, -1, 0.5, 3, -2]
    cls, pip = _exact_runs(M, b, 4)
    assert cls == pip


def test_fraction_oracle_follows_exact_run_for_one_step(orc):
    """First-iteration scalars of the rounded oracle sit within a few ulps of
    the exact-rational run (a dropped term or wrong sign would not)."""
    M = np.array([[4, -1, 0, 0.5, 0, 0], [-2, 5, -1, 0, 0, 0], [0, -1, 6, -2, 0, 1],
                  [1, 0, -1, 4, -1, 0], [0, 0, 0, -3, 5, -1], [0, 0.5, 0, 0, -1, 3]], float)
    b = np.array([1, 2, -1, 0.5, 3, -2], float)
    A = _csr_from_dense(M)
    cls, pip = _exact_runs(M.tolist(), b.tolist(), 2)
    for variant in (0, 1):
        c = orc.solve(A, b, tol=1e-300, maxit=2, variant=variant)
        h = c["hist"]
        ia, io, ib = (1, 4, 8) if variant == 0 else (None, 2, 9)
        for j in range(2):
            alpha_c = h[j][ia] if ia is not None else (c["alpha0"] if j == 0 else h[j - 1][11])
            for got, ex in ((alpha_c, cls[j][0]), (h[j][io], cls[j][1]), (h[j][ib], cls[j][2])):
                # rounding error grows per step; a transcription slip is O(1) off
                assert abs(Fraction(got) - ex) <= abs(ex) * Fraction(1, 2 ** (44 - 8 * j)), (variant, j)


# ---- closed forms ----------------------------------------------------------------

@pytest.mark.parametrize("variant", [0, 1])
def test_manufactured_solution_poisson(orc, variant):
    A = gen.poisson3d(10)
    b = orc.spmv(A, np.ones(A.n))
    c = orc.solve(A, b, tol=1e-12, maxit=1000, variant=variant)
    assert c["status"] == 0 and c["converged"] == 1
    # kappa(A) ~ 50 here; 1e-12 relative residual -> x within ~1e-10 of ones
    assert np.max(np.abs(c["x"] - 1.0)) < 1e-9
    # the recursive residual tracks the true residual
    true_r = b - orc.spmv(A, c["x"])
    assert np.linalg.norm(true_r) <= 100 * c["tau_final"] + 1e-300


@pytest.mark.parametrize("variant", [0, 1])
def test_diagonal_system_converges_in_one_step(orc, variant):
    n = 16
    d = 2.0 ** np.arange(-4, 12, dtype=np.float64)
    A = gen.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d, "diag")
    b = gen.random_vector(n, 3)
    c = orc.solve(A, b, tol=1e-14, maxit=50, variant=variant)
    assert c["status"] == 0 and c["converged"] == 1 and c["iters"] == 1
    assert (c["x"] == b / d).all()
    assert c["tau_final"] == 0.0


def test_breakdown_sigma_zero(orc):
    # <r0, A D^-1 r0> = 0 for A = [[1,0],[-2,1]], r0 = b = (1,1)
    A = _csr_from_dense([[1.0, 0.0], [-2.0, 1.0]])
    c = orc.solve(A, np.array([1.0, 1.0]), tol=1e-8, maxit=10, variant=0)
    assert c["status"] == 4 and c["iters"] == 0 and c["converged"] == 0
    p = fr.solve(A, [1.0, 1.0], 1e-8, 10, 0)
    assert p["status"] == 4 and p["iters"] == 0


def test_breakdown_mu_zero_pipelined(orc):
    A = _csr_from_dense([[1.0, 0.0], [-2.0, 1.0]])
    c = orc.solve(A, np.array([1.0, 1.0]), tol=1e-8, maxit=10, variant=1)
    assert c["status"] == 4 and c["iters"] == 0


@pytest.mark.parametrize("variant", [0, 1])
def test_input_errors_and_trivial_cases(orc, variant):
    A = gen.poisson3d(3)
    b = np.ones(A.n)
    assert orc.solve(A, b, diag=np.zeros(A.n), variant=variant)["status"] == 1
    z = orc.solve(A, np.zeros(A.n), variant=variant)
    assert z["status"] == 0 and z["iters"] == 0 and z["converged"] == 1
    assert not np.signbit(z["x"]).any() and (z["x"] == 0).all()
    m0 = orc.solve(A, b, maxit=0, variant=variant)
    assert m0["iters"] == 0 and m0["converged"] == 0 and m0["status"] == 0
    bn = b.copy()
    bn[3] = np.nan
    assert orc.solve(A, bn, variant=variant)["status"] == 5
    m3 = orc.solve(A, orc.spmv(A, np.ones(A.n)), tol=1e-14, maxit=3, variant=variant)
    assert m3["iters"] == 3 and m3["converged"] == 0 and m3["status"] == 0
