"""Second, independent CPU oracle in pure Python with exact rationals.

TEST INFRASTRUCTURE ONLY. It pins the C oracle: it shares no code with it (or
with the GPU library) and computes every rounding from its definition:
fma(a, b, c) = RN(a*b + c) with the exact value taken as a Fraction and
rounded by ``float(Fraction)`` (CPython rounds integer ratios correctly, to
nearest even); the dot is RN of the exact Fraction sum (Sec. 2, Sec. 3.2).
Plain float *, / and math.sqrt are IEEE-754 correctly rounded.

It is slow (tiny systems only) and follows Fig. 2 and Fig. 4 with the same
readings as the C oracle (listed in oracle/solver.c).
"""
from __future__ import annotations

import math
import struct
from fractions import Fraction

QNAN = struct.unpack("<d", struct.pack("<Q", 0x7FF8000000000000))[0]


def _rn(q: Fraction, neg_hint: bool) -> float:
    """Round an exact rational to binary64 (nearest even). A zero exact value
    takes the sign neg_hint (IEEE zero-sum rule, decided by the caller)."""
    if q == 0:
        return -0.0 if neg_hint else 0.0
    try:
        v = float(q)
    except OverflowError:
        return math.inf if q > 0 else -math.inf
    if v == 0.0:  # a nonzero value that underflows keeps its sign
        return -0.0 if q < 0 else 0.0
    return v


def _signbit(v: float) -> bool:
    return math.copysign(1.0, v) < 0


def fma(a: float, b: float, c: float) -> float:
    """IEEE fma for finite operands: RN(a*b + c) with one rounding."""
    prod = Fraction(a) * Fraction(b)
    q = prod + Fraction(c)
    if q == 0:
        # exact zero: -0 only if both addends are zeros of negative sign
        pneg = _signbit(a) != _signbit(b)
        if prod == 0 and c == 0:
            return -0.0 if (pneg and _signbit(c)) else 0.0
        return 0.0
    return _rn(q, False)


def exdot(x, y) -> float:
    """RN(sum x_i y_i) with the sum exact; an exact zero gives +0.0."""
    s = Fraction(0)
    for a, b in zip(x, y):
        s += Fraction(a) * Fraction(b)
    return _rn(s, False)


def spmv(n, rowptr, col, val, x):
    """y_i = fma(a_last, x_last, ... fma(a_0, x_0, +0.0)) in stored order."""
    y = [0.0] * n
    for i in range(n):
        acc = 0.0
        for k in range(int(rowptr[i]), int(rowptr[i + 1])):
            acc = fma(float(val[k]), float(x[int(col[k])]), acc)
        y[i] = acc
    return y


def _diag(n, rowptr, col, val):
    d = []
    for i in range(n):
        v = None
        for k in range(int(rowptr[i]), int(rowptr[i + 1])):
            if int(col[k]) == i:
                v = float(val[k])
                break
        if v is None or v == 0.0:
            raise ValueError("zero or missing diagonal")
        d.append(v)
    return d


def solve(A, b, tol, maxit, variant, x0=None):
    """Classic (variant 0, Fig. 2) or pipelined (variant 1, Fig. 4) PBiCGStab.
    Returns dict(x, iters, converged, status, tau0, hist) with hist a list of
    12-field records in the C oracle's layout."""
    n = A.n
    rowptr, col, val = A.rowptr, A.col, A.val
    invd = [1.0 / d for d in _diag(n, rowptr, col, val)]
    jac = lambda v: [v[i] * invd[i] for i in range(n)]  # noqa: E731
    mv = lambda v: spmv(n, rowptr, col, val, v)  # noqa: E731
    bl = [float(t) for t in b]
    if x0 is not None:
        x = [float(t) for t in x0]
        ax = mv(x)
        r = [bl[i] - ax[i] for i in range(n)]
    else:
        x = [0.0] * n
        r = list(bl)
    r0 = list(r)
    hist = []
    status = 0
    if variant == 0:
        p = list(r)
        rho = exdot(r0, r)
        tau = math.sqrt(rho)
        tau_max = tol * tau
        tau0 = tau
        j = 0
        while tau > tau_max and j < maxit:
            rec = [QNAN] * 12
            ph = jac(p)
            s = mv(ph)
            sigma = exdot(r0, s)
            if sigma == 0.0:
                status = 4
                break
            alpha = rho / sigma
            q = [fma(-alpha, s[i], r[i]) for i in range(n)]
            qh = jac(q)
            y = mv(qh)
            gamma = exdot(q, y)
            delta = exdot(y, y)
            omega = 0.0 if delta == 0.0 else gamma / delta
            x = [fma(omega, qh[i], fma(alpha, ph[i], x[i])) for i in range(n)]
            r = [fma(-omega, y[i], q[i]) for i in range(n)]
            rho1 = exdot(r0, r)
            theta = exdot(r, r)
            tau = math.sqrt(theta)
            j += 1
            rec[0:8] = [sigma, alpha, gamma, delta, omega, rho1, theta, tau]
            if not (tau > tau_max):
                hist.append(rec)
                break
            if omega == 0.0 or rho1 == 0.0:
                hist.append(rec)
                status = 4
                break
            beta = (rho1 / rho) * (alpha / omega)
            rec[8] = beta
            hist.append(rec)
            p = [fma(beta, fma(-omega, s[i], p[i]), r[i]) for i in range(n)]
            rho = rho1
        return dict(x=x, iters=j, converged=int(status == 0 and not (tau > tau_max)),
                    status=status, tau0=tau0, hist=hist)

    # pipelined
    rh = jac(r)
    w = mv(rh)
    wh = jac(w)
    t = mv(wh)
    rho = exdot(r0, r)
    mu = exdot(r0, w)
    tau = math.sqrt(rho)
    tau_max = tol * tau
    tau0 = tau
    alpha = beta = omega = 0.0
    if tau > tau_max and maxit > 0:
        if mu == 0.0:
            return dict(x=x, iters=0, converged=0, status=4, tau0=tau0, hist=hist)
        alpha = rho / mu
    ph = s = sh = z = zh = v = None
    j = 0
    while tau > tau_max and j < maxit:
        rec = [QNAN] * 12
        if j == 0:
            ph, s, sh, z = list(rh), list(w), list(wh), list(t)
        else:
            ph_n = [fma(beta, fma(-omega, sh[i], ph[i]), rh[i]) for i in range(n)]
            s_n = [fma(beta, fma(-omega, z[i], s[i]), w[i]) for i in range(n)]
            sh_n = [fma(beta, fma(-omega, zh[i], sh[i]), wh[i]) for i in range(n)]
            z_n = [fma(beta, fma(-omega, v[i], z[i]), t[i]) for i in range(n)]
            ph, s, sh, z = ph_n, s_n, sh_n, z_n
        q = [fma(-alpha, s[i], r[i]) for i in range(n)]
        qh = [fma(-alpha, sh[i], rh[i]) for i in range(n)]
        y = [fma(-alpha, z[i], w[i]) for i in range(n)]
        gamma = exdot(q, y)
        delta = exdot(y, y)
        zh = jac(z)
        v = mv(zh)
        omega = 0.0 if delta == 0.0 else gamma / delta
        x = [fma(omega, qh[i], fma(alpha, ph[i], x[i])) for i in range(n)]
        r = [fma(-omega, y[i], q[i]) for i in range(n)]
        rh = [fma(-omega, fma(-alpha, zh[i], wh[i]), qh[i]) for i in range(n)]
        w = [fma(-omega, fma(-alpha, v[i], t[i]), y[i]) for i in range(n)]
        rho1 = exdot(r0, r)
        a = exdot(r0, w)
        c = exdot(r0, s)
        e = exdot(r0, z)
        theta = exdot(r, r)
        tau = math.sqrt(theta)
        j += 1
        rec[0:9] = [gamma, delta, omega, rho1, a, c, e, theta, tau]
        if not (tau > tau_max):
            hist.append(rec)
            break
        if omega == 0.0 or rho1 == 0.0:
            hist.append(rec)
            status = 4
            break
        wh = jac(w)
        t = mv(wh)
        beta = (rho1 / rho) * (alpha / omega)
        bw = beta * omega
        den = fma(-bw, e, fma(beta, c, a))
        rec[9] = beta
        rec[10] = den
        if den == 0.0:
            hist.append(rec)
            status = 4
            break
        alpha = rho1 / den
        rec[11] = alpha
        hist.append(rec)
        rho = rho1
    return dict(x=x, iters=j, converged=int(status == 0 and not (tau > tau_max)),
                status=status, tau0=tau0, hist=hist)
