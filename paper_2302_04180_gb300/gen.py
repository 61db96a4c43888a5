"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds inputs: sparse matrices in CSR, vectors, and dot
operands with a known exact result. It holds none of the method's arithmetic
(no SpMV, no dot, no solver step); both the GPU library's tests and the CPU
oracle's tests draw from it, and nothing here depends on either.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014; the constants
are Vigna's published ones), evaluated counter-style: word i of stream s is
mix(s * 2^32 + i), so a draw never depends on how many draws came before, and
the streams match on any machine and numpy version.

Workloads (the paper's SuiteSparse matrices and its 27-point stencil are not
available; these stand in for them):
  * 3D Poisson, 7-point, N^3 interior grid, Dirichlet boundary eliminated,
    lexicographic index i + N*j + N^2*k, columns ascending
    (k-1, j-1, i-1, diag, i+1, j+1, k+1), 6 on the diagonal, -1 off it.
  * 3D (and 2D) convection-diffusion with first-order upwinding on the unit
    cube, h = 1/(N+1), unit direction d, Peclet number Pe, P_m = Pe*h*|d_m|;
    row scaled by h^2: diagonal 2*dim + sum_m P_m, upwind neighbour along m
    -(1 + P_m), downwind neighbour -1.
  * Ill-conditioned dot operands whose exact dot is known by construction
    (exact cancellation, see ``ill_conditioned_dot``).
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64(stream: int, count: int, start: int = 0) -> np.ndarray:
    """Words start..start+count-1 of SplitMix64 stream ``stream`` (uint64)."""
    with np.errstate(over="ignore"):
        ctr = (np.arange(start, start + count, dtype=np.uint64)
               + np.uint64((int(stream) & 0xFFFFFFFF) << 32))
        z = (ctr + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(stream: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (splitmix64(stream, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def stream_id(seed: int, tag: int) -> int:
    return (int(seed) * 1000003 + int(tag)) & 0xFFFFFFFF


@dataclass
class CSR:
    """CSR matrix: int64 rowptr[n+1], int32 col[nnz], float64 val[nnz].
    The stored order of a row is its fma order."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _stencil_csr(n: int, cols_list, vals_list, masks, name: str) -> CSR:
    k = len(cols_list)
    mask = np.empty((n, k), dtype=bool)
    cols = np.empty((n, k), dtype=np.int32)
    vals = np.empty((n, k), dtype=np.float64)
    for t in range(k):
        mask[:, t] = masks[t]
        cols[:, t] = cols_list[t]
        vals[:, t] = vals_list[t]
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[mask]
    val = vals[mask]
    return CSR(n, rowptr, np.ascontiguousarray(col), np.ascontiguousarray(val), name)


def poisson3d(N: int) -> CSR:
    """3D Poisson 7-point on an N^3 grid (nnz = N^3 + 6 (N-1) N^2)."""
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    i = idx % N
    j = (idx // N) % N
    k = idx // (N * N)
    NN = N * N
    offs = [(-NN, k > 0), (-N, j > 0), (-1, i > 0), (0, None),
            (1, i < N - 1), (N, j < N - 1), (NN, k < N - 1)]
    cols_list, vals_list, masks = [], [], []
    for off, m in offs:
        c = idx + off
        cols_list.append(np.where((m if m is not None else True), c, 0).astype(np.int32))
        vals_list.append(6.0 if off == 0 else -1.0)
        masks.append(np.ones(n, dtype=bool) if m is None else m)
    return _stencil_csr(n, cols_list, vals_list, masks, f"poisson3d_{N}")


def convdiff3d(N: int, Pe: float, direction=(1.0, 1.0, 1.0)) -> CSR:
    """Nonsymmetric 3D convection-diffusion, 7-point, first-order upwind."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.sqrt(np.sum(d * d))
    h = 1.0 / (N + 1)
    P = [Pe * h * abs(float(d[m])) for m in range(3)]
    diag = 6.0 + P[0] + P[1] + P[2]
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    coord = [idx % N, (idx // N) % N, idx // (N * N)]
    stride = [1, N, N * N]
    lo_val = [-(1.0 + P[m]) if d[m] > 0 else -1.0 for m in range(3)]
    hi_val = [-(1.0 + P[m]) if d[m] < 0 else -1.0 for m in range(3)]
    cols_list, vals_list, masks = [], [], []
    for m in (2, 1, 0):  # k-1, j-1, i-1
        msk = coord[m] > 0
        cols_list.append(np.where(msk, idx - stride[m], 0).astype(np.int32))
        vals_list.append(lo_val[m])
        masks.append(msk)
    cols_list.append(idx.astype(np.int32))
    vals_list.append(diag)
    masks.append(np.ones(n, dtype=bool))
    for m in (0, 1, 2):  # i+1, j+1, k+1
        msk = coord[m] < N - 1
        cols_list.append(np.where(msk, idx + stride[m], 0).astype(np.int32))
        vals_list.append(hi_val[m])
        masks.append(msk)
    return _stencil_csr(n, cols_list, vals_list, masks, f"convdiff3d_{N}_Pe{Pe:g}")


def convdiff2d(N: int, Pe: float, direction=(1.0, 1.0)) -> CSR:
    """Nonsymmetric 2D convection-diffusion, 5-point, first-order upwind."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.sqrt(np.sum(d * d))
    h = 1.0 / (N + 1)
    P = [Pe * h * abs(float(d[m])) for m in range(2)]
    diag = 4.0 + P[0] + P[1]
    n = N ** 2
    idx = np.arange(n, dtype=np.int64)
    coord = [idx % N, idx // N]
    stride = [1, N]
    lo_val = [-(1.0 + P[m]) if d[m] > 0 else -1.0 for m in range(2)]
    hi_val = [-(1.0 + P[m]) if d[m] < 0 else -1.0 for m in range(2)]
    cols_list, vals_list, masks = [], [], []
    for m in (1, 0):
        msk = coord[m] > 0
        cols_list.append(np.where(msk, idx - stride[m], 0).astype(np.int32))
        vals_list.append(lo_val[m])
        masks.append(msk)
    cols_list.append(idx.astype(np.int32))
    vals_list.append(diag)
    masks.append(np.ones(n, dtype=bool))
    for m in (0, 1):
        msk = coord[m] < N - 1
        cols_list.append(np.where(msk, idx + stride[m], 0).astype(np.int32))
        vals_list.append(hi_val[m])
        masks.append(msk)
    return _stencil_csr(n, cols_list, vals_list, masks, f"convdiff2d_{N}_Pe{Pe:g}")


def random_csr(n: int, max_row: int, seed: int, empty_frac: float = 0.0,
               dup_frac: float = 0.0, diag_dominant: bool = False,
               ncols: int | None = None) -> CSR:
    """Unstructured CSR with ragged rows, optional empty rows and duplicate
    column entries (kept in stored order); with diag_dominant every row holds
    its diagonal entry, larger than the sum of the row's other magnitudes."""
    ncols = n if ncols is None else ncols
    u = uniform(stream_id(seed, 1), n)
    lens = (u * (max_row + 1)).astype(np.int64)
    if empty_frac > 0:
        e = uniform(stream_id(seed, 2), n) < empty_frac
        lens[e] = 0
    if diag_dominant:
        lens = np.maximum(lens, 1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = (splitmix64(stream_id(seed, 3), nnz) % np.uint64(max(ncols, 1))).astype(np.int64)
    if dup_frac > 0 and nnz > 1:
        dmask = uniform(stream_id(seed, 4), nnz) < dup_frac
        dmask[0] = False
        prev = np.roll(col, 1)
        col = np.where(dmask, prev, col)
    val = uniform(stream_id(seed, 5), nnz) * 2.0 - 1.0
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    if diag_dominant:
        first = rowptr[:-1][lens > 0]
        col[first] = np.arange(n, dtype=np.int64)[lens > 0]
        absrow = np.zeros(n)
        np.add.at(absrow, rows, np.abs(val))
        val[first] = absrow[lens > 0] + 1.0 + uniform(stream_id(seed, 6), int((lens > 0).sum()))
    return CSR(n, rowptr, col.astype(np.int32), val, f"random_{n}_{max_row}_{seed}")


def ones_like_rows(A: CSR) -> np.ndarray:
    return np.ones(A.n, dtype=np.float64)


def random_vector(n: int, seed: int, tag: int = 7, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform(stream_id(seed, tag), n)


def _mantissas(stream: int, count: int) -> np.ndarray:
    """Doubles in [1, 2) with random 52-bit fractions."""
    frac = splitmix64(stream, count) >> np.uint64(12)
    bits = frac | np.uint64(0x3FF0000000000000)
    return bits.view(np.float64)


def ill_conditioned_dot(n: int, cond: float, seed: int):
    """Dot operands (x, y) of length n and their exact dot as a Fraction.

    cond <= 2 is read as the well-conditioned case: x, y uniform in (0, 1),
    all products positive (condition number 2); the exact dot is then not
    known in closed form and None is returned for it.

    Otherwise, in the style of Ogita, Rump & Oishi's dot generator, products
    spread over 2^0 .. 2^(2b), b = log2(cond)/2, and cancel exactly:
    groups (x, y), (x, -y_hi), (x, -y_lo) with y = y_hi + y_lo split exactly
    at a random bit, and pairs (x, y), (-x, y) to fill. One residual pair
    (u, v) with an exactly representable product u*v of magnitude about
    2 sum|x_i y_i| / cond stays, so the exact dot is u*v and the condition
    number 2 sum|x_i y_i| / |sum x_i y_i| is about cond. All elements are
    shuffled.
    """
    if n <= 0:
        return np.zeros(0), np.zeros(0), Fraction(0)
    s = lambda tag: stream_id(seed, 100 + tag)  # noqa: E731
    if cond <= 2.0:
        x = uniform(s(1), n)
        y = uniform(s(2), n)
        x[x == 0.0] = 0.5
        y[y == 0.0] = 0.5
        return x, y, None
    b = max(1, int(round(np.log2(cond) / 2.0)))
    body = n - 1
    ntrip = body // 3
    npair = (body - 3 * ntrip) // 2
    nzero = body - 3 * ntrip - 2 * npair  # 0 or 1 element left: (x, 0)
    m = ntrip + npair
    ex = (splitmix64(s(3), m) % np.uint64(b + 1)).astype(np.int64)
    ey = (splitmix64(s(4), m) % np.uint64(b + 1)).astype(np.int64)
    sx = np.where(splitmix64(s(5), m) & np.uint64(1), -1.0, 1.0)
    sy = np.where(splitmix64(s(6), m) & np.uint64(1), -1.0, 1.0)
    xb = sx * np.ldexp(_mantissas(s(7), m), ex)
    yb = sy * np.ldexp(_mantissas(s(8), m), ey)
    xs, ys = [], []
    # triples: y = y_hi + y_lo exactly, y_hi = y with its low `cut` bits cleared
    xt, yt = xb[:ntrip], yb[:ntrip]
    cut = (splitmix64(s(9), ntrip) % np.uint64(51)).astype(np.uint64) + np.uint64(1)
    ybits = yt.view(np.uint64)
    yhi = (ybits & ~((np.uint64(1) << cut) - np.uint64(1))).view(np.float64)
    ylo = yt - yhi  # exact: yhi is y truncated toward zero
    xs += [xt, xt, xt]
    ys += [yt, -yhi, -ylo]
    # pairs: (x, y) and (-x, y)
    xp, yp = xb[ntrip:], yb[ntrip:]
    xs += [xp, -xp]
    ys += [yp, yp]
    absum = 2.0 * float(np.sum(np.abs(xt * yt))) + 2.0 * float(np.sum(np.abs(xp * yp)))
    target = max(2.0 * absum / cond, 2.0 ** -900)
    # residual u * v exact: 26-bit significands
    mu = int(splitmix64(s(10), 1)[0] >> np.uint64(38)) | (1 << 25)
    mv = int(splitmix64(s(11), 1)[0] >> np.uint64(38)) | (1 << 25)
    e_t = int(np.floor(np.log2(target))) - 50
    eu = e_t // 2
    ev = e_t - eu
    sgn = -1.0 if (int(splitmix64(s(12), 1)[0]) & 1) else 1.0
    u = sgn * float(np.ldexp(float(mu), eu))
    v = float(np.ldexp(float(mv), ev))
    xs.append(np.array([u]))
    ys.append(np.array([v]))
    if nzero:
        xs.append(np.array([1.5]))
        ys.append(np.array([0.0]))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    assert x.size == n
    perm = np.argsort(splitmix64(s(13), n), kind="stable")
    exact = Fraction(u) * Fraction(v)
    return np.ascontiguousarray(x[perm]), np.ascontiguousarray(y[perm]), exact


def batch_workload(count: int, seed: int, n_min: int = 1000, n_max: int = 300000):
    """Independent nonsymmetric convection-diffusion systems for batched solves.

    Per system (SplitMix64, stream per field): 2D 5-point or 3D 7-point with
    probability 1/2; target size n drawn log-uniform in [n_min, n_max], grid side
    round(n^(1/dim)) (at least 3); Peclet number uniform in [0, 50]; a random unit
    velocity direction; classic or pipelined with probability 1/2. Returns a list
    of (CSR, variant) pairs.
    """
    sid = lambda tag: stream_id(seed, 900 + tag)  # noqa: E731
    u_dim = uniform(sid(1), count)
    u_n = uniform(sid(2), count)
    u_pe = uniform(sid(3), count)
    u_var = uniform(sid(4), count)
    dirs = uniform(sid(5), 3 * count).reshape(count, 3) * 2.0 - 1.0
    out = []
    for k in range(count):
        dim = 2 if u_dim[k] < 0.5 else 3
        n_target = float(np.exp(np.log(n_min) + u_n[k] * (np.log(n_max) - np.log(n_min))))
        side = max(3, int(round(n_target ** (1.0 / dim))))
        pe = 50.0 * float(u_pe[k])
        d = dirs[k, :dim]
        if not np.any(d):
            d = np.ones(dim)
        A = convdiff2d(side, pe, tuple(d)) if dim == 2 else convdiff3d(side, pe, tuple(d))
        out.append((A, 1 if u_var[k] >= 0.5 else 0))
    return out


def stencil27(N: int, perturb: float = 1e-4) -> CSR:
    """3D 27-point stencil on an N^3 grid, the 'e-type' unsymmetric model of the
    paper's scalability study (Sec. 5.2): the 27-point Poisson matrix (26 on the
    diagonal, -1 for each of the up to 26 neighbours), with every neighbour below
    the central point (lower column index) perturbed to -(1 - perturb). Columns
    ascending (lexicographic i + N j + N^2 k)."""
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    coord = [idx % N, (idx // N) % N, idx // (N * N)]
    cols_list, vals_list, masks = [], [], []
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                off = di + N * dj + N * N * dk
                msk = np.ones(n, dtype=bool)
                for c, d in zip(coord, (di, dj, dk)):
                    if d < 0:
                        msk &= c > 0
                    elif d > 0:
                        msk &= c < N - 1
                cols_list.append(np.where(msk, idx + off, 0).astype(np.int32))
                if off == 0:
                    vals_list.append(26.0)
                elif off < 0:
                    vals_list.append(-(1.0 - perturb))
                else:
                    vals_list.append(-1.0)
                masks.append(msk)
    return _stencil_csr(n, cols_list, vals_list, masks, f"stencil27_{N}")


def banded(n: int, band: int, perturb: float = 1e-4) -> CSR:
    """Band matrix with bandL = bandU = band (nnz = (2 band + 1) n away from the
    edges), the stand-in for the paper's weak-scaling band matrices (Sec. 5.2):
    -1 above the diagonal, -(1 - perturb) below it, and a diagonal of 2 band + 1
    (strictly dominant)."""
    idx = np.arange(n, dtype=np.int64)
    cols_list, vals_list, masks = [], [], []
    for off in range(-band, band + 1):
        c = idx + off
        msk = (c >= 0) & (c < n)
        cols_list.append(np.where(msk, c, 0).astype(np.int32))
        vals_list.append(float(2 * band + 1) if off == 0 else (-(1.0 - perturb) if off < 0 else -1.0))
        masks.append(msk)
    return _stencil_csr(n, cols_list, vals_list, masks, f"banded_{n}_{band}")


def serving_pool(count: int, seed: int, n_side_max: int = 128):
    """Distinct systems that serving requests draw from: half 3D upwind
    convection-diffusion (side log-uniform in [12, 64], Pe uniform in [0, 50],
    random unit direction), half 3D Poisson (side log-uniform in [12,
    n_side_max]); classic or pipelined with probability 1/2. Returns a list of
    (CSR, variant) pairs."""
    sid = lambda tag: stream_id(seed, 700 + tag)  # noqa: E731
    u_kind, u_side, u_pe, u_var = (uniform(sid(t), count) for t in range(4))
    dirs = uniform(sid(5), 3 * count).reshape(count, 3) * 2.0 - 1.0
    out = []
    for k in range(count):
        if u_kind[k] < 0.5:
            side = int(round(np.exp(np.log(12) + u_side[k] * (np.log(64) - np.log(12)))))
            d = dirs[k] if np.any(dirs[k]) else np.ones(3)
            A = convdiff3d(side, 50.0 * float(u_pe[k]), tuple(d))
        else:
            side = int(round(np.exp(np.log(12) + u_side[k] * (np.log(n_side_max) - np.log(12)))))
            A = poisson3d(side)
        out.append((A, 1 if u_var[k] >= 0.5 else 0))
    return out


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    u = uniform(stream_id(seed, 800), count)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)
