"""GPU parity of the fma-ordered CSR SpMV (Sec. 4.1, Sec. 3.3) and the Jacobi
preconditioner (Sec. 4) against the CPU oracle, bit for bit, including empty
rows, duplicate entries, signed zeros, the full 128^3 Poisson matrix, launch
shapes, and a bad column index reported as an error (never read)."""
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
    yield m
    m.rbs_set_param("spmv.block", 0)
    m.rbs_set_param("spmv.mode", 0)


def _spmv(rbs, dev, A, x):
    import torch
    Ad = rbs.to_device(A, dev)
    return rbs.rbs_spmv_csr(Ad, torch.from_numpy(x).to(dev)).cpu().numpy()


@pytest.mark.parametrize("n,mr,empty,dup", [(1, 1, 0.0, 0.0), (7, 3, 0.3, 0.2), (1000, 12, 0.1, 0.3),
                                            (33333, 40, 0.05, 0.1)])
def test_random_csr(rbs, dev, orc, n, mr, empty, dup):
    A = gen.random_csr(n, mr, seed=n, empty_frac=empty, dup_frac=dup)
    x = gen.random_vector(n, 3) * 10.0 ** gen.random_vector(n, 3, 9, -100, 100)
    x[::5] = -0.0
    ref = orc.spmv(A, x)
    for mode in (0, 1, 2, 3):  # long spans (mr=40) also exercise the staged path's fallback
        rbs.rbs_set_param("spmv.mode", mode)
        assert same_array(_spmv(rbs, dev, A, x), ref), mode
    rbs.rbs_set_param("spmv.mode", 0)


@pytest.mark.parametrize("make", [lambda: gen.poisson3d(17), lambda: gen.convdiff3d(19, 10.0),
                                  lambda: gen.convdiff2d(101, 50.0, (0.6, -0.8))])
def test_stencils(rbs, dev, orc, make):
    A = make()
    x = gen.random_vector(A.n, 5)
    assert same_array(_spmv(rbs, dev, A, x), orc.spmv(A, x))
    ones = np.ones(A.n)
    assert same_array(_spmv(rbs, dev, A, ones), orc.spmv(A, ones))


def test_poisson_128_full_size(rbs, dev, orc):
    A = gen.poisson3d(128)
    assert A.n == 2097152 and A.nnz == 14581760
    x = gen.random_vector(A.n, 6)
    ref = orc.spmv(A, x)
    for mode in (0, 1, 2, 3):
        rbs.rbs_set_param("spmv.mode", mode)
        for block in (0, 64, 256):
            rbs.rbs_set_param("spmv.block", block)
            assert same_array(_spmv(rbs, dev, A, x), ref), (mode, block)
    rbs.rbs_set_param("spmv.block", 0)
    rbs.rbs_set_param("spmv.mode", 0)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_bad_column_is_reported_not_read(rbs, dev, mode):
    import torch
    A = gen.random_csr(100, 5, seed=1) if mode != 3 else gen.stencil27(7)
    col = A.col.copy()
    col[len(col) // 2] = 1 << 30
    bad = gen.CSR(A.n, A.rowptr, col, A.val)
    Ad = rbs.to_device(bad, dev)
    try:
        rbs.rbs_set_param("spmv.mode", mode)
        rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
        with pytest.raises(rbs.RbsError) as e:
            rbs.rbs_stream_status()
        assert e.value.code == rbs.RBS_EINVAL
        rbs.rbs_stream_status()  # cleared
    finally:
        rbs.rbs_set_param("spmv.mode", 0)


@pytest.mark.parametrize("long_rows", [False, True])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_malformed_row_pointers_are_reported(rbs, dev, mode, long_rows):
    """A row pointer that runs backwards, or past nnz, is caught by the kernel's
    own checks under every schedule (the chunk is not staged and the row is
    skipped), reported as RBS_EINVAL; the next call is clean."""
    import torch
    A = gen.stencil27(9) if long_rows else gen.poisson3d(10)
    for bad_value in (int(A.rowptr[A.n // 2 + 1]) + 5, A.nnz + 1000):
        rp = A.rowptr.copy()
        rp[A.n // 2] = bad_value
        bad = gen.CSR(A.n, rp, A.col, A.val)
        Bd = rbs.to_device(bad, dev)
        try:
            rbs.rbs_set_param("spmv.mode", mode)
            rbs.rbs_spmv_csr(Bd, torch.ones(A.n, dtype=torch.float64, device=dev))
            with pytest.raises(rbs.RbsError) as e:
                rbs.rbs_stream_status()
            assert e.value.code == rbs.RBS_EINVAL
            rbs.rbs_stream_status()  # cleared
        finally:
            rbs.rbs_set_param("spmv.mode", 0)


@pytest.mark.parametrize("side", [7, 21, 33])
def test_stencil27_ragged_chunks(rbs, dev, orc, side):
    """Long rows (27 nonzeros) through the register-staged schedule: n = 343,
    9261 and 35937 leave tails of 23, 13 and 1 rows after the 32-row chunks;
    the edge rows (8 to 18 nonzeros) share chunks with the interior ones."""
    A = gen.stencil27(side)
    x = gen.random_vector(A.n, side) * 10.0 ** gen.random_vector(A.n, side + 1, 9, -30, 30)
    x[::7] = -0.0
    ref = orc.spmv(A, x)
    for mode in (0, 3):
        rbs.rbs_set_param("spmv.mode", mode)
        assert same_array(_spmv(rbs, dev, A, x), ref), mode
    rbs.rbs_set_param("spmv.mode", 0)


def _lengthen_rows(A, every, extra):
    """A copy of A in which every `every`-th row gets `extra` more entries:
    repeats of its own first entries (duplicates sum in stored order)."""
    rows, cols, vals = [0], [], []
    for i in range(A.n):
        b, e = int(A.rowptr[i]), int(A.rowptr[i + 1])
        c, v = list(A.col[b:e]), list(A.val[b:e])
        if i % every == 0 and e > b:
            c += [c[k % len(c)] for k in range(extra)]
            v += [v[k % len(v)] * 0.5 for k in range(extra)]
        cols += c
        vals += v
        rows.append(len(cols))
    return gen.CSR(A.n, np.array(rows, np.int64), np.array(cols, np.int32), np.array(vals, np.float64))


def test_long_rows_past_the_register_length(rbs, dev, orc):
    """Chunks of the long-row schedule holding rows of more than 28 nonzeros
    (every 37th row of a 27-point matrix lengthened to 35) are computed
    from the staged buffer before it is refilled; the others from registers."""
    A = _lengthen_rows(gen.stencil27(15), 37, 8)
    x = gen.random_vector(A.n, 15)
    ref = orc.spmv(A, x)
    for mode in (0, 3):
        rbs.rbs_set_param("spmv.mode", mode)
        assert same_array(_spmv(rbs, dev, A, x), ref), mode
    rbs.rbs_set_param("spmv.mode", 0)


def test_long_rows_unaligned_arrays(rbs, dev, orc):
    """col and val views 4 and 8 bytes past a 16-byte boundary: no bulk
    copies; every chunk is staged by per-lane element copies."""
    import torch
    A = gen.stencil27(17)
    colb = torch.zeros(A.nnz + 1, dtype=torch.int32, device=dev)
    valb = torch.zeros(A.nnz + 1, dtype=torch.float64, device=dev)
    colb[1:] = torch.from_numpy(A.col.astype(np.int32)).to(dev)
    valb[1:] = torch.from_numpy(A.val).to(dev)
    Ad = rbs.DeviceCSR(A.n, torch.from_numpy(A.rowptr.astype(np.int64)).to(dev), colb[1:], valb[1:])
    assert Ad.col.data_ptr() % 16 == 4 and Ad.val.data_ptr() % 16 == 8
    x = gen.random_vector(A.n, 17)
    ref = orc.spmv(A, x)
    for mode in (0, 2, 3):
        rbs.rbs_set_param("spmv.mode", mode)
        assert same_array(rbs.rbs_spmv_csr(Ad, torch.from_numpy(x).to(dev)).cpu().numpy(), ref), mode
    rbs.rbs_set_param("spmv.mode", 0)


def test_stencil27_159_full_size(rbs, dev, orc):
    """The 27-point e-type matrix at the benchmark's size (n = 4,019,679,
    nnz = 107,171,875), every row bitwise the oracle's."""
    A = gen.stencil27(159)
    assert A.n == 159 ** 3 and A.nnz == (3 * 159 - 2) ** 3
    x = gen.random_vector(A.n, 27)
    assert same_array(_spmv(rbs, dev, A, x), orc.spmv(A, x))


def test_jacobi(rbs, dev, orc):
    import torch
    A = gen.convdiff3d(9, 30.0, (0.2, 1.0, -0.4))
    Ad = rbs.to_device(A, dev)
    invd = rbs.rbs_jacobi_invd(Ad)
    ref = orc.jacobi_invd(A)
    assert (bits(invd.cpu().numpy()) == bits(ref)).all()
    p = gen.random_vector(A.n, 2)
    ph = rbs.rbs_jacobi_apply(invd, torch.from_numpy(p).to(dev))
    assert (bits(ph.cpu().numpy()) == bits(orc.jacobi_apply(ref, p))).all()
    d = gen.random_vector(A.n, 3, lo=0.5, hi=2.0)
    assert (bits(rbs.rbs_jacobi_invd(Ad, torch.from_numpy(d).to(dev)).cpu().numpy())
            == bits(orc.jacobi_invd(A, d))).all()
    with pytest.raises(rbs.RbsError):
        rbs.rbs_jacobi_invd(Ad, torch.zeros(A.n, dtype=torch.float64, device=dev))
