"""Row-block ranks on CPU (gloo, world_size 2 and 4), the paper's partition
(Sec. 3.1, Sec. 4.1): every rank owns a block of rows of A and the matching
pieces of every vector. The exchange steps are an integer sum-Allreduce of the
ranks' long accumulators for every dot, after which every rank rounds locally
(Sec. 3.2), and an Allgather of the SpMV operand. A sharded exact dot, and a
whole sharded classic PBiCGStab (Fig. 2) run on the oracle's primitives, must
be bitwise the one-rank results, whatever the split. The GPU library's limb
export (rbs_exdot_partial) round-trips through the same Allreduce."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, cond, seed, out_q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2302_04180_gb300 import gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, y, _ = gen.ill_conditioned_dot(n, cond, seed)
        # uneven row blocks, as in the paper's p_k partition (Sec. 3)
        cuts = np.linspace(0, n, world + 1).astype(np.int64)
        cuts[1:-1] += (np.arange(1, world) * 37) % 101
        a, b = int(cuts[rank]), int(cuts[rank + 1])
        limbs, flags = oracle.exdot_limbs(x[a:b], y[a:b])
        t = torch.from_numpy(limbs.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        f = torch.tensor([flags], dtype=torch.int64)
        # flags are disjoint bits; a per-bit MAX is their OR
        fb = torch.tensor([(flags >> k) & 1 for k in range(3)], dtype=torch.int64)
        dist.all_reduce(fb, op=dist.ReduceOp.MAX)
        fl = int(sum(int(v) << k for k, v in enumerate(fb.tolist())))
        del f
        val = oracle.round_limbs(t.numpy(), fl)
        out_q.put((rank, float(val), float(oracle.exdot(x, y))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_exdot_integer_allreduce(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, 30011, 1e40, 5, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    vals = {r: (v, ref) for r, v, ref in res}
    ref_bits = np.float64(vals[0][1]).view(np.uint64)
    for r in range(world):
        assert np.float64(vals[r][0]).view(np.uint64) == ref_bits


def _cuts(n, world):
    """Uneven row blocks, as in the paper's p_k partition (Sec. 3)."""
    cuts = np.linspace(0, n, world + 1).astype(np.int64)
    cuts[1:-1] += (np.arange(1, world) * 37) % 101
    return cuts


def _allreduce_dot(oracle, x, y):
    """One exact dot over the ranks: local limbs, integer sum-Allreduce, OR of
    the non-finite flags (a per-bit MAX), one local rounding."""
    limbs, flags = oracle.exdot_limbs(x, y)
    t = torch.from_numpy(limbs.copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    fb = torch.tensor([(flags >> k) & 1 for k in range(3)], dtype=torch.int64)
    dist.all_reduce(fb, op=dist.ReduceOp.MAX)
    return float(oracle.round_limbs(t.numpy(), int(sum(int(v) << k for k, v in enumerate(fb.tolist())))))


def _allgather(local, cuts):
    """The full vector from every rank's piece (Allgatherv of the SpMV operand)."""
    world = len(cuts) - 1
    size = int(max(cuts[1:] - cuts[:-1]))
    buf = torch.zeros(size, dtype=torch.float64)
    buf[: local.size] = torch.from_numpy(local)
    parts = [torch.zeros(size, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, buf)
    return np.concatenate([parts[k].numpy()[: int(cuts[k + 1] - cuts[k])] for k in range(world)])


def _solve_worker(rank, world, port, out_q):
    """Fig. 2 on this rank's rows, in the order of the oracle's loop."""
    import math
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2302_04180_gb300 import gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for A in (gen.poisson3d(10), gen.convdiff3d(9, 25.0, (0.3, -1.0, 0.5))):
            tol, maxit = 1e-10, 400
            bfull = oracle.spmv(A, np.ones(A.n))
            cuts = _cuts(A.n, world)
            a, b = int(cuts[rank]), int(cuts[rank + 1])
            rows = gen.CSR(b - a, A.rowptr[a:b + 1] - A.rowptr[a], A.col[A.rowptr[a]:A.rowptr[b]],
                           A.val[A.rowptr[a]:A.rowptr[b]])
            invd = oracle.jacobi_invd(A)[a:b]  # RN(1 / a_ii) of this rank's rows
            spmv = lambda v: oracle.spmv(rows, _allgather(v, cuts))  # noqa: E731
            dot = lambda u, v: _allreduce_dot(oracle, u, v)  # noqa: E731
            x = np.zeros(b - a)
            r = bfull[a:b].copy()
            r0, p = r.copy(), r.copy()
            rho = dot(r0, r)
            tau = math.sqrt(rho)
            tau_max = tol * tau
            hist, j = [], 0
            while tau > tau_max and j < maxit:
                ph = oracle.jacobi_apply(invd, p)
                s = spmv(ph)
                sigma = dot(r0, s)
                alpha = rho / sigma
                q = oracle.fma_vec(-alpha, s, r)
                qh = oracle.jacobi_apply(invd, q)
                y = spmv(qh)
                gamma, delta = dot(q, y), dot(y, y)
                omega = 0.0 if delta == 0.0 else gamma / delta
                x = oracle.fma_vec(omega, qh, oracle.fma_vec(alpha, ph, x))
                r = oracle.fma_vec(-omega, y, q)
                rho1, theta = dot(r0, r), dot(r, r)
                tau = math.sqrt(theta)
                j += 1
                rec = [sigma, alpha, gamma, delta, omega, rho1, theta, tau, float("nan")]
                if not tau > tau_max:
                    hist.append(rec)
                    break
                beta = (rho1 / rho) * (alpha / omega)
                rec[8] = beta
                hist.append(rec)
                p = oracle.fma_vec(beta, oracle.fma_vec(-omega, s, p), r)
                rho = rho1
            xfull = _allgather(x, cuts)
            ref = oracle.solve(A, bfull, tol=tol, maxit=maxit, variant=0)
            out.append((j, np.array(hist), xfull, ref["iters"], ref["hist"][:, :9], ref["x"]))
        out_q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _bits(a):
    a = np.asarray(a, dtype=np.float64)
    b = a.view(np.uint64).copy()
    b[np.isnan(a)] = 0x7FF8000000000000
    return b


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_classic_solve_is_the_one_rank_solve(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        for j, hist, x, ref_iters, ref_hist, ref_x in res[r]:
            assert j == ref_iters > 5
            assert (_bits(hist) == _bits(ref_hist)).all()
            assert (_bits(x) == _bits(ref_x)).all()


def _partial_worker(rank, world, port, out_q):
    """The GPU library's partial limbs of this rank's slice, summed over the
    ranks with the same Allreduce and rounded by the library."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cuda:0")
        vals = []
        for n, cond, seed in ((100003, 1e32, 3), (4099, 1e48, 4), (65536, 1.0, 5)):
            x, y, _ = gen.ill_conditioned_dot(n, cond, seed)
            cuts = _cuts(n, world)
            a, b = int(cuts[rank]), int(cuts[rank + 1])
            xt, yt = torch.from_numpy(x[a:b].copy()).to(dev), torch.from_numpy(y[a:b].copy()).to(dev)
            limbs, flags = rbs.rbs_exdot_partial(xt, yt)
            t = limbs.cpu()
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            f = int(flags.cpu().item())
            fb = torch.tensor([(f >> k) & 1 for k in range(3)], dtype=torch.int64)
            dist.all_reduce(fb, op=dist.ReduceOp.MAX)
            fl = torch.tensor([int(sum(int(v) << k for k, v in enumerate(fb.tolist())))], dtype=torch.int32)
            got = float(rbs.rbs_round_limbs(t.to(dev), fl.to(dev)).item())
            full = float(rbs.rbs_exdot(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)).item())
            vals.append((got, full))
        out_q.put((rank, vals))
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_library_partial_limbs_through_the_allreduce():
    """Ranks share the one GPU only as independent callers (no kernel waits
    on another rank's); the exchange is gloo on the host."""
    import __graft_entry__ as g
    g.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partial_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        for got, full in res[r]:
            assert np.float64(got).view(np.uint64) == np.float64(full).view(np.uint64)
