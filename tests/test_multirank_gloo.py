"""Row-block ranks on CPU (gloo, world_size 2 and 4): the one exchange step of a
sharded exact dot is an integer sum-Allreduce of long accumulators (Sec. 3.2),
after which every rank rounds locally. The result must be bitwise the 1-rank
exdot, whatever the split. The ranks here use the oracle's accumulator export;
the GPU library exports the same kind of limb array (rbs_exdot_partial)."""
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
