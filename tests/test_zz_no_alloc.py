"""The allocation-free exact dot, rbs_exdot_noalloc.

It exists for callers that cannot allocate device memory when they call: code
running inside a CUDA graph capture, latency-critical loops that cannot take an
allocation's implicit synchronisation, and applications whose own pool owns the
device memory. Its only scratch is an 8 KiB array inside the library.

The test calls it through the C ABI twice in a row (the shared array keeps the
previous call's contents, which the entry point must clear) and checks every
result against the existing rbs_exdot_multi entry point, the CPU oracle and
the exact value the generator knows. Exact dots are compared bit for bit, the
tolerance all exact-dot tests here use. This file is named to be collected
last; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_common import cuda_device, same
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


def test_noalloc_matches_exdot_multi_two_calls_in_a_row(orc):
    import torch
    dev = cuda_device()
    import paper_2302_04180_gb300 as rbs
    lib = rbs.load()
    f = lib.rbs_exdot_noalloc
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call, (n, cond, k) in enumerate([(300007, 1e32, 3), (1 << 20, 1e48, 6)]):
        vs, refs = [], []
        for j in range(k):
            x, y, exact = gen.ill_conditioned_dot(n, cond, seed=10 * call + j)
            vs.append((torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)))
            refs.append((orc.exdot(x, y), exact))
        xa = (C.c_void_p * k)(*[v[0].data_ptr() for v in vs])
        ya = (C.c_void_p * k)(*[v[1].data_ptr() for v in vs])
        out = torch.full((k,), float("nan"), dtype=torch.float64, device=dev)
        rc = f(k, xa, ya, n, C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == rbs.RBS_OK, lib.rbs_last_error()
        ref = rbs.rbs_exdot_multi([v[0] for v in vs], [v[1] for v in vs])
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        for j in range(k):
            assert same(got[j], want[j]), (call, j, got[j], want[j])
            assert same(got[j], refs[j][0]), (call, j, got[j], refs[j][0])
            if refs[j][1] is not None:
                assert same(got[j], float(refs[j][1])), (call, j)


def test_noalloc_rejects_more_dots_than_its_scratch_holds():
    import torch
    dev = cuda_device()
    import paper_2302_04180_gb300 as rbs
    lib = rbs.load()
    x = torch.ones(10, dtype=torch.float64, device=dev)
    k = rbs.RBS_NOALLOC_MAX_DOTS + 1 if hasattr(rbs, "RBS_NOALLOC_MAX_DOTS") else 7
    xa = (C.c_void_p * k)(*[x.data_ptr()] * k)
    out = torch.empty(k, dtype=torch.float64, device=dev)
    rc = lib.rbs_exdot_noalloc(k, xa, xa, 10, C.c_void_p(out.data_ptr()), None)
    assert rc == rbs.RBS_EINVAL
    assert b"6" in lib.rbs_last_error()
    host = np.ones(10)
    xh = (C.c_void_p * 1)(host.ctypes.data)
    assert lib.rbs_exdot_noalloc(1, xh, xh, 10, C.c_void_p(out.data_ptr()), None) == rbs.RBS_EINVAL
