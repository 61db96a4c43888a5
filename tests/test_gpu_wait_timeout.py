"""The staged SpMV's bounded wait, made to run out on purpose without any
fault: the test mode (knob test.stall_staging) has the issuing lane announce a
chunk's bulk copies on the mbarrier but not issue them, so the wait (a phase
that nothing completes) hits its poll limit. The kernel records the timeout, the warp reads its remaining
rows from global memory, and the call reports RBS_ETIMEOUT. The product is
still exact; after the hooks are reset everything runs normally."""
import numpy as np
import pytest

from gpu_common import cuda_device, same_array
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make", [lambda: gen.poisson3d(24), lambda: gen.stencil27(19)],
                         ids=["short_rows", "long_rows"])
def test_bounded_wait_runs_out_and_is_reported(orc, make):
    import torch
    dev = cuda_device()
    import paper_2302_04180_gb300 as rbs
    A = make()
    Ad = rbs.to_device(A, dev)
    x = gen.random_vector(A.n, 8)
    xt = torch.from_numpy(x).to(dev)
    ref = orc.spmv(A, x)
    b = torch.from_numpy(orc.spmv(A, np.ones(A.n))).to(dev)
    try:
        rbs.rbs_set_param("test.stall_staging", 1)
        y = rbs.rbs_spmv_csr(Ad, xt)
        with pytest.raises(rbs.RbsError) as e:
            rbs.rbs_stream_status()
        assert e.value.code == rbs.RBS_ETIMEOUT
        assert same_array(y.cpu().numpy(), ref)  # the fallback rows are the same fma chains
        with pytest.raises(rbs.RbsError) as e:
            rbs.rbs_solve(Ad, b, tol=1e-8, maxit=50, variant=0)
        assert e.value.code == rbs.RBS_ETIMEOUT
    finally:
        rbs.rbs_set_param("test.stall_staging", 0)
    y = rbs.rbs_spmv_csr(Ad, xt)
    rbs.rbs_stream_status()
    assert same_array(y.cpu().numpy(), ref)
    g = rbs.rbs_solve(Ad, b, tol=1e-8, maxit=500, variant=0)
    assert g["status"] == 0 and g["converged"] == 1
