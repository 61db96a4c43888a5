"""Whole-run parity of the full-size single solves (the benchmark workload and
its nonsymmetric companion): every scalar of every iteration, the iteration
count and x, bit for bit against the CPU oracle (Fig. 2, Fig. 4; the method of
Sec. 5.3). The oracle's runs take minutes at these sizes, so they are stored as
digests written by tests/golden/make_c3_digests.py, which calls only oracle/."""
import hashlib
import os
import sys

import numpy as np
import pytest

from gpu_common import cuda_device
from paper_2302_04180_gb300 import gen

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_c3_digests as D  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


@pytest.fixture(scope="module")
def rbs(dev):
    import paper_2302_04180_gb300 as m
    return m


@pytest.mark.parametrize("name", list(D.WORKLOADS))
def test_whole_run_matches_oracle_digest(rbs, dev, name):
    import torch
    want = D.read(name)
    fn, args, variant = D.WORKLOADS[name]
    A = getattr(gen, fn)(*args)
    Ad = rbs.to_device(A, dev)
    b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    loops = (0, 1) if name == "poisson256_classic" else (0,)
    for loop_mode in loops:  # the device-side graph loop, and the host loop the bench times
        g = rbs.rbs_solve(Ad, b, tol=D.TOL, maxit=D.MAXIT, variant=variant, loop_mode=loop_mode)
        assert g["iters"] == int(want["iters"]) and g["status"] == int(want["status"])
        assert g["converged"] == int(want["converged"]) == 1
        # alpha0 and mu0 are pipelined set-up scalars (rbs_info leaves them NaN / 0 for classic)
        for k in ("tau0", "tau_final", "rho0", "tau_max") + (("alpha0", "mu0") if variant == 1 else ()):
            assert D.hx(g[k]) == want[k], k
        if D.history_sha(g["hist"]) != want["history_sha256"]:
            col = 7 if variant == 0 else 8
            first = next((j for j in range(g["iters"]) if D.hx(g["hist"][j, col]) != want["tau"][j]), None)
            pytest.fail(f"{name}: history differs (first differing tau at iteration {first})")
        x = g["x"].cpu().numpy()
        for i, h in want["x"].items():
            assert D.hx(x[i]) == h, i
        assert D.x_sha(x) == want["x_sha256"]
