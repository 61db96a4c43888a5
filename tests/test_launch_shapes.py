"""Launch-shape invariants of the solver kernels, checked from the compiler's
register report (CPU only: nvcc cross-compiles for sm_103a).

The vector kernels of one solver variant share a persistent grid sized from the
occupancy of one of them (K4 for the classic loop, P1 for the pipelined one). A
kernel of the group that fits fewer blocks per SM than that one runs the grid in
more than one wave: K2 once took 80 registers, fitted three 256-thread blocks
where K4 fits four, and ran 1.33 waves. These tests pin the register budgets that
keep every kernel of a group at least as resident as the kernel sizing its grid,
and that the exact reducers' windows stay out of local memory where the launch
shape was chosen for that.
"""
import re
import shutil
import subprocess

import pytest

from paper_2302_04180_gb300 import build as B

REGS_PER_SM = 65536
BLOCK = 256


def _ptxas_report(tmp_path_factory, source):
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    obj = tmp_path_factory.mktemp("ptxas") / source.replace(".cu", ".o")
    cmd = [B.nvcc(), "-Xptxas=-v", *B.ARCH, *B.NVCC_FLAGS, "-c", f"{B.CSRC}/{source}", "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, name, spill = {}, None, 0
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            name = m.group(1)
        m = re.search(r"(\d+) bytes spill stores", line)
        if m:
            spill = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            out[name] = (int(m.group(1)), spill)
            name = None
    return out


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    return _ptxas_report(tmp_path_factory, "kernels_solver.cu")


@pytest.fixture(scope="module")
def step_report(tmp_path_factory):
    return _ptxas_report(tmp_path_factory, "kernels_step.cu")


def _find(report, *parts):
    hits = [k for k in report if all(p in k for p in parts)]
    assert len(hits) == 1, (parts, hits)
    return report[hits[0]]


def _blocks(regs):
    per_warp = ((regs + 7) // 8) * 8 * 32  # registers are allocated per warp, 8 per thread at a time
    return REGS_PER_SM // (per_warp * (BLOCK // 32))


EXACT, PLAIN = "ExactR", "PlainR"


@pytest.mark.parametrize("red", [EXACT, PLAIN])
def test_classic_vector_kernels_fit_the_k4_grid(report, red):
    k4 = _blocks(_find(report, "k_cls_k4", red)[0])
    assert k4 >= 4
    for kern in ("k_cls_k2", "k_cls_k5"):
        assert _blocks(_find(report, kern)[0]) >= k4, kern
    assert _blocks(_find(report, "k_cls_setup", red)[0]) >= k4


@pytest.mark.parametrize("red", [EXACT, PLAIN])
def test_pipelined_setup_fits_the_p1_grid(report, red):
    p1 = _blocks(_find(report, "k_pipe_p1", red)[0])
    assert _blocks(_find(report, "k_pipe_setup1")[0]) >= p1


def test_chosen_pipelined_shapes(report):
    # exact P1: three blocks per SM; exact P3: two, with its five windows in registers
    assert _blocks(_find(report, "k_pipe_p1", EXACT)[0]) == 3
    regs, spill = _find(report, "k_pipe_p3", EXACT)
    assert _blocks(regs) == 2 and spill == 0


def test_streaming_kernels_do_not_spill(report):
    for parts in (("k_cls_k2",), ("k_cls_k5",), ("k_cls_k4", EXACT), ("k_cls_k4", PLAIN)):
        assert _find(report, *parts)[1] == 0, parts


def test_step_kernels_as_resident_as_the_solve_kernels(step_report):
    """The per-step kernels (batched solves and the serving engine) run the
    same element steps with per-system task indexing on top; left free, the
    five-dot P3 took 138 registers and fitted one block per SM. They keep the
    solve kernels' residency: P3 two blocks, P1 three, K4 four."""
    assert _blocks(_find(step_report, "k_step_pipe_p3")[0]) >= 2
    assert _blocks(_find(step_report, "k_step_pipe_p1")[0]) >= 3
    regs, spill = _find(step_report, "k_step_cls_k4")
    assert _blocks(regs) >= 4 and spill == 0
    assert _blocks(_find(step_report, "k_step_cls_k1")[0]) >= 3
    assert _blocks(_find(step_report, "k_step_cls_k3")[0]) >= 3


@pytest.fixture(scope="module")
def dot_report(tmp_path_factory):
    return _ptxas_report(tmp_path_factory, "kernels_spmv.cu")


def _blocks_of(regs, threads):
    per_warp = ((regs + 7) // 8) * 8 * 32
    return REGS_PER_SM // (per_warp * (threads // 32))


def test_long_row_kernels_fit_three_four_warp_blocks(dot_report, report):
    """The register-staged long-row SpMV holds each row's values and x entries
    in registers and relies on three 128-thread blocks per SM (12 warps) to keep
    a chain of fmas ready on every SM sub-partition: at most 168 registers, and
    the standalone kernel without spills. The fused classic K1/K3 on long rows
    keep the same residency."""
    for name in ("k_spmv_regILb0", "k_spmv_regILb1"):
        regs, spill = _find(dot_report, name)
        assert _blocks_of(regs, 128) >= 3 and spill == 0, (name, regs, spill)
    for kern, red in (("k_cls_k1", "ExactRILi1"), ("k_cls_k3", "ExactRILi2")):
        regs, _ = _find(report, kern, red, "Li1024E")
        assert _blocks_of(regs, 128) >= 3, (kern, regs)
