"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads
without a GPU, and exports every entry point include/rbs.h declares. No
compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbs_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_04180_gb300 import build
    build.build()
    import paper_2302_04180_gb300 as rbs
    return rbs.load()


def test_header_declarations_are_exported(lib):
    import paper_2302_04180_gb300 as rbs
    names = _declared()
    assert len(names) >= 15
    assert set(names) == set(rbs.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_library_is_in_tree_and_sm103a(lib):
    from paper_2302_04180_gb300 import build
    assert os.path.dirname(build.LIB).startswith(ROOT)
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert "-fmad=false" in build.NVCC_FLAGS
    assert "sm_103a" in lib.rbs_version().decode()


def test_param_knobs_without_gpu(lib):
    import paper_2302_04180_gb300 as rbs
    rbs.rbs_set_param("exdot.window", 2)
    assert rbs.rbs_get_param("exdot.window") == 2
    rbs.rbs_set_param("exdot.window", 0)
    with pytest.raises(rbs.RbsError):
        rbs.rbs_set_param("no.such.knob", 1)


def test_no_cpu_fallback_when_library_missing(tmp_path):
    import paper_2302_04180_gb300 as rbs
    saved = rbs._lib
    try:
        rbs._lib = None
        with pytest.raises(RuntimeError):
            rbs.load(str(tmp_path / "missing.so"))
    finally:
        rbs._lib = saved
