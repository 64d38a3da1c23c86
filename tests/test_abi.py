"""The C-ABI library loads and exports every call include/dpd.h declares;
argument validation of dpd_create needs no GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "dpd.h")).read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(dpd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def binding():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def test_every_declared_symbol_is_exported(binding):
    names = _declared()
    assert len(names) >= 14
    lib = C.CDLL(binding.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(binding.EXPORTED)


def test_strerror_and_defaults(binding):
    assert binding.strerror(binding.DPD_EINVAL) == "invalid argument"
    assert binding.strerror(binding.DPD_EUNSTABLE).startswith("non-finite")
    o = binding.default_options()
    assert abs(o.lambda_ - 0.65) < 1e-15 and o.precision == binding.DPD_FP32
    assert o.use_graph == 0 and o.cuda_stream is None


@pytest.mark.parametrize("case", ["small_box", "asym_a", "bad_type", "bad_bond", "dt0",
                                  "self_bond", "ntypes"])
def test_create_rejects_bad_arguments(binding, case):
    L, types, a = 5.0, np.zeros(4, np.int32), np.array([[25.0]])
    bonds, dt = None, 0.04
    if case == "small_box":
        L = (5.0, 2.5, 5.0)
    elif case == "asym_a":
        types = np.array([0, 1, 0, 1], np.int32)
        a = np.array([[25.0, 30.0], [31.0, 25.0]])
    elif case == "bad_type":
        types = np.array([0, 0, 3, 0], np.int32)
    elif case == "bad_bond":
        bonds = dict(i=[0], j=[9], kind=[1], r0=[0.0], k=[4.0], alpha=[0.0])
    elif case == "self_bond":
        bonds = dict(i=[1], j=[1], kind=[1], r0=[0.0], k=[4.0], alpha=[0.0])
    elif case == "dt0":
        dt = 0.0
    elif case == "ntypes":
        a = np.full((17, 17), 25.0)
    with pytest.raises(binding.DPDError) as e:
        binding.System(L, types, a, 4.5, 1.0, dt, bonds=bonds)
    assert e.value.code == binding.DPD_EINVAL


def test_wait_check_rejects_bad_arguments(binding):
    # argument checks come before any CUDA call
    assert binding.wait_check(True, tries=0) == binding.DPD_EINVAL
    assert binding.wait_check(True, tries=binding.WAIT_CHECK_MAX_TRIES + 1) == binding.DPD_EINVAL


def test_noalloc_rejects_overflowing_boxes_before_touching_memory(binding):
    # host-side checks: the pointers are never dereferenced for these sizes
    fake = 0x1000
    big = float(binding.NOALLOC_MAX_CELLS)
    for L in ((big, big, big), (big + 1.0, 3.0, 3.0), (2048.0, 2048.0, 2048.0),
              (1e300, 3.0, 3.0), (float("inf"), 3.0, 3.0), (float("nan"), 3.0, 3.0)):
        assert binding.cells_noalloc(fake, 10, L, fake, fake, fake) == binding.DPD_EINVAL, L
    assert binding.cells_noalloc(fake, binding.NOALLOC_MAX_N + 1, 50.0, fake, fake,
                                 fake) == binding.DPD_EINVAL
    assert binding.cells_noalloc(fake, 0, 50.0, fake, fake, fake) == binding.DPD_EINVAL


@pytest.mark.parametrize("L", [(4194304.0, 4194304.0, 4194304.0), (2.0 ** 31, 3.0, 3.0),
                               (1e10, 1e10, 1e10), (65536.0, 65536.0, 3.0)])
def test_create_rejects_boxes_with_too_many_cells(binding, L):
    # rejected while validating the box, before any device allocation
    with pytest.raises(binding.DPDError) as e:
        binding.System(L, np.zeros(4, np.int32), np.array([[25.0]]), 4.5, 1.0, 0.04)
    assert e.value.code == binding.DPD_EINVAL
    assert "too many cells" in str(e.value)


def test_grid_wait_check_rejects_bad_arguments(binding):
    # argument checks come before any CUDA call
    assert binding.grid_wait_check(True, budget_cycles=0) == binding.DPD_EINVAL
    assert binding.grid_wait_check(
        True, budget_cycles=binding.GRID_WAIT_CHECK_MAX_CYCLES + 1) == binding.DPD_EINVAL
