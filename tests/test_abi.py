"""Host-side checks of the C ABI library: it loads without a GPU and exports every
symbol include/trg.h declares; argument errors are reported, not raised."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "trg.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:trg_status|const char \*)\s*(trg_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_2507_21909_b300 as pkg
    path = pkg.library_path()
    if not os.path.exists(path):
        from paper_2507_21909_b300 import build
        build.build()
    return ctypes.CDLL(path)


def test_header_lists_the_four_core_calls():
    syms = declared_symbols()
    for s in ("trg_init_ising", "trg_step", "trg_free_energy", "trg_magnetisation_impurity"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    import paper_2507_21909_b300 as pkg
    assert sorted(pkg.EXPORTED) == declared_symbols()


def test_argument_errors_without_gpu(lib):
    lib.trg_set_params.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_int]
    assert lib.trg_set_params(0, 4, 1, 0) == -1          # q_swap >= 1
    assert lib.trg_set_params(4, -1, 1, 0) == -1         # q_rho >= 0
    assert lib.trg_set_params(4, 4, 1, 9) == -1          # precision (0..8)
    assert lib.trg_set_params(4, 4, 0x5EED, 0) == 0
    lib.trg_set_bond_overspan.argtypes = [ctypes.c_int]
    assert lib.trg_set_bond_overspan(0) == -1            # r_bond >= 1
    assert lib.trg_set_bond_overspan(9) == -1            # r_bond <= 8
    assert lib.trg_set_bond_overspan(1) == 0
    lib.trg_last_error.restype = ctypes.c_char_p
    assert lib.trg_last_error() == b"ok"


def test_set_state_rejects_bad_state_without_gpu(lib):
    """The state is validated before anything touches the device."""
    lib.trg_set_state.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double]
    lib.trg_last_error.restype = ctypes.c_char_p
    buf = (ctypes.c_double * 32)()
    dims = (ctypes.c_int * 5)(2, 2, 2, 2, 2)
    good_axes = (ctypes.c_int * 4)(1, 2, 3, 0)
    for axes in ((0, 1, 2, 2), (0, 1, 2, 4), (-1, 1, 2, 3)):
        a = (ctypes.c_int * 4)(*axes)
        assert lib.trg_set_state(0.1, dims, buf, buf, None, a, 0, 0.0) == -1
        assert b"permutation" in lib.trg_last_error()
    bad_dims = (ctypes.c_int * 5)(2, 0, 2, 2, 2)
    assert lib.trg_set_state(0.1, bad_dims, buf, buf, None, good_axes, 0, 0.0) == -1
    assert lib.trg_set_state(float("nan"), dims, buf, buf, None, good_axes, 0, 0.0) == -1
    assert lib.trg_set_state(0.1, dims, buf, buf, None, good_axes, -1, 0.0) == -1
    assert lib.trg_set_state(0.1, dims, None, buf, None, good_axes, 0, 0.0) == -1


def test_new_entry_points_reject_without_gpu(lib):
    """Argument and state checks of the ATRG comparator and the impurity pair come before
    any device work."""
    lib.trg_atrg_init_ising.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.trg_atrg_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.trg_internal_energy.argtypes = [ctypes.c_void_p]
    assert lib.trg_atrg_init_ising(1, 0.2, 0.0) == -1         # d in 2..4
    assert lib.trg_atrg_init_ising(5, 0.2, 0.0) == -1
    assert lib.trg_atrg_init_ising(2, -0.1, 0.0) == -1        # beta >= 0
    assert lib.trg_atrg_step(0, 4, 8) == -6                   # no ATRG model yet
    assert lib.trg_set_impurity_pair() == -6                  # no model yet
    assert lib.trg_internal_energy(None) == -1                # NULL output


def test_set_state_rejects_nonfinite_buffers_without_gpu(lib):
    """NaN or Inf in a host state buffer is reported (TRG_ERR_NONFINITE) before upload."""
    lib.trg_set_state.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double]
    lib.trg_last_error.restype = ctypes.c_char_p
    dims = (ctypes.c_int * 5)(2, 2, 2, 2, 2)
    axes = (ctypes.c_int * 4)(0, 1, 2, 3)
    good = (ctypes.c_double * 32)(*([1.0] * 32))
    for bad_value, where in ((float("nan"), 5), (float("inf"), 31), (-float("inf"), 0)):
        bad = (ctypes.c_double * 32)(*([1.0] * 32))
        bad[where] = bad_value
        for args in ((bad, good, None), (good, bad, None), (good, good, bad)):
            assert lib.trg_set_state(0.2, dims, *args, axes, 0, 0.0) == -4
            assert f"index {where}".encode() in lib.trg_last_error()


def test_sketch_calls_without_network_without_gpu(lib):
    """The learned-sketch calls report a missing network before any device work."""
    x = (ctypes.c_float * 5)()
    u = (ctypes.c_float * 1)()
    lib.trg_sketch_forward.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                       ctypes.c_int]
    lib.trg_sketch_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                    ctypes.c_void_p, ctypes.c_void_p]
    lib.trg_sketch_train.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_ulonglong, ctypes.c_void_p]
    assert lib.trg_sketch_forward(x, 1, u, 1) == -6
    g = (ctypes.c_float * 67585)()
    assert lib.trg_sketch_grad(x, u, 1, None, g) == -6
    assert lib.trg_sketch_train(x, u, 1, 1, 1, ctypes.c_float(1e-3), 0, None) == -6
    assert lib.trg_sketch_forward(None, 1, u, 1) == -1
    assert lib.trg_set_sketch_mode(1) == -6
