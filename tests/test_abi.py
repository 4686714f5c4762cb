"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/platelet_fsi.h declares; host-side validation rejects bad
arguments before anything reaches the device (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1312_2234_b300 import build, fsi, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return fsi.lib()


def declared():
    h = open(os.path.join(ROOT, "include", "platelet_fsi.h")).read()
    return re.findall(r"^\s*int\s+(\w+)\s*\(", h, re.M)


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 20
    for n in ("lb_create", "lb_step", "ib_interp", "ib_spread", "membrane_forces", "bonds_step", "sim_step"):
        assert n in names
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []
    assert set(fsi._SIGS) == set(names)
    assert L.pfsi_version() >= 100


def test_lb_query_sizes_validation(L):
    s = fsi.lb_sizes()
    p = fsi.lb_params(128, 64, 64, 0.8, (ctypes.c_float * 3)(0, 0, 0), (ctypes.c_float * 3)(0, 0, 0))
    assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == 0
    N = 128 * 64 * 64
    assert s.n_cells == N and s.f_bytes == 19 * 4 * N and s.g_bytes == 16 * N and s.flag_bytes == 4 * 64 * 64
    p.nz = 1
    assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == -1
    assert "nz" in fsi.last_error()
    p.nz, p.nx = 64, 2 ** 20
    assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == -1
    assert L.lb_query_sizes(None, ctypes.byref(s)) == -1


def test_lb_query_sizes_mixed_storage(L):
    s = fsi.lb_sizes()
    z = (ctypes.c_float * 3)(0, 0, 0)
    N = 48 * 40 * 36
    for mode in (fsi.LB_BF16, fsi.LB_FP16):
        p = fsi.lb_params(48, 40, 36, 0.8, z, z, mode, 12)
        assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == 0
        assert s.f_bytes == 19 * 2 * N and s.v_bytes == 16 * N
    p = fsi.lb_params(48, 40, 36, 0.8, z, z, 3, 0)
    assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == -1
    assert "storage" in fsi.last_error()
    p = fsi.lb_params(48, 40, 36, 0.8, z, z, fsi.LB_FP16, 61)
    assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == -1
    assert "fp16_exponent" in fsi.last_error()
    p = fsi.lb_params(48, 40, 36, 0.8, z, z, fsi.LB_FP32, 0, 2)
    assert L.lb_query_sizes(ctypes.byref(p), ctypes.byref(s)) == -1
    assert "wall" in fsi.last_error()


def test_lb_create_checks_the_storage_mode(L):
    z = (ctypes.c_float * 3)(0, 0, 0)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    p = fsi.lb_params(8, 8, 8, 0.8, z, z, fsi.LB_BF16, 0)
    assert L.lb_create(ctypes.byref(p), fake, fake, fake, fake, fake, ctypes.byref(h)) == -1
    assert "PFSI_LB_FP32" in fsi.last_error()
    p.storage = fsi.LB_FP32
    assert L.lb_create_mixed(ctypes.byref(p), fake, fake, fake, fake, fake, fake, ctypes.byref(h)) == -1
    assert "PFSI_LB_BF16" in fsi.last_error()
    p.storage = fsi.LB_FP16
    odd = ctypes.c_void_p(0x1008)
    assert L.lb_create_mixed(ctypes.byref(p), fake, fake, odd, fake, fake, fake, ctypes.byref(h)) == -1
    assert "aligned" in fsi.last_error()


def test_default_fp16_exponent_keeps_shear_fneq_normal():
    """The first-order f^neq of a Couette flow, w tau |u_top| / nz, scaled by
    the default 2^s, lands in FP16's normal range with room above it."""
    for u, nz, tau in [(2.2e-4, 64, 0.8), (4e-3, 19, 0.8), (0.05, 32, 1.379), (0.0, 16, 0.9)]:
        s = fsi.default_fp16_exponent(nz, tau, (u, 0.0, 0.0))
        fneq = (1 / 36) * tau * max(u / nz, 1e-6) * 2.0 ** s
        assert 2.0 ** -14 < fneq < 1.0


def test_lb_create_rejects_bad_buffers(L):
    p = fsi.lb_params(8, 8, 8, 0.8, (ctypes.c_float * 3)(0, 0, 0), (ctypes.c_float * 3)(0, 0, 0))
    h = ctypes.c_void_p()
    assert L.lb_create(ctypes.byref(p), None, None, None, None, None, ctypes.byref(h)) == -1
    fake = ctypes.c_void_p(0x1000)
    odd = ctypes.c_void_p(0x1004)
    assert L.lb_create(ctypes.byref(p), odd, fake, fake, fake, fake, ctypes.byref(h)) == -1
    assert "aligned" in fsi.last_error()
    p.tau = 0.5
    assert L.lb_create(ctypes.byref(p), fake, fake, fake, fake, fake, ctypes.byref(h)) == -1
    assert "tau" in fsi.last_error()


def test_membrane_workspace_query_and_validation(L):
    w = workload.config_small()
    m = w["mesh"]
    nb = fsi.membrane_query_workspace(w["M"], m["tri"], len(m["pairs"]), 1)
    assert nb > 0 and nb % 256 == 0
    bad = np.array(m["tri"], copy=True)
    bad[0, 0] = w["M"] + 5
    with pytest.raises(RuntimeError, match="out of range"):
        fsi.membrane_query_workspace(w["M"], bad, 0, 1)
    flipped = np.array(m["tri"], copy=True)
    flipped[0] = flipped[0, [0, 2, 1]]
    with pytest.raises(RuntimeError, match="orient"):
        fsi.membrane_query_workspace(w["M"], flipped, 0, 1)


def test_bond_workspace_query_and_validation(L):
    w = workload.config_small()
    p = fsi.bond_params_from(w["bonds"])
    assert fsi.bonds_query_workspace(p, 100) >= 256 * 16 * 4
    p.lig_i0 = 30
    with pytest.raises(RuntimeError, match="patch"):
        fsi.bonds_query_workspace(p, 100)
    # capture beyond one lattice spacing is accepted (the 2r x 2r window)
    assert fsi.bonds_query_workspace(fsi.bond_params_from(dict(w["bonds"], d_capture=1.5)), 100) > 0
    for bad in (0.0, -0.5, 8.5, float("nan"), 16.5):
        p = fsi.bond_params_from(dict(w["bonds"], d_capture=bad))
        with pytest.raises(RuntimeError, match="d_capture"):
            fsi.bonds_query_workspace(p, 100)
    # the window must fit the box once: 2 ceil(d_capture) <= box lengths
    p = fsi.bond_params_from(dict(w["bonds"], d_capture=4.5, box_nx=9, lig_i0=0, lig_ni=8))
    with pytest.raises(RuntimeError, match="d_capture"):
        fsi.bonds_query_workspace(p, 100)


def test_fem_workspace_and_validation(L):
    """Six-node element lists are checked on the host before any copy."""
    w = workload.config_small()
    e6 = np.ascontiguousarray(w["mesh"]["elem6"], dtype=np.int32)
    assert e6.shape == (320, 6)
    nb = ctypes.c_size_t()
    assert L.fem_query_workspace(w["M"], len(e6), ctypes.byref(nb)) == 0
    assert nb.value % 256 == 0 and nb.value >= len(e6) * 6 * (16 + 8)
    assert L.fem_query_workspace(0, len(e6), ctypes.byref(nb)) == -1
    fake = ctypes.c_void_p(1 << 20)     # never dereferenced: validation fails first
    h = ctypes.c_void_p()
    for bad, msg in ((w["M"] + 1, "out of range"), (e6[0, 1], "repeated")):
        b = e6.copy()
        b[0, 0] = bad
        assert L.fem_create(w["M"], len(b), b.ctypes.data_as(ctypes.c_void_p), fake, ctypes.c_size_t(nb.value),
                            ctypes.byref(h)) == -1
        assert msg in fsi.last_error()
    assert L.fem_create(w["M"], len(e6), e6.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p((1 << 20) + 8),
                        ctypes.c_size_t(nb.value), ctypes.byref(h)) == -1
    assert "aligned" in fsi.last_error()


def test_bridge_workspace_and_parameter_validation(L):
    """Bridge parameters are checked on the host (capture distance, kT and
    the periodic box positive, rates non-negative) and the workspace grows
    with the sites, platelets and nodes."""
    w = workload.config_pair(seed=0, level=2, n_sce=10, n_sites=100)
    ok = fsi.bridge_params_from(w["bridges"])
    nb = ctypes.c_size_t()
    assert L.bridges_query_workspace(ctypes.byref(ok), 200, 2, w["M"], ctypes.byref(nb)) == 0
    small = nb.value
    assert small % 256 == 0
    assert L.bridges_query_workspace(ctypes.byref(ok), 20000, 2, w["M"], ctypes.byref(nb)) == 0
    assert nb.value > small
    for bad in (dict(d_capture=0.0), dict(kT=0.0), dict(kon0_dt=-1.0), dict(koff0_dt=-1.0), dict(box_nx=0)):
        p = fsi.bridge_params_from(dict(w["bridges"], **bad))
        assert L.bridges_query_workspace(ctypes.byref(p), 200, 2, w["M"], ctypes.byref(nb)) == -1
        assert "invalid parameters" in fsi.last_error()
    assert L.bridges_query_workspace(ctypes.byref(ok), 200, 0, w["M"], ctypes.byref(nb)) == -1
    assert L.bridges_query_workspace(ctypes.byref(ok), 200, 2, 0, ctypes.byref(nb)) == -1


def test_lattice_batch_validates_its_arguments(L):
    h = ctypes.c_void_p()
    assert L.lb_batch_create(None, 2, ctypes.byref(h)) == -1
    arr = (ctypes.c_void_p * 1)(None)
    assert L.lb_batch_create(ctypes.cast(arr, ctypes.c_void_p), 0, ctypes.byref(h)) == -1
    assert L.lb_batch_create(ctypes.cast(arr, ctypes.c_void_p), 1, ctypes.byref(h)) == -1
    assert "null lattice" in fsi.last_error()
    assert L.lb_batch_step(None, 1, None) == -1
    assert L.lb_batch_autotune(None, 1, None, None) == -1
    assert L.lb_batch_get_shapes(None, None) == -1
    assert L.lb_batch_set_shapes(None, None) == -1
    assert L.lb_batch_destroy(None) == 0
    assert L.batch_autotune(None, 1, None, None) == -1


def test_product_path_fails_loudly_without_the_library(monkeypatch):
    monkeypatch.setattr(fsi, "_lib", None)
    monkeypatch.setattr(fsi, "LIB_PATH", "/nonexistent/libplatelet_fsi.so")
    with pytest.raises(RuntimeError, match="not built"):
        fsi.lib()


def test_wait_selftest_rejects_bad_arguments():
    L = fsi.lib()
    assert L.pfsi_wait_selftest(0, None, None) == -1
    assert L.pfsi_wait_selftest(5, None, None) == -1


def test_tether_calls_validate_their_arguments():
    L = fsi.lib()
    n = ctypes.c_size_t()
    assert L.tether_query_workspace(-1, 2, ctypes.byref(n)) == -1
    assert L.tether_query_workspace(10, 3, None) == -1
    assert L.tether_query_workspace(10, 3, ctypes.byref(n)) == 0 and n.value >= 4 * 4 + 4 * 10
    h = ctypes.c_void_p()
    assert L.tether_create(None, 3, None, None, 0, None, None, 0, None, ctypes.byref(h)) == -1
    assert L.tether_update(None, 0, None) == -1
    assert L.sim_set_tether(None, None) == -1
