"""membrane_measure_static, the entry point for callers that cannot allocate
device memory: through the C ABI it must give the per-platelet area and
volume that membrane_measure gives (same tolerance as the membrane tests,
1e-6 relative), on two calls in a row (the static scratch keeps the previous
call's sums and must be cleared), and reject a context with more platelets
than its static scratch holds.  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu


def test_matches_membrane_measure_twice():
    w = workload.config_channel(seed=3)
    mem = fsi.Membrane(w["membrane"], w["mesh"])
    rng = np.random.default_rng(4)
    X = w["X"] + 0.02 * rng.standard_normal(w["X"].shape)
    Xd = torch.from_numpy(X).cuda()
    ref = mem.measure(Xd)
    for _ in range(2):
        got = fsi.membrane_measure_static(mem.h, Xd, mem.n_plt)
        assert np.allclose(got, ref, rtol=1e-6, atol=0)
    # a different input on the next call: no leftover sums
    X2 = Xd * 1.01
    ref2 = mem.measure(X2)
    got2 = fsi.membrane_measure_static(mem.h, X2, mem.n_plt)
    assert np.allclose(got2, ref2, rtol=1e-6, atol=0)
    assert not np.allclose(got2, ref, rtol=1e-6)


def tetrahedra(n_plt):
    """One small tetrahedron per platelet, platelet p scaled by 1 + p / n_plt
    (so each platelet's area and volume differ, the last one included)."""
    base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    tet = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    X = np.vstack([(1.0 + p / n_plt) * base + [3.0 * (p % 100), 3.0 * (p // 100), 5.0] for p in range(n_plt)])
    tri = np.vstack([tet + 4 * p for p in range(n_plt)])
    mesh = dict(X0=np.ascontiguousarray(X.T).ravel(), tri=tri, pairs=np.zeros((0, 2), np.int32),
                node_plt=np.repeat(np.arange(n_plt, dtype=np.int32), 4),
                is_membrane=np.ones(4 * n_plt, np.uint8), n_plt=n_plt)
    params = dict(k_spring=1.0, k_s=1.0, k_t=1.0, k_v=1.0, k_b=0.0, morse_D=0.0, morse_a=1.0,
                  rep_F0=0.0, rep_tau=1.0, rep_eps_min=1e-3, z_wall=-0.5)
    return fsi.Membrane(params, mesh), torch.from_numpy(mesh["X0"]).cuda()


def test_largest_context_uses_the_last_slot():
    """Exactly PFSI_STATIC_MAX_PLATELETS = 8192 platelets: every slot of the
    static array is used, the last platelet's included, on two calls."""
    n_plt = 8192
    mem, Xd = tetrahedra(n_plt)
    ref = mem.measure(Xd)
    for _ in range(2):
        got = fsi.membrane_measure_static(mem.h, Xd, n_plt)
        assert np.allclose(got, ref, rtol=1e-6, atol=0)
    s = 1.0 + (n_plt - 1) / n_plt
    assert np.allclose(got[-1], [s * s * (1.5 + 0.5 * np.sqrt(3.0)), s ** 3 / 6.0], rtol=1e-12)


def test_rejects_more_platelets_than_the_scratch_holds():
    n_plt = 8193
    mem, Xd = tetrahedra(n_plt)
    out = (ctypes.c_double * (2 * n_plt))()
    rc = fsi.lib().membrane_measure_static(mem.h, fsi._ptr(Xd), out, fsi._stream())
    assert rc == -1
    assert "exceed" in fsi.last_error() and "8192" in fsi.last_error()
