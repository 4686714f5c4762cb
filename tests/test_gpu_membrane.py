"""GPU parity of membrane_forces / membrane_measure (Section 3.1, Eq. 2-11;
wall term of 3.4.1) against the FP64 oracle, term by term and in total, on
deformed platelets of the paper's shape.

Tolerance: the kernel forms every neighbour offset in FP64 and rounds it
once to FP32, then works in FP32.  The cancelling differences (|R| - L0,
S_t - S0, phi - phi0) then carry an absolute error ~2^-24 of the rest
length/area/angle, i.e. a relative error ~6e-8 / strain.  At the 2-3 %
random strains used here that is < 1e-5 of the largest nodal force, the
bound checked below; at the rest shape the force is zero to ~1e-6 of the
force a 1 % strain produces."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu
TERMS = ("spring", "area_local", "area_global", "volume", "bend", "morse", "wall")
OFF = dict(k_spring=0.0, k_s=0.0, k_t=0.0, k_v=0.0, k_b=0.0, morse_D=0.0, rep_F0=0.0)
ONLY = {"spring": ("k_spring",), "area_local": ("k_t",), "area_global": ("k_s",), "volume": ("k_v",),
        "bend": ("k_b",), "morse": ("morse_D",), "wall": ("rep_F0",)}


def f32(d):
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in d.items()}


def deformed(w, strain, seed):
    rng = np.random.default_rng(seed)
    X = w["X"].reshape(3, -1).copy()
    mem = w["mesh"]["is_membrane"].astype(bool)
    h = 0.5 * np.mean([np.linalg.norm(X[:, t[0]] - X[:, t[1]]) for t in w["mesh"]["tri"][:200]])
    X += strain * h * rng.standard_normal(X.shape)
    X[2, mem] = np.maximum(X[2, mem], -0.5 + 0.004)   # keep the surface off the wall
    return np.ascontiguousarray(X).ravel()


def setup(w, params, path=0):
    mem = fsi.Membrane(params, w["mesh"])
    mem.set_path(path)
    assert mem.fused == (path == 1)
    om = oracle.Mesh(w["mesh"]["X0"], w["mesh"]["tri"], w["mesh"]["pairs"], w["mesh"]["node_plt"],
                     w["mesh"]["is_membrane"], w["mesh"]["n_plt"])
    return mem, om


def gpu_forces(mem, X):
    Xd = torch.from_numpy(X).cuda()
    Fd = torch.empty(X.size, dtype=torch.float32, device="cuda")
    mem.forces(Xd, Fd)
    torch.cuda.synchronize()
    return Fd.cpu().numpy().astype(np.float64)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def small_workload():
    # the config's platelet moved down so that the wall term is active
    return workload.build(32, 32, 64, 0.8, 100.0, 1, 3, 200, 100, 0, patch=(8, 8, 16, 16), orient="flat",
                          gap=0.02, centers=[(16.0, 16.0, -0.5 + 0.02 + 1.25)])


# path 0: the three passes through slots; 1: the fused per-platelet pass
@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("term", TERMS)
def test_each_term(term, path):
    w = small_workload()
    base = f32(w["membrane"])
    params = dict(base, **{k: 0.0 for k in OFF})
    for k in ONLY[term]:
        params[k] = base[k]
    mem, om = setup(w, params, path)
    X = deformed(w, 0.03, 5)
    F = gpu_forces(mem, X)
    Fo = om.forces(params, X)
    assert np.max(np.abs(Fo)) > 0
    assert rel_err(F, Fo) < 1e-5, term


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("which", ["small", "channel"])
def test_total_force_and_measure(which, path):
    w = small_workload() if which == "small" else workload.config_channel()
    params = f32(w["membrane"])
    mem, om = setup(w, params, path)
    X = deformed(w, 0.02, 6)
    assert rel_err(gpu_forces(mem, X), om.forces(params, X)) < 1e-5
    SV = mem.measure(torch.from_numpy(X).cuda())
    S, V = om.measure(X)
    assert np.allclose(SV[:, 0], S, rtol=1e-6)
    assert np.allclose(SV[:, 1], V, rtol=1e-6)


@pytest.mark.parametrize("path", [0, 1])
def test_rest_shape_force_free(path):
    w = workload.build(32, 32, 64, 0.8, 100.0, 1, 3, 200, 100, 0, orient="random", gap=3.0)
    params = dict(f32(w["membrane"]), rep_F0=0.0)
    mem, _ = setup(w, params, path)
    F0 = gpu_forces(mem, w["X"])
    F1 = gpu_forces(mem, deformed(w, 0.01, 1))
    assert np.max(np.abs(F0)) < 1e-4 * np.max(np.abs(F1))


def test_fused_pass_falls_back_when_elements_are_not_grouped():
    """A mesh whose Morse pairs of one platelet come in two runs (or whose
    platelets exceed the shared memory) runs the three passes even with
    path 1; the forces still match the oracle, and the two paths agree on
    the grouped mesh to FP32 summation order (1e-6 of the largest force);
    the fused pass's exact sums give the same bits on a repeated call."""
    w = workload.config_channel()
    params = f32(w["membrane"])
    X = deformed(w, 0.02, 7)
    fused, _ = setup(w, params, 1)
    three, om = setup(w, params, 0)
    assert np.array_equal(gpu_forces(fused, X), gpu_forces(fused, X))
    Fo = om.forces(params, X)
    assert rel_err(gpu_forces(fused, X), gpu_forces(three, X)) < 1e-6
    mesh = dict(w["mesh"])
    pairs = np.asarray(mesh["pairs"]).reshape(-1, 2)
    n_first = int(np.sum(np.asarray(mesh["node_plt"])[pairs[:, 0]] == 0))
    assert n_first > 2
    order = np.r_[np.arange(1, n_first, 2), np.arange(n_first, len(pairs)), np.arange(0, n_first, 2)]
    mesh["pairs"] = pairs[order]
    mem = fsi.Membrane(params, mesh)
    mem.set_path(1)
    assert not mem.fused
    assert rel_err(gpu_forces(mem, X), Fo) < 1e-5
    big = workload.build(64, 64, 64, 0.8, 100.0, 1, 5, 0, 0, 0, orient="flat", gap=3.0)
    big_mem = fsi.Membrane(f32(big["membrane"]), big["mesh"])
    big_mem.set_path(1)
    assert not big_mem.fused
