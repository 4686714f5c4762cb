"""GPU parity of the finite-element bending term (Section 3.1, Eq. 6-10)
against the FP64 oracle, node by node: normals, areas, K, K_G, Lap_S K and
the force, on platelet meshes of the channel workload with smooth
deformations, and the coupled step with the finite-element bending selected.

Tolerances.  The kernels work in FP32 on coordinates relative to each
element's first corner, so each first derivative (tangents, normal
derivatives) carries a relative rounding error of a few u = 2^-24 of the
element's size, and each further derivative divides the error of the
previous field by the element size again: a few u for normals and areas,
~10 u for K and K_G, ~100 u for Lap_S K and the force (three derivative
levels of the positions), each relative to the field's largest value.
Measured on the deformed channel meshes: 3e-7 (normals), 2e-7 (areas),
1.1e-6 (K), 1.9e-6 (K_G), 6.3e-6 (Lap_S K), 6.5e-6 (force).  The membrane
fields are held to the 1e-5 relative bound of the other membrane parity
tests (1e-6 for normals and areas); the coupled step keeps the same 1e-5
(measured 3e-7 .. 6e-7)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fem
from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def deformed_channel_mesh(seed=0):
    """Channel workload meshes (10 discoid platelets, level 4, with SCE
    nodes) under a smooth, low-mode deformation of every platelet."""
    w = workload.config_channel(seed=seed)
    m = w["mesh"]
    M = w["M"]
    X = w["X"].reshape(3, M).T.copy()
    plt = np.asarray(m["node_plt"])
    rng = np.random.default_rng(seed + 1)
    for p in range(int(m["n_plt"])):
        sel = plt == p
        c = X[sel].mean(0)
        Y = X[sel] - c
        k = rng.uniform(0.1, 0.3, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        X[sel] = c + Y + 0.15 * np.stack([np.sin(k[0] * Y[:, 1] + ph[0]), np.sin(k[1] * Y[:, 2] + ph[1]),
                                          np.sin(k[2] * Y[:, 0] + ph[2])], axis=1)
    return w, X


def test_fields_and_forces_match_the_oracle():
    w, X = deformed_channel_mesh()
    E = np.asarray(w["mesh"]["elem6"]).reshape(-1, 6)
    fb = fsi.FemBending(w["mesh"])
    Xd = torch.as_tensor(np.ascontiguousarray(X.T).ravel()).cuda()
    f = {k: v.cpu().numpy().astype(np.float64) for k, v in fb.fields(Xd).items()}
    ref = fem.bending_fields(X, E)
    mem = np.asarray(w["mesh"]["is_membrane"]).astype(bool)
    errs = {
        "n": rel(np.stack([f["nx"], f["ny"], f["nz"]], 1)[mem], ref["n"][mem]),
        "A": rel(f["A"], ref["A"]),
        "K": rel(f["K"], ref["K"]),
        "KG": rel(f["KG"], ref["KG"]),
        "lapK": rel(f["lapK"], ref["lapK"]),
    }
    k0 = 2.5e-3
    F = torch.zeros(3 * w["M"], device="cuda")
    fb.forces(k0, Xd, F)
    Fr = fem.bending_forces(X, E, k0)
    errs["F"] = rel(F.reshape(3, -1).T.cpu().numpy(), Fr)
    print("fem rel errors", errs)
    assert errs["n"] < 1e-6 and errs["A"] < 1e-6
    assert errs["K"] < 1e-5 and errs["KG"] < 1e-5
    assert errs["lapK"] < 1e-5 and errs["F"] < 1e-5
    # SCE nodes (no element) get nothing
    assert float(F.reshape(3, -1)[:, torch.as_tensor(~mem).cuda()].abs().max()) == 0.0


def test_far_from_the_origin_and_accumulate():
    """Moving the mesh by 1000 lattice units changes nothing beyond FP32
    rounding of the force (the element arithmetic is relative to each
    element's corner), and accumulate adds to F."""
    w, X = deformed_channel_mesh(seed=3)
    fb = fsi.FemBending(w["mesh"])
    k0 = 1e-3
    Xd = torch.as_tensor(np.ascontiguousarray(X.T).ravel()).cuda()
    Xf = torch.as_tensor(np.ascontiguousarray((X + np.array([1000.25, -700.5, 0.0])).T).ravel()).cuda()
    F0 = torch.zeros(3 * w["M"], device="cuda")
    F1 = torch.zeros_like(F0)
    fb.forces(k0, Xd, F0)
    fb.forces(k0, Xf, F1)
    scale = float(F0.abs().max())
    print("fem translated rel change", float((F1 - F0).abs().max()) / scale)
    assert float((F1 - F0).abs().max()) < 1e-5 * scale
    base = torch.randn_like(F0)
    F2 = base.clone()
    fb.forces(k0, Xd, F2, accumulate=True)
    assert torch.allclose(F2, base + F0, rtol=0, atol=1e-6 * (1 + scale))
    # deterministic: fixed-order node sums
    F3 = torch.zeros_like(F0)
    fb.forces(k0, Xd, F3)
    assert torch.equal(F3, F0)


def f32_workload(w):
    w = dict(w)
    w["membrane"] = {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in w["membrane"].items()}
    g = dict(w["grid"])
    g["tau"] = float(np.float32(g["tau"]))
    g["u_top"] = tuple(float(np.float32(u)) for u in g["u_top"])
    w["grid"] = g
    return w


@pytest.mark.parametrize("level", [2, 3])
def test_coupled_step_with_fem_bending(level):
    """The coupled step with the finite-element bending in place of the
    dihedral term (modulus raised 100x so that it shapes the motion) against
    the oracle's coupled step: displacements and node velocities within
    1e-5 of their largest entries after 10 steps."""
    w = workload.tiny(seed=2, level=level, n_sce=20, n_sites=60, shear=3.0e4)
    w["membrane"] = dict(w["membrane"], bending="fem", k0=100.0 * w["membrane"]["k0"])
    w = f32_workload(w)
    sim = fsi.Simulation(w)
    ora = oracle.Sim(w)
    steps = 10
    sim.step(steps)
    for _ in range(steps):
        ora.step()
    torch.cuda.synchronize()
    X0 = w["X"]
    ex = rel(sim.X.cpu().numpy() - X0, ora.X - X0)
    eu = rel(sim.U.cpu().numpy(), ora.U)
    print("coupled fem level", level, ex, eu)
    assert ex < 1e-5 and eu < 1e-5
    if sim.bonds is not None:
        assert np.array_equal(sim.bonds.bound.cpu().numpy(), ora.bound)
