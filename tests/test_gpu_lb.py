"""GPU parity of lb_init_shear / lb_step (Section 3.3) against the FP64
oracle, element by element on the populations (stored shifted, f - w_q) and on
the force-corrected velocity written in forced rows.

Tolerance (FP32 populations, FP32 collision): each step rounds every shifted
population once (relative 2^-24 of |f~|) and the collision adds a few more
roundings of terms of the same size, so after n steps the error stays below
~n * 1e-7 of max |f~|; the bound 1e-5 * max |f~| holds for the windows used."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi

pytestmark = pytest.mark.gpu
TOL = 1e-5


def shifted_oracle(f):
    _, w = oracle.lattice()
    N = f.size // 19
    return f.reshape(19, N) - w[:, None]


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("dims", [(37, 23, 19), (128, 64, 64), (5, 3, 2)])
def test_init_and_free_steps(dims):
    nx, ny, nz = dims
    u_top = (4e-3, -1.5e-3, 0.0)
    lat = fsi.Lattice(nx, ny, nz, 0.8, u_top, (2e-6, 0.0, -1e-6))
    lat.init_shear()
    p = oracle.lb_params(nx, ny, nz, float(np.float32(0.8)),
                         tuple(float(np.float32(u)) for u in u_top),
                         (float(np.float32(2e-6)), 0.0, float(np.float32(-1e-6))))
    f = oracle.lb_init_shear(p)
    torch.cuda.synchronize()
    assert rel_err(lat.current().cpu().numpy(), shifted_oracle(f)) < 1e-6
    n = 12
    lat.step(n)
    for _ in range(n):
        f, rho, v = oracle.lb_step(p, f)
    torch.cuda.synchronize()
    assert rel_err(lat.current().cpu().numpy(), shifted_oracle(f)) < TOL


def test_forced_rows_step():
    """Force in flagged rows only: populations, velocity/density output, and
    the force field cleared where it was consumed."""
    nx, ny, nz = 45, 17, 13
    N = nx * ny * nz
    rng = np.random.default_rng(7)
    lat = fsi.Lattice(nx, ny, nz, 0.7, (2e-3, 0.0, 0.0))
    lat.init_shear()
    flags = (rng.uniform(size=ny * nz) < 0.3).astype(np.int32)
    g = np.zeros((N, 4), np.float32)
    rows = np.repeat(flags, nx).astype(bool)
    g[rows, :3] = (1e-4 * rng.standard_normal((rows.sum(), 3))).astype(np.float32)
    lat.g.copy_(torch.from_numpy(g))
    lat.flags.copy_(torch.from_numpy(flags))
    lat.step(1)
    p = oracle.lb_params(nx, ny, nz, float(np.float32(0.7)), (float(np.float32(2e-3)), 0.0, 0.0))
    f0 = oracle.lb_init_shear(p)
    g64 = np.ascontiguousarray(g[:, :3].astype(np.float64).T).ravel()
    f1, rho, v = oracle.lb_step(p, f0, g64)
    torch.cuda.synchronize()
    assert rel_err(lat.current().cpu().numpy(), shifted_oracle(f1)) < TOL
    vg = lat.v.cpu().numpy()
    V = v.reshape(3, N).T
    assert rel_err(vg[rows, :3], V[rows]) < TOL
    assert np.max(np.abs(vg[rows, 3] - rho[rows])) < 1e-6
    assert np.all(lat.g.cpu().numpy()[rows] == 0)
    # rows that were not flagged got no force: the populations match the
    # oracle run with zero force there (already checked above globally)


def test_conservation_fp64_moments():
    """Still walls, no force: FP64 sums of mass and momentum on the device
    match the oracle's state after each window."""
    nx, ny, nz = 24, 20, 16
    lat = fsi.Lattice(nx, ny, nz, 0.9, (0.0, 0.0, 0.0))
    lat.init_shear()
    rng = np.random.default_rng(3)
    f = lat.current()
    f.add_(torch.from_numpy((1e-4 * rng.standard_normal(f.shape)).astype(np.float32)).cuda())
    m0 = lat.moments_fp64()
    f_or = f.double().cpu().numpy()
    _, w = oracle.lattice()
    f_or = (f_or + w[:, None]).ravel()
    p = oracle.lb_params(nx, ny, nz, float(np.float32(0.9)))
    lat.step(50)
    for _ in range(50):
        f_or, rho, v = oracle.lb_step(p, f_or)
    m1 = lat.moments_fp64()
    assert abs(m1[0] - m0[0]) < 1e-6 * m0[0]
    c, _ = oracle.lattice()
    F = f_or.reshape(19, -1)
    mom = (c.T.astype(np.float64) @ F).sum(1)
    assert abs(m1[0] - F.sum()) < 1e-6 * F.sum()
    assert np.allclose(m1[1:], mom, atol=1e-6 * np.abs(F - w[:, None]).sum())


@pytest.mark.parametrize("dims", [(37, 23, 19), (5, 3, 2)])
def test_onsite_walls(dims):
    """On-site velocity walls (Eq. 23-30) on the end layers, with a body
    force and a random perturbation of the developed profile: populations
    and velocities against the oracle after 12 steps."""
    nx, ny, nz = dims
    u_top = (4e-3, -1.5e-3, 0.0)
    body = (2e-6, 0.0, -1e-6)
    lat = fsi.Lattice(nx, ny, nz, 0.8, u_top, body, walls=1)
    lat.init_shear()
    p = oracle.lb_params(nx, ny, nz, float(np.float32(0.8)), tuple(float(np.float32(u)) for u in u_top),
                         tuple(float(np.float32(b)) for b in body), walls=1)
    f = oracle.lb_init_shear(p)
    torch.cuda.synchronize()
    assert rel_err(lat.current().cpu().numpy(), shifted_oracle(f)) < 1e-6
    rng = np.random.default_rng(5)
    pert = (1e-5 * rng.standard_normal(lat.current().shape)).astype(np.float32)
    lat.current().add_(torch.from_numpy(pert).cuda())
    f = f + pert.astype(np.float64).ravel()
    n = 12
    lat.step(n)
    for _ in range(n):
        f, rho, v = oracle.lb_step(p, f)
    torch.cuda.synchronize()
    assert rel_err(lat.current().cpu().numpy(), shifted_oracle(f)) < TOL
