"""GPU parity of ib_spread / ib_interp (Section 3.4.2, Eq. 33-36) against the
FP64 oracle: nodes across the periodic seams, on cell centres, next to and
inside the wall layers (scattered nodes: the per-node path), and the
platelet meshes of the channel workload (the shared-memory tile path);
spreading accumulates with FP32 atomics (any order), so the spread field is
compared within 1e-5 of its largest entry.  Row flags cover the support rows
(every row of a chunk's box when the chunk is tiled) and interpolation
clears them all."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def nodes(rng, nx, ny, nz, M):
    X = np.vstack([rng.uniform(-3, nx + 3, M), rng.uniform(-2, ny + 2, M), rng.uniform(-1.4, nz + 0.4, M)])
    X[:, 0] = (0.0, 0.0, 0.0)
    X[:, 1] = (nx - 1e-9, ny - 0.5, -0.5)
    X[:, 2] = (3.0, 4.0, nz - 1.0)
    X[:, 3] = (-1e3 * nx + 0.25, 2.5, 1.75)     # far periodic image
    return X


def support_rows(X, ny, nz):
    rows = set()
    for m in range(X.shape[1]):
        by, bz = int(np.floor(X[1, m])) - 1, int(np.floor(X[2, m])) - 1
        for c in range(4):
            k = bz + c
            if 0 <= k < nz:
                for b in range(4):
                    rows.add(k * ny + (by + b) % ny)
    return rows


def expected_rows(X, nx, ny, nz, chunk=64, cap=768):
    """Rows the spreading kernel flags: per chunk of 64 nodes, every row of the
    supports' bounding box when the box fits the 768-cell tile and is no
    wider than the grid, else the support rows."""
    rows = set()
    for s0 in range(0, X.shape[1], chunk):
        Xc = X[:, s0:s0 + chunk]
        b = np.floor(Xc).astype(np.int64) - 1
        z0, z1 = max(b[2].min(), 0), min(b[2].max() + 3, nz - 1)
        ex, ey, ez = b[0].max() + 4 - b[0].min(), b[1].max() + 4 - b[1].min(), z1 - z0 + 1
        if ez > 0 and ex <= nx and ey <= ny and ex * ey * ez <= cap:
            rows |= {k * ny + j % ny for k in range(z0, z1 + 1) for j in range(b[1].min(), b[1].max() + 4)}
        else:
            rows |= support_rows(Xc, ny, nz)
    return rows


def platelet_nodes():
    from paper_1312_2234_b300 import workload
    w = workload.config_channel(seed=1)
    return w["X"].reshape(3, -1).copy(), (128, 64, 64)


@pytest.mark.parametrize("dims,M", [((29, 21, 17), 700), ((128, 64, 64), 33620), ("platelets", 0)])
def test_spread_parity_and_flags(dims, M):
    rng = np.random.default_rng(11)
    if dims == "platelets":
        X, dims = platelet_nodes()
        M = X.shape[1]
    else:
        X = nodes(rng, *dims, M)
    nx, ny, nz = dims
    F = rng.standard_normal((3, M)).astype(np.float32)
    lat = fsi.Lattice(nx, ny, nz, 0.8)
    Xd = torch.from_numpy(np.ascontiguousarray(X).ravel()).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(F).ravel()).cuda()
    fsi.ib_spread(lat.h, Xd, Fd, M)
    p = oracle.lb_params(nx, ny, nz, 0.8)
    g = oracle.ib_spread(p, np.ascontiguousarray(X).ravel(), np.ascontiguousarray(F.astype(np.float64)).ravel())
    torch.cuda.synchronize()
    gg = lat.g.cpu().numpy()
    assert rel_err(gg[:, :3].T.ravel(), g) < TOL
    assert np.all(gg[:, 3] == 0)
    flags = lat.flags.cpu().numpy()
    assert set(np.nonzero(flags)[0].tolist()) == expected_rows(X, nx, ny, nz)


@pytest.mark.parametrize("dims,M", [((29, 21, 17), 700), ((128, 64, 64), 33620), ("platelets", 0)])
def test_interp_parity_advect_and_flag_clear(dims, M):
    rng = np.random.default_rng(12)
    if dims == "platelets":
        X, dims = platelet_nodes()
        M = X.shape[1]
    else:
        X = nodes(rng, *dims, M)
    nx, ny, nz = dims
    N = nx * ny * nz
    lat = fsi.Lattice(nx, ny, nz, 0.8)
    v = rng.standard_normal((N, 4)).astype(np.float32) * 1e-3
    lat.v.copy_(torch.from_numpy(v))
    Xd = torch.from_numpy(np.ascontiguousarray(X).ravel()).cuda()
    Ud = torch.zeros(3 * M, dtype=torch.float32, device="cuda")
    Fd = torch.zeros(3 * M, dtype=torch.float32, device="cuda")
    fsi.ib_spread(lat.h, Xd, Fd, M)                   # sets the flags
    fsi.ib_interp(lat.h, Xd, Ud, M, advect=True)
    p = oracle.lb_params(nx, ny, nz, 0.8)
    v64 = np.ascontiguousarray(v[:, :3].astype(np.float64).T).ravel()
    U = oracle.ib_interp(p, np.ascontiguousarray(X).ravel(), v64)
    torch.cuda.synchronize()
    Ug = Ud.cpu().numpy()
    assert rel_err(Ug, U) < TOL
    Xn = Xd.cpu().numpy()
    assert np.max(np.abs(Xn - (np.ascontiguousarray(X).ravel() + Ug.astype(np.float64)))) == 0.0
    assert np.max(np.abs(Xn - (np.ascontiguousarray(X).ravel() + U))) < 1e-9
    assert int(lat.flags.sum().item()) == 0


def test_adjoint_on_gpu():
    nx, ny, nz = 33, 19, 14
    N = nx * ny * nz
    M = 500
    rng = np.random.default_rng(13)
    X = nodes(rng, nx, ny, nz, M)
    F = rng.standard_normal((3, M)).astype(np.float32)
    v = rng.standard_normal((N, 4)).astype(np.float32)
    lat = fsi.Lattice(nx, ny, nz, 0.8)
    lat.v.copy_(torch.from_numpy(v))
    Xd = torch.from_numpy(np.ascontiguousarray(X).ravel()).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(F).ravel()).cuda()
    Ud = torch.zeros(3 * M, dtype=torch.float32, device="cuda")
    fsi.ib_spread(lat.h, Xd, Fd, M)
    fsi.ib_interp(lat.h, Xd, Ud, M, advect=False)
    torch.cuda.synchronize()
    lhs = float((lat.g[:, :3].double() * torch.from_numpy(v[:, :3]).double().cuda()).sum())
    rhs = float((Fd.double() * Ud.double()).sum())
    assert abs(lhs - rhs) < 1e-5 * (abs(lhs) + np.abs(F).sum())
    assert np.array_equal(Xd.cpu().numpy(), np.ascontiguousarray(X).ravel())
