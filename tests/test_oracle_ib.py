"""Pins of the oracle's immersed-boundary part (Section 3.4.2, Eq. 33-36):
printed kernel values, the kernel's partition of unity and its sum of
squares (closed forms), brute-force Eq. 34 over the whole grid, force
conservation, adjointness of spreading and interpolation, exact
interpolation of a uniform flow."""
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))


def test_phi_printed_values(oracle_lib):
    for r, val in GOLD["delta_kernel_eq36"]["samples"]:
        assert math.isclose(oracle_lib.phi(r), val, rel_tol=0, abs_tol=1e-15)
    for r in (2.0001, -2.5, 7.0):
        assert oracle_lib.phi(r) == 0.0


def test_partition_of_unity_and_squares(oracle_lib):
    rng = np.random.default_rng(0)
    for x in rng.uniform(-3, 3, size=200):
        js = np.arange(math.floor(x) - 1, math.floor(x) + 3)
        vals = np.array([oracle_lib.phi(x - j) for j in js])
        assert abs(vals.sum() - 1.0) < 1e-14
        assert abs((vals ** 2).sum() - 3.0 / 8.0) < 1e-14
        # nothing outside the 4-point support
        assert abs(oracle_lib.phi(x - (math.floor(x) - 2))) < 1e-16
        assert oracle_lib.phi(x - (math.floor(x) + 3)) == 0.0


def _brute_spread(nx, ny, nz, X, F):
    """Eq. 34 summed over every cell of the grid and over the periodic images
    in x and y, cells outside 0 <= k < nz dropped."""
    M = X.shape[1]
    g = np.zeros((3, nz, ny, nx))
    ph = lambda r: np.where(np.abs(r) <= 2, 0.25 * (1 + np.cos(np.pi * r / 2)), 0.0)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for m in range(M):
        for sx in (-nx, 0, nx):
            for sy in (-ny, 0, ny):
                w = ph(I + sx - X[0, m]) * ph(J + sy - X[1, m]) * ph(K - X[2, m])
                g += F[:, m][:, None, None, None] * w
    return g.reshape(3, -1)


def test_spread_matches_brute_force(oracle_lib):
    rng = np.random.default_rng(1)
    nx, ny, nz = 7, 6, 9
    p = oracle_lib.lb_params(nx, ny, nz, 0.8)
    M = 12
    X = np.vstack([rng.uniform(-1, nx + 1, M), rng.uniform(-1, ny + 1, M), rng.uniform(-1.2, nz, M)])
    X[:, 0] = (0.0, 0.0, 0.0)    # exactly on a cell centre and on the periodic seam
    X[:, 1] = (nx - 0.5, 2.0, -0.49)
    F = rng.standard_normal((3, M))
    g = oracle_lib.ib_spread(p, np.ascontiguousarray(X).ravel(), np.ascontiguousarray(F).ravel())
    assert np.allclose(g, _brute_spread(nx, ny, nz, X, F).ravel(), atol=1e-14)


def test_force_conservation_and_adjointness(oracle_lib):
    rng = np.random.default_rng(2)
    nx, ny, nz = 8, 7, 10
    N = nx * ny * nz
    p = oracle_lib.lb_params(nx, ny, nz, 0.8)
    M = 30
    # interior nodes: total force is conserved by spreading
    X = np.vstack([rng.uniform(0, nx, M), rng.uniform(0, ny, M), rng.uniform(2.0, nz - 3.0, M)])
    F = rng.standard_normal((3, M))
    g = oracle_lib.ib_spread(p, X.ravel(), F.ravel())
    assert np.allclose(g.reshape(3, N).sum(1), F.sum(1), atol=1e-13)
    # anywhere (also near the walls): <g, v> = sum_m F_m . U_m
    X[2] = rng.uniform(-0.5, nz - 0.5, M)
    g = oracle_lib.ib_spread(p, X.ravel(), F.ravel())
    v = rng.standard_normal(3 * N)
    U = oracle_lib.ib_interp(p, X.ravel(), v)
    assert math.isclose(float(g @ v), float(F.ravel() @ U), rel_tol=1e-12)


def test_uniform_flow_interpolated_exactly(oracle_lib):
    rng = np.random.default_rng(4)
    nx, ny, nz = 6, 6, 9
    N = nx * ny * nz
    p = oracle_lib.lb_params(nx, ny, nz, 0.8)
    u0 = np.array([0.3, -0.1, 0.05])
    v = np.repeat(u0, N)
    X = np.vstack([rng.uniform(-2, 8, 20), rng.uniform(0, 6, 20), rng.uniform(2.0, nz - 3.0, 20)])
    U = oracle_lib.ib_interp(p, X.ravel(), v).reshape(3, -1)
    assert np.allclose(U, u0[:, None], atol=1e-14)
