"""Pins of the FP64 finite-element bending oracle (Section 3.1, Eq. 6-10)
against what the mathematics fixes, not against itself:

* the quadratic six-node basis (Eq. 7): partition of unity, Kronecker
  property at the nodes, exact reproduction of every quadratic polynomial and
  its derivatives;
* the six-node elements of the icosphere cover its triangles exactly once;
* curvatures (Eq. 9-10) converge to the closed forms on a sphere and on a
  triaxial ellipsoid, K = (a^2+b^2+c^2-|x|^2)/(2 a^2 b^2 c^2 p^(3/2)),
  K_G = 1/(a^2 b^2 c^2 p^2), p = x^2/a^4 + y^2/b^4 + z^2/c^4;
* the surface Laplacian converges to the spherical-harmonic eigenvalues
  (Lap_S z = -2 z, Lap_S xy = -6 xy on the unit sphere);
* the bending force is the negative first variation of the energy of Eq. 6:
  its work along a smooth deformation converges to -dH/d(eps), which fixes
  the sign, the factor k0/2 and the Gaussian-curvature term (a force without
  it, or with another factor, fails by far);
* rigid motions rotate the forces, and scaling all positions by s scales the
  forces by 1/s (exact, up to rounding)."""
import numpy as np
import pytest

from oracle import fem
from paper_1312_2234_b300 import workload


def sphere(level, R=1.0):
    U, T, E = workload.icosphere_elements(level)
    return U * R, T, E


def test_basis_partition_kronecker_and_quadratic_reproduction():
    for j, (xi, eta) in enumerate(fem.NODE_XI):
        N, _, _ = fem.shape(xi, eta)
        assert np.allclose(N, np.eye(6)[j], atol=1e-15)
    rng = np.random.default_rng(0)
    c = rng.standard_normal(6)

    def poly(x, y):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y

    def dpoly(x, y):
        return c[1] + 2 * c[3] * x + c[4] * y, c[2] + c[4] * x + 2 * c[5] * y

    u = np.array([poly(x, y) for x, y in fem.NODE_XI])
    for _ in range(20):
        r = rng.uniform(size=2)
        if r.sum() > 1:
            r = 1 - r
        N, dxi, deta = fem.shape(*r)
        assert abs(N.sum() - 1) < 1e-14 and abs(dxi.sum()) < 1e-13 and abs(deta.sum()) < 1e-13
        assert abs(N @ u - poly(*r)) < 1e-13
        gx, gy = dpoly(*r)
        assert abs(dxi @ u - gx) < 1e-12 and abs(deta @ u - gy) < 1e-12


@pytest.mark.parametrize("level", [1, 2, 3])
def test_elements_cover_the_triangles(level):
    X, T, E = sphere(level)
    assert len(E) * 4 == len(T)
    sub = np.sort(E[:, fem.SUB_TRI].reshape(-1, 3), axis=1)
    assert np.array_equal(np.unique(sub, axis=0), np.unique(np.sort(T, axis=1), axis=0))
    # midpoint nodes: two elements each, at the normalised midpoint of their edge
    counts = np.bincount(E[:, 3:].ravel(), minlength=len(X))
    assert set(counts[E[:, 3:].ravel()]) == {2}
    for m, (a, b) in zip((3, 4, 5), ((0, 1), (1, 2), (2, 0))):
        mid = X[E[:, a]] + X[E[:, b]]
        assert np.allclose(X[E[:, m]], mid / np.linalg.norm(mid, axis=1, keepdims=True), atol=1e-14)
    # outward orientation of every element
    n = np.cross(X[E[:, 1]] - X[E[:, 0]], X[E[:, 2]] - X[E[:, 0]])
    assert np.all(np.einsum("ij,ij->i", n, X[E[:, 0]]) > 0)


def test_sphere_curvatures_converge():
    R = 2.5
    errs = []
    for level in (3, 4, 5):
        X, _, E = sphere(level, R)
        K, KG = fem.curvatures(X, E)
        errs.append((np.abs(K * R - 1).max(), np.abs(KG * R * R - 1).max()))
    for (k1, g1), (k2, g2) in zip(errs, errs[1:]):
        assert k2 < k1 / 2.5 and g2 < g1 / 2.5
    assert errs[-1][0] < 1e-4 and errs[-1][1] < 2e-4


def test_ellipsoid_curvatures_closed_form():
    a, b, c = 1.0, 0.8, 0.6
    errs = []
    for level in (3, 4):
        U, _, E = workload.icosphere_elements(level)
        X = U * np.array([a, b, c])
        x, y, z = X.T
        p = x * x / a ** 4 + y * y / b ** 4 + z * z / c ** 4
        KG = 1.0 / (a * a * b * b * c * c * p * p)
        K = (a * a + b * b + c * c - (x * x + y * y + z * z)) / (2 * a * a * b * b * c * c * p ** 1.5)
        Kh, KGh = fem.curvatures(X, E)
        errs.append((np.abs(Kh - K).max() / K.max(), np.abs(KGh - KG).max() / KG.max()))
    assert errs[1][0] < errs[0][0] / 2.5 and errs[1][1] < errs[0][1] / 2.5
    assert errs[1][0] < 1e-2 and errs[1][1] < 2e-2


def test_laplace_beltrami_spherical_harmonics():
    prev = None
    for level in (3, 4, 5):
        X, _, E = sphere(level)
        e1 = np.abs(fem.laplace_beltrami(X, E, X[:, 2]) + 2 * X[:, 2]).max()
        e2 = np.abs(fem.laplace_beltrami(X, E, X[:, 0] * X[:, 1]) + 6 * X[:, 0] * X[:, 1]).max()
        assert np.abs(fem.laplace_beltrami(X, E, np.full(len(X), 3.0))).max() < 1e-10
        if prev is not None:
            assert e1 < prev[0] / 2.5 and e2 < prev[1] / 1.4
        prev = (e1, e2)
    assert prev[0] < 2e-2 and prev[1] < 3e-2


def _work_and_energy_rate(level, scale_axis, eps0, k0=1.7, force=fem.bending_forces):
    U, _, E = workload.icosphere_elements(level)

    def X(e):
        s = np.ones(3)
        s[scale_axis] += e
        return U * s

    h = 1e-5
    dE = (fem.bending_energy(X(eps0 + h), E, k0) - fem.bending_energy(X(eps0 - h), E, k0)) / (2 * h)
    dX = (X(eps0 + h) - X(eps0 - h)) / (2 * h)
    return float(np.sum(force(X(eps0), E, k0) * dX)), -dE


@pytest.mark.parametrize("axis,eps0,tol4", [(2, -0.3, 4e-3), (0, 0.2, 1.6e-2), (2, -0.75, 3e-2)])
def test_force_is_the_energy_variation(axis, eps0, tol4):
    rel = []
    for level in (3, 4):
        W, mdE = _work_and_energy_rate(level, axis, eps0)
        rel.append(abs(W - mdE) / abs(mdE))
    assert rel[1] < tol4 and rel[1] < rel[0]


def test_energy_variation_rejects_planted_mistakes():
    """Forces with the printed 2 K^3 term, with the opposite sign or without
    the factor 1/2 miss the energy rate by far more than the discretisation
    error of the correct form."""
    def literal(X, E, k0):
        f = fem.bending_fields(X, E)
        return (f["A"] * 0.5 * k0 * (f["lapK"] + 2 * f["K"] ** 3))[:, None] * f["n"]

    W, mdE = _work_and_energy_rate(4, 2, -0.3)
    good = abs(W - mdE) / abs(mdE)
    for bad in (literal, lambda X, E, k0: -fem.bending_forces(X, E, k0),
                lambda X, E, k0: 2 * fem.bending_forces(X, E, k0)):
        Wb, _ = _work_and_energy_rate(4, 2, -0.3, force=bad)
        assert abs(Wb - mdE) / abs(mdE) > 20 * good


def test_rigid_motion_and_scaling():
    U, _, E = workload.icosphere_elements(3)
    X = U * np.array([1.0, 0.9, 0.35])
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    F = fem.bending_forces(X, E, 2.0)
    Fm = fem.bending_forces(X @ Q.T + np.array([3.0, -7.0, 11.0]), E, 2.0)
    assert np.abs(Fm - F @ Q.T).max() < 1e-9 * np.abs(F).max()
    s = 3.7
    Fs = fem.bending_forces(s * X, E, 2.0)
    assert np.abs(Fs - F / s).max() < 1e-10 * np.abs(F).max()


def test_soa_layout_matches():
    U, _, E = workload.icosphere_elements(2)
    X = U * np.array([1.0, 1.0, 0.5])
    F = fem.bending_forces(X, E, 1.0)
    Fs = fem.forces_soa(np.ascontiguousarray(X.T).ravel(), E, 1.0).reshape(3, -1).T
    assert np.array_equal(F, Fs)
