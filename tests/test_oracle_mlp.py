"""Pins of the FP64 surrogate reference (oracle/mlp.py) against facts that do
not come from its own formulas: the exact-erf GELU, finite differences,
icosahedron geometry, rigid-motion invariance, the closed form of a first
Adam step, and the linearity of the membrane force in its coefficients."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1312_2234_b300 import workload


def test_gelu_identities():
    z = np.linspace(-6, 6, 241)
    g = mlp.gelu(z)
    # tanh is odd: g(z) - g(-z) = z exactly
    assert np.allclose(g - mlp.gelu(-z), z, atol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # the tanh form stays within 1e-3 of the exact x Phi(x)
    exact = np.array([0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0))) for x in z])
    assert np.max(np.abs(g - exact)) < 1e-3
    assert abs(mlp.gelu(np.array([30.0]))[0] - 30.0) < 1e-12
    assert abs(mlp.gelu(np.array([-30.0]))[0]) < 1e-12


def test_gelu_grad_by_central_differences():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


def ico(level):
    U, T = workload.icosphere(level)
    return U, T


def test_one_rings_follow_face_orientation():
    U, T = ico(1)
    ring, deg = mlp.one_rings(T, len(U))
    assert set(deg.tolist()) == {5, 6} and (deg == 5).sum() == 12
    faces = {tuple(np.roll(f, -k)) for f in T.tolist() for k in range(3)}
    for i in range(len(U)):
        d = deg[i]
        assert ring[i, 0] == min(ring[i, :d])
        for k in range(d):
            assert (i, ring[i, k], ring[i, (k + 1) % d]) in faces


def test_rest_features_and_icosahedron_curvature():
    U, T = ico(0)
    ring, deg = mlp.one_rings(T, len(U))
    f, R, mag = mlp.features(U, U, ring, deg, np.arange(12))
    assert np.all(f[:, :18] == 0) and np.all(mag == 0)
    # all edges of the regular icosahedron are equal: rest-length ratios 1,
    # the sixth slot of a degree-5 node empty
    assert np.allclose(f[:, 21:26], 1.0, atol=1e-14) and np.all(f[:, 26] == 0)
    # regular icosahedron on the unit sphere: the five neighbours sit at
    # polar angle acos(1/sqrt 5), so the mean neighbour offset is
    # (1/sqrt 5 - 1) along the outward normal and the edge is sqrt(2 - 2/sqrt 5)
    kz = (1 / math.sqrt(5) - 1) / math.sqrt(2 - 2 / math.sqrt(5))
    assert np.allclose(f[:, 18:20], 0, atol=1e-14)
    assert np.allclose(f[:, 20], kz, atol=1e-14)
    # frames are orthonormal, right-handed, z outward
    for r, i in enumerate(range(12)):
        assert np.allclose(R[r] @ R[r].T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R[r]) - 1) < 1e-14
        assert R[r][2] @ U[i] > 0.99


def rotation(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_features_invariant_and_forces_equivariant_under_rigid_motion():
    rng = np.random.default_rng(1)
    U, T = ico(2)
    U = U * np.array([5.0, 5.0, 1.25])
    ring, deg = mlp.one_rings(T, len(U))
    X = U + 0.02 * rng.standard_normal(U.shape)
    Q = rotation(rng)
    c = np.array([3.0, -2.0, 7.5])
    nodes = np.arange(len(U))
    f1, _, m1 = mlp.features(X, U, ring, deg, nodes)
    f2, _, m2 = mlp.features(X @ Q.T + c, U, ring, deg, nodes)
    assert np.allclose(f1, f2, atol=1e-12) and np.allclose(m1, m2, atol=1e-12)
    p = mlp.init_params(rng)
    F1 = mlp.predict_forces(p, X, U, ring, deg, nodes)
    F2 = mlp.predict_forces(p, X @ Q.T + c, U, ring, deg, nodes)
    assert np.allclose(F2, F1 @ Q.T, atol=1e-12)


def test_uniform_dilation():
    """Under X -> (1 + a) X every edge vector grows by a in an unchanged
    frame: delta_k = a R0 e0_k / l, so the direction inputs are R0 e0_k / l
    over its norm for any a, the magnitude is a times that norm, and the rest
    inputs do not move."""
    U, T = ico(1)
    ring, deg = mlp.one_rings(T, len(U))
    f0, _, _ = mlp.features(U, U, ring, deg, np.arange(len(U)))
    for a in (1e-6, 0.01):
        f, _, mag = mlp.features((1 + a) * U, U, ring, deg, np.arange(len(U)))
        for i in range(len(U)):
            d = deg[i]
            nb = ring[i, :d]
            e0 = U[nb] - U[i]
            ell = np.linalg.norm(e0, axis=1).mean()
            R0 = mlp.frame(e0, d)
            c = np.concatenate([(R0 @ e0[k]) / ell for k in range(d)])
            assert abs(mag[i] - a * np.linalg.norm(c)) < 1e-9 * a
            assert np.allclose(f[i, :3 * d], c / np.linalg.norm(c), atol=1e-7)
            assert np.allclose(f[i, 18:], f0[i, 18:], atol=1e-15)
            assert np.all(f[i, 3 * d:18] == 0) and np.all(f[i, 21 + d:] == 0)


def test_surrogate_force_is_homogeneous_in_the_deformation():
    """Scaling a deformation of the rest shape by s scales the predicted
    local force by s (and it vanishes at rest)."""
    rng = np.random.default_rng(6)
    U, T = ico(2)
    ring, deg = mlp.one_rings(T, len(U))
    p = mlp.init_params(rng)
    D = rng.standard_normal(U.shape)
    nodes = np.arange(len(U))
    F1 = mlp.predict_forces(p, U + 1e-5 * D, U, ring, deg, nodes)
    F2 = mlp.predict_forces(p, U + 2e-5 * D, U, ring, deg, nodes)
    assert np.all(mlp.predict_forces(p, U, U, ring, deg, nodes) == 0)
    # the inputs are linear in the displacement only to first order (the
    # frame turns with it), so the ratio is 2 up to a relative O(strain)
    # (here ~2e-4)
    assert np.allclose(F2, 2 * F1, rtol=0, atol=1e-3 * np.abs(F1).max())


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    p = mlp.init_params(rng)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    f = rng.standard_normal((7, mlp.N_IN))
    t = rng.standard_normal((7, mlp.N_OUT))
    o, cache = mlp.forward(p, f)
    g = mlp.backward(p, cache, o, t)
    h = 1e-6
    for k in mlp.TRAINED:
        idx = [tuple(rng.integers(0, s) for s in p[k].shape) for _ in range(6)]
        for ix in idx:
            old = p[k][ix]
            p[k][ix] = old + h
            lp = mlp.loss(mlp.forward(p, f)[0], t)
            p[k][ix] = old - h
            lm = mlp.loss(mlp.forward(p, f)[0], t)
            p[k][ix] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k][ix] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, ix, g[k][ix], fd)


def test_first_adam_steps_closed_form():
    """With zero moments, bias correction makes m_hat = g and v_hat = g^2 at
    every step while the gradient stays the same, so each step moves a
    parameter by lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    p = mlp.init_params(rng)
    g = {k: rng.standard_normal(p[k].shape) for k in mlp.TRAINED}
    p0 = {k: p[k].copy() for k in mlp.TRAINED}
    state = {}
    lr, eps = 1e-3, 1e-8
    mlp.adam_step(p, g, state, lr, eps=eps)
    mlp.adam_step(p, g, state, lr, eps=eps)
    for k in mlp.TRAINED:
        step = lr * g[k] / (np.abs(g[k]) + eps)
        assert np.allclose(p[k], p0[k] - 2 * step, rtol=0, atol=1e-12)


def test_local_and_global_terms_split_the_membrane_force():
    w = workload.tiny(seed=4)
    m = w["mesh"]
    mesh = oracle.Mesh(m["X0"], m["tri"], m["pairs"], m["node_plt"], m["is_membrane"], m["n_plt"])
    rng = np.random.default_rng(5)
    X = w["X"] + 0.03 * rng.standard_normal(w["X"].shape)
    full = mesh.forces(w["membrane"], X)
    loc = mesh.forces(mlp.local_params(w["membrane"]), X)
    glo = mesh.forces(mlp.global_params(w["membrane"]), X)
    assert np.allclose(loc + glo, full, rtol=0, atol=1e-12 * np.abs(full).max())
    # the local terms vanish at rest
    assert np.abs(mesh.forces(mlp.local_params(w["membrane"]), m["X0"])).max() < 1e-12 * np.abs(full).max()
