"""Pins of the FP64 surrogate reference (oracle/mlp.py) against facts that do
not come from its own formulas: the C reference's per-element membrane
forces and energy (a separate derivation of the same local terms), the
closed-form strains of a uniform dilation, regular-icosahedron geometry, the
exact-erf GELU, finite differences, rigid-motion invariance and equivariance,
the closed form of a first Adam step, and the linearity of the membrane force
in its coefficients."""
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


def tiny_state(seed=4, amp=0.03, level=2):
    w = workload.tiny(seed=seed, level=level)
    m = w["mesh"]
    n = m["node_plt"].size
    rng = np.random.default_rng(seed)
    X = w["X"] + amp * rng.standard_normal(w["X"].shape)
    ring, deg = mlp.one_rings(m["tri"], n)
    nodes = np.where((deg > 0) & (np.asarray(m["is_membrane"]) > 0))[0]
    mesh = oracle.Mesh(m["X0"], m["tri"], m["pairs"], m["node_plt"], m["is_membrane"], m["n_plt"])
    return w, mesh, X, m["X0"].reshape(3, n).T, X.reshape(3, n).T, ring, deg, nodes


def test_exact_stresses_reproduce_the_local_membrane_force():
    """The node shares' stresses through the strain gradients give the plain
    solver's local force (springs, local area, bending: the C reference's
    per-element formulas, a separate derivation)."""
    w, mesh, Xsoa, X0, X, ring, deg, nodes = tiny_state()
    x, m, _ = mlp.strains(X, X0, ring, deg, nodes)
    F = mlp.assemble(X, X0, ring, deg, nodes, mlp.exact_stresses(x, m, w["membrane"]))
    ref = mesh.forces(mlp.local_params(w["membrane"]), Xsoa).reshape(3, -1).T
    assert np.max(np.abs(F - ref)) < 1e-10 * np.abs(ref).max()
    # each term on its own (a dropped factor in one of them cannot hide)
    for only in ("k_spring", "k_t", "k_b"):
        q = dict(mlp.local_params(w["membrane"]))
        for k in ("k_spring", "k_t", "k_b"):
            if k != only:
                q[k] = 0.0
        F = mlp.assemble(X, X0, ring, deg, nodes, mlp.exact_stresses(x, m, q))
        ref = mesh.forces(q, Xsoa).reshape(3, -1).T
        assert np.max(np.abs(F - ref)) < 1e-10 * np.abs(ref).max(), only


def test_node_shares_sum_to_the_local_energy():
    w, mesh, Xsoa, X0, X, ring, deg, nodes = tiny_state(seed=6)
    t = mesh.energy_terms(w["membrane"], Xsoa)
    E = mlp.node_energy(X, X0, ring, deg, nodes, w["membrane"])
    ref = t[0] + t[1] + t[4]
    assert abs(E - ref) < 1e-11 * abs(ref)


def test_strains_of_a_uniform_dilation():
    """X -> (1 + a) X0: every spoke stretches by a, every face area by
    (1 + a)^2 - 1, no bending angle changes."""
    w, mesh, Xsoa, X0, X, ring, deg, nodes = tiny_state()
    for a in (1e-6, 0.02):
        x, m, r = mlp.strains((1 + a) * X0, X0, ring, deg, nodes)
        present = m[:, :6] > 0
        # FP64 differences of O(10) coordinates: ~1e-14 absolute
        assert np.allclose(x[:, :6][present], a, rtol=1e-9, atol=1e-13)
        assert np.allclose(x[:, 6:12][present], (1 + a) ** 2 - 1, rtol=1e-9, atol=1e-13)
        assert np.max(np.abs(x[:, 12:][present])) < 1e-12
        assert np.all(x[:, :6][~present] == 0) and np.all(r[:, :6][~present] == 0)


def test_rest_descriptors_of_the_regular_icosahedron():
    """All edges equal: L0/l = 1, S0/l^2 = sqrt(3)/4; every hinge at the
    icosahedron's dihedral angle arccos(-sqrt(5)/3), so |cos phi0| = sqrt(5)/3
    and |sin phi0| = 2/3; degree 5 leaves the sixth slot empty."""
    U, T = ico(0)
    ring, deg = mlp.one_rings(T, len(U))
    x, m, r = mlp.strains(U, U, ring, deg, np.arange(12))
    assert np.all(x == 0)
    assert np.allclose(r[:, 0:5], 1.0, atol=1e-14) and np.all(r[:, 5] == 0)
    assert np.allclose(r[:, 6:11], math.sqrt(3) / 4, atol=1e-14)
    assert np.allclose(r[:, 12:17], -math.sqrt(5) / 3, atol=1e-14)
    assert np.allclose(np.abs(r[:, 18:23]), 2.0 / 3.0, atol=1e-14)
    assert np.allclose(m[:, 0:5], np.linalg.norm(U[T[0, 0]] - U[T[0, 1]]) ** 2, atol=1e-14)


def rotation(rng):
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_strains_invariant_and_forces_equivariant_under_rigid_motion():
    rng = np.random.default_rng(1)
    U, T = ico(2)
    U = U * np.array([5.0, 5.0, 1.25])
    ring, deg = mlp.one_rings(T, len(U))
    X = U + 0.02 * rng.standard_normal(U.shape)
    Q = rotation(rng)
    c = np.array([3.0, -2.0, 7.5])
    nodes = np.arange(len(U))
    x1, m1, r1 = mlp.strains(X, U, ring, deg, nodes)
    x2, m2, r2 = mlp.strains(X @ Q.T + c, U, ring, deg, nodes)
    assert np.allclose(x1, x2, atol=1e-12) and np.array_equal(m1, m2) and np.array_equal(r1, r2)
    p = mlp.init_params(rng)
    F1 = mlp.predict_forces(p, X, U, ring, deg, nodes)
    F2 = mlp.predict_forces(p, X @ Q.T + c, U, ring, deg, nodes)
    assert np.allclose(F2, F1 @ Q.T, atol=1e-12 * np.abs(F1).max())
    # the internal forces of any stresses sum to zero (translation
    # invariance of every strain)
    assert np.max(np.abs(F1.sum(0))) < 1e-12 * np.abs(F1).max()


def test_inputs_direction_and_rest_descriptors():
    rng = np.random.default_rng(3)
    U, T = ico(1)
    ring, deg = mlp.one_rings(T, len(U))
    X = U + 1e-3 * rng.standard_normal(U.shape)
    nodes = np.arange(len(U))
    x, m, r = mlp.strains(X, U, ring, deg, nodes)
    p = mlp.init_params(rng, in_scale=rng.uniform(0.5, 2.0, mlp.N_IN))
    p["in_shift"] = rng.uniform(-1, 1, mlp.N_IN)
    f = mlp.inputs(p, x, r)
    assert np.allclose(np.linalg.norm(f[:, :18], axis=1), 1.0, atol=1e-14)
    d5 = deg == 5
    for q in range(4):
        assert np.all(f[d5, 18 + 6 * q + 5] == 0)
        k = 18 + 6 * q
        assert np.allclose(f[~d5, k:k + 6], (r[~d5, 6 * q:6 * q + 6] - p["in_shift"][k:k + 6]) * p["in_scale"][k:k + 6])
    assert np.all(mlp.inputs(p, 0 * x, r)[:, :18] == 0)


def test_network_with_the_exact_moduli_gives_the_plain_force():
    """Output o = 1 with out_scale = the stress coefficients (zero last
    layer, unit bias) reproduces the plain local force up to the bending's
    sin x - x (relative x^2/6: below 1e-6 at these bending angles)."""
    w, mesh, Xsoa, X0, X, ring, deg, nodes = tiny_state(amp=3e-4)
    cs, ca, cb = mlp.stress_coefficients(w["membrane"])
    p = mlp.init_params(np.random.default_rng(0), out_scale=np.repeat([cs, ca, cb], 6))
    p["W3"][:] = 0.0
    p["b3"][:] = 1.0
    F = mlp.predict_forces(p, X, X0, ring, deg, nodes)
    ref = mesh.forces(mlp.local_params(w["membrane"]), Xsoa).reshape(3, -1).T
    assert np.max(np.abs(F - ref)) < 1e-6 * np.abs(ref).max()


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
    # strains are linear in the displacement to first order: the ratio is 2
    # up to a relative O(strain) (~1e-4 here)
    assert np.allclose(F2, 2 * F1, rtol=0, atol=1e-3 * np.abs(F1).max())


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    p = mlp.init_params(rng)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    f = rng.standard_normal((7, mlp.N_IN))
    a = rng.standard_normal((7, mlp.N_OUT))
    b = rng.standard_normal((7, mlp.N_OUT))
    o, cache = mlp.forward(p, f)
    g = mlp.backward(p, cache, o, a, b)
    h = 1e-6
    for k in mlp.TRAINED:
        idx = [tuple(rng.integers(0, s) for s in p[k].shape) for _ in range(6)]
        for ix in idx:
            old = p[k][ix]
            p[k][ix] = old + h
            lp = mlp.loss(mlp.forward(p, f)[0], a, b)
            p[k][ix] = old - h
            lm = mlp.loss(mlp.forward(p, f)[0], a, b)
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
