"""Pins of the oracle's hybrid membrane (Section 3.1, Eq. 2-11; wall term of
Section 3.4.1): closed forms on a regular octahedron (area, volume, and every
energy under uniform scaling), a hinged pair of triangles for the bending
term, a single Morse pair, the wall potential, hand values for one spring
(Eq. 3), zero force at the rest shape, translation and rotation invariance,
and central-difference gradients of each energy term (F = -grad H)."""
import math

import numpy as np
import pytest

TERMS = ("spring", "area_local", "area_global", "volume", "bend", "morse", "wall")


def params(**on):
    base = dict(k_spring=0.0, k_s=0.0, k_t=0.0, k_v=0.0, k_b=0.0, morse_D=0.0, morse_a=2.0,
                rep_F0=0.0, rep_tau=3.0, rep_eps_min=1e-3, z_wall=-0.5)
    base.update(on)
    return base


def octahedron(r=1.0):
    X = np.array([[r, 0, 0], [-r, 0, 0], [0, r, 0], [0, -r, 0], [0, 0, r], [0, 0, -r]], float)
    T = []
    for a in (0, 1):
        for b in (2, 3):
            for c in (4, 5):
                t = [a, b, c]
                n = np.cross(X[b] - X[a], X[c] - X[a])
                if n @ (X[a] + X[b] + X[c]) < 0:
                    t = [a, c, b]
                T.append(t)
    return X, np.array(T, np.int32)


def make_mesh(oracle_lib, X, T, pairs=None, is_mem=None, plt=None, n_plt=1):
    n = len(X)
    pairs = np.zeros((0, 2), np.int32) if pairs is None else np.asarray(pairs, np.int32)
    is_mem = np.ones(n, np.uint8) if is_mem is None else np.asarray(is_mem, np.uint8)
    plt = np.zeros(n, np.int32) if plt is None else np.asarray(plt, np.int32)
    return oracle_lib.Mesh(np.ascontiguousarray(X.T).ravel(), T, pairs, plt, is_mem, n_plt)


def soa(X):
    return np.ascontiguousarray(np.asarray(X, float).T).ravel()


def test_octahedron_closed_forms(oracle_lib):
    r = 1.7
    X, T = octahedron(r)
    m = make_mesh(oracle_lib, X, T)
    S, V = m.measure(soa(X))
    assert m.n_edges == 12
    assert math.isclose(S[0], 4 * math.sqrt(3) * r * r, rel_tol=1e-14)
    assert math.isclose(V[0], 4.0 / 3.0 * r ** 3, rel_tol=1e-14)


def test_uniform_scaling_energies(oracle_lib):
    r, s = 1.3, 1.07
    X, T = octahedron(r)
    m = make_mesh(oracle_lib, X, T)
    S0, V0 = 4 * math.sqrt(3) * r * r, 4.0 / 3.0 * r ** 3
    k, kt, ks, kv, kb = 0.7, 1.1, 2.3, 0.9, 0.4
    e = m.energy_terms(params(k_spring=k, k_t=kt, k_s=ks, k_v=kv, k_b=kb), soa(s * X))
    # 12 edges of rest length r sqrt(2): sum k/2 (sL - L)^2
    assert math.isclose(e[0], 12 * 0.5 * k * ((s - 1) * r * math.sqrt(2)) ** 2, rel_tol=1e-12)
    # Eq. 4: both area terms scale as (s^2 - 1)^2 S0 / 2
    assert math.isclose(e[1], kt * (s * s - 1) ** 2 * S0 / 2, rel_tol=1e-12)
    assert math.isclose(e[2], ks * (s * s - 1) ** 2 * S0 / 2, rel_tol=1e-12)
    # Eq. 5
    assert math.isclose(e[3], kv * (s ** 3 - 1) ** 2 * V0 / 2, rel_tol=1e-12)
    # dihedral angles do not change under scaling
    assert abs(e[4]) < 1e-14


def test_hinged_triangles_bending(oracle_lib):
    X = np.array([[0, 0, 0], [1, 0, 0], [0.5, 1.0, 0], [0.5, -1.0, 0]], float)
    T = np.array([[0, 1, 2], [1, 0, 3]], np.int32)
    m = make_mesh(oracle_lib, X, T)
    kb = 0.8
    for beta in (0.1, 0.7, -0.4, 2.0):
        Y = X.copy()
        Y[3] = [0.5, -math.cos(beta), -math.sin(beta)]
        e = m.energy_terms(params(k_b=kb), soa(Y))
        assert math.isclose(e[4], kb * (1 - math.cos(beta)), rel_tol=1e-12)


def test_morse_pair(oracle_lib):
    X = np.array([[0, 0, 0], [1.0, 0.2, 0.1]], float)
    r0 = float(np.linalg.norm(X[1] - X[0]))
    m = make_mesh(oracle_lib, X, np.zeros((0, 3), np.int32), pairs=[[0, 1]], is_mem=[0, 0])
    D, a = 0.3, 1.7
    for r in (0.8 * r0, r0, 1.3 * r0):
        Y = X.copy()
        Y[1] = X[1] / r0 * r
        e = m.energy_terms(params(morse_D=D, morse_a=a), soa(Y))
        assert math.isclose(e[5], D * ((1 - math.exp(-a * (r - r0))) ** 2 - 1), rel_tol=1e-13)
        F = m.forces(params(morse_D=D, morse_a=a), soa(Y)).reshape(3, 2)
        mag = 2 * D * a * (1 - math.exp(-a * (r - r0))) * math.exp(-a * (r - r0))
        assert np.allclose(F[:, 0], mag * (Y[1] - Y[0]) / r, atol=1e-14)
        assert np.allclose(F[:, 0] + F[:, 1], 0, atol=1e-15)


def test_wall_potential(oracle_lib):
    X = np.array([[0.3, 0.2, 0.1]], float)
    m = make_mesh(oracle_lib, X, np.zeros((0, 3), np.int32))
    F0, tau, zw = 0.02, 5.0, -0.5
    for z in (-0.45, -0.2, 0.4):
        Y = X.copy()
        Y[0, 2] = z
        eps = z - zw
        P = params(rep_F0=F0, rep_tau=tau, rep_eps_min=1e-4, z_wall=zw)
        e = m.energy_terms(P, soa(Y))
        assert math.isclose(e[6], -F0 * math.log(1 - math.exp(-tau * eps)), rel_tol=1e-13)
        F = m.forces(P, soa(Y))
        assert math.isclose(F[2], F0 * tau / math.expm1(tau * eps), rel_tol=1e-12)
        assert F[0] == 0 and F[1] == 0


def test_single_spring_by_hand(oracle_lib):
    """Eq. 3 on one triangle: vertex 1 pulled from (1,0,0) to (1.1,0,0)."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    T = np.array([[0, 1, 2]], np.int32)
    m = make_mesh(oracle_lib, X, T)
    Y = X.copy()
    Y[1, 0] = 1.1
    k = 2.0
    F = m.forces(params(k_spring=k), soa(Y)).reshape(3, 3).T
    d12 = Y[2] - Y[1]
    L12 = np.linalg.norm(d12)
    f12 = k * (L12 - math.sqrt(2)) * d12 / L12      # pulls 1 toward 2
    assert np.allclose(F[0], [k * 0.1, 0, 0], atol=1e-14)
    assert np.allclose(F[1], [-k * 0.1, 0, 0] + f12, atol=1e-14)
    assert np.allclose(F[2], -f12, atol=1e-14)


def platelet(oracle_lib, level=1, n_sce=6, seed=0, deform=0.0, z_shift=0.0):
    from paper_1312_2234_b300 import workload
    rng = np.random.default_rng(seed)
    tp = workload.platelet_template(level, n_sce, 0, 5.0, 0.25, rng)
    X0 = np.vstack([tp["Xm"], tp["Xs"]])
    X0[:, 2] += z_shift
    nm = len(tp["Xm"])
    is_mem = np.r_[np.ones(nm), np.zeros(len(tp["Xs"]))]
    m = make_mesh(oracle_lib, X0, tp["T"], tp["pairs"], is_mem)
    Y = X0 + deform * rng.standard_normal(X0.shape)
    return m, X0, Y, tp


ALL_ON = params(k_spring=1.0, k_t=0.8, k_s=1.3, k_v=0.6, k_b=0.5, morse_D=0.4, morse_a=1.5,
                rep_F0=0.01, rep_tau=4.0, rep_eps_min=1e-3, z_wall=-0.5)


def test_zero_force_at_rest(oracle_lib):
    m, X0, _, tp = platelet(oracle_lib, level=2, n_sce=20, z_shift=40.0)
    assert len(tp["pairs"]) > 0
    P = dict(ALL_ON, rep_F0=0.0)
    F = m.forces(P, soa(X0))
    assert np.max(np.abs(F)) < 1e-12
    assert np.max(np.abs(m.energy_terms(P, soa(X0))[:5])) < 1e-20


def test_translation_rotation_invariance(oracle_lib):
    m, X0, Y, _ = platelet(oracle_lib, level=2, n_sce=20, deform=0.05)
    P = dict(ALL_ON, rep_F0=0.0)
    F = m.forces(P, soa(Y)).reshape(3, -1).T
    scale = np.abs(F).max()
    assert scale > 1e-3
    assert np.allclose(F.sum(0), 0, atol=1e-12 * scale * len(F))
    torque = np.cross(Y, F).sum(0)
    assert np.allclose(torque, 0, atol=1e-11 * scale * len(F))


@pytest.mark.parametrize("term", TERMS)
def test_forces_are_minus_energy_gradient(oracle_lib, term):
    m, X0, Y, _ = platelet(oracle_lib, level=1, n_sce=6, deform=0.08, seed=3, z_shift=0.9)
    single = {
        "spring": dict(k_spring=1.0), "area_local": dict(k_t=1.0), "area_global": dict(k_s=1.0),
        "volume": dict(k_v=1.0), "bend": dict(k_b=1.0), "morse": dict(morse_D=1.0, morse_a=1.5),
        "wall": dict(rep_F0=0.05, rep_tau=2.0, rep_eps_min=1e-4),
    }[term]
    P = params(**single)
    x = soa(Y)
    F = m.forces(P, x)
    idx = TERMS.index(term)
    h = 1e-6
    num = np.empty_like(x)
    for i in range(x.size):
        xp = x.copy()
        xm = x.copy()
        xp[i] += h
        xm[i] -= h
        num[i] = -(m.energy_terms(P, xp)[idx] - m.energy_terms(P, xm)[idx]) / (2 * h)
    scale = np.abs(F).max()
    assert scale > 0
    assert np.max(np.abs(num - F)) < 2e-7 * scale
