"""Pins of the oracle's lattice Boltzmann part (Section 3.3) against what the
paper prints and what the mathematics fixes: the D3Q19 table and numbering
(Eq. 21, Eq. 23-30), moment identities of the equilibrium (Eq. 20) and of
Guo's forcing (Eq. 19), streaming against an independent numpy shift, and the
closed-form Couette and Poiseuille profiles."""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))


def test_weights_and_isotropy(oracle_lib):
    c, w = oracle_lib.lattice()
    g = GOLD["d3q19_weights_eq21"]
    assert np.allclose(w[:6], g["axis"][0] / g["axis"][1])
    assert np.allclose(w[6:18], g["diagonal"][0] / g["diagonal"][1])
    assert np.isclose(w[18], g["rest"][0] / g["rest"][1])
    assert np.isclose(w.sum(), 1.0)
    assert np.allclose((w[:, None] * c).sum(0), 0.0)
    # second and fourth moments of an isotropic lattice with c_s^2 = 1/3
    M2 = np.einsum("q,qa,qb->ab", w, c, c)
    assert np.allclose(M2, np.eye(3) / 3.0)
    M4 = np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(M4, iso)
    # the 18 moving directions are distinct and have unit or sqrt(2) length
    assert len({tuple(v) for v in c}) == 19
    assert sorted(int(v @ v) for v in c) == [0] + [1] * 6 + [2] * 12


def test_numbering_matches_eq23_30(oracle_lib):
    c, _ = oracle_lib.lattice()
    cz = {i + 1: int(c[i, 2]) for i in range(19)}
    assert sorted(k for k, v in cz.items() if v == +1) == GOLD["unknown_at_bottom_wall"]["ids"]
    assert sorted(k for k, v in cz.items() if v <= 0) == GOLD["known_at_bottom_wall"]["ids"]
    assert sorted(k for k, v in cz.items() if v == -1) == GOLD["outgoing_in_eq23"]["ids"]
    for a, b in GOLD["opposite_pairs_eq24_28"]["pairs"]:
        assert np.array_equal(c[a - 1], -c[b - 1])
    s = GOLD["eq25_28_tangential_sign"]
    assert c[s["x_plus"] - 1, 0] == 1 and c[s["x_minus"] - 1, 0] == -1
    assert c[s["y_plus"] - 1, 1] == 1 and c[s["y_minus"] - 1, 1] == -1
    for key, axis in (("eq29_groups", 0), ("eq30_groups", 1)):
        grp = GOLD[key]
        assert all(c[i - 1, axis] == 1 and c[i - 1, 2] == 0 for i in grp["plus"])
        assert all(c[i - 1, axis] == -1 and c[i - 1, 2] == 0 for i in grp["minus"])


def test_time_step_of_section_3_3():
    from paper_1312_2234_b300 import workload
    t = GOLD["time_step"]
    nu = t["mu_Pa_s"] / t["rho_kg_m3"]
    L = workload.lattice_units(t["tau"])
    assert abs(L["dt"] - t["dt_s"]) / t["dt_s"] < 1e-3
    assert abs((t["tau"] - 0.5) * t["h_m"] ** 2 / (3 * nu) - t["dt_s"]) / t["dt_s"] < 1e-3
    k = GOLD["spring_constant"]
    assert math.isclose(2 * k["E_Pa"] * k["dx_m"] / 5, k["k_N_per_m"], rel_tol=1e-12)


def _numpy_stream(f_in, c, nx, ny, nz, u_top):
    """Independent streaming: np.roll per direction, halfway bounce-back at z."""
    N = nx * ny * nz
    F = f_in.reshape(19, nz, ny, nx)
    w = np.array([2 / 36] * 6 + [1 / 36] * 12 + [12 / 36])
    out = np.empty_like(F)
    opp = [int(np.nonzero((c == -c[q]).all(1))[0][0]) for q in range(19)]
    for q in range(19):
        cx, cy, cz = c[q]
        out[q] = np.roll(F[q], shift=(cz, cy, cx), axis=(0, 1, 2))
        if cz == 1:
            out[q][0] = F[opp[q]][0]
        if cz == -1:
            out[q][nz - 1] = F[opp[q]][nz - 1] + 6 * w[q] * (c[q] @ np.array(u_top))
    return out.reshape(19, N)


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_streaming_and_collision_moments(oracle_lib, tau):
    """Per cell: mass kept, momentum += F, momentum flux relaxed with the Guo
    second moment (1 - 1/2tau)(vF + Fv); the streamed moments come from an
    independent numpy shift."""
    rng = np.random.default_rng(3)
    nx, ny, nz = 5, 4, 6
    N = nx * ny * nz
    u_top = (2e-2, -1e-2, 0.0)
    p = oracle_lib.lb_params(nx, ny, nz, tau, u_top, (1e-4, 0, -2e-4))
    c, w = oracle_lib.lattice()
    f_in = np.repeat(w, N) + 1e-2 * rng.standard_normal(19 * N)
    g = 1e-3 * rng.standard_normal(3 * N)
    f_out, rho, v = oracle_lib.lb_step(p, f_in, g)
    fs = _numpy_stream(f_in, c, nx, ny, nz, u_top)
    F = g.reshape(3, N) + np.array([1e-4, 0, -2e-4])[:, None]
    rho_s = fs.sum(0)
    m_s = np.einsum("qa,qn->an", c, fs)
    assert np.allclose(rho, rho_s, rtol=0, atol=1e-14)
    assert np.allclose(v.reshape(3, N), (m_s + F / 2) / rho_s, rtol=0, atol=1e-14)
    fo = f_out.reshape(19, N)
    assert np.allclose(fo.sum(0), rho_s, atol=1e-14)
    assert np.allclose(np.einsum("qa,qn->an", c, fo), m_s + F, atol=1e-14)
    V = v.reshape(3, N)
    Pi_s = np.einsum("qa,qb,qn->abn", c, c, fs)
    Pi_eq = rho_s * (np.eye(3)[:, :, None] / 3.0 + V[:, None, :] * V[None, :, :])
    guo2 = (1 - 1 / (2 * tau)) * (V[:, None, :] * F[None, :, :] + F[:, None, :] * V[None, :, :])
    Pi_out = np.einsum("qa,qb,qn->abn", c, c, fo)
    assert np.allclose(Pi_out, Pi_s - (Pi_s - Pi_eq) / tau + guo2, atol=1e-14)


def test_moving_wall_conserves_mass(oracle_lib):
    rng = np.random.default_rng(5)
    nx, ny, nz = 6, 5, 7
    N = nx * ny * nz
    p = oracle_lib.lb_params(nx, ny, nz, 0.7, (3e-2, 1e-2, 0.0))
    c, w = oracle_lib.lattice()
    f = np.repeat(w, N) * (1 + 1e-2 * rng.standard_normal(19 * N))
    m0 = f.sum()
    for _ in range(50):
        f, rho, v = oracle_lib.lb_step(p, f)
    assert abs(f.sum() - m0) < 1e-12 * m0


def test_couette_steady_state(oracle_lib):
    """BGK with halfway bounce-back holds the linear Couette profile exactly;
    started from rest it converges to u_x = U (k + 1/2) / nz."""
    nx, ny, nz, U = 3, 2, 8, 1e-3
    p0 = oracle_lib.lb_params(nx, ny, nz, 0.8, (0, 0, 0))
    f = oracle_lib.lb_init_shear(p0)  # rest
    p = oracle_lib.lb_params(nx, ny, nz, 0.8, (U, 0, 0))
    for _ in range(4000):
        f, rho, v = oracle_lib.lb_step(p, f)
    N = nx * ny * nz
    ux = v[:N].reshape(nz, ny, nx)
    exact = U * (np.arange(nz) + 0.5) / nz
    assert np.allclose(ux, exact[:, None, None], rtol=1e-10, atol=0)
    assert np.allclose(v[N:], 0.0, atol=1e-11 * U)
    # the shear initial state is the converged one
    f0 = oracle_lib.lb_init_shear(p)
    _, _, v0 = oracle_lib.lb_step(p, f0)
    assert np.allclose(v0[:N].reshape(nz, ny, nx), exact[:, None, None], rtol=1e-9)


@pytest.mark.parametrize("tau,tol", [(0.5 + math.sqrt(3.0) / 4.0, 1e-9), (0.8, 5e-3)])
def test_poiseuille(oracle_lib, tau, tol):
    """Body-force Poiseuille flow between still walls at z = -1/2, nz - 1/2:
    u = G/(2 nu)(k + 1/2)(nz - 1/2 - k), nu = (tau - 1/2)/3.  Halfway
    bounce-back places the wall exactly for (tau - 1/2)^2 = 3/16; at tau = 0.8
    the slip error is O(1/nz^2)."""
    nx, ny, nz, G = 2, 2, 12, 1e-6
    p = oracle_lib.lb_params(nx, ny, nz, tau, (0, 0, 0), (G, 0, 0))
    f = oracle_lib.lb_init_shear(p)
    for _ in range(12000):
        f, rho, v = oracle_lib.lb_step(p, f)
    N = nx * ny * nz
    nu = (tau - 0.5) / 3.0
    k = np.arange(nz)
    exact = G / (2 * nu) * (k + 0.5) * (nz - 0.5 - k)
    ux = v[:N].reshape(nz, ny, nx)[:, 0, 0]
    assert np.max(np.abs(ux - exact)) / exact.max() < tol


@pytest.mark.parametrize("nz,u_top,tau", [(9, (1e-3, 0.0, 0.0), 0.8), (12, (1e-3, -6e-4, 0.0), 1.379)])
def test_onsite_walls_couette_is_exact(oracle_lib, nz, u_top, tau):
    """On-site velocity walls (Eq. 23-30) on the node planes k = 0 and nz - 1:
    started from rest, the flow converges to the linear profile
    u = u_top k/(nz - 1) exactly (BGK with velocity walls on the nodes
    reproduces a linear shear with no slip), and the shear initial state is
    that profile."""
    nx, ny = 3, 2
    p0 = oracle_lib.lb_params(nx, ny, nz, tau, (0, 0, 0), walls=1)
    f = oracle_lib.lb_init_shear(p0)  # rest
    p = oracle_lib.lb_params(nx, ny, nz, tau, u_top, walls=1)
    for _ in range(6000):
        f, rho, v = oracle_lib.lb_step(p, f)
    N = nx * ny * nz
    prof = np.arange(nz) / (nz - 1)
    for d in range(2):
        exact = u_top[d] * prof
        assert np.allclose(v[d * N:(d + 1) * N].reshape(nz, ny, nx), exact[:, None, None], rtol=1e-10,
                           atol=1e-12 * abs(u_top[0]))
    assert np.allclose(v[2 * N:], 0.0, atol=1e-11 * abs(u_top[0]))
    assert np.allclose(rho, 1.0, atol=1e-12)
    f0 = oracle_lib.lb_init_shear(p)
    _, _, v0 = oracle_lib.lb_step(p, f0)
    assert np.allclose(v0[:N].reshape(nz, ny, nx), (u_top[0] * prof)[:, None, None], rtol=1e-9, atol=1e-15)


def test_onsite_walls_impose_the_wall_velocity(oracle_lib):
    """For any state, the wall nodes' populations after streaming carry
    exactly the wall velocity (no force): the rule's defining property,
    checked on the moments rather than on its formulas."""
    nx, ny, nz = 6, 5, 7
    u_top = (0.015, 0.004, 0.0)
    p = oracle_lib.lb_params(nx, ny, nz, 0.9, u_top, walls=1)
    rng = np.random.default_rng(4)
    f = oracle_lib.lb_init_shear(p) + 1e-3 * rng.standard_normal(19 * nx * ny * nz)
    _, rho, v = oracle_lib.lb_step(p, f)
    V = v.reshape(3, nz, ny, nx)
    assert np.max(np.abs(V[:, 0])) < 1e-14
    for d in range(3):
        assert np.max(np.abs(V[d, nz - 1] - u_top[d])) < 1e-14
    # the bulk is untouched by the wall mode: same result as bounce-back walls
    pb = oracle_lib.lb_params(nx, ny, nz, 0.9, u_top, walls=0)
    _, rho_b, v_b = oracle_lib.lb_step(pb, f)
    inner = slice(2, nz - 2)
    assert np.array_equal(v.reshape(3, nz, ny, nx)[:, inner], v_b.reshape(3, nz, ny, nx)[:, inner])


def test_thread_count_does_not_change_results(oracle_lib):
    """The oracle's parallel loops (independent cells and nodes) give the
    same bits on one host thread and on several."""
    p = oracle_lib.lb_params(23, 17, 11, 0.8, (3e-3, 1e-3, 0.0))
    rng = np.random.default_rng(5)
    f0 = oracle_lib.lb_init_shear(p)
    g = 1e-5 * rng.standard_normal(3 * 23 * 17 * 11)
    X = np.vstack([rng.uniform(0, 23, 300), rng.uniform(0, 17, 300), rng.uniform(-0.4, 10.4, 300)]).ravel()
    out = []
    for n in (1, 4):
        oracle_lib.set_threads(n)
        f = oracle_lib.lb_init_shear(p)
        f1, rho, v = oracle_lib.lb_step(p, f, g)
        U = oracle_lib.ib_interp(p, X, v)
        out.append((f, f1, rho, v, U))
    oracle_lib.set_threads(1)
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][0], f0)
