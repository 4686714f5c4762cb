"""Pins of the oracle's adhesion part (Section 3.2, Eq. 12-14): Philox4x32-10
against NVIDIA's cuRAND host generator (an independent library routine that
runs on the CPU), uniformity, closed-form bond survival under a fixed force
(Bell model), the capacity and capture rules, and the bond spring force."""
import ctypes
import math
import os

import numpy as np
import pytest


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator(oracle_lib):
    """cuRAND's host PHILOX4_32_10 generator seeded with s emits, for a request
    of 256 numbers, the blocks Philox4x32-10(counter (0, 0, i, 0), key s)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x0123456789ABCDEF, 2 ** 64 - 1):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(256, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(256)) == 0
        lib.curandDestroyGenerator(gen)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for i in range(64):
            assert oracle_lib.philox4x32_10((0, 0, i, 0), key) == [int(x) for x in out[4 * i: 4 * i + 4]]


def test_uniform_draws(oracle_lib):
    u = np.array([oracle_lib.uniform(7, s, 11, p) for s in range(20000) for p in (0, 1)])
    assert u.min() >= 0.0 and u.max() < 1.0
    hist, _ = np.histogram(u, bins=20, range=(0, 1))
    exp = len(u) / 20
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45.0            # 19 d.o.f., p ~ 1e-3
    # different purposes and steps give different draws
    assert oracle_lib.uniform(7, 3, 11, 0) != oracle_lib.uniform(7, 3, 11, 1)
    assert oracle_lib.uniform(7, 3, 11, 0) != oracle_lib.uniform(7, 3, 12, 0)
    assert oracle_lib.uniform(7, 3, 2 ** 32 + 11, 0) != oracle_lib.uniform(7, 3, 11, 0)


def bond_params(**kw):
    p = dict(lig_i0=0, lig_j0=0, lig_ni=8, lig_nj=8, box_nx=8, box_ny=8, max_per_ligand=4,
             z_wall=-0.5, sigma=1.0, l_b=0.64, d_capture=0.64, gamma=0.1, kT=0.05,
             kon0_dt=0.0, koff0_dt=0.0, seed=12345)
    p.update(kw)
    return p


def sites_at(points):
    """One node per site (weights (1, 0, 0)) on degenerate triangles (v, v, v)."""
    n = len(points)
    X = np.ascontiguousarray(np.asarray(points, float).T).ravel()
    tri = np.repeat(np.arange(n, dtype=np.int32), 3)
    site_tri = np.arange(n, dtype=np.int32)
    site_w = np.tile([1.0, 0.0], n)
    return X, tri, site_tri, site_w


@pytest.mark.parametrize("Fb_target", [0.0, 0.2])
def test_survival_under_fixed_force(oracle_lib, Fb_target):
    """N0 bonds held at a fixed length: survivors after n steps are binomial
    with p = exp(-k_off(F) n dt), k_off(F) = k_off0 exp(gamma F / kT)."""
    p = bond_params(koff0_dt=2e-3)
    N0 = 4000
    # site straight above ligand (1, 1): x_b = l_b + Fb / sigma
    xb = p["l_b"] + Fb_target / p["sigma"]
    X, tri, st, sw = sites_at([[1.0, 1.0, -0.5 + xb]] * N0)
    bound = np.full(N0, 9, np.int32)             # ligand id 9 = (1, 1)
    lig = np.zeros(64, np.int32)
    lig[9] = N0                                   # capacity bookkeeping only
    n = 150
    for step in range(n):
        oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, step)
    koff_dt = p["koff0_dt"] * math.exp(p["gamma"] * Fb_target / p["kT"])
    ps = (1 - (-math.expm1(-koff_dt))) ** n
    mean, sd = N0 * ps, math.sqrt(N0 * ps * (1 - ps))
    surv = int((bound >= 0).sum())
    assert abs(surv - mean) < 5 * sd, (surv, mean, sd)
    assert lig[9] == surv


def test_capacity_four_lowest_sites(oracle_lib):
    """Ten free sites all within capture of one ligand with P_f = 1: exactly
    four bind, the four lowest site ids."""
    p = bond_params(kon0_dt=1e6)
    pts = [[2.0 + 0.01 * s, 3.0, -0.5 + 0.3] for s in range(10)]
    X, tri, st, sw = sites_at(pts)
    bound = np.full(10, -1, np.int32)
    lig = np.zeros(64, np.int32)
    nr, nf = oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, 0)
    assert (nr, nf) == (0, 4)
    assert list(bound) == [3 * 8 + 2] * 4 + [-1] * 6
    assert lig[3 * 8 + 2] == 4
    # the ligand is full: nothing forms on later steps
    for step in range(1, 5):
        assert oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, step) == (0, 0)


def test_capture_distance_and_lowest_ligand(oracle_lib):
    p = bond_params(kon0_dt=1e6)
    pts = [[2.0, 3.0, -0.5 + 0.7],      # 0.7 above the ligand: out of reach
           [2.5, 3.0, -0.5 + 0.2],      # between ligands (2,3) and (3,3): lowest id wins
           [5.0, 5.0, -0.5 + 0.63]]     # just inside 0.64
    X, tri, st, sw = sites_at(pts)
    bound = np.full(3, -1, np.int32)
    lig = np.zeros(64, np.int32)
    oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, 0)
    assert list(bound) == [-1, 3 * 8 + 2, 5 * 8 + 5]


def test_rupture_then_no_reformation_same_step(oracle_lib):
    p = bond_params(koff0_dt=1e6, kon0_dt=1e6)
    X, tri, st, sw = sites_at([[4.0, 4.0, -0.5 + 0.3]] * 3)
    bound = np.array([36, 36, -1], np.int32)
    lig = np.zeros(64, np.int32)
    lig[36] = 2
    nr, nf = oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, 0)
    assert (nr, nf) == (2, 1)          # both bonds break; only the free site binds
    assert list(bound) == [-1, -1, 36] and lig[36] == 1


def test_formation_probability(oracle_lib):
    """Free sites with one candidate each form with P_f = 1 - exp(-k_on dt),
    k_on from Eq. 13 at the site's distance."""
    p = bond_params(kon0_dt=0.3)
    n = 6000
    h = 0.5
    X, tri, st, sw = sites_at([[6.0, 6.0, -0.5 + h]] * n)
    bound = np.full(n, -1, np.int32)
    lig = np.zeros(64, np.int32)
    lig[6 * 8 + 6] = -10 ** 6                     # unlimited capacity for this check
    oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, 0)
    dev = abs(h - p["l_b"])
    kon = p["kon0_dt"] * math.exp(p["sigma"] * dev * (p["gamma"] - 0.5 * dev) / p["kT"])
    Pf = -math.expm1(-kon)
    k = int((bound >= 0).sum())
    assert abs(k - n * Pf) < 5 * math.sqrt(n * Pf * (1 - Pf))


def test_bond_force_eq14(oracle_lib):
    p = bond_params(sigma=2.5)
    X, tri, st, sw = sites_at([[1.2, 0.9, -0.5 + 0.9]])
    bound = np.array([9], np.int32)              # ligand (1, 1) at (1, 1, -0.5)
    F = np.zeros(3)
    oracle_lib.bond_forces(p, st, sw, tri, bound, X, F)
    d = np.array([0.2, -0.1, 0.9])
    xb = np.linalg.norm(d)
    assert np.allclose(F, -2.5 * (xb - 0.64) * d / xb, atol=1e-15)
    # barycentric split on a real triangle
    X = np.ascontiguousarray(np.array([[1, 1, 0.5], [2, 1, 0.5], [1, 2, 0.5]], float).T).ravel()
    tri = np.array([0, 1, 2], np.int32)
    st = np.array([0], np.int32)
    sw = np.array([0.2, 0.5])
    F = np.zeros(9)
    oracle_lib.bond_forces(p, st, sw, tri, bound, X, F)
    r = 0.2 * np.array([1, 1, 0.5]) + 0.5 * np.array([2, 1, 0.5]) + 0.3 * np.array([1, 2, 0.5])
    d = r - np.array([1, 1, -0.5])
    f = -2.5 * (np.linalg.norm(d) - 0.64) * d / np.linalg.norm(d)
    assert np.allclose(F.reshape(3, 3).T, np.outer([0.2, 0.5, 0.3], f), atol=1e-15)


def _brute_force_first_ligand(p, pts):
    """Every ligand node of the patch at its minimum-image distance from each
    point: the ids in reach (ascending) per point, by a scan of the whole
    patch."""
    li = np.arange(p["lig_ni"] * p["lig_nj"])
    gx = p["lig_i0"] + li % p["lig_ni"]
    gy = p["lig_j0"] + li // p["lig_ni"]
    out = []
    for x, y, z in pts:
        dx = x - gx
        dx -= p["box_nx"] * np.round(dx / p["box_nx"])
        dy = y - gy
        dy -= p["box_ny"] * np.round(dy / p["box_ny"])
        d = np.sqrt(dx * dx + dy * dy + (z - p["z_wall"]) ** 2)
        out.append(li[d < p["d_capture"]])
    return out


def test_capture_beyond_one_spacing_matches_brute_force(oracle_lib):
    """d_capture = 1.7 lattice spacings (128 nm at a lattice spacing of
    75 nm): a free site may reach up to a few dozen ligands, outside the 2x2
    nodes around it.  With P_f = 1 every free site proposes to the lowest
    ligand id within reach, and each ligand takes the four lowest site ids:
    the same bonds as a scan of the whole patch, including across the
    periodic seam (patch columns 0..7 of a 10-wide box)."""
    p = bond_params(lig_ni=8, lig_nj=7, box_nx=10, box_ny=9, d_capture=1.7, l_b=1.0, kon0_dt=1e6)
    rng = np.random.default_rng(3)
    n = 400
    pts = np.column_stack([rng.uniform(0, 10, n), rng.uniform(0, 9, n), rng.uniform(-0.5, 1.4, n)])
    pts[:20, 0] += 10.0 * rng.integers(-2, 3, 20)          # unwrapped coordinates
    X, tri, st, sw = sites_at(pts)
    bound = np.full(n, -1, np.int32)
    lig = np.zeros(p["lig_ni"] * p["lig_nj"], np.int32)
    oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, 0)
    reach = _brute_force_first_ligand(p, pts)
    # the case the 2x2 block would miss occurs: a lowest in-reach ligand
    # outside the nodes floor(x) + {0, 1}, floor(y) + {0, 1}
    outside = 0
    for (x, y, _), ids in zip(pts, reach):
        if len(ids):
            l0 = ids[0]
            di = (p["lig_i0"] + l0 % p["lig_ni"] - math.floor(x % 10)) % 10
            dj = (p["lig_j0"] + l0 // p["lig_ni"] - math.floor(y % 9)) % 9
            outside += not (di in (0, 1) and dj in (0, 1))
    assert outside > 20 and max(len(r) for r in reach) > 4
    want = np.full(n, -1, np.int32)
    taken = np.zeros_like(lig)
    for s in range(n):                          # ascending site id per ligand
        if len(reach[s]) and taken[reach[s][0]] < 4:
            want[s] = reach[s][0]
            taken[reach[s][0]] += 1
    assert np.array_equal(bound, want)
    assert np.array_equal(lig, taken)


def test_every_candidate_in_reach_draws_once(oracle_lib):
    """With sigma = 0, k_on = k_on0 for every candidate, so a site with n
    ligands in reach proposes with probability 1 - (1 - p)^n and picks the
    k-th lowest of them with probability p (1 - p)^(k-1): n independent
    draws, one per ligand, the lowest id kept.  At d_capture = 1.5 a site
    0.1 above the wall plane over a node centre reaches 9 ligands (offsets
    in {-1, 0, 1}^2); with capacity unlimited 20000 sites give the law."""
    p = bond_params(d_capture=1.5, sigma=0.0, kon0_dt=0.15)
    n = 20000
    X, tri, st, sw = sites_at([[4.0, 4.0, -0.5 + 0.1]] * n)
    bound = np.full(n, -1, np.int32)
    lig = np.full(64, -10 ** 6, np.int32)
    oracle_lib.bonds_step(p, st, sw, tri, X, bound, lig, 7)
    reach = _brute_force_first_ligand(p, [[4.0, 4.0, -0.4]])[0]
    assert len(reach) == 9
    P = -math.expm1(-p["kon0_dt"])
    probs = [P * (1 - P) ** k for k in range(9)] + [(1 - P) ** 9]
    counts = [int((bound == l).sum()) for l in reach] + [int((bound < 0).sum())]
    exp = np.array(probs) * n
    chi2 = float((((np.array(counts) - exp) ** 2) / exp).sum())
    assert chi2 < 33.7, (counts, exp)      # 9 d.o.f., p ~ 1e-4
