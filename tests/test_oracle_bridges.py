"""Pins of the FP64 oracle of the platelet-platelet bridges (Section 3.2,
GPIb-alpha - vWF - GPIb-alpha bonds "treated similarly" to the wall bonds):

* formation of one pair is Bernoulli with P_f = 1 - exp(-k_on dt), k_on of
  Eq. 13, at two separations (binomial test over independent steps), and
  never at or beyond the capture distance;
* survival of one bridge is Bernoulli with P_r = 1 - exp(-k_off dt), Bell
  k_off of Eq. 12 at the bridge's force, at two lengths;
* the matching rule on hand-built cases: the lowest-index successful partner,
  mutual choices only, a chain resolved over two steps;
* one bond per site: wall-bound sites do not bridge and bridged sites take no
  wall bond; a ruptured bridge does not re-form in the same step;
* the minimum image across the periodic x boundary;
* the spring force (Eq. 14 form) by hand: equal and opposite, of size
  sigma |x - l_b| along the pair, split by the barycentric weights."""
import math

import numpy as np

import oracle


def two_sites(sep, box=(64, 48), axis=0, shift=(10.0, 10.0, 5.0)):
    """Two one-triangle 'platelets' whose first corners carry one site each
    (weights (1, 0, 0)), separated by `sep` along `axis`."""
    X = np.zeros((6, 3))
    X[:3] = np.array(shift) + np.array([[0, 0, 0], [0.3, 0, 0], [0, 0.3, 0]])
    off = np.zeros(3)
    off[axis] = sep
    X[3:] = X[:3] + off
    tri = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    node_plt = np.array([0, 0, 0, 1, 1, 1], dtype=np.int32)
    site_tri = np.array([0, 1], dtype=np.int32)
    site_w = np.array([1.0, 0.0, 1.0, 0.0])
    return np.ascontiguousarray(X.T).ravel(), tri, node_plt, site_tri, site_w


def params(**kw):
    p = dict(sigma=0.05, l_b=1.0, d_capture=1.2, gamma=0.1, kT=0.05, kon0_dt=0.4, koff0_dt=0.02,
             box_nx=64, box_ny=48, seed=11)
    p.update(kw)
    return p


def kon_dt(p, x):
    dev = abs(x - p["l_b"])
    return p["kon0_dt"] * math.exp(p["sigma"] * dev * (p["gamma"] - 0.5 * dev) / p["kT"])


def koff_dt(p, x):
    return p["koff0_dt"] * math.exp(p["gamma"] * p["sigma"] * abs(x - p["l_b"]) / p["kT"])


def within(k, n, prob, sigmas=4.5):
    return abs(k - n * prob) <= sigmas * math.sqrt(n * prob * (1 - prob)) + 1


def step_pair(p, X, tri, plt, st, sw, partner, step, bound=None):
    if bound is None:
        bound = np.full(len(st), -1, dtype=np.int32)
    site_plt = oracle.site_platelets(st, tri, plt)
    return oracle.bridges_step(p, st, sw, tri, site_plt, X, bound, partner, step)


def test_formation_is_bernoulli_with_eq13():
    for sep in (0.8, 1.15):
        p = params()
        X, tri, plt, st, sw = two_sites(sep)
        n, k = 6000, 0
        for step in range(n):
            partner = np.full(2, -1, dtype=np.int32)
            step_pair(p, X, tri, plt, st, sw, partner, step)
            k += int(partner[0] == 1)
            assert partner[1] == (0 if partner[0] == 1 else -1)
        assert within(k, n, -math.expm1(-kon_dt(p, sep))), (sep, k)
    # at and beyond the capture distance: never
    p = params()
    for sep in (1.2 + 1e-9, 1.3):
        X, tri, plt, st, sw = two_sites(sep)
        for step in range(300):
            partner = np.full(2, -1, dtype=np.int32)
            step_pair(p, X, tri, plt, st, sw, partner, step)
            assert partner[0] == -1


def test_rupture_is_bernoulli_with_bell():
    for sep in (0.6, 1.1):
        p = params(kon0_dt=0.0, koff0_dt=0.01)
        X, tri, plt, st, sw = two_sites(sep)
        n, k = 6000, 0
        for step in range(n):
            partner = np.array([1, 0], dtype=np.int32)
            step_pair(p, X, tri, plt, st, sw, partner, step)
            k += int(partner[0] == -1)
        assert within(k, n, -math.expm1(-koff_dt(p, sep))), (sep, k)


def sites_on_platelets(points, plts, box=(64, 48)):
    """One one-triangle platelet per site; site s sits on corner 0 of
    triangle s, which belongs to platelet plts[s]."""
    n = len(points)
    X = np.zeros((3 * n, 3))
    for s, q in enumerate(points):
        X[3 * s:3 * s + 3] = np.array(q) + np.array([[0, 0, 0], [0.2, 0, 0], [0, 0.2, 0]])
    tri = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    node_plt = np.repeat(np.asarray(plts, dtype=np.int32), 3)
    st = np.arange(n, dtype=np.int32)
    sw = np.tile([1.0, 0.0], n)
    return np.ascontiguousarray(X.T).ravel(), tri, node_plt, st, sw


def test_matching_rule_lowest_index_and_mutual():
    p = params(kon0_dt=60.0)   # P_f = 1 for every pair in reach
    # three sites on three platelets, all within reach of each other
    X, tri, plt, st, sw = sites_on_platelets([(10, 10, 5), (10.5, 10, 5), (10, 10.5, 5)], [0, 1, 2])
    partner = np.full(3, -1, dtype=np.int32)
    ev = step_pair(p, X, tri, plt, st, sw, partner, 0)
    assert list(partner) == [1, 0, -1] and ev == (0, 1)
    ev = step_pair(p, X, tri, plt, st, sw, partner, 1)     # 2 has no free partner left
    assert list(partner) == [1, 0, -1] and ev == (0, 0)
    # a chain 0-1-2-3 on alternating platelets, neighbours only in reach
    X, tri, plt, st, sw = sites_on_platelets([(10, 10, 5), (11, 10, 5), (12, 10, 5), (13, 10, 5)], [0, 1, 0, 1])
    partner = np.full(4, -1, dtype=np.int32)
    step_pair(p, X, tri, plt, st, sw, partner, 0)
    assert list(partner) == [1, 0, -1, -1]      # 2 chose 1, so 3's choice of 2 is not mutual
    step_pair(p, X, tri, plt, st, sw, partner, 1)
    assert list(partner) == [1, 0, 3, 2]
    # sites on the same platelet never bridge
    X, tri, plt, st, sw = sites_on_platelets([(10, 10, 5), (10.5, 10, 5)], [4, 4])
    partner = np.full(2, -1, dtype=np.int32)
    step_pair(p, X, tri, plt, st, sw, partner, 0)
    assert list(partner) == [-1, -1]


def test_one_bond_per_site_and_no_reformation_in_the_same_step():
    p = params(kon0_dt=60.0)
    X, tri, plt, st, sw = sites_on_platelets([(10, 10, 5), (10.5, 10, 5)], [0, 1])
    partner = np.full(2, -1, dtype=np.int32)
    bound = np.array([7, -1], dtype=np.int32)      # site 0 holds a wall bond
    step_pair(p, X, tri, plt, st, sw, partner, 0, bound)
    assert list(partner) == [-1, -1]
    # rupture certain, formation certain: the pair alternates
    p = params(kon0_dt=60.0, koff0_dt=60.0)
    partner = np.full(2, -1, dtype=np.int32)
    seq = []
    for step in range(4):
        step_pair(p, X, tri, plt, st, sw, partner, step)
        seq.append(int(partner[0]))
    assert seq == [1, -1, 1, -1]
    # both ends of a ruptured bridge wait a step, whichever index they have:
    # site 1 (the higher end) does not bridge to site 2 in the step its bridge broke
    X3, tri3, plt3, st3, sw3 = sites_on_platelets([(10, 10, 5), (10.5, 10, 5), (10.5, 10.5, 5)], [0, 1, 2])
    partner = np.array([1, 0, -1], dtype=np.int32)
    step_pair(p, X3, tri3, plt3, st3, sw3, partner, 0)
    assert list(partner) == [-1, -1, -1]
    step_pair(params(kon0_dt=60.0), X3, tri3, plt3, st3, sw3, partner, 1)
    assert list(partner) == [1, 0, -1]
    # a bridged site takes no wall bond even when one is certain
    w = {"lig_i0": 0, "lig_j0": 0, "lig_ni": 64, "lig_nj": 48, "box_nx": 64, "box_ny": 48, "max_per_ligand": 4,
         "z_wall": 4.9, "sigma": 0.05, "l_b": 0.1, "d_capture": 0.9, "gamma": 0.0, "kT": 1.0, "kon0_dt": 60.0,
         "koff0_dt": 0.0, "seed": 3}
    bound = np.full(2, -1, dtype=np.int32)
    lig = np.zeros(64 * 48, dtype=np.int32)
    oracle.bonds_step(w, st, sw, tri, X, bound, lig, 0, np.array([1, 0], dtype=np.int32))
    assert list(bound) == [-1, -1]
    oracle.bonds_step(w, st, sw, tri, X, bound, lig, 0, np.full(2, -1, dtype=np.int32))
    assert (bound >= 0).all()


def test_minimum_image_across_the_periodic_boundary():
    p = params(kon0_dt=60.0)
    X, tri, plt, st, sw = sites_on_platelets([(63.7, 10, 5), (0.2, 10, 5)], [0, 1])
    partner = np.full(2, -1, dtype=np.int32)
    step_pair(p, X, tri, plt, st, sw, partner, 0)
    assert list(partner) == [1, 0]


def test_spring_force_by_hand():
    p = params()
    X, tri, plt, st, sw = two_sites(0.7, axis=1)
    sw = np.array([0.2, 0.5, 0.6, 0.1])
    partner = np.array([1, 0], dtype=np.int32)
    F = np.zeros_like(X)
    oracle.bridge_forces(p, st, sw, tri, partner, X, F)
    Xn = X.reshape(3, -1).T
    r0 = 0.2 * Xn[0] + 0.5 * Xn[1] + 0.3 * Xn[2]
    r1 = 0.6 * Xn[3] + 0.1 * Xn[4] + 0.3 * Xn[5]
    d = r0 - r1
    L = np.linalg.norm(d)
    f0 = -p["sigma"] * (L - p["l_b"]) * d / L          # on site 0
    Fn = F.reshape(3, -1).T
    assert np.allclose(Fn[0], 0.2 * f0) and np.allclose(Fn[1], 0.5 * f0) and np.allclose(Fn[2], 0.3 * f0)
    assert np.allclose(Fn[3], -0.6 * f0) and np.allclose(Fn[4], -0.1 * f0) and np.allclose(Fn[5], -0.3 * f0)
    assert np.allclose(Fn.sum(0), 0.0, atol=1e-15)
    assert abs(np.linalg.norm(f0) - p["sigma"] * abs(L - p["l_b"])) < 1e-15


def test_pair_draws_are_symmetric_and_distinct_from_the_wall_draws():
    seed, step = 0x1234_5678_9ABC, (3 << 32) + 17
    u = oracle.pair_uniform(seed, 5, 9, step, 17)
    assert 0.0 <= u < 1.0
    assert u != oracle.pair_uniform(seed, 9, 5, step, 17)     # ordered pairs are distinct counters
    assert u != oracle.pair_uniform(seed, 5, 9, step, 16)
    assert u != oracle.pair_uniform(seed, 5, 9, step + (1 << 32), 17)   # the step's high word enters the key
    r = oracle.philox4x32_10([5, 9, step & 0xFFFFFFFF, 17], [seed & 0xFFFFFFFF, (seed >> 32) ^ (step >> 32)])
    assert u == float((r[0] << 21) | (r[1] >> 11)) * 2.0 ** -53
