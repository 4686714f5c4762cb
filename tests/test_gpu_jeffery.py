"""Jeffery-orbit check of the coupled fluid-membrane step (Section 4.1): a
discoid platelet (oblate spheroid, aspect r = 0.25) lying in the
flow-vorticity plane at mid-height of a Couette channel (walls 10 radii
away) tumbles in the shear plane.  Jeffery's period for a rigid spheroid in
unbounded shear is T = (2 pi / shear)(r + 1/r); the axis line returns after
T/2.

* Membrane only (642 nodes, a = 5 lattice units, shear 2e-4 per step:
  Reynolds number shear a^2 / nu = 0.05, fluid stress ~1e-3 of the membrane
  modulus): the capsule, fluid inside, deforms as it turns (aspect ratio
  0.25 -> 0.32) and its half period lies within 10 % of T/2 (measured 0.93).
* With the SCE interior (the configurations' platelet: 2562 membrane nodes,
  800 Morse-coupled interior points) the platelet stays rigid (aspect ratio
  within 0.24-0.25 throughout) and turns faster than Jeffery's rigid spheroid
  at finite resolution: the immersed boundary spreads each node's force over
  +-2 lattice spacings, so the body acts ~0.7 h thicker, which at a = 5 h
  (a platelet only 2.5 h thick) moves the effective aspect ratio from 0.25 to
  ~0.33.  At fixed physical shear and capillary number the error of the half
  period falls linearly with h: measured 1 - t/(T/2) = 0.235, 0.181, 0.157,
  0.129 at a = 5, 6, 7.5, 10 lattice units (least-squares intercept 0.02 at
  h -> 0).  The test runs a = 5 and a = 10 and checks rigidity, convergence
  and the first-order extrapolation 2 t_10 - t_5 within 10 % of T/2
  (measured 0.977)."""
import numpy as np
import pytest

from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu


def half_period(a_cells, level, n_sce, shear_lat5=2e-4, every5=500, frac=0.65):
    """Half period / (T/2) of a flat platelet of radius a_cells lattice
    units (the lattice spacing scaled, the physical shear and properties
    kept: the a = 5 run has shear 2e-4 per step), and the range of its
    membrane's aspect ratio over the run."""
    phys = dict(workload.PHYSICAL)
    scale = a_cells / 5.0
    phys["h"] = phys["h"] / scale
    L = workload.lattice_units(0.8, phys)
    shear_phys = shear_lat5 / workload.lattice_units(0.8)["dt"]
    shear_lat = shear_phys * L["dt"]
    nx = ny = int(round(48 * scale))
    nz = int(round(100 * scale))
    w = workload.build(nx, ny, nz, 0.8, shear_phys, 1, level, n_sce, 0, 0, orient="flat",
                       centers=[(nx / 2, ny / 2, nz / 2 - 0.5)], phys=phys)
    sim = fsi.Simulation(w)
    M = w["M"]
    mem = np.asarray(w["mesh"]["is_membrane"]).astype(bool)
    T = 2 * np.pi / shear_lat * (0.25 + 1 / 0.25)
    every = int(every5 * scale * scale)
    ts, ang, asp = [], [], []
    step = 0
    while step < frac * T:
        X = sim.X.cpu().numpy().reshape(3, M)
        lam, V = np.linalg.eigh(np.cov(X[:, mem]))
        a = V[:, 0]                       # symmetry axis: least spread
        ts.append(step)
        ang.append(np.arctan2(a[2], a[0]))
        asp.append(float(np.sqrt(lam[0] / lam[2])))
        sim.step(every)
        step += every
    turn = np.abs(np.unwrap(2 * np.array(ang)) / 2 - ang[0])   # the axis line: period pi
    assert turn.max() >= np.pi, "the platelet did not turn over"
    k = int(np.argmax(turn >= np.pi))
    t_half = ts[k - 1] + (np.pi - turn[k - 1]) / (turn[k] - turn[k - 1]) * (ts[k] - ts[k - 1])
    # tumbling, not spinning in place: the slow phase (axis near the gradient
    # direction, platelet aligned with the flow) takes most of the time
    assert turn[k // 4] < np.pi / 4
    return t_half / (T / 2), min(asp), max(asp)


def test_half_period_of_the_jeffery_orbit():
    ratio, _, asp_max = half_period(5, 3, 0)
    assert abs(ratio - 1.0) < 0.10, ratio
    assert asp_max > 0.28   # the membrane-only capsule deforms as it turns


def test_jeffery_orbit_with_the_sce_interior_converges():
    r5, lo5, hi5 = half_period(5, 4, 800)
    r10, lo10, hi10 = half_period(10, 4, 800)
    for lo, hi in ((lo5, hi5), (lo10, hi10)):
        assert 0.23 < lo and hi < 0.26, (lo, hi)   # rigid: the interior holds the shape
    assert r5 < r10 < 1.0, (r5, r10)               # faster than Jeffery, less so when finer
    assert abs((2 * r10 - r5) - 1.0) < 0.10, (r5, r10)
