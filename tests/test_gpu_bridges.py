"""GPU parity of the platelet-platelet bridges (Section 3.2, GPIb-alpha - vWF
- GPIb-alpha, modelled like the wall bonds) against the FP64 oracle.

Bridge events are integer decisions taken in FP64 with the oracle's rounding
order, so the partner arrays must agree bit for bit (the one exception, a
uniform within an ulp of its probability, where CUDA's and glibc's exp may
differ, has not occurred).  Kinetic constants are raised above the
physiological ones so that tens to hundreds of events happen per step.
Workloads: the two stacked platelets of the platelet-platelet study, and a
cube of 27 small platelets straddling the periodic x boundary whose centre
platelet has more than 16 neighbours (the neighbour-list overflow path)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu

FAST = dict(sigma=0.02, kT=0.05, gamma=0.05, kon0_dt=0.3, koff0_dt=0.05)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def cube(seed=3):
    P = dict(workload.PHYSICAL, a=0.4e-6, aspect=1.0)
    cs = [(0.3 + 4.4 * i, 12.2 + 4.4 * j, 3.0 + 4.4 * k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (0, 1, 2)]
    return workload.build(32, 24, 24, 0.8, 500.0, 27, 1, 0, 60, seed, gap=0.3, orient="flat", centers=cs,
                          bridges=True, phys=P)


class State:
    """Wall bonds + bridges on the device for a workload, and the same state
    for the oracle."""

    def __init__(self, w, bp):
        m = w["mesh"]
        self.w = w
        self.bp = bp
        self.st = np.ascontiguousarray(w["sites"]["tri"], dtype=np.int32)
        self.sw = np.ascontiguousarray(w["sites"]["w"], dtype=np.float64).ravel()
        self.tri = np.ascontiguousarray(m["tri"], dtype=np.int32).ravel()
        self.site_plt = oracle.site_platelets(self.st, self.tri, m["node_plt"])
        self.tri_dev = torch.as_tensor(self.tri).cuda()
        self.bonds = fsi.Bonds(w["bonds"], self.st, self.sw.reshape(-1, 2), self.tri_dev, w["bound"], w["lig_count"])
        self.br = fsi.Bridges(bp, self.bonds, m["node_plt"], m["n_plt"])
        self.partner = np.full(len(self.st), -1, dtype=np.int32)
        self.bound = np.full(len(self.st), -1, dtype=np.int32)
        self.M = w["M"]

    def step_both(self, X, step):
        Xd = torch.as_tensor(X).cuda()
        self.br.step(Xd, step)
        ev = oracle.bridges_step(self.bp, self.st, self.sw, self.tri, self.site_plt, X, self.bound, self.partner,
                                 step)
        torch.cuda.synchronize()
        return ev


@pytest.mark.parametrize("which", ["pair", "cube"])
def test_bridge_events_match_the_oracle(which):
    if which == "pair":
        w = workload.config_pair(seed=1, level=3, n_sce=100, n_sites=1500)
    else:
        w = cube()
    bp = dict(w["bridges"], **FAST)
    S = State(w, bp)
    X = w["X"].copy()
    rng = np.random.default_rng(5)
    tot = np.zeros(2, dtype=np.int64)
    for step in range(6):
        ev = S.step_both(X, step)
        tot += ev
        assert np.array_equal(S.br.partner.cpu().numpy(), S.partner), step
        # move the nodes a little: new lengths, new rupture forces
        X = X + 0.05 * rng.standard_normal(X.shape)
    st = S.br.status()
    assert (st[0], st[1]) == (int(tot[0]), int(tot[1]))
    assert tot[1] > 20 and tot[0] > 0, tot
    if which == "cube":
        assert st[2] > 0      # the centre platelet's neighbour list overflowed
    # forces of the bridges that stand now
    F = torch.zeros(3 * S.M, device="cuda")
    S.br.forces(torch.as_tensor(X).cuda(), F)
    Fr = oracle.bridge_forces(bp, S.st, S.sw, S.tri, S.partner, X, np.zeros(3 * S.M))
    torch.cuda.synchronize()
    assert rel(F.cpu().numpy(), Fr) < 1e-6


def test_bridged_sites_take_no_wall_bond():
    """Wall kinetics fast as well: the wall and bridge states of the device
    match the oracle's, and no site holds both."""
    w = workload.config_pair(seed=2, level=3, n_sce=100, n_sites=1500)
    w["bonds"] = dict(w["bonds"], kon0_dt=0.5, kT=0.05, sigma=0.02, gamma=0.05, koff0_dt=0.02)
    bp = dict(w["bridges"], **FAST)
    S = State(w, bp)
    X = w["X"].copy()
    lig = np.zeros_like(w["lig_count"])
    Xd = torch.as_tensor(X).cuda()
    for step in range(5):
        S.bonds.step(Xd, S.M, step)
        oracle.bonds_step(w["bonds"], S.st, S.sw, S.tri, X, S.bound, lig, step, S.partner)
        S.step_both(X, step)
        assert np.array_equal(S.bonds.bound.cpu().numpy(), S.bound)
        assert np.array_equal(S.br.partner.cpu().numpy(), S.partner)
    assert (S.bound >= 0).sum() > 0 and (S.partner >= 0).sum() > 0
    assert not np.any((S.bound >= 0) & (S.partner >= 0))


def f32_workload(w):
    w = dict(w)
    w["membrane"] = {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in w["membrane"].items()}
    g = dict(w["grid"])
    g["tau"] = float(np.float32(g["tau"]))
    g["u_top"] = tuple(float(np.float32(u)) for u in g["u_top"])
    w["grid"] = g
    return w


def test_coupled_step_with_bridges():
    """The coupled step of two stacked platelets with wall bonds and bridges
    (fast kinetics) against the oracle's: displacement and node velocity
    within 1e-5 of their largest entries, bond and bridge states equal."""
    w = workload.config_pair(seed=4, level=3, n_sce=100, n_sites=1500, shear=2.0e4)
    w["bridges"] = dict(w["bridges"], **FAST)
    w = f32_workload(w)
    sim = fsi.Simulation(w)
    ora = oracle.Sim(w)
    steps = 6
    sim.step(steps)
    for _ in range(steps):
        ora.step()
    torch.cuda.synchronize()
    X0 = w["X"]
    assert rel(sim.X.cpu().numpy() - X0, ora.X - X0) < 1e-5
    assert rel(sim.U.cpu().numpy(), ora.U) < 1e-5
    assert np.array_equal(sim.bridges.partner.cpu().numpy(), ora.partner)
    assert np.array_equal(sim.bonds.bound.cpu().numpy(), ora.bound)
    assert (ora.partner >= 0).sum() > 0
