"""Instability check and checkpoint/resume of the coupled step.

lb_check / sim_check count non-finite cells, cells with rho <= 0, cells faster
than u_max and non-finite node coordinates; a healthy state reads zero and
each planted defect is counted (the defects are written into the state on
the host side of the test: nothing faults on the device).

A run checkpointed after 4 steps and restored into a fresh simulation takes
the next 4 steps as the uninterrupted run does: the same random decisions
(Philox keyed by site and step) and the same states up to the run-to-run
rounding of force spreading, whose tile sums are added with FP32 atomics in
no fixed order (1e-6 of the largest entry).  With 16-bit population storage
such a difference can move a stored f*neq across a rounding boundary: one
BF16 step is at most 2^-7 of the stored value, so the populations agree to
2^-7 of the largest population (positions and bond states as for FP32)."""
import numpy as np
import pytest
import torch

from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_check_counts_planted_defects_fp32():
    w = workload.tiny(seed=1, shear=2.0e4)
    sim = fsi.Simulation(w)
    sim.step(3)
    counts, ok = sim.check(0.3)
    assert ok and counts == (0, 0, 0, 0)
    f = sim.lattice.current()
    N = f.shape[1]
    f[0, 10] = float("nan")                    # non-finite population
    f[:, 20] = -1.0                             # rho = 1 - 19 < 0
    f[0, 30] += 0.5                             # +x momentum 0.5 at rho ~ 1.5: |u| ~ 0.33
    sim.X[5] = float("inf")
    counts, ok = sim.check(0.3)
    assert not ok
    assert counts == (1, 1, 1, 1), counts
    lat_counts, lat_ok = sim.lattice.check(0.3)
    assert not lat_ok and lat_counts == (1, 1, 1)
    assert N > 30


def test_check_mixed_storage():
    lat = fsi.Lattice(24, 20, 18, 0.8, (3e-3, 0.0, 0.0), storage="bf16")
    lat.init_shear()
    lat.step(2)
    counts, ok = lat.check(0.3)
    assert ok and counts == (0, 0, 0)
    live = 0 if lat.velocity().data_ptr() == lat.m[0].data_ptr() else 1
    lat.f[live].view(torch.int16)[3, 7] = 0x7fc0            # BF16 NaN in a stored f*neq
    lat.m[live][11, 0] = 0.5                                 # fast cell
    lat.m[live][12, 3] = -1.5                                # rho - 1 = -1.5
    counts, ok = lat.check(0.3)
    assert not ok and counts == (1, 1, 1), counts


def fast_pair():
    w = workload.config_pair(seed=5, level=3, n_sce=100, n_sites=1500, shear=2.0e4)
    w["bonds"] = dict(w["bonds"], kon0_dt=0.5, kT=0.05, sigma=0.02, gamma=0.05, koff0_dt=0.02)
    w["bridges"] = dict(w["bridges"], sigma=0.02, kT=0.05, gamma=0.05, kon0_dt=0.3, koff0_dt=0.05)
    return w


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_checkpoint_resume_continues_the_run(storage, tmp_path):
    w = fast_pair()
    a = fsi.Simulation(w, storage=storage)
    a.step(4)
    ck = a.checkpoint()
    np.savez(tmp_path / "ck.npz", **ck)
    a.step(4)
    loaded = dict(np.load(tmp_path / "ck.npz"))
    b = fsi.Simulation.restore(w, loaded)
    assert b.step_index == 4
    b.step(4)
    torch.cuda.synchronize()
    assert a.step_index == b.step_index == 8
    X0 = w["X"]
    assert rel(b.X.cpu().numpy() - X0, a.X.cpu().numpy() - X0) < 1e-6
    tol_f = 1e-6 if storage == "fp32" else 2.0 ** -7
    assert rel(b.lattice.export().cpu().numpy(), a.lattice.export().cpu().numpy()) < tol_f
    assert np.array_equal(b.bonds.bound.cpu().numpy(), a.bonds.bound.cpu().numpy())
    assert np.array_equal(b.bonds.lig_count.cpu().numpy(), a.bonds.lig_count.cpu().numpy())
    assert np.array_equal(b.bridges.partner.cpu().numpy(), a.bridges.partner.cpu().numpy())
    assert (a.bonds.bound.cpu().numpy() >= 0).any() and (a.bridges.partner.cpu().numpy() >= 0).any()


def test_blown_up_positions_are_left_out_not_indexed():
    """Nodes whose coordinates are not finite or lie far outside the grid (a
    run that blew up) take no part in spreading and interpolation -- their
    support cells would overflow the integer cell indices -- so the step
    completes, and sim_check reports the state."""
    w = workload.tiny(seed=2, shear=2.0e4)
    sim = fsi.Simulation(w)
    sim.step(2)
    M = sim.M
    sim.X[3] = float("nan")
    sim.X[M + 7] = 1.0e30
    sim.X[2 * M + 11] = -3.0e12
    sim.step(5)
    torch.cuda.synchronize()
    counts, ok = sim.check(0.3)
    assert not ok and counts[3] >= 1
