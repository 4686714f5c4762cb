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
2^-7 of the largest population, and a node velocity can move by up to that
step, 2^-7 max|f*neq| (~9e-6 x 2^-7 in this fast shear flow, against node
velocities ~1e-4): positions within 1e-4 of the largest displacement
(measured 8e-6), bond states as for FP32."""
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
    tol_x = 1e-6 if storage == "fp32" else 1e-4
    assert rel(b.X.cpu().numpy() - X0, a.X.cpu().numpy() - X0) < tol_x
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
    completes, and sim_check counts exactly the planted coordinates, NaN or
    far but finite.  The planted coordinates are interior (SCE) nodes: their
    Morse pairs give no force at such distances, so the rest of the state
    stays as it was (planted on membrane nodes, the elastic forces of their
    neighbours grow without bound and the run blows up for real, which
    sim_check then reports cell by cell)."""
    w = workload.tiny(seed=2, shear=2.0e4)
    sim = fsi.Simulation(w)
    sim.step(2)
    M = sim.M
    sce = np.nonzero(np.asarray(w["mesh"]["is_membrane"]) == 0)[0]
    a, b, c = (int(v) for v in sce[[1, 3, 5]])
    sim.X[M + a] = 1.0e30
    sim.X[2 * M + b] = -3.0e12
    sim.X[c] = 1.0e8
    counts, ok = sim.check(0.3)
    assert not ok and counts[3] == 3, counts
    sim.step(5)
    torch.cuda.synchronize()
    counts, ok = sim.check(0.3)
    assert not ok and counts[3] == 3, counts
    U = sim.U.reshape(3, M).cpu().numpy()
    assert np.isnan(U[:, [a, b, c]]).all()
    sim.X[3] = float("nan")
    counts, ok = sim.check(0.3)
    assert not ok and counts[3] == 4, counts


def test_left_out_nodes_do_not_disturb_the_others():
    """Spreading and interpolation with a few nodes planted far away give the
    other nodes the same result as a run without the planted nodes whose
    force is zero (their chunks keep the tile of the nodes in range), within
    the run-to-run rounding of spreading; the planted nodes read U = NaN and
    keep their positions.  Spreading adds each chunk's tile into the cell
    forces with FP32 atomics in no fixed order, so two runs of the same input
    already differ: up to 5.2e-7 of max|f| on this channel (about 7 ULPs of a
    4e-5 shifted population); the bound is 4e-6, a few times that floor."""
    w = workload.config_channel(seed=0)
    M = w["M"]
    runs = []
    rng = np.random.default_rng(4)
    F = torch.as_tensor(rng.standard_normal(3 * M).astype(np.float32) * 1e-4).cuda()
    planted = np.array([5, 1300, 20000])
    F.reshape(3, M)[:, planted] = 0.0
    for plant in (False, True):
        lat = fsi.Lattice(w["grid"]["nx"], w["grid"]["ny"], w["grid"]["nz"], w["grid"]["tau"], w["grid"]["u_top"])
        lat.init_shear()
        X = torch.as_tensor(np.ascontiguousarray(w["X"])).cuda()
        if plant:
            X.reshape(3, M)[0, planted[0]] = float("nan")
            X.reshape(3, M)[1, planted[1]] = 2.0e8
            X.reshape(3, M)[2, planted[2]] = -1.0e20
        Xs = X.clone()
        U = torch.zeros(3 * M, device="cuda")
        fsi.ib_spread(lat.h, X, F, M)
        fsi.lb_step(lat.h, 1)
        fsi.ib_interp(lat.h, X, U, M, advect=True)
        torch.cuda.synchronize()
        runs.append((lat.export().cpu().numpy(), U.reshape(3, M).cpu().numpy(), X.reshape(3, M).cpu().numpy(),
                     Xs.reshape(3, M).cpu().numpy()))
    (f0, U0, X0, _), (f1, U1, X1, Xs1) = runs
    keep = np.ones(M, bool)
    keep[planted] = False
    assert rel(f1, f0) < 4e-6
    assert rel(U1[:, keep], U0[:, keep]) < 4e-6
    assert np.isfinite(U1[:, keep]).all() and np.isnan(U1[:, planted]).all()
    assert np.array_equal(X1[:, planted], Xs1[:, planted], equal_nan=True)
    assert rel(X1[:, keep] - Xs1[:, keep], X0[:, keep] - runs[0][3][:, keep]) < 4e-6
