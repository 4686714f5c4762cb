"""Tether (pause-time) tracking on the GPU (Section 4.2; reading in
oracle/pause.py) against the FP64 oracle.

* Fixed node positions, accelerated kinetics: the wall-bond events are
  bit-exact (FP64 decision path, Philox keyed by site and step), so the
  device tracker's pause times (sorted: the device appends them in no fixed
  order) and open-tether state equal the oracle tracker's exactly.
* Full coupled runs (flow, membrane, IB, bonds) on a small channel with four
  discoid platelets over the ligand patch and accelerated kinetics (k_on0 dt
  = 0.01, k_off0 dt = 0.3, so tethers form and break every few steps): the
  GPU's and the oracle's pause-time samples are statistically matched.
  With the same seed the two runs share their random draws and their
  samples nearly coincide (two-sample KS p > 0.01); with an independent
  seed for the GPU run they are independent samples of one law (KS
  p > 1e-3)."""
import numpy as np
import pytest
import torch
from scipy import stats

import oracle
from oracle.pause import TetherTracker
from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu


def test_device_tracker_matches_the_oracle_on_fixed_positions():
    ni = nj = 16
    p = dict(lig_i0=0, lig_j0=0, lig_ni=ni, lig_nj=nj, box_nx=ni, box_ny=nj, max_per_ligand=4,
             z_wall=-0.5, sigma=1.0, l_b=0.64, d_capture=0.64, gamma=0.1, kT=0.05,
             kon0_dt=0.2, koff0_dt=0.2, seed=77)
    rng = np.random.default_rng(3)
    n = 2 * ni * nj
    # sites scattered over the patch at heights within and beyond reach
    pts = np.column_stack([rng.uniform(0, ni, n), rng.uniform(0, nj, n), rng.uniform(-0.45, 0.4, n)])
    X = np.ascontiguousarray(pts.T).ravel()
    tri = np.repeat(np.arange(n, dtype=np.int32), 3)
    site_tri = np.arange(n, dtype=np.int32)
    site_w = np.tile([1.0, 0.0], n)
    n_plt = 37
    site_plt = (np.arange(n) * 7919) % n_plt            # sites of a platelet spread over the patch
    bound = np.full(n, -1, dtype=np.int32)
    lig = np.zeros(ni * nj, dtype=np.int32)
    tri_dev = torch.as_tensor(tri).cuda()
    bonds = fsi.Bonds(p, site_tri, site_w.reshape(-1, 2), tri_dev, bound, lig)
    tr_dev = fsi.Tethers(bonds, site_plt, n_plt, capacity=4096)
    tr_ora = TetherTracker(site_plt, n_plt)
    Xd = torch.as_tensor(X).cuda()
    for step in range(400):
        bonds.step(Xd, n, step)
        tr_dev.update(step)
        oracle.bonds_step(p, site_tri, site_w, tri, X, bound, lig, step)
        tr_ora.update(bound, step + 1)
    torch.cuda.synchronize()
    assert np.array_equal(bonds.bound.cpu().numpy(), bound)
    assert len(tr_ora.pauses) > 300
    assert tr_dev.events() == len(tr_ora.pauses)
    assert np.array_equal(tr_dev.pauses(), np.sort(tr_ora.pauses))
    assert np.array_equal(tr_dev.state.cpu().numpy(), tr_ora.state)


def pause_workload(seed):
    """32x24x16 channel at shear 1000/s, four flat discoid platelets (162-node
    meshes, radius 0.6 um) just above a wall-wide ligand patch, 120 receptor
    sites each, accelerated kinetics; parameters rounded to FP32 so both
    sides start from the same numbers."""
    P = dict(workload.PHYSICAL, a=0.6e-6)
    w = workload.build(32, 24, 16, 0.8, 1000.0, 4, 2, 0, 120, 0, patch=(0, 0, 32, 24), gap=0.3,
                       orient="flat", phys=P, z_max=1.2)
    w["bonds"] = dict(w["bonds"], kon0_dt=0.01, koff0_dt=0.3, kT=0.05, sigma=0.02, gamma=0.05, seed=seed)
    w["membrane"] = {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in w["membrane"].items()}
    g = dict(w["grid"])
    g["tau"] = float(np.float32(g["tau"]))
    g["u_top"] = tuple(float(np.float32(u)) for u in g["u_top"])
    w["grid"] = g
    return w


def gpu_pauses(w, steps):
    sim = fsi.Simulation(w, track_tethers=1 << 16)
    sim.step(steps)
    torch.cuda.synchronize()
    return sim.tethers.pauses()


def test_coupled_pause_times_match_the_oracle():
    steps = 1500
    w = pause_workload(seed=11)
    g_same = gpu_pauses(w, steps)
    g_other = gpu_pauses(pause_workload(seed=12345), steps)
    ora = oracle.Sim(w)
    site_plt = oracle.site_platelets(ora.site_tri, w["mesh"]["tri"], w["mesh"]["node_plt"])
    tr = TetherTracker(site_plt, w["mesh"]["n_plt"])
    for _ in range(steps):
        ora.step()
        tr.update(ora.bound, ora.step_index)
    o = np.array(tr.pauses)
    assert min(len(o), len(g_same), len(g_other)) >= 200, (len(o), len(g_same), len(g_other))
    p_same = stats.ks_2samp(g_same, o).pvalue
    p_other = stats.ks_2samp(g_other, o).pvalue
    assert p_same > 0.01, (p_same, np.mean(g_same), np.mean(o))
    assert p_other > 1e-3, (p_other, np.mean(g_other), np.mean(o))
    # means within a few standard errors of each other as well
    se = np.sqrt(np.var(o) / len(o) + np.var(g_other) / len(g_other))
    assert abs(np.mean(g_other) - np.mean(o)) < 4.5 * se
