"""GPU parity of the adhesion update (Section 3.2, Eq. 12-14) against the
oracle: with positions held fixed, every bond event (which site binds which
ligand, which bonds break, per-ligand counts) is bit-exact step by step; the
bond spring forces match within FP32 rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu


def sheet_workload(n_sites=3000, seed=0, **rates):
    """A flat platelet resting 0.05 lattice units above a ligand patch, so that
    many receptor sites are within the capture distance."""
    w = workload.build(32, 32, 64, 0.8, 100.0, 1, 3, 0, n_sites, seed, patch=(8, 8, 16, 16), orient="flat",
                       gap=0.05, centers=[(16.3, 15.8, -0.5 + 0.05 + 1.25)])
    w["bonds"].update(rates)
    return w


def run_both(w, steps, X=None):
    X = w["X"] if X is None else X
    tri = np.ascontiguousarray(w["mesh"]["tri"], dtype=np.int32).ravel()
    tri_d = torch.from_numpy(tri).cuda()
    b = fsi.Bonds(w["bonds"], w["sites"]["tri"], w["sites"]["w"], tri_d, w["bound"], w["lig_count"])
    Xd = torch.from_numpy(X).cuda()
    bound = w["bound"].copy()
    lig = w["lig_count"].copy()
    st = np.ascontiguousarray(w["sites"]["tri"], dtype=np.int32)
    sw = np.ascontiguousarray(w["sites"]["w"], dtype=np.float64).ravel()
    history = []
    for step in range(steps):
        b.step(Xd, w["M"], step)
        ev = oracle.bonds_step(w["bonds"], st, sw, tri, X, bound, lig, step)
        torch.cuda.synchronize()
        gb = b.bound.cpu().numpy()
        gl = b.lig_count.cpu().numpy()
        assert np.array_equal(gb, bound), "bound sites differ at step %d" % step
        assert np.array_equal(gl, lig), "ligand counts differ at step %d" % step
        history.append(ev)
    return b, bound, history


def test_events_bit_exact_fixed_positions():
    w = sheet_workload(kon0_dt=0.3, koff0_dt=0.02, sigma=0.05, kT=0.02, gamma=0.05)
    b, bound, hist = run_both(w, 40)
    nr = sum(h[0] for h in hist)
    nf = sum(h[1] for h in hist)
    assert nf > 100 and nr > 20, (nr, nf)
    rc, counters = b.status()
    assert rc == 0 and counters[0] == nr and counters[1] == nf and counters[2] == 0
    assert (np.asarray(bound) >= -1).all()


def test_capacity_saturates_all_ligands():
    w = sheet_workload(n_sites=3000, kon0_dt=50.0, koff0_dt=0.0, sigma=0.05, kT=0.02, gamma=0.05)
    b, bound, hist = run_both(w, 6)
    lig = b.lig_count.cpu().numpy()
    assert lig.max() == 4 and (lig <= 4).all()
    counts = np.bincount(bound[bound >= 0], minlength=lig.size)
    assert np.array_equal(counts, lig)


def test_bond_forces_parity():
    w = sheet_workload(kon0_dt=0.3, koff0_dt=0.0, sigma=0.05, kT=0.02, gamma=0.05)
    b, bound, _ = run_both(w, 5)
    rng = np.random.default_rng(2)
    X = w["X"] + 0.05 * rng.standard_normal(w["X"].shape)   # stretch and compress the bonds
    Fd = torch.zeros(X.size, dtype=torch.float32, device="cuda")
    b.forces(torch.from_numpy(X).cuda(), Fd, w["M"])
    F = np.zeros(X.size)
    oracle.bond_forces(w["bonds"], np.ascontiguousarray(w["sites"]["tri"], dtype=np.int32),
                       np.ascontiguousarray(w["sites"]["w"]).ravel(),
                       np.ascontiguousarray(w["mesh"]["tri"], dtype=np.int32).ravel(), bound, X, F)
    torch.cuda.synchronize()
    Fg = Fd.cpu().numpy()
    assert np.max(np.abs(F)) > 0
    assert np.max(np.abs(Fg - F)) < 1e-5 * np.max(np.abs(F))


@pytest.mark.parametrize("d_capture", [1.0, 1.7])
def test_events_bit_exact_capture_beyond_one_spacing(d_capture):
    """Capture distances of one and more lattice spacings (128 nm on a finer
    lattice): each site's candidates come from the 2r x 2r nodes around it
    (r = ceil(d_capture); 4 x 4 at 1.7), every draw and event as the
    oracle's scan of the whole patch."""
    w = sheet_workload(kon0_dt=0.05, koff0_dt=0.05, sigma=0.05, kT=0.02, gamma=0.05, d_capture=d_capture,
                       l_b=0.8 * d_capture)
    b, bound, hist = run_both(w, 30)
    nr = sum(h[0] for h in hist)
    nf = sum(h[1] for h in hist)
    assert nf > 100 and nr > 20, (nr, nf)
    rc, counters = b.status()
    assert rc == 0 and counters[0] == nr and counters[1] == nf


def test_capture_distance_argument_checks():
    w = sheet_workload()
    for bad in (0.0, -1.0, 8.5, float("nan")):
        with pytest.raises(RuntimeError):
            run_both(dict(w, bonds=dict(w["bonds"], d_capture=bad)), 1)
