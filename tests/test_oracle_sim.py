"""The oracle's coupled step (Fig. 1 order): a platelet at its rest shape in
fluid at rest stays put; mass is conserved to round-off while a platelet is
advected by the shear flow; the spread force equals the total nodal force."""
import numpy as np

from paper_1312_2234_b300 import workload as W


def test_rest_state_is_stationary(oracle_lib):
    w = W.tiny(seed=1, shear=0.0, gap=2.0)
    sim = oracle_lib.Sim(w)
    X0 = sim.X.copy()
    f0 = sim.f.copy()
    for _ in range(4):
        sim.step()
    assert np.max(np.abs(sim.X - X0)) < 1e-12
    assert np.max(np.abs(sim.f - f0)) < 1e-12


def test_coupled_mass_and_force_balance(oracle_lib):
    w = W.tiny(seed=2, shear=2.0e5, gap=2.5)  # strong shear; clear of the wall (no truncation)
    sim = oracle_lib.Sim(w)
    m0 = sim.f.sum()
    X0 = sim.X.copy().reshape(3, -1)
    for _ in range(6):
        sim.step()
        assert abs(sim.f.sum() - m0) < 1e-11 * m0
        N = sim.N
        assert np.allclose(sim.g.reshape(3, N).sum(1), sim.F.reshape(3, -1).sum(1), atol=1e-12)
    X = sim.X.reshape(3, -1)
    dx = (X - X0)[0]
    assert (dx > 0).all()                     # carried downstream by the shear flow
    u_c = w["grid"]["u_top"][0] * (X0[2].mean() + 0.5) / w["grid"]["nz"]
    assert 0.3 < dx.mean() / (6 * u_c) < 1.5
