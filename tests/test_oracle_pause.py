"""Pins of the oracle's tether (pause-time) bookkeeping (Section 4.2; the
reading is stated in oracle/pause.py):

* hand-built bond-count sequences give the pause times of the definition
  (one platelet and several, a tether still open at the end, adjacent
  events);
* with the adhesion update of Section 3.2 at a fixed bond length, certain
  formation and the Bell rupture probability P_r of Eq. 12, every pause is a
  run of survived rupture tests: pause times are geometric,
  P(T = n) = (1 - P_r)^(n - 1) P_r, mean 1/P_r.  An off-by-one in the
  bookkeeping moves the mean by 1, ~30 standard errors."""
import math

import numpy as np

import oracle
from oracle.pause import TetherTracker, pauses_from_counts


def test_hand_built_sequences():
    assert pauses_from_counts([0, 1, 2, 0, 0, 3, 0, 1]) == [2, 1]
    assert pauses_from_counts([1, 1, 1]) == []            # still tethered at the end
    assert pauses_from_counts([1, 0, 1, 0]) == [1, 1]
    assert pauses_from_counts([0, 0, 0]) == []
    assert pauses_from_counts([5, 5, 0]) == [2]
    # three platelets, sites 0-1 on platelet 0, 2 on 1, 3-5 on 2
    tr = TetherTracker([0, 0, 1, 2, 2, 2], 3)
    seq = [[-1, 3, -1, -1, -1, -1],     # step count 1: platelet 0 tethered
           [-1, -1, 4, -1, 7, -1],      # 2: 0 free (pause 1), 1 and 2 tethered
           [2, -1, 4, -1, -1, 9],       # 3: 0 tethered again
           [-1, -1, -1, -1, -1, 9],     # 4: 0 and 1 free (pauses 1, 2)
           [-1, -1, -1, -1, -1, -1]]    # 5: 2 free (pause 3)
    for k, b in enumerate(seq):
        tr.update(np.array(b), k + 1)
    assert tr.pauses == [1, 1, 2, 3]
    assert list(tr.state) == [-1, -1, -1]
    # a saved state continues a tether across a restart
    tr = TetherTracker([0], 1, state=[7])
    tr.update(np.array([-1]), 10)
    assert tr.pauses == [3]


def test_pause_times_are_geometric_under_a_fixed_force():
    ni = nj = 32
    p = dict(lig_i0=0, lig_j0=0, lig_ni=ni, lig_nj=nj, box_nx=ni, box_ny=nj, max_per_ligand=4,
             z_wall=-0.5, sigma=1.0, l_b=0.64, d_capture=0.64, gamma=0.1, kT=0.05,
             kon0_dt=60.0, koff0_dt=0.05, seed=2024)
    # one site straight above every ligand (no other ligand within reach),
    # each on its own platelet: bond length 0.5, force sigma |0.5 - l_b|
    n = ni * nj
    pts = np.array([[i, j, -0.5 + 0.5] for j in range(nj) for i in range(ni)], dtype=float)
    X = np.ascontiguousarray(pts.T).ravel()
    tri = np.repeat(np.arange(n, dtype=np.int32), 3)
    site_tri = np.arange(n, dtype=np.int32)
    site_w = np.tile([1.0, 0.0], n)
    bound = np.full(n, -1, dtype=np.int32)
    lig = np.zeros(ni * nj, dtype=np.int32)
    tr = TetherTracker(np.arange(n), n)
    # formation on for 700 steps, then off until every tether has ended: all
    # tethers that began are counted, whatever their length (stopping with
    # tethers still open would drop the long ones preferentially)
    step = 0
    while step < 700 or (bound >= 0).any():
        q = p if step < 700 else dict(p, kon0_dt=0.0)
        oracle.bonds_step(q, site_tri, site_w, tri, X, bound, lig, step)
        tr.update(bound, step + 1)
        step += 1
        assert step < 1400
    assert (tr.state == -1).all()
    Fb = p["sigma"] * abs(0.5 - p["l_b"])
    Pr = -math.expm1(-p["koff0_dt"] * math.exp(p["gamma"] * Fb / p["kT"]))
    T = np.array(tr.pauses)
    N = len(T)
    assert N > 35000
    mean, se = T.mean(), math.sqrt(1.0 - Pr) / Pr / math.sqrt(N)
    assert abs(mean - 1.0 / Pr) < 4.5 * se, (mean, 1.0 / Pr, se)
    # the whole law: chi-square over n = 1..40 and the tail
    K = 40
    obs = np.array([(T == k).sum() for k in range(1, K + 1)] + [(T > K).sum()], dtype=float)
    prob = np.array([(1 - Pr) ** (k - 1) * Pr for k in range(1, K + 1)] + [(1 - Pr) ** K])
    exp = N * prob
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < 90.0, chi2            # 40 d.o.f.: p ~ 1e-5
