"""Tether (pause-time) bookkeeping of the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.

Section 4.2 characterises adhesion by pause times: how long a platelet that
has been captured by the vWF-coated wall stays held there before it moves on,
the rupture rate k_off following from how the number of pauses decays with
their length.  The paper gives no bookkeeping rule.  Reading (used by the
CUDA tracker as well): after every step's adhesion update a platelet is
tethered when at least one of its receptor sites holds a wall bond; a tether
event starts at the first update after which the platelet is tethered and
ends at the first later update after which it is not; its pause time is the
number of updates between the two, i.e. the number of consecutive
post-update states in which the platelet held a bond.  A bond formed in
step s and broken in step s + n gives a pause of n steps.

"Step count" below is the number of completed steps: after the update of
step s it is s + 1.
"""
from __future__ import annotations

import numpy as np


class TetherTracker:
    """Per-platelet tether state and the pause times of completed events.

    site_plt: the platelet of every receptor site; n_plt: number of
    platelets; state: optional saved state (step count at which each
    platelet's open tether began, -1 when free).
    """

    def __init__(self, site_plt, n_plt, state=None):
        self.site_plt = np.asarray(site_plt, dtype=np.int64)
        self.n_plt = int(n_plt)
        if state is None:
            self.state = np.full(self.n_plt, -1, dtype=np.int64)
        else:
            self.state = np.array(state, dtype=np.int64)
        self.pauses: list[int] = []

    def update(self, bound, now):
        """bound: every site's wall-bond state after the adhesion update
        (>= 0: bound); now: the step count after that update."""
        bonds_per_platelet = np.bincount(self.site_plt[np.asarray(bound) >= 0], minlength=self.n_plt)
        for p in range(self.n_plt):
            tethered = bonds_per_platelet[p] > 0
            if tethered and self.state[p] < 0:
                self.state[p] = now
            elif not tethered and self.state[p] >= 0:
                self.pauses.append(int(now - self.state[p]))
                self.state[p] = -1


def pauses_from_counts(counts):
    """Pause times of one platelet from its bond counts after successive
    updates (counts[k] after the update that brings the step count to k + 1);
    a tether still open at the end is not counted."""
    tr = TetherTracker(np.zeros(1, dtype=np.int64), 1)
    for k, n in enumerate(counts):
        tr.update(np.zeros(1, dtype=np.int64) if n > 0 else np.full(1, -1), k + 1)
    return tr.pauses
