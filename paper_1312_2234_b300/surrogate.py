"""Training and use of the learned membrane-force surrogate.

The network (42 -> 128 -> 128 -> 18, GELU) sets the element stresses of the
local membrane terms (springs, local area, bending) in a node-share split of
their energy; the CUDA library computes its element strains and inputs, its
forward and backward passes (BF16 tensor cores, or FP32 in check mode), Adam,
the training records (the plain terms' stresses at a state), and the
surrogate force inside the coupled step (stresses times the exact strain
gradients).  This module only organises the data: membrane states from the
plain method's trajectories (plus random perturbations of them, so that the
training set also covers deformations a short run does not reach), the
input, output and target scales, the batches, and the judge that compares
the surrogate with the plain solver and falls back to it.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fsi

N_IN, N_HID, N_OUT = 42, 128, 18


def local_params(params):
    """Membrane coefficients of the local terms only (springs, local area,
    bending): the force the surrogate stands for."""
    q = dict(params)
    for k in ("k_s", "k_v", "morse_D", "rep_F0"):
        q[k] = 0.0
    return q


def init_params(rng, in_scale=None, out_scale=None):
    """Weights with variance 1/fan_in, zero biases, zero input shifts, unit
    target scales (reference layout)."""
    p = dict(W1=rng.standard_normal((N_HID, N_IN)) / np.sqrt(N_IN), b1=np.zeros(N_HID),
             W2=rng.standard_normal((N_HID, N_HID)) / np.sqrt(N_HID), b2=np.zeros(N_HID),
             W3=rng.standard_normal((N_OUT, N_HID)) / np.sqrt(N_HID), b3=np.zeros(N_OUT))
    p["in_shift"] = np.zeros(N_IN)
    p["in_scale"] = np.ones(N_IN) if in_scale is None else np.asarray(in_scale, float)
    p["out_scale"] = np.ones(N_OUT) if out_scale is None else np.asarray(out_scale, float)
    p["tgt_scale"] = np.ones(N_OUT)
    return p


def perturbed_states(X_list, mesh, amplitudes, copies, rng):
    """Each state of X_list (double [3][M]) plus `copies` random perturbations
    per amplitude (Gaussian, amplitude x the mean rest edge length, membrane
    nodes only)."""
    X0 = np.asarray(mesh["X0"]).reshape(3, -1)
    tri = np.asarray(mesh["tri"])
    ell = float(np.mean(np.linalg.norm(X0[:, tri[:, 0]] - X0[:, tri[:, 1]], axis=0)))
    mem = np.asarray(mesh["is_membrane"]).astype(bool)
    out = []
    for X in X_list:
        out.append(np.ascontiguousarray(X, dtype=np.float64))
        for a in amplitudes:
            for _ in range(copies):
                d = np.zeros((3, X0.shape[1]))
                d[:, mem] = a * ell * rng.standard_normal((3, int(mem.sum())))
                out.append(np.ascontiguousarray((np.asarray(X).reshape(3, -1) + d).ravel()))
    return out


class Dataset:
    """Inputs and training records (stress targets) of many membrane states,
    on the GPU.  membrane_params: the chamber's membrane coefficients (the
    local ones, k_spring, k_t and k_b, give the stresses)."""

    def __init__(self, sg, params, membrane_params, states, device="cuda"):
        feats, targets = [], []
        for X in states:
            Xd = torch.as_tensor(X, device=device)
            feat, xs, ms = sg.features(params, Xd)
            t = sg.targets(params, membrane_params, xs, ms)
            feats.append(feat[:sg.rows])
            targets.append(t[:sg.rows])
        self.feat = torch.cat(feats)
        self.target = torch.cat(targets)

    def __len__(self):
        return self.feat.shape[0]


KINDS = (slice(0, 6), slice(6, 12), slice(12, 18))   # stretch, area, bending outputs


def fit_scales(sg, params, membrane_params, states):
    """Rest-descriptor, output and target scales from raw (unit-scale)
    statistics over the states, per kind of slot (the six slots of a kind
    share them): shift and scale of a rest descriptor = its mean and 1 / its
    std (1 where it does not vary); out_scale = the
    least-squares modulus sum(y x m) / sum((x m)^2), so that the stresses are
    about x m out_scale and the network output about 1; tgt_scale =
    1 / rms(x m)."""
    p = params.get()
    p["in_shift"] = np.zeros(N_IN)
    p["in_scale"] = np.ones(N_IN)
    p["out_scale"] = np.ones(N_OUT)
    p["tgt_scale"] = np.ones(N_OUT)
    params.set(p)
    raw = Dataset(sg, params, membrane_params, states)
    f = raw.feat.float().cpu().numpy().astype(np.float64)
    t = raw.target.cpu().numpy().astype(np.float64)
    a, b = t[:, :N_OUT], t[:, N_OUT:]
    present = f[:, 18:24] != 0          # L0/l > 0 in every present slot
    for q in range(4):
        cols = slice(18 + 6 * q, 24 + 6 * q)
        v = f[:, cols][present]
        mu, sd = float(v.mean()), float(v.std())
        p["in_shift"][cols] = mu
        p["in_scale"][cols] = 1.0 / sd if sd > 1e-6 * max(1.0, abs(mu)) else 1.0
    for kind in KINDS:
        ak, bk = a[:, kind][present], b[:, kind][present]
        den = float(np.sum(ak * ak))
        p["out_scale"][kind] = float(np.sum(ak * bk)) / den if den > 0 else 1.0
        rms = math.sqrt(den / max(1, ak.size))
        p["tgt_scale"][kind] = 1.0 / rms if rms > 0 else 1.0
    params.set(p)
    return p


def fit_strain_scales(sg, params, states):
    """in_scale of the strain directions: 1 / rms of each kind's strains over
    the states (present slots)."""
    p = params.get()
    sums = np.zeros(3)
    counts = np.zeros(3)
    for X in states:
        feat, xs, ms = sg.features(params, torch.as_tensor(X, device=params.device))
        x = xs[:sg.rows].cpu().numpy().astype(np.float64)
        on = ms[:sg.rows, :6].cpu().numpy() > 0
        for q, kind in enumerate(KINDS):
            sums[q] += float(np.sum(x[:, kind][on] ** 2))
            counts[q] += on.sum()
    for q, kind in enumerate(KINDS):
        rms = math.sqrt(sums[q] / max(1.0, counts[q]))
        p["in_scale"][kind] = 1.0 / rms if rms > 0 else 1.0
    params.set(p)
    return p


def prepare(sg, params, membrane_params, states):
    """All scales (fit_scales, then fit_strain_scales) and the dataset."""
    fit_scales(sg, params, membrane_params, states)
    fit_strain_scales(sg, params, states)
    return Dataset(sg, params, membrane_params, states)


def train(params, data, steps, batch=1024, lr=1e-3, mode="bf16", seed=0, log_every=0, decay=True):
    """Adam on random batches of the dataset (learning rate decayed to 2 % of
    lr on a cosine schedule when decay).  Returns [(step, loss)]."""
    g = torch.Generator(device=data.feat.device)
    g.manual_seed(seed)
    B = fsi.SurrogateBatch(batch, device=data.feat.device)
    hist = []
    n = len(data)
    for it in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g, device=data.feat.device)
        feat = data.feat.index_select(0, idx).contiguous()
        tgt = data.target.index_select(0, idx).contiguous()
        loss = B.grad(params, feat, tgt, mode)
        rate = lr * (0.02 + 0.98 * 0.5 * (1.0 + math.cos(math.pi * it / max(1, steps)))) if decay else lr
        fsi.sg_adam(params, rate)
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, float(loss.item())))
    return hist


def rel_force_error(F_test, F_ref, mask):
    """max |F_test - F_ref| / max |F_ref| over the nodes in mask."""
    a = F_test.reshape(3, -1)[:, mask]
    b = F_ref.reshape(3, -1)[:, mask]
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-30))


class Judge:
    """Keeps the plain solver as the judge of the surrogate: every `every`
    steps it computes the plain and the surrogate membrane force at the
    current positions and, if they differ by more than `tol` of the largest
    plain force on a membrane node, switches the simulation back to the plain
    solver (the fallback) for the rest of the run."""

    def __init__(self, sim, sg, params, membrane_plain, is_membrane, every=100, tol=0.05):
        self.sim, self.sg, self.params = sim, sg, params
        self.plain = membrane_plain
        self.every, self.tol = every, tol
        self.active = True
        self.errors = []
        M = sim.M
        self.Fp = torch.zeros(3 * M, dtype=torch.float32, device=sim.X.device)
        self.Fs = torch.zeros_like(self.Fp)
        self.mask = torch.as_tensor(np.asarray(is_membrane).astype(bool), device=sim.X.device)
        fsi.sim_set_surrogate(sim, sg, params)

    def error(self):
        self.plain.forces(self.sim.X, self.Fp)
        self.sg.forces(self.params, self.plain, self.sim.X, self.Fs)
        return rel_force_error(self.Fs, self.Fp, self.mask)

    def step(self, n):
        done = 0
        while done < n:
            k = min(self.every, n - done)
            self.sim.step(k)
            done += k
            if self.active:
                e = self.error()
                self.errors.append(e)
                if e > self.tol:
                    fsi.sim_set_surrogate(self.sim, None, None)
                    self.active = False
        return self.active
