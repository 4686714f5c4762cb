"""Training and use of the learned membrane-force surrogate.

The network (27 -> 128 -> 128 -> 3, GELU) stands for the local membrane terms
(springs, local area, bending); the CUDA library computes its features, its
forward and backward passes (BF16 tensor cores, or FP32 in check mode), Adam,
and the surrogate force inside the coupled step.  This module only organises
the data: membrane states from the plain method's trajectories (plus random
perturbations of them, so that the training set also covers deformations
larger than a short run reaches), the per-input and per-output scales, the
batches, and the judge that compares the surrogate with the plain solver and
falls back to it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fsi


def local_params(params):
    """Membrane coefficients of the local terms only (springs, local area,
    bending): the force the surrogate is trained to reproduce."""
    q = dict(params)
    for k in ("k_s", "k_v", "morse_D", "rep_F0"):
        q[k] = 0.0
    return q


def init_params(rng, in_scale=None, out_scale=None):
    """Weights with variance 1/fan_in, zero biases (reference layout)."""
    p = dict(W1=rng.standard_normal((128, 27)) / np.sqrt(27.0), b1=np.zeros(128),
             W2=rng.standard_normal((128, 128)) / np.sqrt(128.0), b2=np.zeros(128),
             W3=rng.standard_normal((3, 128)) / np.sqrt(128.0), b3=np.zeros(3))
    p["in_scale"] = np.ones(27) if in_scale is None else np.asarray(in_scale, float)
    p["out_scale"] = np.ones(3) if out_scale is None else np.asarray(out_scale, float)
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
    """Features and local-frame targets of many membrane states, on the GPU."""

    def __init__(self, sg, params, membrane_local, states, device="cuda"):
        feats, targets = [], []
        F = torch.zeros(3 * sg.n, dtype=torch.float32, device=device)
        for X in states:
            Xd = torch.as_tensor(X, device=device)
            feat, frames, mags = sg.features(params, Xd)
            membrane_local.forces(Xd, F)
            t = sg.targets(params, F, frames, mags)
            feats.append(feat[:sg.rows])
            targets.append(t[:sg.rows])
        self.feat = torch.cat(feats)
        self.target = torch.cat(targets)

    def __len__(self):
        return self.feat.shape[0]


def fit_scales(sg, params, membrane_local, states):
    """Per-input and per-output scales from raw (unit-scale) statistics:
    in_scale = 1 / std of each input over the states (1 where constant),
    out_scale = std of each local force component."""
    p = params.get()
    p["in_scale"] = np.ones(27)
    p["out_scale"] = np.ones(3)
    params.set(p)
    raw = Dataset(sg, params, membrane_local, states)
    f = raw.feat.float().cpu().numpy()[:, :27]
    t = raw.target.cpu().numpy()
    sd = f.std(0)
    p["in_scale"] = np.where(sd > 1e-12, 1.0 / np.maximum(sd, 1e-30), 1.0)
    ts = t.std(0)
    p["out_scale"] = np.where(ts > 0, ts, 1.0)
    params.set(p)
    return p


def train(params, data, steps, batch=1024, lr=1e-3, mode="bf16", seed=0, log_every=0):
    """Adam on random batches of the dataset.  Returns [(step, loss)]."""
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
        fsi.sg_adam(params, lr)
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
