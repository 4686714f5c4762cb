"""FP64 reference of the learned membrane-force surrogate.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it).

The paper has no learned component; the surrogate is defined by this project
and written out here plainly, in FP64 numpy, one definition per function:

* one-ring features of a membrane node (27 per node, in a local frame),
* the network 27 -> 128 -> 128 -> 3 with the tanh form of GELU,
  g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
* its mean-squared-error loss, the gradients of every parameter by the chain
  rule, and one Adam step (Kingma and Ba, Algorithm 1),
* the forces it stands for: the local membrane terms of Section 3.1 (edge
  springs, Eq. 3; local area, Eq. 4 second term; dihedral bending), i.e. the
  membrane force with the global-area, volume, Morse and wall coefficients
  set to zero.

Features of node i with one-ring neighbours n_0 .. n_{d-1} (d <= 6, counter-
clockwise seen from outside, starting at the neighbour of smallest index):
  e_k = X[n_k] - X[i];  nu = sum_k e_k x e_{k+1} (cyclic);  z = nu/|nu|;
  x = unit(e_0 - (e_0.z) z);  y = z x x;  R = rows (x, y, z).
The same construction on the rest positions X0 gives R0, e0_k, and the
node's length scale l = mean_k |e0_k|.  Then
  delta_k = (R e_k - R0 e0_k) / l,  mag = |(delta_0 .. delta_5)|
  delta_k / mag                            18 inputs (zero for k >= d, and
                                           all zero when mag = 0)
  kappa0  = R0 (mean_k e0_k) / l           3 inputs (rest curvature normal)
  rho_k   = |e0_k| / l                     6 inputs (rest-length ratios,
                                           zero for k >= d)
each multiplied by a fixed per-input scale.  The deformation enters through
the direction delta / mag and the magnitude mag; kappa0 and rho_k describe
the node's rest one-ring, on which its stiffness depends.  The network output
o (3) times mag times a fixed per-component scale is the local force in the
frame R: the force is R^T (o * mag * out_scale), zero at rest and
homogeneous of degree one in the deformation, as the local membrane forces
are in the linear-elastic range (where the strains of a platelet in shear
flow lie).

It shares no code with the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 27, 128, 3
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


# --------------------------------------------------------------------- GELU
def gelu(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * z * (1.0 + t)


def gelu_grad(z):
    u = GELU_C * (z + GELU_A * z ** 3)
    t = np.tanh(u)
    du = GELU_C * (1.0 + 3.0 * GELU_A * z ** 2)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


# ------------------------------------------------------------------ one ring
def one_rings(tri, n_nodes):
    """Cyclic one-ring of every node of a closed, outward-oriented triangle
    mesh: for a face (i, a, b) counter-clockwise, b follows a around i.
    Returns (ring[n_nodes][6] int, -1 padded; degree[n_nodes]).  Nodes in no
    triangle get degree 0."""
    nxt = [dict() for _ in range(n_nodes)]
    for a, b, c in np.asarray(tri, dtype=np.int64):
        for i, p, q in ((a, b, c), (b, c, a), (c, a, b)):
            nxt[i][int(p)] = int(q)
    ring = -np.ones((n_nodes, 6), dtype=np.int64)
    deg = np.zeros(n_nodes, dtype=np.int64)
    for i in range(n_nodes):
        if not nxt[i]:
            continue
        d = len(nxt[i])
        if d > 6:
            raise ValueError("node %d has %d neighbours (at most 6 supported)" % (i, d))
        start = min(nxt[i])
        k, cur = 0, start
        while True:
            ring[i, k] = cur
            k += 1
            cur = nxt[i][cur]
            if cur == start:
                break
            if k >= d:
                raise ValueError("node %d: open or non-manifold one-ring" % i)
        if k != d:
            raise ValueError("node %d: one-ring does not close" % i)
        deg[i] = d
    return ring, deg


def frame(e, d):
    """Local frame R (rows x, y, z) from the first d edge vectors e[k]."""
    nu = np.zeros(3)
    for k in range(d):
        nu += np.cross(e[k], e[(k + 1) % d])
    z = nu / np.linalg.norm(nu)
    x = e[0] - np.dot(e[0], z) * z
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z])


def features(X, X0, ring, deg, nodes):
    """Unscaled features [len(nodes)][27], frames [len(nodes)][3][3] and
    deformation magnitudes [len(nodes)].  X, X0: positions [n][3]."""
    out = np.zeros((len(nodes), N_IN))
    frames = np.zeros((len(nodes), 3, 3))
    mags = np.zeros(len(nodes))
    for r, i in enumerate(nodes):
        d = int(deg[i])
        nb = ring[i, :d]
        e = X[nb] - X[i]
        e0 = X0[nb] - X0[i]
        R = frame(e, d)
        R0 = frame(e0, d)
        L0 = np.linalg.norm(e0, axis=1)
        ell = L0.mean()
        for k in range(d):
            out[r, 3 * k:3 * k + 3] = (R @ e[k] - R0 @ e0[k]) / ell
            out[r, 21 + k] = L0[k] / ell
        mag = np.linalg.norm(out[r, :18])
        out[r, :18] = out[r, :18] / mag if mag > 0 else 0.0
        out[r, 18:21] = R0 @ e0.mean(axis=0) / ell
        frames[r] = R
        mags[r] = mag
    return out, frames, mags


# ------------------------------------------------------------------ network
def init_params(rng, scale_in=None, scale_out=None):
    """Weights with variance 1/fan_in (rows = outputs), zero biases."""
    p = dict(
        W1=rng.standard_normal((N_HID, N_IN)) / math.sqrt(N_IN), b1=np.zeros(N_HID),
        W2=rng.standard_normal((N_HID, N_HID)) / math.sqrt(N_HID), b2=np.zeros(N_HID),
        W3=rng.standard_normal((N_OUT, N_HID)) / math.sqrt(N_HID), b3=np.zeros(N_OUT),
    )
    p["in_scale"] = np.ones(N_IN) if scale_in is None else np.asarray(scale_in, float)
    p["out_scale"] = np.ones(N_OUT) if scale_out is None else np.asarray(scale_out, float)
    return p


TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(p, f):
    """f: scaled features [B][27].  Returns output o [B][3] and the cache."""
    z1 = f @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, dict(f=f, z1=z1, h1=h1, z2=z2, h2=h2)


def loss(o, t):
    """Mean over the batch and the 3 components of the squared error."""
    return float(np.mean((o - t) ** 2))


def backward(p, cache, o, t):
    """Gradients of loss(o, t) for every trained parameter."""
    B = o.shape[0]
    do = 2.0 * (o - t) / (B * N_OUT)
    g = dict(W3=do.T @ cache["h2"], b3=do.sum(0))
    dz2 = (do @ p["W3"]) * gelu_grad(cache["z2"])
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(cache["z1"])
    g["W1"] = dz1.T @ cache["f"]
    g["b1"] = dz1.sum(0)
    return g


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the trained parameters (state: m, v, t)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in TRAINED:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1.0 - beta1) * g[k]
        v[...] = beta2 * v + (1.0 - beta2) * g[k] * g[k]
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return p


def predict_forces(p, X, X0, ring, deg, nodes):
    """Surrogate local forces [len(nodes)][3] in the global frame."""
    f, R, mag = features(X, X0, ring, deg, nodes)
    o, _ = forward(p, f * p["in_scale"])
    Fl = o * mag[:, None] * p["out_scale"]
    return np.einsum("nij,ni->nj", R, Fl)


def local_targets(F_local, frames, mags, out_scale):
    """Training targets: the plain solver's local forces in each node's frame,
    divided by the deformation magnitude and the output scale (zero where
    the node is undeformed)."""
    t = np.einsum("nij,nj->ni", frames, F_local) / out_scale
    safe = np.where(mags > 0, mags, 1.0)
    return np.where(mags[:, None] > 0, t / safe[:, None], 0.0)


def local_params(params):
    """Membrane coefficients of the local terms only (edge springs, local
    area, bending): global area, volume, Morse and wall terms switched off."""
    q = dict(params)
    for k in ("k_s", "k_v", "morse_D", "rep_F0"):
        q[k] = 0.0
    return q


def global_params(params):
    """The complement of local_params: global area, volume, Morse, wall."""
    q = dict(params)
    for k in ("k_spring", "k_t", "k_b"):
        q[k] = 0.0
    return q
