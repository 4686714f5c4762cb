"""FP64 reference of the learned membrane-force surrogate.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it).

The paper has no learned component; the surrogate is defined by this project
and written out here plainly, in FP64 numpy, one definition per function.

What the network stands for: the local membrane terms of Section 3.1 (edge
springs, Eq. 2-3; local area, Eq. 4 second term; dihedral bending), i.e. the
membrane energy with the global-area, volume, Morse and wall coefficients
set to zero.  That energy is a sum over membrane nodes i of a node share

  E_i = sum_k [ (k_s/4) (L_k - L0_k)^2 + (k_t/6) (S_k - S0_k)^2 / S0_k
                + (k_b/2) (1 - cos(phi_k - phi0_k)) ]

over the node's one-ring slots k: spoke k is the edge (i, n_k) of length L_k
(each edge is a spoke of both its ends: half its spring each), fan triangle
k is the face (i, n_k, n_{k+1}) of area S_k (each face is in the fans of its
three corners: a third each), and the spoke's bending angle phi_k is the
torsion of the chain n_{k+1} - i - n_k - n_{k-1} across it (half each).  In
the element strains of slot k

  x_s = (L - L0)/L0,   x_a = (S - S0)/S0,   x_b = phi - phi0 (wrapped to +-pi)

the node share's stresses are y = dE_i/dx:

  y_s = (k_s/2) L0^2 x_s,   y_a = (k_t/3) S0 x_a,   y_b = (k_b/2) sin x_b

and the local force is F = - sum_i sum_(slots, kinds) y dx/dX, with the
strain gradients dx/dX written out below (exact kinematics).  The network
replaces the stresses: per node it sees 42 inputs

  f[0..17]  = the strain direction x * s / |x * s| (s = in_scale[0..17];
              slot order: 6 stretches, 6 area strains, 6 bending angles;
              zero for empty slots and at rest),
  f[18..41] = rest descriptors of each slot: L0/l, S0/l^2, cos phi0, sin phi0
              (l = mean rest spoke length), each (r - in_shift) * in_scale,
              zero for empty slots,

and its output o (18) sets the stresses y = x * m * out_scale * o with the
rest moduli scales m = (L0^2, S0, 1): the surrogate force is zero at rest,
each stress has the sign of its strain, and the force is homogeneous of
degree one in the deformation.  Training minimises the mean over rows and
the 18 outputs of (a o - b)^2 with a = x m t, b = y t / out_scale (t a
per-output target scale): the error of the predicted stress.

The network is 42 -> 128 -> 128 -> 18 with the tanh form of GELU,
g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))); its gradients follow by
the chain rule, and Adam is Kingma and Ba, Algorithm 1.

The one-ring of node i: neighbours n_0 .. n_{d-1} (3 <= d <= 6) in cyclic
order (for an outward-oriented face (i, a, b), b follows a), starting at the
neighbour of smallest index.

It shares no code with the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 42, 128, 18
N_STRAIN = 18
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


# ----------------------------------------------------------- element geometry
def torsion(r1, r2, r3, r4):
    """Torsion angle of the chain r1-r2-r3-r4 and its gradient with respect
    to the four points (Blondel and Karplus, J. Comput. Chem. 17, 1996):
    F = r1 - r2, G = r2 - r3, H = r4 - r3, A = F x G, B = H x G,
    phi = atan2((B x A).G / (|A||B||G|), A.B / (|A||B|))."""
    F, G, H = r1 - r2, r2 - r3, r4 - r3
    A, B = np.cross(F, G), np.cross(H, G)
    A2, B2, gn = A @ A, B @ B, math.sqrt(G @ G)
    phi = math.atan2(np.cross(B, A) @ G / (math.sqrt(A2 * B2) * gn), (A @ B) / math.sqrt(A2 * B2))
    FG, HG = F @ G, H @ G
    g1 = -gn / A2 * A
    g4 = gn / B2 * B
    g2 = gn / A2 * A + FG / (A2 * gn) * A - HG / (B2 * gn) * B
    g3 = -gn / B2 * B - FG / (A2 * gn) * A + HG / (B2 * gn) * B
    return phi, (g1, g2, g3, g4)


def wrap(a):
    """Angle a in (-pi, pi]."""
    return a - 2.0 * math.pi * math.ceil((a - math.pi) / (2.0 * math.pi))


def slot_geometry(P, i, nb, k):
    """For node position P[i] and ring positions P[nb] (d of them), slot k:
    the spoke vector e_k, the fan triangle (i, n_k, n_{k+1}) cross product
    and the bending torsion of the chain n_{k+1} - i - n_k - n_{k-1} with its
    gradient (order: n_{k+1}, i, n_k, n_{k-1})."""
    d = len(nb)
    e = P[nb] - P[i]
    ek, en, ep = e[k], e[(k + 1) % d], e[(k - 1) % d]
    c = np.cross(ek, en)
    phi, g = torsion(P[nb[(k + 1) % d]], P[i], P[nb[k]], P[nb[(k - 1) % d]])
    return ek, c, phi, g


def strains(X, X0, ring, deg, nodes):
    """Element strains x [len(nodes)][18] (stretch, area, bending of slots
    0..5), rest moduli scales m [.][18] = (L0^2, S0, 1) and rest descriptors
    r [.][24] = (L0/l, S0/l^2, cos phi0, sin phi0) per slot; empty slots 0.
    X, X0: positions [n][3]."""
    x = np.zeros((len(nodes), N_STRAIN))
    m = np.zeros((len(nodes), N_STRAIN))
    r = np.zeros((len(nodes), 24))
    for row, i in enumerate(nodes):
        d = int(deg[i])
        nb = ring[i, :d]
        L0 = np.array([np.linalg.norm(slot_geometry(X0, i, nb, k)[0]) for k in range(d)])
        ell = L0.mean()
        for k in range(d):
            e, c, phi, _ = slot_geometry(X, i, nb, k)
            e0, c0, phi0, _ = slot_geometry(X0, i, nb, k)
            L, S, S0 = np.linalg.norm(e), 0.5 * np.linalg.norm(c), 0.5 * np.linalg.norm(c0)
            x[row, k] = (L - L0[k]) / L0[k]
            x[row, 6 + k] = (S - S0) / S0
            x[row, 12 + k] = wrap(phi - phi0)
            m[row, k], m[row, 6 + k], m[row, 12 + k] = L0[k] ** 2, S0, 1.0
            r[row, k] = L0[k] / ell
            r[row, 6 + k] = S0 / ell ** 2
            r[row, 12 + k] = math.cos(phi0)
            r[row, 18 + k] = math.sin(phi0)
    return x, m, r


def stress_coefficients(params):
    """(k_s/2, k_t/3, k_b/2) of a membrane parameter dict."""
    return 0.5 * params["k_spring"], params["k_t"] / 3.0, 0.5 * params["k_b"]


def exact_stresses(x, m, params):
    """The node shares' stresses y = dE_i/dx of the plain local terms."""
    cs, ca, cb = stress_coefficients(params)
    y = np.zeros_like(x)
    y[:, 0:6] = cs * m[:, 0:6] * x[:, 0:6]
    y[:, 6:12] = ca * m[:, 6:12] * x[:, 6:12]
    y[:, 12:18] = cb * np.sin(x[:, 12:18])
    return y


def node_energy(X, X0, ring, deg, nodes, params):
    """Sum over the rows of the node shares E_i (the local membrane energy)."""
    x, m, _ = strains(X, X0, ring, deg, nodes)
    cs, ca, cb = stress_coefficients(params)
    present = m[:, 0:6] > 0
    return float(np.sum(0.5 * cs * m[:, 0:6] * x[:, 0:6] ** 2) + np.sum(0.5 * ca * m[:, 6:12] * x[:, 6:12] ** 2)
                 + np.sum(cb * (1.0 - np.cos(x[:, 12:18])) * present))


def assemble(X, X0, ring, deg, nodes, y):
    """F = - sum_rows sum_slots y dx/dX with the strain gradients
    dx_s/dX = +-e_k/(L L0) at n_k / i, dx_a/dX_v = (1/2) nhat x (P_{v+2} -
    P_{v+1}) / S0 over the corners v of the fan triangle, dx_b/dX = the
    torsion gradient.  Returns [n][3]."""
    F = np.zeros_like(X)
    for row, i in enumerate(nodes):
        d = int(deg[i])
        nb = ring[i, :d]
        for k in range(d):
            e, c, _, g = slot_geometry(X, i, nb, k)
            e0, c0, _, _ = slot_geometry(X0, i, nb, k)
            L0, S0 = np.linalg.norm(e0), 0.5 * np.linalg.norm(c0)
            u = e / np.linalg.norm(e)
            F[nb[k]] -= y[row, k] * u / L0
            F[i] += y[row, k] * u / L0
            nh = c / np.linalg.norm(c)
            tri = (i, nb[k], nb[(k + 1) % d])
            for a in range(3):
                opp = X[tri[(a + 2) % 3]] - X[tri[(a + 1) % 3]]
                F[tri[a]] -= y[row, 6 + k] * 0.5 * np.cross(nh, opp) / S0
            chain = (nb[(k + 1) % d], i, nb[k], nb[(k - 1) % d])
            for a in range(4):
                F[chain[a]] -= y[row, 12 + k] * g[a]
    return F


# ------------------------------------------------------------------ network
def init_params(rng, in_scale=None, out_scale=None):
    """Weights with variance 1/fan_in (rows = outputs), zero biases, unit
    scales and zero shifts unless given."""
    p = dict(
        W1=rng.standard_normal((N_HID, N_IN)) / math.sqrt(N_IN), b1=np.zeros(N_HID),
        W2=rng.standard_normal((N_HID, N_HID)) / math.sqrt(N_HID), b2=np.zeros(N_HID),
        W3=rng.standard_normal((N_OUT, N_HID)) / math.sqrt(N_HID), b3=np.zeros(N_OUT),
    )
    p["in_shift"] = np.zeros(N_IN)
    p["in_scale"] = np.ones(N_IN) if in_scale is None else np.asarray(in_scale, float)
    p["out_scale"] = np.ones(N_OUT) if out_scale is None else np.asarray(out_scale, float)
    p["tgt_scale"] = np.ones(N_OUT)
    return p


TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")


def inputs(p, x, r):
    """Network inputs [B][42] from strains x and rest descriptors r."""
    f = np.zeros((x.shape[0], N_IN))
    xs = x * p["in_scale"][:N_STRAIN]
    mag = np.linalg.norm(xs, axis=1)
    nz = mag > 0
    f[nz, :N_STRAIN] = xs[nz] / mag[nz, None]
    present = np.tile(r[:, 0:6] > 0, 4)
    f[:, N_STRAIN:] = np.where(present, (r - p["in_shift"][N_STRAIN:]) * p["in_scale"][N_STRAIN:], 0.0)
    return f


def forward(p, f):
    """f: inputs [B][42].  Returns output o [B][18] and the cache."""
    z1 = f @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, dict(f=f, z1=z1, h1=h1, z2=z2, h2=h2)


def targets(p, x, m, y):
    """Training record of each row: a = x m t, b = y t / out_scale."""
    t = p["tgt_scale"]
    return x * m * t, y * t / p["out_scale"]


def loss(o, a, b):
    """Mean over the batch and the 18 outputs of (a o - b)^2."""
    return float(np.mean((a * o - b) ** 2))


def backward(p, cache, o, a, b):
    """Gradients of loss(o, a, b) for every trained parameter."""
    B = o.shape[0]
    do = 2.0 * a * (a * o - b) / (B * N_OUT)
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


def predicted_stresses(p, x, m, r):
    """Stresses the network sets: y = x m out_scale o."""
    o, _ = forward(p, inputs(p, x, r))
    return x * m * p["out_scale"] * o


def predict_forces(p, X, X0, ring, deg, nodes):
    """Surrogate local forces [n][3] (global frame) of the rows `nodes`."""
    x, m, r = strains(X, X0, ring, deg, nodes)
    return assemble(X, X0, ring, deg, nodes, predicted_stresses(p, x, m, r))


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
