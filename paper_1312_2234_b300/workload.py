"""Seeded synthetic workloads for the platelet fluid-structure step.

This module builds inputs only: geometry (icosphere-derived platelet meshes,
interior SCE points, receptor sites, platelet placement), the topology lists
given to the solvers (triangles, Morse pair lists) and the conversion of the
paper's physical parameters (Table 2) to lattice units.  It holds none of the
method's arithmetic (no forces, no lattice Boltzmann, no delta kernel, no bond
kinetics); both the CUDA library's tests and the oracle take their inputs from
here.  Every random choice is drawn from ``numpy.random.default_rng(seed)``.

Shapes and sizes follow the paper's workloads: a discoid platelet is the
oblate ellipsoid x^2/a^2 + y^2/a^2 + z^2/(lambda a)^2 = 1 with a = 1 um and
lambda = 0.25 (Section 3.1), meshed by a triangulated surface; receptors are
point sites placed uniformly by area on the membrane (Section 3.2); vWF
ligands cover a patch of the bottom wall at one per lattice node (25 per
um^2 at h = 0.2 um, Section 3.2/3.3).
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Physical parameters (Table 2 and Sections 3.1-3.4).  Entries marked
# "reading" are not fixed by the paper; the value is this project's choice.
# ---------------------------------------------------------------------------
PHYSICAL = dict(
    h=0.2e-6,            # lattice spacing (Section 3.3)
    rho=1023.9,          # plasma density, kg/m^3 (Table 2)
    mu=1.2e-3,           # plasma viscosity, Pa s (Table 2)
    a=1.0e-6,            # platelet radius (Table 2)
    aspect=0.25,         # platelet aspect ratio (Table 2)
    E=25e3,              # elastic modulus, Pa (Table 2)
    dx_link=0.1e-6,      # unit link length in k = 2 E dx / 5 (Eq. 3 text)
    l0=75e-9,            # average initial spring length (Table 2)
    T=300.0,             # temperature (Table 2)
    kB=1.380649e-23,
    area_factor=6000.0,  # k_s = k_t = 6000 kBT / l0^2 (Table 2)
    vol_factor=6000.0,   # k_v = 6000 kBT / l0^3 (Table 2)
    bend_factor=200.0,   # k0 = 200 kBT (Table 2)
    koff0=3.45,          # 1/s (Table 2)
    kon0=1.0e4,          # 1/s; reading (Table 2 prints 1e-5, which forms no bonds)
    rep_F0=500e-12 * 1e-9,  # 500 pN nm; reading of "500 pN m" (Section 3.4.1)
    rep_tau=2000e6,      # 2000 per um (Section 3.4.1)
    rep_eps_min=0.5e-9,  # reading: clamp of the wall gap
    sigma=1.0e-3,        # bond spring constant, N/m; reading (not given)
    l_b=128e-9,          # equilibrium bond length = capture distance (Section 3.2)
    d_capture=128e-9,    # 128 nm (Section 3.2)
    gamma=0.1e-9,        # reactive compliance; reading (not given)
    morse_width=0.1e-6,  # Morse range 1/a; reading
)


def lattice_units(tau: float, phys: dict | None = None) -> dict:
    """Lattice-unit constants for relaxation time ``tau`` (h = dt = rho0 = 1).

    dt follows from the viscosity relation of Section 3.3 (Eq. 22 and the
    parameter choice after it): dt = (tau - 1/2) h^2 / (3 nu), nu = mu / rho.
    """
    P = dict(PHYSICAL if phys is None else phys)
    h = P["h"]
    nu = P["mu"] / P["rho"]
    dt = (tau - 0.5) * h * h / (3.0 * nu)
    m_u = P["rho"] * h ** 3
    F_u = m_u * h / dt ** 2
    E_u = F_u * h
    kBT = P["kB"] * P["T"]
    k_spring = 2.0 * P["E"] * P["dx_link"] / 5.0
    k_area = P["area_factor"] * kBT / P["l0"] ** 2
    k_vol = P["vol_factor"] * kBT / P["l0"] ** 3
    k0 = P["bend_factor"] * kBT
    a_m = h / P["morse_width"]                 # Morse a in 1/lattice length
    k_lat = k_spring / (F_u / h)
    return dict(
        dt=dt, F_u=F_u, E_u=E_u, h=h,
        membrane=dict(
            k_spring=k_lat,
            k_s=k_area / (E_u / h ** 2),
            k_t=k_area / (E_u / h ** 2),
            k_v=k_vol / (E_u / h ** 3),
            k_b=(2.0 * k0 / math.sqrt(3.0)) / E_u,
            k0=k0 / E_u,            # Eq. 6 modulus, for the finite-element bending
            bending="dihedral",     # or "fem": Eq. 6-10 on quadratic six-node elements
            morse_D=k_lat / (2.0 * a_m * a_m),  # reading: 2 D a^2 = k
            morse_a=a_m,
            rep_F0=P["rep_F0"] / E_u,
            rep_tau=P["rep_tau"] * h,
            rep_eps_min=P["rep_eps_min"] / h,
            z_wall=-0.5,
        ),
        bonds=dict(
            sigma=P["sigma"] / (F_u / h),
            l_b=P["l_b"] / h,
            d_capture=P["d_capture"] / h,
            gamma=P["gamma"] / h,
            kT=kBT / E_u,
            kon0_dt=P["kon0"] * dt,
            koff0_dt=P["koff0"] * dt,
            z_wall=-0.5,
            max_per_ligand=4,
        ),
    )


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------
def icosphere(level: int):
    """Unit icosphere: 10*4^level + 2 vertices, outward counter-clockwise faces."""
    V, F, _ = icosphere_elements(level)
    return V, F


def icosphere_elements(level: int):
    """Unit icosphere with its quadratic six-node elements.

    Returns (V, F, E6).  For level >= 1 every triangle of the previous level
    is split into four by its edge midpoints; E6[e] = (a, b, c, m_ab, m_bc,
    m_ca) lists that parent triangle's corners (outward counter-clockwise)
    and its three midpoint nodes, which is the node set of a quadratic
    six-node triangle (corners at (xi, eta) = (0,0), (1,0), (0,1); midpoints
    at (1/2,0), (1/2,1/2), (0,1/2)).  Level 0 has no midpoint nodes and
    returns an empty E6."""
    if level not in _ICO:
        _ICO[level] = _icosphere(level)
    V, F, E6 = _ICO[level]
    return V.copy(), F.copy(), E6.copy()


_ICO = {}


def _icosphere(level: int):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    E6 = []
    for _ in range(level):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = V[i] + V[j]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        E6 = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
            E6.append((a, b, c, ab, bc, ca))
        F = nf
    X = np.array(V)
    T = np.array(F, dtype=np.int32)
    # orient outward
    n = np.cross(X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]])
    flip = np.einsum("ij,ij->i", n, X[T[:, 0]]) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    E = np.array(E6, dtype=np.int32).reshape(-1, 6)
    if len(E):
        n = np.cross(X[E[:, 1]] - X[E[:, 0]], X[E[:, 2]] - X[E[:, 0]])
        flip = np.einsum("ij,ij->i", n, X[E[:, 0]] + X[E[:, 1]] + X[E[:, 2]]) < 0
        # (a, c, b) with midpoints (m_ac, m_cb, m_ba)
        E[flip] = E[flip][:, [0, 2, 1, 5, 4, 3]]
    return X, T, E


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def sce_points(n, a, c, rng, shrink=0.8):
    """n points uniform inside the ellipsoid (a, a, c) scaled by ``shrink``."""
    if n == 0:
        return np.zeros((0, 3))
    out = []
    while len(out) < n:
        p = rng.uniform(-1.0, 1.0, size=(4 * n + 16, 3))
        p = p[np.einsum("ij,ij->i", p, p) <= 1.0]
        out.extend(p[: n - len(out)])
    P = np.array(out[:n]) * shrink
    P[:, 0] *= a
    P[:, 1] *= a
    P[:, 2] *= c
    return P


def morse_pairs(Xm, Xs, r_cut):
    """Index pairs (into [Xm; Xs]) of SCE-SCE and SCE-membrane points closer
    than r_cut in the rest shape, ordered by SCE point, then partner index."""
    from scipy.spatial import cKDTree

    nm = len(Xm)
    if len(Xs) == 0:
        return np.zeros((0, 2), dtype=np.int32)
    allX = np.vstack([Xm, Xs])
    near = cKDTree(allX).query_ball_point(Xs, r_cut, return_sorted=True)
    pairs = []
    for s, idx in enumerate(near):
        for j in idx:
            if j < nm or j > nm + s:  # membrane partner, or a later SCE
                pairs.append((nm + s, j) if j > nm + s else (j, nm + s))
    return np.array(pairs, dtype=np.int32).reshape(-1, 2)


def receptor_sites(X, T, n_sites, rng):
    """Area-uniform points: (triangle id, w0, w1) with weights (w0, w1, 1-w0-w1)."""
    if n_sites == 0:
        return np.zeros(0, dtype=np.int32), np.zeros((0, 2))
    area = 0.5 * np.linalg.norm(np.cross(X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]]), axis=1)
    tri = rng.choice(len(T), size=n_sites, p=area / area.sum()).astype(np.int32)
    r = rng.uniform(size=(n_sites, 2))
    over = r.sum(axis=1) > 1.0
    r[over] = 1.0 - r[over]
    w = np.stack([1.0 - r[:, 0] - r[:, 1], r[:, 0]], axis=1)
    return tri, w


def platelet_template(level, n_sce, n_sites, a_lat, aspect, rng):
    """One platelet in its body frame: membrane nodes, SCE points, triangles,
    Morse pairs and receptor sites."""
    U, T, E6 = icosphere_elements(level)
    Xm = U * np.array([a_lat, a_lat, a_lat * aspect])
    Xs = sce_points(n_sce, a_lat, a_lat * aspect, rng)
    edges = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    mean_edge = np.linalg.norm(Xm[edges[:, 0]] - Xm[edges[:, 1]], axis=1).mean()
    pairs = morse_pairs(Xm, Xs, 2.0 * mean_edge)
    st, sw = receptor_sites(Xm, T, n_sites, rng)
    return dict(Xm=Xm, Xs=Xs, T=T, E6=E6, pairs=pairs, site_tri=st, site_w=sw, mean_edge=mean_edge)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def bridge_params(bonds):
    """Platelet-platelet bridge parameters from the wall-bond ones (lattice
    units).  Reading of "treated similarly": a bridge is two GPIb-alpha - vWF
    links in series, so its rest length and capture distance are twice the
    single link's and its spring constant half; the kinetic constants of
    Eq. 12-13 are the single link's."""
    return dict(sigma=0.5 * bonds["sigma"], l_b=2.0 * bonds["l_b"], d_capture=2.0 * bonds["d_capture"],
                gamma=bonds["gamma"], kT=bonds["kT"], kon0_dt=bonds["kon0_dt"], koff0_dt=bonds["koff0_dt"],
                box_nx=bonds["box_nx"], box_ny=bonds["box_ny"], seed=bonds["seed"])


def build(nx, ny, nz, tau, shear, n_plt, level, n_sce, n_sites, seed,
          patch=None, gap=0.5, z_max=None, orient="random", stiffness=1.0,
          phys=None, centers=None, bridges=False):
    """A channel workload in lattice units.

    shear: wall shear rate in 1/s (top wall moves at shear * nz * dt).
    patch: (i0, j0, ni, nj) ligand patch; default a centred patch of half the
           wall length in x and y.
    gap: lowest membrane point at least this far (lattice units) above the wall.
    z_max: highest centroid height above the wall (lattice units); default 3 um.
    orient: "flat" (axis along z) or "random".
    """
    rng = np.random.default_rng(seed)
    L = lattice_units(tau, phys)
    P = dict(PHYSICAL if phys is None else phys)
    a_lat = P["a"] / P["h"]
    aspect = P["aspect"]
    if z_max is None:
        z_max = 3.0e-6 / P["h"]
    z_wall = -0.5
    Xs_all, tris, pairs, node_plt, is_mem, site_tri, site_w, elems = [], [], [], [], [], [], [], []
    placed = []
    off = 0
    toff = 0
    for p in range(n_plt):
        tp = platelet_template(level, n_sce, n_sites, a_lat, aspect, rng)
        body = np.vstack([tp["Xm"], tp["Xs"]])
        for _attempt in range(100000):
            R = np.eye(3) if orient == "flat" else random_rotation(rng)
            Y = body @ R.T
            if centers is not None:
                c = np.array(centers[p], dtype=np.float64)
            else:
                lo = z_wall + gap - Y[:, 2].min()
                c = np.array([rng.uniform(0, nx), rng.uniform(0, ny),
                              rng.uniform(lo, max(lo, z_wall + z_max))])
            if Y[:, 2].min() + c[2] < z_wall + gap - 1e-12:
                if centers is not None:
                    raise ValueError("platelet %d would touch the wall" % p)
                continue
            ok = True
            for q in placed:  # non-overlap of bounding spheres, periodic in x, y
                d = c - q
                d[0] -= nx * round(d[0] / nx)
                d[1] -= ny * round(d[1] / ny)
                if np.linalg.norm(d) < 2.0 * a_lat + 1.0:
                    ok = False
                    break
            if ok or centers is not None:
                break
        else:
            raise RuntimeError("could not place platelet %d" % p)
        placed.append(c)
        Xs_all.append(Y + c)
        nm = len(tp["Xm"])
        tris.append(tp["T"] + off)
        elems.append(tp["E6"] + off)
        pairs.append(tp["pairs"] + off)
        node_plt.append(np.full(len(body), p, dtype=np.int32))
        is_mem.append(np.r_[np.ones(nm, np.uint8), np.zeros(len(tp["Xs"]), np.uint8)])
        site_tri.append(tp["site_tri"] + toff)
        site_w.append(tp["site_w"])
        off += len(body)
        toff += len(tp["T"])
    X = np.vstack(Xs_all)                      # (M, 3)
    M = len(X)
    if patch is None:
        patch = (nx // 4, ny // 4, nx // 2, ny // 2)
    mem = dict(L["membrane"])
    mem["k_spring"] *= stiffness
    mem["morse_D"] *= stiffness
    bonds = dict(L["bonds"])
    bonds.update(lig_i0=patch[0], lig_j0=patch[1], lig_ni=patch[2], lig_nj=patch[3],
                 box_nx=nx, box_ny=ny, seed=seed)
    Xsoa = np.ascontiguousarray(X.T).ravel()   # [3][M]
    st = np.concatenate(site_tri).astype(np.int32)
    w = dict(
        grid=dict(nx=nx, ny=ny, nz=nz, tau=tau, u_top=(shear * L["dt"] * nz, 0.0, 0.0),
                  body=(0.0, 0.0, 0.0)),
        dt=L["dt"], shear=shear,
        mesh=dict(X0=Xsoa.copy(), tri=np.concatenate(tris).astype(np.int32),
                  elem6=np.concatenate(elems).astype(np.int32).reshape(-1, 6),
                  pairs=np.concatenate(pairs).astype(np.int32).reshape(-1, 2),
                  node_plt=np.concatenate(node_plt), is_membrane=np.concatenate(is_mem),
                  n_plt=n_plt),
        membrane=mem, bonds=bonds,
        sites=dict(tri=st, w=np.concatenate(site_w).reshape(-1, 2)),
        X=Xsoa, M=M,
        bound=np.full(len(st), -1, dtype=np.int32),
        lig_count=np.zeros(patch[2] * patch[3], dtype=np.int32),
    )
    if bridges:
        w["bridges"] = bridge_params(bonds)
        w["partner"] = np.full(len(st), -1, dtype=np.int32)
    return w


def config_small(seed=0):
    """D3Q19 Couette shear channel 32x32x64, tau = 0.8, wall shear 100/s,
    bottom-wall ligand patch 16x16 at 1 ligand/node; one discoid platelet
    (642-node icosphere-derived mesh, 200 SCE elements, 100 receptor sites),
    lying flat just above the patch."""
    return build(32, 32, 64, 0.8, 100.0, 1, 3, 200, 100, seed, patch=(8, 8, 16, 16),
                 orient="flat", centers=[(16.0, 16.0, -0.5 + 0.5 + 1.25)])


def config_channel(seed=0):
    """128x64x64 channel, shear 1000/s, 10 platelets of 2562 membrane nodes
    and 800 SCE elements each, random orientation, non-overlapping, centroids
    within 3 um of the wall, 5000 receptor sites each."""
    return build(128, 64, 64, 0.8, 1000.0, 10, 4, 800, 5000, seed)


def tiny(seed=0, nx=24, ny=20, nz=18, level=1, n_sce=8, n_sites=40, n_plt=1, shear=500.0,
         tau=0.8, orient="flat", gap=0.3, centers=None):
    """Small case for quick parity checks (several tiles and ragged edges)."""
    if centers is None and n_plt == 1:
        centers = [(nx / 2.0 + 0.37, ny / 2.0 - 0.21, -0.5 + gap + 1.25 + 0.05)]
    return build(nx, ny, nz, tau, shear, n_plt, level, n_sce, n_sites, seed,
                 patch=(nx // 4, ny // 4, nx // 2, ny // 2), orient=orient, gap=gap,
                 centers=centers)


def config_pair(seed=0, gap=0.4, nx=64, ny=48, nz=40, shear=1000.0, level=4, n_sce=800, n_sites=5000):
    """Two interacting platelets near the wall (the platelet-platelet
    adhesion study, Section 4.3.3): discoid platelets lying flat, the lower
    one `gap` above the wall over the ligand patch, the upper one stacked on
    it `gap` higher and shifted by a quarter radius in x; receptor sites on
    both, wall bonds and platelet-platelet bridges."""
    a = PHYSICAL["a"] / PHYSICAL["h"]
    c = a * PHYSICAL["aspect"]
    z0 = -0.5 + gap + c
    centers = [(nx / 2.0 + 0.37, ny / 2.0 - 0.21, z0), (nx / 2.0 + 0.37 + 0.25 * a, ny / 2.0 - 0.21, z0 + 2 * c + gap)]
    return build(nx, ny, nz, 0.8, shear, 2, level, n_sce, n_sites, seed, orient="flat", gap=gap,
                 centers=centers, bridges=True)


def config_batched(seed=0, n_chambers=64):
    """Independent chambers of uneven sizes: each (nx, ny, nz) drawn from
    48..128, wall shear from 500..3000/s, receptor count from 2000..25000,
    membrane stiffness (spring constant and Morse depth) scaled by a factor
    from 0.5..2; one platelet of 2562 membrane nodes and 800 SCE elements per
    chamber, ligand patch centred on the bottom wall.  Returns the list of
    chamber workloads."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_chambers):
        nx, ny, nz = (int(v) for v in rng.integers(48, 129, size=3))
        shear = float(rng.uniform(500.0, 3000.0))
        sites = int(rng.integers(2000, 25001))
        stiff = float(rng.uniform(0.5, 2.0))
        out.append(build(nx, ny, nz, 0.8, shear, 1, 4, 800, sites, 1000 * seed + c, stiffness=stiff))
    return out


def config_surrogate(seed=0):
    """Learned-surrogate workload: 256x128x128 channel at wall shear 1500/s,
    100 platelets of 2562 membrane nodes (no SCE, no receptors), random
    orientation, centroids within 3 um of the wall."""
    return build(256, 128, 128, 0.8, 1500.0, 100, 4, 0, 0, seed)


def config_full(seed=0, n_plt=500):
    """Full scale: 512x256x256 channel (33.5 M cells) at wall shear 3000/s,
    500 platelets of 2562 membrane nodes and 800 SCE elements with 5000
    receptor sites each, ligands on every node of the bottom wall (the
    configuration names no patch; with the whole wall adhesive, the sites
    that start within the capture distance can bind)."""
    return build(512, 256, 256, 0.8, 3000.0, n_plt, 4, 800, 5000, seed, patch=(0, 0, 512, 256))


def config_full_sample(seed=0, nx=32):
    """A bounded sample of the full-scale workload for host timings: the same
    256 x 256 cross section, shear and platelet kind, nx cells long instead of
    512 (periodic in x), with the same number of platelets per cell
    (500 nx / 512, rounded) and ligands on the whole bottom wall."""
    n_plt = max(1, int(round(500 * nx / 512)))
    return build(nx, 256, 256, 0.8, 3000.0, n_plt, 4, 800, 5000, seed, patch=(0, 0, nx, 256))
