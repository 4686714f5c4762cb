"""FP64 CPU oracle of the platelet fluid-structure step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
restatement in ``oracle.c`` (double precision, plain loops) with ctypes and
numpy and strings the pieces together in the per-step order of the paper's
flow chart (Fig. 1; Section 3, the coupling paragraph of 3.4.2):

  1. membrane forces (Section 3.1, Eq. 2-11) + wall repulsion (3.4.1) + bond
     forces (Eq. 14),
  2. immersed-boundary spreading (Eq. 34-36),
  3. lattice Boltzmann step (Eq. 16-21),
  4. immersed-boundary interpolation (Eq. 33) and X += U dt (Eq. 31),
  5. Monte-Carlo adhesion update: rupture, then formation (Section 3.2).

It shares no code with the CUDA library: nothing here imports it and it
imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

DP = ctypes.POINTER(ctypes.c_double)
IP = ctypes.POINTER(ctypes.c_int)
UP = ctypes.POINTER(ctypes.c_uint32)
BP = ctypes.POINTER(ctypes.c_ubyte)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, IEEE arithmetic)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
             "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class LBParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("u_top", ctypes.c_double * 3),
                ("body", ctypes.c_double * 3), ("walls", ctypes.c_int)]


class MemParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "k_spring", "k_s", "k_t", "k_v", "k_b", "morse_D", "morse_a",
        "rep_F0", "rep_tau", "rep_eps_min", "z_wall")]


class BondParams(ctypes.Structure):
    _fields_ = [("lig_i0", ctypes.c_int), ("lig_j0", ctypes.c_int),
                ("lig_ni", ctypes.c_int), ("lig_nj", ctypes.c_int),
                ("box_nx", ctypes.c_int), ("box_ny", ctypes.c_int),
                ("max_per_ligand", ctypes.c_int),
                ("z_wall", ctypes.c_double), ("sigma", ctypes.c_double),
                ("l_b", ctypes.c_double), ("d_capture", ctypes.c_double),
                ("gamma", ctypes.c_double), ("kT", ctypes.c_double),
                ("kon0_dt", ctypes.c_double), ("koff0_dt", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class BridgeParams(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("l_b", ctypes.c_double), ("d_capture", ctypes.c_double),
                ("gamma", ctypes.c_double), ("kT", ctypes.c_double),
                ("kon0_dt", ctypes.c_double), ("koff0_dt", ctypes.c_double),
                ("box_nx", ctypes.c_int), ("box_ny", ctypes.c_int), ("seed", ctypes.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.ora_set_threads.argtypes = [ctypes.c_int]
        L.ora_get_threads.restype = ctypes.c_int
        L.ora_philox4x32_10.argtypes = [UP, UP, UP]
        L.ora_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
        L.ora_uniform.restype = ctypes.c_double
        L.ora_lb_lattice.argtypes = [IP, DP]
        L.ora_lb_init_shear.argtypes = [ctypes.POINTER(LBParams), DP]
        L.ora_lb_step.argtypes = [ctypes.POINTER(LBParams), DP, DP, DP, DP, DP]
        L.ora_phi.argtypes = [ctypes.c_double]
        L.ora_phi.restype = ctypes.c_double
        L.ora_ib_spread.argtypes = [ctypes.POINTER(LBParams), ctypes.c_int, DP, DP, DP]
        L.ora_ib_interp.argtypes = [ctypes.POINTER(LBParams), ctypes.c_int, DP, DP, DP]
        L.ora_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, IP, ctypes.c_int, IP,
                                      ctypes.c_int, IP, BP, DP]
        L.ora_mesh_create.restype = ctypes.c_void_p
        L.ora_mesh_destroy.argtypes = [ctypes.c_void_p]
        L.ora_mesh_n_edges.argtypes = [ctypes.c_void_p]
        L.ora_mesh_measure.argtypes = [ctypes.c_void_p, DP, DP, DP]
        L.ora_mesh_energy.argtypes = [ctypes.c_void_p, ctypes.POINTER(MemParams), DP, DP]
        L.ora_mesh_forces.argtypes = [ctypes.c_void_p, ctypes.POINTER(MemParams), DP, DP]
        L.ora_bond_forces.argtypes = [ctypes.POINTER(BondParams), ctypes.c_int, IP, DP, IP,
                                      ctypes.c_int, IP, DP, DP]
        L.ora_bonds_step.argtypes = [ctypes.POINTER(BondParams), ctypes.c_int, IP, DP, IP,
                                     ctypes.c_int, DP, IP, IP, ctypes.c_uint64, IP, IP]
        L.ora_pair_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint32]
        L.ora_pair_uniform.restype = ctypes.c_double
        L.ora_bridge_forces.argtypes = [ctypes.POINTER(BridgeParams), ctypes.c_int, IP, DP, IP, ctypes.c_int, IP,
                                        DP, DP]
        L.ora_bridges_step.argtypes = [ctypes.POINTER(BridgeParams), ctypes.c_int, IP, DP, IP, IP, ctypes.c_int,
                                       DP, IP, IP, ctypes.c_uint64, IP]
        _lib = L
    return _lib


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(DP)


def _i(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(IP)


# ---------------------------------------------------------------- Philox
def set_threads(n):
    """Host threads of the oracle's parallel loops (lattice step, initial
    state, interpolation); results do not depend on the count."""
    lib().ora_set_threads(int(n))


def get_threads():
    return int(lib().ora_get_threads())


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(seed, site, step, purpose):
    return lib().ora_uniform(seed, site, step, purpose)


# ---------------------------------------------------------------- LB
def lattice():
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    lib().ora_lb_lattice(_i(c), _d(w))
    return c.reshape(19, 3), w


def lb_params(nx, ny, nz, tau, u_top=(0.0, 0.0, 0.0), body=(0.0, 0.0, 0.0), walls=0):
    return LBParams(nx, ny, nz, tau, (ctypes.c_double * 3)(*u_top), (ctypes.c_double * 3)(*body), int(walls))


def lb_init_shear(p):
    f = np.zeros(19 * p.nx * p.ny * p.nz)
    lib().ora_lb_init_shear(ctypes.byref(p), _d(f))
    return f


def lb_step(p, f_in, g=None):
    N = p.nx * p.ny * p.nz
    f_out = np.empty_like(f_in)
    rho = np.empty(N)
    v = np.empty(3 * N)
    lib().ora_lb_step(ctypes.byref(p), _d(f_in), _d(g) if g is not None else None,
                      _d(f_out), _d(rho), _d(v))
    return f_out, rho, v


# ---------------------------------------------------------------- IB
def phi(r):
    return lib().ora_phi(float(r))


def ib_spread(p, X, F, g=None):
    N = p.nx * p.ny * p.nz
    M = X.size // 3
    if g is None:
        g = np.zeros(3 * N)
    lib().ora_ib_spread(ctypes.byref(p), M, _d(X), _d(F), _d(g))
    return g


def ib_interp(p, X, v):
    M = X.size // 3
    U = np.empty(3 * M)
    lib().ora_ib_interp(ctypes.byref(p), M, _d(X), _d(v), _d(U))
    return U


# ---------------------------------------------------------------- membrane
def mem_params(d):
    return MemParams(*[float(d[n]) for n, _ in MemParams._fields_])


class Mesh:
    """Membrane topology plus its rest state, derived from the rest shape X0."""

    def __init__(self, X0, tri, pairs, node_plt, is_membrane, n_plt):
        self.n = X0.size // 3
        self._tri = np.ascontiguousarray(tri, dtype=np.int32).ravel()
        self._pairs = np.ascontiguousarray(pairs, dtype=np.int32).ravel()
        self._plt = np.ascontiguousarray(node_plt, dtype=np.int32)
        self._mem = np.ascontiguousarray(is_membrane, dtype=np.uint8)
        self.n_plt = int(n_plt)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        self.h = lib().ora_mesh_create(
            self.n, self._tri.size // 3, _i(self._tri), self._pairs.size // 2, _i(self._pairs),
            self.n_plt, _i(self._plt), self._mem.ctypes.data_as(BP), _d(X0))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_mesh_destroy(self.h)
            self.h = None

    @property
    def n_edges(self):
        return lib().ora_mesh_n_edges(self.h)

    def measure(self, X):
        S = np.zeros(self.n_plt)
        V = np.zeros(self.n_plt)
        lib().ora_mesh_measure(self.h, _d(np.ascontiguousarray(X, dtype=np.float64)), _d(S), _d(V))
        return S, V

    def energy_terms(self, params, X):
        t = np.zeros(7)
        mp = mem_params(params)
        lib().ora_mesh_energy(self.h, ctypes.byref(mp), _d(np.ascontiguousarray(X, dtype=np.float64)), _d(t))
        return t

    def forces(self, params, X):
        F = np.zeros(3 * self.n)
        mp = mem_params(params)
        lib().ora_mesh_forces(self.h, ctypes.byref(mp), _d(np.ascontiguousarray(X, dtype=np.float64)), _d(F))
        return F


# ---------------------------------------------------------------- bonds
def bond_params(d):
    return BondParams(int(d["lig_i0"]), int(d["lig_j0"]), int(d["lig_ni"]), int(d["lig_nj"]),
                      int(d["box_nx"]), int(d["box_ny"]), int(d["max_per_ligand"]),
                      float(d["z_wall"]), float(d["sigma"]), float(d["l_b"]),
                      float(d["d_capture"]), float(d["gamma"]), float(d["kT"]),
                      float(d["kon0_dt"]), float(d["koff0_dt"]), int(d["seed"]))


def bond_forces(params, site_tri, site_w, tri, bound, X, F):
    bp = bond_params(params)
    M = X.size // 3
    lib().ora_bond_forces(ctypes.byref(bp), site_tri.size, _i(site_tri), _d(site_w),
                          _i(np.ascontiguousarray(tri, dtype=np.int32).ravel()), M, _i(bound), _d(X), _d(F))
    return F


def bonds_step(params, site_tri, site_w, tri, X, bound, lig_count, step, partner=None):
    """Updates bound / lig_count in place; returns (n_ruptures, n_formations).
    partner: bridge partners (sites with one hold no wall bond), or None."""
    bp = bond_params(params)
    M = X.size // 3
    ev = np.zeros(2, dtype=np.int32)
    lib().ora_bonds_step(ctypes.byref(bp), site_tri.size, _i(site_tri), _d(site_w),
                         _i(np.ascontiguousarray(tri, dtype=np.int32).ravel()), M, _d(X),
                         _i(bound), _i(lig_count), int(step), _i(partner) if partner is not None else None, _i(ev))
    return int(ev[0]), int(ev[1])


# ---------------------------------------------------------------- bridges
def bridge_params(d):
    return BridgeParams(float(d["sigma"]), float(d["l_b"]), float(d["d_capture"]), float(d["gamma"]),
                        float(d["kT"]), float(d["kon0_dt"]), float(d["koff0_dt"]), int(d["box_nx"]),
                        int(d["box_ny"]), int(d["seed"]))


def pair_uniform(seed, i, j, step, purpose):
    return lib().ora_pair_uniform(seed, i, j, step, purpose)


def site_platelets(site_tri, tri, node_plt):
    """Platelet of each receptor site (that of its triangle's first node)."""
    t = np.asarray(tri, dtype=np.int32).reshape(-1, 3)
    return np.ascontiguousarray(np.asarray(node_plt, dtype=np.int32)[t[np.asarray(site_tri), 0]])


def bridge_forces(params, site_tri, site_w, tri, partner, X, F):
    bp = bridge_params(params)
    M = X.size // 3
    lib().ora_bridge_forces(ctypes.byref(bp), site_tri.size, _i(site_tri), _d(site_w),
                            _i(np.ascontiguousarray(tri, dtype=np.int32).ravel()), M, _i(partner), _d(X), _d(F))
    return F


def bridges_step(params, site_tri, site_w, tri, site_plt, X, bound, partner, step):
    """Updates partner in place; returns (n_ruptures, n_formations)."""
    bp = bridge_params(params)
    M = X.size // 3
    ev = np.zeros(2, dtype=np.int32)
    lib().ora_bridges_step(ctypes.byref(bp), site_tri.size, _i(site_tri), _d(site_w),
                           _i(np.ascontiguousarray(tri, dtype=np.int32).ravel()), _i(site_plt), M, _d(X),
                           _i(bound), _i(partner), int(step), _i(ev))
    return int(ev[0]), int(ev[1])


# ---------------------------------------------------------------- coupled step
class Sim:
    """The coupled per-step loop of the paper (Fig. 1), FP64 throughout.

    ``w`` is a workload dictionary (lattice-unit parameters, the rest mesh,
    receptor sites, initial positions and bond state).
    """

    def __init__(self, w):
        g = w["grid"]
        self.p = lb_params(g["nx"], g["ny"], g["nz"], g["tau"], g["u_top"], g.get("body", (0, 0, 0)),
                           g.get("walls", 0))
        self.N = g["nx"] * g["ny"] * g["nz"]
        m = w["mesh"]
        self.mesh = Mesh(m["X0"], m["tri"], m["pairs"], m["node_plt"], m["is_membrane"], m["n_plt"])
        self.tri = np.ascontiguousarray(m["tri"], dtype=np.int32).ravel()
        self.memp = w["membrane"]
        # finite-element bending (Eq. 6-10) in place of the dihedral term
        self.fem = self.memp.get("bending", "dihedral") == "fem"
        if self.fem:
            self.memp = dict(self.memp, k_b=0.0)
            self.elem6 = np.asarray(m["elem6"], dtype=np.int64).reshape(-1, 6)
            self.k0 = float(w["membrane"]["k0"])
        self.bondp = w["bonds"]
        self.site_tri = np.ascontiguousarray(w["sites"]["tri"], dtype=np.int32)
        self.site_w = np.ascontiguousarray(w["sites"]["w"], dtype=np.float64).ravel()
        self.X = np.ascontiguousarray(w["X"], dtype=np.float64).ravel().copy()
        self.bound = np.ascontiguousarray(w["bound"], dtype=np.int32).copy()
        # platelet-platelet bridges (optional)
        self.bridgep = w.get("bridges")
        self.partner = None
        if self.bridgep is not None:
            self.site_plt = site_platelets(self.site_tri, m["tri"], m["node_plt"])
            self.partner = np.ascontiguousarray(w.get("partner", np.full(len(self.site_tri), -1)), dtype=np.int32).copy()
        self.bridge_events = (0, 0)
        self.lig_count = np.ascontiguousarray(w["lig_count"], dtype=np.int32).copy()
        self.f = lb_init_shear(self.p)
        self.step_index = int(w.get("step0", 0))
        self.M = self.X.size // 3
        self.F = np.zeros(3 * self.M)
        self.U = np.zeros(3 * self.M)
        self.g = np.zeros(3 * self.N)
        self.rho = None
        self.v = None
        self.events = (0, 0)

    def step(self):
        # 1. forces on the Lagrangian nodes
        self.F = self.mesh.forces(self.memp, self.X)
        if self.fem:
            from . import fem
            self.F += fem.forces_soa(self.X, self.elem6, self.k0)
        bond_forces(self.bondp, self.site_tri, self.site_w, self.tri, self.bound, self.X, self.F)
        if self.partner is not None:
            bridge_forces(self.bridgep, self.site_tri, self.site_w, self.tri, self.partner, self.X, self.F)
        # 2. spread
        self.g = ib_spread(self.p, self.X, self.F)
        # 3. fluid
        self.f, self.rho, self.v = lb_step(self.p, self.f, self.g)
        # 4. interpolate and move
        self.U = ib_interp(self.p, self.X, self.v)
        self.X += self.U
        # 5. adhesion
        self.events = bonds_step(self.bondp, self.site_tri, self.site_w, self.tri, self.X,
                                 self.bound, self.lig_count, self.step_index, self.partner)
        if self.partner is not None:
            self.bridge_events = bridges_step(self.bridgep, self.site_tri, self.site_w, self.tri, self.site_plt,
                                              self.X, self.bound, self.partner, self.step_index)
        self.step_index += 1
