"""Thin ctypes binding of the C ABI in include/platelet_fsi.h.

Functions keep the C names and only marshal arguments: torch tensors become
device pointers, the current torch CUDA stream becomes the cudaStream_t.
Every computation runs in libplatelet_fsi.so; if the library has not been
built, or a call fails, a RuntimeError is raised (there is no fallback).

The classes at the end (:class:`Lattice`, :class:`Membrane`, :class:`Bonds`,
:class:`Simulation`) allocate the caller-owned device buffers with torch and
hold the handles.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libplatelet_fsi.so")
_lib = None

c_int, c_double, c_float, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_size_t, ctypes.c_void_p
c_uint64, c_longlong = ctypes.c_uint64, ctypes.c_longlong


LB_FP32, LB_BF16, LB_FP16 = 0, 1, 2
STORAGE = {"fp32": LB_FP32, "bf16": LB_BF16, "fp16": LB_FP16}


class lb_params(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("tau", c_float),
                ("u_top", c_float * 3), ("body", c_float * 3), ("storage", c_int), ("fp16_exponent", c_int),
                ("walls", c_int)]


class lb_sizes(ctypes.Structure):
    _fields_ = [("f_bytes", c_size_t), ("g_bytes", c_size_t), ("v_bytes", c_size_t),
                ("flag_bytes", c_size_t), ("n_cells", c_longlong)]


class mem_params(ctypes.Structure):
    _fields_ = [(n, c_float) for n in ("k_spring", "k_s", "k_t", "k_v", "k_b", "morse_D", "morse_a",
                                        "rep_F0", "rep_tau", "rep_eps_min", "z_wall")]


class bond_params(ctypes.Structure):
    _fields_ = [("lig_i0", c_int), ("lig_j0", c_int), ("lig_ni", c_int), ("lig_nj", c_int),
                ("box_nx", c_int), ("box_ny", c_int), ("max_per_ligand", c_int),
                ("z_wall", c_double), ("sigma", c_double), ("l_b", c_double), ("d_capture", c_double),
                ("gamma", c_double), ("kT", c_double), ("kon0_dt", c_double), ("koff0_dt", c_double),
                ("seed", c_uint64)]


class bridge_params(ctypes.Structure):
    _fields_ = [("sigma", c_double), ("l_b", c_double), ("d_capture", c_double), ("gamma", c_double),
                ("kT", c_double), ("kon0_dt", c_double), ("koff0_dt", c_double), ("box_nx", c_int),
                ("box_ny", c_int), ("seed", c_uint64)]


P = c_void_p
_SIGS = {
    "pfsi_last_error": [ctypes.c_char_p, c_size_t],
    "pfsi_version": [],
    "lb_query_sizes": [ctypes.POINTER(lb_params), ctypes.POINTER(lb_sizes)],
    "lb_create": [ctypes.POINTER(lb_params), P, P, P, P, P, ctypes.POINTER(P)],
    "lb_create_mixed": [ctypes.POINTER(lb_params), P, P, P, P, P, P, ctypes.POINTER(P)],
    "lb_export": [P, P, P],
    "lb_velocity": [P, ctypes.POINTER(P)],
    "lb_destroy": [P],
    "lb_init_shear": [P, P],
    "lb_step": [P, c_int, P],
    "lb_current": [P, ctypes.POINTER(P)],
    "lb_moments_fp64": [P, P, ctypes.POINTER(c_double), P],
    "lb_check": [P, c_float, P, ctypes.POINTER(c_longlong), P],
    "sim_check": [P, c_float, P, ctypes.POINTER(c_longlong), P],
    "ib_spread": [P, P, P, c_int, P],
    "ib_interp": [P, P, P, c_int, c_int, P],
    "membrane_query_workspace": [c_int, c_int, P, c_int, c_int, ctypes.POINTER(c_size_t)],
    "membrane_create": [ctypes.POINTER(mem_params), c_int, c_int, P, c_int, P, c_int, P, P, P, P,
                        c_size_t, ctypes.POINTER(P)],
    "membrane_destroy": [P],
    "membrane_set_params": [P, ctypes.POINTER(mem_params)],
    "membrane_forces": [P, P, P, P],
    "membrane_set_path": [P, c_int],
    "membrane_get_path": [P, ctypes.POINTER(c_int)],
    "membrane_measure": [P, P, ctypes.POINTER(c_double), P],
    "membrane_measure_static": [P, P, ctypes.POINTER(c_double), P],
    "membrane_centroids": [P, P, P, P],
    "bonds_query_workspace": [ctypes.POINTER(bond_params), c_int, ctypes.POINTER(c_size_t)],
    "bonds_create": [ctypes.POINTER(bond_params), c_int, P, P, P, P, P, P, c_size_t, ctypes.POINTER(P)],
    "bonds_destroy": [P],
    "bonds_forces": [P, P, P, c_int, P],
    "bonds_step": [P, P, c_int, c_uint64, P],
    "tether_query_workspace": [c_int, c_int, ctypes.POINTER(c_size_t)],
    "tether_create": [P, c_int, P, P, c_size_t, P, P, c_int, P, ctypes.POINTER(P)],
    "tether_destroy": [P],
    "tether_update": [P, c_uint64, P],
    "sim_set_tether": [P, P],
    "bonds_status": [P, ctypes.POINTER(c_longlong)],
    "sim_create": [P, P, P, P, P, P, c_int, c_uint64, ctypes.POINTER(P)],
    "sim_destroy": [P],
    "sim_step": [P, c_int, P],
    "sim_step_index": [P, ctypes.POINTER(c_uint64)],
    "sim_time_lb": [P, c_int],
    "sim_set_surrogate": [P, P, P],
    "bridges_query_workspace": [ctypes.POINTER(bridge_params), c_int, c_int, c_int, ctypes.POINTER(c_size_t)],
    "bridges_create": [ctypes.POINTER(bridge_params), P, c_int, P, c_int, P, P, c_size_t, ctypes.POINTER(P)],
    "bridges_destroy": [P],
    "bridges_forces": [P, P, P, c_int, P],
    "bridges_step": [P, P, c_int, c_uint64, P],
    "bridges_status": [P, ctypes.POINTER(c_longlong)],
    "bridges_partner": [P, ctypes.POINTER(P)],
    "sim_set_bridges": [P, P],
    "pfsi_wait_selftest": [c_int, P, P],
    "fem_query_workspace": [c_int, c_int, ctypes.POINTER(c_size_t)],
    "fem_create": [c_int, c_int, P, P, c_size_t, ctypes.POINTER(P)],
    "fem_destroy": [P],
    "fem_bending_forces": [P, c_float, P, P, c_int, P],
    "fem_fields": [P, P, P, P],
    "sim_set_fem_bending": [P, P, c_float],
    "sim_step_record": [P, c_int, P, P, c_int, P],
    "sim_step_track": [P, c_int, P, P, P],
    "lb_set_shape": [P, c_int],
    "lb_get_shape": [P, ctypes.POINTER(c_int)],
    "lb_autotune": [P, c_int, P, ctypes.POINTER(ctypes.c_float)],
    "batch_create": [P, c_int, c_int, ctypes.POINTER(P)],
    "batch_destroy": [P],
    "batch_step": [P, c_int, P],
    "batch_autotune": [P, c_int, P, ctypes.POINTER(ctypes.c_float)],
    "batch_set_layout": [P, c_int, c_int],
    "lb_batch_set_grid": [P, c_int],
    "lb_batch_create": [P, c_int, ctypes.POINTER(P)],
    "lb_batch_destroy": [P],
    "lb_batch_step": [P, c_int, P],
    "lb_batch_autotune": [P, c_int, P, ctypes.POINTER(ctypes.c_float)],
    "lb_batch_get_shapes": [P, ctypes.POINTER(c_int)],
    "lb_batch_set_shapes": [P, ctypes.POINTER(c_int)],
    "sg_params_bytes": [ctypes.POINTER(c_size_t)],
    "sg_sync_shadows": [P, P],
    "sg_query_work": [c_int, ctypes.POINTER(c_size_t)],
    "sg_grad": [P, P, P, c_int, c_int, P, P, P, c_size_t, P],
    "sg_work_status": [P, c_int, ctypes.POINTER(c_int)],
    "sg_adam": [P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, c_int, P],
    "sg_query_workspace": [c_int, ctypes.POINTER(c_size_t)],
    "sg_create": [c_int, c_int, P, P, P, c_int, P, c_size_t, ctypes.POINTER(P)],
    "sg_destroy": [P],
    "sg_rows": [P, ctypes.POINTER(c_int), ctypes.POINTER(P)],
    "sg_features": [P, P, P, P, P, P, P],
    "sg_membrane_forces": [P, P, P, P, P, P],
    "sg_targets": [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P, P, P],
    "sg_status": [P, ctypes.POINTER(c_int)],
    "sim_lb_ms": [P, ctypes.POINTER(ctypes.c_float)],
}


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libplatelet_fsi.so is not built: run `python -m paper_1312_2234_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = c_int
        _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().pfsi_last_error(buf, 1024)
    return buf.value.decode()


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed (%d): %s" % (what, rc, last_error()))


def _call(name, *args):
    _ok(getattr(lib(), name)(*args), name)


PFSI_ERR_UNSTABLE = -7
PFSI_ERR_TIMEOUT = -8


def wait_selftest(limit, stream=None):
    """Bounded device wait on an mbarrier phase nothing completes, with at
    most `limit` polls: True when it gave up (PFSI_ERR_TIMEOUT), False if the
    phase completed."""
    word = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib().pfsi_wait_selftest(int(limit), _ptr(word), _stream(stream))
    if rc not in (0, PFSI_ERR_TIMEOUT):
        _ok(rc, "pfsi_wait_selftest")
    return rc == PFSI_ERR_TIMEOUT


def _check(name, h, u_max, scratch, n, stream=None):
    """lb_check / sim_check: (counts, ok); a non-physical state is a result,
    not an exception."""
    out = (c_longlong * n)()
    rc = getattr(lib(), name)(h, float(u_max), _ptr(scratch), out, _stream(stream))
    if rc not in (0, PFSI_ERR_UNSTABLE):
        _ok(rc, name)
    return tuple(int(v) for v in out), rc == 0


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous()
        return c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return c_void_p(t.ctypes.data)
    return t


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- C-named calls
def lb_query_sizes(p):
    s = lb_sizes()
    _call("lb_query_sizes", ctypes.byref(p), ctypes.byref(s))
    return s


def lb_create(p, f_a, f_b, g, v, flags):
    h = c_void_p()
    _call("lb_create", ctypes.byref(p), _ptr(f_a), _ptr(f_b), _ptr(g), _ptr(v), _ptr(flags), ctypes.byref(h))
    return h


def lb_destroy(h):
    _call("lb_destroy", h)


def lb_create_mixed(p, n_a, n_b, m_a, m_b, g, flags):
    h = c_void_p()
    _call("lb_create_mixed", ctypes.byref(p), _ptr(n_a), _ptr(n_b), _ptr(m_a), _ptr(m_b), _ptr(g), _ptr(flags),
          ctypes.byref(h))
    return h


def lb_velocity(h):
    out = c_void_p()
    _call("lb_velocity", h, ctypes.byref(out))
    return out.value


def lb_export(h, f_out, stream=None):
    _call("lb_export", h, _ptr(f_out), _stream(stream))


def lb_init_shear(h, stream=None):
    _call("lb_init_shear", h, _stream(stream))


def lb_step(h, nsteps=1, stream=None):
    _call("lb_step", h, int(nsteps), _stream(stream))


def lb_current(h):
    out = c_void_p()
    _call("lb_current", h, ctypes.byref(out))
    return out.value


def lb_moments_fp64(h, scratch, stream=None):
    out = (c_double * 4)()
    _call("lb_moments_fp64", h, _ptr(scratch), out, _stream(stream))
    return np.array(out[:])


def ib_spread(h, X, F, M, stream=None):
    _call("ib_spread", h, _ptr(X), _ptr(F), int(M), _stream(stream))


def ib_interp(h, X, U, M, advect=True, stream=None):
    _call("ib_interp", h, _ptr(X), _ptr(U), int(M), int(bool(advect)), _stream(stream))


def membrane_query_workspace(n_nodes, tri, n_pairs, n_plt):
    b = c_size_t()
    tri = np.ascontiguousarray(tri, dtype=np.int32).ravel()
    _call("membrane_query_workspace", int(n_nodes), tri.size // 3, _ptr(tri), int(n_pairs), int(n_plt), ctypes.byref(b))
    return b.value


def membrane_create(p, n_nodes, tri, pairs, n_plt, node_plt, is_membrane, X0, ws):
    tri = np.ascontiguousarray(tri, dtype=np.int32).ravel()
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).ravel()
    node_plt = np.ascontiguousarray(node_plt, dtype=np.int32)
    is_mem = np.ascontiguousarray(is_membrane, dtype=np.uint8)
    X0 = np.ascontiguousarray(X0, dtype=np.float64).ravel()
    h = c_void_p()
    _call("membrane_create", ctypes.byref(p), int(n_nodes), tri.size // 3, _ptr(tri), pairs.size // 2, _ptr(pairs),
          int(n_plt), _ptr(node_plt), _ptr(is_mem), _ptr(X0), _ptr(ws), ws.numel() * ws.element_size(),
          ctypes.byref(h))
    return h


def membrane_destroy(h):
    _call("membrane_destroy", h)


def membrane_set_params(h, p):
    _call("membrane_set_params", h, ctypes.byref(p))


def membrane_forces(h, X, F, stream=None):
    _call("membrane_forces", h, _ptr(X), _ptr(F), _stream(stream))


def membrane_measure(h, X, n_plt, stream=None):
    out = (c_double * (2 * n_plt))()
    _call("membrane_measure", h, _ptr(X), out, _stream(stream))
    return np.array(out[:]).reshape(n_plt, 2)


def membrane_measure_static(h, X, n_plt, stream=None):
    """membrane_measure without the context's scratch (library-owned static
    device array; for callers that cannot allocate device memory)."""
    out = (c_double * (2 * n_plt))()
    _call("membrane_measure_static", h, _ptr(X), out, _stream(stream))
    return np.array(out[:]).reshape(n_plt, 2)


def bonds_query_workspace(p, n_sites):
    b = c_size_t()
    _call("bonds_query_workspace", ctypes.byref(p), int(n_sites), ctypes.byref(b))
    return b.value


def bonds_create(p, n_sites, site_tri, site_w, tri, bound, lig_count, ws):
    h = c_void_p()
    _call("bonds_create", ctypes.byref(p), int(n_sites), _ptr(site_tri), _ptr(site_w), _ptr(tri), _ptr(bound),
          _ptr(lig_count), _ptr(ws), ws.numel() * ws.element_size(), ctypes.byref(h))
    return h


def bonds_destroy(h):
    _call("bonds_destroy", h)


def bonds_forces(h, X, F, M, stream=None):
    _call("bonds_forces", h, _ptr(X), _ptr(F), int(M), _stream(stream))


def bonds_step(h, X, M, step, stream=None):
    _call("bonds_step", h, _ptr(X), int(M), int(step), _stream(stream))


def bonds_status(h):
    out = (c_longlong * 3)()
    rc = lib().bonds_status(h, out)
    return rc, [int(x) for x in out]


def sim_create(lb, mem, bonds, X, F, U, M, first_step=0):
    h = c_void_p()
    _call("sim_create", lb, mem, bonds, _ptr(X), _ptr(F), _ptr(U), int(M), int(first_step), ctypes.byref(h))
    return h


def sim_destroy(h):
    _call("sim_destroy", h)


def sim_step(h, nsteps=1, stream=None):
    _call("sim_step", h, int(nsteps), _stream(stream))


def sim_step_index(h):
    out = c_uint64()
    _call("sim_step_index", h, ctypes.byref(out))
    return out.value


def sim_time_lb(h, on=True):
    _call("sim_time_lb", h, int(bool(on)))


def sim_lb_ms(h):
    out = ctypes.c_float()
    _call("sim_lb_ms", h, ctypes.byref(out))
    return out.value


# ---------------------------------------------------------------- owners
def _bytes(n, device):
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    t = torch.empty(max(int(n), 1), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


def default_fp16_exponent(nz, tau, u_top):
    """Power-of-two scale for FP16 f^neq storage.  The first-order
    non-equilibrium part of a shear flow is about w tau |du/dz| (|du/dz| ~
    |u_top| / nz); 2^s of its inverse over 4 keeps it a normal FP16 number
    with ~2^14 of headroom for the steeper gradients near immersed bodies."""
    grad = max(math.hypot(u_top[0], u_top[1]) / nz, 1e-6)
    return int(max(-60, min(60, math.floor(math.log2(1.0 / (tau * grad))) - 2)))


class Lattice:
    """D3Q19 lattice with caller-owned (torch) buffers.  storage is "fp32"
    (shifted populations) or "bf16" / "fp16" (16-bit f^neq + FP32 moments)."""

    def __init__(self, nx, ny, nz, tau, u_top=(0.0, 0.0, 0.0), body=(0.0, 0.0, 0.0), device="cuda",
                 storage="fp32", fp16_exponent=None, walls=0):
        mode = STORAGE[storage]
        if fp16_exponent is None:
            fp16_exponent = default_fp16_exponent(nz, tau, u_top) if mode == LB_FP16 else 0
        self.storage = storage
        self.p = lb_params(nx, ny, nz, tau, (c_float * 3)(*u_top), (c_float * 3)(*body), mode, int(fp16_exponent),
                           int(walls))
        s = lb_query_sizes(self.p)
        self.N = int(s.n_cells)
        self.shape = (nz, ny, nx)
        self.g = torch.zeros(self.N, 4, dtype=torch.float32, device=device)
        self.flags = torch.zeros(ny * nz, dtype=torch.int32, device=device)
        self.scratch = torch.zeros(4, dtype=torch.float64, device=device)
        if mode == LB_FP32:
            self.f = [torch.empty(19, self.N, dtype=torch.float32, device=device) for _ in range(2)]
            self.v = torch.zeros(self.N, 4, dtype=torch.float32, device=device)
            self.h = lb_create(self.p, self.f[0], self.f[1], self.g, self.v, self.flags)
        else:
            dt = torch.bfloat16 if mode == LB_BF16 else torch.float16
            self.f = [torch.zeros(19, self.N, dtype=dt, device=device) for _ in range(2)]
            self.m = [torch.zeros(self.N, 4, dtype=torch.float32, device=device) for _ in range(2)]
            self.h = lb_create_mixed(self.p, self.f[0], self.f[1], self.m[0], self.m[1], self.g, self.flags)

    @property
    def mixed(self):
        return self.storage != "fp32"

    def current(self):
        """The live FP32 population buffer (FP32 storage only)."""
        ptr = lb_current(self.h)
        return self.f[0] if ptr == self.f[0].data_ptr() else self.f[1]

    def velocity(self):
        """The float4 velocity field ib_interp reads: (v, rho) in the last
        step's forced rows (FP32 storage) or (v, rho - 1) everywhere (mixed)."""
        if not self.mixed:
            return self.v
        ptr = lb_velocity(self.h)
        return self.m[0] if ptr == self.m[0].data_ptr() else self.m[1]

    def export(self, stream=None):
        """The current post-collision state as FP32 shifted populations, [19, N]."""
        out = torch.empty(19, self.N, dtype=torch.float32, device=self.g.device)
        lb_export(self.h, out, stream)
        return out

    def init_shear(self):
        lb_init_shear(self.h)

    def step(self, n=1):
        lb_step(self.h, n)

    def moments_fp64(self):
        return lb_moments_fp64(self.h, self.scratch)

    def check(self, u_max=0.3):
        """Instability check: ((non-finite cells, rho <= 0, |u| > u_max), ok)."""
        return _check("lb_check", self.h, u_max, self.scratch, 3)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.lb_destroy(self.h)
            self.h = None


def mem_params_from(d):
    return mem_params(*[float(d[n]) for n, _ in mem_params._fields_])


def bond_params_from(d):
    return bond_params(int(d["lig_i0"]), int(d["lig_j0"]), int(d["lig_ni"]), int(d["lig_nj"]),
                       int(d["box_nx"]), int(d["box_ny"]), int(d["max_per_ligand"]), float(d["z_wall"]),
                       float(d["sigma"]), float(d["l_b"]), float(d["d_capture"]), float(d["gamma"]),
                       float(d["kT"]), float(d["kon0_dt"]), float(d["koff0_dt"]), int(d["seed"]))


class Membrane:
    """Membrane mesh (rest state from X0) in a caller-owned workspace."""

    def __init__(self, params, mesh, device="cuda"):
        n = int(mesh["X0"].size // 3)
        self.n = n
        self.n_plt = int(mesh["n_plt"])
        self.p = mem_params_from(params)
        pairs = np.asarray(mesh["pairs"], dtype=np.int32).reshape(-1, 2)
        ws_bytes = membrane_query_workspace(n, mesh["tri"], len(pairs), self.n_plt)
        self.ws = _bytes(ws_bytes, device)
        self.h = membrane_create(self.p, n, mesh["tri"], pairs, self.n_plt, mesh["node_plt"],
                                 mesh["is_membrane"], mesh["X0"], self.ws)

    def forces(self, X, F):
        membrane_forces(self.h, X, F)

    def set_path(self, path):
        """0: the three passes through per-element slots (default); 1: the
        fused per-platelet pass with exact fixed-point sums, where it applies."""
        _call("membrane_set_path", self.h, int(path))

    @property
    def fused(self):
        v = c_int()
        _call("membrane_get_path", self.h, ctypes.byref(v))
        return bool(v.value)

    def measure(self, X):
        return membrane_measure(self.h, X, self.n_plt)

    def centroids(self, X, out=None, stream=None):
        """Per-platelet node centroids [n_plt][3] on the device (out: device
        float64 buffer of 4 * n_plt, reused if given)."""
        if out is None:
            out = torch.empty(4 * self.n_plt, dtype=torch.float64, device=X.device)
        _call("membrane_centroids", self.h, _ptr(X), _ptr(out), _stream(stream))
        return out[:3 * self.n_plt].view(self.n_plt, 3)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.membrane_destroy(self.h)
            self.h = None


class Bonds:
    """Receptor sites and bond state on the device."""

    def __init__(self, params, site_tri, site_w, tri_dev, bound, lig_count, device="cuda"):
        self.p = bond_params_from(params)
        self.R = int(len(site_tri))
        n_tri = int(tri_dev.numel() // 3)
        st = np.asarray(site_tri)
        sw = np.asarray(site_w, dtype=np.float64).reshape(-1, 2)
        bd = np.asarray(bound)
        if self.R and (st.min() < 0 or st.max() >= n_tri):
            raise ValueError("receptor site on a triangle id outside [0, %d)" % n_tri)
        if self.R and (sw.min() < 0 or (sw.sum(1) > 1 + 1e-12).any()):
            raise ValueError("barycentric weights must be >= 0 with w0 + w1 <= 1")
        if self.R and (bd.min() < -1 or bd.max() >= self.p.lig_ni * self.p.lig_nj):
            raise ValueError("bound ligand id out of range")
        self.site_tri = torch.as_tensor(np.ascontiguousarray(site_tri, dtype=np.int32), device=device)
        self.site_w = torch.as_tensor(np.ascontiguousarray(site_w, dtype=np.float64).ravel(), device=device)
        self.tri = tri_dev
        self.bound = torch.as_tensor(np.ascontiguousarray(bound, dtype=np.int32), device=device).clone()
        self.lig_count = torch.as_tensor(np.ascontiguousarray(lig_count, dtype=np.int32), device=device).clone()
        self.ws = _bytes(bonds_query_workspace(self.p, self.R), device)
        self.h = bonds_create(self.p, self.R, self.site_tri, self.site_w, self.tri, self.bound, self.lig_count,
                              self.ws)

    def forces(self, X, F, M):
        bonds_forces(self.h, X, F, M)

    def step(self, X, M, step):
        bonds_step(self.h, X, M, step)

    def status(self):
        return bonds_status(self.h)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.bonds_destroy(self.h)
            self.h = None


class Tethers:
    """Tether (pause-time) tracking over a Bonds object (Section 4.2): per
    platelet the step count at which its current tether began (-1: free) and
    the pause times, in steps, of completed tether events.  site_plt: the
    platelet of every site (host array); state: optional saved per-platelet
    state (a continued run)."""

    def __init__(self, bonds, site_plt, n_plt, capacity=1 << 20, state=None, device="cuda"):
        sp = np.ascontiguousarray(site_plt, dtype=np.int32)
        if len(sp) != bonds.R:
            raise ValueError("one platelet id per receptor site")
        self.bonds = bonds                   # the tracker reads its bond state
        self.n_plt = int(n_plt)
        st = np.full(self.n_plt, -1, dtype=np.int64) if state is None else np.asarray(state, dtype=np.int64)
        self.state = torch.as_tensor(st, device=device).clone()
        self.pause_buf = torch.zeros(max(int(capacity), 1), dtype=torch.int64, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        n = c_size_t()
        _call("tether_query_workspace", bonds.R, self.n_plt, ctypes.byref(n))
        self.ws = _bytes(n.value, device)
        h = P()
        _call("tether_create", bonds.h, self.n_plt, _ptr(sp), _ptr(self.ws), n.value, _ptr(self.state),
              _ptr(self.pause_buf), int(capacity), _ptr(self.count), ctypes.byref(h))
        self.h = h

    def update(self, step, stream=None):
        """After the bonds_step of step `step`."""
        _call("tether_update", self.h, int(step), _stream(stream))

    def pauses(self):
        """Completed pause times in steps, sorted (the device appends them in
        no fixed order)."""
        n = min(int(self.count.item()), self.pause_buf.numel())
        return np.sort(self.pause_buf[:n].cpu().numpy())

    def events(self):
        return int(self.count.item())

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tether_destroy(self.h)
            self.h = None


def bridge_params_from(d):
    return bridge_params(float(d["sigma"]), float(d["l_b"]), float(d["d_capture"]), float(d["gamma"]),
                         float(d["kT"]), float(d["kon0_dt"]), float(d["koff0_dt"]), int(d["box_nx"]),
                         int(d["box_ny"]), int(d["seed"]))


class Bridges:
    """Platelet-platelet bridges between the receptor sites of a Bonds set
    (which this object keeps alive: the bridges go first)."""

    def __init__(self, params, bonds, node_plt, n_plt, partner=None, device="cuda"):
        self.p = bridge_params_from(params)
        self.bonds = bonds
        node_plt = np.ascontiguousarray(node_plt, dtype=np.int32)
        self.M = int(node_plt.size)
        R = bonds.R
        if partner is None:
            partner = np.full(R, -1, dtype=np.int32)
        pa = np.asarray(partner, dtype=np.int32)
        if R and (pa.min() < -1 or pa.max() >= R):
            raise ValueError("partner ids out of range")
        idx = np.where(pa >= 0)[0]
        if np.any(pa[pa[idx]] != idx) or np.any(pa[idx] == idx):
            raise ValueError("partner array must pair distinct sites symmetrically")
        self.partner = torch.as_tensor(np.ascontiguousarray(pa), device=device).clone()
        nb = c_size_t()
        _call("bridges_query_workspace", ctypes.byref(self.p), R, int(n_plt), self.M, ctypes.byref(nb))
        self.ws = _bytes(nb.value, device)
        h = c_void_p()
        _call("bridges_create", ctypes.byref(self.p), bonds.h, int(n_plt), _ptr(node_plt), self.M,
              _ptr(self.partner), _ptr(self.ws), nb.value, ctypes.byref(h))
        self.h = h

    def forces(self, X, F, stream=None):
        _call("bridges_forces", self.h, _ptr(X), _ptr(F), self.M, _stream(stream))

    def step(self, X, step, stream=None):
        _call("bridges_step", self.h, _ptr(X), self.M, int(step), _stream(stream))

    def status(self):
        out = (c_longlong * 3)()
        _call("bridges_status", self.h, out)
        return tuple(int(v) for v in out)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.bridges_destroy(self.h)
            self.h = None


class Simulation:
    """The coupled step on one workload (see :mod:`paper_1312_2234_b300.workload`)."""

    def __init__(self, w, device="cuda", first_step=0, storage="fp32", fp16_exponent=None, tune=False,
                 track_tethers=0):
        """track_tethers: capacity of the pause-time record (0: no tether
        tracking; see Tethers)."""
        g = w["grid"]
        self.lattice = Lattice(g["nx"], g["ny"], g["nz"], g["tau"], g["u_top"], g.get("body", (0, 0, 0)), device,
                               storage, fp16_exponent, g.get("walls", 0))
        if tune:   # pick the lattice kernel's launch shape for this grid (before the state is set)
            self.shape, _ = lb_autotune(self.lattice)
        self.lattice.init_shear()
        memp = w["membrane"]
        self.fem = None
        if memp.get("bending", "dihedral") == "fem":   # Eq. 6-10 in place of the dihedral term
            memp = dict(memp, k_b=0.0)
            self.fem = FemBending(w["mesh"], device)
        self.membrane = Membrane(memp, w["mesh"], device)
        self.M = int(w["M"])
        self.X = torch.as_tensor(np.ascontiguousarray(w["X"], dtype=np.float64), device=device).clone()
        self.F = torch.zeros(3 * self.M, dtype=torch.float32, device=device)
        self.U = torch.zeros(3 * self.M, dtype=torch.float32, device=device)
        self.tri = torch.as_tensor(np.ascontiguousarray(w["mesh"]["tri"], dtype=np.int32).ravel(), device=device)
        self.bonds = None
        if len(w["sites"]["tri"]) > 0:
            self.bonds = Bonds(w["bonds"], w["sites"]["tri"], w["sites"]["w"], self.tri, w["bound"],
                               w["lig_count"], device)
        self.h = sim_create(self.lattice.h, self.membrane.h, self.bonds.h if self.bonds else None,
                            self.X, self.F, self.U, self.M, first_step)
        if self.fem is not None:
            _call("sim_set_fem_bending", self.h, self.fem.h, float(w["membrane"]["k0"]))
        self.bridges = None
        if w.get("bridges") is not None and self.bonds is not None:
            self.bridges = Bridges(w["bridges"], self.bonds, w["mesh"]["node_plt"], w["mesh"]["n_plt"],
                                   w.get("partner"), device)
            _call("sim_set_bridges", self.h, self.bridges.h)
        self.tethers = None
        if track_tethers and self.bonds is not None:
            tri = np.asarray(w["mesh"]["tri"], dtype=np.int64).reshape(-1, 3)
            site_plt = np.asarray(w["mesh"]["node_plt"])[tri[np.asarray(w["sites"]["tri"]), 0]]
            self.tethers = Tethers(self.bonds, site_plt, w["mesh"]["n_plt"], int(track_tethers), device=device)
            _call("sim_set_tether", self.h, self.tethers.h)

    def step(self, n=1, stream=None):
        sim_step(self.h, n, stream)

    def step_record(self, n, dev_ring, host_ring, stream=None):
        """n steps, each step's positions copied to the pinned host ring
        [ring][3M] through the device ring [ring][3M], overlapping the next
        step (see sim_step_record)."""
        ring = int(host_ring.shape[0])
        assert host_ring.is_pinned() and dev_ring.shape == host_ring.shape
        _call("sim_step_record", self.h, int(n), _ptr(dev_ring), _ptr(host_ring), ring, _stream(stream))

    def step_track(self, n, dev_scratch, host_out, stream=None):
        """n steps; after step k the platelet centroids go to host_out[k]
        (pinned, [n][n_plt][3] float64) through dev_scratch (device, 72 n_plt)."""
        assert host_out.is_pinned() and host_out.shape[0] >= n
        _call("sim_step_track", self.h, int(n), _ptr(dev_scratch), _ptr(host_out), _stream(stream))

    @property
    def step_index(self):
        return sim_step_index(self.h)

    def check(self, u_max=0.3):
        """((non-finite cells, rho <= 0, |u| > u_max, non-finite node
        coordinates), ok) of the current state."""
        return _check("sim_check", self.h, u_max, self.lattice.scratch, 4)

    def _live_populations(self):
        lat = self.lattice
        if not lat.mixed:
            return {"f": lat.current()}
        live = 0 if lat.velocity().data_ptr() == lat.m[0].data_ptr() else 1
        return {"fneq": lat.f[live], "m": lat.m[live]}

    def checkpoint(self):
        """The state a later run needs to continue this one: the step index,
        the lattice populations (FP32, or 16-bit f*neq with the moments), the
        node positions, the wall-bond and bridge state and the open tethers.  Philox draws are keyed
        by (site, step), so the continued run takes the same random decisions.
        Returns a dict of host arrays (np.savez-able)."""
        torch.cuda.synchronize()
        ck = {"step": np.array(self.step_index, dtype=np.int64), "storage": np.array(self.lattice.storage),
              "fp16_exponent": np.array(int(self.lattice.p.fp16_exponent)), "X": self.X.cpu().numpy()}
        for k, v in self._live_populations().items():
            ck[k] = v.cpu().numpy() if v.dtype != torch.bfloat16 else v.view(torch.int16).cpu().numpy()
        if self.bonds is not None:
            ck["bound"] = self.bonds.bound.cpu().numpy()
            ck["lig_count"] = self.bonds.lig_count.cpu().numpy()
        if self.bridges is not None:
            ck["partner"] = self.bridges.partner.cpu().numpy()
        if self.tethers is not None:
            ck["tether_state"] = self.tethers.state.cpu().numpy()
        return ck

    @classmethod
    def restore(cls, w, ck, device="cuda", **kw):
        """A simulation of workload `w` continuing from checkpoint `ck`."""
        sim = cls(w, device=device, first_step=int(ck["step"]), storage=str(ck["storage"]),
                  fp16_exponent=int(ck["fp16_exponent"]), **kw)
        for k, v in sim._live_populations().items():
            src = torch.as_tensor(ck[k])
            v.copy_(src.view(torch.bfloat16) if v.dtype == torch.bfloat16 else src)
        sim.X.copy_(torch.as_tensor(ck["X"]))
        if sim.bonds is not None:
            sim.bonds.bound.copy_(torch.as_tensor(ck["bound"]))
            sim.bonds.lig_count.copy_(torch.as_tensor(ck["lig_count"]))
        if sim.bridges is not None:
            sim.bridges.partner.copy_(torch.as_tensor(ck["partner"]))
        if sim.tethers is not None and "tether_state" in ck:
            sim.tethers.state.copy_(torch.as_tensor(ck["tether_state"]))
        torch.cuda.synchronize()
        return sim

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.sim_destroy(self.h)
            self.h = None


# ---------------------------------------------------------------- finite-element bending
FEM_FIELDS = ("nx", "ny", "nz", "A", "K", "KG", "lapK")


class FemBending:
    """Six-node element mesh of the finite-element bending term (Eq. 6-10)."""

    def __init__(self, mesh, device="cuda"):
        n = int(np.asarray(mesh["node_plt"]).size)
        e6 = np.ascontiguousarray(mesh["elem6"], dtype=np.int32).ravel()
        nb = c_size_t()
        _call("fem_query_workspace", n, e6.size // 6, ctypes.byref(nb))
        self.ws = _bytes(nb.value, device)
        h = c_void_p()
        _call("fem_create", n, e6.size // 6, _ptr(e6), _ptr(self.ws), nb.value, ctypes.byref(h))
        self.h = h
        self.n = n
        self.device = device

    def forces(self, k0, X, F, accumulate=False, stream=None):
        _call("fem_bending_forces", self.h, float(k0), _ptr(X), _ptr(F), int(bool(accumulate)), _stream(stream))

    def fields(self, X, stream=None):
        """Nodal normals, areas and curvatures: dict of float32 device tensors."""
        out = torch.empty(7, self.n, dtype=torch.float32, device=self.device)
        _call("fem_fields", self.h, _ptr(X), _ptr(out), _stream(stream))
        return {k: out[i] for i, k in enumerate(FEM_FIELDS)}

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.fem_destroy(self.h)
            self.h = None


# ---------------------------------------------------------------- learned membrane surrogate
SG_BF16, SG_FP32 = 0, 1
SG_MODE = {"bf16": SG_BF16, "fp32": SG_FP32}
SG = dict(IN=42, IN_PAD=64, HID=128, OUT=18, OUT_PAD=32, W1=0, B1=8192, W2=8320, B2=24704, W3=24832, B3=28928,
          N_TRAINED=28960, IN_SHIFT=28960, IN_SCALE=29024, OUT_SCALE=29088, TGT_SCALE=29120, N_FLOATS=29152,
          PARAM_BYTES=215040)


class SurrogateParams:
    """Caller-owned parameter buffer of the surrogate (FP32 master block +
    BF16 copies) with its Adam moments and gradient buffer."""

    def __init__(self, device="cuda"):
        n = c_size_t()
        _call("sg_params_bytes", ctypes.byref(n))
        assert n.value == SG["PARAM_BYTES"]
        self.buf = _bytes(n.value, device).zero_()
        self.floats = self.buf[:SG["N_FLOATS"] * 4].view(torch.float32)
        self.m = torch.zeros(SG["N_TRAINED"], dtype=torch.float32, device=device)
        self.v = torch.zeros_like(self.m)
        self.grad = torch.zeros_like(self.m)
        self.t = 0
        self.device = device

    def set(self, p):
        """p: dict of numpy arrays W1 [128][42], b1, W2, b2, W3 [18][128], b3,
        in_shift [42], in_scale [42], out_scale [18], tgt_scale [18] (the
        reference's layout)."""
        ni, no = SG["IN"], SG["OUT"]
        f = np.zeros(SG["N_FLOATS"], np.float32)
        W1 = np.zeros((128, SG["IN_PAD"]), np.float32)
        W1[:, :ni] = p["W1"]
        f[SG["W1"]:SG["B1"]] = W1.ravel()
        f[SG["B1"]:SG["W2"]] = p["b1"]
        f[SG["W2"]:SG["B2"]] = np.asarray(p["W2"], np.float32).ravel()
        f[SG["B2"]:SG["W3"]] = p["b2"]
        W3 = np.zeros((SG["OUT_PAD"], 128), np.float32)
        W3[:no] = p["W3"]
        f[SG["W3"]:SG["B3"]] = W3.ravel()
        f[SG["B3"]:SG["B3"] + no] = p["b3"]
        f[SG["IN_SHIFT"]:SG["IN_SHIFT"] + ni] = p.get("in_shift", np.zeros(ni))
        f[SG["IN_SCALE"]:SG["IN_SCALE"] + ni] = p["in_scale"]
        f[SG["OUT_SCALE"]:SG["OUT_SCALE"] + no] = p["out_scale"]
        f[SG["TGT_SCALE"]:SG["TGT_SCALE"] + no] = p.get("tgt_scale", np.ones(no))
        self.floats.copy_(torch.from_numpy(f))
        _call("sg_sync_shadows", _ptr(self.buf), None)

    def get(self):
        ni, no, nip, nop = SG["IN"], SG["OUT"], SG["IN_PAD"], SG["OUT_PAD"]
        f = self.floats.cpu().numpy().astype(np.float64)
        return dict(W1=f[SG["W1"]:SG["B1"]].reshape(128, nip)[:, :ni].copy(), b1=f[SG["B1"]:SG["W2"]].copy(),
                    W2=f[SG["W2"]:SG["B2"]].reshape(128, 128).copy(), b2=f[SG["B2"]:SG["W3"]].copy(),
                    W3=f[SG["W3"]:SG["B3"]].reshape(nop, 128)[:no].copy(), b3=f[SG["B3"]:SG["B3"] + no].copy(),
                    in_shift=f[SG["IN_SHIFT"]:SG["IN_SHIFT"] + ni].copy(),
                    in_scale=f[SG["IN_SCALE"]:SG["IN_SCALE"] + ni].copy(),
                    out_scale=f[SG["OUT_SCALE"]:SG["OUT_SCALE"] + no].copy(),
                    tgt_scale=f[SG["TGT_SCALE"]:SG["TGT_SCALE"] + no].copy())

    def grads(self):
        """The last gradient as a dict in the reference's layout."""
        ni, no, nip, nop = SG["IN"], SG["OUT"], SG["IN_PAD"], SG["OUT_PAD"]
        g = self.grad.cpu().numpy().astype(np.float64)
        return dict(W1=g[SG["W1"]:SG["B1"]].reshape(128, nip)[:, :ni].copy(), b1=g[SG["B1"]:SG["W2"]].copy(),
                    W2=g[SG["W2"]:SG["B2"]].reshape(128, 128).copy(), b2=g[SG["B2"]:SG["W3"]].copy(),
                    W3=g[SG["W3"]:SG["B3"]].reshape(nop, 128)[:no].copy(), b3=g[SG["B3"]:SG["B3"] + no].copy())


class SurrogateBatch:
    """Workspace of sg_grad for a fixed batch size (multiple of 128)."""

    def __init__(self, batch, device="cuda"):
        assert batch % 128 == 0
        n = c_size_t()
        _call("sg_query_work", int(batch), ctypes.byref(n))
        self.batch = batch
        self.work = _bytes(n.value, device)
        self.nbytes = n.value
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)

    def grad(self, params, feat, target, mode="bf16", stream=None):
        """Gradients into params.grad; returns the device loss tensor."""
        _call("sg_grad", _ptr(params.buf), _ptr(feat), _ptr(target), self.batch, SG_MODE[mode], _ptr(params.grad),
              _ptr(self.loss), _ptr(self.work), self.nbytes, _stream(stream))
        return self.loss

    def status(self):
        f = c_int()
        _call("sg_work_status", _ptr(self.work), self.batch, ctypes.byref(f))
        return f.value


def sg_adam(params, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    params.t += 1
    _call("sg_adam", _ptr(params.buf), _ptr(params.grad), _ptr(params.m), _ptr(params.v), float(lr), float(beta1),
          float(beta2), float(eps), params.t, _stream(stream))


class Surrogate:
    """Surrogate mesh context (one-rings and rest data of the membrane nodes)."""

    def __init__(self, mesh, mode="bf16", device="cuda"):
        n = int(np.asarray(mesh["node_plt"]).size)
        tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32).ravel()
        X0 = np.ascontiguousarray(mesh["X0"], dtype=np.float64)
        ism = np.ascontiguousarray(mesh["is_membrane"], dtype=np.uint8)
        nb = c_size_t()
        _call("sg_query_workspace", n, ctypes.byref(nb))
        self.ws = _bytes(nb.value, device)
        self.mode = mode
        self.n = n
        h = c_void_p()
        _call("sg_create", n, tri.size // 3, _ptr(tri), _ptr(X0), _ptr(ism), SG_MODE[mode], _ptr(self.ws), nb.value,
              ctypes.byref(h))
        self.h = h
        rows = c_int()
        node = c_void_p()
        _call("sg_rows", self.h, ctypes.byref(rows), ctypes.byref(node))
        self.rows = rows.value
        self.rows_pad = (self.rows + 127) // 128 * 128
        self.device = device

    def features(self, params, X, stream=None):
        """(feat [rows_pad][64] BF16 or float, strains xs [rows_pad][18],
        rest moduli scales ms [rows_pad][18])."""
        dt = torch.bfloat16 if self.mode == "bf16" else torch.float32
        feat = torch.zeros(self.rows_pad, SG["IN_PAD"], dtype=dt, device=self.device)
        xs = torch.zeros(self.rows_pad, SG["OUT"], dtype=torch.float32, device=self.device)
        ms = torch.zeros(self.rows_pad, SG["OUT"], dtype=torch.float32, device=self.device)
        _call("sg_features", self.h, _ptr(params.buf), _ptr(X), _ptr(feat), _ptr(xs), _ptr(ms), _stream(stream))
        return feat, xs, ms

    def targets(self, params, membrane_params, xs, ms, stream=None):
        """Training records [rows_pad][36] (a, b) of the plain local terms'
        stresses (membrane_params: k_spring, k_t, k_b)."""
        t = torch.zeros(self.rows_pad, 2 * SG["OUT"], dtype=torch.float32, device=self.device)
        q = membrane_params
        _call("sg_targets", self.h, _ptr(params.buf), float(q["k_spring"]), float(q["k_t"]), float(q["k_b"]),
              _ptr(xs), _ptr(ms), _ptr(t), _stream(stream))
        return t

    def forces(self, params, membrane, X, F, stream=None):
        _call("sg_membrane_forces", self.h, _ptr(params.buf), membrane.h, _ptr(X), _ptr(F), _stream(stream))

    def status(self):
        f = c_int()
        _call("sg_status", self.h, ctypes.byref(f))
        return f.value

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.sg_destroy(self.h)
            self.h = None


def sim_set_surrogate(sim, sg, params):
    _call("sim_set_surrogate", sim.h, sg.h if sg is not None else None,
          _ptr(params.buf) if params is not None else None)


# ---------------------------------------------------------------- launch shapes, batches
def lb_autotune(lat, reps=5, stream=None):
    """Times every launch shape of the lattice step, keeps the fastest;
    returns (shape, ms per step).  The lattice advances: tune before init."""
    ms = ctypes.c_float()
    _call("lb_autotune", lat.h, int(reps), _stream(stream), ctypes.byref(ms))
    sh = c_int()
    _call("lb_get_shape", lat.h, ctypes.byref(sh))
    return sh.value, ms.value


def lb_set_shape(lat, shape):
    _call("lb_set_shape", lat.h, int(shape))


def lb_get_shape(lat):
    sh = c_int()
    _call("lb_get_shape", lat.h, ctypes.byref(sh))
    return sh.value


class LatticeBatch:
    """Lattices of any sizes and storage modes stepped together: one
    persistent kernel launch per storage mode and step (lb_batch_step)."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        arr = (c_void_p * len(self.lattices))(*[lat.h.value if isinstance(lat.h, c_void_p) else lat.h
                                                 for lat in self.lattices])
        h = c_void_p()
        _call("lb_batch_create", ctypes.cast(arr, c_void_p), len(self.lattices), ctypes.byref(h))
        self.h = h

    def step(self, n=1, stream=None):
        _call("lb_batch_step", self.h, int(n), _stream(stream))

    def autotune(self, reps=5, stream=None):
        """Picks each mixed lattice's column shape by timing; the state is
        unchanged (no spread force pending).  Returns ms per batched step."""
        ms = ctypes.c_float()
        _call("lb_batch_autotune", self.h, int(reps), _stream(stream), ctypes.byref(ms))
        return ms.value

    def set_grid(self, blocks_per_sm):
        """blocks per SM of the batched launches (0: every resident block)."""
        _call("lb_batch_set_grid", self.h, int(blocks_per_sm))

    def shapes(self):
        out = (c_int * len(self.lattices))()
        _call("lb_batch_get_shapes", self.h, out)
        return list(out)

    def set_shapes(self, shapes):
        _call("lb_batch_set_shapes", self.h, (c_int * len(self.lattices))(*[int(s) for s in shapes]))

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.lb_batch_destroy(self.h)
            self.h = None


class Batch:
    """Independent chambers stepped by one CUDA graph launch: each chamber's
    small kernels on parallel branches, the lattice update of all chambers
    as one batched launch per storage mode."""

    def __init__(self, sims, steps_per_graph=1, tune=False):
        """tune: pick the mixed chambers' column shapes by timing (between
        steps; the state is unchanged)."""
        self.sims = list(sims)
        arr = (c_void_p * len(self.sims))(*[s.h.value if isinstance(s.h, c_void_p) else s.h for s in self.sims])
        h = c_void_p()
        _call("batch_create", ctypes.cast(arr, c_void_p), len(self.sims), int(steps_per_graph), ctypes.byref(h))
        self.h = h
        self.k = steps_per_graph
        self.lb_ms = self.autotune() if tune else None

    def step(self, n=1, stream=None):
        _call("batch_step", self.h, int(n), _stream(stream))

    def set_layout(self, groups, blocks_per_sm=0):
        """Chamber groups of the step graph and the lattice launches' blocks
        per SM (0: persistent grid of every resident block)."""
        _call("batch_set_layout", self.h, int(groups), int(blocks_per_sm))

    def autotune(self, reps=5, stream=None):
        """Returns ms per batched lattice step after tuning."""
        ms = ctypes.c_float()
        _call("batch_autotune", self.h, int(reps), _stream(stream), ctypes.byref(ms))
        return ms.value

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.batch_destroy(self.h)
            self.h = None
