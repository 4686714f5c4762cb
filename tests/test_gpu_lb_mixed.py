"""GPU parity of the mixed-precision lattice storage (16-bit post-collision
f^neq + FP32 (v, rho - 1), Section 3.3 step unchanged) against the FP64
oracle, and of the coupled step run on it.

Error bound.  The only difference from the FP32 path is that every step
rounds each stored f*neq_q once, by at most u |f*neq_q| with u = 2^-9 (BF16)
or 2^-12 (FP16 scaled into its normal range), plus 2^-25 2^-s absolute for
FP16 values that stay subnormal.  BGK with tau > 1/2 does not amplify a
perturbation of the populations, so after n steps

    |f_gpu - f_oracle| <= (FP32 bound: 1e-5 max|f~|) + n u max_t |f*neq|,

and a velocity component, a sum of at most 10 populations divided by
rho ~ 1, is off by at most 10 times that.  Each test asserts these bounds;
the measured errors sit about an order of magnitude below them."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu
UNIT = {"bf16": 2.0 ** -9, "fp16": 2.0 ** -12}


def f32(x):
    return float(np.float32(x))


def feq_shifted(rho, v):
    c, w = oracle.lattice()
    cv = c.astype(np.float64) @ v
    vv = (v * v).sum(0)
    return w[:, None] * ((rho - 1.0) + rho * (3.0 * cv + 4.5 * cv * cv - 1.5 * vv))


def run_pair(storage, dims, tau, u_top, body, n, g=None, flags=None, walls=0):
    nx, ny, nz = dims
    N = nx * ny * nz
    lat = fsi.Lattice(nx, ny, nz, tau, u_top, body, storage=storage, walls=walls)
    lat.init_shear()
    p = oracle.lb_params(nx, ny, nz, f32(tau), tuple(f32(u) for u in u_top), tuple(f32(b) for b in body),
                         walls=walls)
    f = oracle.lb_init_shear(p)
    _, w = oracle.lattice()
    fneq_max = 0.0
    rho = v = None
    for s in range(n):
        if g is not None:
            lat.g.copy_(torch.from_numpy(g))
            lat.flags.copy_(torch.from_numpy(flags))
            g64 = np.ascontiguousarray(g[:, :3].astype(np.float64).T).ravel()
            f, rho, v = oracle.lb_step(p, f, g64)
        else:
            f, rho, v = oracle.lb_step(p, f)
        lat.step(1)
        fs = f.reshape(19, N) - w[:, None]
        fneq_max = max(fneq_max, float(np.abs(fs - feq_shifted(rho, v.reshape(3, N))).max()))
    torch.cuda.synchronize()
    return lat, f.reshape(19, N) - w[:, None], rho, v.reshape(3, N), fneq_max


@pytest.mark.parametrize("walls", [0, 1])
@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("dims", [(37, 23, 19), (128, 64, 16), (5, 3, 2)])
def test_free_steps(storage, dims, walls):
    n = 30
    lat, fs, rho, v, fneq_max = run_pair(storage, dims, 0.8, (4e-3, -1.5e-3, 0.0), (2e-6, 0.0, -1e-6), n,
                                         walls=walls)
    # an on-site wall node builds each entering population from up to seven
    # known ones (Eq. 23-30), adding their rounding errors: a factor 4 on
    # the storage term where every layer is a wall (nz = 2)
    amp = 4.0 if walls else 1.0
    bound_f = 1e-5 * np.abs(fs).max() + amp * n * UNIT[storage] * fneq_max
    err_f = np.abs(lat.export().cpu().numpy() - fs).max()
    assert err_f <= bound_f, (err_f, bound_f)
    m = lat.velocity().cpu().numpy()
    assert np.abs(m[:, :3].T - v).max() <= 10 * bound_f
    assert np.abs(m[:, 3] - (rho - 1.0)).max() <= 19 * bound_f


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_forced_rows(storage):
    """Forced rows: the moments buffer carries the force-corrected velocity
    everywhere, the consumed force is cleared."""
    dims = (45, 17, 13)
    nx, ny, nz = dims
    rng = np.random.default_rng(7)
    flags = (rng.uniform(size=ny * nz) < 0.3).astype(np.int32)
    g = np.zeros((nx * ny * nz, 4), np.float32)
    rows = np.repeat(flags, nx).astype(bool)
    g[rows, :3] = (1e-4 * rng.standard_normal((rows.sum(), 3))).astype(np.float32)
    n = 8
    lat, fs, rho, v, fneq_max = run_pair(storage, dims, 0.7, (2e-3, 0.0, 0.0), (0.0, 0.0, 0.0), n, g, flags)
    bound_f = 1e-5 * np.abs(fs).max() + n * UNIT[storage] * fneq_max
    assert np.abs(lat.export().cpu().numpy() - fs).max() <= bound_f
    m = lat.velocity().cpu().numpy()
    assert np.abs(m[:, :3].T - v).max() <= 10 * bound_f
    assert np.all(lat.g.cpu().numpy()[rows] == 0)


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_mass_momentum_fp64(storage):
    """Still walls and no force: the FP64 device sums of mass and momentum
    of the rebuilt populations stay put (collision and bounce-back conserve
    them; each step's rounding of f*neq is the only change)."""
    nx, ny, nz = 24, 20, 16
    lat = fsi.Lattice(nx, ny, nz, 0.9, (0.0, 0.0, 0.0), storage=storage, fp16_exponent=20)
    lat.init_shear()
    m0 = lat.moments_fp64()
    lat.step(50)
    m1 = lat.moments_fp64()
    assert abs(m0[0] - nx * ny * nz) < 1e-9 * nx * ny * nz
    assert abs(m1[0] - m0[0]) < 1e-6 * m0[0]
    assert np.all(np.abs(m1[1:]) < 1e-9)


def test_export_fp32_is_the_live_buffer():
    lat = fsi.Lattice(16, 8, 8, 0.8, (1e-3, 0.0, 0.0))
    lat.init_shear()
    lat.step(3)
    assert torch.equal(lat.export(), lat.current())


@pytest.mark.parametrize("storage,tol_x,tol_u", [("bf16", 2e-4, 1e-3), ("fp16", 3e-5, 1e-4)])
def test_coupled_step(storage, tol_x, tol_u):
    """The whole coupled step on mixed storage: displacement and node
    velocity against the FP64 oracle within the stated per-output error
    (measured ~2e-5 / 8e-5 for BF16 and ~4e-6 / 9e-6 for FP16 after 200
    steps), and the bond states compared site by site: at these position
    errors no adhesion decision flips."""
    w = workload.tiny(seed=3, shear=3.0e4)
    w["membrane"] = {k: (f32(v) if isinstance(v, float) else v) for k, v in w["membrane"].items()}
    g = dict(w["grid"])
    g["tau"] = f32(g["tau"])
    g["u_top"] = tuple(f32(u) for u in g["u_top"])
    w["grid"] = g
    sim = fsi.Simulation(w, storage=storage)
    ora = oracle.Sim(w)
    X0 = w["X"].copy()
    steps = 200
    sim.step(steps)
    for _ in range(steps):
        ora.step()
    torch.cuda.synchronize()
    dX = sim.X.cpu().numpy() - X0
    assert np.abs(dX - (ora.X - X0)).max() <= tol_x * np.abs(ora.X - X0).max()
    assert np.abs(sim.U.cpu().numpy() - ora.U).max() <= tol_u * np.abs(ora.U).max()
    if sim.bonds is not None:
        assert np.array_equal(sim.bonds.bound.cpu().numpy(), ora.bound)


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("dims", [(37, 23, 19), (46, 17, 13), (3, 5, 4)])
def test_state_varying_along_x(storage, dims):
    """A state that varies from cell to cell (the developed shear flow plus a
    random perturbation of the stored f*neq): every pulled population comes
    from a different value, so a wrong source column (periodic wrap, the
    last cell of an odd row) shows.  The exported state is the oracle's
    initial state; bounds as in test_free_steps."""
    nx, ny, nz = dims
    N = nx * ny * nz
    lat = fsi.Lattice(nx, ny, nz, 0.8, (4e-3, -1.5e-3, 0.0), (2e-6, 0.0, -1e-6), storage=storage)
    lat.init_shear()
    rng = np.random.default_rng(11)
    live = 0 if lat.velocity().data_ptr() == lat.m[0].data_ptr() else 1   # f*neq buffer paired with the moments
    cur = lat.f[live]
    noise = torch.from_numpy((3e-5 * rng.standard_normal(tuple(cur.shape))).astype(np.float32)).cuda()
    cur.copy_((cur.float() + noise * (1.0 if storage == "bf16" else 2.0 ** lat.p.fp16_exponent)).to(cur.dtype))
    f0 = lat.export().cpu().numpy().astype(np.float64)
    _, w = oracle.lattice()
    p = oracle.lb_params(nx, ny, nz, f32(0.8), (f32(4e-3), f32(-1.5e-3), 0.0), (f32(2e-6), 0.0, f32(-1e-6)))
    f = (f0 + w[:, None]).ravel()
    n = 12
    fneq_max = 0.0
    for _ in range(n):
        f, rho, v = oracle.lb_step(p, f)
        fs = f.reshape(19, N) - w[:, None]
        fneq_max = max(fneq_max, float(np.abs(fs - feq_shifted(rho, v.reshape(3, N))).max()))
    lat.step(n)
    torch.cuda.synchronize()
    bound_f = 1e-5 * np.abs(fs).max() + n * UNIT[storage] * fneq_max
    err_f = np.abs(lat.export().cpu().numpy() - fs).max()
    assert err_f <= bound_f, (err_f, bound_f)


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("dims", [(48, 17, 13), (8, 5, 4), (64, 9, 6), (16, 3, 5), (40, 24, 7)])
def test_launch_shapes_rows_on_16_byte_boundaries(storage, shape, dims):
    """Grids whose x rows start on 16-byte boundaries (nx a multiple of 8):
    shape 0 runs the staged pair kernel (64x4 columns, two cells a thread,
    the 16-bit values of interior planes staged in shared memory), 1 the pair
    kernel (64x4), 2 the one-cell kernel (32x8 columns), 3 the TMA-staged
    kernel (32x8 columns).  Columns wider or taller than the grid,
    partial columns at the far edges, the periodic halo of every edge column
    and both wall planes; a state that varies from cell to cell and a
    flagged force, against the oracle with the bounds of test_free_steps."""
    nx, ny, nz = dims
    N = nx * ny * nz
    lat = fsi.Lattice(nx, ny, nz, 0.8, (4e-3, -1.5e-3, 0.0), (2e-6, 0.0, -1e-6), storage=storage)
    fsi.lb_set_shape(lat, shape)
    lat.init_shear()
    rng = np.random.default_rng(13)
    live = 0 if lat.velocity().data_ptr() == lat.m[0].data_ptr() else 1
    cur = lat.f[live]
    noise = torch.from_numpy((3e-5 * rng.standard_normal(tuple(cur.shape))).astype(np.float32)).cuda()
    cur.copy_((cur.float() + noise * (1.0 if storage == "bf16" else 2.0 ** lat.p.fp16_exponent)).to(cur.dtype))
    f0 = lat.export().cpu().numpy().astype(np.float64)
    flags = (rng.uniform(size=ny * nz) < 0.4).astype(np.int32)
    g = np.zeros((N, 4), np.float32)
    rows = np.repeat(flags, nx).astype(bool)
    g[rows, :3] = (1e-5 * rng.standard_normal((rows.sum(), 3))).astype(np.float32)
    g64 = np.ascontiguousarray(g[:, :3].astype(np.float64).T).ravel()
    _, w = oracle.lattice()
    p = oracle.lb_params(nx, ny, nz, f32(0.8), (f32(4e-3), f32(-1.5e-3), 0.0), (f32(2e-6), 0.0, f32(-1e-6)))
    f = (f0 + w[:, None]).ravel()
    n = 6
    fneq_max = 0.0
    for _ in range(n):
        lat.g.copy_(torch.from_numpy(g))
        lat.flags.copy_(torch.from_numpy(flags))
        lat.step(1)
        f, rho, v = oracle.lb_step(p, f, g64)
        fs = f.reshape(19, N) - w[:, None]
        fneq_max = max(fneq_max, float(np.abs(fs - feq_shifted(rho, v.reshape(3, N))).max()))
    torch.cuda.synchronize()
    bound_f = 1e-5 * np.abs(fs).max() + n * UNIT[storage] * fneq_max
    err_f = np.abs(lat.export().cpu().numpy() - fs).max()
    assert err_f <= bound_f, (err_f, bound_f)
    m = lat.velocity().cpu().numpy()
    assert np.abs(m[:, :3].T - v.reshape(3, N)).max() <= 10 * bound_f
    assert np.all(lat.g.cpu().numpy()[rows] == 0)
    assert fsi.lb_get_shape(lat) == shape


def test_shapes_share_one_state():
    """All 16-bit kernels read and write the same stored state with the same
    per-cell operation sequence: alternating them step by step gives the
    populations of one kernel bit for bit."""
    dims = (64, 24, 10)
    runs = []
    for order in ([2] * 8, [0, 2, 1, 3, 0, 2, 1, 3]):
        lat = fsi.Lattice(*dims, 0.8, (4e-3, 0.0, 0.0), storage="bf16")
        lat.init_shear()
        for s in order:
            fsi.lb_set_shape(lat, s)
            lat.step(1)
        runs.append(lat.export().cpu().numpy())
    assert np.array_equal(runs[0], runs[1])


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
@pytest.mark.parametrize("walls", [0, 1])
@pytest.mark.parametrize("dims", [(64, 24, 10), (136, 9, 3), (8, 5, 4), (16, 3, 5), (8, 2, 2), (54, 20, 9),
                                  (53, 17, 13), (130, 7, 5), (3, 5, 4), (1, 4, 3)])
def test_every_shape_bit_identical(storage, walls, dims):
    """Every launch shape (staged pair, pair, one-cell and TMA-staged kernels
    where nx is a multiple of 8; pair and one-cell kernels otherwise) gives
    the same populations and moment records bit for bit: even nx (the pair
    kernel's 32-bit words; a multiple of 8 takes the staged kernels, with
    windows wrapped per chunk at both x edges and per row in y; one interior
    plane, none), odd nx (the last pair of a row has one cell), more than
    two pair columns along x, grids narrower than one column, both wall
    modes, a state that varies from cell to cell and flagged forces, over 4
    steps."""
    nx, ny, nz = dims
    N = nx * ny * nz
    rng = np.random.default_rng(nx * 100 + ny)
    flags = (rng.uniform(size=ny * nz) < 0.4).astype(np.int32)
    g = np.zeros((N, 4), np.float32)
    rows = np.repeat(flags, nx).astype(bool)
    g[rows, :3] = (1e-5 * rng.standard_normal((rows.sum(), 3))).astype(np.float32)
    noise = (3e-5 * rng.standard_normal((19, N))).astype(np.float32)
    out = []
    for shape in range(4):
        lat = fsi.Lattice(nx, ny, nz, 0.8, (4e-3, -1.5e-3, 0.0), (2e-6, 0.0, -1e-6), storage=storage, walls=walls)
        fsi.lb_set_shape(lat, shape)
        lat.init_shear()
        live = 0 if lat.velocity().data_ptr() == lat.m[0].data_ptr() else 1
        cur = lat.f[live]
        scale = 1.0 if storage == "bf16" else 2.0 ** lat.p.fp16_exponent
        cur.copy_((cur.float() + torch.from_numpy(noise).cuda() * scale).to(cur.dtype))
        for _ in range(4):
            lat.g.copy_(torch.from_numpy(g))
            lat.flags.copy_(torch.from_numpy(flags))
            lat.step(1)
        torch.cuda.synchronize()
        out.append((lat.export().cpu().numpy(), lat.velocity().cpu().numpy()))
    for f, m in out[1:]:
        assert np.array_equal(f, out[0][0])
        assert np.array_equal(m, out[0][1])
    assert np.isfinite(out[0][0]).all()
