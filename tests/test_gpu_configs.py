"""The large configurations at their full sizes.

Surrogate channel (256x128x128, 100 platelets of 2562 nodes): small enough for
the FP64 oracle, so two coupled steps of the plain FP32 form are compared with
it element by element (tolerance 1e-5, as for the channel), and the surrogate
force on 400 sampled nodes with the reference network, node by node.

Full scale (512x256x256 = 33.5 M cells, 500 platelets with SCE and 2.5 M
receptor sites): the oracle would need ~10 GB of host
arrays per step, so the test checks what holds at any size, on the GPU run
itself:
  * a developed Couette flow is a fixed point of the lattice step (exact for
    BGK with halfway bounce-back), so 5 steps of the 33.5 M-cell lattice leave
    every population within FP32 rounding of its start;
  * the coupled step (BF16 storage, surrogate membrane, Philox bonds) keeps
    the mass of the lattice (FP64 device sums) and leaves finite positions;
  * the membrane's internal forces sum to zero per platelet (translation
    invariance of the energy);
  * spreading conserves force: the FP64 sum of the spread field equals the
    FP64 sum of the nodal forces of the nodes out of reach of the walls;
  * the bond state is consistent: every ligand's count equals the number of
    sites bound to it and stays <= 4;
  * the surrogate force on sampled nodes matches the reference network."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_1312_2234_b300 import fsi, surrogate, workload

pytestmark = pytest.mark.gpu


def f32_workload(w):
    w = dict(w)
    w["membrane"] = {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in w["membrane"].items()}
    g = dict(w["grid"])
    g["tau"] = float(np.float32(g["tau"]))
    g["u_top"] = tuple(float(np.float32(u)) for u in g["u_top"])
    w["grid"] = g
    return w


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def bf16_round(a):
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def check_surrogate_sampled(w, X, params_np, n_sample=400, seed=0, amp=3e-3):
    """Surrogate force (exact global terms removed) on sampled nodes against
    the reference network evaluated node by node on the BF16-rounded weights,
    at X plus a deformation of the membrane nodes (Gaussian, amp lattice
    units): the surrogate's bending angles are accurate to ~1e-7 absolute, so
    a state a few steps from rest (strains ~1e-7) would compare rounding."""
    m = w["mesh"]
    n = w["M"]
    mem_nodes = np.asarray(m["is_membrane"]).astype(bool)
    D = np.random.default_rng(seed + 1).standard_normal((3, n)) * mem_nodes
    X = (np.asarray(X).reshape(3, n) + amp * D).ravel()
    sg = fsi.Surrogate(m, "bf16")
    params = fsi.SurrogateParams()
    params.set(params_np)
    mem = fsi.Membrane(w["membrane"], m)
    glob = fsi.Membrane(dict(w["membrane"], k_spring=0.0, k_t=0.0, k_b=0.0), m)
    Xd = torch.as_tensor(X).cuda()
    Fs = torch.zeros(3 * n, device="cuda")
    Fg = torch.zeros(3 * n, device="cuda")
    sg.forces(params, mem, Xd, Fs)
    glob.forces(Xd, Fg)
    loc = (Fs - Fg).reshape(3, n).cpu().numpy()
    rng = np.random.default_rng(seed)
    ring, deg = mlp.one_rings(m["tri"], n)
    nodes = np.sort(rng.choice(np.where(deg > 0)[0], size=n_sample, replace=False))
    pr = dict(params_np)
    for k in ("W1", "W2", "W3"):
        pr[k] = bf16_round(params_np[k])
    # a node's force comes from its own row and its neighbours' rows
    Xn, X0n = X.reshape(3, n).T, m["X0"].reshape(3, n).T
    ref = np.zeros((len(nodes), 3))
    for q, v in enumerate(nodes):
        rows = np.concatenate([[v], ring[v, :deg[v]]])
        ref[q] = mlp.predict_forces(pr, Xn, X0n, ring, deg, rows)[v]
    assert sg.status() == 0
    # the global terms cancel to FP32 rounding of the larger of the two force
    # fields: bound the comparison by that as well
    floor = 2e-6 * float(Fg.abs().max())
    err = np.abs(loc[:, nodes].T - ref).max()
    assert err <= 2e-2 * np.abs(ref).max() + floor, (err, np.abs(ref).max(), floor)


def test_surrogate_channel_full_size():
    w = f32_workload(workload.config_surrogate(seed=0))
    sim = fsi.Simulation(w)
    ora = oracle.Sim(w)
    X0 = w["X"].copy()
    steps = 2
    sim.step(steps)
    for _ in range(steps):
        ora.step()
    torch.cuda.synchronize()
    assert rel(sim.X.cpu().numpy() - X0, ora.X - X0) < 1e-5
    assert rel(sim.U.cpu().numpy(), ora.U) < 1e-5
    _, wq = oracle.lattice()
    assert rel(sim.lattice.current().cpu().numpy(), ora.f.reshape(19, -1) - wq[:, None]) < 1e-5
    rng = np.random.default_rng(1)
    p = surrogate.init_params(rng, in_scale=rng.uniform(0.5, 2, 42), out_scale=rng.uniform(0.5, 2, 18))
    check_surrogate_sampled(w, sim.X.cpu().numpy(), p)


def test_full_scale_invariants():
    w = workload.config_full(seed=0)
    g = w["grid"]
    # Couette fixed point of the full-size lattice, FP32 storage
    lat = fsi.Lattice(g["nx"], g["ny"], g["nz"], g["tau"], g["u_top"])
    lat.init_shear()
    f0 = lat.current().clone()
    lat.step(5)
    torch.cuda.synchronize()
    assert float((lat.current() - f0).abs().max()) <= 1e-5 * float(f0.abs().max())
    del lat, f0
    torch.cuda.empty_cache()

    # the coupled step: BF16 storage, surrogate membrane, Philox bonds
    rng = np.random.default_rng(2)
    p = surrogate.init_params(rng)
    p["W3"] *= 1e-3     # a small untrained network keeps the run physical
    params = fsi.SurrogateParams()
    params.set(p)
    sim = fsi.Simulation(w, storage="bf16")
    sg = fsi.Surrogate(w["mesh"], "bf16")
    fsi.sim_set_surrogate(sim, sg, params)
    m0 = sim.lattice.moments_fp64()[0]
    sim.step(3)
    torch.cuda.synchronize()
    assert torch.isfinite(sim.X).all()
    assert abs(sim.lattice.moments_fp64()[0] - m0) < 1e-6 * m0
    assert sg.status() == 0
    # bonds: counts match the bound sites, capacity kept
    bound = sim.bonds.bound.cpu().numpy()
    counts = np.bincount(bound[bound >= 0], minlength=sim.bonds.lig_count.numel())
    assert np.array_equal(counts, sim.bonds.lig_count.cpu().numpy())
    assert counts.max(initial=0) <= w["bonds"]["max_per_ligand"]

    # membrane internal forces sum to zero per platelet (no wall term)
    X = sim.X
    M = w["M"]
    inner = fsi.Membrane(dict(w["membrane"], rep_F0=0.0), w["mesh"])
    F = torch.zeros(3 * M, device="cuda")
    inner.forces(X, F)
    plt = torch.as_tensor(np.asarray(w["mesh"]["node_plt"]), device="cuda", dtype=torch.long)
    Fd = F.double().reshape(3, M)
    sums = torch.zeros(3, int(w["mesh"]["n_plt"]), dtype=torch.float64, device="cuda")
    sums.index_add_(1, plt, Fd)
    scale = torch.zeros_like(sums).index_add_(1, plt, Fd.abs())
    assert float((sums.abs() / scale.clamp_min(1e-300)).max()) < 1e-5

    # spreading conserves force for nodes whose support stays off the walls
    # (the support is cut at the walls): spread only those
    z = X.reshape(3, M)[2]
    far = ((z > 1.5) & (z < g["nz"] - 2.5)).float()
    F2 = (F.reshape(3, M) * far).reshape(-1).contiguous()
    lat = fsi.Lattice(g["nx"], g["ny"], g["nz"], g["tau"], g["u_top"])
    fsi.ib_spread(lat.h, X, F2, M)
    torch.cuda.synchronize()
    assert torch.allclose(lat.g[:, :3].double().sum(0), F2.double().reshape(3, M).sum(1), rtol=0,
                          atol=1e-5 * float(F2.abs().sum()))
    del lat

    # surrogate force on sampled nodes
    check_surrogate_sampled(w, X.cpu().numpy(), p, n_sample=300)


def lattice_block(f, nx, ny, i, j, k0, wq):
    """The 3x3x3 block of full populations (FP64, f~ + w) around column
    (i, j), planes k0 .. k0 + 2, periodic in x and y: [19][3][3][3]."""
    ii = (np.arange(i - 1, i + 2) % nx)
    jj = (np.arange(j - 1, j + 2) % ny)
    b = f[:, k0:k0 + 3][:, :, jj][:, :, :, ii].astype(np.float64)
    return b + wq[:, None, None, None]


def test_full_scale_sampled_parity():
    """Sampled outputs at the full size, in the launch configuration the
    benchmark times (512x256x256 lattice, 500 platelets): the lattice step
    of cells in the bulk, on both walls and under the platelets' spread
    force, each recomputed by the oracle from its 3x3x3 neighbourhood (a cell
    pulls only from its neighbours, so the oracle's step of the block gives
    the centre cell's exact FP64 result); and the membrane force of whole
    platelets, each by the oracle's membrane of that platelet alone.  Bounds
    as in the element-wise tests: 1e-5 of the largest population or force."""
    w = f32_workload(workload.config_full(seed=0))
    g = w["grid"]
    nx, ny, nz = g["nx"], g["ny"], g["nz"]
    N = nx * ny * nz
    M = w["M"]
    sim = fsi.Simulation(w)
    sim.step(3)                                  # the platelets disturb the flow
    # membrane forces on a deformed state, then spread them and take one
    # lattice step on the simulation's own lattice
    rng = np.random.default_rng(7)
    Xh = sim.X.cpu().numpy() + 0.01 * rng.standard_normal(3 * M)
    X = torch.from_numpy(Xh).cuda()
    F = torch.zeros(3 * M, device="cuda")
    fsi.membrane_forces(sim.membrane.h, X, F)
    lat = sim.lattice
    fsi.ib_spread(lat.h, X, F, M)
    torch.cuda.synchronize()
    f_pre = lat.current().cpu().numpy().reshape(19, nz, ny, nx)
    gf = lat.g[:, :3].cpu().numpy().astype(np.float64).T.reshape(3, nz, ny, nx)
    fsi.lb_step(lat.h, 1)
    torch.cuda.synchronize()
    f_post = lat.current().cpu().numpy().reshape(19, nz, ny, nx)
    _, wq = oracle.lattice()
    wq = np.asarray(wq)
    scale = float(np.abs(f_post).max())
    forced = np.argwhere(np.abs(gf).sum(0) > 0)
    cells = [tuple(c) for c in forced[rng.choice(len(forced), 120, replace=False)]]
    cells += [(int(rng.integers(1, nz - 1)), int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(120)]
    cells += [(0, int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(40)]
    cells += [(nz - 1, int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(40)]
    worst = 0.0
    for (k, j, i) in cells:
        k0 = min(max(k - 1, 0), nz - 3)
        kc = k - k0
        p = oracle.lb_params(3, 3, 3, g["tau"], g["u_top"])
        fb = lattice_block(f_pre, nx, ny, i, j, k0, wq)
        gb = gf[:, k0:k0 + 3][:, :, (np.arange(j - 1, j + 2) % ny)][:, :, :, (np.arange(i - 1, i + 2) % nx)]
        out, _, _ = oracle.lb_step(p, np.ascontiguousarray(fb).ravel(), np.ascontiguousarray(gb).ravel())
        want = out.reshape(19, 3, 3, 3)[:, kc, 1, 1] - wq
        worst = max(worst, float(np.abs(f_post[:, k, j, i] - want).max()))
    print("full-scale lattice sampled parity: %d cells (%d forced), max err %.2e of max |f~|"
          % (len(cells), 120, worst / scale))
    assert worst < 1e-5 * scale

    # membrane: whole platelets by the oracle's membrane of that platelet alone
    m = w["mesh"]
    plt = np.asarray(m["node_plt"])
    tri = np.asarray(m["tri"]).reshape(-1, 3)
    pairs = np.asarray(m["pairs"]).reshape(-1, 2)
    Fg = F.cpu().numpy().reshape(3, M)
    X0 = np.asarray(m["X0"]).reshape(3, M)
    Xd = Xh.reshape(3, M)
    for pid in (0, 137, 499):
        nodes = np.nonzero(plt == pid)[0]
        lo, hi = nodes[0], nodes[-1] + 1
        assert np.array_equal(nodes, np.arange(lo, hi))
        t = tri[(tri >= lo).all(1) & (tri < hi).all(1)] - lo
        pr = pairs[(pairs >= lo).all(1) & (pairs < hi).all(1)] - lo
        mesh = oracle.Mesh(np.ascontiguousarray(X0[:, lo:hi]).ravel(), t, pr, np.zeros(hi - lo, np.int32),
                           np.asarray(m["is_membrane"])[lo:hi], 1)
        Fo = mesh.forces(w["membrane"], np.ascontiguousarray(Xd[:, lo:hi]).ravel()).reshape(3, -1)
        err = rel(Fg[:, lo:hi], Fo)
        print("full-scale membrane parity, platelet %d: %.2e" % (pid, err))
        assert err < 1e-5
