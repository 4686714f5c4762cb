"""GPU parity of the learned membrane surrogate against the FP64 reference
(oracle/mlp.py): element strains, moduli scales and inputs, training
records, forward output and every gradient in the FP32 check mode (CUDA
cores, tolerance 1e-5 of the largest entry of each tensor) and on the BF16
tensor cores (1e-2), Adam, the exact global terms of the surrogate force,
the stress-to-force path against the plain solver, training, the surrogate
form against the plain method on the same run, and the fallback to the plain
solver.

Tolerances.  FP32 check mode: strains are formed from small differences of
the split positions (relative accuracy ~1e-7 of each strain; the bending
angle ~1e-7 absolute), the layers accumulate <= 128 products in FP32, so
outputs and gradients agree with FP64 to ~1e-6 of their largest entry; the
bound is 1e-5.  BF16 mode: operands and activations are rounded to BF16
(2^-9 relative) before each product; the reference is evaluated on the same
BF16-rounded inputs and weights, so what remains is the rounding of the two
hidden activations and of the backward signals, a few 2^-9 of the largest
entry: the bound is 1e-2."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_1312_2234_b300 import fsi, surrogate, workload

pytestmark = pytest.mark.gpu


def bf16_round(a):
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def f32(d):
    return {k: (float(np.float32(v)) if isinstance(v, float) else v) for k, v in d.items()}


def mesh_and_state(seed=4, amp=0.03, level=2):
    w = workload.tiny(seed=seed, level=level)
    m = w["mesh"]
    rng = np.random.default_rng(seed)
    X = w["X"] + amp * rng.standard_normal(w["X"].shape)
    return w, m, X


def oracle_rows(m):
    n = m["node_plt"].size
    ring, deg = mlp.one_rings(m["tri"], n)
    nodes = np.where((deg > 0) & (np.asarray(m["is_membrane"]) > 0))[0]
    return ring, deg, nodes


def random_scales(rng, p):
    p["in_scale"] = rng.uniform(0.5, 2.0, mlp.N_IN)
    p["in_shift"] = rng.uniform(-0.5, 0.5, mlp.N_IN)
    p["out_scale"] = rng.uniform(0.5, 2.0, mlp.N_OUT)
    p["tgt_scale"] = rng.uniform(0.5, 2.0, mlp.N_OUT)
    return p


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_strains_and_inputs(mode):
    w, m, X = mesh_and_state()
    rng = np.random.default_rng(1)
    p = random_scales(rng, mlp.init_params(rng))
    p["in_scale"][:18] = rng.uniform(5.0, 50.0, 18)
    params = fsi.SurrogateParams()
    params.set(p)
    sg = fsi.Surrogate(m, mode)
    feat, xs, ms = sg.features(params, torch.as_tensor(X).cuda())
    ring, deg, nodes = oracle_rows(m)
    assert sg.rows == len(nodes)
    n = m["node_plt"].size
    x_or, m_or, r_or = mlp.strains(X.reshape(3, n).T, m["X0"].reshape(3, n).T, ring, deg, nodes)
    xs = xs.cpu().numpy()[:sg.rows]
    for kind in surrogate.KINDS:
        assert rel(xs[:, kind], x_or[:, kind]) < 1e-5
    assert rel(ms.cpu().numpy()[:sg.rows], m_or) < 1e-6
    f_or = mlp.inputs(p, x_or, r_or)
    got = feat.float().cpu().numpy()[:sg.rows]
    assert np.all(got[:, mlp.N_IN:] == 0)
    if mode == "fp32":
        assert np.max(np.abs(got[:, :mlp.N_IN] - f_or)) < 1e-5 * max(1.0, np.abs(f_or).max())
    else:
        assert np.all(np.abs(got[:, :mlp.N_IN] - f_or) <= 2.0 ** -8 * np.abs(f_or) + 1e-4)


def test_training_records_are_the_plain_stresses():
    w, m, X = mesh_and_state(seed=5)
    rng = np.random.default_rng(2)
    p = random_scales(rng, mlp.init_params(rng))
    params = fsi.SurrogateParams()
    params.set(p)
    sg = fsi.Surrogate(m, "fp32")
    mp = f32(w["membrane"])
    feat, xs, ms = sg.features(params, torch.as_tensor(X).cuda())
    t = sg.targets(params, mp, xs, ms).cpu().numpy()[:sg.rows]
    ring, deg, nodes = oracle_rows(m)
    n = m["node_plt"].size
    x_or, m_or, _ = mlp.strains(X.reshape(3, n).T, m["X0"].reshape(3, n).T, ring, deg, nodes)
    pf = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}
    a, b = mlp.targets(pf, x_or, m_or, mlp.exact_stresses(x_or, m_or, mp))
    for kind in surrogate.KINDS:
        assert rel(t[:, :18][:, kind], a[:, kind]) < 1e-5
        assert rel(t[:, 18:][:, kind], b[:, kind]) < 1e-5


def random_problem(batch, seed):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(rng)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    f = rng.standard_normal((batch, mlp.N_IN))
    a = rng.standard_normal((batch, mlp.N_OUT))
    b = rng.standard_normal((batch, mlp.N_OUT))
    return p, f, a, b


def gpu_grads(p, f, a, b, mode):
    params = fsi.SurrogateParams()
    params.set(p)
    B = f.shape[0]
    dt = torch.bfloat16 if mode == "bf16" else torch.float32
    feat = torch.zeros(B, fsi.SG["IN_PAD"], dtype=dt, device="cuda")
    feat[:, :mlp.N_IN] = torch.as_tensor(f, dtype=torch.float32).to(dt)
    tgt = torch.as_tensor(np.ascontiguousarray(np.hstack([a, b]), dtype=np.float32)).cuda()
    batch = fsi.SurrogateBatch(B)
    loss = batch.grad(params, feat, tgt, mode)
    torch.cuda.synchronize()
    assert batch.status() == 0
    return params.grads(), float(loss.item()), params


def r32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("B", [128, 384])
def test_gradients_fp32_check_mode(B):
    p, f, a, b = random_problem(B, 7)
    g, loss, _ = gpu_grads(p, f, a, b, "fp32")
    pf = {k: (r32(v) if k in mlp.TRAINED else v) for k, v in p.items()}
    o, cache = mlp.forward(pf, r32(f))
    g_or = mlp.backward(pf, cache, o, r32(a), r32(b))
    ref = mlp.loss(o, r32(a), r32(b))
    assert abs(loss - ref) <= 1e-5 * ref
    for k in mlp.TRAINED:
        assert rel(g[k], g_or[k]) < 1e-5, k


@pytest.mark.parametrize("B", [128, 1024])
def test_gradients_bf16_tensor_cores(B):
    p, f, a, b = random_problem(B, 8)
    g, loss, _ = gpu_grads(p, f, a, b, "bf16")
    pb = dict(p)
    for k in ("W1", "W2", "W3"):
        pb[k] = bf16_round(p[k])
    for k in ("b1", "b2", "b3"):
        pb[k] = r32(p[k])
    o, cache = mlp.forward(pb, bf16_round(f))
    g_or = mlp.backward(pb, cache, o, r32(a), r32(b))
    ref = mlp.loss(o, r32(a), r32(b))
    assert abs(loss - ref) <= 1e-2 * ref
    for k in mlp.TRAINED:
        assert rel(g[k], g_or[k]) < 1e-2, (k, rel(g[k], g_or[k]))


def test_adam_matches_reference():
    p, f, a, b = random_problem(256, 9)
    params = fsi.SurrogateParams()
    params.set(p)
    feat = torch.zeros(256, fsi.SG["IN_PAD"], dtype=torch.float32, device="cuda")
    feat[:, :mlp.N_IN] = torch.as_tensor(f, dtype=torch.float32)
    tgt = torch.as_tensor(np.ascontiguousarray(np.hstack([a, b]), dtype=np.float32)).cuda()
    batch = fsi.SurrogateBatch(256)
    pf = {k: (r32(v) if k in mlp.TRAINED else v) for k, v in p.items()}
    state = {}
    # eps well above the FP32 gradient error keeps the update a smooth function
    # of the gradient (with eps ~ 1e-8 a component whose gradient is within
    # rounding of zero could step by +lr on one side and -lr on the other)
    eps = 1e-4
    for _ in range(3):
        batch.grad(params, feat, tgt, "fp32")
        fsi.sg_adam(params, 1e-3, eps=eps)
        o, cache = mlp.forward(pf, r32(f))
        mlp.adam_step(pf, mlp.backward(pf, cache, o, r32(a), r32(b)), state, 1e-3, eps=eps)
    got = params.get()
    for k in mlp.TRAINED:
        assert np.max(np.abs(got[k] - pf[k])) < 1e-5 * max(1.0, np.abs(pf[k]).max()), k


@pytest.mark.parametrize("n_sce,mode", [(8, "bf16"), (0, "bf16"), (0, "fp32")])
def test_global_terms_are_exact(n_sce, mode):
    """A network with zero output leaves exactly the plain solver's global
    area, volume, Morse and wall terms (the area and volume terms and, on a
    mesh without Morse pairs, the wall term applied by the surrogate kernel
    per node)."""
    w = workload.tiny(seed=4, level=2, n_sce=n_sce)
    m = w["mesh"]
    X = w["X"] + 0.03 * np.random.default_rng(4).standard_normal(w["X"].shape)
    assert (len(m["pairs"]) > 0) == (n_sce > 0)
    params = fsi.SurrogateParams()
    p = mlp.init_params(np.random.default_rng(2))
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    params.set(p)
    sg = fsi.Surrogate(m, mode)
    mem = fsi.Membrane(w["membrane"], m)
    Xd = torch.as_tensor(X).cuda()
    F = torch.zeros(3 * sg.n, dtype=torch.float32, device="cuda")
    sg.forces(params, mem, Xd, F)
    mesh = oracle.Mesh(m["X0"], m["tri"], m["pairs"], m["node_plt"], m["is_membrane"], m["n_plt"])
    ref = mesh.forces(mlp.global_params(f32(w["membrane"])), X)
    assert rel(F.cpu().numpy(), ref) < 1e-5
    assert sg.status() == 0


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_exact_moduli_give_the_plain_local_force(mode):
    """Output 1 (zero last layer, unit bias) with out_scale = the stress
    coefficients (k_spring/2, k_t/3, k_b/2): the stresses are the plain ones
    (bending up to sin x - x) and the surrogate's strain gradients and
    scatter reproduce the plain CUDA solver's local force; with W3 = 0 the
    tensor-core path gives o = 1 exactly.  At this deformation the bending
    angles reach ~0.03, where sin x - x is below 2e-4 of the bending stress
    (the FP64 reference gives the same difference)."""
    w, m, X = mesh_and_state(level=3, amp=1e-3)
    mp = f32(w["membrane"])
    p = mlp.init_params(np.random.default_rng(3))
    p["W3"][:] = 0.0
    p["b3"][:] = 1.0
    p["out_scale"] = np.repeat(mlp.stress_coefficients(mp), 6)
    params = fsi.SurrogateParams()
    params.set(p)
    sg = fsi.Surrogate(m, mode)
    Xd = torch.as_tensor(X).cuda()
    glob = fsi.Membrane(surrogate.local_params(w["membrane"]) | {"k_spring": 0.0, "k_t": 0.0, "k_b": 0.0}, m)
    loc = fsi.Membrane(surrogate.local_params(w["membrane"]), m)
    Fs = torch.zeros(3 * sg.n, device="cuda")
    Fl = torch.zeros(3 * sg.n, device="cuda")
    sg.forces(params, glob, Xd, Fs)     # zero global part + surrogate local part
    loc.forces(Xd, Fl)
    assert rel(Fs.cpu().numpy(), Fl.cpu().numpy()) < 1e-4
    assert sg.status() == 0


def test_surrogate_force_matches_reference_network():
    """The surrogate force with a given network, end to end through the
    strains, the tensor-core layers and the stress scatter, against the
    reference network on the BF16-rounded weights."""
    w, m, X = mesh_and_state(level=2)
    rng = np.random.default_rng(3)
    p = random_scales(rng, mlp.init_params(rng))
    p["in_scale"][:18] = rng.uniform(5, 20, 18)
    params = fsi.SurrogateParams()
    params.set(p)
    n = m["node_plt"].size
    ring, deg, nodes = oracle_rows(m)
    mesh = oracle.Mesh(m["X0"], m["tri"], m["pairs"], m["node_plt"], m["is_membrane"], m["n_plt"])
    glob = mesh.forces(mlp.global_params(f32(w["membrane"])), X).reshape(3, n)
    for mode, tol in (("fp32", 1e-5), ("bf16", 2e-2)):
        sg = fsi.Surrogate(m, mode)
        mem = fsi.Membrane(w["membrane"], m)
        F = torch.zeros(3 * n, dtype=torch.float32, device="cuda")
        sg.forces(params, mem, torch.as_tensor(X).cuda(), F)
        loc = F.cpu().numpy().reshape(3, n) - glob
        pr = {k: (r32(v) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
        if mode == "bf16":
            for k in ("W1", "W2", "W3"):
                pr[k] = bf16_round(p[k])
        ref = mlp.predict_forces(pr, X.reshape(3, n).T, m["X0"].reshape(3, n).T, ring, deg, nodes)
        assert rel(loc.T, ref) < tol, (mode, rel(loc.T, ref))


def trained(w, steps=2000, seed=0, flow_steps=0):
    """A surrogate trained on perturbed states of the workload's platelets
    (and, with flow_steps, on snapshots of a plain coupled run)."""
    m = w["mesh"]
    rng = np.random.default_rng(seed)
    params = fsi.SurrogateParams()
    params.set(surrogate.init_params(rng))
    sg = fsi.Surrogate(m, "bf16")
    snaps = [w["X"]]
    if flow_steps:
        sim = fsi.Simulation(w)
        for _ in range(4):
            sim.step(flow_steps // 4)
            snaps.append(sim.X.cpu().numpy())
    states = surrogate.perturbed_states(snaps, m, amplitudes=(0.001, 0.01), copies=8, rng=rng)
    data = surrogate.prepare(sg, params, w["membrane"], states)
    untrained = fsi.SurrogateParams()
    untrained.set(params.get())
    hist = surrogate.train(params, data, steps, batch=1024, lr=2e-3, log_every=100)
    return params, untrained, sg, hist


def local_error(sg, P, w, X):
    m = w["mesh"]
    n = sg.n
    mem = fsi.Membrane(w["membrane"], m)
    local = fsi.Membrane(surrogate.local_params(w["membrane"]), m)
    mask = torch.as_tensor(np.asarray(m["is_membrane"]).astype(bool)).cuda()
    Fl = torch.zeros(3 * n, device="cuda")
    Fp = torch.zeros(3 * n, device="cuda")
    Fs = torch.zeros(3 * n, device="cuda")
    local.forces(X, Fl)             # plain local terms
    mem.forces(X, Fp)               # plain total
    sg.forces(P, mem, X, Fs)        # exact global + surrogate local
    return surrogate.rel_force_error(Fs - Fp + Fl, Fl, mask)


def test_training_reaches_the_stresses_on_fresh_states():
    """Training lowers the loss by more than 100x; on fresh perturbed states
    the trained surrogate's local force is within 5 % of the largest local
    force, the untrained network's is not (the method without the learned
    part, which has no local force, is off by exactly 1)."""
    w = workload.tiny(seed=5, level=3)
    params, untrained, sg, hist = trained(w)
    assert hist[-1][1] < 0.01 * hist[0][1], hist
    rng = np.random.default_rng(11)
    test_states = surrogate.perturbed_states([w["X"]], w["mesh"], amplitudes=(0.003,), copies=3, rng=rng)[1:]
    errs = {name: max(local_error(sg, P, w, torch.as_tensor(X).cuda()) for X in test_states)
            for name, P in (("trained", params), ("untrained", untrained))}
    assert errs["trained"] < 0.05, errs
    assert errs["untrained"] > 0.3, errs


def test_surrogate_form_against_the_plain_method():
    """The same coupled run with the plain membrane solver and with the
    trained surrogate (trained on perturbed snapshots of a plain run of this
    chamber): after 300 steps the surrogate's local force on the surrogate
    run's state is within 5 % of the plain local force there, and the node
    displacements and velocities of the two runs agree within 5 % of the
    plain run's largest entries."""
    w = workload.tiny(seed=5, level=3, shear=3e4)
    params, untrained, sg, hist = trained(w, flow_steps=400)
    plain = fsi.Simulation(w)
    sim = fsi.Simulation(w)
    fsi.sim_set_surrogate(sim, sg, params)
    plain.step(300)
    sim.step(300)
    torch.cuda.synchronize()
    assert torch.isfinite(sim.X).all()
    e = local_error(sg, params, w, sim.X)
    assert e < 0.05, e
    X0 = torch.as_tensor(w["X"]).cuda()
    dp, ds = plain.X - X0, sim.X - X0
    assert float((ds - dp).abs().max() / dp.abs().max()) < 0.05
    assert float((sim.U - plain.U).abs().max() / plain.U.abs().max()) < 0.05
    assert sg.status() == 0


def test_coupled_step_with_surrogate_and_fallback():
    """The judge at its default 5 % tolerance: an untrained network falls
    back to the plain solver at the first check, the trained one keeps
    running on the surrogate."""
    w = workload.tiny(seed=5, level=3)
    params, untrained, sg, hist = trained(w)
    m = w["mesh"]
    plain = fsi.Membrane(w["membrane"], m)
    # a network that is far off triggers the fallback at the first check
    sim_bad = fsi.Simulation(w)
    judge = surrogate.Judge(sim_bad, sg, untrained, plain, m["is_membrane"], every=5, tol=0.05)
    assert not judge.step(10)
    X_after = sim_bad.X.clone()
    # with the trained network the coupled step runs on the surrogate
    sim = fsi.Simulation(w)
    judge = surrogate.Judge(sim, sg, params, plain, m["is_membrane"], every=10, tol=0.05)
    assert judge.step(40), judge.errors
    assert max(judge.errors) < 0.05
    torch.cuda.synchronize()
    assert torch.isfinite(sim.X).all()
    assert judge.errors and all(np.isfinite(judge.errors))
    assert sg.status() == 0
    assert torch.isfinite(X_after).all()


@pytest.mark.parametrize("amp", [1e-6, 1e-4])
def test_strains_keep_their_accuracy_at_small_deformations(amp):
    """The strains are formed from small quantities (split positions minus
    split rest edges), so they keep their relative accuracy where forming
    them from FP32 positions would lose them: at a displacement of 1e-6 of
    the platelet radius the stretch and area strains agree with the FP64
    reference to 1e-3 of the largest."""
    w = workload.tiny(seed=4, level=2)
    m = w["mesh"]
    n = m["node_plt"].size
    rng = np.random.default_rng(9)
    X = m["X0"] + amp * rng.standard_normal(m["X0"].shape)
    params = fsi.SurrogateParams()
    params.set(mlp.init_params(rng))
    sg = fsi.Surrogate(m, "fp32")
    feat, xs, ms = sg.features(params, torch.as_tensor(X).cuda())
    ring, deg, nodes = oracle_rows(m)
    x_or, _, _ = mlp.strains(X.reshape(3, n).T, m["X0"].reshape(3, n).T, ring, deg, nodes)
    got = xs.cpu().numpy()[:sg.rows]
    for kind in surrogate.KINDS[:2]:
        assert rel(got[:, kind], x_or[:, kind]) < 1e-3


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The bounded mbarrier wait the tensor-core kernels use gives up after
    its limit on a phase nothing completes (no asynchronous copy or MMA is in
    flight) and reports PFSI_ERR_TIMEOUT; the context then runs the
    tensor-core gradients as before."""
    assert fsi.wait_selftest(1000)
    assert fsi.wait_selftest(1)
    torch.cuda.synchronize()
    test_gradients_bf16_tensor_cores(128)
