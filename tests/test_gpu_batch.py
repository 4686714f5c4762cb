"""Batches of independent chambers (one CUDA graph per step: each kernel of
the step one launch for a group of chambers, the lattice update one batched
launch per storage mode) and the launch-shape autotuners.

A chamber stepped inside a batch computes what it computes alone: the same
kernels on its own buffers.  Force spreading adds tile sums with
floating-point atomics whose order is not fixed, so two runs agree to FP32
rounding (1e-6 of the largest entry here), not bit for bit.  The launch
shapes do not change any cell's arithmetic: every shape gives bit-identical
populations."""
import numpy as np
import pytest
import torch

import oracle
from paper_1312_2234_b300 import fsi, workload

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


def small_chambers():
    return [f32_workload(workload.tiny(seed=1, nx=24, ny=20, nz=18, shear=2.0e4)),
            f32_workload(workload.tiny(seed=2, nx=30, ny=17, nz=21, shear=3.5e4)),
            f32_workload(workload.tiny(seed=3, nx=19, ny=26, nz=16, shear=1.0e4))]


@pytest.mark.parametrize("k,layout", [(1, None), (2, None), (1, (1, 0)), (2, (2, 3)), (1, (0, 0))])
def test_batch_matches_individual_chambers_and_oracle(k, layout):
    """layout (groups, blocks per SM): one group (every kernel one launch for
    all chambers), two groups, per-chamber chains; None: the default."""
    ws = small_chambers()
    storage = ["fp32", "bf16", "fp32"]
    batched = [fsi.Simulation(w, storage=s) for w, s in zip(ws, storage)]
    alone = [fsi.Simulation(w, storage=s) for w, s in zip(ws, storage)]
    batch = fsi.Batch(batched, steps_per_graph=k)
    if layout is not None:
        batch.set_layout(*layout)
    steps = 4
    batch.step(steps)
    for s in alone:
        s.step(steps)
    torch.cuda.synchronize()
    for w, a, b in zip(ws, batched, alone):
        assert a.step_index == b.step_index == steps
        X0 = w["X"]
        assert rel(a.X.cpu().numpy() - X0, b.X.cpu().numpy() - X0) < 1e-6
        assert rel(a.U.cpu().numpy(), b.U.cpu().numpy()) < 1e-6
        assert rel(a.lattice.export().cpu().numpy(), b.lattice.export().cpu().numpy()) < 1e-6
        if a.bonds is not None:
            assert np.array_equal(a.bonds.bound.cpu().numpy(), b.bonds.bound.cpu().numpy())
    # the FP32 chambers against the oracle
    for i in (0, 2):
        ora = oracle.Sim(ws[i])
        for _ in range(steps):
            ora.step()
        X0 = ws[i]["X"]
        assert rel(batched[i].X.cpu().numpy() - X0, ora.X - X0) < 1e-5
        assert rel(batched[i].U.cpu().numpy(), ora.U) < 1e-5


@pytest.mark.parametrize("groups", [1, 2])
def test_group_with_a_finite_element_chamber(groups):
    """A chamber with the finite-element bending keeps its group on
    per-chamber branches (the plain groups launch each kernel once for all
    their chambers); every chamber still matches its lone steps."""
    ws = small_chambers()
    w = workload.tiny(seed=4, level=2, n_sce=20, n_sites=60, shear=3.0e4)
    w["membrane"] = dict(w["membrane"], bending="fem", k0=100.0 * w["membrane"]["k0"])
    ws.append(f32_workload(w))
    batched = [fsi.Simulation(w) for w in ws]
    alone = [fsi.Simulation(w) for w in ws]
    batch = fsi.Batch(batched, steps_per_graph=2)
    batch.set_layout(groups, 0)
    batch.step(4)
    for s in alone:
        s.step(4)
    torch.cuda.synchronize()
    for w, a, b in zip(ws, batched, alone):
        X0 = w["X"]
        assert rel(a.X.cpu().numpy() - X0, b.X.cpu().numpy() - X0) < 1e-6
        assert rel(a.U.cpu().numpy(), b.U.cpu().numpy()) < 1e-6
        if a.bonds is not None:
            assert np.array_equal(a.bonds.bound.cpu().numpy(), b.bonds.bound.cpu().numpy())


def test_a_chamber_stepped_alone_stops_the_batch():
    sims = [fsi.Simulation(w) for w in small_chambers()[:2]]
    batch = fsi.Batch(sims)
    batch.step(1)
    sims[0].step(1)
    with pytest.raises(RuntimeError, match="parit"):
        batch.step(1)


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp16"])
def test_every_launch_shape_gives_the_same_populations(storage):
    out = []
    for shape in range(4):
        lat = fsi.Lattice(53, 37, 29, 0.8, (3e-3, 1e-3, 0.0), (1e-6, 0.0, 0.0), storage=storage)
        fsi.lb_set_shape(lat, shape)
        lat.init_shear()
        lat.step(3)
        out.append(lat.export().cpu().numpy())
    for o in out[1:]:
        assert np.array_equal(o, out[0])


def test_autotune_picks_a_shape_and_keeps_results():
    lat = fsi.Lattice(96, 64, 48, 0.8, (2e-3, 0.0, 0.0), storage="bf16")
    shape, ms = fsi.lb_autotune(lat, reps=3)
    assert 0 <= shape < 4 and ms > 0
    lat.init_shear()
    lat.step(2)
    ref = fsi.Lattice(96, 64, 48, 0.8, (2e-3, 0.0, 0.0), storage="bf16")
    ref.init_shear()
    ref.step(2)
    assert np.array_equal(lat.export().cpu().numpy(), ref.export().cpu().numpy())


def test_batched_chambers_full_size():
    """The batched workload at full size: 64 chambers of 48..128 cells per
    side with BF16 (even) and FP16 (odd) population storage, one graph launch
    per step.  Every chamber keeps its mass (FP64 sums on the device; the
    walls and the periodic sides conserve it), and the two smallest chambers
    match the FP64 oracle within the mixed-storage bounds of
    test_gpu_lb_mixed (displacement 2e-4, node velocity 1e-3 of their
    largest entries, BF16; a tenth of that, FP16) after 3 steps."""
    ws = [f32_workload(w) for w in workload.config_batched(seed=0)]
    storage = ["bf16" if i % 2 == 0 else "fp16" for i in range(len(ws))]
    sims = [fsi.Simulation(w, storage=s) for w, s in zip(ws, storage)]
    m0 = [s.lattice.moments_fp64()[0] for s in sims]
    batch = fsi.Batch(sims, steps_per_graph=1)
    steps = 3
    batch.step(steps)
    torch.cuda.synchronize()
    for s, m in zip(sims, m0):
        assert torch.isfinite(s.X).all()
        assert abs(s.lattice.moments_fp64()[0] - m) < 1e-6 * m
    cells = [w["grid"]["nx"] * w["grid"]["ny"] * w["grid"]["nz"] for w in ws]
    for i in np.argsort(cells)[:2]:
        ora = oracle.Sim(ws[i])
        for _ in range(steps):
            ora.step()
        X0 = ws[i]["X"]
        tx, tu = (2e-4, 1e-3) if storage[i] == "bf16" else (2e-5, 1e-4)
        assert rel(sims[i].X.cpu().numpy() - X0, ora.X - X0) < tx, i
        assert rel(sims[i].U.cpu().numpy(), ora.U) < tu, i
        if sims[i].bonds is not None:
            assert np.array_equal(sims[i].bonds.bound.cpu().numpy(), ora.bound)
