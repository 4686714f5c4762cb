"""Batched lattice step (lb_batch_*): lattices of uneven sizes and mixed
storage modes advanced by one persistent launch per storage mode that walks
the tile list of all of them.  Every tile runs the per-cell arithmetic of
lb_step, so each lattice's populations and velocity field must be
bit-identical to lb_step on it alone: for every column shape, after the
autotuner, with wall, body and spread-row forcing, and on ragged sizes
(sides that are not multiples of any tile side, nz below the column depth)."""
import numpy as np
import pytest
import torch

from paper_1312_2234_b300 import fsi, workload

pytestmark = pytest.mark.gpu

# (nx, ny, nz, storage, walls): ragged in x and y for every column shape
# (pair 64x4, 32x4, 16x8), nz below and above the 16-plane column depth, a
# two-plane lattice, both wall modes
SPECS = [(53, 37, 29, "fp32", 0), (48, 40, 36, "bf16", 0), (33, 19, 17, "fp16", 1), (64, 8, 3, "bf16", 1),
         (17, 70, 21, "fp32", 1), (100, 27, 40, "fp16", 0), (7, 5, 2, "bf16", 0), (130, 3, 18, "fp32", 0)]


def make(spec, seed):
    nx, ny, nz, storage, walls = spec
    rng = np.random.default_rng(seed)
    tau = float(np.float32(rng.uniform(0.6, 1.2)))
    u = (float(rng.uniform(1e-3, 5e-3)), float(rng.uniform(-2e-3, 2e-3)), 0.0)
    body = (float(rng.uniform(0.0, 1e-6)), 0.0, float(rng.uniform(-1e-7, 1e-7)))
    lat = fsi.Lattice(nx, ny, nz, tau, u, body, storage=storage, walls=walls)
    lat.init_shear()
    return lat


def set_forces(lat, rng):
    """Spread forces in a random seventh of the rows (g and the row flags
    written directly, as ib_spread leaves them)."""
    nz, ny, nx = lat.shape
    rows = rng.choice(ny * nz, size=max(1, ny * nz // 7), replace=False)
    g = np.zeros((ny * nz, nx, 4), np.float32)
    g[rows, :, :3] = rng.uniform(-1e-4, 1e-4, size=(len(rows), nx, 3))
    flags = np.zeros(ny * nz, np.int32)
    flags[rows] = 1
    return torch.as_tensor(g.reshape(-1, 4)), torch.as_tensor(flags)


def state(lat):
    """Populations and the velocity field ib_interp reads: every cell with
    mixed storage; with FP32 storage only the rows flagged at the last step
    hold it (the other rows keep whatever an earlier step left)."""
    v = lat.velocity().cpu().numpy()
    if not lat.mixed:
        nz, ny, nx = lat.shape
        live = np.repeat(lat.flags.cpu().numpy() != 0, nx)
        v = np.where(live[:, None], v, 0.0)
    return lat.export().cpu().numpy(), v


def pairs(specs=SPECS, seed=0):
    batched = [make(s, seed + i) for i, s in enumerate(specs)]
    alone = [make(s, seed + i) for i, s in enumerate(specs)]
    return batched, alone


def step_both(batch, batched, alone, steps, seed=7):
    rng = np.random.default_rng(seed)
    for _ in range(steps):
        for a, b in zip(batched, alone):
            g, fl = set_forces(a, rng)
            for lat in (a, b):
                lat.g.copy_(g)
                lat.flags.copy_(fl)
        batch.step(1)
        for b in alone:
            b.step(1)
    torch.cuda.synchronize()


def assert_identical(batched, alone):
    for i, (a, b) in enumerate(zip(batched, alone)):
        fa, va = state(a)
        fb, vb = state(b)
        assert np.array_equal(fa, fb), (i, SPECS[i] if i < len(SPECS) else None)
        assert np.array_equal(va, vb), i
        assert np.isfinite(fa).all()


def test_batch_is_bit_identical_to_lone_steps():
    batched, alone = pairs()
    batch = fsi.LatticeBatch(batched)
    shapes = batch.shapes()
    assert [s < 0 for s in shapes] == [sp[3] == "fp32" for sp in SPECS]
    step_both(batch, batched, alone, 3)
    assert_identical(batched, alone)


@pytest.mark.parametrize("shape", [0, 1, 2])
def test_every_column_shape_gives_the_same_populations(shape):
    batched, alone = pairs(seed=10)
    batch = fsi.LatticeBatch(batched)
    batch.set_shapes([shape] * len(batched))
    assert all(s == shape for s, sp in zip(batch.shapes(), SPECS) if sp[3] != "fp32")
    step_both(batch, batched, alone, 2, seed=11)
    assert_identical(batched, alone)


def test_autotune_keeps_the_state_and_the_results():
    batched, alone = pairs(seed=20)
    batch = fsi.LatticeBatch(batched)
    step_both(batch, batched, alone, 1, seed=21)
    before = [state(a) for a in batched]
    ms = batch.autotune(reps=2)
    assert ms > 0
    assert all(0 <= s < 3 for s, sp in zip(batch.shapes(), SPECS) if sp[3] != "fp32")
    for (f0, v0), a in zip(before, batched):
        f1, v1 = state(a)
        assert np.array_equal(f0, f1)
        if a.mixed:          # FP32: v of the still-flagged rows is rewritten (with g consumed)
            assert np.array_equal(v0, v1)
    # the pending forces were consumed before tuning; set them on both again
    step_both(batch, batched, alone, 2, seed=22)
    assert_identical(batched, alone)


def test_shape_and_parity_errors():
    batched, _ = pairs(SPECS[:2], seed=30)
    batch = fsi.LatticeBatch(batched)
    with pytest.raises(RuntimeError, match="shape"):
        batch.set_shapes([0, 5])
    batched[1].step(1)          # stepped alone: the parities now differ
    with pytest.raises(RuntimeError, match="parit"):
        batch.step(1)
    with pytest.raises(RuntimeError, match="twice"):
        fsi.LatticeBatch([batched[0], batched[0]])


def test_batched_chamber_sizes_full_scale():
    """The 64 chamber lattices of the batched workload (sides 48..128, 45 M
    cells) in BF16 and FP16, stepped as one batch; three chambers (the
    smallest, the largest, one between) stepped alone alongside."""
    ws = workload.config_batched(seed=0)
    specs = [(w["grid"]["nx"], w["grid"]["ny"], w["grid"]["nz"], "bf16" if i % 2 == 0 else "fp16", 0)
             for i, w in enumerate(ws)]
    cells = [s[0] * s[1] * s[2] for s in specs]
    order = np.argsort(cells)
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    batched = [make(s, 100 + i) for i, s in enumerate(specs)]
    alone = {i: make(specs[i], 100 + i) for i in pick}
    batch = fsi.LatticeBatch(batched)
    batch.step(2)
    for lat in alone.values():
        lat.step(2)
    torch.cuda.synchronize()
    for i, lat in alone.items():
        fa, va = state(batched[i])
        fb, vb = state(lat)
        assert np.array_equal(fa, fb), i
        assert np.array_equal(va, vb), i
