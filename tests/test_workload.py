"""The seeded workload generator: mesh sizes of the configured icospheres, a
closed, outward-oriented surface (Euler characteristic 2), platelet shape of
Section 3.1 (a = 1 um, aspect 0.25), receptor and SCE counts, placement above
the wall, determinism under a seed."""
import numpy as np

from paper_1312_2234_b300 import workload as W


def test_icosphere_counts_and_orientation():
    for level, nv in ((0, 12), (1, 42), (3, 642), (4, 2562)):
        X, T = W.icosphere(level)
        assert len(X) == nv and len(T) == 2 * nv - 4
        E = {tuple(sorted(e)) for t in T for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
        assert len(X) - len(E) + len(T) == 2
        n = np.cross(X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]])
        assert (np.einsum("ij,ij->i", n, X[T[:, 0]]) > 0).all()


def test_config_small_shape():
    w = W.config_small(seed=0)
    X = w["X"].reshape(3, -1)
    mem = w["mesh"]["is_membrane"].astype(bool)
    assert mem.sum() == 642 and (~mem).sum() == 200 and len(w["sites"]["tri"]) == 100
    c = X[:, mem].mean(1)
    ext = X[:, mem].max(1) - X[:, mem].min(1)
    h = W.PHYSICAL["h"]
    assert np.allclose(ext[:2], 2 * W.PHYSICAL["a"] / h, rtol=2e-2)
    assert np.isclose(ext[2], 2 * W.PHYSICAL["a"] * W.PHYSICAL["aspect"] / h, rtol=5e-2)
    assert X[2, mem].min() >= -0.5 + 0.5 - 1e-9
    assert w["lig_count"].size == 256 and (w["bound"] == -1).all()
    assert np.allclose(c[:2], [16, 16])


def test_seeded_determinism():
    a, b = W.tiny(seed=4), W.tiny(seed=4)
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["sites"]["w"], b["sites"]["w"])
    c = W.tiny(seed=5)
    assert not np.array_equal(a["sites"]["w"], c["sites"]["w"])
