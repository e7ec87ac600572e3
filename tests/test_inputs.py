"""The seeded input generators: determinism and complete neighbour lists."""
import numpy as np

from paper_2604_24994_gb300 import inputs


def brute_lists(sc, K):
    P = sc.pos.astype(np.float64)
    W = sc.w.astype(np.float64)
    out = []
    for i in range(sc.n):
        a = P - P[i]
        L2 = (a * a).sum(1)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (L2 + W[i] - W) / (2 * np.sqrt(L2))
        t[i] = np.inf
        o = np.lexsort((np.arange(sc.n), t))
        out.append((o[:K], t[o[K]]))
    return out


def test_neighbour_lists_are_the_k_smallest_plane_distances():
    # capture-shaped (very uneven weights) and uniform scenes
    for sc, K in ((inputs.capture_scene(3000, seed=4, K=12), 12), (inputs.tiny_scene(), 16)):
        ref = brute_lists(sc, K)
        P = sc.pos.astype(np.float64)
        W = sc.w.astype(np.float64)
        for i in range(sc.n):
            js, tk1 = ref[i]
            assert np.array_equal(np.sort(sc.nbr[i]), np.sort(js)), i
            # complete: no unlisted site's plane reaches the (clipped) ball
            assert float(sc.R[i]) <= tk1 + 1e-12


def test_generators_are_deterministic():
    a = inputs.uniform_scene(500, seed=7, K=8)
    b = inputs.uniform_scene(500, seed=7, K=8)
    for k in a.PARAMS + ("nbr",):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c = inputs.uniform_scene(500, seed=8, K=8)
    assert not np.array_equal(a.pos, c.pos)


def test_scene_file_round_trip(tmp_path):
    """The binary scene format (one .npz) stores every array bit for bit,
    the optional extended face model included, and refuses other files."""
    import numpy as np
    import pytest
    from paper_2604_24994_gb300 import inputs
    sc = inputs.uniform_scene(500, seed=4, K=8)
    rng = np.random.default_rng(0)
    sc.disp = rng.normal(size=(sc.n, 4)).astype(np.float32)
    sc.sv = rng.normal(size=(sc.n, 4, 8, 6)).astype(np.float32)
    p = tmp_path / "scene.npz"
    sc.save(str(p))
    back = inputs.load_scene(str(p))
    for f in ("pos", "w", "R", "sigma", "rgb", "normal", "offset", "tex", "nbr", "disp", "sv"):
        a, b = getattr(sc, f), getattr(back, f)
        assert a.dtype == b.dtype and a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8)), f
    assert back.sites is None and back.n_clipped == sc.n_clipped
    np.savez(tmp_path / "other.npz", format=np.array("x"))
    with pytest.raises(ValueError):
        inputs.load_scene(str(tmp_path / "other.npz"))
