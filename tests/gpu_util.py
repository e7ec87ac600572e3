"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle."""
import numpy as np

RGB_TOL = 1e-4      # max abs per RGB channel vs the FP64 oracle
T_TOL = 1e-5        # max abs in transmittance
GRAD_TOL = 1e-3     # relative L2 per parameter tensor


def gpu_forward(scene, cams, capacity=None, stats=False):
    import torch
    from paper_2604_24994_gb300 import DeviceScene, Renderer
    ds = DeviceScene.from_numpy(scene, "cuda")
    r = Renderer(ds.n, ds.k, cams, capacity=capacity)
    if stats:
        r.enable_stats(True)
    rgb, T, last = r.forward(ds)
    torch.cuda.synchronize()
    out = (rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64),
           last.cpu().numpy())
    return (out, r, ds) if stats else out


def pixel_index(cams, view, pix):
    """Flat indices into the concatenated outputs for pixels (u, v) of a view."""
    base = sum(c.width * c.height for c in cams[:view])
    pix = np.asarray(pix).reshape(-1, 2)
    return base + pix[:, 1] * cams[view].width + pix[:, 0]


def sample_pixels(cam, n, seed=0, include_corners=True):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, cam.width, n)
    v = rng.integers(0, cam.height, n)
    pix = np.stack([u, v], 1)
    if include_corners:
        extra = np.array([[0, 0], [cam.width - 1, 0], [0, cam.height - 1], [cam.width - 1, cam.height - 1],
                          [cam.width // 2, cam.height // 2]])
        pix = np.concatenate([pix, extra])
    return pix.astype(np.int32)


def assert_close_image(rgb, T, rgb_o, T_o, what=""):
    ec = float(np.abs(rgb - rgb_o).max()) if rgb.size else 0.0
    et = float(np.abs(T - T_o).max()) if T.size else 0.0
    assert ec < RGB_TOL and et < T_TOL, f"{what}: max |drgb| {ec:.3e} (tol {RGB_TOL}), max |dT| {et:.3e} (tol {T_TOL})"
    return ec, et


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
