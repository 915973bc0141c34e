"""The CUDA library's image-energy arithmetic (render.cuh), built for the host with g++,
against the oracle (oracle/softras.py) on the CPU: rendered image, silhouette, energy and
dE/dx."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from oracle import softras as S  # noqa: E402
from paper_2203_11938_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def host_lib(tmp_path_factory):
    global _lib
    if _lib is None:
        out = str(tmp_path_factory.mktemp("render") / "librender_host.so")
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                               os.path.join(HERE, "render_host.cpp")])
        _lib = ctypes.CDLL(out)
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        _lib.host_image_energy.argtypes = [ctypes.c_int, ctypes.c_int, ip, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp,
                                           ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
        _lib.host_image_energy.restype = ctypes.c_double
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def scene(seed, width=24, height=20):
    """A perturbed 4 x 4 sheet and the frame (width x height) of another perturbation.  At 96 x 80 most
    pixels lie tens of pixels from the sheet, where every coverage underflows and the
    colour is the background's."""
    rng = np.random.default_rng(seed)
    N = 4
    rest, tris = W.grid_mesh(N)
    x = rest + np.c_[0.02 * rng.normal(size=(N * N, 2)), 0.05 * rng.normal(size=N * N)]
    uv = np.c_[rest[:, 0], 1.0 - rest[:, 1]]
    tex = rng.uniform(0, 1, (8, 8, 3))
    cam = (26.0, 0.5, 0.5, 2.0)
    xt = rest + np.c_[0.02 * rng.normal(size=(N * N, 2)), 0.05 * rng.normal(size=N * N)]
    tri = [tuple(int(i) for i in t) for t in tris]
    img, A = S.render(xt, tri, uv, tex, cam, width, height)
    return x, tris.astype(np.int32), tri, uv, tex, cam, img.numpy(), (A.numpy() > 0.5).astype(np.float64)


@pytest.mark.parametrize("seed,W,H", [(1, 24, 20), (2, 24, 20), (3, 96, 80)])
def test_host_build_matches_oracle(tmp_path_factory, seed, W, H):
    lib = host_lib(tmp_path_factory)
    x, tris, tri, uv, tex, cam, image, mask = scene(seed, W, H)
    n, m = x.shape[0], tris.shape[0]
    grad = np.zeros_like(x)
    out_img = np.zeros((H, W, 3))
    out_sil = np.zeros((H, W))
    E = lib.host_image_energy(n, m, tris.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(np.ascontiguousarray(x)),
                              _d(np.ascontiguousarray(uv)), 8, 8, _d(np.ascontiguousarray(tex)),
                              _d(np.array(cam, float)), W, H, _d(np.ascontiguousarray(image)),
                              _d(np.ascontiguousarray(mask)), _d(grad), _d(out_img), _d(out_sil))
    img_o, A_o = S.render(x, tri, uv, tex, cam, W, H)
    assert np.isfinite(img_o.numpy()).all() and np.isfinite(out_img).all()
    np.testing.assert_allclose(out_img, img_o.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(out_sil, A_o.numpy(), rtol=1e-10, atol=1e-12)
    E_o, g_o = S.energy_and_grad(np.stack([x, x]), tri, uv, tex, cam, [None, image], [None, mask])
    assert E == pytest.approx(E_o, rel=1e-10)
    np.testing.assert_allclose(grad, g_o[1], rtol=1e-7, atol=1e-9 * np.abs(g_o[1]).max())
