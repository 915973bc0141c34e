"""CPU-side checks of the C-ABI boundary: the library builds, loads without a GPU and
exports every entry point that include/cloth_sim.h declares; host-side validation
rejects bad meshes and options without touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2203_11938_gb300 import build as B
from paper_2203_11938_gb300 import sim
from paper_2203_11938_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cloth_sim.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sim.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cloth_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sim.EXPORTS)


def test_opts_struct_layout_matches_header(lib):
    o = sim.default_opts()
    assert ctypes.sizeof(sim.ClothOpts) == 104  # = sizeof(cloth_opts) in C (checked with gcc)
    assert o.precision == sim.FP32 and o.steps == 1 and o.cg_max_iter == 2000
    assert o.gravity[2] == pytest.approx(-9.8) and o.clamp_eta == pytest.approx(1e-3)
    assert o.exec == sim.EXEC_GRAPH and o.cg_poll_every == 16 and o.precond == 1 and o.cg_schedule == -1
    assert o.cg_handover == 0 and o.force_mode == 0 and o.air_density == 0.0 and o.cg_warm_start == 0


def test_mesh_create_counts(lib):
    for N in (2, 10, 33):
        rest, tris = W.grid_mesh(N)
        m = sim.Mesh(rest, tris, W.pins(N, "top2"))
        assert m.info() == W.grid_counts(N)


def test_mesh_validation_errors(lib):
    rest, tris = W.grid_mesh(3)
    bad = tris.copy()
    bad[0, 0] = 99
    with pytest.raises(sim.ClothError, match="-1"):
        sim.Mesh(rest, bad)
    deg = rest.copy()
    deg[1] = deg[0]
    with pytest.raises(sim.ClothError, match="-3"):
        sim.Mesh(deg, tris)
    flipped = tris.copy()
    flipped[1] = flipped[1][::-1]
    with pytest.raises(sim.ClothError, match="-2"):
        sim.Mesh(rest, flipped)
    # three triangles on one edge
    r3 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], float)
    t3 = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], np.int32)
    with pytest.raises(sim.ClothError, match="-2"):
        sim.Mesh(r3, t3)
    msg = lib.cloth_last_error().decode()
    assert "more than two" in msg


def test_batch_create_rejects_bad_options_on_host(lib):
    rest, tris = W.grid_mesh(3)
    m = sim.Mesh(rest, tris)
    arr = (ctypes.c_void_p * 1)(m._h)
    h = ctypes.c_void_p()
    for field, value in (("steps", 0), ("dt", -1.0), ("cg_max_iter", 0), ("precision", 7), ("exec", 9),
                         ("clamp_eta", -1.0), ("cg_poll_every", 0), ("precond", 5),
                         ("cg_schedule", 32), ("cg_schedule", -2), ("cg_handover", -1),
                         ("force_mode", 2), ("air_density", -1.0), ("cg_warm_start", 2)):
        o = sim.default_opts()
        setattr(o, field, value)
        rc = lib.cloth_batch_create(arr, 1, ctypes.byref(o), ctypes.byref(h))
        assert rc == -1, field
    assert lib.cloth_batch_create(arr, 0, ctypes.byref(sim.default_opts()), ctypes.byref(h)) == -1
    assert lib.cloth_forward(None, None, None, None, None, None, None, None) == -1
    assert lib.cloth_backward(None, None, None, None, None, None, None, None) == -1


def test_host_validation_of_the_newer_entry_points(lib):
    """Entry points added for the force modes, the wind and the image energies reject a
    null batch or bad arguments on the host, before any device work."""
    p = ctypes.c_void_p(1)  # never dereferenced: validation fails first
    assert lib.cloth_set_wind(None, None) == -1
    assert lib.cloth_wind_gradient(None, p, None) == -1
    assert lib.cloth_sheet_iterations(None, 0, None, None) == -1
    assert lib.cloth_kernel_bytes(None, 0, None) == -1
    cam = (ctypes.c_double * 4)(30.0, 0.5, 0.5, 2.0)
    bad = np.array([[0, 1, 5]], np.int32)  # vertex 5 of a 3-vertex mesh
    good = np.array([[0, 1, 2]], np.int32)
    args = lambda n, tris: (n, tris.shape[0], tris.ctypes.data_as(ctypes.c_void_p), p, p, 4, 4, p, cam, 8, 8, p, p,  # noqa: E731
                            p, p, None, None, None, None)
    assert lib.cloth_image_energy(*args(3, bad)) == -1
    assert "out of range" in lib.cloth_last_error().decode()
    assert lib.cloth_image_energy(*args(2, good)) == -1
    # scratch: 12 W H + 15 n doubles and the 3 m triangle indices
    assert lib.cloth_image_energy_scratch(3, 1, 8, 8) == 8 * (12 * 64 + 15 * 3 + 21 * 1 + 2)


def test_image_energy_binding_rejects_wrong_shapes_before_any_launch():
    """sim.image_energy checks every array's shape against x, mask and the texture before
    it checks devices or calls the library, so a grey frame, a 4-channel texture or too
    few uv rows never reach a kernel (which would index past their ends)."""
    torch = pytest.importorskip("torch")
    n, H, W = 9, 6, 5
    f = lambda *s: torch.zeros(*s, dtype=torch.float64)  # noqa: E731
    good = dict(x=f(n, 3), tris=np.array([[0, 1, 2]], np.int32), uv=f(n, 2), tex=f(4, 4, 3), camera=(500, 0, 0, 2),
                image=f(H, W, 3), mask=f(H, W))
    bad = {
        "x": dict(x=f(n, 2)), "uv": dict(uv=f(n - 1, 2)), "tex": dict(tex=f(4, 4, 4)),
        "image": dict(image=f(H, W)), "mask": dict(mask=f(H, W, 1)), "tris": dict(tris=np.array([0, 1, 2], np.int32)),
    }
    for name, change in bad.items():
        args = dict(good, **change)
        with pytest.raises(sim.ClothError, match="shape"):
            sim.image_energy(**args)
    # right shapes on the CPU: rejected for the device, still before any launch
    with pytest.raises(sim.ClothError, match="CUDA"):
        sim.image_energy(**good)
