"""The allocation-free loss entry point (cloth_loss_l2_static) against cloth_loss_l2.

cloth_loss_l2_static serves callers that must not allocate device memory where they call
it (another allocator owns the pool, or cudaMalloc's implicit synchronisation is not
acceptable in their loop); its scratch is a static device array shared by all calls.
This file is collected last so that a failure here stops a run only after every other
test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_11938_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_scratch_loss_matches_loss_l2_on_two_calls(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11938_gb300 import build, sim

    build.build()
    lib = sim.load_library()
    rng = np.random.default_rng(7)
    sheets = []
    for N in (5, 9, 12):
        rest, tris = W.grid_mesh(N)
        sheets.append((rest, tris, W.pins(N, "top2")))
    steps = 6
    for precision, dtype in (("f32", torch.float32), ("f64", torch.float64)):
        b = sim.ClothBatch(sheets, steps=steps, dt=1 / 30, precision=precision, cg_tol=1e-8)
        mat = torch.tensor(np.tile([1e3, 0.3, 1e-4, 0.1], (3, 1)), dtype=dtype, device="cuda")
        x0 = torch.tensor(np.concatenate([s[0] for s in sheets]), dtype=dtype, device="cuda")
        traj, _ = b.forward(mat, x0, torch.zeros_like(x0), None)
        offsets = torch.tensor(np.cumsum([0] + b.sheet_sizes), dtype=torch.int32, device="cuda")
        N = b.total_vertices
        for call in range(2):  # two calls in a row share (and reuse) the static scratch
            target = traj + torch.tensor(rng.normal(scale=0.01, size=traj.shape), dtype=dtype, device="cuda")
            ref_loss, ref_grad = b.loss_l2(traj, target)
            loss = torch.empty(b.count, dtype=torch.float64, device="cuda")
            grad = torch.full_like(traj, float("nan"))
            rc = lib.cloth_loss_l2_static(b.count, ctypes.c_void_p(offsets.data_ptr()), steps, N,
                                          sim.FP32 if precision == "f32" else sim.FP64,
                                          ctypes.c_void_p(traj.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                          ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0, lib.cloth_last_error()
            torch.cuda.synchronize()
            np.testing.assert_allclose(loss.cpu().numpy(), ref_loss.cpu().numpy(), rtol=1e-12, atol=0)
            np.testing.assert_allclose(grad.cpu().numpy(), ref_grad.cpu().numpy(), rtol=1e-12, atol=0)
            # and both against the oracle's loss of each sheet on the same values
            tr, tg = traj.double().cpu().numpy(), target.double().cpu().numpy()
            off = np.cumsum([0] + b.sheet_sizes)
            for k in range(b.count):
                L_o, g_o = oracle_mod.loss_l2(tr[:, off[k]:off[k + 1]], tg[:, off[k]:off[k + 1]])
                assert float(loss[k]) == pytest.approx(L_o, rel=1e-12 if precision == "f64" else 1e-6)
                np.testing.assert_allclose(grad.double().cpu().numpy()[:, off[k]:off[k + 1]], g_o,
                                           rtol=1e-12 if precision == "f64" else 1e-6,
                                           atol=1e-300 if precision == "f64" else 1e-7)
    # sizes beyond the static scratch are rejected with a clear error
    rc = lib.cloth_loss_l2_static(70000, ctypes.c_void_p(offsets.data_ptr()), 1, N, sim.FP32,
                                  ctypes.c_void_p(traj.data_ptr()), ctypes.c_void_p(traj.data_ptr()),
                                  ctypes.c_void_p(loss.data_ptr()), None, None)
    assert rc == -1 and b"exceeds the static scratch" in lib.cloth_last_error()
