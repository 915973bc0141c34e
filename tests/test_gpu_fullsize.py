"""Full-size checks of the two long single-sheet workloads, in the launch configuration
bench.py uses (FP32, captured graph, checkpoint-and-recompute).

The FP64 oracle cannot run 300 steps of a 10,000-vertex sheet or one solve of a
65,536-vertex sheet in test time, so these tests check sampled outputs the oracle can
compute one by one (the first step, the loss on the whole trajectory, forces and the step
matrix applied to a vector at the final state) and properties that
hold at any size (checkpoint-and-recompute gives bitwise the same gradients as keeping
every state; every solve converges).
"""
import numpy as np
import pytest

from paper_2203_11938_gb300 import workloads as W

from gpu_util import make_batch, max_entry_err, rel, to_cuda, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

f32r = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11938_gb300 import build

    build.build()


def _project(traj, cam):
    f, cx, cy, cz = cam
    Xc = traj[..., 0] - cx
    Yc = -(traj[..., 1] - cy)
    Zc = cz - traj[..., 2]
    return torch.stack([f * Xc / Zc, f * Yc / Zc], dim=-1).contiguous()


def test_grid100_pinhole_300_steps_full_size(oracle_mod):
    """100x100 sheet, two top corners, 300 steps of 1/30 s, smooth wind, pinhole loss against
    tracks of the ground-truth material, checkpoint every 30 steps."""
    cfg = W.config3()
    s = cfg.sheets[0]
    f32 = torch.float32
    runs = {}
    for ckpt in (cfg.checkpoint_every, 0):
        b = make_batch(cfg.sheets, steps=cfg.steps, dt=cfg.dt, precision="f32", tol=cfg.cg_tol,
                       max_iter=cfg.cg_max_iter, ckpt=ckpt)
        x0 = to_cuda(s.rest, f32)
        v0 = torch.zeros_like(x0)
        F = to_cuda(s.forces, f32)
        truth, _ = b.forward(to_cuda(W.config3_truth(), f32)[None], x0, v0, F)
        uv = _project(truth.double(), cfg.camera).to(f32)
        traj, st = b.forward(to_cuda(s.material, f32)[None], x0, v0, F)
        loss, dL = b.loss_pinhole(traj, uv, cfg.camera)
        g = b.backward(dL)
        torch.cuda.synchronize()
        assert int(st[0]) == 0 and int(g["status"][0]) == 0
        runs[ckpt] = (to_np(traj), float(loss[0]), to_np(dL), to_np(g["material"]), to_np(g["x0"]),
                      to_np(g["forces"]), to_np(uv))
    a, c = runs[cfg.checkpoint_every], runs[0]
    for k in (0, 3, 4, 5):
        np.testing.assert_array_equal(a[k], c[k])  # recompute reproduces the states bitwise
    assert np.isfinite(a[3]).all() and np.abs(a[3][0, [0, 2, 3]]).min() > 0
    # the pinhole loss and its gradient on the whole trajectory, recomputed by the oracle
    L_o, g_o = oracle_mod.loss_pinhole(a[0], a[6], cfg.camera)
    assert a[1] == pytest.approx(L_o, rel=1e-9)
    assert rel(a[2], g_o) < 1e-6 and max_entry_err(a[2], g_o) < 1e-6
    # the first step, recomputed by the oracle on the same (float-rounded) inputs
    o = oracle_mod.OracleSim(s.rest, s.tris, s.pinned)
    tx, _, _, st = o.forward(f32r(s.material), f32r(s.rest), np.zeros_like(s.rest), f32r(s.forces[:1]), dt=cfg.dt,
                             steps=1, tol=1e-10, max_iter=20000, gravity=W.GRAVITY)
    assert st == 0
    assert np.abs(a[0][1] - tx[1]).max() <= 1e-6


def test_grid256_corners_200_steps_full_size(oracle_mod):
    """256x256 sheet, four corners, 200 steps of 1/60 s, smooth wind, checkpoint every 20
    steps: bitwise the same gradients as without checkpoints; forces and A p of the final
    state against the oracle."""
    cfg = W.config5()
    s = cfg.sheets[0]
    f32 = torch.float32
    runs = {}
    for ckpt in (cfg.checkpoint_every, 0):
        b = make_batch(cfg.sheets, steps=cfg.steps, dt=cfg.dt, precision="f32", tol=cfg.cg_tol,
                       max_iter=cfg.cg_max_iter, ckpt=ckpt)
        x0 = to_cuda(s.rest, f32)
        v0 = torch.zeros_like(x0)
        F = to_cuda(s.forces, f32)
        mat = to_cuda(s.material, f32)[None]
        tgt, _ = b.forward(mat * torch.tensor(cfg.target_scale, dtype=f32, device="cuda"), x0, v0, F)
        tgt = tgt.clone()
        traj, st = b.forward(mat, x0, v0, F)
        _, dL = b.loss_l2(traj, tgt)
        g = b.backward(dL)
        torch.cuda.synchronize()
        assert int(st[0]) == 0 and int(g["status"][0]) == 0
        runs[ckpt] = (to_np(traj), to_np(g["material"]), to_np(g["x0"]), to_np(g["forces"]), b)
    a, c = runs[cfg.checkpoint_every], runs[0]
    for k in (0, 1, 2, 3):
        np.testing.assert_array_equal(a[k], c[k])
    # final state (x_T, v_T = (x_T - x_{T-1}) / h) through the single-stage entry points
    b = a[4]
    xT = a[0][-1]
    vT = (a[0][-1] - a[0][-2]) / cfg.dt
    rng = np.random.default_rng(3)
    p = rng.normal(size=xT.shape)
    mat = to_cuda(s.material, f32)[None]
    fm, fb = b.internal_forces(mat, to_cuda(xT, f32))
    y = b.spmv(mat, to_cuda(xT, f32), to_cuda(vT, f32), to_cuda(p, f32))
    o = oracle_mod.OracleSim(s.rest, s.tris, s.pinned)
    m64 = f32r(s.material)
    x64 = f32r(xT)
    v64 = f32r(vT)
    _, om, ob = o.energy_forces(m64, x64)
    fm, fb = to_np(fm), to_np(fb)
    assert rel(fm, om) < 1e-4 and max_entry_err(fm, om) < 1e-4, (rel(fm, om), max_entry_err(fm, om))
    assert rel(fb, ob) < 1e-3 and max_entry_err(fb, ob) < 1e-3, (rel(fb, ob), max_entry_err(fb, ob))
    yo, bo = o.system_matvec(m64, cfg.dt, W.GRAVITY, x64, v64, f32r(s.forces[-1]), f32r(p))
    y = to_np(y)
    assert rel(y, yo) < 1e-5 and max_entry_err(y, yo) < 1e-5, (rel(y, yo), max_entry_err(y, yo))
