"""GPU parity: every stage of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances: FP64 mode must agree to 1e-10 (relative) on gradients and to round-off on
states (both sides run the same Jacobi-PCG recurrence); FP32 mode must keep the max
vertex position error within 1e-5 of the 1 m sheet and the parameter gradients within
1e-3 relative of the oracle.  Element-level FP32 checks use 1e-4 relative of the
field's scale (float has 6e-8 unit round-off; the Green strain near rest cancels about
three digits).
"""
import numpy as np
import pytest

from paper_2203_11938_gb300 import workloads as W

from gpu_util import MAT, make_batch, max_entry_err, oracle_sims, rel, sheets_mixed, split, to_cuda, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11938_gb300 import build

    build.build()


def close(a, b, tol):
    """Norm-relative error and largest entry-wise error (relative to the field's largest
    entry) both within tol."""
    return rel(a, b) < tol and max_entry_err(a, b) < tol


def _dtype(prec):
    return torch.float64 if prec == "f64" else torch.float32


def _perturbed(sheets, seed=0, amp=0.03):
    rng = np.random.default_rng(seed)
    xs = [s.rest * np.array([0.97, 1.03, 1.0]) + amp * rng.normal(size=s.rest.shape) for s in sheets]
    vs = [0.1 * rng.normal(size=s.rest.shape) * (s.pinned == 0)[:, None] for s in sheets]
    return xs, vs


def _materials(sheets):
    return np.stack([s.material for s in sheets])


# --------------------------------------------------------------------- element stages
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_internal_forces_match_oracle(oracle_mod, prec):
    sheets = sheets_mixed()
    b = make_batch(sheets, steps=1, dt=1 / 30, precision=prec, tol=1e-10)
    xs, _ = _perturbed(sheets)
    mat = _materials(sheets)
    dt = _dtype(prec)
    fm, fb = b.internal_forces(to_cuda(mat, dt), to_cuda(np.concatenate(xs), dt))
    fm, fb = split(to_np(fm), b.sheet_sizes), split(to_np(fb), b.sheet_sizes)
    tol = 1e-11 if prec == "f64" else 1e-4
    for k, (s, o) in enumerate(zip(sheets, oracle_sims(oracle_mod, sheets))):
        _, om, ob = o.energy_forces(s.material, xs[k])
        assert close(fm[k], om, tol), (rel(fm[k], om), max_entry_err(fm[k], om))
        assert close(fb[k], ob, tol * (10 if prec == "f32" else 1)), (rel(fb[k], ob), max_entry_err(fb[k], ob))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_assembled_system_matches_oracle(oracle_mod, prec):
    """A = M + h^2 H~ and b = h (f + M g + F) - h^2 H~ v, pinned rows identity."""
    sheets = sheets_mixed()
    b = make_batch(sheets, steps=1, dt=1 / 30, precision=prec, tol=1e-10)
    xs, vs = _perturbed(sheets, seed=1)
    rng = np.random.default_rng(2)
    Fs = [1e-3 * rng.normal(size=s.rest.shape) for s in sheets]
    dt = _dtype(prec)
    mat = _materials(sheets)
    A, bv = b.system_dense(to_cuda(mat, dt), to_cuda(np.concatenate(xs), dt), to_cuda(np.concatenate(vs), dt),
                           to_cuda(np.concatenate(Fs), dt))
    bv = split(to_np(bv), b.sheet_sizes)
    tol = 1e-11 if prec == "f64" else 1e-5
    for k, (s, o) in enumerate(zip(sheets, oracle_sims(oracle_mod, sheets))):
        Ao, bo = o.system_dense(s.material, 1 / 30, W.GRAVITY, xs[k], vs[k], Fs[k], eta=1e-3)
        Ag = to_np(A[k])
        assert np.abs(Ag - Ao).max() < tol * np.abs(Ao).max()
        assert close(bv[k].ravel(), bo, tol * 10), (rel(bv[k].ravel(), bo), max_entry_err(bv[k].ravel(), bo))
        if prec == "f64":  # symmetric to round-off (the diagonal block is rebuilt from the row sum)
            np.testing.assert_allclose(Ag, Ag.T, rtol=0, atol=1e-14 * np.abs(Ag).max())


def test_spmv_matches_dense_product(oracle_mod):
    sheets = sheets_mixed()
    b = make_batch(sheets, steps=1, dt=1 / 30, precision="f64", tol=1e-10)
    xs, vs = _perturbed(sheets, seed=4)
    rng = np.random.default_rng(5)
    ps = [rng.normal(size=s.rest.shape) for s in sheets]
    mat = to_cuda(_materials(sheets), torch.float64)
    y = b.spmv(mat, to_cuda(np.concatenate(xs), torch.float64), to_cuda(np.concatenate(vs), torch.float64),
               to_cuda(np.concatenate(ps), torch.float64))
    y = split(to_np(y), b.sheet_sizes)
    for k, (s, o) in enumerate(zip(sheets, oracle_sims(oracle_mod, sheets))):
        Ao, _ = o.system_dense(s.material, 1 / 30, W.GRAVITY, xs[k], vs[k], None, eta=1e-3)
        assert close(y[k].ravel(), Ao @ ps[k].ravel(), 1e-12)


@pytest.mark.parametrize("eta", [0.0, 1e-3])
def test_third_contraction_matches_oracle(oracle_mod, eta):
    sheets = sheets_mixed()
    b = make_batch(sheets, steps=1, dt=1 / 30, precision="f64", tol=1e-10, eta=eta)
    xs, _ = _perturbed(sheets, seed=6)
    rng = np.random.default_rng(7)
    As = [rng.normal(size=s.rest.shape) for s in sheets]
    Bs = [rng.normal(size=s.rest.shape) for s in sheets]
    f64 = torch.float64
    out = b.third(to_cuda(_materials(sheets), f64), to_cuda(np.concatenate(xs), f64), to_cuda(np.concatenate(As), f64),
                  to_cuda(np.concatenate(Bs), f64))
    out = split(to_np(out), b.sheet_sizes)
    for k, (s, o) in enumerate(zip(sheets, oracle_sims(oracle_mod, sheets))):
        ref = o.third(s.material, xs[k], As[k], Bs[k], eta=eta)
        assert close(out[k], ref, 1e-10), (rel(out[k], ref), max_entry_err(out[k], ref))


# --------------------------------------------------------------------- trajectories
def _rollout_both(oracle_mod, sheets, *, steps, dt, prec, tol, oracle_tol, forces=None, exec_mode="graph", ckpt=0,
                  v0s=None, precond="block"):
    b = make_batch(sheets, steps=steps, dt=dt, precision=prec, tol=tol, exec_mode=exec_mode, ckpt=ckpt,
                   precond=precond)
    dtp = _dtype(prec)
    x0 = np.concatenate([s.rest for s in sheets])
    v0 = np.zeros_like(x0) if v0s is None else np.concatenate(v0s)
    F = None if forces is None else np.concatenate(forces, axis=1)
    traj, status = b.forward(to_cuda(_materials(sheets), dtp), to_cuda(x0, dtp), to_cuda(v0, dtp),
                             None if F is None else to_cuda(F, dtp))
    torch.cuda.synchronize()
    refs = []
    for k, (s, o) in enumerate(zip(sheets, oracle_sims(oracle_mod, sheets))):
        vk = np.zeros_like(s.rest) if v0s is None else v0s[k]
        refs.append(o.forward(s.material, s.rest, vk, None if forces is None else forces[k], dt=dt, steps=steps,
                              tol=oracle_tol, max_iter=20000, gravity=W.GRAVITY,
                              precond=1 if precond == "block" else 0))
    return b, traj, status, refs


@pytest.mark.parametrize("precond", ["block", "scalar"])
def test_config1_fp64_trajectory_and_gradients(oracle_mod, precond):
    """10x10 sheet, two top corners pinned, 20 steps of 1/30 s, FP64 (config 1 of the
    benchmark list): positions to 1e-10 m, gradients of the target-trajectory loss
    w.r.t. Y, k_b, rho, x0, v0 and the per-step forces to 1e-10 relative (by norm and
    entry by entry); block and scalar Jacobi."""
    cfg = W.config1()
    s = cfg.sheets[0]
    tol = 1e-12
    pc = 1 if precond == "block" else 0
    b, traj, status, refs = _rollout_both(oracle_mod, cfg.sheets, steps=cfg.steps, dt=cfg.dt, prec="f64", tol=tol,
                                          oracle_tol=tol, precond=precond)
    tx, tv, it, st = refs[0]
    assert int(status[0]) == 0 and st == 0
    assert np.abs(to_np(traj) - tx).max() < 1e-10
    # target trajectory from scaled parameters (oracle), loss and adjoint
    o = oracle_sims(oracle_mod, cfg.sheets)[0]
    tgt_mat = s.material * np.array(cfg.target_scale)
    target = o.forward(tgt_mat, s.rest, np.zeros_like(s.rest), None, dt=cfg.dt, steps=cfg.steps, tol=tol,
                       max_iter=20000, gravity=W.GRAVITY, precond=pc)[0]
    L_o, dL = oracle_mod.loss_l2(tx, target)
    loss, grad = b.loss_l2(traj, to_cuda(target, torch.float64))
    assert float(loss[0]) == pytest.approx(L_o, rel=1e-9)
    assert close(to_np(grad), dL, 1e-9)
    g = b.backward(to_cuda(dL, torch.float64))
    go = o.backward(s.material, tx, tv, dL, dt=cfg.dt, steps=cfg.steps, tol=tol, max_iter=20000, gravity=W.GRAVITY,
                    precond=pc)
    gm = to_np(g["material"])[0]
    for k in (0, 2, 3):
        assert gm[k] == pytest.approx(go["material"][k], rel=1e-10)
    assert gm[1] == 0.0
    # every gradient of phi (Eq. 2) to the FP64 bar of 1e-10, by norm and entry by entry
    for name in ("x0", "v0", "forces"):
        a, r = to_np(g[name]), go[name]
        assert close(a, r, 1e-10), (name, rel(a, r), max_entry_err(a, r))
    assert int(g["status"][0]) == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_velocity_increment_forces_match_oracle(oracle_mod, prec):
    """Corrective forces as velocity increments (force_mode "velocity"): 10x10 sheet, two
    top corners pinned, 20 steps, seeded increments of 1e-3 m/s (also on the pinned
    vertices, where they must have no effect), against the oracle in the same mode:
    FP64 positions to 1e-10 m and gradients to 1e-10; FP32 positions to 1e-5 m and
    gradients to 1e-3.  Checkpoint-and-recompute (every 3 steps) gives bitwise the same
    gradients."""
    from paper_2203_11938_gb300 import sim

    cfg = W.config1()
    s = cfg.sheets[0]
    T = cfg.steps
    rng = np.random.Generator(np.random.PCG64(7))
    F = 1e-3 * rng.normal(size=(T, s.n, 3))
    dtype = torch.float64 if prec == "f64" else torch.float32
    rnd = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if prec == "f32" else (lambda a: np.asarray(a))
    x0, Fi, mat = rnd(s.rest), rnd(F), rnd(s.material)
    tol = 1e-12 if prec == "f64" else 1e-8
    o = oracle_sims(oracle_mod, cfg.sheets)[0]
    kw = dict(dt=cfg.dt, steps=T, tol=1e-12, max_iter=20000, gravity=W.GRAVITY)
    tx, tv, _, st = o.forward(mat, x0, np.zeros_like(x0), Fi, force_mode=1, **kw)
    target = o.forward(mat * np.array(cfg.target_scale), x0, np.zeros_like(x0), Fi, force_mode=1, **kw)[0]
    _, dL = oracle_mod.loss_l2(tx, target)
    go = o.backward(mat, tx, tv, dL, forces=Fi, force_mode=1, **kw)
    assert st == 0 and go["status"] == 0
    res = []
    for ckpt in (0, 3):
        b = sim.ClothBatch([(s.rest, s.tris, s.pinned)], steps=T, dt=cfg.dt, precision=prec, cg_tol=tol,
                           cg_max_iter=20000, checkpoint_every=ckpt, force_mode="velocity")
        dF = to_cuda(Fi, dtype)
        traj, status = b.forward(to_cuda(mat[None], dtype), to_cuda(x0, dtype), torch.zeros(s.n, 3, dtype=dtype,
                                 device="cuda"), dF)
        _, dLg = b.loss_l2(traj, to_cuda(target, dtype))
        g = b.backward(dLg)
        torch.cuda.synchronize()
        assert int(status[0]) == 0 and int(g["status"][0]) == 0
        res.append((to_np(traj), to_np(g["material"])[0], to_np(g["forces"]), to_np(g["x0"]), to_np(g["v0"])))
    for a, c in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, c)
    traj, gm, gF, gx, gv = res[0]
    pos_tol, g_tol = (1e-10, 1e-10) if prec == "f64" else (1e-5, 1e-3)
    assert np.abs(traj - tx).max() <= pos_tol
    for k in (0, 2, 3):
        assert gm[k] == pytest.approx(go["material"][k], rel=g_tol), k
    for name, a in (("forces", gF), ("v0", gv), ("x0", gx)):
        assert close(a, go[name], g_tol), (name, rel(a, go[name]), max_entry_err(a, go[name]))
    pin = s.pinned.astype(bool)
    assert np.all(gF[:, pin] == 0.0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_air_drag_matches_oracle(oracle_mod, prec):
    """Air drag of a wind (rho_air = 1 kg/m^3, wind 0.5 m/s sideways and 0.1 m/s up) on the
    10x10 sheet with seeded forces, 20 steps, against the oracle with the same drag:
    FP64 positions to 1e-10 m and gradients (material, forces, x0, v0, wind) to 1e-10;
    FP32 positions to 1e-5 m and gradients to 1e-3.  Checkpoint-and-recompute (every 3
    steps) gives bitwise the same gradients."""
    from paper_2203_11938_gb300 import sim

    cfg = W.config1()
    s = cfg.sheets[0]
    T = cfg.steps
    rng = np.random.Generator(np.random.PCG64(11))
    F = 1e-4 * rng.normal(size=(T, s.n, 3))
    w = np.array([0.5, 0.0, 0.1])
    dtype = torch.float64 if prec == "f64" else torch.float32
    rnd = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if prec == "f32" else (lambda a: np.asarray(a))
    x0, Fi, mat, wi = rnd(s.rest), rnd(F), rnd(s.material), rnd(w)
    tol = 1e-12 if prec == "f64" else 1e-8
    o = oracle_sims(oracle_mod, cfg.sheets)[0]
    kw = dict(dt=cfg.dt, steps=T, tol=1e-12, max_iter=20000, gravity=W.GRAVITY, air_density=1.0)
    tx, tv, _, st = o.forward(mat, x0, np.zeros_like(x0), Fi, wind=wi, **kw)
    target = o.forward(mat * np.array(cfg.target_scale), x0, np.zeros_like(x0), Fi, wind=0.5 * wi, **kw)[0]
    _, dL = oracle_mod.loss_l2(tx, target)
    go = o.backward(mat, tx, tv, dL, forces=Fi, wind=wi, **kw)
    assert st == 0 and go["status"] == 0
    res = []
    for ckpt in (0, 3):
        b = sim.ClothBatch([(s.rest, s.tris, s.pinned)], steps=T, dt=cfg.dt, precision=prec, cg_tol=tol,
                           cg_max_iter=20000, checkpoint_every=ckpt, air_density=1.0)
        b.set_wind(to_cuda(wi[None], dtype))
        traj, status = b.forward(to_cuda(mat[None], dtype), to_cuda(x0, dtype),
                                 torch.zeros(s.n, 3, dtype=dtype, device="cuda"), to_cuda(Fi, dtype))
        _, dLg = b.loss_l2(traj, to_cuda(target, dtype))
        g = b.backward(dLg)
        gw = b.wind_gradient()
        torch.cuda.synchronize()
        assert int(status[0]) == 0 and int(g["status"][0]) == 0
        res.append((to_np(traj), to_np(g["material"])[0], to_np(g["forces"]), to_np(g["x0"]), to_np(g["v0"]),
                    to_np(gw)[0]))
    for a, c in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, c)
    traj, gm, gF, gx, gv, gwv = res[0]
    pos_tol, g_tol = (1e-10, 1e-10) if prec == "f64" else (1e-5, 1e-3)
    assert np.abs(traj - tx).max() <= pos_tol
    for k in (0, 2, 3):
        assert gm[k] == pytest.approx(go["material"][k], rel=g_tol), k
    for name, a in (("forces", gF), ("x0", gx), ("v0", gv), ("wind", gwv)):
        assert close(a, go[name], g_tol), (name, rel(a, go[name]), max_entry_err(a, go[name]))


@pytest.mark.parametrize("warm", [False, True])
def test_config2_fp32_positions_and_gradients(oracle_mod, warm):
    """32x32 sheet, top edge pinned, 60 steps of 1/60 s with seeded per-vertex forces,
    FP32 path (CG tol 1e-8) vs the FP64 oracle (tol 1e-10) run on the same inputs (the
    FP32 API receives x0, forces and material rounded to float; the oracle is given
    those values): max position error <= 1e-5 m, gradients w.r.t. Y, k_b, rho, forces
    and x0 within 1e-3 relative, with solves started from zero, and warm-started (each from
    the previous step's solution) at CG tol 1e-9."""
    cfg = W.config2()
    s = cfg.sheets[0]
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    x0, F, mat = f32(s.rest), f32(s.forces), f32(s.material)
    # warm starts stop at a different point within the tolerance: at 1e-8 the forces'
    # gradient is off by 1.08e-3 in its largest entry, at 1e-9 well inside the bounds
    b = make_batch(cfg.sheets, steps=cfg.steps, dt=cfg.dt, precision="f32", tol=cfg.cg_tol * (0.1 if warm else 1.0),
                   warm=warm)
    traj, status = b.forward(to_cuda(mat[None], torch.float32), to_cuda(x0, torch.float32),
                             torch.zeros(s.n, 3, dtype=torch.float32, device="cuda"), to_cuda(F, torch.float32))
    o = oracle_sims(oracle_mod, cfg.sheets)[0]
    tx, tv, _, st = o.forward(mat, x0, np.zeros_like(x0), F, dt=cfg.dt, steps=cfg.steps, tol=1e-10, max_iter=20000,
                              gravity=W.GRAVITY)
    assert int(status[0]) == 0 and st == 0
    err = np.abs(to_np(traj)[-1] - tx[-1]).max()
    assert err <= 1e-5, err
    tgt = o.forward(mat * np.array(cfg.target_scale), x0, np.zeros_like(x0), F, dt=cfg.dt, steps=cfg.steps,
                    tol=1e-10, max_iter=20000, gravity=W.GRAVITY)[0]
    _, dL = oracle_mod.loss_l2(tx, tgt)
    _, dLg = b.loss_l2(traj, to_cuda(tgt, torch.float32))
    g = b.backward(dLg)
    go = o.backward(mat, tx, tv, dL, dt=cfg.dt, steps=cfg.steps, tol=1e-10, max_iter=20000, gravity=W.GRAVITY)
    gm = to_np(g["material"])[0]
    for k in (0, 2, 3):
        assert gm[k] == pytest.approx(go["material"][k], rel=1e-3), k
    for name in ("forces", "x0"):
        a = to_np(g[name])
        assert close(a, go[name], 1e-3), (name, rel(a, go[name]), max_entry_err(a, go[name]))



def test_config2_gradients_vs_finite_differences():
    """Adjoint against central differences (h = 1e-3 relative) of the forward map for Y,
    k_b and rho on the 32x32 workload.  The differences are taken on the FP64 path
    (tol 1e-12) and Richardson-extrapolated from h and h/2 (error O(h^4)); the FP64
    adjoint must agree to 1e-7 and the FP32 adjoint to 1e-3."""
    cfg = W.config2()
    s = cfg.sheets[0]
    mat = s.material.copy()
    grads = {}
    for prec, tol in (("f64", 1e-12), ("f32", cfg.cg_tol)):
        dt_ = _dtype(prec)
        b = make_batch(cfg.sheets, steps=cfg.steps, dt=cfg.dt, precision=prec, tol=tol)
        x0 = to_cuda(s.rest, dt_)
        v0 = torch.zeros_like(x0)
        F = to_cuda(s.forces, dt_)
        tgt, _ = b.forward(to_cuda(mat * np.array(cfg.target_scale), dt_)[None], x0, v0, F)
        tgt = tgt.clone()
        traj, _ = b.forward(to_cuda(mat, dt_)[None], x0, v0, F)
        _, dL = b.loss_l2(traj, tgt)
        grads[prec] = to_np(b.backward(dL, want=("material",))["material"])[0]
        if prec == "f64":
            fd = {}
            for k in (0, 2, 3):
                cd = []
                for h in (1e-3 * mat[k], 0.5e-3 * mat[k]):
                    Ls = []
                    for sgn in (1.0, -1.0):
                        m2 = mat.copy()
                        m2[k] += sgn * h
                        tr, _ = b.forward(to_cuda(m2, dt_)[None], x0, v0, F)
                        Ls.append(float(b.loss_l2(tr, tgt, want_grad=False)[0][0]))
                    cd.append((Ls[0] - Ls[1]) / (2 * h))
                fd[k] = (4 * cd[1] - cd[0]) / 3
    for k in (0, 2, 3):
        assert grads["f64"][k] == pytest.approx(fd[k], rel=1e-7), k
        assert grads["f32"][k] == pytest.approx(fd[k], rel=1e-3), k


def test_batch256_full_size_sampled_sheets(oracle_mod):
    """The 256-sheet benchmark batch at full size (100 steps, FP32, CG tol 1e-7, captured
    graph): the two smallest sheets, recomputed one by one by the oracle, match in
    positions (1e-5 m) and material gradients (1e-3 relative)."""
    cfg = W.config4()
    f32 = torch.float32
    b = make_batch(cfg.sheets, steps=cfg.steps, dt=cfg.dt, precision="f32", tol=cfg.cg_tol, max_iter=cfg.cg_max_iter)
    mat = np.stack([s.material for s in cfg.sheets])
    x0 = np.concatenate([s.rest for s in cfg.sheets])
    traj, status = b.forward(to_cuda(mat, f32), to_cuda(x0, f32), torch.zeros(x0.shape, dtype=f32, device="cuda"), None)
    dL = torch.zeros_like(traj)
    dL[1:] = 0.1  # loss = 0.1 * sum of all coordinates over t >= 1
    g = b.backward(dL)
    traj_np = split(to_np(traj), b.sheet_sizes, axis=1)
    gm = to_np(g["material"])
    order = np.argsort([s.n for s in cfg.sheets])[:2]
    f32r = lambda a: np.asarray(a, np.float32).astype(np.float64)
    for k in order:
        s = cfg.sheets[k]
        o = oracle_mod.OracleSim(s.rest, s.tris, s.pinned)
        m = f32r(s.material)
        tx, tv, _, st = o.forward(m, f32r(s.rest), np.zeros_like(s.rest), None, dt=cfg.dt, steps=cfg.steps, tol=1e-10,
                                  max_iter=20000, gravity=W.GRAVITY)
        assert np.abs(traj_np[k][-1] - tx[-1]).max() <= 1e-5
        dl = np.zeros_like(tx)
        dl[1:] = 0.1
        go = o.backward(m, tx, tv, dl, dt=cfg.dt, steps=cfg.steps, tol=1e-10, max_iter=20000, gravity=W.GRAVITY)
        for q in (0, 2, 3):
            assert gm[k, q] == pytest.approx(go["material"][q], rel=1e-3), (k, q)


def test_batched_sheets_match_their_own_oracles(oracle_mod):
    """Three sheets of different sizes and materials in one batch, FP64: each sheet's
    trajectory and material gradient equals its own oracle run."""
    sheets = sheets_mixed(seed=11)
    steps, dt, tol = 8, 1 / 30, 1e-12
    b, traj, status, refs = _rollout_both(oracle_mod, sheets, steps=steps, dt=dt, prec="f64", tol=tol, oracle_tol=tol)
    parts = split(to_np(traj), b.sheet_sizes, axis=1)
    for k, ref in enumerate(refs):
        assert np.abs(parts[k] - ref[0]).max() < 1e-10
    rng = np.random.default_rng(12)
    dLs = [rng.normal(size=ref[0].shape) for ref in refs]
    g = b.backward(to_cuda(np.concatenate(dLs, axis=1), torch.float64))
    gm = to_np(g["material"])
    for k, (s, o) in enumerate(zip(sheets, oracle_sims(oracle_mod, sheets))):
        go = o.backward(s.material, refs[k][0], refs[k][1], dLs[k], dt=dt, steps=steps, tol=tol, max_iter=20000,
                        gravity=W.GRAVITY)
        for q in (0, 2, 3):
            assert gm[k, q] == pytest.approx(go["material"][q], rel=1e-9)


@pytest.mark.parametrize("warm", [False, True])
def test_checkpointing_and_exec_modes_agree(oracle_mod, warm):
    """Checkpoint-and-recompute (C = 3 of 10 steps), the plain host-polled CG and the CG
    kernel schedules (resident or per-entry grid, with or without a per-sheet cluster solver
    and its on-chip and dense variants, and the autotuned one) give bitwise the same
    trajectory and gradients as the captured-graph run without checkpoints; with
    warm-started solves too (the recompute replays the stored starting vectors)."""
    sheets = sheets_mixed(seed=21)[:2]
    steps, dt = 10, 1 / 30
    res = []
    for exec_mode, ckpt, sched in (("graph", 0, 3), ("graph", 3, 2), ("plain", 3, 3), ("plain", 0, 2), ("graph", 0, -1),
                                   ("graph", 3, 6), ("plain", 0, 7), ("graph", 0, 22), ("plain", 3, 15)):
        b = make_batch(sheets, steps=steps, dt=dt, precision="f32", tol=1e-6, exec_mode=exec_mode, ckpt=ckpt,
                       schedule=sched, warm=warm)
        x0 = to_cuda(np.concatenate([s.rest for s in sheets]), torch.float32)
        mat = to_cuda(_materials(sheets), torch.float32)
        traj, st = b.forward(mat, x0, torch.zeros_like(x0), None)
        dL = torch.ones_like(traj)
        g = b.backward(dL)
        g2 = b.backward(dL)  # a second backward on the same forward recomputes every segment
        res.append((to_np(traj), to_np(g["material"]), to_np(g["x0"]), to_np(g2["material"])))
    for r in res[1:]:
        np.testing.assert_array_equal(r[0], res[0][0])
        np.testing.assert_array_equal(r[1], res[0][1])
        np.testing.assert_array_equal(r[2], res[0][2])
    for r in res:
        np.testing.assert_array_equal(r[3], r[1])


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_sheet_solver_matches_device_loop_bitwise(precision):
    """The per-sheet cluster solver (schedule bit 2) and its on-chip variant (bit 3: matrix
    and gathered vectors in the shared memory of up to 16 CTAs, neighbours read through
    distributed shared memory) and its dense classes (bit 4: two work entries per CTA, two
    CTAs per SM) against the device loop alone, on sheets of 1 to 40 work entries (every
    cluster size and entries-per-CTA class, including the 16-CTA clusters of 2 and 3 entries
    per CTA; in FP64 the largest sheets do not fit on chip and take the first solver):
    bitwise the same trajectory, gradients and per-sheet iteration counts, in graph and
    plain execution."""
    rng = np.random.Generator(np.random.PCG64(8))
    sheets = []
    for N in (16, 20, 30, 40, 50, 64, 70, 100):
        rest, tris = W.grid_mesh(N)
        sheets.append(W.Sheet(N, rest, tris, W.pins(N, "top2"), W.sample_material(rng), None))
    dtype = torch.float32 if precision == "f32" else torch.float64
    res = []
    for exec_mode, sched in (("graph", 2), ("graph", 6), ("plain", 7), ("graph", 14), ("plain", 15), ("graph", 22),
                             ("plain", 23)):
        b = make_batch(sheets, steps=4, dt=1 / 30, precision=precision, tol=1e-7, exec_mode=exec_mode, schedule=sched)
        assert b.matrix_info()["cg_schedule"] == sched  # bit 3: the on-chip solver holds at least one sheet
        x0 = to_cuda(np.concatenate([s.rest for s in sheets]), dtype)
        mat = to_cuda(_materials(sheets), dtype)
        traj, st = b.forward(mat, x0, torch.zeros_like(x0), None)
        g = b.backward(torch.ones_like(traj))
        torch.cuda.synchronize()
        assert int(st.max()) == 0 and int(g["status"].max()) == 0
        it = [b.sheet_iterations(ph) for ph in ("forward", "adjoint")]
        res.append((to_np(traj), to_np(g["material"]), to_np(g["x0"]), it))
    for r in res[1:]:
        np.testing.assert_array_equal(r[0], res[0][0])
        np.testing.assert_array_equal(r[1], res[0][1])
        np.testing.assert_array_equal(r[2], res[0][2])
        for (m1, t1), (m0, t0) in zip(r[3], res[0][3]):
            np.testing.assert_array_equal(m1, m0)
            np.testing.assert_array_equal(t1, t0)


@pytest.mark.parametrize("sched", [6, 22])
def test_launch_order_changes_no_result(sched):
    """The per-sheet solver launches each size class's sheets in order of their last
    solve's iteration counts (k_order_lists).  The first call of a batch runs in the
    classes' own order (no counts yet), later calls in the sorted order, so repeated calls
    with the same inputs check that the order changes no result: bitwise the same
    trajectory and gradients, on 24 sheets of 4 to 16 work
    entries with sampled materials (several sheets per class, so the order moves)."""
    rng = np.random.Generator(np.random.PCG64(11))
    sheets = []
    for N in (30, 32, 34, 40, 44, 48, 52, 56, 60, 64, 30, 36, 42, 50, 58, 64, 32, 46, 54, 62, 28, 38, 56, 64):
        rest, tris = W.grid_mesh(N)
        sheets.append(W.Sheet(N, rest, tris, W.pins(N, "top2"), W.sample_material(rng), None))
    f32 = torch.float32
    b = make_batch(sheets, steps=6, dt=1 / 30, precision="f32", tol=1e-7, schedule=sched)
    assert b.matrix_info()["cg_schedule"] == sched
    x0 = to_cuda(np.concatenate([s.rest for s in sheets]), f32)
    mat = to_cuda(_materials(sheets), f32)
    res = []
    for _ in range(3):
        traj, st = b.forward(mat, x0, torch.zeros_like(x0), None)
        g = b.backward(torch.ones_like(traj))
        torch.cuda.synchronize()
        assert int(st.max()) == 0 and int(g["status"].max()) == 0
        res.append((to_np(traj), to_np(g["material"]), to_np(g["x0"])))
    # the iteration counts differ between sheets of a class, so the sorted order is not
    # the classes' own order
    its = b.sheet_iterations("forward")[1]
    assert len(set(int(v) for v in its)) > 8
    for r in res[1:]:
        for a, a0 in zip(r, res[0]):
            np.testing.assert_array_equal(a, a0)


def test_cg_maxiter_status_and_free_fall():
    """cg_max_iter = 1 marks every sheet CG_MAXITER without failing the call; an
    unpinned sheet under gravity falls exactly as implicit Euler predicts."""
    from paper_2203_11938_gb300 import sim

    rest, tris = W.grid_mesh(6)
    b = sim.ClothBatch([(rest, tris, None)], steps=5, dt=1 / 30, precision="f64", cg_tol=1e-12, cg_max_iter=4000)
    x0 = to_cuda(rest, torch.float64)
    traj, status = b.forward(to_cuda(MAT[None], torch.float64), x0, torch.zeros_like(x0), None)
    assert int(status[0]) == 0
    g = np.array(W.GRAVITY)
    h = 1 / 30
    for t in range(6):
        np.testing.assert_allclose(to_np(traj[t]), rest + h * h * g * t * (t + 1) / 2, atol=1e-9)
    rng = np.random.default_rng(0)
    b1 = sim.ClothBatch([(rest, tris, W.pins(6, "top2"))], steps=2, dt=1 / 30, precision="f32", cg_tol=1e-9,
                        cg_max_iter=1)
    x1 = to_cuda(rest + 0.01 * rng.normal(size=rest.shape), torch.float32)
    _, status = b1.forward(to_cuda(MAT[None], torch.float32), x1, torch.zeros_like(x1), None)
    assert int(status[0]) & sim.STATUS_CG_MAXITER


def test_pinhole_loss_matches_oracle(oracle_mod):
    cfg = W.config1()
    s = cfg.sheets[0]
    b = make_batch(cfg.sheets, steps=4, dt=cfg.dt, precision="f64", tol=1e-10)
    rng = np.random.default_rng(3)
    traj = s.rest[None] + 0.05 * rng.normal(size=(5, s.n, 3))
    uv = rng.normal(scale=20.0, size=(5, s.n, 2))
    cam = (500.0, 0.5, 0.5, 2.0)
    L_o, g_o = oracle_mod.loss_pinhole(traj, uv, cam)
    loss, grad = b.loss_pinhole(to_cuda(traj, torch.float64), to_cuda(uv, torch.float64), cam)
    assert float(loss[0]) == pytest.approx(L_o, rel=1e-12)
    assert close(to_np(grad), g_o, 1e-12)


def test_autograd_function_matches_direct_calls():
    from paper_2203_11938_gb300 import sim

    sheets = sheets_mixed(seed=5)[:2]
    b = make_batch(sheets, steps=4, dt=1 / 30, precision="f64", tol=1e-12)
    mat = to_cuda(_materials(sheets), torch.float64).requires_grad_(True)
    x0 = to_cuda(np.concatenate([s.rest for s in sheets]), torch.float64).requires_grad_(True)
    v0 = torch.zeros_like(x0, requires_grad=True)
    traj = sim.cloth_trajectory(b, mat, x0, v0)
    (traj ** 2).sum().backward()
    g = b.backward(2 * traj.detach())
    torch.testing.assert_close(mat.grad, g["material"], rtol=0, atol=0)
    torch.testing.assert_close(x0.grad, g["x0"], rtol=0, atol=0)


def test_pinned_vertex_with_initial_velocity_is_flagged():
    """A nonzero v0 on a pinned vertex sets PINNED_VELOCITY_NONZERO on that sheet only (the
    kinematic pin then moves at v0); v0 = 0 on every pin leaves the status clear."""
    from paper_2203_11938_gb300 import sim

    sheets = sheets_mixed(seed=31)[:2]
    b = make_batch(sheets, steps=2, dt=1 / 30, precision="f64", tol=1e-10)
    x0 = to_cuda(np.concatenate([s.rest for s in sheets]), torch.float64)
    mat = to_cuda(_materials(sheets), torch.float64)
    v0 = torch.zeros_like(x0)
    _, st = b.forward(mat, x0, v0, None)
    assert int(st.max()) == 0
    n0 = sheets[0].n
    k = int(np.flatnonzero(sheets[1].pinned)[0])
    v0[n0 + k, 2] = 1e-3
    traj, st = b.forward(mat, x0, v0, None)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    assert int(st[1]) & sim.STATUS_PINNED_VELOCITY_NONZERO
    # the pin moved at its starting velocity
    np.testing.assert_allclose(to_np(traj)[2, n0 + k], sheets[1].rest[k] + np.array([0, 0, 2e-3 / 30]), atol=1e-15)
