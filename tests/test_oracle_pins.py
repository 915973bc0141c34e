"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

The oracle restates Sec. 3.1 (Eq. 3-5) with the energy readings R1/R2 and the
clamped geometric stiffness R6.  Nothing here re-derives its formulas: each test
checks a property that a dropped term, a wrong sign, a wrong index or a
transposed operand would break (closed forms, invariances, finite differences,
a textbook dense solve, the implicit-Euler free fall, and the adjoint against
Richardson-extrapolated central differences of the forward map).
"""
import math

import numpy as np
import pytest

from paper_2203_11938_gb300 import workloads as W

MAT = np.array([1.0e3, 0.3, 1.0e-4, 0.1])


def _lame(Y, nu):
    return Y / (2 * (1 + nu)), Y * nu / (1 - nu * nu)


def _rand_rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _small_sheet(oracle_mod, N=4, pin="top2"):
    rest, tris = W.grid_mesh(N)
    return oracle_mod.OracleSim(rest, tris, W.pins(N, pin)), rest


# ----------------------------------------------------------------- membrane
def test_membrane_uniaxial_closed_form(oracle_mod):
    """Uniform stretch s along e1 of a right triangle: G = diag(g, 0), g = (s^2-1)/2,
    so E = A0 (mu g^2 + lambda/2 g^2) (StVK with plane-stress Lame constants)."""
    rest = np.array([0, 0, 0, 1.0, 0, 0, 0, 1.0, 0])
    for s in (0.7, 1.0, 1.3):
        x = rest.reshape(3, 3) * np.array([s, 1.0, 1.0])
        E, _, _ = oracle_mod.membrane_element(rest, x.ravel(), 1e3, 0.3)
        mu, lam = _lame(1e3, 0.3)
        g = (s * s - 1) / 2
        assert E == pytest.approx(0.5 * (mu * g * g + 0.5 * lam * g * g), rel=1e-13, abs=1e-15)


def test_membrane_biaxial_and_shear_closed_form(oracle_mod):
    """Equi-biaxial stretch s: G = g I, E = A0 (2 mu g^2 + 2 lambda g^2);
    simple shear x += k y: G = [[0, k/2], [k/2, k^2/2]], E = A0 (mu (k^2/2 + k^4/4) + lambda k^4/8)."""
    rest = np.array([0, 0, 0, 2.0, 0, 0, 0, 1.0, 0])  # A0 = 1
    mu, lam = _lame(2e3, 0.25)
    s = 1.2
    x = rest.reshape(3, 3) * np.array([s, s, 1.0])
    E, _, _ = oracle_mod.membrane_element(rest, x.ravel(), 2e3, 0.25)
    g = (s * s - 1) / 2
    assert E == pytest.approx(2 * mu * g * g + 2 * lam * g * g, rel=1e-13)
    k = 0.3
    x = rest.reshape(3, 3).copy()
    x[:, 0] += k * x[:, 1]
    E, _, _ = oracle_mod.membrane_element(rest, x.ravel(), 2e3, 0.25)
    assert E == pytest.approx(mu * (k * k / 2 + k ** 4 / 4) + lam * k ** 4 / 8, rel=1e-13)


def test_membrane_rigid_invariance_and_rest(oracle_mod):
    rng = np.random.default_rng(3)
    rest = rng.normal(size=9)
    E0, g0, H0 = oracle_mod.membrane_element(rest, rest, 1e3, 0.3)
    assert abs(E0) < 1e-20 and np.abs(g0).max() < 1e-12
    x = rest + 0.1 * rng.normal(size=9)
    E1, _, _ = oracle_mod.membrane_element(rest, x, 1e3, 0.3)
    R = _rand_rot(rng)
    xr = (x.reshape(3, 3) @ R.T + rng.normal(size=3)).ravel()
    E2, _, _ = oracle_mod.membrane_element(rest, xr, 1e3, 0.3)
    assert E2 == pytest.approx(E1, rel=1e-12)
    # Hessian at rest annihilates the 6 rigid modes
    rig = []
    for c in range(3):
        t = np.zeros((3, 3)); t[:, c] = 1; rig.append(t.ravel())
    P = rest.reshape(3, 3)
    for axis in np.eye(3):
        rig.append(np.cross(axis, P).ravel())
    for r in rig:
        assert np.abs(H0 @ r).max() < 1e-9 * np.abs(H0).max()


def test_membrane_grad_hess_vs_fd(oracle_mod):
    rng = np.random.default_rng(4)
    rest = rng.normal(size=9)
    x = rest + 0.2 * rng.normal(size=9)
    E, g, H = oracle_mod.membrane_element(rest, x, 1e3, 0.3)
    h = 1e-6
    for i in range(9):
        d = np.zeros(9); d[i] = h
        Ep, gp, _ = oracle_mod.membrane_element(rest, x + d, 1e3, 0.3)
        Em, gm, _ = oracle_mod.membrane_element(rest, x - d, 1e3, 0.3)
        assert (Ep - Em) / (2 * h) == pytest.approx(g[i], rel=1e-6, abs=1e-6)
        np.testing.assert_allclose((gp - gm) / (2 * h), H[i], rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(H, H.T, atol=1e-10)


# ------------------------------------------------------------------ bending
def _hinge(theta):
    """Shared edge (0,0,0)-(1,0,0); wing a = (0.5, 1, 0) fixed; wing b rotated about
    the edge so the two triangles are folded by `theta` from flat."""
    return np.array([0, 0, 0, 1, 0, 0, 0.5, 1, 0, 0.5, -math.cos(theta), math.sin(theta)], float)


def test_dihedral_closed_form(oracle_mod):
    for th in (-2.0, -0.5, 0.0, 0.3, 1.0, 2.5):
        assert abs(oracle_mod.dihedral(_hinge(th))) == pytest.approx(abs(th), abs=1e-13)
    # sign flips with the fold direction, magnitude equal
    assert oracle_mod.dihedral(_hinge(0.4)) == pytest.approx(-oracle_mod.dihedral(_hinge(-0.4)), abs=1e-14)


def test_bending_energy_hinge_closed_form(oracle_mod):
    """Two-triangle hinge: E = 1/2 kb w theta^2 with w = 3 |e|^2 / (A1 + A2) = 3 here."""
    rest = _hinge(0.0).reshape(4, 3)
    tris = np.array([[0, 1, 2], [1, 0, 3]], np.int32)
    sim = oracle_mod.OracleSim(rest, tris)
    v, w, th0 = sim.hinges()
    assert v.shape == (1, 4) and w[0] == pytest.approx(3.0) and th0[0] == pytest.approx(0.0, abs=1e-15)
    for th in (0.2, -0.7, 1.4):
        E, fm, fb = sim.energy_forces([0.0, 0.3, 2e-3, 0.1], _hinge(th).reshape(4, 3))
        assert E == pytest.approx(0.5 * 2e-3 * 3.0 * th * th, rel=1e-12)
        assert np.abs(fm).max() < 1e-14  # Y = 0: no membrane force


# --------------------------------------------------------------- mesh level
def test_grid_topology_counts(oracle_mod):
    for N in (2, 3, 10, 17):
        rest, tris = W.grid_mesh(N)
        sim = oracle_mod.OracleSim(rest, tris)
        n, m, e = W.grid_counts(N)
        assert (sim.n, sim.m, sim.hinges()[0].shape[0]) == (n, m, e)


def test_lumped_mass_totals(oracle_mod):
    sim, rest = _small_sheet(oracle_mod, 7)
    m = sim.mass(0.25)
    assert m.sum() == pytest.approx(0.25 * 1.0, rel=1e-13)  # rho * area of the 1 m^2 sheet
    assert (m > 0).all()


def _grid_vertex_mass(a, b, N, rho):
    """Lumped mass of grid vertex (a, b) of the alternating-diagonal N x N sheet (Eq. 3:
    each triangle gives a third of rho A0 to each of its corners), counted from the
    geometry alone.  Cell (i, j) is cut along the diagonal from (i, j) to (i+1, j+1) when
    i + j is even, else from (i+1, j) to (i, j+1); a corner on the cut belongs to both of
    the cell's triangles, the other two corners to one each.  A0 = h^2 / 2, h = 1/(N-1)."""
    h = 1.0 / (N - 1)
    count = 0
    for i, j in ((a - 1, b - 1), (a, b - 1), (a - 1, b), (a, b)):
        if not (0 <= i < N - 1 and 0 <= j < N - 1):
            continue
        ends = {(i, j), (i + 1, j + 1)} if (i + j) % 2 == 0 else {(i + 1, j), (i, j + 1)}
        count += 2 if (a, b) in ends else 1
    return rho * count * (h * h / 2.0) / 3.0


@pytest.mark.parametrize("N", [2, 3, 6, 7, 12])
def test_lumped_mass_per_vertex_closed_form(oracle_mod, N):
    """Every vertex's lumped mass against the count of incident triangles on the grid:
    interior vertices alternate between 8 triangles (i + j even: every surrounding cell is
    cut through them) and 4 (odd), edge and corner vertices take the cells that exist.
    A mass lumped onto the wrong corners keeps the total and fails here."""
    rest, tris = W.grid_mesh(N)
    sim = oracle_mod.OracleSim(rest, tris)
    rho = 0.37
    m = sim.mass(rho)
    expect = np.array([_grid_vertex_mass(k % N, k // N, N, rho) for k in range(N * N)])
    np.testing.assert_allclose(m, expect, rtol=1e-13, atol=0)
    if N >= 4:  # the two interior classes really differ (8 vs 4 triangles)
        h2 = (1.0 / (N - 1)) ** 2
        assert m[1 * N + 1] == pytest.approx(rho * 8 * h2 / 6, rel=1e-13)
        assert m[1 * N + 2] == pytest.approx(rho * 4 * h2 / 6, rel=1e-13)


def test_forces_zero_at_rest_net_force_torque(oracle_mod):
    rng = np.random.default_rng(5)
    sim, rest = _small_sheet(oracle_mod, 6, "none")
    E, fm, fb = sim.energy_forces(MAT, rest)
    assert abs(E) < 1e-25 and np.abs(fm).max() < 1e-12 and np.abs(fb).max() < 1e-16
    x = rest + 0.05 * rng.normal(size=rest.shape)
    E, fm, fb = sim.energy_forces(MAT, x)
    for f in (fm, fb):
        scale = np.abs(f).max()
        assert np.abs(f.sum(0)).max() < 1e-11 * scale * sim.n
        assert np.abs(np.cross(x, f).sum(0)).max() < 1e-11 * scale * sim.n
    R = _rand_rot(rng)
    E2, _, _ = sim.energy_forces(MAT, x @ R.T + 3.0)
    assert E2 == pytest.approx(E, rel=1e-11)


def test_forces_are_negative_energy_gradient(oracle_mod):
    rng = np.random.default_rng(6)
    sim, rest = _small_sheet(oracle_mod, 4, "none")
    x = rest + 0.05 * rng.normal(size=rest.shape)
    E, fm, fb = sim.energy_forces(MAT, x)
    f = fm + fb
    h = 1e-6
    for _ in range(12):
        i, c = rng.integers(sim.n), rng.integers(3)
        xp = x.copy(); xp[i, c] += h
        xm = x.copy(); xm[i, c] -= h
        fd = (sim.energy_forces(MAT, xp)[0] - sim.energy_forces(MAT, xm)[0]) / (2 * h)
        assert -fd == pytest.approx(f[i, c], rel=1e-6, abs=1e-8)


def test_exact_hessian_symmetric_and_fd_of_forces(oracle_mod):
    rng = np.random.default_rng(7)
    sim, rest = _small_sheet(oracle_mod, 4, "none")
    x = rest + 0.05 * rng.normal(size=rest.shape)
    H = sim.hessian_dense(MAT, x, eta=0.0)
    np.testing.assert_allclose(H, H.T, atol=1e-9 * np.abs(H).max())
    h = 1e-6
    for k in rng.choice(3 * sim.n, 8, replace=False):
        d = np.zeros(3 * sim.n); d[k] = h
        _, fmp, fbp = sim.energy_forces(MAT, (x.ravel() + d).reshape(-1, 3))
        _, fmm, fbm = sim.energy_forces(MAT, (x.ravel() - d).reshape(-1, 3))
        col = -((fmp + fbp) - (fmm + fbm)).ravel() / (2 * h)
        np.testing.assert_allclose(col, H[:, k], rtol=1e-5, atol=1e-5 * np.abs(H).max())


def test_clamped_hessian_psd_in_compression(oracle_mod):
    """R6: the clamped Hessian is symmetric PSD on a compressed, crumpled sheet where
    the exact Hessian is indefinite."""
    rng = np.random.default_rng(8)
    sim, rest = _small_sheet(oracle_mod, 5, "none")
    xc = rest * 0.9 + 0.01 * rng.normal(size=rest.shape)  # compressed
    Hc = sim.hessian_dense(MAT, xc, eta=1e-3)
    He = sim.hessian_dense(MAT, xc, eta=0.0)
    np.testing.assert_allclose(Hc, Hc.T, atol=1e-9 * np.abs(Hc).max())
    assert np.linalg.eigvalsh(He).min() < -1e-3  # the exact one is indefinite here
    assert np.linalg.eigvalsh(Hc).min() > -1e-8 * np.abs(Hc).max()


@pytest.mark.parametrize("stretch", [0.9, 1.0, 1.1])
def test_clamped_hessian_closed_form_uniform_biaxial(oracle_mod, stretch):
    """Single right triangle (Dm = I, A0 = 1/2) under uniform biaxial stretch s: the
    2nd Piola-Kirchhoff stress is sigma I, sigma = 2 g (mu + lambda), g = (s^2 - 1)/2.
    The clamp changes only the geometric term, so
    H - H~ = A0 * (sigma - sigma~+) * (L kron I3),  sigma~+ = (sigma + sqrt(sigma^2 + eps^2)) / 2,
    with L the Gram matrix of the nodal shape-function gradients [[2,-1,-1],[-1,1,0],[-1,0,1]]."""
    rest = np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]])
    sim = oracle_mod.OracleSim(rest, np.array([[0, 1, 2]], np.int32))
    x = rest * np.array([stretch, stretch, 1.0])
    eta = 1e-3
    He = sim.hessian_dense(MAT, x, eta=0.0)
    Hc = sim.hessian_dense(MAT, x, eta=eta)
    mu, lam = _lame(MAT[0], MAT[1])
    g = (stretch ** 2 - 1) / 2
    sigma = 2 * g * (mu + lam)
    eps = eta * MAT[0]
    splus = 0.5 * (sigma + math.sqrt(sigma * sigma + eps * eps))
    L = np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]], float)
    np.testing.assert_allclose(He - Hc, 0.5 * (sigma - splus) * np.kron(L, np.eye(3)), atol=1e-10 * np.abs(He).max())


def test_third_contraction_vs_fd_of_hessian(oracle_mod):
    """D(a^T H~(x) b)/dx against central differences of the assembled Hessian."""
    rng = np.random.default_rng(9)
    sim, rest = _small_sheet(oracle_mod, 4, "none")
    x = rest * np.array([0.97, 1.02, 1.0]) + 0.03 * rng.normal(size=rest.shape)
    a = rng.normal(size=rest.shape)
    b = rng.normal(size=rest.shape)
    for eta in (0.0, 1e-3):
        T = sim.third(MAT, x, a, b, eta=eta)
        h = 1e-6
        for k in rng.choice(3 * sim.n, 8, replace=False):
            d = np.zeros(3 * sim.n); d[k] = h
            Hp = sim.hessian_dense(MAT, (x.ravel() + d).reshape(-1, 3), eta=eta)
            Hm = sim.hessian_dense(MAT, (x.ravel() - d).reshape(-1, 3), eta=eta)
            fd = a.ravel() @ ((Hp - Hm) / (2 * h)) @ b.ravel()
            assert T.ravel()[k] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(T).max())


# -------------------------------------------------------------------- step
@pytest.mark.parametrize("precond", [0, 1])
def test_pcg_matches_dense_solve(oracle_mod, precond):
    """One step with PCG to tol 1e-13 (exact Hessian, eta = 0) equals numpy's dense
    solve of (M + h^2 H) dv = b, with the dense system built from finite differences of
    the forces (not from the oracle's own Hessian) on a stretched (all-tension) state."""
    rng = np.random.default_rng(10)
    sim, rest = _small_sheet(oracle_mod, 4, "top2")
    x = rest * np.array([1.05, 1.08, 1.0])
    x[:, 2] += 0.0
    v = 0.1 * rng.normal(size=rest.shape)
    v[sim.pinned.astype(bool)] = 0
    dt = 1.0 / 30.0
    g = np.array(W.GRAVITY)
    # H by central differences of the exact forces (all triangles in tension => H~ = H)
    N = 3 * sim.n
    H = np.zeros((N, N))
    h = 1e-6
    for k in range(N):
        d = np.zeros(N); d[k] = h
        _, a1, b1 = sim.energy_forces(MAT, (x.ravel() + d).reshape(-1, 3))
        _, a2, b2 = sim.energy_forces(MAT, (x.ravel() - d).reshape(-1, 3))
        H[:, k] = -((a1 + b1) - (a2 + b2)).ravel() / (2 * h)
    H = 0.5 * (H + H.T)
    mass = np.repeat(sim.mass(MAT[3]), 3)
    _, fm, fb = sim.energy_forces(MAT, x)
    f = (fm + fb).ravel() + mass * np.tile(g, sim.n)
    A = np.diag(mass) + dt * dt * H
    b = dt * (f - dt * H @ v.ravel())
    free = np.repeat(sim.pinned == 0, 3)
    dv = np.zeros(N)
    dv[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    tx, tv, it, st = sim.forward(MAT, x, v, None, dt=dt, steps=1, tol=1e-13, max_iter=10000, gravity=W.GRAVITY,
                                 eta=0.0, precond=precond)
    assert st == 0
    np.testing.assert_allclose(tv[1].ravel() - v.ravel(), dv, rtol=0, atol=1e-7 * np.abs(dv).max())
    np.testing.assert_allclose(tx[1], x + dt * tv[1], rtol=0, atol=1e-15)


def test_system_matvec_matches_dense_system(oracle_mod):
    """The sparse one-step operator used for large-mesh checks equals the dense system."""
    rng = np.random.default_rng(14)
    sim, rest = _small_sheet(oracle_mod, 5, "top2")
    x = rest + 0.02 * rng.normal(size=rest.shape)
    v = 0.1 * rng.normal(size=rest.shape)
    F = 1e-3 * rng.normal(size=rest.shape)
    p = rng.normal(size=rest.shape)
    A, b = sim.system_dense(MAT, 1 / 30, W.GRAVITY, x, v, F)
    y, b2 = sim.system_matvec(MAT, 1 / 30, W.GRAVITY, x, v, F, p)
    np.testing.assert_allclose(y.ravel(), A @ p.ravel(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b2.ravel(), b, rtol=1e-12, atol=1e-16)


def test_free_fall_closed_form(oracle_mod):
    """Unpinned sheet at rest, gravity only: K annihilates uniform motion, so
    dv = h g exactly, v_t = t h g and x_t = x_0 + h^2 g t (t+1)/2."""
    sim, rest = _small_sheet(oracle_mod, 6, "none")
    dt, T = 1.0 / 30.0, 12
    tx, tv, it, st = sim.forward(MAT, rest, np.zeros_like(rest), None, dt=dt, steps=T, tol=1e-12,
                                 max_iter=1000, gravity=W.GRAVITY)
    assert st == 0
    g = np.array(W.GRAVITY)
    for t in range(T + 1):
        np.testing.assert_allclose(tv[t], np.broadcast_to(t * dt * g, rest.shape), atol=1e-9)
        np.testing.assert_allclose(tx[t], rest + dt * dt * g * t * (t + 1) / 2, atol=1e-9)


def test_velocity_increments_free_fall_closed_form(oracle_mod):
    """Corrective forces as velocity increments: an unpinned sheet at rest receiving the
    same increment c at every vertex and step moves rigidly (K annihilates uniform
    motion), so v_{t+1} = v_t + c + h g, i.e. v_t = t (c + h g) and
    x_t = x_0 + h (c + h g) t (t+1)/2; as a force (mode 0) the same c gives h c / m per step."""
    sim, rest = _small_sheet(oracle_mod, 6, "none")
    dt, T = 1.0 / 30.0, 10
    c = np.array([0.02, -0.01, 0.03])
    F = np.broadcast_to(c, (T, sim.n, 3)).copy()
    tx, tv, _, st = sim.forward(MAT, rest, np.zeros_like(rest), F, dt=dt, steps=T, tol=1e-12, max_iter=1000,
                                gravity=W.GRAVITY, force_mode=1)
    assert st == 0
    w = c + dt * np.array(W.GRAVITY)
    for t in range(T + 1):
        np.testing.assert_allclose(tv[t], np.broadcast_to(t * w, rest.shape), atol=1e-9)
        np.testing.assert_allclose(tx[t], rest + dt * w * t * (t + 1) / 2, atol=1e-9)
    tx0, _, _, _ = sim.forward(MAT, rest, np.zeros_like(rest), F, dt=dt, steps=T, tol=1e-12, max_iter=1000,
                               gravity=W.GRAVITY, force_mode=0)
    assert np.abs(tx0[-1] - tx[-1]).max() > 1e-3  # the two readings differ


def test_velocity_increments_ignore_pinned_vertices(oracle_mod):
    """Increments on pinned vertices change nothing (pins are kinematic), in both the
    trajectory and the gradients; their force gradients are zero."""
    rng = np.random.default_rng(5)
    sim, rest = _small_sheet(oracle_mod, 5, "top2")
    pin = W.pins(5, "top2").astype(bool)
    dt, T = 1.0 / 30.0, 5
    F = 1e-2 * rng.normal(size=(T, sim.n, 3))
    Fm = F.copy()
    Fm[:, pin] = 0.0
    kw = dict(dt=dt, steps=T, tol=1e-13, max_iter=5000, gravity=W.GRAVITY)
    tx, tv, _, _ = sim.forward(MAT, rest, np.zeros_like(rest), F, force_mode=1, **kw)
    txm, tvm, _, _ = sim.forward(MAT, rest, np.zeros_like(rest), Fm, force_mode=1, **kw)
    np.testing.assert_array_equal(tx, txm)
    np.testing.assert_array_equal(tv, tvm)
    dL = rng.normal(size=tx.shape)
    g = sim.backward(MAT, tx, tv, dL, forces=F, force_mode=1, **kw)
    gm = sim.backward(MAT, txm, tvm, dL, forces=Fm, force_mode=1, **kw)
    np.testing.assert_array_equal(g["material"], gm["material"])
    assert np.all(g["forces"][:, pin] == 0.0)


def test_implicit_euler_dissipates_energy_linear_regime(oracle_mod):
    """Backward Euler on a linear elastic system with SPD stiffness dissipates the
    energy 1/2 v^T M v + 1/2 u^T H u at every step.  A tiny in-plane perturbation of
    a sheet pinned along its top edge, without gravity, is in that regime; a step with
    a wrong sign or a dropped h^2 K v term gains energy."""
    rng = np.random.default_rng(13)
    sim, rest = _small_sheet(oracle_mod, 6, "top")
    u0 = 1e-6 * rng.normal(size=rest.shape)
    u0[:, 2] = 0.0
    u0[sim.pinned.astype(bool)] = 0.0
    v0 = np.zeros_like(rest)
    dt, T = 1.0 / 30.0, 15
    tx, tv, it, st = sim.forward(MAT, rest + u0, v0, None, dt=dt, steps=T, tol=1e-13, max_iter=5000,
                                 gravity=(0.0, 0.0, 0.0))
    assert st == 0
    m = sim.mass(MAT[3])
    tot = [sim.energy_forces(MAT, tx[t])[0] + 0.5 * (m[:, None] * tv[t] ** 2).sum() for t in range(T + 1)]
    assert all(b < a for a, b in zip(tot, tot[1:]))
    assert tot[-1] < 0.9 * tot[0]


# ------------------------------------------------------------------ losses
def test_loss_l2_and_pinhole(oracle_mod):
    rng = np.random.default_rng(11)
    traj = rng.normal(size=(4, 5, 3))
    tgt = rng.normal(size=(4, 5, 3))
    L, g = oracle_mod.loss_l2(traj, tgt)
    assert L == pytest.approx(((traj[1:] - tgt[1:]) ** 2).sum())
    assert np.abs(g[0]).max() == 0
    cam = (500.0, 0.5, 0.5, 2.0)
    # a point on the optical axis projects to the principal point; one metre off-axis
    # at 2 m depth lands f/2 = 250 px away (closed form of the pinhole model)
    pts = np.zeros((2, 2, 3))
    pts[1, 0] = (0.5, 0.5, 0.0)
    pts[1, 1] = (1.5, 0.5, 0.0)
    uv = np.zeros((2, 2, 2))
    L, _ = oracle_mod.loss_pinhole(pts, uv, cam)
    assert L == pytest.approx(250.0 ** 2)
    # gradient by central differences
    traj = rng.normal(scale=0.3, size=(3, 4, 3)) + np.array([0.5, 0.5, -0.2])
    uvt = rng.normal(scale=50, size=(3, 4, 2))
    L, g = oracle_mod.loss_pinhole(traj, uvt, cam)
    h = 1e-6
    for idx in [(1, 0, 0), (2, 3, 1), (1, 2, 2), (2, 1, 2)]:
        tp = traj.copy(); tp[idx] += h
        tm = traj.copy(); tm[idx] -= h
        fd = (oracle_mod.loss_pinhole(tp, uvt, cam)[0] - oracle_mod.loss_pinhole(tm, uvt, cam)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6)


# ----------------------------------------------------------------- adjoint
def _rollout_loss(sim, mat, x0, v0, F, target, dt, T, tol, force_mode=0):
    tx, tv, _, st = sim.forward(mat, x0, v0, F, dt=dt, steps=T, tol=tol, max_iter=20000, gravity=W.GRAVITY,
                                force_mode=force_mode)
    from oracle import loss_l2
    return loss_l2(tx, target)[0], tx, tv


def _richardson(fun, h):
    d1 = (fun(h) - fun(-h)) / (2 * h)
    d2 = (fun(h / 2) - fun(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("N,T", [(4, 6), (10, 20)])
def test_adjoint_matches_finite_differences(oracle_mod, N, T):
    """Gradients of the trajectory loss w.r.t. Y, kb, rho, a random force direction,
    a random initial-position and initial-velocity direction: adjoint vs Richardson-
    extrapolated central differences of the forward map (tight CG tolerance)."""
    rng = np.random.default_rng(12 + N)
    rest, tris = W.grid_mesh(N)
    pin = W.pins(N, "top2")
    sim = oracle_mod.OracleSim(rest, tris, pin)
    dt, tol = 1.0 / 30.0, 1e-13
    mat = MAT.copy()
    F = 1e-4 * rng.normal(size=(T, sim.n, 3))
    x0 = rest.copy()
    v0 = np.zeros_like(rest)
    tgt_mat = mat * np.array([2.0, 1.0, 0.5, 1.0])
    target, _, _, _ = sim.forward(tgt_mat, x0, v0, F, dt=dt, steps=T, tol=tol, max_iter=20000, gravity=W.GRAVITY)
    L, tx, tv = _rollout_loss(sim, mat, x0, v0, F, target, dt, T, tol)
    _, dL = oracle_mod.loss_l2(tx, target)
    gr = sim.backward(mat, tx, tv, dL, dt=dt, steps=T, tol=tol, max_iter=20000, gravity=W.GRAVITY)
    assert gr["status"] == 0
    assert gr["material"][1] == 0.0

    def check(fd, an, what):
        assert an == pytest.approx(fd, rel=2e-6, abs=1e-9 * max(1.0, abs(L))), what

    for k, name in ((0, "Y"), (2, "kb"), (3, "rho")):
        h = 1e-3 * mat[k]

        def f(e, k=k):
            m2 = mat.copy(); m2[k] += e
            return _rollout_loss(sim, m2, x0, v0, F, target, dt, T, tol)[0]
        check(_richardson(f, h), gr["material"][k], name)

    free = (pin == 0)[:, None].astype(float)
    dF = rng.normal(size=F.shape) * free
    dx = rng.normal(size=rest.shape)
    dv = rng.normal(size=rest.shape) * free
    for d, key, base, scale in ((dF, "forces", F, 1e-4), (dx, "x0", x0, 1e-3), (dv, "v0", v0, 1e-3)):
        def f(e, d=d, key=key):
            args = {"F": F, "x0": x0, "v0": v0}
            name = {"forces": "F", "x0": "x0", "v0": "v0"}[key]
            args[name] = args[name] + e * d
            return _rollout_loss(sim, mat, args["x0"], args["v0"], args["F"], target, dt, T, tol)[0]
        check(_richardson(f, 1e-3 * scale), float((gr[key] * d).sum()), key)


def test_adjoint_velocity_increments_matches_finite_differences(oracle_mod):
    """Corrective forces as velocity increments (v'_t = v_t + F_t before each step): the
    adjoint's gradients w.r.t. Y, kb, rho, the increments, x0 and v0 against Richardson-
    extrapolated central differences of the forward map."""
    rng = np.random.default_rng(31)
    N, T = 4, 6
    rest, tris = W.grid_mesh(N)
    pin = W.pins(N, "top2")
    sim = oracle_mod.OracleSim(rest, tris, pin)
    dt, tol = 1.0 / 30.0, 1e-13
    mat = MAT.copy()
    F = 1e-3 * rng.normal(size=(T, sim.n, 3))
    x0 = rest.copy()
    v0 = np.zeros_like(rest)
    target, _, _, _ = sim.forward(mat * np.array([2.0, 1.0, 0.5, 1.0]), x0, v0, F, dt=dt, steps=T, tol=tol,
                                  max_iter=20000, gravity=W.GRAVITY, force_mode=1)
    L, tx, tv = _rollout_loss(sim, mat, x0, v0, F, target, dt, T, tol, force_mode=1)
    _, dL = oracle_mod.loss_l2(tx, target)
    gr = sim.backward(mat, tx, tv, dL, dt=dt, steps=T, tol=tol, max_iter=20000, gravity=W.GRAVITY, forces=F,
                      force_mode=1)
    assert gr["status"] == 0

    def check(fd, an, what):
        assert an == pytest.approx(fd, rel=2e-6, abs=1e-9 * max(1.0, abs(L))), what

    for k, name in ((0, "Y"), (2, "kb"), (3, "rho")):
        def f(e, k=k):
            m2 = mat.copy(); m2[k] += e
            return _rollout_loss(sim, m2, x0, v0, F, target, dt, T, tol, force_mode=1)[0]
        check(_richardson(f, 1e-3 * mat[k]), gr["material"][k], name)
    free = (pin == 0)[:, None].astype(float)
    for d, key, scale in ((rng.normal(size=F.shape) * free, "forces", 1e-3), (rng.normal(size=rest.shape), "x0", 1e-3),
                          (rng.normal(size=rest.shape) * free, "v0", 1e-3)):
        def f(e, d=d, key=key):
            a = {"forces": F, "x0": x0, "v0": v0}
            a[key] = a[key] + e * d
            return _rollout_loss(sim, mat, a["x0"], a["v0"], a["forces"], target, dt, T, tol, force_mode=1)[0]
        check(_richardson(f, 1e-3 * scale), float((gr[key] * d).sum()), key)


# ----------------------------------------------------------------- air drag (wind)
def test_drag_terminal_velocity(oracle_mod):
    """An unpinned sheet falling through still air reaches the terminal velocity where
    drag balances gravity: m g + rho_air A |d|_e d = 0 with d = -v and m = rho A, i.e.
    |v|_e v = (rho / rho_air) g.  Implicit Euler's fixed point (dv = 0) is exactly that
    balance, whatever the step."""
    sim, rest = _small_sheet(oracle_mod, 5, "none")
    dt, T = 1.0 / 30.0, 200
    rho_air = 1.0
    tx, tv, _, st = sim.forward(MAT, rest, np.zeros_like(rest), None, dt=dt, steps=T, tol=1e-13, max_iter=2000,
                                gravity=W.GRAVITY, air_density=rho_air, wind=np.zeros(3))
    assert st == 0
    a = MAT[3] / rho_air * 9.8
    eps = 1e-3
    # s sqrt(s^2 + eps^2) = a  =>  s^2 = (-eps^2 + sqrt(eps^4 + 4 a^2)) / 2
    s = np.sqrt((-eps ** 2 + np.sqrt(eps ** 4 + 4 * a * a)) / 2)
    np.testing.assert_allclose(tv[-1], np.broadcast_to([0.0, 0.0, -s], rest.shape), atol=1e-10)


def test_drag_galilean_invariance(oracle_mod):
    """Wind w on a sheet starting at v0 = 0 is the same motion as still air with the sheet
    starting at -w, seen from a frame moving with the wind: x^w_t = x^0_t + t h w and
    v^w_t = v^0_t + w (internal forces see only relative positions, H annihilates uniform
    velocities, drag sees only v - w)."""
    rng = np.random.default_rng(9)
    sim, rest = _small_sheet(oracle_mod, 5, "none")
    x0 = rest + 0.01 * rng.normal(size=rest.shape)
    dt, T = 1.0 / 30.0, 12
    w = np.array([0.7, -0.3, 0.2])
    kw = dict(dt=dt, steps=T, tol=1e-13, max_iter=5000, gravity=W.GRAVITY, air_density=1.0)
    txw, tvw, _, _ = sim.forward(MAT, x0, np.zeros_like(rest), None, wind=w, **kw)
    tx0, tv0, _, _ = sim.forward(MAT, x0, np.broadcast_to(-w, rest.shape), None, wind=np.zeros(3), **kw)
    for t in range(T + 1):
        np.testing.assert_allclose(txw[t], tx0[t] + t * dt * w, atol=1e-10)
        np.testing.assert_allclose(tvw[t], tv0[t] + w, atol=1e-10)


def test_drag_zero_density_is_no_drag(oracle_mod):
    rng = np.random.default_rng(2)
    sim, rest = _small_sheet(oracle_mod, 4, "top2")
    kw = dict(dt=1 / 30, steps=5, tol=1e-13, max_iter=5000, gravity=W.GRAVITY)
    a = sim.forward(MAT, rest, np.zeros_like(rest), None, **kw)
    b = sim.forward(MAT, rest, np.zeros_like(rest), None, air_density=0.0, wind=rng.normal(size=3), **kw)
    np.testing.assert_array_equal(a[0], b[0])


@pytest.mark.parametrize("force_mode", [0, 1])
def test_adjoint_with_drag_matches_finite_differences(oracle_mod, force_mode):
    """Air drag on (rho_air = 1, wind 0.5 m/s sideways plus a seeded part): the adjoint's
    gradients w.r.t. the wind components, Y, kb, rho, the forces (or increments), x0 and
    v0 against Richardson-extrapolated central differences of the forward map."""
    rng = np.random.default_rng(40 + force_mode)
    N, T = 4, 6
    rest, tris = W.grid_mesh(N)
    pin = W.pins(N, "top2")
    sim = oracle_mod.OracleSim(rest, tris, pin)
    dt, tol = 1.0 / 30.0, 1e-13
    mat = MAT.copy()
    F = (1e-4 if force_mode == 0 else 1e-3) * rng.normal(size=(T, sim.n, 3))
    w = np.array([0.5, 0.0, 0.1]) + 0.1 * rng.normal(size=3)
    x0, v0 = rest.copy(), np.zeros_like(rest)
    kw = dict(dt=dt, steps=T, tol=tol, max_iter=20000, gravity=W.GRAVITY, force_mode=force_mode, air_density=1.0)
    target = sim.forward(mat * np.array([2.0, 1.0, 0.5, 1.0]), x0, v0, F, wind=w * 0.5, **kw)[0]

    def loss(m=mat, x=x0, v=v0, f=F, wi=w):
        tx = sim.forward(m, x, v, f, wind=wi, **kw)[0]
        return oracle_mod.loss_l2(tx, target)[0]

    tx, tv, _, _ = sim.forward(mat, x0, v0, F, wind=w, **kw)
    L, dL = oracle_mod.loss_l2(tx, target)
    gr = sim.backward(mat, tx, tv, dL, forces=F, wind=w, **kw)
    assert gr["status"] == 0

    def check(fd, an, what):
        assert an == pytest.approx(fd, rel=2e-6, abs=1e-9 * max(1.0, abs(L))), what

    for k in range(3):
        e = np.zeros(3); e[k] = 1.0
        check(_richardson(lambda h: loss(wi=w + h * e), 1e-3), gr["wind"][k], f"wind{k}")
    for k, name in ((0, "Y"), (2, "kb"), (3, "rho")):
        def f(h, k=k):
            m2 = mat.copy(); m2[k] += h
            return loss(m=m2)
        check(_richardson(f, 1e-3 * mat[k]), gr["material"][k], name)
    free = (pin == 0)[:, None].astype(float)
    dF = rng.normal(size=F.shape) * free
    dx = rng.normal(size=rest.shape)
    dv = rng.normal(size=rest.shape) * free
    check(_richardson(lambda h: loss(f=F + h * dF), 1e-3 * np.abs(F).max()), float((gr["forces"] * dF).sum()), "forces")
    check(_richardson(lambda h: loss(x=x0 + h * dx), 1e-6), float((gr["x0"] * dx).sum()), "x0")
    check(_richardson(lambda h: loss(v=v0 + h * dv), 1e-6), float((gr["v0"] * dv).sum()), "v0")
