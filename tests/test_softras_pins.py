"""Pins of the image-energy oracle (soft rasteriser, E_p, E_s) against closed forms,
special cases and finite differences (CPU)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from oracle import softras as S  # noqa: E402

sig = lambda z: 1.0 / (1.0 + math.exp(-z))  # noqa: E731


def test_edge_and_corner_probabilities():
    """A pixel centre on an edge has D = 1/2; inside pixels follow sigmoid(+d^2/sigma)
    with d the distance to the nearest edge line, outside pixels below an edge
    sigmoid(-d^2/sigma) (right triangle with legs on pixel-centre lines)."""
    q = torch.tensor([[2.5, 2.5], [14.5, 2.5], [2.5, 14.5]], dtype=torch.float64)
    s_, _ = S.coverage(q, [(0, 1, 2)], 16, 16)
    D = torch.sigmoid(s_)[0].numpy()
    assert D[2, 6] == pytest.approx(0.5, abs=1e-15)  # centre (6.5, 2.5) on the edge y = 2.5
    for (v, u) in [(5, 5), (4, 7), (6, 4), (8, 3)]:
        x, y = u + 0.5, v + 0.5
        d = min(x - 2.5, y - 2.5, (17.0 - x - y) / math.sqrt(2))
        assert D[v, u] == pytest.approx(sig(d * d / S.SIGMA_R), rel=1e-12)
    for u in (4, 8, 11):
        d = 2.5 - 0.5  # pixel row 0 (y = 0.5) lies 2 px below the edge y = 2.5
        assert D[0, u] == pytest.approx(sig(-d * d / S.SIGMA_R), rel=1e-12)


def test_soft_union_on_a_shared_edge():
    """Two triangles of a square share the diagonal: at a pixel centre on it both have
    D = 1/2, so the silhouette is 1 - (1/2)^2 = 3/4; at (10.5, 4.5), 2 px from the square's
    bottom and right edges and 6/sqrt(2) px from the diagonal, it is
    1 - (1 - sigmoid(4)) (1 - sigmoid(-18))."""
    q = torch.tensor([[2.5, 2.5], [12.5, 2.5], [12.5, 12.5], [2.5, 12.5]], dtype=torch.float64)
    s_, _ = S.coverage(q, [(0, 1, 2), (0, 2, 3)], 16, 16)
    A = S.silhouette(torch.sigmoid(s_)).numpy()
    assert A[7, 7] == pytest.approx(0.75, abs=1e-12)  # centre (7.5, 7.5) on the diagonal
    assert A[4, 10] == pytest.approx(1 - (1 - sig(4.0)) * (1 - sig(-18.0)), rel=1e-12)


def _sheet_quad(z, half=0.3, cx=0.5, cy=0.5):
    x = np.array([[cx - half, cy - half, z], [cx + half, cy - half, z], [cx + half, cy + half, z],
                  [cx - half, cy + half, z]])
    uv = np.array([[0.0, 1.0], [1.0, 1.0], [1.0, 0.0], [0.0, 0.0]])
    return x, [(0, 1, 2), (0, 2, 3)], uv


def test_colour_blend_closed_form_constant_texture():
    """One triangle parallel to the image plane with a constant texture c: every pixel
    shows c D / (D + exp((EPS - zn)/GAMMA)) with zn the normalised inverse depth."""
    cam = (40.0, 0.5, 0.5, 2.0)
    x, _, uv = _sheet_quad(0.0)
    tris = [(0, 1, 2)]
    c = np.array([0.2, 0.5, 0.9])
    tex = np.broadcast_to(c, (4, 4, 3)).copy()
    img, A = S.render(x, tris, uv, tex, cam, 32, 32)
    q, depth = S.project(torch.as_tensor(x), cam, 32, 32)
    s_, _ = S.coverage(q, tris, 32, 32)
    D = torch.sigmoid(s_)[0].numpy()
    zn = (1 / 2.0 - 1 / S.Z_FAR) / (1 / S.Z_NEAR - 1 / S.Z_FAR)
    wb = math.exp((S.EPS - zn) / S.GAMMA)
    expect = c[None, None, :] * (D / (D + wb))[..., None]
    np.testing.assert_allclose(img.numpy(), expect, rtol=1e-12, atol=1e-300)


def _logsig(z):
    """log sigmoid(z), written out for the closed forms below."""
    return -math.log1p(math.exp(-z)) if z >= 0 else z - math.log1p(math.exp(z))


def _one_triangle_at_pixels(corners_px, depth, cam, W, H):
    """World corners at `depth` in front of the camera whose images are the given pixel
    coordinates (the inverse of the pinhole with the principal point at the centre)."""
    f, cx, cy, cz = cam
    return np.array([[cx + (u - W / 2) * depth / f, cy - (v - H / 2) * depth / f, cz - depth] for u, v in corners_px])


def test_colour_blend_away_from_the_sheet_closed_form():
    """Outside a triangle the colour is c D e^{zn/GAMMA} / (D e^{zn/GAMMA} + e^{EPS/GAMMA})
    = c sigmoid(zn/GAMMA + log D - EPS/GAMMA), D = sigmoid(-d^2/SIGMA_R): at depth 4 m
    (zn = 1/36) a pixel centre 16.5 px above the triangle's top edge shows about 1 % of
    the texture colour, a value that dropping the coverage term, the depth term or the
    background would each change."""
    W = H = 128
    cam = (100.0, 0.5, 0.5, 4.0)
    x = _one_triangle_at_pixels([(40.0, 64.0), (90.0, 64.0), (64.0, 110.0)], 4.0, cam, W, H)
    c = np.array([0.2, 0.5, 0.9])
    tex = np.broadcast_to(c, (4, 4, 3)).copy()
    uv = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0]])
    img, _ = S.render(x, [(0, 1, 2)], uv, tex, cam, W, H)
    zn = (1 / 4.0 - 1 / S.Z_FAR) / (1 / S.Z_NEAR - 1 / S.Z_FAR)
    d = 64.0 - 47.5  # pixel (64, 47): centre (64.5, 47.5), nearest point (64.5, 64) on the top edge
    share = 1.0 / (1.0 + math.exp(-(zn / S.GAMMA + _logsig(-d * d / S.SIGMA_R) - S.EPS / S.GAMMA)))
    assert 1e-3 < share < 0.1
    np.testing.assert_allclose(img[47, 64].numpy(), c * share, rtol=1e-9)


def test_background_far_from_every_triangle_is_black_not_nan():
    """Where every coverage underflows (a pixel tens of pixels from the sheet, here at
    2 m, zn = 1/6) the blend is the black background: 0, finite, with a finite gradient."""
    W = H = 96
    cam = (100.0, 0.5, 0.5, 2.0)
    x = torch.tensor(_one_triangle_at_pixels([(60.0, 60.0), (90.0, 60.0), (75.0, 90.0)], 2.0, cam, W, H),
                     requires_grad=True)
    tex = np.full((4, 4, 3), 0.7)
    uv = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0]])
    img, A = S.render(x, [(0, 1, 2)], uv, tex, cam, W, H)
    assert torch.isfinite(img).all() and torch.isfinite(A).all()
    assert float(img[0, 0].abs().max()) == 0.0 and float(A[0, 0]) == 0.0  # ~80 px from the triangle
    assert float(img[75, 75].min()) > 0.69  # inside: the texture colour
    (g,) = torch.autograd.grad(img.sum(), x)
    assert torch.isfinite(g).all()


def test_nearer_triangle_wins():
    """Two overlapping parallel quads at different depths, red near, blue far: each
    pixel blends them with weights D exp(zn/GAMMA) (exactly), so where both cover the
    pixel the near colour dominates."""
    cam = (40.0, 0.5, 0.5, 2.0)
    xn, tris, uv = _sheet_quad(0.2)
    xf, _, _ = _sheet_quad(0.0)
    x = np.concatenate([xn, xf])
    tris2 = tris + [(a + 4, b + 4, c + 4) for (a, b, c) in tris]
    red = np.zeros((2, 2, 3)); red[..., 0] = 1.0
    blue = np.zeros((2, 2, 3)); blue[..., 2] = 1.0
    # one texture: red in the left half (u < 1/2), blue in the right half; near quad uses u
    # in [0, 0.25], far quad u in [0.75, 1]
    tex = np.concatenate([red, blue], axis=1)
    uv2 = np.concatenate([uv * [0.25, 1.0], uv * [0.25, 1.0] + [0.75, 0.0]])
    img, _ = S.render(x, tris2, uv2, tex, cam, 32, 32)
    centre = img.numpy()[16, 16]
    assert centre[0] > 1 - 1e-9 and centre[2] < 1e-9


def test_gaussian_filter_impulse_response():
    """The filter of a unit impulse is the normalised sampled Gaussian (outer product)."""
    img = torch.zeros(61, 61, dtype=torch.float64)
    img[30, 30] = 1.0
    out = S.gaussian_filter(img).numpy()
    r = int(math.ceil(3 * S.SIGMA_S))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / S.SIGMA_S) ** 2)
    k /= k.sum()
    np.testing.assert_allclose(out[30 - r:30 + r + 1, 30 - r:30 + r + 1], np.outer(k, k), rtol=1e-12, atol=1e-18)
    assert out.sum() == pytest.approx(1.0, abs=1e-12)


def test_bilinear_texture_sampling():
    tex = torch.as_tensor(np.arange(2 * 3 * 3, dtype=np.float64).reshape(2, 3, 3))
    # texel centres return the texels; the midpoint of four texels their mean
    assert torch.allclose(S.sample_texture(tex, torch.tensor([[0.5 / 3, 0.5 / 2]], dtype=torch.float64))[0], tex[0, 0])
    assert torch.allclose(S.sample_texture(tex, torch.tensor([[2.5 / 3, 1.5 / 2]], dtype=torch.float64))[0], tex[1, 2])
    mid = S.sample_texture(tex, torch.tensor([[1.0 / 3, 1.0 / 2]], dtype=torch.float64))[0]
    assert torch.allclose(mid, (tex[0, 0] + tex[0, 1] + tex[1, 0] + tex[1, 1]) / 4)


def test_projection_is_the_tracking_losss_pinhole(oracle_mod):
    """Image points minus the principal point are the pinhole tracks of the tracking loss:
    the pinhole loss against them vanishes."""
    rng = np.random.default_rng(3)
    x = np.c_[rng.uniform(0, 1, (7, 2)), rng.uniform(-0.2, 0.2, 7)]
    cam = (500.0, 0.5, 0.5, 2.0)
    q, _ = S.project(torch.as_tensor(x), cam, 64, 48)
    uv = q.numpy() - [32, 24]
    L, _ = oracle_mod.loss_pinhole(np.stack([x, x]), np.stack([uv, uv]), cam)
    assert L == pytest.approx(0.0, abs=1e-20)


def test_energy_zero_at_the_rendered_frame_and_gradient_by_differences():
    """E vanishes when the inputs are the rendering itself (image and soft silhouette); at
    a perturbed sheet its autograd gradient matches central differences."""
    cam = (40.0, 0.5, 0.5, 2.0)
    x, tris, uv = _sheet_quad(0.0)
    rng = np.random.default_rng(4)
    tex = rng.uniform(0, 1, (8, 8, 3))
    img, A = S.render(x, tris, uv, tex, cam, 24, 24)
    assert float(S.frame_energy(x, tris, uv, tex, cam, img, A)) == pytest.approx(0.0, abs=1e-12)
    xp = x + 0.01 * rng.normal(size=x.shape)
    traj = np.stack([x, xp])
    E, g = S.energy_and_grad(traj, tris, uv, tex, cam, [None, img], [None, (A > 0.5).double()])
    assert np.all(g[0] == 0)
    h = 1e-6
    for (i, k) in [(0, 0), (1, 1), (2, 2), (3, 0)]:
        xa, xb = xp.copy(), xp.copy()
        xa[i, k] += h
        xb[i, k] -= h
        fd = (float(S.frame_energy(xa, tris, uv, tex, cam, img, (A > 0.5).double()))
              - float(S.frame_energy(xb, tris, uv, tex, cam, img, (A > 0.5).double()))) / (2 * h)
        assert g[1, i, k] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_image_energy_gradient_through_the_simulator(oracle_mod):
    """dE/dx_t of the image energy, fed to the simulator's adjoint, gives dE/dY, dE/dk_b,
    dE/drho of E(render(simulate(material))): against Richardson differences of the
    whole pipeline (4x4 sheet, 4 steps, 20 x 20 images of a target trajectory)."""
    from paper_2203_11938_gb300 import workloads as W

    N, T, dt = 4, 4, 1.0 / 30.0
    rest, tris = W.grid_mesh(N)
    pin = W.pins(N, "top2")
    sim = oracle_mod.OracleSim(rest, tris, pin)
    tri = [tuple(int(i) for i in t) for t in tris]
    uvv = np.c_[rest[:, 0], 1.0 - rest[:, 1]]
    rng = np.random.default_rng(8)
    tex = rng.uniform(0, 1, (6, 6, 3))
    cam = (30.0, 0.5, 0.5, 2.0)
    mat = np.array([1.0e3, 0.3, 1.0e-4, 0.1])
    kw = dict(dt=dt, steps=T, tol=1e-13, max_iter=5000, gravity=W.GRAVITY)
    tgt = sim.forward(mat * np.array([0.5, 1.0, 2.0, 1.0]), rest, np.zeros_like(rest), None, **kw)[0]
    images, masks = [None], [None]
    for t in range(1, T + 1):
        img, A = S.render(tgt[t], tri, uvv, tex, cam, 20, 20)
        images.append(img)
        masks.append((A > 0.5).double())

    def energy(m):
        tx = sim.forward(m, rest, np.zeros_like(rest), None, **kw)[0]
        return S.energy_and_grad(tx, tri, uvv, tex, cam, images, masks)[0]

    tx, tv, _, _ = sim.forward(mat, rest, np.zeros_like(rest), None, **kw)
    E, dE = S.energy_and_grad(tx, tri, uvv, tex, cam, images, masks)
    g = sim.backward(mat, tx, tv, dE, **kw)["material"]
    for k in (0, 2, 3):
        def f(h, k=k):
            m2 = mat.copy(); m2[k] += h
            return energy(m2)
        h = 1e-3 * mat[k]
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        assert g[k] == pytest.approx((4 * d2 - d1) / 3, rel=1e-4), k
