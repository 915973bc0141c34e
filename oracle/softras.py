"""FP64 CPU oracle of the image energies of phi-SfT (Sec. 3.2): a soft rasteriser of the
textured sheet and the photometric and silhouette energies E_p, E_s.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): a plain, slow restatement in
PyTorch CPU float64 tensors, shares no code with the CUDA library.  The energies are
written out directly; their gradients with respect to the vertex positions are the exact
derivatives of these definitions (torch.autograd on the CPU).

Definitions (the paper names the Soft Rasterizer of Liu et al. for R and fixes
sigma = 7 px and lambda = 0.5; the rasteriser's own constants are readings):

* camera: the pinhole of the tracking loss, pi(x) = f ((x - cx)/(cz - z), -(y - cy)/(cz - z)),
  image of W x H pixels, pixel centres at (u + 1/2, v + 1/2), image point p = (W/2, H/2) + pi(x);
* triangle j, projected corners a, b, c: signed squared distance of a pixel centre p to
  the triangle, +d^2 inside and -d^2 outside (d = distance to the nearest edge segment),
  and its coverage probability D_j(p) = sigmoid(+-d^2 / SIGMA_R);
* silhouette A(p) = 1 - prod_j (1 - D_j(p));
* colour: each triangle's texture colour at p (bilinear texel sampling of the uv
  coordinates interpolated with the barycentric coordinates of p, clamped to the
  triangle), blended with weights w_j = D_j exp(zn_j / GAMMA) against a black background
  of weight exp(EPS / GAMMA), where zn_j is the normalised inverse depth at p
  (1 nearest at Z_NEAR, 0 at Z_FAR), interpolated with the same barycentric coordinates;
  the weights are evaluated as exp(zn_j / GAMMA + log D_j - top) with top the largest of
  these exponents and EPS / GAMMA (a stable softmax that keeps the background's weight at
  pixels where every D_j underflows);
* E_p = sum_p sum_rgb |I(p) - I_hat(p)|;  E_s = sum_p |G(A)(p) - G(B_hat)(p)| with G the
  Gaussian filter of standard deviation SIGMA_S px (truncated at 3 sigma, zero outside the
  image); the energy of a frame is E_p + LAMBDA E_s.
"""
from __future__ import annotations

import math

import numpy as np
import torch

SIGMA_R = 1.0      # px^2, sharpness of the coverage probabilities
GAMMA = 1e-4       # depth-softmax temperature
EPS = 1e-3         # background's normalised inverse depth
Z_NEAR, Z_FAR = 0.5, 5.0
SIGMA_S = 7.0      # px, silhouette blur (the paper's sigma)
LAMBDA = 0.5       # weight of E_s (the paper's lambda)


def _t(a):
    return a if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a, np.float64))


def project(x, camera, W, H):
    """Image points [n, 2] (pixels) and camera depths [n] of vertices x [n, 3]."""
    f, cx, cy, cz = camera
    depth = cz - x[:, 2]
    px = W / 2 + f * (x[:, 0] - cx) / depth
    py = H / 2 - f * (x[:, 1] - cy) / depth
    return torch.stack([px, py], dim=1), depth


def pixel_centres(W, H):
    v, u = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64), indexing="ij")
    return torch.stack([u + 0.5, v + 0.5], dim=-1)  # [H, W, 2]


def _segment_distance2(p, a, b):
    """Squared distance of points p [..., 2] to the segment a-b ([2] each)."""
    ab = b - a
    t = ((p - a) * ab).sum(-1) / (ab * ab).sum()
    t = t.clamp(0.0, 1.0)
    q = a + t[..., None] * ab
    return ((p - q) ** 2).sum(-1)


def _barycentric(p, a, b, c):
    """Barycentric coordinates [..., 3] of points p [..., 2] in the triangle a, b, c."""
    v0, v1, v2 = b - a, c - a, p - a
    d00, d01, d11 = (v0 * v0).sum(), (v0 * v1).sum(), (v1 * v1).sum()
    d20, d21 = (v2 * v0).sum(-1), (v2 * v1).sum(-1)
    den = d00 * d11 - d01 * d01
    l1 = (d11 * d20 - d01 * d21) / den
    l2 = (d00 * d21 - d01 * d20) / den
    return torch.stack([1 - l1 - l2, l1, l2], dim=-1)


def coverage(q, tris, W, H):
    """Signed sigmoid arguments s = +-d^2 / SIGMA_R [m, H, W] (coverage D = sigmoid(s)) and
    barycentric coordinates [m, H, W, 3] of every pixel centre in every projected triangle
    (q: image points [n, 2])."""
    P = pixel_centres(W, H)
    S, L = [], []
    for (i, j, k) in tris:
        a, b, c = q[i], q[j], q[k]
        lam = _barycentric(P, a, b, c)
        inside = (lam >= 0).all(-1)
        d2 = torch.minimum(torch.minimum(_segment_distance2(P, a, b), _segment_distance2(P, b, c)),
                           _segment_distance2(P, c, a))
        S.append(torch.where(inside, d2, -d2) / SIGMA_R)
        L.append(lam)
    return torch.stack(S), torch.stack(L)


def silhouette(D):
    return 1.0 - torch.prod(1.0 - D, dim=0)


def sample_texture(tex, uv):
    """Bilinear sample of texture tex [Ht, Wt, 3] at uv [..., 2] in [0, 1]^2 (u along the
    width, v along the height, texel centres at (k + 1/2) / size, clamped at the border)."""
    Ht, Wt = tex.shape[0], tex.shape[1]
    x = (uv[..., 0] * Wt - 0.5).clamp(0.0, Wt - 1.0)
    y = (uv[..., 1] * Ht - 0.5).clamp(0.0, Ht - 1.0)
    x0 = x.floor().clamp(max=Wt - 2 if Wt > 1 else 0).long()
    y0 = y.floor().clamp(max=Ht - 2 if Ht > 1 else 0).long()
    x1 = (x0 + 1).clamp(max=Wt - 1)
    y1 = (y0 + 1).clamp(max=Ht - 1)
    fx = (x - x0.double())[..., None]
    fy = (y - y0.double())[..., None]
    return ((1 - fx) * (1 - fy) * tex[y0, x0] + fx * (1 - fy) * tex[y0, x1] + (1 - fx) * fy * tex[y1, x0]
            + fx * fy * tex[y1, x1])


def render(x, tris, uv, tex, camera, W, H):
    """Soft-rasterised colour image [H, W, 3] and silhouette [H, W] of the sheet x [n, 3]
    with per-vertex texture coordinates uv [n, 2] and texture tex [Ht, Wt, 3]."""
    x, uv, tex = _t(x), _t(uv), _t(tex)
    q, depth = project(x, camera, W, H)
    Sarg, L = coverage(q, tris, W, H)
    D = torch.sigmoid(Sarg)
    Lc = L.clamp(min=0.0)
    Lc = Lc / Lc.sum(-1, keepdim=True)
    tri = torch.as_tensor(np.asarray(tris, np.int64))
    inv = 1.0 / depth
    zn = ((Lc * inv[tri][:, None, None, :]).sum(-1) - 1.0 / Z_FAR) / (1.0 / Z_NEAR - 1.0 / Z_FAR)
    uvp = (Lc[..., None] * uv[tri][:, None, None, :, :]).sum(-2)  # [m, H, W, 2]
    C = sample_texture(tex, uvp)                                  # [m, H, W, 3]
    # w_j = D_j exp(zn_j / GAMMA) and the background's exp(EPS / GAMMA), every exponent taken
    # relative to the largest one present (log D_j = log sigmoid(s_j)): where every D_j has
    # underflowed the background term stays 1 instead of 0 / 0
    logw = zn / GAMMA + torch.nn.functional.logsigmoid(Sarg)
    top = torch.maximum(logw.max(dim=0).values, torch.full_like(zn[0], EPS / GAMMA))
    w = torch.exp(logw - top)
    wb = torch.exp(EPS / GAMMA - top)
    img = (w[..., None] * C).sum(0) / (w.sum(0) + wb)[..., None]  # black background
    return img, silhouette(D)


def gaussian_filter(img, sigma=SIGMA_S):
    """Separable Gaussian filter of an [H, W] image, truncated at 3 sigma, zero padding."""
    r = int(math.ceil(3 * sigma))
    k = torch.exp(-0.5 * (torch.arange(-r, r + 1, dtype=torch.float64) / sigma) ** 2)
    k = k / k.sum()
    H, W = img.shape
    pad = torch.nn.functional.pad(img[None, None], (r, r, r, r))
    out = torch.nn.functional.conv2d(pad, k.view(1, 1, 1, -1))
    out = torch.nn.functional.conv2d(out, k.view(1, 1, -1, 1))
    return out[0, 0]


def frame_energy(x, tris, uv, tex, camera, image, mask):
    """E_p + LAMBDA E_s of one frame against the input image [H, W, 3] and binary mask [H, W]."""
    image, mask = _t(image), _t(mask)
    H, W = mask.shape
    img, A = render(x, tris, uv, tex, camera, W, H)
    Ep = (img - image).abs().sum()
    Es = (gaussian_filter(A) - gaussian_filter(mask)).abs().sum()
    return Ep + LAMBDA * Es


def energy_and_grad(traj, tris, uv, tex, camera, images, masks):
    """E = sum_{t>=1} (E_p + LAMBDA E_s) over a trajectory [T+1, n, 3] and dE/dx_t
    [T+1, n, 3] (row 0 is zero: the first frame is the given template)."""
    traj = _t(traj)
    E = 0.0
    grad = torch.zeros_like(traj)
    for t in range(1, traj.shape[0]):
        xt = traj[t].clone().requires_grad_(True)
        e = frame_energy(xt, tris, uv, tex, camera, images[t], masks[t])
        (g,) = torch.autograd.grad(e, xt)
        E += float(e.detach())
        grad[t] = g
    return E, grad.numpy()
