// Host build of the image-energy pipeline of the CUDA library, for CPU tests: the same
// per-pixel functions (paper_2203_11938_gb300/csrc/render.cuh) driven by plain loops in
// place of the kernels, so the arithmetic can be checked against the oracle without a GPU.
#include <cmath>
#include <vector>

#include "../paper_2203_11938_gb300/csrc/render.cuh"

using namespace cloth::render;

static void blur(int W, int H, int dir, double norm, const double* src, double* dst) {
  const int r = blur_radius();
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      double acc = 0.0;
      for (int k = -r; k <= r; ++k) {
        const int uu = dir == 0 ? u + k : u, vv = dir == 0 ? v : v + k;
        if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
        acc += blur_tap(k, norm) * src[(size_t)vv * W + uu];
      }
      dst[(size_t)v * W + u] = acc;
    }
}

extern "C" double host_image_energy(int n, int m, const int* tris, const double* x, const double* uv, int Wt, int Ht,
                                    const double* tex, const double* camera, int W, int H, const double* image,
                                    const double* mask, double* grad, double* out_image, double* out_sil) {
  const Camera cam = {camera[0], camera[1], camera[2], camera[3], W, H};
  std::vector<P2> q(n);
  std::vector<double> inv(n), J(9 * (size_t)n);
  for (int v = 0; v < n; ++v) project(cam, x + 3 * v, &q[v], &inv[v], &J[9 * v]);
  const Scene s = {tris, m, q.data(), inv.data(), uv, tex, Wt, Ht};
  const size_t WH = (size_t)W * H;
  std::vector<double> I(3 * WH), A(WH), tmp(WH), ga(WH), gb(WH), sg(WH), gA(WH);
  double E = 0.0;
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      const size_t pix = (size_t)v * W + u;
      pixel_forward(s, P2{u + 0.5, v + 0.5}, &I[3 * pix], &A[pix]);
      for (int k = 0; k < 3; ++k) E += std::fabs(I[3 * pix + k] - image[3 * pix + k]);
    }
  const double norm = blur_norm();
  blur(W, H, 0, norm, A.data(), tmp.data());
  blur(W, H, 1, norm, tmp.data(), ga.data());
  blur(W, H, 0, norm, mask, tmp.data());
  blur(W, H, 1, norm, tmp.data(), gb.data());
  for (size_t p = 0; p < WH; ++p) {
    const double d = ga[p] - gb[p];
    E += LAMBDA * std::fabs(d);
    sg[p] = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
  }
  if (out_image)
    for (size_t k = 0; k < 3 * WH; ++k) out_image[k] = I[k];
  if (out_sil)
    for (size_t k = 0; k < WH; ++k) out_sil[k] = A[k];
  if (grad) {
    blur(W, H, 0, norm, sg.data(), tmp.data());
    blur(W, H, 1, norm, tmp.data(), gA.data());
    std::vector<double> gq(3 * (size_t)n, 0.0);
    for (int v = 0; v < H; ++v)
      for (int u = 0; u < W; ++u) {
        const size_t pix = (size_t)v * W + u;
        double gI[3];
        for (int k = 0; k < 3; ++k) {
          const double d = I[3 * pix + k] - image[3 * pix + k];
          gI[k] = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
        }
        pixel_backward(s, P2{u + 0.5, v + 0.5}, gI, LAMBDA * gA[pix], [&](int vv, double gx, double gy, double gi) {
          gq[3 * vv] += gx;
          gq[3 * vv + 1] += gy;
          gq[3 * vv + 2] += gi;
        });
      }
    for (int v = 0; v < n; ++v)
      for (int c = 0; c < 3; ++c)
        grad[3 * v + c] = J[9 * v + c] * gq[3 * v] + J[9 * v + 3 + c] * gq[3 * v + 1] + J[9 * v + 6 + c] * gq[3 * v + 2];
  }
  return E;
}
