// Image energies of a sheet (Sec. 3.2): soft rasterisation, photometric and silhouette
// energies and their gradient with respect to the vertex positions (cloth_image_energy in
// include/cloth_sim.h).  The per-pixel arithmetic is in render.cuh; these kernels map one
// thread to one pixel (or one vertex) and move the data.
#include <cuda_runtime.h>

#include <string>

#include "engine.h"
#include "render.cuh"

namespace cloth {
namespace {

using namespace render;

constexpr int kPix = 256;

__global__ void k_project(int n, Camera cam, const double* __restrict__ x, P2* __restrict__ q,
                          double* __restrict__ inv, double* __restrict__ J) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  project(cam, x + 3 * (size_t)v, &q[v], &inv[v], J + 9 * (size_t)v);
}

// colour, silhouette and the per-pixel photometric energy |I - I_hat|_1
__global__ void k_render(Scene s, int W, int H, const double* __restrict__ image, double* __restrict__ I,
                         double* __restrict__ A, double* __restrict__ ep) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= W * H) return;
  const P2 p = {(pix % W) + 0.5, (pix / W) + 0.5};
  double c[3], a;
  pixel_forward(s, p, c, &a);
  double e = 0.0;
  for (int k = 0; k < 3; ++k) {
    I[3 * (size_t)pix + k] = c[k];
    e += fabs(c[k] - image[3 * (size_t)pix + k]);
  }
  A[pix] = a;
  ep[pix] = e;
}

// one pass of the separable Gaussian filter (dir 0: along rows, 1: along columns)
__global__ void k_blur(int W, int H, int dir, double norm, const double* __restrict__ src, double* __restrict__ dst) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= W * H) return;
  const int u = pix % W, v = pix / W, r = blur_radius();
  double acc = 0.0;
  for (int k = -r; k <= r; ++k) {
    const int uu = dir == 0 ? u + k : u, vv = dir == 0 ? v : v + k;
    if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
    acc += blur_tap(k, norm) * src[(size_t)vv * W + uu];
  }
  dst[pix] = acc;
}

// per-pixel silhouette energy |G(A) - G(B)| and its sign
__global__ void k_sil(int n, const double* __restrict__ ga, const double* __restrict__ gb, double* __restrict__ es,
                      double* __restrict__ sg) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= n) return;
  const double d = ga[pix] - gb[pix];
  es[pix] = fabs(d);
  sg[pix] = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
}

// E = sum ep + LAMBDA sum es, in a fixed order (one CTA)
__global__ void k_energy(int n, const double* __restrict__ ep, const double* __restrict__ es, double* __restrict__ E) {
  __shared__ double sh[kPix];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += ep[i] + LAMBDA * es[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *E = sh[0];
}

// dE/d(image point, inverse depth) of every vertex: per pixel, every triangle's share
// (gA: the filtered sign of G(A) - G(B); dE/dA = LAMBDA gA)
__global__ void k_render_backward(Scene s, int W, int H, const double* __restrict__ image,
                                  const double* __restrict__ I, const double* __restrict__ gA,
                                  double* __restrict__ gq) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= W * H) return;
  const P2 p = {(pix % W) + 0.5, (pix / W) + 0.5};
  double gI[3];
  for (int k = 0; k < 3; ++k) {
    const double d = I[3 * (size_t)pix + k] - image[3 * (size_t)pix + k];
    gI[k] = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
  }
  pixel_backward(s, p, gI, LAMBDA * gA[pix], [&](int v, double gx, double gy, double gi) {
    atomicAdd(&gq[3 * (size_t)v], gx);
    atomicAdd(&gq[3 * (size_t)v + 1], gy);
    atomicAdd(&gq[3 * (size_t)v + 2], gi);
  });
}

// chain to the 3-D positions: dE/dx = J^T (dE/dq, dE/dinv)
__global__ void k_chain(int n, const double* __restrict__ J, const double* __restrict__ gq, double* __restrict__ gx) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double* j = J + 9 * (size_t)v;
  const double* g = gq + 3 * (size_t)v;
  for (int c = 0; c < 3; ++c) gx[3 * (size_t)v + c] = j[c] * g[0] + j[3 + c] * g[1] + j[6 + c] * g[2];
}

int fail(const std::string& msg, int code) {
  set_last_error("cloth_image_energy: " + msg);
  return code;
}

}  // namespace
}  // namespace cloth

extern "C" size_t cloth_image_energy_scratch(int32_t n, int32_t m, int32_t W, int32_t H) {
  return sizeof(double) * (12 * (size_t)W * H + 15 * (size_t)n + ((3 * (size_t)m + 1) / 2));
}

extern "C" int cloth_image_energy(int32_t n, int32_t m, const int32_t* tris, const double* x, const double* uv,
                                  int32_t tex_w, int32_t tex_h, const double* tex, const double* camera, int32_t W,
                                  int32_t H, const double* image, const double* mask, void* scratch, double* energy,
                                  double* dE_dx, double* out_image, double* out_silhouette, void* stream) {
  using namespace cloth;
  using namespace cloth::render;
  if (n < 3 || m < 1 || W < 1 || H < 1 || tex_w < 1 || tex_h < 1 || (long long)tex_w * tex_h > MAX_TEX ||
      (long long)W * H > (1LL << 28) || !tris || !x || !uv || !tex || !camera || !image || !mask || !scratch ||
      !energy)
    return fail("need n >= 3, m >= 1, an image and a texture of positive size and non-null arrays",
                CLOTH_ERR_INVALID_ARG);
  for (long long k = 0; k < 3LL * m; ++k)
    if (tris[k] < 0 || tris[k] >= n) return fail("triangle vertex index out of range", CLOTH_ERR_INVALID_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t WH = (size_t)W * H;
  double* base = (double*)scratch;
  double* I = base;            // 3 WH
  double* A = I + 3 * WH;      // WH
  double* ep = A + WH;
  double* ga = ep + WH;
  double* gb = ga + WH;
  double* tmp = gb + WH;
  double* es = tmp + WH;
  double* sg = es + WH;
  double* gA = sg + WH;        // up to 12 WH
  double* q = base + 12 * WH;  // 2 n (P2)
  double* inv = q + 2 * (size_t)n;
  double* J = inv + n;         // 9 n
  double* gq = J + 9 * (size_t)n;  // 3 n
  int* dtris = (int*)(gq + 3 * (size_t)n);  // 3 m
  cudaError_t e = cudaMemcpyAsync(dtris, tris, sizeof(int) * 3 * (size_t)m, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(cudaGetErrorString(e), CLOTH_ERR_CUDA);
  const Camera cam = {camera[0], camera[1], camera[2], camera[3], W, H};
  const int gp = (int)((WH + kPix - 1) / kPix), gv = (n + kPix - 1) / kPix;
  k_project<<<gv, kPix, 0, st>>>(n, cam, x, (P2*)q, inv, J);
  const Scene s = {dtris, m, (const P2*)q, inv, uv, tex, tex_w, tex_h};
  k_render<<<gp, kPix, 0, st>>>(s, W, H, image, I, A, ep);
  if (out_image) cudaMemcpyAsync(out_image, I, sizeof(double) * 3 * WH, cudaMemcpyDeviceToDevice, st);
  if (out_silhouette) cudaMemcpyAsync(out_silhouette, A, sizeof(double) * WH, cudaMemcpyDeviceToDevice, st);
  const double norm = blur_norm();
  k_blur<<<gp, kPix, 0, st>>>(W, H, 0, norm, A, tmp);
  k_blur<<<gp, kPix, 0, st>>>(W, H, 1, norm, tmp, ga);
  k_blur<<<gp, kPix, 0, st>>>(W, H, 0, norm, mask, tmp);
  k_blur<<<gp, kPix, 0, st>>>(W, H, 1, norm, tmp, gb);
  k_sil<<<gp, kPix, 0, st>>>((int)WH, ga, gb, es, sg);
  k_energy<<<1, kPix, 0, st>>>((int)WH, ep, es, energy);
  if (dE_dx) {
    // the filter is symmetric with zero padding, so its adjoint is the same filter
    k_blur<<<gp, kPix, 0, st>>>(W, H, 0, norm, sg, tmp);
    k_blur<<<gp, kPix, 0, st>>>(W, H, 1, norm, tmp, gA);
    cudaMemsetAsync(gq, 0, sizeof(double) * 3 * n, st);
    k_render_backward<<<gp, kPix, 0, st>>>(s, W, H, image, I, gA, gq);
    k_chain<<<gv, kPix, 0, st>>>(n, J, gq, dE_dx);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(cudaGetErrorString(e), CLOTH_ERR_CUDA);
  return CLOTH_OK;
}
