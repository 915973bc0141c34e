// Image energies of a sheet (Sec. 3.2): soft rasterisation, photometric and silhouette
// energies and their gradient with respect to the vertex positions (cloth_image_energy in
// include/cloth_sim.h).  The per-pixel arithmetic is in render.cuh; the rasterising kernels
// take one 16 x 16 screen tile per CTA and run each per-pixel pass over the triangles that
// can reach the tile (exactly the same values as a pass over every triangle, see
// tri_reach); the others map one thread to one pixel (or one vertex) and move the data.
#include <cuda_runtime.h>

#include <algorithm>

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

// ---- screen tiles: 16 x 16 pixels per CTA, each pass over the triangles that reach the tile
constexpr int kTile = 16;

// every triangle's record (corners, inverse depths, texture coordinates) and reach
__global__ void k_tri_setup(Scene s, TriRec* __restrict__ rec, TriReach* __restrict__ reach) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s.m) return;
  const TriRec r = corners(s, j);
  rec[j] = r;
  reach[j] = tri_reach(r);
}

// The tile's triangles among [c0, c0 + kPix), in ascending order, into list / srec (the
// triangles left out contribute exactly nothing to the tile's pixels, see tri_reach).
// Returns their number; every thread of the CTA calls it.
__device__ int tile_list(const Scene& s, const TriRec* __restrict__ rec, const TriReach* __restrict__ reach, int c0,
                         double ax, double ay, double bx, double by, int* list, TriRec* srec, int* wcount) {
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int j = c0 + t;
  const bool in = j < s.m && reaches(reach[j], ax, ay, bx, by);
  const unsigned bal = __ballot_sync(0xffffffffu, in);
  if (lane == 0) wcount[wp] = __popc(bal);
  __syncthreads();
  int off = 0, n = 0;
  for (int w = 0; w < kPix / 32; ++w) {
    off += w < wp ? wcount[w] : 0;
    n += wcount[w];
  }
  if (in) {
    const int pos = off + __popc(bal & ((1u << lane) - 1u));
    list[pos] = j;
    srec[pos] = rec[j];
  }
  __syncthreads();
  return n;
}

// colour, silhouette and the per-pixel photometric energy |I - I_hat|_1 (the passes of
// pixel_forward over the tile's triangles, in the same order)
__global__ void __launch_bounds__(kPix) k_render(Scene s, const TriRec* __restrict__ rec,
                                                 const TriReach* __restrict__ reach, int W, int H,
                                                 const double* __restrict__ image, double* __restrict__ I,
                                                 double* __restrict__ A, double* __restrict__ ep) {
  __shared__ int list[kPix], wcount[kPix / 32];
  __shared__ TriRec srec[kPix];
  const int tx0 = blockIdx.x * kTile, ty0 = blockIdx.y * kTile;
  const int u = tx0 + (threadIdx.x % kTile), v = ty0 + (threadIdx.x / kTile);
  const bool on = u < W && v < H;
  const P2 p = {u + 0.5, v + 0.5};
  const double ax = tx0 + 0.5, ay = ty0 + 0.5, bx = min(tx0 + kTile - 1, W - 1) + 0.5,
               by = min(ty0 + kTile - 1, H - 1) + 0.5;
  double top = EPS / GAMMA;
  for (int c0 = 0; c0 < s.m; c0 += kPix) {
    const int n = tile_list(s, rec, reach, c0, ax, ay, bx, by, list, srec, wcount);
    if (on)
      for (int e = 0; e < n; ++e) pass_top(p, srec[e], s.tex, s.Wt, s.Ht, &top);
    __syncthreads();
  }
  PixAcc a = pix_acc_begin(top);
  for (int c0 = 0; c0 < s.m; c0 += kPix) {
    const int n = tile_list(s, rec, reach, c0, ax, ay, bx, by, list, srec, wcount);
    if (on)
      for (int e = 0; e < n; ++e) pass_acc(p, srec[e], s.tex, s.Wt, s.Ht, top, false, &a);
    __syncthreads();
  }
  if (!on) return;
  const size_t pix = (size_t)v * W + u;
  double e = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double c = a.acc[k] / a.S;
    I[3 * pix + k] = c;
    e += fabs(c - image[3 * pix + k]);
  }
  A[pix] = 1.0 - a.prod;
  ep[pix] = e;
}

// one pass of the separable Gaussian filter (dir 0: along rows, 1: along columns)
// (the 2r + 1 taps are formed once per CTA, by the same function, into shared memory)
__global__ void k_blur(int W, int H, int dir, double norm, const double* __restrict__ src, double* __restrict__ dst) {
  constexpr int kMaxTaps = 2 * 32 + 1;
  static_assert(3.0 * SIGMA_S <= 32.0 && kPix >= kMaxTaps, "radius up to 32 px, one thread per tap");
  __shared__ double tap[kMaxTaps];
  const int r = blur_radius();
  if ((int)threadIdx.x <= 2 * r) tap[threadIdx.x] = blur_tap((int)threadIdx.x - r, norm);
  __syncthreads();
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= W * H) return;
  const int u = pix % W, v = pix / W;
  double acc = 0.0;
  for (int k = -r; k <= r; ++k) {
    const int uu = dir == 0 ? u + k : u, vv = dir == 0 ? v : v + k;
    if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
    acc += tap[k + r] * src[(size_t)vv * W + uu];
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

// Sums of a[i] + lam b[i] (b may be null): CTA c sums its contiguous chunk of [0, n)
// (thread-strided, then a shared-memory tree) into out[c].  E = sum ep + LAMBDA sum es takes
// two launches, one partial per CTA and then one CTA over the partials: a fixed order, so
// the energy is deterministic.
constexpr int kEnergyParts = 1024;
__global__ void k_energy_sum(int n, const double* __restrict__ a, const double* __restrict__ b, double lam,
                             double* __restrict__ out) {
  __shared__ double sh[kPix];
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double acc = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += b ? a[i] + lam * b[i] : a[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// dE/d(image point, inverse depth) of every vertex: the passes of pixel_backward over the
// tile's triangles; each triangle's share is summed over the warp's 32 pixels and added
// once per warp (gA: the filtered sign of G(A) - G(B); dE/dA = LAMBDA gA)
__global__ void __launch_bounds__(kPix) k_render_backward(Scene s, const TriRec* __restrict__ rec,
                                                          const TriReach* __restrict__ reach, int W, int H,
                                                          const double* __restrict__ image,
                                                          const double* __restrict__ I,
                                                          const double* __restrict__ gA_img,
                                                          double* __restrict__ gq) {
  __shared__ int list[kPix], wcount[kPix / 32];
  __shared__ TriRec srec[kPix];
  const int tx0 = blockIdx.x * kTile, ty0 = blockIdx.y * kTile;
  const int u = tx0 + (threadIdx.x % kTile), v = ty0 + (threadIdx.x / kTile);
  const int lane = threadIdx.x & 31;
  const bool on = u < W && v < H;
  const P2 p = {u + 0.5, v + 0.5};
  const double ax = tx0 + 0.5, ay = ty0 + 0.5, bx = min(tx0 + kTile - 1, W - 1) + 0.5,
               by = min(ty0 + kTile - 1, H - 1) + 0.5;
  const size_t pix = on ? (size_t)v * W + u : 0;
  double gI[3] = {0.0, 0.0, 0.0}, gA = 0.0;
  if (on) {
    for (int k = 0; k < 3; ++k) {
      const double d = I[3 * pix + k] - image[3 * pix + k];
      gI[k] = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
    }
    gA = LAMBDA * gA_img[pix];
  }
  double top = EPS / GAMMA;
  for (int c0 = 0; c0 < s.m; c0 += kPix) {
    const int n = tile_list(s, rec, reach, c0, ax, ay, bx, by, list, srec, wcount);
    if (on)
      for (int e = 0; e < n; ++e) pass_top(p, srec[e], s.tex, s.Wt, s.Ht, &top);
    __syncthreads();
  }
  PixAcc a = pix_acc_begin(top);
  for (int c0 = 0; c0 < s.m; c0 += kPix) {
    const int n = tile_list(s, rec, reach, c0, ax, ay, bx, by, list, srec, wcount);
    if (on)
      for (int e = 0; e < n; ++e) pass_acc(p, srec[e], s.tex, s.Wt, s.Ht, top, true, &a);
    __syncthreads();
  }
  const double Ip[3] = {a.acc[0] / a.S, a.acc[1] / a.S, a.acc[2] / a.S};
  for (int c0 = 0; c0 < s.m; c0 += kPix) {
    const int n = tile_list(s, rec, reach, c0, ax, ay, bx, by, list, srec, wcount);
    for (int e = 0; e < n; ++e) {  // every lane takes every entry (warp-uniform loop)
      P2 g2[3];
      double gi[3];
      const bool nz = on && pass_grad(p, srec[e], s.tex, s.Wt, s.Ht, top, a, Ip, gI, gA, g2, gi);
      if (!__any_sync(0xffffffffu, nz)) continue;
      double val[9];
      for (int k = 0; k < 3; ++k) {
        val[3 * k] = nz ? g2[k].x : 0.0;
        val[3 * k + 1] = nz ? g2[k].y : 0.0;
        val[3 * k + 2] = nz ? gi[k] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val[q] += __shfl_down_sync(0xffffffffu, val[q], o);
      if (lane == 0) {
        const int j = list[e];
        for (int k = 0; k < 3; ++k) {
          const int vtx = s.tris[3 * j + k];
          atomicAdd(&gq[3 * (size_t)vtx], val[3 * k]);
          atomicAdd(&gq[3 * (size_t)vtx + 1], val[3 * k + 1]);
          atomicAdd(&gq[3 * (size_t)vtx + 2], val[3 * k + 2]);
        }
      }
    }
    __syncthreads();
  }
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
  // 12 planes of W x H, 15 per vertex (image point, inverse depth, Jacobian, gradient),
  // 21 per triangle (record and reach), then the triangle indices
  return sizeof(double) * (12 * (size_t)W * H + 15 * (size_t)n + 21 * (size_t)m + ((3 * (size_t)m + 1) / 2));
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
  static_assert(sizeof(TriRec) == 15 * sizeof(double) && sizeof(TriReach) <= 6 * sizeof(double), "record sizes");
  TriRec* rec = (TriRec*)(gq + 3 * (size_t)n);              // 15 m
  TriReach* reach = (TriReach*)((double*)rec + 15 * (size_t)m);  // 6 m
  int* dtris = (int*)((double*)reach + 6 * (size_t)m);      // 3 m
  cudaError_t e = cudaMemcpyAsync(dtris, tris, sizeof(int) * 3 * (size_t)m, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(cudaGetErrorString(e), CLOTH_ERR_CUDA);
  const Camera cam = {camera[0], camera[1], camera[2], camera[3], W, H};
  const int gp = (int)((WH + kPix - 1) / kPix), gv = (n + kPix - 1) / kPix;
  k_project<<<gv, kPix, 0, st>>>(n, cam, x, (P2*)q, inv, J);
  const Scene s = {dtris, m, (const P2*)q, inv, uv, tex, tex_w, tex_h};
  k_tri_setup<<<(m + kPix - 1) / kPix, kPix, 0, st>>>(s, rec, reach);
  const dim3 tiles((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  k_render<<<tiles, kPix, 0, st>>>(s, rec, reach, W, H, image, I, A, ep);
  if (out_image) cudaMemcpyAsync(out_image, I, sizeof(double) * 3 * WH, cudaMemcpyDeviceToDevice, st);
  if (out_silhouette) cudaMemcpyAsync(out_silhouette, A, sizeof(double) * WH, cudaMemcpyDeviceToDevice, st);
  const double norm = blur_norm();
  k_blur<<<gp, kPix, 0, st>>>(W, H, 0, norm, A, tmp);
  k_blur<<<gp, kPix, 0, st>>>(W, H, 1, norm, tmp, ga);
  k_blur<<<gp, kPix, 0, st>>>(W, H, 0, norm, mask, tmp);
  k_blur<<<gp, kPix, 0, st>>>(W, H, 1, norm, tmp, gb);
  k_sil<<<gp, kPix, 0, st>>>((int)WH, ga, gb, es, sg);
  // the partials go to tmp, which the filter passes below overwrite only after this
  const int parts = (int)std::min<size_t>(kEnergyParts, (WH + kPix - 1) / kPix);
  k_energy_sum<<<parts, kPix, 0, st>>>((int)WH, ep, es, LAMBDA, tmp);
  k_energy_sum<<<1, kPix, 0, st>>>(parts, tmp, nullptr, 0.0, energy);
  if (dE_dx) {
    // the filter is symmetric with zero padding, so its adjoint is the same filter
    k_blur<<<gp, kPix, 0, st>>>(W, H, 0, norm, sg, tmp);
    k_blur<<<gp, kPix, 0, st>>>(W, H, 1, norm, tmp, gA);
    cudaMemsetAsync(gq, 0, sizeof(double) * 3 * n, st);
    k_render_backward<<<tiles, kPix, 0, st>>>(s, rec, reach, W, H, image, I, gA, gq);
    k_chain<<<gv, kPix, 0, st>>>(n, J, gq, dE_dx);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(cudaGetErrorString(e), CLOTH_ERR_CUDA);
  return CLOTH_OK;
}
