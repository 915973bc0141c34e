// Cloth step + adjoint engine: CUDA kernels and host driver, templated on the real type.
//
// One time step (phi-SfT Sec. 3.1, Eq. 3-5, df/dv = 0):
//   element kernels   f_e, H~_e per triangle (membrane) and per interior edge (bending)
//   assembly          A = M + h^2 H~ (3x3-block SELL-32, pinned rows/cols -> identity),
//                     b = h (f + M g + F_t) - h^2 H~ v, D^{-1} = 1/diag(A); each block sums a
//                     fixed list of element blocks (no atomics, fixed order)
//   Jacobi PCG        per-sheet FP64 dot products by deterministic segmented reduction
//   update            v' = v + dv, x' = x + h v'
// Adjoint of step t (implicit differentiation of the solve):
//   A lam = mask(v_bar + h x_bar);  x_bar += -h H lam - h^2 d(lam^T H~ u)/dx + dL/dx_t,
//   v_bar += h x_bar - h^2 H~ lam,  F_bar_t = h lam,  with u = v_{t+1};
//   Y_bar += lam^T (h f_mem - h^2 H~_mem u) / Y, kb_bar likewise, rho_bar += lam^T M_1 (h g - dv).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "elements.cuh"
#include "engine.h"
#include "ffloat.cuh"

namespace cloth {

constexpr int kThreads = kRowsPerBlock;  // row kernels: one CTA per work entry
constexpr int kElemThreads = 128;

// Per-sheet CG scalars.  FP64 mode computes in the doubles; FP32 mode computes r.z,
// alpha and the stopping threshold as float-float and keeps beta as the float the
// direction update takes (the doubles then hold the values at the start of the solve).
struct CGSheet {
  double rz, rr, bb, pAp, alpha, beta;
  double stop_rr;         // (tol |b|)^2: the solve ends when r.r <= stop_rr
  FF rz_f, stop_f, alpha_f;
  float beta_f;
  int iters, done, status;
  int zero_rhs;  // b = 0: the solution is 0 (matters when the solve starts from a guess)
};

// CG dot-product accumulator of one thread: FP64 in FP64 mode; in FP32 mode a
// float-float, so the sums run on the FP32 pipe at near-FP64 accuracy.
template <class R> struct CGAcc { using T = double; };
template <> struct CGAcc<float> { using T = FF; };
template <class R> using acc_t = typename CGAcc<R>::T;

// kPhaseTimed: the solves cloth_time_kernel times (their counts kept apart)
enum Phase { kPhaseForward = 0, kPhaseBackward = 1, kPhaseRecompute = 2, kPhaseTimed = 3 };

template <class R>
struct Dev {
  int S, Np, Nu, M, E, nslices, NW;
  const int *tri_v, *tri_sheet;
  const R* tri_rest;
  const double* tri_rest_d;  // [5][M] the same rest data in FP64 (force path)
  const double* tri_metric;  // [3][M] rest edge metric
  const int *hin_v, *hin_sheet;
  const R* hin_rest;
  const double* hin_rest_d;  // [2][E] FP64 copy (force path)
  const int *i2u, *u2i;
  const uint8_t* pinned;
  const R* area3;
  const int *vsheet, *usheet;
  const int *slice_base, *slice_K, *cols, *contrib_ptr, *contrib;
  const int *vf_ptr, *vf;
  const int *work_sheet, *work_row0, *work_rows, *sheet_wfirst;
  const int *sheet_uoff, *sheet_voff, *sheet_toff, *sheet_hoff;
  // scratch
  double *tri_f, *hin_f;  // element force vectors f_e - h H~_e v_e, FP64
  R *tri_H, *hin_H, *tri_r, *hin_r;
  double *tri_sc, *hin_sc, *row_sc;
  R *Aval, *bvec, *r, *Ap;
  R* zp;  // CG gather records [2][Np][8]: buffer k & 1 holds (z_k, p_{k-1}) of iteration k
  R* pg;  // a solve's starting guess in the direction layout (warm start), or null
  R* dinv;  // [9][Np] inverse of each vertex's 3x3 diagonal block (block Jacobi) or its diagonal
  double* dv;  // CG solution (dv, or lambda in the adjoint): FP64 after each solve
  float *dvh, *dvl;  // FP32 mode: the solution accumulated as float-float hi + lo [Np][3]
  CGSheet* cg;
  acc_t<R> *part_a, *part_b, *part_c;  // per-warp partial sums [NW * 8] (r.z, r.r, p.Ap)
  int tail_threshold;                 // the device loop hands over when <= this many sheets remain
  int* active;
  unsigned long long* iter_total;
  unsigned long long* body_runs;  // [3] CG loop-body executions per phase
  unsigned* sheet_iters;          // [3][S][2] per phase and sheet: largest solve, sum over solves
  unsigned* last_iters;           // [S] iterations of each sheet's last finished solve
  double* gacc;  // [S][3] dL/dY, dL/dkb, dL/drho
  double* gacc_w;  // [S][3] dL/dw (wind velocity)
  double* row_w;   // [Np][3] per-vertex shares of dL/dw (adjoint scratch)
  double air_density;  // > 0: air drag of the relative wind on every free vertex
  const R* wind;       // [S][3] wind velocity per sheet, or null (still air)
  // parameters
  R h, gx, gy, gz, eta;
  double tol;
  int maxit;
  int precond;  // 0 scalar Jacobi, 1 block Jacobi
  bool clamp;
  const R* material;  // [S][4]
};

// ------------------------------------------------------------------ helpers
template <class R> __device__ __forceinline__ V3<R> ld3(const R* a, int i) {
  return {a[3 * (size_t)i], a[3 * (size_t)i + 1], a[3 * (size_t)i + 2]};
}
template <class R> __device__ __forceinline__ void st3(R* a, int i, V3<R> v) {
  a[3 * (size_t)i] = v.x;
  a[3 * (size_t)i + 1] = v.y;
  a[3 * (size_t)i + 2] = v.z;
}
template <class R> __device__ __forceinline__ V3<R> add3(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }

// Explicitly rounded operations for the CG row arithmetic: every kernel that computes a
// CG row (the device loop and the per-sheet solver) evaluates it through these, so the
// compiler has no freedom in fusing multiplies and adds and the kernels agree bitwise.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
// a0 v.x + a1 v.y + a2 v.z as one fixed chain
template <class R> __device__ __forceinline__ R dot3_fixed(R a0, R a1, R a2, V3<R> v) {
  return fma_rn(a2, v.z, fma_rn(a1, v.y, mul_rn(a0, v.x)));
}
// y = B v and y += B v for a row-major 3x3 block B
template <class R> __device__ __forceinline__ V3<R> block_mul(const R (&b)[9], V3<R> v) {
  return {dot3_fixed(b[0], b[1], b[2], v), dot3_fixed(b[3], b[4], b[5], v), dot3_fixed(b[6], b[7], b[8], v)};
}
template <class R> __device__ __forceinline__ void block_acc(V3<R>& y, const R (&b)[9], V3<R> v) {
  y.x = add_rn(y.x, dot3_fixed(b[0], b[1], b[2], v));
  y.y = add_rn(y.y, dot3_fixed(b[3], b[4], b[5], v));
  y.z = add_rn(y.z, dot3_fixed(b[6], b[7], b[8], v));
}

// CG direction vectors are the gathered operand of the SpMV: in FP32 they are stored as
// 16-byte float4 (x, y, z, 0) so a neighbour gather is one aligned load.
template <class R> struct PStride { static constexpr int v = 3; };
template <> struct PStride<float> { static constexpr int v = 4; };
template <class R> __device__ __forceinline__ V3<R> ldp(const R* a, int i) { return ld3(a, i); }
template <> __device__ __forceinline__ V3<float> ldp<float>(const float* a, int i) {
  const float4 q = reinterpret_cast<const float4*>(a)[i];
  return {q.x, q.y, q.z};
}
template <class R> __device__ __forceinline__ void stp(R* a, int i, V3<R> v) { st3(a, i, v); }
template <> __device__ __forceinline__ void stp<float>(float* a, int i, V3<float> v) {
  reinterpret_cast<float4*>(a)[i] = make_float4(v.x, v.y, v.z, 0.f);
}
// CG gather records.  In iteration k every row's SpMV reads, for itself and each
// neighbour j, z_k[j] and the previous direction p_{k-1}[j]; both live in one record of
// 8 reals (x, y, z, 0 of z_k, then of p_{k-1}), so a neighbour costs one aligned 32-byte
// load in FP32 (two 32-byte loads in FP64).  Buffer k & 1 holds the records of iteration
// k; iteration k writes p_k and z_{k+1} into buffer (k + 1) & 1.
template <class R> struct Rec {
  V3<R> z, p;
};
template <class R> __device__ __forceinline__ R* rec(const Dev<R>& d, int k, int i) {
  return d.zp + ((size_t)(k & 1) * d.Np + i) * 8;
}
// a record through L1 (values written by earlier kernels) or L2 only (values written by
// other SMs during the same kernel, after a cluster barrier)
template <class R> __device__ __forceinline__ Rec<R> ld_rec(const R* a) {
  return {ld3(a, 0), {a[4], a[5], a[6]}};
}
template <class R> __device__ __forceinline__ Rec<R> ld_rec_l2(const R* a) {
  return {{__ldcg(a), __ldcg(a + 1), __ldcg(a + 2)}, {__ldcg(a + 4), __ldcg(a + 5), __ldcg(a + 6)}};
}
template <> __device__ __forceinline__ Rec<float> ld_rec<float>(const float* a) {
  float v[8];
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(a));
  return {{v[0], v[1], v[2]}, {v[4], v[5], v[6]}};
}
template <> __device__ __forceinline__ Rec<float> ld_rec_l2<float>(const float* a) {
  float v[8];
  asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(a));
  return {{v[0], v[1], v[2]}, {v[4], v[5], v[6]}};
}
template <class R> __device__ __forceinline__ void st_rec_z(R* a, V3<R> z) { st3(a, 0, z); }
template <class R> __device__ __forceinline__ void st_rec_p(R* a, V3<R> p) { st3(a + 4, 0, p); }
template <> __device__ __forceinline__ void st_rec_z<float>(float* a, V3<float> z) {
  *reinterpret_cast<float4*>(a) = make_float4(z.x, z.y, z.z, 0.f);
}
template <> __device__ __forceinline__ void st_rec_p<float>(float* a, V3<float> p) {
  *reinterpret_cast<float4*>(a + 4) = make_float4(p.x, p.y, p.z, 0.f);
}

// streamed (read-once) matrix data: do not keep in L1
template <class R> __device__ __forceinline__ R lds(const R* a) { return __ldcs(a); }
template <class R> __device__ __forceinline__ V3<R> axpy3(R s, V3<R> x, V3<R> y) {
  return {s * x.x + y.x, s * x.y + y.y, s * x.z + y.z};
}
template <class R> __device__ __forceinline__ double ddot3(V3<R> a, V3<R> b) {
  return (double)a.x * (double)b.x + (double)a.y * (double)b.y + (double)a.z * (double)b.z;
}

template <class R> __device__ __forceinline__ acc_t<R> acc_zero() { return 0.0; }
template <> __device__ __forceinline__ FF acc_zero<float>() { return {0.f, 0.f}; }
template <class R> __device__ __forceinline__ acc_t<R> acc_dot3(V3<R> a, V3<R> b) {
  return (double)dot3_fixed(a.x, a.y, a.z, b);
}
template <> __device__ __forceinline__ FF acc_dot3<float>(V3<float> a, V3<float> b) {
  return {dot3_fixed(a.x, a.y, a.z, b), 0.f};
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}
// warp sum (valid in lane 0), sum, broadcast of lane 0
__device__ __forceinline__ double acc_warp_total(double x) { return warp_sum(x); }
__device__ __forceinline__ FF acc_warp_total(FF x) { return ff_warp_sum(x); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ FF acc_add(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ double acc_bcast0(double x) { return __shfl_sync(0xffffffffu, x, 0); }
__device__ __forceinline__ FF acc_bcast0(FF x) {
  return {__shfl_sync(0xffffffffu, x.hi, 0), __shfl_sync(0xffffffffu, x.lo, 0)};
}
__device__ __forceinline__ bool acc_finite(double x) { return isfinite(x); }
__device__ __forceinline__ bool acc_finite(FF x) { return isfinite(x.hi) && isfinite(x.lo); }

// alpha and beta of a sheet in the form the row kernels take
template <class R> __device__ __forceinline__ acc_t<R> alpha_of(const CGSheet& c) { return c.alpha; }
template <> __device__ __forceinline__ FF alpha_of<float>(const CGSheet& c) { return c.alpha_f; }
template <class R> __device__ __forceinline__ R beta_of(const CGSheet& c) { return (R)c.beta; }
template <> __device__ __forceinline__ float beta_of<float>(const CGSheet& c) { return c.beta_f; }

// ------------------------------------------------------------------ CG scalar steps
// Shared by the device loop's per-sheet scalar kernels and the per-sheet solver, so both
// form alpha, beta and the stopping decisions bitwise alike.  Each returns true when the
// sheet's solve is over (converged, or stopped with a status bit).
// After the initial sums r.z, r.r and |b|^2 (b = r when the solve starts from 0).
template <class R> __device__ __forceinline__ bool cg_init_step(CGSheet& c, acc_t<R> rz, acc_t<R> rr, acc_t<R> bb, double tol);
template <> __device__ __forceinline__ bool cg_init_step<double>(CGSheet& c, double rz, double rr, double bb, double tol) {
  c.rz = rz;
  c.rr = rr;
  c.bb = bb;
  c.stop_rr = tol * tol * bb;
  c.beta = 0.0;
  c.iters = 0;
  c.done = 0;
  c.zero_rhs = bb == 0.0;
  if (!isfinite(rr) || !isfinite(bb)) {
    c.status |= CLOTH_STATUS_NONFINITE;
    return true;
  }
  return bb == 0.0 || rr <= c.stop_rr;
}
template <> __device__ __forceinline__ bool cg_init_step<float>(CGSheet& c, FF rz, FF rr, FF bb, double tol) {
  const double bbd = ff_to_double(bb);
  c.rz = ff_to_double(rz);
  c.rr = ff_to_double(rr);
  c.bb = bbd;
  c.stop_rr = tol * tol * bbd;
  c.rz_f = rz;
  c.stop_f = ff_from_double(c.stop_rr);
  c.beta = 0.0;
  c.beta_f = 0.f;
  c.iters = 0;
  c.done = 0;
  c.zero_rhs = bb.hi == 0.f;
  if (!acc_finite(rr) || !acc_finite(bb)) {
    c.status |= CLOTH_STATUS_NONFINITE;
    return true;
  }
  return bb.hi == 0.f || ff_le(rr, c.stop_f);
}
// After the sum p.Ap: alpha = r.z / p.Ap.
template <class R> __device__ __forceinline__ bool cg_alpha_step(CGSheet& c, acc_t<R> pAp);
template <> __device__ __forceinline__ bool cg_alpha_step<double>(CGSheet& c, double pAp) {
  c.pAp = pAp;
  if (!isfinite(pAp)) {
    c.status |= CLOTH_STATUS_NONFINITE;
    return true;
  }
  if (pAp <= 0.0) {
    c.status |= CLOTH_STATUS_INDEFINITE;
    return true;
  }
  c.alpha = c.rz / pAp;
  return false;
}
template <> __device__ __forceinline__ bool cg_alpha_step<float>(CGSheet& c, FF pAp) {
  if (!acc_finite(pAp)) {
    c.status |= CLOTH_STATUS_NONFINITE;
    return true;
  }
  if (pAp.hi <= 0.f) {
    c.status |= CLOTH_STATUS_INDEFINITE;
    return true;
  }
  c.alpha_f = ff_div(c.rz_f, pAp);
  return false;
}
// After the update's sums r.z, r.r: beta = r.z / previous r.z, one iteration done.
template <class R> __device__ __forceinline__ bool cg_beta_step(CGSheet& c, acc_t<R> rz, acc_t<R> rr, int maxit);
template <> __device__ __forceinline__ bool cg_beta_step<double>(CGSheet& c, double rz, double rr, int maxit) {
  c.beta = rz / c.rz;
  c.rz = rz;
  c.rr = rr;
  c.iters += 1;
  if (!isfinite(rr) || !isfinite(rz)) {
    c.status |= CLOTH_STATUS_NONFINITE;
    return true;
  }
  if (rr <= c.stop_rr) return true;
  if (c.iters >= maxit) {
    c.status |= CLOTH_STATUS_CG_MAXITER;
    return true;
  }
  return false;
}
template <> __device__ __forceinline__ bool cg_beta_step<float>(CGSheet& c, FF rz, FF rr, int maxit) {
  c.beta_f = ff_div(rz, c.rz_f).hi;
  c.rz_f = rz;
  c.iters += 1;
  if (!acc_finite(rr) || !acc_finite(rz)) {
    c.status |= CLOTH_STATUS_NONFINITE;
    return true;
  }
  if (ff_le(rr, c.stop_f)) return true;
  if (c.iters >= maxit) {
    c.status |= CLOTH_STATUS_CG_MAXITER;
    return true;
  }
  return false;
}
__device__ __forceinline__ double alpha_cast(double a) { return a; }
__device__ __forceinline__ float alpha_cast(FF a) { return a.hi; }  // = (float) alpha

// z = D^{-1} r with the stored 3x3 inverse (SoA [9][Np])
template <class R>
__device__ __forceinline__ V3<R> apply_dinv(const R* __restrict__ D, int Np, int i, V3<R> r) {
  const size_t n = (size_t)Np;
  return {dot3_fixed(D[i], D[n + i], D[2 * n + i], r), dot3_fixed(D[3 * n + i], D[4 * n + i], D[5 * n + i], r),
          dot3_fixed(D[6 * n + i], D[7 * n + i], D[8 * n + i], r)};
}

// Block sum of NV doubles (blockDim.x == kThreads); result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < kThreads / 32 ? sh[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
  __syncthreads();
}

template <class R>
__device__ __forceinline__ void finish_sheet(const Dev<R>& d, int s, int phase, cudaGraphConditionalHandle cond,
                                             int use_cond) {
  d.cg[s].done = 1;
  atomicAdd(&d.iter_total[phase], (unsigned long long)d.cg[s].iters);
  // one thread finishes sheet s of a solve, so these need no atomics
  unsigned* si = d.sheet_iters + 2 * ((size_t)phase * d.S + s);
  si[0] = max(si[0], (unsigned)d.cg[s].iters);
  si[1] += (unsigned)d.cg[s].iters;
  d.last_iters[s] = (unsigned)d.cg[s].iters;
  const int left = atomicSub(d.active, 1) - 1;
  // exactly one thread sees each value of `left`: the one reaching the hand-over point
  // ends the device loop (the per-sheet cluster solver finishes the remaining sheets)
  if (left == d.tail_threshold && use_cond) cudaGraphSetConditional(cond, 0);
}

// ------------------------------------------------------------------ layout moves
template <class R, class Tin, class Tout>
__global__ void k_gather(Dev<R> d, const Tin* __restrict__ in, Tout* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const int u = d.i2u[i];
  V3<Tout> v = {Tout(0), Tout(0), Tout(0)};
  if (u >= 0 && in) {
    const V3<Tin> w = ld3(in, u);
    v = {(Tout)w.x, (Tout)w.y, (Tout)w.z};
  }
  st3(out, i, v);
}

template <class R, class Tin>
__global__ void k_scatter(Dev<R> d, const Tin* __restrict__ in, R* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const int u = d.i2u[i];
  if (u < 0) return;
  const V3<Tin> v = ld3(in, i);
  st3(out, u, V3<R>{(R)v.x, (R)v.y, (R)v.z});
}

// Element positions relative to the element's first vertex: the differences are
// formed from the FP64 state before rounding to R, so FP32 element arithmetic sees
// edge vectors with full relative precision.
template <class R, int K>
__device__ __forceinline__ void load_relative(const double* __restrict__ x, const int* idx, V3<R>* out) {
  const V3<double> x0 = ld3(x, idx[0]);
  out[0] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 1; a < K; ++a) {
    const V3<double> xa = ld3(x, idx[a]);
    out[a] = {(R)(xa.x - x0.x), (R)(xa.y - x0.y), (R)(xa.z - x0.z)};
  }
}

// out_a = sum_b H_ab v_b from the upper 3x3 blocks of a K-vertex element (H_ba = H_ab^T).
template <class R, int K>
__device__ __forceinline__ void block_matvec(const R (*H)[9], const V3<R>* v, V3<R>* out) {
#pragma unroll
  for (int a = 0; a < K; ++a) {
    R o[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int b = 0; b < K; ++b) {
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      const R* Hb = H[lo * K - lo * (lo - 1) / 2 + (hi - lo)];
      const R vb[3] = {v[b].x, v[b].y, v[b].z};
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) o[c] += (a <= b ? Hb[3 * c + e] : Hb[3 * e + c]) * vb[e];
    }
    out[a] = {o[0], o[1], o[2]};
  }
}

// Relative vectors of an element (u_a - u_0), differences formed in FP64: every
// element operator here annihilates uniform translations, so dropping the common
// part first removes the cancellation of large, nearly rigid motions.
template <class R, int K>
__device__ __forceinline__ void load_relative_dir(const R* __restrict__ u, const int* idx, V3<R>* out) {
  const V3<R> u0 = ld3(u, idx[0]);
  out[0] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 1; a < K; ++a) {
    const V3<R> ua = ld3(u, idx[a]);
    out[a] = {(R)((double)ua.x - (double)u0.x), (R)((double)ua.y - (double)u0.y), (R)((double)ua.z - (double)u0.z)};
  }
}

template <class R>
__device__ __forceinline__ V3<R> ld3r(const double* __restrict__ x, int i) {
  const V3<double> v = ld3(x, i);
  return {(R)v.x, (R)v.y, (R)v.z};
}

// ------------------------------------------------------------------ element kernels
template <class R>
__device__ __forceinline__ TriConst<R> tri_const(const Dev<R>& d, int t) {
  TriConst<R> k;
  const int s = d.tri_sheet[t];
  const R b00 = d.tri_rest[t], b01 = d.tri_rest[(size_t)d.M + t];
  const R b10 = d.tri_rest[2 * (size_t)d.M + t], b11 = d.tri_rest[3 * (size_t)d.M + t];
  k.g[1][0] = b00;
  k.g[1][1] = b01;
  k.g[2][0] = b10;
  k.g[2][1] = b11;
  k.g[0][0] = -(b00 + b10);
  k.g[0][1] = -(b01 + b11);
  k.A0 = d.tri_rest[4 * (size_t)d.M + t];
  const R Y = d.material[4 * s], nu = d.material[4 * s + 1];
  k.mu = Y / (R(2) * (R(1) + nu));
  k.lam = Y * nu / (R(1) - nu * nu);
  k.eps = d.eta * Y;
  return k;
}

// Green strain G = Bm^T (Ds^T Ds - Dm^T Dm) Bm / 2 with the edge metric difference
// formed in FP64 from the FP64 state (no cancellation of the identity in F^T F - I).
template <class R>
__device__ __forceinline__ Sym2<R> green_strain(const Dev<R>& d, int t, const double* __restrict__ x,
                                                const int* idx) {
  const V3<double> x0 = ld3(x, idx[0]), x1 = ld3(x, idx[1]), x2 = ld3(x, idx[2]);
  const V3<double> e1 = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
  const V3<double> e2 = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
  const double m00 = e1.x * e1.x + e1.y * e1.y + e1.z * e1.z - d.tri_metric[t];
  const double m11 = e2.x * e2.x + e2.y * e2.y + e2.z * e2.z - d.tri_metric[(size_t)d.M + t];
  const double m01 = e1.x * e2.x + e1.y * e2.y + e1.z * e2.z - d.tri_metric[2 * (size_t)d.M + t];
  const double b00 = d.tri_rest[t], b01 = d.tri_rest[(size_t)d.M + t];
  const double b10 = d.tri_rest[2 * (size_t)d.M + t], b11 = d.tri_rest[3 * (size_t)d.M + t];
  // (dM Bm) then Bm^T (dM Bm)
  const double q00 = m00 * b00 + m01 * b10, q01 = m00 * b01 + m01 * b11;
  const double q10 = m01 * b00 + m11 * b10, q11 = m01 * b01 + m11 * b11;
  const double g00 = 0.5 * (b00 * q00 + b10 * q10);
  const double g11 = 0.5 * (b01 * q01 + b11 * q11);
  const double g01 = 0.5 * (b00 * q01 + b10 * q11);
  return {(R)g00, (R)g11, (R)g01};
}

template <class R>
__device__ __forceinline__ HingeConst<R> hinge_const(const Dev<R>& d, int e) {
  const int s = d.hin_sheet[e];
  return {d.material[4 * s + 2] * d.hin_rest[e], d.hin_rest[(size_t)d.E + e]};
}

// Membrane force -dE/dx_a = -A0 F S g_a in FP64.  Element forces of a tensioned sheet
// are tens to hundreds of times larger than the net force per vertex, so they are
// formed and summed in FP64 whatever the batch precision (the Hessian stays in R).
template <class R>
__device__ __forceinline__ void membrane_force_fp64(const Dev<R>& d, int t, const V3<double>* xr, V3<double>* f) {
  TriConst<double> k;
  const double b00 = d.tri_rest_d[t], b01 = d.tri_rest_d[(size_t)d.M + t];
  const double b10 = d.tri_rest_d[2 * (size_t)d.M + t], b11 = d.tri_rest_d[3 * (size_t)d.M + t];
  k.g[1][0] = b00;
  k.g[1][1] = b01;
  k.g[2][0] = b10;
  k.g[2][1] = b11;
  k.g[0][0] = -(b00 + b10);
  k.g[0][1] = -(b01 + b11);
  k.A0 = d.tri_rest_d[4 * (size_t)d.M + t];
  const int s = d.tri_sheet[t];
  const double Y = (double)d.material[4 * s], nu = (double)d.material[4 * s + 1];
  k.mu = Y / (2.0 * (1.0 + nu));
  k.lam = Y * nu / (1.0 - nu * nu);
  k.eps = 0.0;
  // G from the edge metric difference (exact zero at rest)
  const V3<double> e1 = xr[1], e2 = xr[2];
  const double m00 = dot(e1, e1) - d.tri_metric[t];
  const double m11 = dot(e2, e2) - d.tri_metric[(size_t)d.M + t];
  const double m01 = dot(e1, e2) - d.tri_metric[2 * (size_t)d.M + t];
  const double q00 = m00 * b00 + m01 * b10, q01 = m00 * b01 + m01 * b11;
  const double q10 = m01 * b00 + m11 * b10, q11 = m01 * b01 + m11 * b11;
  const Sym2<double> G = {0.5 * (b00 * q00 + b10 * q10), 0.5 * (b01 * q01 + b11 * q11), 0.5 * (b00 * q01 + b10 * q11)};
  double F[3][2];
  deformation_gradient(k, xr, F);
  const Sym2<double> S = stvk_stress_G(k, G);
#pragma unroll
  for (int a = 0; a < 3; ++a) f[a] = scale(-k.A0, mat32_sym_vec(F, S, k.g[a]));
}

template <class R>
__device__ __forceinline__ void bending_force_fp64(const Dev<R>& d, int e, const V3<double>* xr, V3<double>* f) {
  const int s = d.hin_sheet[e];
  const double kw = (double)d.material[4 * s + 2] * d.hin_rest_d[e];
  double th;
  V3<double> g[4];
  dihedral_grad(xr, th, g);
  const double c = -kw * (th - d.hin_rest_d[(size_t)d.E + e]);
#pragma unroll
  for (int a = 0; a < 4; ++a) f[a] = scale(c, g[a]);
}

template <class R, int K>
__device__ __forceinline__ void load_relative_d(const double* __restrict__ x, const int* idx, V3<double>* out) {
  const V3<double> x0 = ld3(x, idx[0]);
  out[0] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 1; a < K; ++a) {
    const V3<double> xa = ld3(x, idx[a]);
    out[a] = {xa.x - x0.x, xa.y - x0.y, xa.z - x0.z};
  }
}

// N values of v to p with 8-byte stores (p 8-byte aligned, N even: the element records
// of 54 and 90 FP32 values, 216 and 360 bytes) or, in FP64, 16-byte stores (p 16-byte
// aligned)
template <int N>
__device__ __forceinline__ void st_record(float* p, const float* v) {
  static_assert(N % 2 == 0, "record size");
#pragma unroll
  for (int c = 0; c < N / 2; ++c) reinterpret_cast<float2*>(p)[c] = make_float2(v[2 * c], v[2 * c + 1]);
}
template <int N>
__device__ __forceinline__ void st_record(double* p, const double* v) {
  static_assert(N % 2 == 0, "record size");
#pragma unroll
  for (int c = 0; c < N / 2; ++c) reinterpret_cast<double2*>(p)[c] = make_double2(v[2 * c], v[2 * c + 1]);
}

// NT: threads per CTA (the autotuner picks 64, 128 or 256 per element kind)
template <class R, int NT = kElemThreads>
__global__ void __launch_bounds__(NT) k_elem_tri(Dev<R> d, const double* __restrict__ x,
                                                 const double* __restrict__ v) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.M) return;
  TriConst<R> k = tri_const(d, t);
  V3<R> xe[3], f[3];
  R H[6][9];
  int idx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) idx[a] = d.tri_v[(size_t)a * d.M + t];
  load_relative<R, 3>(x, idx, xe);
  membrane_force_hessian(k, xe, green_strain(d, t, x, idx), d.clamp, f, H);
  V3<double> xr[3], fd[3];
  load_relative_d<R, 3>(x, idx, xr);
  membrane_force_fp64(d, t, xr, fd);
  if (v) {  // store f - h H~ v (the element's share of b / h)
    V3<R> ve[3], Hv[3];
    load_relative<R, 3>(v, idx, ve);
    block_matvec<R, 3>(H, ve, Hv);
    const double h = (double)d.h;
#pragma unroll
    for (int a = 0; a < 3; ++a) fd[a] = {fd[a].x - h * Hv[a].x, fd[a].y - h * Hv[a].y, fd[a].z - h * Hv[a].z};
  }
  double* fo = d.tri_f + 9 * (size_t)t;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fo[3 * a] = fd[a].x;
    fo[3 * a + 1] = fd[a].y;
    fo[3 * a + 2] = fd[a].z;
  }
  st_record<54>(d.tri_H + 54 * (size_t)t, &H[0][0]);
}

template <class R, int NT = kElemThreads>
__global__ void __launch_bounds__(NT) k_elem_hinge(Dev<R> d, const double* __restrict__ x,
                                                   const double* __restrict__ v) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  HingeConst<R> k = hinge_const(d, e);
  V3<R> xe[4], f[4];
  R H[10][9];
  int idx[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) idx[a] = d.hin_v[(size_t)a * d.E + e];
  load_relative<R, 4>(x, idx, xe);
  bending_force_hessian(k, xe, f, H);
  V3<double> xr[4], fd[4];
  load_relative_d<R, 4>(x, idx, xr);
  bending_force_fp64(d, e, xr, fd);
  if (v) {
    V3<R> ve[4], Hv[4];
    load_relative<R, 4>(v, idx, ve);
    block_matvec<R, 4>(H, ve, Hv);
    const double h = (double)d.h;
#pragma unroll
    for (int a = 0; a < 4; ++a) fd[a] = {fd[a].x - h * Hv[a].x, fd[a].y - h * Hv[a].y, fd[a].z - h * Hv[a].z};
  }
  {  // 12 FP64 force entries (96 bytes per hinge, 16-byte aligned)
    const double fv[12] = {fd[0].x, fd[0].y, fd[0].z, fd[1].x, fd[1].y, fd[1].z,
                           fd[2].x, fd[2].y, fd[2].z, fd[3].x, fd[3].y, fd[3].z};
    st_record<12>(d.hin_f + 12 * (size_t)e, fv);
  }
  st_record<90>(d.hin_H + 90 * (size_t)e, &H[0][0]);
}

// element-vertex force slot -> pointer to 3 reals
template <class R>
__device__ __forceinline__ const double* force_slot(const Dev<R>& d, int slot) {
  return slot < 3 * d.M ? d.tri_f + 3 * (size_t)slot : d.hin_f + 3 * (size_t)(slot - 3 * d.M);
}

// Sum of the element Hessian blocks of SELL entry `ent` (fixed order, transposes applied).
template <class R>
__device__ __forceinline__ void gather_block(const Dev<R>& d, int ent, R (&Hb)[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) Hb[q] = R(0);
  const int q0 = d.contrib_ptr[ent], q1 = d.contrib_ptr[ent + 1];
  for (int q = q0; q < q1; ++q) {
    const int code = d.contrib[q];
    const int blk = code >> 1;
    const R* src = blk < 6 * d.M ? d.tri_H + 9 * (size_t)blk : d.hin_H + 9 * (size_t)(blk - 6 * d.M);
    if (code & 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) Hb[3 * c + e] += src[3 * e + c];
    } else {
#pragma unroll
      for (int q2 = 0; q2 < 9; ++q2) Hb[q2] += src[q2];
    }
  }
}

// Assembly of A, b, D^{-1} (one thread per row; a warp is one SELL slice).
// The element kernels stored f_e - h H~_e v_e per element vertex, so
// b_i = h (sum_e (f_e - h H~_e v_e)_i + m_i g + F_i)  (= h (f + M g + F) - h^2 H~ v).
// Fext: user-layout external force of this step or null.
// Air drag on a free vertex: the air moves at the sheet's wind velocity w; the vertex
// with lumped rest area A feels f = rho_air A s(d) d for the relative air velocity
// d = w - v, with the smoothed speed s(d) = sqrt(|d|^2 + eps^2).  df/dv = -rho_air A G(d),
// G(d) = s I + d d^T / s, symmetric positive definite: it adds h rho_air A G to the
// vertex's diagonal block of the step matrix (Eq. 5 with df/dv nonzero).
constexpr double kAirEps = 1e-3;  // m/s

template <class R>
__device__ __forceinline__ V3<double> relative_wind(const Dev<R>& d, int s, V3<double> v) {
  const V3<double> w = d.wind ? V3<double>{(double)d.wind[3 * s], (double)d.wind[3 * s + 1], (double)d.wind[3 * s + 2]}
                              : V3<double>{0.0, 0.0, 0.0};
  return {w.x - v.x, w.y - v.y, w.z - v.z};
}

__device__ __forceinline__ double air_speed(V3<double> r) { return sqrt(r.x * r.x + r.y * r.y + r.z * r.z + kAirEps * kAirEps); }

// G(r) a
__device__ __forceinline__ V3<double> air_G(V3<double> r, V3<double> a) {
  const double s = air_speed(r), ra = (r.x * a.x + r.y * a.y + r.z * a.z) / s;
  return {s * a.x + ra * r.x, s * a.y + ra * r.y, s * a.z + ra * r.z};
}

// the vector k -> a^T (dG/dr_k) b
__device__ __forceinline__ V3<double> air_dG(V3<double> r, V3<double> a, V3<double> b) {
  const double s = air_speed(r);
  const double ab = a.x * b.x + a.y * b.y + a.z * b.z, ar = a.x * r.x + a.y * r.y + a.z * r.z;
  const double rb = r.x * b.x + r.y * b.y + r.z * b.z, k = ar * rb / (s * s * s);
  return {r.x * ab / s + (a.x * rb + ar * b.x) / s - k * r.x, r.y * ab / s + (a.y * rb + ar * b.y) / s - k * r.y,
          r.z * ab / s + (a.z * rb + ar * b.z) / s - k * r.z};
}

// v: the velocity the step starts from (FP64, internal layout), or null (no drag terms)
template <class R>
__global__ void __launch_bounds__(kThreads) k_assemble(Dev<R> d, const R* __restrict__ Fext,
                                                      const double* __restrict__ v) {
  const int w = blockIdx.x;
  const int s = d.work_sheet[w];
  if (threadIdx.x >= d.work_rows[w]) return;
  const int i = d.work_row0[w] + threadIdx.x;
  const int sl = i >> 5, lane = i & 31;
  const int K = d.slice_K[sl], base = d.slice_base[sl];
  const bool pin_i = d.pinned[i] != 0;
  const R rho = d.material[4 * s + 3];
  const R mass = rho * d.area3[i];
  const R h2 = d.h * d.h;
  V3<double> f = {0.0, 0.0, 0.0};
  for (int q = d.vf_ptr[i]; q < d.vf_ptr[i + 1]; ++q) {
    const double* src = force_slot(d, d.vf[q]);
    f.x += src[0];
    f.y += src[1];
    f.z += src[2];
  }
  // Slot 0 stores the row sum R_i = sum_j A_ij instead of A_ii, which the SpMV uses in
  // difference form (A p)_i = R_i p_i + sum_{j != i} A_ij (p_j - p_i).  H annihilates
  // uniform translations, so R_i = m_i I - h^2 sum_{pinned j} H_ij exactly (no
  // cancellation), and smooth p no longer cancels large terms in the product.
  double dblk[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  R rsum[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) rsum[q] = R(0);
  for (int k = 0; k < K; ++k) {
    const int ent = (base + k) * 32 + lane;
    const int j = d.cols[ent];
    R Hb[9];
    gather_block(d, ent, Hb);
    const bool pin_j = d.pinned[j] != 0;
    const bool zero = pin_i || pin_j;
    R* dst = d.Aval + (size_t)(base + k) * 32 * 9 + lane;
    if (k == 0) {
      if (!pin_i) {
#pragma unroll
        for (int q = 0; q < 9; ++q)
          dblk[q] = (double)h2 * (double)Hb[q] + ((q == 0 || q == 4 || q == 8) ? (double)mass : 0.0);
      }
      continue;  // written after the loop
    }
    if (!pin_i && pin_j && j != i) {
#pragma unroll
      for (int q = 0; q < 9; ++q) rsum[q] += Hb[q];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) dst[q * 32] = zero ? R(0) : h2 * Hb[q];
  }
  // air drag: h rho_air A G(d) on the diagonal block, the force into b
  double dg[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  V3<double> fw = {0.0, 0.0, 0.0};
  if (d.air_density > 0.0 && v && !pin_i) {
    const V3<double> r = relative_wind(d, s, ld3(v, i));
    const double c = d.air_density * (double)d.area3[i], sp = air_speed(r), hc = (double)d.h * c;
    const double rr[3] = {r.x, r.y, r.z};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 3; ++q) dg[3 * a + q] = hc * ((a == q ? sp : 0.0) + rr[a] * rr[q] / sp);
    fw = {c * sp * r.x, c * sp * r.y, c * sp * r.z};
#pragma unroll
    for (int q = 0; q < 9; ++q) dblk[q] += dg[q];
  }
  {
    R* dst = d.Aval + (size_t)base * 32 * 9 + lane;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const R dq = (q == 0 || q == 4 || q == 8) ? (pin_i ? R(1) : mass) : R(0);
      dst[q * 32] = pin_i ? dq : dq + (R)dg[q] - h2 * rsum[q];
    }
  }
  V3<R> b = {R(0), R(0), R(0)};
  if (!pin_i) {
    const int u = d.i2u[i];
    V3<R> fe = Fext && u >= 0 ? ld3(Fext, u) : V3<R>{R(0), R(0), R(0)};
    const double h = (double)d.h, md = (double)mass;
    b.x = (R)(h * (f.x + md * (double)d.gx + (double)fe.x + fw.x));
    b.y = (R)(h * (f.y + md * (double)d.gy + (double)fe.y + fw.y));
    b.z = (R)(h * (f.z + md * (double)d.gz + (double)fe.z + fw.z));
  }
  st3(d.bvec, i, b);
  // preconditioner: inverse of the 3x3 diagonal block (adjugate / determinant, in FP64)
  double inv[9];
  if (d.precond) {
    const double* m = dblk;
    const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
    const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    const double id = 1.0 / det;
    inv[0] = c00 * id;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    inv[3] = c01 * id;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    inv[6] = c02 * id;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) * id;
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) inv[q] = (q == 0 || q == 4 || q == 8) ? 1.0 / dblk[q] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) d.dinv[(size_t)q * d.Np + i] = (R)inv[q];
}

// ------------------------------------------------------------------ CG
template <class R>
__global__ void k_solve_begin(Dev<R> d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *d.active = d.S;
}

template <class R>
__global__ void k_cond_set(Dev<R> d, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(cond, *d.active > d.tail_threshold ? 1u : 0u);
}

// Jacobi-PCG over all sheets at once.  The streaming kernels (init, SpMV, update) write one
// partial sum per warp and use no barrier, fence or atomic; a per-sheet scalar kernel (one
// warp per sheet, fixed summation order, hence deterministic) then forms alpha, or beta and
// the convergence test.  Iteration k of a sheet uses p_k = z_k + beta_k p_{k-1}
// (beta_0 = 0), which the SpMV forms from the gather records for the own row and every
// neighbour (the same fused multiply-add everywhere, so every copy is bitwise the same).
template <class R>
__device__ __forceinline__ V3<R> next_dir(V3<R> z, R beta, V3<R> pold) {
  return {fma_rn(beta, pold.x, z.x), fma_rn(beta, pold.y, z.y), fma_rn(beta, pold.z, z.z)};
}

// partial of warp `wp` (0..7) of work entry w: index w * 8 + wp
constexpr int kWarpsPerEntry = kThreads / 32;

// r = rhs, dv = 0, z_0 = D^{-1} r, p_{-1} = 0 (record buffer 0); partials of r.z and r.r.
template <class R>
__global__ void __launch_bounds__(kThreads) k_cg_init(Dev<R> d, const R* __restrict__ rhs) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < d.NW; w += gridDim.x) {
    const bool on = threadIdx.x < d.work_rows[w];
    const int i = d.work_row0[w] + threadIdx.x;
    acc_t<R> v0 = acc_zero<R>(), v1 = acc_zero<R>();
    if (on) {
      const V3<R> r = ld3(rhs, i);
      const V3<R> z = apply_dinv(d.dinv, d.Np, i, r);
      st3(d.r, i, r);
      st_rec_z(rec(d, 0, i), z);                      // z_0
      st_rec_p(rec(d, 0, i), V3<R>{R(0), R(0), R(0)});  // p_{-1} = 0
      if constexpr (std::is_same<R, float>::value) {
        st3(d.dvh, i, V3<float>{0.f, 0.f, 0.f});
        st3(d.dvl, i, V3<float>{0.f, 0.f, 0.f});
      } else {
        st3(d.dv, i, V3<double>{0.0, 0.0, 0.0});
      }
      v0 = acc_dot3(r, z);
      v1 = acc_dot3(r, r);
    }
    const acc_t<R> t0 = acc_warp_total(v0), t1 = acc_warp_total(v1);
    if (lane == 0) {
      d.part_a[(size_t)w * kWarpsPerEntry + wp] = t0;
      d.part_b[(size_t)w * kWarpsPerEntry + wp] = t1;
    }
  }
}

// Sum over the warp partials of sheet s (one warp, lane-strided then shuffle tree).
template <class R>
__device__ __forceinline__ acc_t<R> sheet_sum(const Dev<R>& d, const acc_t<R>* part, int s) {
  const int lane = threadIdx.x & 31;
  const int p0 = d.sheet_wfirst[s] * kWarpsPerEntry, p1 = d.sheet_wfirst[s + 1] * kWarpsPerEntry;
  acc_t<R> acc = acc_zero<R>();
  for (int q = p0 + lane; q < p1; q += 32) acc = acc_add(acc, part[q]);
  return acc_bcast0(acc_warp_total(acc));
}

// Per sheet after k_cg_init (guess: after k_cg_init_guess, whose |b|^2 partials are in
// part_c): r.z, r.r, |b|^2; a sheet with b = 0 (or non-finite), or whose guess already
// meets the tolerance, is done at once.
template <class R>
__global__ void k_cg_scalar_init(Dev<R> d, int phase, int guess) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= d.S) return;
  const acc_t<R> rz = sheet_sum(d, d.part_a, s), rr = sheet_sum(d, d.part_b, s);
  const acc_t<R> bb = guess ? sheet_sum(d, d.part_c, s) : rr;
  if ((threadIdx.x & 31) != 0) return;
  if (cg_init_step<R>(d.cg[s], rz, rr, bb, d.tol)) finish_sheet(d, s, phase, 0, 0);
}

// One row of A v in difference form, (A v)_i = R_i v_i + sum_{j != i} A_ij (v_j - v_i), for
// the row's own value vi and gather(j) giving v_j (two slots per loop iteration: more loads
// in flight).
template <class R, class G>
__device__ __forceinline__ V3<R> spmv_core(const Dev<R>& d, int i, V3<R> vi, G gather) {
  const int sl = i >> 5, lane = i & 31;
  const int K = d.slice_K[sl], base = d.slice_base[sl];
  const R* a0 = d.Aval + (size_t)base * 32 * 9 + lane;
  R ab[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) ab[t] = lds(a0 + 32 * t);
  V3<R> y = block_mul(ab, vi);
  int q = 1;
  for (; q + 1 < K; q += 2) {
    const int e0 = (base + q) * 32 + lane, e1 = e0 + 32;
    const int j0 = lds(d.cols + e0), j1 = lds(d.cols + e1);
    const R* a = d.Aval + (size_t)(base + q) * 32 * 9 + lane;
    const R* b = a + 32 * 9;
    R av[9], bv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      av[t] = lds(a + 32 * t);
      bv[t] = lds(b + 32 * t);
    }
    const V3<R> p0 = gather(j0), p1 = gather(j1);
    block_acc(y, av, V3<R>{p0.x - vi.x, p0.y - vi.y, p0.z - vi.z});
    block_acc(y, bv, V3<R>{p1.x - vi.x, p1.y - vi.y, p1.z - vi.z});
  }
  if (q < K) {
    const int e0 = (base + q) * 32 + lane;
    const int j0 = lds(d.cols + e0);
    const R* a = d.Aval + (size_t)(base + q) * 32 * 9 + lane;
    R av[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) av[t] = lds(a + 32 * t);
    const V3<R> p0 = gather(j0);
    block_acc(y, av, V3<R>{p0.x - vi.x, p0.y - vi.y, p0.z - vi.z});
  }
  return y;
}

// One row of the CG SpMV of iteration k: p_k = z_k + beta_k p_{k-1} formed from the records
// for the row (and stored as the row's p_k) and for every neighbour, Ap_i = (A p_k)_i;
// returns p_i . Ap_i.
template <class R>
__device__ __forceinline__ acc_t<R> spmv_row(const Dev<R>& d, int i, R beta, int k) {
  const Rec<R> own = ld_rec(rec(d, k, i));
  const V3<R> pi = next_dir(own.z, beta, own.p);
  st_rec_p(rec(d, k + 1, i), pi);
  const V3<R> y = spmv_core(d, i, pi, [&](int j) {
    const Rec<R> n = ld_rec(rec(d, k, j));
    return next_dir(n.z, beta, n.p);
  });
  st3(d.Ap, i, y);
  return acc_dot3(pi, y);
}

// One row of the update: dv += alpha p_k (FP64, or float-float in FP32 mode),
// r -= alpha Ap, z = D^{-1} r (stored).
template <class R>
__device__ __forceinline__ void update_row(const Dev<R>& d, int i, acc_t<R> al, int k, acc_t<R>& rz,
                                           acc_t<R>& rr) {
  const R alpha = alpha_cast(al);
  R* rk1 = rec(d, k + 1, i);  // holds p_k (written by this iteration's SpMV); receives z_{k+1}
  const V3<R> p = ld_rec(rk1).p, Ap = ld3(d.Ap, i);
  V3<R> r = ld3(d.r, i);
  if constexpr (std::is_same<R, float>::value) {
    const V3<float> xh = ld3(d.dvh, i), xl = ld3(d.dvl, i);
    const FF a = ff_add({xh.x, xl.x}, ff_mul(al, p.x));
    const FF b = ff_add({xh.y, xl.y}, ff_mul(al, p.y));
    const FF c = ff_add({xh.z, xl.z}, ff_mul(al, p.z));
    st3(d.dvh, i, V3<float>{a.hi, b.hi, c.hi});
    st3(d.dvl, i, V3<float>{a.lo, b.lo, c.lo});
  } else {
    V3<double> x = ld3(d.dv, i);
    x = {fma_rn(al, (double)p.x, x.x), fma_rn(al, (double)p.y, x.y), fma_rn(al, (double)p.z, x.z)};
    st3(d.dv, i, x);
  }
  r = {fma_rn(-alpha, Ap.x, r.x), fma_rn(-alpha, Ap.y, r.y), fma_rn(-alpha, Ap.z, r.z)};
  st3(d.r, i, r);
  const V3<R> z = apply_dinv(d.dinv, d.Np, i, r);
  st_rec_z(rk1, z);
  rz = acc_dot3(r, z);
  rr = acc_dot3(r, r);
}

// Starting guess of a solve (FP64, internal layout): kept as the solution accumulator and,
// rounded to the batch precision, in the gatherable layout the SpMV reads (d.pg).
template <class R>
__global__ void k_cg_guess(Dev<R> d, const double* __restrict__ guess) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const V3<double> g = ld3(guess, i);
  stp(d.pg, i, V3<R>{(R)g.x, (R)g.y, (R)g.z});
  if constexpr (std::is_same<R, float>::value) {
    const V3<float> h = {(float)g.x, (float)g.y, (float)g.z};
    st3(d.dvh, i, h);
    st3(d.dvl, i, V3<float>{(float)(g.x - (double)h.x), (float)(g.y - (double)h.y), (float)(g.z - (double)h.z)});
  } else {
    st3(d.dv, i, g);
  }
}

// Solve started from the guess of k_cg_guess: r = rhs - A g (the SpMV's difference form),
// z_0 = D^{-1} r, p_{-1} = 0; partials of r.z, r.r and |rhs|^2 (the stopping test
// stays |r| <= tol |b|).
template <class R>
__global__ void __launch_bounds__(kThreads) k_cg_init_guess(Dev<R> d, const R* __restrict__ rhs) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < d.NW; w += gridDim.x) {
    const bool on = threadIdx.x < d.work_rows[w];
    const int i = d.work_row0[w] + threadIdx.x;
    acc_t<R> v0 = acc_zero<R>(), v1 = acc_zero<R>(), v2 = acc_zero<R>();
    if (on) {
      const V3<R> ag = spmv_core(d, i, ldp(d.pg, i), [&](int j) { return ldp(d.pg, j); });  // A g
      const V3<R> b = ld3(rhs, i);
      const V3<R> r = {add_rn(b.x, -ag.x), add_rn(b.y, -ag.y), add_rn(b.z, -ag.z)};
      const V3<R> z = apply_dinv(d.dinv, d.Np, i, r);
      st3(d.r, i, r);
      st_rec_z(rec(d, 0, i), z);                      // z_0
      st_rec_p(rec(d, 0, i), V3<R>{R(0), R(0), R(0)});  // p_{-1} = 0
      v0 = acc_dot3(r, z);
      v1 = acc_dot3(r, r);
      v2 = acc_dot3(b, b);
    }
    const acc_t<R> t0 = acc_warp_total(v0), t1 = acc_warp_total(v1), t2 = acc_warp_total(v2);
    if (lane == 0) {
      d.part_a[(size_t)w * kWarpsPerEntry + wp] = t0;
      d.part_b[(size_t)w * kWarpsPerEntry + wp] = t1;
      d.part_c[(size_t)w * kWarpsPerEntry + wp] = t2;
    }
  }
}

// End of a solve: the solution as FP64 (FP32 mode: dv = hi + lo), 0 on sheets with b = 0
// (a solve started from a guess keeps the guess there otherwise); optionally also kept in
// `keep` as the next solve's guess.
template <class R>
__global__ void k_cg_solution(Dev<R> d, double* __restrict__ keep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  V3<double> x;
  if constexpr (std::is_same<R, float>::value) {
    const V3<float> h = ld3(d.dvh, i), l = ld3(d.dvl, i);
    x = {(double)h.x + (double)l.x, (double)h.y + (double)l.y, (double)h.z + (double)l.z};
  } else {
    x = ld3(d.dv, i);
  }
  if (d.cg[d.vsheet[i]].zero_rhs) x = {0.0, 0.0, 0.0};
  st3(d.dv, i, x);
  if (keep) st3(keep, i, x);
}

// Ap = A p_k over all active sheets; warp partials of p.Ap.
template <class R>
__global__ void __launch_bounds__(kThreads) k_cg_spmv(Dev<R> d) {
  const int lane_w = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < d.NW; w += gridDim.x) {
    const int s = d.work_sheet[w];
    if (d.cg[s].done) continue;  // uniform over the CTA
    const int k = d.cg[s].iters;
    const R beta = beta_of<R>(d.cg[s]);
    acc_t<R> v = acc_zero<R>();
    if (threadIdx.x < d.work_rows[w])
      v = spmv_row<R>(d, d.work_row0[w] + threadIdx.x, beta, k);
    const acc_t<R> t = acc_warp_total(v);
    if (lane_w == 0) d.part_c[(size_t)w * kWarpsPerEntry + wp] = t;
  }
}

// Per sheet: pAp, alpha = rz / pAp; p.Ap <= 0 or non-finite ends the sheet's solve.
template <class R>
__global__ void k_cg_scalar_alpha(Dev<R> d, int phase, cudaGraphConditionalHandle cond, int use_cond) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= d.S || d.cg[s].done) return;  // uniform over the warp
  const acc_t<R> pAp = sheet_sum(d, d.part_c, s);
  if ((threadIdx.x & 31) != 0) return;
  if (cg_alpha_step<R>(d.cg[s], pAp)) finish_sheet(d, s, phase, cond, use_cond);
}

// dv += alpha p_k (FP64), r -= alpha Ap, z = D^{-1} r (stored); warp partials of r.z, r.r.
template <class R>
__global__ void __launch_bounds__(kThreads) k_cg_update(Dev<R> d) {
  const int lane_w = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < d.NW; w += gridDim.x) {
    const int s = d.work_sheet[w];
    if (d.cg[s].done) continue;
    const int k = d.cg[s].iters;
    acc_t<R> v0 = acc_zero<R>(), v1 = acc_zero<R>();
    if (threadIdx.x < d.work_rows[w])
      update_row(d, d.work_row0[w] + threadIdx.x, alpha_of<R>(d.cg[s]), k, v0, v1);
    const acc_t<R> t0 = acc_warp_total(v0), t1 = acc_warp_total(v1);
    if (lane_w == 0) {
      d.part_a[(size_t)w * kWarpsPerEntry + wp] = t0;
      d.part_b[(size_t)w * kWarpsPerEntry + wp] = t1;
    }
  }
}

// Per sheet: beta = rz_new / rz, iteration count, convergence |r| <= tol |b|, max_iter.
// Also counts the loop-body executions of this phase.
template <class R>
__global__ void k_cg_scalar_beta(Dev<R> d, int phase, cudaGraphConditionalHandle cond, int use_cond) {
  if (blockIdx.x == 0 && threadIdx.x == 0) d.body_runs[phase] += 1ull;
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= d.S || d.cg[s].done) return;
  const acc_t<R> rz = sheet_sum(d, d.part_a, s), rr = sheet_sum(d, d.part_b, s);
  if ((threadIdx.x & 31) != 0) return;
  if (cg_beta_step<R>(d.cg[s], rz, rr, d.maxit)) finish_sheet(d, s, phase, cond, use_cond);
}

// ------------------------------------------------------------------ per-sheet cluster solver
// Each sheet is solved to the end by one thread-block cluster of CL CTAs (CL = 1, 2, 4 or 8,
// by the sheet's size) holding EPC work entries (256 rows each) per CTA, one row per
// thread.  The row's CG state (r, z, its own direction, the solution) and its column
// indices stay in registers for the whole solve, so an iteration reads from memory only
// the matrix row and the neighbours' z and p_{k-1} (L2-resident while the sheet runs).
// The per-warp partial sums go through shared memory (distributed shared memory across
// the cluster) and the two reductions of an iteration are separated by CTA or cluster
// barriers (hardware barriers, release/acquire at cluster scope).  Sheets are independent,
// so a launch may hold more clusters than fit on the GPU at once: they run as others end.
// Every CTA forms alpha, beta and the stopping test from the same partial sums in the same
// order, so all take the same branches.  The arithmetic and the summation orders are those
// of the device loop above, so the results are bitwise the same.
// Launch order of the per-sheet solver's clusters.  The hardware starts a launch's clusters
// roughly in index order, and a solve ends with its slowest sheet, so each size class's
// sheets are put in order of the iterations their last finished solve took, most first
// (ties keep the class's own order): the sheets that run longest start first.  A rank sort
// in one CTA per class (seg: the classes' offsets into the lists, then the total); a class
// of more than kOrderMax sheets keeps its own order.  The order changes no sheet's
// arithmetic, only when its cluster runs.
constexpr int kOrderMax = 2048;
template <class R>
__global__ void k_order_lists(Dev<R> d, const int* __restrict__ seg, const int* __restrict__ base,
                              int* __restrict__ order) {
  __shared__ unsigned key[kOrderMax];
  const int c0 = seg[blockIdx.x], n = seg[blockIdx.x + 1] - c0;
  const int* b = base + c0;
  int* o = order + c0;
  if (n > kOrderMax) {
    for (int q = threadIdx.x; q < n; q += blockDim.x) o[q] = b[q];
    return;
  }
  for (int q = threadIdx.x; q < n; q += blockDim.x) key[q] = d.last_iters[b[q]];
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const unsigned kq = key[q];
    int rank = 0;
    for (int u = 0; u < n; ++u) rank += (key[u] > kq || (key[u] == kq && u < q)) ? 1 : 0;
    o[rank] = b[q];
  }
}

constexpr int kColCache = 16;  // column indices kept in registers per row (further slots are loaded)
constexpr int kSmemCols = 12;  // off-diagonal column indices per row kept in shared memory, classes without
                               // the register cache (a grid sheet's interior rows have 12: 6 edge and
                               // 6 hinge neighbours)
constexpr int kSmemColsWide = 8;  // the same for four entries per CTA (static shared memory stays < 48 KB)
constexpr int kColSmemCarveout = 50;  // percent of the SM's shared storage given to shared memory there

// CG solution of one row in registers: FP64, or float-float in FP32 mode
template <class R> struct DvReg {
  V3<double> x;
  __device__ __forceinline__ void load(const Dev<R>& d, int i) { x = ld3(d.dv, i); }
  __device__ __forceinline__ void axpy(double al, V3<R> p) {
    x = {fma_rn(al, (double)p.x, x.x), fma_rn(al, (double)p.y, x.y), fma_rn(al, (double)p.z, x.z)};
  }
  __device__ __forceinline__ void store(const Dev<R>& d, int i) const { st3(d.dv, i, x); }
};
template <> struct DvReg<float> {
  FF a, b, c;
  __device__ __forceinline__ void load(const Dev<float>& d, int i) {
    const V3<float> h = ld3(d.dvh, i), l = ld3(d.dvl, i);
    a = {h.x, l.x};
    b = {h.y, l.y};
    c = {h.z, l.z};
  }
  __device__ __forceinline__ void axpy(FF al, V3<float> p) {
    a = ff_add(a, ff_mul(al, p.x));
    b = ff_add(b, ff_mul(al, p.y));
    c = ff_add(c, ff_mul(al, p.z));
  }
  __device__ __forceinline__ void store(const Dev<float>& d, int i) const {
    st3(d.dvh, i, V3<float>{a.hi, b.hi, c.hi});
    st3(d.dvl, i, V3<float>{a.lo, b.lo, c.lo});
  }
};

// The matrix, its column indices and the block-Jacobi inverse do not change during a
// solve and are read through the read-only (L1) path; the gather records written by other
// CTAs in the previous phase are read through L2 (ld_rec_l2).

// MINB: CTAs per SM the register budget is sized for (2 for the dense classes of two
// entries per CTA, which put two sheets' CTAs on each SM so that one sheet's barrier waits
// overlap another's work).
template <class R, int EPC, int MINB = (EPC == 1 ? 2 : 1)>
__global__ void __launch_bounds__(kThreads * EPC, MINB) k_cg_sheet(Dev<R> d, const int* __restrict__ sheets, int nsheets,
                                                                   int CL, int phase) {
  namespace cgrp = cooperative_groups;
  // column indices kept in registers per row: only where the launch leaves 128 registers
  // per thread (fewer than 768 threads per SM); the others (the dense classes, three or
  // more entries per CTA) keep the first SC off-diagonal indices of each row in shared
  // memory, so that a gather waits on one L2 access (the neighbour's record) rather than two
  constexpr int CC = EPC * MINB >= 3 ? 0 : kColCache;
  constexpr int SC = CC > 0 ? 0 : EPC >= 4 ? kSmemColsWide : kSmemCols;
  const int cid = blockIdx.x / CL;
  const int rank = blockIdx.x - cid * CL;  // = the CTA's rank in its (1-D) cluster
  if (cid >= nsheets) return;               // uniform over the cluster
  const int s = sheets[cid];
  if (d.cg[s].done) return;  // uniform: written only at the end of this sheet's solve

  // partial sums of the CTA's warps: [0] p.Ap, [1] r.z, [2] r.r, per local entry and warp
  __shared__ acc_t<R> sp[3][EPC][kWarpsPerEntry];
  __shared__ acc_t<R> bc_alpha;
  __shared__ R bc_beta;
  __shared__ int bc_stop;
  __shared__ int scol[SC > 0 ? SC : 1][kThreads * EPC];  // [slot - 1][thread]
  // the dense classes also keep each row's block-Jacobi inverse in shared memory (the
  // update phase then makes no global load; FP32 only: in FP64 the static shared memory
  // would pass 48 KB)
  constexpr bool SD = EPC * MINB >= 4 && EPC <= 2 && sizeof(R) == 4;
  __shared__ R sdinv[SD ? 9 : 1][SD ? kThreads * EPC : 1];

  const int jl = threadIdx.x / kThreads, t = threadIdx.x - jl * kThreads;
  const int lane = threadIdx.x & 31, wp = t >> 5;
  const int w0 = d.sheet_wfirst[s], w1 = d.sheet_wfirst[s + 1];
  const int w = w0 + rank + CL * jl;
  const bool on = w < w1 && t < d.work_rows[w];
  const int i = on ? d.work_row0[w] + t : 0;

  auto barrier = [&]() {
    if (CL > 1) cgrp::this_cluster().sync();
    else __syncthreads();
  };
  // the sheet's sum of one partial array, in the order of sheet_sum (lane-strided, then a
  // shuffle tree); called by one full warp
  // The sheet's sums of one or two partial arrays, each in the order of sheet_sum
  // (lane-strided, then a shuffle tree); the partials are loaded four at a time before they
  // are added, so the (distributed) shared memory loads overlap.  Called by one full warp.
  auto sheet_totals = [&](int wa, int wb, acc_t<R>* ta, acc_t<R>* tb) {
    const int q0 = w0 * kWarpsPerEntry, q1 = w1 * kWarpsPerEntry;
    acc_t<R> a = acc_zero<R>(), b = acc_zero<R>();
    for (int qb = q0 + lane; qb < q1; qb += 128) {
      acc_t<R> va[4], vb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = qb + 32 * u;
        va[u] = acc_zero<R>();
        vb[u] = acc_zero<R>();
        if (q < q1) {
          const int e = q / kWarpsPerEntry - w0, pw = q % kWarpsPerEntry;
          const int rk = e % CL, jj = e / CL;
          const acc_t<R>* sa = &sp[wa][jj][pw];
          const acc_t<R>* sb = &sp[wb][jj][pw];
          if (CL > 1) {
            sa = cgrp::this_cluster().map_shared_rank(sa, rk);
            sb = cgrp::this_cluster().map_shared_rank(sb, rk);
          }
          va[u] = *sa;
          if (tb) vb[u] = *sb;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (qb + 32 * u < q1) {
          a = acc_add(a, va[u]);
          b = acc_add(b, vb[u]);
        }
    }
    *ta = acc_warp_total(a);
    if (tb) *tb = acc_warp_total(b);
  };

  // row state
  int k = d.cg[s].iters;
  R beta_r = beta_of<R>(d.cg[s]);
  V3<R> r = {R(0), R(0), R(0)}, z = r, pold = r, Ap = r;
  DvReg<R> x;
  int K = 0, base = 0, col[CC > 0 ? CC : 1];
  const int sl_lane = i & 31;
  if (on) {
    r = ld3(d.r, i);
    const Rec<R> own = ld_rec_l2(rec(d, k, i));
    z = own.z;
    pold = own.p;
    x.load(d, i);
    const int sl = i >> 5;
    K = d.slice_K[sl];
    base = d.slice_base[sl];
  }
#pragma unroll
  for (int q = 0; q < CC; ++q) col[q] = (on && q + 1 < K) ? d.cols[(base + q + 1) * 32 + sl_lane] : 0;
  // each thread reads back only its own row's entries: no barrier needed
#pragma unroll
  for (int q = 0; q < SC; ++q)
    if (on && q + 1 < K) scol[q][threadIdx.x] = __ldg(d.cols + (base + q + 1) * 32 + sl_lane);
  if (SD && on) {
#pragma unroll
    for (int m = 0; m < 9; ++m) sdinv[m][SD ? threadIdx.x : 0] = __ldg(d.dinv + (size_t)m * d.Np + i);
  }
  // the sheet's scalars, advanced by thread 0 with the loop's scalar steps (in shared memory:
  // a register copy in every thread would cost ~26 registers per thread)
  __shared__ CGSheet c;
  if (threadIdx.x == 0) c = d.cg[s];

  while (true) {
    // ---- Ap = A p_k, p_k = z_k + beta_k p_{k-1} formed on the fly (own row and neighbours)
    acc_t<R> vpart = acc_zero<R>();
    V3<R> pi = {R(0), R(0), R(0)};
    if (on) {
      pi = next_dir(z, beta_r, pold);
      st_rec_p(rec(d, k + 1, i), pi);  // read by the neighbours as p_k in the next iteration
      const R* a0 = d.Aval + (size_t)base * 32 * 9 + sl_lane;
      R ab[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) ab[m] = __ldg(a0 + 32 * m);
      V3<R> y = block_mul(ab, pi);
#pragma unroll
      for (int q = 1; q <= CC; ++q) {
        if (q < K) {
          const int j = col[q - 1];
          const R* a = d.Aval + (size_t)(base + q) * 32 * 9 + sl_lane;
          R av[9];
#pragma unroll
          for (int m = 0; m < 9; ++m) av[m] = __ldg(a + 32 * m);
          const Rec<R> nj = ld_rec_l2(rec(d, k, j));
          const V3<R> pj = next_dir(nj.z, beta_r, nj.p);
          block_acc(y, av, V3<R>{pj.x - pi.x, pj.y - pi.y, pj.z - pi.z});
        }
      }
      // two slots per trip: both slots' blocks and neighbour records are requested before
      // either is used, so two L2 round trips overlap (accumulation order unchanged)
      auto col_of = [&](int q) {
        return q <= SC ? scol[q - 1][threadIdx.x] : __ldg(d.cols + (base + q) * 32 + sl_lane);
      };
      int q = CC + 1;
      for (; q + 1 < K; q += 2) {
        const int j0 = col_of(q), j1 = col_of(q + 1);
        const R* a = d.Aval + (size_t)(base + q) * 32 * 9 + sl_lane;
        R av[9], bv[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) {
          av[m] = __ldg(a + 32 * m);
          bv[m] = __ldg(a + 32 * 9 + 32 * m);
        }
        const Rec<R> n0 = ld_rec_l2(rec(d, k, j0)), n1 = ld_rec_l2(rec(d, k, j1));
        const V3<R> p0 = next_dir(n0.z, beta_r, n0.p), p1 = next_dir(n1.z, beta_r, n1.p);
        block_acc(y, av, V3<R>{p0.x - pi.x, p0.y - pi.y, p0.z - pi.z});
        block_acc(y, bv, V3<R>{p1.x - pi.x, p1.y - pi.y, p1.z - pi.z});
      }
      if (q < K) {
        const int j = col_of(q);
        const R* a = d.Aval + (size_t)(base + q) * 32 * 9 + sl_lane;
        R av[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) av[m] = __ldg(a + 32 * m);
        const Rec<R> nj = ld_rec_l2(rec(d, k, j));
        const V3<R> pj = next_dir(nj.z, beta_r, nj.p);
        block_acc(y, av, V3<R>{pj.x - pi.x, pj.y - pi.y, pj.z - pi.z});
      }
      Ap = y;
      vpart = acc_dot3(pi, y);
    }
    {
      const acc_t<R> tw = acc_warp_total(vpart);
      if (lane == 0) sp[0][jl][wp] = tw;
    }
    barrier();
    if (threadIdx.x < 32) {
      acc_t<R> tsum;
      sheet_totals(0, 0, &tsum, nullptr);
      if (threadIdx.x == 0) {
        bc_stop = cg_alpha_step<R>(c, tsum);
        bc_alpha = alpha_of<R>(c);
      }
    }
    __syncthreads();
    if (bc_stop) break;
    // ---- dv += alpha p_k, r -= alpha Ap, z = D^{-1} r
    acc_t<R> va = acc_zero<R>(), vb = acc_zero<R>();
    if (on) {
      const acc_t<R> alpha = bc_alpha;
      x.axpy(alpha, pi);
      const R am = -alpha_cast(alpha);
      r = {fma_rn(am, Ap.x, r.x), fma_rn(am, Ap.y, r.y), fma_rn(am, Ap.z, r.z)};
      {
        R dm[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) dm[m] = SD ? sdinv[m][SD ? threadIdx.x : 0] : __ldg(d.dinv + (size_t)m * d.Np + i);
        z = block_mul(dm, r);  // = apply_dinv
      }
      st_rec_z(rec(d, k + 1, i), z);  // gathered by the neighbours in the next iteration
      va = acc_dot3(r, z);
      vb = acc_dot3(r, r);
      pold = pi;
    }
    {
      const acc_t<R> ta = acc_warp_total(va), tb = acc_warp_total(vb);
      if (lane == 0) {
        sp[1][jl][wp] = ta;
        sp[2][jl][wp] = tb;
      }
    }
    barrier();
    k += 1;
    if (threadIdx.x < 32) {
      acc_t<R> a, b;
      sheet_totals(1, 2, &a, &b);
      if (threadIdx.x == 0) {
        bc_stop = cg_beta_step<R>(c, a, b, d.maxit);
        bc_beta = beta_of<R>(c);
      }
    }
    __syncthreads();
    if (bc_stop) break;
    beta_r = bc_beta;
  }
  if (on) {
    x.store(d, i);
    st3(d.r, i, r);
    st3(d.Ap, i, Ap);
  }
  // no CTA leaves while another may still read its shared memory
  if (CL > 1) cgrp::this_cluster().sync();
  if (rank == 0 && threadIdx.x == 0) {
    d.cg[s] = c;
    finish_sheet(d, s, phase, 0, 0);
  }
}

// ------------------------------------------------------------------ on-chip per-sheet cluster solver
// The same per-sheet solve as k_cg_sheet, with the sheet's data on chip: the sheet's SELL
// slices are split into contiguous ranges, one per CTA of a thread-block cluster (up to 16
// CTAs, one row per thread), and each CTA copies its rows' matrix values into shared
// memory once per solve.  The vectors the SpMV gathers (z and the previous direction) live
// in the owning CTA's shared memory and are read by the neighbours through distributed
// shared memory, so an iteration touches neither L2 nor HBM.  Row arithmetic, per-warp
// partial sums and the sheet-wide summation order are those of the device loop (one warp
// per 32-row slice, the sheet's slice partials summed lane-strided then by a shuffle tree),
// so results are bitwise the same.
constexpr int kSmMaxRanks = 16;    // CTAs per cluster (non-portable cluster size)
constexpr int kSmMaxThreads = 512;  // rows per CTA (keeps 128 registers per thread)
constexpr int kSmSlots = 16;       // blocks per row the kernel keeps column addresses for
constexpr int kSmMaxSlices = kSmMaxRanks * (kSmMaxThreads / 32);
constexpr size_t kSmDynMax = 227 * 1024 - 1024;   // dynamic shared memory per CTA (the static part aside)
constexpr size_t kSmBudget = kSmDynMax - 3072;      // what a partition may plan per CTA (slack for a class's
                                                    // largest CTA against its largest row count)

// Partition of one sheet: rank g holds the slices [sl0[g], sl0[g + 1]) (absolute slice ids).
struct SmSheet {
  int sheet;
  int sl0[kSmMaxRanks + 1];
};

template <class R>
__global__ void __launch_bounds__(kSmMaxThreads, 1) k_cg_sheet_sm(Dev<R> d, const SmSheet* __restrict__ list, int CL,
                                                                  int phase) {
  namespace cgrp = cooperative_groups;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int sl0s[kSmMaxRanks + 1];
  __shared__ unsigned char srank[kSmMaxSlices];
  __shared__ acc_t<R> bc_alpha;
  __shared__ R bc_beta;
  __shared__ int bc_stop;

  const int cid = blockIdx.x / CL;
  const int rank = blockIdx.x - cid * CL;  // = the CTA's rank in its (1-D) cluster
  const int s = list[cid].sheet;
  if (d.cg[s].done) return;  // uniform over the cluster: written only at the end of this sheet's solve

  constexpr int PS = PStride<R>::v;
  const int MR = blockDim.x;
  R* zs = reinterpret_cast<R*>(sm_raw);  // [MR][PS] z of this CTA's rows
  R* pb = zs + (size_t)PS * MR;          // [2][MR][PS] directions p_k, p_{k-1} (by parity of k)
  acc_t<R>* part = reinterpret_cast<acc_t<R>*>(pb + 2 * (size_t)PS * MR);  // [3][32] warp partials
  R* vals = reinterpret_cast<R*>(part + 3 * 32);                          // this CTA's matrix values

  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  if (t <= CL) sl0s[t] = list[cid].sl0[t];
  __syncthreads();
  const int sl_first = sl0s[0], nsl = sl0s[CL] - sl0s[0];
  for (int q = t; q < nsl; q += MR) {
    int g = 0;
    while (sl0s[g + 1] <= sl_first + q) ++g;
    srank[q] = (unsigned char)g;
  }
  const int sl0 = sl0s[rank], sl1 = sl0s[rank + 1];
  const int nrows = (sl1 - sl0) * 32;
  const bool on = t < nrows;
  const int i = sl0 * 32 + t;
  // this CTA's matrix values: one contiguous range of the SELL value array, 16-byte aligned
  {
    const int lb0 = d.slice_base[sl0];
    const size_t n16 = ((size_t)(d.slice_base[sl1] - lb0) * 32 * 9 * sizeof(R)) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(d.Aval + (size_t)lb0 * 32 * 9);
    uint4* dst = reinterpret_cast<uint4*>(vals);
    for (size_t q = t; q < n16; q += MR) dst[q] = __ldg(src + q);
  }
  // row state
  int k = d.cg[s].iters;
  R beta_r = beta_of<R>(d.cg[s]);
  V3<R> r = {R(0), R(0), R(0)}, z = r, pold = r, Ap = r;
  DvReg<R> x;
  R dm[9];
  int K = 0, lb = 0, col[kSmSlots - 1];
  if (on) {
    r = ld3(d.r, i);
    const Rec<R> own = ld_rec_l2(rec(d, k, i));
    z = own.z;
    pold = own.p;
    x.load(d, i);
    const int sl = i >> 5;
    K = d.slice_K[sl];
    lb = d.slice_base[sl] - d.slice_base[sl0];
#pragma unroll
    for (int m = 0; m < 9; ++m) dm[m] = d.dinv[(size_t)m * d.Np + i];
    // column j -> (rank of its CTA) << 16 | row within that CTA
#pragma unroll
    for (int q = 1; q < kSmSlots; ++q) {
      int a = 0;
      if (q < K) {
        const int j = d.cols[(size_t)(d.slice_base[sl] + q) * 32 + lane];
        int g = 0;
        while (sl0s[g + 1] * 32 <= j) ++g;
        a = (g << 16) | (j - sl0s[g] * 32);
      }
      col[q - 1] = a;
    }
    stp(zs, t, z);
    stp(pb + (size_t)PS * MR * ((k + 1) & 1), t, pold);
  } else {
#pragma unroll
    for (int m = 0; m < 9; ++m) dm[m] = R(0);
#pragma unroll
    for (int q = 0; q < kSmSlots - 1; ++q) col[q] = 0;
  }
  const int ne8 = (d.sheet_wfirst[s + 1] - d.sheet_wfirst[s]) * kWarpsPerEntry;

  auto barrier = [&]() {
    if (CL > 1) cgrp::this_cluster().sync();
    else __syncthreads();
  };
  auto remote = [&](const R* p, int g) -> const R* {
    return CL > 1 ? cgrp::this_cluster().map_shared_rank(const_cast<R*>(p), g) : p;
  };
  // the sheet's sum of one partial array in the order of sheet_sum (called by one warp)
  // (two totals at once; every partial loaded before the first add, as in k_cg_sheet)
  constexpr int kPerLane = kSmMaxSlices / 32;
  auto sheet_totals = [&](int wa, int wb, acc_t<R>* ta, acc_t<R>* tb) {
    acc_t<R> va[kPerLane], vb[kPerLane];
#pragma unroll
    for (int u = 0; u < kPerLane; ++u) {
      const int q = lane + 32 * u;
      va[u] = acc_zero<R>();
      vb[u] = acc_zero<R>();
      if (q < nsl) {
        const int g = srank[q];
        const acc_t<R>* sa = part + wa * 32 + (sl_first + q - sl0s[g]);
        const acc_t<R>* sb = part + wb * 32 + (sl_first + q - sl0s[g]);
        if (CL > 1) {
          sa = cgrp::this_cluster().map_shared_rank(const_cast<acc_t<R>*>(sa), g);
          sb = cgrp::this_cluster().map_shared_rank(const_cast<acc_t<R>*>(sb), g);
        }
        va[u] = *sa;
        if (tb) vb[u] = *sb;
      }
    }
    acc_t<R> a = acc_zero<R>(), b = acc_zero<R>();
#pragma unroll
    for (int u = 0; u < kPerLane; ++u)
      if (lane + 32 * u < ne8) {
        a = acc_add(a, va[u]);
        b = acc_add(b, vb[u]);
      }
    *ta = acc_warp_total(a);
    if (tb) *tb = acc_warp_total(b);
  };

  __shared__ CGSheet c;  // advanced by thread 0 (see k_cg_sheet)
  if (t == 0) c = d.cg[s];
  barrier();  // every CTA's vectors are in place before the first gather
  while (true) {
    // ---- Ap = A p_k, p_k = z_k + beta_k p_{k-1} formed on the fly (own row and neighbours)
    acc_t<R> vpart = acc_zero<R>();
    V3<R> pi = {R(0), R(0), R(0)};
    if (on) {
      const R* pprev = pb + (size_t)PS * MR * ((k + 1) & 1);
      pi = next_dir(z, beta_r, pold);
      stp(pb + (size_t)PS * MR * (k & 1), t, pi);  // read by the neighbours as p_{k} next iteration
      const R* a0 = vals + (size_t)lb * 288 + lane;
      R ab[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) ab[m] = a0[32 * m];
      V3<R> y = block_mul(ab, pi);
#pragma unroll
      for (int q = 1; q < kSmSlots; ++q) {
        if (q < K) {
          const int g = col[q - 1] >> 16, l = col[q - 1] & 0xffff;
          const R* a = a0 + (size_t)q * 288;
          R av[9];
#pragma unroll
          for (int m = 0; m < 9; ++m) av[m] = a[32 * m];
          const V3<R> pj = next_dir(ldp(remote(zs, g), l), beta_r, ldp(remote(pprev, g), l));
          block_acc(y, av, V3<R>{pj.x - pi.x, pj.y - pi.y, pj.z - pi.z});
        }
      }
      Ap = y;
      vpart = acc_dot3(pi, y);
    }
    {
      const acc_t<R> tw = acc_warp_total(vpart);
      if (lane == 0) part[wp] = tw;
    }
    barrier();
    if (t < 32) {
      acc_t<R> tsum;
      sheet_totals(0, 0, &tsum, nullptr);
      if (t == 0) {
        bc_stop = cg_alpha_step<R>(c, tsum);
        bc_alpha = alpha_of<R>(c);
      }
    }
    __syncthreads();
    if (bc_stop) break;
    // ---- dv += alpha p_k, r -= alpha Ap, z = D^{-1} r
    acc_t<R> va = acc_zero<R>(), vb = acc_zero<R>();
    if (on) {
      const acc_t<R> alpha = bc_alpha;
      x.axpy(alpha, pi);
      const R am = -alpha_cast(alpha);
      r = {fma_rn(am, Ap.x, r.x), fma_rn(am, Ap.y, r.y), fma_rn(am, Ap.z, r.z)};
      z = block_mul(dm, r);  // = apply_dinv
      stp(zs, t, z);         // gathered by the neighbours in the next iteration
      va = acc_dot3(r, z);
      vb = acc_dot3(r, r);
      pold = pi;
    }
    {
      const acc_t<R> ta = acc_warp_total(va), tb = acc_warp_total(vb);
      if (lane == 0) {
        part[32 + wp] = ta;
        part[64 + wp] = tb;
      }
    }
    barrier();
    k += 1;
    if (t < 32) {
      acc_t<R> a, b;
      sheet_totals(1, 2, &a, &b);
      if (t == 0) {
        bc_stop = cg_beta_step<R>(c, a, b, d.maxit);
        bc_beta = beta_of<R>(c);
      }
    }
    __syncthreads();
    if (bc_stop) break;
    beta_r = bc_beta;
  }
  if (on) {
    x.store(d, i);
    st3(d.r, i, r);
    st3(d.Ap, i, Ap);
  }
  // no CTA leaves while another may still read its shared memory
  barrier();
  if (rank == 0 && t == 0) {
    d.cg[s] = c;
    finish_sheet(d, s, phase, 0, 0);
  }
}

// Velocity increments: out = v + F_t on free vertices (F_t in the user layout), v elsewhere.
template <class R>
__global__ void k_add_increment(Dev<R> d, const double* __restrict__ v, const R* __restrict__ F,
                                double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  V3<double> w = ld3(v, i);
  const int u = d.i2u[i];
  if (u >= 0 && !d.pinned[i]) {
    const V3<R> f = ld3(F, u);
    w = {w.x + (double)f.x, w.y + (double)f.y, w.z + (double)f.z};
  }
  st3(out, i, w);
}

// v' = v + dv, x' = x + h v'; optional user-layout copy of x'.
template <class R>
__global__ void k_state_update(Dev<R> d, const double* __restrict__ x, const double* __restrict__ v,
                               double* __restrict__ xn, double* __restrict__ vn, R* __restrict__ traj_row) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const V3<double> dv = ld3(d.dv, i);
  const V3<double> v0 = ld3(v, i), x0 = ld3(x, i);
  const V3<double> v1 = {v0.x + dv.x, v0.y + dv.y, v0.z + dv.z};
  const double h = (double)d.h;
  const V3<double> x1 = {x0.x + h * v1.x, x0.y + h * v1.y, x0.z + h * v1.z};
  st3(vn, i, v1);
  st3(xn, i, x1);
  const int u = d.i2u[i];
  if (traj_row && u >= 0) st3(traj_row, u, V3<R>{(R)x1.x, (R)x1.y, (R)x1.z});
}

// A pinned vertex keeps its starting velocity (dv = 0): flag a sheet whose pinned vertices
// do not start at rest (their pins would drift), including non-finite values.
template <class R>
__global__ void k_check_pins(Dev<R> d, const double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np || !d.pinned[i]) return;
  const V3<double> w = ld3(v, i);
  if (!(w.x == 0.0 && w.y == 0.0 && w.z == 0.0))
    atomicOr(&d.cg[d.vsheet[i]].status, (int)CLOTH_STATUS_PINNED_VELOCITY_NONZERO);
}

template <class R>
__global__ void k_reset_status(Dev<R> d, int phase) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < d.S) {
    d.cg[s].status = 0;
    d.sheet_iters[2 * ((size_t)phase * d.S + s)] = 0;
    d.sheet_iters[2 * ((size_t)phase * d.S + s) + 1] = 0;
  }
  if (s == 0) {
    d.iter_total[phase] = 0;
    d.body_runs[phase] = 0;
  }
}

// Re-open every sheet's CG (kernel timing on the last assembled system).
template <class R>
__global__ void k_reopen(Dev<R> d) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < d.S) d.cg[s].done = 0;
}

template <class R>
__global__ void k_status_out(Dev<R> d, int32_t* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < d.S) status[s] = d.cg[s].status;
}

// ------------------------------------------------------------------ adjoint kernels
// mode 0: adjoint step contributions; mode 1: third-derivative contraction only.
template <class R>
__global__ void __launch_bounds__(kElemThreads) k_adj_tri(Dev<R> d, const double* __restrict__ x,
                                                         const double* __restrict__ lam,
                                                         const double* __restrict__ u, int mode) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.M) return;
  TriConst<R> k = tri_const(d, t);
  V3<R> xe[3], le[3], ue[3], f[3], Hx[3], Hl[3], Hu[3], th[3];
  int idx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) idx[a] = d.tri_v[(size_t)a * d.M + t];
  load_relative<R, 3>(x, idx, xe);
  load_relative<R, 3>(lam, idx, le);
  load_relative<R, 3>(u, idx, ue);
  membrane_adjoint(k, xe, green_strain(d, t, x, idx), le, ue, d.clamp, f, Hx, Hl, Hu, th);
  const R h = d.h, h2 = d.h * d.h;
  R* ro = d.tri_r + 18 * (size_t)t;
  double sc = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (mode == 0) {
      ro[6 * a + 0] = -h * Hx[a].x - h2 * th[a].x;
      ro[6 * a + 1] = -h * Hx[a].y - h2 * th[a].y;
      ro[6 * a + 2] = -h * Hx[a].z - h2 * th[a].z;
      ro[6 * a + 3] = -h2 * Hl[a].x;
      ro[6 * a + 4] = -h2 * Hl[a].y;
      ro[6 * a + 5] = -h2 * Hl[a].z;
      sc += (double)le[a].x * (double)(h * f[a].x - h2 * Hu[a].x) + (double)le[a].y * (double)(h * f[a].y - h2 * Hu[a].y) +
            (double)le[a].z * (double)(h * f[a].z - h2 * Hu[a].z);
    } else {
      ro[6 * a + 0] = th[a].x;
      ro[6 * a + 1] = th[a].y;
      ro[6 * a + 2] = th[a].z;
      ro[6 * a + 3] = R(0);
      ro[6 * a + 4] = R(0);
      ro[6 * a + 5] = R(0);
    }
  }
  const int s = d.tri_sheet[t];
  d.tri_sc[t] = sc / (double)d.material[4 * s];
}

template <class R>
__global__ void __launch_bounds__(kElemThreads) k_adj_hinge(Dev<R> d, const double* __restrict__ x,
                                                           const double* __restrict__ lam,
                                                           const double* __restrict__ u, int mode) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  HingeConst<R> k = hinge_const(d, e);
  V3<R> xe[4], le[4], ue[4], f[4], Hl[4], Hu[4], th[4];
  int idx[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) idx[a] = d.hin_v[(size_t)a * d.E + e];
  load_relative<R, 4>(x, idx, xe);
  load_relative<R, 4>(lam, idx, le);
  load_relative<R, 4>(u, idx, ue);
  bending_adjoint(k, xe, le, ue, f, Hl, Hu, th);
  const R h = d.h, h2 = d.h * d.h;
  R* ro = d.hin_r + 24 * (size_t)e;
  double sc = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (mode == 0) {
      ro[6 * a + 0] = -h * Hl[a].x - h2 * th[a].x;
      ro[6 * a + 1] = -h * Hl[a].y - h2 * th[a].y;
      ro[6 * a + 2] = -h * Hl[a].z - h2 * th[a].z;
      ro[6 * a + 3] = -h2 * Hl[a].x;
      ro[6 * a + 4] = -h2 * Hl[a].y;
      ro[6 * a + 5] = -h2 * Hl[a].z;
      sc += (double)le[a].x * (double)(h * f[a].x - h2 * Hu[a].x) + (double)le[a].y * (double)(h * f[a].y - h2 * Hu[a].y) +
            (double)le[a].z * (double)(h * f[a].z - h2 * Hu[a].z);
    } else {
      ro[6 * a + 0] = th[a].x;
      ro[6 * a + 1] = th[a].y;
      ro[6 * a + 2] = th[a].z;
      ro[6 * a + 3] = R(0);
      ro[6 * a + 4] = R(0);
      ro[6 * a + 5] = R(0);
    }
  }
  const int s = d.hin_sheet[e];
  d.hin_sc[e] = sc / (double)d.material[4 * s + 2];
}

template <class R>
__device__ __forceinline__ const R* adj_slot(const Dev<R>& d, int slot) {
  return slot < 3 * d.M ? d.tri_r + 6 * (size_t)slot : d.hin_r + 6 * (size_t)(slot - 3 * d.M);
}

// RHS of the adjoint solve: mask(v_bar + h x_bar)
template <class R>
__global__ void k_adj_rhs(Dev<R> d, const double* __restrict__ ax, const double* __restrict__ av) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  V3<R> g = {R(0), R(0), R(0)};
  if (!d.pinned[i]) {
    const V3<double> gd = axpy3((double)d.h, ld3(ax, i), ld3(av, i));
    g = {(R)gd.x, (R)gd.y, (R)gd.z};
  }
  st3(d.bvec, i, g);
}

// Per-vertex adjoint update after the element pass; lam = d.dv.
// v_t: the velocity the step started from; fmode 0: gF = h lam (F_t a force), 1: gF = the
// adjoint of the starting velocity on free vertices (F_t a velocity increment).
template <class R>
__global__ void k_adj_vertex(Dev<R> d, double* __restrict__ ax, double* __restrict__ av, const double* __restrict__ v_t,
                             const double* __restrict__ v_t1, const R* __restrict__ dLdx_row, R* __restrict__ gF_row,
                             int fmode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  // element contributions are large and cancel at a vertex: summed in FP64
  V3<double> r1 = {0.0, 0.0, 0.0}, r2 = {0.0, 0.0, 0.0};
  for (int q = d.vf_ptr[i]; q < d.vf_ptr[i + 1]; ++q) {
    const R* src = adj_slot(d, d.vf[q]);
    r1.x += (double)src[0];
    r1.y += (double)src[1];
    r1.z += (double)src[2];
    r2.x += (double)src[3];
    r2.y += (double)src[4];
    r2.z += (double)src[5];
  }
  const int u = d.i2u[i];
  const V3<double> a_x = ld3(ax, i), a_v = ld3(av, i), lam = ld3(d.dv, i);
  const V3<R> dl = (dLdx_row && u >= 0) ? ld3(dLdx_row, u) : V3<R>{R(0), R(0), R(0)};
  const double h = (double)d.h;
  st3(ax, i, V3<double>{a_x.x + (double)r1.x + (double)dl.x, a_x.y + (double)r1.y + (double)dl.y,
                        a_x.z + (double)r1.z + (double)dl.z});
  V3<double> nv = {a_v.x + h * a_x.x + (double)r2.x, a_v.y + h * a_x.y + (double)r2.y,
                   a_v.z + h * a_x.z + (double)r2.z};
  // air drag: b depends on w and on the starting velocity through f, A through G(d);
  // q = h rho_air A (G lam - dG[lam, dv]) goes to the wind gradient and leaves v_bar
  V3<double> qw = {0.0, 0.0, 0.0};
  if (d.air_density > 0.0 && !d.pinned[i]) {
    const V3<double> vs = ld3(v_t, i), vn1 = ld3(v_t1, i);
    const V3<double> r = relative_wind(d, d.vsheet[i], vs);
    const V3<double> dvi = {vn1.x - vs.x, vn1.y - vs.y, vn1.z - vs.z};
    const V3<double> gl = air_G(r, lam), tl = air_dG(r, lam, dvi);
    const double hc = h * d.air_density * (double)d.area3[i];
    qw = {hc * (gl.x - tl.x), hc * (gl.y - tl.y), hc * (gl.z - tl.z)};
    nv = {nv.x - qw.x, nv.y - qw.y, nv.z - qw.z};
  }
  if (d.row_w) st3(d.row_w, i, qw);
  st3(av, i, nv);
  if (gF_row && u >= 0) {
    if (fmode == 0) st3(gF_row, u, V3<R>{(R)(h * lam.x), (R)(h * lam.y), (R)(h * lam.z)});
    else st3(gF_row, u, d.pinned[i] ? V3<R>{R(0), R(0), R(0)} : V3<R>{(R)nv.x, (R)nv.y, (R)nv.z});
  }
  const V3<double> vt = ld3(v_t, i), vt1 = ld3(v_t1, i);
  const double m1 = (double)d.area3[i];
  d.row_sc[i] = m1 * ((double)lam.x * ((double)d.h * (double)d.gx - (vt1.x - vt.x)) +
                      (double)lam.y * ((double)d.h * (double)d.gy - (vt1.y - vt.y)) +
                      (double)lam.z * ((double)d.h * (double)d.gz - (vt1.z - vt.z)));
}

// Per-sheet accumulation of the material gradients (deterministic).
template <class R>
__global__ void __launch_bounds__(kThreads) k_param_acc(Dev<R> d) {
  const int s = blockIdx.x;
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = d.sheet_toff[s] + threadIdx.x; t < d.sheet_toff[s + 1]; t += kThreads) v[0] += d.tri_sc[t];
  for (int e = d.sheet_hoff[s] + threadIdx.x; e < d.sheet_hoff[s + 1]; e += kThreads) v[1] += d.hin_sc[e];
  for (int i = d.sheet_voff[s] + threadIdx.x; i < d.sheet_voff[s + 1]; i += kThreads) {
    v[2] += d.row_sc[i];
    if (d.air_density > 0.0) {
      v[3] += d.row_w[3 * (size_t)i];
      v[4] += d.row_w[3 * (size_t)i + 1];
      v[5] += d.row_w[3 * (size_t)i + 2];
    }
  }
  block_sum<6>(v);
  if (threadIdx.x == 0) {
    d.gacc[3 * s] += v[0];
    d.gacc[3 * s + 1] += v[1];
    d.gacc[3 * s + 2] += v[2];
    d.gacc_w[3 * s] += v[3];
    d.gacc_w[3 * s + 1] += v[4];
    d.gacc_w[3 * s + 2] += v[5];
  }
}

template <class R>
__global__ void k_grad_material(Dev<R> d, R* __restrict__ g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.S) return;
  g[4 * s] = (R)d.gacc[3 * s];
  g[4 * s + 1] = R(0);
  g[4 * s + 2] = (R)d.gacc[3 * s + 1];
  g[4 * s + 3] = (R)d.gacc[3 * s + 2];
}

template <class R>
__global__ void k_grad_wind(Dev<R> d, R* __restrict__ g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.S) return;
  for (int k = 0; k < 3; ++k) g[3 * s + k] = (R)d.gacc_w[3 * s + k];
}

// ------------------------------------------------------------------ test-only kernels
// per-vertex force of one kind (kind 0 membrane, 1 bending) in user layout
template <class R>
__global__ void k_vertex_force(Dev<R> d, int kind, R* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const int u = d.i2u[i];
  if (u < 0) return;
  V3<double> f = {0.0, 0.0, 0.0};
  for (int q = d.vf_ptr[i]; q < d.vf_ptr[i + 1]; ++q) {
    const int slot = d.vf[q];
    if ((slot < 3 * d.M) != (kind == 0)) continue;
    const double* src = force_slot(d, slot);
    f = add3(f, V3<double>{src[0], src[1], src[2]});
  }
  st3(out, u, V3<R>{(R)f.x, (R)f.y, (R)f.z});
}

template <class R>
__global__ void k_vertex_third(Dev<R> d, R* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const int u = d.i2u[i];
  if (u < 0) return;
  V3<R> f = {R(0), R(0), R(0)};
  for (int q = d.vf_ptr[i]; q < d.vf_ptr[i + 1]; ++q) {
    const R* src = adj_slot(d, d.vf[q]);
    f = add3(f, V3<R>{src[0], src[1], src[2]});
  }
  st3(out, u, f);
}

// Expand the SELL matrix of each sheet into a dense row-major block (user order).
template <class R>
__global__ void k_dense(Dev<R> d, const long long* __restrict__ dense_off, R* __restrict__ A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const int u = d.i2u[i];
  if (u < 0) return;
  const int s = d.vsheet[i];
  const int n = d.sheet_uoff[s + 1] - d.sheet_uoff[s];
  const int ul = u - d.sheet_uoff[s];
  const int sl = i >> 5, lane = i & 31;
  double diag[9];
  {
    const R* a0 = d.Aval + (size_t)d.slice_base[sl] * 32 * 9 + lane;
    for (int q = 0; q < 9; ++q) diag[q] = (double)a0[q * 32];
  }
  for (int k = 1; k < d.slice_K[sl]; ++k) {
    const int ent = (d.slice_base[sl] + k) * 32 + lane;
    const int j = d.cols[ent];
    const int uj = d.i2u[j];
    if (uj < 0 || j == i) continue;  // padding slot
    const int ujl = uj - d.sheet_uoff[s];
    const R* a = d.Aval + (size_t)(d.slice_base[sl] + k) * 32 * 9 + lane;
    for (int q = 0; q < 9; ++q) {
      diag[q] -= (double)a[q * 32];
      A[dense_off[s] + (size_t)(3 * ul + q / 3) * (3 * n) + 3 * ujl + q % 3] = a[q * 32];
    }
  }
  for (int q = 0; q < 9; ++q) A[dense_off[s] + (size_t)(3 * ul + q / 3) * (3 * n) + 3 * ul + q % 3] = (R)diag[q];
}

// y = A p outside CG (for the single-kernel entry point)
template <class R>
__global__ void k_spmv_plain(Dev<R> d, const R* __restrict__ p, R* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.Np) return;
  const int sl = i >> 5, lane = i & 31;
  const V3<R> pi = ld3(p, i);
  const R* a0 = d.Aval + (size_t)d.slice_base[sl] * 32 * 9 + lane;
  V3<R> acc = {a0[0] * pi.x + a0[32] * pi.y + a0[64] * pi.z, a0[96] * pi.x + a0[128] * pi.y + a0[160] * pi.z,
               a0[192] * pi.x + a0[224] * pi.y + a0[256] * pi.z};
  for (int k = 1; k < d.slice_K[sl]; ++k) {
    const int ent = (d.slice_base[sl] + k) * 32 + lane;
    const R* a = d.Aval + (size_t)(d.slice_base[sl] + k) * 32 * 9 + lane;
    const V3<R> pj = ld3(p, d.cols[ent]);
    const V3<R> dp = {pj.x - pi.x, pj.y - pi.y, pj.z - pi.z};
    acc.x += a[0] * dp.x + a[32] * dp.y + a[64] * dp.z;
    acc.y += a[96] * dp.x + a[128] * dp.y + a[160] * dp.z;
    acc.z += a[192] * dp.x + a[224] * dp.y + a[256] * dp.z;
  }
  st3(y, i, acc);
}

// ------------------------------------------------------------------ losses
template <class R>
__global__ void __launch_bounds__(kThreads) k_loss_l2(Dev<R> d, int T, const R* __restrict__ traj,
                                                      const R* __restrict__ tgt, R* __restrict__ grad,
                                                      double* __restrict__ lpart) {
  const int s = blockIdx.x, t = blockIdx.y + 1;
  const int u0 = d.sheet_uoff[s], u1 = d.sheet_uoff[s + 1];
  const size_t row = (size_t)t * d.Nu;
  double v[1] = {0.0};
  for (int u = u0 + threadIdx.x; u < u1; u += kThreads) {
    const V3<R> x = ld3(traj + 3 * row, u), y = ld3(tgt + 3 * row, u);
    const V3<R> df = {x.x - y.x, x.y - y.y, x.z - y.z};
    v[0] += ddot3(df, df);
    if (grad) st3(grad + 3 * row, u, V3<R>{R(2) * df.x, R(2) * df.y, R(2) * df.z});
  }
  block_sum<1>(v);
  if (threadIdx.x == 0) lpart[(size_t)s * T + (t - 1)] = v[0];
}

template <class R>
__global__ void __launch_bounds__(kThreads) k_loss_pinhole(Dev<R> d, int T, const R* __restrict__ traj,
                                                           const R* __restrict__ uv, double f, double cx, double cy,
                                                           double cz, R* __restrict__ grad,
                                                           double* __restrict__ lpart) {
  const int s = blockIdx.x, t = blockIdx.y + 1;
  const int u0 = d.sheet_uoff[s], u1 = d.sheet_uoff[s + 1];
  const size_t row = (size_t)t * d.Nu;
  double v[1] = {0.0};
  for (int u = u0 + threadIdx.x; u < u1; u += kThreads) {
    const V3<R> x = ld3(traj + 3 * row, u);
    const double Xc = (double)x.x - cx, Yc = -((double)x.y - cy), Zc = cz - (double)x.z;
    if (!(Zc > 0.0)) {
      v[0] += NAN;
      continue;
    }
    const double pu = f * Xc / Zc, pv = f * Yc / Zc;
    const double du = pu - (double)uv[2 * (row + u)], dw = pv - (double)uv[2 * (row + u) + 1];
    v[0] += du * du + dw * dw;
    if (grad)
      st3(grad + 3 * row, u,
          V3<R>{(R)(2.0 * du * f / Zc), (R)(-2.0 * dw * f / Zc), (R)(2.0 * (du * f * Xc + dw * f * Yc) / (Zc * Zc))});
  }
  block_sum<1>(v);
  if (threadIdx.x == 0) lpart[(size_t)s * T + (t - 1)] = v[0];
}

template <class R>
__global__ void k_loss_final(Dev<R> d, int T, const double* __restrict__ lpart, double* __restrict__ loss) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.S) return;
  double acc = 0.0;
  for (int t = 0; t < T; ++t) acc += lpart[(size_t)s * T + t];
  loss[s] = acc;
}

}  // namespace cloth
