// Element physics of the cloth step (device code), templated on the real type.
//
// Membrane (St. Venant-Kirchhoff on the Green strain, isotropic, plane stress):
//   F = sum_a x_a g_a^T (3x2), g_1 / g_2 = rows of Dm^{-1}, g_0 = -(g_1 + g_2)
//   G = (F^T F - I)/2, S = 2 mu G + lambda tr(G) I, E = A0 (mu |G|^2 + lambda/2 tr(G)^2)
//   dE/dx_a = A0 F S g_a
//   d2E/dx_a dx_b [c][d] = A0 ( delta_cd g_a.S g_b                       (geometric)
//                             + mu ((F F^T)_cd g_a.g_b + w_b[c] w_a[d])    (material)
//                             + lambda w_a[c] w_b[d] ),   w_a = F g_a
// The matrix of the implicit solve may use S+ = (S + (S^2 + eps^2 I)^{1/2})/2 in the
// geometric term (positive definite, smooth), which keeps A = M + h^2 H~ SPD when the
// cloth is compressed (phi-SfT leaves the material model open, Sec. 3.1).
//
// Bending (per interior edge, hinge x0-x1 with wings xa, xb):
//   n1 = e x (xa - x0), n2 = (xb - x0) x e, e = x1 - x0,
//   theta = atan2((n1 x n2).e/|e|, n1.n2),  E = 1/2 kb w (theta - theta0)^2
//   dtheta/dxa = -|e| n1/|n1|^2, dtheta/dxb = -|e| n2/|n2|^2,
//   dtheta/dx1 = -ta dtheta/dxa - tb dtheta/dxb,
//   dtheta/dx0 = -(1 - ta) dtheta/dxa - (1 - tb) dtheta/dxb,
//   ta = (xa - x0).e/|e|^2, tb = (xb - x0).e/|e|^2.
// Second and third derivatives of theta come from forward-mode dual numbers applied to
// this analytic gradient.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace cloth {

// ------------------------------------------------------------------ dual numbers
template <class T> struct Dual;
template <class T> struct Base { using type = T; };
template <class T> struct Base<Dual<T>> { using type = typename Base<T>::type; };

template <class T>
struct Dual {
  T v, d;
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
  // a constant (zero derivative at every nesting level)
  __host__ __device__ Dual(typename Base<T>::type a) : v(a), d(typename Base<T>::type(0)) {}
};

template <class T> __host__ __device__ inline Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __host__ __device__ inline Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __host__ __device__ inline Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __host__ __device__ inline Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <class T> __host__ __device__ inline Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T, class S> __host__ __device__ inline Dual<T> operator*(S s, Dual<T> a) { return {T(s) * a.v, T(s) * a.d}; }
template <class T, class S> __host__ __device__ inline Dual<T> operator*(Dual<T> a, S s) { return {a.v * T(s), a.d * T(s)}; }
template <class T, class S> __host__ __device__ inline Dual<T> operator+(Dual<T> a, S s) { return {a.v + T(s), a.d}; }
template <class T, class S> __host__ __device__ inline Dual<T> operator-(Dual<T> a, S s) { return {a.v - T(s), a.d}; }

__device__ inline float dsqrt(float a) { return sqrtf(a); }
__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline float datan2(float y, float x) { return atan2f(y, x); }
__device__ inline double datan2(double y, double x) { return atan2(y, x); }
template <class T> __device__ inline Dual<T> dsqrt(Dual<T> a) {
  T s = dsqrt(a.v);
  return {s, a.d / (s + s)};
}
template <class T> __device__ inline Dual<T> datan2(Dual<T> y, Dual<T> x) {
  T r2 = x.v * x.v + y.v * y.v;
  return {datan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2};
}

// nested constant construction
template <class T> struct ConstOf { __device__ static T make(typename Base<T>::type a) { return a; } };
template <class T> struct ConstOf<Dual<T>> {
  __device__ static Dual<T> make(typename Base<T>::type a) { return Dual<T>(ConstOf<T>::make(a), ConstOf<T>::make(0)); }
};
template <class T> __device__ inline T cst(typename Base<T>::type a) { return ConstOf<T>::make(a); }

// ------------------------------------------------------------------ small vectors
template <class T> struct V3 { T x, y, z; };
template <class T> __device__ inline V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> __device__ inline V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S> __device__ inline V3<T> scale(S s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> __device__ inline T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __device__ inline V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// --------------------------------------------------------------- membrane parts
// 2x2 symmetric matrices are kept as (m00, m11, m01).
template <class T> struct Sym2 { T a, b, c; };

// S+ = (S + (S^2 + eps^2 I)^{1/2}) / 2 with the closed-form 2x2 SPD square root
// sqrt(P) = (P + sqrt(det P) I) / sqrt(tr P + 2 sqrt(det P)).
template <class T, class R>
__device__ inline Sym2<T> smooth_positive(Sym2<T> S, R eps) {
  T p00 = S.a * S.a + S.c * S.c + eps * eps;
  T p11 = S.b * S.b + S.c * S.c + eps * eps;
  T p01 = S.c * (S.a + S.b);
  T sd = dsqrt(p00 * p11 - p01 * p01);
  T tn = dsqrt(p00 + p11 + sd + sd);
  T hr = cst<T>(0.5) / tn;
  return {cst<T>(0.5) * S.a + hr * (p00 + sd), cst<T>(0.5) * S.b + hr * (p11 + sd),
          cst<T>(0.5) * S.c + hr * p01};
}

template <class R>
struct TriConst {
  R g[3][2];  // shape-function gradients
  R A0, mu, lam, eps;
};

// F (3x2, row-major) from the three positions.
template <class T, class R>
__device__ inline void deformation_gradient(const TriConst<R>& k, const V3<T>* x, T F[3][2]) {
  for (int j = 0; j < 2; ++j) {
    F[0][j] = x[0].x * k.g[0][j] + x[1].x * k.g[1][j] + x[2].x * k.g[2][j];
    F[1][j] = x[0].y * k.g[0][j] + x[1].y * k.g[1][j] + x[2].y * k.g[2][j];
    F[2][j] = x[0].z * k.g[0][j] + x[1].z * k.g[1][j] + x[2].z * k.g[2][j];
  }
}

template <class T, class R>
__device__ inline Sym2<T> stvk_stress(const TriConst<R>& k, const T F[3][2]) {
  T c00 = F[0][0] * F[0][0] + F[1][0] * F[1][0] + F[2][0] * F[2][0];
  T c11 = F[0][1] * F[0][1] + F[1][1] * F[1][1] + F[2][1] * F[2][1];
  T c01 = F[0][0] * F[0][1] + F[1][0] * F[1][1] + F[2][0] * F[2][1];
  T g00 = cst<T>(0.5) * (c00 - cst<T>(1)), g11 = cst<T>(0.5) * (c11 - cst<T>(1)), g01 = cst<T>(0.5) * c01;
  T ltr = k.lam * (g00 + g11);
  return {R(2) * k.mu * g00 + ltr, R(2) * k.mu * g11 + ltr, R(2) * k.mu * g01};
}

// S = 2 mu G + lambda tr(G) I from a Green strain computed elsewhere
template <class R>
__device__ inline Sym2<R> stvk_stress_G(const TriConst<R>& k, Sym2<R> G) {
  const R ltr = k.lam * (G.a + G.b);
  return {R(2) * k.mu * G.a + ltr, R(2) * k.mu * G.b + ltr, R(2) * k.mu * G.c};
}

// C : X for symmetric X:  2 mu X + lambda tr(X) I
template <class T, class R>
__device__ inline Sym2<T> elastic_map(const TriConst<R>& k, Sym2<T> X) {
  T ltr = k.lam * (X.a + X.b);
  return {R(2) * k.mu * X.a + ltr, R(2) * k.mu * X.b + ltr, R(2) * k.mu * X.c};
}

// sym(F^T dF) for 3x2 F, dF
template <class T, class U>
__device__ inline Sym2<T> sym_FtdF(const T F[3][2], const U dF[3][2]) {
  T a = F[0][0] * dF[0][0] + F[1][0] * dF[1][0] + F[2][0] * dF[2][0];
  T b = F[0][1] * dF[0][1] + F[1][1] * dF[1][1] + F[2][1] * dF[2][1];
  T c01 = F[0][0] * dF[0][1] + F[1][0] * dF[1][1] + F[2][0] * dF[2][1];
  T c10 = F[0][1] * dF[0][0] + F[1][1] * dF[1][0] + F[2][1] * dF[2][0];
  return {a, b, cst<T>(0.5) * (c01 + c10)};
}

// (A S g) for 3x2 A, symmetric S, 2-vector g
template <class T, class R>
__device__ inline V3<T> mat32_sym_vec(const T A[3][2], Sym2<T> S, const R* g) {
  T s0 = S.a * g[0] + S.c * g[1];
  T s1 = S.c * g[0] + S.b * g[1];
  return {A[0][0] * s0 + A[0][1] * s1, A[1][0] * s0 + A[1][1] * s1, A[2][0] * s0 + A[2][1] * s1};
}

// Forces and upper Hessian blocks of one triangle.
// f[3]: -dE/dx_a.  H[6][9]: blocks (0,0),(0,1),(0,2),(1,1),(1,2),(2,2), row-major 3x3.
// G: the Green strain of the element (formed by the caller from edge metrics, so it
// keeps its relative precision when the strain is small); clamp: the geometric term
// uses S+ (eps = k.eps) instead of S.
template <class R>
__device__ inline void membrane_force_hessian(const TriConst<R>& k, const V3<R>* x, Sym2<R> G, bool clamp, V3<R>* f,
                                              R (*H)[9]) {
  R F[3][2];
  deformation_gradient(k, x, F);
  Sym2<R> S = stvk_stress_G(k, G);
  Sym2<R> Sg = clamp ? smooth_positive(S, k.eps) : S;
  V3<R> w[3];
  for (int a = 0; a < 3; ++a) {
    f[a] = scale(-k.A0, mat32_sym_vec(F, S, k.g[a]));
    w[a] = {F[0][0] * k.g[a][0] + F[0][1] * k.g[a][1], F[1][0] * k.g[a][0] + F[1][1] * k.g[a][1],
            F[2][0] * k.g[a][0] + F[2][1] * k.g[a][1]};
  }
  R FF[3][3];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) FF[c][d] = F[c][0] * F[d][0] + F[c][1] * F[d][1];
  int blk = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b, ++blk) {
      const R* ga = k.g[a];
      const R* gb = k.g[b];
      R geo = ga[0] * (Sg.a * gb[0] + Sg.c * gb[1]) + ga[1] * (Sg.c * gb[0] + Sg.b * gb[1]);
      R gg = ga[0] * gb[0] + ga[1] * gb[1];
      const R wa[3] = {w[a].x, w[a].y, w[a].z};
      const R wb[3] = {w[b].x, w[b].y, w[b].z};
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          R v = k.mu * (FF[c][d] * gg + wb[c] * wa[d]) + k.lam * (wa[c] * wb[d]);
          if (c == d) v += geo;
          H[blk][3 * c + d] = k.A0 * v;
        }
    }
}

// dF = sum_a u_a g_a^T for a nodal direction u
template <class R>
__device__ inline void direction_gradient(const TriConst<R>& k, const V3<R>* u, R dF[3][2]) {
  for (int j = 0; j < 2; ++j) {
    dF[0][j] = u[0].x * k.g[0][j] + u[1].x * k.g[1][j] + u[2].x * k.g[2][j];
    dF[1][j] = u[0].y * k.g[0][j] + u[1].y * k.g[1][j] + u[2].y * k.g[2][j];
    dF[2][j] = u[0].z * k.g[0][j] + u[1].z * k.g[1][j] + u[2].z * k.g[2][j];
  }
}

// Everything the adjoint needs from one triangle at positions x, for the adjoint
// vector lam and the new velocity u = v_{t+1}:
//   Hx_lam = H lam (exact Hessian),  Hc_lam = H~ lam,  Hc_u = H~ u,  f = -dE/dx,
//   third = d/dx (lam^T H~(x) u).
template <class R>
__device__ inline void membrane_adjoint(const TriConst<R>& k, const V3<R>* x, Sym2<R> G, const V3<R>* lam,
                                        const V3<R>* u, bool clamp, V3<R>* f, V3<R>* Hx_lam, V3<R>* Hc_lam,
                                        V3<R>* Hc_u, V3<R>* third) {
  R F[3][2], dFl[3][2], dFu[3][2];
  deformation_gradient(k, x, F);
  direction_gradient(k, lam, dFl);
  direction_gradient(k, u, dFu);
  Sym2<R> S = stvk_stress_G(k, G);
  Sym2<R> Sg = clamp ? smooth_positive(S, k.eps) : S;
  Sym2<R> dGl = sym_FtdF(F, dFl), dGu = sym_FtdF(F, dFu);
  Sym2<R> dSl = elastic_map(k, dGl), dSu = elastic_map(k, dGu);
  // N = d(M : S+)/dS with M = sym(dFl^T dFu), by three dual directions of S
  Sym2<R> M = sym_FtdF(dFl, dFu);
  Sym2<R> N;
  if (clamp) {
    R nn[3];
    for (int q = 0; q < 3; ++q) {
      Sym2<Dual<R>> Sd = {Dual<R>(S.a, q == 0 ? R(1) : R(0)), Dual<R>(S.b, q == 1 ? R(1) : R(0)),
                          Dual<R>(S.c, q == 2 ? R(1) : R(0))};
      Sym2<Dual<R>> P = smooth_positive(Sd, k.eps);
      nn[q] = M.a * P.a.d + M.b * P.b.d + R(2) * M.c * P.c.d;
    }
    N = {nn[0], nn[1], R(0.5) * nn[2]};  // direction q=2 moves both off-diagonal entries
  } else {
    N = M;
  }
  Sym2<R> CN = elastic_map(k, N);
  // ds/dF = A0 (F C:N + dFl C:dGu + dFu C:dGl)
  for (int a = 0; a < 3; ++a) {
    const R* g = k.g[a];
    f[a] = scale(-k.A0, mat32_sym_vec(F, S, g));
    V3<R> t1 = mat32_sym_vec(dFl, S, g) + mat32_sym_vec(F, dSl, g);
    Hx_lam[a] = scale(k.A0, t1);
    Hc_lam[a] = scale(k.A0, mat32_sym_vec(dFl, Sg, g) + mat32_sym_vec(F, dSl, g));
    Hc_u[a] = scale(k.A0, mat32_sym_vec(dFu, Sg, g) + mat32_sym_vec(F, dSu, g));
    third[a] = scale(k.A0, mat32_sym_vec(F, CN, g) + mat32_sym_vec(dFl, dSu, g) + mat32_sym_vec(dFu, dSl, g));
  }
}

// ------------------------------------------------------------------ bending parts
// theta and its gradient for one hinge (p[0] = x0, p[1] = x1, p[2] = xa, p[3] = xb).
template <class T>
__device__ inline void dihedral_grad(const V3<T>* p, T& theta, V3<T>* g) {
  V3<T> e = p[1] - p[0];
  V3<T> ua = p[2] - p[0];
  V3<T> ub = p[3] - p[0];
  V3<T> n1 = cross(e, ua);
  V3<T> n2 = cross(ub, e);
  T le2 = dot(e, e);
  T le = dsqrt(le2);
  theta = datan2(dot(cross(n1, n2), e) / le, dot(n1, n2));
  T ca = -le / dot(n1, n1);
  T cb = -le / dot(n2, n2);
  g[2] = {ca * n1.x, ca * n1.y, ca * n1.z};
  g[3] = {cb * n2.x, cb * n2.y, cb * n2.z};
  T ta = dot(ua, e) / le2;
  T tb = dot(ub, e) / le2;
  T one = cst<T>(1);
  g[1] = {-(ta * g[2].x + tb * g[3].x), -(ta * g[2].y + tb * g[3].y), -(ta * g[2].z + tb * g[3].z)};
  T sa = one - ta, sb = one - tb;
  g[0] = {-(sa * g[2].x + sb * g[3].x), -(sa * g[2].y + sb * g[3].y), -(sa * g[2].z + sb * g[3].z)};
}

template <class R>
struct HingeConst {
  R kw;      // k_b * w_e
  R theta0;  // rest angle
};

template <class R>
__device__ inline R comp(const V3<R>& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : v.z);
}

// Forces and upper Hessian blocks of one hinge: H = kw (g g^T + (theta - theta0) d2theta),
// d2theta column by column from dual numbers on the analytic gradient.
// H[10][9]: blocks (0,0),(0,1),(0,2),(0,3),(1,1),(1,2),(1,3),(2,2),(2,3),(3,3).
template <class R>
__device__ inline void bending_force_hessian(const HingeConst<R>& k, const V3<R>* x, V3<R>* f, R (*H)[9]) {
  R theta;
  V3<R> g[4];
  dihedral_grad(x, theta, g);
  const R dth = theta - k.theta0;
  for (int a = 0; a < 4; ++a) f[a] = scale(-k.kw * dth, g[a]);
  // column (b, d) of the Hessian
  for (int b = 0; b < 4; ++b)
    for (int d = 0; d < 3; ++d) {
      V3<Dual<R>> xd[4];
      for (int a = 0; a < 4; ++a) {
        xd[a].x = Dual<R>(x[a].x, (a == b && d == 0) ? R(1) : R(0));
        xd[a].y = Dual<R>(x[a].y, (a == b && d == 1) ? R(1) : R(0));
        xd[a].z = Dual<R>(x[a].z, (a == b && d == 2) ? R(1) : R(0));
      }
      Dual<R> th;
      V3<Dual<R>> gd[4];
      dihedral_grad(xd, th, gd);
      const R gbd = comp(g[b], d);
      for (int a = 0; a <= b; ++a) {
        const int blk = a * 4 - a * (a - 1) / 2 + (b - a);
        R col[3] = {gd[a].x.d, gd[a].y.d, gd[a].z.d};
        for (int c = 0; c < 3; ++c) H[blk][3 * c + d] = k.kw * (comp(g[a], c) * gbd + dth * col[c]);
      }
    }
  // exact symmetry of the diagonal blocks
  const int diag[4] = {0, 4, 7, 9};
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c)
      for (int d = c + 1; d < 3; ++d) {
        R m = R(0.5) * (H[diag[a]][3 * c + d] + H[diag[a]][3 * d + c]);
        H[diag[a]][3 * c + d] = m;
        H[diag[a]][3 * d + c] = m;
      }
}

// Adjoint quantities of one hinge (the bending Hessian is exact, so H~ = H):
//   f, H lam, H u and third = d/dx (lam^T H u) = D(H u)[lam] (symmetric third derivative),
// from one evaluation of the gradient in nested duals (outer along lam, inner along u).
template <class R>
__device__ inline void bending_adjoint(const HingeConst<R>& k, const V3<R>* x, const V3<R>* lam, const V3<R>* u,
                                       V3<R>* f, V3<R>* H_lam, V3<R>* H_u, V3<R>* third) {
  using D1 = Dual<R>;
  using D2 = Dual<D1>;
  V3<D2> xd[4];
  for (int a = 0; a < 4; ++a) {
    xd[a].x = D2(D1(x[a].x, u[a].x), D1(lam[a].x, R(0)));
    xd[a].y = D2(D1(x[a].y, u[a].y), D1(lam[a].y, R(0)));
    xd[a].z = D2(D1(x[a].z, u[a].z), D1(lam[a].z, R(0)));
  }
  D2 th;
  V3<D2> g[4];
  dihedral_grad(xd, th, g);
  const R dth = th.v.v - k.theta0;
  const R th_u = th.v.d, th_l = th.d.v, th_ul = th.d.d;
  for (int a = 0; a < 4; ++a) {
    for (int c = 0; c < 3; ++c) {
      const D2& gc = c == 0 ? g[a].x : (c == 1 ? g[a].y : g[a].z);
      const R g0 = gc.v.v, gu = gc.v.d, gl = gc.d.v, gul = gc.d.d;
      const R fv = -k.kw * dth * g0;
      const R hl = k.kw * (g0 * th_l + dth * gl);
      const R hu = k.kw * (g0 * th_u + dth * gu);
      const R t3 = k.kw * (gl * th_u + g0 * th_ul + th_l * gu + dth * gul);
      if (c == 0) { f[a].x = fv; H_lam[a].x = hl; H_u[a].x = hu; third[a].x = t3; }
      else if (c == 1) { f[a].y = fv; H_lam[a].y = hl; H_u[a].y = hu; third[a].y = t3; }
      else { f[a].z = fv; H_lam[a].z = hl; H_u[a].z = hu; third[a].z = t3; }
    }
  }
}

}  // namespace cloth
