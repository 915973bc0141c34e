// FP64 CPU oracle for the phi-SfT cloth simulator step and its adjoint.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
// this file: only the test-suite, the smoke check and the CPU-baseline leg of the
// benchmark use it.  It shares no code with the CUDA library (no headers, no
// helpers, no tables); the two meet only through seeded inputs.
//
// What it computes (phi-SfT, Sec. 3.1 "Deformation Model"):
//   * state S_t = {x_t, v_t} per vertex, fixed topology                  (Sec. 3.1)
//   * lumped diagonal mass from density and rest area                   (Eq. 3)
//   * internal forces from a membrane energy and a bending energy.  The
//     paper names a data-driven anisotropic model without formulas; the
//     reading taken here is an isotropic St. Venant-Kirchhoff membrane on
//     the Green strain and a dihedral-angle bending energy per interior
//     edge (reading R1/R2, stated in the design notes).
//   * external forces: gravity (M g) plus a per-step per-vertex force F_t  (Eq. 2)
//   * one implicit backward-Euler step linearised as in Eq. 4-5 with
//     df/dv = 0:  (M - h^2 K) dv = h (f + h K v),  v' = v + dv,  x' = x + h v'
//   * the linear system solved by Jacobi-preconditioned conjugate gradients
//     (the paper does not name its solver); pinned vertices keep dv = 0.
//   * the adjoint of the whole trajectory by implicit differentiation of the
//     linear solve (Sec. 3.1, backward pass after Liang et al.).
//
// Derivatives are NOT hand-derived here: the only physics written by hand is the
// two element energies.  Forces, Hessians and the third-derivative contraction
// needed by the adjoint all come from forward-mode automatic differentiation
// (nested dual numbers) of those energies, so a reader checks two short energy
// functions against the definitions and nothing else.
//
// Layout: every per-vertex array is AoS, vertex-major, [n][3] doubles.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>
#include <algorithm>

namespace {

// ---------------------------------------------------------------- dual numbers
template <class T> struct Dual {
  T v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(const T& a, const T& b) : v(a), d(b) {}
};
template <class T> Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return {a.v + b.v, a.d + b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return {a.v - b.v, a.d - b.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a) { return {-a.v, -a.d}; }
template <class T> Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
template <class T> Dual<T> operator*(double s, const Dual<T>& a) { return {s * a.v, s * a.d}; }
template <class T> Dual<T> operator*(const Dual<T>& a, double s) { return {s * a.v, s * a.d}; }
template <class T> Dual<T> operator+(const Dual<T>& a, double s) { return {a.v + s, a.d}; }
template <class T> Dual<T> operator-(const Dual<T>& a, double s) { return {a.v - s, a.d}; }

inline double dsqrt(double x) { return std::sqrt(x); }
inline double datan2(double y, double x) { return std::atan2(y, x); }
template <class T> Dual<T> dsqrt(const Dual<T>& a) {
  T s = dsqrt(a.v);
  return {s, a.d / (2.0 * s)};
}
// d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
template <class T> Dual<T> datan2(const Dual<T>& y, const Dual<T>& x) {
  return {datan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
}

inline double value_of(double a) { return a; }
template <class T> double value_of(const Dual<T>& a) { return value_of(a.v); }

template <class T> struct V3 { T x, y, z; };
template <class T> V3<T> sub(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// --------------------------------------------------------------- rest geometry
// Rest 2-D frame of a triangle: e1 along X1-X0, e2 = n x e1 in the plane.
// Dm = [[e1.(X1-X0), e1.(X2-X0)], [e2.(X1-X0), e2.(X2-X0)]], A0 = |det Dm| / 2.
struct TriRest {
  double Bm[4];  // Dm^{-1}, row-major 2x2
  double A0;
};

bool tri_rest(const double* X0, const double* X1, const double* X2, TriRest* out) {
  V3<double> a{X1[0] - X0[0], X1[1] - X0[1], X1[2] - X0[2]};
  V3<double> b{X2[0] - X0[0], X2[1] - X0[1], X2[2] - X0[2]};
  double la = std::sqrt(dot(a, a));
  V3<double> nrm = cross(a, b);
  double ln = std::sqrt(dot(nrm, nrm));
  if (la <= 0.0 || ln <= 1e-300) return false;
  V3<double> e1{a.x / la, a.y / la, a.z / la};
  V3<double> nh{nrm.x / ln, nrm.y / ln, nrm.z / ln};
  V3<double> e2 = cross(nh, e1);
  double d00 = dot(e1, a), d01 = dot(e1, b), d10 = dot(e2, a), d11 = dot(e2, b);
  double det = d00 * d11 - d01 * d10;
  if (std::fabs(det) <= 1e-300) return false;
  out->Bm[0] = d11 / det;
  out->Bm[1] = -d01 / det;
  out->Bm[2] = -d10 / det;
  out->Bm[3] = d00 / det;
  out->A0 = 0.5 * std::fabs(det);
  return true;
}

// ---------------------------------------------------------------- the energies
// Membrane (reading R1): F = Ds Dm^{-1} (3x2), G = (F^T F - I)/2,
// Psi = mu |G|_F^2 + (lambda/2) tr(G)^2, E = A0 Psi.
// Plane-stress Lame constants from the stretch stiffness Y [N/m] and Poisson nu:
// mu = Y / (2 (1 + nu)), lambda = Y nu / (1 - nu^2).
template <class T>
T membrane_energy(const TriRest& r, double mu, double lam, const T* x /*9*/) {
  T ds[3][2];
  for (int c = 0; c < 3; ++c) {
    ds[c][0] = x[3 + c] - x[c];
    ds[c][1] = x[6 + c] - x[c];
  }
  T F[3][2];
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 2; ++j) F[c][j] = ds[c][0] * r.Bm[0 * 2 + j] + ds[c][1] * r.Bm[1 * 2 + j];
  T C[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) C[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  T g00 = 0.5 * (C[0][0] - 1.0), g11 = 0.5 * (C[1][1] - 1.0), g01 = 0.5 * C[0][1];
  T frob = g00 * g00 + g11 * g11 + 2.0 * (g01 * g01);
  T tr = g00 + g11;
  return r.A0 * (mu * frob + 0.5 * lam * (tr * tr));
}

// Dihedral angle of a hinge (e0, e1, a, b).  Triangle 1 is (e0, e1, a) in its
// own winding, triangle 2 is (e1, e0, b).  n1 = (x_e1 - x_e0) x (x_a - x_e0),
// n2 = (x_b - x_e0) x (x_e1 - x_e0); theta = atan2((n1 x n2).e_hat, n1.n2).
template <class T>
T dihedral(const T* x /*12*/) {
  V3<T> p0{x[0], x[1], x[2]}, p1{x[3], x[4], x[5]}, pa{x[6], x[7], x[8]}, pb{x[9], x[10], x[11]};
  V3<T> e = sub(p1, p0);
  V3<T> n1 = cross(e, sub(pa, p0));
  V3<T> n2 = cross(sub(pb, p0), e);
  T le = dsqrt(dot(e, e));
  T s = dot(cross(n1, n2), e) / le;
  T c = dot(n1, n2);
  return datan2(s, c);
}

// Bending (reading R2): E = 1/2 k_b w_e (theta - theta_rest)^2 with
// w_e = 3 |e_rest|^2 / (A1_rest + A2_rest).
struct HingeRest {
  int v[4];
  double w;      // 3 |e|^2 / (A1 + A2), rest
  double theta0; // rest dihedral angle
};

template <class T>
T bending_energy(const HingeRest& h, double kb, const T* x /*12*/) {
  T d = dihedral(x) - h.theta0;
  return 0.5 * kb * h.w * (d * d);
}

// Clamped geometric stiffness (reading R6).  Under compression the StVK Hessian's
// geometric term tr(dF^T dF' S) is indefinite and A = M - h^2 K loses definiteness.
// The clamped Hessian replaces the second Piola-Kirchhoff stress S in that term by
// a smooth positive part  S+ = (S + (S^2 + eps^2 I)^{1/2}) / 2,  eps = eta * Y,
// which is positive definite, infinitely differentiable (no kink at S = 0, where
// every rollout starts) and tends to max(S, 0) for |S| >> eps.  Hence
//   H~_mem(x) = d^2E_mem/dx^2 (x) - A0 tr(dF^T dF' S-(x)),   S- = S - S+,
// i.e. S- = (S - (S^2 + eps^2 I)^{1/2}) / 2.  The 2x2 SPD square root is the closed
// form  sqrt(P) = (P + sqrt(det P) I) / sqrt(tr P + 2 sqrt(det P)).
// Forces stay the exact -dE/dx; only the matrix of the linear solve changes.
template <class T>
void stvk_negative_stress(const TriRest& r, double mu, double lam, double eps, const T* x /*9*/, T Sm[2][2]) {
  T F[3][2];
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 2; ++j)
      F[c][j] = (x[3 + c] - x[c]) * r.Bm[0 * 2 + j] + (x[6 + c] - x[c]) * r.Bm[1 * 2 + j];
  T G[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      G[i][j] = 0.5 * (F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j] - (i == j ? 1.0 : 0.0));
  T tr = G[0][0] + G[1][1];
  T S[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) S[i][j] = 2.0 * mu * G[i][j] + (i == j ? lam * tr : T(0.0));
  T P[2][2];  // S^2 + eps^2 I
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) P[i][j] = S[i][0] * S[0][j] + S[i][1] * S[1][j] + (i == j ? eps * eps : 0.0);
  T sdet = dsqrt(P[0][0] * P[1][1] - P[0][1] * P[1][0]);
  T tnorm = dsqrt(P[0][0] + P[1][1] + 2.0 * sdet);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      T root = (P[i][j] + (i == j ? sdet : T(0.0))) / tnorm;
      Sm[i][j] = 0.5 * (S[i][j] - root);
    }
}

// Deformation-gradient differential dF = dDs Dm^{-1} for a nodal direction a (9).
inline void dF_of(const TriRest& r, const double* a, double dF[3][2]) {
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 2; ++j)
      dF[c][j] = (a[3 + c] - a[c]) * r.Bm[0 * 2 + j] + (a[6 + c] - a[c]) * r.Bm[1 * 2 + j];
}

// g(x) = A0 tr(dF_a^T dF_b S-(x)) for fixed nodal directions a, b.
template <class T>
T neg_geometric_form(const TriRest& r, double mu, double lam, double eps, const double* a, const double* b,
                     const T* x) {
  T Sm[2][2];
  stvk_negative_stress(r, mu, lam, eps, x, Sm);
  double Fa[3][2], Fb[3][2];
  dF_of(r, a, Fa);
  dF_of(r, b, Fb);
  T acc = T(0.0);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double M = Fa[0][i] * Fb[0][j] + Fa[1][i] * Fb[1][j] + Fa[2][i] * Fb[2][j];  // (dF_a^T dF_b)_ij
      acc = acc + M * Sm[j][i];
    }
  return r.A0 * acc;
}

// ------------------------------------------------------------ AD element kernels
// Gradient and Hessian of an element energy with k DOFs by nested duals.
// H[j][l] is the eps1*eps2 coefficient of E(x + eps1 e_l + eps2 e_j).
template <int K, class EnergyFn>
void ad_grad_hess(const double* x, EnergyFn energy, double* E, double* g, double* H) {
  using D1 = Dual<double>;
  using D2 = Dual<D1>;
  for (int j = 0; j < K; ++j) {
    for (int l = j; l < K; ++l) {
      D2 xs[K];
      for (int i = 0; i < K; ++i) xs[i] = D2(D1(x[i], i == l ? 1.0 : 0.0), D1(i == j ? 1.0 : 0.0, 0.0));
      D2 e = energy(xs);
      if (H) {
        H[j * K + l] = e.d.d;
        H[l * K + j] = e.d.d;
      }
      if (j == 0 && g) g[l] = e.v.d;
      if (j == 0 && l == 0 && E) *E = e.v.v;
    }
  }
}

template <int K, class EnergyFn>
void ad_grad(const double* x, EnergyFn energy, double* E, double* g) {
  using D1 = Dual<double>;
  for (int l = 0; l < K; ++l) {
    D1 xs[K];
    for (int i = 0; i < K; ++i) xs[i] = D1(x[i], i == l ? 1.0 : 0.0);
    D1 e = energy(xs);
    g[l] = e.d;
    if (l == 0 && E) *E = e.v;
  }
}

// out[q] = sum_{i,j} d^3E / (dx_i dx_j dx_q) a_i b_j  (third derivative contracted
// with two directions), the eps1*eps2*eps3 coefficient of E(x + eps1 a + eps2 b + eps3 e_q).
template <int K, class EnergyFn>
void ad_third(const double* x, const double* a, const double* b, EnergyFn energy, double* out) {
  using D1 = Dual<double>;
  using D2 = Dual<D1>;
  using D3 = Dual<D2>;
  for (int q = 0; q < K; ++q) {
    D3 xs[K];
    for (int i = 0; i < K; ++i)
      xs[i] = D3(D2(D1(x[i], a[i]), D1(b[i], 0.0)), D2(D1(i == q ? 1.0 : 0.0, 0.0), D1(0.0, 0.0)));
    D3 e = energy(xs);
    out[q] = e.d.d.d;
  }
}

// ----------------------------------------------------------------- the system
struct Sim {
  int n = 0, m = 0;
  std::vector<double> rest;        // [n][3]
  std::vector<int> tris;           // [m][3]
  std::vector<unsigned char> pinned;
  std::vector<TriRest> trest;      // [m]
  std::vector<HingeRest> hinges;   // [ne]
  std::vector<double> area3;       // [n] sum over incident triangles of A0/3 (mass per unit density)
};

struct Mat {
  double Y, nu, kb, rho;
  double eta;  // > 0: membrane geometric stiffness uses the smooth positive stress, eps = eta * Y (R6)
  int precond = 1;  // CG preconditioner: 0 scalar Jacobi, 1 3x3 block Jacobi
  double mu() const { return Y / (2.0 * (1.0 + nu)); }
  double lam() const { return Y * nu / (1.0 - nu * nu); }
};

void gather(const double* x, const int* idx, int k, double* out) {
  for (int a = 0; a < k; ++a)
    for (int c = 0; c < 3; ++c) out[3 * a + c] = x[3 * idx[a] + c];
}

// Sparse symmetric matrix kept as one ordered map per row: slow, plain.
struct Sparse {
  std::vector<std::map<int, double>> rows;
  explicit Sparse(int dof) : rows(dof) {}
  void add(int i, int j, double v) { rows[i][j] += v; }
  void matvec(const std::vector<double>& p, std::vector<double>& y) const {
    for (size_t i = 0; i < rows.size(); ++i) {
      double s = 0.0;
      for (const auto& kv : rows[i]) s += kv.second * p[kv.first];
      y[i] = s;
    }
  }
  double at(int i, int j) const {
    auto it = rows[i].find(j);
    return it == rows[i].end() ? 0.0 : it->second;
  }
};

// Internal elastic energy and force f = -dE/dx, split by term.
void internal_forces(const Sim& s, const Mat& mt, const double* x, double* f_mem, double* f_bend, double* Eout) {
  const int n3 = 3 * s.n;
  std::fill(f_mem, f_mem + n3, 0.0);
  std::fill(f_bend, f_bend + n3, 0.0);
  double Etot = 0.0;
  const double mu = mt.mu(), lam = mt.lam();
  for (int t = 0; t < s.m; ++t) {
    double xe[9], g[9], E;
    gather(x, &s.tris[3 * t], 3, xe);
    const TriRest& r = s.trest[t];
    ad_grad<9>(xe, [&](const auto* xs) { return membrane_energy(r, mu, lam, xs); }, &E, g);
    Etot += E;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) f_mem[3 * s.tris[3 * t + a] + c] -= g[3 * a + c];
  }
  for (const HingeRest& h : s.hinges) {
    double xe[12], g[12], E;
    gather(x, h.v, 4, xe);
    ad_grad<12>(xe, [&](const auto* xs) { return bending_energy(h, mt.kb, xs); }, &E, g);
    Etot += E;
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 3; ++c) f_bend[3 * h.v[a] + c] -= g[3 * a + c];
  }
  if (Eout) *Eout = Etot;
}

// Hessian of the internal energy H = d^2E/dx^2 (so the stiffness K = -H),
// membrane and bending parts accumulated into separate sparse matrices.
void internal_hessian(const Sim& s, const Mat& mt, const double* x, Sparse& Hm, Sparse& Hb) {
  const double mu = mt.mu(), lam = mt.lam();
  for (int t = 0; t < s.m; ++t) {
    double xe[9], H[81];
    const int* v = &s.tris[3 * t];
    gather(x, v, 3, xe);
    const TriRest& r = s.trest[t];
    ad_grad_hess<9>(xe, [&](const auto* xs) { return membrane_energy(r, mu, lam, xs); }, nullptr, nullptr, H);
    if (mt.eta > 0.0) {
      for (int j = 0; j < 9; ++j)
        for (int l = 0; l < 9; ++l) {
          double ej[9] = {0}, el[9] = {0};
          ej[j] = 1.0;
          el[l] = 1.0;
          H[j * 9 + l] -= neg_geometric_form(r, mu, lam, mt.eta * mt.Y, ej, el, xe);
        }
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) Hm.add(3 * v[a] + c, 3 * v[b] + d, H[(3 * a + c) * 9 + 3 * b + d]);
  }
  for (const HingeRest& h : s.hinges) {
    double xe[12], H[144];
    gather(x, h.v, 4, xe);
    ad_grad_hess<12>(xe, [&](const auto* xs) { return bending_energy(h, mt.kb, xs); }, nullptr, nullptr, H);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) Hb.add(3 * h.v[a] + c, 3 * h.v[b] + d, H[(3 * a + c) * 12 + 3 * b + d]);
  }
}

// out = d/dx [ a^T H(x) b ] = D^3E[a, b, .], membrane and bending parts summed.
void third_contraction(const Sim& s, const Mat& mt, const double* x, const double* a, const double* b, double* out) {
  const double mu = mt.mu(), lam = mt.lam();
  std::fill(out, out + 3 * s.n, 0.0);
  for (int t = 0; t < s.m; ++t) {
    double xe[9], ae[9], be[9], o[9];
    const int* v = &s.tris[3 * t];
    gather(x, v, 3, xe);
    gather(a, v, 3, ae);
    gather(b, v, 3, be);
    const TriRest& r = s.trest[t];
    ad_third<9>(xe, ae, be, [&](const auto* xs) { return membrane_energy(r, mu, lam, xs); }, o);
    if (mt.eta > 0.0) {
      double gneg[9];
      ad_grad<9>(xe, [&](const auto* xs) { return neg_geometric_form(r, mu, lam, mt.eta * mt.Y, ae, be, xs); },
                 nullptr, gneg);
      for (int q = 0; q < 9; ++q) o[q] -= gneg[q];
    }
    for (int q = 0; q < 3; ++q)
      for (int c = 0; c < 3; ++c) out[3 * v[q] + c] += o[3 * q + c];
  }
  for (const HingeRest& h : s.hinges) {
    double xe[12], ae[12], be[12], o[12];
    gather(x, h.v, 4, xe);
    gather(a, h.v, 4, ae);
    gather(b, h.v, 4, be);
    ad_third<12>(xe, ae, be, [&](const auto* xs) { return bending_energy(h, mt.kb, xs); }, o);
    for (int q = 0; q < 4; ++q)
      for (int c = 0; c < 3; ++c) out[3 * h.v[q] + c] += o[3 * q + c];
  }
}

// Inverse of a 3x3 matrix by the adjugate (cofactor transpose over the determinant).
void inv3(const double m[9], double out[9]) {
  const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  out[0] = c00 / det;
  out[1] = (m[2] * m[7] - m[1] * m[8]) / det;
  out[2] = (m[1] * m[5] - m[2] * m[4]) / det;
  out[3] = c01 / det;
  out[4] = (m[0] * m[8] - m[2] * m[6]) / det;
  out[5] = (m[2] * m[3] - m[0] * m[5]) / det;
  out[6] = c02 / det;
  out[7] = (m[1] * m[6] - m[0] * m[7]) / det;
  out[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

// The same matrix as flat row arrays (columns ascending, as the map iterates), made once
// per solve: its product sums every row in the same order as Sparse::matvec, so every
// result is identical; it only spares walking the maps in each CG iteration.
struct Csr {
  std::vector<size_t> ptr;
  std::vector<int> col;
  std::vector<double> val;
  explicit Csr(const Sparse& A) : ptr(A.rows.size() + 1, 0) {
    for (size_t i = 0; i < A.rows.size(); ++i) ptr[i + 1] = ptr[i] + A.rows[i].size();
    col.reserve(ptr.back());
    val.reserve(ptr.back());
    for (const auto& row : A.rows)
      for (const auto& kv : row) {
        col.push_back(kv.first);
        val.push_back(kv.second);
      }
  }
  void matvec(const std::vector<double>& p, std::vector<double>& y) const {
    for (size_t i = 0; i + 1 < ptr.size(); ++i) {
      double s = 0.0;
      for (size_t q = ptr[i]; q < ptr[i + 1]; ++q) s += val[q] * p[col[q]];
      y[i] = s;
    }
  }
};

// Jacobi-preconditioned CG on A y = rhs from y = 0, stopping when
// |r|_2 <= tol |rhs|_2 (checked before each iteration) or after max_iter.
// precond 0: scalar Jacobi z_i = r_i / A_ii;  1: block Jacobi with the 3x3 diagonal
// block of each vertex, z_v = A_vv^{-1} r_v.
// Returns 0 converged, 1 max_iter reached, 2 p^T A p <= 0 (indefinite), 3 non-finite.
int pcg(const Sparse& A, const std::vector<double>& rhs, double tol, int max_iter, int precond, std::vector<double>& y,
        int* iters) {
  const size_t N = rhs.size();
  const Csr C(A);
  std::vector<double> r(rhs), z(N), p(N), Ap(N), dinv(N), binv(precond ? 3 * N : 0);
  y.assign(N, 0.0);
  if (precond) {
    for (size_t v = 0; v < N / 3; ++v) {
      double blk[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) blk[3 * a + b] = A.at((int)(3 * v + a), (int)(3 * v + b));
      inv3(blk, &binv[9 * v]);
    }
  } else {
    for (size_t i = 0; i < N; ++i) dinv[i] = 1.0 / A.at((int)i, (int)i);
  }
  auto apply_prec = [&]() {
    if (precond) {
      for (size_t v = 0; v < N / 3; ++v)
        for (int a = 0; a < 3; ++a) {
          double acc = 0.0;
          for (int b = 0; b < 3; ++b) acc += binv[9 * v + 3 * a + b] * r[3 * v + b];
          z[3 * v + a] = acc;
        }
    } else {
      for (size_t i = 0; i < N; ++i) z[i] = dinv[i] * r[i];
    }
  };
  auto dotv = [&](const std::vector<double>& u, const std::vector<double>& w) {
    double acc = 0.0;
    for (size_t i = 0; i < N; ++i) acc += u[i] * w[i];
    return acc;
  };
  const double bnorm = std::sqrt(dotv(rhs, rhs));
  *iters = 0;
  if (!std::isfinite(bnorm)) return 3;
  if (bnorm == 0.0) return 0;
  apply_prec();
  p = z;
  double rz = dotv(r, z);
  double rr = dotv(r, r);
  for (int k = 0; k < max_iter; ++k) {
    if (std::sqrt(rr) <= tol * bnorm) return 0;
    C.matvec(p, Ap);
    double pAp = dotv(p, Ap);
    if (!std::isfinite(pAp)) return 3;
    if (pAp <= 0.0) return 2;
    double alpha = rz / pAp;
    for (size_t i = 0; i < N; ++i) {
      y[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    apply_prec();
    double rz_new = dotv(r, z);
    rr = dotv(r, r);
    double beta = rz_new / rz;
    rz = rz_new;
    for (size_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    *iters = k + 1;
  }
  return std::sqrt(rr) <= tol * bnorm ? 0 : 1;
}

struct Opts {
  double dt, tol, gravity[3];
  int steps, max_iter;
};

// A = M - h^2 K = M + h^2 (Hm + Hb); rows/cols of pinned DOFs replaced by identity.
Sparse system_matrix(const Sim& s, const Mat& mt, double h, const Sparse& Hm, const Sparse& Hb) {
  const int N = 3 * s.n;
  Sparse A(N);
  for (int i = 0; i < N; ++i) {
    const int vi = i / 3;
    if (s.pinned[vi]) {
      A.add(i, i, 1.0);
      continue;
    }
    A.add(i, i, mt.rho * s.area3[vi]);
    for (const Sparse* H : {&Hm, &Hb})
      for (const auto& kv : H->rows[i])
        if (!s.pinned[kv.first / 3]) A.add(i, kv.first, h * h * kv.second);
  }
  return A;
}

// ------------------------------------------------------------------- air drag
// Wind: the air moves at the sheet's wind velocity w (density rho_air).  Each free vertex
// feels the quadratic drag of the relative air velocity d = w - v on its lumped rest area
// A_i (the area that also lumps its mass):  f_i = rho_air A_i |d|_e d,  with the smooth
// magnitude |d|_e = sqrt(d.d + e^2), e = kDragEps.  Its velocity Jacobian is
// df/dv = -rho_air A_i G(d),  G(d) = |d|_e I + d d^T / |d|_e  (symmetric positive
// definite), which enters the step matrix as + h rho_air A_i G (Eq. 5 with df/dv != 0).
constexpr double kDragEps = 1e-3;

double drag_norm(const double d[3]) { return std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + kDragEps * kDragEps); }

void drag_G(const double d[3], double G[9]) {
  const double n = drag_norm(d);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[3 * a + b] = (a == b ? n : 0.0) + d[a] * d[b] / n;
}

// out_k = a^T (dG/dd_k) b, k = 0..2 (the derivative of G(d) contracted with a and b)
void drag_dG(const double d[3], const double a[3], const double b[3], double out[3]) {
  const double n = drag_norm(d);
  const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  const double ad = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
  const double db = d[0] * b[0] + d[1] * b[1] + d[2] * b[2];
  for (int k = 0; k < 3; ++k)
    out[k] = d[k] / n * ab + (a[k] * db + ad * b[k]) / n - ad * db * d[k] / (n * n * n);
}

}  // namespace

// ============================================================== C interface
extern "C" {

// Status / error codes (oracle-local).
enum { OR_OK = 0, OR_INVALID = -1, OR_DEGENERATE = -2, OR_NONMANIFOLD = -3 };

// Build the simulation handle: rest positions [n][3], triangles [m][3], pinned[n].
// Precomputes per-triangle rest frames, interior-edge hinges and lumped areas.
int oracle_create(int n, const double* rest, int m, const int* tris, const unsigned char* pinned, void** out) {
  if (n <= 0 || m <= 0 || !rest || !tris || !out) return OR_INVALID;
  Sim* s = new Sim();
  s->n = n;
  s->m = m;
  s->rest.assign(rest, rest + 3 * n);
  s->tris.assign(tris, tris + 3 * m);
  s->pinned.assign(n, 0);
  if (pinned)
    for (int i = 0; i < n; ++i) s->pinned[i] = pinned[i] ? 1 : 0;
  s->trest.resize(m);
  s->area3.assign(n, 0.0);
  for (int t = 0; t < m; ++t) {
    const int* v = &tris[3 * t];
    for (int a = 0; a < 3; ++a)
      if (v[a] < 0 || v[a] >= n) { delete s; return OR_INVALID; }
    if (!tri_rest(&rest[3 * v[0]], &rest[3 * v[1]], &rest[3 * v[2]], &s->trest[t])) { delete s; return OR_DEGENERATE; }
    for (int a = 0; a < 3; ++a) s->area3[v[a]] += s->trest[t].A0 / 3.0;
  }
  // Interior edges: an undirected edge seen by exactly two triangles.  The first
  // triangle found traverses it as (e0 -> e1) and supplies wing a; the second
  // must traverse it as (e1 -> e0) (consistent winding) and supplies wing b.
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> seen;  // key (min,max) -> (tri, local edge)
  for (int t = 0; t < m; ++t)
    for (int k = 0; k < 3; ++k) {
      int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
      seen[{std::min(a, b), std::max(a, b)}].push_back({t, k});
    }
  for (const auto& kv : seen) {
    if (kv.second.size() > 2) { delete s; return OR_NONMANIFOLD; }
    if (kv.second.size() != 2) continue;
    int t1 = kv.second[0].first, k1 = kv.second[0].second;
    int t2 = kv.second[1].first, k2 = kv.second[1].second;
    int e0 = tris[3 * t1 + k1], e1 = tris[3 * t1 + (k1 + 1) % 3], wa = tris[3 * t1 + (k1 + 2) % 3];
    int f0 = tris[3 * t2 + k2], f1 = tris[3 * t2 + (k2 + 1) % 3], wb = tris[3 * t2 + (k2 + 2) % 3];
    if (!(f0 == e1 && f1 == e0)) { delete s; return OR_NONMANIFOLD; }  // inconsistent winding
    HingeRest h;
    h.v[0] = e0; h.v[1] = e1; h.v[2] = wa; h.v[3] = wb;
    double d[3] = {rest[3 * e1] - rest[3 * e0], rest[3 * e1 + 1] - rest[3 * e0 + 1], rest[3 * e1 + 2] - rest[3 * e0 + 2]};
    double l2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    h.w = 3.0 * l2 / (s->trest[t1].A0 + s->trest[t2].A0);
    double xe[12];
    gather(rest, h.v, 4, xe);
    h.theta0 = dihedral(xe);
    s->hinges.push_back(h);
  }
  *out = s;
  return OR_OK;
}

void oracle_destroy(void* h) { delete static_cast<Sim*>(h); }

int oracle_num_hinges(void* h) { return (int)static_cast<Sim*>(h)->hinges.size(); }

// hinges out: [ne][4] vertex ids (e0, e1, a, b); w and theta0 out: [ne]
void oracle_hinges(void* h, int* v, double* w, double* theta0) {
  const Sim* s = static_cast<Sim*>(h);
  for (size_t i = 0; i < s->hinges.size(); ++i) {
    for (int k = 0; k < 4; ++k) v[4 * i + k] = s->hinges[i].v[k];
    if (w) w[i] = s->hinges[i].w;
    if (theta0) theta0[i] = s->hinges[i].theta0;
  }
}

// Lumped mass per vertex m_i = rho * sum_{t ∋ i} A0_t / 3  (Eq. 3: diagonal M
// from density and surface area).
void oracle_mass(void* h, double rho, double* mass) {
  const Sim* s = static_cast<Sim*>(h);
  for (int i = 0; i < s->n; ++i) mass[i] = rho * s->area3[i];
}

// material = {Y, nu, kb, rho}.  Energy of the internal forces and f = -dE/dx.
double oracle_energy_forces(void* h, const double* material, const double* x, double* f_mem, double* f_bend) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], 0.0};
  std::vector<double> fm(3 * s->n), fb(3 * s->n);
  double E;
  internal_forces(*s, mt, x, fm.data(), fb.data(), &E);
  if (f_mem) std::copy(fm.begin(), fm.end(), f_mem);
  if (f_bend) std::copy(fb.begin(), fb.end(), f_bend);
  return E;
}

// Dense Hessian H = d^2E/dx^2 [3n][3n] (small meshes only).
void oracle_hessian_dense(void* h, const double* material, double eta, const double* x, double* H) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], eta};
  const int N = 3 * s->n;
  Sparse Hm(N), Hb(N);
  internal_hessian(*s, mt, x, Hm, Hb);
  std::fill(H, H + (size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i) {
    for (const auto& kv : Hm.rows[i]) H[(size_t)i * N + kv.first] += kv.second;
    for (const auto& kv : Hb.rows[i]) H[(size_t)i * N + kv.first] += kv.second;
  }
}

// out = D^3E(x)[a, b, .]  (n x 3)
void oracle_third(void* h, const double* material, double eta, const double* x, const double* a, const double* b,
                  double* out) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], eta};
  third_contraction(*s, mt, x, a, b, out);
}

// Element-level helpers for the closed-form pins.
// rest/x: 3 vertices x 3 coords.  Returns 0 or OR_DEGENERATE.
int oracle_membrane_element(const double* rest, const double* x, double Y, double nu, double* E, double* g, double* H) {
  TriRest r;
  if (!tri_rest(rest, rest + 3, rest + 6, &r)) return OR_DEGENERATE;
  double mu = Y / (2.0 * (1.0 + nu)), lam = Y * nu / (1.0 - nu * nu);
  ad_grad_hess<9>(x, [&](const auto* xs) { return membrane_energy(r, mu, lam, xs); }, E, g, H);
  return OR_OK;
}

double oracle_dihedral(const double* x /*12*/) { return dihedral(x); }

// One linearised implicit step's system (small meshes): A dense [3n][3n] and b [3n],
// with pinned rows/cols replaced by identity and b_pinned = 0.
void oracle_system_dense(void* h, const double* material, double eta, double dt, const double* gravity,
                         const double* x, const double* v, const double* F, double* A, double* b) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], eta};
  const int N = 3 * s->n;
  Sparse Hm(N), Hb(N);
  internal_hessian(*s, mt, x, Hm, Hb);
  Sparse As = system_matrix(*s, mt, dt, Hm, Hb);
  std::fill(A, A + (size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (const auto& kv : As.rows[i]) A[(size_t)i * N + kv.first] = kv.second;
  std::vector<double> fm(N), fb(N), Hv(N), Hv2(N);
  internal_forces(*s, mt, x, fm.data(), fb.data(), nullptr);
  std::vector<double> vv(v, v + N);
  Hm.matvec(vv, Hv);
  Hb.matvec(vv, Hv2);
  for (int i = 0; i < N; ++i) {
    const int vi = i / 3;
    if (s->pinned[vi]) { b[i] = 0.0; continue; }
    double f = fm[i] + fb[i] + mt.rho * s->area3[vi] * gravity[i % 3] + (F ? F[i] : 0.0);
    b[i] = dt * (f - dt * (Hv[i] + Hv2[i]));
  }
}

// One step's system applied to a vector (any mesh size): y = A p and the right-hand
// side b, with A = M + h^2 H~ and b = h (f + M g + F) - h^2 H~ v (pinned rows identity, b = 0).
void oracle_system_matvec(void* h, const double* material, double eta, double dt, const double* gravity,
                          const double* x, const double* v, const double* F, const double* p, double* y, double* b) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], eta};
  const int N = 3 * s->n;
  Sparse Hm(N), Hb(N);
  internal_hessian(*s, mt, x, Hm, Hb);
  Sparse A = system_matrix(*s, mt, dt, Hm, Hb);
  std::vector<double> pv(p, p + N), yv(N), fm(N), fb(N), Hv(N), Hv2(N), vv(v, v + N);
  A.matvec(pv, yv);
  std::copy(yv.begin(), yv.end(), y);
  internal_forces(*s, mt, x, fm.data(), fb.data(), nullptr);
  Hm.matvec(vv, Hv);
  Hb.matvec(vv, Hv2);
  for (int i = 0; i < N; ++i) {
    const int vi = i / 3;
    if (s->pinned[vi]) {
      b[i] = 0.0;
      continue;
    }
    double f = fm[i] + fb[i] + mt.rho * s->area3[vi] * gravity[i % 3] + (F ? F[i] : 0.0);
    b[i] = dt * (f - dt * (Hv[i] + Hv2[i]));
  }
}

// Forward trajectory.  x0, v0: [n][3]; forces: [steps][n][3] or NULL;
// force_mode 0: F_t is a force [N] added to f (Eq. 3); 1: F_t is a velocity increment
// [m/s] added to the free vertices' velocities before step t (the corrective forces'
// form in the paper's implementation details, Sec. 3.4), v'_t = v_t + F_t, and the step
// runs from (x_t, v'_t).
// traj_x, traj_v: [steps+1][n][3] (traj_v holds v_t, before any increment); cg_iters [steps];
// status: worst per-step solver status (0 ok, 1 maxiter, 2 indefinite, 3 non-finite).
// air_density > 0 with wind (double[3]): the air drag above acts on every free vertex.
int oracle_forward(void* h, const double* material, double eta, int precond, double dt, int steps, double tol,
                   int max_iter, const double* gravity, const double* x0, const double* v0, const double* forces,
                   int force_mode, double air_density, const double* wind, double* traj_x, double* traj_v,
                   int* cg_iters, int* status) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], eta, precond};
  const int N = 3 * s->n;
  std::copy(x0, x0 + N, traj_x);
  std::copy(v0, v0 + N, traj_v);
  int worst = 0;
  std::vector<double> fm(N), fb(N), b(N), Hv(N), Hv2(N), dv;
  for (int t = 0; t < steps; ++t) {
    const double* x = traj_x + (size_t)t * N;
    const double* v = traj_v + (size_t)t * N;
    const double* F = forces ? forces + (size_t)t * N : nullptr;
    Sparse Hm(N), Hb(N);
    internal_hessian(*s, mt, x, Hm, Hb);
    internal_forces(*s, mt, x, fm.data(), fb.data(), nullptr);
    std::vector<double> vv(v, v + N);  // the step's starting velocity
    if (F && force_mode == 1)
      for (int i = 0; i < N; ++i)
        if (!s->pinned[i / 3]) vv[i] += F[i];
    Hm.matvec(vv, Hv);
    Hb.matvec(vv, Hv2);
    for (int i = 0; i < N; ++i) {
      const int vi = i / 3;
      double f = fm[i] + fb[i] + mt.rho * s->area3[vi] * gravity[i % 3] + (F && force_mode == 0 ? F[i] : 0.0);
      b[i] = s->pinned[vi] ? 0.0 : dt * (f - dt * (Hv[i] + Hv2[i]));
    }
    Sparse A = system_matrix(*s, mt, dt, Hm, Hb);
    if (air_density > 0.0 && wind)
      for (int vi = 0; vi < s->n; ++vi) {
        if (s->pinned[vi]) continue;
        const double d[3] = {wind[0] - vv[3 * vi], wind[1] - vv[3 * vi + 1], wind[2] - vv[3 * vi + 2]};
        const double c = air_density * s->area3[vi], n = drag_norm(d);
        double G[9];
        drag_G(d, G);
        for (int a = 0; a < 3; ++a) {
          b[3 * vi + a] += dt * c * n * d[a];
          for (int q = 0; q < 3; ++q) A.add(3 * vi + a, 3 * vi + q, dt * c * G[3 * a + q]);
        }
      }
    int it = 0;
    int st = pcg(A, b, tol, max_iter, mt.precond, dv, &it);
    if (cg_iters) cg_iters[t] = it;
    worst = std::max(worst, st);
    double* xn = traj_x + (size_t)(t + 1) * N;
    double* vn = traj_v + (size_t)(t + 1) * N;
    for (int i = 0; i < N; ++i) {
      vn[i] = vv[i] + dv[i];
      xn[i] = x[i] + dt * vn[i];
    }
  }
  if (status) *status = worst;
  return OR_OK;
}

// Adjoint of the whole trajectory (implicit differentiation of each linear solve,
// reverse sweep over the stored forward states).
// dL_dx: [steps+1][n][3] (gradient of the loss w.r.t. every x_t, t = 0..steps).
// Outputs (any may be NULL): g_material[4] (dL/dY, dL/dnu := 0, dL/dkb, dL/drho),
// g_forces [steps][n][3], g_x0 [n][3], g_v0 [n][3]; cg_iters [steps]; status.
// forces, force_mode: as given to oracle_forward (the forces are read only in mode 1,
// where the step started from v'_t = v_t + F_t; then dL/dF_t = dL/dv'_t on free vertices).
// air_density, wind: as given to oracle_forward; g_wind (double[3] or NULL): dL/dw.
int oracle_backward(void* h, const double* material, double eta, int precond, double dt, int steps, double tol,
                    int max_iter, const double* gravity, const double* traj_x, const double* traj_v,
                    const double* forces, int force_mode, double air_density, const double* wind,
                    const double* dL_dx, double* g_material, double* g_forces, double* g_x0, double* g_v0,
                    double* g_wind, int* cg_iters, int* status) {
  const Sim* s = static_cast<Sim*>(h);
  Mat mt{material[0], material[1], material[2], material[3], eta, precond};
  const int N = 3 * s->n;
  std::vector<double> ax(dL_dx + (size_t)steps * N, dL_dx + (size_t)(steps + 1) * N), av(N, 0.0);
  std::vector<double> g(N), lam, Hl(N), Hl2(N), third(N), fm(N), fb(N), Hu(N), Hu2(N), u(N), dv(N);
  double gY = 0.0, gkb = 0.0, grho = 0.0, gw[3] = {0.0, 0.0, 0.0};
  const bool drag = air_density > 0.0 && wind;
  std::vector<double> vst(N);
  int worst = 0;
  for (int t = steps - 1; t >= 0; --t) {
    const double* x = traj_x + (size_t)t * N;
    const double* v = traj_v + (size_t)t * N;
    const double* vn = traj_v + (size_t)(t + 1) * N;
    const double* F = (forces && force_mode == 1) ? forces + (size_t)t * N : nullptr;
    for (int i = 0; i < N; ++i) {
      u[i] = vn[i];
      const double vstart = v[i] + ((F && !s->pinned[i / 3]) ? F[i] : 0.0);  // v'_t
      vst[i] = vstart;
      dv[i] = vn[i] - vstart;
      // adjoint of dv: v_{t+1} = v_t + dv and x_{t+1} = x_t + h v_{t+1}
      g[i] = s->pinned[i / 3] ? 0.0 : av[i] + dt * ax[i];
    }
    Sparse Hm(N), Hb(N);
    internal_hessian(*s, mt, x, Hm, Hb);
    Sparse A = system_matrix(*s, mt, dt, Hm, Hb);
    if (drag)
      for (int vi = 0; vi < s->n; ++vi) {
        if (s->pinned[vi]) continue;
        const double d[3] = {wind[0] - vst[3 * vi], wind[1] - vst[3 * vi + 1], wind[2] - vst[3 * vi + 2]};
        double G[9];
        drag_G(d, G);
        for (int a = 0; a < 3; ++a)
          for (int q = 0; q < 3; ++q) A.add(3 * vi + a, 3 * vi + q, dt * air_density * s->area3[vi] * G[3 * a + q]);
      }
    int it = 0;
    int st = pcg(A, g, tol, max_iter, mt.precond, lam, &it);
    worst = std::max(worst, st);
    if (cg_iters) cg_iters[t] = it;
    // The matrix term of b and A uses the (possibly clamped) Hessian H~ = Hm + Hb;
    // the force term of b differentiates to the exact Hessian: db/dx = -h H - h^2 d(H~ v)/dx.
    Hm.matvec(lam, Hl);
    Hb.matvec(lam, Hl2);
    std::vector<double> Hxl(N), Hxl2(N);
    if (mt.eta > 0.0) {
      Mat exact = mt;
      exact.eta = 0.0;
      Sparse Em(N), Eb(N);
      internal_hessian(*s, exact, x, Em, Eb);
      Em.matvec(lam, Hxl);
      Eb.matvec(lam, Hxl2);
    } else {
      Hxl = Hl;
      Hxl2 = Hl2;
    }
    third_contraction(*s, mt, x, lam.data(), u.data(), third.data());
    internal_forces(*s, mt, x, fm.data(), fb.data(), nullptr);
    Hm.matvec(u, Hu);
    Hb.matvec(u, Hu2);
    for (int i = 0; i < N; ++i) {
      const double Klam = -(Hl[i] + Hl2[i]);       // K~ lambda (matrix of the solve)
      const double Kxlam = -(Hxl[i] + Hxl2[i]);    // K lambda, exact force Jacobian
      const double vtot = av[i] + dt * ax[i];
      if (g_forces && force_mode == 0) g_forces[(size_t)t * N + i] = dt * lam[i];
      // parameters: dL/dp += lam^T (db/dp - dA/dp dv)
      gY += lam[i] * (dt * fm[i] - dt * dt * Hu[i]) / mt.Y;     // f_mem, K_mem linear in Y
      gkb += lam[i] * (dt * fb[i] - dt * dt * Hu2[i]) / mt.kb;  // f_bend, K_bend linear in kb
      grho += lam[i] * s->area3[i / 3] * (dt * gravity[i % 3] - dv[i]);
      ax[i] = ax[i] + dt * Kxlam - dt * dt * third[i] + dL_dx[(size_t)t * N + i];
      av[i] = vtot + dt * dt * Klam;  // adjoint of the step's starting velocity (= of v_t)
    }
    // air drag: b depends on w and on the starting velocity through f = c |d|_e d, A
    // through G(d); with q = h c (G lam - (dG/dd)[lam, dv]):  w_bar += q, v_bar -= q
    if (drag)
      for (int vi = 0; vi < s->n; ++vi) {
        if (s->pinned[vi]) continue;
        const double d[3] = {wind[0] - vst[3 * vi], wind[1] - vst[3 * vi + 1], wind[2] - vst[3 * vi + 2]};
        const double c = air_density * s->area3[vi];
        double G[9], T[3];
        drag_G(d, G);
        drag_dG(d, &lam[3 * vi], &dv[3 * vi], T);
        for (int a = 0; a < 3; ++a) {
          double Gl = 0.0;
          for (int q = 0; q < 3; ++q) Gl += G[3 * a + q] * lam[3 * vi + q];
          const double qa = dt * c * (Gl - T[a]);
          gw[a] += qa;
          av[3 * vi + a] -= qa;
        }
      }
    if (g_forces && force_mode == 1)
      for (int i = 0; i < N; ++i) g_forces[(size_t)t * N + i] = s->pinned[i / 3] ? 0.0 : av[i];

  }
  if (g_material) {
    g_material[0] = gY;
    g_material[1] = 0.0;
    g_material[2] = gkb;
    g_material[3] = grho;
  }
  if (g_wind)
    for (int a = 0; a < 3; ++a) g_wind[a] = gw[a];
  if (g_x0) std::copy(ax.begin(), ax.end(), g_x0);
  if (g_v0) std::copy(av.begin(), av.end(), g_v0);
  if (status) *status = worst;
  return OR_OK;
}

// Trajectory loss sum_{t=1..steps} sum_i |x_t^i - target_t^i|^2 and its gradient
// (dL/dx_0 = 0).  traj, target, grad: [steps+1][n][3].
double oracle_loss_l2(int n, int steps, const double* traj, const double* target, double* grad) {
  const size_t N = 3 * (size_t)n;
  double L = 0.0;
  if (grad) std::fill(grad, grad + N * (steps + 1), 0.0);
  for (int t = 1; t <= steps; ++t)
    for (size_t i = 0; i < N; ++i) {
      double d = traj[t * N + i] - target[t * N + i];
      L += d * d;
      if (grad) grad[t * N + i] = 2.0 * d;
    }
  return L;
}

// Pinhole reprojection loss.  Camera centre c = cam[1..3], focal cam[0] in px,
// looking along -z with camera axes (x, -y, -z): X_c = x - cx, Y_c = -(y - cy),
// Z_c = cz - z;  pi(x) = f (X_c / Z_c, Y_c / Z_c).  target_uv: [steps+1][n][2].
// L = sum_{t=1..steps} sum_i |pi(x_t^i) - uv_t^i|^2.  Returns NaN if any Z_c <= 0.
double oracle_loss_pinhole(int n, int steps, const double* cam, const double* traj, const double* target_uv, double* grad) {
  const double f = cam[0], cx = cam[1], cy = cam[2], cz = cam[3];
  double L = 0.0;
  if (grad) std::fill(grad, grad + 3 * (size_t)n * (steps + 1), 0.0);
  for (int t = 1; t <= steps; ++t)
    for (int i = 0; i < n; ++i) {
      const double* p = traj + ((size_t)t * n + i) * 3;
      double Xc = p[0] - cx, Yc = -(p[1] - cy), Zc = cz - p[2];
      if (!(Zc > 0.0)) return NAN;
      double u = f * Xc / Zc, w = f * Yc / Zc;
      const double* q = target_uv + ((size_t)t * n + i) * 2;
      double du = u - q[0], dw = w - q[1];
      L += du * du + dw * dw;
      if (grad) {
        double* gp = grad + ((size_t)t * n + i) * 3;
        // du/dx = f/Zc; dw/dy = -f/Zc; du/dz = f Xc / Zc^2; dw/dz = f Yc / Zc^2
        gp[0] = 2.0 * du * f / Zc;
        gp[1] = -2.0 * dw * f / Zc;
        gp[2] = 2.0 * (du * f * Xc + dw * f * Yc) / (Zc * Zc);
      }
    }
  return L;
}

}  // extern "C"
