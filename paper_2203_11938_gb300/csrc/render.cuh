// Soft rasteriser of the textured sheet and the image energies of phi-SfT (Sec. 3.2):
// per-pixel math, compiled for the device and (for host-side tests of this same code)
// for the host.
//
// Image of W x H pixels, pixel centres at (u + 1/2, v + 1/2); a vertex x projects to
// (W/2 + f (x - cx)/(cz - z), H/2 - f (y - cy)/(cz - z)) (the tracking loss's pinhole
// with the principal point at the image centre).  Triangle j, projected corners a, b, c:
//   coverage      D_j(p) = sigmoid(+-d^2 / SIGMA_R), d = distance of p to the nearest
//                 edge segment, + inside (all barycentric coordinates >= 0), - outside;
//   silhouette    A(p) = 1 - prod_j (1 - D_j(p));
//   colour        texture sampled (bilinear, texel centres at (k + 1/2)/size, clamped) at
//                 the uv interpolated with the clamped, renormalised barycentric
//                 coordinates of p; blended with weights D_j exp(zn_j / GAMMA) against a
//                 black background of weight exp(EPS / GAMMA), zn_j the normalised inverse
//                 depth (1 at Z_NEAR, 0 at Z_FAR) interpolated the same way, evaluated
//                 relative to the largest exponent (zn_j / GAMMA + log D_j, EPS / GAMMA);
//   energies      E_p = sum |I - I_hat|_1,  E_s = sum |G(A) - G(B_hat)|_1, G the Gaussian
//                 of SIGMA_S px truncated at 3 SIGMA_S with zero padding; E = E_p + LAMBDA E_s.
// The backward pass differentiates these definitions with respect to the vertex positions
// (the texture and the inputs are constants).
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define RS_HD __host__ __device__ __forceinline__
#else
#define RS_HD inline
#endif

namespace cloth {
namespace render {

constexpr double SIGMA_R = 1.0;   // px^2
constexpr double GAMMA = 1e-4;
constexpr double EPS = 1e-3;
constexpr double Z_NEAR = 0.5, Z_FAR = 5.0;
constexpr double SIGMA_S = 7.0;   // px
constexpr double LAMBDA = 0.5;
constexpr int MAX_TEX = 1 << 24;  // texels

struct P2 {
  double x, y;
};
RS_HD P2 sub2(P2 a, P2 b) { return {a.x - b.x, a.y - b.y}; }
RS_HD double dot2(P2 a, P2 b) { return a.x * b.x + a.y * b.y; }
RS_HD double cross2(P2 a, P2 b) { return a.x * b.y - a.y * b.x; }

struct Camera {
  double f, cx, cy, cz;
  int W, H;
};

// image point and inverse depth of a vertex; J: d(px, py, inv)/d(x, y, z), row-major 3x3
// A vertex at or behind the camera (depth <= 0) gets NaN image point, inverse depth and
// Jacobian, so the frame's energy and gradient come out NaN (as the tracking loss does).
RS_HD void project(const Camera& c, const double* x, P2* q, double* inv, double* J) {
  const double dep = c.cz - x[2], id = dep > 0.0 ? 1.0 / dep : NAN;
  q->x = 0.5 * c.W + c.f * (x[0] - c.cx) * id;
  q->y = 0.5 * c.H - c.f * (x[1] - c.cy) * id;
  *inv = id;
  if (J) {
    J[0] = c.f * id;  J[1] = 0.0;         J[2] = c.f * (x[0] - c.cx) * id * id;
    J[3] = 0.0;       J[4] = -c.f * id;   J[5] = -c.f * (x[1] - c.cy) * id * id;
    J[6] = 0.0;       J[7] = 0.0;         J[8] = id * id;
  }
}

// squared distance of p to the segment a-b
RS_HD double seg_d2(P2 p, P2 a, P2 b) {
  const P2 e = sub2(b, a), u = sub2(p, a);
  double t = dot2(u, e) / dot2(e, e);
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const P2 r = {u.x - t * e.x, u.y - t * e.y};
  return dot2(r, r);
}

// gradient of seg_d2 with respect to a and b (g: scale)
RS_HD void seg_d2_grad(P2 p, P2 a, P2 b, double g, P2* ga, P2* gb) {
  const P2 e = sub2(b, a), u = sub2(p, a);
  const double ee = dot2(e, e), t = dot2(u, e) / ee;
  if (t <= 0.0) {  // nearest point a: d2 = |p - a|^2
    ga->x += -2.0 * u.x * g;
    ga->y += -2.0 * u.y * g;
  } else if (t >= 1.0) {  // nearest point b
    const P2 w = sub2(p, b);
    gb->x += -2.0 * w.x * g;
    gb->y += -2.0 * w.y * g;
  } else {  // d2 = u.u - t (u.e): dd2/du = 2u - 2t e, dd2/de = -2t u + 2t^2 e
    const P2 du = {2.0 * u.x - 2.0 * t * e.x, 2.0 * u.y - 2.0 * t * e.y};
    const P2 de = {-2.0 * t * u.x + 2.0 * t * t * e.x, -2.0 * t * u.y + 2.0 * t * t * e.y};
    ga->x += (-du.x - de.x) * g;
    ga->y += (-du.y - de.y) * g;
    gb->x += de.x * g;
    gb->y += de.y * g;
  }
}

// bilinear texture sample (tex [Ht][Wt][3]) at (u, v); dC/du, dC/dv when wanted
RS_HD void sample(const double* tex, int Wt, int Ht, double u, double v, double* C, double* dCdu, double* dCdv) {
  double x = u * Wt - 0.5, y = v * Ht - 0.5;
  const bool cx = !(x >= 0.0 && x <= Wt - 1.0), cy = !(y >= 0.0 && y <= Ht - 1.0);  // clamped: no gradient
  // written so that a NaN coordinate (degenerate projected triangle) clamps to texel 0
  // and never reaches the integer conversion
  x = !(x >= 0.0) ? 0.0 : (x > Wt - 1.0 ? Wt - 1.0 : x);
  y = !(y >= 0.0) ? 0.0 : (y > Ht - 1.0 ? Ht - 1.0 : y);
  int x0 = (int)floor(x), y0 = (int)floor(y);
  const int xm = Wt > 1 ? Wt - 2 : 0, ym = Ht > 1 ? Ht - 2 : 0;
  x0 = x0 > xm ? xm : x0;
  y0 = y0 > ym ? ym : y0;
  const int x1 = x0 + 1 > Wt - 1 ? Wt - 1 : x0 + 1, y1 = y0 + 1 > Ht - 1 ? Ht - 1 : y0 + 1;
  const double fx = x - x0, fy = y - y0;
  const double* t00 = tex + 3 * ((size_t)y0 * Wt + x0);
  const double* t01 = tex + 3 * ((size_t)y0 * Wt + x1);
  const double* t10 = tex + 3 * ((size_t)y1 * Wt + x0);
  const double* t11 = tex + 3 * ((size_t)y1 * Wt + x1);
  for (int k = 0; k < 3; ++k) {
    C[k] = (1 - fx) * (1 - fy) * t00[k] + fx * (1 - fy) * t01[k] + (1 - fx) * fy * t10[k] + fx * fy * t11[k];
    if (dCdu) dCdu[k] = cx ? 0.0 : Wt * ((1 - fy) * (t01[k] - t00[k]) + fy * (t11[k] - t10[k]));
    if (dCdv) dCdv[k] = cy ? 0.0 : Ht * ((1 - fx) * (t10[k] - t00[k]) + fx * (t11[k] - t01[k]));
  }
}

RS_HD double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }
// log sigmoid(z), without overflow or cancellation on either side
RS_HD double log_sigmoid(double z) { return z >= 0.0 ? -log1p(exp(-z)) : z - log1p(exp(z)); }

// Everything one triangle contributes at one pixel.
struct TriPix {
  double D, zn, C[3];
  double s;        // signed sigmoid argument +-d^2 / SIGMA_R (D = sigmoid(s))
  double logw;     // zn / GAMMA + log D: the log of the triangle's colour weight
  double lam[3];   // barycentric coordinates (unclamped)
  double lc[3];    // clamped, renormalised
  double msum;     // sum of the clamped coordinates
  int edge;        // nearest edge (0: a-b, 1: b-c, 2: c-a)
  bool inside;
};

RS_HD double zn_scale() { return 1.0 / (1.0 / Z_NEAR - 1.0 / Z_FAR); }

RS_HD void tri_pixel(P2 p, const P2* q, const double* inv, const double* uv, const double* tex, int Wt, int Ht,
                     TriPix* o) {
  const P2 a = q[0], b = q[1], c = q[2];
  const double area = cross2(sub2(b, a), sub2(c, a));
  o->lam[0] = cross2(sub2(b, p), sub2(c, p)) / area;
  o->lam[1] = cross2(sub2(c, p), sub2(a, p)) / area;
  o->lam[2] = cross2(sub2(a, p), sub2(b, p)) / area;
  o->inside = o->lam[0] >= 0.0 && o->lam[1] >= 0.0 && o->lam[2] >= 0.0;
  const double d0 = seg_d2(p, a, b), d1 = seg_d2(p, b, c), d2 = seg_d2(p, c, a);
  double d = d0;
  o->edge = 0;
  if (d1 < d) d = d1, o->edge = 1;
  if (d2 < d) d = d2, o->edge = 2;
  o->s = (o->inside ? d : -d) / SIGMA_R;
  o->D = sigmoid(o->s);
  double m[3], s = 0.0;
  for (int k = 0; k < 3; ++k) {
    m[k] = o->lam[k] > 0.0 ? o->lam[k] : 0.0;
    s += m[k];
  }
  o->msum = s;
  double zsum = 0.0, u = 0.0, v = 0.0;
  for (int k = 0; k < 3; ++k) {
    o->lc[k] = m[k] / s;
    zsum += o->lc[k] * inv[k];
    u += o->lc[k] * uv[2 * k];
    v += o->lc[k] * uv[2 * k + 1];
  }
  o->zn = (zsum - 1.0 / Z_FAR) * zn_scale();
  o->logw = o->zn / GAMMA + log_sigmoid(o->s);
  sample(tex, Wt, Ht, u, v, o->C, nullptr, nullptr);
}

// Backward of one triangle at one pixel: given dE/ds (s the signed sigmoid argument),
// dE/dzn and dE/dC, accumulate dE/d(corner image points) gq[3] and dE/d(corner inverse
// depths) ginv[3].
RS_HD void tri_pixel_backward(P2 p, const P2* q, const double* inv, const double* uv, const double* tex, int Wt,
                              int Ht, const TriPix& t, double gs, double gzn, const double* gC, P2* gq,
                              double* ginv) {
  // s = +-d^2 / SIGMA_R
  const double gd2 = gs * (t.inside ? 1.0 : -1.0) / SIGMA_R;
  const int e0 = t.edge, e1 = (t.edge + 1) % 3;
  seg_d2_grad(p, q[e0], q[e1], gd2, &gq[e0], &gq[e1]);
  // zn and the texture coordinates through the clamped barycentric coordinates
  double u = 0.0, v = 0.0;
  for (int k = 0; k < 3; ++k) {
    u += t.lc[k] * uv[2 * k];
    v += t.lc[k] * uv[2 * k + 1];
  }
  double Cs[3], dCdu[3], dCdv[3];
  sample(tex, Wt, Ht, u, v, Cs, dCdu, dCdv);
  const double gu = gC[0] * dCdu[0] + gC[1] * dCdu[1] + gC[2] * dCdu[2];
  const double gv = gC[0] * dCdv[0] + gC[1] * dCdv[1] + gC[2] * dCdv[2];
  double glc[3];
  for (int k = 0; k < 3; ++k) {
    glc[k] = gzn * zn_scale() * inv[k] + gu * uv[2 * k] + gv * uv[2 * k + 1];
    ginv[k] += gzn * zn_scale() * t.lc[k];
  }
  // lc_k = m_k / sum m,  m = max(lam, 0)
  double glam[3];
  double dot = 0.0;
  for (int k = 0; k < 3; ++k) dot += glc[k] * t.lc[k];
  for (int k = 0; k < 3; ++k) glam[k] = t.lam[k] >= 0.0 ? (glc[k] - dot) / t.msum : 0.0;
  // lam_0 = cross(b - p, c - p) / area (cyclic), area = cross(b - a, c - a)
  const P2 a = q[0], b = q[1], c = q[2];
  const double area = cross2(sub2(b, a), sub2(c, a));
  const P2 pa = sub2(a, p), pb = sub2(b, p), pc = sub2(c, p);
  // numerators n0 = cross(pb, pc), n1 = cross(pc, pa), n2 = cross(pa, pb); lam_k = n_k / area
  // dn/d(first) = (second.y, -second.x), dn/d(second) = (-first.y, first.x)
  const double g0 = glam[0] / area, g1 = glam[1] / area, g2 = glam[2] / area;
  const double garea = -(glam[0] * t.lam[0] + glam[1] * t.lam[1] + glam[2] * t.lam[2]) / area;
  gq[1].x += g0 * pc.y;   gq[1].y += -g0 * pc.x;    // n0 wrt b
  gq[2].x += -g0 * pb.y;  gq[2].y += g0 * pb.x;     // n0 wrt c
  gq[2].x += g1 * pa.y;   gq[2].y += -g1 * pa.x;    // n1 wrt c
  gq[0].x += -g1 * pc.y;  gq[0].y += g1 * pc.x;     // n1 wrt a
  gq[0].x += g2 * pb.y;   gq[0].y += -g2 * pb.x;    // n2 wrt a
  gq[1].x += -g2 * pa.y;  gq[1].y += g2 * pa.x;     // n2 wrt b
  // area = cross(b - a, c - a): d/db = ((c-a).y, -(c-a).x), d/dc = (-(b-a).y, (b-a).x), d/da = -(d/db + d/dc)
  // (garea is zero up to rounding: the renormalised coordinates do not change when all
  // three are scaled together; kept as the exact derivative of lam)
  const P2 ba = sub2(b, a), ca = sub2(c, a);
  const P2 dab = {ca.y, -ca.x}, dac = {-ba.y, ba.x};
  gq[1].x += garea * dab.x;  gq[1].y += garea * dab.y;
  gq[2].x += garea * dac.x;  gq[2].y += garea * dac.y;
  gq[0].x -= garea * (dab.x + dac.x);
  gq[0].y -= garea * (dab.y + dac.y);
}

// ---------------------------------------------------------------- one pixel
// A projected triangle as the per-pixel functions read it: corner image points, inverse
// depths and texture coordinates.
struct TriRec {
  P2 q[3];
  double inv[3], uv[6];
};

// Projected corners of every triangle: q [n] image points, inv [n] inverse depths.
struct Scene {
  const int* tris;    // [m][3]
  int m;
  const P2* q;        // [n]
  const double* inv;  // [n]
  const double* uv;   // [n][2]
  const double* tex;  // [Ht][Wt][3]
  int Wt, Ht;
};

RS_HD TriRec corners(const Scene& s, int j) {
  TriRec r;
  for (int k = 0; k < 3; ++k) {
    const int v = s.tris[3 * j + k];
    r.q[k] = s.q[v];
    r.inv[k] = s.inv[v];
    r.uv[2 * k] = s.uv[2 * v];
    r.uv[2 * k + 1] = s.uv[2 * v + 1];
  }
  return r;
}

// Screen-space reach of a triangle: beyond R from its bounding box it contributes exactly
// nothing to any pixel.  There d^2 > R^2 >= 750 SIGMA_R, so exp(d^2 / SIGMA_R) overflows and
// its coverage D is exactly 0 (its silhouette factor 1 - D exactly 1), and its colour
// exponent zn / GAMMA + log D <= zn_max / GAMMA - d^2 / SIGMA_R < EPS / GAMMA - 746 lies more
// than 746 below the blend's largest exponent, so its weight exp(.) underflows to exactly 0.
// A triangle with a non-finite corner reaches everywhere (its NaN must reach the energy).
struct TriReach {
  double x0, y0, x1, y1, r2;  // bounding box of the corners, R^2
  bool all;
};
RS_HD TriReach tri_reach(const TriRec& t) {
  TriReach b;
  b.x0 = fmin(t.q[0].x, fmin(t.q[1].x, t.q[2].x));
  b.x1 = fmax(t.q[0].x, fmax(t.q[1].x, t.q[2].x));
  b.y0 = fmin(t.q[0].y, fmin(t.q[1].y, t.q[2].y));
  b.y1 = fmax(t.q[0].y, fmax(t.q[1].y, t.q[2].y));
  const double zmax = (fmax(t.inv[0], fmax(t.inv[1], t.inv[2])) - 1.0 / Z_FAR) * zn_scale();
  b.r2 = SIGMA_R * (fmax(zmax - EPS, 0.0) / GAMMA + 750.0);
  // x - x is 0 exactly for finite x and NaN for infinities and NaNs
  bool fin = true;
  for (int k = 0; k < 3; ++k) fin = fin && t.q[k].x - t.q[k].x == 0.0 && t.q[k].y - t.q[k].y == 0.0 &&
                                    t.inv[k] - t.inv[k] == 0.0;
  b.all = !fin;
  return b;
}
// true when the triangle may touch a pixel centre in [ax, bx] x [ay, by]
RS_HD bool reaches(const TriReach& b, double ax, double ay, double bx, double by) {
  if (b.all) return true;
  const double dx = fmax(0.0, fmax(b.x0 - bx, ax - b.x1)), dy = fmax(0.0, fmax(b.y0 - by, ay - b.y1));
  return dx * dx + dy * dy <= b.r2;
}

// Per-pixel passes over the triangles (each called for the triangles in ascending order):
// 1. the largest colour exponent, starting from EPS / GAMMA
RS_HD void pass_top(P2 p, const TriRec& r, const double* tex, int Wt, int Ht, double* top) {
  TriPix t;
  tri_pixel(p, r.q, r.inv, r.uv, tex, Wt, Ht, &t);
  *top = t.logw > *top ? t.logw : *top;
}
// 2. the blend's denominator S, numerator acc[3] and the silhouette's product of (1 - D)
//    (forward), or of its non-zero factors with the count of zero factors (backward)
struct PixAcc {
  double S, acc[3], prod;
  int zeros;
};
RS_HD PixAcc pix_acc_begin(double top) { return {exp(EPS / GAMMA - top), {0.0, 0.0, 0.0}, 1.0, 0}; }
RS_HD void pass_acc(P2 p, const TriRec& r, const double* tex, int Wt, int Ht, double top, bool split_zeros,
                    PixAcc* a) {
  TriPix t;
  tri_pixel(p, r.q, r.inv, r.uv, tex, Wt, Ht, &t);
  const double w = exp(t.logw - top);
  a->S += w;
  for (int k = 0; k < 3; ++k) a->acc[k] += w * t.C[k];
  if (split_zeros && 1.0 - t.D == 0.0) ++a->zeros;
  else a->prod *= 1.0 - t.D;
}

// 3. (backward) one triangle's share of dE/d(corner image points) gq[3] and dE/d(corner
//    inverse depths) ginv[3], given dE/dI gI[3], dE/dA gA and the pixel's I = acc / S;
//    returns false (and leaves gq, ginv at 0) where the share is exactly 0 (weight and
//    coverage both underflowed)
RS_HD bool pass_grad(P2 p, const TriRec& r, const double* tex, int Wt, int Ht, double top, const PixAcc& a,
                     const double* I, const double* gI, double gA, P2* gq, double* ginv) {
  TriPix t;
  tri_pixel(p, r.q, r.inv, r.uv, tex, Wt, Ht, &t);
  const double w = exp(t.logw - top);
  for (int k = 0; k < 3; ++k) {
    gq[k] = {0.0, 0.0};
    ginv[k] = 0.0;
  }
  if (w == 0.0 && t.D == 0.0) return false;
  const double S = a.S;
  const double gw = (gI[0] * (t.C[0] - I[0]) + gI[1] * (t.C[1] - I[1]) + gI[2] * (t.C[2] - I[2])) / S;
  const double gC[3] = {gI[0] * w / S, gI[1] * w / S, gI[2] * w / S};
  const double om = 1.0 - t.D;
  const double others = om == 0.0 ? (a.zeros == 1 ? a.prod : 0.0) : (a.zeros == 0 ? a.prod / om : 0.0);
  // dw/ds = w (1 - D) (d log sigmoid(s) / ds = 1 - D), dA/ds = others D (1 - D), dw/dzn = w / GAMMA
  const double gs = (gw * w + gA * others * t.D) * om;
  const double gzn = gw * w / GAMMA;
  tri_pixel_backward(p, r.q, r.inv, r.uv, tex, Wt, Ht, t, gs, gzn, gC, gq, ginv);
  return true;
}

// Colour I[3] and silhouette A of the pixel centre p over every triangle.
// The colour weights w_j = D_j exp(zn_j / GAMMA) and the background's exp(EPS / GAMMA) are
// evaluated relative to the largest of their exponents (zn_j / GAMMA + log D_j and
// EPS / GAMMA), so a pixel where every D_j underflows keeps the background's weight 1.
RS_HD void pixel_forward(const Scene& s, P2 p, double* I, double* A) {
  double top = EPS / GAMMA;
  for (int j = 0; j < s.m; ++j) pass_top(p, corners(s, j), s.tex, s.Wt, s.Ht, &top);
  PixAcc a = pix_acc_begin(top);
  for (int j = 0; j < s.m; ++j) pass_acc(p, corners(s, j), s.tex, s.Wt, s.Ht, top, false, &a);
  for (int k = 0; k < 3; ++k) I[k] = a.acc[k] / a.S;
  *A = 1.0 - a.prod;
}

// Backward at one pixel: gI[3] = dE/dI, gA = dE/dA; add(v, gqx, gqy, ginv) receives the
// gradient with respect to vertex v's image point and inverse depth.
template <class Add>
RS_HD void pixel_backward(const Scene& s, P2 p, const double* gI, double gA, Add add) {
  double top = EPS / GAMMA;
  for (int j = 0; j < s.m; ++j) pass_top(p, corners(s, j), s.tex, s.Wt, s.Ht, &top);
  PixAcc a = pix_acc_begin(top);
  for (int j = 0; j < s.m; ++j) pass_acc(p, corners(s, j), s.tex, s.Wt, s.Ht, top, true, &a);
  const double I[3] = {a.acc[0] / a.S, a.acc[1] / a.S, a.acc[2] / a.S};
  // per triangle (the largest exponent cancels in I: no gradient through it)
  for (int j = 0; j < s.m; ++j) {
    P2 gq[3];
    double ginv[3];
    if (!pass_grad(p, corners(s, j), s.tex, s.Wt, s.Ht, top, a, I, gI, gA, gq, ginv)) continue;
    for (int k = 0; k < 3; ++k) add(s.tris[3 * j + k], gq[k].x, gq[k].y, ginv[k]);
  }
}

// Gaussian filter taps: weight of offset k in [-r, r], r = ceil(3 SIGMA_S)
RS_HD int blur_radius() { return (int)ceil(3.0 * SIGMA_S); }
RS_HD double blur_norm() {
  const int r = blur_radius();
  double z = 0.0;
  for (int k = -r; k <= r; ++k) z += exp(-0.5 * (k / SIGMA_S) * (k / SIGMA_S));
  return z;
}
RS_HD double blur_tap(int k, double norm) { return exp(-0.5 * (k / SIGMA_S) * (k / SIGMA_S)) / norm; }

}  // namespace render
}  // namespace cloth
