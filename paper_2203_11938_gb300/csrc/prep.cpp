// Host-side mesh preparation (see prep.h).
#include "prep.h"

#include <algorithm>
#include <cmath>
#include <numeric>

#include "../../include/cloth_sim.h"

namespace cloth {
namespace {

struct HalfEdge {
  int lo, hi;    // undirected key
  int tri, k;    // triangle and local edge k: vertices (k, k+1 mod 3)
};

// Rest frame of a triangle: e1 along X1 - X0, e2 = unit normal x e1.
// Dm = [e1.(X1-X0) e1.(X2-X0); e2.(X1-X0) e2.(X2-X0)] (2x2), A0 = |det Dm|/2.
bool rest_frame(const double* X0, const double* X1, const double* X2, double* out5) {
  double a[3], b[3];
  for (int c = 0; c < 3; ++c) {
    a[c] = X1[c] - X0[c];
    b[c] = X2[c] - X0[c];
  }
  double nrm[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double ln = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
  if (!(la > 0.0) || !(ln > 1e-14 * la * la)) return false;
  double e1[3], nh[3], e2[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = a[c] / la;
    nh[c] = nrm[c] / ln;
  }
  e2[0] = nh[1] * e1[2] - nh[2] * e1[1];
  e2[1] = nh[2] * e1[0] - nh[0] * e1[2];
  e2[2] = nh[0] * e1[1] - nh[1] * e1[0];
  double m00 = 0, m01 = 0, m10 = 0, m11 = 0;
  for (int c = 0; c < 3; ++c) {
    m00 += e1[c] * a[c];
    m01 += e1[c] * b[c];
    m10 += e2[c] * a[c];
    m11 += e2[c] * b[c];
  }
  double det = m00 * m11 - m01 * m10;
  if (!(std::fabs(det) > 0.0)) return false;
  out5[0] = m11 / det;
  out5[1] = -m01 / det;
  out5[2] = -m10 / det;
  out5[3] = m00 / det;
  out5[4] = 0.5 * std::fabs(det);
  return true;
}

// Dihedral angle of hinge (p0, p1, pa, pb) with n1 = e x (pa - p0), n2 = (pb - p0) x e,
// theta = atan2((n1 x n2) . e/|e|, n1 . n2).
double rest_dihedral(const double* p0, const double* p1, const double* pa, const double* pb) {
  double e[3], u[3], w[3];
  for (int c = 0; c < 3; ++c) {
    e[c] = p1[c] - p0[c];
    u[c] = pa[c] - p0[c];
    w[c] = pb[c] - p0[c];
  }
  auto cross = [](const double* x, const double* y, double* z) {
    z[0] = x[1] * y[2] - x[2] * y[1];
    z[1] = x[2] * y[0] - x[0] * y[2];
    z[2] = x[0] * y[1] - x[1] * y[0];
  };
  double n1[3], n2[3], c12[3];
  cross(e, u, n1);
  cross(w, e, n2);
  cross(n1, n2, c12);
  double le = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  double s = (c12[0] * e[0] + c12[1] * e[1] + c12[2] * e[2]) / le;
  double co = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
  return std::atan2(s, co);
}

inline int upper_pair(int a, int b, int k) {  // a <= b
  return a * k - a * (a - 1) / 2 + (b - a);
}

}  // namespace

int build_mesh(const double* rest, int n, const int* tris, int m, const uint8_t* pinned, MeshData* out,
               std::string* err) {
  if (!rest || !tris || !out || n < 3 || m < 1) {
    *err = "mesh needs n >= 3 vertices, m >= 1 triangles and non-null arrays";
    return CLOTH_ERR_INVALID_ARG;
  }
  MeshData& d = *out;
  d.n = n;
  d.m = m;
  d.rest.assign(rest, rest + 3 * (size_t)n);
  d.tris.assign(tris, tris + 3 * (size_t)m);
  d.pinned.assign(n, 0);
  if (pinned)
    for (int i = 0; i < n; ++i) d.pinned[i] = pinned[i] ? 1 : 0;
  for (size_t i = 0; i < d.rest.size(); ++i)
    if (!std::isfinite(d.rest[i])) {
      *err = "non-finite rest position";
      return CLOTH_ERR_INVALID_ARG;
    }
  d.tri_rest.resize(5 * (size_t)m);
  d.tri_metric.resize(3 * (size_t)m);
  d.area3.assign(n, 0.0);
  for (int t = 0; t < m; ++t) {
    const int* v = &tris[3 * t];
    for (int a = 0; a < 3; ++a)
      if (v[a] < 0 || v[a] >= n) {
        *err = "triangle " + std::to_string(t) + " has a vertex index out of range";
        return CLOTH_ERR_INVALID_ARG;
      }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2] ||
        !rest_frame(&rest[3 * v[0]], &rest[3 * v[1]], &rest[3 * v[2]], &d.tri_rest[5 * (size_t)t])) {
      *err = "triangle " + std::to_string(t) + " has zero rest area";
      return CLOTH_ERR_DEGENERATE;
    }
    for (int a = 0; a < 3; ++a) d.area3[v[a]] += d.tri_rest[5 * (size_t)t + 4] / 3.0;
    double E1[3], E2[3];
    for (int c = 0; c < 3; ++c) {
      E1[c] = rest[3 * v[1] + c] - rest[3 * v[0] + c];
      E2[c] = rest[3 * v[2] + c] - rest[3 * v[0] + c];
    }
    d.tri_metric[3 * (size_t)t] = E1[0] * E1[0] + E1[1] * E1[1] + E1[2] * E1[2];
    d.tri_metric[3 * (size_t)t + 1] = E2[0] * E2[0] + E2[1] * E2[1] + E2[2] * E2[2];
    d.tri_metric[3 * (size_t)t + 2] = E1[0] * E2[0] + E1[1] * E2[1] + E1[2] * E2[2];
  }
  // Interior edges: sort the 3m half-edges by undirected key; a run of two is a hinge.
  std::vector<HalfEdge> he;
  he.reserve(3 * (size_t)m);
  for (int t = 0; t < m; ++t)
    for (int k = 0; k < 3; ++k) {
      int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
      he.push_back({std::min(a, b), std::max(a, b), t, k});
    }
  std::sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
    return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : x.tri < y.tri);
  });
  d.hinges.clear();
  d.hinge_rest.clear();
  for (size_t i = 0; i < he.size();) {
    size_t j = i;
    while (j < he.size() && he[j].lo == he[i].lo && he[j].hi == he[i].hi) ++j;
    if (j - i > 2) {
      *err = "edge shared by more than two triangles";
      return CLOTH_ERR_NONMANIFOLD;
    }
    if (j - i == 2) {
      const HalfEdge& A = he[i];
      const HalfEdge& B = he[i + 1];
      int e0 = tris[3 * A.tri + A.k], e1 = tris[3 * A.tri + (A.k + 1) % 3], wa = tris[3 * A.tri + (A.k + 2) % 3];
      int f0 = tris[3 * B.tri + B.k], f1 = tris[3 * B.tri + (B.k + 1) % 3], wb = tris[3 * B.tri + (B.k + 2) % 3];
      if (f0 != e1 || f1 != e0) {
        *err = "triangles sharing an edge have inconsistent winding";
        return CLOTH_ERR_NONMANIFOLD;
      }
      d.hinges.insert(d.hinges.end(), {e0, e1, wa, wb});
      double l2 = 0;
      for (int c = 0; c < 3; ++c) {
        double q = rest[3 * e1 + c] - rest[3 * e0 + c];
        l2 += q * q;
      }
      double w = 3.0 * l2 / (d.tri_rest[5 * (size_t)A.tri + 4] + d.tri_rest[5 * (size_t)B.tri + 4]);
      d.hinge_rest.push_back(w);
      d.hinge_rest.push_back(rest_dihedral(&rest[3 * e0], &rest[3 * e1], &rest[3 * wa], &rest[3 * wb]));
    }
    i = j;
  }
  return CLOTH_OK;
}

void build_layout(const std::vector<const MeshData*>& sheets, BatchLayout* Lp) {
  BatchLayout& L = *Lp;
  L = BatchLayout();
  L.S = (int)sheets.size();
  L.sheet_uoff.assign(L.S + 1, 0);
  L.sheet_voff.assign(L.S + 1, 0);
  L.sheet_toff.assign(L.S + 1, 0);
  L.sheet_hoff.assign(L.S + 1, 0);
  for (int s = 0; s < L.S; ++s) {
    const MeshData& d = *sheets[s];
    int npad = (d.n + kSlice - 1) / kSlice * kSlice;
    L.sheet_uoff[s + 1] = L.sheet_uoff[s] + d.n;
    L.sheet_voff[s + 1] = L.sheet_voff[s] + npad;
    L.sheet_toff[s + 1] = L.sheet_toff[s] + d.m;
    L.sheet_hoff[s + 1] = L.sheet_hoff[s] + d.num_hinges();
  }
  L.Nu = L.sheet_uoff[L.S];
  L.Np = L.sheet_voff[L.S];
  L.M = L.sheet_toff[L.S];
  L.E = L.sheet_hoff[L.S];
  L.i2u.assign(L.Np, -1);
  L.u2i.assign(L.Nu, -1);
  L.pinned.assign(L.Np, 1);
  L.rest.assign(3 * (size_t)L.Np, 0.0);
  L.area3.assign(L.Np, 0.0);
  L.vsheet.assign(L.Np, 0);
  L.usheet.assign(L.Nu, 0);
  L.tri_v.assign(3 * (size_t)L.M, 0);
  L.tri_sheet.assign(L.M, 0);
  L.tri_rest.assign(5 * (size_t)L.M, 0.0);
  L.tri_metric.assign(3 * (size_t)L.M, 0.0);
  L.hin_v.assign(4 * (size_t)L.E, 0);
  L.hin_sheet.assign(L.E, 0);
  L.hin_rest.assign(2 * (size_t)L.E, 0.0);

  // per internal row: sorted neighbour list (diagonal first)
  std::vector<std::vector<int>> rowcols(L.Np);
  for (int s = 0; s < L.S; ++s) {
    const MeshData& d = *sheets[s];
    const int ne = d.num_hinges();
    // block pattern in local user ids
    std::vector<std::vector<int>> nb(d.n);
    for (int i = 0; i < d.n; ++i) nb[i].push_back(i);
    auto couple = [&](int a, int b) {
      nb[a].push_back(b);
      nb[b].push_back(a);
    };
    for (int t = 0; t < d.m; ++t) {
      const int* v = &d.tris[3 * t];
      couple(v[0], v[1]);
      couple(v[1], v[2]);
      couple(v[0], v[2]);
    }
    for (int e = 0; e < ne; ++e) couple(d.hinges[4 * e + 2], d.hinges[4 * e + 3]);
    std::vector<int> cnt(d.n);
    for (int i = 0; i < d.n; ++i) {
      std::sort(nb[i].begin(), nb[i].end());
      nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
      cnt[i] = (int)nb[i].size();
    }
    // internal order: block count descending, stable (keeps slices homogeneous)
    std::vector<int> order(d.n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] > cnt[b]; });
    std::vector<int> loc2int(d.n);
    const int voff = L.sheet_voff[s], uoff = L.sheet_uoff[s];
    for (int r = 0; r < d.n; ++r) loc2int[order[r]] = voff + r;
    for (int u = 0; u < d.n; ++u) {
      int i = loc2int[u];
      L.i2u[i] = uoff + u;
      L.u2i[uoff + u] = i;
      L.pinned[i] = d.pinned[u];
      L.area3[i] = d.area3[u];
      for (int c = 0; c < 3; ++c) L.rest[3 * (size_t)i + c] = d.rest[3 * (size_t)u + c];
      L.usheet[uoff + u] = s;
      std::vector<int>& rc = rowcols[i];
      rc.push_back(i);
      std::vector<int> others;
      for (int j : nb[u])
        if (j != u) others.push_back(loc2int[j]);
      std::sort(others.begin(), others.end());
      rc.insert(rc.end(), others.begin(), others.end());
    }
    for (int i = voff; i < L.sheet_voff[s + 1]; ++i) {
      L.vsheet[i] = s;
      if (L.i2u[i] < 0) rowcols[i].push_back(i);  // padding row: diagonal only
    }
    const int toff = L.sheet_toff[s], hoff = L.sheet_hoff[s];
    for (int t = 0; t < d.m; ++t) {
      for (int a = 0; a < 3; ++a) L.tri_v[(size_t)a * L.M + toff + t] = loc2int[d.tris[3 * t + a]];
      for (int q = 0; q < 5; ++q) L.tri_rest[(size_t)q * L.M + toff + t] = d.tri_rest[5 * (size_t)t + q];
      for (int q = 0; q < 3; ++q) L.tri_metric[(size_t)q * L.M + toff + t] = d.tri_metric[3 * (size_t)t + q];
      L.tri_sheet[toff + t] = s;
    }
    for (int e = 0; e < ne; ++e) {
      for (int a = 0; a < 4; ++a) L.hin_v[(size_t)a * L.E + hoff + e] = loc2int[d.hinges[4 * e + a]];
      for (int q = 0; q < 2; ++q) L.hin_rest[(size_t)q * L.E + hoff + e] = d.hinge_rest[2 * (size_t)e + q];
      L.hin_sheet[hoff + e] = s;
    }
  }

  // SELL-32 slices
  L.nslices = L.Np / kSlice;
  L.slice_K.assign(L.nslices, 0);
  L.slice_base.assign(L.nslices + 1, 0);
  for (int sl = 0; sl < L.nslices; ++sl) {
    int K = 0;
    for (int r = 0; r < kSlice; ++r) K = std::max(K, (int)rowcols[sl * kSlice + r].size());
    L.slice_K[sl] = K;
    L.slice_base[sl + 1] = L.slice_base[sl] + K;
  }
  const size_t nent = (size_t)L.slice_base[L.nslices] * kSlice;
  L.cols.assign(nent, 0);
  // entry lookup per row: column -> entry index
  std::vector<std::vector<std::pair<int, int>>> rowent(L.Np);
  for (int sl = 0; sl < L.nslices; ++sl)
    for (int r = 0; r < kSlice; ++r) {
      int i = sl * kSlice + r;
      const std::vector<int>& rc = rowcols[i];
      for (int k = 0; k < L.slice_K[sl]; ++k) {
        size_t ent = ((size_t)L.slice_base[sl] + k) * kSlice + r;
        int col = k < (int)rc.size() ? rc[k] : i;
        L.cols[ent] = col;
        if (k < (int)rc.size()) rowent[i].push_back({col, (int)ent});
      }
      std::sort(rowent[i].begin(), rowent[i].end());
    }
  auto entry_of = [&](int i, int j) {
    const auto& v = rowent[i];
    auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(j, -1));
    return it->second;  // the pattern contains every coupled pair by construction
  };
  // contributor lists: counting pass, then fill
  std::vector<int> count(nent + 1, 0);
  auto visit = [&](auto&& fn) {
    for (int t = 0; t < L.M; ++t) {
      int v[3];
      for (int a = 0; a < 3; ++a) v[a] = L.tri_v[(size_t)a * L.M + t];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          int blk = a <= b ? 6 * t + upper_pair(a, b, 3) : 6 * t + upper_pair(b, a, 3);
          fn(entry_of(v[a], v[b]), (blk << 1) | (a > b ? 1 : 0));
        }
    }
    for (int e = 0; e < L.E; ++e) {
      int v[4];
      for (int a = 0; a < 4; ++a) v[a] = L.hin_v[(size_t)a * L.E + e];
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          int base = 6 * L.M + 10 * e;
          int blk = a <= b ? base + upper_pair(a, b, 4) : base + upper_pair(b, a, 4);
          fn(entry_of(v[a], v[b]), (blk << 1) | (a > b ? 1 : 0));
        }
    }
  };
  visit([&](int ent, int) { count[ent + 1]++; });
  for (size_t i = 0; i < nent; ++i) count[i + 1] += count[i];
  L.contrib_ptr = count;
  L.contrib.assign(count[nent], 0);
  std::vector<int> fill(count.begin(), count.end() - 1);
  visit([&](int ent, int code) { L.contrib[fill[ent]++] = code; });
  // keep each list in ascending code order (fixed summation order)
  for (size_t i = 0; i < nent; ++i) std::sort(L.contrib.begin() + L.contrib_ptr[i], L.contrib.begin() + L.contrib_ptr[i + 1]);

  // per-vertex force slots
  std::vector<int> vc(L.Np + 1, 0);
  for (int t = 0; t < L.M; ++t)
    for (int a = 0; a < 3; ++a) vc[L.tri_v[(size_t)a * L.M + t] + 1]++;
  for (int e = 0; e < L.E; ++e)
    for (int a = 0; a < 4; ++a) vc[L.hin_v[(size_t)a * L.E + e] + 1]++;
  for (int i = 0; i < L.Np; ++i) vc[i + 1] += vc[i];
  L.vf_ptr = vc;
  L.vf.assign(vc[L.Np], 0);
  std::vector<int> vfill(vc.begin(), vc.end() - 1);
  for (int t = 0; t < L.M; ++t)
    for (int a = 0; a < 3; ++a) L.vf[vfill[L.tri_v[(size_t)a * L.M + t]]++] = 3 * t + a;
  for (int e = 0; e < L.E; ++e)
    for (int a = 0; a < 4; ++a) L.vf[vfill[L.hin_v[(size_t)a * L.E + e]]++] = 3 * L.M + 4 * e + a;

  // work table
  L.sheet_wfirst.assign(L.S + 1, 0);
  for (int s = 0; s < L.S; ++s) {
    int r0 = L.sheet_voff[s], r1 = L.sheet_voff[s + 1];
    int nb = 0;
    for (int r = r0; r < r1; r += kRowsPerBlock) {
      L.work_sheet.push_back(s);
      L.work_row0.push_back(r);
      L.work_rows.push_back(std::min(kRowsPerBlock, r1 - r));
      ++nb;
    }
    L.sheet_wfirst[s + 1] = L.sheet_wfirst[s] + nb;
    L.max_sheet_blocks = std::max(L.max_sheet_blocks, nb);
  }
}

}  // namespace cloth
