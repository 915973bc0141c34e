// Host-side mesh preparation for the cloth step kernels.
//
// Turns each sheet's template mesh S_1 (phi-SfT Sec. 3.1: fixed topology, per-vertex
// state) into the flat arrays the kernels read: interior-edge hinges, rest-frame data,
// lumped areas, an internal vertex order, the 3x3-block SELL-32 pattern of the step
// matrix A = M - h^2 K (Eq. 4-5) and, for every block, the list of element Hessian
// blocks that sum into it (assembly without atomics).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace cloth {

// One validated sheet.
struct MeshData {
  int n = 0, m = 0;
  std::vector<double> rest;        // [n][3]
  std::vector<int> tris;           // [m][3]
  std::vector<uint8_t> pinned;     // [n]
  std::vector<int> hinges;         // [e][4]: edge (e0, e1), wing of the first triangle, wing of the second
  std::vector<double> tri_rest;    // [m][5]: Dm^{-1} row-major (4), rest area A0
  std::vector<double> tri_metric;  // [m][3]: rest metric E1.E1, E2.E2, E1.E2 of the edges E1 = X1-X0, E2 = X2-X0
  std::vector<double> hinge_rest;  // [e][2]: w_e = 3|e|^2/(A1+A2), rest dihedral angle
  std::vector<double> area3;       // [n]: sum over incident triangles of A0/3 (mass per unit density)
  int num_hinges() const { return (int)hinges.size() / 4; }
};

// Returns 0 or a negative CLOTH_ERR_* code with a message in *err.
int build_mesh(const double* rest, int n, const int* tris, int m, const uint8_t* pinned, MeshData* out,
               std::string* err);

constexpr int kSlice = 32;       // rows per SELL slice (one warp)
constexpr int kRowsPerBlock = 256;  // rows per work-table entry (one CTA of the row kernels)

// Concatenated layout of a batch (all vertex ids are internal unless noted).
struct BatchLayout {
  int S = 0;   // sheets
  int Nu = 0;  // user vertices (packed)
  int Np = 0;  // internal vertices (each sheet padded to a multiple of kSlice)
  int M = 0, E = 0;  // triangles, hinges
  std::vector<int> sheet_uoff, sheet_voff, sheet_toff, sheet_hoff;  // [S+1]
  std::vector<int> i2u;            // [Np] internal -> user index, -1 for padding
  std::vector<int> u2i;            // [Nu]
  std::vector<uint8_t> pinned;     // [Np] padding rows count as pinned
  std::vector<double> rest;        // [Np][3] rest positions (0 for padding rows)
  std::vector<double> area3;       // [Np]
  std::vector<int> vsheet;         // [Np]
  std::vector<int> usheet;         // [Nu] sheet of each user vertex
  // elements, structure of arrays
  std::vector<int> tri_v;          // [3][M]
  std::vector<int> tri_sheet;      // [M]
  std::vector<double> tri_rest;    // [5][M]
  std::vector<double> tri_metric;  // [3][M]
  std::vector<int> hin_v;          // [4][E]
  std::vector<int> hin_sheet;      // [E]
  std::vector<double> hin_rest;    // [2][E]
  // SELL-32 block pattern: slice s covers internal rows [32 s, 32 s + 32) and has
  // slice_K[s] slots; block (slot k, lane r) of slice s has entry index
  // (slice_base[s] + k) * 32 + r into `cols` and `contrib_ptr`.
  int nslices = 0;
  std::vector<int> slice_base;     // [nslices + 1] cumulative slot count
  std::vector<int> slice_K;        // [nslices]
  std::vector<int> cols;           // [slots * 32] column vertex (self for padding slots)
  std::vector<int> contrib_ptr;    // [slots * 32 + 1]
  std::vector<int> contrib;        // element Hessian block id << 1 | transpose
  // per-vertex force contributions: element-vertex slot ids
  std::vector<int> vf_ptr;         // [Np + 1]
  std::vector<int> vf;
  // row work table: entry w covers rows [work_row0[w], work_row0[w] + work_rows[w]) of work_sheet[w]
  std::vector<int> work_sheet, work_row0, work_rows;
  std::vector<int> sheet_wfirst;   // [S + 1]
  int max_sheet_blocks = 0;
  long long total_slots() const { return slice_base.empty() ? 0 : slice_base.back(); }
};

// Element Hessian block ids: triangle t, upper pair p (0..5) -> 6 t + p;
// hinge e, upper pair p (0..9) -> 6 M + 10 e + p.  Force slots: triangle t vertex a ->
// 3 t + a; hinge e vertex a -> 3 M + 4 e + a.
void build_layout(const std::vector<const MeshData*>& sheets, BatchLayout* L);

}  // namespace cloth
