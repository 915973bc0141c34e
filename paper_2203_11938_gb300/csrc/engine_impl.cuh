// Host driver of the cloth engine (buffers, trajectory segments, execution modes).
#pragma once

#include <cstdio>
#include <cstdlib>
#include <filesystem>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "engine.cuh"

namespace cloth {

#define CLOTH_CUDA(expr)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      set_last_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                        \
      return CLOTH_ERR_CUDA;                                                                     \
    }                                                                                            \
  } while (0)

#define CLOTH_TRY(expr)        \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != CLOTH_OK) return rc_; \
  } while (0)

template <class R>
class Engine final : public EngineBase {
  // a size class of the per-sheet cluster solver: CL CTAs per cluster, EPC work entries per CTA
  struct SheetClass {
    int CL = 1, EPC = 1, offset = 0, n = 0;
    bool dense = false;  // k_cg_sheet<R, 2, 2>: two CTAs of two entries per SM
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
  };

  // a size class of the on-chip solver: clusters of CL CTAs of MR threads, smem bytes each
  struct SmClass {
    int CL = 1, MR = 32, offset = 0, n = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
  };

  // Every host-issued kernel launch goes through here so the launch count of a call
  // is known (CG loop-body kernels are counted on the device instead).
  template <class... P, class... A>
  void launch(void (*kern)(P...), dim3 g, dim3 b, cudaStream_t st, A&&... args) {
    kern<<<g, b, 0, st>>>(std::forward<A>(args)...);
    ++launches_;
  }

 public:
  Engine(const BatchLayout& L, const cloth_opts& o) : L_(L), o_(o) {}

  ~Engine() override {
    for (auto& g : graphs_)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    if (body_stream_) cudaStreamDestroy(body_stream_);
    if (host_active_) cudaFreeHost(host_active_);
    if (ev0_) cudaEventDestroy(ev0_);
    if (ev1_) cudaEventDestroy(ev1_);
    if (fork_ev_) cudaEventDestroy(fork_ev_);
    for (auto* cl : {&classes_, &rest_classes_, &dense_classes_})
      for (auto& c : *cl) {
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
      }
    for (auto& c : sm_classes_) {
      if (c.stream) cudaStreamDestroy(c.stream);
      if (c.done) cudaEventDestroy(c.done);
    }
    for (void* p : allocs_) cudaFree(p);
  }

  int init(std::string* err) {
    T_ = o_.steps;
    C_ = (o_.checkpoint_every >= 1 && o_.checkpoint_every < T_) ? o_.checkpoint_every : T_;
    nseg_ = (T_ + C_ - 1) / C_;
    Dev<R>& d = d_;
    std::memset(&d, 0, sizeof(d));
    d.S = L_.S;
    d.Np = L_.Np;
    d.Nu = L_.Nu;
    d.M = L_.M;
    d.E = L_.E;
    d.nslices = L_.nslices;
    d.NW = (int)L_.work_sheet.size();
    d.h = (R)o_.dt;
    d.gx = (R)o_.gravity[0];
    d.gy = (R)o_.gravity[1];
    d.gz = (R)o_.gravity[2];
    d.eta = (R)o_.clamp_eta;
    d.clamp = o_.clamp_eta > 0.0;
    d.tol = o_.cg_tol;
    d.maxit = o_.cg_max_iter;
    d.precond = o_.precond;
    int rc = CLOTH_OK;
    auto up_i = [&](const std::vector<int>& v) -> const int* { return upload(v, &rc); };
    auto up_r = [&](const std::vector<double>& v) -> const R* {
      std::vector<R> c(v.begin(), v.end());
      return upload(c, &rc);
    };
    d.tri_v = up_i(L_.tri_v);
    d.tri_sheet = up_i(L_.tri_sheet);
    d.tri_rest = up_r(L_.tri_rest);
    d.tri_rest_d = upload(L_.tri_rest, &rc);
    d.tri_metric = upload(L_.tri_metric, &rc);
    d.hin_v = up_i(L_.hin_v);
    d.hin_sheet = up_i(L_.hin_sheet);
    d.hin_rest = up_r(L_.hin_rest);
    d.hin_rest_d = upload(L_.hin_rest, &rc);
    d.i2u = up_i(L_.i2u);
    d.u2i = up_i(L_.u2i);
    d.pinned = upload(L_.pinned, &rc);
    d.area3 = up_r(L_.area3);
    d.vsheet = up_i(L_.vsheet);
    d.usheet = up_i(L_.usheet);
    d.slice_base = up_i(L_.slice_base);
    d.slice_K = up_i(L_.slice_K);
    d.cols = up_i(L_.cols);
    d.contrib_ptr = up_i(L_.contrib_ptr);
    d.contrib = up_i(L_.contrib);
    d.vf_ptr = up_i(L_.vf_ptr);
    d.vf = up_i(L_.vf);
    d.work_sheet = up_i(L_.work_sheet);
    d.work_row0 = up_i(L_.work_row0);
    d.work_rows = up_i(L_.work_rows);
    d.sheet_wfirst = up_i(L_.sheet_wfirst);
    d.sheet_uoff = up_i(L_.sheet_uoff);
    d.sheet_voff = up_i(L_.sheet_voff);
    d.sheet_toff = up_i(L_.sheet_toff);
    d.sheet_hoff = up_i(L_.sheet_hoff);
    const size_t n3 = 3 * (size_t)L_.Np;
    const size_t M = L_.M, E = L_.E;
    d.tri_f = alloc<double>(9 * M, &rc);
    d.tri_H = alloc<R>(54 * M, &rc);
    d.hin_f = alloc<double>(12 * E, &rc);
    d.hin_H = alloc<R>(90 * E, &rc);
    d.tri_r = alloc<R>(18 * M, &rc);
    d.hin_r = alloc<R>(24 * E, &rc);
    d.tri_sc = alloc<double>(M, &rc);
    d.hin_sc = alloc<double>(E, &rc);
    d.row_sc = alloc<double>(L_.Np, &rc);
    d.Aval = alloc<R>((size_t)L_.total_slots() * 32 * 9, &rc);
    d.bvec = alloc<R>(n3, &rc);
    d.dinv = alloc<R>(9 * (size_t)L_.Np, &rc);
    d.r = alloc<R>(n3, &rc);
    d.zp = alloc<R>(2 * 8 * (size_t)L_.Np, &rc);
    d.Ap = alloc<R>(n3, &rc);
    d.dv = alloc<double>(n3, &rc);
    if (o_.cg_warm_start) {
      // warm start: the guess in the direction layout, the forward and adjoint guess chains
      // and the forward chain's value at every checkpoint (so a recompute replays it)
      d.pg = alloc<R>((size_t)PStride<R>::v * L_.Np, &rc);
      guess_f_ = alloc<double>(n3, &rc);
      guess_a_ = alloc<double>(n3, &rc);
      if (nseg_ > 1) ck_g_ = alloc<double>(n3 * nseg_, &rc);
    }
    if (std::is_same<R, float>::value) {
      d.dvh = alloc<float>(n3, &rc);
      d.dvl = alloc<float>(n3, &rc);
    }
    d.cg = alloc<CGSheet>(L_.S, &rc);
    d.part_a = alloc<acc_t<R>>((size_t)d.NW * kWarpsPerEntry, &rc);
    d.part_b = alloc<acc_t<R>>((size_t)d.NW * kWarpsPerEntry, &rc);
    d.part_c = alloc<acc_t<R>>((size_t)d.NW * kWarpsPerEntry, &rc);
    d.active = alloc<int>(1, &rc);
    d.iter_total = alloc<unsigned long long>(4, &rc);
    d.body_runs = alloc<unsigned long long>(4, &rc);
    d.sheet_iters = alloc<unsigned>(8 * (size_t)L_.S, &rc);
    d.last_iters = alloc<unsigned>(L_.S, &rc);
    d.gacc = alloc<double>(3 * (size_t)L_.S, &rc);
    d.gacc_w = alloc<double>(3 * (size_t)L_.S, &rc);
    d.air_density = o_.air_density;
    d.wind = nullptr;
    if (o_.air_density > 0.0) d.row_w = alloc<double>(n3, &rc);
    // the state (x, v) is carried in FP64 in both precisions
    seg_x_ = alloc<double>(n3 * (C_ + 1), &rc);
    seg_v_ = alloc<double>(n3 * (C_ + 1), &rc);
    if (nseg_ > 1) {
      ck_x_ = alloc<double>(n3 * nseg_, &rc);
      ck_v_ = alloc<double>(n3 * nseg_, &rc);
    }
    ax_ = alloc<double>(n3, &rc);  // adjoint accumulators x_bar, v_bar in FP64
    av_ = alloc<double>(n3, &rc);
    tmp_a_ = alloc<R>(n3, &rc);
    tmp_b_ = alloc<R>(n3, &rc);
    tmp_xd_ = alloc<double>(n3, &rc);
    tmp_vd_ = alloc<double>(n3, &rc);
    tmp_ud_ = alloc<double>(n3, &rc);
    vin_ = alloc<double>(n3, &rc);
    mat_ = alloc<R>(4 * (size_t)L_.S, &rc);
    mat_tmp_ = alloc<R>(4 * (size_t)L_.S, &rc);
    d.material = mat_;
    lpart_ = alloc<double>((size_t)L_.S * T_, &rc);
    if (rc != CLOTH_OK) {
      *err = "device allocation failed";
      return rc;
    }
    if (cudaMemset(d.cg, 0, sizeof(CGSheet) * L_.S) != cudaSuccess ||
        cudaMemset(d.iter_total, 0, sizeof(unsigned long long) * 4) != cudaSuccess ||
        cudaMemset(d.body_runs, 0, sizeof(unsigned long long) * 4) != cudaSuccess ||
        cudaMemset(d.sheet_iters, 0, sizeof(unsigned) * 8 * L_.S) != cudaSuccess ||
        cudaMemset(d.last_iters, 0, sizeof(unsigned) * L_.S) != cudaSuccess ||
        cudaEventCreate(&ev0_) != cudaSuccess || cudaEventCreate(&ev1_) != cudaSuccess ||
        cudaMallocHost(&host_active_, sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&body_stream_, cudaStreamNonBlocking) != cudaSuccess) {
      *err = "CUDA setup failed";
      return CLOTH_ERR_CUDA;
    }
    // CG kernels of the resident-grid schedules: as many CTAs as can be resident at once
    // (each kernel by its own occupancy), each looping over work entries
    int dev = 0, sms = 0, per_sm = 0, per_sm2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_spmv<R>, kThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_cg_update<R>, kThreads, 0) != cudaSuccess) {
      *err = "CUDA occupancy query failed";
      return CLOTH_ERR_CUDA;
    }
    auto resident = [&](int per) { return std::max(1, std::min(d.NW, sms * std::max(1, per))); };
    res_spmv_ = resident(per_sm);
    res_upd_ = resident(per_sm2);
    spmv_grid_ = upd_grid_ = d.NW;
    // per-sheet cluster solvers: every sheet of at most 8 x 4 work entries (8192 rows) gets a
    // cluster of CL CTAs with EPC entries each (k_cg_sheet); sheets whose rows fit the
    // shared memory of at most 16 CTAs also get a partition for the on-chip solver
    // (k_cg_sheet_sm)
    {
      // clusters of 16 CTAs (a non-portable size): 2 entries per CTA for sheets of 17-32
      // entries, 3 (without the register cache) for 33-48, where the device can launch them
      wide2_ok_ = wide_cluster_ok(k_cg_sheet<R, 2>, 2 * kThreads);
      wide3_ok_ = wide_cluster_ok(k_cg_sheet<R, 3>, 3 * kThreads);
      int max_entries = 0;
      for (int s2 = 0; s2 < L_.S; ++s2) max_entries = std::max(max_entries, L_.sheet_wfirst[s2 + 1] - L_.sheet_wfirst[s2]);
      sheet_solver_ok_ = max_entries <= (wide3_ok_ ? 48 : 32);
      if (sheet_solver_ok_) {
        std::vector<int> all(L_.S);
        for (int s2 = 0; s2 < L_.S; ++s2) all[s2] = s2;
        CLOTH_TRY(make_classes(all, &classes_, &sheet_lists_, err));
        std::vector<int> rest;
        CLOTH_TRY(make_sm_classes(&rest, err));
        CLOTH_TRY(make_classes(rest, &rest_classes_, &rest_lists_, err));
        CLOTH_TRY(make_dense_classes(all, err));
        // the classes with the register column cache need little shared memory: leave the
        // rest of the SM's storage to L1, which holds the matrix rows they reread every
        // iteration; the others keep column indices in shared memory (up to 37 KB per CTA)
        cudaFuncSetAttribute(k_cg_sheet<R, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxL1);
        cudaFuncSetAttribute(k_cg_sheet<R, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxL1);
        cudaFuncSetAttribute(k_cg_sheet<R, 3>, cudaFuncAttributePreferredSharedMemoryCarveout, kColSmemCarveout);
        cudaFuncSetAttribute(k_cg_sheet<R, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, kColSmemCarveout);
        if (cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming) != cudaSuccess) {
          *err = "CUDA setup failed";
          return CLOTH_ERR_CUDA;
        }
      }
      cudaGetLastError();
    }
    if (o_.cg_handover > 0) handover_ = o_.cg_handover;
    if (o_.cg_schedule >= 0) {
      set_schedule(o_.cg_schedule);
    } else {
      int rc2 = autotune(err);
      if (rc2 != CLOTH_OK) return rc2;
    }
    return CLOTH_OK;
  }

  size_t workspace_bytes() const override { return bytes_; }
  int total_vertices() const override { return L_.Nu; }
  int count() const override { return L_.S; }

  // ---------------------------------------------------------------- forward
  int forward(const void* material, const void* x0, const void* v0, const void* forces, void* traj_x,
              int32_t* status, void* stream_) override {
    if (!material || !x0 || !v0 || !traj_x || !status) {
      set_last_error("cloth_forward: material, x0, v0, traj_x and status must be non-null");
      return CLOTH_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream_;
    last_stream_ = st;
    d_.material = mat_;
    d_.wind = wind_;
    fwd_forces_ = forces;
    if (o_.exec == CLOTH_EXEC_GRAPH) {
      GraphKey key{0, {material, x0, v0, forces, traj_x, status, wind_, nullptr, nullptr, nullptr}, 0};
      CLOTH_TRY(run_graph(key, st, &fixed_fwd_, [&](cudaStream_t s) {
        return forward_body(material, x0, v0, forces, traj_x, status, s, true);
      }));
    } else {
      launches_ = 0;
      CLOTH_TRY(forward_body(material, x0, v0, forces, traj_x, status, st, false));
      fixed_fwd_ = launches_;
    }
    fixed_bwd_ = 0;
    have_forward_ = true;
    seg_valid_ = nseg_ - 1;
    return CLOTH_OK;
  }

  int backward(const void* dL_dx, void* g_material, void* g_forces, void* g_x0, void* g_v0, int32_t* status,
               void* stream_) override {
    if (!have_forward_) {
      set_last_error("cloth_backward: no forward pass on this handle");
      return CLOTH_ERR_STATE;
    }
    if (!dL_dx || !status) {
      set_last_error("cloth_backward: dL_dx and status must be non-null");
      return CLOTH_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream_;
    last_stream_ = st;
    d_.material = mat_;
    d_.wind = wind_;
    const int seg_valid = seg_valid_;
    if (o_.exec == CLOTH_EXEC_GRAPH) {
      GraphKey key{1, {fwd_forces_, dL_dx, g_material, g_forces, g_x0, g_v0, status, wind_, nullptr, nullptr},
                   seg_valid};
      CLOTH_TRY(run_graph(key, st, &fixed_bwd_, [&](cudaStream_t s) {
        return backward_body(dL_dx, g_material, g_forces, g_x0, g_v0, status, s, true, seg_valid);
      }));
    } else {
      launches_ = 0;
      CLOTH_TRY(backward_body(dL_dx, g_material, g_forces, g_x0, g_v0, status, st, false, seg_valid));
      fixed_bwd_ = launches_;
    }
    seg_valid_ = 0;
    return CLOTH_OK;
  }

  int stats(int64_t* fwd, int64_t* bwd, int64_t* rec, int64_t* launches) override {
    CLOTH_CUDA(cudaStreamSynchronize(last_stream_));
    unsigned long long h[3], b[3];
    CLOTH_CUDA(cudaMemcpy(h, d_.iter_total, sizeof(h), cudaMemcpyDeviceToHost));
    CLOTH_CUDA(cudaMemcpy(b, d_.body_runs, sizeof(b), cudaMemcpyDeviceToHost));
    if (fwd) *fwd = (int64_t)h[0];
    if (bwd) *bwd = (int64_t)h[1];
    if (rec) *rec = (int64_t)h[2];
    if (launches) *launches = fixed_fwd_ + fixed_bwd_ + 4 * (int64_t)(b[0] + b[1] + b[2]);
    return CLOTH_OK;
  }

  int set_wind(const void* wind) override {
    wind_ = (const R*)wind;
    d_.wind = wind_;
    return CLOTH_OK;
  }

  int wind_gradient(void* g, void* stream) override {
    if (!g) return invalid("cloth_wind_gradient: null output");
    launch(k_grad_wind<R>, dim3((L_.S + 127) / 128), dim3(128), (cudaStream_t)stream, d_, (R*)g);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  int sheet_iterations(int phase, int32_t* max_iters, int64_t* total_iters) override {
    CLOTH_CUDA(cudaStreamSynchronize(last_stream_));
    std::vector<unsigned> h(2 * (size_t)L_.S);
    CLOTH_CUDA(cudaMemcpy(h.data(), d_.sheet_iters + 2 * (size_t)phase * L_.S, sizeof(unsigned) * h.size(),
                          cudaMemcpyDeviceToHost));
    for (int s = 0; s < L_.S; ++s) {
      if (max_iters) max_iters[s] = (int32_t)h[2 * s];
      if (total_iters) total_iters[s] = (int64_t)h[2 * s + 1];
    }
    return CLOTH_OK;
  }

  int64_t nonzero_blocks() const {
    int64_t nb = 0;
    for (size_t i = 0; i + 1 < L_.contrib_ptr.size(); ++i) nb += L_.contrib_ptr[i + 1] > L_.contrib_ptr[i] ? 1 : 0;
    // rows without element blocks (padding) still hold their identity diagonal
    for (int i = 0; i < L_.Np; ++i) nb += L_.i2u[i] < 0 ? 1 : 0;
    return nb;
  }

  int matrix_info(int64_t* rows, int64_t* blocks, int64_t* slots, int32_t* schedule) override {
    if (schedule) *schedule = schedule_;
    if (rows) *rows = L_.Np;
    if (blocks) *blocks = nonzero_blocks();
    if (slots) *slots = (int64_t)L_.total_slots() * 32;
    return CLOTH_OK;
  }

  // Algorithmic (compulsory) bytes of one launch of a kernel cloth_time_kernel times:
  // every input the kernel needs and every output it writes, once.
  int kernel_bytes(int which, int64_t* out) override {
    if (!out) return invalid("cloth_kernel_bytes: null output");
    const int64_t es = sizeof(R), rows = L_.Np, M = L_.M, E = L_.E;
    const int64_t stored = (int64_t)L_.total_slots() * 32;
    switch (which) {
      case 0:  // 3x3 values + column per nonzero block; z, p_{k-1} read and p_k, Ap written
        *out = nonzero_blocks() * (9 * es + 4) + rows * 4 * 3 * es;
        break;
      case 1:  // p, Ap, r read; r, z written; 3x3 inverse; the solution read and written (24 B each)
        *out = rows * (5 * 3 * es + 9 * es + 48);
        break;
      case 2:  // per row: pin flag, mass area, two index words, b and the 3x3 inverse written;
               // per force contribution: index + 3 doubles; per stored block: column, pin flag
               // of the column, contributor range, 9 values written; per contribution: index +
               // the element's 3x3 block
        *out = rows * (1 + es + 8 + 12 * es) + (int64_t)L_.vf.size() * 28 + stored * (9 + 9 * es) +
               (int64_t)L_.contrib.size() * (4 + 9 * es);
        break;
      case 3:  // per triangle: 3 vertex ids, sheet id, rest data (batch precision and FP64),
               // rest metric, FP64 force vector and 6 Hessian blocks written; x, v once per row
        *out = M * (16 + 5 * es + 40 + 24 + 72 + 54 * es) + rows * 48;
        break;
      case 4:  // per hinge: 4 vertex ids, sheet id, rest data (both precisions), FP64 force
               // vector and 10 Hessian blocks written; x, v once per row
        *out = E * (20 + 2 * es + 16 + 96 + 90 * es) + rows * 48;
        break;
      case 5:  // whole CG solve: every iteration of every sheet moves what kernels 0 and 1 move
               // for that sheet's rows (matrix once per iteration, as a streaming solve reads it)
        if (timed_solve_bytes_ < 0) return invalid("cloth_kernel_bytes: kernel 5 needs cloth_time_kernel(5) first");
        *out = timed_solve_bytes_;
        break;
      default:
        return invalid("cloth_kernel_bytes: kernel must be 0..5");
    }
    return CLOTH_OK;
  }

  // Average duration of `reps` back-to-back launches of one step kernel on the
  // system left by the last call (0: CG SpMV with its per-sheet p^T A p reduction,
  // 1: CG vector update, 2: assembly, 3: membrane element kernel, 4: bending element
  // kernel), timed with CUDA events on `stream`.
  int time_kernel(int which, int reps, double* avg_ms, void* stream_) override {
    if (!have_forward_ || reps < 1 || !avg_ms) return invalid("cloth_time_kernel: needs a forward and reps >= 1");
    cudaStream_t st = (cudaStream_t)stream_;
    d_.material = mat_;
    auto one = [&]() {
      switch (which) {
        case 0:
          k_cg_spmv<R><<<spmv_grid_, kThreads, 0, st>>>(d_);
          break;
        case 1: k_cg_update<R><<<upd_grid_, kThreads, 0, st>>>(d_); break;
        case 2: k_assemble<R><<<d_.NW, kThreads, 0, st>>>(d_, nullptr, nullptr); break;
        case 3: elements_of(0, sx(0), sv(0), st); break;
        default: elements_of(1, sx(0), sv(0), st); break;
      }
    };
    if (which < 0 || which > 5) return invalid("cloth_time_kernel: unknown kernel id");
    if (which == 5) return time_whole_solve(reps, avg_ms, st);
    k_reopen<R><<<(L_.S + 255) / 256, 256, 0, st>>>(d_);
    one();  // warm-up
    k_reopen<R><<<(L_.S + 255) / 256, 256, 0, st>>>(d_);
    CLOTH_CUDA(cudaEventRecord(ev0_, st));
    for (int k = 0; k < reps; ++k) one();
    CLOTH_CUDA(cudaEventRecord(ev1_, st));
    CLOTH_CUDA(cudaEventSynchronize(ev1_));
    float ms = 0.f;
    CLOTH_CUDA(cudaEventElapsedTime(&ms, ev0_, ev1_));
    *avg_ms = ms / reps;
    // leave the CG state closed again
    k_reset_status<R><<<(L_.S + 255) / 256, 256, 0, st>>>(d_, kPhaseForward);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  // Kernel id 5: whole solves of the system the last call assembled last (right-hand side
  // in bvec), in the schedule in use, captured once and replayed `reps` times; records the
  // algorithmic bytes of one solve from its per-sheet iteration counts.
  int time_whole_solve(int reps, double* avg_ms, cudaStream_t st) {
    CLOTH_CUDA(cudaStreamSynchronize(st));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CLOTH_CUDA(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeRelaxed));
    const int rc = solve(d_.bvec, kPhaseTimed, cap_stream_, true);
    const cudaError_t ec = cudaStreamEndCapture(cap_stream_, &g);
    if (rc != CLOTH_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc != CLOTH_OK) return rc;
      CLOTH_CUDA(ec);
    }
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CLOTH_CUDA(ei);
    cudaError_t e = cudaGraphLaunch(ge, st);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(ev0_, st);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev1_, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1_);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0_, ev1_);
    cudaGraphExecDestroy(ge);
    CLOTH_CUDA(e);
    *avg_ms = ms / reps;
    // iterations of one solve: the counters of the timed phase hold reps + 1 identical solves
    std::vector<unsigned> h(2 * (size_t)L_.S);
    CLOTH_CUDA(cudaMemcpy(h.data(), d_.sheet_iters + 2 * (size_t)kPhaseTimed * L_.S, sizeof(unsigned) * h.size(),
                          cudaMemcpyDeviceToHost));
    const int64_t es = sizeof(R);
    int64_t bytes = 0;
    for (int s2 = 0; s2 < L_.S; ++s2) {
      const int64_t rows = L_.sheet_voff[s2 + 1] - L_.sheet_voff[s2];
      const int64_t per_iter = sheet_nonzero_blocks(s2) * (9 * es + 4) + rows * 4 * 3 * es +
                               rows * (5 * 3 * es + 9 * es + 48);
      bytes += (int64_t)(h[2 * s2 + 1] / (unsigned)(reps + 1)) * per_iter;
    }
    timed_solve_bytes_ = bytes;
    k_reset_status<R><<<(L_.S + 255) / 256, 256, 0, st>>>(d_, kPhaseTimed);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  // nonzero 3x3 blocks of one sheet's rows (padding rows count their identity diagonal)
  int64_t sheet_nonzero_blocks(int s2) const {
    int64_t nb = 0;
    for (int i = L_.sheet_voff[s2]; i < L_.sheet_voff[s2 + 1]; ++i) {
      if (L_.i2u[i] < 0) {
        ++nb;
        continue;
      }
      const int sl = i / kSlice, lane = i % kSlice;
      for (int k = 0; k < L_.slice_K[sl]; ++k) {
        const size_t ent = ((size_t)L_.slice_base[sl] + k) * kSlice + lane;
        nb += L_.contrib_ptr[ent + 1] > L_.contrib_ptr[ent] ? 1 : 0;
      }
    }
    return nb;
  }

  // ---------------------------------------------------------------- losses
  int loss_l2(const void* traj, const void* target, double* loss, void* grad, void* stream_) override {
    if (!traj || !target || !loss) {
      set_last_error("cloth_loss_l2: traj, target and loss must be non-null");
      return CLOTH_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream_;
    if (grad) CLOTH_CUDA(cudaMemsetAsync(grad, 0, sizeof(R) * 3 * (size_t)L_.Nu, st));
    dim3 grid(L_.S, T_);
    k_loss_l2<R><<<grid, kThreads, 0, st>>>(d_, T_, (const R*)traj, (const R*)target, (R*)grad, lpart_);
    k_loss_final<R><<<(L_.S + 127) / 128, 128, 0, st>>>(d_, T_, lpart_, loss);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  int loss_pinhole(const void* traj, const void* uv, const double* cam, double* loss, void* grad,
                   void* stream_) override {
    if (!traj || !uv || !cam || !loss) {
      set_last_error("cloth_loss_pinhole: traj, target_uv, camera and loss must be non-null");
      return CLOTH_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream_;
    if (grad) CLOTH_CUDA(cudaMemsetAsync(grad, 0, sizeof(R) * 3 * (size_t)L_.Nu, st));
    dim3 grid(L_.S, T_);
    k_loss_pinhole<R><<<grid, kThreads, 0, st>>>(d_, T_, (const R*)traj, (const R*)uv, cam[0], cam[1], cam[2],
                                                 cam[3], (R*)grad, lpart_);
    k_loss_final<R><<<(L_.S + 127) / 128, 128, 0, st>>>(d_, T_, lpart_, loss);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  // ---------------------------------------------------------------- single stages
  int internal_forces(const void* material, const void* x, void* fm, void* fb, void* stream_) override {
    if (!material || !x) return invalid("cloth_internal_forces: material and x must be non-null");
    cudaStream_t st = (cudaStream_t)stream_;
    CLOTH_TRY(use_material(material, st));
    gather_state((const R*)x, tmp_xd_, st);
    elements(tmp_xd_, nullptr, st);
    if (fm) k_vertex_force<R><<<grid_rows(), 256, 0, st>>>(d_, 0, (R*)fm);
    if (fb) k_vertex_force<R><<<grid_rows(), 256, 0, st>>>(d_, 1, (R*)fb);
    d_.material = mat_;
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  int system_dense(const void* material, const void* x, const void* v, const void* F, void* A, void* b,
                   void* stream_) override {
    if (!material || !x || !v || !A || !b) return invalid("cloth_system_dense: null argument");
    cudaStream_t st = (cudaStream_t)stream_;
    CLOTH_TRY(use_material(material, st));
    CLOTH_TRY(assemble_at(x, v, F, st));
    std::vector<long long> off(L_.S + 1, 0);
    for (int s = 0; s < L_.S; ++s) {
      long long n3 = 3LL * (L_.sheet_uoff[s + 1] - L_.sheet_uoff[s]);
      off[s + 1] = off[s] + n3 * n3;
    }
    long long* doff = nullptr;
    CLOTH_CUDA(cudaMallocAsync((void**)&doff, sizeof(long long) * off.size(), st));
    CLOTH_CUDA(cudaMemcpyAsync(doff, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
    CLOTH_CUDA(cudaMemsetAsync(A, 0, sizeof(R) * off[L_.S], st));
    k_dense<R><<<grid_rows(), 256, 0, st>>>(d_, doff, (R*)A);
    k_scatter<R, R><<<grid_rows(), 256, 0, st>>>(d_, d_.bvec, (R*)b);
    d_.material = mat_;
    CLOTH_CUDA(cudaGetLastError());
    CLOTH_CUDA(cudaFreeAsync(doff, st));
    return CLOTH_OK;
  }

  int spmv(const void* material, const void* x, const void* v, const void* p, void* y, void* stream_) override {
    if (!material || !x || !v || !p || !y) return invalid("cloth_spmv: null argument");
    cudaStream_t st = (cudaStream_t)stream_;
    CLOTH_TRY(use_material(material, st));
    CLOTH_TRY(assemble_at(x, v, nullptr, st));
    gather((const R*)p, tmp_a_, st);
    k_spmv_plain<R><<<grid_rows(), 256, 0, st>>>(d_, tmp_a_, tmp_b_);
    k_scatter<R, R><<<grid_rows(), 256, 0, st>>>(d_, tmp_b_, (R*)y);
    d_.material = mat_;
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  int third(const void* material, const void* x, const void* a, const void* b, void* out, void* stream_) override {
    if (!material || !x || !a || !b || !out) return invalid("cloth_third_contraction: null argument");
    cudaStream_t st = (cudaStream_t)stream_;
    CLOTH_TRY(use_material(material, st));
    gather_state((const R*)x, tmp_xd_, st);
    gather_state((const R*)a, tmp_vd_, st);
    gather_state((const R*)b, tmp_ud_, st);
    k_adj_tri<R><<<(L_.M + kElemThreads - 1) / kElemThreads, kElemThreads, 0, st>>>(d_, tmp_xd_, tmp_vd_, tmp_ud_, 1);
    if (L_.E)
      k_adj_hinge<R><<<(L_.E + kElemThreads - 1) / kElemThreads, kElemThreads, 0, st>>>(d_, tmp_xd_, tmp_vd_, tmp_ud_,
                                                                                       1);
    k_vertex_third<R><<<grid_rows(), 256, 0, st>>>(d_, (R*)out);
    d_.material = mat_;
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

 private:
  struct GraphKey {
    int kind;
    const void* p[10];
    int extra;
    bool operator==(const GraphKey& o) const {
      if (kind != o.kind || extra != o.extra) return false;
      for (int i = 0; i < 10; ++i)
        if (p[i] != o.p[i]) return false;
      return true;
    }
  };
  struct CachedGraph {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    int64_t fixed = 0;  // host-issued kernel nodes (CG loop bodies excluded)
  };

  int invalid(const char* msg) {
    set_last_error(msg);
    return CLOTH_ERR_INVALID_ARG;
  }

  template <class U>
  U* alloc(size_t n, int* rc) {
    if (n == 0) n = 1;
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(U)) != cudaSuccess) {
      *rc = CLOTH_ERR_OOM;
      return nullptr;
    }
    allocs_.push_back(p);
    bytes_ += n * sizeof(U);
    return (U*)p;
  }
  template <class U>
  const U* upload(const std::vector<U>& v, int* rc) {
    U* p = alloc<U>(v.size(), rc);
    if (p && !v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice) != cudaSuccess)
      *rc = CLOTH_ERR_CUDA;
    return p;
  }

  int grid_rows() const { return (L_.Np + 255) / 256; }
  size_t n3() const { return 3 * (size_t)L_.Np; }
  double* sx(int j) const { return seg_x_ + n3() * j; }
  double* sv(int j) const { return seg_v_ + n3() * j; }

  void gather(const R* in, R* out, cudaStream_t st) { launch(k_gather<R, R, R>, dim3(grid_rows()), dim3(256), st, d_, in, out); }
  void gather_state(const R* in, double* out, cudaStream_t st) {
    launch(k_gather<R, R, double>, dim3(grid_rows()), dim3(256), st, d_, in, out);
  }

  // single-stage entry points read their own material buffer
  int use_material(const void* material, cudaStream_t st) {
    CLOTH_CUDA(cudaMemcpyAsync(mat_tmp_, material, sizeof(R) * 4 * L_.S, cudaMemcpyDeviceToDevice, st));
    d_.material = mat_tmp_;
    return CLOTH_OK;
  }

  // element forces and Hessian blocks at x; with v, the stored element vectors are f - h H~ v
  void elements(const double* x, const double* v, cudaStream_t st) {
    elements_of(0, x, v, st);
    elements_of(1, x, v, st);
  }
  // the membrane (kind 0) or bending (kind 1) element kernel at its tuned block size
  void elements_of(int kind, const double* x, const double* v, cudaStream_t st) {
    const int n = kind == 0 ? L_.M : L_.E, nt = kind == 0 ? tri_nt_ : hin_nt_;
    if (!n) return;
    const dim3 g((unsigned)((n + nt - 1) / nt)), b((unsigned)nt);
    if (kind == 0) {
      if (nt == 64) launch(k_elem_tri<R, 64>, g, b, st, d_, x, v);
      else if (nt == 256) launch(k_elem_tri<R, 256>, g, b, st, d_, x, v);
      else launch(k_elem_tri<R, 128>, g, b, st, d_, x, v);
    } else {
      if (nt == 64) launch(k_elem_hinge<R, 64>, g, b, st, d_, x, v);
      else if (nt == 256) launch(k_elem_hinge<R, 256>, g, b, st, d_, x, v);
      else launch(k_elem_hinge<R, 128>, g, b, st, d_, x, v);
    }
  }
  // Block sizes of the element kernels (64, 128 or 256 threads per CTA), per element kind:
  // the fastest in three rounds of five launches on the state the autotuner set up.
  int tune_element_shapes(cudaStream_t st) {
    for (int kind = 0; kind < 2; ++kind) {
      if ((kind == 0 ? L_.M : L_.E) == 0) continue;
      int& nt = kind == 0 ? tri_nt_ : hin_nt_;
      float best = 1e30f;
      int best_nt = kElemThreads;
      for (int round = 0; round < 3; ++round)
        for (int c : {128, 64, 256}) {
          nt = c;
          elements_of(kind, tmp_xd_, tmp_vd_, st);  // warm-up
          CLOTH_CUDA(cudaEventRecord(ev0_, st));
          for (int k = 0; k < 5; ++k) elements_of(kind, tmp_xd_, tmp_vd_, st);
          CLOTH_CUDA(cudaEventRecord(ev1_, st));
          CLOTH_CUDA(cudaEventSynchronize(ev1_));
          float ms = 0.f;
          CLOTH_CUDA(cudaEventElapsedTime(&ms, ev0_, ev1_));
          if (ms < best) {
            best = ms;
            best_nt = c;
          }
        }
      nt = best_nt;
    }
    return CLOTH_OK;
  }
  static int nt_code(int nt) { return nt == 64 ? 1 : nt == 256 ? 2 : 0; }
  static int nt_of(int code) { return code == 1 ? 64 : code == 2 ? 256 : kElemThreads; }

  int assemble_at(const void* x, const void* v, const void* F, cudaStream_t st) {
    gather_state((const R*)x, tmp_xd_, st);
    gather_state((const R*)v, tmp_vd_, st);
    const double* vs = start_velocity(tmp_vd_, (const R*)F, st);
    elements(tmp_xd_, vs, st);
    k_assemble<R><<<d_.NW, kThreads, 0, st>>>(d_, o_.force_mode == CLOTH_FORCES_VELOCITY ? nullptr : (const R*)F, vs);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  // Size classes (CL, EPC) of k_cg_sheet over the given sheets, each listed largest first,
  // with a stream and an event each; the sheet lists go to the device.
  // dense: one work entry per CTA (cluster of E CTAs for a sheet of E <= 16 entries, four
  // CTAs per SM); sheets of more entries take the (8, 4) class.
  int make_classes(const std::vector<int>& sheets, std::vector<SheetClass>* out, const int** dev_lists,
                   std::string* err, bool dense = false) {
    std::map<std::pair<int, int>, std::vector<int>> cls;
    for (int s2 : sheets) {
      const int E = L_.sheet_wfirst[s2 + 1] - L_.sheet_wfirst[s2];
      int CL = 1, EPC = 1;
      if (dense && E <= 16) CL = (E + 1) / 2, EPC = 2;
      else if (E <= 1) CL = 1, EPC = 1;
      else if (E <= 2) CL = 1, EPC = 2;
      else if (E <= 4) CL = 2, EPC = 2;
      else if (E <= 8) CL = 4, EPC = 2;
      else if (E <= 16) CL = 8, EPC = 2;
      else if (E <= 32 && wide2_ok_) CL = 16, EPC = 2;
      else if (E <= 32) CL = 8, EPC = 4;
      else CL = 16, EPC = 3;  // E <= 48 (wide3_ok_ checked by the caller)
      cls[{CL, EPC}].push_back(s2);
    }
    std::vector<int> lists;
    for (auto& kv : cls) {
      auto& v = kv.second;
      std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
        return L_.sheet_wfirst[a + 1] - L_.sheet_wfirst[a] > L_.sheet_wfirst[b + 1] - L_.sheet_wfirst[b];
      });
      SheetClass c;
      c.CL = kv.first.first;
      c.EPC = kv.first.second;
      c.dense = dense && c.EPC == 2 && c.CL <= 8;
      c.offset = (int)lists.size();
      c.n = (int)v.size();
      lists.insert(lists.end(), v.begin(), v.end());
      if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess) {
        *err = "CUDA stream setup failed";
        return CLOTH_ERR_CUDA;
      }
      out->push_back(c);
    }
    int rc = CLOTH_OK;
    *dev_lists = lists.empty() ? nullptr : upload(lists, &rc);
    if (!lists.empty() && rc == CLOTH_OK) {
      // the classes' offsets and the total, for the launch-order kernel, and its output
      std::vector<int> seg;
      int off = 0;
      for (auto& kv : cls) {
        seg.push_back(off);
        off += (int)kv.second.size();
      }
      seg.push_back(off);
      ListOrder lo;
      lo.seg = upload(seg, &rc);
      lo.order = alloc<int>(lists.size(), &rc);
      lo.nclasses = (int)cls.size();
      orders_[*dev_lists] = lo;
    }
    if (rc != CLOTH_OK) *err = "device allocation failed";
    return rc;
  }

  // true when one cluster of 16 CTAs of `threads` threads of `kern` can be resident
  template <class K>
  bool wide_cluster_ok(K kern, int threads) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(16);
    lc.blockDim = dim3((unsigned)threads);
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 16;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    lc.attrs = &at;
    lc.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, kern, &lc) == cudaSuccess && n >= 1;
    cudaGetLastError();
    return ok;
  }

  // Dense classes (schedule bit 4), kept only if every cluster shape can be launched.
  int make_dense_classes(const std::vector<int>& all, std::string* err) {
    std::vector<SheetClass> cl;
    const int* lists = nullptr;
    CLOTH_TRY(make_classes(all, &cl, &lists, err, true));
    // two CTAs per SM, each with ~25 KB of column indices (and in FP32 ~18 KB of
    // block-Jacobi inverses) in shared memory; clusters of at most 8 CTAs
    bool ok = cudaFuncSetAttribute(k_cg_sheet<R, 2, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   kColSmemCarveout) == cudaSuccess;
    for (const auto& c : cl) {
      if (!ok || !c.dense) continue;
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3((unsigned)c.CL);
      lc.blockDim = dim3(2 * kThreads);
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = (unsigned)c.CL;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      lc.attrs = &at;
      lc.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_cg_sheet<R, 2, 2>, &lc) != cudaSuccess || n < 1) ok = false;
    }
    cudaGetLastError();
    dense_classes_ = cl;  // destroyed with the engine either way
    dense_lists_ = lists;
    dense_ok_ = ok;
    return CLOTH_OK;
  }

  // Partitions for the on-chip solver: each sheet's slices split into the fewest contiguous
  // ranges (CTAs, at most 16) whose matrix values and gathered vectors fit one CTA's shared
  // memory, balanced by bytes; sheets grouped by cluster size (one launch each, largest
  // first), each group checked to be launchable (cudaOccupancyMaxActiveClusters).  The
  // sheets that do not fit are returned in *rest.
  int make_sm_classes(std::vector<int>* rest, std::string* err) {
    constexpr int PS = PStride<R>::v;
    const size_t vec_row = 3 * PS * sizeof(R), part_bytes = 3 * 32 * sizeof(acc_t<R>);
    const size_t budget = kSmBudget - part_bytes;
    std::map<int, std::vector<std::pair<int, SmSheet>>> by_cl;  // CL -> (sheet, partition)
    std::map<int, std::pair<int, size_t>> need;                 // CL -> (max rows, max value bytes)
    for (int s2 = 0; s2 < L_.S; ++s2) {
      const int a = L_.sheet_voff[s2] / kSlice, b = L_.sheet_voff[s2 + 1] / kSlice;
      bool fits = true;
      std::vector<size_t> vb(b - a);
      size_t total = 0;
      for (int sl = a; sl < b; ++sl) {
        if (L_.slice_K[sl] > kSmSlots) fits = false;
        vb[sl - a] = (size_t)L_.slice_K[sl] * 32 * 9 * sizeof(R);
        total += vb[sl - a] + 32 * vec_row;
      }
      int G = 0;
      SmSheet ps = {};
      ps.sheet = s2;
      size_t rows_max = 0, vals_max = 0;
      for (int g = 1; fits && g <= kSmMaxRanks && !G; ++g) {
        if (total > budget * g || b - a < g) continue;
        // cut where the running byte count crosses total * k / g
        std::vector<int> cut(g + 1, a);
        cut[g] = b;
        size_t run = 0;
        int k = 1;
        for (int sl = a; sl < b && k < g; ++sl) {
          run += vb[sl - a] + 32 * vec_row;
          if (run * g >= total * (size_t)k) cut[k++] = sl + 1;
        }
        bool ok = k == g;
        size_t rmax = 0, vmax = 0;
        for (int q = 0; ok && q < g; ++q) {
          size_t v = 0;
          for (int sl = cut[q]; sl < cut[q + 1]; ++sl) v += vb[sl - a];
          const size_t rows = (size_t)(cut[q + 1] - cut[q]) * 32;
          if (rows == 0 || rows > (size_t)kSmMaxThreads || v + rows * vec_row > budget) ok = false;
          rmax = std::max(rmax, rows);
          vmax = std::max(vmax, v);
        }
        if (!ok) continue;
        G = g;
        for (int q = 0; q <= g; ++q) ps.sl0[q] = cut[q];
        rows_max = rmax;
        vals_max = vmax;
      }
      if (!G) {
        rest->push_back(s2);
        continue;
      }
      by_cl[G].push_back({s2, ps});
      auto& nd = need[G];
      nd.first = std::max(nd.first, (int)rows_max);
      nd.second = std::max(nd.second, vals_max);
    }
    size_t max_smem = 0;
    bool nonportable = false;
    for (auto& kv : need) {
      const size_t smem = kv.second.first * vec_row + part_bytes + kv.second.second;
      max_smem = std::max(max_smem, smem);
      nonportable = nonportable || kv.first > 8;
    }
    if (by_cl.empty()) return CLOTH_OK;
    if (cudaFuncSetAttribute(k_cg_sheet_sm<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem) !=
            cudaSuccess ||
        (nonportable && cudaFuncSetAttribute(k_cg_sheet_sm<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                            cudaSuccess)) {
      cudaGetLastError();  // no on-chip solver on this device: every sheet to the other one
      for (auto& kv : by_cl)
        for (auto& e : kv.second) rest->push_back(e.first);
      std::sort(rest->begin(), rest->end());
      return CLOTH_OK;
    }
    std::vector<SmSheet> lists;
    for (auto& kv : by_cl) {
      const int CL = kv.first;
      SmClass c;
      c.CL = CL;
      c.MR = need[CL].first;
      c.smem = c.MR * vec_row + part_bytes + need[CL].second;
      // launchable: at least one cluster of this shape fits the device
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3((unsigned)CL);
      lc.blockDim = dim3((unsigned)c.MR);
      lc.dynamicSmemBytes = c.smem;
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = (unsigned)CL;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      lc.attrs = &at;
      lc.numAttrs = 1;
      int nclusters = 0;
      if (c.smem > kSmDynMax ||
          cudaOccupancyMaxActiveClusters(&nclusters, k_cg_sheet_sm<R>, &lc) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        for (auto& e : kv.second) rest->push_back(e.first);
        continue;
      }
      auto& v = kv.second;
      std::stable_sort(v.begin(), v.end(), [&](const std::pair<int, SmSheet>& x, const std::pair<int, SmSheet>& y) {
        return L_.sheet_voff[x.first + 1] - L_.sheet_voff[x.first] > L_.sheet_voff[y.first + 1] - L_.sheet_voff[y.first];
      });
      c.offset = (int)lists.size();
      c.n = (int)v.size();
      for (auto& e : v) lists.push_back(e.second);
      if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess) {
        *err = "CUDA stream setup failed";
        return CLOTH_ERR_CUDA;
      }
      sm_classes_.push_back(c);
    }
    std::sort(rest->begin(), rest->end());
    if (!lists.empty()) {
      int rc = CLOTH_OK;
      sm_lists_ = upload(lists, &rc);
      if (rc != CLOTH_OK) {
        *err = "device allocation failed";
        return rc;
      }
    }
    return CLOTH_OK;
  }

  // CG schedules (bitwise-identical results): bit 1 = direction update folded into the
  // SpMV (2 kernels per iteration) else a separate direction kernel (3); bit 0 = grid of
  // resident CTAs looping over work entries else one CTA per work entry; bit 2 = per-sheet
  // cluster solver after the hand-over point; bit 3 = its on-chip variant where it fits.
  void set_schedule(int sched) {
    schedule_ = sched & 31;
    // bit 3: sheets that fit go to the on-chip per-sheet solver; bit 4: the dense classes of
    // the per-sheet solver (each reported only where it exists)
    use_sm_ = (schedule_ & 8) != 0 && !sm_classes_.empty();
    use_dense_ = (schedule_ & 16) != 0 && !use_sm_ && dense_ok_;
    if (!use_sm_) schedule_ &= ~8;
    if (!use_dense_) schedule_ &= ~16;
    schedule_ |= 2;  // the direction update is always folded into the SpMV
    spmv_grid_ = (schedule_ & 1) ? res_spmv_ : d_.NW;
    upd_grid_ = (schedule_ & 1) ? res_upd_ : d_.NW;
    // bit 2: every sheet is solved by the per-sheet cluster solver (the device loop
    // hands over at once)
    d_.tail_threshold = ((schedule_ & 4) && sheet_solver_ok_) ? std::min(L_.S, handover_) : 0;
  }

  int scalar_grid() const { return (L_.S * 32 + 255) / 256; }

  void emit_cg_body(cudaStream_t s, int phase, cudaGraphConditionalHandle cond, int use_cond) {
    k_cg_spmv<R><<<spmv_grid_, kThreads, 0, s>>>(d_);
    k_cg_scalar_alpha<R><<<scalar_grid(), 256, 0, s>>>(d_, phase, cond, use_cond);
    k_cg_update<R><<<upd_grid_, kThreads, 0, s>>>(d_);
    k_cg_scalar_beta<R><<<scalar_grid(), 256, 0, s>>>(d_, phase, cond, use_cond);
  }

  static std::string tune_cache_path() {
    if (const char* p = std::getenv("CLOTH_TUNE_CACHE")) return p;
    const char* base = std::getenv("XDG_CACHE_HOME");
    std::string dir = base ? std::string(base) : (std::getenv("HOME") ? std::string(std::getenv("HOME")) + "/.cache" : "");
    if (dir.empty()) return "";
    return dir + "/cloth_sim/tune.json";
  }

  // Flat JSON object {"key": value, ...} of integer schedule choices.
  static std::map<std::string, int> read_tune_cache(const std::string& path) {
    std::map<std::string, int> m;
    std::ifstream f(path);
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    size_t i = 0;
    while ((i = t.find('"', i)) != std::string::npos) {
      const size_t j = t.find('"', i + 1);
      if (j == std::string::npos) break;
      const size_t c = t.find(':', j);
      if (c == std::string::npos) break;
      m[t.substr(i + 1, j - i - 1)] = std::atoi(t.c_str() + c + 1);
      i = t.find_first_of(",}", c);
      if (i == std::string::npos) break;
    }
    return m;
  }

  static void write_tune_cache(const std::string& path, const std::map<std::string, int>& m) {
    std::error_code ec;
    std::filesystem::create_directories(std::filesystem::path(path).parent_path(), ec);
    std::ofstream f(path, std::ios::trunc);
    if (!f) return;
    f << "{";
    bool first = true;
    for (const auto& kv : m) {
      f << (first ? "" : ",") << "\n  \"" << kv.first << "\": " << kv.second;
      first = false;
    }
    f << "\n}\n";
  }

  // Autotuner: time CG iterations of every loop schedule on this batch's matrix (assembled
  // at the rest state with a nominal material), then whole solves with and without the
  // per-sheet solver at several hand-over points, and keep the fastest; the choice is
  // cached per device and matrix shape in a JSON file.
  int autotune(std::string* err) {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
      *err = "device query failed";
      return CLOTH_ERR_CUDA;
    }
    std::ostringstream key;
    key << prop.name << "|" << (sizeof(R) == 4 ? "f32" : "f64") << "|rows=" << L_.Np << "|entries=" << d_.NW
        << "|slots=" << L_.total_slots() << "|sheets=" << L_.S << "|handover=" << o_.cg_handover << "|v5";
    const std::string path = tune_cache_path();
    auto cache = path.empty() ? std::map<std::string, int>() : read_tune_cache(path);
    auto it = cache.find(key.str());
    if (it != cache.end()) {
      // value: schedule (bits 0-4), membrane and bending block-size codes (bits 5-6, 7-8),
      // hand-over point (bits 9 and up)
      if (o_.cg_handover == 0 && (it->second >> 9) > 0) handover_ = it->second >> 9;
      tri_nt_ = nt_of((it->second >> 5) & 3);
      hin_nt_ = nt_of((it->second >> 7) & 3);
      set_schedule(it->second & 31);
      return CLOTH_OK;
    }
    cudaStream_t st = cap_stream_;
    std::vector<R> mat(4 * (size_t)L_.S);
    for (int s = 0; s < L_.S; ++s) {
      mat[4 * s] = R(1e3);
      mat[4 * s + 1] = R(0.3);
      mat[4 * s + 2] = R(1e-4);
      mat[4 * s + 3] = R(0.1);
    }
    CLOTH_CUDA(cudaMemcpy(mat_tmp_, mat.data(), sizeof(R) * mat.size(), cudaMemcpyHostToDevice));
    CLOTH_CUDA(cudaMemcpy(tmp_xd_, L_.rest.data(), sizeof(double) * L_.rest.size(), cudaMemcpyHostToDevice));
    CLOTH_CUDA(cudaMemset(tmp_vd_, 0, sizeof(double) * n3()));
    d_.material = mat_tmp_;
    CLOTH_TRY(tune_element_shapes(st));
    elements(tmp_xd_, tmp_vd_, st);
    k_assemble<R><<<d_.NW, kThreads, 0, st>>>(d_, nullptr, nullptr);
    // loop schedules (bit 0: resident or per-entry grid): the best of three rounds of 30
    // iterations each (bit 2 and above are decided below)
    float best_ms[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    const int iters = 30;
    for (int round = 0; round < 3; ++round) {
      for (int sched = 2; sched < 4; ++sched) {
        set_schedule(sched);
        k_solve_begin<R><<<1, 32, 0, st>>>(d_);
        k_cg_init<R><<<upd_grid_, kThreads, 0, st>>>(d_, d_.bvec);
        k_cg_scalar_init<R><<<scalar_grid(), 256, 0, st>>>(d_, kPhaseForward, 0);
        emit_cg_body(st, kPhaseForward, 0, 0);  // warm-up
        CLOTH_CUDA(cudaEventRecord(ev0_, st));
        for (int k = 0; k < iters; ++k) emit_cg_body(st, kPhaseForward, 0, 0);
        CLOTH_CUDA(cudaEventRecord(ev1_, st));
        CLOTH_CUDA(cudaEventSynchronize(ev1_));
        float ms = 0.f;
        CLOTH_CUDA(cudaEventElapsedTime(&ms, ev0_, ev1_));
        best_ms[sched] = std::min(best_ms[sched], ms);
      }
    }
    int best_s = 2;
    if (best_ms[3] < best_ms[2]) best_s = 3;
    // then whole solves of this system: the loop alone, and the loop handing over to the
    // per-sheet cluster solver at several points (unless the caller fixed the point)
    if (sheet_solver_ok_) {
      std::vector<int> points;
      if (o_.cg_handover > 0) {
        points.push_back(handover_);
      } else {
        for (int f : {16, 8, 4, 2, 1}) {
          const int p = std::max(1, L_.S / f);
          if (points.empty() || points.back() != p) points.push_back(p);
        }
      }
      set_schedule(best_s);
      float t_best = 0.f;
      CLOTH_TRY(time_solve(&t_best));
      int best_h = 0, best_tail = 0;
      std::vector<int> tails = {4};
      if (!sm_classes_.empty()) tails.push_back(12);  // the on-chip variant
      if (dense_ok_) tails.push_back(20);             // the dense classes
      for (int tail : tails)
        for (int p : points) {
          handover_ = p;
          set_schedule(best_s | tail);
          float t = 0.f;
          CLOTH_TRY(time_solve(&t));
          if (t < t_best) {
            t_best = t;
            best_h = p;
            best_tail = tail;
          }
        }
      if (best_h > 0) {
        handover_ = best_h;
        best_s |= best_tail;
      }
    }
    set_schedule(best_s);
    d_.material = mat_;
    k_reset_status<R><<<(L_.S + 255) / 256, 256, 0, st>>>(d_, kPhaseForward);
    CLOTH_CUDA(cudaStreamSynchronize(st));
    if (!path.empty()) {
      cache[key.str()] = best_s | nt_code(tri_nt_) << 5 | nt_code(hin_nt_) << 7 | ((best_s & 4) ? handover_ << 9 : 0);
      write_tune_cache(path, cache);
    }
    return CLOTH_OK;
  }

  // Device time [ms] of one solve of the assembled system, captured as it runs in a call
  // (autotuner): one untimed replay, then one timed.
  int time_solve(float* ms) {
    cudaStream_t st = cap_stream_;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CLOTH_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    const int rc = solve(d_.bvec, kPhaseForward, st, true);
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (rc != CLOTH_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc != CLOTH_OK) return rc;
      CLOTH_CUDA(ec);
    }
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CLOTH_CUDA(ei);
    cudaError_t e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev0_, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev1_, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1_);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ev0_, ev1_);
    cudaGraphExecDestroy(ge);
    CLOTH_CUDA(e);
    return CLOTH_OK;
  }

  // Solve A y = rhs (y left in d_.dv) for every sheet.  In graph mode the CG loop is a
  // conditional WHILE node whose condition the kernels clear when the last sheet ends.
  // guess: FP64 starting vector (internal layout) or null for 0; keep: where the solution
  // is also written (the next solve's guess) or null.
  int solve(const R* rhs, int phase, cudaStream_t st, bool capturing, const double* guess = nullptr,
            double* keep = nullptr) {
    launch(k_solve_begin<R>, dim3(1), dim3(32), st, d_);
    if (guess) {
      launch(k_cg_guess<R>, dim3(grid_rows()), dim3(256), st, d_, guess);
      launch(k_cg_init_guess<R>, dim3(upd_grid_), dim3(kThreads), st, d_, rhs);
    } else {
      launch(k_cg_init<R>, dim3(upd_grid_), dim3(kThreads), st, d_, rhs);
    }
    launch(k_cg_scalar_init<R>, dim3(scalar_grid()), dim3(256), st, d_, phase, guess ? 1 : 0);
    CLOTH_CUDA(cudaGetLastError());
    if (capturing) {
      cudaStreamCaptureStatus cs;
      cudaGraph_t g;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      CLOTH_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
      cudaGraphConditionalHandle cond;
      CLOTH_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
      launch(k_cond_set<R>, dim3(1), dim3(32), st, d_, cond);
      CLOTH_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &ndeps));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      CLOTH_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
      CLOTH_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      CLOTH_CUDA(cudaStreamBeginCaptureToGraph(body_stream_, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      emit_cg_body(body_stream_, phase, cond, 1);
      cudaGraph_t out = nullptr;
      CLOTH_CUDA(cudaStreamEndCapture(body_stream_, &out));
      CLOTH_CUDA(cudaGetLastError());
      CLOTH_TRY(emit_tail(st, phase));
      emit_solution(st, guess != nullptr, keep);
      return CLOTH_OK;
    }
    const int poll = std::max(1, o_.cg_poll_every);
    int launched = 0;
    while (true) {
      CLOTH_CUDA(cudaMemcpyAsync(host_active_, d_.active, sizeof(int), cudaMemcpyDeviceToHost, st));
      CLOTH_CUDA(cudaStreamSynchronize(st));
      if (*host_active_ <= d_.tail_threshold || launched >= o_.cg_max_iter) break;
      for (int k = 0; k < poll; ++k) {
        emit_cg_body(st, phase, 0, 0);
      }
      launched += poll;
      CLOTH_CUDA(cudaGetLastError());
    }
    CLOTH_TRY(emit_tail(st, phase));
    emit_solution(st, guess != nullptr, keep);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  // FP32 mode accumulates the solution as float-float; its consumers read FP64.  A solve
  // from a guess also needs its b = 0 sheets set to 0, and a kept solution its copy.
  void emit_solution(cudaStream_t st, bool guessed, double* keep) {
    if (std::is_same<R, float>::value || guessed || keep)
      launch(k_cg_solution<R>, dim3(grid_rows()), dim3(256), st, d_, keep);
  }

  // the sheets still running after the device loop finish in the per-sheet cluster
  // solver: one launch per size class, on its own stream so the classes run side by side
  template <int EPC, int MINB = (EPC == 1 ? 2 : 1)>
  cudaError_t launch_class(const SheetClass& c, int phase, const int* lists) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(c.n * c.CL));
    lc.blockDim = dim3(kThreads * EPC);
    lc.stream = c.stream;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)c.CL;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    lc.attrs = &at;
    lc.numAttrs = c.CL > 1 ? 1 : 0;
    ++launches_;
    return cudaLaunchKernelEx(&lc, k_cg_sheet<R, EPC, MINB>, d_, (const int*)(lists + c.offset), c.n, c.CL, phase);
  }

  cudaError_t launch_sm_class(const SmClass& c, int phase) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(c.n * c.CL));
    lc.blockDim = dim3((unsigned)c.MR);
    lc.dynamicSmemBytes = c.smem;
    lc.stream = c.stream;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)c.CL;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    lc.attrs = &at;
    lc.numAttrs = c.CL > 1 ? 1 : 0;
    ++launches_;
    return cudaLaunchKernelEx(&lc, k_cg_sheet_sm<R>, d_, (const SmSheet*)(sm_lists_ + c.offset), c.CL, phase);
  }

  int emit_tail(cudaStream_t st, int phase) {
    if (d_.tail_threshold <= 0) return CLOTH_OK;
    auto& set = use_sm_ ? rest_classes_ : use_dense_ ? dense_classes_ : classes_;
    const int* lists = use_sm_ ? rest_lists_ : use_dense_ ? dense_lists_ : sheet_lists_;
    // the classes' sheets in launch order, longest last solve first
    auto lo = orders_.find(lists);
    if (lo != orders_.end()) {
      launch(k_order_lists<R>, dim3(lo->second.nclasses), dim3(256), st, d_, lo->second.seg, lists,
             lo->second.order);
      lists = lo->second.order;
    }
    CLOTH_CUDA(cudaEventRecord(fork_ev_, st));
    if (use_sm_) {
      for (auto& c : sm_classes_) {
        CLOTH_CUDA(cudaStreamWaitEvent(c.stream, fork_ev_, 0));
        CLOTH_CUDA(launch_sm_class(c, phase));
        CLOTH_CUDA(cudaEventRecord(c.done, c.stream));
        CLOTH_CUDA(cudaStreamWaitEvent(st, c.done, 0));
      }
    }
    for (auto& c : set) {
      CLOTH_CUDA(cudaStreamWaitEvent(c.stream, fork_ev_, 0));
      const cudaError_t le = c.dense ? launch_class<2, 2>(c, phase, lists)
                             : c.EPC == 1 ? launch_class<1>(c, phase, lists)
                             : c.EPC == 2 ? launch_class<2>(c, phase, lists)
                             : c.EPC == 3 ? launch_class<3>(c, phase, lists) : launch_class<4>(c, phase, lists);
      CLOTH_CUDA(le);
      CLOTH_CUDA(cudaEventRecord(c.done, c.stream));
      CLOTH_CUDA(cudaStreamWaitEvent(st, c.done, 0));
    }
    return CLOTH_OK;
  }

  // The velocity a step starts from: v, or v + F_t with velocity-increment forces.
  const double* start_velocity(const double* v, const R* F, cudaStream_t st) {
    if (o_.force_mode != CLOTH_FORCES_VELOCITY || !F) return v;
    launch(k_add_increment<R>, dim3(grid_rows()), dim3(256), st, d_, v, F, vin_);
    return vin_;
  }

  // One implicit step from (x, v) to (xn, vn); F: user-layout force row (or velocity
  // increments, by the force mode) or null.
  int step(const double* x, const double* v0, const R* F, double* xn, double* vn, R* traj_row, int phase,
           cudaStream_t st, bool cap) {
    const double* v = start_velocity(v0, F, st);
    if (o_.force_mode == CLOTH_FORCES_VELOCITY) F = nullptr;
    elements(x, v, st);
    launch(k_assemble<R>, dim3(d_.NW), dim3(kThreads), st, d_, F, v);
    CLOTH_CUDA(cudaGetLastError());
    CLOTH_TRY(solve(d_.bvec, phase, st, cap, guess_f_, guess_f_));
    launch(k_state_update<R>, dim3(grid_rows()), dim3(256), st, d_, x, v, xn, vn, traj_row);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  const R* force_row(const void* forces, int t) const {
    return forces ? (const R*)forces + (size_t)t * 3 * L_.Nu : nullptr;
  }

  int forward_body(const void* material, const void* x0, const void* v0, const void* forces, void* traj_x,
                   int32_t* status, cudaStream_t st, bool cap) {
    const size_t nu3 = 3 * (size_t)L_.Nu;
    CLOTH_CUDA(cudaMemcpyAsync(mat_, material, sizeof(R) * 4 * L_.S, cudaMemcpyDeviceToDevice, st));
    launch(k_reset_status<R>, dim3((L_.S + 255) / 256), dim3(256), st, d_, (int)kPhaseForward);
    gather_state((const R*)x0, sx(0), st);
    gather_state((const R*)v0, sv(0), st);
    launch(k_check_pins<R>, dim3(grid_rows()), dim3(256), st, d_, (const double*)sv(0));
    if (guess_f_) CLOTH_CUDA(cudaMemsetAsync(guess_f_, 0, sizeof(double) * n3(), st));
    CLOTH_CUDA(cudaMemcpyAsync(traj_x, x0, sizeof(R) * nu3, cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k < nseg_; ++k) {
      const int t0 = k * C_, t1 = std::min(T_, t0 + C_);
      if (k > 0) {
        CLOTH_CUDA(cudaMemcpyAsync(sx(0), sx(C_), sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
        CLOTH_CUDA(cudaMemcpyAsync(sv(0), sv(C_), sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
      }
      if (nseg_ > 1) {
        CLOTH_CUDA(cudaMemcpyAsync(ck_x_ + n3() * k, sx(0), sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
        CLOTH_CUDA(cudaMemcpyAsync(ck_v_ + n3() * k, sv(0), sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
        if (ck_g_)
          CLOTH_CUDA(cudaMemcpyAsync(ck_g_ + n3() * k, guess_f_, sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
      }
      for (int t = t0; t < t1; ++t) {
        const int j = t - t0;
        R* row = (R*)traj_x + (size_t)(t + 1) * nu3;
        CLOTH_TRY(step(sx(j), sv(j), force_row(forces, t), sx(j + 1), sv(j + 1), row, kPhaseForward, st, cap));
      }
    }
    launch(k_status_out<R>, dim3((L_.S + 255) / 256), dim3(256), st, d_, status);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  int backward_body(const void* dL_dx, void* g_material, void* g_forces, void* g_x0, void* g_v0, int32_t* status,
                    cudaStream_t st, bool cap, int seg_valid) {
    const size_t nu3 = 3 * (size_t)L_.Nu;
    launch(k_reset_status<R>, dim3((L_.S + 255) / 256), dim3(256), st, d_, (int)kPhaseBackward);
    launch(k_reset_status<R>, dim3((L_.S + 255) / 256), dim3(256), st, d_, (int)kPhaseRecompute);
    CLOTH_CUDA(cudaMemsetAsync(d_.gacc, 0, sizeof(double) * 3 * L_.S, st));
    CLOTH_CUDA(cudaMemsetAsync(d_.gacc_w, 0, sizeof(double) * 3 * L_.S, st));
    gather_state((const R*)dL_dx + (size_t)T_ * nu3, ax_, st);
    CLOTH_CUDA(cudaMemsetAsync(av_, 0, sizeof(double) * n3(), st));
    if (guess_a_) CLOTH_CUDA(cudaMemsetAsync(guess_a_, 0, sizeof(double) * n3(), st));
    const int gm = (L_.M + kElemThreads - 1) / kElemThreads, ge = (L_.E + kElemThreads - 1) / kElemThreads;
    for (int k = nseg_ - 1; k >= 0; --k) {
      const int t0 = k * C_, t1 = std::min(T_, t0 + C_);
      // The segment buffer still holds segment k only if it is the first one swept
      // (the last segment of the forward); any other segment is recomputed.
      if (!(k == nseg_ - 1 && seg_valid == nseg_ - 1)) {
        CLOTH_CUDA(cudaMemcpyAsync(sx(0), ck_x_ + n3() * k, sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
        CLOTH_CUDA(cudaMemcpyAsync(sv(0), ck_v_ + n3() * k, sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
        if (ck_g_)
          CLOTH_CUDA(cudaMemcpyAsync(guess_f_, ck_g_ + n3() * k, sizeof(double) * n3(), cudaMemcpyDeviceToDevice, st));
        for (int t = t0; t < t1; ++t) {
          const int j = t - t0;
          CLOTH_TRY(step(sx(j), sv(j), force_row(fwd_forces_, t), sx(j + 1), sv(j + 1), nullptr, kPhaseRecompute, st,
                         cap));
        }
      }
      for (int t = t1 - 1; t >= t0; --t) {
        const int j = t - t0;
        // A_t at x_t (the RHS of the step matrix is not needed)
        const double* vstart = start_velocity(sv(j), force_row(fwd_forces_, t), st);
        elements(sx(j), nullptr, st);
        launch(k_assemble<R>, dim3(d_.NW), dim3(kThreads), st, d_, (const R*)nullptr, vstart);
        launch(k_adj_rhs<R>, dim3(grid_rows()), dim3(256), st, d_, (const double*)ax_, (const double*)av_);
        CLOTH_CUDA(cudaGetLastError());
        CLOTH_TRY(solve(d_.bvec, kPhaseBackward, st, cap, guess_a_, guess_a_));
        if (L_.M) launch(k_adj_tri<R>, dim3(gm), dim3(kElemThreads), st, d_, (const double*)sx(j), (const double*)d_.dv, (const double*)sv(j + 1), 0);
        if (L_.E) launch(k_adj_hinge<R>, dim3(ge), dim3(kElemThreads), st, d_, (const double*)sx(j), (const double*)d_.dv, (const double*)sv(j + 1), 0);
        R* gF = g_forces ? (R*)g_forces + (size_t)t * nu3 : nullptr;
        launch(k_adj_vertex<R>, dim3(grid_rows()), dim3(256), st, d_, ax_, av_, vstart, (const double*)sv(j + 1),
               (const R*)dL_dx + (size_t)t * nu3, gF, (int)o_.force_mode);
        launch(k_param_acc<R>, dim3(L_.S), dim3(kThreads), st, d_);
        CLOTH_CUDA(cudaGetLastError());
      }
    }
    if (g_material) launch(k_grad_material<R>, dim3((L_.S + 127) / 128), dim3(128), st, d_, (R*)g_material);
    if (g_x0) launch(k_scatter<R, double>, dim3(grid_rows()), dim3(256), st, d_, (const double*)ax_, (R*)g_x0);
    if (g_v0) launch(k_scatter<R, double>, dim3(grid_rows()), dim3(256), st, d_, (const double*)av_, (R*)g_v0);
    launch(k_status_out<R>, dim3((L_.S + 255) / 256), dim3(256), st, d_, status);
    CLOTH_CUDA(cudaGetLastError());
    return CLOTH_OK;
  }

  // Capture `body` into a graph once per argument set, then launch it on `st`.
  template <class Body>
  int run_graph(const GraphKey& key, cudaStream_t st, int64_t* fixed, Body body) {
    for (auto& g : graphs_)
      if (g.key == key) {
        *fixed = g.fixed;
        CLOTH_CUDA(cudaGraphLaunch(g.exec, st));
        return CLOTH_OK;
      }
    launches_ = 0;
    CLOTH_CUDA(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeRelaxed));
    int rc = body(cap_stream_);
    *fixed = launches_;
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cap_stream_, &graph);
    if (rc != CLOTH_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) {
      set_last_error(std::string("graph capture failed: ") + cudaGetErrorString(ec));
      return CLOTH_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      set_last_error(std::string("graph instantiation failed: ") + cudaGetErrorString(ei));
      return CLOTH_ERR_CUDA;
    }
    if (graphs_.size() >= 8) {
      cudaGraphExecDestroy(graphs_.front().exec);
      graphs_.erase(graphs_.begin());
    }
    graphs_.push_back({key, exec, *fixed});
    CLOTH_CUDA(cudaGraphLaunch(exec, st));
    return CLOTH_OK;
  }

  BatchLayout L_;
  const void* fwd_forces_ = nullptr;  // force input of the last forward (the recompute reads it again)
  cloth_opts o_;
  Dev<R> d_ = {};
  int T_ = 0, C_ = 0, nseg_ = 0, seg_valid_ = -1;
  bool have_forward_ = false;
  double *seg_x_ = nullptr, *seg_v_ = nullptr, *ck_x_ = nullptr, *ck_v_ = nullptr;
  double *tmp_xd_ = nullptr, *tmp_vd_ = nullptr, *tmp_ud_ = nullptr;
  double* vin_ = nullptr;  // a step's starting velocity v_t + F_t (velocity-increment forces)
  const R* wind_ = nullptr;  // per-sheet wind velocity [S][3] given by cloth_set_wind
  double *ax_ = nullptr, *av_ = nullptr;
  // warm start (cloth_opts.cg_warm_start): each forward (and recomputed) solve starts from
  // the previous step's dv, each adjoint solve from the lambda of the step after it
  double *guess_f_ = nullptr, *guess_a_ = nullptr, *ck_g_ = nullptr;
  R *tmp_a_ = nullptr, *tmp_b_ = nullptr;
  R *mat_ = nullptr, *mat_tmp_ = nullptr;
  double* lpart_ = nullptr;
  int* host_active_ = nullptr;
  cudaStream_t cap_stream_ = nullptr, body_stream_ = nullptr, last_stream_ = nullptr;
  std::vector<CachedGraph> graphs_;
  int64_t launches_ = 0, fixed_fwd_ = 0, fixed_bwd_ = 0;
  int64_t timed_solve_bytes_ = -1;  // algorithmic bytes of the last solve timed as kernel 5
  int spmv_grid_ = 1, upd_grid_ = 1;  // CTAs of the SpMV and of the other CG row kernels
  std::vector<SheetClass> classes_;  // size classes of the per-sheet cluster solver
  const int* sheet_lists_ = nullptr;  // their sheets, class after class
  struct ListOrder {
    const int* seg = nullptr;  // [classes + 1] offsets of the classes in the list
    int* order = nullptr;      // the list in launch order (k_order_lists)
    int nclasses = 0;
  };
  std::map<const int*, ListOrder> orders_;  // by class list
  // on-chip solver: its size classes (one cluster size each), their partitions, and the
  // k_cg_sheet classes of the sheets it cannot hold
  std::vector<SmClass> sm_classes_;
  const SmSheet* sm_lists_ = nullptr;
  std::vector<SheetClass> rest_classes_;
  const int* rest_lists_ = nullptr;
  bool use_sm_ = false;
  std::vector<SheetClass> dense_classes_;  // schedule bit 4
  const int* dense_lists_ = nullptr;
  bool dense_ok_ = false, use_dense_ = false;
  bool sheet_solver_ok_ = false;      // every sheet fits one cluster
  int tri_nt_ = kElemThreads, hin_nt_ = kElemThreads;  // element kernels' block sizes (autotuned)
  bool wide2_ok_ = false, wide3_ok_ = false;  // 16-CTA clusters of 2 or 3 entries per CTA launchable
  int handover_ = 1 << 30;            // sheets left when the device loop hands over
  cudaEvent_t fork_ev_ = nullptr;
  int res_spmv_ = 1, res_upd_ = 1;  // CTAs resident at once (SpMV, update)
  int schedule_ = 3;
  cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
  std::vector<void*> allocs_;
  size_t bytes_ = 0;
};

template <class R>
std::unique_ptr<EngineBase> make_engine(const BatchLayout& L, const cloth_opts& o, int* rc, std::string* err) {
  auto e = std::make_unique<Engine<R>>(L, o);
  *rc = e->init(err);
  if (*rc != CLOTH_OK) return nullptr;
  return e;
}

}  // namespace cloth
