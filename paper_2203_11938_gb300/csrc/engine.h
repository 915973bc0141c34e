// Precision-independent interface of the simulation engine (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <string>

#include "../../include/cloth_sim.h"
#include "prep.h"

namespace cloth {

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual int forward(const void* material, const void* x0, const void* v0, const void* forces, void* traj_x,
                      int32_t* status, void* stream) = 0;
  virtual int backward(const void* dL_dx, void* g_material, void* g_forces, void* g_x0, void* g_v0, int32_t* status,
                       void* stream) = 0;
  virtual int loss_l2(const void* traj, const void* target, double* loss, void* grad, void* stream) = 0;
  virtual int loss_pinhole(const void* traj, const void* uv, const double* cam, double* loss, void* grad,
                           void* stream) = 0;
  virtual int stats(int64_t* fwd, int64_t* bwd, int64_t* rec, int64_t* launches) = 0;
  virtual int sheet_iterations(int phase, int32_t* max_iters, int64_t* total_iters) = 0;
  virtual int matrix_info(int64_t* rows, int64_t* blocks, int64_t* slots, int32_t* schedule) = 0;
  virtual int time_kernel(int which, int reps, double* avg_ms, void* stream) = 0;
  virtual int kernel_bytes(int which, int64_t* bytes) = 0;
  virtual int set_wind(const void* wind) = 0;
  virtual int wind_gradient(void* g_wind, void* stream) = 0;
  virtual int internal_forces(const void* material, const void* x, void* fm, void* fb, void* stream) = 0;
  virtual int system_dense(const void* material, const void* x, const void* v, const void* F, void* A, void* b,
                           void* stream) = 0;
  virtual int spmv(const void* material, const void* x, const void* v, const void* p, void* y, void* stream) = 0;
  virtual int third(const void* material, const void* x, const void* a, const void* b, void* out, void* stream) = 0;
  virtual size_t workspace_bytes() const = 0;
  virtual int total_vertices() const = 0;
  virtual int count() const = 0;
};

// Creates the engine for opts->precision; returns nullptr and sets *err on failure.
std::unique_ptr<EngineBase> make_engine_f32(const BatchLayout& L, const cloth_opts& o, int* rc, std::string* err);
std::unique_ptr<EngineBase> make_engine_f64(const BatchLayout& L, const cloth_opts& o, int* rc, std::string* err);

void set_last_error(const std::string& msg);

}  // namespace cloth
