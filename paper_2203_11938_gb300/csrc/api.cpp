// extern "C" entry points of include/cloth_sim.h (argument checks, handles, dispatch).
#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/cloth_sim.h"
#include "engine.h"
#include "prep.h"

struct cloth_mesh {
  cloth::MeshData data;
};

struct cloth_batch {
  cloth_opts opts;
  std::unique_ptr<cloth::EngineBase> engine;
};

namespace cloth {
namespace {
thread_local std::string g_last_error;
}
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace cloth

using cloth::set_last_error;

namespace {
int fail(int rc, const std::string& msg) {
  set_last_error(msg);
  return rc;
}
}  // namespace

extern "C" {

const char* cloth_last_error(void) { return cloth::g_last_error.c_str(); }

void cloth_default_opts(cloth_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = CLOTH_FP32;
  o->steps = 1;
  o->dt = 1.0 / 30.0;
  o->cg_tol = 1e-6;
  o->cg_max_iter = 2000;
  o->checkpoint_every = 0;
  o->gravity[2] = -9.8;
  o->clamp_eta = 1e-3;
  o->exec = CLOTH_EXEC_GRAPH;
  o->cg_poll_every = 16;
  o->precond = CLOTH_PRECOND_BLOCK_JACOBI;
  o->cg_schedule = -1;
  o->cg_handover = 0;
  o->force_mode = CLOTH_FORCES_FORCE;
  o->air_density = 0.0;
  o->cg_warm_start = 0;
}

int cloth_mesh_create(const double* rest_xyz, int32_t n, const int32_t* tris, int32_t m, const uint8_t* pinned,
                      cloth_mesh** out) {
  if (!out) return fail(CLOTH_ERR_INVALID_ARG, "cloth_mesh_create: out is null");
  *out = nullptr;
  auto mesh = std::make_unique<cloth_mesh>();
  std::string err;
  int rc = cloth::build_mesh(rest_xyz, n, tris, m, pinned, &mesh->data, &err);
  if (rc != CLOTH_OK) return fail(rc, "cloth_mesh_create: " + err);
  *out = mesh.release();
  set_last_error("");
  return CLOTH_OK;
}

int cloth_mesh_destroy(cloth_mesh* mesh) {
  delete mesh;
  return CLOTH_OK;
}

int cloth_mesh_info(const cloth_mesh* mesh, int32_t* n, int32_t* m, int32_t* hinges) {
  if (!mesh) return fail(CLOTH_ERR_INVALID_ARG, "cloth_mesh_info: mesh is null");
  if (n) *n = mesh->data.n;
  if (m) *m = mesh->data.m;
  if (hinges) *hinges = mesh->data.num_hinges();
  return CLOTH_OK;
}

int cloth_batch_create(const cloth_mesh* const* meshes, int32_t count, const cloth_opts* opts, cloth_batch** out) {
  if (!out) return fail(CLOTH_ERR_INVALID_ARG, "cloth_batch_create: out is null");
  *out = nullptr;
  if (!meshes || count < 1 || !opts) return fail(CLOTH_ERR_INVALID_ARG, "cloth_batch_create: need >= 1 mesh and opts");
  const cloth_opts& o = *opts;
  if (o.precision != CLOTH_FP32 && o.precision != CLOTH_FP64)
    return fail(CLOTH_ERR_INVALID_ARG, "cloth_batch_create: precision must be CLOTH_FP32 or CLOTH_FP64");
  if (o.steps < 1 || !(o.dt > 0.0) || !(o.cg_tol >= 0.0) || o.cg_max_iter < 1 || o.checkpoint_every < 0 ||
      !(o.clamp_eta >= 0.0) || (o.exec != CLOTH_EXEC_PLAIN && o.exec != CLOTH_EXEC_GRAPH) || o.cg_poll_every < 1 ||
      (o.precond != CLOTH_PRECOND_JACOBI && o.precond != CLOTH_PRECOND_BLOCK_JACOBI) || o.cg_schedule < -1 ||
      o.cg_schedule > 31 || o.cg_handover < 0 ||
      (o.force_mode != CLOTH_FORCES_FORCE && o.force_mode != CLOTH_FORCES_VELOCITY) ||
      !(o.air_density >= 0.0) || (o.cg_warm_start != 0 && o.cg_warm_start != 1))
    return fail(CLOTH_ERR_INVALID_ARG, "cloth_batch_create: invalid option value");
  std::vector<const cloth::MeshData*> sheets;
  for (int i = 0; i < count; ++i) {
    if (!meshes[i]) return fail(CLOTH_ERR_INVALID_ARG, "cloth_batch_create: null mesh");
    sheets.push_back(&meshes[i]->data);
  }
  auto b = std::make_unique<cloth_batch>();
  b->opts = o;
  cloth::BatchLayout L;
  cloth::build_layout(sheets, &L);
  std::string err;
  int rc = CLOTH_OK;
  b->engine = o.precision == CLOTH_FP32 ? cloth::make_engine_f32(L, o, &rc, &err)
                                        : cloth::make_engine_f64(L, o, &rc, &err);
  if (!b->engine) return fail(rc == CLOTH_OK ? CLOTH_ERR_CUDA : rc, "cloth_batch_create: " + err);
  *out = b.release();
  set_last_error("");
  return CLOTH_OK;
}

int cloth_batch_destroy(cloth_batch* batch) {
  delete batch;
  return CLOTH_OK;
}

int cloth_batch_info(const cloth_batch* batch, int32_t* total_vertices, int32_t* count, size_t* workspace_bytes) {
  if (!batch) return fail(CLOTH_ERR_INVALID_ARG, "cloth_batch_info: batch is null");
  if (total_vertices) *total_vertices = batch->engine->total_vertices();
  if (count) *count = batch->engine->count();
  if (workspace_bytes) *workspace_bytes = batch->engine->workspace_bytes();
  return CLOTH_OK;
}

#define CLOTH_NEED_BATCH(name) \
  if (!batch) return fail(CLOTH_ERR_INVALID_ARG, name ": batch is null")

int cloth_forward(cloth_batch* batch, const void* material, const void* x0, const void* v0, const void* forces,
                  void* traj_x, int32_t* status, void* stream) {
  CLOTH_NEED_BATCH("cloth_forward");
  return batch->engine->forward(material, x0, v0, forces, traj_x, status, stream);
}

int cloth_backward(cloth_batch* batch, const void* dL_dx, void* g_material, void* g_forces, void* g_x0, void* g_v0,
                   int32_t* status, void* stream) {
  CLOTH_NEED_BATCH("cloth_backward");
  return batch->engine->backward(dL_dx, g_material, g_forces, g_x0, g_v0, status, stream);
}

int cloth_loss_l2(cloth_batch* batch, const void* traj_x, const void* target, double* loss, void* dL_dx,
                  void* stream) {
  CLOTH_NEED_BATCH("cloth_loss_l2");
  return batch->engine->loss_l2(traj_x, target, loss, dL_dx, stream);
}

int cloth_loss_pinhole(cloth_batch* batch, const void* traj_x, const void* target_uv, const double* camera,
                       double* loss, void* dL_dx, void* stream) {
  CLOTH_NEED_BATCH("cloth_loss_pinhole");
  return batch->engine->loss_pinhole(traj_x, target_uv, camera, loss, dL_dx, stream);
}

int cloth_stats(cloth_batch* batch, int64_t* fwd, int64_t* bwd, int64_t* rec, int64_t* launches) {
  CLOTH_NEED_BATCH("cloth_stats");
  return batch->engine->stats(fwd, bwd, rec, launches);
}

int cloth_sheet_iterations(cloth_batch* batch, int32_t phase, int32_t* max_iters, int64_t* total_iters) {
  CLOTH_NEED_BATCH("cloth_sheet_iterations");
  if (phase < 0 || phase > 3) {
    cloth::set_last_error(
        "cloth_sheet_iterations: phase must be 0 (forward), 1 (adjoint), 2 (recomputed forward) or 3 (timed)");
    return CLOTH_ERR_INVALID_ARG;
  }
  return batch->engine->sheet_iterations(phase, max_iters, total_iters);
}

int cloth_matrix_info(const cloth_batch* batch, int64_t* rows, int64_t* blocks, int64_t* stored_blocks,
                      int32_t* cg_schedule) {
  CLOTH_NEED_BATCH("cloth_matrix_info");
  return batch->engine->matrix_info(rows, blocks, stored_blocks, cg_schedule);
}

int cloth_set_wind(cloth_batch* batch, const void* wind) {
  CLOTH_NEED_BATCH("cloth_set_wind");
  return batch->engine->set_wind(wind);
}

int cloth_wind_gradient(cloth_batch* batch, void* g_wind, void* stream) {
  CLOTH_NEED_BATCH("cloth_wind_gradient");
  return batch->engine->wind_gradient(g_wind, stream);
}

int cloth_kernel_bytes(cloth_batch* batch, int32_t kernel, int64_t* bytes) {
  CLOTH_NEED_BATCH("cloth_kernel_bytes");
  return batch->engine->kernel_bytes(kernel, bytes);
}

int cloth_time_kernel(cloth_batch* batch, int32_t kernel, int32_t reps, double* avg_ms, void* stream) {
  CLOTH_NEED_BATCH("cloth_time_kernel");
  return batch->engine->time_kernel(kernel, reps, avg_ms, stream);
}

int cloth_internal_forces(cloth_batch* batch, const void* material, const void* x, void* f_membrane,
                          void* f_bending, void* stream) {
  CLOTH_NEED_BATCH("cloth_internal_forces");
  return batch->engine->internal_forces(material, x, f_membrane, f_bending, stream);
}

int cloth_system_dense(cloth_batch* batch, const void* material, const void* x, const void* v, const void* F,
                       void* A, void* b, void* stream) {
  CLOTH_NEED_BATCH("cloth_system_dense");
  return batch->engine->system_dense(material, x, v, F, A, b, stream);
}

int cloth_spmv(cloth_batch* batch, const void* material, const void* x, const void* v, const void* p, void* y,
               void* stream) {
  CLOTH_NEED_BATCH("cloth_spmv");
  return batch->engine->spmv(material, x, v, p, y, stream);
}

int cloth_third_contraction(cloth_batch* batch, const void* material, const void* x, const void* a, const void* b,
                            void* out, void* stream) {
  CLOTH_NEED_BATCH("cloth_third_contraction");
  return batch->engine->third(material, x, a, b, out, stream);
}

}  // extern "C"
