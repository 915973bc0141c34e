// FP32 instantiation of the cloth engine (element Hessians, the assembled matrix, SpMV and
// CG vectors in float; CG dot products, residual norms, alpha and the CG solution in
// float-float; state, element force vectors and gradient reductions in double).
#include "engine_impl.cuh"

namespace cloth {
std::unique_ptr<EngineBase> make_engine_f32(const BatchLayout& L, const cloth_opts& o, int* rc, std::string* err) {
  return make_engine<float>(L, o, rc, err);
}
}  // namespace cloth
