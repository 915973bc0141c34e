// FP64 instantiation of the cloth engine (every stage in double).
#include "engine_impl.cuh"

namespace cloth {
std::unique_ptr<EngineBase> make_engine_f64(const BatchLayout& L, const cloth_opts& o, int* rc, std::string* err) {
  return make_engine<double>(L, o, rc, err);
}
}  // namespace cloth
