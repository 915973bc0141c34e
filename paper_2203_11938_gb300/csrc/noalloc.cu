// Trajectory L2 loss without any device allocation (see cloth_loss_l2_static in
// include/cloth_sim.h).  The kernels are the ones cloth_loss_l2 runs; only the scratch
// that holds one partial sum per (sheet, time step) differs: here it is a file-scope
// device array instead of memory the batch handle allocated.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "engine.cuh"

namespace cloth {
namespace {

constexpr int kStaticPartials = 1 << 16;  // 65,536 doubles = 512 KiB per device
constexpr int kMaxDevices = 64;

// One array per device that loads this library, kept until the process exits.  In host
// code `g_loss_partials` names a host-side stand-in, never the device address: the
// address is obtained per device with cudaGetSymbolAddress below.
static __device__ __align__(256) double g_loss_partials[kStaticPartials];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the static array for the current device (first call per device does
// the lookup and keeps it for the life of the process; a cudaDeviceReset of that device
// unloads the module, after which the kept address is stale, so the entry point must not
// be used on a device after it was reset).  Returns CLOTH_OK, CLOTH_ERR_INVALID_ARG or
// CLOTH_ERR_CUDA.
int static_partials(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_last_error(std::string("cloth_loss_l2_static: cudaGetDevice failed: ") + cudaGetErrorString(e));
    return CLOTH_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("cloth_loss_l2_static: device index " + std::to_string(dev) + " is beyond the " +
                   std::to_string(kMaxDevices) + " devices this entry point keeps an address for");
    return CLOTH_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loss_partials);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cloth_loss_l2_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return CLOTH_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<double*>(g_addr[dev]);
  return CLOTH_OK;
}

template <class R>
int loss_static(int count, const int* sheet_offsets, int steps, int n_total, const void* traj, const void* target,
                double* loss, void* grad, cudaStream_t st) {
  double* partials = nullptr;
  int rc = static_partials(&partials);
  if (rc != CLOTH_OK) return rc;
  // The loss kernels read only these fields of the batch description.
  Dev<R> d;
  std::memset(&d, 0, sizeof(d));
  d.S = count;
  d.Nu = n_total;
  d.sheet_uoff = sheet_offsets;
  if (grad) {
    // row t = 0 of the gradient is zero (the loss sums t = 1..steps)
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(R) * 3 * (size_t)n_total, st);
    if (e != cudaSuccess) {
      set_last_error(std::string("cloth_loss_l2_static: ") + cudaGetErrorString(e));
      return CLOTH_ERR_CUDA;
    }
  }
  // Every partial (s, t) is written by k_loss_l2 before k_loss_final reads it, so the
  // array needs no clearing between calls.
  k_loss_l2<R><<<dim3(count, steps), kThreads, 0, st>>>(d, steps, (const R*)traj, (const R*)target, (R*)grad,
                                                       partials);
  k_loss_final<R><<<(count + 127) / 128, 128, 0, st>>>(d, steps, partials, loss);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("cloth_loss_l2_static: launch failed: ") + cudaGetErrorString(e));
    return CLOTH_ERR_CUDA;
  }
  return CLOTH_OK;
}

}  // namespace
}  // namespace cloth

extern "C" int cloth_loss_l2_static(int32_t count, const int32_t* sheet_offsets, int32_t steps, int32_t n_total,
                                    int32_t precision, const void* traj_x, const void* target, double* loss,
                                    void* dL_dx, void* stream) {
  using namespace cloth;
  if (count < 1 || steps < 1 || n_total < 1 || !sheet_offsets || !traj_x || !target || !loss ||
      (precision != CLOTH_FP32 && precision != CLOTH_FP64)) {
    set_last_error("cloth_loss_l2_static: need count, steps, n_total >= 1, a valid precision and non-null arrays");
    return CLOTH_ERR_INVALID_ARG;
  }
  if ((long long)count * steps > kStaticPartials || count > 65535 || steps > 65535) {
    set_last_error("cloth_loss_l2_static: count * steps = " + std::to_string((long long)count * steps) +
                   " exceeds the static scratch of " + std::to_string(kStaticPartials) +
                   " partial sums (and each of count, steps must be <= 65535)");
    return CLOTH_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return precision == CLOTH_FP32
             ? loss_static<float>(count, sheet_offsets, steps, n_total, traj_x, target, loss, dL_dx, st)
             : loss_static<double>(count, sheet_offsets, steps, n_total, traj_x, target, loss, dL_dx, st);
}
