// An MVM entry point that allocates no device memory.
//
// The lattice MVM needs work space beyond its inputs and outputs: two [m][k] buffers of
// lattice values and the splat partials.  sgp_mvm / sgp_mvm_ex allocate it on first use
// with cudaMallocAsync.  Some callers cannot allocate at the moment they need a product:
// a serving loop must not call cudaMalloc/cudaFree on its hot path (those calls can
// synchronise the device and stall every other stream), and a process whose device
// memory is already reserved by another allocator's pool has nothing left to hand out.
// sgp_mvm_static serves them from a fixed work area compiled into this library.
#include <mutex>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr size_t kStaticScratchFloats = kStaticScratchBytes / sizeof(float);
constexpr int kMaxDevices = 64;

// The work area.  Every GPU that loads this library holds it until the process exits.
__device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

std::mutex g_scratch_mu;
float* g_scratch_addr[kMaxDevices] = {};

// Device address of the work area on device `dev` (the current device), looked up once
// per device.  The host-side symbol is only a stand-in and must never reach a kernel.
sgp_status scratch_address(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sgp_mvm_static: device ordinal out of range");
    return SGP_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_status(e, "sgp_mvm_static: locating the static work area");
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return SGP_OK;
}

}  // namespace
}  // namespace sgp

using namespace sgp;

extern "C" sgp_status sgp_mvm_static(sgp_lattice* h, const float* V, int k, int blur,
                                     float alpha, float beta, float* out) {
  if (!h) {
    set_error("sgp_mvm_static: null lattice handle");
    return SGP_ERR_INVALID_ARG;
  }
  if (!V || !out || V == out || k < 1 || k > kMaxK || blur < SGP_BLUR_SEQUENTIAL ||
      blur > SGP_BLUR_SYMMETRIC) {
    set_error("sgp_mvm_static: need V, out (not aliasing V), 1 <= k <= 256 and an "
              "SGP_BLUR_* operator");
    return SGP_ERR_INVALID_ARG;
  }
  const size_t need = mvm_work_bytes(h, k);
  if (need > kStaticScratchBytes) {
    set_error("sgp_mvm_static: this lattice needs " + std::to_string(need) +
              " bytes of work space for k = " + std::to_string(k) +
              ", more than the 64 MiB static work area");
    return SGP_ERR_INVALID_ARG;
  }
  clear_pending_error();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "sgp_mvm_static: cudaGetDevice");
  // the work area is per device: the one of the lattice's device must be the one used
  if (dev != h->device) {
    set_error("sgp_mvm_static: the current device (" + std::to_string(dev) +
              ") is not the device the lattice was built on (" + std::to_string(h->device) +
              "); make that device current");
    return SGP_ERR_INVALID_ARG;
  }
  float* base = nullptr;
  if (sgp_status s = scratch_address(dev, &base)) return s;
  // Every element of the value buffers, partials and permuted input is written before it
  // is read, so the contents left by an earlier call need no clearing.
  enqueue_mvm_into(h, V, k, blur, alpha, beta, out, base, h->stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "sgp_mvm_static: launching the lattice MVM");
  return SGP_OK;
}
