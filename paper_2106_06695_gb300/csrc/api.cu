// C-ABI entry points of the lattice library (declared in include/sgp.h): argument
// validation, handle lifetime and error reporting around the build, MVM and CG paths.
#include <atomic>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sgp_internal.cuh"

namespace sgp {

int injected_fault() {
  const char* f = getenv("SGP_FAULT");
  if (!f || !f[0]) return FAULT_NONE;
  if (!strcmp(f, "oom")) return FAULT_OOM;
  if (!strcmp(f, "cuda_err")) return FAULT_CUDA;
  if (!strcmp(f, "hash_full")) return FAULT_HASH_FULL;
  if (!strcmp(f, "nan_input")) return FAULT_NAN_INPUT;
  return FAULT_NONE;
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

// The library's stream-ordered memory pool per device: freed blocks stay mapped (release
// threshold: all of them) so that the next build or solve reuses them instead of mapping
// fresh pages; sgp_trim_memory returns them.
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kPoolDevices] = {};

cudaError_t pool_of(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    cudaError_t e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      (void)cudaMemPoolDestroy(p);
      return e;
    }
    g_pools[dev] = p;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

bool have_device() {
  int count = 0;
  return cudaGetDeviceCount(&count) == cudaSuccess && count > 0;
}

void free_lattice(Lattice* L) {
  if (!L) return;
  cudaStream_t st = L->stream;
  void* arrays[] = {L->perm, L->idx, L->w, L->rank, L->row_ptr, L->items, L->nbr, L->keys, L->err,
                    L->act, L->act_off_dev, L->epoch, L->act_tmp, L->g0pow,
                    L->lat[0], L->lat[1], L->seg, L->med_rows, L->huge_rows, L->partial,
                    L->vperm};
  for (void* p : arrays)
    if (p) (void)cudaFreeAsync(p, st);
  for (cudaEvent_t ev : L->prof_ev)
    if (ev) (void)cudaEventDestroy(ev);
  delete L;
  clear_pending_error();
}

sgp_status check_handle(const sgp_lattice* h) {
  if (!h) {
    set_error("null lattice handle");
    return SGP_ERR_INVALID_ARG;
  }
  return SGP_OK;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

void clear_pending_error() {
  // SGP_TRACE=1 reports such leftovers on stderr (diagnostics only)
  static const bool trace = getenv("SGP_TRACE") && getenv("SGP_TRACE")[0] == '1';
  const cudaError_t e = cudaGetLastError();
  if (trace && e != cudaSuccess)
    fprintf(stderr, "[sgp] cleared a pending CUDA error: %s\n", cudaGetErrorName(e));
}

void note_launches(int64_t count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  if (e == cudaSuccess) e = pool_of(dev, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

sgp_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    set_error(std::string(what) + ": out of device memory");
    return SGP_ERR_OOM;
  }
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return SGP_ERR_CUDA;
}

}  // namespace sgp

using namespace sgp;

extern "C" {

void sgp_opts_init(sgp_opts* o) {
  if (!o) return;
  o->order_r = 1;
  o->kernel = SGP_KERNEL_RBF_BINOMIAL;
  o->spacing_s = 0.0;
  o->outputscale = 1.0f;
  o->value_dtype = SGP_VALUES_F32;
  o->check_every = 8;
  o->stream = nullptr;
  o->precond_rank = 0;
  o->precond_seed = 0;
  o->precond_power_iters = 1;
}

sgp_status sgp_stencil(int kernel, int order_r, double spacing_override, double* spacing_s,
                       double* coef, double* half_coef) {
  double s = 0.0, c[kMaxOrder + 1], g[kMaxOrder + 1];
  if (!make_stencil(kernel, order_r, spacing_override, &s, c, g)) {
    set_error("sgp_stencil: kernel must be an SGP_KERNEL_* value and 1 <= order_r <= 4");
    return SGP_ERR_INVALID_ARG;
  }
  if (spacing_s) *spacing_s = s;
  for (int t = 0; t <= order_r; ++t) {
    if (coef) coef[t] = c[t];
    if (half_coef) half_coef[t] = g[t];
  }
  return SGP_OK;
}

sgp_status sgp_lattice_build(const float* X, const float* lengthscales, int64_t n, int d,
                             const sgp_opts* opts, sgp_lattice** out) {
  if (!out) {
    set_error("sgp_lattice_build: out is null");
    return SGP_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sgp_opts o;
  sgp_opts_init(&o);
  if (opts) o = *opts;
  if (!X || !lengthscales || n < 1 || d < 1 || d + 1 > kMaxD) {
    set_error("sgp_lattice_build: need X, lengthscales, n >= 1 and 1 <= d <= 127");
    return SGP_ERR_INVALID_ARG;
  }
  if (n * (int64_t)(d + 1) > (int64_t)0x7fffffff) {
    set_error("sgp_lattice_build: n * (d + 1) must stay below 2^31");
    return SGP_ERR_INVALID_ARG;
  }
  if (o.value_dtype != SGP_VALUES_F32 && o.value_dtype != SGP_VALUES_BF16) {
    set_error("sgp_lattice_build: unknown value_dtype");
    return SGP_ERR_INVALID_ARG;
  }
  if (!have_device()) {
    set_error("sgp_lattice_build: no CUDA device (this library has no CPU path)");
    return SGP_ERR_CUDA;
  }
  clear_pending_error();
  NvtxRange nvtx("sgp_build");
  const int fault = injected_fault();
  if (fault == FAULT_OOM) {
    set_error("sgp_lattice_build: out of device memory (injected by SGP_FAULT=oom)");
    return SGP_ERR_OOM;
  }
  if (fault == FAULT_CUDA) {
    set_error("sgp_lattice_build: CUDA error (injected by SGP_FAULT=cuda_err)");
    return SGP_ERR_CUDA;
  }
  Lattice* L = new Lattice();
  L->fault = fault;
  L->n = n;
  L->d = d;
  L->D = d + 1;
  L->r = o.order_r;
  L->kernel = o.kernel;
  L->outputscale = o.outputscale;
  L->value_dtype = o.value_dtype;
  L->check_every = o.check_every > 0 ? o.check_every : 8;
  if (o.precond_rank < 0 || o.precond_rank > kMaxLibRank || o.precond_power_iters < 0 ||
      o.precond_power_iters > 1) {
    delete L;
    set_error("sgp_lattice_build: precond_rank must be in 0..4096 and precond_power_iters "
              "0 or 1");
    return SGP_ERR_INVALID_ARG;
  }
  L->precond_rank = o.precond_rank;
  L->precond_power_iters = o.precond_power_iters;
  L->precond_seed = o.precond_seed;
  L->stream = (cudaStream_t)o.stream;
  if (cudaGetDevice(&L->device) != cudaSuccess) L->device = -1;
  if (!make_stencil(o.kernel, o.order_r, o.spacing_s, &L->s, L->coef, L->half)) {
    delete L;
    set_error("sgp_lattice_build: kernel must be an SGP_KERNEL_* value and 1 <= order_r <= 4");
    return SGP_ERR_INVALID_ARG;
  }
  cudaError_t e = dev_malloc((void**)&L->err, sizeof(unsigned), L->stream);
  if (e != cudaSuccess) {
    delete L;
    return cuda_status(e, "sgp_lattice_build: allocating the error word");
  }
  sgp_status s = build_lattice(L, X, lengthscales);
  if (s != SGP_OK) {
    free_lattice(L);
    return s;
  }
  *out = L;
  return SGP_OK;
}

sgp_status sgp_lattice_info(const sgp_lattice* h, int64_t* m, size_t* device_bytes) {
  if (sgp_status s = check_handle(h)) return s;
  if (m) *m = h->m;
  if (device_bytes) *device_bytes = h->bytes;
  return SGP_OK;
}

sgp_status sgp_lattice_blur_lists(const sgp_lattice* h, int* sparse, int64_t* pairs) {
  if (sgp_status s = check_handle(h)) return s;
  if (sparse) *sparse = h->sparse ? 1 : 0;
  if (pairs) *pairs = h->sparse ? h->act_off.back() : -1;
  return SGP_OK;
}

sgp_status sgp_lattice_stencil(const sgp_lattice* h, int* order_r, double* spacing_s,
                               double* coef, double* half_coef) {
  if (sgp_status s = check_handle(h)) return s;
  if (order_r) *order_r = h->r;
  if (spacing_s) *spacing_s = h->s;
  for (int t = 0; t <= h->r; ++t) {
    if (coef) coef[t] = h->coef[t];
    if (half_coef) half_coef[t] = h->half[t];
  }
  return SGP_OK;
}

sgp_status sgp_lattice_export(const sgp_lattice* h, int16_t* keys, int32_t* idx, float* w) {
  if (sgp_status s = check_handle(h)) return s;
  const int64_t n = h->n, D = h->D, nD = n * D;
  cudaStream_t st = h->stream;
  if (keys) {
    cudaError_t e = cudaMemcpyAsync(keys, h->keys, h->m * D * sizeof(int16_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e, "sgp_lattice_export: keys");
  }
  if (idx || w) {
    std::vector<int32_t> perm(n), hidx(nD);
    std::vector<float> hw(nD);
    cudaError_t e = cudaMemcpyAsync(perm.data(), h->perm, n * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hidx.data(), h->idx, nD * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hw.data(), h->w, nD * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "sgp_lattice_export: idx/w");
    for (int64_t p = 0; p < n; ++p) {
      const int64_t i = perm[p];
      for (int64_t c = 0; c < D; ++c) {
        if (idx) idx[i * D + c] = hidx[p * D + c];
        if (w) w[i * D + c] = hw[p * D + c];
      }
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "sgp_lattice_export");
  return SGP_OK;
}

sgp_status sgp_set_stream(sgp_lattice* h, void* stream) {
  if (sgp_status s = check_handle(h)) return s;
  h->stream = (cudaStream_t)stream;
  return SGP_OK;
}

static sgp_status check_mvm_args(const sgp_lattice* h, const float* V, int k, int blur,
                                 const float* out, const char* who) {
  if (sgp_status s = check_handle(h)) return s;
  if (!V || !out || k < 1 || k > kMaxK || blur < SGP_BLUR_SEQUENTIAL || blur > SGP_BLUR_SYMMETRIC) {
    set_error(std::string(who) + ": need V, out, 1 <= k <= 256 and an SGP_BLUR_* operator");
    return SGP_ERR_INVALID_ARG;
  }
  if (V == out) {
    set_error(std::string(who) + ": out must not alias the input");
    return SGP_ERR_INVALID_ARG;
  }
  return SGP_OK;
}

sgp_status sgp_mvm(sgp_lattice* h, const float* V, int k, float* out) {
  if (sgp_status s = check_mvm_args(h, V, k, SGP_BLUR_SEQUENTIAL, out, "sgp_mvm")) return s;
  clear_pending_error();
  NvtxRange nvtx("sgp_mvm");
  return run_mvm(h, V, k, SGP_BLUR_SEQUENTIAL, h->outputscale, 0.f, out);
}

sgp_status sgp_mvm_ex(sgp_lattice* h, const float* V, int k, int blur, float alpha, float beta,
                      float* out) {
  if (sgp_status s = check_mvm_args(h, V, k, blur, out, "sgp_mvm_ex")) return s;
  clear_pending_error();
  NvtxRange nvtx("sgp_mvm");
  return run_mvm(h, V, k, blur, alpha, beta, out);
}

sgp_status sgp_cg_solve_ex(sgp_lattice* h, const float* B, int k, int blur, float noise_var,
                           float tol, int max_iter, float* X, int* iters, double* rel_res) {
  if (sgp_status s = check_mvm_args(h, B, k, blur, X, "sgp_cg_solve")) return s;
  if (!(noise_var >= 0.f) || !(tol >= 0.f) || max_iter < 0) {
    set_error("sgp_cg_solve: need noise_var >= 0, tol >= 0 and max_iter >= 0");
    return SGP_ERR_INVALID_ARG;
  }
  clear_pending_error();
  NvtxRange nvtx("sgp_cg");
  return run_cg(h, B, k, blur, noise_var, tol, max_iter, X, iters, rel_res, h->precond_rank,
                h->precond_seed);
}

sgp_status sgp_cg_solve_history(sgp_lattice* h, const float* B, int k, int blur,
                                float noise_var, float tol, int max_iter, float* X, int* iters,
                                double* rel_res, double* history) {
  if (sgp_status s = check_mvm_args(h, B, k, blur, X, "sgp_cg_solve_history")) return s;
  if (!(noise_var >= 0.f) || !(tol >= 0.f) || max_iter < 0 || !history) {
    set_error("sgp_cg_solve_history: need noise_var >= 0, tol >= 0, max_iter >= 0 and a "
              "history buffer");
    return SGP_ERR_INVALID_ARG;
  }
  clear_pending_error();
  NvtxRange nvtx("sgp_cg");
  return run_cg(h, B, k, blur, noise_var, tol, max_iter, X, iters, rel_res, h->precond_rank,
                h->precond_seed, nullptr, history);
}

sgp_status sgp_cg_solve(sgp_lattice* h, const float* B, int k, float noise_var, float tol,
                        int max_iter, float* X, int* iters, double* rel_res) {
  return sgp_cg_solve_ex(h, B, k, SGP_BLUR_SYMMETRIC, noise_var, tol, max_iter, X, iters,
                         rel_res);
}

sgp_status sgp_mvm_backward(sgp_lattice* h, const float* X, const float* lengthscales,
                            const float* V, const float* G, int k, int blur, float alpha,
                            int grad, float* dV, float* dX, float* dls) {
  if (sgp_status s = check_handle(h)) return s;
  const bool want_x = dX || dls;
  if (k < 1 || k > kMaxK || blur < SGP_BLUR_SEQUENTIAL || blur > SGP_BLUR_SYMMETRIC ||
      (grad != SGP_GRAD_LATTICE && grad != SGP_GRAD_FILTER) || !G || (want_x && (!V || !X || !lengthscales))) {
    set_error("sgp_mvm_backward: need G, 1 <= k <= 256, an SGP_BLUR_* blur, an SGP_GRAD_* "
              "mode, and V, X and lengthscales when dX or dls is requested");
    return SGP_ERR_INVALID_ARG;
  }
  if (grad == SGP_GRAD_FILTER && want_x && h->kernel == SGP_KERNEL_MATERN32_COVERAGE) {
    set_error("sgp_mvm_backward: SGP_GRAD_FILTER needs an RBF handle (k' = -k / 2)");
    return SGP_ERR_INVALID_ARG;
  }
  if (!dV && !want_x) return SGP_OK;
  clear_pending_error();
  NvtxRange nvtx("sgp_backward");
  return run_mvm_backward(h, X, lengthscales, V, G, k, blur, alpha, grad, dV, dX, dls);
}

sgp_status sgp_logdet(sgp_lattice* h, const float* Z, int s, float noise_var, int max_lanczos,
                      float tol, double* logdet, double* quad) {
  if (sgp_status st = check_handle(h)) return st;
  if (!Z || !logdet || s < 1 || s > kMaxK || max_lanczos < 1 || max_lanczos > 256 ||
      !(noise_var >= 0.f) || !(tol >= 0.f)) {
    set_error("sgp_logdet: need Z, logdet, 1 <= s <= 256, 1 <= max_lanczos <= 256, "
              "noise_var >= 0 and tol >= 0");
    return SGP_ERR_INVALID_ARG;
  }
  clear_pending_error();
  NvtxRange nvtx("sgp_logdet");
  return run_logdet(h, Z, s, noise_var, max_lanczos, tol, logdet, quad);
}

void sgp_lattice_free(sgp_lattice* h) { free_lattice(h); }

sgp_status sgp_profile_blur(sgp_lattice* h, int enable) {
  if (sgp_status s = check_handle(h)) return s;
  for (int i = 0; i < 8 && enable; ++i) {
    if (!h->prof_ev[i]) {
      cudaError_t e = cudaEventCreate(&h->prof_ev[i]);
      if (e != cudaSuccess) return cuda_status(e, "sgp_profile_blur");
    }
  }
  h->profile = enable ? 1 : 0;
  h->prof_ms = 0.0;
  h->prof_passes = 0;
  for (double& v : h->prof_stage_ms) v = 0.0;
  h->prof_mvms = 0;
  return SGP_OK;
}

sgp_status sgp_profile_read_stages(const sgp_lattice* h, double* stage_ms, int64_t* samples) {
  if (sgp_status s = check_handle(h)) return s;
  if (stage_ms)
    for (int i = 0; i < kProfStages; ++i) stage_ms[i] = h->prof_stage_ms[i];
  if (samples) *samples = h->prof_mvms;
  return SGP_OK;
}

sgp_status sgp_profile_read(const sgp_lattice* h, double* blur_ms, int64_t* blur_passes) {
  if (sgp_status s = check_handle(h)) return s;
  if (blur_ms) *blur_ms = h->prof_ms;
  if (blur_passes) *blur_passes = h->prof_passes;
  return SGP_OK;
}

int64_t sgp_kernel_launches(void) { return launches_so_far(); }

sgp_status sgp_trim_memory(void) {
  clear_pending_error();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  if (e == cudaSuccess) e = pool_of(dev, &pool);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  return e == cudaSuccess ? SGP_OK : cuda_status(e, "sgp_trim_memory");
}

const char* sgp_last_error(void) { return g_last_error.c_str(); }

int sgp_version(void) { return SGP_VERSION; }

}  // extern "C"
