// Internal declarations of the sm_103a Simplex-GP library (not part of the C-ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sgp.h"

namespace sgp {

// Device error word bits, OR-ed by kernels and read back by the host.
enum : unsigned {
  ERRBIT_NONFINITE = 1u,
  ERRBIT_RANGE = 2u,
  ERRBIT_HASH_FULL = 4u,
};

// Faults injected on the host through SGP_FAULT (tests of the error paths).
enum { FAULT_NONE = 0, FAULT_OOM, FAULT_CUDA, FAULT_HASH_FULL, FAULT_NAN_INPUT };
int injected_fault();

// NVTX range for the lifetime of a scope (timeline profilers; no-op without one).
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
};

constexpr int kMaxOrder = 4;  // stencil order r
constexpr int kMaxD = 128;    // d + 1
constexpr int kMaxK = 256;    // right-hand sides per call
constexpr int kProfStages = 5;     // splat, blur, slice, B^T r, z (sgp_profile_read_stages)
constexpr int kSplatSeg = 32;      // splat items per segment
constexpr int kSplatMedSegs = 16;  // segments a single thread-group sums in the fix-up
// A lattice blurs in sparse mode when the direction lists hold at most this fraction of
// the D m (vertex, direction) pairs.
constexpr double kSparseFrac = 0.3;

// Stencil taps passed by value to the blur kernels.
struct Taps {
  float t[kMaxOrder + 1];
};

}  // namespace sgp

// The lattice handle: every array below is device memory owned by the handle.
struct sgp_lattice {
  int64_t n = 0;
  int d = 0, D = 0, r = 1;
  int kernel = 0;
  int64_t m = 0;
  double s = 0.0;
  double coef[sgp::kMaxOrder + 1] = {};
  double half[sgp::kMaxOrder + 1] = {};
  float outputscale = 1.f;
  int value_dtype = 0;
  int check_every = 8;
  int precond_rank = 0;
  int precond_power_iters = 1;
  uint64_t precond_seed = 0;
  int fault = 0;  // sgp::FAULT_* injected by SGP_FAULT into this lattice's construction
  int device = -1;  // CUDA device current at build time (the arrays live there)
  cudaStream_t stream = nullptr;

  // Points are processed in a locality order p = 0..n-1; perm[p] is the caller's index.
  int32_t* perm = nullptr;   // [n]
  int32_t* idx = nullptr;    // [n][D] vertex id of vertex k of point perm[p]
  float* w = nullptr;        // [n][D] barycentric weight, same order
  int32_t* row_ptr = nullptr;  // [m+1] splat lists: vertex v gathers items[row_ptr[v]..]
  int2* items = nullptr;       // [n*D] (locality-ordered point index p, weight bits)
  // Splat work split into segments of at most kSplatSeg items (load balance: a dense
  // cluster gives a vertex thousands of points).  seg[s] = (vertex, begin, end, slot):
  // slot < 0 writes the vertex directly, else the partial goes to partial[slot] and a
  // fix-up sums a vertex's partials in order.  med_rows / huge_rows: (vertex, first slot,
  // number of slots) of vertices with 2..kSplatMedSegs / more segments.
  int4* seg = nullptr;
  int64_t nseg = 0;
  int4* med_rows = nullptr;
  int64_t nmed = 0;
  int4* huge_rows = nullptr;
  int64_t nhuge = 0;
  int64_t nslots = 0;
  float* partial = nullptr;  // [nslots][k], sized with the lattice values
  float* vperm = nullptr;    // [n][k] the caller's V in locality order (public MVMs)
  int32_t* nbr = nullptr;      // [D][r][2][m] neighbour id of v - t u_j (0) / v + t u_j (1)
  int16_t* keys = nullptr;     // [m][D] vertex coordinates
  // Sparse lattices (few vertices with a neighbour along each direction, e.g. isolated
  // simplices at high d): act[act_off[j] .. act_off[j+1]) lists the vertices with at least
  // one neighbour along direction j, and the blur updates only those (sgp::kSparseFrac).
  bool sparse = false;
  int32_t* act = nullptr;
  std::vector<int64_t> act_off;  // [D + 1], host
  int64_t* act_off_dev = nullptr;  // [D + 1], device copy
  int64_t act_max = 0;           // largest list
  int32_t* epoch = nullptr;      // [m] pass after which a vertex's stored row was written
  void* act_tmp = nullptr;       // [act_max][k] new values of one pass
  size_t act_tmp_elems = 0;
  float* g0pow = nullptr;        // [2D + 1] powers of the symmetric blur's centre tap
  uint8_t* rank = nullptr;     // [n][D] rank of each elevated coordinate, locality order
  unsigned* err = nullptr;     // device error word

  // Lattice values (fp32 or bf16 per value_dtype), allocated on first use, grown on demand.
  void* lat[2] = {nullptr, nullptr};
  size_t lat_elems = 0;
  size_t lat_bytes = 0;  // value buffers + splat partials + permuted input
  size_t vperm_elems = 0;

  // Optional blur timing: events bracket the blur passes of one MVM inside the CG graph
  // and are read at every flag check (sgp_profile_blur / sgp_profile_read).
  // prof_ev: [0] after the splat, [1] after the blur, [2] before the splat, [3] after the
  // slice of the MVM inside the CG graph; [4] .. [7] around the preconditioner's B^T r
  // kernel ([4], [5]) and its z kernel ([6], [7]).
  int profile = 0;
  cudaEvent_t prof_ev[8] = {};
  double prof_ms = 0.0;
  int64_t prof_passes = 0;
  double prof_stage_ms[sgp::kProfStages] = {};  // SGP_STAGE_* order
  int64_t prof_mvms = 0;

  size_t bytes = 0;
};

namespace sgp {

using Lattice = ::sgp_lattice;

// ---- error reporting and launch accounting (api.cu) ----
void set_error(const std::string& msg);
sgp_status cuda_status(cudaError_t e, const char* what);
// Clear a pending non-sticky runtime error left by earlier calls of this thread (ours or
// the caller's), so that the launch checks of the current call report only its own
// launches.  A sticky error (a failed context) is returned again by the next call anyway.
void clear_pending_error();
// Count kernels enqueued by this library (graph replays count every kernel node).
void note_launches(int64_t count);
int64_t launches_so_far();
// Stream-ordered device allocation from the library's pool on the current device (freed
// with cudaFreeAsync; freed blocks stay mapped for reuse until sgp_trim_memory).
cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t st);

// ---- stencils (stencil.cpp) ----
// Spacing s and taps c[0..r] (kernel values k(t s)) and g[0..r] (half-kernel taps).
// Returns false when the kernel id or order is invalid.
bool make_stencil(int kernel, int r, double spacing_override, double* s, double* coef,
                  double* half);

// ---- primitives (scan_sort.cu) ----
// Exclusive scan of n uint32 values in place; *total (device, may be null) receives the
// sum.  `tmp` must hold scan_temp_elems(n) uint32.
size_t scan_temp_elems(int64_t n);
void exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* total, uint32_t* tmp,
                        cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the key.  Uses
// the *_alt buffers as ping-pong storage; returns true when the result ended in *_alt.
size_t radix_temp_elems(int64_t n);
bool radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                      int64_t n, int bits, uint32_t* tmp, cudaStream_t st);

// ---- lattice construction (build.cu) ----
sgp_status build_lattice(Lattice* L, const float* X, const float* ls);

// ---- MVM (mvm.cu) ----
// Make sure the lattice value buffers, splat partials and permuted-input buffer hold
// what a k-column product needs (allocated on `st`).
sgp_status ensure_lattice_values(Lattice* L, int k, cudaStream_t st);
// Enqueue out = alpha * W B W^T V + beta * V on `st` (buffers must be ready).  With
// internal = false, V and out are in the caller's point order (V is first permuted into
// locality order); with internal = true both are already in locality order (CG).  When
// `ev` is given, ev[0] / ev[1] are recorded around the blur passes.  Returns the number
// of blur passes.
int enqueue_mvm(const Lattice* L, const float* V, int k, int blur, float alpha, float beta,
                float* out, cudaStream_t st, cudaEvent_t* ev = nullptr, bool internal = false,
                double* dot_partial = nullptr);
// out = alpha K V (V and out in locality order) with the lattice values held in bf16 whatever
// the lattice's value type, in the lattice's own value buffers, which
// ensure_lattice_values(L, k) must have sized (a bf16 value takes half the room of an fp32
// one); every sum stays fp32.
void enqueue_mvm_bf16_values(const Lattice* L, const float* V, int k, int blur, float alpha,
                             float* out, cudaStream_t st);
// With internal = true and dot_partial set, the slice also writes per-block column sums of
// V * out (the CG's <p, A p>) to dot_partial[block][k]; this many blocks (grid-stride).
int64_t slice_dot_blocks(const Lattice* L, int k);
constexpr int kVecBlocks = 8 * 152;  // blocks of the grid-stride column-owning kernels
// Bytes of work space one k-column product needs (value buffers, partials, permuted
// input, each rounded up to 256 bytes).
size_t mvm_work_bytes(const Lattice* L, int k);
// As enqueue_mvm (caller's point order) with all work space carved out of `work`
// (mvm_work_bytes(L, k) bytes, 256-byte aligned); allocates nothing.
void enqueue_mvm_into(const Lattice* L, const float* V, int k, int blur, float alpha,
                      float beta, float* out, void* work, cudaStream_t st);
// Pieces of the operator for the backward: splat a locality-ordered Vp and blur it (the
// result ends in the returned buffer, lat0 or lat1, of the handle's value type); gather
// the caller's rows into locality order; out (caller's order) = alpha W lat.
void* enqueue_splat_blur(const Lattice* L, const float* Vp, int k, int blur, void* lat0,
                         void* lat1, float* partial, cudaStream_t st);
void enqueue_permute(const Lattice* L, const float* V, int k, float* Vp, cudaStream_t st);
void enqueue_slice_caller(const Lattice* L, const void* lat, int k, float alpha, float* out,
                          cudaStream_t st);
size_t lattice_value_bytes(const Lattice* L, int k);
// Full operator on the handle's stream, allocating value buffers when needed.
sgp_status run_mvm(Lattice* L, const float* V, int k, int blur, float alpha, float beta,
                   float* out);

// ---- Nystrom preconditioners of the CG (server: nystrom.cu + serve.cu; library: precond.cu) ----
constexpr int kMaxRank = 128;       // server requests (kb_* ring kernels)
constexpr int kMaxLibRank = 4096;   // library CG (ShiftedNystrom)

// Large-rank shifted Nystrom preconditioner of the library CG (precond.cu):
// P = B B^T + tau I with B B^T a rank-l Nystrom approximation of outputscale K~ (q power
// iterations) and tau = lambda_min(B^T B) + noise.
struct ShiftedNystrom {
  int l = 0, ld = 0;
  int64_t n = 0;
  float tau = 0.f;
  bool ok = false;
  // [n][ld] bf16 (the factor rounded to bf16; P is defined by these values), locality
  // order, padding columns zero
  void* B = nullptr;
  float* Minv = nullptr;   // [ld][ld] fp32 (tau I + B^T B)^-1 of the stored B, zero padded
  float* tpart = nullptr;  // [bt_splits][ld][16] B^T r partials
  float* tvec = nullptr;   // [ld][16]
  void* u = nullptr;       // [3][16][ld] bf16: Minv B^T r split in three bf16 parts
  void* r3 = nullptr;      // [ldr][64] bf16: r split in three bf16 parts (columns 16 p + c
                           // hold part p of column c; 48..63 zero)
  int* err = nullptr;      // set when a per-iteration kernel's bounded wait gave up
  int64_t ldr = 0;         // n rounded up to 64
  int bt_splits = 0;
  int64_t bt_rows = 0;
  int z_blocks = 0;
  // TMA maps: B as [n][ld] in 128 x 64 boxes (A of B u) and 64 x 64 boxes (A of B^T r),
  // u as [48][ld] in 48 x 64 boxes and r3 as [n][64] in 64 x 64 boxes
  CUtensorMap map_b_k, map_b_mn, map_u, map_r;
  std::vector<void*> ptrs;
  sgp_status build(Lattice* L, int rank, uint64_t seed, float noise, int blur, int power_iters,
                   cudaStream_t st);
  // partial rows apply() writes per column: one per block of the z kernel
  int64_t dot_blocks() const;
  // z = P^-1 r (r = rh + rl, locality order [n][k]) and per-block column sums of r z into
  // dot[block][c] (fp64).  split_ready: r3 already holds the split of columns 0..15 of r
  // (written by the CG's x, r update).
  void apply(const float* rh, const float* rl, int k, float* z, double* dot, cudaStream_t st,
             cudaEvent_t* ev = nullptr, bool split_ready = false) const;
  // SGP_ERR_CUDA when a per-iteration kernel gave up waiting (synchronizes st)
  sgp_status check(cudaStream_t st) const;
  void release(cudaStream_t st);
};

// Nystrom factor of the training block of a joint lattice's operator, for the GP
// posterior server: A = outputscale K~ restricted to the rows p with perm[p] < n_train
// (the other rows are masked: zero sketch rows, zero rows of Y and B).  The l sketch
// columns go through the lattice kp at a time (V, KV: [n][kp] device scratch, lattice
// values already sized for kp columns), so that no l-column value buffer is needed.
// Writes B (fp32 [n][ld], locality order, columns l..ld-1 zero) into Bh and
// (noise I + B^T B)^-1 (fp64 [l][l]) into Minv; scratch: nystrom_masked_scratch_bytes(l, n)
// device bytes.  Enqueued on st; *status_dev (device int) is set to 1 when a Cholesky
// pivot fails (the factor must then not be used); the caller reads it.
size_t nystrom_masked_scratch_bytes(int l, int64_t n);
sgp_status nystrom_build_masked(Lattice* L, int64_t n_train, int l, int ld, uint64_t seed,
                                float noise, int kp, float* V, float* KV, float* Bh,
                                double* Minv, void* scratch, int* status_dev, cudaStream_t st);

// ---- backward (backward.cu) ----
sgp_status run_mvm_backward(Lattice* L, const float* X, const float* ls, const float* V,
                            const float* G, int k, int blur, float alpha, int grad, float* dV,
                            float* dX, float* dls);

// ---- CG (cg.cu) ----
// Device buffers that receive the CG coefficients of every column for the Lanczos
// quadrature: alpha_j / beta_j of column c at [j][k] for j < cap, ||b_c|| and the
// iteration count per column.
struct LanczosRecord {
  double* alpha;
  double* beta;
  int cap;
  double* bnorm;
  int* iters;
};
// precond_rank > 0: preconditioned CG with a rank-precond_rank Nystrom preconditioner
// (not with a Lanczos record, which needs the plain CG's coefficients).
sgp_status run_cg(Lattice* L, const float* B, int k, int blur, float noise, float tol,
                  int max_iter, float* X, int* iters, double* rel_res, int precond_rank = 0,
                  uint64_t seed = 0, const LanczosRecord* rec = nullptr,
                  double* history = nullptr);
// log det(outputscale K~ + noise I) by stochastic Lanczos quadrature over the probe
// columns Z (device [n][s], caller's order); quad (host [s], may be null) receives each
// probe's ||z||^2 e1^T log(T) e1 (lanczos.cu).
sgp_status run_logdet(Lattice* L, const float* Z, int s, float noise, int max_lanczos,
                      float tol, double* logdet, double* quad);

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Per-column sums of per-thread fp64 partials inside one block, for kernels whose threads
// own VEC consecutive columns of one row: thread t owns columns (t % G) VEC .. + VEC - 1
// of block row t / G, with G = k / VEC threads per row and blockDim.x a multiple of G.
// The block's column sums go to out[0..k) in a fixed order (deterministic).  Every
// thread of the block must call it.
template <int VEC>
__device__ __forceinline__ void block_column_sums(const double (&acc)[VEC], int k, double* out) {
  __shared__ double s[256 * VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) s[threadIdx.x * VEC + j] = acc[j];
  __syncthreads();
  const int G = k / VEC;
  const int rows = blockDim.x / G;
  for (int col = threadIdx.x; col < k; col += blockDim.x) {
    const int chunk = col / VEC, lane = col % VEC;
    double t = 0.0;
    for (int r = 0; r < rows; ++r) t += s[(r * G + chunk) * VEC + lane];
    out[col] = t;
  }
}

// ---- double-float arithmetic -------------------------------------------------------
// FP64 throughput on this part is a small fraction of FP32, so quantities that need more
// than fp32 precision per element (CG iterate and residual, dot-product accumulation) are
// kept as unevaluated sums hi + lo of two fp32 numbers and updated with error-free
// transformations: TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|) and TwoProd through a
// fused multiply-add.  The _rn intrinsics keep the compiler from contracting or
// reordering the steps.  About 48 significant bits.
struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// (a.hi + a.lo) + (b.hi + b.lo)
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const dfloat s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, e);
}
// (a.hi + a.lo) * b
__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
  const dfloat p = df_two_prod(a.hi, b);
  return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ dfloat df_from_double(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

// Threads per block for the column-owning kernels: a whole number of rows of G threads.
inline int column_block_threads(int k, int vec) {
  const int G = k / vec;
  return G * (256 / G);
}

}  // namespace sgp
