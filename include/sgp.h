/* sgp.h -- C-ABI of the GB300 (sm_103a) Simplex-GP lattice library.
 *
 * The library computes the permutohedral-lattice approximation of a stationary-kernel
 * matrix-vector product,  K V ~= W B W^T V  (Sec. 3.2 and Eq. ski_to_bf: splat W^T,
 * blur B, slice W), and solves (outputscale K~ + noise I) X = B with batched conjugate
 * gradients that touch K~ only through these products (Sec. 2).
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major fp32: X is [n][d], V/out/B/X-solutions are [n][k].
 *   - Pointers marked "device" are CUDA device pointers on the current device (for
 *     example torch.Tensor.data_ptr() of a contiguous CUDA tensor); pointers marked
 *     "host" are ordinary host memory.  The caller owns every buffer it passes in.
 *   - The library owns the lattice handle and the device arrays inside it; it allocates
 *     them with stream-ordered cudaMallocAsync on the handle's stream and frees them in
 *     sgp_lattice_free().
 *   - Work is enqueued on the handle's stream (opts->stream at build time, or the one set
 *     with sgp_set_stream).  sgp_mvm / sgp_mvm_ex never synchronise; sgp_lattice_build
 *     synchronises once (to read the vertex count and the device error word);
 *     sgp_cg_solve synchronises every opts->check_every iterations to read the
 *     per-column convergence flags, and once at the end.
 *   - No C++ exception crosses this boundary.  Every call returns an sgp_status; on a
 *     failure sgp_last_error() returns a thread-local message, the outputs are
 *     unspecified and an existing handle stays valid.
 *   - There is no CPU fallback: without a CUDA device every call fails with SGP_ERR_CUDA.
 *   - Fault injection for tests of the error paths, read by sgp_lattice_build from the
 *     environment variable SGP_FAULT: "oom" (fails as out of memory before allocating),
 *     "cuda_err" (fails as a CUDA error before any device work), "hash_full" (builds with
 *     a 1024-slot vertex table, so that the bounded probes of a larger lattice run out and
 *     the build returns SGP_ERR_HASH_FULL), "nan_input" (the elevation kernel treats the
 *     first point as NaN: SGP_ERR_NONFINITE).  None of them faults the device.
 *   - Each stage pushes an NVTX range (sgp_build, sgp_mvm, sgp_cg, sgp_backward,
 *     sgp_logdet, sgp_serve_step) for timeline profilers.
 */
#ifndef SGP_H_
#define SGP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGP_VERSION 1

typedef struct sgp_lattice sgp_lattice; /* opaque; created by sgp_lattice_build */

typedef enum {
  SGP_OK = 0,
  SGP_ERR_INVALID_ARG = 1, /* a size, pointer or option is out of range            */
  SGP_ERR_OOM = 2,         /* a device allocation failed                            */
  SGP_ERR_RANGE = 3,       /* a lattice coordinate does not fit in int16            */
  SGP_ERR_HASH_FULL = 4,   /* the vertex hash table ran out of probes               */
  SGP_ERR_NONFINITE = 5,   /* X holds NaN/Inf, or a lengthscale is <= 0 / not finite */
  SGP_ERR_CUDA = 6,        /* a CUDA runtime call failed (message has the CUDA error) */
  SGP_ERR_TIMEOUT = 7,     /* a served request passed its deadline (sgp_serve.h)     */
} sgp_status;

/* Stationary kernel and its stencil (Sec. 4.1).  Stencil taps are kernel values at the
 * lattice points, c_t = k(t s), t = -r..r, with spacing s in lengthscale units:
 *   SGP_KERNEL_RBF_BINOMIAL      RBF, s = sqrt(2 ln 2) so that r = 1 gives the binomial
 *                                stencil [.5, 1, .5] of Sec. 3.2 "Blur" (the default);
 *   SGP_KERNEL_RBF_COVERAGE      RBF, s balancing spatial and Fourier coverage
 *                                (Eq. balance_coverage) by numerical integration;
 *   SGP_KERNEL_MATERN32_COVERAGE Matern-3/2, s from Eq. balance_coverage. */
enum {
  SGP_KERNEL_RBF_BINOMIAL = 0,
  SGP_KERNEL_RBF_COVERAGE = 1,
  SGP_KERNEL_MATERN32_COVERAGE = 2,
};

/* Blur operator B.
 *   SGP_BLUR_SEQUENTIAL  the paper's blur (Sec. 3.2 "Blur"): the 1-D stencil c along
 *                        lattice directions j = 0, 1, ..., d in turn, vertex set fixed.
 *   SGP_BLUR_TRANSPOSE   the exact adjoint of the above: directions d, ..., 0.
 *   SGP_BLUR_SYMMETRIC   M^T M, with M the sequential blur built from the taps g of the
 *                        half kernel (the kernel whose self-convolution is proportional
 *                        to k), g normalised so that sum_t g_t^2 = 1: passes 0..d then
 *                        d..0.  Symmetric positive semi-definite, as K_UU of Eq. k_ski
 *                        is; the per-direction blurs of a truncated lattice do not
 *                        commute, so the sequential operator is not symmetric. */
enum {
  SGP_BLUR_SEQUENTIAL = 0,
  SGP_BLUR_TRANSPOSE = 1,
  SGP_BLUR_SYMMETRIC = 2,
};

/* Storage type of the lattice values during an MVM.  Arithmetic is fp32 in both. */
enum {
  SGP_VALUES_F32 = 0,
  SGP_VALUES_BF16 = 1,
};

typedef struct {
  int order_r;        /* stencil order r, 1..4 (taps -r..r); default 1                  */
  int kernel;         /* SGP_KERNEL_*; default SGP_KERNEL_RBF_BINOMIAL                  */
  double spacing_s;   /* > 0 overrides the kernel rule's spacing s; default 0 (rule)    */
  float outputscale;  /* multiplies K~ in sgp_mvm and in the CG system; default 1       */
  int value_dtype;    /* SGP_VALUES_*; default SGP_VALUES_F32                           */
  int check_every;    /* CG iterations between host reads of the flags; default 8       */
  void* stream;       /* cudaStream_t for all work on this handle; NULL = default stream */
  int precond_rank;   /* CG preconditioner rank l (0 = none, <= 4096); App. A uses 100;
                         default 0 (see sgp_cg_solve_ex)                                */
  unsigned long long precond_seed; /* seed of the preconditioner's random sketch; 0    */
  int precond_power_iters; /* subspace iterations of the sketch, 0 or 1; default 1      */
} sgp_opts;

/* Fill *opts with the defaults listed above. */
void sgp_opts_init(sgp_opts* opts);

/* Stencil of a kernel without building a lattice (host only, no device needed; Sec. 4.1,
 * Eq. balance_coverage): spacing *spacing_s, taps coef[0..order_r] = k(t s) and
 * symmetric-blur taps half_coef[0..order_r] (host arrays of order_r + 1 doubles).
 * spacing_override > 0 replaces the kernel rule's spacing.  SGP_ERR_INVALID_ARG for an
 * unknown kernel or order_r outside 1..4. */
sgp_status sgp_stencil(int kernel, int order_r, double spacing_override, double* spacing_s,
                       double* coef, double* half_coef);

/* Build the lattice of n points (Sec. 3.2 "Splat"): scale each point by the
 * lengthscales, elevate it into H_d, find its enclosing simplex by rounding and ranking,
 * compute its d+1 barycentric weights, insert the simplex vertices into a device hash
 * table, number the distinct vertices, and precompute the per-direction neighbour table
 * used by the blur and the vertex-to-point lists used by the splat.
 *   X            device, [n][d] fp32, finite.
 *   lengthscales device, [d] fp32, each > 0 and finite (ARD lengthscales).
 *   n >= 1; 1 <= d <= 127.  opts may be NULL (defaults).
 *   *out         receives the new handle; release it with sgp_lattice_free.
 * Errors: SGP_ERR_INVALID_ARG (sizes/options), SGP_ERR_NONFINITE, SGP_ERR_RANGE (a
 * vertex coordinate beyond int16: lengthscales far smaller than the data's spread),
 * SGP_ERR_HASH_FULL, SGP_ERR_OOM, SGP_ERR_CUDA.  On error *out is set to NULL. */
sgp_status sgp_lattice_build(const float* X, const float* lengthscales, int64_t n, int d,
                             const sgp_opts* opts, sgp_lattice** out);

/* Number of lattice vertices m (m <= n (d+1), Sec. 5.2 Table n_lattice) and the device
 * bytes the handle holds.  Either output may be NULL. */
sgp_status sgp_lattice_info(const sgp_lattice* h, int64_t* m, size_t* device_bytes);

/* Blur work of the handle: *pairs (may be NULL) receives the number of (vertex,
 * direction) pairs whose vertex has a neighbour along that direction when the lattice is
 * sparse, else -1; *sparse (may be NULL) is 1 when those pairs are at most 30 % of the
 * (d+1) m pairs, and the blur then updates
 * only those vertices in each pass (the others keep their rows; the centre tap's factor
 * is applied lazily), 0 when every pass sweeps all m vertices.  The operator is the same
 * either way. */
sgp_status sgp_lattice_blur_lists(const sgp_lattice* h, int* sparse, int64_t* pairs);

/* Stencil actually used (Sec. 4.1): the spacing s, the paper's taps c[0..r] and the
 * symmetric-blur taps g[0..r] (host arrays of order_r + 1 doubles).  Any may be NULL. */
sgp_status sgp_lattice_stencil(const sgp_lattice* h, int* order_r, double* spacing_s,
                               double* coef, double* half_coef);

/* Copy the lattice structure to host memory (for inspection and tests; synchronises):
 *   keys  host [m][d+1] int16: integer coordinates of vertex id v (Eq. canon_simplex
 *         lattice points, coordinate sum 0);
 *   idx   host [n][d+1] int32: vertex id of vertex k of point i (point i in the caller's
 *         order; vertex k has all coordinates congruent to k mod d+1);
 *   w     host [n][d+1] fp32: barycentric weight of vertex k of point i.
 * Any pointer may be NULL.  Vertex ids are the library's own numbering. */
sgp_status sgp_lattice_export(const sgp_lattice* h, int16_t* keys, int32_t* idx, float* w);

/* Set the stream used by subsequent calls on this handle (cudaStream_t; NULL = default). */
sgp_status sgp_set_stream(sgp_lattice* h, void* stream);

/* out = outputscale * W B W^T V with the sequential blur (Sec. 3.2, Eq. ski_to_bf).
 *   V    device [n][k] fp32;  out device [n][k] fp32 (must not alias V);  1 <= k <= 256.
 * Stream-ordered, no synchronisation, may be captured in a CUDA graph. */
sgp_status sgp_mvm(sgp_lattice* h, const float* V, int k, float* out);

/* out = alpha * W B W^T V + beta * V for the blur selected by `blur` (SGP_BLUR_*).
 * Same layout and rules as sgp_mvm; outputscale is not applied (alpha replaces it). */
sgp_status sgp_mvm_ex(sgp_lattice* h, const float* V, int k, int blur, float alpha,
                      float beta, float* out);

/* As sgp_mvm_ex, but allocating no device memory: the lattice value buffers and splat
 * partials and the input in the lattice's point order (2 m k lattice values of the
 * handle's value type plus (nslots + n) k floats) come from a 64 MiB work area compiled
 * into the
 * library (a file-scope __device__ array, held by every GPU that loads the library until
 * the process exits).  The paper has no counterpart; this entry point exists for callers
 * that cannot allocate when they need a product: serving loops that must keep
 * cudaMalloc/cudaFree (which can synchronise the device) off their hot path, and
 * processes whose device memory is already reserved by another allocator's pool.
 *   V, out  device [n][k] fp32 as in sgp_mvm_ex (the handle must already be built).
 * A lattice whose work space for this k exceeds 64 MiB is rejected with
 * SGP_ERR_INVALID_ARG before anything is launched, and so is every call made while a
 * device other than the one the lattice was built on is current (each device has its
 * own work area).  Sparse lattices (sgp_lattice_blur_lists) are blurred by full sweeps
 * here, since the fixed area holds no direction-list buffers: at high d (isolated
 * simplices) such a product is several times slower than sgp_mvm_ex's (about 6x at
 * d = 90).  The first call on a device looks up
 * the work area's device address (cudaGetSymbolAddress, with that device current); make
 * that first call before any stream capture.  All calls in the process share the one
 * work area and it keeps the last call's contents (every element is rewritten before it
 * is read): calls whose execution overlaps on the GPU -- concurrent streams, threads or
 * handles -- race on it and must be ordered by the caller. */
sgp_status sgp_mvm_static(sgp_lattice* h, const float* V, int k, int blur, float alpha,
                          float beta, float* out);

/* Batched conjugate gradients (Sec. 2; App. A: at most max_iter = 500 iterations) on
 *   (outputscale * W B W^T + noise_var I) X = B,   B = SGP_BLUR_SYMMETRIC,
 * every column independent: column c stops when ||r_c|| / ||b_c|| <= tol (recurrence
 * residual), after max_iter iterations, or when <p_c, A p_c> <= 0.  The iterate and the
 * residual are carried on the device as double-float pairs (two fp32 numbers, about 48
 * significant bits), the search direction and its product in fp32 (the MVM operands);
 * dot products and norms are accumulated in double-float per thread and fp64 across
 * threads.  Work space: 24 n k bytes plus the handle's lattice value buffers, allocated
 * per call.
 *   B      device [n][k] fp32;  X device [n][k] fp32 (solution; must not alias B).
 *   iters  host [k] int (iterations per column) or NULL;
 *   rel_res host [k] double (final recurrence residual ratio per column) or NULL.
 * Non-convergence is not an error: it shows in iters / rel_res.  noise_var >= 0,
 * tol >= 0, max_iter >= 0, 1 <= k <= 256. */
sgp_status sgp_cg_solve(sgp_lattice* h, const float* B, int k, float noise_var, float tol,
                        int max_iter, float* X, int* iters, double* rel_res);

/* As sgp_cg_solve with the blur operator chosen by `blur` (SGP_BLUR_*).  CG assumes a
 * symmetric positive-definite matrix; only SGP_BLUR_SYMMETRIC guarantees one.
 *
 * Preconditioning (opts->precond_rank = l > 0 at build time, noise_var > 0; App. A: CG
 * pre-conditioner): CG runs preconditioned with P = B B^T + tau I, where B B^T is a
 * rank-l randomized Nystrom approximation of K = outputscale W B W^T (B here the blur):
 *   Omega  n x l Rademacher sketch, Omega[i][j] = sign bit of SplitMix64 at counter
 *          i l + j + 1 from precond_seed (i the caller's point index);
 *   Q      Omega (precond_power_iters = 0) or a basis of the range of K Omega (1), by
 *          Cholesky QR (a second pass only when the first needed a raised shift: the
 *          approximation depends only on the range, so K Omega is formed with bf16
 *          lattice values and fp32 sums);
 *   Y      = K Q,  C = (Q^T Y + Y^T Q)/2 + eps I (eps = 1e-6 max_j C_jj, raised when its
 *          Cholesky fails) = R R^T,  B = Y R^-T;
 *   tau    = lambda_min(B^T B) (inverse power iteration) + noise_var.
 * B is stored rounded to bf16 (P is defined by the stored values) and
 * P^-1 r = (r - B (tau I + B^T B)^-1 B^T r) / tau.  The l-column products with K run in
 * chunks of 128 columns; the tall n x l products on the tensor cores (bf16 operands: the
 * set-up's panels held as three bf16 parts, B exact with three-part r and u per
 * iteration), the l x l factorizations in fp64.  Work space: about 14 n l + 1100 n bytes
 * during the set-up, 2 n l + 96 n kept for the solve.  When a Cholesky fails after its retries the solve runs
 * unpreconditioned.  The stopping rule is unchanged (unpreconditioned residual
 * ||r_c|| / ||b_c||). */
sgp_status sgp_cg_solve_ex(sgp_lattice* h, const float* B, int k, int blur, float noise_var,
                           float tol, int max_iter, float* X, int* iters, double* rel_res);

/* As sgp_cg_solve_ex, also recording the convergence history (Sec. 2): history is host
 * [max_iter][k] doubles; entry (j, c) receives ||r_c|| / ||b_c|| (the recurrence residual
 * the stopping rule tests) after iteration j + 1 of column c, and NaN for iterations the
 * column did not run.  Work space grows by 8 max_iter k bytes.  SGP_ERR_INVALID_ARG when
 * history is NULL; other rules as sgp_cg_solve_ex. */
sgp_status sgp_cg_solve_history(sgp_lattice* h, const float* B, int k, int blur,
                                float noise_var, float tol, int max_iter, float* X, int* iters,
                                double* rel_res, double* history);

/* log det(outputscale * W B W^T + noise_var I), B = SGP_BLUR_SYMMETRIC: the second term of
 * the marginal log-likelihood (Eq. gp_mll), by stochastic Lanczos quadrature.  For each
 * probe column z_s, plain CG on A x = z_s (at most max_lanczos iterations; App. A uses
 * 100; stopping early at ||r|| / ||z|| <= tol) gives the Lanczos tridiagonal T_s from its
 * coefficients (T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T[j+1][j] =
 * sqrt(beta_j)/alpha_j); quad_s = ||z_s||^2 e1^T log(T_s) e1 (from T_s's eigenvalues and
 * the first components of its eigenvectors, implicit QL on the GPU), and
 *   *logdet = (1/s) sum_s quad_s,
 * an unbiased estimate of tr log A when E[z z^T] = I (e.g. Rademacher probes).
 *   Z       device [n][s] fp32 probes (caller's order), 1 <= s <= 256.
 *   max_lanczos 1..256;  noise_var >= 0;  tol >= 0.
 *   logdet  host double;  quad host [s] doubles or NULL.
 * Synchronises (CG flag reads and the result).  SGP_ERR_NONFINITE when a tridiagonal is
 * not positive definite (e.g. noise_var = 0 on a singular operator). */
sgp_status sgp_logdet(sgp_lattice* h, const float* Z, int s, float noise_var, int max_lanczos,
                      float tol, double* logdet, double* quad);

/* Input gradients of the backward (sgp_mvm_backward).
 *   SGP_GRAD_LATTICE  the exact derivative of the product the forward computes, through
 *                     the barycentric weights (Sec. 3.2): piecewise linear in the elevated
 *                     points, with ranks and vertex ids piecewise constant.
 *   SGP_GRAD_FILTER   Sec. 4.2: the kernel's own input gradient estimated with ONE lattice
 *                     filtering of the 2k(d+1) columns [z (.) G, G, z (.) V, V], z = X / l,
 *                     with k' = dk/d(d^2) (= -k/2 for the RBF kernels; not available for
 *                     Matern-3/2). */
enum {
  SGP_GRAD_LATTICE = 0,
  SGP_GRAD_FILTER = 1,
};

/* Backward of out = alpha * W B W^T V (B per `blur`, as in sgp_mvm_ex) for a scalar loss
 * with upstream gradient G = dLoss/dout:
 *   dV   = alpha * W B^T W^T G   (the transpose product on the same lattice)
 *   dX   = dLoss/dX  and  dls = dLoss/dlengthscales  through the lattice's dependence on
 *          the scaled points z = X / l, computed as selected by `grad` (SGP_GRAD_*);
 *          dls_j = -sum_i dX_ij X_ij / l_j.
 *   X, lengthscales  device, the [n][d] points and [d] lengthscales the handle was built
 *                    from (needed when dX or dls is requested; may be NULL otherwise).
 *   V, G     device [n][k] fp32 (V may be NULL when only dV is requested).
 *   dV       device [n][k], dX device [n][d], dls device [d] fp32; each may be NULL.
 * Work space: two extra lattice value buffers (SGP_GRAD_LATTICE) or 2 n min(256, 2k(d+1))
 * floats and the value buffers of that many columns (SGP_GRAD_FILTER), allocated per
 * call; stream-ordered on the handle's stream, no synchronisation.  1 <= k <= 256.
 * SGP_ERR_INVALID_ARG for a missing input, an unknown blur or grad, or SGP_GRAD_FILTER on
 * a Matern-3/2 handle. */
sgp_status sgp_mvm_backward(sgp_lattice* h, const float* X, const float* lengthscales,
                            const float* V, const float* G, int k, int blur, float alpha,
                            int grad, float* dV, float* dX, float* dls);

/* Blur timing for measurement tools.  While enabled, every CG solve on this handle
 * brackets the blur passes of one MVM with CUDA events recorded on the solve's stream (as
 * nodes of its graph) and, at each flag check, adds the elapsed time of the last replay
 * to a running total.  Enabling (or disabling) resets the totals. */
sgp_status sgp_profile_blur(sgp_lattice* h, int enable);

/* Totals collected since sgp_profile_blur: milliseconds spent in the sampled blur passes
 * and the number of passes those samples cover.  Either output may be NULL. */
sgp_status sgp_profile_read(const sgp_lattice* h, double* blur_ms, int64_t* blur_passes);

/* Per-stage totals collected since sgp_profile_blur, over the iterations sampled inside
 * the CG graph (one per flag check): stage_ms (host, 5 doubles, or NULL) receives the
 * milliseconds of SGP_STAGE_SPLAT (splat with its fix-ups), SGP_STAGE_BLUR (all blur
 * passes), SGP_STAGE_SLICE (slice with its <p, Ap> partials) of the MVM and, in a
 * preconditioned solve, SGP_STAGE_PRECOND_BT (the B^T r kernel) and SGP_STAGE_PRECOND_Z
 * (the z = (r - B u) / tau kernel) of the first 16 columns; *samples (or NULL) the number of
 * sampled iterations. */
enum {
  SGP_STAGE_SPLAT = 0,
  SGP_STAGE_BLUR = 1,
  SGP_STAGE_SLICE = 2,
  SGP_STAGE_PRECOND_BT = 3,
  SGP_STAGE_PRECOND_Z = 4,
};
sgp_status sgp_profile_read_stages(const sgp_lattice* h, double* stage_ms, int64_t* samples);

/* Number of kernels this library has enqueued in this process (a replayed CUDA graph
 * counts each of its kernels), for launch accounting in benchmarks. */
int64_t sgp_kernel_launches(void);

/* Device memory: the library allocates its work space and handle arrays stream-ordered
 * from a memory pool of its own per device, which keeps the blocks freed by a finished call
 * mapped so that the next build, product or solve reuses them (at n = 2M a preconditioner
 * set-up frees and re-takes about 30 GB; mapping it afresh cost 65 ms per solve).
 * sgp_trim_memory synchronizes the current device and returns every unused pooled block of
 * it to the driver.  SGP_ERR_CUDA without a device. */
sgp_status sgp_trim_memory(void);

/* Release the handle and every device array it owns (stream-ordered on its stream). */
void sgp_lattice_free(sgp_lattice* h);

/* Message of the last failed call on this thread ("" if none). */
const char* sgp_last_error(void);

/* SGP_VERSION of the loaded library. */
int sgp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SGP_H_ */
