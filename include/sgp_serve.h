/* sgp_serve.h -- C-ABI of the continuous-batching GP posterior server (sm_103a).
 *
 * A request is one exact-GP prediction (Sec. 2, Eq. gp_pred_mean and Eq. gp_pred_cov with
 * a zero prior mean): training inputs X [n][d] with targets y [n], test inputs Xs
 * [ns][d], ARD lengthscales, outputscale and noise variance sigma^2.  The server returns
 *   mean[t] = (K*X (K + sigma^2 I)^-1 y)[t]
 *   var[t]  = outputscale - (1/S) sum_s z_s[t] (K*X (K + sigma^2 I)^-1 KX* z_s)[t]
 * where K = outputscale K~ is the lattice kernel (symmetric blur SGP_BLUR_SYMMETRIC) on
 * one lattice built over the joint point set [X; Xs] (so that K*X is a slice at the test
 * rows of the same operator), and z_1..z_S are Rademacher probe vectors over the test
 * points: z_s[t] = -1 if the top bit of SplitMix64 at counter t S + s + 1 (seed =
 * request seed) is set, else +1.  The variance term is the probe (Hutchinson-type)
 * estimate of the diagonal of K*X (K + sigma^2 I)^-1 KX*; its expectation over the probes
 * is that diagonal.  The prior diagonal is outputscale (k(0) = 1 for the kernels here).
 *
 * Each request needs one linear solve with k = 1 + S right-hand sides (y and KX* z_s):
 * batched CG as in sgp_cg_solve (double-float iterate and residual, fp64 dot products,
 * per-column stopping ||r|| / ||b|| <= tol or max_iter iterations).
 *
 * Preconditioning (App. A: CG preconditioner of rank 100): the set-up computes the
 * condition estimate kappa = (outputscale max_i (K~_XX 1)_i + noise) / noise (Gershgorin:
 * K~ has non-negative entries, so its largest eigenvalue is at most its largest row sum;
 * one extra column of the probe product).  When precond_rank > 0 and kappa >=
 * precond_min_kappa, the request's CG is preconditioned with P = B B^T + noise I, the
 * rank-l randomized Nystrom approximation of outputscale K~_XX (l = min(precond_rank,
 * n)): Omega n x l Rademacher over the training points (Omega[i][j] = sign bit of
 * SplitMix64 at counter i l + j + 1, seed = request seed XOR 0x6A09E667F3BCC909), Y =
 * A Omega + 1e-3 noise Omega, Omega^T Y = R R^T, B = Y R^-T, and P^-1 r = (r - B (noise I
 * + B^T B)^-1 B^T r) / noise.  The stopping rule stays on the unpreconditioned residual.
 * Smooth kernels over many points per lattice vertex (low d, long lengthscales, small
 * noise) give kappa in the 10^4..10^6 range, where plain CG stalls; isolated points (high
 * d) give kappa near 1 / noise and converge in a few plain iterations.
 *
 * Continuous batching: requests are admitted in arrival order while the number of active
 * requests is below max_active and the device bytes they may hold stay within
 * hbm_budget (an upper bound per request from sgp_request_bytes_bound until its lattice
 * is built, then its actual allocation).  Active requests are grouped into lanes of
 * similar dimension and per-iteration work; every CG iteration of all requests of a lane
 * runs as one sequence of kernels over a device table of those requests (fixed grids,
 * per-request and per-column convergence masks), replayed from a CUDA graph, and lanes
 * run concurrently on their own streams.  A request leaves its lane as soon as its
 * columns have stopped, and new requests join at the lane's next round.  Each request's
 * arithmetic is partitioned by its own sizes only, so its results are bitwise the same
 * alone and in any mix.  max_active = 1 gives the plain one-request-at-a-time path with
 * the same kernels.
 *
 * Threading: a server is used by one host thread at a time.  Host buffers of a request
 * (X, y, Xs, lengthscales, mean, var) must stay valid until the request has completed
 * (sgp_request_stats.done != 0).  Errors follow sgp.h: every call returns an sgp_status
 * and sgp_last_error() has the message; a request whose build fails completes with its
 * own status and does not stop the server.  The preconditioner's kernels wait on
 * bulk-copy barriers with a bounded number of polls; should a wait give up, the kernel
 * records it and returns, and the requests of that round complete with SGP_ERR_CUDA
 * (their mean/var are not written) while the server keeps running.  For tests of that
 * path, SGP_FAULT=ring_wait in the environment of sgp_server_create makes the first lane
 * round that applies a preconditioner wait with a limit of 0 polls: its first chunk wait
 * gives up at once, the block still waits (bounded) for its copies in flight before it
 * returns, and the next rounds run with the normal limit.  Nothing faults the device.
 */
#ifndef SGP_SERVE_H_
#define SGP_SERVE_H_

#include "sgp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgp_server sgp_server; /* opaque; created by sgp_server_create */

typedef struct {
  unsigned long long hbm_budget; /* device bytes the active requests may hold; default
                                    half of the device's total memory                    */
  int max_active;     /* requests in the batch at once, 1..64; default 16 (1 = plain)     */
  int probes;         /* Rademacher probes S of the variance estimate, 0..30; default 8   */
  int order_r;        /* stencil order (as sgp_opts); default 1                           */
  int kernel;         /* SGP_KERNEL_*; default SGP_KERNEL_RBF_BINOMIAL                    */
  double spacing_s;   /* > 0 overrides the kernel rule's spacing; default 0               */
  int value_dtype;    /* SGP_VALUES_F32 / SGP_VALUES_BF16 lattice value storage.  With
                         BF16 a request keeps bf16 values only when its condition estimate
                         kappa is at most 100: the ~2^-8 relative error of bf16 products
                         grows with the conditioning of the solve, so a worse-conditioned
                         request is rebuilt with fp32 values (same lattice) before its
                         right-hand sides and solve, and serves at the fp32 accuracy.
                         Admission reserves the fp32 bound in either mode.               */
  double tol;         /* CG tolerance on ||r|| / ||b||; default 1e-3                      */
  int max_iter;       /* CG iteration cap; default 1000                                   */
  int check_every;    /* CG iterations per sgp_server_step between flag reads; default 8 */
  int precond_rank;   /* rank l of the Nystrom preconditioner, 0..128 (0 = none); default
                         100 (App. A)                                                     */
  double precond_min_kappa; /* precondition requests whose condition estimate kappa is at
                         least this; default 1e3 (0 = every request)                      */
  int lane_classes;   /* 1 (default): lanes by dimension class, work class and value type;
                         0: one lane per value type for all requests (every iteration round
                         then runs the blur passes of the largest active d for all)       */
} sgp_server_opts;

typedef struct {
  const float* X;            /* host [n][d] training inputs                               */
  const float* y;            /* host [n] training targets                                 */
  long long n;               /* >= 1                                                      */
  const float* Xs;           /* host [ns][d] test inputs                                  */
  long long ns;              /* >= 1; n + ns <= 2^31 / (d + 1)                            */
  int d;                     /* 1..127                                                    */
  const float* lengthscales; /* host [d], each > 0                                        */
  float outputscale;         /* > 0                                                       */
  float noise;               /* sigma^2 > 0                                               */
  unsigned long long seed;   /* probe seed                                                */
  float* mean;               /* host [ns] output                                          */
  float* var;                /* host [ns] output (may be NULL when probes = 0)            */
  double arrival_us;         /* arrival time on the server clock (sgp_server_clock_us), or
                                < 0 for "now"; latency is measured from it                */
  double timeout_us;         /* > 0: deadline arrival_us + timeout_us; a request still
                                queued or iterating at a step past it completes with
                                SGP_ERR_TIMEOUT (mean/var not written); <= 0: none        */
  unsigned long long lattice_key; /* != 0: requests with the same key promise the same X,
                                Xs, lengthscales and outputscale; the server keeps the
                                lattice of a finished one resident (within hbm_budget,
                                least recently used evicted first) and a later one reuses
                                it instead of uploading and building; 0: no reuse        */
} sgp_request;

typedef struct {
  int done;                  /* 1 once mean/var are written (or the request failed)      */
  int status;                /* sgp_status of the request                                 */
  int iters;                 /* CG iterations the request ran                             */
  double rel_res;            /* largest final ||r|| / ||b|| over its columns              */
  double arrival_us, admit_us, done_us; /* server clock                                   */
  long long m;               /* lattice vertices                                          */
  unsigned long long bytes;  /* device bytes the request held while active                */
  double setup_us;           /* host time of its set-up (upload, lattice build, right-hand
                                sides) on a set-up thread                                 */
  int lattice_reused;        /* 1 when it ran on a resident lattice (lattice_key)         */
  int precond_rank;          /* rank of its preconditioner (0: plain CG)                  */
  double kappa_est;          /* its condition estimate (0 when precond_rank option is 0
                                and the server stores fp32 values)                        */
  int value_dtype;           /* SGP_VALUES_* its solve used (see value_dtype below)       */
} sgp_request_stats;

/* Fill *opts with the defaults listed above (hbm_budget from the current device, or 0
 * without one). */
void sgp_server_opts_init(sgp_server_opts* opts);

/* Upper bound of the device bytes one request holds at its peak (lattice build work
 * space included) for n_points = n + ns points in d dimensions, stencil order r, k
 * columns (the server uses k = 1 + probes + 1: y, the probes and the row-sum column),
 * the value type and the preconditioner rank (0..128; its factor, apply buffers and
 * factorisation scratch): every size taken at its bound m = n_points (d + 1) (Sec. 5.2:
 * at most d + 1 vertices per point).  0 for invalid arguments.  Host only. */
unsigned long long sgp_request_bytes_bound(long long n_points, int d, int order_r, int k,
                                           int value_dtype, int precond_rank);

/* Create a server on the current device (its own CUDA streams).  opts may be NULL. */
sgp_status sgp_server_create(const sgp_server_opts* opts, sgp_server** out);

/* Queue a request (nothing is copied or launched yet); *id receives its id.
 * SGP_ERR_INVALID_ARG for bad sizes or pointers, or a request whose bound exceeds the
 * whole budget (it could never be admitted). */
sgp_status sgp_server_submit(sgp_server* srv, const sgp_request* req, long long* id);

/* One scheduling round: for every lane whose round of check_every CG iterations has
 * ended, finish the requests that stopped (predictive slice, copy of mean/var to the
 * host, release of their memory) and cancel those past their deadline; complete queued
 * requests past their deadline with SGP_ERR_TIMEOUT; admit and set up queued requests
 * (lattice build, right-hand sides) on a set-up stream while the other lanes run;
 * relaunch idle lanes; then, if nothing finished, wait up to 2 ms for a lane to end its
 * round.  *completed (may be NULL) receives the number of requests finished by this
 * call.  Returns at once when nothing is queued or active. */
sgp_status sgp_server_step(sgp_server* srv, int* completed);

/* Statistics of request `id` (valid at any time; done = 0 while it is queued/active). */
sgp_status sgp_server_stats(const sgp_server* srv, long long id, sgp_request_stats* out);

/* Queue and batch state: queued and active request counts, device bytes held by active
 * requests (as accounted against the budget), and the largest batch seen so far. */
sgp_status sgp_server_info(const sgp_server* srv, int* queued, int* active,
                           unsigned long long* bytes_in_use, int* peak_active);

/* Resident lattices kept for reuse (lattice_key) and their device bytes (counted in
 * bytes_in_use of sgp_server_info). */
sgp_status sgp_server_cache_info(const sgp_server* srv, int* lattices,
                                 unsigned long long* bytes);

/* Microseconds since the server was created (steady clock). */
double sgp_server_clock_us(const sgp_server* srv);

/* Wait for the device, release every request's memory, the streams and the graphs. */
void sgp_server_destroy(sgp_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* SGP_SERVE_H_ */
