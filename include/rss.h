/*
 * rss.h -- C ABI of the GB300 strong-recursive-skeletonization (RS-S) library.
 *
 * RS-S factors a dense kernel matrix A (A_ij = K(x_i, x_j), i != j, paper
 * Eq. 3) for points on a uniform planar grid into the product of per-box
 * operators of Eq. (9) (Algorithm 1), then applies the factorization to
 * right-hand sides (Section 2.5).  Every numerical step runs in the library's
 * own sm_103a CUDA kernels; there is no CPU fallback.
 *
 * Conventions
 *  - Every call returns an rss_status; nothing throws across the ABI.  On a
 *    non-OK status, rss_last_error() gives a message (thread-local).
 *  - Handles are opaque and owned by the library; release them with rss_free.
 *  - Complex values are interleaved (re, im) pairs of doubles, the layout of
 *    C99 double _Complex, numpy complex128 and torch.complex128.
 *  - Matrices of right-hand sides are column-major: entry (i, j) at
 *    b[i + j * ldb], i a point index in the caller's order.
 *  - Input errors (bad sizes, points that are not a complete uniform grid,
 *    unsupported parameters) return RSS_EINVAL before any GPU work.
 *  - CUDA failures return RSS_ECUDA; device memory exhaustion RSS_ENOMEM; a
 *    zero pivot in an LU returns RSS_ENUMERIC (Eq. 8 supposes X_RR non-singular);
 *    a bounded device wait that runs out returns RSS_ETIMEOUT.
 */
#ifndef RSS_GB300_H
#define RSS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rss_tree rss_tree;
typedef struct rss_factorization rss_factorization;
typedef struct rss_server rss_server;

typedef enum {
  RSS_OK = 0,
  RSS_EINVAL = 1,   /* invalid argument; nothing was launched */
  RSS_ENOMEM = 2,   /* device or host allocation failed */
  RSS_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  RSS_ENUMERIC = 4, /* exact zero pivot in an LU factorization */
  RSS_ETIMEOUT = 5, /* a bounded device wait expired (the tensor-core barrier of
                       the Schur update; see rss_params.wait_polls) */
  RSS_EBUSY = 6     /* reserved */
} rss_status;

/* Kernel kinds.
 *  RSS_LAPLACE    A_ij = -(h^2 / 2 pi) log |x_i - x_j|, real (paper Eq. 15).
 *  RSS_HELMHOLTZ  A_ij = h^2 (i/4) H0^(1)(kappa |x_i - x_j|), complex (Eq. 18
 *                 without the kappa^2 sqrt(b_i b_j) factor of Eq. 19).
 *  RSS_TEST_POLY  A_ij = scale conj(w_i) w_j sum_d coef[d] (z_i - z_j)^d,
 *                 z = x + i y, w = exp(i (phase_x x + phase_y y)), complex.
 *  RSS_TEST_RPOLY the real part of sum_d coef[d] (z_i - z_j)^d times scale.
 *  RSS_HELMHOLTZ_LS  the symmetrised Lippmann-Schwinger system of Eqs. 19-20:
 *                 A_ij = w_i w_j h^2 (i/4) H0^(1)(kappa |x_i - x_j|) with
 *                 w = kappa sqrt(b(x)), b(x) = exp(-bump_a |x - (bump_cx, bump_cy)|^2),
 *                 and A_ii = 1 + w_i^2 d, d = diag_re + i diag_im (or, with
 *                 diag_rule = 1, the self-cell integral of (i/4) H0^(1) of Eq. 20);
 *                 complex.  Proxy points (Eq. 6) take the weight kappa.
 * The two test kinds have an exactly low-rank far field, so the whole
 * factorization is exact up to rounding; they exist to verify the elimination
 * bookkeeping against a dense solve and are not a workload of the paper. */
enum { RSS_LAPLACE = 0, RSS_HELMHOLTZ = 1, RSS_TEST_POLY = 2, RSS_TEST_RPOLY = 3, RSS_HELMHOLTZ_LS = 4 };

#define RSS_MAX_COEF 8

typedef struct {
  int kind;                       /* one of the kinds above */
  double h;                       /* entry scale h (h^2 multiplies K); <= 0: the grid spacing */
  double kappa;                   /* Helmholtz wavenumber */
  double diag_re, diag_im;        /* A_ii */
  int proxy_n;                    /* points on the proxy circle (Eq. 6); 0: 64 */
  double proxy_radius_over_side;  /* proxy-circle radius / box side; 0: 1.25 */
  double eps;                     /* ID tolerance (Definition 1), >= 0 */
  int ncoef;                      /* test kernels: number of coefficients (<= RSS_MAX_COEF) */
  double coef_re[RSS_MAX_COEF], coef_im[RSS_MAX_COEF];
  double scale, phase_x, phase_y; /* test kernels */
  int id_rows;                    /* 0: for a real symmetric kernel (Laplace with a real
                                     diagonal) compress [A_MB; K_PB] only, which equals the
                                     full stack of Eq. 4 up to rounding; 1: always the full
                                     stack [A_MB; K_PB; A_BM^*; K_BP^*] */
  int schur_path;                 /* 0: the dense products of the elimination on the tensor
                                     cores where they apply: the Schur update A_CC -= E F
                                     (any rank) and
                                     E = A_CB W_E and
                                     F^T = A_BC^T W_F (real factors with n_B <= 128,
                                     complex with any n_B); operands split into eight 7-bit
                                     slices with row and column scales, exact integer
                                     products, FP64 recombination (accuracy of an FP64
                                     product); the Schur update runs on tcgen05
                                     (tensor memory accumulators) when every r <= 384
                                     (real) or r <= 192 (complex);
                                     1: FP64 FMA kernels everywhere; 2: as 0 with the real
                                     Schur update on warp-level MMAs (mma.sync), the same
                                     integer arithmetic and, for real factors, the same
                                     result */
  int id_cluster;                 /* colour classes with fewer boxes than the GPU has room for:
                                     0 spreads each box's ID over a thread-block cluster of
                                     up to 8 CTAs, > 0 sets the largest cluster size (1: one
                                     CTA per box; at most 16, above 8 a non-portable cluster
                                     size), -1 is the same as 1 */
  double bump_cx, bump_cy, bump_a;/* RSS_HELMHOLTZ_LS: b(x) = exp(-bump_a |x - c|^2); bump_a
                                     <= 0 selects the paper's (0.5, 0.5) and 32 */
  int diag_rule;                  /* 0: the diagonal is diag_re + i diag_im; 1: the paper's
                                     quadrature, the integral of the kernel over the point's
                                     own h x h cell (Eq. 16 for Laplace, Eq. 20 for Helmholtz
                                     and Lippmann-Schwinger), see rss_self_integral */
  int per_box;                    /* 0: all boxes of a colour class in one launch per phase;
                                     1: the plain per-box form, one box per launch in the same
                                     order (for comparison: same mathematics, slower) */
  int class_order;                /* 0: the boxes of a colour class in row-major order; any
                                     other value: a permutation of each class drawn from this
                                     seed (same-colour boxes are independent, Algorithm 1 with
                                     nine colours, so the factorization must not change) */
  int wait_polls;                 /* device waits are bounded: a CTA of the tensor-core Schur
                                     update polls its barrier at most this many times before it
                                     gives up, and rss_factor then returns RSS_ETIMEOUT (after
                                     the products already issued have finished, so nothing is
                                     left running); a CTA of the persistent solve sweeps polls a
                                     grid barrier at most this many times, and a solve whose
                                     barrier ran out writes NaN into every entry of its result.
                                     0: the default limits (2^22 and 2^24 polls); n > 0: n polls;
                                     -1: give up without polling, which exercises the timeout
                                     paths on purpose (for tests) */
  const char* tune_table;         /* NULL, or the JSON object rss_tune_solve returned (read during
                                     the call): its last "launch", "spread", "ctas_per_sm" and
                                     "tail_boxes" set the launch form of the solve sweeps without
                                     measuring again.
                                     A form changes the time of a solve, never its result */
} rss_params;

/* Build the quadtree of Section 2.1 for n points given as pts_xy[2*i],
 * pts_xy[2*i+1] (host memory, read only during the call).  The points must be
 * the n = s*s nodes of a uniform square grid (any origin and spacing, any
 * order).  leaf is the number of points per leaf box, a square l*l with s/l
 * a power of two.  On success *out holds a tree the caller releases with
 * rss_free; a tree may be shared by several factorizations. */
rss_status rss_build_tree(const double* pts_xy, int64_t n, int leaf, rss_tree** out);

/* Factor A for the tree's points (Algorithm 1: per level, all boxes of one
 * colour class in one batched launch per phase; the ID of Eq. 6, the
 * elimination of Eq. 8, the Schur update of Remark 2, the merge of Section
 * 2.4, a dense LU at the top).  stream is a cudaStream_t (NULL: the legacy
 * default stream) on the current device.  The call returns when the
 * factorization is complete.  *out is released with rss_free; the factor
 * keeps its own copy of everything it needs from tree and params. */
rss_status rss_factor(const rss_tree* tree, const rss_params* params, void* stream,
                      rss_factorization** out);

/* Overwrite b (n x nrhs, column-major, leading dimension ldb >= n, entries in
 * the caller's point order) with the RS-S approximation of A^{-1} b
 * (Section 2.5).  b may be device memory (the call is then asynchronous on
 * stream) or host memory (the library stages it through the device and
 * returns after the result is back).  Real factors take double, complex
 * factors interleaved complex double.  Calls on distinct streams may run
 * concurrently on the same factor (the factor is read only). */
rss_status rss_solve(const rss_factorization* f, void* b, int64_t nrhs, int64_t ldb, void* stream);

/* rss_solve without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory at call time --
 * a process whose framework allocator already holds the device's free memory,
 * or a latency-bound serving loop that must not pay for (or synchronise on) a
 * fresh allocation.  Results are those of rss_solve.
 *  - b must be device memory (n x nrhs, column-major, ldb >= n); the call is
 *    asynchronous on stream.
 *  - The working copy of b lives in a fixed 16 MiB array compiled into the
 *    library, held on every GPU that loads it until the process exits:
 *    n * nrhs * sizeof(scalar) must be <= 16 MiB (8 or 16 bytes per scalar),
 *    else RSS_EINVAL with nothing launched.
 *  - The first call on a device looks up that array's device address (once
 *    per device, with the device current); make that first call before any
 *    stream capture.
 *  - All calls share the one array: calls whose work overlaps on the GPU
 *    (for example on two streams at once) race and corrupt each other; order
 *    them on one stream or synchronise between them.  Each call overwrites
 *    the whole region it uses before reading it. */
rss_status rss_solve_noalloc(const rss_factorization* f, void* b, int64_t nrhs, int64_t ldb,
                             void* stream);

/* Autotuner of the solve's launch form.  The FP64 sweeps (fewer than 32
 * right-hand sides) run in one of three forms, which add the same products in
 * the same order, so results are bitwise the same under any of them:
 *  - "per_class": kernels per colour class (two or three launches each);
 *  - "persistent": two cooperative launches that walk all colour classes of the
 *    factorization, meeting at grid barriers; a class with few boxes is split
 *    across CTAs by rows of C (one more barrier);
 *  - "hybrid": per-class kernels for the fine levels and persistent launches for
 *    the tail of colour classes with fewer than "tail_boxes" boxes each (the
 *    coarse levels, where per-class launches are bound by latency).
 * The persistent part has two knobs: "spread", the target number of work items
 * per CTA and class, and "ctas_per_sm" (0: as many as fit).  rss_tune_solve
 * times the solve of nrhs zero right-hand sides under eleven candidates (the
 * per-class form, four persistent and six hybrid schedules; median of three
 * after one untimed run, CUDA events on stream), keeps the fastest for the
 * later solves of f, and writes the table to json (may be NULL) as {"nrhs": ..,
 * "path": .., "candidates": [..], "launch": .., "spread": .., "ctas_per_sm":
 * .., "tail_boxes": .., "ms": ..}; passing that text back as
 * rss_params.tune_table applies it without measuring.  With 32 or more
 * right-hand sides (tensor-core sweeps) there is nothing to tune and the table
 * says so.  The paper has no counterpart.  Synchronises stream; allocates
 * n * nrhs scalars for the duration of the call; solves that run meanwhile on
 * other streams may take either form. */
rss_status rss_tune_solve(rss_factorization* f, int64_t nrhs, void* stream, char* json, size_t len);

/* ---- Serving: resident factorizations, continuous batching of solves ----
 * A server owns a worker thread and, per registered factorization, a CUDA
 * stream.  Whenever a factorization's stream is idle, the worker packs all of
 * its pending requests (up to max_batch_rhs columns, and only as far as the
 * device-memory budget allows) into one right-hand-side panel and solves it
 * with one rss_solve; requests arriving meanwhile join the next panel, and
 * panels of different factorizations run concurrently on their own streams.
 * Every column goes through the same operations whatever it is batched with,
 * so a result equals the one rss_solve gives for the request alone.  This is
 * the serving pattern the workloads ask for (requests of 1-64 right-hand sides
 * against several resident factorizations); the paper has no counterpart. */

/* Start a server that may hold at most device_bytes of device memory for
 * panels and solve workspaces, with at most max_batch_rhs columns per panel.
 * A panel of c columns is charged n * c scalars for itself plus what the solve
 * allocates for it (its working copy of the panel and the sweep workspace). */
rss_status rss_server_create(size_t device_bytes, int64_t max_batch_rhs, rss_server** out);

/* Register a factorization (it must outlive the server); *factor_id names it.
 * Caches that the factorization's solves would build on first use (the digit
 * slices of E and F that real factors use for 32 or more columns) are built
 * here, on the server's stream for this factorization, and charged to the
 * budget for the server's lifetime; RSS_ENOMEM if they and a one-column panel
 * do not fit. */
rss_status rss_server_add(rss_server* s, const rss_factorization* f, int32_t* factor_id);

/* Queue a solve: b and x are host arrays of n x nrhs scalars, column-major with
 * leading dimension n; both must stay valid until rss_server_wait returns for
 * *ticket.  x receives A^{-1} b.  Returns at once. */
rss_status rss_server_submit(rss_server* s, int32_t factor_id, const void* b, void* x, int64_t nrhs,
                             int64_t* ticket);

/* Block until the request is done (timeout_s <= 0: no limit; RSS_ETIMEOUT if
 * it is still pending then).  *latency_s (may be NULL) receives the time from
 * submission to the result being in x.  A request that can never fit the
 * budget fails with RSS_ENOMEM. */
rss_status rss_server_wait(rss_server* s, int64_t ticket, double timeout_s, double* latency_s);

/* JSON counters: requests, panels, columns, largest panel, memory in use. */
rss_status rss_server_stats(rss_server* s, char* buf, size_t len);


/* Integral of the kernel over one h x h cell centred on the singularity
 * (paper Eqs. 16 and 20): kind RSS_LAPLACE gives the closed form
 * -(1/2pi) 2 a^2 (2 log a + log 2 - 3 + pi/2), a = h/2; RSS_HELMHOLTZ and
 * RSS_HELMHOLTZ_LS give the integral of (i/4) H0^(1)(kappa |x|), reduced by the
 * cell's symmetry to 8 (i/4) int_0^{pi/4} [rho H1^(1)(kappa rho)/kappa + 2i/(pi kappa^2)]
 * dtheta, rho = a / cos(theta), by Gauss-Legendre quadrature.  Host only, no
 * GPU work.  EINVAL for other kinds, h <= 0, or kappa <= 0 where it is needed. */
rss_status rss_self_integral(int kind, double h, double kappa, double* re, double* im);

/* y = A x for the factored matrix (the exact A of Eq. 3, not its
 * factorization), applied by FFT: on the uniform grid the off-diagonal part is
 * a two-level Toeplitz convolution, embedded in a 2s x 2s circulant (s points
 * per side); the diagonal and the Lippmann-Schwinger weights are applied
 * pointwise.  x and y: device buffers of n x nrhs scalars, leading dimension
 * ld >= n, in the caller's point order; x and y must not overlap.  The first
 * call builds the circulant's spectrum (16 (2s)^2 bytes kept with the factor)
 * and a cuFFT plan.  Asynchronous on stream. */
rss_status rss_matvec(const rss_factorization* f, const void* x, void* y, int64_t nrhs, int64_t ld,
                      void* stream);

/* Solve A x = b to a relative residual ||b - A x|| / ||b|| <= tol with the
 * factorization as preconditioner (Section 5): method 1 is preconditioned
 * conjugate gradients (symmetric positive definite A: the Laplace kernel with
 * the quadrature diagonal), method 2 right-preconditioned GMRES(restart)
 * (restart <= 0: 20), method 0 picks PCG for real factors and GMRES for complex
 * ones.  Both start from x0 = (factorization)^{-1} b.  b and x: device buffers
 * of n scalars in the caller's order (one right-hand side).  *iters receives
 * the iterations (GMRES: Arnoldi steps) and *relres the final relative residual
 * of b - A x (either may be NULL).  At most maxit iterations (<= 0: 200); not
 * reaching tol is not an error.  Synchronises stream. */
rss_status rss_solve_iterative(const rss_factorization* f, const void* b, void* x, double tol, int maxit,
                               int restart, int method, int* iters, double* relres, void* stream);

/* Release a tree, a factor or a server (the handle is tagged; a server first
 * finishes its in-flight panels).  NULL is ignored. */
void rss_free(void* handle);

/* Device memory.  Every device allocation of the library (factor storage,
 * per-level stencil slabs and workspaces, solve and server panels) comes from
 * one stream-ordered pool per device, owned by the library.  Freed blocks stay
 * reserved for the next factorization or solve instead of going back to the
 * driver, so repeated calls do not map and unmap memory.  rss_trim_memory
 * waits for the current device, then returns reserved but unused memory of
 * its pool to the driver until at most keep_bytes stay reserved.  Errors:
 * RSS_ECUDA if the device cannot be queried or synchronised. */
rss_status rss_trim_memory(size_t keep_bytes);

/* Measurement, not part of the method (the paper has no counterpart): the FP64
 * fused multiply-add throughput of the current device, from a loop of
 * independent DFMA chains over 8 CTAs of 256 threads per SM, best of five timed
 * launches (CUDA events on stream) after one warm-up.  *tflops receives
 * 2 x FMAs / time in TFLOP/s and *ms (may be NULL) the launch time.  It is the
 * peak against which the FP64-bound phases (the ID, the small LUs) are reported.
 * Synchronises stream; takes about half a second. */
rss_status rss_probe_fp64(double* tflops, double* ms, void* stream);

/* Measurement, as rss_probe_fp64, of the FP64 tensor-core MMA (mma.sync m8n8k4
 * f64, 512 flops per warp-wide product): eight independent accumulator chains per
 * warp, 8 CTAs of 256 threads per SM, best of five timed launches after one
 * warm-up.  It shows whether FP64 tensor products would beat plain DFMA. */
rss_status rss_probe_dmma(double* tflops, double* ms, void* stream);

/* Message for the last non-OK status returned on this thread. */
const char* rss_last_error(void);

/* JSON summary of a factor: sizes, ranks per level, phase times, bytes held. */
rss_status rss_info(const rss_factorization* f, char* buf, size_t len);

/* Inspection (used by the tests): skeleton ranks of the boxes of the level
 * whose box grid has side `side` (row-major boxes), into k_out[side*side]. */
rss_status rss_level_ranks(const rss_factorization* f, int side, int32_t* k_out);

/* Inspection: the factor record of box `box` at level `side`, copied to host
 * buffers (any pointer may be NULL to skip it).  Sizes are returned in
 * sizes[0..3] = k, r, c, n.  Index lists are in the caller's point order:
 * S (k), R (r), C (c, starting with S).  T is k x r, LU r x r (packed, with
 * 0-based getrf pivots piv[r]), E is c x r, F is r x c, all column-major with
 * leading dimension equal to the row count.  Returns RSS_EINVAL if the box
 * had no redundant points at that level. */
rss_status rss_box_record(const rss_factorization* f, int side, int box, int32_t* sizes,
                          int64_t* S, int64_t* R, int64_t* C, void* T, void* LU,
                          int32_t* piv, void* E, void* F);

#ifdef __cplusplus
}
#endif
#endif
