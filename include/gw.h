/*
 * gw.h - C ABI of the GB300 fast Gromov-Wasserstein gradient library.
 *
 * The library computes, on one GPU, the gradient of the discrete
 * Gromov-Wasserstein objective for distributions on uniform grids and runs
 * the entropic mirror-descent solver built on it, following
 * "Fast Gradient Computation for Gromov-Wasserstein Distance"
 * (Zhang, Wang, Fan, Wu, Zhang; arXiv 2404.08970).
 *
 * Notation (Sec. 2 of the paper): X has n points (the paper's M), Y has m
 * points (the paper's N).  Distances on a uniform 1D grid are
 * d_ij = h^k |i - j|^k (eq. "1d distance matrices"); on an s x s 2D grid a
 * point (a, b) has index a*s + b.  A coupling T is an n x m row-major array,
 * T[i*m + p].
 *
 * The gradient returned by gw_grad is
 *     G = L(C_X, C_Y) (x) T = c_x 1^T + 1 c_y^T - 2 D_X T D_Y,
 *     c_x = (D_X o D_X) r,  c_y = (D_Y o D_Y) c,
 * which is half the paper's grad E = C1 - 4 D_X Gamma D_Y (Sec. 2.1,
 * gradient decomposition).  r, c are either the target marginals (u, v), as
 * in the paper's C1, or T's own marginals (T 1, T^T 1), which makes G exact
 * for any T.
 *
 * Conventions shared by every entry point:
 *  - Device pointers (prefix d_) are caller-owned device memory; the library
 *    never frees or keeps them beyond the call's stream work.
 *  - Host pointers (prefix h_) are caller-owned host memory.
 *  - stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue work and return without synchronising unless stated.
 *  - Each call returns a gw_status.  On an error the call enqueues nothing
 *    and gw_last_error(ctx) describes the cause.
 *  - Calls that share a context share its device workspace: order them on
 *    one stream (or use one context per stream).  Host-side state of a
 *    context is protected by a mutex.
 */
#ifndef GW_FGC_H
#define GW_FGC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GW_OK = 0,
  GW_NOT_READY = 1,
  GW_ERR_INVALID = -1,   /* bad argument or descriptor */
  GW_ERR_OOM = -2,       /* device allocation failed */
  GW_ERR_CUDA = -3,      /* a CUDA call failed */
  GW_ERR_TIMEOUT = -4,   /* a bounded device wait gave up */
  GW_ERR_NONFINITE = -5, /* a non-finite value reached an output */
  GW_ERR_SHUTDOWN = -6   /* the server is shutting down */
} gw_status;

typedef enum { GW_F32 = 0, GW_F64 = 1 } gw_dtype;

/* Distance on 2D grids.  GW_COST_POW: Manhattan distance to the power k,
 * h^k (|a-a'| + |b-b'|)^k (Sec. 3.1, eq. "2d Dx"); on 1D grids it is the
 * only cost, h^k |i-j|^k.  GW_COST_SQEUCLID: h^2 ((a-a')^2 + (b-b')^2). */
typedef enum { GW_COST_POW = 0, GW_COST_SQEUCLID = 1 } gw_cost;

/* Arithmetic of the dense comparison gradient (gw_grad_dense). */
typedef enum {
  GW_DENSE_FP32 = 0,
  GW_DENSE_TF32 = 1,
  GW_DENSE_BF16 = 2,
  GW_DENSE_FP64 = 3,
  GW_DENSE_TC_TF32 = 4, /* the library's own tcgen05 kernels, TF32 inputs */
  GW_DENSE_TC_BF16 = 5  /* the library's own tcgen05 kernels, BF16 inputs */
} gw_dense_precision;

/* Which marginals build the constant term c_x, c_y of the gradient. */
typedef enum { GW_MARG_TARGET = 0, GW_MARG_EXACT = 1 } gw_marginals;

/* Problem descriptor, following the paper's problem statement (Sec. 2). */
typedef struct gw_problem {
  int dim;       /* 1, 2 or 3 */
  int nx, ny;    /* 1D: points of X and Y; 2D, 3D: grid sides (points =
                    side^dim) */
  double hx, hy; /* grid spacings h_X, h_Y (> 0) */
  int k;         /* distance exponent, integer >= 1 (k_X = k_Y = k) */
  int cost;      /* gw_cost (2D and 3D; 1D uses GW_COST_POW) */
  double eps;    /* entropic regularisation (> 0), solver only */
  int n_outer;   /* mirror-descent iterations, solver only */
  int n_inner;   /* Sinkhorn iterations per mirror-descent step, solver only */
  double theta;  /* fused-GW weight of the GW term, in [0, 1]; 1 = plain GW */
  int feat_dim;  /* fused-GW feature dimension (0 = none) */
  int dtype;     /* gw_dtype of T, G (and of the solver's arithmetic) */
  double tau;    /* mirror-descent proximal weight (eq. "GW proximal gradient"),
                    solver only: > 0, or 0 for tau = eps (the Remark's choice) */
  int warm_start; /* solver only: 1 starts each mirror-descent step's Sinkhorn
                    iteration from the previous step's potentials, 0 from
                    f = g = 0 */
  double rho;    /* solver only: 0 for balanced (F)GW; > 0 solves entropic
                    unbalanced GW with marginal relaxation rho (Remark
                    "Entropic algorithm for UGW") */
  int ky;        /* 1D: exponent of Y's distance when it differs from X's
                    (Sec. 2 allows k_X != k_Y); 0 means ky = k.  Mixed pairs
                    (k, ky) = (1, 2) or (2, 1), rows of at most 8192 columns
                    (4096 in double) */
} gw_problem;

typedef struct gw_ctx gw_ctx;

/* Creates a context on CUDA device `device` (made current for the calls of
 * this context).  *ctx receives the handle.  GW_ERR_CUDA if the device is
 * unusable.  With the environment variable GW_FORCE_GENERIC set to a value
 * other than "0" at creation, the context's 1D gradients use the generic row
 * kernel (one thread block per band, no warp specialisation) even where the
 * warp-specialised one applies: same results within rounding, for testing
 * that kernel on shapes the fast one would take. */
gw_status gw_ctx_create(gw_ctx** ctx, int device);

/* Frees the context and its device workspace (synchronises the device). */
void gw_ctx_destroy(gw_ctx* ctx);

/* Text of the last error on this context ("" if none).  The string stays
 * valid until the next call on the context. */
const char* gw_last_error(const gw_ctx* ctx);

/* Synchronises `stream`, then reads and clears the context's device status
 * word.  GW_ERR_TIMEOUT if a bounded device wait gave up since the last
 * check, GW_ERR_NONFINITE if a kernel flagged a non-finite output, GW_OK
 * otherwise. */
gw_status gw_ctx_check(gw_ctx* ctx, void* stream);

/* Switches per-kernel timing on (enable = 1) or off (0).  While on, every
 * kernel the library launches for this context is bracketed by CUDA events
 * recorded on the call's stream (a small cost per launch). */
gw_status gw_ctx_profile(gw_ctx* ctx, int enable);

/* Waits for the recorded events, folds them into per-kernel totals and
 * writes the totals to buf as JSON text:
 *   {"kernel": {"launches": L, "ms": T}, ...}
 * reset = 1 clears the totals afterwards.  GW_ERR_INVALID if buf (len bytes)
 * is too small or NULL. */
gw_status gw_ctx_profile_report(gw_ctx* ctx, char* buf, size_t len, int reset);

/*
 * gw_grad - the structured gradient G = L(C_X, C_Y) (x) T (Sec. 3, eqs. "Dx",
 * "1d y", "1d recursive relation"; Sec. 3.1, eqs. "2d gradient" and
 * "2D kronecker"; 3D grids by the same construction with a third axis, which
 * Sec. 3.1 says differs in nothing essential).
 *
 *   prob       dim 1: any k >= 1 up to 3, nx, ny >= 1, ny <= 16384.
 *              dim 2: grid sides nx, ny in [1, 256] (n = nx^2, m = ny^2
 *              points, index a * side + b), cost GW_COST_SQEUCLID, or
 *              GW_COST_POW with k = 1 (Manhattan): the costs that split over
 *              the two axes, so that D_X T D_Y reduces to four side x side
 *              partial sums of T (k = 1 case of eq. "2D kronecker");
 *              GW_COST_POW with k = 2, 3 (Manhattan^k, image transforms by
 *              the paper's recursion) for sides up to 128 in float.
 *              dim 3: grid sides nx, ny in [1, 32] (n = nx^3, m = ny^3
 *              points, index (a * side + b) * side + c), cost
 *              GW_COST_SQEUCLID or GW_COST_POW with k = 1: D_X T D_Y reduces
 *              to nine side x side partial sums of T.
 *              Only dim, nx, ny, hx, hy, k, cost, dtype are read.
 *   d_u, d_v   target marginals, double, lengths n and m; read only with
 *              marginals == GW_MARG_TARGET (may be NULL otherwise).
 *   d_T        the coupling, n x m row-major, prob->dtype.
 *   d_G        output, n x m row-major, prob->dtype; must not overlap d_T.
 *   marginals  GW_MARG_TARGET or GW_MARG_EXACT.
 *
 * Cost O(n m): the DP recursion along columns and rows (1D), or one pass
 * over T plus side x side transforms (2D, 3D), replaces the dense products.
 * With dtype GW_F32 the arithmetic is float with compensated sums and
 * carries; GW_F64 computes in double throughout.
 * Errors: GW_ERR_INVALID for a bad descriptor or a NULL required pointer.
 */
gw_status gw_grad(gw_ctx* ctx, const gw_problem* prob, const double* d_u, const double* d_v,
                  const void* d_T, void* d_G, int marginals, void* stream);

/*
 * gw_grad_host - gw_grad on host buffers: the same gradient (Sec. 3, eqs.
 * "Dx", "1d y", "1d recursive relation"; Sec. 3.1 for dim 2), for callers
 * whose T lives in host memory.
 *
 *   prob, marginals   as for gw_grad.
 *   h_u, h_v          host marginals (double, n and m); read only with
 *                     GW_MARG_TARGET.
 *   h_T               host coupling, n x m row-major, prob->dtype.
 *   h_G               host output, n x m row-major, prob->dtype; must not
 *                     overlap h_T.
 *   stream            the caller's stream: work enqueued on it after this
 *                     call runs after h_G has been written, so
 *                     cudaStreamSynchronize(stream) (or gw_ctx_check with
 *                     the same stream) makes h_G ready to read.
 *
 * Asynchronous: the call returns once the copy of h_T to the device, the
 * gradient and the copy of G back are enqueued on the context's own streams.
 * It does not wait for earlier work on `stream`, so h_u, h_v and h_T must
 * hold their values when the call is made, and none of the host buffers may
 * be changed or freed until `stream` has been synchronised.  Two device
 * slots (T and G each) owned by the context are used in turn, so a call's
 * copy-in overlaps the previous call's gradient and copy-out.  Page-locked
 * host buffers (cudaHostAlloc) make the copies fully asynchronous; pageable
 * ones are still correct, at copy speeds the driver chooses.  The slots are
 * grown on demand (the device is synchronised when that happens).
 * Errors: as gw_grad; GW_ERR_OOM if the slots cannot be allocated.
 */
gw_status gw_grad_host(gw_ctx* ctx, const gw_problem* prob, const double* h_u, const double* h_v,
                       const void* h_T, void* h_G, int marginals, void* stream);

/*
 * gw_grad_noalloc - gw_grad without any device allocation (the paper has no
 * counterpart; this is a deployment convenience).
 *
 * For callers that cannot allocate device memory when they need a gradient:
 * a process whose device memory is fully reserved by another framework's
 * caching allocator, a thread that must not block in cudaMalloc/cudaFree
 * (both can synchronise the device), or code that must keep a fixed memory
 * footprint after start-up.  The scratch comes from one static device array
 * of 32 MiB that every device loading the library reserves until exit; no
 * context is needed and nothing is allocated.
 *
 *   Arguments as for gw_grad (dim 1 only), on the current CUDA device.  Problems whose
 *   scratch need exceeds 32 MiB (about 4096 x 4096 floats with k <= 2) return
 *   GW_ERR_INVALID; so do invalid descriptors or NULL required pointers.
 *   The first call on each device looks up the array's device address (make
 *   that first call before any stream capture).  All calls share the array:
 *   calls that overlap on the GPU (different streams, no ordering) race.
 *   hx and hy must be finite and positive.  The kernels' bounded device
 *   waits share one static status word too, cleared on `stream` before each
 *   launch, so that a launch whose wait has run out ends quickly; such a
 *   failure leaves G invalid and is not reported by the return value (the
 *   call returns before the kernels run).
 */
gw_status gw_grad_noalloc(const gw_problem* prob, const double* d_u, const double* d_v, const void* d_T,
                          void* d_G, int marginals, void* stream);

/*
 * gw_grad_dense - the same gradient G as gw_grad, computed the original way
 * (Sec. 2.1, gradient decomposition): the distance matrices D_X (n x n) and
 * D_Y (m x m) are materialised and G = c_x 1^T + 1 c_y^T - 2 (D_X T) D_Y is
 * formed with two cuBLAS matrix products, O(n^2 m + n m^2).  It exists as the
 * comparison baseline of the structured method.
 *
 *   precision  GW_DENSE_FP32 (FP32 CUDA cores), GW_DENSE_TF32 or GW_DENSE_BF16
 *              (tensor cores, FP32 accumulation; BF16 rounds T, D and the
 *              intermediate D_X T to bfloat16), GW_DENSE_FP64: products by
 *              cuBLAS.  GW_DENSE_TC_TF32 and GW_DENSE_TC_BF16: the same
 *              products on the library's own tcgen05 kernels (TMA-fed
 *              128 x 256 tiles, FP32 accumulators in tensor memory, the
 *              constant terms added in the second product's epilogue, so Z
 *              is never stored); inputs rounded as for the cuBLAS forms
 *              (TF32 keeps the top 19 bits of each float).
 *   prob->dtype must be GW_F64 for GW_DENSE_FP64 and GW_F32 otherwise; the
 *   other arguments are as for gw_grad (dim 1, 2 or 3; on grids the
 *   distance matrices are n x n and m x m over the grid points).  The dense distance
 *   matrices are cached in the context between calls.
 */
gw_status gw_grad_dense(gw_ctx* ctx, const gw_problem* prob, const double* d_u, const double* d_v,
                        const void* d_T, void* d_G, int marginals, int precision, void* stream);

/*
 * gw_solve - entropic (fused) Gromov-Wasserstein by mirror descent (Sec.
 * 2.1, eqs. "GW proximal gradient" and "GW sinkhorn", with the Remark's
 * tau = eps unless prob->tau is set; fused GW by the Remark "FGW").
 *
 * Starting from T^0 = u v^T, each of prob->n_outer steps forms the cost
 *     Pi = 2 theta G(T) + (1 - theta) C o C + (eps - tau) ln T,
 *     G = L(C_X, C_Y) (x) T with the target marginals (gw_grad),
 *     C o C_ip = ||phi_i - psi_p||^2 (the last term vanishes for tau = eps;
 *     an entry of T that underflowed to 0 counts as the smallest normal),
 * and runs prob->n_inner log-domain Sinkhorn iterations at regularisation
 * tau from f = g = 0 (with prob->warm_start, from the previous step's f, g
 * after the first step), f then g each iteration, then sets
 * T_ip = exp((f_i + g_p - Pi_ip) / tau).
 *
 *   prob         dim 1, 2 or 3; nx, ny, hx, hy, k, cost as for gw_grad, with
 *                at most 16384 points in Y (ny, or ny^dim on grids; 10240 with
 *                GW_F64); eps > 0;
 *                tau = 0 (tau = eps) or > 0; warm_start 0 or 1;
 *                n_outer >= 0; n_inner >= 1; theta in [0, 1]; feat_dim in
 *                [1, 64] when theta < 1; dtype GW_F32 or GW_F64 (the
 *                arithmetic precision of the whole solve).
 *   d_u, d_v     target marginals (double, lengths n and m, positive).
 *   d_phi,d_psi  fused-GW features, double, row-major n x feat_dim and
 *                m x feat_dim; read only when theta < 1 (else may be NULL).
 *   d_T          output plan, n x m row-major, prob->dtype.
 *   d_f, d_g     output potentials of the last Sinkhorn solve (double,
 *                lengths n and m, in the units of its regularisation tau)
 *                or NULL.
 *   d_stats      NULL or 8 doubles on the device: [0] objective
 *                (1 - theta) <C o C, T> + theta E(T), [1] E(T) (the GW
 *                energy, Sec. 2), [2] <C o C, T>, [3] eps H(T),
 *                [4] sum_i |(T 1)_i - u_i|, [5] sum_p |(T^T 1)_p - v_p|,
 *                [6] outer iterations run, [7] 0.
 *
 * The call enqueues the whole solve on `stream` and returns.  The context
 * workspace holds Pi (n*m reals) plus O(n + m) state.
 */
gw_status gw_solve(gw_ctx* ctx, const gw_problem* prob, const double* d_u, const double* d_v,
                   const double* d_phi, const double* d_psi, void* d_T, double* d_f, double* d_g,
                   double* d_stats, void* stream);

/*
 * gw_solve_batch - `count` independent solves (as gw_solve, without the
 * potentials) in one call: the batched workload of many problems of mixed
 * sizes (the paper solves one problem at a time; batching is a throughput
 * mode of the same method).
 *
 *   probs[i]            descriptor of problem i (validated as for gw_solve).
 *   d_u[i], d_v[i]      target marginals of problem i (device, double).
 *   d_phi, d_psi        NULL, or arrays whose entry i is problem i's feature
 *                       array (NULL where theta == 1).
 *   d_T[i]              output plan of problem i (device, probs[i].dtype).
 *   d_stats             NULL, or an array whose entry i is NULL or 8 device
 *                       doubles (layout as for gw_solve).
 *   The pointer arrays themselves are host memory, read during the call.
 *
 * Problems of one dtype and schedule whose rows fit the 512-thread row
 * configurations (up to 8192 columns in float, 4096 in double) advance in
 * lock step and share every Sinkhorn launch: each pass is one launch over all
 * of their row bands (bands of at least 32 rows), each block running its own
 * problem's row configuration; the gradients and statistics run per problem
 * on worker streams.  Longer rows form groups of one row configuration (up
 * to 32 problems per launch) beside them.  The worker streams belong to the
 * context and are forked from and joined back into `stream`; each problem
 * gets its own region of a batch workspace owned by the context.
 * The whole batch is captured once into one CUDA graph and relaunched while
 * the arguments are unchanged.  Results agree with gw_solve on each problem
 * alone up to rounding (the batch's longer row bands group the partial sums
 * differently).
 * Errors: GW_ERR_INVALID naming the first bad problem; GW_ERR_OOM if the
 * batch workspace cannot be allocated.
 */
gw_status gw_solve_batch(gw_ctx* ctx, int count, const gw_problem* probs, const double* const* d_u,
                         const double* const* d_v, const double* const* d_phi, const double* const* d_psi,
                         void* const* d_T, double* const* d_stats, void* stream);

/* Fixed-support GW barycenter problem (gw_barycenter). */
typedef struct gw_barycenter_problem {
  int count;    /* input spaces, 1 .. 64 */
  int N;        /* barycenter points, 1 .. 4096 */
  int k;        /* distance exponent of the input grids, 1 or 2 */
  int dtype;    /* GW_F32 or GW_F64: plans, C and the solves' arithmetic */
  double eps;   /* entropic regularisation of every GW solve (> 0) */
  int n_iter;   /* barycenter rounds (>= 1) */
  int n_outer;  /* mirror-descent steps per GW solve (>= 1) */
  int n_inner;  /* Sinkhorn iterations per step (>= 1) */
} gw_barycenter_problem;

/*
 * gw_barycenter - fixed-support GW barycenter of spaces on 1D grids (the
 * conclusion names the barycenter among the GW variants that the fast
 * gradient accelerates; the iteration is the cited barycenter method's
 * block coordinate descent with the square loss).
 *
 * Input s is the grid of n[s] points i h[s] with distances h[s]^k |i - j|^k
 * and marginal d_ps[s]; the barycenter has N points with weights d_p and a
 * dense distance matrix C.  Each of prob->n_iter rounds solves entropic GW
 * between (C, p) and every input by mirror descent (as gw_solve: T^0 = p
 * p_s^T, cost 2 G with G = (C o C) p 1^T + 1 ((D_s o D_s) p_s)^T - 2 C T D_s,
 * prob->n_outer steps of prob->n_inner Sinkhorn iterations at eps) and then
 * sets
 *     C = sum_s lambda[s] T_s D_s T_s^T / ((sum_s lambda[s]) p p^T).
 * T D_s is the paper's O(N n) transform along the rows of T (double
 * arithmetic); C (T D_s) and (T_s D_s) T_s^T are dense products accumulated
 * in double.
 *
 *   n, h, lambda  host arrays of prob->count entries: grid sizes (1 .. 16384,
 *                 10240 with GW_F64), spacings (finite, > 0), weights
 *                 (finite, >= 0, positive sum).
 *   d_ps          host array of prob->count device pointers to the inputs'
 *                 marginals (double, n[s] each).
 *   d_p           barycenter weights (device, double, N, positive).
 *   d_C           device N x N row-major array of prob->dtype: the initial
 *                 distance matrix on entry, the barycenter's on return.
 *   d_stats       NULL, or 8 * count device doubles: for each input the
 *                 statistics of its last round's solve (layout as gw_solve's
 *                 stats, against the C of that round).
 *
 * The whole computation is captured once into a CUDA graph keyed by the
 * arguments and relaunched while they are unchanged.  Errors: GW_ERR_INVALID
 * for a bad descriptor, size or pointer; GW_ERR_OOM if the workspace cannot
 * be allocated.
 */
gw_status gw_barycenter(gw_ctx* ctx, const gw_barycenter_problem* prob, const int* n, const double* h,
                        const double* lambda, const double* const* d_ps, const double* d_p, void* d_C,
                        double* d_stats, void* stream);

/*
 * Serving: independent (fused) GW solves arriving over time (a deployment
 * mode of the same method; the paper has no counterpart).
 *
 * gw_server_create starts `max_slots` (1..64) worker threads on CUDA device
 * `device`, each with its own stream.  A free worker takes the oldest queued
 * request that fits in the unused part of the device-memory budget
 * `hbm_budget_bytes` (inputs, plan, statistics and solve workspace), so a
 * large request waiting for memory does not hold up smaller ones behind it;
 * once the oldest request has been passed over 32 times, nothing else is
 * admitted until it fits (no starvation).  A finished request frees its
 * memory and slot for the next one.  Up to max_slots requests run
 * concurrently.  Inputs are copied to the device from page-locked staging
 * buffers; the plan is copied into h_T as given (page-locked h_T copies
 * fastest).
 */
typedef struct gw_server gw_server;

gw_status gw_server_create(gw_server** server, int device, size_t hbm_budget_bytes, int max_slots);

/* Stops the workers after their running requests; queued requests end with
 * GW_ERR_SHUTDOWN.  Frees the server. */
void gw_server_destroy(gw_server* server);

/*
 * gw_submit - queues one solve (as gw_solve) and returns at once.
 *   prob                 validated as for gw_solve.
 *   h_u, h_v             host marginals (double, n and m); copied.
 *   h_phi, h_psi         host features (double, n x feat_dim, m x feat_dim)
 *                        when theta < 1, else may be NULL; copied.
 *   h_T                  NULL, or a host buffer of n*m reals (prob->dtype)
 *                        that receives the plan; it must stay valid until
 *                        gw_poll reports the request finished.
 *   *ticket              receives the request's ticket.
 * GW_ERR_INVALID for a bad descriptor or a request larger than the budget
 * (it could never run); GW_ERR_SHUTDOWN after gw_server_destroy began.
 */
gw_status gw_submit(gw_server* server, const gw_problem* prob, const double* h_u, const double* h_v,
                    const double* h_phi, const double* h_psi, void* h_T, uint64_t* ticket);

/*
 * gw_poll - GW_NOT_READY while the request is queued or running.  Once it
 * has finished: its status (GW_OK, or the error of its solve), the 8
 * statistics of gw_solve in stats (if not NULL) and the seconds from
 * gw_submit to completion in *latency_s (if not NULL).  A finished ticket
 * is reported once; afterwards (or for an unknown ticket) GW_ERR_INVALID.
 */
gw_status gw_poll(gw_server* server, uint64_t ticket, double* stats, double* latency_s);

/* Text of the last failed request ("" if none); valid until the calling
 * thread's next call of this function. */
const char* gw_server_last_error(gw_server* server);

/* Queued requests, requests completed so far, device bytes held by running
 * requests (any pointer may be NULL). */
gw_status gw_server_info(gw_server* server, long* queued, long* completed, size_t* bytes_in_use);

/*
 * Tuned row configurations (process-wide).
 *
 * Each pass of the Sinkhorn kernels splits a row of Pi over a row group of
 * 32*NW threads holding VPT values each (32*NW*VPT >= m), with NG row groups
 * per block.  The built-in choice depends on the row length m and the dtype.
 * A tuning table replaces it per row-length range: the sweep in
 * paper_2404_08970_gb300/tune.py times every candidate on the GPU, keeps
 * only candidates whose plan matches the built-in configuration's, and writes
 * the table.  The configuration sets the order of a row's reductions, so
 * every entry point (gw_solve, gw_solve_batch, the server) reads the same
 * table and gives the same results for it; change the table only while no
 * solve is running.  With no table the built-in choice is used.
 *
 * At the first gw_ctx_create of the process the library loads the table named
 * by the environment variable GW_TUNE_TABLE, or else tune_table.txt beside
 * the library if that file exists.  Format: one entry per line,
 *     <kernel> <dtype> <m_lo> <m_hi> <config>
 * with '#' starting a comment.  Later entries take precedence.
 */
typedef enum { GW_TUNE_SINKHORN = 0 } gw_tune_kernel;

/* Use configuration `config` for rows of m_lo <= m <= m_hi columns of dtype.
 * GW_ERR_INVALID for an unknown kernel, dtype or configuration, an empty
 * range, or a configuration that does not cover m_hi columns. */
gw_status gw_tune_set(int kernel, int dtype, int m_lo, int m_hi, int config);

/* Drops every table entry (the built-in choice applies again). */
gw_status gw_tune_clear(void);

/* Adds the entries of a table file (format above).  GW_ERR_INVALID if the
 * file cannot be read or a line is malformed or invalid; the entries read
 * before the bad line stay. */
gw_status gw_tune_load(const char* path);

/* The configuration in effect for rows of m columns (table entry, or the
 * built-in choice); -1 for an unknown kernel or dtype, or m outside
 * [1, 16384]. */
int gw_tune_config(int kernel, int dtype, int m);

/* The candidate configurations for rows of m columns: the built-in choice
 * first, then every other configuration that covers m columns but at most
 * four times the built-in choice's.  Writes at most `cap` of them to out (out
 * may be NULL when cap is 0) and returns how many there are; -1 for an
 * unknown kernel or dtype, or m outside [1, 16384]. */
int gw_tune_candidates(int kernel, int dtype, int m, int* out, int cap);

/* Shape of a configuration: warps per row group, values per thread, row
 * groups per block.  GW_ERR_INVALID for an unknown configuration. */
gw_status gw_tune_shape(int kernel, int config, int* nw, int* vpt, int* ng);

#ifdef __cplusplus
}
#endif

#endif /* GW_FGC_H */
