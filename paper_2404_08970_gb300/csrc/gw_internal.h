// Internal host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gw.h"

namespace gw {

// Device workspace of one context: a single growing allocation carved into
// regions by each call.  Calls on one context are ordered on their stream.
struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
};

struct Carve {
  char* p;
  size_t left;
  void* take(size_t n, size_t align = 256) {
    uintptr_t a = ((uintptr_t)p + align - 1) & ~(uintptr_t)(align - 1);
    size_t used = (size_t)(a - (uintptr_t)p) + n;
    if (used > left) return nullptr;
    p += used;
    left -= used;
    return (void*)a;
  }
};

// Optional per-kernel timing: when a context has profiling switched on, each
// launch site brackets its kernel with begin()/end(), which record CUDA
// events on the launch stream.
struct Tracer {
  virtual void begin(const char* name, cudaStream_t st) = 0;
  virtual void end(cudaStream_t st) = 0;
  virtual ~Tracer() {}
};

struct TraceScope {
  Tracer* t;
  cudaStream_t st;
  TraceScope(Tracer* tr, const char* name, cudaStream_t s) : t(tr), st(s) {
    if (t) t->begin(name, st);
  }
  ~TraceScope() {
    if (t) t->end(st);
  }
};

// Layout of the 1D row bands used by the structured gradient.
struct Bands {
  int B;  // number of bands
  int R;  // rows per band (the last band may be shorter)
};

Bands choose_bands(int n, int target);

struct Grad1DArgs {
  int n, m, k;
  int ky;               // exponent of Y's distance when it differs from k (0: same as k)
  double hx, hy;
  int dtype;            // GW_F32 or GW_F64
  const void* T;        // n x m row-major, dtype
  void* G;              // n x m row-major, dtype
  const double* u;      // target marginals (device) or nullptr with exact
  const double* v;
  int exact;            // 1: constant term from T's own marginals
  double out_scale;     // G := out_scale * (c_x + c_y - 2 D_X T D_Y)
  // With regen_F set (float, target marginals), T is not read: `T` points to
  // the cost Pi of the previous mirror-descent step and the kernels form the
  // plan T_ip = 2^(regen_F[i] + regen_G[p] - regen_c Pi_ip) as they load it
  // (the expression of the plan pass).  G may then be Pi itself: each row is
  // read before it is written.
  const float* regen_F;
  const float* regen_G;
  float regen_c;
  cudaStream_t stream;
  unsigned* status;     // device status word
  int num_sms;
  Tracer* tracer;       // nullable
  int force_generic;    // 1: use the block-scan row kernel even where the warp-specialised one applies
  // Optional: a second stream and two events, to run the constant terms
  // (target marginals) concurrently with the band passes.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// Host-side failure notes (per thread): the launch helpers record what
// failed before returning an error status, for the callers' messages.
void note_failure(const char* what);
const char* last_failure();

// Lets `func` use the device's largest opt-in dynamic shared memory.  Every
// caller sets the same value, so threads launching concurrently with
// different shared-memory sizes do not undo each other's setting.  Returns
// false if the attribute cannot be set or `need` exceeds the limit.
bool allow_dynamic_smem(const void* func, size_t need);

// Encodes a TMA tensor map over the rows of an n x m row-major array of
// elem_bytes-sized reals, viewed as [n][m / E][E] with E*elem_bytes = 128,
// 128-byte swizzle, box {E, box_cols, 1}, box_cols the largest divisor of
// m / E up to 256.  False if m is not a multiple of E or the driver rejects
// the map.
bool encode_rows_tmap(void* tmap, const void* base, int n, int m, int elem_bytes, int* box_cols);
bool encode_rows_tmap_box(void* tmap, const void* base, int n, int m, int elem_bytes, int box_cols);

// Bytes of workspace the structured 1D gradient needs.
size_t grad1d_workspace_bytes(int n, int m, int k, int dtype, int num_sms);
// Launches the structured 1D gradient.  Returns GW_OK or an error.
int grad1d_launch(const Grad1DArgs& a, void* ws, size_t ws_bytes);
// Whether the 1D gradient can form T from (Pi, F, G) as it loads it (the
// TMA-fed band-moment pass and the warp-specialised row kernel run).
bool grad1d_regen_supported(int n, int m, int k, int ky, int dtype, int force_generic);

// Per-exponent entry points (one translation unit each).
int grad1d_launch_k1(const Grad1DArgs& a, void* ws, size_t ws_bytes);
int grad1d_launch_k2(const Grad1DArgs& a, void* ws, size_t ws_bytes);
int grad1d_launch_k3(const Grad1DArgs& a, void* ws, size_t ws_bytes);
int grad1d_launch_mixed(const Grad1DArgs& a, void* ws, size_t ws_bytes);  // k != ky (1 and 2)

// c[i] = h^{2k} sum_j |i - j|^{2k} w_j for i < len (the constant term of the
// gradient), from a double vector w on the device.  part must hold
// marg_part_doubles(len, k) doubles.
size_t marg_part_doubles(int len, int k);
int marg_const_launch(const double* w, int len, int k, double h, void* out, int dtype,
                      double* part, cudaStream_t stream, Tracer* tracer = nullptr);
// Both constant terms in one pair of launches; part must hold
// marg_part_doubles(n, k) + marg_part_doubles(m, k) doubles.
int marg_const2_launch(const double* wx, int n, double fx, void* outx, const double* wy, int m, double fy,
                       void* outy, int k, int dtype, double* part, cudaStream_t stream, Tracer* tracer);

// Structured gradient on side x side grids with an axis-separable cost
// (grad2d.cu): Manhattan with k = 1, or squared Euclidean.
constexpr int kMax2DSide = 256;
// Mixed distance exponents (1D): supported pairs and row lengths.
inline bool mixed_k_supported(int k, int ky, int m, int dtype) {
  if (ky == 0 || ky == k) return true;
  if (!((k == 1 && ky == 2) || (k == 2 && ky == 1))) return false;
  return m <= (dtype == GW_F32 ? 8192 : 4096);
}
// Longest row a double-precision Sinkhorn pass holds in shared memory.
constexpr int kMaxSolveF64Y = 10240;
// Structured gradient on side^3 grids with an axis-separable cost
// (grad3d.cu): Manhattan with k = 1, or squared Euclidean.
constexpr int kMax3DSide = 32;
struct Grad2DArgs {
  int sx, sy;           // grid sides; n = sx^dim points of X, m = sy^dim points of Y
  int dim;              // 2 (side x side grids) or 3 (side^3 grids); 0 reads as 2
  int cost;             // GW_COST_POW (Manhattan^k) or GW_COST_SQEUCLID
  int k;                // exponent of the Manhattan distance (GW_COST_POW)
  double hx, hy;
  int dtype;
  const void* T;        // n x m row-major, dtype
  void* G;              // n x m row-major, dtype
  const double* u;      // target marginals (n and m) or nullptr with exact
  const double* v;
  int exact;
  double out_scale;
  cudaStream_t stream;
  unsigned* status;
  int num_sms;
  Tracer* tracer;
};
// Workspace of the 2D gradient for this cost and exponent (the separable
// costs, or Manhattan^k with k >= 2).
size_t grad2d_workspace_bytes(int sx, int sy, int dtype, int cost, int k);
int grad2d_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes);
size_t grad3d_workspace_bytes(int sx, int sy, int dtype);
int grad3d_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes);
// Workspace of the grid gradient of a problem with dim 2 or 3.
inline size_t grid_grad_workspace_bytes(int dim, int sx, int sy, int dtype, int cost, int k) {
  return dim == 3 ? grad3d_workspace_bytes(sx, sy, dtype) : grad2d_workspace_bytes(sx, sy, dtype, cost, k);
}
// Manhattan^k, k = 2, 3 (grad2d_powk.cu): supported grid sides and dtype.
bool grad2d_powk_supported(int sx, int sy, int k, int dtype);
size_t grad2d_powk_workspace_bytes(int sx, int sy, int k, int dtype);
int grad2d_powk_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes);

// Dense comparison gradient through cuBLAS (dense.cu).
struct DenseArgs {
  int dim, cost, sx, sy;  // dim 2, 3: sx, sy grid sides, n = sx^dim, m = sy^dim
  int n, m, k, prec, exact;
  int ky;                 // 1D: exponent of Y's distance (0: same as k)
  double hx, hy;
  const double *u, *v;
  const void* T;
  void* G;
  cudaStream_t stream;
  Tracer* tracer;
  unsigned* status;  // device status word (bounded waits of the tcgen05 kernels)
  int num_sms;
};
// C = A B^T on the tcgen05 tensor cores (dense_tc.cu).  A: M x K row-major
// (pitch lda elements), B: N x K row-major (pitch ldb), BF16 (tf32 = false)
// or FP32 read as TF32; pitches a multiple of 16 bytes, bases 16-byte
// aligned.  mode 0 stores C as bf16, 1 as float rounded to TF32, 2 stores
// fma(-scale, C, cx[row] + cy[col]) as float; out_rows x out_cols outputs
// are written (row pitch ldo).
int tc_gemm_abt_launch(bool tf32, const void* A, long long lda, const void* B, long long ldb, int M, int N, int K,
                       int mode, void* out, long long ldo, int out_rows, int out_cols, const float* cx,
                       const float* cy, float scale, unsigned* status, int num_sms, cudaStream_t st,
                       Tracer* tracer);
void* dense_state_create();
void dense_state_destroy(void* state);
size_t dense_workspace_bytes(int n, int m, int prec);
int dense_grad_launch(void* state, const DenseArgs& a, void* ws, size_t ws_bytes);

// Entropic (fused) GW by mirror descent (sinkhorn.cu).  dim 1: n = nx and
// m = ny points; dim 2, 3: nx, ny are grid sides (n = nx^dim, m = ny^dim).
struct SolveArgs {
  int dim, cost;
  int nx, ny;
  int n, m, k, dtype;
  double hx, hy, eps, theta;
  double tau;      // Sinkhorn regularisation of each step (= eps unless set)
  int warm_start;  // 1: Sinkhorn starts from the previous step's potentials
  double rho;      // > 0: entropic unbalanced GW with marginal relaxation rho
  int ky;          // 1D: exponent of Y's distance (0: same as k)
  int n_outer, n_inner, feat_dim;
  const double *u, *v, *phi, *psi;
  void* T;
  double *f, *g, *stats;
  cudaStream_t stream;
  unsigned* status;
  int num_sms;
  Tracer* tracer;
  int force_generic;
  int batch;  // 1: part of a batch (row bands of at least 32 rows)
  // Barycenter solves: X is a dense N x N distance matrix (Real, row-major)
  // instead of a grid; Y is the 1D grid of m points (hy, k).
  const void* dense_x;
};

// Gradient with a dense X side (barycenter.cu): G = out_scale ((C o C) u 1^T +
// 1 ((D o D) v)^T - 2 C T D) with C dense N x N and D the 1D grid distance
// of n points (hy, k = 1 or 2); T and G are N x n in dtype.
struct DenseXGradArgs {
  int N, n, k, dtype, exact;
  double hy, out_scale;
  const void* C;
  const void* T;
  void* G;
  const double *u, *v;
  cudaStream_t stream;
  Tracer* tracer;
};
size_t dense_x_workspace_bytes(int N, int n, int dtype);
int dense_x_grad_launch(const DenseXGradArgs& a, void* ws, size_t ws_bytes);

// Fixed-support GW barycenter of `count` 1D grid spaces (n[s] points, spacing
// h[s], exponent k, marginals ps[s]) with weights lambda, on N points with
// weights p; C (N x N, dtype) is the initial distance matrix and receives
// the result; values (8 doubles per input, nullable) the statistics of the
// last round's solves.
struct BarycenterArgs {
  int count, N, k, dtype;
  const int* n;
  const double* h;
  const double* lambda;
  const double* const* ps;
  const double* p;
  void* C;
  double* values;
  double eps;
  int n_iter, n_outer, n_inner;
  cudaStream_t stream;
  unsigned* status;
  int num_sms;
  Tracer* tracer;
};

size_t solve_workspace_bytes(const SolveArgs& a);
int solve_launch(const SolveArgs& a, void* ws, size_t ws_bytes);
// Batched solves: problems with equal solve_group_key, dtype and schedule
// (n_outer, n_inner) form a group that solve_group_launch advances in lock
// step on one stream (each Sinkhorn pass one launch per 32 problems).
int solve_group_key(const SolveArgs& a);
int solve_group_launch(const SolveArgs* const* a, void* const* ws, const size_t* ws_bytes, int count,
                       cudaStream_t stream);

// Mixed batches (sinkhorn.cu): problems of one dtype and schedule whose row
// configurations all run 512-thread blocks share every Sinkhorn launch.  The
// host image of the problems' device table (solve_mixed_table_bytes bytes)
// is written by solve_mixed_table and must be on the device before
// solve_mixed_launch enqueues the solves: per-problem work on the worker
// streams, the shared Sinkhorn passes on `main` (fork/join by the events).
bool solve_mixable(const SolveArgs& A);
size_t solve_mixed_table_bytes(int count, int dtype);
int solve_mixed_table(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count, void* host);
int solve_mixed_launch(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count,
                       const void* dev_table, cudaStream_t main, const cudaStream_t* workers, int nworkers,
                       cudaEvent_t fork, const cudaEvent_t* join);

size_t barycenter_workspace_bytes(const BarycenterArgs& a);
int barycenter_launch(const BarycenterArgs& a, void* ws, size_t ws_bytes);
SolveArgs barycenter_solve_args(const BarycenterArgs& a, int s, const void* C, void* T, double* stats);

// Sinkhorn row configurations (sinkhorn.cu): the built-in choice for m
// columns, the shape of a configuration id, and every id (count returned, at
// most cap written).
int sk_default_config(int m, int dtype);
bool sk_config_shape(int id, int* dtype, int* nw, int* vpt, int* ng);
int sk_config_ids(int* out, int cap);

// Tuning table (tune.cu): the entry for m columns (-1 if none), a counter
// that changes whenever the table does (part of every cached graph's key),
// and the one-time load at the first context creation.
int tune_lookup(int kernel, int dtype, int m);
unsigned tune_generation();
void tune_autoload();

}  // namespace gw
