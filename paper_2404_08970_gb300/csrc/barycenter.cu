// Fixed-support GW barycenter of spaces on 1D grids.  The conclusion names
// the barycenter among the GW variants the fast gradient accelerates; the
// iteration is the cited barycenter method's block coordinate descent with
// the square loss:
//   (i)  for each input s, an entropic GW solve between the barycenter
//        (C, p), a dense N x N distance matrix, and the grid space (D_s, p_s)
//        by the library's mirror descent, whose gradient
//          G = (C o C) p 1^T + 1 ((D_s o D_s) p_s)^T - 2 C T D_s
//        keeps the grid structure on its Y side: Z = T D_s is the paper's
//        O(N n) transform along each row of T, and only C Z is a dense
//        product;
//   (ii) C = sum_s lambda_s T_s D_s T_s^T / ((sum_s lambda_s) p p^T), again
//        with T_s D_s by the row transform.
// The dense products accumulate in double for both data types (the GW value
// cancels against the constant terms), with FP64 row transforms.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gw_common.cuh"
#include "gw_internal.h"

namespace gw {
namespace {

// ---------------------------------------------------------------------------
// Z[i][p] = h^k sum_q |p - q|^k T[i][q], k = 1 or 2, one block of 256 threads
// per row, double arithmetic.  k = 2 needs only the row's moments
// (|p - q|^2 = (p - q)^2); k = 1 splits at p with inclusive prefix sums
//   A_p = sum_{q <= p} T_q, B_p = sum_{q <= p} q T_q:
//   z_p = 2 p A_p - 2 B_p + B_n - p A_n.
// Each thread takes a contiguous chunk of the row; chunk sums are scanned in
// shared memory.
// ---------------------------------------------------------------------------
constexpr int kRtThreads = 256;

template <typename Real>
__global__ void __launch_bounds__(kRtThreads) bary_row_transform(const Real* __restrict__ T, int N, int n, int k,
                                                                 double hk, Real* __restrict__ Z) {
  __shared__ double sa[kRtThreads], sb[kRtThreads], sc[kRtThreads];
  const int i = blockIdx.x;
  if (i >= N) return;
  const Real* row = T + (size_t)i * n;
  Real* out = Z + (size_t)i * n;
  const int tid = threadIdx.x;
  const int per = (n + kRtThreads - 1) / kRtThreads;
  const int q0 = min(n, tid * per), q1 = min(n, q0 + per);
  double a = 0.0, b = 0.0, c = 0.0;
  for (int q = q0; q < q1; ++q) {
    const double x = (double)row[q];
    a += x;
    b += (double)q * x;
    c += (double)q * (double)q * x;
  }
  sa[tid] = a;
  sb[tid] = b;
  sc[tid] = c;
  __syncthreads();
  // Inclusive scan of the chunk sums (Hillis-Steele, double).
  for (int d = 1; d < kRtThreads; d <<= 1) {
    const double xa = tid >= d ? sa[tid - d] : 0.0;
    const double xb = tid >= d ? sb[tid - d] : 0.0;
    __syncthreads();
    sa[tid] += xa;
    sb[tid] += xb;
    __syncthreads();
  }
  const double An = sa[kRtThreads - 1], Bn = sb[kRtThreads - 1];
  if (k == 2) {
    // Totals of q^2 T: a block sum of sc.
    __syncthreads();
    for (int d = kRtThreads / 2; d > 0; d >>= 1) {
      if (tid < d) sc[tid] += sc[tid + d];
      __syncthreads();
    }
    const double Cn = sc[0];
    for (int p = q0; p < q1; ++p) {
      const double pp = (double)p;
      out[p] = (Real)(hk * (pp * pp * An - 2.0 * pp * Bn + Cn));
    }
    return;
  }
  double Ap = tid > 0 ? sa[tid - 1] : 0.0, Bp = tid > 0 ? sb[tid - 1] : 0.0;
  for (int p = q0; p < q1; ++p) {
    const double x = (double)row[p];
    const double pp = (double)p;
    Ap += x;
    Bp += pp * x;
    out[p] = (Real)(hk * (2.0 * pp * Ap - 2.0 * Bp + Bn - pp * An));
  }
}

// ---------------------------------------------------------------------------
// Dense products with double accumulation, 64 x 64 output tiles, 256 threads
// (4 x 4 outputs each), K in steps of 16 through shared memory.
//   NN: acc = A (M x K) B (K x Nc);   NT: acc = A (M x K) B^T, B (Nc x K).
//   EPI 0: out (double) += alpha acc;
//   EPI 1: out (Real) = scale (cx[i] + cy[j] - 2 acc).
// ---------------------------------------------------------------------------
constexpr int kGT = 64, kGK = 16;

template <typename Real, bool NT, int EPI>
__global__ void __launch_bounds__(256) bary_gemm(const Real* __restrict__ A, const Real* __restrict__ B, int M,
                                                 int Nc, int K, double alpha, const double* __restrict__ cx,
                                                 const double* __restrict__ cy, double scale, void* out) {
  __shared__ double As[kGK][kGT + 1];
  __shared__ double Bs[kGK][kGT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += kGK) {
    // A tile: rows i0.., columns k0..  (64 x 16), B tile: (16 x 64).
    for (int e = threadIdx.x; e < kGT * kGK; e += 256) {
      const int r = e / kGK, kk = e % kGK;
      const int gi = i0 + r, gk = k0 + kk;
      As[kk][r] = (gi < M && gk < K) ? (double)A[(size_t)gi * K + gk] : 0.0;
    }
    for (int e = threadIdx.x; e < kGT * kGK; e += 256) {
      int kk, cidx;
      if (NT) {
        cidx = e / kGK;
        kk = e % kGK;
      } else {
        kk = e / kGT;
        cidx = e % kGT;
      }
      const int gj = j0 + cidx, gk = k0 + kk;
      double v = 0.0;
      if (gj < Nc && gk < K) v = NT ? (double)B[(size_t)gj * K + gk] : (double)B[(size_t)gk * Nc + gj];
      Bs[kk][cidx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= Nc) continue;
      const size_t o = (size_t)gi * Nc + gj;
      if constexpr (EPI == 0) {
        double* D = reinterpret_cast<double*>(out);
        D[o] += alpha * acc[a][b];
      } else {
        Real* D = reinterpret_cast<Real*>(out);
        D[o] = (Real)(scale * (cx[gi] + cy[gj] - 2.0 * acc[a][b]));
      }
    }
  }
}

// cx[i] = sum_j C_ij^2 w_j (one block per row, double).
template <typename Real>
__global__ void __launch_bounds__(256) bary_const_x(const Real* __restrict__ C, const double* __restrict__ w, int N,
                                                    double* __restrict__ cx) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < N; j += 256) {
    const double c = (double)C[(size_t)i * N + j];
    s += c * c * w[j];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) cx[i] = red[0];
}

// Moments mom[r] = sum_q q^r w_q, r = 0 .. 2k (one block, double).
__global__ void __launch_bounds__(256) bary_moments(const double* __restrict__ w, int n, int k2,
                                                    double* __restrict__ mom) {
  __shared__ double red[256];
  for (int r = 0; r <= k2; ++r) {
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 256) {
      double t = w[q];
      for (int e = 0; e < r; ++e) t *= (double)q;
      s += t;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
      if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
      __syncthreads();
    }
    if (threadIdx.x == 0) mom[r] = red[0];
    __syncthreads();
  }
}

// cy[p] = h^{2k} sum_q (p - q)^{2k} w_q = h^{2k} sum_r C(2k, r) p^{2k-r} (-1)^r mom[r].
__global__ void bary_const_y(const double* __restrict__ mom, int n, int k2, double h2k, double* __restrict__ cy) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double s = 0.0;
  for (int r = 0; r <= k2; ++r) {
    double t = (double)binom(k2, r) * mom[r];
    for (int e = 0; e < k2 - r; ++e) t *= (double)p;
    s += (r & 1) ? -t : t;
  }
  cy[p] = h2k * s;
}

// Row sums r_i = sum_p T_ip (one warp per row) and column sums c_p = sum_i T_ip.
template <typename Real>
__global__ void bary_row_sums(const Real* __restrict__ T, int N, int n, double* __restrict__ r) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= N) return;
  double s = 0.0;
  for (int p = threadIdx.x & 31; p < n; p += 32) s += (double)T[(size_t)i * n + p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) r[i] = s;
}
template <typename Real>
__global__ void bary_col_sums(const Real* __restrict__ T, int N, int n, double* __restrict__ c) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += (double)T[(size_t)i * n + p];
  c[p] = s;
}

// C = B / (wsum p p^T) in the data type.
template <typename Real>
__global__ void bary_finish(const double* __restrict__ B, const double* __restrict__ p, int N, double wsum,
                            Real* __restrict__ C) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)N * N) return;
  const int i = (int)(e / N), j = (int)(e % N);
  C[e] = (Real)(B[e] / (wsum * p[i] * p[j]));
}

__global__ void fill_zero_d(double* x, size_t len) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    x[e] = 0.0;
}

struct DxLayout {
  size_t Z, cx, cy, mom, r, c, total;
};
DxLayout dx_layout(int N, int n, size_t rb) {
  DxLayout L{};
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = (off + b + 255) / 256 * 256;
    return o;
  };
  L.Z = take((size_t)N * n * rb);
  L.cx = take((size_t)N * 8);
  L.cy = take((size_t)n * 8);
  L.mom = take(16 * 8);
  L.r = take((size_t)N * 8);
  L.c = take((size_t)n * 8);
  L.total = off;
  return L;
}

template <typename Real>
int dense_x_typed(const DenseXGradArgs& g, void* wsv, size_t ws_bytes) {
  const DxLayout L = dx_layout(g.N, g.n, sizeof(Real));
  if (L.total > ws_bytes) return GW_ERR_OOM;
  char* ws = (char*)wsv;
  cudaStream_t st = g.stream;
  const Real* T = (const Real*)g.T;
  Real* Z = (Real*)(ws + L.Z);
  double* cx = (double*)(ws + L.cx);
  double* cy = (double*)(ws + L.cy);
  double* mom = (double*)(ws + L.mom);
  const double* wx = g.u;
  const double* wy = g.v;
  TraceScope ts(g.tracer, "bary_grad", st);
  if (g.exact) {
    bary_row_sums<Real><<<(g.N + 7) / 8, 256, 0, st>>>(T, g.N, g.n, (double*)(ws + L.r));
    bary_col_sums<Real><<<(g.n + 255) / 256, 256, 0, st>>>(T, g.N, g.n, (double*)(ws + L.c));
    wx = (const double*)(ws + L.r);
    wy = (const double*)(ws + L.c);
  }
  bary_const_x<Real><<<g.N, 256, 0, st>>>((const Real*)g.C, wx, g.N, cx);
  bary_moments<<<1, 256, 0, st>>>(wy, g.n, 2 * g.k, mom);
  bary_const_y<<<(g.n + 255) / 256, 256, 0, st>>>(mom, g.n, 2 * g.k, std::pow(g.hy, 2 * g.k), cy);
  bary_row_transform<Real><<<g.N, kRtThreads, 0, st>>>(T, g.N, g.n, g.k, std::pow(g.hy, g.k), Z);
  const dim3 grid((g.n + kGT - 1) / kGT, (g.N + kGT - 1) / kGT);
  bary_gemm<Real, false, 1><<<grid, 256, 0, st>>>((const Real*)g.C, Z, g.N, g.n, g.N, 1.0, cx, cy, g.out_scale,
                                                  g.G);
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

}  // namespace

size_t dense_x_workspace_bytes(int N, int n, int dtype) {
  return dx_layout(N, n, dtype == GW_F32 ? 4 : 8).total + 4096;
}

int dense_x_grad_launch(const DenseXGradArgs& a, void* ws, size_t ws_bytes) {
  if (a.N < 1 || a.n < 1 || a.k < 1 || a.k > 2) return GW_ERR_INVALID;
  if (a.dtype == GW_F32) return dense_x_typed<float>(a, ws, ws_bytes);
  return dense_x_typed<double>(a, ws, ws_bytes);
}

// ---------------------------------------------------------------------------
// The barycenter iteration (host side): per round, one mirror-descent solve
// against each input (plan in the workspace), then the update of C.
// Workspace: B (N x N double) | per input: solve workspace, plan T_s (N x n_s)
// | Z (N x max n_s, Real).
// ---------------------------------------------------------------------------
size_t barycenter_workspace_bytes(const BarycenterArgs& a) {
  const size_t rb = a.dtype == GW_F32 ? 4 : 8;
  size_t b = ((size_t)a.N * a.N * 8 + 255) / 256 * 256;
  int nmax = 1;
  for (int s = 0; s < a.count; ++s) {
    // Sized for the solves' dense-X gradient (a.C marks the dense side).
    SolveArgs sa = barycenter_solve_args(a, s, a.C, nullptr, nullptr);
    b += (solve_workspace_bytes(sa) + 255) / 256 * 256;
    b += ((size_t)a.N * a.n[s] * rb + 255) / 256 * 256;
    nmax = std::max(nmax, a.n[s]);
  }
  b += ((size_t)a.N * nmax * rb + 255) / 256 * 256;
  return b + 4096;
}

SolveArgs barycenter_solve_args(const BarycenterArgs& a, int s, const void* C, void* T, double* stats) {
  SolveArgs sa{};
  sa.dim = 1;
  sa.cost = GW_COST_POW;
  sa.nx = a.N;
  sa.ny = a.n[s];
  sa.n = a.N;
  sa.m = a.n[s];
  sa.k = a.k;
  sa.ky = 0;
  sa.dtype = a.dtype;
  sa.hx = 1.0;
  sa.hy = a.h[s];
  sa.eps = a.eps;
  sa.tau = a.eps;
  sa.theta = 1.0;
  sa.n_outer = a.n_outer;
  sa.n_inner = a.n_inner;
  sa.u = a.p;
  sa.v = a.ps[s];
  sa.T = T;
  sa.stats = stats;
  sa.dense_x = C;
  sa.stream = a.stream;
  sa.status = a.status;
  sa.num_sms = a.num_sms;
  sa.tracer = a.tracer;
  return sa;
}

namespace {
template <typename Real>
int barycenter_typed(const BarycenterArgs& a, void* wsv, size_t ws_bytes) {
  if (barycenter_workspace_bytes(a) > ws_bytes) return GW_ERR_OOM;
  char* ws = (char*)wsv;
  size_t off = 0;
  auto take = [&](size_t b) {
    char* p = ws + off;
    off = (off + b + 255) / 256 * 256;
    return p;
  };
  cudaStream_t st = a.stream;
  const size_t NN = (size_t)a.N * a.N;
  double* B = (double*)take(NN * 8);
  std::vector<char*> sws(a.count), Ts(a.count);
  std::vector<size_t> swb(a.count);
  int nmax = 1;
  for (int s = 0; s < a.count; ++s) {
    SolveArgs sa = barycenter_solve_args(a, s, a.C, nullptr, nullptr);
    swb[s] = solve_workspace_bytes(sa);
    sws[s] = take(swb[s]);
    Ts[s] = take((size_t)a.N * a.n[s] * sizeof(Real));
    nmax = std::max(nmax, a.n[s]);
  }
  Real* Z = (Real*)take((size_t)a.N * nmax * sizeof(Real));
  double wsum = 0.0;
  for (int s = 0; s < a.count; ++s) wsum += a.lambda[s];
  for (int it = 0; it < a.n_iter; ++it) {
    const bool last = it + 1 == a.n_iter;
    for (int s = 0; s < a.count; ++s) {
      SolveArgs sa = barycenter_solve_args(a, s, a.C, Ts[s], last && a.values ? a.values + 8 * s : nullptr);
      const int rc = solve_launch(sa, sws[s], swb[s]);
      if (rc != GW_OK) return rc;
    }
    TraceScope ts(a.tracer, "bary_update", st);
    fill_zero_d<<<4 * a.num_sms, 256, 0, st>>>(B, NN);
    for (int s = 0; s < a.count; ++s) {
      bary_row_transform<Real><<<a.N, kRtThreads, 0, st>>>((const Real*)Ts[s], a.N, a.n[s], a.k,
                                                           std::pow(a.h[s], a.k), Z);
      const dim3 grid((a.N + kGT - 1) / kGT, (a.N + kGT - 1) / kGT);
      bary_gemm<Real, true, 0><<<grid, 256, 0, st>>>(Z, (const Real*)Ts[s], a.N, a.N, a.n[s], a.lambda[s], nullptr,
                                                    nullptr, 0.0, B);
    }
    bary_finish<Real><<<(unsigned)((NN + 255) / 256), 256, 0, st>>>(B, a.p, a.N, wsum, (Real*)a.C);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}
}  // namespace

int barycenter_launch(const BarycenterArgs& a, void* ws, size_t ws_bytes) {
  if (a.count < 1 || a.N < 1 || a.k < 1 || a.k > 2) return GW_ERR_INVALID;
  if (a.dtype == GW_F32) return barycenter_typed<float>(a, ws, ws_bytes);
  return barycenter_typed<double>(a, ws, ws_bytes);
}

}  // namespace gw
