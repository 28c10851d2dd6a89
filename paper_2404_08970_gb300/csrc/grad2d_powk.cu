// Structured 2D gradient for the Manhattan distance to a power k >= 2 (Sec.
// 3.1, eqs. "2d Dx", "2d gradient", "2D kronecker").
//
// On a side x side grid (point (a, b) at index a * side + b) the distance
// matrix is h^k D-hat with D-hat = (|a-a'| + |b-b'|)^k, which expands as
//     D-hat = sum_s C(k, s) A_{k-s} (x) A_s,   A_j = |i - j|^j,  A_0 = J.
// For k >= 2 the middle terms (0 < s < k) do not reduce to partial sums of T,
// so D_X T D_Y is formed in two passes, each applying D-hat to images:
//   pass 1 (g2k_images<.., 0>): row i of T is an sy x sy image Y; it becomes
//       W_i = sum_s C(k, s) A_{k-s} Y A_s  (A_{k-s} along the image's first
//       axis, A_s along its second), written as row i of W (n x m);
//   pass 2 (g2k_images<.., 1>): column p of W is an sx x sx image; the same
//       transform gives column p of D-hat_X T D-hat_Y, and the epilogue writes
//       G = c_x 1^T + 1 c_y^T - 2 h_X^k h_Y^k Z.
// In one image transform the two end terms are rank-one: s = 0 gives
// A_k (Y 1) along the first axis, s = k gives (1^T Y) A_k along the second;
// only the k - 1 middle terms transform the whole image, first along the
// second axis (R_s = Y A_s), then along the first.  Every line transform is
// the paper's recursion run forward and backward over the states
// F_s(i) = sum_{j<i} (i - j)^s x_j, s = 0..order (Sec. 3, eqs. "1d y" and
// "1d recursive relation"); all terms are non-negative, so plain float
// arithmetic loses no digits to cancellation.
//
// Memory traffic: read T, write W, read W, write G (16 bytes per element in
// float).  Pass 2 reads and writes tiles of P consecutive columns (P * 4
// bytes per row), holding P column images in shared memory.
//
// The constant terms c = h^{2k} (|da| + |db|)^{2k} w are two separable sums
// in double: M_r[a', b] = sum_b' |b - b'|^r w[a', b'] for r = 0..2k, then
// c[a, b] = sum_r C(2k, r) sum_a' |a - a'|^{2k-r} M_r[a', b].
#include <algorithm>
#include <cmath>

#include "gw_common.cuh"
#include "gw_internal.h"

namespace gw {

namespace {

// Shared-memory budget of one image-transform block (leaves room for the
// runtime's reservation within the 227 KB per-block limit).
constexpr size_t kPowKSmemLimit = 200 * 1024;
constexpr int kMaxPow = 2 * 3;     // highest exponent of the constant terms (2k, k <= 3)
constexpr int kMaxConstSide = 128;

__host__ __device__ constexpr int binom_c(int n, int r) {
  int b = 1;
  for (int i = 1; i <= r; ++i) b = b * (n - r + i) / i;
  return b;
}

// Image layout in shared memory: row pitch L + 1 (conflict-free line walks in
// both directions), image stride L (L + 1) + 1.
__host__ __device__ inline int img_stride(int L) { return L * (L + 1) + 1; }

// One line of length L read at x[j * step]: forward and backward recursions
// with states of orders 0..Q, adding w * (A_Q x)(i) to out[i * ostep] (set
// instead of add when `first`).
template <int Q, typename Real>
__device__ __forceinline__ void line_pow(const Real* x, int step, int L, Real* out, int ostep, Real w, bool first) {
  Real S[Q + 1];
#pragma unroll
  for (int s = 0; s <= Q; ++s) S[s] = 0;
#pragma unroll 4
  for (int i = 0; i < L; ++i) {
    const Real xi = x[i * step];
    Real* o = out + i * ostep;
    *o = first ? w * S[Q] : fma(w, S[Q], *o);
#pragma unroll
    for (int s = Q; s >= 0; --s) {
      Real acc = S[s] + xi;
#pragma unroll
      for (int u = 0; u < s; ++u) acc = fma((Real)binom_c(s, u), S[u], acc);
      S[s] = acc;
    }
  }
#pragma unroll
  for (int s = 0; s <= Q; ++s) S[s] = 0;
#pragma unroll 4
  for (int i = L - 1; i >= 0; --i) {
    const Real xi = x[i * step];
    Real* o = out + i * ostep;
    *o = fma(w, S[Q], *o);
#pragma unroll
    for (int s = Q; s >= 0; --s) {
      Real acc = S[s] + xi;
#pragma unroll
      for (int u = 0; u < s; ++u) acc = fma((Real)binom_c(s, u), S[u], acc);
      S[s] = acc;
    }
  }
}

// R_s = A_s x along one line for s = 1..Q (each written to R[s-1]), and the
// line's sum: the same recursion, all orders at once.
template <int Q, typename Real>
__device__ __forceinline__ Real line_orders(const Real* x, int step, int L, Real* const* R, int ostep) {
  Real S[Q + 1];
#pragma unroll
  for (int s = 0; s <= Q; ++s) S[s] = 0;
#pragma unroll 4
  for (int i = 0; i < L; ++i) {
    const Real xi = x[i * step];
#pragma unroll
    for (int s = 1; s <= Q; ++s) R[s - 1][i * ostep] = S[s];
#pragma unroll
    for (int s = Q; s >= 0; --s) {
      Real acc = S[s] + xi;
#pragma unroll
      for (int u = 0; u < s; ++u) acc = fma((Real)binom_c(s, u), S[u], acc);
      S[s] = acc;
    }
  }
  const Real total = S[0];
#pragma unroll
  for (int s = 0; s <= Q; ++s) S[s] = 0;
#pragma unroll 4
  for (int i = L - 1; i >= 0; --i) {
    const Real xi = x[i * step];
#pragma unroll
    for (int s = 1; s <= Q; ++s) R[s - 1][i * ostep] += S[s];
#pragma unroll
    for (int s = Q; s >= 0; --s) {
      Real acc = S[s] + xi;
#pragma unroll
      for (int u = 0; u < s; ++u) acc = fma((Real)binom_c(s, u), S[u], acc);
      S[s] = acc;
    }
  }
  return total;
}

struct PowKIO {
  const void* in;        // pass 1: T; pass 2: W
  void* out;             // pass 1: W; pass 2: G
  int n, m;              // points of X and Y
  int L;                 // image side: sy (pass 1) or sx (pass 2)
  int P;                 // images per CTA iteration (pass 1: 1)
  double* rowsum;        // pass 1, exact marginals: T 1 (double) or nullptr
  const void* cxh;       // pass 2: constant terms, high and low parts (Real;
  const void* cxl;       // the low parts are zero for double)
  const void* cyh;
  const void* cyl;
  double scale;          // pass 2: 2 h_X^k h_Y^k
};

// i / L for 0 <= i < 2^20 and 1 <= L <= 256 without an integer division:
// (i + 1/2) / L is at least 1/(2L) away from an integer, far more than the
// float product's rounding error.
__device__ __forceinline__ int div_small(int i, float invL) { return __float2int_rz(((float)i + 0.5f) * invL); }

// MODE 0: pass 1 over rows of T; MODE 1: pass 2 over column tiles of W.
template <int K, typename Real, int MODE>
__global__ void __launch_bounds__(512) g2k_images(PowKIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);
  const int L = io.L, P = io.P;
  const int IS = img_stride(L);
  const int PL = P * L;
  Real* Y = sm;                              // images; later the middle-term sums
  Real* Rb = Y + (size_t)P * IS;             // K - 1 buffers of R_s, s = 1..K-1
  Real* rs = Rb + (size_t)(K - 1) * P * IS;  // [P][L] sums over the second axis
  Real* cs = rs + PL;                        // [P][L] sums over the first axis
  Real* e0 = cs + PL;                        // [P][L] A_K rs
  Real* ek = e0 + PL;                        // [P][L] A_K cs
  const int tid = threadIdx.x, NT = blockDim.x;
  const int img_elems = L * L;
  const float invL = 1.0f / (float)L;
  const int lp = P == 1 ? 0 : (P == 2 ? 1 : (P == 4 ? 2 : 3));  // P is a power of two
  const int units = MODE == 0 ? io.n : (io.m + P - 1) / P;

  for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
    const int p0 = MODE == 0 ? 0 : unit * P;
    // ---- load the P images
    if (MODE == 0) {
      const Real* src = reinterpret_cast<const Real*>(io.in) + (size_t)unit * io.m;
      for (int e = tid; e < img_elems; e += NT) Y[e + div_small(e, invL)] = src[e];
    } else {
      const Real* src = reinterpret_cast<const Real*>(io.in);
      for (int e = tid; e < P * img_elems; e += NT) {
        const int q = e & (P - 1), i = e >> lp;
        const int p = p0 + q;
        Y[q * IS + i + div_small(i, invL)] = p < io.m ? src[(size_t)i * io.m + p] : (Real)0;
      }
    }
    __syncthreads();
    // ---- lines along the second axis (R_s, row sums), column sums
    if (tid < PL) {
      const int q = tid / L, c = tid % L;
      const Real* x = Y + (size_t)q * IS + c * (L + 1);
      Real* Rp[K - 1];
#pragma unroll
      for (int s = 0; s < K - 1; ++s) Rp[s] = Rb + (size_t)s * P * IS + (size_t)q * IS + c * (L + 1);
      rs[tid] = line_orders<K - 1, Real>(x, 1, L, Rp, 1);
    } else if (tid < 2 * PL) {
      const int t = tid - PL;
      const int q = t / L, d = t % L;
      const Real* x = Y + (size_t)q * IS + d;
      Real acc = 0;
      for (int c = 0; c < L; ++c) acc += x[c * (L + 1)];
      cs[t] = acc;
    }
    __syncthreads();
    // ---- lines along the first axis: middle terms into Y; the end vectors
    if (tid < PL) {
      const int q = tid / L, d = tid % L;
      Real* o = Y + (size_t)q * IS + d;
      bool first = true;
#pragma unroll
      for (int s = 1; s < K; ++s) {
        const Real* x = Rb + (size_t)(s - 1) * P * IS + (size_t)q * IS + d;
        const Real w = (Real)binom_c(K, s);
        if (K - s == 1) line_pow<1, Real>(x, L + 1, L, o, L + 1, w, first);
        else if (K - s == 2) line_pow<2, Real>(x, L + 1, L, o, L + 1, w, first);
        else line_pow<3, Real>(x, L + 1, L, o, L + 1, w, first);
        first = false;
      }
    } else if (tid < PL + 2 * P) {
      const int t = tid - PL;
      const int q = t >> 1;
      if (t & 1) line_pow<K, Real>(cs + q * L, 1, L, ek + q * L, 1, (Real)1, true);
      else line_pow<K, Real>(rs + q * L, 1, L, e0 + q * L, 1, (Real)1, true);
    }
    __syncthreads();
    // ---- write
    if (MODE == 0) {
      Real* dst = reinterpret_cast<Real*>(io.out) + (size_t)unit * io.m;
      for (int e = tid; e < img_elems; e += NT) {
        const int c = div_small(e, invL), d = e - c * L;
        dst[e] = Y[e + c] + e0[c] + ek[d];
      }
      if (io.rowsum && tid == 0) {
        double r = 0.0;
        for (int c = 0; c < L; ++c) r += (double)rs[c];
        io.rowsum[unit] = r;
      }
    } else {
      Real* dst = reinterpret_cast<Real*>(io.out);
      const Real s = (Real)io.scale;
      const Real* cxh = reinterpret_cast<const Real*>(io.cxh);
      const Real* cxl = reinterpret_cast<const Real*>(io.cxl);
      const Real* cyh = reinterpret_cast<const Real*>(io.cyh);
      const Real* cyl = reinterpret_cast<const Real*>(io.cyl);
      for (int e = tid; e < P * img_elems; e += NT) {
        const int q = e & (P - 1), i = e >> lp;
        const int p = p0 + q;
        if (p >= io.m) continue;
        const int a = div_small(i, invL), b = i - a * L;
        const Real z = Y[q * IS + i + a] + e0[q * L + a] + ek[q * L + b];
        dst[(size_t)i * io.m + p] = fma(-s, z, cxh[i] + cyh[p]) + (cxl[i] + cyl[p]);
      }
    }
    __syncthreads();
  }
}

// Column sums of T in double (exact marginals): one thread per column, rows
// split over blockIdx.y, partial sums added atomically.
template <typename Real>
__global__ void g2k_colsum(const Real* __restrict__ T, int n, int m, int rows_per, double* __restrict__ c) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const int i0 = blockIdx.y * rows_per, i1 = min(n, i0 + rows_per);
  double acc = 0.0;
  for (int i = i0; i < i1; ++i) acc += (double)T[(size_t)i * m + p];
  atomicAdd(&c[p], acc);
}

// Constant term, stage 1: M[r][a'][b] = sum_b' |b - b'|^r w[a' L + b'],
// r = 0..2K.  One thread per output; the two marginals side by side.
struct ConstJob {
  const double* w;
  int L;
  double* M;    // [2K + 1][L][L]
  void* hi;     // [L * L] constant term, rounded to the compute type,
  void* lo;     // and the rounding remainder (zero for double)
  double factor;
  int pad, pad2;  // first job's thread range, rounded to whole blocks (stage 1, stage 2)
};
// Powers d^r, d = 0..L-1, r = 0..P2, in shared memory (exact in double).
__device__ __forceinline__ void fill_pow_table(double* tab, int L, int P2) {
  for (int t = threadIdx.x; t < L * (P2 + 1); t += blockDim.x) {
    const int r = t / L, d = t % L;
    double x = 1.0;
    for (int i = 0; i < r; ++i) x *= (double)d;
    tab[t] = x;
  }
  __syncthreads();
}
__global__ void g2k_const1(ConstJob X, ConstJob Yj, int P2) {
  __shared__ double tab[(kMaxPow + 1) * kMaxConstSide];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nx = (P2 + 1) * X.L * X.L;
  // A block never straddles the two jobs (the first job's range is padded
  // to whole blocks by the launcher).
  const bool isx = (int)(blockIdx.x * blockDim.x) < X.pad;
  const ConstJob& J = isx ? X : Yj;
  const int L = J.L;
  fill_pow_table(tab, L, P2);
  const int t = isx ? idx : idx - X.pad;
  if (t >= (P2 + 1) * L * L || (isx && idx >= nx)) return;
  const int r = t / (L * L), a = (t / L) % L, b = t % L;
  const double* pw = tab + r * L;
  const double* w = J.w + a * L;
  double acc = 0.0;
  for (int bp = 0; bp < L; ++bp) acc = fma(pw[abs(b - bp)], w[bp], acc);
  J.M[t] = acc;
}
// Stage 2: c[a L + b] = factor sum_r C(2K, r) sum_a' |a - a'|^{2K - r} M[r][a'][b].
template <typename Real>
__global__ void g2k_const2(ConstJob X, ConstJob Yj, int P2) {
  __shared__ double tab[(kMaxPow + 1) * kMaxConstSide];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool isx = (int)(blockIdx.x * blockDim.x) < X.pad2;
  const ConstJob& J = isx ? X : Yj;
  const int L = J.L;
  fill_pow_table(tab, L, P2);
  const int t = isx ? idx : idx - X.pad2;
  if (t >= L * L) return;
  const int a = t / L, b = t % L;
  double acc = 0.0;
  for (int r = 0; r <= P2; ++r) {
    const double* pw = tab + (P2 - r) * L;
    const double* M = J.M + (size_t)r * L * L + b;
    double inner = 0.0;
    for (int ap = 0; ap < L; ++ap) inner = fma(pw[abs(a - ap)], M[(size_t)ap * L], inner);
    acc = fma((double)binom_c(P2, r), inner, acc);
  }
  const double c = J.factor * acc;
  const Real h = (Real)c;
  reinterpret_cast<Real*>(J.hi)[t] = h;
  reinterpret_cast<Real*>(J.lo)[t] = (Real)(c - (double)h);
}

size_t images_smem(int K, int L, int P, size_t rb) {
  return ((size_t)K * P * img_stride(L) + 4 * (size_t)P * L) * rb;
}

// Column-tile width of pass 2: the widest of 8, 4, 2, 1 whose images leave
// room for two blocks per SM, else the widest that fits at all.
int pass2_tile(int K, int L, size_t rb) {
  for (int P : {8, 4, 2, 1})
    if (images_smem(K, L, P, rb) <= kPowKSmemLimit / 2 && 2 * P * L <= 512) return P;
  for (int P : {8, 4, 2, 1})
    if (images_smem(K, L, P, rb) <= kPowKSmemLimit && 2 * P * L <= 512) return P;
  return 0;
}

struct PowKLayout {
  size_t W, cxh, cxl, cyh, cyl, rowsum, colsum, Mx, My, total;
};

PowKLayout powk_layout(int sx, int sy, int k, int dtype) {
  const size_t rb = dtype == GW_F32 ? 4 : 8;
  const size_t n = (size_t)sx * sx, m = (size_t)sy * sy;
  PowKLayout l{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) / 256 * 256;
    return o;
  };
  l.W = take(n * m * rb);
  l.cxh = take(n * rb);
  l.cxl = take(n * rb);
  l.cyh = take(m * rb);
  l.cyl = take(m * rb);
  l.rowsum = take(n * 8);
  l.colsum = take(m * 8);
  l.Mx = take((size_t)(2 * k + 1) * n * 8);
  l.My = take((size_t)(2 * k + 1) * m * 8);
  l.total = off;
  return l;
}

template <int K, typename Real>
int powk_typed(const Grad2DArgs& A, char* ws) {
  cudaStream_t st = A.stream;
  const int sx = A.sx, sy = A.sy;
  const int n = sx * sx, m = sy * sy;
  const size_t rb = sizeof(Real);
  const PowKLayout lay = powk_layout(sx, sy, K, A.dtype);
  double* rowsum = (double*)(ws + lay.rowsum);
  double* colsum = (double*)(ws + lay.colsum);

  // Pass 1 (also T 1 for exact marginals).
  {
    const size_t smem = images_smem(K, sy, 1, rb);
    auto kern = g2k_images<K, Real, 0>;
    if (!allow_dynamic_smem((const void*)kern, smem)) return GW_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    const int grid = std::max(1, std::min(n, std::max(1, per_sm) * A.num_sms));
    PowKIO io{A.T, ws + lay.W, n, m, sy, 1, A.exact ? rowsum : nullptr, nullptr, nullptr, nullptr, nullptr, 0.0};
    TraceScope ts(A.tracer, "g2k_rows", st);
    kern<<<grid, 256, smem, st>>>(io);
  }
  // Constant terms from the target marginals or from T's own marginals.
  const double* wx = A.u;
  const double* wy = A.v;
  if (A.exact) {
    TraceScope ts(A.tracer, "g2k_colsum", st);
    cudaMemsetAsync(colsum, 0, (size_t)m * 8, st);
    const int rows_per = std::max(1, (n + 63) / 64);
    g2k_colsum<Real><<<dim3((m + 255) / 256, (n + rows_per - 1) / rows_per), 256, 0, st>>>((const Real*)A.T, n, m,
                                                                                           rows_per, colsum);
    wx = rowsum;
    wy = colsum;
  }
  {
    // The constant terms carry out_scale (the solver's Pi = 2 theta G).
    TraceScope ts(A.tracer, "g2k_const", st);
    const int P2 = 2 * K;
    const int pad1 = ((P2 + 1) * n + 255) / 256 * 256, pad2 = (n + 255) / 256 * 256;
    ConstJob jx{wx, sx, (double*)(ws + lay.Mx), ws + lay.cxh, ws + lay.cxl, std::pow(A.hx, 2 * K) * A.out_scale,
                pad1, pad2};
    ConstJob jy{wy, sy, (double*)(ws + lay.My), ws + lay.cyh, ws + lay.cyl, std::pow(A.hy, 2 * K) * A.out_scale, 0, 0};
    g2k_const1<<<(pad1 + (P2 + 1) * m + 255) / 256, 256, 0, st>>>(jx, jy, P2);
    g2k_const2<Real><<<(pad2 + m + 255) / 256, 256, 0, st>>>(jx, jy, P2);
  }
  // Pass 2 with the epilogue.
  {
    const int P = pass2_tile(K, sx, rb);
    if (P == 0) return GW_ERR_INVALID;
    const size_t smem = images_smem(K, sx, P, rb);
    auto kern = g2k_images<K, Real, 1>;
    if (!allow_dynamic_smem((const void*)kern, smem)) return GW_ERR_CUDA;
    const int threads = std::max(256, ((std::max(2 * P * sx, P * sx + 2 * P) + 31) / 32) * 32);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    const int tiles = (m + P - 1) / P;
    const int grid = std::max(1, std::min(tiles, std::max(1, per_sm) * A.num_sms));
    PowKIO io{ws + lay.W, A.G, n, m, sx, P, nullptr, ws + lay.cxh, ws + lay.cxl, ws + lay.cyh, ws + lay.cyl,
              2.0 * std::pow(A.hx, K) * std::pow(A.hy, K) * A.out_scale};
    TraceScope ts(A.tracer, "g2k_cols", st);
    kern<<<grid, threads, smem, st>>>(io);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

}  // namespace

bool grad2d_powk_supported(int sx, int sy, int k, int dtype) {
  if (k < 2 || k > 3 || sx > kMaxConstSide || sy > kMaxConstSide) return false;
  const size_t rb = dtype == GW_F32 ? 4 : 8;
  if (2 * sy > 512 || 2 * sx > 512) return false;
  if (images_smem(k, sy, 1, rb) > kPowKSmemLimit) return false;
  return pass2_tile(k, sx, rb) > 0;
}

size_t grad2d_powk_workspace_bytes(int sx, int sy, int k, int dtype) {
  return powk_layout(sx, sy, k, dtype).total + 4096;
}

int grad2d_powk_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes) {
  if (!grad2d_powk_supported(a.sx, a.sy, a.k, a.dtype)) return GW_ERR_INVALID;
  if (grad2d_powk_workspace_bytes(a.sx, a.sy, a.k, a.dtype) > ws_bytes) return GW_ERR_OOM;
  char* w = (char*)ws;
  if (a.dtype == GW_F32) return a.k == 2 ? powk_typed<2, float>(a, w) : powk_typed<3, float>(a, w);
  return a.k == 2 ? powk_typed<2, double>(a, w) : powk_typed<3, double>(a, w);
}

}  // namespace gw
