// Device helpers shared by the grid gradients with an axis-separable cost
// (2D in grad2d.cu, 3D in grad3d.cu): accumulator helpers, the axis weight,
// the column sums of T for exact marginals and the small transforms by the
// axis matrix.  Included inside namespace gw's anonymous namespace.
#pragma once

template <typename Real>
using AccOf = typename AccT<Real>::type;

__device__ __forceinline__ ff acc_add_d(ff a, double x) { return ff_add(a, ff_from_double(x)); }
__device__ __forceinline__ double acc_add_d(double a, double x) { return a + x; }
__device__ __forceinline__ ff acc_mul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ double acc_mul(double a, double b) { return a * b; }
__device__ __forceinline__ void acc_from(ff* o, double x) { *o = ff_from_double(x); }
__device__ __forceinline__ void acc_from(double* o, double x) { *o = x; }
__device__ __forceinline__ void acc_split(ff a, float& hi, float& lo) {
  hi = a.hi;
  lo = a.lo;
}
__device__ __forceinline__ void acc_split(double a, double& hi, double& lo) {
  hi = a;
  lo = 0.0;
}

// Axis weight A(delta): |delta| or delta^2 (exact in float for |delta| < 4096).
__device__ __forceinline__ float axis_w(int delta, int sq) {
  const float a = (float)(delta < 0 ? -delta : delta);
  return sq ? a * a : a;
}
__device__ __forceinline__ ff acc_w(ff x, float w) { return ff_mul(x, w); }
__device__ __forceinline__ double acc_w(double x, float w) { return x * (double)w; }

// Column sums of T over row bands (exact marginals only), then over bands.
template <typename Real>
__global__ void g2_colsum(const Real* __restrict__ T, int n, int m, int rows_per, AccOf<Real>* __restrict__ part) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const int i0 = blockIdx.y * rows_per, i1 = min(n, i0 + rows_per);
  Real s = 0, cmp = 0;
  for (int i = i0; i < i1; ++i) {
    const Real y = T[(size_t)i * m + p] - cmp;
    const Real s2 = s + y;
    cmp = (s2 - s) - y;
    s = s2;
  }
  part[(size_t)blockIdx.y * m + p] = acc_of(s, -cmp);
}

template <typename Acc>
__global__ void g2_colsum_fin(const Acc* __restrict__ part, int nb, int m, Acc* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  Acc s = acc_zero((Acc*)nullptr);
  for (int b = 0; b < nb; ++b) s = acc_add(s, part[(size_t)b * m + p]);
  out[p] = s;
}

// One butterfly step of a warp reduction on accumulators.
__device__ __forceinline__ ff acc_shfl_xor(ff a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ double acc_shfl_xor(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }

// Small transforms by the axis matrix A (entries A(i - l)^pw):
//   left:  out[b][i][j] = sum_l A(i - l)^pw in[b][l][j]
//   right: out[b][i][j] = sum_l in[b][i][l] A(l - j)^pw
struct TxJob {
  const void* in;
  void* out;
  int batch, rows, cols;
  int right, sq, pw;
  int start;  // first thread of this job
};
constexpr int kMaxTxJobs = 8;
struct TxJobs {
  TxJob j[kMaxTxJobs];
  int n, total;
};

template <typename Acc>
__global__ void g2_tx(const __grid_constant__ TxJobs jobs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= jobs.total) return;
  int q = 0;
  while (q + 1 < jobs.n && t >= jobs.j[q + 1].start) ++q;
  const TxJob J = jobs.j[q];
  const int e = t - J.start;
  const int per = J.rows * J.cols;
  const int b = e / per, i = (e % per) / J.cols, j = e % J.cols;
  const Acc* in = (const Acc*)J.in + (size_t)b * per;
  const int len = J.right ? J.cols : J.rows;
  // Element l of the contracted line and the weight's offset from it.
  const Acc* x0 = J.right ? in + (size_t)i * J.cols : in + j;
  const int stride = J.right ? 1 : J.cols;
  const int ref = J.right ? j : i;
  constexpr int U = 8;
  Acc s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q] = acc_zero((Acc*)nullptr);
  int l = 0;
  for (; l + U <= len; l += U) {
    Acc x[U];
#pragma unroll
    for (int q = 0; q < U; ++q) x[q] = x0[(size_t)(l + q) * stride];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const float w = axis_w(l + q - ref, J.sq);
      Acc y = acc_w(x[q], w);
      if (J.pw == 2) y = acc_w(y, w);
      s[q & 3] = acc_add(s[q & 3], y);
    }
  }
  for (; l < len; ++l) {
    const float w = axis_w(l - ref, J.sq);
    Acc y = acc_w(x0[(size_t)l * stride], w);
    if (J.pw == 2) y = acc_w(y, w);
    s[0] = acc_add(s[0], y);
  }
  ((Acc*)J.out)[e] = acc_add(acc_add(s[0], s[1]), acc_add(s[2], s[3]));
}

// Blocks of `threads` threads (with `smem` bytes of dynamic shared memory)
// that one SM holds at once for kernel f.
template <typename F>
int resident_blocks(F f, int threads, size_t smem = 0) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, smem) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}
