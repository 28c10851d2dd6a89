// Dense comparison gradient: G = c_x 1^T + 1 c_y^T - 2 D_X T D_Y with the
// distance matrices materialised and the two products D_X T and (D_X T) D_Y
// done by cuBLAS (the "original" O(n^2 m + n m^2) route of Sec. 2.1 that the
// structured recursion replaces).  Precisions: FP32 (CUDA cores), TF32 and
// BF16 tensor cores with FP32 accumulation, FP64.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "gw_common.cuh"
#include "gw_internal.h"

namespace gw {

// Absolute coordinate differences of grid points i and j on a side^dims grid
// (row-major, the last axis fastest; dims = 2 or 3).
__device__ __forceinline__ void grid_deltas(long long i, long long j, int side, int dims, double (&d)[3]) {
  for (int t = dims - 1; t >= 0; --t) {
    d[t] = (double)llabs(i % side - j % side);
    i /= side;
    j /= side;
  }
  if (dims < 3) d[2] = 0.0;
}

// Grid distance from coordinate differences: Manhattan^k (sq = 0) or squared
// Euclidean (sq = 1), without the spacing factor.
__device__ __forceinline__ double grid_metric(const double (&d)[3], int k, int sq) {
  if (sq) return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double s = d[0] + d[1] + d[2];
  double v = 1.0;
  for (int e = 0; e < k; ++e) v *= s;
  return v;
}

// D[i][j] = d(i, j) for n points: 1D grid (side = 0): h^k |i - j|^k; grid of
// side^dims points (row-major): Manhattan h^k (sum_t |x_t - x'_t|)^k (sq = 0)
// or squared Euclidean h^2 sum_t (x_t - x'_t)^2 (sq = 1).
template <typename Out>
__global__ void build_dist(Out* __restrict__ D, int n, double hk, int k, int side, int dims, int sq, int pitch,
                           int tf32) {
  const size_t N = (size_t)n * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    const long long i = (long long)(idx / n), j = (long long)(idx % n);
    double v;
    if (side > 0) {
      double d[3];
      grid_deltas(i, j, side, dims, d);
      v = grid_metric(d, k, sq);
    } else {
      const double d = (double)(i > j ? i - j : j - i);
      v = 1.0;
      for (int e = 0; e < k; ++e) v *= d;
    }
    Out o = (Out)(hk * v);
    if constexpr (sizeof(Out) == 4) {
      if (tf32) {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)(hk * v)));
        o = (Out)__uint_as_float(r);
      }
    }
    D[(size_t)i * pitch + j] = o;
  }
}

// Four floats -> four bfloat16 per thread (16-byte loads, 8-byte stores);
// N a multiple of 4, both arrays 16-byte aligned.
__global__ void to_bf16(const float4* __restrict__ x, __nv_bfloat162* __restrict__ y, size_t N4) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = x[i];
    y[2 * i] = __floats2bfloat162_rn(v.x, v.y);
    y[2 * i + 1] = __floats2bfloat162_rn(v.z, v.w);
  }
}
__global__ void to_bf16_tail(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, size_t from, size_t N) {
  for (size_t i = from + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// Float rounded to the nearest TF32 value (10 mantissa bits), kept in a
// float: the tensor cores then read it exactly instead of dropping the low
// bits.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
template <typename Out> __device__ __forceinline__ Out to_input(float x);
template <> __device__ __forceinline__ float to_input<float>(float x) { return round_tf32(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_input<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// Four floats -> four TF32-rounded floats per thread (16-byte accesses).
__global__ void to_tf32(const float4* __restrict__ x, float4* __restrict__ y, size_t N4) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = x[i];
    y[i] = make_float4(round_tf32(v.x), round_tf32(v.y), round_tf32(v.z), round_tf32(v.w));
  }
}

// Rows of a float matrix (n x m) copied to pitch mp >= m in the tensor-core
// input type Out (TF32 values in floats, or bfloat16), the padding zero.
template <typename Out>
__global__ void pad_rows(const float* __restrict__ T, int n, int m, Out* __restrict__ Tp, int mp) {
  const size_t N = (size_t)n * mp;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t i = idx / mp, p = idx % mp;
    Tp[idx] = to_input<Out>(p < (size_t)m ? T[i * m + p] : 0.f);
  }
}

// G = cx_i + cy_p - s * Z_ip, in place on Z (= G).  cx, cy hold hi parts first.
// One block per matrix row, 16-byte accesses when the rows allow them.
template <typename Real>
__global__ void dense_epilogue(Real* __restrict__ G, int n, int m, const Real* __restrict__ cx,
                               const Real* __restrict__ cy, Real s) {
  constexpr int PER = 16 / sizeof(Real);
  const int i = blockIdx.x;
  Real* row = G + (size_t)i * m;
  const Real ci = cx[i];
  if (m % PER == 0 && ((reinterpret_cast<uintptr_t>(G) & 15) == 0)) {
    for (int q = threadIdx.x; q < m / PER; q += blockDim.x) {
      float4 z = reinterpret_cast<float4*>(row)[q];
      Real* e = reinterpret_cast<Real*>(&z);
#pragma unroll
      for (int w = 0; w < PER; ++w) e[w] = fma(-s, e[w], ci + cy[q * PER + w]);
      reinterpret_cast<float4*>(row)[q] = z;
    }
  } else {
    for (int p = threadIdx.x; p < m; p += blockDim.x) row[p] = fma(-s, row[p], ci + cy[p]);
  }
}

// Constant term on a 2D or 3D grid, pointwise: c[i] = scale * sum_j d(i,j)^2
// w_j with d the Manhattan^k or squared Euclidean grid distance (one block
// per i).
template <typename Real>
__global__ void dist2_const_grid(const double* __restrict__ w, int side, int dims, int sq, int k, double scale,
                                 Real* __restrict__ out) {
  const int n = dims == 3 ? side * side * side : side * side;
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double dd[3];
    grid_deltas(i, j, side, dims, dd);
    const double d = grid_metric(dd, k, sq);
    acc += d * d * w[j];
  }
  __shared__ double sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
    t *= scale;
    // hi part, then the rounding remainder (read by the epilogue as cx + cy).
    out[i] = (Real)t;
    out[n + i] = (Real)(t - (double)(Real)t);
  }
}

template <typename Real>
__global__ void row_sums(const Real* __restrict__ T, int n, int m, double* __restrict__ r) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double acc = 0.0;
  for (int p = threadIdx.x & 31; p < m; p += 32) acc += (double)T[(size_t)i * m + p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) r[i] = acc;
}

template <typename Real>
__global__ void col_sums(const Real* __restrict__ T, int n, int m, double* __restrict__ c) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += (double)T[(size_t)i * m + p];
  c[p] = acc;
}

struct DenseCache {
  int n = 0, k = 0, prec = -1, side = 0, dims = 0, sq = 0, pitch = 0;
  double h = 0;
  void* D = nullptr;
};

// Row pitch (elements) of the matrices the tcgen05 kernels read: a multiple
// of 16 bytes, padding zero.
int tc_pitch(int n, int prec) {
  const int q = prec == GW_DENSE_TC_BF16 ? 8 : 4;
  return (n + q - 1) / q * q;
}
bool is_tc(int prec) { return prec == GW_DENSE_TC_BF16 || prec == GW_DENSE_TC_TF32; }

struct DenseState {
  cublasHandle_t handle = nullptr;
  DenseCache X, Y;
};

static int ensure_dist(DenseCache& c, int n, double h, int k, int side, int dims, int sq, int prec,
                       cudaStream_t st) {
  if (c.D && c.n == n && c.h == h && c.k == k && c.side == side && c.dims == dims && c.sq == sq && c.prec == prec)
    return GW_OK;
  if (c.D) {
    cudaStreamSynchronize(st);
    cudaFree(c.D);
    c.D = nullptr;
  }
  const bool bf = prec == GW_DENSE_BF16 || prec == GW_DENSE_TC_BF16;
  const size_t esz = bf ? 2 : (prec == GW_DENSE_FP64 ? 8 : 4);
  const int pitch = is_tc(prec) ? tc_pitch(n, prec) : n;
  if (cudaMalloc(&c.D, (size_t)pitch * pitch * esz) != cudaSuccess) {
    cudaGetLastError();
    c.D = nullptr;
    return GW_ERR_OOM;
  }
  const double hk = side > 0 && sq ? h * h : std::pow(h, k);
  if (pitch != n) cudaMemsetAsync(c.D, 0, (size_t)pitch * pitch * esz, st);
  const int tf = prec == GW_DENSE_TC_TF32;
  if (bf)
    build_dist<__nv_bfloat16><<<1024, 256, 0, st>>>((__nv_bfloat16*)c.D, n, hk, k, side, dims, sq, pitch, 0);
  else if (prec == GW_DENSE_FP64)
    build_dist<double><<<1024, 256, 0, st>>>((double*)c.D, n, hk, k, side, dims, sq, pitch, 0);
  else
    build_dist<float><<<1024, 256, 0, st>>>((float*)c.D, n, hk, k, side, dims, sq, pitch, tf);
  c.pitch = pitch;
  c.n = n;
  c.h = h;
  c.k = k;
  c.side = side;
  c.dims = dims;
  c.sq = sq;
  c.prec = prec;
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

void* dense_state_create() { return new DenseState(); }

void dense_state_destroy(void* p) {
  DenseState* s = (DenseState*)p;
  if (!s) return;
  if (s->X.D) cudaFree(s->X.D);
  if (s->Y.D) cudaFree(s->Y.D);
  if (s->handle) cublasDestroy(s->handle);
  delete s;
}

size_t dense_workspace_bytes(int n, int m, int prec) {
  const size_t nm = (size_t)n * m;
  size_t b = 0;
  if (is_tc(prec)) {
    // T with padded rows (n x mp) and C1 = D_Y T^T (m x np), in the input type.
    const size_t es = prec == GW_DENSE_TC_BF16 ? 2 : 4;
    b += (size_t)n * tc_pitch(m, prec) * es + (size_t)m * tc_pitch(n, prec) * es + 1024;
  } else if (prec == GW_DENSE_BF16) b += 2 * nm * 2;   // T and Y in bf16
  else if (prec == GW_DENSE_FP64) b += nm * 8;          // Y
  else b += nm * 4;                                     // Y
  b += ((size_t)2 * (n + m) * 8) + (size_t)(n + m) * 8 + marg_part_doubles(n, 3) * 8 + marg_part_doubles(m, 3) * 8 + 8192;
  return b;
}

int dense_grad_launch(void* state, const DenseArgs& a, void* wsv, size_t ws_bytes) {
  DenseState* S = (DenseState*)state;
  cudaStream_t st = a.stream;
  if (!S->handle) {
    if (cublasCreate(&S->handle) != CUBLAS_STATUS_SUCCESS) return GW_ERR_CUDA;
  }
  cublasSetStream(S->handle, st);
  const int n = a.n, m = a.m;
  const bool grid = a.dim >= 2;
  const int sq = grid && a.cost == GW_COST_SQEUCLID;
  int rc = ensure_dist(S->X, n, a.hx, a.k, grid ? a.sx : 0, a.dim, sq, a.prec, st);
  if (rc != GW_OK) return rc;
  const int ky = a.ky > 0 ? a.ky : a.k;
  rc = ensure_dist(S->Y, m, a.hy, ky, grid ? a.sy : 0, a.dim, sq, a.prec, st);
  if (rc != GW_OK) return rc;
  char* ws = (char*)wsv;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = ws + off;
    off = (off + bytes + 255) / 256 * 256;
    return p;
  };
  const size_t nm = (size_t)n * m;
  const bool dbl = a.prec == GW_DENSE_FP64;
  const size_t rb = dbl ? 8 : 4;
  void* Tin = (void*)a.T;
  void* Y = nullptr;
  const bool tc = is_tc(a.prec);
  const int np = tc ? tc_pitch(n, a.prec) : n, mp = tc ? tc_pitch(m, a.prec) : m;
  if (tc) {
    const size_t es = a.prec == GW_DENSE_TC_BF16 ? 2 : 4;
    Tin = take((size_t)n * mp * es);
    Y = take((size_t)m * np * es);
  } else if (a.prec == GW_DENSE_BF16) {
    Tin = take(nm * 2);
    Y = take(nm * 2);
  } else {
    Y = take(nm * rb);
  }
  void* cx = take((size_t)2 * n * rb);
  void* cy = take((size_t)2 * m * rb);
  double* r = (double*)take((size_t)n * 8);
  double* cc = (double*)take((size_t)m * 8);
  double* part = (double*)take((marg_part_doubles(n, 3) + marg_part_doubles(m, 3)) * 8 + 512);
  if (off > ws_bytes) return GW_ERR_OOM;

  const double* wx = a.u;
  const double* wy = a.v;
  if (a.exact) {
    TraceScope ts(a.tracer, "dense_marginals", st);
    if (dbl) {
      row_sums<double><<<(n + 7) / 8, 256, 0, st>>>((const double*)a.T, n, m, r);
      col_sums<double><<<(m + 255) / 256, 256, 0, st>>>((const double*)a.T, n, m, cc);
    } else {
      row_sums<float><<<(n + 7) / 8, 256, 0, st>>>((const float*)a.T, n, m, r);
      col_sums<float><<<(m + 255) / 256, 256, 0, st>>>((const float*)a.T, n, m, cc);
    }
    wx = r;
    wy = cc;
  }
  if (grid) {
    TraceScope ts(a.tracer, "dense_const", st);
    const double fx = sq ? a.hx * a.hx : std::pow(a.hx, a.k), fy = sq ? a.hy * a.hy : std::pow(a.hy, a.k);
    if (dbl) {
      dist2_const_grid<double><<<n, 256, 0, st>>>(wx, a.sx, a.dim, sq, a.k, fx * fx, (double*)cx);
      dist2_const_grid<double><<<m, 256, 0, st>>>(wy, a.sy, a.dim, sq, a.k, fy * fy, (double*)cy);
    } else {
      dist2_const_grid<float><<<n, 256, 0, st>>>(wx, a.sx, a.dim, sq, a.k, fx * fx, (float*)cx);
      dist2_const_grid<float><<<m, 256, 0, st>>>(wy, a.sy, a.dim, sq, a.k, fy * fy, (float*)cy);
    }
  } else {
    if (ky == a.k) {
      rc = marg_const2_launch(wx, n, std::pow(a.hx, 2 * a.k), cx, wy, m, std::pow(a.hy, 2 * a.k), cy, a.k,
                              dbl ? GW_F64 : GW_F32, part, st, a.tracer);
    } else {
      rc = marg_const_launch(wx, n, a.k, std::pow(a.hx, 2 * a.k), cx, dbl ? GW_F64 : GW_F32, part, st, a.tracer);
      if (rc == GW_OK)
        rc = marg_const_launch(wy, m, ky, std::pow(a.hy, 2 * ky), cy, dbl ? GW_F64 : GW_F32,
                               part + marg_part_doubles(n, a.k), st, a.tracer);
    }
    if (rc != GW_OK) return rc;
  }

  if (tc) {
    // C1 = D_Y T^T (m x np), then G = c_x + c_y - 2 D_X C1^T in the second
    // product's epilogue.  T is copied with zero-padded rows (pitch mp) in the
    // input type; the padding columns of C1 come out zero.
    const bool tf32 = a.prec == GW_DENSE_TC_TF32;
    const void* Tk = Tin;
    {
      TraceScope ts(a.tracer, "dense_pad_T", st);
      const bool vec = mp == m && nm % 4 == 0 && (reinterpret_cast<uintptr_t>(a.T) & 15) == 0;
      if (vec && tf32)
        to_tf32<<<8 * 152, 256, 0, st>>>((const float4*)a.T, (float4*)Tin, nm / 4);
      else if (vec)
        to_bf16<<<8 * 152, 256, 0, st>>>((const float4*)a.T, (__nv_bfloat162*)Tin, nm / 4);
      else if (tf32)
        pad_rows<float><<<8 * 152, 256, 0, st>>>((const float*)a.T, n, m, (float*)Tin, mp);
      else
        pad_rows<__nv_bfloat16><<<8 * 152, 256, 0, st>>>((const float*)a.T, n, m, (__nv_bfloat16*)Tin, mp);
    }
    rc = tc_gemm_abt_launch(tf32, S->Y.D, mp, Tk, mp, m, n, mp, tf32 ? 1 : 0, Y, np, m, np, nullptr, nullptr, 0.f,
                            a.status, a.num_sms, st, a.tracer);
    if (rc != GW_OK) return rc;
    rc = tc_gemm_abt_launch(tf32, S->X.D, np, Y, np, n, m, np, 2, a.G, m, n, m, (const float*)cx, (const float*)cy,
                            2.f, a.status, a.num_sms, st, a.tracer);
    if (rc != GW_OK) return rc;
    return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
  }

  // Row-major n x m arrays are column-major m x n.  Y^T = T^T D_X and
  // Z^T = D_Y Y^T in column-major terms.
  cublasStatus_t cs;
  {
    TraceScope ts(a.tracer, "dense_gemm", st);
    if (a.prec == GW_DENSE_BF16) {
      if ((reinterpret_cast<uintptr_t>(a.T) & 15) == 0) {
        to_bf16<<<8 * 152, 256, 0, st>>>((const float4*)a.T, (__nv_bfloat162*)Tin, nm / 4);
        if (nm % 4) to_bf16_tail<<<1, 256, 0, st>>>((const float*)a.T, (__nv_bfloat16*)Tin, nm / 4 * 4, nm);
      } else {
        to_bf16_tail<<<8 * 152, 256, 0, st>>>((const float*)a.T, (__nv_bfloat16*)Tin, 0, nm);
      }
      const float one = 1.f, zero = 0.f;
      cs = cublasGemmEx(S->handle, CUBLAS_OP_N, CUBLAS_OP_N, m, n, n, &one, Tin, CUDA_R_16BF, m, S->X.D,
                        CUDA_R_16BF, n, &zero, Y, CUDA_R_16BF, m, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
      if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasGemmEx(S->handle, CUBLAS_OP_N, CUBLAS_OP_N, m, n, m, &one, S->Y.D, CUDA_R_16BF, m, Y,
                          CUDA_R_16BF, m, &zero, a.G, CUDA_R_32F, m, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    } else if (dbl) {
      const double one = 1.0, zero = 0.0;
      cs = cublasDgemm(S->handle, CUBLAS_OP_N, CUBLAS_OP_N, m, n, n, &one, (const double*)Tin, m,
                       (const double*)S->X.D, n, &zero, (double*)Y, m);
      if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasDgemm(S->handle, CUBLAS_OP_N, CUBLAS_OP_N, m, n, m, &one, (const double*)S->Y.D, m,
                         (const double*)Y, m, &zero, (double*)a.G, m);
    } else {
      const float one = 1.f, zero = 0.f;
      const cublasComputeType_t ct = a.prec == GW_DENSE_TF32 ? CUBLAS_COMPUTE_32F_FAST_TF32 : CUBLAS_COMPUTE_32F;
      cs = cublasGemmEx(S->handle, CUBLAS_OP_N, CUBLAS_OP_N, m, n, n, &one, Tin, CUDA_R_32F, m, S->X.D, CUDA_R_32F,
                        n, &zero, Y, CUDA_R_32F, m, ct, CUBLAS_GEMM_DEFAULT);
      if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasGemmEx(S->handle, CUBLAS_OP_N, CUBLAS_OP_N, m, n, m, &one, S->Y.D, CUDA_R_32F, m, Y, CUDA_R_32F,
                          m, &zero, a.G, CUDA_R_32F, m, ct, CUBLAS_GEMM_DEFAULT);
    }
  }
  if (cs != CUBLAS_STATUS_SUCCESS) return GW_ERR_CUDA;
  {
    TraceScope ts(a.tracer, "dense_epilogue", st);
    if (dbl)
      dense_epilogue<double><<<n, 256, 0, st>>>((double*)a.G, n, m, (const double*)cx, (const double*)cy, 2.0);
    else
      dense_epilogue<float><<<n, 256, 0, st>>>((float*)a.G, n, m, (const float*)cx, (const float*)cy, 2.f);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

}  // namespace gw
