// Host dispatch of the structured 1D gradient and the constant-term kernels.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "grad1d_impl.cuh"

namespace gw {

// Bands of at least 8 rows, about `target` of them (one CTA each).
Bands choose_bands(int n, int target) {
  const int Rmin = 8;
  int B = std::max(1, std::min(target, (n + Rmin - 1) / Rmin));
  int R = (n + B - 1) / B;
  B = (n + R - 1) / R;
  return {B, R};
}

__global__ void rowsum_finish(const void* rowpart, int nchunks, int n, int is_f32, double* r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  if (is_f32) {
    const float* rp = (const float*)rowpart;
    for (int c = 0; c < nchunks; ++c) {
      const size_t o = ((size_t)c * n + i) * 2;
      acc += (double)rp[o] + (double)rp[o + 1];
    }
  } else {
    const double* rp = (const double*)rowpart;
    for (int c = 0; c < nchunks; ++c) {
      const size_t o = ((size_t)c * n + i) * 2;
      acc += rp[o] + rp[o + 1];
    }
  }
  r[i] = acc;
}

// Constant term c[i] = factor * sum_j (i - j)^P w_j, P = 2k (even), written as
// a polynomial in (i - ctr) whose coefficients are the centred moments
// M_t = sum_j (j - ctr)^t w_j (binomial expansion of ((i-ctr) - (j-ctr))^P).
// FP64 throughout.  Both vectors (X and Y) go through the same two launches;
// the work is spread over many blocks because FP64 throughput per SM is low.
constexpr int kMargBlock = 256;

struct MargVec {
  const double* w;
  int len;
  double factor;
  void* out;
};

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ ff warp_sum_ff(ff x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
    x = ff_add(x, y);
  }
  return x;
}

// Float output: float-float arithmetic on the FP32 pipe (the constant term
// keeps about 48 bits, ample for a float result; FP64 throughput per SM is
// too low to be worth it here).  Partials are stored as (hi, lo) floats.
__global__ void marg_moments2_ff(MargVec X, MargVec Y, int nbx, int P, float* __restrict__ part) {
  __shared__ ff sm[kMargBlock / 32][16];
  const bool isx = (int)blockIdx.x < nbx;
  const MargVec V = isx ? X : Y;
  const int blk = isx ? blockIdx.x : blockIdx.x - nbx;
  const int j = blk * kMargBlock + threadIdx.x;
  const float d = (float)(j - V.len / 2);
  ff pw = (j < V.len) ? ff_from_double(V.w[j]) : ff{0.f, 0.f};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t <= P; ++t) {
    const ff s = warp_sum_ff(pw);
    if (lane == 0) sm[warp][t] = s;
    pw = ff_mul(pw, d);
  }
  __syncthreads();
  if (threadIdx.x <= P) {
    ff acc{0.f, 0.f};
    for (int w = 0; w < kMargBlock / 32; ++w) acc = ff_add(acc, sm[w][threadIdx.x]);
    part[((size_t)blockIdx.x * (P + 1) + threadIdx.x) * 2 + 0] = acc.hi;
    part[((size_t)blockIdx.x * (P + 1) + threadIdx.x) * 2 + 1] = acc.lo;
  }
}

__global__ void marg_eval2_ff(MargVec X, MargVec Y, int nbx, int nby, int P, const float* __restrict__ part,
                              float fxh, float fxl, float fyh, float fyl) {
  __shared__ ff M[16];
  const bool isx = (int)blockIdx.x < nbx;
  const MargVec V = isx ? X : Y;
  const int blk = isx ? blockIdx.x : blockIdx.x - nbx;
  const int p0 = isx ? 0 : nbx, np = isx ? nbx : nby;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t <= P; t += kMargBlock / 32) {
    ff acc{0.f, 0.f};
    for (int b = lane; b < np; b += 32) {
      const size_t o = ((size_t)(p0 + b) * (P + 1) + t) * 2;
      acc = ff_add(acc, ff{part[o], part[o + 1]});
    }
    acc = warp_sum_ff(acc);
    if (lane == 0) M[t] = acc;
  }
  __syncthreads();
  const int i = blk * kMargBlock + threadIdx.x;
  if (i >= V.len) return;
  const float x = (float)(i - V.len / 2);
  // sum_t C(P,t) x^{P-t} (-1)^t M_t, Horner in x.
  ff acc{0.f, 0.f};
  for (int t = 0; t <= P; ++t) {
    ff c = ff_mul(M[t], (float)binom(P, t));
    if (t & 1) c = ff_neg(c);
    acc = ff_add(ff_mul(acc, x), c);
  }
  const ff val = ff_mul(acc, ff{isx ? fxh : fyh, isx ? fxl : fyl});
  float* out = (float*)V.out;
  out[i] = val.hi;
  out[V.len + i] = val.lo;
}

__global__ void marg_moments2(MargVec X, MargVec Y, int nbx, int P, double* __restrict__ part) {
  __shared__ double sm[kMargBlock / 32][16];
  const bool isx = (int)blockIdx.x < nbx;
  const MargVec V = isx ? X : Y;
  const int blk = isx ? blockIdx.x : blockIdx.x - nbx;
  const int j = blk * kMargBlock + threadIdx.x;
  const double ctr = (double)(V.len / 2);
  const double d = (double)j - ctr;
  double pw = (j < V.len) ? V.w[j] : 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t <= P; ++t) {
    const double s = warp_sum_d(pw);
    if (lane == 0) sm[warp][t] = s;
    pw *= d;
  }
  __syncthreads();
  if (threadIdx.x <= P) {
    double acc = 0.0;
    for (int w = 0; w < kMargBlock / 32; ++w) acc += sm[w][threadIdx.x];
    part[(size_t)blockIdx.x * (P + 1) + threadIdx.x] = acc;
  }
}

// Writes out[0..len) = hi part and out[len..2 len) = lo part of each value
// (lo = 0 for double output).
__global__ void marg_eval2(MargVec X, MargVec Y, int nbx, int nby, int nex, int P, const double* __restrict__ part) {
  __shared__ double M[16];
  const bool isx = (int)blockIdx.x < nex;
  const MargVec V = isx ? X : Y;
  const int blk = isx ? blockIdx.x : blockIdx.x - nex;
  const int p0 = isx ? 0 : nbx, np = isx ? nbx : nby;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t <= P; t += kMargBlock / 32) {
    double acc = 0.0;
    for (int b = lane; b < np; b += 32) acc += part[(size_t)(p0 + b) * (P + 1) + t];
    acc = warp_sum_d(acc);
    if (lane == 0) M[t] = acc;
  }
  __syncthreads();
  const int i = blk * kMargBlock + threadIdx.x;
  if (i >= V.len) return;
  const double x = (double)i - (double)(V.len / 2);
  double acc = 0.0;
  for (int t = 0; t <= P; ++t) {
    const double c = (double)binom(P, t) * ((t & 1) ? -M[t] : M[t]);
    acc = acc * x + c;
  }
  double* out = (double*)V.out;
  out[i] = V.factor * acc;
  out[V.len + i] = 0.0;
}

size_t marg_part_doubles(int len, int k) {
  const int nblk = (len + kMargBlock - 1) / kMargBlock;
  return (size_t)nblk * (2 * k + 1);
}

int marg_const2_launch(const double* wx, int n, double fx, void* outx, const double* wy, int m, double fy,
                       void* outy, int k, int dtype, double* part, cudaStream_t stream, Tracer* tracer) {
  const int P = 2 * k;
  const int nbx = (n + kMargBlock - 1) / kMargBlock, nby = (m + kMargBlock - 1) / kMargBlock;
  MargVec X{wx, n, fx, outx}, Y{wy, m, fy, outy};
  if (dtype == GW_F32) {
    const float fxh = (float)fx, fyh = (float)fy;
    const float fxl = (float)(fx - (double)fxh), fyl = (float)(fy - (double)fyh);
    {
      TraceScope ts(tracer, "marg_moments", stream);
      marg_moments2_ff<<<nbx + nby, kMargBlock, 0, stream>>>(X, Y, nbx, P, (float*)part);
    }
    TraceScope ts(tracer, "marg_eval", stream);
    marg_eval2_ff<<<nbx + nby, kMargBlock, 0, stream>>>(X, Y, nbx, nby, P, (const float*)part, fxh, fxl, fyh, fyl);
  } else {
    {
      TraceScope ts(tracer, "marg_moments", stream);
      marg_moments2<<<nbx + nby, kMargBlock, 0, stream>>>(X, Y, nbx, P, part);
    }
    TraceScope ts(tracer, "marg_eval", stream);
    marg_eval2<<<nbx + nby, kMargBlock, 0, stream>>>(X, Y, nbx, nby, nbx, P, part);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

int marg_const_launch(const double* w, int len, int k, double factor, void* out, int dtype, double* part,
                      cudaStream_t stream, Tracer* tracer) {
  return marg_const2_launch(w, len, factor, out, w, 0, 0.0, nullptr, k, dtype, part, stream, tracer);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_rows_tmap(void* tmap, const void* base, int n, int m, int elem_bytes, int* box_cols) {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  if (!fn) return false;
  const int E = 128 / elem_bytes;
  if (m % E != 0 || n < 1) return false;
  // Box height: the largest divisor of m / E that is at most 256, so that a
  // row is a whole number of boxes with no out-of-range fill.
  int bc = std::min(256, m / E);
  while ((m / E) % bc != 0) --bc;
  cuuint64_t dims[3] = {(cuuint64_t)E, (cuuint64_t)(m / E), (cuuint64_t)n};
  cuuint64_t strides[2] = {128, (cuuint64_t)m * (cuuint64_t)elem_bytes};
  cuuint32_t box[3] = {(cuuint32_t)E, (cuuint32_t)bc, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn((CUtensorMap*)tmap, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                  3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  *box_cols = bc;
  return r == CUDA_SUCCESS;
}

bool encode_rows_tmap_box(void* tmap, const void* base, int n, int m, int elem_bytes, int box_cols) {
  // Same shape as encode_rows_tmap ({128-byte chunk, chunks per row, rows},
  // 128-byte swizzle) with a given box height, for tensor stores.
  int dummy = 0;
  if (!encode_rows_tmap(tmap, base, n, m, elem_bytes, &dummy)) return false;  // checks shape and driver
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  const int E = 128 / elem_bytes;
  if (!fn || box_cols < 1 || box_cols > 256 || box_cols > m / E) return false;
  cuuint64_t dims[3] = {(cuuint64_t)E, (cuuint64_t)(m / E), (cuuint64_t)n};
  cuuint64_t strides[2] = {128, (cuuint64_t)m * (cuuint64_t)elem_bytes};
  cuuint32_t box[3] = {(cuuint32_t)E, (cuuint32_t)box_cols, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn((CUtensorMap*)tmap, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                  3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {
thread_local char g_failure[256] = "";
}
void note_failure(const char* what) { snprintf(g_failure, sizeof g_failure, "%s", what); }
const char* last_failure() { return g_failure; }

namespace {
// Functions whose attribute is already set, per device, with their limit.
struct SmemGrant {
  const void* func;
  int dev, limit;
};
std::mutex g_grant_mu;
std::vector<SmemGrant> g_grants;
}  // namespace

bool allow_dynamic_smem(const void* func, size_t need) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    note_failure("cudaGetDevice failed");
    return false;
  }
  {
    std::lock_guard<std::mutex> lk(g_grant_mu);
    for (const auto& gr : g_grants)
      if (gr.func == func && gr.dev == dev) {
        if (need <= (size_t)gr.limit) return true;
        snprintf(g_failure, sizeof g_failure, "kernel needs %zu bytes of dynamic shared memory, limit %d", need,
                 gr.limit);
        return false;
      }
  }
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_failure, sizeof g_failure, "shared-memory limit query: %s", cudaGetErrorString(e));
    return false;
  }
  // The limit covers static and dynamic shared memory together.
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_failure, sizeof g_failure, "cudaFuncGetAttributes: %s", cudaGetErrorString(e));
    return false;
  }
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if (need > (size_t)dyn_max) {
    snprintf(g_failure, sizeof g_failure, "kernel needs %zu bytes of dynamic shared memory, limit %d", need, dyn_max);
    return false;
  }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_failure, sizeof g_failure, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return false;
  }
  std::lock_guard<std::mutex> lk(g_grant_mu);
  g_grants.push_back({func, dev, dyn_max});
  return true;
}

size_t grad1d_workspace_bytes(int n, int m, int k, int dtype, int num_sms) {
  return k1_layout(n, m, k, dtype == GW_F32 ? 4 : 8, num_sms).end;
}

bool grad1d_regen_supported(int n, int m, int k, int ky, int dtype, int force_generic) {
  const int kk = ky > 0 ? ky : k;
  return dtype == GW_F32 && !force_generic && n >= 1 && m % 32 == 0 && m >= 32 && m <= 8192 && k >= 1 &&
         k <= 2 && kk >= 1 && kk <= 2;
}

int grad1d_launch(const Grad1DArgs& a, void* ws, size_t ws_bytes) {
  if (a.ky != 0 && a.ky != a.k) return grad1d_launch_mixed(a, ws, ws_bytes);
  switch (a.k) {
    case 1: return grad1d_launch_k1(a, ws, ws_bytes);
    case 2: return grad1d_launch_k2(a, ws, ws_bytes);
    case 3: return grad1d_launch_k3(a, ws, ws_bytes);
    default: return GW_ERR_INVALID;
  }
}

}  // namespace gw
