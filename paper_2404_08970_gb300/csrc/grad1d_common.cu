// Host dispatch of the structured 1D gradient and the constant-term kernels.
#include <algorithm>
#include <cmath>

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
// FP64 throughout; the work is spread over ceil(len/256) blocks.
constexpr int kMargBlock = 256;

__global__ void marg_moments(const double* __restrict__ w, int len, int P, double ctr, double* __restrict__ part) {
  __shared__ double sm[kMargBlock];
  const int j = blockIdx.x * kMargBlock + threadIdx.x;
  const double d = (double)j - ctr;
  const double wj = (j < len) ? w[j] : 0.0;
  double pw = wj;
  for (int t = 0; t <= P; ++t) {
    sm[threadIdx.x] = pw;
    __syncthreads();
    for (int o = kMargBlock / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * (P + 1) + t] = sm[0];
    __syncthreads();
    pw *= d;
  }
}

// Writes out[0..len) = hi part and out[len..2 len) = lo part of each value
// (lo = 0 for double output), so that float consumers keep the constant term
// to float-float accuracy.
template <typename Real>
__global__ void marg_eval(const double* __restrict__ part, int nblk, int len, int P, double ctr, double factor,
                          Real* __restrict__ out) {
  __shared__ double M[16];
  if (threadIdx.x <= P) {
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * (P + 1) + threadIdx.x];
    M[threadIdx.x] = acc;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const double x = (double)i - ctr;
  // sum_t C(P,t) x^{P-t} (-1)^t M_t, Horner in x.
  double acc = 0.0;
  for (int t = 0; t <= P; ++t) {
    double c = (double)binom(P, t) * ((t & 1) ? -M[t] : M[t]);
    acc = acc * x + c;
  }
  const double val = factor * acc;
  const Real hi = (Real)val;
  out[i] = hi;
  out[len + i] = (Real)(val - (double)hi);
}

size_t marg_part_doubles(int len, int k) {
  const int nblk = (len + kMargBlock - 1) / kMargBlock;
  return (size_t)nblk * (2 * k + 1);
}

int marg_const_launch(const double* w, int len, int k, double factor, void* out, int dtype, double* part,
                      cudaStream_t stream, Tracer* tracer) {
  TraceScope ts(tracer, "marg_const", stream);
  const int P = 2 * k;
  const int nblk = (len + kMargBlock - 1) / kMargBlock;
  const double ctr = (double)(len / 2);
  marg_moments<<<nblk, kMargBlock, 0, stream>>>(w, len, P, ctr, part);
  if (dtype == GW_F32)
    marg_eval<float><<<nblk, kMargBlock, 0, stream>>>(part, nblk, len, P, ctr, factor, (float*)out);
  else
    marg_eval<double><<<nblk, kMargBlock, 0, stream>>>(part, nblk, len, P, ctr, factor, (double*)out);
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

size_t grad1d_workspace_bytes(int n, int m, int k, int dtype, int num_sms) {
  return k1_layout(n, m, k, dtype == GW_F32 ? 4 : 8, num_sms).end;
}

int grad1d_launch(const Grad1DArgs& a, void* ws, size_t ws_bytes) {
  switch (a.k) {
    case 1: return grad1d_launch_k1(a, ws, ws_bytes);
    case 2: return grad1d_launch_k2(a, ws, ws_bytes);
    case 3: return grad1d_launch_k3(a, ws, ws_bytes);
    default: return GW_ERR_INVALID;
  }
}

}  // namespace gw
