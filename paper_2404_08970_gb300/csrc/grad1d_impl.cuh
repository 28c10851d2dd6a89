// Structured 1D gradient G = c_x 1^T + 1 c_y^T - 2 D_X T D_Y on uniform grids.
//
// D_X T D_Y = h_X^k h_Y^k D~ T D~ with D~ = L + L^T (Sec. 3, eq. "Dx").  The
// paper applies L with a dynamic-programming recursion over the states
//   a_{i,r} = sum_{j<i} (i-j)^{r-1} x_j,  a_{i+1,r} = x_i + sum_{s<=r} C(r-1,s-1) a_{i,s}
// (Sec. 3, eqs. "1d y" and "1d recursive relation"), and L^T the same way
// on the reversed sequence.  Here the states are indexed from 0
// (S_r = a_{.,r+1}, r = 0..k), so S_r(pos) = sum_{q<pos} (pos-q)^r y_q.
//
// GB300 layout of the work (one read of T for the band statistics, one read
// of T and one write of G for the output):
//   k1a  per row band a (rows s_a .. s_a+R_a-1) and column p, the band
//        moments about the band's end nu_r = sum_t (R_a - t)^r T[s_a+t, p]
//        (nu_0 compensated).
//   k1b  per column, scans the band moments in float-float across bands and
//        turns them into, for every band, a degree-k polynomial Q_a,p(t) with
//        Q(t) = sum_{j < s_a} (i-j)^k x_j + sum_{j >= s_a} (j-i)^k x_j,
//        i = s_a + t.  Since L^T x = P - (-1)^k L x with
//        P_i = sum_j (j-i)^k x_j, the column transform becomes
//        (D~ x)_i = Q(t) + (1 - (-1)^k) F_t, where F_t is the recursion above
//        run inside the band from a zero state: one forward sweep per band.
//   k1c  one CTA per band streams the band's rows (TMA bulk copies into a
//        shared-memory ring), runs the column recursion on each row, applies
//        D~ along the row (the whole row is on chip) with the same identity:
//        a forward block scan of the recursion plus the row's moments, adds
//        the constant term and writes G.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "gw_common.cuh"
#include "gw_internal.h"
#include "gw_tma.cuh"

namespace gw {

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  float y = __fsub_rn(x, c);
  float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}
__device__ __forceinline__ void kahan_add(double& s, double& c, double x) {
  double y = __dsub_rn(x, c);
  double t = __dadd_rn(s, y);
  c = __dsub_rn(__dsub_rn(t, s), y);
  s = t;
}

// a * c for a float c that is exact (an integer below 2^24).
__device__ __forceinline__ ff acc_mulf(ff a, float c) { return ff_mul(a, c); }
__device__ __forceinline__ double acc_mulf(double a, double c) { return a * c; }
template <typename A> struct AccReal;
template <> struct AccReal<ff> { using type = float; };
template <> struct AccReal<double> { using type = double; };

// Shifts moments measured at a position x to position x + d (or, for moments
// of elements to the right, from x to x - d):
//   S_r <- sum_{u<=r} C(r,u) d^{r-u} S_u,
// evaluated by Horner in d (d < 2^24, so every multiplier is exact).
template <int K, typename A>
__device__ __forceinline__ void shift_acc(A (&S)[K + 1], int d) {
  using F = typename AccReal<A>::type;
  const F df = (F)d;
#pragma unroll
  for (int r = K; r >= 1; --r) {
    A acc = S[0];
#pragma unroll
    for (int u = 1; u <= r; ++u) {
      acc = acc_mulf(acc, df);
      const int c = binom(r, u);
      acc = acc_add(acc, c == 1 ? S[u] : acc_mulf(S[u], (F)c));
    }
    S[r] = acc;
  }
}

// Same shift in plain Real arithmetic (in-CTA scans; d small).
template <int K, typename Real>
__device__ __forceinline__ void shift_real(Real (&S)[K + 1], Real d) {
#pragma unroll
  for (int r = K; r >= 1; --r) {
    Real acc = S[r];
    Real dp = d;
#pragma unroll
    for (int u = r - 1; u >= 0; --u) {
      acc = fma((Real)binom(r, u) * dp, S[u], acc);
      dp *= d;
    }
    S[r] = acc;
  }
}

// One step of the paper's recursion: S(pos+1) from S(pos) and y_pos.
template <int K, typename Real>
__device__ __forceinline__ void pascal_step(Real (&S)[K + 1], Real y) {
#pragma unroll
  for (int r = K; r >= 1; --r) {
    Real acc = S[r] + y;
#pragma unroll
    for (int u = 0; u < r; ++u) acc = fma((Real)binom(r, u), S[u], acc);
    S[r] = acc;
  }
  S[0] += y;
}


// Accumulator helpers used by the row stage (float-float for float data,
// plain double for double data).
__device__ __forceinline__ ff acc_shfl_up(ff a, int d) {
  return {__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ double acc_shfl_up(double a, int d) { return __shfl_up_sync(0xffffffffu, a, d); }
__device__ __forceinline__ ff acc_shfl(ff a, int src) {
  return {__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
}
__device__ __forceinline__ double acc_shfl(double a, int src) { return __shfl_sync(0xffffffffu, a, src); }
// Exact scaling by a power of two.
__device__ __forceinline__ ff acc_pow2(ff a, float c) { return {a.hi * c, a.lo * c}; }
__device__ __forceinline__ double acc_pow2(double a, double c) { return a * c; }
__device__ __forceinline__ float acc_hi(ff a) { return a.hi; }
__device__ __forceinline__ float acc_lo(ff a) { return a.lo; }
__device__ __forceinline__ double acc_hi(double a) { return a; }
__device__ __forceinline__ double acc_lo(double) { return 0.0; }

// Shift of accumulator moments by d = 2^j * base (all powers exact).
template <int K, typename A, typename Real>
__device__ __forceinline__ void shift_acc_pow2(A (&S)[K + 1], Real d) {
#pragma unroll
  for (int r = K; r >= 1; --r) {
    A acc = S[r];
    Real dp = d;
#pragma unroll
    for (int u = r - 1; u >= 0; --u) {
      const int c = binom(r, u);
      acc = acc_add(acc, acc_pow2(c == 1 ? S[u] : acc_mulf(S[u], (typename AccReal<A>::type)c), dp));
      dp *= d;
    }
    S[r] = acc;
  }
}

// ---------------------------------------------------------------------------
// k1a: band moments.  One CTA per band covers the whole row width: thread t
// owns CPT groups of VEC consecutive columns, group g starting at column
// (g*NT + t)*VEC.  Rows are read bottom-up so that the rows the main kernel
// reads first (each band's top rows) are the most recently cached in L2.
// mu layout [band][K+2][m]: slot 0 = nu_0, slot 1 = its compensation (true
// nu_0 = slot0 + slot1), slots 2.. = nu_1..nu_K,
// nu_r = sum_t (R_a - t)^r T[s_a+t, p] (moments about the band's end).
// rowpart (exact marginals only) layout [wchunk][n][2]: (hi, lo) partial row
// sums over the 32*VEC columns of warp-chunk wchunk = g*(NT/32) + warp.
// ---------------------------------------------------------------------------
template <int K, typename Real, int VEC, int CPT>
__global__ void __launch_bounds__(1024) k1a_band_moments(const Real* __restrict__ T, int n, int m, int R,
                                                         Real* __restrict__ mu, Real* __restrict__ rowpart,
                                                         int exact) {
  const int a = blockIdx.x;
  const int s = a * R;
  const int Ra = min(R, n - s);
  const int NT = blockDim.x;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // blockIdx.y splits the row into column slices of NT*VEC*CPT columns.
  const int col0 = blockIdx.y * NT * VEC * CPT;
  const int wbase = blockIdx.y * (NT >> 5) * CPT;
  Real m0[CPT][VEC], c0[CPT][VEC], mr[CPT][K][VEC];
#pragma unroll
  for (int g = 0; g < CPT; ++g)
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      m0[g][v] = 0;
      c0[g][v] = 0;
#pragma unroll
      for (int r = 0; r < K; ++r) mr[g][r][v] = 0;
    }
#pragma unroll 2
  for (int t = Ra - 1; t >= 0; --t) {
    const Real* row = T + (size_t)(s + t) * m;
    Real x[CPT][VEC];
#pragma unroll
    for (int g = 0; g < CPT; ++g) {
      const int p0 = col0 + (g * NT + (int)threadIdx.x) * VEC;
      if (VEC > 1 && p0 + VEC <= m) {
        if constexpr (VEC == 4 && sizeof(Real) == 4) {
          float4 f = __ldg(reinterpret_cast<const float4*>(row + p0));
          x[g][0] = f.x; x[g][1] = f.y; x[g][2] = f.z; x[g][3] = f.w;
        } else if constexpr (VEC == 2 && sizeof(Real) == 8) {
          double2 d = __ldg(reinterpret_cast<const double2*>(row + p0));
          x[g][0] = d.x; x[g][1] = d.y;
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) x[g][v] = __ldg(row + p0 + v);
        }
      } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) x[g][v] = (p0 + v < m) ? __ldg(row + p0 + v) : (Real)0;
      }
    }
    const Real tr = (Real)(Ra - t);
#pragma unroll
    for (int g = 0; g < CPT; ++g)
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        kahan_add(m0[g][v], c0[g][v], x[g][v]);
        Real tp = tr;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          mr[g][r][v] = fma(tp, x[g][v], mr[g][r][v]);
          tp *= tr;
        }
      }
    if (exact) {
#pragma unroll
      for (int g = 0; g < CPT; ++g) {
        const int wchunk = wbase + g * (NT >> 5) + warp;
        if (wchunk * 32 * VEC >= m) continue;  // warp-uniform
        Real loc = 0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) loc += x[g][v];
        const size_t o = ((size_t)wchunk * n + s + t) * 2;
        if constexpr (sizeof(Real) == 4) {
          ff acc = ff_make(loc);
#pragma unroll
          for (int d = 16; d >= 1; d >>= 1) {
            ff other;
            other.hi = __shfl_xor_sync(0xffffffffu, acc.hi, d);
            other.lo = __shfl_xor_sync(0xffffffffu, acc.lo, d);
            acc = ff_add(acc, other);
          }
          if (lane == 0) {
            rowpart[o] = acc.hi;
            rowpart[o + 1] = acc.lo;
          }
        } else {
          Real acc = loc;
#pragma unroll
          for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
          if (lane == 0) {
            rowpart[o] = acc;
            rowpart[o + 1] = 0;
          }
        }
      }
    }
  }
#pragma unroll
  for (int g = 0; g < CPT; ++g)
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int p = col0 + (g * NT + (int)threadIdx.x) * VEC + v;
      if (p < m) {
        Real* base = mu + (size_t)a * (K + 2) * m + p;
        base[0] = m0[g][v];
        base[(size_t)m] = -c0[g][v];
#pragma unroll
        for (int r = 0; r < K; ++r) base[(size_t)(r + 2) * m] = mr[g][r][v];
      }
    }
}

// ---------------------------------------------------------------------------
// k1a, streamed form (float, target marginals, m a multiple of 32 up to 8192):
// the band's rows come into a shared-memory ring of kA_STAGES whole rows by
// TMA tensor copies (128-byte swizzle), bottom-up like k1a_band_moments, so
// the loads in flight no longer depend on registers.  Thread t owns the 8
// consecutive columns 8t .. 8t+7.  Same moments and layout as
// k1a_band_moments.
// ---------------------------------------------------------------------------
constexpr int kA_STAGES = 4;
constexpr int kA_VPT = 8;

template <int K>
__global__ void __launch_bounds__(1024, 1)
    k1a_band_moments_tma(const __grid_constant__ CUtensorMap tmT, int n, int m, int R, int slot_bytes,
                         int box_cols, int ncopies, float* __restrict__ mu, const float* __restrict__ rF,
                         const float* __restrict__ rG, float rc, unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  unsigned char* ring = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + (size_t)kA_STAGES * slot_bytes);
  const int a = blockIdx.x;
  const int s = a * R;
  const int Ra = min(R, n - s);
  const int tid = threadIdx.x;
  const int c0 = tid * kA_VPT;
  auto issue = [&](int j) {  // j-th row from the bottom of the band
    const int slot = j % kA_STAGES;
    mbar_arrive_expect_tx(&bars[slot], (unsigned)(m * sizeof(float)));
    for (int c = 0; c < ncopies; ++c)
      tma_load_3d(ring + (size_t)slot * slot_bytes + (size_t)c * box_cols * 128, &tmT, 0, c * box_cols,
                  s + Ra - 1 - j, &bars[slot]);
  };
  if (tid == 0) {
    for (int st = 0; st < kA_STAGES; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
    for (int j = 0; j < kA_STAGES && j < Ra; ++j) issue(j);
  }
  __syncthreads();
  float m0[kA_VPT], c0k[kA_VPT], mr[K][kA_VPT];
  // With rF set the ring holds rows of Pi: the plan's columns' potentials.
  float gp[kA_VPT];
  const bool active = c0 < m;
#pragma unroll
  for (int v = 0; v < kA_VPT; ++v) {
    m0[v] = 0.f;
    c0k[v] = 0.f;
    gp[v] = (rF && active) ? rG[c0 + v] : 0.f;
#pragma unroll
    for (int r = 0; r < K; ++r) mr[r][v] = 0.f;
  }
  for (int j = 0; j < Ra; ++j) {
    const int slot = j % kA_STAGES;
    mbar_wait_bounded(&bars[slot], (unsigned)((j / kA_STAGES) & 1), status);
    if (active) {
      float x[kA_VPT];
      lds_swz<float, kA_VPT>(ring + (size_t)slot * slot_bytes, c0, x);
      if (rF) {
        const float fi = rF[s + Ra - 1 - j];
#pragma unroll
        for (int v = 0; v < kA_VPT; ++v) x[v] = ex2(fmaf(-rc, x[v], gp[v] + fi));
      }
      const float tr = (float)(j + 1);  // R_a - t for row t = R_a - 1 - j
#pragma unroll
      for (int v = 0; v < kA_VPT; ++v) {
        kahan_add(m0[v], c0k[v], x[v]);
        float tp = tr;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          mr[r][v] = fmaf(tp, x[v], mr[r][v]);
          tp *= tr;
        }
      }
    }
    __syncthreads();  // every thread has read the slot
    if (tid == 0 && j + kA_STAGES < Ra) {
      fence_proxy_async_smem();
      issue(j + kA_STAGES);
    }
  }
  if (!active) return;
  float* base = mu + (size_t)a * (K + 2) * m + c0;
  auto put = [&](float* dst, const float (&v)[kA_VPT]) {
    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
  };
  float negc[kA_VPT];
#pragma unroll
  for (int v = 0; v < kA_VPT; ++v) negc[v] = -c0k[v];
  put(base, m0);
  put(base + (size_t)m, negc);
#pragma unroll
  for (int r = 0; r < K; ++r) put(base + (size_t)(r + 2) * m, mr[r]);
}

// ---------------------------------------------------------------------------
// k1b: carries across bands -> per-band polynomial coefficients
//   A_r(a)  = sum_{j < s_a} (s_a - j)^r x_j      (forward, exclusive)
//   Bk_r(a) = sum_{j >= s_a} (j - s_a)^r x_j     (from the band start on)
//   q_e(a)  = C(K, K-e) [A_{K-e}(a) + (-1)^e Bk_{K-e}(a)],  Q(t) = sum_e q_e t^e
// in one kernel, all in float-float (double for double data).  A block
// covers 32 columns (one per lane); its kGroups warps split the bands into
// kGroups consecutive groups:
//   1. each warp: its group's moments about the group's end;
//   2. warp 0: the exclusive prefix over the groups (A at each group's start)
//      and the column's moments about row n (all groups), via shared memory;
//   3. each warp walks its bands with A, takes Bk from the column moments,
//      writes q.
// q layout [band][K+1][m].
// ---------------------------------------------------------------------------
template <int K, typename Real>
struct K1bOps {
  using A = typename AccT<Real>::type;
  static __device__ __forceinline__ void load_mu(const Real* mu, int m, int a, int p, A (&M)[K + 1]) {
    const Real* base = mu + (size_t)a * (K + 2) * m + p;
    M[0] = acc_of(base[0], base[(size_t)m]);
#pragma unroll
    for (int r = 1; r <= K; ++r) M[r] = acc_of(base[(size_t)(r + 1) * m]);
  }
};

constexpr int kGroups = 32;

template <int K, typename Real>
__global__ void __launch_bounds__(32 * kGroups) k1b_carries(const Real* __restrict__ mu, int n, int m, int R, int B,
                                                          Real* __restrict__ q, double* __restrict__ colsum) {
  using A = typename AccT<Real>::type;
  using O = K1bOps<K, Real>;
  using F = typename AccReal<A>::type;
  __shared__ A gagg[kGroups][K + 1][32];  // group aggregates, then exclusive prefixes
  __shared__ A gtot[K + 1][32];           // the column's moments about row n
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  const int per = (B + kGroups - 1) / kGroups;
  auto group_bands = [&](int g, int& g0, int& g1) {
    g0 = min(B, g * per);
    g1 = min(B, g0 + per);
  };
  int a0, a1;
  group_bands(w, a0, a1);
  A N[K + 1];
  // 1. group aggregate about the group's end
  A FA[K + 1];
#pragma unroll
  for (int r = 0; r <= K; ++r) FA[r] = acc_zero((A*)nullptr);
  if (p < m) {
#pragma unroll 4
    for (int a = a0; a < a1; ++a) {
      const int Ra = min(R, n - a * R);
      O::load_mu(mu, m, a, p, N);  // moments about the band's end
      shift_acc<K>(FA, Ra);
#pragma unroll
      for (int r = 0; r <= K; ++r) FA[r] = acc_add(FA[r], N[r]);
    }
  }
#pragma unroll
  for (int r = 0; r <= K; ++r) gagg[w][r][lane] = FA[r];
  __syncthreads();
  // 2. warp 0: exclusive prefixes at each group's start (in place) and the
  // column total.
  if (w == 0) {
    A Nt[K + 1];
#pragma unroll
    for (int r = 0; r <= K; ++r) Nt[r] = acc_zero((A*)nullptr);
    for (int g = 0; g < kGroups; ++g) {
      int g0, g1;
      group_bands(g, g0, g1);
      const int L = g1 > g0 ? min(n, g1 * R) - g0 * R : 0;
      A ag[K + 1];
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        ag[r] = gagg[g][r][lane];
        gagg[g][r][lane] = Nt[r];
      }
      shift_acc<K>(Nt, L);
#pragma unroll
      for (int r = 0; r <= K; ++r) Nt[r] = acc_add(Nt[r], ag[r]);
    }
#pragma unroll
    for (int r = 0; r <= K; ++r) gtot[r][lane] = Nt[r];
  }
  __syncthreads();
  A Nt[K + 1], Af[K + 1];
#pragma unroll
  for (int r = 0; r <= K; ++r) {
    Nt[r] = gtot[r][lane];
    Af[r] = gagg[w][r][lane];
  }
  if (p >= m) return;
  if (colsum && w == 0) {
    if constexpr (sizeof(Real) == 4) colsum[p] = ff_to_double(Nt[0]);
    else colsum[p] = Nt[0];
  }
  // 3. walk the group's bands
#pragma unroll 4
  for (int a = a0; a < a1; ++a) {
    const int sa = a * R;
    const F dn = (F)(n - sa);
    // Moments about s_a of the whole column (Horner in n - s_a, alternating
    // signs), then Bk = those minus (-1)^u A.
    A Bk[K + 1];
#pragma unroll
    for (int u = 0; u <= K; ++u) {
      A acc = Nt[0];
#pragma unroll
      for (int w2 = 1; w2 <= u; ++w2) {
        acc = acc_mulf(acc, dn);
        const int c = binom(u, w2);
        const A term = c == 1 ? Nt[w2] : acc_mulf(Nt[w2], (F)c);
        acc = (w2 & 1) ? acc_sub(acc, term) : acc_add(acc, term);
      }
      Bk[u] = (u & 1) ? acc_add(acc, Af[u]) : acc_sub(acc, Af[u]);
    }
#pragma unroll
    for (int e = 0; e <= K; ++e) {
      const int r = K - e;
      A t = (e & 1) ? acc_sub(Af[r], Bk[r]) : acc_add(Af[r], Bk[r]);
      const int cb = binom(K, r);
      if (cb != 1) t = acc_mulf(t, (F)cb);
      q[((size_t)a * (K + 1) + e) * m + p] = (Real)acc_round(t);
    }
    const int Ra = min(R, n - a * R);
    O::load_mu(mu, m, a, p, N);
    shift_acc<K>(Af, Ra);
#pragma unroll
    for (int r = 0; r <= K; ++r) Af[r] = acc_add(Af[r], N[r]);
  }
}

// ---------------------------------------------------------------------------
// k1c: one CTA per band.  Thread `tid` owns the VPT consecutive columns
// [c0, c0 + VPT), c0 = tid*VPT.  Per row i = s_a + t:
//   y_p = Q_p(t) + c_K F_t,p                        (column transform)
//   z_p = sum_q |p-q|^K y_q                          (row transform)
// with c_K = 1 - (-1)^K.  Along the row, z at chunk offset v is the value at
// the chunk start, Zc = Al_K + Bc_K, plus a degree-K polynomial in v plus
// c_K times the recursion run inside the chunk, where Al are the moments of
// the columns left of the chunk and Bc those of the columns from the chunk on
// (same identity as the column direction).  Al and Bc come from scans of the
// chunk moments: lanes in float (in-warp partial sums), warps in float-float.
// z is kept split into the float-float Zc and a small float part, so that
// the constant term cancels against Zc in one exactly-rounded fma:
//   G = (fma(-s, Zc.hi, cx.hi) + cy.hi) + fma(-s, small, cx.lo + cy.lo).
// Rows arrive through a ring of `stages` shared-memory row buffers filled by
// 1D TMA bulk copies (or, if rows are not 16-byte aligned, by a cooperative
// copy into one buffer).
// ---------------------------------------------------------------------------
template <int K, int NT, int VPT, typename Real>
struct K1cSmem {
  using A = typename AccT<Real>::type;
  static constexpr int NW = NT / 32;
  // warp totals [2][NW][K+1] Real, then warp prefixes and suffixes [2][NW][K+1] A
  static constexpr size_t scan_bytes = sizeof(Real) * 2 * NW * (K + 1) + sizeof(A) * 2 * NW * (K + 1) + 32;
  static size_t bytes(int m_pad, int stages) {
    size_t ring = (size_t)stages * m_pad * sizeof(Real);
    ring = (ring + 15) & ~(size_t)15;
    return ring + 8 * (size_t)stages + scan_bytes + 16;
  }
};

template <int K, int NT, int VPT, typename Real>
__global__ void __launch_bounds__(NT, 1)
    k1c_grad_rows(const Real* __restrict__ T, Real* __restrict__ G, int n, int m, int R,
                  const Real* __restrict__ q, const Real* __restrict__ cxh, const Real* __restrict__ cxl,
                  const Real* __restrict__ cyh, const Real* __restrict__ cyl, Real scale, int use_tma, int stages,
                  int m_pad, unsigned* status) {
  using A = typename AccT<Real>::type;
  constexpr int NW = NT / 32;
  constexpr Real CK = (K & 1) ? (Real)2 : (Real)0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* ring = reinterpret_cast<Real*>(smem_raw);
  const size_t ring_bytes = ((size_t)stages * m_pad * sizeof(Real) + 15) & ~(size_t)15;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + ring_bytes);
  Real* wtot = reinterpret_cast<Real*>(smem_raw + ring_bytes + 8 * (size_t)stages);  // [2][NW][K+1]
  unsigned char* wpraw = reinterpret_cast<unsigned char*>(wtot + 2 * NW * (K + 1));
  A* wpre = reinterpret_cast<A*>(wpraw + ((16u - (smem_u32(wpraw) & 15u)) & 15u));

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int a = blockIdx.x;
  const int s = a * R;
  const int Ra = min(R, n - s);
  const int c0 = tid * VPT;
  const unsigned row_bytes = (unsigned)(m * sizeof(Real));

  if (use_tma) {
    if (tid == 0) {
      for (int st = 0; st < stages; ++st) mbar_init(&bars[st], 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      for (int st = 0; st < stages - 1 && st < Ra; ++st) {
        mbar_arrive_expect_tx(&bars[st], row_bytes);
        bulk_g2s(ring + (size_t)st * m_pad, T + (size_t)(s + st) * m, row_bytes, &bars[st]);
      }
    }
  }

  // Per-thread column state.
  Real qv[VPT][K + 1];
  Real cs[VPT][K + 1];  // column recursion states (odd K only)
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int p = c0 + v;
    const bool ok = p < m;
#pragma unroll
    for (int e = 0; e <= K; ++e) {
      qv[v][e] = ok ? q[((size_t)a * (K + 1) + e) * m + p] : (Real)0;
      cs[v][e] = 0;
    }
  }

  for (int t = 0; t < Ra; ++t) {
    const int i = s + t;
    int slot = 0;
    if (use_tma) {
      slot = t % stages;
      if (tid == 0) {
        const int nt = t + stages - 1;
        if (nt < Ra) {
          const int ns = nt % stages;
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&bars[ns], row_bytes);
          bulk_g2s(ring + (size_t)ns * m_pad, T + (size_t)(s + nt) * m, row_bytes, &bars[ns]);
        }
      }
      mbar_wait_bounded(&bars[slot], (unsigned)((t / stages) & 1), status);
    } else {
      const Real* src = T + (size_t)i * m;
      for (int idx = tid; idx < m; idx += NT) ring[idx] = src[idx];
      __syncthreads();
    }
    const Real* xr = ring + (size_t)slot * m_pad;

    // Column transform.
    Real y[VPT];
    const Real tr = (Real)t;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int p = c0 + v;
      const Real x = (p < m) ? xr[p] : (Real)0;
      Real Qt = qv[v][K];
#pragma unroll
      for (int e = K - 1; e >= 0; --e) Qt = fma(Qt, tr, qv[v][e]);
      if constexpr (K & 1) {
        y[v] = fma(CK, cs[v][K], Qt);
        pascal_step<K>(cs[v], x);
      } else {
        y[v] = Qt;
      }
      if (p >= m) y[v] = 0;
    }

    // Row transform, local part: forward walk inside the chunk (y[v] is
    // replaced by the local forward state, odd K only) and the chunk's
    // moments about its start (for the suffix scan).
    Real agg[K + 1], bag[K + 1];
#pragma unroll
    for (int r = 0; r <= K; ++r) {
      agg[r] = 0;
      bag[r] = 0;
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const Real yv = y[v];
      if constexpr (K & 1) y[v] = agg[K];
      pascal_step<K>(agg, yv);
      Real pw = yv;
      bag[0] += yv;
#pragma unroll
      for (int r = 1; r <= K; ++r) {
        pw *= (Real)v;
        bag[r] += pw;
      }
    }
    // Lane scans (float): forward inclusive moments about my chunk end,
    // backward inclusive moments about my chunk start.
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Real o[K + 1], ob[K + 1];
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        o[r] = __shfl_up_sync(0xffffffffu, agg[r], d);
        ob[r] = __shfl_down_sync(0xffffffffu, bag[r], d);
      }
      shift_real<K>(o, (Real)(d * VPT));
      shift_real<K>(ob, (Real)(d * VPT));
      if (lane >= d) {
#pragma unroll
        for (int r = 0; r <= K; ++r) agg[r] += o[r];
      }
      if (lane + d < 32) {
#pragma unroll
        for (int r = 0; r <= K; ++r) bag[r] += ob[r];
      }
    }
    Real ex[K + 1];
#pragma unroll
    for (int r = 0; r <= K; ++r) {
      ex[r] = __shfl_up_sync(0xffffffffu, agg[r], 1);
      if (lane == 0) ex[r] = 0;
    }
    if (lane == 31) {
#pragma unroll
      for (int r = 0; r <= K; ++r) wtot[warp * (K + 1) + r] = agg[r];
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r <= K; ++r) wtot[(NW + warp) * (K + 1) + r] = bag[r];
    }
    __syncthreads();
    // Warp 0 scans the warp totals in float-float: exclusive forward prefix
    // (about each warp's start) and exclusive backward suffix (about the
    // start of the next warp).
    if (warp == 0) {
      A W[K + 1], V[K + 1];
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        W[r] = (lane < NW) ? acc_of(wtot[lane * (K + 1) + r]) : acc_zero((A*)nullptr);
        V[r] = (lane < NW) ? acc_of(wtot[(NW + lane) * (K + 1) + r]) : acc_zero((A*)nullptr);
      }
#pragma unroll
      for (int d = 1; d < NW; d <<= 1) {
        A o[K + 1], ob[K + 1];
#pragma unroll
        for (int r = 0; r <= K; ++r) {
          o[r] = acc_shfl_up(W[r], d);
          ob[r] = acc_shfl_down(V[r], d);
        }
        shift_acc_pow2<K>(o, (Real)(d * 32 * VPT));
        shift_acc_pow2<K>(ob, (Real)(d * 32 * VPT));
        if (lane >= d) {
#pragma unroll
          for (int r = 0; r <= K; ++r) W[r] = acc_add(W[r], o[r]);
        }
        if (lane + d < NW) {
#pragma unroll
          for (int r = 0; r <= K; ++r) V[r] = acc_add(V[r], ob[r]);
        }
      }
      A P[K + 1], S2[K + 1];
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        P[r] = acc_shfl_up(W[r], 1);
        S2[r] = acc_shfl_down(V[r], 1);
        if (lane == 0) P[r] = acc_zero((A*)nullptr);
        if (lane >= NW - 1) S2[r] = acc_zero((A*)nullptr);
      }
      if (lane < NW) {
#pragma unroll
        for (int r = 0; r <= K; ++r) {
          wpre[lane * (K + 1) + r] = P[r];
          wpre[(NW + lane) * (K + 1) + r] = S2[r];
        }
      }
    }
    __syncthreads();
    // Left moments about my chunk start (Al) and moments of everything from
    // my chunk start on, about my chunk start (Bc): both positive sums.
    A Al[K + 1], Bc[K + 1];
#pragma unroll
    for (int r = 0; r <= K; ++r) {
      Al[r] = wpre[warp * (K + 1) + r];
      Bc[r] = wpre[(NW + warp) * (K + 1) + r];
    }
    shift_acc<K>(Al, lane * VPT);
    shift_acc<K>(Bc, (32 - lane) * VPT);
#pragma unroll
    for (int r = 0; r <= K; ++r) {
      Al[r] = acc_add(Al[r], acc_of(ex[r]));
      Bc[r] = acc_add(Bc[r], acc_of(bag[r]));
    }
    // z at chunk offset v: Zc + sum_{e>=1} s_e v^e + c_K F_local(v), with
    // s_e = C(K, K-e) [Al_{K-e} + (-1)^e Bc_{K-e}] and Zc = Al_K + Bc_K.
    const A Zc = acc_add(Al[K], Bc[K]);
    Real se[K + 1];
    se[0] = 0;
#pragma unroll
    for (int e = 1; e <= K; ++e) {
      const int u = K - e;
      A t2 = (e & 1) ? acc_sub(Al[u], Bc[u]) : acc_add(Al[u], Bc[u]);
      se[e] = (Real)binom(K, u) * (Real)acc_round(t2);
    }
    const Real zc_hi = (Real)acc_hi(Zc);
    const Real zc_lo = (Real)acc_lo(Zc);

    // Epilogue.
    const Real cxi_h = cxh[i];
    const Real cxi_l = cxl[i];
    const Real big0 = fma(-scale, zc_hi, cxi_h);
    Real* grow = G + (size_t)i * m + c0;
    Real out[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int p = c0 + v;
      const Real vv = (Real)v;
      Real small = se[K];
#pragma unroll
      for (int e = K - 1; e >= 1; --e) small = fma(small, vv, se[e]);
      small = fma(small, vv, zc_lo);
      if constexpr (K & 1) small = fma(CK, y[v], small);
      const Real cyh_p = (p < m) ? __ldg(cyh + p) : (Real)0;
      const Real cyl_p = (p < m) ? __ldg(cyl + p) : (Real)0;
      out[v] = (big0 + cyh_p) + fma(-scale, small, cxi_l + cyl_p);
    }
    const bool vec_ok = (c0 + VPT <= m) && ((((uintptr_t)grow) & 15) == 0);
    if (vec_ok) {
      if constexpr (sizeof(Real) == 4 && VPT % 4 == 0) {
#pragma unroll
        for (int v = 0; v < VPT; v += 4)
          *reinterpret_cast<float4*>(grow + v) = make_float4(out[v], out[v + 1], out[v + 2], out[v + 3]);
      } else if constexpr (sizeof(Real) == 8 && VPT % 2 == 0) {
#pragma unroll
        for (int v = 0; v < VPT; v += 2) *reinterpret_cast<double2*>(grow + v) = make_double2(out[v], out[v + 1]);
      } else {
#pragma unroll
        for (int v = 0; v < VPT; ++v) grow[v] = out[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < VPT; ++v)
        if (c0 + v < m) grow[v] = out[v];
    }
    if (!use_tma) __syncthreads();
  }
}

}  // namespace gw

#include "grad1d_fast.cuh"

namespace gw {

// ---------------------------------------------------------------------------
// Host launcher for one exponent K.
// ---------------------------------------------------------------------------
struct K1Layout {
  Bands bands;
  size_t mu_off, q_off, rowpart_off, r_off, c_off, cx_off, cy_off, partx_off,
      party_off, end;
  int nwchunks;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline K1Layout k1_layout(int n, int m, int k, size_t real_bytes, int target_bands) {
  K1Layout L;
  L.bands = choose_bands(n, target_bands);
  const int B = L.bands.B;
  L.nwchunks = (m + 31) / 32;  // warp chunks of the narrowest (VEC = 1) k1a layout
  size_t off = 0;
  L.mu_off = off;      off = align_up(off + (size_t)B * (k + 2) * m * real_bytes, 256);
  L.q_off = off;       off = align_up(off + (size_t)B * (k + 1) * m * real_bytes, 256);

  L.rowpart_off = off; off = align_up(off + (size_t)L.nwchunks * n * 2 * real_bytes, 256);
  L.r_off = off;       off = align_up(off + (size_t)n * 8, 256);
  L.c_off = off;       off = align_up(off + (size_t)m * 8, 256);
  L.cx_off = off;      off = align_up(off + (size_t)2 * n * real_bytes, 256);  // hi, lo
  L.cy_off = off;      off = align_up(off + (size_t)2 * m * real_bytes, 256);
  L.partx_off = off;   off = align_up(off + marg_part_doubles(n, k) * 8, 256);
  L.party_off = off;   off = align_up(off + marg_part_doubles(m, 3) * 8, 256);
  L.end = off;
  return L;
}

__global__ void rowsum_finish(const void* rowpart, int nchunks, int n, int is_f32, double* r);

template <int K, int NT, int VPT, typename Real>
int launch_k1c(const Grad1DArgs& g, const K1Layout& L, char* ws, int use_tma, cudaStream_t st) {
  const int m_pad = (int)align_up((size_t)g.m, 4);
  int stages = 1;
  if (use_tma) {
    size_t row = (size_t)m_pad * sizeof(Real);
    stages = (int)std::min<size_t>(4, (size_t)(190 * 1024) / row);
    if (stages < 2) {
      use_tma = 0;
      stages = 1;
    }
  }
  const size_t smem = K1cSmem<K, NT, VPT, Real>::bytes(m_pad, stages);
  auto kern = k1c_grad_rows<K, NT, VPT, Real>;
  TraceScope ts(g.tracer, "k1c_grad_rows", st);
  if (!allow_dynamic_smem((const void*)kern, smem))
    return GW_ERR_CUDA;
  const Real scale = (Real)(2.0 * g.out_scale * std::pow(g.hx, g.k) * std::pow(g.hy, g.k));
  const Real* cx = (const Real*)(ws + L.cx_off);
  const Real* cy = (const Real*)(ws + L.cy_off);
  kern<<<L.bands.B, NT, smem, st>>>((const Real*)g.T, (Real*)g.G, g.n, g.m, L.bands.R,
                                     (const Real*)(ws + L.q_off), cx, cx + g.n, cy, cy + g.m, scale, use_tma,
                                     stages, m_pad, g.status);
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

template <int KX, int K, int NW, int VPT, typename Real, bool REGEN>
int launch_k1c_fast_as(const Grad1DArgs& g, const K1Layout& L, char* ws, cudaStream_t st) {
  CUtensorMap tm, tmg;
  memset(&tm, 0, sizeof tm);
  memset(&tmg, 0, sizeof tmg);
  int box_cols = 0;
  const int use_tma = ((((uintptr_t)g.T) & 15) == 0) && encode_rows_tmap(&tm, g.T, g.n, g.m, sizeof(Real), &box_cols);
  // G leaves by one tensor store per warp segment (32 VPT reals) when its
  // rows fit the same 128-byte-chunk tensor shape.
  const int seg_chunks = 32 * VPT * (int)sizeof(Real) / 128;
  // The segments must start on 1024-byte boundaries of the staging buffer so
  // that the swizzle pattern (address bits 4-9) is the staging layout's.
  const int use_tma_store = use_tma && seg_chunks % 8 == 0 && ((((uintptr_t)g.G) & 15) == 0) &&
                            (g.m * (int)sizeof(Real)) % 128 == 0 &&
                            encode_rows_tmap_box(&tmg, g.G, g.n, g.m, sizeof(Real), std::min(seg_chunks, g.m * (int)sizeof(Real) / 128));
  const int cover = 32 * NW * VPT;
  const int vec_bytes = (int)align_up((size_t)cover * sizeof(Real), 1024);
  const int slot_bytes = vec_bytes;
  int stages = 2;
  const int fl_bytes = (int)FastSmem<K, NW, VPT, Real>::fl_bytes;
  if (use_tma) stages = std::max(2, std::min(4, (200 * 1024 - 3 * vec_bytes - fl_bytes) / slot_bytes));
  const size_t smem = FastSmem<K, NW, VPT, Real>::bytes(slot_bytes, vec_bytes, stages);
  auto kern = k1c_fast_rows<KX, K, NW, VPT, Real, REGEN>;
  TraceScope ts(g.tracer, "k1c_fast_rows", st);
  if (!allow_dynamic_smem((const void*)kern, smem))
    return GW_ERR_CUDA;
  const Real scale = (Real)(2.0 * g.out_scale * std::pow(g.hx, KX) * std::pow(g.hy, K));
  const Real* cx = (const Real*)(ws + L.cx_off);
  const Real* cy = (const Real*)(ws + L.cy_off);
  const Real* rF = nullptr;
  const Real* rG = nullptr;
  if constexpr (REGEN) {
    rF = g.regen_F;
    rG = g.regen_G;
  }
  kern<<<L.bands.B, 32 * (NW + 1), smem, st>>>(tm, tmg, use_tma_store, (const Real*)g.T, (Real*)g.G, g.n, g.m,
                                                L.bands.R,
                                                (const Real*)(ws + L.q_off), cx, cx + g.n, cy, cy + g.m, scale,
                                                use_tma, stages, slot_bytes, vec_bytes, box_cols, 1, rF, rG,
                                                (Real)g.regen_c, g.status);
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

template <int KX, int K, int NW, int VPT, typename Real>
int launch_k1c_fast(const Grad1DArgs& g, const K1Layout& L, char* ws, cudaStream_t st) {
  if constexpr (sizeof(Real) == 4) {
    if (g.regen_F) return launch_k1c_fast_as<KX, K, NW, VPT, Real, true>(g, L, ws, st);
  }
  return launch_k1c_fast_as<KX, K, NW, VPT, Real, false>(g, L, ws, st);
}

template <int K, typename Real, int VEC, int CPT>
void launch_k1a(const Grad1DArgs& g, int B, int R, Real* mu, Real* rowpart, cudaStream_t st) {
  int nt = (g.m + VEC * CPT - 1) / (VEC * CPT);
  nt = std::min(1024, (nt + 31) / 32 * 32);
  dim3 grid(B, 1);
  k1a_band_moments<K, Real, VEC, CPT><<<grid, nt, 0, st>>>((const Real*)g.T, g.n, g.m, R, mu, rowpart, g.exact);
}

// Constant terms c_x (exponent 2 KX) and c_y (exponent 2 KY) as hi/lo
// pairs on `st`; one launch pair for equal exponents, one per vector else.
template <int KX, int KY>
int const_terms(const Grad1DArgs& g, const double* wx, const double* wy, char* ws, const K1Layout& L, int dt,
                cudaStream_t st) {
  const double fx = std::pow(g.hx, 2 * KX) * g.out_scale, fy = std::pow(g.hy, 2 * KY) * g.out_scale;
  if constexpr (KX == KY)
    return marg_const2_launch(wx, g.n, fx, ws + L.cx_off, wy, g.m, fy, ws + L.cy_off, KX, dt,
                              (double*)(ws + L.partx_off), st, g.tracer);
  int rc = marg_const_launch(wx, g.n, KX, fx, ws + L.cx_off, dt, (double*)(ws + L.partx_off), st, g.tracer);
  if (rc != GW_OK) return rc;
  return marg_const_launch(wy, g.m, KY, fy, ws + L.cy_off, dt, (double*)(ws + L.party_off), st, g.tracer);
}

// KX: the exponent of X's distance (column transform, band moments, c_x);
// KY: Y's (row transform, c_y).  Mixed exponents run the warp-specialised
// row kernel only (KX, KY <= 2, rows of at most 8192 columns).
template <int KX, typename Real, int KY = KX>
int grad1d_launch_typed(const Grad1DArgs& g, void* wsv, size_t ws_bytes) {
  const int n = g.n, m = g.m;
  const K1Layout L = k1_layout(n, m, KX, sizeof(Real), g.num_sms);
  if (L.end > ws_bytes) return GW_ERR_OOM;
  char* ws = (char*)wsv;
  cudaStream_t st = g.stream;
  const int B = L.bands.B, R = L.bands.R;
  Real* mu = (Real*)(ws + L.mu_off);
  Real* rowpart = (Real*)(ws + L.rowpart_off);

  // With target marginals the constant terms do not depend on T: given a
  // side stream, they run there concurrently with k1b.
  const int dt = sizeof(Real) == 4 ? GW_F32 : GW_F64;
  const bool overlap = !g.exact && g.side && g.ev_fork && g.ev_join;
  auto fork_consts = [&]() -> int {
    if (cudaEventRecord(g.ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(g.side, g.ev_fork, 0) != cudaSuccess)
      return GW_ERR_CUDA;
    int rc = const_terms<KX, KY>(g, g.u, g.v, ws, L, dt, g.side);
    if (rc != GW_OK) return rc;
    if (cudaEventRecord(g.ev_join, g.side) != cudaSuccess) return GW_ERR_CUDA;
    return GW_OK;
  };

  // k1a: VEC columns per vector load, CPT column groups per thread.
  const bool vec_ok = (m % 4 == 0) && ((((uintptr_t)g.T) & 15) == 0);
  int vec_used = 1;
  {
    TraceScope ts(g.tracer, "k1a_band_moments", st);
    bool done = false;
    if constexpr (sizeof(Real) == 4) {
      // Streamed form: target marginals (no row partials), m a multiple of 32
      // up to 1024 threads x 8 columns, a row tensor map for T.
      if (!g.exact && m % 32 == 0 && m <= 1024 * kA_VPT && vec_ok) {
        CUtensorMap tm;
        memset(&tm, 0, sizeof tm);
        int box_cols = 0;
        if (encode_rows_tmap(&tm, g.T, n, m, 4, &box_cols)) {
          const int slot_bytes = (int)align_up((size_t)m * 4, 1024);
          const size_t smem = 1024 + (size_t)kA_STAGES * slot_bytes + 8 * kA_STAGES;
          auto kern = k1a_band_moments_tma<KX>;
          if (allow_dynamic_smem((const void*)kern, smem)) {
            const int nt = std::max(32, (m / kA_VPT + 31) / 32 * 32);
            kern<<<B, nt, smem, st>>>(tm, n, m, R, slot_bytes, box_cols, (m / 32) / box_cols, (float*)mu,
                                      g.regen_F, g.regen_G, g.regen_c, g.status);
            done = true;
          }
        }
      }
    }
    if (!done && g.regen_F) {
      note_failure("forming T from Pi needs the TMA-fed band-moment pass (float, target marginals, m a multiple "
                   "of 32 up to 8192)");
      return GW_ERR_INVALID;
    }
    if (done) {
    } else if constexpr (sizeof(Real) == 4) {
      if (vec_ok) {
        vec_used = 4;
        if (m <= 4096) launch_k1a<KX, Real, 4, 1>(g, B, R, mu, rowpart, st);
        else if (m <= 8192) launch_k1a<KX, Real, 4, 2>(g, B, R, mu, rowpart, st);
        else launch_k1a<KX, Real, 4, 4>(g, B, R, mu, rowpart, st);
      } else {
        if (m <= 1024) launch_k1a<KX, Real, 1, 1>(g, B, R, mu, rowpart, st);
        else if (m <= 4096) launch_k1a<KX, Real, 1, 4>(g, B, R, mu, rowpart, st);
        else launch_k1a<KX, Real, 1, 16>(g, B, R, mu, rowpart, st);
      }
    } else {
      if (vec_ok) {
        vec_used = 2;
        if (m <= 2048) launch_k1a<KX, Real, 2, 1>(g, B, R, mu, rowpart, st);
        else if (m <= 8192) launch_k1a<KX, Real, 2, 4>(g, B, R, mu, rowpart, st);
        else launch_k1a<KX, Real, 2, 8>(g, B, R, mu, rowpart, st);
      } else {
        if (m <= 1024) launch_k1a<KX, Real, 1, 1>(g, B, R, mu, rowpart, st);
        else if (m <= 4096) launch_k1a<KX, Real, 1, 4>(g, B, R, mu, rowpart, st);
        else launch_k1a<KX, Real, 1, 16>(g, B, R, mu, rowpart, st);
      }
    }
  }
  if (cudaPeekAtLastError() != cudaSuccess) return GW_ERR_CUDA;
  // Forked after k1a, which streams T on every SM: the constant terms then
  // share the GPU with k1b's second wave of blocks instead (172 against 174 us
  // per 8192^2 gradient when forked before k1a).
  if (overlap) {
    int rc = fork_consts();
    if (rc != GW_OK) return rc;
  }
  const int nchunks = (m + 32 * vec_used - 1) / (32 * vec_used);

  // k1b
  double* r = (double*)(ws + L.r_off);
  double* c = (double*)(ws + L.c_off);
  {
    TraceScope ts(g.tracer, "k1b_band_carries", st);
    k1b_carries<KX, Real><<<(m + 31) / 32, 32 * kGroups, 0, st>>>(mu, n, m, R, B, (Real*)(ws + L.q_off),
                                                                g.exact ? c : nullptr);
  }
  if (cudaPeekAtLastError() != cudaSuccess) return GW_ERR_CUDA;

  // Constant terms (hi, lo pairs).
  const double* wx = g.u;
  const double* wy = g.v;
  if (g.exact) {
    TraceScope ts(g.tracer, "rowsum_finish", st);
    rowsum_finish<<<(n + 255) / 256, 256, 0, st>>>(rowpart, nchunks, n, sizeof(Real) == 4, r);
    wx = r;
    wy = c;
  }
  if (overlap) {
    if (cudaStreamWaitEvent(st, g.ev_join, 0) != cudaSuccess) return GW_ERR_CUDA;
  } else {
    int rc = const_terms<KX, KY>(g, wx, wy, ws, L, dt, st);
    if (rc != GW_OK) return rc;
  }

  // k1c
  if constexpr (KX <= 2 && KY <= 2) {
    if (!g.force_generic) {
      if constexpr (sizeof(Real) == 4) {
        if (m <= 512) return launch_k1c_fast<KX, KY, 4, 4, Real>(g, L, ws, st);
        if (m <= 1024) return launch_k1c_fast<KX, KY, 8, 4, Real>(g, L, ws, st);
        if (m <= 2048) return launch_k1c_fast<KX, KY, 8, 8, Real>(g, L, ws, st);
        if (m <= 4096) return launch_k1c_fast<KX, KY, 16, 8, Real>(g, L, ws, st);
        if (m <= 8192) return launch_k1c_fast<KX, KY, 16, 16, Real>(g, L, ws, st);
      } else {
        if (m <= 1024) return launch_k1c_fast<KX, KY, 8, 4, Real>(g, L, ws, st);
        if (m <= 4096) return launch_k1c_fast<KX, KY, 16, 8, Real>(g, L, ws, st);
      }
    }
  }
  if (g.regen_F) {
    note_failure("forming T from Pi needs the warp-specialised row kernel (float, k <= 2, m <= 8192)");
    return GW_ERR_INVALID;
  }
  if constexpr (KX != KY) {
    note_failure("mixed distance exponents need rows of at most 8192 columns (4096 in double)");
    return GW_ERR_INVALID;
  } else {
  constexpr int K = KX;
  const int use_tma = ((m * sizeof(Real)) % 16 == 0) && ((((uintptr_t)g.T) & 15) == 0);
  if constexpr (sizeof(Real) == 4) {
    if (m <= 512) return launch_k1c<K, 128, 4, Real>(g, L, ws, use_tma, st);
    if (m <= 1024) return launch_k1c<K, 256, 4, Real>(g, L, ws, use_tma, st);
    if (m <= 2048) return launch_k1c<K, 256, 8, Real>(g, L, ws, use_tma, st);
    if (m <= 4096) return launch_k1c<K, 512, 8, Real>(g, L, ws, use_tma, st);
    if (m <= 8192) return launch_k1c<K, 512, 16, Real>(g, L, ws, use_tma, st);
    return launch_k1c<K, 1024, 16, Real>(g, L, ws, use_tma, st);
  } else {
    if (m <= 1024) return launch_k1c<K, 256, 4, Real>(g, L, ws, use_tma, st);
    if (m <= 4096) return launch_k1c<K, 512, 8, Real>(g, L, ws, use_tma, st);
    return launch_k1c<K, 1024, 16, Real>(g, L, ws, use_tma, st);
  }
  }
}

}  // namespace gw
