// Entropic mirror descent for 1D grids: log-domain Sinkhorn on a stored cost
// Pi, the plan, and the solve statistics.
//
// Mirror descent with tau = eps (Sec. 2.1, eq. "GW sinkhorn" and the Remark
// on tau = eps) solves, at every outer step, the entropic OT problem whose
// cost is Pi = 2 theta G(T) + (1 - theta) C o C (Remark "FGW"), then replaces
// T by that problem's plan T_ip = exp((f_i + g_p - Pi_ip) / eps).  The inner
// Sinkhorn iterations update f then g (log-sum-exp along rows, then columns)
// from f = g = 0, for a fixed count.
//
// Arithmetic is in base 2: F = f log2(e) / eps, G = g log2(e) / eps and
// c = log2(e) / eps, so a plan entry is 2^(F_i + G_p - c Pi_ip) and every
// exponential is one exp2.  One pass over Pi per iteration:
//   sk_pass  one CTA per band of rows streams the band's rows of Pi (TMA
//            ring).  Per row: S_i = sum_p 2^(F_i + G_p - c Pi_ip) (previous
//            F as reference; after a column update every term is <= v_p), the
//            new F_i = F_i + log2 u_i - log2 S_i; then, per column, the band's
//            partial sum of 2^(F_i + G_p - c Pi_ip) with the new F (every term
//            <= u_i).
//   sk_cols  per column: sums the band partials (FP64 combine) into the new
//            G_p.  A column whose total underflows (a cold start far from the
//            fixed point) is recomputed over all rows with a running max.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "gw_common.cuh"
#include "gw_internal.h"

namespace gw {

__device__ __forceinline__ float lg2(float x) { return log2f(x); }
__device__ __forceinline__ double lg2(double x) { return log2(x); }

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
template <typename Real>
__device__ __forceinline__ Real warp_max(Real x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Pairwise sums (short dependency chains; a fixed order, so results do not
// depend on scheduling).
template <int N, typename Real>
__device__ __forceinline__ Real tree_sum(const Real (&x)[N]) {
  Real t[N];
#pragma unroll
  for (int v = 0; v < N; ++v) t[v] = x[v];
#pragma unroll
  for (int w = 1; w < N; w *= 2)
#pragma unroll
    for (int v = 0; v + w < N; v += 2 * w) t[v] += t[v + w];
  return t[0];
}
// p 16-byte aligned (shared memory): read with 16-byte loads.
template <int N, typename Real>
__device__ __forceinline__ Real tree_sum_smem(const Real* p) {
  constexpr int PER = 16 / sizeof(Real);
  Real t[N];
  if constexpr (N % PER == 0) {
#pragma unroll
    for (int j = 0; j < N / PER; ++j) {
      const float4 q = reinterpret_cast<const float4*>(p)[j];
      const Real* e = reinterpret_cast<const Real*>(&q);
#pragma unroll
      for (int w = 0; w < PER; ++w) t[j * PER + w] = e[w];
    }
  } else {
#pragma unroll
    for (int v = 0; v < N; ++v) t[v] = p[v];
  }
  return tree_sum<N>(t);
}

// A row or column sum below this is redone with a max shift.  In FP32 the
// exp2 results below 2^-126 are flushed, so a sum of up to 2^20 terms above
// 1e-24 is short by at most 2^20 * 2^-126 / 1e-24 ~ 1e-8 of itself.
template <typename Real> __device__ __forceinline__ Real tiny_sum();
template <> __device__ __forceinline__ float tiny_sum<float>() { return 1e-24f; }
template <> __device__ __forceinline__ double tiny_sum<double>() { return 1e-250; }

// ---------------------------------------------------------------------------
// Row streaming.  Rows of Pi are brought into a shared-memory ring with 1D
// bulk copies (cp.async.bulk) completing on mbarriers.  A copy must start and
// end on 16-byte boundaries, so row i is copied from the 16-byte boundary at
// or below its first byte to the boundary at or above its end, and its
// element p sits at index off + p of the slot (off < 16 / sizeof(Real)); any
// row length works.  The copies may read up to 15 bytes past the end of Pi,
// which lies inside the workspace.
// ---------------------------------------------------------------------------
struct RowGeom {
  int slot_bytes, stages;
};

template <typename Real>
__device__ __forceinline__ void row_span(const Real* Pi, int m, int row, const char** src, unsigned* bytes,
                                         int* off) {
  const size_t start = (size_t)row * (size_t)m * sizeof(Real);
  const size_t a0 = start & ~(size_t)15;
  const size_t a1 = (start + (size_t)m * sizeof(Real) + 15) & ~(size_t)15;
  *src = reinterpret_cast<const char*>(Pi) + a0;
  *bytes = (unsigned)(a1 - a0);
  *off = (int)((start - a0) / sizeof(Real));
}

// Column ownership in the row kernels: value v = j * PER + e of thread t
// (PER = 16 / sizeof(Real)) is column col_of(t, v) = PER * (j * NT + t) + e,
// so the j-th 16-byte load of a warp reads 512 contiguous bytes (no bank
// conflicts without a swizzle) and every thread's columns are interleaved
// across the row.
template <typename Real>
__host__ __device__ __forceinline__ int col_of(int t, int v, int NT) {
  constexpr int PER = 16 / sizeof(Real);
  return PER * ((v / PER) * NT + t) + v % PER;
}

// x[v] = row[col_of(t, v)] by 16-byte loads (two per group when the row's
// start is not 16-byte aligned).  A 16-byte group that starts at or past
// column m is not read (zeros); the group straddling m reads up to PER - 1
// values past the row, and the unaligned form up to one group more, inside
// the slot's slack (finite, see sk_pass).  `row` is derived from the shared
// array.
template <int VPT, int NT, typename Real>
__device__ __forceinline__ void load_vals(const Real* row, int tid, int m, Real (&x)[VPT]) {
  constexpr int PER = 16 / sizeof(Real);
  static_assert(VPT % PER == 0, "VPT must be a multiple of the 16-byte vector");
  if ((smem_u32(row) & 15u) == 0) {
#pragma unroll
    for (int j = 0; j < VPT / PER; ++j) {
      const bool in = PER * (j * NT + tid) < m;
      const float4 q = in ? reinterpret_cast<const float4*>(row)[j * NT + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
      const Real* e = reinterpret_cast<const Real*>(&q);
#pragma unroll
      for (int w = 0; w < PER; ++w) x[j * PER + w] = e[w];
    }
  } else {
    // The row starts `off` elements into a 16-byte group of the slot: each
    // 16-byte group of the row spans two aligned slot groups, read whole
    // (consecutive lanes read consecutive groups, so no bank conflicts) and
    // recombined with the row-uniform shift.
    const uint32_t mis = smem_u32(row) & 15u;
    const float4* base = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(row) - mis);
    const int off = (int)(mis / sizeof(Real));
#pragma unroll
    for (int j = 0; j < VPT / PER; ++j) {
      const int q = j * NT + tid;
      Real* o = x + j * PER;
      if (PER * q < m) {
        const float4 a4 = base[q], b4 = base[q + 1];
        const Real* A = reinterpret_cast<const Real*>(&a4);
        const Real* B = reinterpret_cast<const Real*>(&b4);
        if constexpr (PER == 4) {
          if (off == 1) {
            o[0] = A[1]; o[1] = A[2]; o[2] = A[3]; o[3] = B[0];
          } else if (off == 2) {
            o[0] = A[2]; o[1] = A[3]; o[2] = B[0]; o[3] = B[1];
          } else {
            o[0] = A[3]; o[1] = B[0]; o[2] = B[1]; o[3] = B[2];
          }
        } else {
          o[0] = A[1];
          o[1] = B[0];
        }
      } else {
#pragma unroll
        for (int w = 0; w < PER; ++w) o[w] = (Real)0;
      }
    }
  }
}

// One problem of a (possibly batched) launch: its cost matrix, potentials,
// outputs and row-band layout.  Launches take up to MAXP of these as one
// __grid_constant__ parameter block; blocks are numbered across the problems.
template <typename Real>
struct SkProb {
  RowGeom geo;
  const Real* Pi;
  const Real* lu;  // log2 u
  const Real* lv;  // log2 v
  Real* F;
  Real* G;
  Real* part;           // [B][m] column partials of one Sinkhorn pass
  Real* T;              // plan output
  const double* u;      // row targets (plan statistics)
  double* colpart;      // [B][m] plan column sums
  double* cta_stats;    // [B][2] entropy and row-error partials
  int n, m, R, B;
  Real c;
  Real kappa;  // unbalanced GW: new potentials = kappa * balanced update (1 when balanced)
};
template <typename Real, int MAXP>
struct SkBatch {
  SkProb<Real> p[MAXP];
  int block0[MAXP + 1];  // first block of each problem; block0[count] = grid size
  int count;
};
template <typename Real, int MAXP>
__device__ __forceinline__ int batch_problem(const SkBatch<Real, MAXP>& P) {
  int pi = 0;
  while (pi + 1 < P.count && (int)blockIdx.x >= P.block0[pi + 1]) ++pi;
  return pi;
}

// r = 2^lu / S: the factor that turns the row pass's exponentials into the
// new plan's entries (float: hardware exp2 and a correctly rounded
// reciprocal, about 2 ulp in all; double: exact library operations).
__device__ __forceinline__ float scale_of(float lu, float S) { return ex2(lu) * __frcp_rn(S); }
__device__ __forceinline__ double scale_of(double lu, double S) { return exp2(lu) / S; }

// Shared memory of sk_pass (128-byte aligned base):
//   ring [NG][stages][slot_bytes] (reused at the end for the groups' column
//   sums, [NG][cover] Real) | red [NG][2][NW] Real | sfb [NG][NW] Real |
//   Fold, LU [R] Real | full [NG][stages] mbarriers | (VPT >= kGvSmemVpt) the
//   columns' potentials G [cover] Real, 16-byte aligned.
// With 32 values per thread the column potentials do not fit in the register
// budget of a 512-thread block (128 per thread) beside the row values and the
// column sums; they are read from shared memory with the row's 16-byte loads.
constexpr int kGvSmemVpt = 32;
template <int NW, int VPT, int NG, typename Real>
size_t pass_smem_bytes(const RowGeom& g, int R) {
  const size_t ring = std::max((size_t)NG * g.stages * g.slot_bytes, (size_t)NG * 32 * NW * VPT * sizeof(Real));
  const size_t gvs = VPT >= kGvSmemVpt ? 16 + (size_t)32 * NW * VPT * sizeof(Real) : 0;
  return 128 + ring + sizeof(Real) * (3 * NG * NW + 2 * (size_t)R) + 16 + 8 * (size_t)NG * g.stages + gvs;
}
// Shared memory of sk_plan: ring | full [stages] mbarriers.
inline size_t plan_smem_bytes(const RowGeom& g) { return 128 + (size_t)g.stages * g.slot_bytes + 8 * g.stages + 16; }

// Barrier of the NW warps of row group g (named barrier 1 + g; a group of
// one warp needs only a warp barrier).
template <int NW>
__device__ __forceinline__ void group_sync(int g) {
  if constexpr (NW == 1) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(32 * NW) : "memory");
  }
}

// Row sum out of range: redo the row from the ring with a max shift,
// M = max_p e_p, S2 = sum_p 2^(e_p - M), e = F_old + G - c Pi (all threads of
// the row group call it for the same row; padded columns have G = -inf).
// Returns the new potential and adds the row's plan entries to acc.  The
// row is read again from the ring, so nothing of the row pass stays live
// across the group barrier.
template <int NW, int VPT, typename Real, typename GvAt>
__device__ __forceinline__ Real row_redo(const Real* row, int gt, int g, int m, Real c, GvAt Gv,
                                         Real Fo, Real lut, Real kappa, Real (&acc)[VPT], Real* sfb) {
  const int lane = gt & 31, wig = gt >> 5;
  Real x[VPT];
  load_vals<VPT, 32 * NW>(row, gt, m, x);
  Real e[VPT];
  Real lm = -INFINITY;
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    e[v] = fma(-c, x[v], Gv(v) + Fo);
    lm = fmax(lm, e[v]);
  }
  lm = warp_max(lm);
  if (lane == 0) sfb[wig] = lm;
  group_sync<NW>(g);
  Real M = -INFINITY;
#pragma unroll
  for (int q = 0; q < NW; ++q) M = fmax(M, sfb[q]);
  Real s2 = 0;
#pragma unroll
  for (int v = 0; v < VPT; ++v) s2 += ex2(e[v] - M);
  s2 = warp_sum(s2);
  group_sync<NW>(g);
  if (lane == 0) sfb[wig] = s2;
  group_sync<NW>(g);
  Real S2 = 0;
#pragma unroll
  for (int q = 0; q < NW; ++q) S2 += sfb[q];
  Real Fn = Fo + lut - (M + lg2(S2));
  if (kappa != (Real)1) Fn *= kappa;
#pragma unroll
  for (int v = 0; v < VPT; ++v) acc[v] += ex2(Fn + e[v] - Fo);
  group_sync<NW>(g);
  return Fn;
}

// ---------------------------------------------------------------------------
// sk_pass: one Sinkhorn iteration over one row band of one problem.
//
// Row j: w_j,p = 2^(F_old,j + G_p - c Pi_jp) (every w <= v_p after a column
// update), S_j = sum_p w_j,p.  The new potential is F_j + log2(u_j / S_j) and
// the column sums need 2^(F_new,j + G_p - c Pi_jp) = (u_j / S_j) w_j,p, so one
// exp2 per element serves both.
//
// The block holds NG row groups of NW warps; group g takes the band's rows
// g, g + NG, g + 2 NG, ... through its own ring of bulk-copied rows, so short
// rows do not leave the block idle behind one barrier per row.  In a group,
// thread t owns the columns col_of(t, v); per row: the row pass, one group
// barrier (the row sum needs every warp of the group; none for a one-warp
// group), then the group's first thread refills the slot and every thread
// adds r_j w_j to its column sums.  At the end the groups' column sums are
// added in shared memory.  A row sum out of range is redone from the ring
// with a max shift (group-uniform branch).
// ---------------------------------------------------------------------------
// The pass over band `a` of problem `pr` by one block of 32 NW NG threads
// (smem_dyn: the block's dynamic shared memory).
template <int NW, int VPT, int NG, typename Real>
__device__ __forceinline__ void pass_band(const SkProb<Real>& pr, int a, unsigned* status,
                                          unsigned char* smem_dyn) {
  constexpr int GT = 32 * NW;  // threads of a row group
  constexpr int NT = GT * NG;
  constexpr int COVER = GT * VPT;
  const int S = pr.geo.stages, slot_bytes = pr.geo.slot_bytes;
  const Real* __restrict__ Pi = pr.Pi;
  Real* __restrict__ F = pr.F;
  Real* __restrict__ part = pr.part;
  const int n = pr.n, m = pr.m, R = pr.R;
  const Real c = pr.c;

  unsigned char* sm = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  unsigned char* ring = sm;
  const size_t ring_bytes = (size_t)NG * S * slot_bytes > (size_t)NG * COVER * sizeof(Real)
                                ? (size_t)NG * S * slot_bytes
                                : (size_t)NG * COVER * sizeof(Real);
  Real* red = reinterpret_cast<Real*>(ring + ring_bytes);  // 16-byte aligned
  Real* sfb = red + 2 * NG * NW;
  Real* Fold = sfb + NG * NW;
  Real* LU = Fold + R;
  unsigned char* braw = reinterpret_cast<unsigned char*>(LU + R);
  uint64_t* full = reinterpret_cast<uint64_t*>(braw + ((8u - (smem_u32(braw) & 7u)) & 7u));
  constexpr bool GVS = VPT >= kGvSmemVpt;
  unsigned char* graw = reinterpret_cast<unsigned char*>(full + NG * S);
  Real* gvs = reinterpret_cast<Real*>(graw + ((16u - (smem_u32(graw) & 15u)) & 15u));

  const int tid = threadIdx.x, g = tid / GT, gt = tid % GT, lane = tid & 31, wig = gt >> 5;
  const int s = a * R, Ra = min(R, n - s);
  unsigned char* gring = ring + (size_t)g * S * slot_bytes;
  uint64_t* gfull = full + g * S;
  // Row k of group g is band row g + k NG, in slot k mod S.
  auto issue = [&](int k) {
    const int t = g + k * NG;
    const char* src;
    unsigned bytes;
    int off;
    row_span(Pi, m, s + t, &src, &bytes, &off);
    mbar_arrive_expect_tx(&gfull[k % S], bytes);
    bulk_g2s(gring + (size_t)(k % S) * slot_bytes, src, bytes, &gfull[k % S]);
  };
  // Past the row's end a slot holds up to 24 bytes of what follows the row in
  // Pi (finite), or the zeros written here: finite values that the -inf of the
  // padded columns' G turns into exact zeros, with no per-element masks.  A
  // thread reads at most 2 * 16 bytes past the row's end (alignment offset
  // plus the 16-byte group straddling column m), so 48 bytes per slot are
  // cleared.  Each group's first thread clears its group's slots, sets up
  // their barriers and issues the first copies at once, so that their latency
  // overlaps the loads of the band's potentials below.
  const int row_bytes = m * (int)sizeof(Real);
  const int zw = min((slot_bytes - row_bytes) / 4, 12);
  if (gt == 0) {
    for (int q = 0; q < S; ++q) {
      unsigned* z = reinterpret_cast<unsigned*>(gring + (size_t)q * slot_bytes + row_bytes);
      for (int w = 0; w < zw; ++w) z[w] = 0u;
      mbar_init(&gfull[q], 1);
    }
    fence_mbar_init();
    fence_proxy_async_smem();
    for (int k = 0; k < S && g + k * NG < Ra; ++k) issue(k);
  }
  for (int t = tid; t < Ra; t += NT) {
    Fold[t] = F[s + t];
    LU[t] = pr.lu[s + t];
  }
  if constexpr (GVS) {
    for (int p = tid; p < COVER; p += NT) gvs[p] = p < m ? pr.G[p] : (Real)-INFINITY;
  }
  __syncthreads();
  Real Gv[GVS ? 1 : VPT], acc[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    if constexpr (!GVS) {
      const int p = col_of<Real>(gt, v, GT);
      Gv[v] = p < m ? pr.G[p] : (Real)-INFINITY;
    }
    acc[v] = 0;
  }
  auto gv_at = [&](int v) -> Real {
    if constexpr (GVS) return gvs[col_of<Real>(gt, v, GT)];
    else return Gv[v];
  };
  Real* gred = red + g * 2 * NW;
  Real* gsfb = sfb + g * NW;
  for (int k = 0;; ++k) {
    const int t = g + k * NG;
    if (t >= Ra) break;
    mbar_wait_bounded(&gfull[k % S], (unsigned)((k / S) & 1), status);
    const int off = (int)((((size_t)(s + t) * (size_t)m * sizeof(Real)) & 15) / sizeof(Real));
    const Real* row = reinterpret_cast<const Real*>(gring + (size_t)(k % S) * slot_bytes) + off;
    Real x[VPT], w[VPT];
    load_vals<VPT, GT>(row, gt, m, x);
    const Real Fo = Fold[t];
    if constexpr (GVS) {
      constexpr int PER = 16 / sizeof(Real);
#pragma unroll
      for (int j = 0; j < VPT / PER; ++j) {
        const float4 q = reinterpret_cast<const float4*>(gvs)[j * GT + gt];
        const Real* e = reinterpret_cast<const Real*>(&q);
#pragma unroll
        for (int u = 0; u < PER; ++u) w[j * PER + u] = ex2(fma(-c, x[j * PER + u], e[u] + Fo));
      }
    } else {
#pragma unroll
      for (int v = 0; v < VPT; ++v) w[v] = ex2(fma(-c, x[v], Gv[v] + Fo));
    }
    Real St = warp_sum(tree_sum<VPT>(w));
    if constexpr (NW > 1) {
      Real* rb = gred + (k & 1) * NW;
      if (lane == 0) rb[wig] = St;
      group_sync<NW>(g);
      St = tree_sum_smem<NW>(rb);
    }
    const Real lut = LU[t];
    const bool more = t + S * NG < Ra;
    if (St >= tiny_sum<Real>() && St <= (Real)1e30) {
      // Every thread of the group has read row t: its slot takes row k + S.
      if (gt == 0 && more) {
        fence_proxy_async_smem();
        issue(k + S);
      }
      if (pr.kappa == (Real)1) {
        const Real r = scale_of(lut, St);
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[v] = fma(r, w[v], acc[v]);
        if (gt == 0) F[s + t] = Fo + lut - lg2(St);
      } else {
        // Unbalanced GW: the balanced update scaled by kappa; the column sums
        // take 2^(F_new + G - c Pi) = 2^(F_new - F_old) w.
        const Real Fn = pr.kappa * (Fo + lut - lg2(St));
        const Real r = ex2(Fn - Fo);
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[v] = fma(r, w[v], acc[v]);
        if (gt == 0) F[s + t] = Fn;
      }
    } else {
      const Real Fn = row_redo<NW, VPT, Real>(row, gt, g, m, c, gv_at, Fo, lut, pr.kappa, acc, gsfb);
      if (gt == 0) {
        F[s + t] = Fn;
        if (more) {
          fence_proxy_async_smem();
          issue(k + S);
        }
      }
    }
  }
  // Band partials of the column sums (relative to the current G).
  if constexpr (NG == 1) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int p = col_of<Real>(gt, v, GT);
      if (p < m) part[(size_t)a * m + p] = acc[v];
    }
  } else {
    // Every copy was consumed, so the ring is free: add the groups' sums.
    __syncthreads();
    Real* cs = reinterpret_cast<Real*>(ring);
#pragma unroll
    for (int v = 0; v < VPT; ++v) cs[(size_t)g * COVER + col_of<Real>(gt, v, GT)] = acc[v];
    __syncthreads();
    for (int p = tid; p < m; p += NT) {
      Real sum = 0;
#pragma unroll
      for (int q = 0; q < NG; ++q) sum += cs[(size_t)q * COVER + p];
      part[(size_t)a * m + p] = sum;
    }
  }
}

template <int NW, int VPT, int NG, typename Real, int MAXP>
__global__ void __launch_bounds__(32 * NW * NG, 1)
    sk_pass(const __grid_constant__ SkBatch<Real, MAXP> P, unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  const int pi = batch_problem(P);
  pass_band<NW, VPT, NG, Real>(P.p[pi], (int)blockIdx.x - P.block0[pi], status, smem_dyn);
}

// Per column: S_p = sum_b part_bp (FP32 compensated sums over 8 band groups,
// combined in FP64) and G_p += log2 v_p - log2 S_p.  A block covers 32
// columns.  If any of them has S_p out of range, the block recomputes its 32
// columns from Pi and the new F with a running max (8 warps over the rows,
// one lane per column).
template <typename Real>
__device__ __forceinline__ void cols_block(const SkProb<Real>& pr, int cb) {
  const Real* __restrict__ part = pr.part;
  const Real* __restrict__ lv = pr.lv;
  Real* __restrict__ G = pr.G;
  const Real* __restrict__ Pi = pr.Pi;
  const Real* __restrict__ F = pr.F;
  const int B = pr.B, n = pr.n, m = pr.m;
  const Real c = pr.c;
  __shared__ double sS[8][32];
  __shared__ Real sM[8][32];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int p = cb * 32 + lane;
  const int per = (B + 7) / 8;
  const int b0 = min(B, grp * per), b1 = min(B, b0 + per);
  Real S = 0, C = 0;
  if (p < m) {
    // Loads in batches of 8 (independent, all in flight), then the
    // compensated sum in band order.
    for (int b = b0; b < b1; b += 8) {
      Real x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = b + q < b1 ? part[(size_t)(b + q) * m + p] : (Real)0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const Real yk = x[q] - C;
        const Real tk = S + yk;
        C = (tk - S) - yk;
        S = tk;
      }
    }
  }
  sS[grp][lane] = (double)S - (double)C;
  __syncthreads();
  double St = 0.0;
  for (int g = 0; g < 8; ++g) St += sS[g][lane];
  const bool bad = p < m && !(St >= (double)tiny_sum<Real>() && St <= 1e30);
  const double kap = (double)pr.kappa;
  if (!__syncthreads_or(bad)) {
    if (grp == 0 && p < m) {
      const double gn = (double)G[p] + (double)lv[p] - log2(St);
      G[p] = (Real)(kap == 1.0 ? gn : kap * gn);
    }
    return;
  }
  // Recompute: log2 sum_i 2^(F_i + G_p - c Pi_ip) with a running max.
  const Real Gp = p < m ? G[p] : (Real)0;
  Real M = -INFINITY;
  S = 0;
  if (p < m) {
    constexpr int U = 8;
    int i = grp;
    for (; i + 8 * (U - 1) < n; i += 8 * U) {
      Real e[U];
#pragma unroll
      for (int r = 0; r < U; ++r) e[r] = fma(-c, Pi[(size_t)(i + 8 * r) * m + p], Gp + F[i + 8 * r]);
      Real mx = M;
#pragma unroll
      for (int r = 0; r < U; ++r) mx = fmax(mx, e[r]);
      S = (M == -INFINITY) ? (Real)0 : S * ex2(M - mx);
#pragma unroll
      for (int r = 0; r < U; ++r) S += ex2(e[r] - mx);
      M = mx;
    }
    for (; i < n; i += 8) {
      const Real e = fma(-c, Pi[(size_t)i * m + p], Gp + F[i]);
      const Real mx = fmax(M, e);
      S = ((M == -INFINITY) ? (Real)0 : S * ex2(M - mx)) + ex2(e - mx);
      M = mx;
    }
  }
  __syncthreads();
  sM[grp][lane] = M;
  sS[grp][lane] = (double)S;
  __syncthreads();
  if (grp == 0 && p < m) {
    Real Mt = -INFINITY;
    for (int g = 0; g < 8; ++g) Mt = fmax(Mt, sM[g][lane]);
    double St2 = 0.0;
    for (int g = 0; g < 8; ++g)
      if (sS[g][lane] > 0.0) St2 += sS[g][lane] * exp2((double)(sM[g][lane] - Mt));
    const double gn = (double)Gp + (double)lv[p] - ((double)Mt + log2(St2));
    G[p] = (Real)(kap == 1.0 ? gn : kap * gn);
  }
}

template <typename Real, int MAXP>
__global__ void __launch_bounds__(256) sk_cols(const __grid_constant__ SkBatch<Real, MAXP> P) {
  const int pi = batch_problem(P);
  cols_block<Real>(P.p[pi], (int)blockIdx.x - P.block0[pi]);
}

// ---------------------------------------------------------------------------
// Batched Sinkhorn passes over many problems of different row lengths in one
// launch (gw_solve_batch).  The problems' row-pass configurations all use
// 512-thread blocks; a block finds its problem in a device-resident table
// (binary search over the problems' first blocks) and runs that problem's
// configuration on the band.  Blocks are scheduled onto the SMs as they free
// up, so the small problems' bands fill the SMs beside the large ones'.
// ---------------------------------------------------------------------------
// Problems of one mixed launch: their states in device memory, their
// configurations and first blocks in the (constant-cached) parameter block.
constexpr int kMixMax = 256;
template <typename Real>
struct SkMixTable {
  const SkProb<Real>* probs;    // [count], device memory
  int count;
  int cfg[kMixMax];             // row configuration ids
  int block0[kMixMax + 1];      // first row-pass block of each problem
  int cblock0[kMixMax + 1];     // first column-update block of each problem
};

__device__ __forceinline__ int find_owner(const int* first, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kMixThreads = 512;

template <typename Real>
__global__ void __launch_bounds__(kMixThreads, 1) sk_pass_mix(const __grid_constant__ SkMixTable<Real> T,
                                                              unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  const int pi = find_owner(T.block0, T.count, (int)blockIdx.x);
  const SkProb<Real> pr = T.probs[pi];
  const int a = (int)blockIdx.x - T.block0[pi];
  if constexpr (sizeof(Real) == 4) {
    switch (T.cfg[pi]) {
      case 0: pass_band<1, 16, 16, float>(pr, a, status, smem_dyn); break;
      case 1: pass_band<2, 16, 8, float>(pr, a, status, smem_dyn); break;
      case 2: pass_band<4, 16, 4, float>(pr, a, status, smem_dyn); break;
      case 3: pass_band<8, 16, 2, float>(pr, a, status, smem_dyn); break;
      case 4: pass_band<16, 16, 1, float>(pr, a, status, smem_dyn); break;
      case 20: pass_band<2, 8, 8, float>(pr, a, status, smem_dyn); break;
      case 21: pass_band<4, 8, 4, float>(pr, a, status, smem_dyn); break;
      case 22: pass_band<8, 8, 2, float>(pr, a, status, smem_dyn); break;
      case 40: pass_band<1, 12, 16, float>(pr, a, status, smem_dyn); break;
      case 41: pass_band<2, 12, 8, float>(pr, a, status, smem_dyn); break;
      case 42: pass_band<4, 12, 4, float>(pr, a, status, smem_dyn); break;
      case 43: pass_band<8, 12, 2, float>(pr, a, status, smem_dyn); break;
      case 44: pass_band<16, 12, 1, float>(pr, a, status, smem_dyn); break;
      case 45: pass_band<2, 24, 8, float>(pr, a, status, smem_dyn); break;
      case 46: pass_band<4, 24, 4, float>(pr, a, status, smem_dyn); break;
      case 47: pass_band<8, 24, 2, float>(pr, a, status, smem_dyn); break;
      case 48: pass_band<1, 24, 16, float>(pr, a, status, smem_dyn); break;
      case 50: pass_band<1, 32, 16, float>(pr, a, status, smem_dyn); break;
      case 51: pass_band<2, 32, 8, float>(pr, a, status, smem_dyn); break;
      case 52: pass_band<4, 32, 4, float>(pr, a, status, smem_dyn); break;
      case 53: pass_band<8, 32, 2, float>(pr, a, status, smem_dyn); break;
      default: pass_band<16, 8, 1, float>(pr, a, status, smem_dyn); break;  // 23
    }
  } else {
    switch (T.cfg[pi]) {
      case 10: pass_band<1, 8, 16, double>(pr, a, status, smem_dyn); break;
      case 11: pass_band<4, 8, 4, double>(pr, a, status, smem_dyn); break;
      case 12: pass_band<16, 8, 1, double>(pr, a, status, smem_dyn); break;
      case 30: pass_band<2, 4, 8, double>(pr, a, status, smem_dyn); break;
      default: pass_band<8, 4, 2, double>(pr, a, status, smem_dyn); break;  // 31
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) sk_cols_mix(const __grid_constant__ SkMixTable<Real> T) {
  const int pi = find_owner(T.cblock0, T.count, (int)blockIdx.x);
  const SkProb<Real> pr = T.probs[pi];
  cols_block<Real>(pr, (int)blockIdx.x - T.cblock0[pi]);
}

// ---------------------------------------------------------------------------
// Plan and statistics: T = 2^(F_i + G_p - c Pi_ip); per CTA the entropy
// partial sum_ip T (ln T - 1), the row-marginal error sum_i |T_i. - u_i| and
// the band's column sums.
// ---------------------------------------------------------------------------
template <int NW, int VPT, typename Real, int MAXP>
__global__ void __launch_bounds__(32 * NW, 1) sk_plan(const __grid_constant__ SkBatch<Real, MAXP> P, unsigned* status) {
  const int pi = batch_problem(P);
  const SkProb<Real>& pr = P.p[pi];
  const int S = pr.geo.stages, slot_bytes = pr.geo.slot_bytes;
  const Real* __restrict__ Pi = pr.Pi;
  const Real* __restrict__ F = pr.F;
  const double* __restrict__ u = pr.u;
  Real* __restrict__ T = pr.T;
  const int n = pr.n, m = pr.m, R = pr.R;
  const Real c = pr.c;
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  unsigned char* sm = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  unsigned char* ring = sm;
  unsigned char* braw = ring + (size_t)S * slot_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(braw);
  __shared__ double dred[2][32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int a = (int)blockIdx.x - P.block0[pi], s = a * R, Ra = min(R, n - s);
  constexpr int NT = 32 * NW;
  auto issue = [&](int t) {
    const char* src;
    unsigned bytes;
    int off;
    row_span(Pi, m, s + t, &src, &bytes, &off);
    mbar_arrive_expect_tx(&full[t % S], bytes);
    bulk_g2s(ring + (size_t)(t % S) * slot_bytes, src, bytes, &full[t % S]);
  };
  if (tid == 0) {
    for (int i = 0; i < S; ++i) mbar_init(&full[i], 1);
    fence_mbar_init();
    for (int t = 0; t < S && t < Ra; ++t) issue(t);
  }
  __syncthreads();
  Real Gv[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int p = col_of<Real>(tid, v, NT);
    Gv[v] = p < m ? pr.G[p] : (Real)0;
  }
  double csum[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) csum[v] = 0.0;
  double ent = 0.0, rowerr = 0.0;
  const Real ln2 = (Real)0.69314718055994530942;
  for (int t = 0; t < Ra; ++t) {
    const int i = s + t;
    mbar_wait_bounded(&full[t % S], (unsigned)((t / S) & 1), status);
    const int off = (int)((((size_t)i * (size_t)m * sizeof(Real)) & 15) / sizeof(Real));
    Real x[VPT];
    load_vals<VPT, NT>(reinterpret_cast<const Real*>(ring + (size_t)(t % S) * slot_bytes) + off, tid, m, x);
    const Real Fi = F[i];
    Real rs = 0, en = 0;
    Real* trow = T + (size_t)i * m;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int p = col_of<Real>(tid, v, NT);
      if (p < m) {
        const Real lt = fma(-c, x[v], Gv[v] + Fi);  // log2 T
        const Real tv = ex2(lt);
        trow[p] = tv;
        rs += tv;
        en += tv * (lt * ln2 - (Real)1);
        csum[v] += (double)tv;
      }
    }
    double rsd = warp_sum((double)rs);
    ent += (double)en;
    if (lane == 0) dred[t & 1][warp] = rsd;
    __syncthreads();
    if (tid == 0 && t + S < Ra) {
      fence_proxy_async_smem();
      issue(t + S);
    }
    if (tid == 0) {
      double r = 0.0;
      for (int w = 0; w < NW; ++w) r += dred[t & 1][w];
      rowerr += fabs(r - u[i]);
    }
  }
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int p = col_of<Real>(tid, v, NT);
    if (p < m) pr.colpart[(size_t)a * m + p] = csum[v];
  }
  ent = warp_sum(ent);
  __syncthreads();
  if (lane == 0) dred[0][warp] = ent;
  __syncthreads();
  if (tid == 0) {
    double e = 0.0;
    for (int w = 0; w < NW; ++w) e += dred[0][w];
    pr.cta_stats[2 * a + 0] = e;
    pr.cta_stats[2 * a + 1] = rowerr;
  }
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void fill_product(const double* __restrict__ u, const double* __restrict__ v, int n, int m,
                             Real* __restrict__ T) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const double vp = v[p];
  for (int i = blockIdx.y; i < n; i += gridDim.y) T[(size_t)i * m + p] = (Real)(u[i] * vp);
}

template <typename Real>
__global__ void log2_scaled(const double* __restrict__ w, int len, Real* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = (Real)log2(w[i]);
}

template <typename Real>
__global__ void fill_val(Real* __restrict__ x, int len, Real val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) x[i] = val;
}

// Pi += w ||phi_i - psi_p||^2 (w = 1 - theta), features as doubles (row-major
// n x D and m x D, D <= 64).  A block covers 256 columns x 16 rows: each
// thread keeps its column's features in registers (in the arithmetic type:
// D squared differences of order-one features add up without cancellation),
// the block's 16 rows of features sit in shared memory.
constexpr int kFeatRows = 16;
template <typename Real>
__global__ void __launch_bounds__(256) add_feature_cost(Real* __restrict__ Pi, int n, int m, int D,
                                                        const double* __restrict__ phi,
                                                        const double* __restrict__ psi, double w) {
  __shared__ Real ph[kFeatRows][64];
  const int p = blockIdx.x * 256 + threadIdx.x;
  const int i0 = blockIdx.y * kFeatRows;
  for (int e = threadIdx.x; e < kFeatRows * D; e += 256) {
    const int r = e / D, d = e % D;
    ph[r][d] = i0 + r < n ? (Real)phi[(size_t)(i0 + r) * D + d] : (Real)0;
  }
  __syncthreads();
  if (p >= m) return;
  Real ps[64];
#pragma unroll
  for (int d = 0; d < 64; ++d) ps[d] = d < D ? (Real)psi[(size_t)p * D + d] : (Real)0;
  const Real wr = (Real)w;
  for (int r = 0; r < kFeatRows && i0 + r < n; ++r) {
    Real acc = 0;
#pragma unroll
    for (int d = 0; d < 64; ++d) {
      if (d < D) {
        const Real diff = ph[r][d] - ps[d];
        acc = fma(diff, diff, acc);
      }
    }
    Real* q = Pi + (size_t)(i0 + r) * m + p;
    *q = fma(wr, acc, *q);
  }
}

// Partial sums of <CC, T>, CC_ip = ||phi_i - psi_p||^2, over the same tiles
// (FP64 accumulation per thread, one partial per block).
template <typename Real>
__global__ void __launch_bounds__(256) feature_dot_tiles(const Real* __restrict__ T, int n, int m, int D,
                                                         const double* __restrict__ phi,
                                                         const double* __restrict__ psi, double* __restrict__ part) {
  __shared__ double ph[kFeatRows][64];
  __shared__ double sm[8];
  const int p = blockIdx.x * 256 + threadIdx.x;
  const int i0 = blockIdx.y * kFeatRows;
  for (int e = threadIdx.x; e < kFeatRows * D; e += 256) {
    const int r = e / D, d = e % D;
    ph[r][d] = i0 + r < n ? phi[(size_t)(i0 + r) * D + d] : 0.0;
  }
  __syncthreads();
  double tot = 0.0;
  if (p < m) {
    double ps[64];
#pragma unroll
    for (int d = 0; d < 64; ++d) ps[d] = d < D ? psi[(size_t)p * D + d] : 0.0;
    for (int r = 0; r < kFeatRows && i0 + r < n; ++r) {
      double cc = 0.0;
#pragma unroll
      for (int d = 0; d < 64; ++d) {
        if (d < D) {
          const double diff = ph[r][d] - ps[d];
          cc = fma(diff, diff, cc);
        }
      }
      tot += cc * (double)T[(size_t)(i0 + r) * m + p];
    }
  }
  tot = warp_sum(tot);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sm[q];
    part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// Sums `count` partials into out[0] (one block, fixed order).
__global__ void sum_partials(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double sm[32];
  double t = 0.0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) t += part[k];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sm[w];
    out[0] = r;
  }
}

// Deterministic dot products: per-block partial sums (FP64), then one block.
template <typename Real>
__global__ void dot_partial(const Real* __restrict__ A, const Real* __restrict__ B, size_t N, double* __restrict__ part) {
  double acc = 0.0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
    acc += (double)A[k] * (double)B[k];
  __shared__ double sm[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w];
    part[blockIdx.x] = s;
  }
}

// stats: [0] objective, [1] E(T), [2] <CC,T>, [3] eps H(T), [4] sum|T1-u|,
// [5] sum|T^T 1 - v|, [6] outer iterations, [7] 0.
__global__ void finish_stats(const double* __restrict__ dotE, int nE, const double* __restrict__ dotC, int nC,
                             const double* __restrict__ cta_stats, int B, const double* __restrict__ colpart, int m,
                             const double* __restrict__ v, double eps, double theta, int n_outer,
                             double* __restrict__ stats) {
  __shared__ double sm[32];
  // column marginal error (all threads), then scalar sums by thread 0
  double ce = 0.0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    double cs = 0.0;
    for (int b = 0; b < B; ++b) cs += colpart[(size_t)b * m + p];
    ce += fabs(cs - v[p]);
  }
  ce = warp_sum(ce);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = ce;
  __syncthreads();
  if (threadIdx.x == 0) {
    double colerr = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) colerr += sm[w];
    double E = 0.0, C = 0.0, H = 0.0, re = 0.0;
    for (int k = 0; k < nE; ++k) E += dotE[k];
    for (int k = 0; k < nC; ++k) C += dotC[k];
    for (int b = 0; b < B; ++b) {
      H += cta_stats[2 * b];
      re += cta_stats[2 * b + 1];
    }
    stats[0] = (1.0 - theta) * C + theta * E;
    stats[1] = E;
    stats[2] = C;
    stats[3] = eps * H;
    stats[4] = re;
    stats[5] = colerr;
    stats[6] = (double)n_outer;
    stats[7] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Unbalanced GW (Remark "Entropic algorithm for UGW").  The scalars of the
// current plan T (mass m = sum T, row sums a = T 1, column sums b = T^T 1):
//   scal[0] g = rho sum a ln(a/u) + rho sum b ln(b/v) + eps sum T ln(T/(u v))
//   scal[1] m
//   scal[2] KL(a (x) a | u (x) u) = 2 m sum a ln(a/u) - m^2 + (sum u)^2
//   scal[3] the same for b and v
//   scal[4] KL(T (x) T | (u v) (x) (u v)) = 2 m sum T ln(T/(u v)) - m^2 + (sum u sum v)^2
//   scal[5] sum |a - u|, scal[6] sum |b - v|
//   scal[8] 1 / sqrt(sum u sum v) (the starting plan's scale)
//   scal[9] sqrt(m_prev / m) (the rescale after each step's plan)
// ---------------------------------------------------------------------------
constexpr int kUgwScal = 16;
// Row-parallel elementwise kernels: columns on the grid's x, rows strided over
// at most kRowGridY blocks in y.
constexpr int kRowGridY = 2048;

// Per row: a_i = sum_p T_ip, e_i = sum_p T_ip ln T_ip (0 ln 0 = 0), in double.
template <typename Real>
__global__ void ugw_rowstats(const Real* __restrict__ T, int n, int m, double* __restrict__ a,
                             double* __restrict__ e) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const Real* row = T + (size_t)i * m;
  double s = 0.0, t = 0.0;
  for (int p = threadIdx.x & 31; p < m; p += 32) {
    const Real xr = row[p];
    const double x = (double)xr;
    s += x;
    // Float plans take x ln x in float (1 ulp logf; the FP64 log costs tens
    // of FP64 operations per element on this GPU); double plans in double.
    if constexpr (sizeof(Real) == 4) {
      if (xr > 0.0f) t += (double)(xr * logf(xr));
    } else {
      if (x > 0.0) t += x * log(x);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if ((threadIdx.x & 31) == 0) {
    a[i] = s;
    e[i] = t;
  }
}

// Per band of R rows: column sums in double, colpart[band][p].
template <typename Real>
__global__ void ugw_colsums(const Real* __restrict__ T, int n, int m, int R, double* __restrict__ colpart) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const int b = blockIdx.y, i0 = b * R, i1 = min(n, i0 + R);
  double s = 0.0;
  for (int i = i0; i < i1; ++i) s += (double)T[(size_t)i * m + p];
  colpart[(size_t)b * m + p] = s;
}

__device__ __forceinline__ double block_sum_d(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// One block: the scalars above from the row statistics and column partials.
__global__ void ugw_finish(const double* __restrict__ a, const double* __restrict__ e,
                           const double* __restrict__ colpart, int B, int n, int m, const double* __restrict__ u,
                           const double* __restrict__ v, double rho, double eps, double* __restrict__ scal) {
  __shared__ double sh[32];
  double mass = 0.0, sa = 0.0, se = 0.0, su = 0.0, ra = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mass += a[i];
    su += u[i];
    if (a[i] > 0.0) sa += a[i] * log(a[i] / u[i]);
    se += e[i] - a[i] * log(u[i]);
    ra += fabs(a[i] - u[i]);
  }
  double sb = 0.0, sv = 0.0, cb = 0.0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    double b = 0.0;
    for (int q = 0; q < B; ++q) b += colpart[(size_t)q * m + p];
    sv += v[p];
    if (b > 0.0) sb += b * log(b / v[p]);
    se -= b * log(v[p]);
    cb += fabs(b - v[p]);
  }
  mass = block_sum_d(mass, sh);
  sa = block_sum_d(sa, sh);
  se = block_sum_d(se, sh);
  su = block_sum_d(su, sh);
  ra = block_sum_d(ra, sh);
  sb = block_sum_d(sb, sh);
  sv = block_sum_d(sv, sh);
  cb = block_sum_d(cb, sh);
  if (threadIdx.x == 0) {
    scal[0] = rho * sa + rho * sb + eps * se;
    scal[1] = mass;
    scal[2] = 2.0 * mass * sa - mass * mass + su * su;
    scal[3] = 2.0 * mass * sb - mass * mass + sv * sv;
    scal[4] = 2.0 * mass * se - mass * mass + (su * sv) * (su * sv);
    scal[5] = ra;
    scal[6] = cb;
  }
}

// scal[8] = 1 / sqrt(sum u sum v).
__global__ void ugw_start_scale(const double* __restrict__ u, int n, const double* __restrict__ v, int m,
                                double* __restrict__ scal) {
  __shared__ double sh[32];
  double su = 0.0, sv = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) su += u[i];
  for (int p = threadIdx.x; p < m; p += blockDim.x) sv += v[p];
  su = block_sum_d(su, sh);
  sv = block_sum_d(sv, sh);
  if (threadIdx.x == 0) scal[8] = 1.0 / sqrt(su * sv);
}

// scal[9] = sqrt(scal[1] / m_new), m_new the plan's mass from its column
// partials (colpart, written by the plan pass).
__global__ void ugw_rescale_factor(const double* __restrict__ colpart, int B, int m, double* __restrict__ scal) {
  __shared__ double sh[32];
  double t = 0.0;
  for (size_t k = threadIdx.x; k < (size_t)B * m; k += blockDim.x) t += colpart[k];
  t = block_sum_d(t, sh);
  if (threadIdx.x == 0) scal[9] = sqrt(scal[1] / t);
}

// x *= *factor elementwise.
template <typename Real>
__global__ void scale_by(Real* __restrict__ x, size_t N, const double* __restrict__ factor) {
  const Real f = (Real)*factor;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

// The unbalanced step's cost in the Sinkhorn kernels' form:
//   Pi_ip <- (Pi_ip + g) / m - eps (ln u_i + ln v_p)
// with Pi = the gradient with T's own marginals on entry; lu, lv are log2 u,
// log2 v.  The balanced update on this cost, scaled by rho / (rho + eps), is
// the unbalanced update with reference measure u v^T.
template <typename Real>
__global__ void ugw_cost_kernel(Real* __restrict__ Pi, int n, int m, const Real* __restrict__ lu,
                                const Real* __restrict__ lv, const double* __restrict__ scal, double eps) {
  const Real g = (Real)scal[0], inv_m = (Real)(1.0 / scal[1]);
  const Real el = (Real)(eps * 0.6931471805599453);
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  const Real lvp = lv[p];
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const size_t k = (size_t)i * m + p;
    Pi[k] = fma(Pi[k] + g, inv_m, -el * (lu[i] + lvp));
  }
}

// Final UGW statistics (after finish_stats has written E and the rest):
// [0] UGW objective, [2] rho (KLx(a|u) + KLx(b|v)), [3] eps KLx(T|u v),
// [4] sum |a - u|, [5] sum |b - v|, [7] mass of T.
__global__ void ugw_stats(const double* __restrict__ scal, double rho, double eps, double* __restrict__ stats) {
  const double E = stats[1];
  stats[2] = rho * (scal[2] + scal[3]);
  stats[3] = eps * scal[4];
  stats[0] = E + stats[2] + stats[3];
  stats[4] = scal[5];
  stats[5] = scal[6];
  stats[7] = scal[1];
}

// Pi += coef * ln T elementwise; an entry of T that underflowed to zero
// counts as the smallest normal number of the type.
template <typename Real>
__global__ void add_log_plan(Real* __restrict__ Pi, const Real* __restrict__ T, size_t N, Real coef) {
  const Real tiny = sizeof(Real) == 4 ? (Real)1.17549435e-38f : (Real)2.2250738585072014e-308;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    Pi[i] = fma(coef, log(fmax(T[i], tiny)), Pi[i]);
}

template <typename Real>
__global__ void potentials_out(const Real* __restrict__ F, int len, double scale, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = (double)F[i] * scale;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Ring slots hold one row, its alignment offset (< 16 bytes) and the few
// elements a thread straddling the row's end reads past it.  Each of the NG
// row groups gets `stages` slots: as many as fit in about 150 KB, from 2 to
// 6.
template <int NW, int VPT, int NG, typename Real>
RowGeom row_geom(int m) {
  RowGeom g{};
  g.slot_bytes = (int)((((size_t)m + 16 + 8) * sizeof(Real) + 127) / 128 * 128);
  g.stages = (int)std::max<size_t>(2, std::min<size_t>(6, (150 * 1024) / ((size_t)NG * g.slot_bytes)));
  return g;
}

// Row bands of the Sinkhorn kernels.  A single solve spreads its rows over
// all SMs.  In a batch, problems share the GPU, and a band is one block's
// whole work: each block pays for its ring set-up, the first copies' latency
// and its column partials, so bands hold at least kBatchBandBytes of Pi (and
// at least 32 rows, at most kBatchBandRowsMax, whose potentials the block
// keeps in shared memory).  Against 32-row bands this takes batched passes
// over rows of 256 columns from 1.0 to 2.5 TB/s and of 1024 columns from 2.6
// to 4.2 TB/s (n = 4096); 1 MB and 2 MB bands were slower on mixed batches.
constexpr size_t kBatchBandBytes = 512 * 1024;
constexpr int kBatchBandRowsMax = 1024;
Bands solve_bands(const SolveArgs& A) {
  if (!A.batch) return choose_bands(A.n, A.num_sms);
  const size_t row_bytes = (size_t)A.m * (A.dtype == GW_F32 ? 4 : 8);
  const int min_rows =
      (int)std::min<size_t>(kBatchBandRowsMax, std::max<size_t>(32, (kBatchBandBytes + row_bytes - 1) / row_bytes));
  const int fewest = (A.n + kBatchBandRowsMax - 1) / kBatchBandRowsMax;
  const int target = std::max(fewest, std::min(A.num_sms, A.n / min_rows));
  return choose_bands(A.n, target);
}

constexpr int kDots = 256;

// One problem's state inside its workspace:
//   Pi | F | G | lu | lv | part | colpart | cta_stats | dots | gradient workspace
template <typename Real>
struct SolveState {
  const SolveArgs* A;
  SkProb<Real> sk;
  double *dotE, *dotC;
  double *ugw_a, *ugw_e, *ugw_scal;  // unbalanced GW: row statistics and scalars
  char* gws;
  size_t gws_bytes;
  size_t smem_pass, smem_plan;
};

template <int NW, int VPT, int NG, typename Real>
int prepare(const SolveArgs& A, void* wsv, size_t ws_bytes, SolveState<Real>* S) {
  const int n = A.n, m = A.m;
  const Bands bands = solve_bands(A);
  char* ws = (char*)wsv;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = ws + off;
    off = (off + bytes + 255) / 256 * 256;
    return p;
  };
  SkProb<Real>& k = S->sk;
  memset(&k, 0, sizeof(k));
  k.n = n;
  k.m = m;
  k.B = bands.B;
  k.R = bands.R;
  k.c = (Real)(1.4426950408889634 / A.tau);  // each step's Sinkhorn regularisation is tau
  k.kappa = A.rho > 0.0 ? (Real)(A.rho / (A.rho + A.eps)) : (Real)1;
  k.Pi = (Real*)take((size_t)n * m * sizeof(Real));
  k.F = (Real*)take((size_t)n * sizeof(Real));
  k.G = (Real*)take((size_t)m * sizeof(Real));
  k.lu = (Real*)take((size_t)n * sizeof(Real));
  k.lv = (Real*)take((size_t)m * sizeof(Real));
  k.part = (Real*)take((size_t)bands.B * m * sizeof(Real));
  k.colpart = (double*)take((size_t)bands.B * m * sizeof(double));
  k.cta_stats = (double*)take((size_t)2 * bands.B * sizeof(double));
  S->dotE = (double*)take((size_t)kDots * sizeof(double));
  S->dotC = (double*)take((size_t)kDots * sizeof(double));
  S->ugw_a = (double*)take((size_t)n * sizeof(double));
  S->ugw_e = (double*)take((size_t)n * sizeof(double));
  S->ugw_scal = (double*)take((size_t)kUgwScal * sizeof(double));
  S->gws = take(0);
  if (off > ws_bytes) return GW_ERR_OOM;
  S->gws_bytes = ws_bytes - off;
  k.T = (Real*)A.T;
  k.u = A.u;
  k.geo = row_geom<NW, VPT, NG, Real>(m);
  S->smem_pass = pass_smem_bytes<NW, VPT, NG, Real>(k.geo, k.R);
  S->smem_plan = plan_smem_bytes(k.geo);
  S->A = &A;
  return GW_OK;
}

// Pi = out_scale * G(T) with target marginals (out_scale = 2 theta), or,
// for the value, G(T) with T's own marginals.
template <typename Real>
int gradient(const SolveState<Real>& S, int exact, double out_scale, cudaStream_t st, bool regen = false) {
  const SolveArgs& A = *S.A;
  if (A.dense_x) {
    DenseXGradArgs d{};
    d.N = A.n;
    d.n = A.m;
    d.k = A.k;
    d.dtype = A.dtype;
    d.exact = exact;
    d.hy = A.hy;
    d.out_scale = out_scale;
    d.C = A.dense_x;
    d.T = A.T;
    d.G = (void*)S.sk.Pi;
    d.u = A.u;
    d.v = A.v;
    d.stream = st;
    d.tracer = A.tracer;
    return dense_x_grad_launch(d, S.gws, S.gws_bytes);
  }
  if (A.dim >= 2) {
    Grad2DArgs g2{};
    g2.dim = A.dim;
    g2.sx = A.nx;
    g2.sy = A.ny;
    g2.cost = A.cost;
    g2.k = A.k;
    g2.hx = A.hx;
    g2.hy = A.hy;
    g2.dtype = A.dtype;
    g2.T = A.T;
    g2.G = (void*)S.sk.Pi;
    g2.u = A.u;
    g2.v = A.v;
    g2.exact = exact;
    g2.out_scale = out_scale;
    g2.stream = st;
    g2.status = A.status;
    g2.num_sms = A.num_sms;
    g2.tracer = A.tracer;
    return grad2d_launch(g2, S.gws, S.gws_bytes);
  }
  Grad1DArgs ga{};
  ga.n = A.n;
  ga.m = A.m;
  ga.k = A.k;
  ga.ky = A.ky;
  ga.hx = A.hx;
  ga.hy = A.hy;
  ga.dtype = A.dtype;
  ga.T = A.T;
  ga.G = (void*)S.sk.Pi;
  ga.u = A.u;
  ga.v = A.v;
  ga.exact = exact;
  ga.out_scale = out_scale;
  ga.stream = st;
  ga.status = A.status;
  ga.num_sms = A.num_sms;
  ga.tracer = A.tracer;
  ga.force_generic = A.force_generic;
  if constexpr (sizeof(Real) == 4) {
    if (regen) {
      // The plan of the previous step is formed from Pi and the potentials
      // as the gradient loads it; the new cost overwrites Pi row by row.
      ga.T = S.sk.Pi;
      ga.regen_F = S.sk.F;
      ga.regen_G = S.sk.G;
      ga.regen_c = S.sk.c;
    }
  }
  return grad1d_launch(ga, S.gws, S.gws_bytes);
}

template <typename Real>
bool fused(const SolveArgs& A) {
  return A.theta != 1.0 && A.feat_dim > 0 && A.phi && A.psi;
}

// T^0 = u v^T and the log-marginals.
template <typename Real>
void step_setup(const SolveState<Real>& S, cudaStream_t st) {
  const SolveArgs& A = *S.A;
  TraceScope ts(A.tracer, "solve_setup", st);
  // The row copies may read up to 15 bytes past Pi: keep them finite.
  cudaMemsetAsync((char*)S.sk.Pi + (size_t)A.n * A.m * sizeof(Real), 0, 16, st);
  log2_scaled<Real><<<(A.n + 255) / 256, 256, 0, st>>>(A.u, A.n, (Real*)S.sk.lu);
  log2_scaled<Real><<<(A.m + 255) / 256, 256, 0, st>>>(A.v, A.m, (Real*)S.sk.lv);
  fill_product<Real><<<dim3((A.m + 255) / 256, std::min(A.n, kRowGridY)), 256, 0, st>>>(A.u, A.v, A.n, A.m,
                                                                                    (Real*)A.T);
  if (A.rho > 0.0) {
    // Unbalanced GW starts at u v^T / sqrt(m(u) m(v)).
    ugw_start_scale<<<1, 256, 0, st>>>(A.u, A.n, A.v, A.m, S.ugw_scal);
    scale_by<Real><<<4 * A.num_sms, 256, 0, st>>>((Real*)A.T, (size_t)A.n * A.m, S.ugw_scal + 8);
  }
}

// Unbalanced GW: the scalars of the plan T (ugw_finish's list).
template <typename Real>
void ugw_scalars(const SolveState<Real>& S, cudaStream_t st) {
  const SolveArgs& A = *S.A;
  ugw_rowstats<Real><<<(A.n + 7) / 8, 256, 0, st>>>((const Real*)A.T, A.n, A.m, S.ugw_a, S.ugw_e);
  ugw_colsums<Real><<<dim3((A.m + 255) / 256, S.sk.B), 256, 0, st>>>((const Real*)A.T, A.n, A.m, S.sk.R,
                                                                      S.sk.colpart);
  ugw_finish<<<1, 1024, 0, st>>>(S.ugw_a, S.ugw_e, S.sk.colpart, S.sk.B, A.n, A.m, A.u, A.v, A.rho, A.eps,
                                S.ugw_scal);
}

// Pi for mirror-descent step l, then f = g = 0 (or, warm-started after the
// first step, the previous step's potentials stay).
// Single solves of 1D float problems whose gradient can read the plan from
// Pi (balanced, tau = eps, at least two steps) never materialise the plan
// between mirror-descent steps: it is formed from the previous step's Pi and
// potentials inside the next gradient, and written only after the last step.
bool plan_on_the_fly(const SolveArgs& A) {
  return !A.batch && !A.dense_x && A.dim == 1 && A.dtype == GW_F32 && !(A.rho > 0.0) && A.tau == A.eps &&
         A.n_outer >= 2 &&
         grad1d_regen_supported(A.n, A.m, A.k, A.ky, A.dtype, A.force_generic);
}

template <typename Real>
int step_cost(const SolveState<Real>& S, cudaStream_t st, int l) {
  const SolveArgs& A = *S.A;
  if (A.rho > 0.0) {
    // Unbalanced GW: cost ((1/2) grad E(T) + g(T)) / m(T) - eps ln(u v), the
    // gradient taken with T's own marginals.
    TraceScope ts(A.tracer, "ugw_cost", st);
    ugw_scalars(S, st);
    int rc = gradient(S, 1, 1.0, st);
    if (rc != GW_OK) return rc;
    ugw_cost_kernel<Real><<<dim3((A.m + 255) / 256, std::min(A.n, kRowGridY)), 256, 0, st>>>(
        (Real*)S.sk.Pi, A.n, A.m, S.sk.lu, S.sk.lv, S.ugw_scal,
                                                         A.eps);
    if (A.warm_start && l > 0) return GW_OK;
    fill_val<Real><<<(A.n + 255) / 256, 256, 0, st>>>(S.sk.F, A.n, (Real)0);
    fill_val<Real><<<(A.m + 255) / 256, 256, 0, st>>>(S.sk.G, A.m, (Real)0);
    return GW_OK;
  }
  int rc = gradient(S, 0, 2.0 * A.theta, st, l > 0 && plan_on_the_fly(A));
  if (rc != GW_OK) return rc;
  if (fused<Real>(A)) {
    TraceScope ts(A.tracer, "add_feature_cost", st);
    const dim3 grid((A.m + 255) / 256, (A.n + kFeatRows - 1) / kFeatRows);
    add_feature_cost<Real><<<grid, 256, 0, st>>>((Real*)S.sk.Pi, A.n, A.m, A.feat_dim, A.phi, A.psi, 1.0 - A.theta);
  }
  if (A.tau != A.eps) {
    // Pi += (eps - tau) grad H(T), grad H(T) = ln T (eq. "GW sinkhorn").
    TraceScope ts(A.tracer, "add_log_plan", st);
    add_log_plan<Real><<<4 * A.num_sms, 256, 0, st>>>((Real*)S.sk.Pi, (const Real*)A.T, (size_t)A.n * A.m,
                                                      (Real)(A.eps - A.tau));
  }
  if (A.warm_start && l > 0) return GW_OK;
  TraceScope ts(A.tracer, "solve_setup", st);
  fill_val<Real><<<(A.n + 255) / 256, 256, 0, st>>>(S.sk.F, A.n, (Real)0);
  fill_val<Real><<<(A.m + 255) / 256, 256, 0, st>>>(S.sk.G, A.m, (Real)0);
  return GW_OK;
}

// After a step's plan: unbalanced GW rescales it to mass sqrt(m(T_prev) m(T)).
template <typename Real>
void step_after_plan(const SolveState<Real>& S, cudaStream_t st) {
  const SolveArgs& A = *S.A;
  if (!(A.rho > 0.0)) return;
  TraceScope ts(A.tracer, "ugw_rescale", st);
  ugw_rescale_factor<<<1, 1024, 0, st>>>(S.sk.colpart, S.sk.B, A.m, S.ugw_scal);
  scale_by<Real><<<4 * A.num_sms, 256, 0, st>>>((Real*)A.T, (size_t)A.n * A.m, S.ugw_scal + 9);
}

// Potentials out and the statistics of the final plan.
template <typename Real>
int step_finish(const SolveState<Real>& S, cudaStream_t st) {
  const SolveArgs& A = *S.A;
  const int n = A.n, m = A.m;
  if (A.f) potentials_out<Real><<<(n + 255) / 256, 256, 0, st>>>(S.sk.F, n, A.tau / 1.4426950408889634, A.f);
  if (A.g) potentials_out<Real><<<(m + 255) / 256, 256, 0, st>>>(S.sk.G, m, A.tau / 1.4426950408889634, A.g);
  if (!A.stats) return GW_OK;
  TraceScope ts(A.tracer, "solve_stats", st);
  // E(T) = <G(T; T's marginals), T>; the gradient overwrites Pi.
  int rc = gradient(S, 1, 1.0, st);
  if (rc != GW_OK) return rc;
  dot_partial<Real><<<kDots, 256, 0, st>>>(S.sk.Pi, (const Real*)A.T, (size_t)n * m, S.dotE);
  if (fused<Real>(A))
  {
    // <CC, T>: tile partials in Pi's storage (free after the dot above), summed
    // into dotC[0]; the other kDots - 1 entries are zero.
    const dim3 grid((m + 255) / 256, (n + kFeatRows - 1) / kFeatRows);
    double* tiles = reinterpret_cast<double*>(const_cast<Real*>(S.sk.Pi));
    feature_dot_tiles<Real><<<grid, 256, 0, st>>>((const Real*)A.T, n, m, A.feat_dim, A.phi, A.psi, tiles);
    fill_val<double><<<1, 256, 0, st>>>(S.dotC, kDots, 0.0);
    sum_partials<<<1, 256, 0, st>>>(tiles, (int)(grid.x * grid.y), S.dotC);
  } else
    fill_val<double><<<1, 256, 0, st>>>(S.dotC, kDots, 0.0);
  finish_stats<<<1, 256, 0, st>>>(S.dotE, kDots, S.dotC, kDots, S.sk.cta_stats, S.sk.B, S.sk.colpart, m, A.v, A.eps,
                                  A.theta, A.n_outer, A.stats);
  if (A.rho > 0.0) {
    ugw_scalars(S, st);
    ugw_stats<<<1, 1, 0, st>>>(S.ugw_scal, A.rho, A.eps, A.stats);
  }
  return GW_OK;
}

// Launches one Sinkhorn pass (rows, then columns), or the plan, over a list
// of problems in parameter blocks of up to MAXP problems each.
template <int NW, int VPT, int NG, typename Real, int MAXP>
int launch_rows(SolveState<Real>* const* S, int count, bool plan, cudaStream_t st, unsigned* status,
                Tracer* tracer) {
  for (int base = 0; base < count; base += MAXP) {
    const int cnt = std::min(MAXP, count - base);
    SkBatch<Real, MAXP> P;
    memset(&P, 0, sizeof(P));
    P.count = cnt;
    size_t smem = 0;
    int blocks = 0;
    for (int q = 0; q < cnt; ++q) {
      P.p[q] = S[base + q]->sk;
      P.block0[q] = blocks;
      blocks += P.p[q].B;
      smem = std::max(smem, plan ? S[base + q]->smem_plan : S[base + q]->smem_pass);
    }
    P.block0[cnt] = blocks;
    auto kern = plan ? sk_plan<NW, VPT, Real, MAXP> : sk_pass<NW, VPT, NG, Real, MAXP>;
    if (!allow_dynamic_smem((const void*)kern, smem))
      return GW_ERR_CUDA;
    {
      TraceScope ts(tracer, plan ? "sk_plan" : "sk_pass", st);
      kern<<<blocks, plan ? 32 * NW : 32 * NW * NG, smem, st>>>(P, status);
    }
    if (plan) continue;
    // Column update: blocks of 32 columns.
    blocks = 0;
    for (int q = 0; q < cnt; ++q) {
      P.block0[q] = blocks;
      blocks += (P.p[q].m + 31) / 32;
    }
    P.block0[cnt] = blocks;
    TraceScope ts(tracer, "sk_cols", st);
    sk_cols<Real, MAXP><<<blocks, 256, 0, st>>>(P);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

template <int NW, int VPT, int NG, typename Real>
int solve_typed(const SolveArgs& A, void* ws, size_t ws_bytes) {
  cudaStream_t st = A.stream;
  SolveState<Real> S;
  int rc = prepare<NW, VPT, NG, Real>(A, ws, ws_bytes, &S);
  if (rc != GW_OK) return rc;
  SolveState<Real>* list[1] = {&S};
  step_setup(S, st);
  for (int l = 0; l < A.n_outer; ++l) {
    rc = step_cost(S, st, l);
    if (rc != GW_OK) return rc;
    for (int it = 0; it < A.n_inner; ++it) {
      rc = launch_rows<NW, VPT, NG, Real, 1>(list, 1, false, st, A.status, A.tracer);
      if (rc != GW_OK) return rc;
    }
    if (l + 1 < A.n_outer && plan_on_the_fly(A)) continue;  // the next gradient forms the plan
    rc = launch_rows<NW, VPT, NG, Real, 1>(list, 1, true, st, A.status, A.tracer);
    if (rc != GW_OK) return rc;
    step_after_plan(S, st);
  }
  rc = step_finish(S, st);
  if (rc != GW_OK) return rc;
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

// A group of problems with the same row configuration and schedule, advanced
// in lock step on one stream: each Sinkhorn pass is one launch (per 32
// problems) over all of the group's row bands.
template <int NW, int VPT, int NG, typename Real>
int solve_group(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count, cudaStream_t st) {
  std::vector<SolveState<Real>> S(count);
  std::vector<SolveState<Real>*> list(count);
  for (int i = 0; i < count; ++i) {
    int rc = prepare<NW, VPT, NG, Real>(*A[i], ws[i], ws_bytes[i], &S[i]);
    if (rc != GW_OK) return rc;
    list[i] = &S[i];
  }
  unsigned* status = A[0]->status;
  Tracer* tracer = A[0]->tracer;
  for (auto& s : S) step_setup(s, st);
  for (int l = 0; l < A[0]->n_outer; ++l) {
    for (auto& s : S) {
      int rc = step_cost(s, st, l);
      if (rc != GW_OK) return rc;
    }
    for (int it = 0; it < A[0]->n_inner; ++it) {
      int rc = launch_rows<NW, VPT, NG, Real, 32>(list.data(), count, false, st, status, tracer);
      if (rc != GW_OK) return rc;
    }
    int rc = launch_rows<NW, VPT, NG, Real, 32>(list.data(), count, true, st, status, tracer);
    if (rc != GW_OK) return rc;
    for (auto& s : S) step_after_plan(s, st);
  }
  for (auto& s : S) {
    int rc = step_finish(s, st);
    if (rc != GW_OK) return rc;
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

// Row configurations of the Sinkhorn kernels: warps per row group NW, values
// per thread VPT (a row group covers 32 NW VPT >= m columns), row groups per
// block NG.  Built-in choices by row length: float 40, 0, 48, 50, 45, 51, 46,
// 52, 47, 53, 55, 54 (covers 384, 512, 768, 1024, ..., 12288, 16384: steps of
// 4/3 and 3/2, so that a row just above a power of two does not pay for a row
// twice its length), double 10-13; the other ids are alternatives for the
// tuning table.  The built-in float covers from 768 columns take 24 or 32
// values per thread and as few warps per row as that allows: a row group's
// fixed work per row (its reductions, barrier and scale) is shared by more
// columns, and a block streams more rows at once.  Against 12 and 16 values
// per thread with twice the warps per row, batched passes run 1.35-1.45x and
// 1.1-1.2x as fast, the 8192-column single solve 1.14x.  with_config below
// has one case per entry.
struct SkConfig {
  int id, dtype, nw, vpt, ng;
};
constexpr SkConfig kSkConfigs[] = {
    {0, GW_F32, 1, 16, 16}, {1, GW_F32, 2, 16, 8},  {2, GW_F32, 4, 16, 4},  {3, GW_F32, 8, 16, 2},
    {4, GW_F32, 16, 16, 1}, {5, GW_F32, 18, 16, 1}, {6, GW_F32, 32, 16, 1}, {10, GW_F64, 1, 8, 16},
    {11, GW_F64, 4, 8, 4},  {12, GW_F64, 16, 8, 1}, {13, GW_F64, 32, 16, 1}, {20, GW_F32, 2, 8, 8},
    {21, GW_F32, 4, 8, 4},  {22, GW_F32, 8, 8, 2},  {23, GW_F32, 16, 8, 1}, {24, GW_F32, 32, 8, 1},
    {30, GW_F64, 2, 4, 8},  {31, GW_F64, 8, 4, 2},  {32, GW_F64, 32, 4, 1},  {40, GW_F32, 1, 12, 16},
    {41, GW_F32, 2, 12, 8}, {42, GW_F32, 4, 12, 4}, {43, GW_F32, 8, 12, 2}, {44, GW_F32, 16, 12, 1},
    {45, GW_F32, 2, 24, 8}, {46, GW_F32, 4, 24, 4}, {47, GW_F32, 8, 24, 2}, {48, GW_F32, 1, 24, 16},
    {50, GW_F32, 1, 32, 16}, {51, GW_F32, 2, 32, 8}, {52, GW_F32, 4, 32, 4}, {53, GW_F32, 8, 32, 2},
    {54, GW_F32, 16, 32, 1}, {55, GW_F32, 16, 24, 1},
};

bool sk_config_shape(int id, int* dtype, int* nw, int* vpt, int* ng) {
  for (const SkConfig& c : kSkConfigs)
    if (c.id == id) {
      if (dtype) *dtype = c.dtype;
      if (nw) *nw = c.nw;
      if (vpt) *vpt = c.vpt;
      if (ng) *ng = c.ng;
      return true;
    }
  return false;
}

int sk_config_ids(int* out, int cap) {
  const int count = (int)(sizeof(kSkConfigs) / sizeof(kSkConfigs[0]));
  for (int i = 0; i < count && i < cap; ++i) out[i] = kSkConfigs[i].id;
  return count;
}

// Built-in row configuration for m columns.
int sk_default_config(int m, int dtype) {
  if (dtype == GW_F32) {
    if (m <= 384) return 40;
    if (m <= 512) return 0;
    if (m <= 768) return 48;
    if (m <= 1024) return 50;
    if (m <= 1536) return 45;
    if (m <= 2048) return 51;
    if (m <= 3072) return 46;
    if (m <= 4096) return 52;
    if (m <= 6144) return 47;
    if (m <= 8192) return 53;
    if (m <= 12288) return 55;
    return 54;
  }
  if (m <= 256) return 10;
  if (m <= 1024) return 11;
  if (m <= 4096) return 12;
  return 13;
}

// Configuration in effect for m columns: the tuning table's entry, else the
// built-in choice.  The index also groups batched problems.
int row_config(int m, int dtype) {
  const int t = tune_lookup(GW_TUNE_SINKHORN, dtype, m);
  return t >= 0 ? t : sk_default_config(m, dtype);
}

template <typename F>
int with_config(int cfg, F&& f) {
  switch (cfg) {
    case 0: return f.template run<1, 16, 16, float>();
    case 1: return f.template run<2, 16, 8, float>();
    case 2: return f.template run<4, 16, 4, float>();
    case 3: return f.template run<8, 16, 2, float>();
    case 4: return f.template run<16, 16, 1, float>();
    case 5: return f.template run<18, 16, 1, float>();
    case 6: return f.template run<32, 16, 1, float>();
    case 10: return f.template run<1, 8, 16, double>();
    case 11: return f.template run<4, 8, 4, double>();
    case 12: return f.template run<16, 8, 1, double>();
    case 20: return f.template run<2, 8, 8, float>();
    case 21: return f.template run<4, 8, 4, float>();
    case 22: return f.template run<8, 8, 2, float>();
    case 23: return f.template run<16, 8, 1, float>();
    case 24: return f.template run<32, 8, 1, float>();
    case 40: return f.template run<1, 12, 16, float>();
    case 41: return f.template run<2, 12, 8, float>();
    case 42: return f.template run<4, 12, 4, float>();
    case 43: return f.template run<8, 12, 2, float>();
    case 44: return f.template run<16, 12, 1, float>();
    case 45: return f.template run<2, 24, 8, float>();
    case 46: return f.template run<4, 24, 4, float>();
    case 47: return f.template run<8, 24, 2, float>();
    case 48: return f.template run<1, 24, 16, float>();
    case 50: return f.template run<1, 32, 16, float>();
    case 51: return f.template run<2, 32, 8, float>();
    case 52: return f.template run<4, 32, 4, float>();
    case 53: return f.template run<8, 32, 2, float>();
    case 54: return f.template run<16, 32, 1, float>();
    case 55: return f.template run<16, 24, 1, float>();
    case 30: return f.template run<2, 4, 8, double>();
    case 31: return f.template run<8, 4, 2, double>();
    case 32: return f.template run<32, 4, 1, double>();
    default: return f.template run<32, 16, 1, double>();
  }
}

size_t solve_workspace_bytes(const SolveArgs& A) {
  const int n = A.n, m = A.m;
  const size_t rb = A.dtype == GW_F32 ? 4 : 8;
  const Bands bands = solve_bands(A);
  size_t b = 0;
  auto add = [&](size_t x) { b = (b + x + 255) / 256 * 256; };
  add((size_t)n * m * rb);
  add(n * rb);
  add(m * rb);
  add(n * rb);
  add(m * rb);
  add((size_t)bands.B * m * rb);
  add((size_t)bands.B * m * 8);
  add((size_t)2 * bands.B * 8);
  add(kDots * 8);
  add(kDots * 8);
  add((size_t)n * 8);
  add((size_t)n * 8);
  add(kUgwScal * 8);
  const size_t g = A.dense_x ? dense_x_workspace_bytes(n, m, A.dtype)
                  : A.dim >= 2 ? grid_grad_workspace_bytes(A.dim, A.nx, A.ny, A.dtype, A.cost, A.k)
                               : grad1d_workspace_bytes(n, m, A.k, A.dtype, A.num_sms);
  return b + g + 4096;
}

namespace {
struct SingleRun {
  const SolveArgs& A;
  void* ws;
  size_t bytes;
  template <int NW, int VPT, int NG, typename Real>
  int run() {
    return solve_typed<NW, VPT, NG, Real>(A, ws, bytes);
  }
};
struct GroupRun {
  const SolveArgs* const* A;
  void* const* ws;
  const size_t* bytes;
  int count;
  cudaStream_t st;
  template <int NW, int VPT, int NG, typename Real>
  int run() {
    return solve_group<NW, VPT, NG, Real>(A, ws, bytes, count, st);
  }
};
}  // namespace

int solve_launch(const SolveArgs& A, void* ws, size_t ws_bytes) {
  SingleRun r{A, ws, ws_bytes};
  return with_config(row_config(A.m, A.dtype), r);
}

int solve_group_key(const SolveArgs& A) { return row_config(A.m, A.dtype); }

// ---------------------------------------------------------------------------
// Mixed batches: problems of one schedule whose row configurations run
// 512-thread blocks share every Sinkhorn launch (sk_pass_mix, sk_cols_mix).
// ---------------------------------------------------------------------------
// Rows above 8192 columns run in groups of their own configuration: their
// variants in the shared kernel would push its register allocation into
// spills for every problem.
bool solve_mixable(const SolveArgs& A) {
  int dt = 0, nw = 0, vpt = 0, ng = 0;
  if (!sk_config_shape(row_config(A.m, A.dtype), &dt, &nw, &vpt, &ng)) return false;
  return 32 * nw * ng == kMixThreads && 32 * nw * vpt <= 8192;
}

namespace {
template <typename Real>
size_t mix_table_bytes(int count) {
  return ((size_t)count * sizeof(SkProb<Real>) + 255) / 256 * 256;
}

template <typename Real>
struct PrepareRun {
  const SolveArgs& A;
  void* ws;
  size_t bytes;
  SolveState<Real>* S;
  template <int NW, int VPT, int NG, typename R>
  int run() {
    if constexpr (std::is_same<R, Real>::value) return prepare<NW, VPT, NG, Real>(A, ws, bytes, S);
    return GW_ERR_INVALID;
  }
};

template <typename Real>
struct PlanRun {
  SolveState<Real>* const* S;
  int count;
  cudaStream_t st;
  unsigned* status;
  Tracer* tracer;
  template <int NW, int VPT, int NG, typename R>
  int run() {
    if constexpr (std::is_same<R, Real>::value) return launch_rows<NW, VPT, NG, Real, 32>(S, count, true, st, status, tracer);
    return GW_ERR_INVALID;
  }
};

// States of all problems (each prepared with its own row configuration),
// their configuration ids, and the host image of the device table.
template <typename Real>
int mixed_prepare(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count,
                  std::vector<SolveState<Real>>& S, std::vector<int>& cfg) {
  S.assign(count, SolveState<Real>{});
  cfg.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    cfg[i] = row_config(A[i]->m, A[i]->dtype);
    PrepareRun<Real> r{*A[i], ws[i], ws_bytes[i], &S[i]};
    const int rc = with_config(cfg[i], r);
    if (rc != GW_OK) return rc;
  }
  return GW_OK;
}

template <typename Real>
int mixed_table_typed(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count, void* host) {
  std::vector<SolveState<Real>> S;
  std::vector<int> cfg;
  int rc = mixed_prepare<Real>(A, ws, ws_bytes, count, S, cfg);
  if (rc != GW_OK) return rc;
  char* h = (char*)host;
  memset(h, 0, mix_table_bytes<Real>(count));
  SkProb<Real>* probs = (SkProb<Real>*)h;
  for (int i = 0; i < count; ++i) probs[i] = S[i].sk;
  return GW_OK;
}

template <typename Real>
int mixed_launch_typed(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count,
                       const void* dev, cudaStream_t main, const cudaStream_t* workers, int nworkers,
                       cudaEvent_t fork, const cudaEvent_t* join) {
  std::vector<SolveState<Real>> S;
  std::vector<int> cfg;
  int rc = mixed_prepare<Real>(A, ws, ws_bytes, count, S, cfg);
  if (rc != GW_OK) return rc;
  // Parameter blocks of at most kMixMax problems each.
  std::vector<SkMixTable<Real>> tabs;
  std::vector<int> tblocks, tcblocks;
  size_t smem = 0;
  for (int base = 0; base < count; base += kMixMax) {
    SkMixTable<Real> T;
    memset(&T, 0, sizeof(T));
    T.probs = (const SkProb<Real>*)dev + base;
    T.count = std::min(kMixMax, count - base);
    int blocks = 0, cblocks = 0;
    for (int q = 0; q < T.count; ++q) {
      const SolveState<Real>& st = S[base + q];
      T.cfg[q] = cfg[base + q];
      T.block0[q] = blocks;
      T.cblock0[q] = cblocks;
      blocks += st.sk.B;
      cblocks += (st.sk.m + 31) / 32;
      smem = std::max(smem, st.smem_pass);
    }
    T.block0[T.count] = blocks;
    T.cblock0[T.count] = cblocks;
    tabs.push_back(T);
    tblocks.push_back(blocks);
    tcblocks.push_back(cblocks);
  }
  if (!allow_dynamic_smem((const void*)sk_pass_mix<Real>, smem)) return GW_ERR_CUDA;
  // Problems with the same configuration share their plan launches.
  std::map<int, std::vector<SolveState<Real>*>> by_cfg;
  for (int i = 0; i < count; ++i) by_cfg[cfg[i]].push_back(&S[i]);
  unsigned* status = A[0]->status;
  Tracer* tracer = A[0]->tracer;
  const int nw = std::max(1, nworkers);
  auto fork_out = [&]() -> int {
    if (cudaEventRecord(fork, main) != cudaSuccess) return GW_ERR_CUDA;
    for (int k = 0; k < nw; ++k)
      if (cudaStreamWaitEvent(workers[k], fork, 0) != cudaSuccess) return GW_ERR_CUDA;
    return GW_OK;
  };
  auto join_in = [&]() -> int {
    for (int k = 0; k < nw; ++k) {
      if (cudaEventRecord(join[k], workers[k]) != cudaSuccess) return GW_ERR_CUDA;
      if (cudaStreamWaitEvent(main, join[k], 0) != cudaSuccess) return GW_ERR_CUDA;
    }
    return GW_OK;
  };
  // Per-problem work (setup, each step's cost, the step's end) runs on the
  // worker streams, problem i on worker i mod nw; the Sinkhorn passes of all
  // problems run on `main`, one launch each.
  if ((rc = fork_out()) != GW_OK) return rc;
  for (int i = 0; i < count; ++i) step_setup(S[i], workers[i % nw]);
  const int n_outer = A[0]->n_outer, n_inner = A[0]->n_inner;
  for (int l = 0; l < n_outer; ++l) {
    for (int i = 0; i < count; ++i)
      if ((rc = step_cost(S[i], workers[i % nw], l)) != GW_OK) return rc;
    if ((rc = join_in()) != GW_OK) return rc;
    for (int it = 0; it < n_inner; ++it) {
      for (size_t t = 0; t < tabs.size(); ++t) {
        TraceScope ts(tracer, "sk_pass", main);
        sk_pass_mix<Real><<<tblocks[t], kMixThreads, smem, main>>>(tabs[t], status);
      }
      for (size_t t = 0; t < tabs.size(); ++t) {
        TraceScope ts(tracer, "sk_cols", main);
        sk_cols_mix<Real><<<tcblocks[t], 256, 0, main>>>(tabs[t]);
      }
    }
    for (auto& kv : by_cfg) {
      PlanRun<Real> r{kv.second.data(), (int)kv.second.size(), main, status, tracer};
      if ((rc = with_config(kv.first, r)) != GW_OK) return rc;
    }
    if ((rc = fork_out()) != GW_OK) return rc;
    for (int i = 0; i < count; ++i) step_after_plan(S[i], workers[i % nw]);
  }
  for (int i = 0; i < count; ++i)
    if ((rc = step_finish(S[i], workers[i % nw])) != GW_OK) return rc;
  if ((rc = join_in()) != GW_OK) return rc;
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}
}  // namespace

size_t solve_mixed_table_bytes(int count, int dtype) {
  return dtype == GW_F32 ? mix_table_bytes<float>(count) : mix_table_bytes<double>(count);
}

int solve_mixed_table(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count, void* host) {
  if (count <= 0) return GW_OK;
  if (A[0]->dtype == GW_F32) return mixed_table_typed<float>(A, ws, ws_bytes, count, host);
  return mixed_table_typed<double>(A, ws, ws_bytes, count, host);
}

int solve_mixed_launch(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count,
                       const void* dev_table, cudaStream_t main, const cudaStream_t* workers, int nworkers,
                       cudaEvent_t fork, const cudaEvent_t* join) {
  if (count <= 0) return GW_OK;
  if (A[0]->dtype == GW_F32)
    return mixed_launch_typed<float>(A, ws, ws_bytes, count, dev_table, main, workers, nworkers, fork, join);
  return mixed_launch_typed<double>(A, ws, ws_bytes, count, dev_table, main, workers, nworkers, fork, join);
}

int solve_group_launch(const SolveArgs* const* A, void* const* ws, const size_t* ws_bytes, int count,
                       cudaStream_t stream) {
  if (count <= 0) return GW_OK;
  GroupRun r{A, ws, ws_bytes, count, stream};
  return with_config(row_config(A[0]->m, A[0]->dtype), r);
}

}  // namespace gw
