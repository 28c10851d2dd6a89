// Warp-specialised row kernel of the structured 1D gradient (k = 1, 2; up to
// 8192 columns).  Same arithmetic as k1c_grad_rows; the work of a row is split
// between NW compute warps and one scan warp, and consecutive rows overlap:
//
//   compute warps, row t (phase A): wait for the row in the shared-memory ring,
//     column recursion, in-chunk forward walk, float lane scan, post the warp
//     total -> named barrier "totals(t)";
//   scan warp: waits on totals(t), refills the ring slot freed by row t-1
//     (TMA), scans the NW warp totals in float-float (forward prefixes and
//     backward suffixes) and posts, per warp, the polynomial ZW(o) of z over
//     the warp's segment -> named barrier "poly(t)";
//   compute warps, row t-1 (phase B, after phase A of row t): wait on
//     poly(t-1), add the in-warp terms, add the constant term, store G.
//
// Barriers are double-buffered by row parity, so neither side can run more
// than one row ahead of the other.  Rows are stored in shared memory with the
// 128-byte swizzle (16-byte chunk index XOR 128-byte row index mod 8), which
// makes the per-thread 16-byte reads conflict-free; TMA tensor copies write
// that layout directly.
#pragma once

#include <cuda.h>

#include "gw_tma.cuh"

namespace gw {

struct FastGeom {
  int slot_bytes;  // ring slot size (multiple of 1024)
  int vec_bytes;   // one swizzled vector of m_pad reals (multiple of 1024)
};

// Odd K: the in-chunk forward states of the pending row go from phase A(t) to
// phase B(t) in registers for float; for double (twice the registers) they go
// through a shared-memory buffer.
template <int K, typename Real>
struct FastFl {
  static constexpr bool in_smem = (K & 1) && sizeof(Real) != 4;
};

template <int K, int NW, int VPT, typename Real>
struct FastSmem {
  static constexpr int NT = 32 * NW;
  static constexpr size_t fl_bytes = FastFl<K, Real>::in_smem ? sizeof(Real) * (size_t)VPT * NT + 16 : 0;
  static size_t bytes(int slot_bytes, int vec_bytes, int stages) {
    size_t b = 1024;  // alignment slack
    b += (size_t)stages * slot_bytes;
    b += 2 * (size_t)vec_bytes;                     // cy hi, lo
    b += (size_t)vec_bytes;                         // output staging, one warp segment per warp
    b += 8 * (size_t)stages;                        // mbarriers
    b += sizeof(Real) * 2 * NW * 2 * (K + 1);       // warp totals [2][NW][2][K+1]
    b += sizeof(Real) * 2 * NW * (K + 2) + 64;      // polynomials [2][NW][K+2]
    b += fl_bytes;                                  // pending in-chunk forward states (double)
    return b;
  }
};

// KX: exponent of the column transform (X); K: of the row transform (Y).
// REGEN: the ring holds rows of Pi and T is formed from them (rF, rG, rc).
template <int KX, int K, int NW, int VPT, typename Real, bool REGEN = false>
__global__ void __launch_bounds__(32 * (NW + 1), 1)
    k1c_fast_rows(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmG,
                  int use_tma_store, const Real* __restrict__ T, Real* __restrict__ G, int n,
                  int m, int R, const Real* __restrict__ q, const Real* __restrict__ cxh,
                  const Real* __restrict__ cxl, const Real* __restrict__ cyh, const Real* __restrict__ cyl, Real scale,
                  int use_tma, int stages, int slot_bytes, int vec_bytes, int box_cols, int ncopies,
                  const Real* __restrict__ rF, const Real* __restrict__ rG, Real rc, unsigned* status) {
  using A = typename AccT<Real>::type;
  constexpr int kL2Ahead = 4;
  constexpr int NT = 32 * NW;        // compute threads
  constexpr int ALL = NT + 32;       // + scan warp
  constexpr int SEG = 32 * VPT;      // columns per compute warp
  constexpr Real CK = (K & 1) ? (Real)2 : (Real)0;
  static_assert((K == 1 || K == 2) && (KX == 1 || KX == 2), "fast row kernel handles k = 1, 2");

  extern __shared__ __align__(16) unsigned char smem_dyn[];
  // 1024-byte aligned start (the 128-byte swizzle repeats every 1 KB); the
  // pointer stays derived from the shared array so accesses stay shared.
  unsigned char* sm = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  unsigned char* ring = sm;
  unsigned char* cyH = ring + (size_t)stages * slot_bytes;
  unsigned char* cyL = cyH + vec_bytes;
  // Output staging: warp w's SEG outputs of a row, swizzled like the ring, so
  // that each warp writes its segment to global memory 512 contiguous bytes
  // per store instruction.
  unsigned char* stg = cyL + vec_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + vec_bytes);
  Real* wtot = reinterpret_cast<Real*>(bars + stages);             // [2][NW][2][K+1]
  Real* zw = wtot + 2 * NW * 2 * (K + 1);                          // [2][NW][K+2]
  // Double only: in-chunk forward states of the pending row, [VPT/PER][NT]
  // 16-byte chunks.
  constexpr bool FL_SMEM = FastFl<K, Real>::in_smem;
  unsigned char* flraw = reinterpret_cast<unsigned char*>(zw + 2 * NW * (K + 2));
  float4* flbuf = reinterpret_cast<float4*>(flraw + ((16u - (smem_u32(flraw) & 15u)) & 15u));

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int a = blockIdx.x;
  const int s = a * R;
  const int Ra = min(R, n - s);
  const int m_pad = vec_bytes / (int)sizeof(Real);

  // Set-up: barriers, constant term of the columns into swizzled smem.
  if (tid == 0 && use_tma) {
    for (int st = 0; st < stages; ++st) mbar_init(&bars[st], 1);
    fence_mbar_init();
  }
  for (int p = tid; p < m_pad; p += ALL) {
    sts_swz<Real>(cyH, p, p < m ? cyh[p] : (Real)0);
    sts_swz<Real>(cyL, p, p < m ? cyl[p] : (Real)0);
  }
  // Columns m .. m_pad of every ring slot stay zero (TMA writes only the
  // first m), so padded columns contribute nothing without per-element masks.
  for (int st = 0; st < stages; ++st)
    for (int p = m + tid; p < m_pad; p += ALL) sts_swz<Real>(ring + (size_t)st * slot_bytes, p, (Real)0);
  __syncthreads();

  if (warp == NW) {
    // ---------------- scan warp ----------------
    auto issue = [&](int row, int slot) {
      mbar_arrive_expect_tx(&bars[slot], (unsigned)(m * sizeof(Real)));
      for (int c = 0; c < ncopies; ++c)
        tma_load_3d(ring + (size_t)slot * slot_bytes + (size_t)c * box_cols * 128, &tmT, 0, c * box_cols, row, &bars[slot]);
    };
    // Rows kL2Ahead beyond the ring are pulled into L2 early, so that more
    // bytes per SM are in flight than the ring's slots hold.
    const unsigned row_bytes = (unsigned)(m * sizeof(Real));
    auto prefetch = [&](int t) {
      if (t < Ra) bulk_prefetch_l2(T + (size_t)(s + t) * m, row_bytes);
    };
    if (use_tma && lane == 0) {
      for (int st = 0; st < stages - 1 && st < Ra; ++st) issue(s + st, st);
      for (int q = 0; q < kL2Ahead; ++q) prefetch(stages - 1 + q);
    }
    for (int t = 0; t < Ra; ++t) {
      named_sync(1 + (t & 1), ALL);  // totals(t) posted
      if (use_tma && lane == 0) {
        const int nt = t + stages - 1;
        if (nt < Ra) issue(s + nt, nt % stages);
        prefetch(nt + kL2Ahead);
      }
      const Real* wt = wtot + (t & 1) * NW * 2 * (K + 1);
      A W[K + 1], V[K + 1];
      // Warp `lane`'s moments about its end (W) and about its start (V).
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        W[r] = (lane < NW) ? acc_of(wt[lane * 2 * (K + 1) + r]) : acc_zero((A*)nullptr);
        V[r] = (lane < NW) ? acc_of(wt[lane * 2 * (K + 1) + K + 1 + r]) : acc_zero((A*)nullptr);
      }
#pragma unroll
      for (int d = 1; d < NW; d <<= 1) {
        A o[K + 1], ob[K + 1];
#pragma unroll
        for (int r = 0; r <= K; ++r) {
          o[r] = acc_shfl_up(W[r], d);
          ob[r] = acc_shfl_down(V[r], d);
        }
        shift_acc_pow2<K>(o, (Real)(d * SEG));
        shift_acc_pow2<K>(ob, (Real)(d * SEG));
        if (lane >= d) {
#pragma unroll
          for (int r = 0; r <= K; ++r) W[r] = acc_add(W[r], o[r]);
        }
        if (lane + d < NW) {
#pragma unroll
          for (int r = 0; r <= K; ++r) V[r] = acc_add(V[r], ob[r]);
        }
      }
      // Exclusive forward prefix (about the warp start); V is already the
      // inclusive suffix about the warp start.
      A P[K + 1];
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        P[r] = acc_shfl_up(W[r], 1);
        if (lane == 0) P[r] = acc_zero((A*)nullptr);
      }
      if (lane < NW) {
        Real* z = zw + ((t & 1) * NW + lane) * (K + 2);
        // ZW_e = C(K, K-e) [P_{K-e} + (-1)^e V_{K-e}]
        const A z0 = acc_add(P[K], V[K]);
        z[0] = (Real)acc_hi(z0);
        z[1] = (Real)acc_lo(z0);
#pragma unroll
        for (int e = 1; e <= K; ++e) {
          const int u = K - e;
          A t2 = (e & 1) ? acc_sub(P[u], V[u]) : acc_add(P[u], V[u]);
          z[1 + e] = (Real)binom(K, u) * (Real)acc_round(t2);
        }
      }
      named_arrive(3 + (t & 1), ALL);  // poly(t) posted
    }
    return;
  }

  // ---------------- compute warps ----------------
  const int c0 = tid * VPT;
  const int o0 = lane * VPT;  // offset inside the warp segment
  // Column state: KX = 1 difference form (y_t, b_t); KX = 2 Horner (q0, q1, q2).
  Real cst[VPT][KX + 1];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int p = c0 + v;
#pragma unroll
    for (int e = 0; e <= KX; ++e) cst[v][e] = (p < m) ? q[((size_t)a * (KX + 1) + e) * m + p] : (Real)0;
  }
  constexpr int PER = 16 / sizeof(Real);
  // REGEN: the ring holds rows of Pi and T = 2^(F_i + G_p - c Pi) is formed
  // from them, with the columns' potentials G_p kept in registers (-inf for
  // the padding columns, whose T stays 0).
  Real gp[REGEN ? VPT : 1];
  if constexpr (REGEN) {
#pragma unroll
    for (int v = 0; v < VPT; ++v) gp[v] = c0 + v < m ? rG[c0 + v] : (Real)-INFINITY;
  }
  Real ex_prev[K + 1];
  // In-chunk forward states of the pending row (odd K, float).
  Real fl_prev[VPT];
  Real cxh_prev = 0, cxl_prev = 0;
#pragma unroll
  for (int r = 0; r <= K; ++r) ex_prev[r] = 0;
#pragma unroll
  for (int v = 0; v < VPT; ++v) fl_prev[v] = 0;

  for (int t = 0; t <= Ra; ++t) {
    Real fl_new[VPT];
    Real ex_new[K + 1];
    Real cxh_new = 0, cxl_new = 0;
    if (t < Ra) {
      // ---- phase A(t)
      const int i = s + t;
      const unsigned char* xr;
      if (use_tma) {
        const int slot = t % stages;
        mbar_wait_bounded(&bars[slot], (unsigned)((t / stages) & 1), status);
        xr = ring + (size_t)slot * slot_bytes;
      } else {
        unsigned char* dst = ring + (size_t)(t & 1) * slot_bytes;
        const Real* src = T + (size_t)i * m;
        for (int p = tid; p < m_pad; p += NT) sts_swz<Real>(dst, p, p < m ? src[p] : (Real)0);
        named_sync(5, NT);
        xr = dst;
      }
      cxh_new = cxh[i];
      cxl_new = cxl[i];
      // Column recursion and in-chunk forward walk, 16 bytes of the row at a
      // time; also the chunk's moments about its end (agg) and about its
      // start (bag, orders >= 1; order 0 is agg[0]).
      Real agg[K + 1], bag[K + 1];
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        agg[r] = 0;
        bag[r] = 0;
      }
      const Real tr = (Real)t;
      float4 xv[VPT / PER];
#pragma unroll
      for (int j = 0; j < VPT / PER; ++j)
        xv[j] = *reinterpret_cast<const float4*>(xr + swz128((uint32_t)((c0 + j * PER) * sizeof(Real))));
      if constexpr (REGEN) {
        const Real fi = rF[i];
#pragma unroll
        for (int j = 0; j < VPT / PER; ++j) {
          Real* x = reinterpret_cast<Real*>(&xv[j]);
#pragma unroll
          for (int w = 0; w < PER; ++w) x[w] = ex2(fma(-rc, x[w], gp[j * PER + w] + fi));
        }
      }
#pragma unroll
      for (int j = 0; j < VPT / PER; ++j) {
        const Real* x = reinterpret_cast<const Real*>(&xv[j]);
#pragma unroll
        for (int w = 0; w < PER; ++w) {
          const int v = j * PER + w;
          Real y;
          if constexpr (KX == 1) {
            y = cst[v][0];
            cst[v][1] = fma((Real)2, x[w], cst[v][1]);
            cst[v][0] += cst[v][1];
          } else {
            y = fma(fma(cst[v][2], tr, cst[v][1]), tr, cst[v][0]);
          }
          if constexpr (K & 1) {
            fl_new[v] = agg[K];
            pascal_step<K>(agg, y);
          } else {
            const Real wv = (Real)(VPT - v);
            agg[0] += y;
            agg[1] = fma(wv, y, agg[1]);
            agg[2] = fma(wv * wv, y, agg[2]);
          }
          const Real vv = (Real)v;
          bag[1] = fma(vv, y, bag[1]);
          if constexpr (K >= 2) bag[2] = fma(vv * vv, y, bag[2]);
        }
      }
      bag[0] = agg[0];
      // The chunk's moments about the warp start: sum_u C(r,u) o0^{r-u} bag_u
      // (non-negative terms).  Summed over the lanes below (plain butterfly).
      Real csum[K + 1];
      {
        const Real of = (Real)o0;
        csum[0] = bag[0];
        csum[1] = fma(of, bag[0], bag[1]);
        if constexpr (K >= 2) csum[2] = fma(of, fma(of, bag[0], (Real)2 * bag[1]), bag[2]);
      }
      // Lane scan of agg (float, inclusive, about my chunk end) interleaved
      // with the butterfly sum of csum.
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        Real o[K + 1], oc[K + 1];
#pragma unroll
        for (int r = 0; r <= K; ++r) {
          o[r] = __shfl_up_sync(0xffffffffu, agg[r], d);
          oc[r] = __shfl_xor_sync(0xffffffffu, csum[r], d);
        }
        shift_real<K>(o, (Real)(d * VPT));
        if (lane >= d) {
#pragma unroll
          for (int r = 0; r <= K; ++r) agg[r] += o[r];
        }
#pragma unroll
        for (int r = 0; r <= K; ++r) csum[r] += oc[r];
      }
#pragma unroll
      for (int r = 0; r <= K; ++r) {
        ex_new[r] = __shfl_up_sync(0xffffffffu, agg[r], 1);
        if (lane == 0) ex_new[r] = 0;
      }
      if (lane == 31) {
        Real* wt = wtot + ((t & 1) * NW + warp) * 2 * (K + 1);
#pragma unroll
        for (int r = 0; r <= K; ++r) wt[r] = agg[r];
      }
      if (lane == 0) {
        Real* wt = wtot + ((t & 1) * NW + warp) * 2 * (K + 1) + (K + 1);
#pragma unroll
        for (int r = 0; r <= K; ++r) wt[r] = csum[r];
      }
      named_arrive(1 + (t & 1), ALL);
    }
    if (t >= 1) {
      // ---- phase B(t-1)
      const int tp = t - 1;
      const int i = s + tp;
      named_sync(3 + (tp & 1), ALL);
      const Real* z = zw + ((tp & 1) * NW + warp) * (K + 2);
      Real ZW[K + 2];
#pragma unroll
      for (int e = 0; e < K + 2; ++e) ZW[e] = z[e];
      // Coefficients in v of z at offset o0 + v:
      //   ZT_e = sum_{e' >= e} C(e', e) ZW_{e'} o0^{e'-e} + c_K C(K, K-e) ex_{K-e}
      // (ZW_{0} in two parts; ZW[1] is its low part, ZW[1+e] the others).
      Real ZT[K + 1];
      const Real of = (Real)o0;
#pragma unroll
      for (int e = 1; e <= K; ++e) {
        Real acc = 0;
        Real op = 1;
#pragma unroll
        for (int e2 = e; e2 <= K; ++e2) {
          acc = fma((Real)binom(e2, e) * op, ZW[1 + e2], acc);
          op *= of;
        }
        if constexpr (K & 1) acc = fma(CK * (Real)binom(K, K - e), ex_prev[K - e], acc);
        ZT[e] = acc;
      }
      Real small0 = ZW[1];
      {
        Real op = of;
#pragma unroll
        for (int e2 = 1; e2 <= K; ++e2) {
          small0 = fma(op, ZW[1 + e2], small0);
          op *= of;
        }
        if constexpr (K & 1) small0 = fma(CK, ex_prev[K], small0);
      }
      const Real big0 = fma(-scale, ZW[0], cxh_prev);
      // lo(v) = cx.lo - s (small0 + sum_e ZT_e v^e + c_K F_local(v)), folded.
      Real LC[K + 1];
      LC[0] = fma(-scale, small0, cxl_prev);
#pragma unroll
      for (int e = 1; e <= K; ++e) LC[e] = -scale * ZT[e];
      const Real cks = -scale * CK;
      // The staging segment is free once the previous row's tensor store has
      // read it.
      if (use_tma_store) {
        if (lane == 0) bulk_wait_read();
        __syncwarp();
      }
      // Four (float) or two (double) columns at a time: their constant term
      // from swizzled shared memory, the outputs into the warp's staging
      // segment at the same swizzled offsets.
#pragma unroll
      for (int j = 0; j < VPT / PER; ++j) {
        const uint32_t b = (uint32_t)((c0 + j * PER) * sizeof(Real));
        const float4 hv = *reinterpret_cast<const float4*>(cyH + swz128(b));
        const float4 lv = *reinterpret_cast<const float4*>(cyL + swz128(b));
        const Real* ch = reinterpret_cast<const Real*>(&hv);
        const Real* cl = reinterpret_cast<const Real*>(&lv);
        if constexpr (FL_SMEM) {
          const float4 flv = flbuf[j * NT + tid];
          const Real* flp = reinterpret_cast<const Real*>(&flv);
#pragma unroll
          for (int w = 0; w < PER; ++w) fl_prev[j * PER + w] = flp[w];
        }
        Real out[PER];
#pragma unroll
        for (int w = 0; w < PER; ++w) {
          const int v = j * PER + w;
          const Real vv = (Real)v;
          Real lo = LC[K];
#pragma unroll
          for (int e = K - 1; e >= 0; --e) lo = fma(lo, vv, LC[e]);
          if constexpr (K & 1) lo = fma(cks, fl_prev[v], lo);
          out[w] = (big0 + ch[w]) + (lo + cl[w]);
        }
        float4 ov;
        Real* op = reinterpret_cast<Real*>(&ov);
#pragma unroll
        for (int w = 0; w < PER; ++w) op[w] = out[w];
        *reinterpret_cast<float4*>(stg + swz128(b)) = ov;
      }
      if (use_tma_store) {
        // One tensor store of the warp's segment (the tensor map's 128-byte
        // swizzle matches the staging layout; columns past m are clipped).
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0 && warp * SEG < m) {
          tma_store_3d(&tmG, 0, warp * (SEG * (int)sizeof(Real) / 128), i, stg + (size_t)warp * SEG * sizeof(Real));
          bulk_commit();
        }
      } else {
        __syncwarp();
        // Store pass: lane `lane` takes the 16 bytes at lane * 16 of each
        // 512-byte piece of the warp's segment.
        Real* grow = G + (size_t)i * m;
        const bool row_vec = ((((uintptr_t)grow) & 15) == 0);
#pragma unroll 2
        for (int j = 0; j < VPT / PER; ++j) {
          const int col = warp * SEG + (j * 32 + lane) * PER;
          const float4 ov = *reinterpret_cast<const float4*>(stg + swz128((uint32_t)(col * sizeof(Real))));
          if (row_vec && col + PER <= m) {
            *reinterpret_cast<float4*>(grow + col) = ov;
          } else {
            const Real* op = reinterpret_cast<const Real*>(&ov);
#pragma unroll
            for (int w = 0; w < PER; ++w)
              if (col + w < m) grow[col + w] = op[w];
          }
        }
        // The next row's outputs overwrite the segment only after every lane
        // has read it.
        __syncwarp();
      }
    }
    if (t < Ra) {
      if constexpr (FL_SMEM) {
#pragma unroll
        for (int j = 0; j < VPT / PER; ++j) {
          float4 f;
          Real* fr = reinterpret_cast<Real*>(&f);
#pragma unroll
          for (int w = 0; w < PER; ++w) fr[w] = fl_new[j * PER + w];
          flbuf[j * NT + tid] = f;
        }
      } else if constexpr (K & 1) {
#pragma unroll
        for (int v = 0; v < VPT; ++v) fl_prev[v] = fl_new[v];
      }
#pragma unroll
      for (int r = 0; r <= K; ++r) ex_prev[r] = ex_new[r];
      cxh_prev = cxh_new;
      cxl_prev = cxl_new;
    }
  }
  // The last tensor stores complete before the block's shared memory goes.
  if (use_tma_store && lane == 0) bulk_wait_all();
}

}  // namespace gw
