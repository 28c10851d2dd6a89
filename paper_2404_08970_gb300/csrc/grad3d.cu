// Structured gradient on 3D grids with an axis-separable cost.  Sec. 3.1
// builds the 2D case and notes that higher-dimensional grids differ in
// nothing essential; this is the 3D case of the construction in grad2d.cu.
//
// Points of a side^3 grid are flattened row-major, x = (x0 * side + x1) * side
// + x2.  For the Manhattan distance (k = 1) and the squared Euclidean distance
//   D_X[x, x'] = s_X sum_t A(x_t - x'_t),   A(d) = |d| or d^2,
// with s_X = h_X or h_X^2, so with T[x][y] (x in X's grid, y in Y's)
//   (D_X T D_Y)[x, y] = s_X s_Y sum_{t,t'} Z_tt'[x_t][y_t'],   Z_tt' = A M_tt' A,
//   M_tt'[a][b] = sum over x with x_t = a and y with y_t' = b of T[x][y]
// for the nine axis pairs (t, t').  The constant term splits the same way:
// with the marginal r read as a side^3 array R, its 1D marginals r_t and its
// 2D marginals R_tt' (t < t'),
//   ((D_X o D_X) r)[x] = s_X^2 ( sum_t (A^2 r_t)[x_t] + 2 sum_{t<t'} (A R_tt' A)[x_t][x_t'] ).
// Everything after the single pass over T works on side x side matrices.
//
// Kernels (in launch order):
//   g3_rows    one warp per row of T: the row's sums over each Y axis pair
//              (three vectors of side entries; the only pass over T).
//   g2_colsum  exact marginals only: column sums of T (second pass).
//   g3_stage1  partial sums of the row sums over one X axis; R and C.
//   g3_stage2  the nine M_tt', and the 2D marginals of R and C.
//   g3_stage3  the 1D marginals of R and C.
//   g2_tx      transforms by A from the left, then from the right.
//   g3_tab     the epilogue tables: c_y per column, and per row of X the
//              parts of G that depend on (row, y0), (row, y1), (row, y2).
//   g3_epi     writes G, one warp per row.
//
// Sums are compensated: Kahan in the row pass, float-float (double for
// double data) everywhere after it; outputs are rounded once.
#include <algorithm>
#include <cmath>

#include "gw_common.cuh"
#include "gw_internal.h"

namespace gw {
namespace {

#include "grid_sep.cuh"

template <typename Real>
__device__ __forceinline__ void kahan(Real& s, Real& c, Real x) {
  const Real y = x - c;
  const Real t = s + y;
  c = (t - s) - y;
  s = t;
}

// ---------------------------------------------------------------------------
// g3_rows: per row i of T (length m = sy^3, element (y0,y1,y2) at
// y0*sy^2 + q, q = y1*sy + y2):
//   R0[i][a] = sum_q T[i][a][q],
//   R1[i][b] = sum_{y0,y2} T[i][y0][b][y2],   R2[i][c] = sum_{y0,y1} T[i][y0][y1][c].
// Lane l owns q = l + 32j (j < NQ) and keeps a Kahan sum over y0 for each,
// plus one Kahan partial per y0 over its own q's.  At the end of the row the
// partials, each rounded once (a Kahan sum of at most 32 terms is accurate to
// about one rounding), go through the warp's shared memory (odd row pitch, so
// that both the writes and the column-wise reads are free of bank
// conflicts) and are summed in compensated arithmetic:
//   pq[y1][y2] (pitch S = sy | 1) -> R1, R2 by lanes over y1 or y2;
//   py0[lane][y0] (pitch S)       -> R0 by lanes over y0.
// One row per warp; the launch keeps at least 32 warps per SM resident so
// that the rows of the benchmark grids (4096) fit one wave.
// ---------------------------------------------------------------------------
__host__ __device__ inline int g3_pitch(int sy) { return sy | 1; }
template <typename Real>
__host__ __device__ inline size_t g3_rows_warp_reals(int sy) {
  const int S = g3_pitch(sy);
  return (size_t)sy * S + 32 * (size_t)S;
}

// Blocks per SM the row kernels ask the compiler to keep resident: 64
// registers a thread where the per-lane state fits them without spills
// (float with at most 16 (y1, y2) pairs per lane), 256 for double with 32,
// else 128.
template <typename Real, int NQ>
constexpr int g3_min_blocks(int at64) {
  return (sizeof(Real) == 4 && NQ <= 16) ? at64 : (sizeof(Real) == 8 && NQ >= 32 ? at64 / 4 : at64 / 2);
}

template <typename Real, int NQ>
__global__ void __launch_bounds__(128, g3_min_blocks<Real, NQ>(8))
    g3_rows(const Real* __restrict__ T, int n, int sy, AccOf<Real>* __restrict__ R0, AccOf<Real>* __restrict__ R1,
            AccOf<Real>* __restrict__ R2) {
  using Acc = AccOf<Real>;
  constexpr int CB = NQ >= 16 ? 1 : (NQ >= 8 ? 2 : 4);  // y0's whose loads are issued together
  extern __shared__ __align__(16) unsigned char g3_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int S = g3_pitch(sy);
  const int q2 = sy * sy;
  Real* pq = reinterpret_cast<Real*>(g3_smem) + (size_t)wib * g3_rows_warp_reals<Real>(sy);
  Real* py = pq + (size_t)sy * S;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const size_t m = (size_t)q2 * sy;
  for (int i = w0; i < n; i += nw) {
    const Real* row = T + (size_t)i * m;
    Real as[NQ], ac[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) as[j] = ac[j] = 0;
    for (int y0 = 0; y0 < sy; y0 += CB) {
      Real t[CB][NQ];
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) {
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
          const int q = lane + 32 * j;
          t[cb][j] = (y0 + cb < sy && q < q2) ? __ldcs(row + (size_t)(y0 + cb) * q2 + q) : (Real)0;
        }
      }
#pragma unroll
      for (int cb = 0; cb < CB; ++cb) {
        if (y0 + cb < sy) {
          Real ps = 0, pc = 0;
#pragma unroll
          for (int j = 0; j < NQ; ++j) {
            kahan(as[j], ac[j], t[cb][j]);
            kahan(ps, pc, t[cb][j]);
          }
          py[lane * S + y0 + cb] = ps - pc;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const int q = lane + 32 * j;
      if (q < q2) {
        const int e = (q / sy) * S + q % sy;
        pq[e] = as[j] - ac[j];
      }
    }
    __syncwarp();
    for (int a = lane; a < sy; a += 32) {
      Acc s0 = acc_zero((Acc*)nullptr), s1 = s0, s2 = s0;
      for (int l = 0; l < 32; ++l) s0 = acc_add(s0, acc_of(py[l * S + a]));
      for (int e = 0; e < sy; ++e) {
        s1 = acc_add(s1, acc_of(pq[a * S + e]));
        s2 = acc_add(s2, acc_of(pq[e * S + a]));
      }
      R0[(size_t)i * sy + a] = s0;
      R1[(size_t)i * sy + a] = s1;
      R2[(size_t)i * sy + a] = s2;
    }
    __syncwarp();  // the next row overwrites the partials
  }
}

// Stage 1, one thread per output:
//   S[t'][x0][x1][b] = sum_{x2} R_t'[x][b],   P[t'][x0][x2][b] = sum_{x1} R_t'[x][b]
// (layout [3][sx][sx][sy] each), and the marginals as cubes: R[x] = r_x from
// the target u or, with exact marginals, T's row sums (sum_a R0[x][a]);
// C[y] from v or from the column sums Cm.
template <typename Acc>
__global__ void g3_stage1(const Acc* __restrict__ R0, const Acc* __restrict__ R1, const Acc* __restrict__ R2, int sx,
                          int sy, const double* __restrict__ u, const double* __restrict__ v,
                          const Acc* __restrict__ Cm, int exact, Acc* __restrict__ Sx, Acc* __restrict__ Px,
                          Acc* __restrict__ R, Acc* __restrict__ C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = sx * sx * sy;  // one t' of S or P
  const int n = sx * sx * sx, m = sy * sy * sy;
  Acc s = acc_zero((Acc*)nullptr);
  if (idx < 6 * per) {
    const int which = idx / (3 * per);  // 0: S, 1: P
    const int e = idx % (3 * per);
    const int tp = e / per, r = e % per;
    const int b = r % sy, o1 = (r / sy) % sx, o0 = r / (sy * sx);
    const Acc* src = tp == 0 ? R0 : (tp == 1 ? R1 : R2);
    // S: x = (o0, o1, l); P: x = (o0, l, o1).
    const size_t base = which == 0 ? ((size_t)o0 * sx + o1) * sx : (size_t)o0 * sx * sx + o1;
    const size_t step = which == 0 ? 1 : (size_t)sx;
    for (int l = 0; l < sx; ++l) s = acc_add(s, src[(base + (size_t)l * step) * sy + b]);
    (which == 0 ? Sx : Px)[e] = s;
  } else if (idx < 6 * per + n) {
    const int x = idx - 6 * per;
    if (exact) {
      for (int a = 0; a < sy; ++a) s = acc_add(s, R0[(size_t)x * sy + a]);
    } else {
      s = acc_add_d(s, u[x]);
    }
    R[x] = s;
  } else if (idx < 6 * per + n + m) {
    const int y = idx - 6 * per - n;
    if (exact)
      s = Cm[y];
    else
      s = acc_add_d(s, v[y]);
    C[y] = s;
  }
}

// Stage 2, one thread per output:
//   M[t][t'][a][b] (layout [3][3][sx][sy]): t = 0: sum_{x1} S[t'][a][x1][b];
//   t = 1: sum_{x0} S[t'][x0][a][b];  t = 2: sum_{x0} P[t'][x0][a][b];
//   the 2D marginals of a side^3 cube Q (R with side sx, C with side sy),
//   layout [3][side][side] for the axis pairs (0,1), (0,2), (1,2):
//   Q01[a][b] = sum_c Q[a][b][c], Q02[a][c] = sum_b Q[a][b][c], Q12[b][c] = sum_a Q[a][b][c].
template <typename Acc>
__device__ __forceinline__ Acc cube_pair_sum(const Acc* Q, int side, int pair, int i, int j) {
  Acc s = acc_zero((Acc*)nullptr);
  const size_t ss = (size_t)side * side;
  for (int l = 0; l < side; ++l) {
    size_t o;
    if (pair == 0)
      o = (size_t)i * ss + (size_t)j * side + l;
    else if (pair == 1)
      o = (size_t)i * ss + (size_t)l * side + j;
    else
      o = (size_t)l * ss + (size_t)i * side + j;
    s = acc_add(s, Q[o]);
  }
  return s;
}

template <typename Acc>
__global__ void g3_stage2(const Acc* __restrict__ Sx, const Acc* __restrict__ Px, const Acc* __restrict__ R,
                          const Acc* __restrict__ C, int sx, int sy, Acc* __restrict__ M, Acc* __restrict__ R2d,
                          Acc* __restrict__ C2d) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int pm = sx * sy;
  const int per = sx * sx * sy;
  if (idx < 9 * pm) {
    const int tt = idx / pm, e = idx % pm;
    const int t = tt / 3, tp = tt % 3;
    const int a = e / sy, b = e % sy;
    Acc s = acc_zero((Acc*)nullptr);
    const Acc* src = (t == 2 ? Px : Sx) + (size_t)tp * per;
    for (int l = 0; l < sx; ++l) {
      const size_t o = t == 0 ? ((size_t)a * sx + l) * sy + b : ((size_t)l * sx + a) * sy + b;
      s = acc_add(s, src[o]);
    }
    M[idx] = s;
  } else if (idx < 9 * pm + 3 * sx * sx) {
    const int e = idx - 9 * pm;
    const int pair = e / (sx * sx), r = e % (sx * sx);
    R2d[e] = cube_pair_sum(R, sx, pair, r / sx, r % sx);
  } else if (idx < 9 * pm + 3 * sx * sx + 3 * sy * sy) {
    const int e = idx - 9 * pm - 3 * sx * sx;
    const int pair = e / (sy * sy), r = e % (sy * sy);
    C2d[e] = cube_pair_sum(C, sy, pair, r / sy, r % sy);
  }
}

// Stage 3: the 1D marginals [3][side] from the 2D ones:
//   q0[a] = sum_b Q01[a][b],  q1[b] = sum_a Q01[a][b],  q2[c] = sum_a Q02[a][c].
template <typename Acc>
__global__ void g3_stage3(const Acc* __restrict__ R2d, const Acc* __restrict__ C2d, int sx, int sy,
                          Acc* __restrict__ r1, Acc* __restrict__ c1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool xs = idx < 3 * sx;
  if (!xs && idx >= 3 * sx + 3 * sy) return;
  const int side = xs ? sx : sy;
  const int e = xs ? idx : idx - 3 * sx;
  const Acc* Q = xs ? R2d : C2d;
  const int ax = e / side, i = e % side;
  const size_t ss = (size_t)side * side;
  Acc s = acc_zero((Acc*)nullptr);
  for (int l = 0; l < side; ++l) {
    const size_t o = ax == 0 ? (size_t)i * side + l : (ax == 1 ? (size_t)l * side + i : ss + (size_t)l * side + i);
    s = acc_add(s, Q[o]);
  }
  (xs ? r1 : c1)[e] = s;
}

// Epilogue tables, all hi/lo (rounded once from the compensated values):
//   Cy[y] = scale_y (py_0[y0] + py_1[y1] + py_2[y2] + 2 (WY01[y0][y1] + WY02[y0][y2] + WY12[y1][y2]))
//   U_0[x][j] = scale_x (px_0[x0] + px_1[x1] + px_2[x2] + 2 (WX01 + WX02 + WX12)[x])
//               - scale_z sum_t Z_t0[x_t][j]
//   U_t'[x][j] = -scale_z sum_t Z_tt'[x_t][j]            (t' = 1, 2)
// with scale_x = out_scale s_X^2, scale_y = out_scale s_Y^2 and scale_z =
// 2 out_scale s_X s_Y, so that G[x][y] = U_0[x][y0] + U_1[x][y1] + U_2[x][y2]
// + Cy[y].  Layout: Cy as [m] hi then [m] lo; U as [n][sy][6] (U_0 hi, lo,
// U_1 hi, lo, U_2 hi, lo).
template <typename Real>
__global__ void g3_tab(const AccOf<Real>* __restrict__ Z, const AccOf<Real>* __restrict__ px,
                       const AccOf<Real>* __restrict__ WX, const AccOf<Real>* __restrict__ py,
                       const AccOf<Real>* __restrict__ WY, int sx, int sy, double scale_x, double scale_y,
                       double scale_z, Real* __restrict__ Cy, Real* __restrict__ U) {
  using Acc = AccOf<Real>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = sy * sy * sy, n = sx * sx * sx;
  if (idx < m) {
    const int y0 = idx / (sy * sy), y1 = (idx / sy) % sy, y2 = idx % sy;
    const int q = sy * sy;
    Acc sc;
    acc_from(&sc, scale_y);
    const Acc w = acc_add(acc_add(WY[y0 * sy + y1], WY[q + y0 * sy + y2]), WY[2 * q + y1 * sy + y2]);
    const Acc p = acc_add(acc_add(py[y0], py[sy + y1]), py[2 * sy + y2]);
    const Acc val = acc_mul(acc_add(p, acc_add(w, w)), sc);
    Real hi, lo;
    acc_split(val, hi, lo);
    Cy[idx] = hi;
    Cy[m + idx] = lo;
  } else if (idx < m + n * sy) {
    const int e = idx - m;
    const int x = e / sy, j = e % sy;
    const int x0 = x / (sx * sx), x1 = (x / sx) % sx, x2 = x % sx;
    const int q = sx * sx, pm = sx * sy;
    Acc scx, scz;
    acc_from(&scx, scale_x);
    acc_from(&scz, scale_z);
    const Acc w = acc_add(acc_add(WX[x0 * sx + x1], WX[q + x0 * sx + x2]), WX[2 * q + x1 * sx + x2]);
    const Acc p = acc_add(acc_add(px[x0], px[sx + x1]), px[2 * sx + x2]);
    const Acc cx = acc_mul(acc_add(p, acc_add(w, w)), scx);
    // Z[t][t'] at (t * 3 + t') * pm.
    auto zsum = [&](int tp) {
      return acc_add(acc_add(Z[(size_t)(0 * 3 + tp) * pm + x0 * sy + j], Z[(size_t)(1 * 3 + tp) * pm + x1 * sy + j]),
                     Z[(size_t)(2 * 3 + tp) * pm + x2 * sy + j]);
    };
    const Acc U0 = acc_sub(cx, acc_mul(zsum(0), scz));
    const Acc U1 = acc_neg_of(acc_mul(zsum(1), scz));
    const Acc U2 = acc_neg_of(acc_mul(zsum(2), scz));
    Real* o = U + (size_t)e * 6;
    acc_split(U0, o[0], o[1]);
    acc_split(U1, o[2], o[3]);
    acc_split(U2, o[4], o[5]);
  }
}

// G rows: one warp per row, lane l on q = l + 32j (q = y1*sy + y2); no block
// barriers.  Per row, each lane forms U_1[y1] + U_2[y2] for its q's once (as
// a compensated pair), and U_0[y0] (lane y0 holds it) reaches every lane by a
// shuffle:
//   G[x][(y0,q)] = (U_0[y0] + U_12[q] + Cy[y])_hi + (...)_lo.
template <typename Real, int NQ>
__global__ void __launch_bounds__(256, g3_min_blocks<Real, NQ>(4))
    g3_epi(Real* __restrict__ G, int n, int sy, const Real* __restrict__ Cy, const Real* __restrict__ U) {
  using Acc = AccOf<Real>;
  constexpr bool kLo = sizeof(Real) == 4;
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int q2 = sy * sy;
  const int m = q2 * sy;
  for (int i = w0; i < n; i += nw) {
    const Real* ur = U + (size_t)i * sy * 6;
    const Real u0h = lane < sy ? ur[lane * 6] : (Real)0;
    const Real u0l = lane < sy ? ur[lane * 6 + 1] : (Real)0;
    Real uh[NQ], ul[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const int q = lane + 32 * j;
      if (q < q2) {
        const int y1 = q / sy, y2 = q % sy;
        const Acc s = acc_add(acc_of(ur[y1 * 6 + 2], ur[y1 * 6 + 3]), acc_of(ur[y2 * 6 + 4], ur[y2 * 6 + 5]));
        acc_split(s, uh[j], ul[j]);
      } else {
        uh[j] = ul[j] = 0;
      }
    }
    Real* grow = G + (size_t)i * m;
    for (int y0 = 0; y0 < sy; ++y0) {
      const Real ah = __shfl_sync(0xffffffffu, u0h, y0);
      const Real al = __shfl_sync(0xffffffffu, u0l, y0);
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        const int q = lane + 32 * j;
        if (q < q2) {
          const int p = y0 * q2 + q;
          Real g = (ah + uh[j]) + __ldg(Cy + p);
          if (kLo) g += (al + ul[j]) + __ldg(Cy + m + p);
          __stcs(grow + p, g);
        }
      }
    }
  }
}

// Float rows with the c_y table staged in shared memory (hi and lo side by
// side, one 8-byte shared load per element): loading the table from L2 for
// every element bounded g3_epi (long-scoreboard stalls).  Plain shared loads
// only; everything else as g3_epi.
template <int NQ>
__global__ void __launch_bounds__(512, 2)
    g3_epi_cs(float* __restrict__ G, int n, int sy, const float* __restrict__ Cy, const float* __restrict__ U) {
  extern __shared__ __align__(16) float2 g3_cys[];
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int q2 = sy * sy;
  const int m = q2 * sy;
  for (int p = threadIdx.x; p < m; p += blockDim.x) g3_cys[p] = make_float2(Cy[p], Cy[m + p]);
  __syncthreads();
  for (int i = w0; i < n; i += nw) {
    const float* ur = U + (size_t)i * sy * 6;
    const float u0h = lane < sy ? ur[lane * 6] : 0.f;
    const float u0l = lane < sy ? ur[lane * 6 + 1] : 0.f;
    float uh[NQ], ul[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const int q = lane + 32 * j;
      if (q < q2) {
        const int y1 = q / sy, y2 = q % sy;
        const ff sum = ff_add(acc_of(ur[y1 * 6 + 2], ur[y1 * 6 + 3]), acc_of(ur[y2 * 6 + 4], ur[y2 * 6 + 5]));
        uh[j] = sum.hi;
        ul[j] = sum.lo;
      } else {
        uh[j] = ul[j] = 0.f;
      }
    }
    float* grow = G + (size_t)i * m;
    for (int y0 = 0; y0 < sy; ++y0) {
      const float ah = __shfl_sync(0xffffffffu, u0h, y0);
      const float al = __shfl_sync(0xffffffffu, u0l, y0);
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        const int q = lane + 32 * j;
        if (q < q2) {
          const int p = y0 * q2 + q;
          const float2 cv = g3_cys[p];
          float g = (ah + uh[j]) + cv.x;
          g += (al + ul[j]) + cv.y;
          __stcs(grow + p, g);
        }
      }
    }
  }
}

// Largest c_y table staged in shared memory: two blocks of g3_epi_cs per SM.
constexpr size_t kEpi3SmemMax = 100 * 1024;

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct G3Layout {
  size_t R0, R1, R2, Sx, Px, R, C, M, R2d, C2d, r1, c1, YM, YR, YC, px, py, Z, WX, WY, Cy, U, part, Cm, total;
  int nb;
};

G3Layout g3_layout(int sx, int sy, int dtype) {
  const size_t acc = 8;  // ff or double
  const size_t rb = dtype == GW_F32 ? 4 : 8;
  const size_t n = (size_t)sx * sx * sx, m = (size_t)sy * sy * sy;
  const size_t pm = (size_t)sx * sy;
  G3Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) / 256 * 256;
    return o;
  };
  L.nb = (int)std::min<size_t>(n, 64);
  L.R0 = take(n * sy * acc);
  L.R1 = take(n * sy * acc);
  L.R2 = take(n * sy * acc);
  L.Sx = take(3 * (size_t)sx * sx * sy * acc);
  L.Px = take(3 * (size_t)sx * sx * sy * acc);
  L.R = take(n * acc);
  L.C = take(m * acc);
  L.M = take(9 * pm * acc);
  L.R2d = take(3 * (size_t)sx * sx * acc);
  L.C2d = take(3 * (size_t)sy * sy * acc);
  L.r1 = take(3 * (size_t)sx * acc);
  L.c1 = take(3 * (size_t)sy * acc);
  L.YM = take(9 * pm * acc);
  L.YR = take(3 * (size_t)sx * sx * acc);
  L.YC = take(3 * (size_t)sy * sy * acc);
  L.px = take(3 * (size_t)sx * acc);
  L.py = take(3 * (size_t)sy * acc);
  L.Z = take(9 * pm * acc);
  L.WX = take(3 * (size_t)sx * sx * acc);
  L.WY = take(3 * (size_t)sy * sy * acc);
  L.Cy = take(2 * m * rb);
  L.U = take(n * sy * 6 * rb);
  L.part = take((size_t)L.nb * m * acc);
  L.Cm = take(m * acc);
  L.total = off;
  return L;
}

template <typename Real, int NQ>
int grad3d_typed(const Grad2DArgs& A, void* wsv, size_t ws_bytes) {
  using Acc = AccOf<Real>;
  const int sx = A.sx, sy = A.sy;
  const int n = sx * sx * sx, m = sy * sy * sy;
  const G3Layout L = g3_layout(sx, sy, A.dtype);
  if (L.total > ws_bytes) return GW_ERR_OOM;
  char* ws = (char*)wsv;
  auto P = [&](size_t o) { return (Acc*)(ws + o); };
  cudaStream_t st = A.stream;
  const Real* T = (const Real*)A.T;
  const int sq = A.cost == GW_COST_SQEUCLID ? 1 : 0;
  const double s_x = sq ? A.hx * A.hx : A.hx;
  const double s_y = sq ? A.hy * A.hy : A.hy;
  {
    TraceScope ts(A.tracer, "g3_rows", st);
    const size_t smem = 4 * g3_rows_warp_reals<Real>(sy) * sizeof(Real);
    if (!allow_dynamic_smem((const void*)g3_rows<Real, NQ>, smem)) return GW_ERR_INVALID;
    const int per_sm = resident_blocks(g3_rows<Real, NQ>, 128, smem);
    const int blocks = std::max(1, std::min((n + 3) / 4, per_sm * A.num_sms));
    g3_rows<Real, NQ><<<blocks, 128, smem, st>>>(T, n, sy, P(L.R0), P(L.R1), P(L.R2));
  }
  if (A.exact) {
    TraceScope ts(A.tracer, "g2_colsum", st);
    const int rows_per = (n + L.nb - 1) / L.nb;
    const int nb = (n + rows_per - 1) / rows_per;
    g2_colsum<Real><<<dim3((m + 255) / 256, nb), 256, 0, st>>>(T, n, m, rows_per, P(L.part));
    g2_colsum_fin<Acc><<<(m + 255) / 256, 256, 0, st>>>(P(L.part), nb, m, P(L.Cm));
  }
  {
    TraceScope ts(A.tracer, "g3_marg", st);
    const int t1 = 6 * sx * sx * sy + n + m;
    g3_stage1<Acc><<<(t1 + 255) / 256, 256, 0, st>>>(P(L.R0), P(L.R1), P(L.R2), sx, sy, A.u, A.v, P(L.Cm), A.exact,
                                                     P(L.Sx), P(L.Px), P(L.R), P(L.C));
    const int t2 = 9 * sx * sy + 3 * sx * sx + 3 * sy * sy;
    g3_stage2<Acc><<<(t2 + 255) / 256, 256, 0, st>>>(P(L.Sx), P(L.Px), P(L.R), P(L.C), sx, sy, P(L.M), P(L.R2d),
                                                     P(L.C2d));
    const int t3 = 3 * sx + 3 * sy;
    g3_stage3<Acc><<<(t3 + 255) / 256, 256, 0, st>>>(P(L.R2d), P(L.C2d), sx, sy, P(L.r1), P(L.c1));
  }
  {
    TraceScope ts(A.tracer, "g2_tx", st);
    int start = 0;
    auto add = [&](TxJobs& js, size_t in, size_t out, int batch, int rows, int cols, int right, int pw) {
      TxJob& j = js.j[js.n++];
      j.in = ws + in;
      j.out = ws + out;
      j.batch = batch;
      j.rows = rows;
      j.cols = cols;
      j.right = right;
      j.sq = sq;
      j.pw = pw;
      j.start = start;
      start += batch * rows * cols;
    };
    TxJobs left{};
    add(left, L.M, L.YM, 9, sx, sy, 0, 1);
    add(left, L.R2d, L.YR, 3, sx, sx, 0, 1);
    add(left, L.C2d, L.YC, 3, sy, sy, 0, 1);
    add(left, L.r1, L.px, 3, sx, 1, 0, 2);
    add(left, L.c1, L.py, 3, sy, 1, 0, 2);
    left.total = start;
    g2_tx<Acc><<<(left.total + 127) / 128, 128, 0, st>>>(left);
    TxJobs right{};
    start = 0;
    add(right, L.YM, L.Z, 9, sx, sy, 1, 1);
    add(right, L.YR, L.WX, 3, sx, sx, 1, 1);
    add(right, L.YC, L.WY, 3, sy, sy, 1, 1);
    right.total = start;
    g2_tx<Acc><<<(right.total + 127) / 128, 128, 0, st>>>(right);
  }
  {
    TraceScope ts(A.tracer, "g3_tab", st);
    const int tab = m + n * sy;
    g3_tab<Real><<<(tab + 255) / 256, 256, 0, st>>>(P(L.Z), P(L.px), P(L.WX), P(L.py), P(L.WY), sx, sy,
                                                     A.out_scale * s_x * s_x, A.out_scale * s_y * s_y,
                                                     A.out_scale * 2.0 * s_x * s_y, (Real*)(ws + L.Cy),
                                                     (Real*)(ws + L.U));
  }
  {
    TraceScope ts(A.tracer, "g3_epi", st);
    const size_t cs_bytes = (size_t)m * sizeof(float2);
    bool staged = false;
    if constexpr (sizeof(Real) == 4) {
      if (cs_bytes <= kEpi3SmemMax && allow_dynamic_smem((const void*)g3_epi_cs<NQ>, cs_bytes)) {
        const int blocks =
            std::max(1, std::min((n + 15) / 16, resident_blocks(g3_epi_cs<NQ>, 512, cs_bytes) * A.num_sms));
        g3_epi_cs<NQ><<<blocks, 512, cs_bytes, st>>>((float*)A.G, n, sy, (const float*)(ws + L.Cy),
                                                     (const float*)(ws + L.U));
        staged = true;
      }
    }
    if (!staged) {
      const int blocks = std::max(1, std::min((n + 7) / 8, resident_blocks(g3_epi<Real, NQ>, 256) * A.num_sms));
      g3_epi<Real, NQ><<<blocks, 256, 0, st>>>((Real*)A.G, n, sy, (const Real*)(ws + L.Cy),
                                               (const Real*)(ws + L.U));
    }
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

template <typename Real>
int grad3d_dispatch(const Grad2DArgs& A, void* ws, size_t ws_bytes) {
  const int q2 = A.sy * A.sy;
  if (q2 <= 32) return grad3d_typed<Real, 1>(A, ws, ws_bytes);
  if (q2 <= 64) return grad3d_typed<Real, 2>(A, ws, ws_bytes);
  if (q2 <= 128) return grad3d_typed<Real, 4>(A, ws, ws_bytes);
  if (q2 <= 256) return grad3d_typed<Real, 8>(A, ws, ws_bytes);
  if (q2 <= 512) return grad3d_typed<Real, 16>(A, ws, ws_bytes);
  return grad3d_typed<Real, 32>(A, ws, ws_bytes);
}

}  // namespace

size_t grad3d_workspace_bytes(int sx, int sy, int dtype) { return g3_layout(sx, sy, dtype).total + 4096; }

int grad3d_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes) {
  if (a.sx < 1 || a.sy < 1 || a.sx > kMax3DSide || a.sy > kMax3DSide) return GW_ERR_INVALID;
  if (!(a.cost == GW_COST_SQEUCLID || (a.cost == GW_COST_POW && a.k == 1))) return GW_ERR_INVALID;
  if (a.dtype == GW_F32) return grad3d_dispatch<float>(a, ws, ws_bytes);
  return grad3d_dispatch<double>(a, ws, ws_bytes);
}

}  // namespace gw
