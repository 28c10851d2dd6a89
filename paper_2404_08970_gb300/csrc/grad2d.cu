// Structured gradient on 2D grids with an axis-separable cost (Sec. 3.1).
//
// Points of a side x side grid are flattened row-major, i = a * side + b.  For
// the Manhattan distance (k = 1) and the squared Euclidean distance the cost
// splits over the two axes:
//   D_X[(a,b),(a',b')] = s_X (A_aa' + A_bb'),  A_aa' = |a - a'| or (a - a')^2,
// with s_X = h_X or h_X^2 (the k = 1 case of the Kronecker expansion,
// eq. "2D kronecker", where the two J-blocks carry the other axis).  With T
// read as a four-index array T[a][b][c][d] (row (a,b) of X, column (c,d) of Y):
//   (D_X T D_Y)_{(a,b),(c,d)} = s_X s_Y (Z1[a][c] + Z2[a][d] + Z3[b][c] + Z4[b][d]),
//   Z_t = A_X M_t A_Y,
// where M1, M2, M3, M4 sum T over (b,d), (b,c), (a,d), (a,c).  The constant
// term splits the same way: with R[a][b] = r_(a,b),
//   ((D_X o D_X) r)_{(a,b)} = s_X^2 ( (A o A) R 1 + 2 A R A + 1^T R (A o A) )_{ab}.
// Everything after the single pass over T works on side x side matrices.
//
// Kernels (in launch order):
//   g2_rows    one warp per row of T: the row's sums over d for every c and
//              over c for every d (the only pass over the n x m input).
//   g2_colsum  exact marginals only: column sums of T (second pass).
//   g2_marg    M1..M4, R and C (the marginals as side x side matrices).
//   g2_vec     row and column sums of R and C.
//   g2_tx      small transforms by A from the left, then from the right.
//   g2_tab     the epilogue tables: c_y per column, and per row of X the parts
//              of G that depend on (row, c) and on (row, d).
//   g2_epi     writes G, one warp per row.
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

// ---------------------------------------------------------------------------
// g2_rows: per row i of T (length m = sy^2, element (c,d) at c*sy + d)
//   Rc[i][c] = sum_d T[i][c][d],  Rd[i][d] = sum_c T[i][c][d].
// Lane l owns d = l + 32q.  Rd is a per-lane Kahan sum over c.  For Rc each
// lane first adds its NQ values of one c, then 32 consecutive c are reduced
// across the warp at once by a transposing butterfly (lane l ends with c =
// base + l): 31 shuffles per 32 sums.
// ---------------------------------------------------------------------------
template <typename Real, int NQ>
__global__ void __launch_bounds__(256, 1)
    g2_rows(const Real* __restrict__ T, int n, int sy, AccOf<Real>* __restrict__ Rc, AccOf<Real>* __restrict__ Rd) {
  constexpr int SG = NQ <= 2 ? 16 : 8;  // c's whose loads are issued together
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const size_t m = (size_t)sy * sy;
  for (int i = w0; i < n; i += nw) {
    const Real* row = T + (size_t)i * m;
    Real rs[NQ], rc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) rs[q] = rc[q] = 0;
    for (int cg = 0; cg < sy; cg += 32) {
      Real xs[32];
#pragma unroll
      for (int sg = 0; sg < 32; sg += SG) {
        Real t[SG][NQ];
#pragma unroll
        for (int cc = 0; cc < SG; ++cc) {
          const int c = cg + sg + cc;
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int d = lane + 32 * q;
            t[cc][q] = (c < sy && d < sy) ? __ldcs(row + (size_t)c * sy + d) : (Real)0;
          }
        }
#pragma unroll
        for (int cc = 0; cc < SG; ++cc) {
          Real x = 0;
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            x += t[cc][q];
            const Real y = t[cc][q] - rc[q];
            const Real s2 = rs[q] + y;
            rc[q] = (s2 - rs[q]) - y;
            rs[q] = s2;
          }
          xs[sg + cc] = x;
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
          const Real send = up ? xs[j] : xs[j + o];
          const Real keep = up ? xs[j + o] : xs[j];
          xs[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      const int c = cg + lane;
      if (c < sy) Rc[(size_t)i * sy + c] = acc_of(xs[0]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int d = lane + 32 * q;
      if (d < sy) Rd[(size_t)i * sy + d] = acc_of(rs[q], -rc[q]);
    }
  }
}

// M1[a][c] = sum_b Rc[(a,b)][c], M2[a][d] = sum_b Rd[(a,b)][d],
// M3[b][c] = sum_a Rc[(a,b)][c], M4[b][d] = sum_a Rd[(a,b)][d] (layout
// [4][sx][sy]); R[a][b] = r_(a,b) and C[c][d] = c_(c,d), from the targets or,
// with exact marginals, from T (row sums via Rc, column sums from g2_colsum).
template <typename Acc>
__global__ void g2_marg(const Acc* __restrict__ Rc, const Acc* __restrict__ Rd, int sx, int sy,
                        const double* __restrict__ u, const double* __restrict__ v, const Acc* __restrict__ Cm,
                        int exact, Acc* __restrict__ M, Acc* __restrict__ R, Acc* __restrict__ C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nM = 4 * sx * sy, nR = sx * sx, nC = sy * sy;
  Acc s = acc_zero((Acc*)nullptr);
  if (idx < nM) {
    const int t = idx / (sx * sy), e = idx % (sx * sy), r = e / sy, col = e % sy;
    const Acc* src = (t == 0 || t == 2) ? Rc : Rd;
    const size_t base = (t < 2) ? (size_t)r * sx * sy + col : (size_t)r * sy + col;
    const size_t step = (t < 2) ? (size_t)sy : (size_t)sx * sy;
    int o = 0;
    for (; o + 8 <= sx; o += 8) {
      Acc x[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) x[e] = src[base + (size_t)(o + e) * step];
#pragma unroll
      for (int e = 0; e < 8; ++e) s = acc_add(s, x[e]);
    }
    for (; o < sx; ++o) s = acc_add(s, src[base + (size_t)o * step]);
    M[idx] = s;
  } else if (idx < nM + nR) {
    const int e = idx - nM;
    if (exact) {
      int c = 0;
      for (; c + 8 <= sy; c += 8) {
        Acc x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = Rc[(size_t)e * sy + c + q];
#pragma unroll
        for (int q = 0; q < 8; ++q) s = acc_add(s, x[q]);
      }
      for (; c < sy; ++c) s = acc_add(s, Rc[(size_t)e * sy + c]);
    } else
      s = acc_add_d(s, u[e]);
    R[e] = s;
  } else if (idx < nM + nR + nC) {
    const int e = idx - nM - nR;
    if (exact)
      s = Cm[e];
    else
      s = acc_add_d(s, v[e]);
    C[e] = s;
  }
}

// rA = R 1, rB = 1^T R, cA = C 1, cB = 1^T C: one warp per output, lanes
// over the summed index, then a fixed-order butterfly.
template <typename Acc>
__global__ void g2_vec(const Acc* __restrict__ R, const Acc* __restrict__ C, int sx, int sy, Acc* __restrict__ rA,
                       Acc* __restrict__ rB, Acc* __restrict__ cA, Acc* __restrict__ cB) {
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (wid >= 2 * sx + 2 * sy) return;
  const Acc* src;
  Acc* dst;
  int s, j, rows;
  if (wid < 2 * sx) {
    src = R;
    s = sx;
    j = wid % sx;
    rows = wid < sx;
    dst = rows ? rA : rB;
  } else {
    src = C;
    s = sy;
    j = (wid - 2 * sx) % sy;
    rows = (wid - 2 * sx) < sy;
    dst = rows ? cA : cB;
  }
  Acc t = acc_zero((Acc*)nullptr);
  for (int o = lane; o < s; o += 32) t = acc_add(t, rows ? src[j * s + o] : src[o * s + j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t = acc_add(t, acc_shfl_xor(t, o));
  if (lane == 0) dst[j] = t;
}

// Epilogue tables, all hi/lo (rounded once from the compensated values):
//   Cy[(c,d)] = scale_y (py[c] + 2 WY[c][d] + qy[d]),   scale_y = out_scale s_Y^2
//   Ux[i][c]  = scale_x (px[a] + 2 WX[a][b] + qx[b]) - scale_z (Z1[a][c] + Z3[b][c])
//   Vx[i][d]  = -scale_z (Z2[a][d] + Z4[b][d])
// for i = (a,b), with scale_x = out_scale s_X^2 and scale_z = 2 out_scale s_X s_Y,
// so that G[(a,b),(c,d)] = Ux[i][c] + Vx[i][d] + Cy[(c,d)].  Layout: Cy as
// [m] hi then [m] lo; UV as [n][sy] (Ux hi, Ux lo, Vx hi, Vx lo) per entry.
template <typename Real>
__global__ void g2_tab(const AccOf<Real>* __restrict__ Z, const AccOf<Real>* __restrict__ px,
                       const AccOf<Real>* __restrict__ qx, const AccOf<Real>* __restrict__ WX,
                       const AccOf<Real>* __restrict__ py, const AccOf<Real>* __restrict__ qy,
                       const AccOf<Real>* __restrict__ WY, int sx, int sy, double scale_x, double scale_y,
                       double scale_z, Real* __restrict__ Cy, Real* __restrict__ UV) {
  using Acc = AccOf<Real>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = sy * sy, n = sx * sx, per_mat = sx * sy;
  if (idx < m) {
    const int c = idx / sy, d = idx % sy;
    Acc sc;
    acc_from(&sc, scale_y);
    const Acc w = WY[idx];
    const Acc v = acc_mul(acc_add(acc_add(py[c], qy[d]), acc_add(w, w)), sc);
    Real hi, lo;
    acc_split(v, hi, lo);
    Cy[idx] = hi;
    Cy[m + idx] = lo;
  } else if (idx < m + n * sy) {
    const int e = idx - m;
    const int i = e / sy, c = e % sy;  // c doubles as d for the V part
    const int a = i / sx, b = i % sx;
    Acc scx, scz;
    acc_from(&scx, scale_x);
    acc_from(&scz, scale_z);
    const Acc w = WX[a * sx + b];
    const Acc cx = acc_mul(acc_add(acc_add(px[a], qx[b]), acc_add(w, w)), scx);
    const Acc U = acc_sub(cx, acc_mul(acc_add(Z[a * sy + c], Z[2 * per_mat + b * sy + c]), scz));
    const Acc V = acc_neg_of(acc_mul(acc_add(Z[per_mat + a * sy + c], Z[3 * per_mat + b * sy + c]), scz));
    Real* o = UV + (size_t)e * 4;
    acc_split(U, o[0], o[1]);
    acc_split(V, o[2], o[3]);
  }
}

// G rows: one warp per row, lane l on d = l + 32q; no block barriers.  The
// row's table entries (Ux, Vx) for index l + 32q sit in lane l's registers
// (loaded one row ahead); Ux[c] reaches every lane by a shuffle.
//   G[(a,b),(c,d)] = (Ux[c] + Vx[d] + Cy[(c,d)])_hi + (...)_lo
template <typename Real>
struct Quad {
  Real uh, ul, vh, vl;
};
__device__ __forceinline__ Quad<float> load_quad(const float* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return {t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ Quad<double> load_quad(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {a.x, a.y, b.x, b.y};
}

template <typename Real, int NQ>
__global__ void __launch_bounds__(256)
    g2_epi(Real* __restrict__ G, int n, int sy, const Real* __restrict__ Cy, const Real* __restrict__ UV) {
  constexpr bool kLo = sizeof(Real) == 4;
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int m = sy * sy;
  Quad<Real> nxt[NQ];
  auto fetch = [&](int i) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int d = lane + 32 * q;
      nxt[q] = (i < n && d < sy) ? load_quad(UV + ((size_t)i * sy + d) * 4) : Quad<Real>{0, 0, 0, 0};
    }
  };
  fetch(w0);
  for (int i = w0; i < n; i += nw) {
    Quad<Real> cur[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) cur[q] = nxt[q];
    fetch(i + nw);
    Real* grow = G + (size_t)i * m;
#pragma unroll
    for (int qc = 0; qc < NQ; ++qc) {
      const int cmax = min(32, sy - 32 * qc);
#pragma unroll 4
      for (int l = 0; l < cmax; ++l) {
        const int c = 32 * qc + l;
        const Real uh = __shfl_sync(0xffffffffu, cur[qc].uh, l);
        const Real ul = __shfl_sync(0xffffffffu, cur[qc].ul, l);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int d = lane + 32 * q;
          if (d < sy) {
            const int p = c * sy + d;
            Real g = (uh + cur[q].vh) + __ldg(Cy + p);
            if (kLo) g += (ul + cur[q].vl) + __ldg(Cy + m + p);
            __stcs(grow + p, g);
          }
        }
      }
    }
  }
}

// Float rows with the c_y table staged in shared memory (hi and lo side by
// side, one 8-byte shared load per element): loading the table from L2 for
// every element bounded g2_epi (long-scoreboard stalls).  The table is read
// with plain shared-memory loads only; everything else as g2_epi.
template <int NQ>
__global__ void __launch_bounds__(512, 2)
    g2_epi_cs(float* __restrict__ G, int n, int sy, const float* __restrict__ Cy, const float* __restrict__ UV) {
  extern __shared__ __align__(16) float2 g2_cys[];
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int m = sy * sy;
  for (int p = threadIdx.x; p < m; p += blockDim.x) g2_cys[p] = make_float2(Cy[p], Cy[m + p]);
  __syncthreads();
  Quad<float> nxt[NQ];
  auto fetch = [&](int i) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int d = lane + 32 * q;
      nxt[q] = (i < n && d < sy) ? load_quad(UV + ((size_t)i * sy + d) * 4) : Quad<float>{0, 0, 0, 0};
    }
  };
  fetch(w0);
  for (int i = w0; i < n; i += nw) {
    Quad<float> cur[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) cur[q] = nxt[q];
    fetch(i + nw);
    float* grow = G + (size_t)i * m;
#pragma unroll
    for (int qc = 0; qc < NQ; ++qc) {
      const int cmax = min(32, sy - 32 * qc);
#pragma unroll 4
      for (int l = 0; l < cmax; ++l) {
        const int c = 32 * qc + l;
        const float uh = __shfl_sync(0xffffffffu, cur[qc].uh, l);
        const float ul = __shfl_sync(0xffffffffu, cur[qc].ul, l);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int d = lane + 32 * q;
          if (d < sy) {
            const int p = c * sy + d;
            const float2 cv = g2_cys[p];
            float g = (uh + cur[q].vh) + cv.x;
            g += (ul + cur[q].vl) + cv.y;
            __stcs(grow + p, g);
          }
        }
      }
    }
  }
}

// Largest c_y table staged in shared memory: two blocks of g2_epi_cs per SM.
constexpr size_t kEpiSmemMax = 100 * 1024;

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct G2Layout {
  size_t Rc, Rd, M, R, C, rA, rB, cA, cB, Y, YR, YC, px, qx, py, qy, Z, WX, WY, Cy, UV, part, Cm, total;
  int nb;
};

G2Layout g2_layout(int sx, int sy, int dtype) {
  const size_t acc = 8;  // ff or double
  const size_t rb = dtype == GW_F32 ? 4 : 8;
  const size_t n = (size_t)sx * sx, m = (size_t)sy * sy;
  G2Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) / 256 * 256;
    return o;
  };
  L.nb = (int)std::min<size_t>(n, 64);
  L.Rc = take(n * sy * acc);
  L.Rd = take(n * sy * acc);
  L.M = take(4 * (size_t)sx * sy * acc);
  L.R = take(n * acc);
  L.C = take(m * acc);
  L.rA = take(sx * acc);
  L.rB = take(sx * acc);
  L.cA = take(sy * acc);
  L.cB = take(sy * acc);
  L.Y = take(4 * (size_t)sx * sy * acc);
  L.YR = take(n * acc);
  L.YC = take(m * acc);
  L.px = take(sx * acc);
  L.qx = take(sx * acc);
  L.py = take(sy * acc);
  L.qy = take(sy * acc);
  L.Z = take(4 * (size_t)sx * sy * acc);
  L.WX = take(n * acc);
  L.WY = take(m * acc);
  L.Cy = take(2 * m * rb);
  L.UV = take(n * sy * 4 * rb);
  L.part = take((size_t)L.nb * m * acc);
  L.Cm = take(m * acc);
  L.total = off;
  return L;
}

template <typename Real, int NQ>
int grad2d_typed(const Grad2DArgs& A, void* wsv, size_t ws_bytes) {
  using Acc = AccOf<Real>;
  const int sx = A.sx, sy = A.sy;
  const int n = sx * sx, m = sy * sy;
  const G2Layout L = g2_layout(sx, sy, A.dtype);
  if (L.total > ws_bytes) return GW_ERR_OOM;
  char* ws = (char*)wsv;
  auto P = [&](size_t o) { return (Acc*)(ws + o); };
  cudaStream_t st = A.stream;
  const Real* T = (const Real*)A.T;
  const int sq = A.cost == GW_COST_SQEUCLID ? 1 : 0;
  const double s_x = sq ? A.hx * A.hx : A.hx;
  const double s_y = sq ? A.hy * A.hy : A.hy;
  {
    TraceScope ts(A.tracer, "g2_rows", st);
    const int blocks = std::max(1, std::min((n + 7) / 8, resident_blocks(g2_rows<Real, NQ>, 256) * A.num_sms));
    g2_rows<Real, NQ><<<blocks, 256, 0, st>>>(T, n, sy, P(L.Rc), P(L.Rd));
  }
  if (A.exact) {
    TraceScope ts(A.tracer, "g2_colsum", st);
    const int rows_per = (n + L.nb - 1) / L.nb;
    const int nb = (n + rows_per - 1) / rows_per;
    g2_colsum<Real><<<dim3((m + 255) / 256, nb), 256, 0, st>>>(T, n, m, rows_per, P(L.part));
    g2_colsum_fin<Acc><<<(m + 255) / 256, 256, 0, st>>>(P(L.part), nb, m, P(L.Cm));
  }
  {
    TraceScope ts(A.tracer, "g2_marg", st);
    const int tot = 4 * sx * sy + n + m;
    g2_marg<Acc><<<(tot + 255) / 256, 256, 0, st>>>(P(L.Rc), P(L.Rd), sx, sy, A.u, A.v, P(L.Cm), A.exact, P(L.M),
                                                    P(L.R), P(L.C));
  }
  {
    TraceScope ts(A.tracer, "g2_tx", st);
    g2_vec<Acc><<<(2 * sx + 2 * sy + 7) / 8, 256, 0, st>>>(P(L.R), P(L.C), sx, sy, P(L.rA), P(L.rB), P(L.cA),
                                                           P(L.cB));
    TxJobs left{};
    int start = 0;
    auto add = [&](TxJobs& js, size_t in, size_t out, int batch, int rows, int cols, int right, int pw) {
      TxJob& j = js.j[js.n++];
      j.in = ws + in;
      j.out = ws + out;
      j.batch = batch;
      j.rows = rows;
      j.cols = cols;
      j.right = right;
      // The left factor acts on X's axes, the right factor on Y's.
      j.sq = sq;
      j.pw = pw;
      j.start = start;
      start += batch * rows * cols;
    };
    add(left, L.M, L.Y, 4, sx, sy, 0, 1);
    add(left, L.R, L.YR, 1, sx, sx, 0, 1);
    add(left, L.C, L.YC, 1, sy, sy, 0, 1);
    add(left, L.rA, L.px, 1, sx, 1, 0, 2);
    add(left, L.rB, L.qx, 1, sx, 1, 0, 2);
    add(left, L.cA, L.py, 1, sy, 1, 0, 2);
    add(left, L.cB, L.qy, 1, sy, 1, 0, 2);
    left.total = start;
    g2_tx<Acc><<<(left.total + 127) / 128, 128, 0, st>>>(left);
    TxJobs right{};
    start = 0;
    add(right, L.Y, L.Z, 4, sx, sy, 1, 1);
    add(right, L.YR, L.WX, 1, sx, sx, 1, 1);
    add(right, L.YC, L.WY, 1, sy, sy, 1, 1);
    right.total = start;
    g2_tx<Acc><<<(right.total + 127) / 128, 128, 0, st>>>(right);
  }
  {
    TraceScope ts(A.tracer, "g2_tab", st);
    const int tab = m + n * sy;
    g2_tab<Real><<<(tab + 255) / 256, 256, 0, st>>>(P(L.Z), P(L.px), P(L.qx), P(L.WX), P(L.py), P(L.qy), P(L.WY),
                                                     sx, sy, A.out_scale * s_x * s_x, A.out_scale * s_y * s_y,
                                                     A.out_scale * 2.0 * s_x * s_y, (Real*)(ws + L.Cy),
                                                     (Real*)(ws + L.UV));
  }
  {
    TraceScope ts(A.tracer, "g2_epi", st);
    const size_t cs_bytes = (size_t)m * sizeof(float2);
    bool staged = false;
    if constexpr (sizeof(Real) == 4) {
      if (cs_bytes <= kEpiSmemMax && allow_dynamic_smem((const void*)g2_epi_cs<NQ>, cs_bytes)) {
        const int blocks =
            std::max(1, std::min((n + 15) / 16, resident_blocks(g2_epi_cs<NQ>, 512, cs_bytes) * A.num_sms));
        g2_epi_cs<NQ><<<blocks, 512, cs_bytes, st>>>((float*)A.G, n, sy, (const float*)(ws + L.Cy),
                                                     (const float*)(ws + L.UV));
        staged = true;
      }
    }
    if (!staged) {
      const int blocks = std::max(1, std::min((n + 7) / 8, resident_blocks(g2_epi<Real, NQ>, 256) * A.num_sms));
      g2_epi<Real, NQ><<<blocks, 256, 0, st>>>((Real*)A.G, n, sy, (const Real*)(ws + L.Cy),
                                               (const Real*)(ws + L.UV));
    }
  }
  return cudaPeekAtLastError() == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}

template <typename Real>
int grad2d_dispatch(const Grad2DArgs& A, void* ws, size_t ws_bytes) {
  switch ((A.sy + 31) / 32) {
    case 1: return grad2d_typed<Real, 1>(A, ws, ws_bytes);
    case 2: return grad2d_typed<Real, 2>(A, ws, ws_bytes);
    case 3: return grad2d_typed<Real, 3>(A, ws, ws_bytes);
    case 4: return grad2d_typed<Real, 4>(A, ws, ws_bytes);
    case 5:
    case 6: return grad2d_typed<Real, 6>(A, ws, ws_bytes);
    default: return grad2d_typed<Real, 8>(A, ws, ws_bytes);
  }
}

}  // namespace

size_t grad2d_workspace_bytes(int sx, int sy, int dtype, int cost, int k) {
  if (cost == GW_COST_POW && k >= 2) return grad2d_powk_workspace_bytes(sx, sy, k, dtype);
  return g2_layout(sx, sy, dtype).total + 4096;
}

int grad2d_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes) {
  if (a.dim == 3) return grad3d_launch(a, ws, ws_bytes);
  if (a.cost == GW_COST_POW && a.k >= 2) return grad2d_powk_launch(a, ws, ws_bytes);
  if (a.sx < 1 || a.sy < 1 || a.sx > kMax2DSide || a.sy > kMax2DSide) return GW_ERR_INVALID;
  if (a.cost != GW_COST_POW && a.cost != GW_COST_SQEUCLID) return GW_ERR_INVALID;
  if (a.dtype == GW_F32) return grad2d_dispatch<float>(a, ws, ws_bytes);
  return grad2d_dispatch<double>(a, ws, ws_bytes);
}

}  // namespace gw
