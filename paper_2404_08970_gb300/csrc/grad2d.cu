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
//   g2_cy      the column constant c_y as a hi/lo table.
//   g2_epi     writes G row by row from per-row tables in shared memory.
//
// Sums are compensated: Kahan in the row pass, float-float (double for
// double data) everywhere after it; outputs are rounded once.
#include <algorithm>
#include <cmath>

#include "gw_common.cuh"
#include "gw_internal.h"

namespace gw {
namespace {

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

// ---------------------------------------------------------------------------
// g2_rows: per row i of T (length m = sy^2, element (c,d) at c*sy + d)
//   Rc[i][c] = sum_d T[i][c][d],  Rd[i][d] = sum_c T[i][c][d].
// Lane l owns d = l + 32q.  Rd is a per-lane Kahan sum over c.  For Rc each
// lane first adds its NQ values of one c, then 32 consecutive c are reduced
// across the warp at once by a transposing butterfly (lane l ends with c =
// base + l): 31 shuffles per 32 sums.
// ---------------------------------------------------------------------------
template <typename Real, int NQ>
__global__ void __launch_bounds__(256, 2)
    g2_rows(const Real* __restrict__ T, int n, int sy, AccOf<Real>* __restrict__ Rc, AccOf<Real>* __restrict__ Rd) {
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
      for (int cc = 0; cc < 32; ++cc) {
        const int c = cg + cc;
        Real x = 0;
        if (c < sy) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int d = lane + 32 * q;
            const Real t = d < sy ? __ldcs(row + (size_t)c * sy + d) : (Real)0;
            x += t;
            const Real y = t - rc[q];
            const Real s2 = rs[q] + y;
            rc[q] = (s2 - rs[q]) - y;
            rs[q] = s2;
          }
        }
        xs[cc] = x;
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
    for (int o = 0; o < sx; ++o) {
      const int i = (t < 2) ? r * sx + o : o * sx + r;
      s = acc_add(s, src[(size_t)i * sy + col]);
    }
    M[idx] = s;
  } else if (idx < nM + nR) {
    const int e = idx - nM;
    if (exact)
      for (int c = 0; c < sy; ++c) s = acc_add(s, Rc[(size_t)e * sy + c]);
    else
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

// rA = R 1, rB = 1^T R, cA = C 1, cB = 1^T C.
template <typename Acc>
__global__ void g2_vec(const Acc* __restrict__ R, const Acc* __restrict__ C, int sx, int sy, Acc* __restrict__ rA,
                       Acc* __restrict__ rB, Acc* __restrict__ cA, Acc* __restrict__ cB) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  Acc s = acc_zero((Acc*)nullptr);
  if (idx < 2 * sx) {
    const int j = idx % sx;
    const bool rows = idx < sx;
    for (int o = 0; o < sx; ++o) s = acc_add(s, rows ? R[j * sx + o] : R[o * sx + j]);
    (rows ? rA : rB)[j] = s;
  } else if (idx < 2 * sx + 2 * sy) {
    const int e = idx - 2 * sx;
    const int j = e % sy;
    const bool rows = e < sy;
    for (int o = 0; o < sy; ++o) s = acc_add(s, rows ? C[j * sy + o] : C[o * sy + j]);
    (rows ? cA : cB)[j] = s;
  }
}

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
  Acc s0 = acc_zero((Acc*)nullptr), s1 = s0;
  const int len = J.right ? J.cols : J.rows;
  int l = 0;
  for (; l + 1 < len; l += 2) {
    const float w0 = axis_w(J.right ? l - j : i - l, J.sq);
    const float w1 = axis_w(J.right ? l + 1 - j : i - l - 1, J.sq);
    Acc x0 = J.right ? in[i * J.cols + l] : in[l * J.cols + j];
    Acc x1 = J.right ? in[i * J.cols + l + 1] : in[(l + 1) * J.cols + j];
    x0 = acc_w(x0, w0);
    x1 = acc_w(x1, w1);
    if (J.pw == 2) {
      x0 = acc_w(x0, w0);
      x1 = acc_w(x1, w1);
    }
    s0 = acc_add(s0, x0);
    s1 = acc_add(s1, x1);
  }
  if (l < len) {
    const float w0 = axis_w(J.right ? l - j : i - l, J.sq);
    Acc x0 = J.right ? in[i * J.cols + l] : in[l * J.cols + j];
    x0 = acc_w(x0, w0);
    if (J.pw == 2) x0 = acc_w(x0, w0);
    s0 = acc_add(s0, x0);
  }
  ((Acc*)J.out)[e] = acc_add(s0, s1);
}

// Column constant: Cy[(c,d)] = scale_y (py[c] + 2 WY[c][d] + qy[d]), with
// scale_y = out_scale s_Y^2, as hi/lo.
template <typename Real>
__global__ void g2_cy(const AccOf<Real>* __restrict__ py, const AccOf<Real>* __restrict__ qy,
                      const AccOf<Real>* __restrict__ WY, int sy, double scale_y, Real* __restrict__ CyH,
                      Real* __restrict__ CyL) {
  using Acc = AccOf<Real>;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= sy * sy) return;
  const int c = p / sy, d = p % sy;
  Acc sc;
  acc_from(&sc, scale_y);
  const Acc w = WY[p];
  Acc s = acc_add(acc_add(py[c], qy[d]), acc_add(w, w));
  s = acc_mul(s, sc);
  Real hi, lo;
  acc_split(s, hi, lo);
  CyH[p] = hi;
  CyL[p] = lo;
}

// G rows.  For row (a,b):
//   Ux[c] = out_scale (s_X^2 (px[a] + 2 WX[a][b] + qx[b]) - 2 s_X s_Y (Z1[a][c] + Z3[b][c]))
//   Vx[d] = -out_scale 2 s_X s_Y (Z2[a][d] + Z4[b][d])
//   G[(a,b),(c,d)] = Ux[c] + Vx[d] + Cy[(c,d)]   (hi parts, then lo parts).
// The per-row tables are double-buffered in shared memory, so each row costs
// one block barrier.
template <typename Real, int NQ>
__global__ void __launch_bounds__(512, 1)
    g2_epi(Real* __restrict__ G, int sx, int sy, const AccOf<Real>* __restrict__ Z, const AccOf<Real>* __restrict__ px,
           const AccOf<Real>* __restrict__ qx, const AccOf<Real>* __restrict__ WX, const Real* __restrict__ CyH,
           const Real* __restrict__ CyL, double scale_x, double scale_z) {
  using Acc = AccOf<Real>;
  constexpr bool kLo = sizeof(Real) == 4;
  __shared__ Real UH[2][256], UL[2][256], VH[2][256], VL[2][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = sx * sx;
  const size_t m = (size_t)sy * sy;
  const int per_mat = sx * sy;
  Acc scx, scz;
  acc_from(&scx, scale_x);
  acc_from(&scz, scale_z);
  int buf = 0;
  for (int i = blockIdx.x; i < n; i += gridDim.x, buf ^= 1) {
    const int a = i / sx, b = i % sx;
    if (tid < sy) {
      const int c = tid;
      const Acc w = WX[a * sx + b];
      Acc cx = acc_add(acc_add(px[a], qx[b]), acc_add(w, w));
      cx = acc_mul(cx, scx);
      const Acc zz = acc_mul(acc_add(Z[a * sy + c], Z[2 * per_mat + b * sy + c]), scz);
      const Acc U = acc_sub(cx, zz);
      acc_split(U, UH[buf][c], UL[buf][c]);
    } else if (tid >= 256 && tid - 256 < sy) {
      const int d = tid - 256;
      const Acc zz = acc_mul(acc_add(Z[per_mat + a * sy + d], Z[3 * per_mat + b * sy + d]), scz);
      const Acc V = acc_neg_of(zz);
      acc_split(V, VH[buf][d], VL[buf][d]);
    }
    __syncthreads();
    Real* grow = G + (size_t)i * m;
    for (int c = warp; c < sy; c += 16) {
      const Real uh = UH[buf][c], ul = UL[buf][c];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int d = lane + 32 * q;
        if (d < sy) {
          const int p = c * sy + d;
          Real g = (uh + VH[buf][d]) + __ldg(CyH + p);
          if (kLo) g += (ul + VL[buf][d]) + __ldg(CyL + p);
          __stcs(grow + p, g);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct G2Layout {
  size_t Rc, Rd, M, R, C, rA, rB, cA, cB, Y, YR, YC, px, qx, py, qy, Z, WX, WY, CyH, CyL, part, Cm, total;
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
  L.CyH = take(m * rb);
  L.CyL = take(m * rb);
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
    const int blocks = std::max(1, std::min((n + 7) / 8, 2 * A.num_sms));
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
    TraceScope ts(A.tracer, "g2_small", st);
    const int tot = 4 * sx * sy + n + m;
    g2_marg<Acc><<<(tot + 255) / 256, 256, 0, st>>>(P(L.Rc), P(L.Rd), sx, sy, A.u, A.v, P(L.Cm), A.exact, P(L.M),
                                                    P(L.R), P(L.C));
    g2_vec<Acc><<<(2 * sx + 2 * sy + 255) / 256, 256, 0, st>>>(P(L.R), P(L.C), sx, sy, P(L.rA), P(L.rB), P(L.cA),
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
    g2_cy<Real><<<(m + 255) / 256, 256, 0, st>>>(P(L.py), P(L.qy), P(L.WY), sy, A.out_scale * s_y * s_y,
                                                  (Real*)(ws + L.CyH), (Real*)(ws + L.CyL));
  }
  {
    TraceScope ts(A.tracer, "g2_epi", st);
    const int blocks = std::max(1, std::min(n, A.num_sms));
    g2_epi<Real, NQ><<<blocks, 512, 0, st>>>((Real*)A.G, sx, sy, P(L.Z), P(L.px), P(L.qx), P(L.WX),
                                             (const Real*)(ws + L.CyH), (const Real*)(ws + L.CyL),
                                             A.out_scale * s_x * s_x, A.out_scale * 2.0 * s_x * s_y);
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

size_t grad2d_workspace_bytes(int sx, int sy, int dtype) { return g2_layout(sx, sy, dtype).total + 4096; }

int grad2d_launch(const Grad2DArgs& a, void* ws, size_t ws_bytes) {
  if (a.sx < 1 || a.sy < 1 || a.sx > kMax2DSide || a.sy > kMax2DSide) return GW_ERR_INVALID;
  if (a.cost != GW_COST_POW && a.cost != GW_COST_SQEUCLID) return GW_ERR_INVALID;
  if (a.dtype == GW_F32) return grad2d_dispatch<float>(a, ws, ws_bytes);
  return grad2d_dispatch<double>(a, ws, ws_bytes);
}

}  // namespace gw
