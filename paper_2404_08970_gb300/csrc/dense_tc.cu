// Dense comparison gradient on the fifth-generation tensor cores, written by
// hand: C = A * B^T with A (M x K) and B (N x K) both row-major ("K-major"),
// BF16 or TF32 inputs, FP32 accumulation in tensor memory.
//
// The "original" gradient of Sec. 2.1 needs D_X T D_Y.  With D_X and D_Y
// symmetric it runs as two such products:
//   C1 = D_Y T^T            (m x n; A = D_Y, B = T, K = m), stored in the input type,
//   Z  = D_X C1^T = D_X T D_Y  (n x m; A = D_X, B = C1, K = n),
// and the second product's epilogue writes G = c_x 1^T + 1 c_y^T - 2 Z
// directly, so Z never reaches memory.
//
// Kernel layout (one persistent CTA per SM, 192 threads):
//   warp 0     TMA producer: 128 x 64 B-byte tiles of A and 256-row tiles of
//              B into a 4-stage shared-memory ring (128-byte swizzle).
//   warp 1     allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//              and one lane issues tcgen05.mma (M = 128, N = 256) per K step.
//   warps 2-5  epilogue: TMEM -> registers (each warp its 32-lane quarter),
//              then the output rows; one accumulator is drained while the
//              MMAs fill the other.
// Every mbarrier wait is bounded; on a timeout the status word is set and
// all roles leave their loops, wait (bounded) for their own copies and MMAs
// in flight, and the TMEM is freed before the kernel returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "gw_internal.h"
#include "gw_tc.cuh"

namespace gw {

namespace {

constexpr int kBM = 128;           // accumulator rows (TMEM lanes)
constexpr int kBN = 256;           // accumulator columns per tile
constexpr int kStages = 4;
constexpr int kThreads = 192;      // producer, MMA, 4 epilogue warps
constexpr uint32_t kTmemCols = 512;

template <bool TF32>
struct TcCfg {
  static constexpr int kElem = TF32 ? 4 : 2;
  static constexpr int kBK = 128 / kElem;       // one 128-byte swizzle row of K
  static constexpr int kUK = TF32 ? 8 : 16;     // K of one MMA instruction (32 bytes)
  static constexpr int kABytes = kBM * 128;     // 16 KB
  static constexpr int kBBytes = kBN * 128;     // 32 KB
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr uint32_t kIdesc = tc::idesc<kBM, kBN>(TF32 ? tc::kFmtTF32 : tc::kFmtBF16);
};

constexpr size_t tc_smem_bytes() {
  // 1024 B alignment slack, the stages, then the barriers and the TMEM word.
  return 1024 + (size_t)kStages * (128 * (kBM + kBN)) + 256;
}

struct TcEpilogue {
  int mode;            // 0: store bf16, 1: store f32 rounded to TF32, 2: G = fma(-scale, z, cx[row] + cy[col]) as f32
  void* out;
  long long ldo;       // elements between output rows
  int rows, cols;      // valid output extent
  const float* cx;     // mode 2: per-row constant term (hi part)
  const float* cy;     // mode 2: per-column constant term (hi part)
  float scale;
};

__device__ __forceinline__ void epi_store(const TcEpilogue& e, int row, int col0, const uint32_t (&r)[32]) {
  if (row >= e.rows) return;
  if (e.mode == 0) {
    __nv_bfloat16* o = (__nv_bfloat16*)e.out + (size_t)row * e.ldo + col0;
    if (col0 + 32 <= e.cols && (e.ldo & 7) == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint4 w;
        uint32_t* wp = &w.x;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          __nv_bfloat162 b = __floats2bfloat162_rn(__uint_as_float(r[q * 8 + 2 * h]), __uint_as_float(r[q * 8 + 2 * h + 1]));
          wp[h] = *reinterpret_cast<uint32_t*>(&b);
        }
        *reinterpret_cast<uint4*>(o + q * 8) = w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (col0 + j < e.cols) o[j] = __float2bfloat16_rn(__uint_as_float(r[j]));
    }
    return;
  }
  float* o = (float*)e.out + (size_t)row * e.ldo + col0;
  float v[32];
  if (e.mode == 2) {
    const float ci = e.cx[row];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = col0 + j;
      const float cyv = c < e.cols ? e.cy[c] : 0.f;
      v[j] = fmaf(-e.scale, __uint_as_float(r[j]), ci + cyv);
    }
  } else {
    // mode 1 feeds the next TF32 product: round to the nearest TF32 value.
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      uint32_t t;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(__uint_as_float(r[j])));
      v[j] = __uint_as_float(t);
    }
  }
  if (col0 + 32 <= e.cols && (e.ldo & 3) == 0 && ((reinterpret_cast<uintptr_t>(e.out) & 15) == 0)) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(o + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (col0 + j < e.cols) o[j] = v[j];
  }
}

// Tile t of the persistent schedule: groups of kGroupRows row tiles, each
// group walked column tile by column tile, so that the ~152 tiles in flight at
// once touch few A and B stripes (they stay in L2).
constexpr int kGroupRows = 8;
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  const int group = t / (kGroupRows * tiles_n);
  const int first = group * kGroupRows;
  const int gsize = min(kGroupRows, tiles_m - first);
  const int r = t - group * kGroupRows * tiles_n;
  tm = first + r % gsize;
  tn = r / gsize;
}

template <bool TF32>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_abt(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                int K, TcEpilogue epi, unsigned* status) {
  using C = TcCfg<TF32>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                                   // kStages x 16 KB
  unsigned char* sB = smem + (size_t)kStages * C::kABytes;    // kStages x 32 KB
  uint64_t* bars = (uint64_t*)(smem + (size_t)kStages * C::kStageBytes);
  uint64_t* full = bars;                     // [kStages] TMA landed
  uint64_t* empty = bars + kStages;          // [kStages] MMAs done reading
  uint64_t* acc_full = bars + 2 * kStages;   // [2] accumulator ready
  uint64_t* acc_empty = bars + 2 * kStages + 2;  // [2] accumulator drained
  uint64_t* drain = bars + 2 * kStages + 4;  // MMA teardown
  uint32_t* tmem_word = (uint32_t*)(bars + 2 * kStages + 5);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (M + kBM - 1) / kBM, tiles_n = (N + kBN - 1) / kBN;
  const int tiles = tiles_m * tiles_n;
  const int kb_count = (K + C::kBK - 1) / C::kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4 * 32);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_word, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_word;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        int tm, tn;
        tile_coords(t, tiles_m, tiles_n, tm, tn);
        for (int kb = 0; kb < kb_count; ++kb) {
          if (!mbar_wait_bounded(&empty[s], ph ^ 1u, status)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], C::kStageBytes);
          tc::tma_load_2d(sA + (size_t)s * C::kABytes, &mapA, kb * C::kBK, tm * kBM, &full[s]);
          tc::tma_load_2d(sB + (size_t)s * C::kBBytes, &mapB, kb * C::kBK, tn * kBN, &full[s]);
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // Own copies in flight: the last load issued into each stage has landed
      // (returns at once on the normal path, where the MMAs consumed them).
      for (int q = 0; q < kStages; ++q) {
        // Stage q's most recent use was in phase ph (q < s) or ph ^ 1 (q >= s).
        const uint32_t last = q < s ? ph : (ph ^ 1u);
        mbar_wait_bounded(&full[q], last, status);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++it) {
        const int a = it & 1;
        const uint32_t aph = (uint32_t)((it >> 1) & 1);
        if (!mbar_wait_bounded(&acc_empty[a], aph ^ 1u, status)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(a * kBN);
        for (int kb = 0; kb < kb_count; ++kb) {
          if (!mbar_wait_bounded(&full[s], ph, status)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint64_t adesc = tc::sw128_kmajor_desc(sA + (size_t)s * C::kABytes);
          const uint64_t bdesc = tc::sw128_kmajor_desc(sB + (size_t)s * C::kBBytes);
#pragma unroll
          for (int k = 0; k < C::kBK / C::kUK; ++k) {
            // +32 bytes of K per instruction inside the swizzled row (>> 4).
            tc::mma<TF32>(d, adesc + (uint64_t)(k * 2), bdesc + (uint64_t)(k * 2), C::kIdesc,
                          (kb > 0 || k > 0) ? 1u : 0u);
          }
          tc::commit(&empty[s]);  // frees the stage once these MMAs are done
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (ok) tc::commit(&acc_full[a]);
      }
      // Every MMA issued by this thread has completed before teardown.
      tc::commit(drain);
      mbar_wait_bounded(drain, 0, status);
    }
    __syncwarp();
  } else {
    // ---------------- Epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;  // TMEM lane quarter this warp may read
    int it = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
      const int a = it & 1;
      const uint32_t aph = (uint32_t)((it >> 1) & 1);
      // The whole warp leaves together: tcgen05.ld below is warp-collective.
      const bool ok = mbar_wait_bounded(&acc_full[a], aph, status);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc::fence_after_sync();
      int tm, tn;
        tile_coords(t, tiles_m, tiles_n, tm, tn);
      const int row = tm * kBM + quarter * 32 + lane;
      const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * kBN);
#pragma unroll 1
      for (int c = 0; c < kBN / 32; ++c) {
        uint32_t r[32];
        tc::ld_32x32b_x32(base + (uint32_t)(c * 32), r);
        tc::wait_ld();
        const int col0 = tn * kBN + c * 32;
        if (col0 < epi.cols) epi_store(epi, row, col0, r);
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&acc_empty[a]);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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
  return fn;
}

// Row-major rows x cols matrix (row pitch `ld` elements, a multiple of 16
// bytes) tiled as boxes of box_rows rows x 128 bytes with the 128-byte
// swizzle; reads past the edges fill zeros.
bool encode_kmajor(CUtensorMap* map, const void* base, int rows, int cols, long long ld, int elem, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base & 15) != 0 || (ld * elem) % 16 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * elem)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int tc_gemm_abt_launch(bool tf32, const void* A, long long lda, const void* B, long long ldb, int M, int N, int K,
                       int mode, void* out, long long ldo, int out_rows, int out_cols, const float* cx,
                       const float* cy, float scale, unsigned* status, int num_sms, cudaStream_t st,
                       Tracer* tracer) {
  if (M < 1 || N < 1 || K < 1) return GW_ERR_INVALID;
  const int elem = tf32 ? 4 : 2;
  CUtensorMap mA, mB;
  if (!encode_kmajor(&mA, A, M, K, lda, elem, kBM) || !encode_kmajor(&mB, B, N, K, ldb, elem, kBN)) {
    note_failure("tc_gemm: tensor map encoding failed (alignment or driver entry point)");
    return GW_ERR_CUDA;
  }
  TcEpilogue e{mode, out, ldo, out_rows, out_cols, cx, cy, scale};
  const size_t smem = tc_smem_bytes();
  const void* fn = tf32 ? (const void*)tc_gemm_abt<true> : (const void*)tc_gemm_abt<false>;
  if (!allow_dynamic_smem(fn, smem)) return GW_ERR_CUDA;
  const int tiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
  const int grid = std::max(1, std::min(tiles, num_sms));
  TraceScope ts(tracer, tf32 ? "tc_gemm_tf32" : "tc_gemm_bf16", st);
  if (tf32)
    tc_gemm_abt<true><<<grid, kThreads, smem, st>>>(mA, mB, M, N, K, e, status);
  else
    tc_gemm_abt<false><<<grid, kThreads, smem, st>>>(mA, mB, M, N, K, e, status);
  const cudaError_t err = cudaPeekAtLastError();
  if (err != cudaSuccess) {
    note_failure(cudaGetErrorString(err));
    return GW_ERR_CUDA;
  }
  return GW_OK;
}

}  // namespace gw
