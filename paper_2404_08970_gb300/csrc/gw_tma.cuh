// TMA tensor copies, the 128-byte shared-memory swizzle and named barriers.
#pragma once

#include <cuda.h>

#include "gw_common.cuh"

namespace gw {

__device__ __forceinline__ uint32_t swz128(uint32_t b) { return b ^ (((b >> 7) & 7u) << 4); }

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst_smem, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst_smem)),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Shared -> global tensor store of one box (bulk async-group completion).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int c0, int c1, int c2, const void* src_smem) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(tm), "r"(c0),
               "r"(c1), "r"(c2), "r"(smem_u32(src_smem))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until the shared-memory sources of this thread's committed bulk
// stores have been read (they may be overwritten afterwards).
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until this thread's committed bulk stores have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <typename Real, int VPT>
__device__ __forceinline__ void lds_swz(const unsigned char* base, int c0, Real (&out)[VPT]) {
  constexpr int PER = 16 / sizeof(Real);
#pragma unroll
  for (int j = 0; j < VPT / PER; ++j) {
    const uint32_t b = (uint32_t)((c0 + j * PER) * sizeof(Real));
    const float4 f = *reinterpret_cast<const float4*>(base + swz128(b));
    if constexpr (sizeof(Real) == 4) {
      out[j * 4 + 0] = f.x;
      out[j * 4 + 1] = f.y;
      out[j * 4 + 2] = f.z;
      out[j * 4 + 3] = f.w;
    } else {
      const double2 d = *reinterpret_cast<const double2*>(&f);
      out[j * 2 + 0] = d.x;
      out[j * 2 + 1] = d.y;
    }
  }
}

template <typename Real>
__device__ __forceinline__ void sts_swz(unsigned char* base, int idx, Real v) {
  *reinterpret_cast<Real*>(base + swz128((uint32_t)(idx * sizeof(Real)))) = v;
}

}  // namespace gw
