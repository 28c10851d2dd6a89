// gw_grad_noalloc: the structured 1D gradient without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// gradient: a process whose device memory is fully reserved by another
// framework's caching allocator (an extra cudaMalloc would fail), a thread
// that must not block (cudaMalloc and cudaFree can synchronise the device),
// or code that must keep its memory footprint fixed after start-up.  For
// them this entry point takes its scratch from one file-scope device array of
// fixed size instead of a context workspace.  Inputs and outputs are still
// passed by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "gw_internal.h"

namespace {

// 32 MiB of scratch, reserved on every device that loads the library and kept
// until the process exits.  Enough for float problems up to about
// 4096 x 4096 (k <= 2); larger problems are rejected.
constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
// Status word of the kernels' bounded waits, shared by all calls like the
// scratch.  Cleared on the caller's stream before every launch; once a wait
// has run out, the other waits of the same launch see the bit and give up at
// once instead of each running to its own limit.
static __device__ __align__(256) unsigned g_noalloc_status;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned* g_status_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Device addresses of the scratch array and the status word on the current
// device.  Their names in host code are only host-side stand-ins, so the
// addresses are looked up once per device, with that device current.
int scratch_for_current_device(void** ptr, unsigned** status, int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GW_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p ||
        cudaGetSymbolAddress(&q, g_noalloc_status) != cudaSuccess || !q) {
      cudaGetLastError();
      return GW_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return GW_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
    g_status_ptr[dev] = (unsigned*)q;
    g_num_sms[dev] = sms;
  }
  *ptr = g_scratch_ptr[dev];
  *status = g_status_ptr[dev];
  *num_sms = g_num_sms[dev];
  return GW_OK;
}

}  // namespace

extern "C" gw_status gw_grad_noalloc(const gw_problem* p, const double* d_u, const double* d_v, const void* d_T,
                                     void* d_G, int marginals, void* stream) {
  if (!p || p->dim != 1 || p->nx < 1 || p->ny < 1 || p->k < 1 || p->k > 3 || p->ny > 16384 ||
      !(std::isfinite(p->hx) && p->hx > 0.0) || !(std::isfinite(p->hy) && p->hy > 0.0) || (p->dtype != GW_F32 && p->dtype != GW_F64))
    return GW_ERR_INVALID;
  if (marginals != GW_MARG_TARGET && marginals != GW_MARG_EXACT) return GW_ERR_INVALID;
  if (!gw::mixed_k_supported(p->k, p->ky, p->ny, p->dtype)) return GW_ERR_INVALID;
  if (!d_T || !d_G || (marginals == GW_MARG_TARGET && (!d_u || !d_v))) return GW_ERR_INVALID;
  const size_t esz = p->dtype == GW_F32 ? 4 : 8;
  const size_t nm = (size_t)p->nx * (size_t)p->ny;
  const char* t0 = (const char*)d_T;
  const char* g0 = (const char*)d_G;
  if (t0 < g0 + nm * esz && g0 < t0 + nm * esz) return GW_ERR_INVALID;
  void* scratch = nullptr;
  unsigned* status = nullptr;
  int num_sms = 0;
  int rc = scratch_for_current_device(&scratch, &status, &num_sms);
  if (rc != GW_OK) return (gw_status)rc;
  // Too large for the fixed scratch: reject rather than allocate.
  if (gw::grad1d_workspace_bytes(p->nx, p->ny, p->k, p->dtype, num_sms) > kNoallocScratchBytes)
    return GW_ERR_INVALID;
  gw::Grad1DArgs a{};
  a.n = p->nx;
  a.m = p->ny;
  a.k = p->k;
  a.ky = p->ky == p->k ? 0 : p->ky;
  a.hx = p->hx;
  a.hy = p->hy;
  a.dtype = p->dtype;
  a.T = d_T;
  a.G = d_G;
  a.u = d_u;
  a.v = d_v;
  a.exact = marginals == GW_MARG_EXACT;
  a.out_scale = 1.0;
  a.stream = (cudaStream_t)stream;
  a.status = status;
  a.num_sms = num_sms;
  a.tracer = nullptr;
  a.force_generic = 0;
  if (cudaMemsetAsync(status, 0, sizeof(unsigned), a.stream) != cudaSuccess) {
    cudaGetLastError();
    return GW_ERR_CUDA;
  }
  rc = gw::grad1d_launch(a, scratch, kNoallocScratchBytes);
  if (rc != GW_OK) {
    cudaGetLastError();
    return (gw_status)rc;
  }
  return GW_OK;
}
