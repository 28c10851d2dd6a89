// Structured 1D gradient, distance exponent k = 2.
#include "grad1d_impl.cuh"

namespace gw {

int grad1d_launch_k2(const Grad1DArgs& a, void* ws, size_t ws_bytes) {
  if (a.dtype == GW_F32) return grad1d_launch_typed<2, float>(a, ws, ws_bytes);
  return grad1d_launch_typed<2, double>(a, ws, ws_bytes);
}

}  // namespace gw
