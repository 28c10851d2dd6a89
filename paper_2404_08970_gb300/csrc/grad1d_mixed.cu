// Structured 1D gradient with different distance exponents on X and Y
// (k_X = 1, k_Y = 2 and k_X = 2, k_Y = 1).
#include "grad1d_impl.cuh"

namespace gw {

int grad1d_launch_mixed(const Grad1DArgs& a, void* ws, size_t ws_bytes) {
  if (a.k == 1 && a.ky == 2)
    return a.dtype == GW_F32 ? grad1d_launch_typed<1, float, 2>(a, ws, ws_bytes)
                             : grad1d_launch_typed<1, double, 2>(a, ws, ws_bytes);
  if (a.k == 2 && a.ky == 1)
    return a.dtype == GW_F32 ? grad1d_launch_typed<2, float, 1>(a, ws, ws_bytes)
                             : grad1d_launch_typed<2, double, 1>(a, ws, ws_bytes);
  note_failure("mixed distance exponents: only (k_X, k_Y) = (1, 2) and (2, 1)");
  return GW_ERR_INVALID;
}

}  // namespace gw
