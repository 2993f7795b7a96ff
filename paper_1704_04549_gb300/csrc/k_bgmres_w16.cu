// Batched GMRES kernels with 16 lanes per system (device code in k_bgmres.cuh), in a
// translation unit of their own so that the three widths compile in parallel.
#include "k_bgmres.cuh"

namespace tpp {
namespace bg {

const void* kernel_w16(bool mixed, int minb) {
  if (minb >= 2)
    return mixed ? reinterpret_cast<const void*>(&k_bgmres<16, true, 2>)
                 : reinterpret_cast<const void*>(&k_bgmres<16, false, 2>);
  return mixed ? reinterpret_cast<const void*>(&k_bgmres<16, true, 1>)
               : reinterpret_cast<const void*>(&k_bgmres<16, false, 1>);
}

}  // namespace bg
}  // namespace tpp
