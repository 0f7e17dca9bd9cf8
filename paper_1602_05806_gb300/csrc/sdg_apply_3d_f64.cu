// Instantiations of the 3D operator kernels (z-marching columns, element boxes) for dim = 3, double.
#include "sdg_apply3.cuh"

namespace sdg {

cudaError_t apply_dispatch_3d(const sdg_handle* h, const ApplyArgs<double>& a, cudaStream_t s) {
  // tile 0: the z-marching column kernel for n1 <= 5; otherwise element boxes
  if (a.tile == 0) {
    switch (h->g.n1) {
      case 1: return launch_apply3m_t<double, 1>(h, a, s);
      case 2: return launch_apply3m_t<double, 2>(h, a, s);
      case 3: return launch_apply3m_t<double, 3>(h, a, s);
      case 4: return launch_apply3m_t<double, 4>(h, a, s);
      case 5: return launch_apply3m_t<double, 5>(h, a, s);
      default: break;
    }
  }
  switch (h->g.n1) {
    case 1: return launch_apply_t<double, 3, 1>(h, a, s);
    case 2: return launch_apply_t<double, 3, 2>(h, a, s);
    case 3: return launch_apply_t<double, 3, 3>(h, a, s);
    case 4: return launch_apply_t<double, 3, 4>(h, a, s);
    case 5: return launch_apply_t<double, 3, 5>(h, a, s);
    case 6: return launch_apply_t<double, 3, 6>(h, a, s);
    case 7: return launch_apply_t<double, 3, 7>(h, a, s);
    case 8: return launch_apply_t<double, 3, 8>(h, a, s);
    case 9: return launch_apply_t<double, 3, 9>(h, a, s);
    case 10: return launch_apply_t<double, 3, 10>(h, a, s);
    case 11: return launch_apply_t<double, 3, 11>(h, a, s);
    case 12: return launch_apply_t<double, 3, 12>(h, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sdg
