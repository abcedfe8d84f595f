// Jet kernel instantiations: register tile of PT = 2 points, fixed-slope tanh networks only.
#include "jet_step.cuh"

namespace xp {

const void* jet_step_kernel_tanh_pt2(int nt) {
  switch (nt) {
    case 256: return reinterpret_cast<const void*>(jet_step_kernel<2, 256, false>);
    case 128: return reinterpret_cast<const void*>(jet_step_kernel<2, 128, false>);
    default: return nullptr;
  }
}

}  // namespace xp
