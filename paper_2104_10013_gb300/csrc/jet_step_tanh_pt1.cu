// Jet kernel instantiations: register tile of PT = 1 points, fixed-slope tanh networks only.
#include "jet_step.cuh"

namespace xp {

const void* jet_step_kernel_tanh_pt1(int nt) {
  switch (nt) {
    case 256: return reinterpret_cast<const void*>(jet_step_kernel<1, 256, false>);
    case 128: return reinterpret_cast<const void*>(jet_step_kernel<1, 128, false>);
    case 512: return reinterpret_cast<const void*>(jet_step_kernel<1, 512, false>);
    default: return nullptr;
  }
}

}  // namespace xp
