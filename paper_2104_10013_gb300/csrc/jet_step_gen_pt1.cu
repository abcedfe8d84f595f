// Jet kernel instantiations: register tile of PT = 1 points, any activation, fixed or trainable slopes.
#include "jet_step.cuh"

namespace xp {

const void* jet_step_kernel_gen_pt1(int nt) {
  switch (nt) {
    case 256: return reinterpret_cast<const void*>(jet_step_kernel<1, 256, true>);
    case 128: return reinterpret_cast<const void*>(jet_step_kernel<1, 128, true>);
    case 512: return reinterpret_cast<const void*>(jet_step_kernel<1, 512, true>);
    default: return nullptr;
  }
}

}  // namespace xp
