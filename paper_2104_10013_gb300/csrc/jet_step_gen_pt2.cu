// Jet kernel instantiations: register tile of PT = 2 points, any activation, fixed or trainable slopes.
#include "jet_step.cuh"

namespace xp {

const void* jet_step_kernel_gen_pt2(int nt) {
  switch (nt) {
    case 256: return reinterpret_cast<const void*>(jet_step_kernel<2, 256, true>);
    case 128: return reinterpret_cast<const void*>(jet_step_kernel<2, 128, true>);
    default: return nullptr;
  }
}

}  // namespace xp
