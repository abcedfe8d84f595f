// Host side of the jet kernel: shared-memory size and attribute, occupancy
// and launch.  The kernel instantiations live in jet_step_{tanh,gen}_pt1.cu
// (PT = 1; 256, 128 and 512 threads) and jet_step_{tanh,gen}_pt2.cu (PT = 2;
// 256 and 128 threads): the tanh family for problems whose networks are all
// fixed-slope tanh networks, the general family for the rest.
#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

const void* jet_step_kernel_tanh_pt1(int nt);
const void* jet_step_kernel_tanh_pt2(int nt);
const void* jet_step_kernel_gen_pt1(int nt);
const void* jet_step_kernel_gen_pt2(int nt);

namespace {

// The kernel for a register tile of pt points and nt threads, or NULL.
const void* kernel_for(int pt, int nt, bool gen) {
  if (nt == 512 && pt != 1) return nullptr;
  if (nt != 128 && nt != 256 && nt != 512) return nullptr;
  if (pt == 1) return gen ? jet_step_kernel_gen_pt1(nt) : jet_step_kernel_tanh_pt1(nt);
  if (pt == 2) return gen ? jet_step_kernel_gen_pt2(nt) : jet_step_kernel_tanh_pt2(nt);
  return nullptr;
}

}  // namespace

size_t jet_step_smem_bytes(const StepArgs& a) {
  // A, B, two weight buffers, U, Ub, point coordinates; 32 doubles for
  // reductions, two mbarriers and, for the general family, the per-warp
  // slope-gradient partials [2 nets][16 warps][MAXL] (see carve in jet_step.cuh)
  const size_t floats = 2 * (size_t)a.szA + 2 * (size_t)a.szW + 2 * (size_t)a.szU + 2 * (size_t)a.pmax;
  return floats * sizeof(float) + 32 * sizeof(double) + 2 * sizeof(uint64_t) +
         (a.gen ? 2 * 16 * MAXL * sizeof(double) : 0);
}

cudaError_t jet_step_configure(size_t smem) {
  const int v = (int)smem;
  const int cfg[5][2] = {{1, 256}, {2, 256}, {1, 128}, {2, 128}, {1, 512}};
  for (const bool gen : {false, true})
    for (const auto& c : cfg) {
      const cudaError_t e =
          cudaFuncSetAttribute(kernel_for(c[0], c[1], gen), cudaFuncAttributeMaxDynamicSharedMemorySize, v);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

int jet_step_blocks_per_sm(int pt, int nt, bool gen, size_t smem) {
  const void* k = kernel_for(nt == 512 ? 1 : pt, nt, gen);
  int n = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, nt, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Launched as a programmatic dependent of the kernel before it on the
// stream: its launch overlaps that kernel's end, and the kernel waits for the
// previous grid's completion (griddepcontrol.wait) before it reads anything.
void launch_jet_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s) {
  const int nt = a.nt == 512 || a.nt == 128 ? a.nt : 256;
  const void* k = kernel_for(nt == 512 || a.pt == 1 ? 1 : 2, nt, a.gen != 0);
  StepArgs arg = a;
  void* params[] = {&arg};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelExC(&cfg, k, params);
}

}  // namespace xp
