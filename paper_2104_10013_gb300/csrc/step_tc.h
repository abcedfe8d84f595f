// Training-step kernel on the tensor cores (step_tc.cu): launch interface for
// the host planner.  A subdomain qualifies when it has one network with
// input (x, y), identity output of at most three components, tanh, sin or
// cos hidden layers with fixed or trained slopes, 3 to 8 weight layers and
// every hidden width within [min_width, 64], and its PDE trains with
// Laplacian jets (Poisson, Navier-Stokes).  Its residual items then run on
// this kernel; its data and interface items stay on the FP32 jet kernel.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

constexpr int STC_MAXL = 8;                  // weight layers (the tensor-memory budget: 128 + 64 (L - 2) columns)
constexpr int STC_W = 64;                    // hidden width of the tiles (narrower layers are zero-padded)
constexpr int STC_PTS = 32;                  // points per tile (128 rows of 4 jet components)
constexpr int STC_IMG = 2 * STC_W * STC_W;   // floats of one weight image (hi, then lo)
// per-CTA scratch (floats): the saved jets of layers 1..L-1, [layer][neuron][row]
constexpr int64_t STC_SCRATCH = (int64_t)(STC_MAXL - 1) * STC_W * 128;

struct StepTcArgs {
  const Item* items;         // IT_RES items of qualifying subdomains (K[0] = 4, lap = 1)
  int n_items;
  int item_base;             // loss_part slot of items[0]
  int* counter;              // work counter (zero before the launch)
  const SubDev* subs;
  const float* params;
  const float* img;          // weight images (pack_tc_train_kernel)
  const int64_t* img_off;    // [n_sub] first float of a subdomain's images, -1: none
  const float2* pts;
  const float* res_f;
  float* partials;
  double* loss_part;
  float* scratch;            // STC_SCRATCH floats per CTA
  int pde;
  float nu, re;
  int gen;                   // 1: some network has a general activation or trained slopes
  int* err;                  // device status word
};

// One weight image: W^k [n_out][n_in] (at params[src]) as the B operand of
// the forward contraction (transpose = 0: N = output neuron, K = input
// neuron) or of the reverse one (transpose = 1: N = input, K = output),
// zero-padded to 64 x 64, hi then lo, at img[dst].
struct TcTrainPack {
  int64_t src, dst;
  int n_out, n_in, transpose;
};

// Host: does network nd of a subdomain qualify (see above)?
bool step_tc_net_ok(const NetDev& nd, int n_nets, int pde, int min_width);
size_t step_tc_smem_bytes();
cudaError_t step_tc_configure();
void launch_step_tc(const StepTcArgs& a, int grid, cudaStream_t s);
void launch_pack_tc_train(const float* params, const TcTrainPack* blocks, int n_blocks, float* img,
                          cudaStream_t s);

}  // namespace xp
