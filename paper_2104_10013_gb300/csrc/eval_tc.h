// Evaluation jets on the tensor cores (eval_tc.cu): launch interface for the
// host planner.  A network qualifies when it is the subdomain's only network,
// its output activation is the identity, its input is (x, y), it has at least
// one hidden-to-hidden layer and every hidden layer has the same width W, a
// width the kernel is built for (32, 64 or 80).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

struct TcArgs {
  const Item* items;        // IT_EVAL items (K[0] = 1, 3 or 5; K[1] = 0)
  int n_items;
  const int* n_items_dev;   // if not NULL: the item count is min(n_items, *n_items_dev)
  int* counter;             // work counter (zero before the launch)
  const SubDev* subs;
  const float* params;
  const float* img;         // tensor-core weight images (pack_tc_kernel)
  const int64_t* img_off;   // [n_sub] first float of each subdomain's images, -1: none
  const float2* pts;
  const float* scale;       // per point factor or NULL
  float* out;
  int dout;                 // floats per output row
  int* err;                 // device status word
};

// One hidden-to-hidden layer's image: W^k [n_out][n_in] from params[src] in
// the tensor cores' K-major layout, hi then lo, at img[dst].
struct TcPack {
  int64_t src, dst;
  int n_out, n_in;
};

bool eval_tc_width_ok(int W);
// Shared memory of the launch for width W and K jet components.
size_t eval_tc_smem_bytes(int W, int K);
// CTAs of one launch that fit on an SM (shared memory and tensor memory).
int eval_tc_ctas_per_sm(int W, int K);
cudaError_t eval_tc_configure();
void launch_eval_tc(int W, int K, const TcArgs& a, int grid, cudaStream_t s);
void launch_pack_tc(const float* params, const TcPack* blocks, int n_blocks, float* img, cudaStream_t s);

}  // namespace xp
