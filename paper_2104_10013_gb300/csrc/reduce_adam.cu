// Deterministic gradient reduction and per-subdomain Adam (Sec. 6).
//
// Every work item of the jet kernel left its gradient contribution in a
// private slice.  Here one thread per parameter sums the slices of its
// subdomain in a fixed order (so the result is bitwise reproducible), then
// applies one bias-corrected Adam step with the subdomain's own learning
// rate: the subdomains are optimised independently, as in Algorithm 1.
#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

constexpr int RT = 256;

// One weight image from the packed parameters (see NetDev), by a CTA.
__device__ __forceinline__ void pack_block(const float* __restrict__ params, const PackBlock& b,
                                           float* __restrict__ wimg) {
  const float* W = params + b.src;
  float* dst = wimg + b.dst;
  if (b.fwd) {
    // [in_p][out_p] = W^T, then [out_p] = b
    const int n_el = (b.in_p + 1) * b.out_p;
    for (int e = threadIdx.x; e < n_el; e += RT) {
      const int j = e / b.out_p, n = e - j * b.out_p;
      float v = 0.f;
      if (n < b.out_w) {
        if (j < b.in_w) v = W[(int64_t)n * b.in_w + j];
        else if (j == b.in_p) v = W[(int64_t)b.out_w * b.in_w + n];
      }
      dst[e] = v;
    }
  } else {
    // [out_p][in_p] = W
    const int n_el = b.out_p * b.in_p;
    for (int e = threadIdx.x; e < n_el; e += RT) {
      const int n = e / b.in_p, j = e - n * b.in_p;
      dst[e] = (n < b.out_w && j < b.in_w) ? W[(int64_t)n * b.in_w + j] : 0.f;
    }
  }
}

// Start of a step, one launch: CTA 0 resets the work counters of the jet
// launches, advances the Adam step count t and the loss-ring slot, and
// stores the bias corrections 1 - beta1^t and 1 - beta2^t (in double, once
// per step, for every CTA of the reduction); CTA b < n_blocks builds weight
// image b.
__global__ void __launch_bounds__(RT) step_start_kernel(StepStart a) {
  asm volatile("griddepcontrol.wait;" ::: "memory");   // see launch_pdl
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < a.n_counters; i += RT) a.counters[i] = 0;
    if (threadIdx.x == 0) {
      if (a.do_adam) {
        const int t = *a.step_t + 1;
        *a.step_t = t;
        a.bc[0] = (float)(1.0 - pow((double)a.beta1, (double)t));
        a.bc[1] = (float)(1.0 - pow((double)a.beta2, (double)t));
      }
      *a.loss_slot += 1;
    }
  }
  if ((int)blockIdx.x < a.n_blocks) pack_block(a.params, a.blocks[blockIdx.x], a.wimg);
}

// Launch as a programmatic dependent of the kernel before it on the stream:
// the launch overlaps that kernel's end; the kernel waits for the previous
// grid's completion (griddepcontrol.wait) before it reads or writes anything.
template <typename Arg>
void launch_pdl(void (*kernel)(Arg), int grid, const Arg& arg, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(RT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, arg);
}

void launch_step_start(const StepStart& a, cudaStream_t s) {
  launch_pdl(step_start_kernel, a.n_blocks > 1 ? a.n_blocks : 1, a, s);
}

__global__ void __launch_bounds__(RT) reduce_adam_kernel(ReduceArgs a) {
  asm volatile("griddepcontrol.wait;" ::: "memory");   // see launch_pdl
  const int2 blk = a.blocks[blockIdx.x];
  const int q = blk.x;
  const SubDev& sd = a.subs[q];
  const int ib = a.q_item_begin[q], ie = a.q_item_begin[q + 1];
  // loss terms of this subdomain (first block of the subdomain only): one
  // warp, lane l takes items l, l + 32, ...; the lanes' sums are combined by a
  // fixed butterfly, so the order is the same in every step
  if (blk.y == 0 && threadIdx.x < 32) {
    double acc[XPINN_N_TERMS];
#pragma unroll
    for (int t = 0; t < XPINN_N_TERMS; ++t) acc[t] = 0.0;
    for (int k = ib + (int)threadIdx.x; k < ie; k += 32) {
      const int ii = a.q_items[k];
      const int kind = a.items[ii].kind;
      const double l0 = a.loss_part[2 * ii], l1 = a.loss_part[2 * ii + 1];
      switch (kind) {
        case IT_DATA0: acc[0] += l0; break;
        case IT_DATA1: acc[1] += l0; break;
        case IT_RES: acc[2] += l0; break;
        case IT_IFACE:
          acc[3] += l0;
          acc[4] += l1;
          break;
        default: break;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int t = 0; t < XPINN_N_TERMS; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    if (threadIdx.x == 0) {
      const int slot = (*a.loss_slot) % a.ring_cap;
      bool finite = true;
#pragma unroll
      for (int t = 0; t < XPINN_N_TERMS; ++t) {
        const float l = (float)acc[t];
        a.loss_ring[((int64_t)slot * a.n_sub + q) * XPINN_N_TERMS + t] = l;
        finite = finite && isfinite(l);
      }
      // sticky until the host reads it at the next synchronising call
      if (!finite && a.err) atomicCAS(a.err, 0, XPINN_ERR_NONFINITE);
      // J(Theta_q) = W_u MSE_u (each net) + W_F MSE_F + W_I MSE_uavg + W_flux|W_IF MSE_flux|MSE_R
      // (Eqs. cPINNLoss, XPINNLoss), from the same float terms that are reported
      if (a.jq) {
        const float w[XPINN_N_TERMS] = {sd.w_data[0], sd.w_data[1], sd.w_res, sd.w_avg, sd.w_iface};
        double j = 0.0;
#pragma unroll
        for (int t = 0; t < XPINN_N_TERMS; ++t) j += (double)w[t] * (double)(float)acc[t];
        a.jq[q] = (float)j;
      }
    }
  }
  // the slice offsets of this subdomain's items, once per block
  constexpr int MAXI = 256;
  __shared__ int64_t s_off[MAXI];
  __shared__ float s_part[RT];
  const int n_it = ie - ib;
  for (int k = threadIdx.x; k < n_it && k < MAXI; k += RT) s_off[k] = a.q_part_off[ib + k];
  __syncthreads();
  // split threads per parameter: thread (s, j) sums items [s * chunk, (s + 1)
  // * chunk) of parameter blk.y + j in their order; the partial sums are
  // then added in s order, so the result is the same in every step
  const int S = a.split > 0 ? a.split : 1, PB = RT / S;
  const int sidx = threadIdx.x / PB, j = threadIdx.x - sidx * PB;
  const int e = blk.y + j;
  const int chunk = (n_it + S - 1) / S;
  const int k0 = min(n_it, sidx * chunk), k1 = min(n_it, k0 + chunk);
  float g = 0.f;
  if (e < sd.n_params) {
    int k = k0;
    if (n_it <= MAXI) {
      for (; k + 8 <= k1; k += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = a.partials[s_off[k + u] + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) g += v[u];
      }
      for (; k < k1; ++k) g += a.partials[s_off[k] + e];
    } else {
      for (; k < k1; ++k) g += a.partials[a.q_part_off[ib + k] + e];
    }
  }
  if (S > 1) {
    s_part[threadIdx.x] = g;
    __syncthreads();
    if (sidx != 0) return;
    for (int q = 1; q < S; ++q) g += s_part[q * PB + j];
  }
  if (e >= sd.n_params) return;
  const int64_t gi = sd.poff + e;
  if (a.grads) a.grads[gi] = g;
  if (a.do_adam) {
    const float b1 = a.beta1, b2 = a.beta2;
    const float m = b1 * a.m[gi] + (1.f - b1) * g;
    const float v = b2 * a.v[gi] + (1.f - b2) * g * g;
    a.m[gi] = m;
    a.v[gi] = v;
    const float mhat = m / a.bc[0];
    const float vhat = v / a.bc[1];
    a.params[gi] -= sd.lr * mhat / (sqrtf(vhat) + a.eps);
  }
}

void launch_reduce_adam(const ReduceArgs& a, cudaStream_t s) {
  if (a.n_blocks > 0) launch_pdl(reduce_adam_kernel, a.n_blocks, a, s);
}

// J(Theta) = sum_q J(Theta_q): lane l sums subdomains l, l + 32, ... in
// order, the lanes' sums are combined by a fixed butterfly.
__global__ void objective_sum_kernel(const float* __restrict__ jq, int n_sub, float* __restrict__ out) {
  double s = 0.0;
  for (int q = threadIdx.x; q < n_sub; q += 32) s += (double)jq[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = (float)s;
}

void launch_objective_sum(const float* jq, int n_sub, float* out, cudaStream_t s) {
  objective_sum_kernel<<<1, 32, 0, s>>>(jq, n_sub, out);
}

// Weight images (layout in xpinn_dev.cuh): one CTA per image; consecutive
// threads write consecutive image floats.
__global__ void __launch_bounds__(RT) pack_weights_kernel(const float* __restrict__ params,
                                                          const PackBlock* __restrict__ blocks,
                                                          float* __restrict__ wimg) {
  pack_block(params, blocks[blockIdx.x], wimg);
}

void launch_pack_weights(const float* params, const PackBlock* blocks, int n_blocks, float* wimg,
                         cudaStream_t s) {
  if (n_blocks > 0) pack_weights_kernel<<<n_blocks, RT, 0, s>>>(params, blocks, wimg);
}

}  // namespace xp
