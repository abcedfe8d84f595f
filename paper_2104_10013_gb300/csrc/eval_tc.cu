// Evaluation jets on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Forward jets of a network (Sec. 3) at query points for the networks
// eval_tc.h describes: the point-by-width contraction of every
// hidden-to-hidden layer runs as tcgen05.mma kind::tf32 in three passes over a
// hi/lo split of both operands (A_hi B_hi + A_hi B_lo + A_lo B_hi), hi and lo
// both rounded to nearest tf32 (the tensor cores would truncate fp32 inputs),
// so each operand is represented to 2^-22 and the dropped lo x lo term is
// below 2^-22 of a product.  The tf32 products are exact; hi x hi accumulates
// in one fp32 accumulator in tensor memory and the two cross terms in a second
// one, summed in the epilogue, so that the accumulation rounding of the cross
// terms stays at their own scale (about 2^-11 of the main term): with one
// accumulator the 3-pass sum erred up to 1.3e-5 of the jet scale on a width-80
// sin network with trained slopes, in emulation and on the GPU alike.  The
// first layer (two inputs) and the output layer (identity, at most three
// outputs) stay on the FP32 pipes.
//
// Tile: 128 rows = the MMA's M, one thread and one tensor-memory lane per row,
// a row per (point, jet component) for K = 1, 3 or 5 components (u; u, u_x,
// u_y; u, u_x, u_y, u_xx, u_yy).  A warp holds 32 / K whole points (its last
// 32 mod K rows are padding, held at zero), so that a point's rows share a
// warp: 128, 40 or 24 points per tile.  Per hidden layer: A = the activation
// rows H [128][W] and B = W^k [W][W], both K-major in shared memory in the
// no-swizzle canonical layout (core matrices of 8 rows x 16 bytes), D = Z
// [128 lanes][W columns] in tensor memory.  The epilogue reads a row of D per
// thread (tcgen05.ld); the value rows publish their pre-activations, all 128
// threads evaluate Phi, Phi', Phi'' once per (point, neuron) into tables that
// live in the A lo image (free between the layer's MMAs and the writing of the
// next A), and every row applies the jet rule
//   h_0 = Phi(v_0), h_i = Phi'(v_0) v_i, h_ii = Phi'(v_0) v_ii + Phi''(v_0) v_i^2
// (v = s z, s the layer's slope), the second-derivative rows taking v_i of
// their point from a third table.  The rows of h are the next A.
// Weight images (hi and lo, built by pack_tc_kernel) come by one bulk copy
// per layer into a single buffer, free again once a layer's MMAs complete: the
// copy of layer k + 1 is in flight while layer k's epilogue runs.  At width 64
// a tile then needs 98 KB of shared memory, so two CTAs (8 warps) share an SM
// to hide the epilogue's latencies.  Every wait is bounded; a wait that gives
// up sets the error word, the launch stops taking items, frees its tensor
// memory and ends.
#include <cuda_runtime.h>

#include <algorithm>

#include "eval_tc.h"
#include "jet_step.cuh"
#include "tc_util.cuh"

namespace xp {

namespace {

template <int W, int K>
struct TcSmem {
  static constexpr int PW = 32 / K;                // points per warp
  static constexpr int TP = 4 * PW;                // points per tile
  static constexpr int A = TC_ROWS * W;            // floats of one A image (hi or lo)
  static constexpr int B = 2 * W * W;              // floats of the weight buffer (hi, lo)
  static constexpr int Z = K > 1 ? W * TP : 0;     // (point, neuron) pairs of the activation tables
  static constexpr int DS = K == 5 ? 2 : 1;        // Phi' (3 components) or Phi', Phi'' (5) per pair
  static constexpr int VS = K == 5 ? 2 : 0;        // v_x, v_y per pair (second-derivative rows read them)
  static_assert((1 + DS + VS) * Z <= A, "the activation tables live in the A lo image");
  static constexpr int floats = 2 * A + B + 2 * TP;
  // tensor-memory columns: the main accumulator (hi x hi) at column 0, the
  // cross terms (hi x lo + lo x hi) at column COLS / 2
  static constexpr int COLS = W <= 32 ? 64 : (W <= 64 ? 128 : 256);
};

// This thread's row of Z = the main accumulator (columns of `main`) plus the
// cross-term accumulator (columns of `cross`), columns 0..W-1, into z.  The
// cross terms (about 2^-11 of the main term) accumulate apart, so that their
// accumulation rounding stays at that scale.
template <int W>
__device__ __forceinline__ void tmem_row(uint32_t main, uint32_t cross, float (&z)[W]) {
  uint32_t v[W], u[W];
#pragma unroll
  for (int c0 = 0; c0 < W; c0 += 16) {
    tmem_ld16(main + (uint32_t)c0, v + c0);
    tmem_ld16(cross + (uint32_t)c0, u + c0);
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c0 = 0; c0 < W; c0 += 8) {
    tmem_fence_regs8(v + c0);
    tmem_fence_regs8(u + c0);
  }
#pragma unroll
  for (int i = 0; i < W; ++i) z[i] = __uint_as_float(v[i]) + __uint_as_float(u[i]);
}

// The jet rule of the layer's activation on this thread's row (component c
// of point p; c = K on padding rows): z (without the bias) in, h out in z and
// in the A images.  With K > 1 the activation tables Zs (Phi) and Ds (Phi',
// and Phi'' for K = 5) and, for K = 5, Vs (v_x, v_y) occupy the A lo image
// until the last barrier.
template <int W, int K>
__device__ __forceinline__ void jet_rows(const Act& act, const float* __restrict__ bias, float (&z)[W], int r,
                                         int p, int c, bool valid, float* Ahi, float* Alo) {
  using S = TcSmem<W, K>;
  constexpr int TP = S::TP;
  if constexpr (K == 1) {
#pragma unroll
    for (int n = 0; n < W; ++n) {
      float d0, d1, d2, d3;
      phi_derivs(act.kind, act.s * (z[n] + __ldg(bias + n)), d0, d1, d2, d3);
      z[n] = valid ? d0 : 0.f;
    }
  } else {
    float* Zs = Alo;
    float* Ds = Alo + S::Z;
    float* Vs = Ds + S::DS * S::Z;   // K = 5: v_x, v_y of every pair
    if (c == 0) {
#pragma unroll
      for (int n = 0; n < W; ++n) Zs[n * TP + p] = z[n] + __ldg(bias + n);
    }
    if constexpr (K == 5) {
      if (c == 1 || c == 2) {
#pragma unroll
        for (int n = 0; n < W; ++n) Vs[(n * TP + p) * 2 + c - 1] = act.s * z[n];
      }
    }
    __syncthreads();
    for (int e = r; e < W * TP; e += TC_ROWS) {
      float d0, d1, d2, d3;
      phi_derivs(act.kind, act.s * Zs[e], d0, d1, d2, d3);
      Zs[e] = d0;
      if constexpr (K == 5)
        reinterpret_cast<float2*>(Ds)[e] = make_float2(d1, d2);
      else
        Ds[e] = d1;
    }
    __syncthreads();
    // second-derivative rows pair with the first-derivative row of their
    // direction (component 3 with 1, 4 with 2), whose v they read from Vs;
    // every lane loads and computes every candidate and selects (no branch)
    const int vsel = c >= 3 && c < K ? c - 3 : 0;
#pragma unroll
    for (int n = 0; n < W; ++n) {
      const int e = n * TP + p;
      const float vc = act.s * z[n];
      const float d0 = Zs[e];
      float h;
      if constexpr (K == 5) {
        const float2 d = reinterpret_cast<const float2*>(Ds)[e];
        const float vi = Vs[2 * e + vsel];
        const float h1 = d.x * vc;
        const float h2 = fmaf(d.y * vi, vi, h1);
        h = c == 0 ? d0 : (c >= 3 ? h2 : h1);
      } else {
        const float h1 = Ds[e] * vc;
        h = c == 0 ? d0 : h1;
      }
      z[n] = valid ? h : 0.f;
    }
    __syncthreads();   // the tables are read; A lo is written next
  }
#pragma unroll
  for (int j = 0; j < W; j += 4) {
    const float2 s0 = tf32_split(z[j]), s1 = tf32_split(z[j + 1]), s2 = tf32_split(z[j + 2]),
                 s3 = tf32_split(z[j + 3]);
    *reinterpret_cast<float4*>(Ahi + a_off(r, j)) = make_float4(s0.x, s1.x, s2.x, s3.x);
    *reinterpret_cast<float4*>(Alo + a_off(r, j)) = make_float4(s0.y, s1.y, s2.y, s3.y);
  }
}

template <int W, int K>
__global__ void __launch_bounds__(TC_ROWS, 1) eval_tc_kernel(TcArgs a) {
  using S = TcSmem<W, K>;
  constexpr int TP = S::TP;
  constexpr uint32_t IMG_BYTES = 4u * S::B;
  extern __shared__ __align__(1024) float tsm[];
  float* Ahi = tsm;
  float* Alo = tsm + S::A;
  float* B = tsm + 2 * S::A;
  float2* sp = reinterpret_cast<float2*>(tsm + 2 * S::A + S::B);
  __shared__ __align__(8) uint64_t bars[2];   // weight buffer, MMA completion
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_stop;
  const int r = threadIdx.x, lane = r & 31, warp = r >> 5;
  // row -> (point, component): whole points per warp, padding rows last (c = K)
  const bool pad = lane >= S::PW * K;
  const int p = pad ? 0 : warp * S::PW + lane / K;
  const int c = pad ? K : lane % K;
  if (r == 0) {
    for (int i = 0; i < 2; ++i) mbar_init(bars + i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "n"(S::COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t t_warp = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's lanes
  const uint32_t idesc = tc_idesc(W), idesc2 = tc_idesc(2 * W);
  const uint32_t sa_hi = smem_u32(Ahi), sa_lo = smem_u32(Alo);
  uint32_t wph = 0, mph = 0;
  const int n_items = a.n_items_dev ? min(a.n_items, *a.n_items_dev) : a.n_items;
  for (;;) {
    // one thread decides, so that every thread leaves the loop together
    if (r == 0) {
      s_item = atomicAdd(a.counter, 1);
      s_stop = *reinterpret_cast<volatile int*>(a.err) == XPINN_ERR_TIMEOUT;
    }
    __syncthreads();
    const int ii = s_item;
    const bool stop = s_stop != 0;
    __syncthreads();
    if (ii >= n_items || stop) break;
    const Item it = a.items[ii];
    const SubDev& sd = a.subs[it.q];
    const NetDev& nd = sd.net[0];
    const int L = nd.L;
    const int64_t io = a.img_off[it.q];
    bool ok = it.K[0] == K && it.K[1] == 0 && io >= 0 && L >= 3 && L <= MAXL && nd.w[0] == 2 &&
              nd.w[L] >= 1 && nd.w[L] <= XPINN_MAX_OUT && nd.out_act == XPINN_ACT_IDENTITY;
    for (int k = 1; k < L && ok; ++k) ok = nd.w[k] == W;
    if (!ok) {
      if (r == 0) atomicCAS(a.err, 0, XPINN_ERR_INVALID);
      continue;
    }
    const float* prm = a.params + sd.poff;
    const float* img = a.img + io;
    const int D = nd.w[L];
    for (int t0 = 0; t0 < it.n_pts; t0 += TP) {
      const int nv = min(TP, it.n_pts - t0);
      const bool valid = p < nv && c < K;
      // the first hidden-to-hidden layer's image (every earlier MMA has completed)
      if (r == 0) bulk_g2s(B, img, IMG_BYTES, bars);
      if (r < TP) sp[r] = r < nv ? a.pts[it.pt_off + t0 + r] : make_float2(0.f, 0.f);
      __syncthreads();
      float z[W];
      // layer 1: z = W^1 x (b^1 is added on the value rows), z_i = W^1[:, i], z_ii = 0
      {
        const float* W1 = prm + nd.off[1];
        const float2 x = sp[p];
#pragma unroll
        for (int n = 0; n < W; ++n) {
          const float w0 = __ldg(W1 + 2 * n), w1 = __ldg(W1 + 2 * n + 1);
          z[n] = c == 0 ? fmaf(w0, x.x, w1 * x.y) : (c == 1 ? w0 : (c == 2 ? w1 : 0.f));
        }
        jet_rows<W, K>(layer_act(nd, prm, 1), W1 + 2 * W, z, r, p, c, valid, Ahi, Alo);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      // hidden-to-hidden layers: Z = H W^T on the tensor cores, then the jet rule
      for (int k = 2; k <= L - 1; ++k) {
        if (r == 0) {
          mbar_wait(bars, wph, a.err);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sb_hi = smem_u32(B), sb_lo = smem_u32(B + W * W);
          constexpr uint32_t B_SBO = (uint32_t)(W / 4) * 128;
#pragma unroll
          for (int ks = 0; ks < W / 8; ++ks) {
            const uint64_t ahi = tc_sdesc(sa_hi + ks * 2 * TC_A_LBO, TC_A_LBO, 128);
            const uint64_t alo = tc_sdesc(sa_lo + ks * 2 * TC_A_LBO, TC_A_LBO, 128);
            const uint64_t bhi = tc_sdesc(sb_hi + ks * 256, 128, B_SBO);
            if constexpr (S::COLS / 2 == W) {
              // the image's hi and lo halves as one operand of N = 2 W (their
              // 8-row groups continue at the same stride): A_hi is read once
              // for hi x hi (columns 0..W-1) and hi x lo (the cross columns)
              tc_mma(tmem, ahi, bhi, idesc2, ks > 0 ? 1u : 0u);
            } else {
              const uint64_t blo = tc_sdesc(sb_lo + ks * 256, 128, B_SBO);
              tc_mma(tmem, ahi, bhi, idesc, ks > 0 ? 1u : 0u);
              tc_mma(tmem + S::COLS / 2, ahi, blo, idesc, ks > 0 ? 1u : 0u);
            }
            tc_mma(tmem + S::COLS / 2, alo, bhi, idesc, 1u);
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(bars + 1))
                       : "memory");
        }
        wph ^= 1u;
        mbar_wait(bars + 1, mph, a.err);
        mph ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the weight buffer is free again: the next layer's image, in flight
        // while this layer's epilogue runs
        if (r == 0 && k + 1 <= L - 1) bulk_g2s(B, img + (int64_t)(k - 1) * S::B, IMG_BYTES, bars);
        tmem_row<W>(t_warp, t_warp + S::COLS / 2, z);
        jet_rows<W, K>(layer_act(nd, prm, k), prm + nd.off[k] + W * W, z, r, p, c, valid, Ahi, Alo);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
      }
      // output layer (identity): y = W^L h + b^L on the value rows, W^L h on the others
      {
        const float* WL = prm + nd.off[L];
        const float* bL = WL + D * W;
        const float sc = (a.scale && p < nv) ? a.scale[it.pt_off + t0 + p] : 1.f;
#pragma unroll
        for (int o = 0; o < XPINN_MAX_OUT; ++o) {
          if (o >= D) break;
          float y = c == 0 ? __ldg(bL + o) : 0.f;
#pragma unroll
          for (int n = 0; n < W; ++n) y = fmaf(__ldg(WL + o * W + n), z[n], y);
          if (valid) a.out[it.out_off + (int64_t)(t0 + p) * a.dout + o * K + c] = sc * y;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(S::COLS) : "memory");
}

// Weight images for the tensor cores: W^k [n_out][n_in] in the no-swizzle
// K-major canonical layout (8-row groups n_in/4 x 128 bytes apart, K-adjacent
// core matrices 128 bytes apart), the hi parts then the lo parts of
// tf32_split.  One CTA per layer.
__global__ void __launch_bounds__(256) pack_tc_kernel(const float* __restrict__ params,
                                                      const TcPack* __restrict__ blocks, float* __restrict__ img) {
  const TcPack b = blocks[blockIdx.x];
  const float* W = params + b.src;
  float* hi = img + b.dst;
  float* lo = hi + b.n_out * b.n_in;
  for (int e = threadIdx.x; e < b.n_out * b.n_in; e += blockDim.x) {
    const int n = e / b.n_in, j = e - n * b.n_in;
    const float2 w = tf32_split(W[e]);
    const int off = (n >> 3) * (b.n_in / 4) * 32 + (j >> 2) * 32 + (n & 7) * 4 + (j & 3);
    hi[off] = w.x;
    lo[off] = w.y;
  }
}

template <int W, int K>
constexpr size_t smem_of() {
  return sizeof(float) * (size_t)TcSmem<W, K>::floats;
}

template <int W>
cudaError_t configure_w() {
  cudaError_t e = cudaFuncSetAttribute(eval_tc_kernel<W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_of<W, 1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eval_tc_kernel<W, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_of<W, 3>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(eval_tc_kernel<W, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_of<W, 5>());
  return e;
}

template <int W>
void launch_w(int K, const TcArgs& a, int grid, cudaStream_t s) {
  switch (K) {
    case 1: eval_tc_kernel<W, 1><<<grid, TC_ROWS, smem_of<W, 1>(), s>>>(a); break;
    case 3: eval_tc_kernel<W, 3><<<grid, TC_ROWS, smem_of<W, 3>(), s>>>(a); break;
    default: eval_tc_kernel<W, 5><<<grid, TC_ROWS, smem_of<W, 5>(), s>>>(a); break;
  }
}

static_assert(smem_of<80, 5>() + 64 <= 227 * 1024, "tensor-core evaluation tile exceeds shared memory");

}  // namespace

bool eval_tc_width_ok(int W) { return W == 32 || W == 64 || W == 80; }

size_t eval_tc_smem_bytes(int W, int K) {
  switch (W) {
    case 32: return K == 1 ? smem_of<32, 1>() : (K == 3 ? smem_of<32, 3>() : smem_of<32, 5>());
    case 64: return K == 1 ? smem_of<64, 1>() : (K == 3 ? smem_of<64, 3>() : smem_of<64, 5>());
    default: return K == 1 ? smem_of<80, 1>() : (K == 3 ? smem_of<80, 3>() : smem_of<80, 5>());
  }
}

int eval_tc_ctas_per_sm(int W, int K) {
  const int by_smem = (int)((227u << 10) / (eval_tc_smem_bytes(W, K) + 1024));
  const int cols = W <= 32 ? 64 : (W <= 64 ? 128 : 256);
  const int by_tmem = 512 / cols;
  // and at most four: registers (up to 255 a thread) allow no more
  return std::max(1, std::min(std::min(by_smem, by_tmem), 4));
}

cudaError_t eval_tc_configure() {
  cudaError_t e = configure_w<32>();
  if (e == cudaSuccess) e = configure_w<64>();
  if (e == cudaSuccess) e = configure_w<80>();
  return e;
}

void launch_eval_tc(int W, int K, const TcArgs& a, int grid, cudaStream_t s) {
  switch (W) {
    case 32: launch_w<32>(K, a, grid, s); break;
    case 64: launch_w<64>(K, a, grid, s); break;
    default: launch_w<80>(K, a, grid, s); break;
  }
}

void launch_pack_tc(const float* params, const TcPack* blocks, int n_blocks, float* img, cudaStream_t s) {
  if (n_blocks > 0) pack_tc_kernel<<<n_blocks, 256, 0, s>>>(params, blocks, img);
}

}  // namespace xp
