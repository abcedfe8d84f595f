// Grouped, persistent jet kernel for the cPINN / XPINN training step
// (device code; the kernel's instantiations are compiled in
// jet_step_{tanh,gen}_pt{1,2}.cu, one kernel family and register tile each,
// so that the translation units build in parallel; jet_step.cu holds the
// host side).
//
// One CTA processes work items pulled from an atomic counter.  An item is a
// range of points of one subdomain and one kind (residual, data, interface
// side, interface exchange, evaluation).  Its points are processed in
// sub-tiles of P points:
//
//   forward   for every network of the subdomain, the Taylor jet of the
//             network (Sec. 3) at the P points: value, first derivatives and
//             diagonal second derivatives, propagated layer by layer as
//             z^k = W^k h^{k-1} + b^k (all jet components share W^k) and
//             h = tanh(z) with the chain rule for the derivative components;
//             the pre-activation jets (t, z_i, z_ii) are saved to per-CTA
//             scratch for the reverse pass;
//   loss      per point, the residual of the PDE (Sec. 2, Sec. 7), the data
//             mismatch, or the interface terms of Eq. cPINNLoss / Eq.
//             XPINNLoss against the neighbour's values read from the exchange
//             buffer (held constant, Algorithm 1); the derivative of the
//             weighted loss with respect to every jet component (the seeds);
//   reverse   back through the jet, layer by layer, accumulating dW^k, db^k
//             into the item's private gradient slice.
//
// Layer contractions are register-tiled FP32 FFMA loops: a thread owns MT=8
// neurons x PT points x K jet components (PT = 1 or 2, a template parameter:
// PT = 1 keeps a thread under 128 registers so that two CTAs share an SM);
// activations live in shared memory laid out [neuron][point][component], so
// a thread's points and components are one contiguous run of a row.
#pragma once
#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

// Jet arrays (activations and adjoints in shared memory, the saved jets in
// global scratch, the output jets) are laid out [row][point][component]: a
// row (neuron or output) holds P x K floats with the K jet components of a
// point adjacent.  A thread's register tile covers PT points ("slots") of K
// components, acc[i][s * K + c].  For K = 4 and PT = 2 the threads in lanes
// 4-7 of every 8 hold their two points in swapped slots (slot s is point
// p0 + (s ^ 1)), so that the 16-byte accesses of 8 consecutive threads fall
// in 8 different bank groups.
template <int K, int PT>
__device__ __forceinline__ int tile_swap() {
  if constexpr (K == 4 && PT == 2)
    return (int)(threadIdx.x >> 2) & 1;
  else
    return 0;
}

// the K components of one point (K = 4: 16-byte aligned; K = 2: 8-byte)
template <int K>
__device__ __forceinline__ void ldk(const float* __restrict__ p, float (&v)[K]) {
  if constexpr (K == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else if constexpr (K == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = p[c];
  }
}
template <int K>
__device__ __forceinline__ void stk(float* __restrict__ p, const float (&v)[K]) {
  if constexpr (K == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (K == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) p[c] = v[c];
  }
}

// The thread's tile of one row, r = row + p0 * K (p0 even when PT = 2, so
// r is 8-byte aligned), in slot order.
template <int K, int PT>
__device__ __forceinline__ void ld_tile(const float* __restrict__ r, float (&v)[PT * K], int sw) {
  if constexpr (K == 4 && PT == 2) {
    const float4 a = *reinterpret_cast<const float4*>(r + 4 * sw);
    const float4 b = *reinterpret_cast<const float4*>(r + 4 - 4 * sw);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else if constexpr (PT == 2) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const float2 t = reinterpret_cast<const float2*>(r)[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  } else {
    float t[K];
    ldk<K>(r, t);
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = t[c];
  }
}
template <int K, int PT>
__device__ __forceinline__ void st_tile(float* __restrict__ r, const float (&v)[PT * K], int sw) {
  if constexpr (K == 4 && PT == 2) {
    *reinterpret_cast<float4*>(r + 4 * sw) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(r + 4 - 4 * sw) = make_float4(v[4], v[5], v[6], v[7]);
  } else if constexpr (PT == 2) {
#pragma unroll
    for (int q = 0; q < K; ++q) reinterpret_cast<float2*>(r)[q] = make_float2(v[2 * q], v[2 * q + 1]);
  } else {
    float t[K];
#pragma unroll
    for (int c = 0; c < K; ++c) t[c] = v[c];
    stk<K>(r, t);
  }
}

struct Smem {
  float* A;      // activations H^{k} / H^{k-1}      [wp][P][K]
  float* B;      // adjoints z-bar^k                 [wp][P][K], rows RSZ apart
  float* W0;     // two weight-image buffers: one layer's image is copied
  float* W1;     //   into one while the other layer's is in use
  float* U;      // output jets of every net         [D][P][K] per net
  float* Ub;     // seeds (adjoints of U)
  float* sx;     // point coordinates, SoA
  float* sy;
  double* red;   // 32 doubles for block reductions
  uint64_t* bar; // 2 mbarriers, one per weight buffer
  double* slope; // [net][warp][layer] partial slope gradients of the current item (general family)
};

// Sizes of the shared-memory regions (floats).  Functions that are not
// inlined receive this by value and rebuild their pointers from the
// extern __shared__ array, so that the compiler knows they address shared
// memory (32-bit shared loads and stores, not generic ones).
struct SmemLayout {
  int szA, szW, szU, pmax;
  int slopes;   // 1: the per-warp slope-gradient partials exist (general kernel family)
};

constexpr int SLOPE_WARPS = 16;   // warps of the largest CTA (512 threads)

__device__ __forceinline__ Smem carve(SmemLayout l) {
  extern __shared__ __align__(16) float sm[];
  Smem s;
  s.A = sm;
  s.B = s.A + l.szA;
  s.W0 = s.B + l.szA;
  s.W1 = s.W0 + l.szW;
  s.U = s.W1 + l.szW;
  s.Ub = s.U + l.szU;
  s.sx = s.Ub + l.szU;
  s.sy = s.sx + l.pmax;
  s.red = reinterpret_cast<double*>(s.sy + l.pmax);
  s.bar = reinterpret_cast<uint64_t*>(s.red + 32);
  s.slope = reinterpret_cast<double*>(s.bar + 2);
  return s;
}

// ---------------------------------------------------------------------------
// Weight images are brought into shared memory by the bulk-copy (TMA) engine:
// one cp.async.bulk per layer, completion counted in bytes on an mbarrier.
// Each of the two buffers has its own mbarrier; the parity of the phase to
// wait for is tracked in the bits of `ph` (bit b for buffer b), which every
// thread updates identically.  Waits are bounded (about a second at 2 GHz);
// a wait that gives up sets the error flag and returns, so the launch ends
// and the host reports XPINN_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One thread: copy `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global memory to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Every thread: wait for the phase of `bar` with parity `parity`, that is
// for the bulk copy it counts.  The wait is bounded: about a second (2^31
// clock cycles), or about a millisecond once some wait has already given up
// (the error word holds XPINN_ERR_TIMEOUT), which still drains a copy in
// flight (a copy of one layer's weights takes microseconds) but keeps a
// launch whose barriers are out of step from waiting a second per layer.
// So a copy in flight (of valid memory, done in microseconds) is waited for
// before the CTA reuses the buffer or exits.  Other codes in the error word
// (a non-finite loss of an earlier step) do not shorten the wait.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  const long long t0 = clock64();
  long long limit = 0;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return;
    if (limit == 0)
      limit = *reinterpret_cast<volatile int*>(err) == XPINN_ERR_TIMEOUT ? (1ll << 21) : (1ll << 31);
    if (clock64() - t0 > limit) {
      atomicCAS(err, 0, XPINN_ERR_TIMEOUT);
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// tanh jet, forward and reverse (Sec. 3 network with Phi = tanh, slope 1).
// Components: 0 value, 1..2 first derivatives, 3..4 second derivatives
// (component 3 pairs with 1, 4 with 2).
//   h = t,  h_i = s z_i,  h_ii = s z_ii - 2 t s z_i^2,  t = tanh(z), s = 1 - t^2
// Laplacian jets (LAP, K = 4): component 3 carries the Laplacian z_11 + z_22,
// whose rule is exact because the diagonal terms add:
//   h_lap = s z_lap - 2 t s (z_1^2 + z_2^2).
// PDEs that only need the Laplacian (Poisson, Navier-Stokes, the diffusion
// u-network) train with 4 components instead of 5.
// ---------------------------------------------------------------------------
template <int K, bool LAP>
__device__ __forceinline__ void tanh_jet(const float (&z)[K], float (&h)[K], float& t_out) {
  const float t = tanhf(z[0]);
  const float s = 1.f - t * t;
  h[0] = t;
  if (K > 1) h[1] = s * z[1];
  if (K > 2) h[2] = s * z[2];
  if (K > 3) h[3] = s * z[3] - 2.f * t * s * (LAP ? z[1] * z[1] + z[2] * z[2] : z[1] * z[1]);
  if (K > 4) h[4] = s * z[4] - 2.f * t * s * z[2] * z[2];
  t_out = t;
}

// h from the saved (t, z_1, z_2, z_11, z_22)
template <int K, bool LAP>
__device__ __forceinline__ void tanh_jet_from_saved(const float (&sv)[K], float (&h)[K]) {
  const float t = sv[0];
  const float s = 1.f - t * t;
  h[0] = t;
  if (K > 1) h[1] = s * sv[1];
  if (K > 2) h[2] = s * sv[2];
  if (K > 3) h[3] = s * sv[3] - 2.f * t * s * (LAP ? sv[1] * sv[1] + sv[2] * sv[2] : sv[1] * sv[1]);
  if (K > 4) h[4] = s * sv[4] - 2.f * t * s * sv[2] * sv[2];
}

// Reverse of tanh_jet: adjoints hb of (h, h_i, h_ii) to adjoints of (z, z_i, z_ii).
template <int K, bool LAP>
__device__ __forceinline__ void tanh_jet_bwd(const float (&sv)[K], const float (&hb)[K], float (&zb)[K]) {
  const float t = sv[0];
  const float s = 1.f - t * t;
  float tb = hb[0];
  if (K > 1) { zb[1] = s * hb[1]; tb -= 2.f * t * sv[1] * hb[1]; }
  if (K > 2) { zb[2] = s * hb[2]; tb -= 2.f * t * sv[2] * hb[2]; }
  if (K > 3) {
    zb[3] = s * hb[3];
    zb[1] -= 4.f * t * s * sv[1] * hb[3];
    if (LAP) zb[2] -= 4.f * t * s * sv[2] * hb[3];
    const float g2 = LAP ? sv[1] * sv[1] + sv[2] * sv[2] : sv[1] * sv[1];
    tb += (-2.f * t * sv[3] + (6.f * t * t - 2.f) * g2) * hb[3];
  }
  if (K > 4) {
    zb[4] = s * hb[4];
    zb[2] -= 4.f * t * s * sv[2] * hb[4];
    tb += (-2.f * t * sv[4] + (6.f * t * t - 2.f) * sv[2] * sv[2]) * hb[4];
  }
  zb[0] = s * tb;
}

// ---------------------------------------------------------------------------
// General hidden activation h = Phi(v), v = s z with the layer's slope
// s = n a^k (Sec. 3) and Phi = tanh, sin or cos.  With d_m = Phi^(m)(v_0):
//   h = d_0,  h_i = d_1 v_i,  h_ii = d_1 v_ii + d_2 v_i^2.
// A tanh network with fixed slopes keeps the cheaper path above (GEN =
// false: saved t); every other network (GEN = true) saves the unscaled
// pre-activation jet z and recomputes Phi in the reverse pass, which also
// needs z for the slope gradient.  GEN is a template parameter of the
// network passes, so the tanh path carries none of the general code.
// ---------------------------------------------------------------------------
struct Act {
  int kind;        // XPINN_PHI_*
  float s;         // slope n a^k of the layer
};

__device__ __forceinline__ Act layer_act(const NetDev& nd, const float* prm, int k) {
  Act a;
  a.kind = nd.act;
  a.s = nd.aoff < 0 ? 1.f : nd.scale * __ldg(prm + nd.aoff + k - 1);
  return a;
}

// sin and cos of v in one call site per kernel: sincosf carries a long
// argument-reduction path for large |v| that would otherwise be inlined at
// every activation of every network pass.
static __device__ __noinline__ float2 sin_cos(float v) {
  float sn, cs;
  sincosf(v, &sn, &cs);
  return make_float2(sn, cs);
}

// Phi and its first three derivatives at v
__device__ __forceinline__ void phi_derivs(int kind, float v, float& d0, float& d1, float& d2, float& d3) {
  if (kind == XPINN_PHI_TANH) {
    const float t = tanhf(v), q = 1.f - t * t;
    d0 = t;
    d1 = q;
    d2 = -2.f * t * q;
    d3 = (6.f * t * t - 2.f) * q;
  } else {
    const float2 sc = sin_cos(v);
    const float sn = sc.x, cs = sc.y;
    if (kind == XPINN_PHI_SIN) {
      d0 = sn; d1 = cs; d2 = -sn; d3 = -cs;
    } else {
      d0 = cs; d1 = -sn; d2 = -cs; d3 = sn;
    }
  }
}

template <int K, bool LAP>
__device__ __forceinline__ void phi_jet(const Act& a, const float (&z)[K], float (&h)[K]) {
  float v[K];
#pragma unroll
  for (int c = 0; c < K; ++c) v[c] = a.s * z[c];
  float d0, d1, d2, d3;
  phi_derivs(a.kind, v[0], d0, d1, d2, d3);
  h[0] = d0;
  if (K > 1) h[1] = d1 * v[1];
  if (K > 2) h[2] = d1 * v[2];
  if (K > 3) h[3] = fmaf(d2 * v[1], v[1], d1 * v[3]) + (LAP ? d2 * v[2] * v[2] : 0.f);
  if (K > 4) h[4] = fmaf(d2 * v[2], v[2], d1 * v[4]);
}

// forward: h from the pre-activation jet z; sv0 is the value to save at component 0
template <int K, bool LAP, bool GEN>
__device__ __forceinline__ void act_jet(const Act& a, const float (&z)[K], float (&h)[K], float& sv0) {
  if constexpr (!GEN) {
    tanh_jet<K, LAP>(z, h, sv0);
  } else {
    phi_jet<K, LAP>(a, z, h);
    sv0 = z[0];
  }
}

template <int K, bool LAP, bool GEN>
__device__ __forceinline__ void act_jet_from_saved(const Act& a, const float (&sv)[K], float (&h)[K]) {
  if constexpr (!GEN)
    tanh_jet_from_saved<K, LAP>(sv, h);
  else
    phi_jet<K, LAP>(a, sv, h);
}

// reverse: adjoints hb of h to adjoints zb of the unscaled z; gs += dJ/ds
// (= sum over components of vb_c z_c, vb the adjoint of v = s z).
template <int K, bool LAP, bool GEN>
__device__ __forceinline__ void act_jet_bwd(const Act& a, const float (&sv)[K], const float (&hb)[K],
                                            float (&zb)[K], float& gs) {
  if constexpr (!GEN) {
    tanh_jet_bwd<K, LAP>(sv, hb, zb);
  } else {
    float v[K], vb[K];
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = a.s * sv[c];
    float d0, d1, d2, d3;
    phi_derivs(a.kind, v[0], d0, d1, d2, d3);
    float b0 = d1 * hb[0];
    if (K > 1) { vb[1] = d1 * hb[1]; b0 += d2 * v[1] * hb[1]; }
    if (K > 2) { vb[2] = d1 * hb[2]; b0 += d2 * v[2] * hb[2]; }
    if (K > 3) {
      vb[3] = d1 * hb[3];
      vb[1] += 2.f * d2 * v[1] * hb[3];
      if (LAP) vb[2] += 2.f * d2 * v[2] * hb[3];
      const float g2 = LAP ? v[1] * v[1] + v[2] * v[2] : v[1] * v[1];
      b0 += (d2 * v[3] + d3 * g2) * hb[3];
    }
    if (K > 4) {
      vb[4] = d1 * hb[4];
      vb[2] += 2.f * d2 * v[2] * hb[4];
      b0 += (d2 * v[4] + d3 * v[2] * v[2]) * hb[4];
    }
    vb[0] = b0;
#pragma unroll
    for (int c = 0; c < K; ++c) {
      gs = fmaf(vb[c], sv[c], gs);
      zb[c] = a.s * vb[c];
    }
  }
}

// Sum over the CTA; the result is valid in thread 0.  Fixed order: warp
// shuffles, then the warps' partial sums in warp order.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// softplus output activation: y = log(1+e^z), y_i = g z_i, y_ii = g z_ii + g(1-g) z_i^2
__device__ __forceinline__ float softplus_f(float z) {
  return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
}
__device__ __forceinline__ float sigmoid_f(float z) {
  return 1.f / (1.f + expf(-z));
}

// ---------------------------------------------------------------------------
// Register-tiled contractions
// ---------------------------------------------------------------------------

// Two fused multiply-adds in one instruction (packed FP32, sm_100 and later):
// (a.x b.x + c.x, a.y b.y + c.y), each rounded as fmaf rounds it.
__device__ __forceinline__ void ffma2(float& c0, float& c1, float a0, float a1, float b0, float b1) {
  uint64_t c = (uint64_t)__float_as_uint(c0) | ((uint64_t)__float_as_uint(c1) << 32);
  const uint64_t a = (uint64_t)__float_as_uint(a0) | ((uint64_t)__float_as_uint(a1) << 32);
  const uint64_t b = (uint64_t)__float_as_uint(b0) | ((uint64_t)__float_as_uint(b1) << 32);
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(a), "l"(b));
  c0 = __uint_as_float((uint32_t)c);
  c1 = __uint_as_float((uint32_t)(c >> 32));
}

// The register-tiled contraction of both passes:
//   acc[i][m] = sum_{r < R} W[r * ws + col0 + i] X[r * xs + xo + m]  (+ bias[col0 + i] on
//   the value component c = 0 of every slot when BIAS),
// for the thread's MT columns col0.. of W (two float4s a row) and its tile of
// PT x K floats at offset xo of every X row (slots as ld_tile).  Forward:
// X = H^{k-1}, W = (W^k)^T, R = the true input width (padded inputs are zero).
// Reverse: X = Z-bar^k, W = W^k, R = the true output width.  Pairs of
// adjacent tile entries share one packed FMA.
template <int K, int PT, bool BIAS>
__device__ __forceinline__ void gemm_tile(const float* __restrict__ X, int xs, int xo, const float* __restrict__ W,
                                          int ws, int col0, int R, const float* __restrict__ bias, int sw,
                                          float (&acc)[MT][PT * K]) {
  constexpr int MK = PT * K;
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    const float b = BIAS ? bias[col0 + i] : 0.f;
#pragma unroll
    for (int m = 0; m < MK; ++m) acc[i][m] = (m % K == 0) ? b : 0.f;
  }
  const float* wp = W + col0;
  const float* xp = X + xo;
#pragma unroll 4
  for (int r = 0; r < R; ++r) {
    const float4 wa = *reinterpret_cast<const float4*>(wp + r * ws);
    const float4 wb = *reinterpret_cast<const float4*>(wp + r * ws + 4);
    const float w[MT] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    float v[MK];
    ld_tile<K, PT>(xp + r * xs, v, sw);
#pragma unroll
    for (int i = 0; i < MT; ++i) {
#pragma unroll
      for (int m = 0; m + 1 < MK; m += 2) ffma2(acc[i][m], acc[i][m + 1], w[i], w[i], v[m], v[m + 1]);
      if constexpr ((MK & 1) != 0) acc[i][MK - 1] = fmaf(w[i], v[MK - 1], acc[i][MK - 1]);
    }
  }
}

// Gradient slices are private to an item: its first sub-tile stores, later
// sub-tiles add with a reduction that does not wait for the old value.  The
// same thread owns the same element in every sub-tile, so the additions of
// one element happen in program order and the result is deterministic.
__device__ __forceinline__ void accum(float* p, float v, bool first) {
  if (first)
    *p = v;
  else
    atomicAdd(p, v);
}

// dW[n][j] += sum_{p,c} Zb[n][p][c] H[j][p][c] for n < out_w, j < in_w, with
// Zb rows at stride RSZ and H given transposed, HT[(p*K + c)][j] (row stride
// RS).  Each thread owns an 8 x TB tile of dW (TB = 4 measured fastest; 8,
// and unrolling the contraction loop, were slower).  Its rows
// n = tn + i * (out_p / 8), i = 0..7, are interleaved so that the threads of
// a warp, which hold consecutive tiles, read adjacent Zb rows (different
// banks when RSZ mod 32 is not 0 or 16) and consecutive HT columns.  Per 4
// contraction steps a thread loads 8 Zb and TB HT float4s for 32 TB FMAs.
// Narrow layers split the contraction: S threads (a power of two, up to 16)
// share a tile as lanes l, l + 32/S, ... of one warp, and their partial
// tiles are added with a fixed butterfly of warp shuffles (deterministic; no
// shared-memory buffer and no block barrier; a shared-memory reduction with
// two barriers was 0.1 ms slower on the default workload).
template <int TB>
__device__ __forceinline__ void dW_tiles_warp(const float* __restrict__ Zb, int RSZ, const float* __restrict__ HT,
                                              int RS, int out_p, int in_p, int out_w, int in_w, int KP,
                                              float* __restrict__ pW, bool first) {
  constexpr int NB = TB / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const int tj_n = in_p / TB, tn_n = out_p >> 3;
  const int T = tj_n * tn_n;
  int S = (int)blockDim.x / T;
  S = S >= 16 ? 16 : (S >= 8 ? 8 : (S >= 4 ? 4 : (S >= 2 ? 2 : 1)));
  const int TPW = 32 / S;   // tiles per warp
  const int KP4 = KP >> 2, RSZ4 = RSZ >> 2;
  const int sp = lane / TPW;
  for (int base = 0; base < T; base += n_warps * TPW) {
    const int tile = base + warp * TPW + (lane - sp * TPW);
    const bool valid = tile < T;
    const int tt = valid ? tile : 0;
    const int tn = tt / tj_n, tj = tt - tn * tj_n;
    const int j0 = tj * TB;
    float acc[8][TB];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int jj = 0; jj < TB; ++jj) acc[i][jj] = 0.f;
    if (valid) {
      const float4* z4 = reinterpret_cast<const float4*>(Zb) + tn * RSZ4;
      const int zstep = tn_n * RSZ4;
      for (int g = sp; g < KP4; g += S) {
        float4 h[4][NB];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float4* hp = reinterpret_cast<const float4*>(HT + (4 * g + t) * RS + j0);
#pragma unroll
          for (int q = 0; q < NB; ++q) h[t][q] = hp[q];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 z = z4[i * zstep + g];
          const float zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int q = 0; q < NB; ++q) {
              ffma2(acc[i][4 * q + 0], acc[i][4 * q + 1], h[t][q].x, h[t][q].y, zv[t], zv[t]);
              ffma2(acc[i][4 * q + 2], acc[i][4 * q + 3], h[t][q].z, h[t][q].w, zv[t], zv[t]);
            }
        }
      }
    }
    for (int o = TPW; o < 32; o <<= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < TB; ++jj) acc[i][jj] += __shfl_xor_sync(0xffffffffu, acc[i][jj], o);
    if (valid && sp == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = tn + i * tn_n;
#pragma unroll
        for (int jj = 0; jj < TB; ++jj)
          if (n < out_w && j0 + jj < in_w) accum(pW + n * in_w + j0 + jj, acc[i][jj], first);
      }
    }
  }
}

// Row dot products with 8 lanes per row pair: out[r] (+)= sum_k X[r][k] Y[r'][k].
// `rows` pairs of 4 * len4 floats; X row r starts at X + xr(r), Y's at
// Y + yr(r) (float offsets, multiples of 4; Y NULL: plain sum).
template <typename XR, typename YR, typename OUT>
__device__ __forceinline__ void group_dots(int rows, int len4, const float* __restrict__ X,
                                           const float* __restrict__ Y, XR xr, YR yr, OUT out) {
  const int lane8 = threadIdx.x & 7;
  const int warp = threadIdx.x >> 5;
  for (int base = warp * 4; base < rows; base += (int)(blockDim.x >> 5) * 4) {
    const int r = base + ((threadIdx.x >> 3) & 3);
    const bool valid = r < rows;
    float acc = 0.f;
    if (valid) {
      const float4* x4 = reinterpret_cast<const float4*>(X + xr(r));
      if (Y) {
        const float4* y4 = reinterpret_cast<const float4*>(Y + yr(r));
        for (int g = lane8; g < len4; g += 8) {
          const float4 x = x4[g], y = y4[g];
          acc = fmaf(x.x, y.x, acc);
          acc = fmaf(x.y, y.y, acc);
          acc = fmaf(x.z, y.z, acc);
          acc = fmaf(x.w, y.w, acc);
        }
      } else {
        for (int g = lane8; g < len4; g += 8) {
          const float4 x = x4[g];
          acc += (x.x + x.y) + (x.z + x.w);
        }
      }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (valid && lane8 == 0) out(r, acc);
  }
}

// Gradients of the first layer (2 inputs), whose jets are z = W x + b,
// z_i = W[:, i] and z_ii = 0: for each neuron n, in one pass over its
// adjoint row (8 lanes per neuron, each over every 8th point; fixed-order sums),
//   dW[n][i] = sum_p zb0[n][p] x_i[p] + sum_p zb_{1+i}[n][p],  db[n] = sum_p zb0[n][p].
template <int K>
__device__ __forceinline__ void layer1_grads(int rows, int P, const float* __restrict__ Zb, int RSZ,
                                             const float* __restrict__ sx, const float* __restrict__ sy,
                                             float* __restrict__ gW, float* __restrict__ gb, bool first) {
  const int lane8 = threadIdx.x & 7;
  const int warp = threadIdx.x >> 5;
  for (int base = warp * 4; base < rows; base += (int)(blockDim.x >> 5) * 4) {
    const int r = base + ((threadIdx.x >> 3) & 3);
    const bool valid = r < rows;
    float ax = 0.f, ay = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f;
    if (valid) {
      const float* zr = Zb + r * RSZ;
      for (int p = lane8; p < P; p += 8) {
        float z[K];
        ldk<K>(zr + p * K, z);
        const float x = sx[p], y = sy[p];
        ax = fmaf(z[0], x, ax);
        ay = fmaf(z[0], y, ay);
        a0 += z[0];
        if (K > 1) a1 += z[1];
        if (K > 2) a2 += z[2];
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (valid && lane8 == 0) {
      accum(gW + 2 * r, ax + a1, first);
      accum(gW + 2 * r + 1, ay + a2, first);
      accum(gb + r, a0, first);
    }
  }
}

// Sums over the points of the value component (c = 0) of `rows` rows of
// P x K floats at stride rs: out(r, sum) with 8 lanes per row, fixed order.
template <int K, typename OUT>
__device__ __forceinline__ void value_sums(int rows, int P, const float* __restrict__ X, int rs, OUT out) {
  const int lane8 = threadIdx.x & 7;
  const int warp = threadIdx.x >> 5;
  for (int base = warp * 4; base < rows; base += (int)(blockDim.x >> 5) * 4) {
    const int r = base + ((threadIdx.x >> 3) & 3);
    const bool valid = r < rows;
    float acc = 0.f;
    if (valid) {
      const float* xr = X + r * rs;
      for (int p = lane8; p < P; p += 8) acc += xr[p * K];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (valid && lane8 == 0) out(r, acc);
  }
}

// The CTA's walk over a row-major [rows][P] array: this thread's elements
// tid, tid + blockDim.x, ... as (row r, column c), stepped without division.
struct Walk {
  int r, c, dr, dc, P;
  __device__ __forceinline__ explicit Walk(int P_) : P(P_) {
    r = (int)threadIdx.x / P;
    c = (int)threadIdx.x - r * P;
    dr = (int)blockDim.x / P;
    dc = (int)blockDim.x - dr * P;
  }
  __device__ __forceinline__ void next() {
    r += dr;
    c += dc;
    if (c >= P) {
      c -= P;
      ++r;
    }
  }
};

// ---------------------------------------------------------------------------
// Network forward with jets.  Leaves the output jets in Uo [D][P][K] and the
// saved pre-activation jets of every layer in S.
// S layout: layer 1..L-1: [wp_k][P][K] each, then layer L: [D][P][K].
// ---------------------------------------------------------------------------
template <int K, bool LAP, int PT, bool GEN>
__device__ __noinline__ uint32_t net_forward(SmemLayout sl, const NetDev& nd, const float* __restrict__ prm,
                                             const float* __restrict__ img, int P, float* __restrict__ S,
                                             int uoff, uint32_t ph, int* err) {
  const Smem s = carve(sl);
  float* __restrict__ Uo = s.U + uoff;
  const int tid = threadIdx.x;
  const int n_pg = P / PT;
  const int L = nd.L;
  // the first hidden-to-hidden layer's image (into buffer 0) while layer 1 runs
  if (tid == 0 && L > 2) bulk_g2s(s.W0, img + nd.imf[2], 4u * layer_img_floats(nd, 2), s.bar);
  // ---- layer 1 (2 inputs): z = W^1 x + b^1, z_i = W^1[:, i], z_ii = 0
  {
    const Act a1 = GEN ? layer_act(nd, prm, 1) : Act{};
    const int w1 = nd.w[1], wp1 = nd.wp[1];
    const float* W1 = prm + nd.off[1];
    const float* b1 = W1 + 2 * w1;
    for (Walk wk(P); wk.r < wp1; wk.next()) {
      const int n = wk.r, p = wk.c;
      float w0 = 0.f, wv = 0.f, b = 0.f;
      if (n < w1) {
        w0 = __ldg(W1 + 2 * n);
        wv = __ldg(W1 + 2 * n + 1);
        b = __ldg(b1 + n);
      }
      float z[K], h[K], t;
      z[0] = fmaf(w0, s.sx[p], fmaf(wv, s.sy[p], b));
      if (K > 1) z[1] = w0;
      if (K > 2) z[2] = wv;
      if (K > 3) z[3] = 0.f;
      if (K > 4) z[4] = 0.f;
      act_jet<K, LAP, GEN>(a1, z, h, t);
      z[0] = t;
      stk<K>(s.A + (n * P + p) * K, h);
      stk<K>(S + (n * P + p) * K, z);
    }
  }
  float* Sk = S + nd.wp[1] * K * P;
  __syncthreads();
  // ---- hidden layers 2 .. L-1.  Activations alternate between A and B (B
  // holds adjoints only in the reverse pass), so one barrier per layer
  // suffices.  Layer k uses weight buffer (k - 2) & 1, and the next layer's
  // image goes into the other buffer, whose last readers (layer k - 1)
  // finished before the barrier that ended that layer.
  float* Ain = s.A;
  float* Aout = s.B;
  for (int k = 2; k <= L - 1; ++k) {
    const int in_p = nd.wp[k - 1], out_p = nd.wp[k], in_w = nd.w[k - 1];
    const Act ak = GEN ? layer_act(nd, prm, k) : Act{};
    const int b = (k - 2) & 1;
    const float* Wt = b ? s.W1 : s.W0;   // [in_p][out_p] = W^k transposed, then b^k
    if (tid == 0 && k + 1 <= L - 1)
      bulk_g2s(b ? s.W0 : s.W1, img + nd.imf[k + 1], 4u * layer_img_floats(nd, k + 1), s.bar + (b ^ 1));
    mbar_wait(s.bar + b, (ph >> b) & 1u, err);
    ph ^= 1u << b;
    const int ng = tid / n_pg, pg = tid - ng * n_pg;
    const bool act = ng < out_p / MT;
    const int n0 = ng * MT, p0 = pg * PT;
    const int sw = tile_swap<K, PT>();
    const int KP = K * P;
    float acc[MT][PT * K];
    if (act) {
      gemm_tile<K, PT, true>(Ain, KP, p0 * K, Wt, out_p, n0, in_w, Wt + in_p * out_p, sw, acc);
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        float sv[PT * K];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
          float z[K], h[K], t;
#pragma unroll
          for (int c = 0; c < K; ++c) z[c] = acc[i][q * K + c];
          act_jet<K, LAP, GEN>(ak, z, h, t);
#pragma unroll
          for (int c = 0; c < K; ++c) {
            sv[q * K + c] = c == 0 ? t : z[c];
            acc[i][q * K + c] = h[c];
          }
        }
        st_tile<K, PT>(Sk + (n0 + i) * KP + p0 * K, sv, sw);
      }
#pragma unroll
      for (int i = 0; i < MT; ++i) st_tile<K, PT>(Aout + (n0 + i) * KP + p0 * K, acc[i], sw);
    }
    __syncthreads();
    Sk += out_p * K * P;
    float* t = Ain;
    Ain = Aout;
    Aout = t;
  }
  // ---- output layer L
  {
    const int in_w = nd.w[L - 1], D = nd.w[L];
    const float* WL = prm + nd.off[L];
    const float* bL = WL + D * in_w;
    for (Walk wk(P); wk.r < D; wk.next()) {
      const int o = wk.r, p = wk.c;
      float z[K];
      z[0] = __ldg(bL + o);
#pragma unroll
      for (int c = 1; c < K; ++c) z[c] = 0.f;
      const float* wrow = WL + o * in_w;
      for (int j = 0; j < in_w; ++j) {
        const float w = __ldg(wrow + j);
        float h[K];
        ldk<K>(Ain + (j * P + p) * K, h);
#pragma unroll
        for (int c = 0; c < K; ++c) z[c] = fmaf(w, h[c], z[c]);
      }
      stk<K>(Sk + (o * P + p) * K, z);
      float y[K];
      if (nd.out_act == XPINN_ACT_SOFTPLUS) {
        const float g = sigmoid_f(z[0]);
        const float g1 = g * (1.f - g);
        y[0] = softplus_f(z[0]);
        if (K > 1) y[1] = g * z[1];
        if (K > 2) y[2] = g * z[2];
        if (K > 3) y[3] = g * z[3] + g1 * (LAP ? z[1] * z[1] + z[2] * z[2] : z[1] * z[1]);
        if (K > 4) y[4] = g * z[4] + g1 * z[2] * z[2];
      } else {
#pragma unroll
        for (int c = 0; c < K; ++c) y[c] = z[c];
      }
      stk<K>(Uo + (o * P + p) * K, y);
    }
  }
  __syncthreads();
  return ph;
}

// H^{k}[n][p][c] = act(saved S^k) into dst, for all n < wp (padded rows give 0)
template <int K, bool LAP, bool GEN>
__device__ __forceinline__ void act_from_saved(const Act& a, float* __restrict__ dst, const float* __restrict__ Sk,
                                               int wp, int P) {
  for (Walk wk(P); wk.r < wp; wk.next()) {
    const int e = (wk.r * P + wk.c) * K;
    float sv[K], h[K];
    ldk<K>(Sk + e, sv);
    act_jet_from_saved<K, LAP, GEN>(a, sv, h);
    stk<K>(dst + e, h);
  }
}

// The same, transposed: HT[(p*K + c) * wp + n] (row stride wp), for the
// weight-gradient contraction, whose contraction index is the position
// p*K + c within a row.  A thread takes one neuron and 4 consecutive points.
template <int K, bool LAP, bool GEN>
__device__ __forceinline__ void act_from_saved_T(const Act& a, float* __restrict__ HT, const float* __restrict__ Sk,
                                                 int wp, int P) {
  const int P4 = P >> 2;
  for (Walk wk(wp); wk.r < P4; wk.next()) {
    const int n = wk.c, p4 = 4 * wk.r;
    float sv[4][K];
#pragma unroll
    for (int t = 0; t < 4; ++t) ldk<K>(Sk + (n * P + p4 + t) * K, sv[t]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float h[K];
      act_jet_from_saved<K, LAP, GEN>(a, sv[t], h);
#pragma unroll
      for (int c = 0; c < K; ++c) HT[((p4 + t) * K + c) * wp + n] = h[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Network reverse pass.  Ub holds the seeds [D][P][K] (overwritten).  The
// gradient slice gslice receives dW^k, db^k at the network's offsets.
// ---------------------------------------------------------------------------
template <int K, bool LAP, int PT, bool GEN>
__device__ __noinline__ uint32_t net_backward(SmemLayout sl, const NetDev& nd, const float* __restrict__ prm,
                                              const float* __restrict__ img, int P, const float* __restrict__ S,
                                              int uoff, float* __restrict__ gslice, bool first, uint32_t ph,
                                              int* err, int net, int hl) {
  const Smem s = carve(sl);
  float* __restrict__ Ub = s.Ub + uoff;
  const int tid = threadIdx.x;
  const int n_pg = P / PT;
  const int L = nd.L;
  const int KP = K * P;
  // reverse image of layer L-1 (into buffer 0) while the output layer runs;
  // layer k uses buffer (L - 1 - k) & 1
  if (tid == 0 && L - 1 >= 2) bulk_g2s(s.W0, img + nd.imb[L - 1], 4u * nd.wp[L - 1] * nd.wp[L - 2], s.bar);
  // saved jets of layer L (top), then walk down layer by layer
  const float* SL = S;
  for (int k = 1; k < L; ++k) SL += nd.wp[k] * KP;

  // ---- output layer
  const int D = nd.w[L], in_w = nd.w[L - 1], in_p = nd.wp[L - 1];
  if (nd.out_act == XPINN_ACT_SOFTPLUS) {
    for (Walk wk(P); wk.r < D; wk.next()) {
      const int o = wk.r, p = wk.c;
      float z[K], yb[K], zb[K];
      ldk<K>(SL + (o * P + p) * K, z);
      ldk<K>(Ub + (o * P + p) * K, yb);
      const float g = sigmoid_f(z[0]);
      const float g1 = g * (1.f - g);
      const float g2 = g1 * (1.f - 2.f * g);
      float b0 = g * yb[0];
      if (K > 1) { zb[1] = g * yb[1]; b0 += g1 * z[1] * yb[1]; }
      if (K > 2) { zb[2] = g * yb[2]; b0 += g1 * z[2] * yb[2]; }
      if (K > 3) {
        zb[3] = g * yb[3];
        zb[1] += 2.f * g1 * z[1] * yb[3];
        if (LAP) zb[2] += 2.f * g1 * z[2] * yb[3];
        b0 += (g1 * z[3] + g2 * (LAP ? z[1] * z[1] + z[2] * z[2] : z[1] * z[1])) * yb[3];
      }
      if (K > 4) { zb[4] = g * yb[4]; zb[2] += 2.f * g1 * z[2] * yb[4]; b0 += (g1 * z[4] + g2 * z[2] * z[2]) * yb[4]; }
      zb[0] = b0;
      stk<K>(Ub + (o * P + p) * K, zb);
    }
  }
  const float* Sk = SL - in_p * KP;   // saved jets of layer L-1
  // H^{L-1}: still in the activation buffer the forward pass left it in when
  // this network's forward pass was the item's last (hl = 0: A, 1: B; the
  // barrier after the loss stage made the seeds visible), else rebuilt into A
  const float* HL = hl == 1 ? s.B : s.A;
  if (hl < 0) {
    act_from_saved<K, LAP, GEN>(GEN ? layer_act(nd, prm, L - 1) : Act{}, s.A, Sk, in_p, P);
    __syncthreads();
  } else if (nd.out_act == XPINN_ACT_SOFTPLUS) {
    __syncthreads();   // the softplus seeds above
  }
  {
    float* gW = gslice + nd.off[L];
    float* gb = gW + D * in_w;
    // dW^L[o][j] = sum_{p,c} zb^L[o][p][c] H^{L-1}[j][p][c]
    group_dots(D * in_w, KP / 4, Ub, HL, [=](int r) { return (r / in_w) * KP; },
               [=](int r) { return (r % in_w) * KP; }, [=](int r, float v) { accum(gW + r, v, first); });
    // db^L[o] = sum_p zb^L[o][p][0]
    value_sums<K>(D, P, Ub, KP, [=](int r, float v) { accum(gb + r, v, first); });
  }
  // h-bar^{L-1} = (W^L)^T zb^L into registers (the thread's tile, slots as ld_tile)
  const int sw = tile_swap<K, PT>();
  float acc[MT][PT * K];
  {
    const float* WL = prm + nd.off[L];
    const int ng = tid / n_pg, pg = tid - ng * n_pg;
    const int j0 = ng * MT, p0 = pg * PT;
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int m = 0; m < PT * K; ++m) acc[i][m] = 0.f;
    if (ng < in_p / MT) {
      for (int o = 0; o < D; ++o) {
        float w[MT];
#pragma unroll
        for (int i = 0; i < MT; ++i) w[i] = (j0 + i < in_w) ? __ldg(WL + o * in_w + j0 + i) : 0.f;
        float zb[PT * K];
        ld_tile<K, PT>(Ub + o * KP + p0 * K, zb, sw);
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
          for (int m = 0; m < PT * K; ++m) acc[i][m] = fmaf(w[i], zb[m], acc[i][m]);
      }
    }
  }
  __syncthreads();

  // ---- hidden layers L-1 .. 1 (Sk points at the saved jets of layer k).
  // Adjoint rows in B are RSZ floats apart (padded so that adjacent rows
  // fall in different banks for the weight-gradient tiles).
  const int RSZ = adj_stride(K, P);
  for (int k = L - 1; k >= 1; --k) {
    const int out_p = nd.wp[k], out_w = nd.w[k];
    const int ng = tid / n_pg, pg = tid - ng * n_pg;
    const int n0 = ng * MT, p0 = pg * PT;
    const Act ak = GEN ? layer_act(nd, prm, k) : Act{};
    const int b = (L - 1 - k) & 1;
    // the next layer's reverse image into the other buffer, last read by the
    // contraction of layer k + 1 (before the barrier that ended it)
    if (tid == 0 && k - 1 >= 2)
      bulk_g2s(b ? s.W0 : s.W1, img + nd.imb[k - 1], 4u * nd.wp[k - 1] * nd.wp[k - 2], s.bar + (b ^ 1));
    float gs = 0.f;   // dJ/ds_k, this thread's part
    if (ng < out_p / MT) {
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        float sv2[PT * K];
        ld_tile<K, PT>(Sk + (n0 + i) * KP + p0 * K, sv2, sw);
#pragma unroll
        for (int q = 0; q < PT; ++q) {
          float sv[K], hb[K], zb[K];
#pragma unroll
          for (int c = 0; c < K; ++c) {
            sv[c] = sv2[q * K + c];
            hb[c] = acc[i][q * K + c];
          }
          act_jet_bwd<K, LAP, GEN>(ak, sv, hb, zb, gs);
#pragma unroll
          for (int c = 0; c < K; ++c) acc[i][q * K + c] = zb[c];
        }
        st_tile<K, PT>(s.B + (n0 + i) * RSZ + p0 * K, acc[i], sw);
      }
    }
    if (GEN && nd.aoff >= 0) {
      // dJ/ds_k: this warp's part, kept per warp over the item's sub-tiles
      // (summed over the warps in order at the end of the item); no barrier
      float w = gs;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if ((tid & 31) == 0) {
        double* sp = s.slope + (net * SLOPE_WARPS + (tid >> 5)) * MAXL + (k - 1);
        *sp = first ? (double)w : *sp + (double)w;
      }
    }
    float* gW = gslice + nd.off[k];
    if (k >= 2) {
      const int in_pk = nd.wp[k - 1], in_wk = nd.w[k - 1];
      const float* Skm1 = Sk - in_pk * KP;
      act_from_saved_T<K, LAP, GEN>(GEN ? layer_act(nd, prm, k - 1) : Act{}, s.A, Skm1, in_pk, P);
      const float* Wn = b ? s.W1 : s.W0;   // [out_p][in_pk] = W^k
      mbar_wait(s.bar + b, (ph >> b) & 1u, err);
      ph ^= 1u << b;
      __syncthreads();
      // h-bar^{k-1} = (W^k)^T zb^k into registers, then dW^k and db^k
      if (ng < in_pk / MT) gemm_tile<K, PT, false>(s.B, RSZ, p0 * K, Wn, in_pk, n0, out_w, nullptr, sw, acc);
      dW_tiles_warp<4>(s.B, RSZ, s.A, in_pk, out_p, in_pk, out_w, in_wk, KP, gW, first);
      float* gb = gW + out_w * in_wk;
      value_sums<K>(out_w, P, s.B, RSZ, [=](int r, float v) { accum(gb + r, v, first); });
      Sk = Skm1;
    } else {
      __syncthreads();
      // layer 1: dW^1[n][i] = sum_p zb0[n][p] x_i[p] + sum_p zb_{1+i}[n][p], db^1[n] = sum_p zb0[n][p]
      layer1_grads<K>(out_w, P, s.B, RSZ, s.sx, s.sy, gW, gW + 2 * out_w, first);
    }
    __syncthreads();
  }
  return ph;
}

// ---------------------------------------------------------------------------
// PDE residuals, fluxes and their derivatives with respect to the jets.
// J[net][o][c]: jets of output o of net `net` (net 1 only for diffusion).
// ---------------------------------------------------------------------------
struct PtJets {
  float u[XPINN_MAX_OUT][KMAX];   // net 0
  float k[KMAX];                  // net 1 (single output)
};

__device__ __forceinline__ int residual_fwd(int pde, const PtJets& J, float f, float nu, float re,
                                            float r[3]) {
  switch (pde) {
    case XPINN_PDE_BURGERS:   // u_t + u u_x - nu u_xx - f
      r[0] = J.u[0][2] + J.u[0][0] * J.u[0][1] - nu * J.u[0][3] - f;
      return 1;
    case XPINN_PDE_POISSON:   // -(u_xx + u_yy) - f
      r[0] = -(J.u[0][3] + J.u[0][4]) - f;
      return 1;
    case XPINN_PDE_NS: {
      const float* u = J.u[0];
      const float* v = J.u[1];
      const float* p = J.u[2];
      const float ire = 1.f / re;
      r[0] = u[0] * u[1] + v[0] * u[2] + p[1] - (u[3] + u[4]) * ire;
      r[1] = u[0] * v[1] + v[0] * v[2] + p[2] - (v[3] + v[4]) * ire;
      r[2] = u[1] + v[2];
      return 3;
    }
    default: {                // K lap u + grad K . grad u - f
      r[0] = J.k[0] * (J.u[0][3] + J.u[0][4]) + J.k[1] * J.u[0][1] + J.k[2] * J.u[0][2] - f;
      return 1;
    }
  }
}

// G += sum_eq e[eq] d r_eq / d J
__device__ __forceinline__ void residual_seed(int pde, const PtJets& J, const float e[3], float nu,
                                              float re, PtJets& G) {
  switch (pde) {
    case XPINN_PDE_BURGERS:
      G.u[0][0] += e[0] * J.u[0][1];
      G.u[0][1] += e[0] * J.u[0][0];
      G.u[0][2] += e[0];
      G.u[0][3] -= nu * e[0];
      break;
    case XPINN_PDE_POISSON:
      G.u[0][3] -= e[0];
      G.u[0][4] -= e[0];
      break;
    case XPINN_PDE_NS: {
      const float* u = J.u[0];
      const float* v = J.u[1];
      const float ire = 1.f / re;
      G.u[0][0] += e[0] * u[1] + e[1] * v[1];
      G.u[0][1] += e[0] * u[0] + e[2];
      G.u[0][2] += e[0] * v[0];
      G.u[0][3] -= e[0] * ire;
      G.u[0][4] -= e[0] * ire;
      G.u[1][0] += e[0] * u[2] + e[1] * v[2];
      G.u[1][1] += e[1] * u[0];
      G.u[1][2] += e[1] * v[0] + e[2];
      G.u[1][3] -= e[1] * ire;
      G.u[1][4] -= e[1] * ire;
      G.u[2][1] += e[0];
      G.u[2][2] += e[1];
      break;
    }
    default:
      G.u[0][1] += e[0] * J.k[1];
      G.u[0][2] += e[0] * J.k[2];
      G.u[0][3] += e[0] * J.k[0];
      G.u[0][4] += e[0] * J.k[0];
      G.k[0] += e[0] * (J.u[0][3] + J.u[0][4]);
      G.k[1] += e[0] * J.u[0][1];
      G.k[2] += e[0] * J.u[0][2];
      break;
  }
}

// normal flux f . n (cPINN)
__device__ __forceinline__ int flux_fwd(int pde, const PtJets& J, float n0, float n1, float nu,
                                        float re, int mode, float phi[3]) {
  switch (pde) {
    case XPINN_PDE_BURGERS: {
      const float u = J.u[0][0], ux = J.u[0][1];
      const float fx = mode == XPINN_FLUX_CONSERVATIVE ? 0.5f * u * u - nu * ux : u * ux - nu * ux;
      phi[0] = n0 * fx + n1 * u;
      return 1;
    }
    case XPINN_PDE_POISSON:
      phi[0] = -(n0 * J.u[0][1] + n1 * J.u[0][2]);
      return 1;
    case XPINN_PDE_NS: {
      const float* u = J.u[0];
      const float* v = J.u[1];
      const float* p = J.u[2];
      const float ire = 1.f / re;
      phi[0] = n0 * (u[0] * u[0] + p[0] - u[1] * ire) + n1 * (u[0] * v[0] - u[2] * ire);
      phi[1] = n0 * (u[0] * v[0] - v[1] * ire) + n1 * (v[0] * v[0] + p[0] - v[2] * ire);
      phi[2] = n0 * u[0] + n1 * v[0];
      return 3;
    }
    default:
      phi[0] = J.k[0] * (n0 * J.u[0][1] + n1 * J.u[0][2]);
      return 1;
  }
}

__device__ __forceinline__ void flux_seed(int pde, const PtJets& J, float n0, float n1, float nu,
                                          float re, int mode, const float e[3], PtJets& G) {
  switch (pde) {
    case XPINN_PDE_BURGERS: {
      const float u = J.u[0][0], ux = J.u[0][1];
      if (mode == XPINN_FLUX_CONSERVATIVE) {
        G.u[0][0] += e[0] * (n0 * u + n1);
        G.u[0][1] += e[0] * (-nu * n0);
      } else {
        G.u[0][0] += e[0] * (n0 * ux + n1);
        G.u[0][1] += e[0] * (n0 * (u - nu));
      }
      break;
    }
    case XPINN_PDE_POISSON:
      G.u[0][1] -= e[0] * n0;
      G.u[0][2] -= e[0] * n1;
      break;
    case XPINN_PDE_NS: {
      const float* u = J.u[0];
      const float* v = J.u[1];
      const float ire = 1.f / re;
      // x-momentum
      G.u[0][0] += e[0] * (2.f * n0 * u[0] + n1 * v[0]);
      G.u[1][0] += e[0] * (n1 * u[0]);
      G.u[2][0] += e[0] * n0;
      G.u[0][1] -= e[0] * n0 * ire;
      G.u[0][2] -= e[0] * n1 * ire;
      // y-momentum
      G.u[0][0] += e[1] * (n0 * v[0]);
      G.u[1][0] += e[1] * (n0 * u[0] + 2.f * n1 * v[0]);
      G.u[2][0] += e[1] * n1;
      G.u[1][1] -= e[1] * n0 * ire;
      G.u[1][2] -= e[1] * n1 * ire;
      // mass
      G.u[0][0] += e[2] * n0;
      G.u[1][0] += e[2] * n1;
      break;
    }
    default: {
      const float gn = n0 * J.u[0][1] + n1 * J.u[0][2];
      G.k[0] += e[0] * gn;
      G.u[0][1] += e[0] * J.k[0] * n0;
      G.u[0][2] += e[0] * J.k[0] * n1;
      break;
    }
  }
}

// ---------------------------------------------------------------------------
// Item processing
// ---------------------------------------------------------------------------
// Network passes for K components.  The tanh kernel (GEN = false) holds only
// the fixed-slope tanh passes; the general kernel picks, per network, the
// tanh passes or the general ones.
template <int PT, bool GEN>
__device__ uint32_t forward_any(int K, bool lap, SmemLayout sl, const NetDev& nd, const float* prm, const float* img,
                                int P, float* S, int uoff, uint32_t ph, int* err) {
#define XP_FWD(KK, L, G) return net_forward<KK, L, PT, G>(sl, nd, prm, img, P, S, uoff, ph, err)
#define XP_SWITCH(G)                         \
  switch (K) {                               \
    case 1: XP_FWD(1, false, G);             \
    case 2: XP_FWD(2, false, G);             \
    case 3: XP_FWD(3, false, G);             \
    case 4:                                  \
      if (lap) XP_FWD(4, true, G);           \
      XP_FWD(4, false, G);                   \
    default: XP_FWD(5, false, G);            \
  }
  if constexpr (GEN) {
    if (net_is_general(nd)) {
      XP_SWITCH(true)
    }
  }
  XP_SWITCH(false)
#undef XP_SWITCH
#undef XP_FWD
}

template <int PT, bool GEN>
__device__ uint32_t backward_any(int K, bool lap, SmemLayout sl, const NetDev& nd, const float* prm,
                                 const float* img, int P, const float* S, int uoff, float* g, bool first,
                                 uint32_t ph, int* err, int net, int hl) {
#define XP_BWD(KK, L, G) return net_backward<KK, L, PT, G>(sl, nd, prm, img, P, S, uoff, g, first, ph, err, net, hl)
#define XP_SWITCH(G)                         \
  switch (K) {                               \
    case 1: XP_BWD(1, false, G);             \
    case 2: XP_BWD(2, false, G);             \
    case 3: XP_BWD(3, false, G);             \
    case 4:                                  \
      if (lap) XP_BWD(4, true, G);           \
      XP_BWD(4, false, G);                   \
    default: XP_BWD(5, false, G);            \
  }
  if constexpr (GEN) {
    if (net_is_general(nd)) {
      XP_SWITCH(true)
    }
  }
  XP_SWITCH(false)
#undef XP_SWITCH
#undef XP_BWD
}

// Jets of point p from U into J (components beyond a net's K stay 0).
__device__ __forceinline__ void load_point_jets(const SubDev& sd, const Item& it, const float* U,
                                                int u1, int P, int p, PtJets& J) {
#pragma unroll
  for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
    for (int c = 0; c < KMAX; ++c) J.u[o][c] = 0.f;
#pragma unroll
  for (int c = 0; c < KMAX; ++c) J.k[c] = 0.f;
  const int K0 = it.K[0], K1 = it.K[1];
  const int D0 = sd.net[0].w[sd.net[0].L];
  if (K0) {
#pragma unroll
    for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
      for (int c = 0; c < KMAX; ++c)
        if (o < D0 && c < K0) J.u[o][c] = U[(o * P + p) * K0 + c];
  }
  if (K1) {
#pragma unroll
    for (int c = 0; c < KMAX; ++c)
      if (c < K1) J.k[c] = U[u1 + p * K1 + c];
  }
}

__device__ __forceinline__ void store_point_seeds(const SubDev& sd, const Item& it, float* Ub, int u1,
                                                  int P, int p, const PtJets& G) {
  const int K0 = it.K[0], K1 = it.K[1];
  const int D0 = sd.net[0].w[sd.net[0].L];
  if (K0) {
#pragma unroll
    for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
      for (int c = 0; c < KMAX; ++c)
        if (o < D0 && c < K0) Ub[(o * P + p) * K0 + c] = G.u[o][c];
  }
  if (K1) {
#pragma unroll
    for (int c = 0; c < KMAX; ++c)
      if (c < K1) Ub[u1 + p * K1 + c] = G.k[c];
  }
}

// Loss terms and seeds of one point (see the kind of item).  Returns the
// point's contributions to the item's two loss sums in l0, l1.
__device__ __forceinline__ void point_stage(const StepArgs& a, const SubDev& sd, const Item& it,
                                            const IfaceDev* ifc, const PtJets& J, PtJets& G, bool valid,
                                            int64_t gp, int64_t ip, double& l0, double& l1) {
  const int D0 = sd.net[0].w[sd.net[0].L];
  switch (it.kind) {
    case IT_RES: {
      float r[3] = {0.f, 0.f, 0.f};
      const float f = valid ? a.res_f[gp] : 0.f;
      const int ne = residual_fwd(a.pde, J, f, a.nu, a.re, r);
      float sq = 0.f, e[3] = {0.f, 0.f, 0.f};
      const float coef = 2.f * sd.w_res * sd.inv_n_res;
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (q < ne) {
          sq += r[q] * r[q];
          e[q] = valid ? coef * r[q] : 0.f;
        }
      if (valid) l0 += (double)sq * sd.inv_n_res;
      residual_seed(a.pde, J, e, a.nu, a.re, G);
      break;
    }
    case IT_DATA0: {
      const float* tg = a.tgt + sd.tgt_off[0] + (gp - sd.data_off[0]) * D0;
      const float coef = 2.f * sd.w_data[0] * sd.inv_n_data[0];
      float sq = 0.f;
#pragma unroll
      for (int o = 0; o < XPINN_MAX_OUT; ++o)
        if (o < D0) {
          const float d = valid ? J.u[o][0] - tg[o] : 0.f;
          sq += d * d;
          G.u[o][0] = coef * d;
        }
      if (valid) l0 += (double)sq * sd.inv_n_data[0];
      break;
    }
    case IT_DATA1: {
      const float* tg = a.tgt + sd.tgt_off[1] + (gp - sd.data_off[1]);
      const float coef = 2.f * sd.w_data[1] * sd.inv_n_data[1];
      const float d = valid ? J.k[0] - tg[0] : 0.f;
      G.k[0] = coef * d;
      if (valid) l0 += (double)(d * d) * sd.inv_n_data[1];
      break;
    }
    case IT_IFACE:
    case IT_IFACE_FWD: {
      // solution vector (all outputs of all nets) and exchanged quantity
      float uv[XPINN_MAX_OUT + 1] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int o = 0; o < XPINN_MAX_OUT; ++o)
        if (o < D0) uv[o] = J.u[o][0];
      const int nu_ = D0 + (sd.n_nets > 1 ? 1 : 0);
      if (sd.n_nets > 1) uv[D0] = J.k[0];
      float qv[3] = {0.f, 0.f, 0.f};
      const int nq = ifc->method == XPINN_CPINN
                         ? flux_fwd(a.pde, J, ifc->nx, ifc->ny, a.nu, a.re, a.flux_mode, qv)
                         : residual_fwd(a.pde, J, 0.f, a.nu, a.re, qv);
      if (it.kind == IT_IFACE_FWD) {
        if (valid) {
          float* d = a.d4 + (ip * 2 + it.side) * a.d4_nv;
#pragma unroll
          for (int v = 0; v < XPINN_MAX_OUT + 1; ++v)
            if (v < nu_) d[v] = uv[v];
#pragma unroll
          for (int v = 0; v < 3; ++v)
            if (v < nq) d[nu_ + v] = qv[v];
        }
        break;
      }
      const float* dsrc = a.d4 + (ip * 2 + (1 - it.side)) * a.d4_nv;
      float d[XPINN_MAX_OUT + 1 + 3];
#pragma unroll
      for (int v = 0; v < XPINN_MAX_OUT + 1 + 3; ++v)
        d[v] = v < a.d4_nv ? __ldcg(dsrc + v) : 0.f;   // written by other CTAs in this launch
      float sa = 0.f, sf = 0.f;
      const float ca = sd.w_avg * ifc->inv_n;          // d/du of W_I/N ((u-u')/2)^2
      const float cf = 2.f * sd.w_iface * ifc->inv_n;
#pragma unroll
      for (int o = 0; o < XPINN_MAX_OUT; ++o)
        if (o < D0) {
          const float dd = valid ? 0.5f * (uv[o] - d[o]) : 0.f;
          sa += dd * dd;
          G.u[o][0] += ca * dd;
        }
      if (sd.n_nets > 1) {
        const float dd = valid ? 0.5f * (uv[D0] - d[D0]) : 0.f;
        sa += dd * dd;
        G.k[0] += ca * dd;
      }
      float e[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (q < nq) {
          const float dd = valid ? qv[q] - d[nu_ + q] : 0.f;
          sf += dd * dd;
          e[q] = cf * dd;
        }
      if (ifc->method == XPINN_CPINN)
        flux_seed(a.pde, J, ifc->nx, ifc->ny, a.nu, a.re, a.flux_mode, e, G);
      else
        residual_seed(a.pde, J, e, a.nu, a.re, G);
      if (valid) {
        l0 += (double)sa * ifc->inv_n;
        l1 += (double)sf * ifc->inv_n;
      }
      break;
    }
    default:
      break;
  }
}

// Wait (thread 0) until `need` exchange items have completed.  Every exchange
// item is claimed before any item that waits, and exchange items never wait,
// so the wait ends; it is still bounded: after about 1 s it sets the error
// flag and returns false; the item then completes on whatever the exchange
// buffer holds, and the call reports XPINN_ERR_TIMEOUT.
static __device__ bool wait_exchange(const StepArgs& a) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned ns = 32;
    for (long it = 0; atomicAdd(a.fwd_done, 0) < a.n_fwd_wait; ++it) {
      if (it > (1l << 20) || atomicAdd(a.err, 0) == XPINN_ERR_TIMEOUT) {   // gave up here or elsewhere
        atomicCAS(a.err, 0, XPINN_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int PT, bool GEN>
__device__ uint32_t process_item(const StepArgs& a, SmemLayout sl, const Item& it, int item_idx,
                                 float* __restrict__ scratch, uint32_t ph, bool wait_x) {
  const Smem s = carve(sl);
  const SubDev& sd = a.subs[it.q];
  const int P = it.P;
  const float* prm = a.params + sd.poff;
  const float* img = a.wimg + sd.img_off;
  const int tid = threadIdx.x;
  const bool has_bwd = it.kind <= IT_IFACE;
  // offsets of net 1 in U and in the scratch (net 0 starts at 0)
  int u1 = 0;
  int64_t s1 = 0;
  if (it.K[0]) {
    const NetDev& nd = sd.net[0];
    u1 = nd.w[nd.L] * it.K[0] * P;
    int64_t rows = 0;
    for (int k = 1; k < nd.L; ++k) rows += nd.wp[k];
    s1 = (rows + nd.w[nd.L]) * it.K[0] * P;
  }
  const IfaceDev* ifc = (it.kind == IT_IFACE || it.kind == IT_IFACE_FWD) ? &a.ifaces[it.edge] : nullptr;
  double l0 = 0.0, l1 = 0.0;
  for (int t0 = 0; t0 < it.n_pts; t0 += P) {
    const int nv = min(P, it.n_pts - t0);
    const bool first = t0 == 0;
    const float2* src = (it.kind == IT_EVAL) ? a.eval_pts : a.pts;
    for (int p = tid; p < P; p += blockDim.x) {
      float2 z = make_float2(0.f, 0.f);
      if (p < nv) z = src[it.pt_off + t0 + p];
      s.sx[p] = z.x;
      s.sy[p] = z.y;
    }
    __syncthreads();
    // net 1 first, so that the network whose reverse pass comes first is the
    // one whose last hidden activations are still in shared memory
    if (it.K[1]) ph = forward_any<PT, GEN>(it.K[1], false, sl, sd.net[1], prm, img, P, scratch + s1, u1, ph, a.err);
    if (it.K[0]) ph = forward_any<PT, GEN>(it.K[0], it.lap != 0, sl, sd.net[0], prm, img, P, scratch, 0, ph, a.err);
    // interface items read the neighbours' values from the exchange buffer:
    // wait for the exchange items only now, after the first forward pass,
    // which does not need them
    if (wait_x && first) wait_exchange(a);
    // ---- per point: loss terms and seeds (or exchange / evaluation output)
    for (int p = tid; p < P; p += blockDim.x) {
      const bool valid = p < nv;
      PtJets J, G;
      load_point_jets(sd, it, s.U, u1, P, p, J);
      if (it.kind == IT_EVAL) {
        if (valid) {
          float* out = a.eval_out + it.out_off + (int64_t)(t0 + p) * a.eval_dout;
          const float sc = a.eval_scale ? a.eval_scale[it.pt_off + t0 + p] : 1.f;
          const int K0 = it.K[0], K1 = it.K[1];
          const int D0 = sd.net[0].w[sd.net[0].L];
          int col = 0;
          if (K0) {
#pragma unroll
            for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
              for (int c = 0; c < KMAX; ++c)
                if (o < D0 && c < K0) out[col++] = sc * J.u[o][c];
          }
          if (K1) {
#pragma unroll
            for (int c = 0; c < KMAX; ++c)
              if (c < K1) out[col++] = sc * J.k[c];
          }
        }
        continue;
      }
#pragma unroll
      for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
        for (int c = 0; c < KMAX; ++c) G.u[o][c] = 0.f;
#pragma unroll
      for (int c = 0; c < KMAX; ++c) G.k[c] = 0.f;
      const int64_t gp = it.pt_off + t0 + p;   // global point index
      const int64_t ip = ifc ? ifc->d4_pt + (it.pt_off - ifc->pt_off) + t0 + p : 0;
      point_stage(a, sd, it, ifc, J, G, valid, gp, ip, l0, l1);
      if (has_bwd) store_point_seeds(sd, it, s.Ub, u1, P, p, G);
    }
    __syncthreads();
    if (has_bwd) {
      float* gs = a.partials + it.part_off;
      // buffer holding the last forward pass's H^{L-1}: A after an even number
      // of hidden-to-hidden layers, B after an odd one
      const int n_last = it.K[0] ? 0 : 1;
      const int hl_last = (sd.net[n_last].L - 2) & 1;
      if (it.K[0])
        ph = backward_any<PT, GEN>(it.K[0], it.lap != 0, sl, sd.net[0], prm, img, P, scratch, 0, gs, first, ph,
                                   a.err, 0, hl_last);
      if (it.K[1])
        ph = backward_any<PT, GEN>(it.K[1], false, sl, sd.net[1], prm, img, P, scratch + s1, u1, gs, first, ph,
                                   a.err, 1, n_last == 1 ? hl_last : -1);
      // a net that is not evaluated by this item contributes zero gradient
      if (first)
        for (int n = 0; n < sd.n_nets; ++n)
          if (!it.K[n]) {
            const NetDev& nd = sd.net[n];
            for (int e = nd.off[1] + tid; e < nd.end; e += blockDim.x) gs[e] = 0.f;
          }
    }
    // no barrier here: the reverse pass ends with one (after its last reads
    // of sx, sy and the buffers), and without it the barrier after the loss
    // stage is the last use of shared memory in this sub-tile
  }
  if (GEN && has_bwd) {
    // slope gradients of the item: the warps' partials in warp order, stored once
    // (the last sub-tile ended with a barrier, so every warp's partial is visible)
    float* gsl = a.partials + it.part_off;
    const int n_warps = (int)(blockDim.x >> 5);
    for (int n = 0; n < sd.n_nets; ++n) {
      const NetDev& nd = sd.net[n];
      if (!it.K[n] || nd.aoff < 0) continue;
      for (int t = tid; t < nd.L - 1; t += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < n_warps; ++w) sum += s.slope[(n * SLOPE_WARPS + w) * MAXL + t];
        gsl[nd.aoff + t] = nd.scale * (float)sum;
      }
    }
  }
  if (has_bwd) {
    const double t0s = block_sum(l0, s.red);
    const double t1s = block_sum(l1, s.red);
    if (tid == 0) {
      a.loss_part[2 * item_idx] = t0s;
      a.loss_part[2 * item_idx + 1] = t1s;
    }
  }
  return ph;
}

// PT = 1 keeps registers <= 128 so that two 256-thread CTAs fit on an SM;
// PT = 2 uses a larger register tile.  NTH = 128 halves the CTA so that two
// (or four) independent CTAs share an SM and one CTA's narrow phases (first
// and output layers, loss, small reductions) overlap another's contractions.
// NTH = 512 with PT = 1 keeps the sub-tile of 256 x PT=2 with twice the warps.
// GEN = false: every network is a fixed-slope tanh network (the passes of
// the general activations are not in this kernel, so they cost it nothing).
template <int PT, int NTH, bool GEN>
__global__ void __launch_bounds__(NTH, NTH == 512 ? 1 : (PT == 1 ? 2 : 1) * (256 / NTH)) jet_step_kernel(StepArgs a) {
  // launched as a programmatic dependent: nothing is read or written before
  // the previous kernel on the stream has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const SmemLayout sl{a.szA, a.szW, a.szU, a.pmax, GEN ? 1 : 0};
  __shared__ int s_item;
  float* scratch = a.scratch + (int64_t)blockIdx.x * a.scratch_per_cta;
  uint32_t ph = 0;   // phase parities of the two weight-buffer mbarriers
  const int n_items = a.n_items_dev ? min(a.n_items, *a.n_items_dev) : a.n_items;
  if (threadIdx.x == 0) {
    const Smem s = carve(sl);
    mbar_init(s.bar, 1);
    mbar_init(s.bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    const bool wait_x = a.n_fwd_wait > 0 && it >= a.wait_from;
    const Item& item = a.items[it];
    ph = process_item<PT, GEN>(a, sl, item, a.item_base + it, scratch, ph, wait_x);
    if (item.kind == IT_IFACE_FWD && a.n_fwd_wait > 0) {
      __syncthreads();                      // every thread's exchange stores issued
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.fwd_done, 1);
      }
    }
  }
}

}  // namespace xp
