// Residual items of the training step on the 5th-generation tensor cores
// (tcgen05, sm_103a).
//
// For an item (a range of residual points of one subdomain whose network
// step_tc.h admits) the kernel computes what the FP32 jet kernel computes for
// it: the Taylor jets of the network (Sec. 3) at the points, the PDE
// residual term of Eq. cPINNLoss / Eq. XPINNLoss (Sec. 4.2) and its gradient
// with respect to every weight and bias, written to the item's gradient
// slice, and the item's loss sum.  The three point-by-width contractions of
// every hidden-to-hidden layer k run on the tensor cores:
//   forward    Z^k  = H^{k-1} (W^k)^T           [128 rows x 64] . [64 x 64]
//   reverse    Hb^{k-1} = Zb^k W^k              [128 rows x 64] . [64 x 64]
//   gradient   dW^k += (Zb^k)^T H^{k-1}         [64 x 128 rows] . [128 rows x 64]
// The first layer (two inputs) and the output layer (at most three outputs),
// their weight gradients included (sums over a warp's points by shuffles,
// accumulated over the item in shared memory), the jet rules and the
// residual stay on the FP32 pipes.
//
// Tile: 128 rows = the MMA's M, 32 points x 4 jet components (u, u_x, u_y,
// lap u), row 4 p + c.  16 compute warps take two roles.  As row threads (four per
// row: warps w, w + 4, w + 8, w + 12 read the same tensor-memory lanes, 16 of
// the 64 neurons each) they move accumulator rows out of tensor memory into a
// staging array [point][component][neuron].  As point threads (lane = point,
// warp = a group of 4 neurons) they apply the jet rule to all four components
// of a point at once, in registers -- for fixed-slope tanh
//   h = t,  h_i = s z_i,  h_lap = s z_lap - 2 t s (z_x^2 + z_y^2),  t = tanh z,
// s = 1 - t^2, for tanh, sin or cos with a slope the jet kernel's general rule
// -- and its reverse, and write the MMA operand images: 4 rows of one neuron
// are one 16-byte run in every image, transposed or not.  The activation is
// evaluated once per (point, neuron) and pass.  The pre-activation jets (t,
// z_x, z_y, z_lap for tanh; z for the general rule) go to per-CTA scratch in
// global memory (L2-resident) for the reverse pass, which rebuilds H^{k-1}
// from them.
//
// Precision: every contraction takes three TF32 products over hi/lo splits
// of both operands (hi = rna(x), lo = rna(x - hi); the dropped lo x lo term
// is below 2^-22 of a product).  Forward and reverse accumulate hi x hi and
// the cross terms in separate tensor-memory accumulators (summed when read).
// The gradient contraction stacks the hi and lo parts of Zb^T as the MMA's
// 128 M-rows (0-63 hi, 64-127 lo) and issues two MMAs, B = H_hi and B = H_lo:
// lanes 0-63 accumulate hi.H_hi + hi.H_lo, lanes 64-127 lo.H_hi + lo.H_lo,
// and dW^k is their sum (all four products at the MMA's full M = 128).  The
// dW^k accumulators stay in tensor memory over 16 tiles and are then added
// into the item's gradient slice in FP32: a single accumulator over the
// whole item (about 80 tiles) erred up to 1.04e-4 of the largest gradient
// element on the full-size Navier-Stokes workload.
//
// A 17th warp issues the MMAs (one thread) and the weight copies.  Issuing
// an MMA stalls the issuing thread for about as long as the tensor core
// takes to run the one before it, so a compute warp that issued the 32 MMAs
// of a weight gradient would hold every later barrier of the tile for their
// whole duration; from the MMA warp they run while the compute warps move on
// to the next layer's reverse rule.  The compute warps hand over each
// operand set with one arrival per warp on an mbarrier (after a proxy fence)
// and synchronise among themselves on a named barrier that the MMA warp
// does not join; the MMA warp follows the same fixed sequence of MMA groups
// per tile, so their order, and the gradient, do not depend on timing.
//
// Operands are K-major, no swizzle.  Images whose K is the tile's rows pad
// every K-step of core matrices by 16 bytes.  Weight images (forward and
// reverse, built by pack_tc_train_kernel) arrive by bulk copy into one buffer,
// the next image's copy issued as soon as an MMA has released it (it lands
// during the epilogue; the first image of the next tile during the reverse
// pass's last layers).  Every wait is bounded; a wait that gives up sets the
// error word, the launch stops taking items, frees its tensor memory and ends.
#include <cuda_runtime.h>

#include "jet_step.cuh"
#include "step_tc.h"
#include "tc_util.cuh"

namespace xp {

namespace {

constexpr int NPT = 16;                  // neurons of a row thread (of the 64)
constexpr int NCW = 16;                  // compute warps: row threads and point threads
constexpr int NTC = 32 * NCW;            // compute threads (four row threads per row)
constexpr int NTH = NTC + 32;            // and one warp that issues the MMAs and the weight copies
static_assert(NTC == 128 * (STC_W / NPT), "four row threads per row");
constexpr int NPG = 4;                   // neurons of a point thread
constexpr int ROWS = 128;
constexpr unsigned FULL = 0xffffffffu;
// K-major images whose K is the tile's rows: floats between K-adjacent core
// matrices, padded by 16 bytes (conflict-free 16-byte stores across points)
constexpr int LB_B = 8 * 32 + 4;    // B' = H^T [N = 64][K = rows]: 1040 bytes
constexpr int LB_T = 16 * 32 + 4;   // At = stacked Zb^T [M = 128][K = rows]: 2064 bytes
constexpr int SZ_B = 32 * LB_B;     // one B' image (hi or lo)
constexpr int SZ_T = 32 * LB_T;
// the row-major A image [128 rows][64 neurons] (K = neuron): core matrices of
// 8 rows x 4 neurons, 8-row groups 144 bytes apart (padded by 16 bytes, so
// that the 16-byte runs of 8 points' rows fall in distinct bank groups),
// 4-neuron groups 16 x 144 bytes apart
constexpr int A_SBO = 144, A_LBO = 16 * A_SBO;
constexpr int SZ_AF = 16 * A_LBO / 4;   // one A image (hi or lo), floats
constexpr int SZ_RA = 2 * SZ_AF;        // region A: A (hi | lo), or B' (hi | lo)
static_assert(2 * SZ_B <= SZ_RA, "region A holds B'");
// region A also holds, between the forward and the reverse pass, the partial
// outputs [4 parts][128 rows][4] and the output jets [32 points][3][4]
constexpr int RA_X = 0, RA_J = RA_X + 4 * ROWS * 4;
static_assert(RA_J + 384 <= SZ_RA && 2 * 64 * 65 <= SZ_RA, "region A");
// staging [point][component][neuron]: component stride 72, point stride 292
// floats, so that a point thread's 16-byte loads (8 points) and a row
// thread's 16-byte stores (8 rows) each fall in distinct bank groups
constexpr int ZS_C = 72, ZS_P = 4 * ZS_C + 4;
constexpr int SZ_ZS = 32 * ZS_P;
// the item's FP32-pipe weights, zero-padded to 64 neurons: W^1 [64][2], b^1,
// b^k (k = 2..L-1) [STC_MAXL - 2][64], W^L [3][64], b^L [4]
constexpr int PW_W1 = 0, PW_B1 = 128, PW_BK = 192, PW_WL = PW_BK + 64 * (STC_MAXL - 2), PW_BL = PW_WL + 192;
constexpr int SZ_PW = PW_BL + 4;
// shared-memory map (floats): region A, At, the weight buffer, the staging
// array, the points of two tiles, the bias-gradient sums [STC_MAXL - 2][64]
// and [32 points][4], the FP32-pipe weights, the slope-gradient sums, the
// output seeds, the first and output layers' weight-gradient sums
constexpr int O_A = 0;
constexpr int O_T = O_A + SZ_RA;
constexpr int O_W = O_T + SZ_T;
constexpr int O_Z = O_W + STC_IMG;
constexpr int O_P = O_Z + SZ_ZS;
constexpr int O_DB = O_P + 128;
constexpr int O_DL = O_DB + (STC_MAXL - 2) * 64;
constexpr int O_PW = O_DL + 128;
constexpr int O_SL = O_PW + SZ_PW;                   // slope-gradient sums [STC_MAXL - 1][16 warps]
constexpr int O_G = O_SL + (STC_MAXL - 1) * 16;      // output seeds [32 points][3][4]
constexpr int O_D1 = O_G + 384;                      // dW^1 | db^1 sums [64][3]
constexpr int O_DLW = O_D1 + 192;                    // dW^L sums [3][64]
constexpr int SMEM_FLOATS = O_DLW + 192;
// tensor-memory columns: Z main [0, 64), Z cross [64, 128), dW^k (k = 2..L-1)
// at 128 + 64 (k - 2)
constexpr int TMEM_COLS = 512;
// tiles a weight-gradient accumulator sums before it is added into the
// item's slice (bounds the length of each tensor-memory accumulation)
constexpr int STC_FLUSH = 16;
static_assert(128 + 64 * (STC_MAXL - 2) <= TMEM_COLS, "tensor memory");

// element offsets in the images whose K is the rows (column n, row r); the 4
// rows of a point (r = 4 p + c) are one 16-byte run
__device__ __forceinline__ int a_off5(int r, int g) { return g * (A_LBO / 4) + (r >> 3) * (A_SBO / 4) + (r & 7) * 4; }
__device__ __forceinline__ int t_off(int m, int r) { return (m >> 3) * 32 + (r >> 2) * LB_T + (m & 7) * 4 + (r & 3); }
__device__ __forceinline__ int b_off(int j, int r) { return (j >> 3) * 32 + (r >> 2) * LB_B + (j & 7) * 4 + (r & 3); }

__device__ __forceinline__ void fence_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// barrier of the compute warps (the MMA warp does not take part)
__device__ __forceinline__ void csync() { asm volatile("bar.sync 1, %0;" ::"n"(NTC) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A compute warp has written its part of the next MMA's operands: its
// writes are made visible to the tensor core, then the warp arrives (once)
// on the operand barrier, which completes when all NCW warps have.
__device__ __forceinline__ void operands_ready(uint64_t* bar, int lane) {
  fence_to_async();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
}

// sum over the compute threads (thread 0 gets it)
__device__ __forceinline__ double compute_sum(double v, double* red, int warp, int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  csync();
  if (lane == 0) red[warp] = v;
  csync();
  double t = 0.0;
  if (warp == 0 && lane == 0)
    for (int w = 0; w < NCW; ++w) t += red[w];
  return t;
}

// mbar_wait with a suspend-time hint: a warp that finds the phase
// incomplete is parked in the barrier until the phase completes (or the hint
// of 10 ms runs out) instead of polling, so that waiting warps take no issue
// slots from working ones.  Bounded like mbar_wait: about a second, then the
// error word holds XPINN_ERR_TIMEOUT.
__device__ __forceinline__ void mbar_park(uint64_t* bar, uint32_t parity, int* err) {
  const long long t0 = clock64();
  long long limit = 0;
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(10000000u)
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

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Descriptors of successive K-steps differ only in the start address (bits
// 0-13, in 16-byte units): each MMA adds its step's offset to a base
// descriptor built once per call, so that issuing a layer's MMAs costs few
// instructions on the issuing thread.
__device__ __forceinline__ uint64_t dstep(int bytes) { return (uint64_t)(bytes >> 4); }

// Z (+)= A . B over K = 64: A the row-major image at a (hi, then lo), read
// K-major; B a weight image at b (hi, then lo); hi x hi into tm, the cross
// terms into tm + 64.  The hi and lo halves of a weight image are one
// operand of N = 128 (their 8-row groups continue at the same stride), so a
// single MMA takes A_hi against both: the A tile is read from shared memory
// twice per K-step instead of three times (the MMAs of this kernel are
// bound by shared-memory reads: 6 KB of operands per N = 64 MMA).
__device__ __forceinline__ void mma_rows(uint32_t tm, uint32_t a, uint32_t b) {
  const uint32_t id2 = tc_idesc(2 * STC_W), id = tc_idesc(STC_W);
  const uint64_t ahi = tc_sdesc(a, A_LBO, A_SBO), alo = tc_sdesc(a + 4 * SZ_AF, A_LBO, A_SBO);
  const uint64_t bhl = tc_sdesc(b, 128, STC_W / 4 * 128);   // hi rows 0-63, lo rows 64-127
#pragma unroll
  for (int ks = 0; ks < STC_W / 8; ++ks) {
    const uint64_t da = dstep(ks * 2 * A_LBO), db = dstep(ks * 256);
    tc_mma(tm, ahi + da, bhl + db, id2, ks > 0 ? 1u : 0u);
    tc_mma(tm + 64, alo + da, bhl + db, id, 1u);
  }
}

// D (+)= At . B over K = 128 rows: At the stacked image at t, B an [N][rows]
// image at b (hi) and b + lo_bytes (lo) with LB bytes between K-adjacent core
// matrices; N = n.  first: the accumulator starts at zero.
template <int LB>
__device__ __forceinline__ void mma_grad(uint32_t tm, uint32_t t, uint32_t b, uint32_t lo_bytes, int n, bool first) {
  const uint32_t id = tc_idesc(n);
  const uint64_t at = tc_sdesc(t, LB_T * 4, 128);
  const uint64_t bh = tc_sdesc(b, LB, 128), bl = tc_sdesc(b + lo_bytes, LB, 128);
#pragma unroll
  for (int ks = 0; ks < ROWS / 8; ++ks) {
    const uint64_t dt = dstep(ks * 2 * LB_T * 4), db = dstep(ks * 2 * LB);
    tc_mma(tm, at + dt, bh + db, id, (first && ks == 0) ? 0u : 1u);
    tc_mma(tm, at + dt, bl + db, id, 1u);
  }
}

// NPT columns of this thread's lane: main + cross accumulators
__device__ __forceinline__ void tmem_rowz(uint32_t main, uint32_t cross, float (&z)[NPT]) {
  uint32_t v[NPT], u[NPT];
#pragma unroll
  for (int c0 = 0; c0 < NPT; c0 += 16) {
    tmem_ld16(main + c0, v + c0);
    tmem_ld16(cross + c0, u + c0);
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c0 = 0; c0 < NPT; c0 += 8) {
    tmem_fence_regs8(v + c0);
    tmem_fence_regs8(u + c0);
  }
#pragma unroll
  for (int i = 0; i < NPT; ++i) z[i] = __uint_as_float(v[i]) + __uint_as_float(u[i]);
}

// N columns (a multiple of 16) of this thread's lane of one accumulator
template <int N>
__device__ __forceinline__ void tmem_cols(uint32_t taddr, float (&z)[N]) {
  uint32_t v[N];
#pragma unroll
  for (int c0 = 0; c0 < N; c0 += 16) tmem_ld16(taddr + c0, v + c0);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c0 = 0; c0 < N; c0 += 8) tmem_fence_regs8(v + c0);
#pragma unroll
  for (int i = 0; i < N; ++i) z[i] = __uint_as_float(v[i]);
}

// ---------------------------------------------------------------------------
// Point threads: lane p = point, warp g = neurons 4 g .. 4 g + 3.  v[c][i] is
// component c (0 value, 1 x, 2 y, 3 Laplacian) of neuron 4 g + i; row 4 p + c.
// ---------------------------------------------------------------------------

// Forward rule from the pre-activation jets z (the value's includes the
// bias): h, and the saved jets sv = (t, z_x, z_y, z_lap) of every neuron.
__device__ __forceinline__ void jet4_fwd(const float (&z)[4][NPG], float (&h)[4][NPG], float (&sv)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float t = tanhf(z[0][i]), s = 1.f - t * t;
    const float q = z[1][i] * z[1][i] + z[2][i] * z[2][i];
    h[0][i] = t;
    h[1][i] = s * z[1][i];
    h[2][i] = s * z[2][i];
    h[3][i] = s * z[3][i] - 2.f * t * s * q;
    sv[0][i] = t;
    sv[1][i] = z[1][i];
    sv[2][i] = z[2][i];
    sv[3][i] = z[3][i];
  }
}

// The same from saved jets (no tanh)
__device__ __forceinline__ void jet4_saved(const float (&sv)[4][NPG], float (&h)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float t = sv[0][i], s = 1.f - t * t;
    const float q = sv[1][i] * sv[1][i] + sv[2][i] * sv[2][i];
    h[0][i] = t;
    h[1][i] = s * sv[1][i];
    h[2][i] = s * sv[2][i];
    h[3][i] = s * sv[3][i] - 2.f * t * s * q;
  }
}

// Reverse rule: adjoints hb of (h, h_x, h_y, h_lap) to adjoints zb of
// (z, z_x, z_y, z_lap):
//   zb_lap = s hb_lap,  zb_i = s hb_i - 4 t s z_i hb_lap,
//   zb = s [hb - 2 t (z_x hb_x + z_y hb_y) + (-2 t z_lap + (6 t^2 - 2)(z_x^2 + z_y^2)) hb_lap]
__device__ __forceinline__ void jet4_bwd(const float (&sv)[4][NPG], const float (&hb)[4][NPG],
                                         float (&zb)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float t = sv[0][i], z1 = sv[1][i], z2 = sv[2][i], z3 = sv[3][i], s = 1.f - t * t;
    const float h3 = hb[3][i];
    zb[3][i] = s * h3;
    zb[1][i] = s * hb[1][i] - 4.f * t * s * z1 * h3;
    zb[2][i] = s * hb[2][i] - 4.f * t * s * z2 * h3;
    float tb = hb[0][i] - 2.f * t * (z1 * hb[1][i] + z2 * hb[2][i]);
    tb += (-2.f * t * z3 + (6.f * t * t - 2.f) * (z1 * z1 + z2 * z2)) * h3;
    zb[0][i] = s * tb;
  }
}

// The operand images take the hi/lo split of a thread's 16 values, formed
// as they are stored (no split copy stays live in registers).
__device__ __forceinline__ void split_store(float* __restrict__ hi_at, float* __restrict__ lo_at, float a, float b,
                                            float c, float d) {
  const float2 sa = tf32_split(a), sb = tf32_split(b), sc = tf32_split(c), sd = tf32_split(d);
  *reinterpret_cast<float4*>(hi_at) = make_float4(sa.x, sb.x, sc.x, sd.x);
  *reinterpret_cast<float4*>(lo_at) = make_float4(sa.y, sb.y, sc.y, sd.y);
}

// Row-major A image (hi at A, lo at A + SZ_AF): per row, the 4 neurons
__device__ __forceinline__ void put_a(float* __restrict__ A, int p, int g, const float (&x)[4][NPG]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int o = a_off5(4 * p + c, g);
    split_store(A + o, A + SZ_AF + o, x[c][0], x[c][1], x[c][2], x[c][3]);
  }
}

// Stacked transposed image (M-row n: hi, 64 + n: lo): per neuron, the 4 rows
__device__ __forceinline__ void put_t(float* __restrict__ T, int p, int g, const float (&x)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const int n = 4 * g + i;
    split_store(T + t_off(n, 4 * p), T + t_off(64 + n, 4 * p), x[0][i], x[1][i], x[2][i], x[3][i]);
  }
}

// Transposed B' image (hi at B, lo at B + SZ_B): per neuron, the 4 rows
__device__ __forceinline__ void put_b(float* __restrict__ B, int p, int g, const float (&x)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const int o = b_off(4 * g + i, 4 * p);
    split_store(B + o, B + SZ_B + o, x[0][i], x[1][i], x[2][i], x[3][i]);
  }
}

// Saved jets of one layer, [neuron][row] (Sk at the layer's first float):
// the 4 rows of a point are (t, z_x, z_y, z_lap), one 16-byte run
__device__ __forceinline__ void save4(float* __restrict__ Sk, int p, int g, const float (&sv)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i)
    *reinterpret_cast<float4*>(Sk + (4 * g + i) * ROWS + 4 * p) = make_float4(sv[0][i], sv[1][i], sv[2][i], sv[3][i]);
}

// (through L1: the reverse pass prefetches a layer's lines there an epilogue
// ahead of this load)
__device__ __forceinline__ void load4(const float* __restrict__ Sk, int p, int g, float (&sv)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float4 v = __ldca(reinterpret_cast<const float4*>(Sk + (4 * g + i) * ROWS + 4 * p));
    sv[0][i] = v.x;
    sv[1][i] = v.y;
    sv[2][i] = v.z;
    sv[3][i] = v.w;
  }
}

// Staging [point][component][neuron]: a point thread's 4 rows x 4 neurons
__device__ __forceinline__ void zs_read4(const float* __restrict__ ZS, int p, int g, float (&v)[4][NPG]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float4 x = *reinterpret_cast<const float4*>(ZS + p * ZS_P + c * ZS_C + 4 * g);
    v[c][0] = x.x;
    v[c][1] = x.y;
    v[c][2] = x.z;
    v[c][3] = x.w;
  }
}

__device__ __forceinline__ void zs_write4(float* __restrict__ ZS, int p, int g, const float (&v)[4][NPG]) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<float4*>(ZS + p * ZS_P + c * ZS_C + 4 * g) = make_float4(v[c][0], v[c][1], v[c][2], v[c][3]);
}

// ... and a row thread's row (r = 4 p + c), neurons nb .. nb + NPT - 1
__device__ __forceinline__ void zs_row_write(float* __restrict__ ZS, int r, int nb, const float (&z)[NPT]) {
  float* d = ZS + (r >> 2) * ZS_P + (r & 3) * ZS_C + nb;
#pragma unroll
  for (int j = 0; j < NPT; j += 4) *reinterpret_cast<float4*>(d + j) = make_float4(z[j], z[j + 1], z[j + 2], z[j + 3]);
}

__device__ __forceinline__ void zs_row_read(const float* __restrict__ ZS, int r, int nb, float (&z)[NPT]) {
  const float* d = ZS + (r >> 2) * ZS_P + (r & 3) * ZS_C + nb;
#pragma unroll
  for (int j = 0; j < NPT; j += 4) {
    const float4 x = *reinterpret_cast<const float4*>(d + j);
    z[j] = x.x;
    z[j + 1] = x.y;
    z[j + 2] = x.z;
    z[j + 3] = x.w;
  }
}

// The same for a general hidden activation h = Phi(s z) (tanh, sin or cos,
// slope s = n a^k), per neuron by the shared jet rules of the jet kernel;
// the saved jets are then the unscaled z, and the reverse rule adds
// dJ/ds = sum over components of vb_c z_c to gs.
__device__ __forceinline__ void jet4_fwd_gen(const Act& act, const float (&z)[4][NPG], float (&h)[4][NPG],
                                             float (&sv)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float zz[4] = {z[0][i], z[1][i], z[2][i], z[3][i]};
    float hh[4];
    phi_jet<4, true>(act, zz, hh);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      h[c][i] = hh[c];
      sv[c][i] = zz[c];
    }
  }
}

__device__ __forceinline__ void jet4_saved_gen(const Act& act, const float (&sv)[4][NPG], float (&h)[4][NPG]) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float zz[4] = {sv[0][i], sv[1][i], sv[2][i], sv[3][i]};
    float hh[4];
    phi_jet<4, true>(act, zz, hh);
#pragma unroll
    for (int c = 0; c < 4; ++c) h[c][i] = hh[c];
  }
}

__device__ __forceinline__ void jet4_bwd_gen(const Act& act, const float (&sv)[4][NPG], const float (&hb)[4][NPG],
                                             float (&zb)[4][NPG], float& gs) {
#pragma unroll
  for (int i = 0; i < NPG; ++i) {
    const float zz[4] = {sv[0][i], sv[1][i], sv[2][i], sv[3][i]};
    const float hh[4] = {hb[0][i], hb[1][i], hb[2][i], hb[3][i]};
    float zr[4];
    act_jet_bwd<4, true, true>(act, zz, hh, zr, gs);
#pragma unroll
    for (int c = 0; c < 4; ++c) zb[c][i] = zr[c];
  }
}

// Sums over the warp's 32 points of the value-row adjoints of the thread's 4
// neurons (fixed butterfly); lane 0 adds them to d[0..3]
__device__ __forceinline__ void value_sums(const float (&zb)[4][NPG], int lane, float* __restrict__ d) {
  float v[NPG];
#pragma unroll
  for (int i = 0; i < NPG; ++i) v[i] = zb[0][i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NPG; ++i) v[i] += __shfl_xor_sync(FULL, v[i], o);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NPG; ++i) d[i] += v[i];
  }
}

// The residual of one point from its output jets J[o][c] (o < D, c < 4:
// value, x, y, Laplacian), and the seeds G[o][c] = coef dr^2/dJ; returns the
// squared residual.  Not inlined: the 40 jet values it holds would raise the
// register peak of the whole kernel, and one warp runs it once per tile.
__device__ __noinline__ float point_residual(int pde, int D, const float* __restrict__ Jo, float* __restrict__ Go,
                                             float f, float coef, float nu, float re) {
  PtJets J, G;
#pragma unroll
  for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
    for (int cc = 0; cc < KMAX; ++cc) {
      J.u[o][cc] = (o < D && cc < 4) ? Jo[o * 4 + cc] : 0.f;
      G.u[o][cc] = 0.f;
    }
#pragma unroll
  for (int cc = 0; cc < KMAX; ++cc) J.k[cc] = G.k[cc] = 0.f;
  float rr[3] = {0.f, 0.f, 0.f};
  const int ne = residual_fwd(pde, J, f, nu, re, rr);
  float sq = 0.f, e[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (q < ne) {
      sq += rr[q] * rr[q];
      e[q] = coef * rr[q];
    }
  residual_seed(pde, J, e, nu, re, G);
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) Go[o * 4 + cc] = o < D ? G.u[o][cc] : 0.f;
  return sq;
}

// The output layer's weight gradient over the warp's 32 points: for the
// thread's 4 neurons m, sum over components c of yb[o][c] h[c][m] (yb the
// point's output seeds [3][4], h = H^{L-1}); fixed butterfly, lane 0 adds
// them to d[o * 64 + m]
__device__ __forceinline__ void out_grad_sums(const float (&h)[4][NPG], const float* __restrict__ yb, int lane,
                                              float* __restrict__ d) {
  float g[3][NPG];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const float4 y = *reinterpret_cast<const float4*>(yb + 4 * o);
#pragma unroll
    for (int m = 0; m < NPG; ++m) g[o][m] = fmaf(y.x, h[0][m], fmaf(y.y, h[1][m], fmaf(y.z, h[2][m], y.w * h[3][m])));
  }
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1)
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
      for (int m = 0; m < NPG; ++m) g[o][m] += __shfl_xor_sync(FULL, g[o][m], sh);
  if (lane == 0) {
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
      for (int m = 0; m < NPG; ++m) d[o * 64 + m] += g[o][m];
  }
}

// The first layer's weight and bias gradients over the warp's 32 points from
// the adjoints zb of z^1 = W^1 x + b^1 (value, x, y rows; the Laplacian row
// of z^1 is constant): dW^1[m] += (zb x + zb_x, zb y + zb_y), db^1[m] += zb;
// fixed butterfly, lane 0 adds them to d[3 m + 0..2]
__device__ __forceinline__ void in_grad_sums(const float (&zb)[4][NPG], float2 x, int lane, float* __restrict__ d) {
  float g[NPG][3];
#pragma unroll
  for (int m = 0; m < NPG; ++m) {
    g[m][0] = fmaf(zb[0][m], x.x, zb[1][m]);
    g[m][1] = fmaf(zb[0][m], x.y, zb[2][m]);
    g[m][2] = zb[0][m];
  }
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1)
#pragma unroll
    for (int m = 0; m < NPG; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) g[m][c] += __shfl_xor_sync(FULL, g[m][c], sh);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NPG; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) d[3 * m + c] += g[m][c];
  }
}

// GEN = false: every network is tanh with fixed slopes (saved t); true: any
// hidden activation and trained slopes (saved z, Phi evaluated again in the
// reverse pass, slope gradients summed per layer).
template <bool GEN>
__global__ void __launch_bounds__(NTH, 1) step_tc_kernel(StepTcArgs a) {
  extern __shared__ __align__(1024) float sm[];
  float* RA = sm + O_A;
  float* RT = sm + O_T;
  float* RW = sm + O_W;
  float* ZS = sm + O_Z;
  float* Xs = RA + RA_X;
  float* Js = RA + RA_J;
  float* Gs = sm + O_G;
  float* d1s = sm + O_D1;
  float* dlw = sm + O_DLW;
  float2* const sp2 = reinterpret_cast<float2*>(sm + O_P);   // points: this tile's and the next one's
  float* dbs = sm + O_DB;
  float* dls = sm + O_DL;
  float* pw = sm + O_PW;
  float* sls = sm + O_SL;
  __shared__ __align__(8) uint64_t bars[4];   // weight buffer, row MMAs, gradient MMAs, operands
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_stop;
  __shared__ double red[NCW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // row-thread view (tensor memory, the output layer)
  const int quad = warp & 3, part = warp >> 2, nb = part * NPT;
  const int r = quad * 32 + lane, pr = r >> 2, cr = r & 3;
  // point-thread view (jet rules, operand images)
  const int p = lane, g = warp;
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(bars + i, 1);
    mbar_init(bars + 3, NCW);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "n"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);   // this warp's lanes
  const uint32_t sa = smem_u32(RA), st = smem_u32(RT), sw = smem_u32(RW);
  float* const scr = a.scratch + (int64_t)blockIdx.x * STC_SCRATCH;
  uint32_t wph = 0, mph = 0, dph = 0, oph = 0;   // phase parities
  bool d_pending = false;               // a gradient-MMA commit not yet waited for
  for (;;) {
    if (tid == 0) {
      s_item = atomicAdd(a.counter, 1);
      s_stop = *reinterpret_cast<volatile int*>(a.err) == XPINN_ERR_TIMEOUT;
    }
    __syncthreads();
    const int ii = s_item;
    const bool stop = s_stop != 0;
    __syncthreads();
    if (ii >= a.n_items || stop) break;
    const Item it = a.items[ii];
    const SubDev& sd = a.subs[it.q];
    const NetDev& nd = sd.net[0];
    const int L = nd.L;
    const int64_t io = a.img_off[it.q];
    bool ok = it.kind == IT_RES && it.K[0] == 4 && it.K[1] == 0 && io >= 0 && L >= 3 && L <= STC_MAXL &&
              nd.w[0] == 2 && nd.w[L] >= 1 && nd.w[L] <= 3 && it.part_off >= 0;
    for (int k = 1; k < L && ok; ++k) ok = nd.w[k] >= 1 && nd.w[k] <= STC_W;
    if (!ok) {
      if (tid == 0) atomicCAS(a.err, 0, XPINN_ERR_INVALID);
      continue;
    }
    const float* prm = a.params + sd.poff;
    const float* img = a.img + io;
    const int D = nd.w[L], wl = nd.w[L - 1];
    const int nimg = 2 * (L - 2);   // images a tile uses: forward k = 2..L-1, then reverse k = L-1..2
    auto img_src = [&](int i) -> const float* {
      const int k = i < L - 2 ? i + 2 : 2 * L - 3 - i;
      return img + (int64_t)((i < L - 2 ? 0 : L - 2) + k - 2) * STC_IMG;
    };
    const float coef = 2.f * sd.w_res * sd.inv_n_res;
    const int n_tiles = (it.n_pts + STC_PTS - 1) / STC_PTS;
    if (warp == NCW) {
      // The MMA warp: one thread issues the item's MMAs in the order in
      // which the compute warps complete their operands, and the weight
      // copies, each as soon as the buffer is free.
      if (lane == 0 && n_tiles > 0) {
        bulk_g2s(RW, img_src(0), 4u * STC_IMG, bars);
        for (int tile = 0; tile < n_tiles; ++tile) {
          const bool first = tile % STC_FLUSH == 0;   // the gradient accumulators start from zero
          for (int k = 2; k <= L - 1; ++k) {            // Z^k = H^{k-1} (W^k)^T
            mbar_park(bars + 3, oph, a.err);
            oph ^= 1u;
            mbar_park(bars, wph, a.err);
            wph ^= 1u;
            after_sync();
            mma_rows(tmem, sa, sw);
            mma_commit(bars + 1);
            mbar_park(bars + 1, mph, a.err);
            mph ^= 1u;
            bulk_g2s(RW, img_src(k - 1), 4u * STC_IMG, bars);
          }
          for (int k = L - 1; k >= 2; --k) {
            mbar_park(bars + 3, oph, a.err);            // Hb^{k-1} = Zb^k W^k
            oph ^= 1u;
            mbar_park(bars, wph, a.err);
            wph ^= 1u;
            after_sync();
            mma_rows(tmem, sa, sw);
            mma_commit(bars + 1);
            mbar_park(bars + 1, mph, a.err);
            mph ^= 1u;
            const int i = (L - 2) + (L - 1 - k);
            if (i + 1 < nimg)
              bulk_g2s(RW, img_src(i + 1), 4u * STC_IMG, bars);
            else if (tile + 1 < n_tiles)
              bulk_g2s(RW, img_src(0), 4u * STC_IMG, bars);
            mbar_park(bars + 3, oph, a.err);            // dW^k: Zb^k and H^{k-1}
            oph ^= 1u;
            after_sync();
            mma_grad<4 * LB_B>(tmem + 128 + 64 * (k - 2), st, sa, 4u * SZ_B, STC_W, first);
            mma_commit(bars + 2);
          }
        }
      }
      __syncwarp();
      continue;
    }
    // the item's FP32-pipe weights, zero-padded (visible after the first tile's barrier)
    for (int e = tid; e < SZ_PW; e += NTC) {
      float v = 0.f;
      if (e < PW_B1) {
        const int n = e >> 1;
        if (n < nd.w[1]) v = prm[nd.off[1] + e];
      } else if (e < PW_BK) {
        const int n = e - PW_B1;
        if (n < nd.w[1]) v = prm[nd.off[1] + 2 * nd.w[1] + n];
      } else if (e < PW_WL) {
        const int k = 2 + (e - PW_BK) / 64, n = (e - PW_BK) % 64;
        if (k < L && n < nd.w[k]) v = prm[nd.off[k] + nd.w[k] * nd.w[k - 1] + n];
      } else if (e < PW_BL) {
        const int o = (e - PW_WL) / 64, n = (e - PW_WL) % 64;
        if (o < D && n < wl) v = prm[nd.off[L] + o * wl + n];
      } else if (e - PW_BL < D) {
        v = prm[nd.off[L] + D * wl + e - PW_BL];
      }
      pw[e] = v;
    }
    for (int e = tid; e < (STC_MAXL - 2) * 64; e += NTC) dbs[e] = 0.f;
    if (tid < 128) dls[tid] = 0.f;
    if (tid < (STC_MAXL - 1) * 16) sls[tid] = 0.f;
    if (tid < 192) {
      d1s[tid] = 0.f;
      dlw[tid] = 0.f;
    }
    double l0 = 0.0;
    if (tid < STC_PTS) sp2[tid] = tid < it.n_pts ? a.pts[it.pt_off + tid] : make_float2(0.f, 0.f);
    for (int tile = 0; tile < n_tiles; ++tile) {
      const int t0 = tile * STC_PTS;
      const int nv = min(STC_PTS, it.n_pts - t0);
      // every MMA of the previous tile has completed: regions A and At are free
      if (d_pending) {
        mbar_park(bars + 2, dph, a.err);
        dph ^= 1u;
        d_pending = false;
      }
      const float2* sp = sp2 + (tile & 1) * STC_PTS;
      csync();
      float v[4][NPG], h[4][NPG], sv[4][NPG];
      // ---- layer 1: z = W^1 x + b^1, z_x = W^1[:, 0], z_y = W^1[:, 1], z_lap = 0
      {
        const float2 x = sp[p];
#pragma unroll
        for (int i = 0; i < NPG; ++i) {
          const float2 w = reinterpret_cast<const float2*>(pw + PW_W1)[4 * g + i];
          v[0][i] = fmaf(w.x, x.x, fmaf(w.y, x.y, pw[PW_B1 + 4 * g + i]));
          v[1][i] = w.x;
          v[2][i] = w.y;
          v[3][i] = 0.f;
        }
        if constexpr (GEN)
          jet4_fwd_gen(layer_act(nd, prm, 1), v, h, sv);
        else
          jet4_fwd(v, h, sv);
        save4(scr, p, g, sv);
        put_a(RA, p, g, h);   // L >= 3: a hidden-to-hidden layer reads it
      }
      // ---- hidden-to-hidden layers on the tensor cores
      for (int k = 2; k <= L - 1; ++k) {
        operands_ready(bars + 3, lane);
        mbar_park(bars + 1, mph, a.err);
        mph ^= 1u;
        after_sync();
        {
          float z[NPT];
          tmem_rowz(tq + nb, tq + 64 + nb, z);
          zs_row_write(ZS, r, nb, z);
        }
        csync();
        zs_read4(ZS, p, g, v);
        {
          const float4 b = *reinterpret_cast<const float4*>(pw + PW_BK + (k - 2) * 64 + 4 * g);
          v[0][0] += b.x;
          v[0][1] += b.y;
          v[0][2] += b.z;
          v[0][3] += b.w;
        }
        if constexpr (GEN)
          jet4_fwd_gen(layer_act(nd, prm, k), v, h, sv);
        else
          jet4_fwd(v, h, sv);
        save4(scr + (k - 1) * STC_W * ROWS, p, g, sv);
        if (k < L - 1)
          put_a(RA, p, g, h);
        else
          zs_write4(ZS, p, g, h);    // H^{L-1}, exact, for the output layer
      }
      // ---- output layer (FP32, row threads): y = W^L h + b^L on the value row, W^L h on the others
      csync();   // H^{L-1} in the staging array
      {
        const float* WL = pw + PW_WL;
        float z[NPT];
        zs_row_read(ZS, r, nb, z);
        float y[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
          for (int j = 0; j < NPT; ++j) y[o] = fmaf(WL[o * 64 + nb + j], z[j], y[o]);
#pragma unroll
        for (int o = 0; o < 3; ++o) Xs[(part * ROWS + r) * 4 + o] = y[o];
        csync();
        if (part == 0) {
#pragma unroll
          for (int o = 0; o < 3; ++o)
            if (o < D) {
              float yy = y[o];
#pragma unroll
              for (int q = 1; q < STC_W / NPT; ++q) yy += Xs[(q * ROWS + r) * 4 + o];
              Js[(pr * 3 + o) * 4 + cr] = yy + (cr == 0 ? pw[PW_BL + o] : 0.f);
            }
        }
        csync();
      }
      // ---- residual and its seeds, one thread per point
      if (tid < STC_PTS) {
        const bool vv = tid < nv;
        const float f = vv ? a.res_f[it.pt_off + t0 + tid] : 0.f;
        const float sq = point_residual(a.pde, D, Js + tid * 12, Gs + tid * 12, f, vv ? coef : 0.f, a.nu, a.re);
        if (vv) l0 += (double)sq * sd.inv_n_res;
      }
      csync();
      // saved jets of layer L - 1 for the first reverse step, in flight
      // during the output layer's reverse pass
      load4(scr + (L - 2) * STC_W * ROWS, p, g, sv);
      // ---- output layer, reverse (row threads): Hb^{L-1} = (W^L)^T yb into the
      // staging array (FP32); its weight gradient follows in the reverse step
      // of layer L - 1 (point threads)
      {
        const float* WL = pw + PW_WL;
        float yb[3], hb[NPT];
#pragma unroll
        for (int o = 0; o < 3; ++o) yb[o] = Gs[(pr * 3 + o) * 4 + cr];
#pragma unroll
        for (int j = 0; j < NPT; ++j)
          hb[j] = fmaf(yb[0], WL[nb + j], fmaf(yb[1], WL[64 + nb + j], yb[2] * WL[128 + nb + j]));
        zs_row_write(ZS, r, nb, hb);
        // the next tile's points, read while this tile's reverse pass runs
        if (tid < STC_PTS && tile + 1 < n_tiles) {
          const int t1 = t0 + STC_PTS + tid;
          sp2[((tile + 1) & 1) * STC_PTS + tid] = t1 < it.n_pts ? a.pts[it.pt_off + t1] : make_float2(0.f, 0.f);
        }
        if (part == 0 && cr == 0) {
#pragma unroll
          for (int o = 0; o < 3; ++o) dls[pr * 4 + o] += yb[o];
        }
        csync();   // Hb^{L-1} in the staging array for the point threads
      }
      // ---- hidden layers, reverse (point threads).  Hb^k is in the staging
      // array: written above for k = L - 1, moved there from tensor memory
      // (the row MMA of the step before, already waited for) for k < L - 1.
      for (int k = L - 1; k >= 1; --k) {
        if (k >= 2) {
          // the saved jets of layer k - 1, loaded after this step's rule:
          // into L1 now, so that the load waits for L1 rather than L2
#pragma unroll
          for (int i = 0; i < NPG; ++i)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(scr + (k - 2) * STC_W * ROWS + (4 * g + i) * ROWS + 4 * p));
        }
        if (k < L - 1) {
          float z[NPT];
          tmem_rowz(tq + nb, tq + 64 + nb, z);
          zs_row_write(ZS, r, nb, z);
          csync();
        }
        zs_read4(ZS, p, g, h);        // Hb^k
        if constexpr (GEN) {
          float gsl = 0.f;
          jet4_bwd_gen(layer_act(nd, prm, k), sv, h, v, gsl);
          // dJ/ds of layer k over the warp's points and neurons, added per warp
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) gsl += __shfl_xor_sync(FULL, gsl, o);
          if (lane == 0 && nd.aoff >= 0) sls[(k - 1) * 16 + warp] += gsl;
        } else {
          jet4_bwd(sv, h, v);         // Zb^k
        }
        if (k == L - 1) {
          // dW^L[o][n] = sum over points and components of yb_o H^{L-1}_n
          // (FP32; H^{L-1} rebuilt from the saved jets still in sv)
          if constexpr (GEN)
            jet4_saved_gen(layer_act(nd, prm, k), sv, h);
          else
            jet4_saved(sv, h);
          out_grad_sums(h, Gs + p * 12, lane, dlw + 4 * g);
        }
        if (k >= 2) {
          value_sums(v, lane, dbs + (k - 2) * 64 + 4 * g);   // db^k
          // saved jets of layer k - 1 (for H^{k-1} below and the next step's
          // reverse rule), in flight while the images are written
          load4(scr + (k - 2) * STC_W * ROWS, p, g, sv);
        } else {
          // dW^1 = sum of Zb x^T + Zb_x e_x^T + Zb_y e_y^T, db^1 = sum of Zb (FP32)
          in_grad_sums(v, sp[p], lane, d1s + 12 * g);
          break;
        }
        if (d_pending) {   // the last gradient MMAs read regions A and At
          mbar_park(bars + 2, dph, a.err);
          dph ^= 1u;
          d_pending = false;
          after_sync();
        }
        put_t(RT, p, g, v);
        put_a(RA, p, g, v);
        operands_ready(bars + 3, lane);
        // H^{k-1} from the saved jets of layer k - 1
        if constexpr (GEN)
          jet4_saved_gen(layer_act(nd, prm, k - 1), sv, h);
        else
          jet4_saved(sv, h);
        mbar_park(bars + 1, mph, a.err);   // region A is free
        mph ^= 1u;
        after_sync();
        put_b(RA, p, g, h);
        operands_ready(bars + 3, lane);
        d_pending = true;
      }
      // ---- flush the weight-gradient accumulators into the item's slice
      // every STC_FLUSH tiles and after the last: each accumulator then sums
      // at most STC_FLUSH tiles, and the flushes add in FP32 in tile order
      if (tile + 1 == n_tiles || (tile + 1) % STC_FLUSH == 0) {
        const bool add = tile >= STC_FLUSH, last = tile + 1 == n_tiles;
        if (d_pending) {
          mbar_park(bars + 2, dph, a.err);
          dph ^= 1u;
          d_pending = false;
        }
        after_sync();
        float* gs = a.partials + it.part_off;
        float* st_hi = RA;             // [64][65]: lanes 0-63 (hi parts)
        float* st_lo = RA + 64 * 65;   // lanes 64-127 (lo parts)
        float* stg = quad < 2 ? st_hi : st_lo;
        const int m = r & 63;
        for (int k = 2; k <= L - 1; ++k) {
          float v[NPT];
          tmem_cols<NPT>(tq + 128 + 64 * (k - 2) + nb, v);
#pragma unroll
          for (int j = 0; j < NPT; ++j) stg[m * 65 + nb + j] = v[j];
          csync();
          const int wo = nd.w[k], wi = nd.w[k - 1];
          float* gw = gs + nd.off[k];
          for (int e = tid; e < wo * wi; e += NTC) {
            const int n = e / wi, j = e - n * wi;
            gw[e] = (add ? gw[e] : 0.f) + (st_hi[n * 65 + j] + st_lo[n * 65 + j]);
          }
          if (last && tid < wo) gw[wo * wi + tid] = dbs[(k - 2) * 64 + tid];
          csync();
        }
        if (last) {
          // dW^1, db^1 and dW^L: FP32 sums over the whole item (shared memory)
          const int w1 = nd.w[1];
          if (tid < w1) {
            float* gw = gs + nd.off[1];
            gw[2 * tid] = d1s[3 * tid];
            gw[2 * tid + 1] = d1s[3 * tid + 1];
            gw[2 * w1 + tid] = d1s[3 * tid + 2];
          }
          float* gw = gs + nd.off[L];
          for (int e = tid; e < D * wl; e += NTC) {
            const int o = e / wl, n = e - o * wl;
            gw[e] = dlw[o * 64 + n];
          }
          if (tid < D) {
            float sb = 0.f;
            for (int q = 0; q < STC_PTS; ++q) sb += dls[q * 4 + tid];
            gw[D * wl + tid] = sb;
          }
          // trained slopes: dJ/da^k = n dJ/ds, the warps' sums in warp order
          if (GEN && nd.aoff >= 0 && tid < L - 1) {
            float sb = 0.f;
            for (int q = 0; q < 16; ++q) sb += sls[tid * 16 + q];
            gs[nd.aoff + tid] = nd.scale * sb;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        csync();   // region A is rewritten by the next tile
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const double ls = compute_sum(l0, red, warp, lane);
    if (tid == 0) {
      a.loss_part[2 * (int64_t)(a.item_base + ii)] = ls;
      a.loss_part[2 * (int64_t)(a.item_base + ii) + 1] = 0.0;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS) : "memory");
}

// Weight images for the training kernel, one CTA per image (see TcTrainPack).
// Layout: [N][K] K-major, core matrix (N/8, K/4) at (N/8) * 512 + (K/4) * 32 floats.
__global__ void __launch_bounds__(256) pack_tc_train_kernel(const float* __restrict__ params,
                                                            const TcTrainPack* __restrict__ blocks,
                                                            float* __restrict__ img) {
  const TcTrainPack b = blocks[blockIdx.x];
  const float* W = params + b.src;
  float* hi = img + b.dst;
  float* lo = hi + STC_W * STC_W;
  for (int e = threadIdx.x; e < STC_W * STC_W; e += blockDim.x) {
    const int nr = e >> 6, kc = e & 63;
    const int n = b.transpose ? kc : nr, j = b.transpose ? nr : kc;
    const float w = (n < b.n_out && j < b.n_in) ? W[n * b.n_in + j] : 0.f;
    const float2 s = tf32_split(w);
    const int off = (nr >> 3) * 512 + (kc >> 2) * 32 + (nr & 7) * 4 + (kc & 3);
    hi[off] = s.x;
    lo[off] = s.y;
  }
}

}  // namespace

bool step_tc_net_ok(const NetDev& nd, int n_nets, int pde, int min_width) {
  if (min_width <= 0 || n_nets != 1 || (pde != XPINN_PDE_POISSON && pde != XPINN_PDE_NS)) return false;
  if (nd.L < 3 || nd.L > STC_MAXL || nd.w[0] != 2 || nd.w[nd.L] < 1 || nd.w[nd.L] > 3) return false;
  if (nd.out_act != XPINN_ACT_IDENTITY) return false;
  for (int k = 1; k < nd.L; ++k)
    if (nd.w[k] < min_width || nd.w[k] > STC_W) return false;
  return true;
}

size_t step_tc_smem_bytes() { return sizeof(float) * (size_t)SMEM_FLOATS; }

cudaError_t step_tc_configure() {
  cudaError_t e = cudaFuncSetAttribute(step_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)step_tc_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_tc_smem_bytes());
  return e;
}

void launch_step_tc(const StepTcArgs& a, int grid, cudaStream_t s) {
  if (grid <= 0 || a.n_items <= 0) return;
  if (a.gen)
    step_tc_kernel<true><<<grid, NTH, step_tc_smem_bytes(), s>>>(a);
  else
    step_tc_kernel<false><<<grid, NTH, step_tc_smem_bytes(), s>>>(a);
}

void launch_pack_tc_train(const float* params, const TcTrainPack* blocks, int n_blocks, float* img,
                          cudaStream_t s) {
  if (n_blocks > 0) pack_tc_train_kernel<<<n_blocks, 256, 0, s>>>(params, blocks, img);
}

}  // namespace xp
