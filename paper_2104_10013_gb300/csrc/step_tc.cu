// Residual items of the training step on the 5th-generation tensor cores
// (tcgen05, sm_103a).
//
// For an item (a range of residual points of one subdomain whose network
// step_tc.h admits) the kernel computes what the FP32 jet kernel computes for
// it: the Taylor jets of the network (Sec. 3) at the points, the PDE
// residual term of Eq. cPINNLoss / Eq. XPINNLoss (Sec. 4.2) and its gradient
// with respect to every weight and bias, written once to the item's gradient
// slice, and the item's loss sum.  The three point-by-width contractions of
// every hidden-to-hidden layer k run on the tensor cores:
//   forward    Z^k  = H^{k-1} (W^k)^T           [128 rows x 64] . [64 x 64]
//   reverse    Hb^{k-1} = Zb^k W^k              [128 rows x 64] . [64 x 64]
//   gradient   dW^k += (Zb^k)^T H^{k-1}         [64 x 128 rows] . [128 rows x 64]
// The first layer (two inputs), the output layer (at most three outputs),
// the jet rules and the residual stay on the FP32 pipes.
//
// Tile: 128 rows = the MMA's M, 32 points x 4 jet components (u, u_x, u_y,
// lap u) with the components of a point in 4 adjacent lanes; four threads per
// row (warps w, w + 4, w + 8 and w + 12 share tensor-memory lanes), each
// owning 16 of the 64 neurons.  The jet rule of tanh (h = t, h_i = s z_i, h_lap = s z_lap -
// 2 t s (z_x^2 + z_y^2), t = tanh z, s = 1 - t^2) and its reverse exchange
// t, hbar_lap and the sums over a point's rows by warp shuffles; tanh itself
// is evaluated once per (point, neuron), spread over the point's 4 lanes.
// Pre-activation jets (t on the value row, z_c on the others) go to per-CTA
// scratch in global memory (L2-resident) for the reverse pass, which
// rebuilds H^{k-1} from them.
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
// Operands are K-major, no swizzle.  Images whose K is the tile's rows pad
// every K-step of core matrices by 16 bytes so that a warp's 32 rows of one
// column store into 32 different banks.  Weight images (forward and reverse,
// built by pack_tc_train_kernel) arrive by bulk copy into two buffers, the
// copy of the image after next issued as soon as an MMA has released its
// buffer.  Every wait is bounded; a wait that gives up sets the error word,
// the launch stops taking items, frees its tensor memory and ends.
#include <cuda_runtime.h>

#include "jet_step.cuh"
#include "step_tc.h"
#include "tc_util.cuh"

namespace xp {

namespace {

constexpr int NPT = 16;                  // neurons of a thread (of the 64)
constexpr int NTH = 128 * (STC_W / NPT); // four threads per row
constexpr int ROWS = 128;
constexpr unsigned FULL = 0xffffffffu;
// K-major images whose K is the tile's rows: floats between K-adjacent core
// matrices, padded by 16 bytes so that a warp's 32 rows of one column store
// into 32 different banks
constexpr int LB_B = 8 * 32 + 4;    // B' = H^T [N = 64][K = rows]: 1040 bytes
constexpr int LB_T = 16 * 32 + 4;   // At = stacked Zb^T [M = 128][K = rows]: 2064 bytes
constexpr int LB_S = 2 * 32 + 4;    // [N = 16][K = rows] (input jets, output seeds): 272 bytes
constexpr int SZ_B = 32 * LB_B;     // one B' image (hi or lo)
constexpr int SZ_T = 32 * LB_T;
constexpr int SZ_S = 32 * LB_S;
constexpr int SZ_AF = ROWS * STC_W;  // one row-major A image (hi or lo)
constexpr int SZ_RA = 2 * SZ_B;      // region A: A (hi | lo), or B' (hi | lo)
// region A also holds, between the forward and the reverse pass, the partial
// outputs [4 parts][128 rows][4] and the output jets and seeds [32 points][3][4]
constexpr int RA_X = 0, RA_J = RA_X + 4 * ROWS * 4, RA_G = RA_J + 384;
static_assert(2 * SZ_AF <= SZ_RA && RA_G + 384 <= SZ_RA && 2 * 64 * 65 <= SZ_RA, "region A");
// the item's FP32-pipe weights, zero-padded to 64 neurons: W^1 [64][2], b^1,
// b^k (k = 2..L-1) [STC_MAXL - 2][64], W^L [3][64], b^L [4]
constexpr int PW_W1 = 0, PW_B1 = 128, PW_BK = 192, PW_WL = PW_BK + 64 * (STC_MAXL - 2), PW_BL = PW_WL + 192;
constexpr int SZ_PW = PW_BL + 4;
// shared-memory map (floats): region A, At, two weight buffers, the [16][rows]
// images, the points of two tiles, the bias-gradient partials [STC_MAXL - 2][4 lane
// quadrants][64] and [32 points][4], the FP32-pipe weights
constexpr int O_A = 0;
constexpr int O_T = O_A + SZ_RA;
constexpr int O_W = O_T + SZ_T;
constexpr int O_S = O_W + 2 * STC_IMG;
constexpr int O_P = O_S + 2 * SZ_S;
constexpr int O_DB = O_P + 128;
constexpr int O_DL = O_DB + (STC_MAXL - 2) * 4 * 64;
constexpr int O_PW = O_DL + 128;
constexpr int SMEM_FLOATS = O_PW + SZ_PW;
// tensor-memory columns: Z main [0, 64), Z cross [64, 128), dW^k (k = 2..L-1)
// at 128 + 64 (k - 2), then dW^1 and dW^L (16 columns each)
constexpr int TMEM_COLS = 512;
// tiles a weight-gradient accumulator sums before it is added into the
// item's slice (bounds the length of each tensor-memory accumulation)
constexpr int STC_FLUSH = 16;
static_assert(128 + 64 * (STC_MAXL - 2) + 32 <= TMEM_COLS, "tensor memory");

// element offsets in the images whose K is the rows (column n, row r); for
// column nb + i with nb a multiple of 8: base + col_step(i)
__device__ __forceinline__ int t_off(int m, int r) { return (m >> 3) * 32 + (r >> 2) * LB_T + (m & 7) * 4 + (r & 3); }
__device__ __forceinline__ int b_off(int j, int r) { return (j >> 3) * 32 + (r >> 2) * LB_B + (j & 7) * 4 + (r & 3); }
__device__ __forceinline__ int s_off(int j, int r) { return (j >> 3) * 32 + (r >> 2) * LB_S + (j & 7) * 4 + (r & 3); }
__device__ __forceinline__ constexpr int col_step(int i) { return (i >> 3) * 32 + (i & 7) * 4; }

__device__ __forceinline__ void fence_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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
// terms into tm + 64.
__device__ __forceinline__ void mma_rows(uint32_t tm, uint32_t a, uint32_t b) {
  const uint32_t id = tc_idesc(STC_W);
  const uint64_t ahi = tc_sdesc(a, TC_A_LBO, 128), alo = tc_sdesc(a + 4 * SZ_AF, TC_A_LBO, 128);
  const uint64_t bhi = tc_sdesc(b, 128, STC_W / 4 * 128);
  const uint64_t blo = tc_sdesc(b + 4 * STC_W * STC_W, 128, STC_W / 4 * 128);
#pragma unroll
  for (int ks = 0; ks < STC_W / 8; ++ks) {
    const uint64_t da = dstep(ks * 2 * TC_A_LBO), db = dstep(ks * 256);
    tc_mma(tm, ahi + da, bhi + db, id, ks > 0 ? 1u : 0u);
    tc_mma(tm + 64, ahi + da, blo + db, id, ks > 0 ? 1u : 0u);
    tc_mma(tm + 64, alo + da, bhi + db, id, 1u);
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

// Forward jet rule of tanh on this thread's row (component c) for its NPT
// neurons: z in (the value row's includes the bias), h out in z.  The saved
// value (t on the value row, z_c on the others) goes to Sk[n][row] (Sk
// points at this thread's first neuron and row).
__device__ __forceinline__ void jet_fwd(float (&z)[NPT], int c, int gb, float* __restrict__ Sk) {
  float t[NPT];
  // tanh of the value row's z, neuron 4g + c evaluated by lane c of the point
#pragma unroll
  for (int g = 0; g < NPT / 4; ++g) {
    const float a0 = __shfl_sync(FULL, z[4 * g], gb), a1 = __shfl_sync(FULL, z[4 * g + 1], gb);
    const float a2 = __shfl_sync(FULL, z[4 * g + 2], gb), a3 = __shfl_sync(FULL, z[4 * g + 3], gb);
    const float tm = tanhf(c == 0 ? a0 : (c == 1 ? a1 : (c == 2 ? a2 : a3)));
#pragma unroll
    for (int j = 0; j < 4; ++j) t[4 * g + j] = __shfl_sync(FULL, tm, gb + j);
  }
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    const float zi = z[i], ti = t[i], s = 1.f - ti * ti;
    float q = (c == 1 || c == 2) ? zi * zi : 0.f;
    q += __shfl_xor_sync(FULL, q, 1);
    q += __shfl_xor_sync(FULL, q, 2);
    Sk[i * ROWS] = c == 0 ? ti : zi;
    z[i] = c == 0 ? ti : (c == 3 ? s * zi - 2.f * ti * s * q : s * zi);
  }
}

// Reverse jet rule: adjoints hb of (h, h_x, h_y, h_lap) on this row to
// adjoints zb of (z, z_x, z_y, z_lap):
//   zb_lap = s hb_lap,  zb_i = s hb_i - 4 t s z_i hb_lap,
//   zb = s [hb - 2 t (z_x hb_x + z_y hb_y) + (-2 t z_lap + (6 t^2 - 2)(z_x^2 + z_y^2)) hb_lap]
// the bracket summed over the point's 4 rows.
__device__ __forceinline__ void jet_bwd(const float (&sv)[NPT], const float (&tv)[NPT], const float (&hb)[NPT],
                                        int c, int gb, float (&zb)[NPT]) {
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    const float zi = sv[i], ti = tv[i], s = 1.f - ti * ti, hbi = hb[i];
    const float h3 = __shfl_sync(FULL, hbi, gb + 3);
    float e = c == 0 ? hbi
                     : (c == 3 ? -2.f * ti * zi * h3
                               : -2.f * ti * zi * hbi + (6.f * ti * ti - 2.f) * zi * zi * h3);
    e += __shfl_xor_sync(FULL, e, 1);
    e += __shfl_xor_sync(FULL, e, 2);
    zb[i] = c == 0 ? s * e : (c == 3 ? s * hbi : s * hbi - 4.f * ti * s * zi * h3);
  }
}

__device__ __forceinline__ void split_all(const float (&v)[NPT], float (&hi)[NPT], float (&lo)[NPT]) {
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    const float2 s = tf32_split(v[i]);
    hi[i] = s.x;
    lo[i] = s.y;
  }
}

// Row-major A image (hi at A, lo at A + SZ_AF); A points at a_off(r, nb)
__device__ __forceinline__ void put_rows(float* __restrict__ A, const float (&hi)[NPT], const float (&lo)[NPT]) {
#pragma unroll
  for (int g = 0; g < NPT / 4; ++g) {
    *reinterpret_cast<float4*>(A + g * (TC_A_LBO / 4)) =
        make_float4(hi[4 * g], hi[4 * g + 1], hi[4 * g + 2], hi[4 * g + 3]);
    *reinterpret_cast<float4*>(A + SZ_AF + g * (TC_A_LBO / 4)) =
        make_float4(lo[4 * g], lo[4 * g + 1], lo[4 * g + 2], lo[4 * g + 3]);
  }
}

// Stacked transposed image (M-row n: hi, 64 + n: lo; K = row); T points at t_off(nb, r)
__device__ __forceinline__ void put_stacked(float* __restrict__ T, const float (&hi)[NPT], const float (&lo)[NPT]) {
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    T[col_step(i)] = hi[i];
    T[8 * 32 + col_step(i)] = lo[i];   // M-row 64 + n: eight 8-row groups further
  }
}

// Transposed B' image (N = neuron, K = row; hi, then lo); B points at b_off(nb, r)
__device__ __forceinline__ void put_bt(float* __restrict__ B, const float (&hi)[NPT], const float (&lo)[NPT]) {
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    B[col_step(i)] = hi[i];
    B[SZ_B + col_step(i)] = lo[i];
  }
}

// H from saved jets: sv (this row's saved value), tv (t of the point)
__device__ __forceinline__ void jet_from_saved(const float (&sv)[NPT], const float (&tv)[NPT], int c,
                                               float (&h)[NPT]) {
#pragma unroll
  for (int i = 0; i < NPT; ++i) {
    const float zi = sv[i], ti = tv[i], s = 1.f - ti * ti;
    float q = (c == 1 || c == 2) ? zi * zi : 0.f;
    q += __shfl_xor_sync(FULL, q, 1);
    q += __shfl_xor_sync(FULL, q, 2);
    h[i] = c == 0 ? ti : (c == 3 ? s * zi - 2.f * ti * s * q : s * zi);
  }
}

// Saved jets of one layer (Sk at this thread's first neuron and row) and t
// of the point on every row
__device__ __forceinline__ void load_saved(const float* __restrict__ Sk, int gb, float (&sv)[NPT],
                                           float (&tv)[NPT]) {
#pragma unroll
  for (int i = 0; i < NPT; ++i) sv[i] = __ldcg(Sk + i * ROWS);
#pragma unroll
  for (int i = 0; i < NPT; ++i) tv[i] = __shfl_sync(FULL, sv[i], gb);
}

// Sum of the value rows' zb over the warp's 8 points, scattered: the value
// lane of point v (lane 4 v) ends with the sums of neurons 2 v and 2 v + 1
// (of the thread's NPT) in out[0], out[1].  Halving exchanges: xor 16
// (neurons 0-7 / 8-15), xor 8, xor 4.
__device__ __forceinline__ void value_row_sums(const float (&zb)[NPT], int lane, float (&out)[2]) {
  static_assert(NPT == 16, "three halving steps");
  float a[8], b[4];
  const bool h16 = (lane >> 4) & 1, h8 = (lane >> 3) & 1, h4 = (lane >> 2) & 1;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float keep = h16 ? zb[8 + j] : zb[j], send = h16 ? zb[j] : zb[8 + j];
    a[j] = keep + __shfl_xor_sync(FULL, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float keep = h8 ? a[4 + j] : a[j], send = h8 ? a[j] : a[4 + j];
    b[j] = keep + __shfl_xor_sync(FULL, send, 8);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float keep = h4 ? b[2 + j] : b[j], send = h4 ? b[j] : b[2 + j];
    out[j] = keep + __shfl_xor_sync(FULL, send, 4);
  }
}

__global__ void __launch_bounds__(NTH, 1) step_tc_kernel(StepTcArgs a) {
  extern __shared__ __align__(1024) float sm[];
  float* RA = sm + O_A;
  float* RT = sm + O_T;
  float* RW = sm + O_W;
  float* RS = sm + O_S;
  float* Xs = RA + RA_X;
  float* Js = RA + RA_J;
  float* Gs = RA + RA_G;
  float2* const sp2 = reinterpret_cast<float2*>(sm + O_P);   // points: this tile's and the next one's
  float* dbs = sm + O_DB;
  float* dls = sm + O_DL;
  float* pw = sm + O_PW;
  __shared__ __align__(8) uint64_t bars[4];   // weight buffers 0 and 1, row MMAs, gradient MMAs
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_stop;
  __shared__ double red[NTH / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2, nb = part * NPT;
  const int r = quad * 32 + lane, p = r >> 2, c = r & 3, gb = lane & ~3;
  // this thread's bases in the images
  float* const A_r = RA + a_off(r, nb);
  float* const T_r = RT + t_off(nb, r);
  float* const B_r = RA + b_off(nb, r);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(bars + i, 1);
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
  const uint32_t sa = smem_u32(RA), st = smem_u32(RT), sw = smem_u32(RW), ss = smem_u32(RS);
  float* const S_r = a.scratch + (int64_t)blockIdx.x * STC_SCRATCH + nb * ROWS + r;
  uint32_t wph = 0, mph = 0, dph = 0;   // phase parities (wph: bit per weight buffer)
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
    // the item's FP32-pipe weights, zero-padded (visible after the first tile's barrier)
    for (int e = tid; e < SZ_PW; e += NTH) {
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
    for (int e = tid; e < (STC_MAXL - 2) * 4 * 64; e += NTH) dbs[e] = 0.f;
    if (tid < 128) dls[tid] = 0.f;
    double l0 = 0.0;
    const int n_tiles = (it.n_pts + STC_PTS - 1) / STC_PTS;
    if (tid < STC_PTS) sp2[tid] = tid < it.n_pts ? a.pts[it.pt_off + tid] : make_float2(0.f, 0.f);
    for (int tile = 0; tile < n_tiles; ++tile) {
      const int t0 = tile * STC_PTS;
      const int nv = min(STC_PTS, it.n_pts - t0);
      // every MMA of the previous tile has completed: both weight buffers and
      // regions A, At and S are free
      if (d_pending) {
        mbar_park(bars + 3, dph, a.err);
        dph ^= 1u;
        d_pending = false;
      }
      if (tid == 0) {
        bulk_g2s(RW, img_src(0), 4u * STC_IMG, bars);
        if (nimg > 1) bulk_g2s(RW + STC_IMG, img_src(1), 4u * STC_IMG, bars + 1);
      }
      const float2* sp = sp2 + (tile & 1) * STC_PTS;
      __syncthreads();
      float z[NPT], zh[NPT], zl[NPT];
      // ---- layer 1: z = W^1 x + b^1, z_x = W^1[:, 0], z_y = W^1[:, 1], z_lap = 0
      {
        const float2 x = sp[p];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
          const float2 w = reinterpret_cast<const float2*>(pw + PW_W1)[nb + i];
          const float b = pw[PW_B1 + nb + i];
          z[i] = c == 0 ? fmaf(w.x, x.x, fmaf(w.y, x.y, b)) : (c == 1 ? w.x : (c == 2 ? w.y : 0.f));
        }
        jet_fwd(z, c, gb, S_r);
        split_all(z, zh, zl);
        put_rows(A_r, zh, zl);   // L >= 3: a hidden-to-hidden layer reads it
      }
      // ---- hidden-to-hidden layers on the tensor cores
      for (int k = 2; k <= L - 1; ++k) {
        const int i = k - 2, buf = i & 1;
        fence_to_async();
        __syncthreads();
        if (tid == 0) {
          mbar_wait(bars + buf, (wph >> buf) & 1u, a.err);
          wph ^= 1u << buf;
          after_sync();
          mma_rows(tmem, sa, sw + 4u * STC_IMG * buf);
          mma_commit(bars + 2);
        }
        mbar_park(bars + 2, mph, a.err);
        mph ^= 1u;
        after_sync();
        if (tid == 0 && i + 2 < nimg) bulk_g2s(RW + STC_IMG * buf, img_src(i + 2), 4u * STC_IMG, bars + buf);
        tmem_rowz(tq + nb, tq + 64 + nb, z);
        const float* bk = pw + PW_BK + (k - 2) * 64 + nb;
#pragma unroll
        for (int j = 0; j < NPT; ++j) z[j] += c == 0 ? bk[j] : 0.f;
        jet_fwd(z, c, gb, S_r + (k - 1) * STC_W * ROWS);
        split_all(z, zh, zl);
        if (k < L - 1)
          put_rows(A_r, zh, zl);
        else
          put_stacked(T_r, zh, zl);   // H^{L-1} for the output layer's weight gradient
      }
      // ---- output layer (FP32): y = W^L h + b^L on the value row, W^L h on the others
      {
        const float* WL = pw + PW_WL;
        float y[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
          for (int j = 0; j < NPT; ++j) y[o] = fmaf(WL[o * 64 + nb + j], z[j], y[o]);
#pragma unroll
        for (int o = 0; o < 3; ++o) Xs[(part * ROWS + r) * 4 + o] = y[o];
        __syncthreads();
        if (part == 0) {
#pragma unroll
          for (int o = 0; o < 3; ++o)
            if (o < D) {
              float v = y[o];
#pragma unroll
              for (int q = 1; q < STC_W / NPT; ++q) v += Xs[(q * ROWS + r) * 4 + o];
              Js[(p * 3 + o) * 4 + c] = v + (c == 0 ? pw[PW_BL + o] : 0.f);
            }
        }
        __syncthreads();
      }
      // ---- residual and its seeds, one thread per point
      if (tid < STC_PTS) {
        const bool v = tid < nv;
        PtJets J, G;
#pragma unroll
        for (int o = 0; o < XPINN_MAX_OUT; ++o)
#pragma unroll
          for (int cc = 0; cc < KMAX; ++cc) {
            J.u[o][cc] = (o < D && cc < 4) ? Js[(tid * 3 + o) * 4 + cc] : 0.f;
            G.u[o][cc] = 0.f;
          }
#pragma unroll
        for (int cc = 0; cc < KMAX; ++cc) J.k[cc] = G.k[cc] = 0.f;
        float rr[3] = {0.f, 0.f, 0.f};
        const float f = v ? a.res_f[it.pt_off + t0 + tid] : 0.f;
        const int ne = residual_fwd(a.pde, J, f, a.nu, a.re, rr);
        float sq = 0.f, e[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < ne) {
            sq += rr[q] * rr[q];
            e[q] = v ? coef * rr[q] : 0.f;
          }
        if (v) l0 += (double)sq * sd.inv_n_res;
        residual_seed(a.pde, J, e, a.nu, a.re, G);
#pragma unroll
        for (int o = 0; o < 3; ++o)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) Gs[(tid * 3 + o) * 4 + cc] = o < D ? G.u[o][cc] : 0.f;
      }
      __syncthreads();
      // ---- output layer, reverse: Hb^{L-1} = (W^L)^T yb (FP32); dW^L on the
      // tensor cores (At = stacked H^{L-1} transposed, B = yb transposed)
      float hb[NPT];
      {
        const float* WL = pw + PW_WL;
        float yb[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) yb[o] = Gs[(p * 3 + o) * 4 + c];
#pragma unroll
        for (int j = 0; j < NPT; ++j)
          hb[j] = fmaf(yb[0], WL[nb + j], fmaf(yb[1], WL[64 + nb + j], yb[2] * WL[128 + nb + j]));
        // the next tile's points, read while this tile's reverse pass runs
        if (tid < STC_PTS && tile + 1 < n_tiles) {
          const int t1 = t0 + STC_PTS + tid;
          sp2[((tile + 1) & 1) * STC_PTS + tid] = t1 < it.n_pts ? a.pts[it.pt_off + t1] : make_float2(0.f, 0.f);
        }
        if (part == 0) {
#pragma unroll
          for (int o = 0; o < 16; ++o) {
            const float2 s2 = tf32_split(o < 3 ? yb[o] : 0.f);
            RS[s_off(o, r)] = s2.x;
            RS[SZ_S + s_off(o, r)] = s2.y;
          }
          if (c == 0) {
#pragma unroll
            for (int o = 0; o < 3; ++o) dls[p * 4 + o] += yb[o];
          }
        }
        fence_to_async();
        __syncthreads();
        if (tid == 0) {
          after_sync();
          mma_grad<4 * LB_S>(tmem + 144 + 64 * (L - 2), st, ss, 4u * SZ_S, 16, tile % STC_FLUSH == 0);
          mma_commit(bars + 3);
        }
        d_pending = true;
      }
      // ---- hidden layers, reverse.  Hb^k of k < L - 1 is in tensor memory
      // (the row MMA of the step before, already waited for).
      float sv[NPT], tv[NPT];
      load_saved(S_r + (L - 2) * STC_W * ROWS, gb, sv, tv);
      for (int k = L - 1; k >= 1; --k) {
        if (k < L - 1) tmem_rowz(tq + nb, tq + 64 + nb, hb);
        jet_bwd(sv, tv, hb, c, gb, z);
        split_all(z, zh, zl);
        if (d_pending) {   // the last gradient MMAs read regions A, At and S
          mbar_park(bars + 3, dph, a.err);
          dph ^= 1u;
          d_pending = false;
          after_sync();
        }
        put_stacked(T_r, zh, zl);
        if (k >= 2) {
          put_rows(A_r, zh, zl);
        } else if (part == 0) {
          // layer 1's input jets, transposed: value row (x, y, 1), x row
          // (1, 0, 0), y row (0, 1, 0), Laplacian row 0; column 2 gives db^1
          const float2 x = sp[p];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float vj = j == 0 ? (c == 0 ? x.x : (c == 1 ? 1.f : 0.f))
                                    : (j == 1 ? (c == 0 ? x.y : (c == 2 ? 1.f : 0.f)) : (j == 2 && c == 0 ? 1.f : 0.f));
            const float2 s2 = tf32_split(vj);
            RS[s_off(j, r)] = s2.x;
            RS[SZ_S + s_off(j, r)] = s2.y;
          }
        }
        fence_to_async();
        __syncthreads();
        if (k == 1) {
          if (tid == 0) {
            after_sync();
            mma_grad<4 * LB_S>(tmem + 128 + 64 * (L - 2), st, ss, 4u * SZ_S, 16, tile % STC_FLUSH == 0);
            mma_commit(bars + 3);
          }
          d_pending = true;
          break;
        }
        const int i = (L - 2) + (L - 1 - k), buf = i & 1;
        if (tid == 0) {
          mbar_wait(bars + buf, (wph >> buf) & 1u, a.err);
          wph ^= 1u << buf;
          after_sync();
          mma_rows(tmem, sa, sw + 4u * STC_IMG * buf);
          mma_commit(bars + 2);
        }
        // bias gradient: sums of the value rows of Zb^k over the warp's points
        {
          float sb[2];
          value_row_sums(z, lane, sb);
          if (c == 0) {
            float* d = dbs + ((k - 2) * 4 + quad) * 64 + nb + 2 * (lane >> 2);
            d[0] += sb[0];
            d[1] += sb[1];
          }
        }
        // H^{k-1} from the saved jets of layer k - 1 (which the next step's
        // reverse rule uses too)
        load_saved(S_r + (k - 2) * STC_W * ROWS, gb, sv, tv);
        jet_from_saved(sv, tv, c, z);
        split_all(z, zh, zl);
        mbar_park(bars + 2, mph, a.err);   // region A and the weight buffer are free
        mph ^= 1u;
        after_sync();
        if (tid == 0 && i + 2 < nimg) bulk_g2s(RW + STC_IMG * buf, img_src(i + 2), 4u * STC_IMG, bars + buf);
        put_bt(B_r, zh, zl);
        fence_to_async();
        __syncthreads();
        if (tid == 0) {
          after_sync();
          mma_grad<4 * LB_B>(tmem + 128 + 64 * (k - 2), st, sa, 4u * SZ_B, STC_W, tile % STC_FLUSH == 0);
          mma_commit(bars + 3);
        }
        d_pending = true;
      }
      // ---- flush the weight-gradient accumulators into the item's slice
      // every STC_FLUSH tiles and after the last: each accumulator then sums
      // at most STC_FLUSH tiles, and the flushes add in FP32 in tile order
      if (tile + 1 == n_tiles || (tile + 1) % STC_FLUSH == 0) {
        const bool add = tile >= STC_FLUSH, last = tile + 1 == n_tiles;
        if (d_pending) {
          mbar_park(bars + 3, dph, a.err);
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
          __syncthreads();
          const int wo = nd.w[k], wi = nd.w[k - 1];
          float* g = gs + nd.off[k];
          for (int e = tid; e < wo * wi; e += NTH) {
            const int n = e / wi, j = e - n * wi;
            g[e] = (add ? g[e] : 0.f) + (st_hi[n * 65 + j] + st_lo[n * 65 + j]);
          }
          if (last && tid < wo) {
            float sb = 0.f;
            for (int q = 0; q < 4; ++q) sb += dbs[((k - 2) * 4 + q) * 64 + tid];
            g[wo * wi + tid] = sb;
          }
          __syncthreads();
        }
        {
          // dW^1 (columns 0, 1) and db^1 (column 2); dW^L (columns o < D), transposed
          float v1[16], vl[16];
          tmem_cols<16>(tq + 128 + 64 * (L - 2), v1);
          tmem_cols<16>(tq + 144 + 64 * (L - 2), vl);
          if (part == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              stg[m * 65 + j] = v1[j];
              stg[m * 65 + 16 + j] = vl[j];
            }
          }
          __syncthreads();
          const int w1 = nd.w[1];
          if (tid < w1) {
            float* g = gs + nd.off[1];
            g[2 * tid] = (add ? g[2 * tid] : 0.f) + (st_hi[tid * 65] + st_lo[tid * 65]);
            g[2 * tid + 1] = (add ? g[2 * tid + 1] : 0.f) + (st_hi[tid * 65 + 1] + st_lo[tid * 65 + 1]);
            g[2 * w1 + tid] = (add ? g[2 * w1 + tid] : 0.f) + (st_hi[tid * 65 + 2] + st_lo[tid * 65 + 2]);
          }
          float* g = gs + nd.off[L];
          for (int e = tid; e < D * wl; e += NTH) {
            const int o = e / wl, n = e - o * wl;
            g[e] = (add ? g[e] : 0.f) + (st_hi[n * 65 + 16 + o] + st_lo[n * 65 + 16 + o]);
          }
          if (last && tid < D) {
            float sb = 0.f;
            for (int q = 0; q < STC_PTS; ++q) sb += dls[q * 4 + tid];
            g[D * wl + tid] = sb;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // region A is rewritten by the next tile
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const double ls = block_sum(l0, red);
    if (tid == 0) {
      a.loss_part[2 * (int64_t)(a.item_base + ii)] = ls;
      a.loss_part[2 * (int64_t)(a.item_base + ii) + 1] = 0.0;
    }
    __syncthreads();
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
  if (nd.out_act != XPINN_ACT_IDENTITY || net_is_general(nd)) return false;
  for (int k = 1; k < nd.L; ++k)
    if (nd.w[k] < min_width || nd.w[k] > STC_W) return false;
  return true;
}

size_t step_tc_smem_bytes() { return sizeof(float) * (size_t)SMEM_FLOATS; }

cudaError_t step_tc_configure() {
  return cudaFuncSetAttribute(step_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)step_tc_smem_bytes());
}

void launch_step_tc(const StepTcArgs& a, int grid, cudaStream_t s) {
  if (grid > 0 && a.n_items > 0) step_tc_kernel<<<grid, NTH, step_tc_smem_bytes(), s>>>(a);
}

void launch_pack_tc_train(const float* params, const TcTrainPack* blocks, int n_blocks, float* img,
                          cudaStream_t s) {
  if (n_blocks > 0) pack_tc_train_kernel<<<n_blocks, 256, 0, s>>>(params, blocks, img);
}

}  // namespace xp
