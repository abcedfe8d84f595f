// Point-to-subdomain router and stitching for the prediction of Eq. FSol:
// u(z) = sum_q u_q(z) 1_{Omega_q}(z), where the indicator is 1/S on a common
// interface shared by S subdomains.  Subdomains are closed boxes; a point on
// a shared edge (or corner) belongs to every box that contains it.
#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

constexpr int RTT = 256;
constexpr int MAXS = 4;   // a point of a box decomposition lies in at most 4 boxes

// Even-odd rule: is z inside the polygon poly[0..m)?  The crossing abscissa
// of every edge is rounded in float32 in a fixed order,
// xc = a.x + ((z.y - a.y) * (b.x - a.x)) / (b.y - a.y), each operation
// rounded to nearest (no fused multiply-add), so that a point on or next to
// an edge is classified the same way by every implementation of that order.
__device__ __forceinline__ bool in_polygon(float2 z, const float2* __restrict__ poly, int m) {
  bool in = false;
  for (int e = 0; e < m; ++e) {
    const float2 a = poly[e], b = poly[e + 1 == m ? 0 : e + 1];
    if ((a.y > z.y) != (b.y > z.y)) {
      const float t = __fmul_rn(__fsub_rn(z.y, a.y), __fsub_rn(b.x, a.x));
      const float xc = __fadd_rn(a.x, __fdiv_rn(t, __fsub_rn(b.y, a.y)));
      if (z.x < xc) in = !in;
    }
  }
  return in;
}

// Squared distance rounded as (dx*dx) + (dy*dy) with no fused multiply-add,
// so that exact ties are the same on every implementation.
__device__ __forceinline__ float dist2(float2 z, const float* s) {
  const float dx = __fsub_rn(z.x, s[0]), dy = __fsub_rn(z.y, s[1]);
  return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Per point: membership count S and the (ascending) subdomain ids.  Counts
// entries per subdomain.  Points in more than MAXS regions raise err = 1.
// Box regions: closed boxes.  Voronoi regions: inside the polygon, nearest
// site (all sites at the minimum distance).
__global__ void route_kernel(const float2* __restrict__ pts, int64_t n, const SubDev* __restrict__ subs,
                             int q0, int nq, int* __restrict__ S, int* __restrict__ memb,
                             int* __restrict__ counts, int* __restrict__ err,
                             const float2* __restrict__ poly, int n_poly) {
  const int64_t i = (int64_t)blockIdx.x * RTT + threadIdx.x;
  if (i >= n) return;
  const float2 z = pts[i];
  int s = 0;
  if (subs[q0].region_kind == XPINN_REGION_VORONOI) {
    if (n_poly >= 3 && in_polygon(z, poly, n_poly)) {
      float dmin = 3.4e38f;
      for (int l = 0; l < nq; ++l) dmin = fminf(dmin, dist2(z, subs[q0 + l].site));
      for (int l = 0; l < nq; ++l)
        if (dist2(z, subs[q0 + l].site) == dmin) {
          if (s < MAXS) {
            memb[i * MAXS + s] = l;
            atomicAdd(counts + l, 1);
          } else {
            atomicCAS(err, 0, 1);
          }
          ++s;
        }
    }
    S[i] = s < MAXS ? s : MAXS;
    return;
  }
  for (int l = 0; l < nq; ++l) {
    const float* r = subs[q0 + l].rect;
    if (z.x >= r[0] && z.x <= r[1] && z.y >= r[2] && z.y <= r[3]) {
      if (s < MAXS) {
        memb[i * MAXS + s] = l;
        atomicAdd(counts + l, 1);
      } else {
        atomicCAS(err, 0, 1);
      }
      ++s;
    }
  }
  S[i] = s < MAXS ? s : MAXS;
}

// Scatter every (point, membership) entry to its subdomain's bucket.  The
// position inside a bucket may vary between runs; each entry's value does not.
__global__ void bucket_kernel(const float2* __restrict__ pts, int64_t n, const int* __restrict__ S,
                              const int* __restrict__ memb, int* __restrict__ cursor,
                              int* __restrict__ pos, float2* __restrict__ epts,
                              float* __restrict__ escale) {
  const int64_t i = (int64_t)blockIdx.x * RTT + threadIdx.x;
  if (i >= n) return;
  const int s = S[i];
  for (int j = 0; j < s; ++j) {
    const int l = memb[i * MAXS + j];
    const int p = atomicAdd(cursor + l, 1);
    pos[i * MAXS + j] = p;
    epts[p] = pts[i];
    escale[p] = 1.f / (float)s;
  }
}

// out[i] = sum over memberships (ascending subdomain) of the entry rows; NaN if none.
__global__ void gather_kernel(int64_t n, int row, const int* __restrict__ S, const int* __restrict__ pos,
                              const float* __restrict__ eout, float* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * RTT + threadIdx.x;
  if (idx >= n * row) return;
  const int64_t i = idx / row;
  const int c = (int)(idx - i * row);
  const int s = S[i];
  float acc = s == 0 ? __int_as_float(0x7fc00000) : 0.f;
  for (int j = 0; j < s; ++j) acc += eout[(int64_t)pos[i * MAXS + j] * row + c];
  out[idx] = acc;
}

// Device-side plan of a routed evaluation (no host round trip): one CTA
// takes the per-subdomain entry counts, writes each bucket's start into
// cursor[l] (exclusive prefix sum, the bucket kernel's insertion cursor) and
// cuts every bucket into items of at most proto[l].chunk entries, written to
// items[]; *n_items receives their number (items beyond max_items are not
// written and raise err = XPINN_ERR_INVALID, which a correct bound excludes).
__global__ void __launch_bounds__(256) eval_plan_kernel(const int* __restrict__ counts, int nq,
                                                        const EvalProto* __restrict__ proto, int q0,
                                                        int row, int* __restrict__ cursor,
                                                        Item* __restrict__ items, int* __restrict__ n_items,
                                                        int max_items, int* __restrict__ err) {
  __shared__ int s_warp[2][8];
  __shared__ int s_carry[2];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_carry[0] = s_carry[1] = 0;
  __syncthreads();
  for (int base = 0; base < nq; base += 256) {
    const int l = base + t;
    const int c = l < nq ? counts[l] : 0;
    const int ch = l < nq ? proto[l].chunk : 1;
    const int ni = (c + ch - 1) / ch;
    // inclusive scans of (c, ni) over the 256 threads: warp shuffles, then the warps' totals
    int a = c, b = ni;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= o) { a += ua; b += ub; }
    }
    if (lane == 31) { s_warp[0][warp] = a; s_warp[1][warp] = b; }
    __syncthreads();
    int pa = s_carry[0], pb = s_carry[1];
    for (int w = 0; w < warp; ++w) { pa += s_warp[0][w]; pb += s_warp[1][w]; }
    const int start = pa + a - c, istart = pb + b - ni;   // exclusive
    if (l < nq) {
      cursor[l] = start;
      const EvalProto pr = proto[l];
      for (int j = 0; j < ni; ++j) {
        const int k = istart + j;
        if (k >= max_items) {
          atomicCAS(err, 0, XPINN_ERR_INVALID);
          break;
        }
        Item it;
        it.kind = IT_EVAL;
        it.q = q0 + l;
        it.edge = -1;
        it.side = 0;
        it.P = pr.P;
        it.K[0] = pr.K0;
        it.K[1] = pr.K1;
        it.lap = 0;
        it.pt_off = (int64_t)start + (int64_t)j * pr.chunk;
        it.n_pts = min(pr.chunk, c - j * pr.chunk);
        it.part_off = -1;
        it.out_off = it.pt_off * row;
        items[k] = it;
      }
    }
    __syncthreads();
    if (t == 255) { s_carry[0] = pa + a; s_carry[1] = pb + b; }
    __syncthreads();
  }
  if (t == 0) *n_items = min(s_carry[1], max_items);
}

void launch_eval_plan(const int* counts, int nq, const EvalProto* proto, int q0, int row, int* cursor,
                      Item* items, int* n_items, int max_items, int* err, cudaStream_t st) {
  eval_plan_kernel<<<1, 256, 0, st>>>(counts, nq, proto, q0, row, cursor, items, n_items, max_items, err);
}

void launch_route(const float2* pts, int64_t n, const SubDev* subs, int q0, int nq, int* S, int* memb,
                  int* counts, int* err, const float2* poly, int n_poly, cudaStream_t st) {
  if (n > 0)
    route_kernel<<<(unsigned)((n + RTT - 1) / RTT), RTT, 0, st>>>(pts, n, subs, q0, nq, S, memb, counts, err,
                                                                  poly, n_poly);
}
void launch_bucket(const float2* pts, int64_t n, const int* S, const int* memb, int* cursor, int* pos,
                   float2* epts, float* escale, cudaStream_t st) {
  if (n > 0) bucket_kernel<<<(unsigned)((n + RTT - 1) / RTT), RTT, 0, st>>>(pts, n, S, memb, cursor, pos, epts, escale);
}
void launch_gather(int64_t n, int row, const int* S, const int* pos, const float* eout, float* out,
                   cudaStream_t st) {
  const int64_t tot = n * row;
  if (tot > 0) gather_kernel<<<(unsigned)((tot + RTT - 1) / RTT), RTT, 0, st>>>(n, row, S, pos, eout, out);
}

}  // namespace xp
