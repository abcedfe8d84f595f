// Point-to-subdomain router and stitching for the prediction of Eq. FSol:
// u(z) = sum_q u_q(z) 1_{Omega_q}(z), where the indicator is 1/S on a common
// interface shared by S subdomains.  Subdomains are closed boxes; a point on
// a shared edge (or corner) belongs to every box that contains it.
#include <cuda_runtime.h>

#include "xpinn_dev.cuh"

namespace xp {

constexpr int RTT = 256;
constexpr int MAXS = 4;   // a point of a box decomposition lies in at most 4 boxes

// Per point: membership count S and the (ascending) subdomain ids.  Counts
// entries per subdomain.  Points in more than MAXS boxes raise err = 1.
__global__ void route_kernel(const float2* __restrict__ pts, int64_t n, const SubDev* __restrict__ subs,
                             int q0, int nq, int* __restrict__ S, int* __restrict__ memb,
                             int* __restrict__ counts, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * RTT + threadIdx.x;
  if (i >= n) return;
  const float2 z = pts[i];
  int s = 0;
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

void launch_route(const float2* pts, int64_t n, const SubDev* subs, int q0, int nq, int* S, int* memb,
                  int* counts, int* err, cudaStream_t st) {
  if (n > 0) route_kernel<<<(unsigned)((n + RTT - 1) / RTT), RTT, 0, st>>>(pts, n, subs, q0, nq, S, memb, counts, err);
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
