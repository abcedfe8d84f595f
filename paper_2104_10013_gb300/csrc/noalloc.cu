// Residual-loss gradient of one network without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// owned by someone else (a host framework with its own caching allocator that
// forbids foreign allocations, an embedded runtime with a fixed memory
// budget, or a region of a program that must not allocate because it is being
// timed or replayed).  xpinn_residual_grad_noalloc serves them: the caller
// passes inputs and outputs in device memory it already owns, and all working
// memory the jet kernel needs (work descriptors, the work counter, weight
// images, saved jets and per-item gradient slices) comes from one fixed array
// in this file, g_noalloc_scratch, of XPINN_NOALLOC_SCRATCH_BYTES.  That array exists on
// every GPU that loads the library, for as long as the library stays loaded.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (the host-side name of a __device__ array is not
// a device address) while that device is current, and caches it.  Make that
// first call before any stream capture.
//
// All calls share the one array, and each call leaves its contents behind.
// The pieces that must start at zero (the work counter) are cleared by every
// call on its stream.  Calls whose kernels overlap on the GPU (different
// streams, or different threads without ordering) race on the array and give
// wrong results: order them on one stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "xpinn_dev.cuh"

namespace xp {

void set_last_error(const char* msg);   // the message xpinn_last_error() returns

namespace {

constexpr int NA_MAX_ITEMS = 128;     // work items (and gradient slices) per call
constexpr int NA_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[XPINN_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_ptr[NA_MAX_DEVICES] = {};

struct NaDesc {
  SubDev sd;
  Item items[NA_MAX_ITEMS];
  int n_items;
  PackBlock pack[2 * MAXL];   // weight images of the hidden-to-hidden layers
  int n_pack;
};

// Layout of the scratch array (byte offsets, each 256-byte aligned).
struct NaLayout {
  size_t sub, items, counter, err, loss_part, pack, img, partials, scratch, total;
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

NaLayout layout(int n_items, int n_params, int grid, int64_t scratch_per_cta, int64_t img_floats) {
  NaLayout l{};
  size_t o = 0;
  l.sub = o; o = up256(o + sizeof(SubDev));
  l.items = o; o = up256(o + sizeof(Item) * NA_MAX_ITEMS);
  l.counter = o; o = up256(o + sizeof(int));
  l.err = o; o = up256(o + sizeof(int));
  l.loss_part = o; o = up256(o + sizeof(double) * 2 * NA_MAX_ITEMS);
  l.pack = o; o = up256(o + sizeof(PackBlock) * 2 * MAXL);
  l.img = o; o = up256(o + sizeof(float) * (size_t)img_floats);
  l.partials = o; o = up256(o + sizeof(float) * (size_t)n_items * n_params);
  l.scratch = o; o = up256(o + sizeof(float) * (size_t)grid * scratch_per_cta);
  l.total = o;
  return l;
}

// Copies the descriptors (passed by value) into the array and clears the
// work counter and the error flag: the only state that must start at zero.
__global__ void na_setup_kernel(NaDesc d, SubDev* sub, Item* items, int* counter, int* err, PackBlock* pack) {
  const int t = threadIdx.x;
  if (t == 0) {
    *sub = d.sd;
    *counter = 0;
    *err = 0;
  }
  for (int i = t; i < d.n_items; i += blockDim.x) items[i] = d.items[i];
  for (int i = t; i < d.n_pack; i += blockDim.x) pack[i] = d.pack[i];
}

// grads[e] = sum over items (in order) of the item's slice; loss = sum of the
// items' residual sums (each already divided by n).
__global__ void na_reduce_kernel(const float* __restrict__ partials, const double* __restrict__ loss_part,
                                 int n_items, int n_params, float* __restrict__ grads,
                                 float* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_params) {
    float g = 0.f;
    for (int i = 0; i < n_items; ++i) g += partials[(size_t)i * n_params + e];
    grads[e] = g;
  }
  if (e == 0) {
    double s = 0.0;
    for (int i = 0; i < n_items; ++i) s += loss_part[2 * i];
    *loss = (float)s;
  }
}

int fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

}  // namespace
}  // namespace xp

using namespace xp;

extern "C" int xpinn_residual_grad_noalloc(int32_t pde, float nu, float re, const xpinn_net_desc* net,
                                           const float* params, const float* xy, const float* f,
                                           int64_t n, float w_res, float* loss, float* grads,
                                           void* stream) {
  set_last_error("");
  if (!net || !params || !xy || !f || !loss || !grads || n < 0)
    return fail(XPINN_ERR_INVALID, "NULL argument or negative point count");
  if (pde != XPINN_PDE_BURGERS && pde != XPINN_PDE_POISSON && pde != XPINN_PDE_NS)
    return fail(XPINN_ERR_UNSUPPORTED, "only single-network PDEs (Burgers, Poisson, Navier-Stokes)");
  if (n > (1ll << 30)) return fail(XPINN_ERR_UNSUPPORTED, "more than 2^30 points");
  const int L = net->n_layers;
  if (L < 2 || L > XPINN_MAX_LAYERS || net->widths[0] != 2)
    return fail(XPINN_ERR_INVALID, "bad network description");
  for (int k = 1; k < L; ++k)
    if (net->widths[k] < 1 || net->widths[k] > XPINN_MAX_WIDTH)
      return fail(XPINN_ERR_INVALID, "hidden width outside [1, XPINN_MAX_WIDTH]");
  if (net->widths[L] != (pde == XPINN_PDE_NS ? 3 : 1)) return fail(XPINN_ERR_INVALID, "wrong output count");
  if (net->out_act != XPINN_ACT_IDENTITY && net->out_act != XPINN_ACT_SOFTPLUS)
    return fail(XPINN_ERR_INVALID, "bad out_act");
  if (net->act != XPINN_PHI_TANH && net->act != XPINN_PHI_SIN && net->act != XPINN_PHI_COS)
    return fail(XPINN_ERR_INVALID, "bad act");
  if ((net->adaptive != 0 && net->adaptive != 1) ||
      (net->adaptive && !(net->slope_scale > 0.f && net->slope_scale < 3.0e38f)))
    return fail(XPINN_ERR_INVALID, "bad adaptive slope settings");
  if (pde == XPINN_PDE_NS && !(re > 0)) return fail(XPINN_ERR_INVALID, "Reynolds number must be > 0");
  cudaStream_t s = (cudaStream_t)stream;

  // ---- one-time set-up on this device: the array's device address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return fail(XPINN_ERR_CUDA, "no usable current CUDA device");
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (rc != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(XPINN_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_ptr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_ptr[dev]);
  }

  // ---- the network and its single work kind (residual points)
  NaDesc d;
  memset(&d, 0, sizeof d);
  SubDev& sd = d.sd;
  sd.n_nets = 1;
  NetDev& nd = sd.net[0];
  const int off = fill_net_dev(nd, *net, 0);
  sd.img_off = 0;
  const int img_floats = assign_images(nd, 0);
  d.n_pack = 0;
  for (int k = 2; k < L; ++k) {
    d.pack[d.n_pack++] = {nd.off[k], nd.imf[k], nd.w[k - 1], nd.w[k], nd.wp[k - 1], nd.wp[k], 1};
    d.pack[d.n_pack++] = {nd.off[k], nd.imb[k], nd.w[k - 1], nd.w[k], nd.wp[k - 1], nd.wp[k], 0};
  }
  int wmax = MT;
  for (int k = 1; k < L; ++k) wmax = std::max(wmax, nd.wp[k]);
  sd.n_params = off;
  sd.w_res = w_res;
  sd.n_res = (int)n;
  sd.inv_n_res = n ? 1.f / (float)n : 0.f;
  // (u, u_x, u_t, u_xx) for Burgers, Laplacian jets (u, u_x, u_y, lap u) otherwise
  const int K = 4;
  const int D = nd.w[L];
  int P = std::min(256, (NT / (wmax / MT)) * 2);
  P = std::min(P, std::max(4, 2048 / (D * K)));
  P = std::max(4, P / 4 * 4);
  int64_t rows = 0;
  for (int k = 1; k < L; ++k) rows += nd.wp[k];
  const int64_t per_cta = (rows + D) * K * P;

  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(XPINN_ERR_CUDA, "cudaDeviceGetAttribute failed");
  }
  // items of whole sub-tiles; as many CTAs as fit the array
  const int64_t tiles = (n + P - 1) / P;
  int n_items = (int)std::min<int64_t>(std::min<int64_t>(NA_MAX_ITEMS, tiles), (int64_t)n_sm);
  int grid = n_items;
  NaLayout lay = layout(n_items, sd.n_params, grid, per_cta, img_floats);
  while (n_items > 1 && lay.total > (size_t)XPINN_NOALLOC_SCRATCH_BYTES) {
    n_items = std::max(1, n_items * 3 / 4);
    grid = n_items;
    lay = layout(n_items, sd.n_params, grid, per_cta, img_floats);
  }
  if (lay.total > (size_t)XPINN_NOALLOC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "needs %zu bytes of scratch, more than the built-in maximum of %d bytes "
             "(XPINN_NOALLOC_SCRATCH_BYTES)", lay.total, XPINN_NOALLOC_SCRATCH_BYTES);
    return fail(XPINN_ERR_UNSUPPORTED, buf);
  }
  const int64_t per_item = n_items ? (tiles + n_items - 1) / n_items * P : 0;
  d.n_items = 0;
  for (int64_t s0 = 0; s0 < n; s0 += per_item) {
    Item& it = d.items[d.n_items];
    it.kind = IT_RES;
    it.q = 0;
    it.edge = -1;
    it.pt_off = s0;
    it.n_pts = (int)std::min<int64_t>(per_item, n - s0);
    it.P = P;
    it.K[0] = K;
    it.lap = pde == XPINN_PDE_BURGERS ? 0 : 1;
    it.part_off = (int64_t)d.n_items * sd.n_params;
    ++d.n_items;
  }

  StepArgs a;
  memset(&a, 0, sizeof a);
  a.items = reinterpret_cast<const Item*>(base + lay.items);
  a.n_items = d.n_items;
  a.item_base = 0;
  a.counter = reinterpret_cast<int*>(base + lay.counter);
  a.subs = reinterpret_cast<const SubDev*>(base + lay.sub);
  a.params = params;
  a.wimg = reinterpret_cast<const float*>(base + lay.img);
  a.pts = reinterpret_cast<const float2*>(xy);
  a.res_f = f;
  a.partials = reinterpret_cast<float*>(base + lay.partials);
  a.loss_part = reinterpret_cast<double*>(base + lay.loss_part);
  a.scratch = reinterpret_cast<float*>(base + lay.scratch);
  a.scratch_per_cta = per_cta;
  a.pde = pde;
  a.nu = nu;
  a.re = re;
  a.n_out_total = D;
  a.n_eq = pde == XPINN_PDE_NS ? 3 : 1;
  a.szA = wmax * adj_stride(K, P);
  a.szW = 4;
  for (int k = 2; k < L; ++k) a.szW = std::max(a.szW, layer_img_floats(nd, k));
  a.szU = (D * K * P + 3) / 4 * 4;
  a.pmax = P;
  a.pt = 2;
  a.nt = NT;
  a.gen = net_is_general(nd) ? 1 : 0;
  a.err = reinterpret_cast<int*>(base + lay.err);
  const size_t smem = jet_step_smem_bytes(a);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the dynamic limit plus the kernel's static shared memory must stay within
  // the opt-in maximum; 1 KB is left for the static part, as handles do
  const size_t limit = optin > 1024 ? (size_t)optin - 1024 : 0;
  if (smem > limit) return fail(XPINN_ERR_UNSUPPORTED, "network too wide for shared memory");
  // raise the kernel's shared-memory limit to that maximum (never lower it:
  // handles created earlier rely on the limit they set, which is below it)
  if (jet_step_configure(limit) != cudaSuccess) {
    cudaGetLastError();
    return fail(XPINN_ERR_CUDA, "cudaFuncSetAttribute failed");
  }

  na_setup_kernel<<<1, 128, 0, s>>>(d, reinterpret_cast<SubDev*>(base + lay.sub),
                                    reinterpret_cast<Item*>(base + lay.items),
                                    reinterpret_cast<int*>(base + lay.counter),
                                    reinterpret_cast<int*>(base + lay.err),
                                    reinterpret_cast<PackBlock*>(base + lay.pack));
  launch_pack_weights(params, reinterpret_cast<const PackBlock*>(base + lay.pack), d.n_pack,
                      reinterpret_cast<float*>(base + lay.img), s);
  if (d.n_items) launch_jet_step(a, grid, smem, s);
  na_reduce_kernel<<<(sd.n_params + 255) / 256, 256, 0, s>>>(a.partials, a.loss_part, d.n_items,
                                                              sd.n_params, grads, loss);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(XPINN_ERR_CUDA, cudaGetErrorString(e));
  return XPINN_OK;
}
