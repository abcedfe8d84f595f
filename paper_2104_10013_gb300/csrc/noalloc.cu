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
// The pieces that must start at zero (the work counter and the error word)
// are cleared by every call on its stream.  Calls whose kernels overlap on
// the GPU (different streams, or different threads without ordering) race on
// the array and give wrong results: order them on one stream.
//
// Errors on the device: the jet kernel's waits are bounded and set the error
// word when they give up; the call has already returned by then, so the last
// kernel writes NaN to the loss and to every gradient element instead of a
// sum that may include slices an earlier call left in the array.
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

constexpr int NA_MAX_ITEMS = 256;     // work items (and gradient slices) per call; one per CTA
constexpr int NA_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[XPINN_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_ptr[NA_MAX_DEVICES] = {};
thread_local int g_preset_err = 0;    // testing: the next call's initial error word

struct NaDesc {
  SubDev sd;
  Item items[NA_MAX_ITEMS];
  int n_items;
  PackBlock pack[2 * MAXL];   // weight images of the hidden-to-hidden layers
  int n_pack;
};
// passed to na_setup_kernel by value: within the 32,764 bytes of kernel parameters
static_assert(sizeof(NaDesc) <= 32000, "descriptor too large for a kernel parameter");

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
// work counter and the error word: the only state that must start at zero
// (err0 is 0 except in the testing hook xpinn_noalloc_debug_preset_error).
__global__ void na_setup_kernel(NaDesc d, SubDev* sub, Item* items, int* counter, int* err, int err0,
                                PackBlock* pack) {
  const int t = threadIdx.x;
  if (t == 0) {
    *sub = d.sd;
    *counter = 0;
    *err = err0;
  }
  for (int i = t; i < d.n_items; i += blockDim.x) items[i] = d.items[i];
  for (int i = t; i < d.n_pack; i += blockDim.x) pack[i] = d.pack[i];
}

// grads[e] = sum over items (in order) of the item's slice; loss = sum of the
// items' residual sums (each already divided by n).  If the jet kernel set the
// error word (a bounded wait gave up, so some slices were never written), the
// outputs are NaN instead: the call is asynchronous and cannot return the
// error, and a stale sum from an earlier call must not pass for a result.
__global__ void na_reduce_kernel(const float* __restrict__ partials, const double* __restrict__ loss_part,
                                 int n_items, int n_params, const int* __restrict__ err,
                                 float* __restrict__ grads, float* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = *reinterpret_cast<const volatile int*>(err) != 0;
  if (e < n_params) {
    float g = 0.f;
    for (int i = 0; i < n_items; ++i) g += partials[(size_t)i * n_params + e];
    grads[e] = bad ? __int_as_float(0x7fc00000) : g;
  }
  if (e == 0) {
    double s = 0.0;
    for (int i = 0; i < n_items; ++i) s += loss_part[2 * i];
    *loss = bad ? __int_as_float(0x7fc00000) : (float)s;
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
  sd.n_params = off;
  sd.w_res = w_res;
  sd.n_res = (int)n;
  sd.inv_n_res = n ? 1.f / (float)n : 0.f;
  // (u, u_x, u_t, u_xx) for Burgers, Laplacian jets (u, u_x, u_y, lap u) otherwise
  const int D = nd.w[L];
  Item proto;
  memset(&proto, 0, sizeof proto);
  proto.kind = IT_RES;
  proto.edge = -1;
  proto.K[0] = 4;
  proto.lap = pde == XPINN_PDE_BURGERS ? 0 : 1;

  int n_sm = 0, optin = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(XPINN_ERR_CUDA, "cudaDeviceGetAttribute failed");
  }
  // the dynamic limit plus the kernel's static shared memory must stay within
  // the opt-in maximum; 1 KB is left for the static part, as handles do
  const size_t limit = optin > 1024 ? (size_t)optin - 1024 : 0;
  // Sub-tile size and shared memory as the handle's planner sizes them
  // (choose_P, item_needs): the largest P the register tiles occupy, lowered
  // in steps of 4 (down to 8) while the shared memory does not fit.
  StepArgs a;
  memset(&a, 0, sizeof a);
  a.pt = 2;
  a.nt = NT;
  a.gen = net_is_general(nd) ? 1 : 0;
  Limits lim;
  size_t smem = 0;
  for (int cap = 256;; cap -= 4) {
    proto.P = choose_P(sd, proto.K, cap, a.pt, a.nt);
    lim = Limits{};
    item_needs(sd, proto, lim);
    a.szA = round_up4(lim.szA);
    a.szW = round_up4(lim.szW);
    a.szU = round_up4(lim.szU);
    a.pmax = round_up4(lim.pmax);
    smem = jet_step_smem_bytes(a);
    if (smem <= limit || cap <= 8) break;
  }
  if (smem > limit) return fail(XPINN_ERR_UNSUPPORTED, "network too wide for shared memory");
  const int P = proto.P;
  const int64_t per_cta = round_up4((int)lim.scratch);

  // items of whole sub-tiles, one per CTA, at most one CTA per SM; fewer
  // when the working set does not fit the array
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
    it = proto;
    it.pt_off = s0;
    it.n_pts = (int)std::min<int64_t>(per_item, n - s0);
    it.part_off = (int64_t)d.n_items * sd.n_params;
    ++d.n_items;
  }

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
  a.err = reinterpret_cast<int*>(base + lay.err);
  // raise the kernel's shared-memory limit to the opt-in maximum (never lower
  // it: handles created earlier rely on the limit they set, which is below it)
  if (jet_step_configure(limit) != cudaSuccess) {
    cudaGetLastError();
    return fail(XPINN_ERR_CUDA, "cudaFuncSetAttribute failed");
  }

  const int err0 = g_preset_err;
  g_preset_err = 0;
  na_setup_kernel<<<1, 128, 0, s>>>(d, reinterpret_cast<SubDev*>(base + lay.sub),
                                    reinterpret_cast<Item*>(base + lay.items),
                                    reinterpret_cast<int*>(base + lay.counter),
                                    reinterpret_cast<int*>(base + lay.err), err0,
                                    reinterpret_cast<PackBlock*>(base + lay.pack));
  launch_pack_weights(params, reinterpret_cast<const PackBlock*>(base + lay.pack), d.n_pack,
                      reinterpret_cast<float*>(base + lay.img), s);
  if (d.n_items) launch_jet_step(a, grid, smem, s);
  na_reduce_kernel<<<(sd.n_params + 255) / 256, 256, 0, s>>>(a.partials, a.loss_part, d.n_items,
                                                              sd.n_params, a.err, grads, loss);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(XPINN_ERR_CUDA, cudaGetErrorString(e));
  return XPINN_OK;
}

extern "C" int xpinn_noalloc_debug_preset_error(int32_t code) {
  g_preset_err = code;
  set_last_error("");
  return XPINN_OK;
}
