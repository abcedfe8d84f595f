// C ABI of the cPINN / XPINN library (declared in include/xpinn.h).
//
// xpinn_create copies the problem to the device and plans the step: it cuts
// every subdomain's point sets into work items of similar cost, sizes shared
// memory and per-CTA scratch, and lays out the gradient slices.  A training
// step (Algorithm 1) is then four launches on one stream, replayed from a
// CUDA graph:
//   step_begin   reset work counters, advance the Adam step and loss slot
//   jet kernel   interface sides, forward only: fills the exchange buffer
//   jet kernel   all residual / data / interface items: jets, loss, reverse
//   reduce_adam  fixed-order sum of the gradient slices, Adam per subdomain
// The per-subdomain loop schedule launches the same kernels once per
// subdomain and phase instead (the baseline the grouped launch replaces).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "eval_tc.h"
#include "step_tc.h"
#include "xpinn_dev.cuh"

namespace xp {
void launch_route(const float2* pts, int64_t n, const SubDev* subs, int q0, int nq, int* S, int* memb,
                  int* counts, int* err, const float2* poly, int n_poly, cudaStream_t st);
void launch_bucket(const float2* pts, int64_t n, const int* S, const int* memb, int* cursor, int* pos,
                   float2* epts, float* escale, cudaStream_t st);
void launch_gather(int64_t n, int row, const int* S, const int* pos, const float* eout, float* out,
                   cudaStream_t st);
void launch_eval_plan(const int* counts, int nq, const EvalProto* proto, int q0, int row, int* cursor,
                      Item* items, int* n_items, int max_items, int* err, cudaStream_t st);
}  // namespace xp

using namespace xp;

namespace {

thread_local std::string g_err;

}  // namespace

namespace xp {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace xp

namespace {

struct Error {
  int code;
};

[[noreturn]] void fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  throw Error{code};
}

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? XPINN_ERR_OOM : XPINN_ERR_CUDA, "%s: %s", what,
         cudaGetErrorString(e));
  }
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  bool owned = true;   // false: a view into memory someone else owns (a caller's workspace)
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p && owned) cudaFree(p);
    p = nullptr;
    n = 0;
    owned = true;
  }
  void view(void* ptr, size_t count) {
    release();
    p = static_cast<T*>(ptr);
    n = count;
    owned = false;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    ck(cudaMalloc(&p, count * sizeof(T)), "cudaMalloc");
    n = count;
  }
  void ensure(size_t count) {
    if (count > n) alloc(count);
  }
  void upload(const T* src, size_t count, cudaStream_t s = 0) {
    alloc(count);
    if (count) ck(cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
  }
};

bool is_device_ptr(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Jet components at residual points.  Burgers needs (u, u_x, u_t, u_xx);
// Poisson, Navier-Stokes and the diffusion u-network need only the Laplacian
// of their second derivatives, carried as one component (Laplacian jets,
// see jet_step.cuh); the diffusion K-network needs (K, K_x, K_y).
int k_res(int pde, int net) {
  if (pde == XPINN_PDE_DIFFUSION) return net == 0 ? 4 : 3;
  return net == 0 ? 4 : 0;
}
// Net 0 of an item with 4 components carries the Laplacian unless the PDE is Burgers.
int lap_of(int pde, int K0) { return K0 == 4 && pde != XPINN_PDE_BURGERS ? 1 : 0; }
int k_iface(int pde, int method, int net) {
  if (method == XPINN_XPINN) return k_res(pde, net);
  if (pde == XPINN_PDE_BURGERS) return net == 0 ? 2 : 0;
  if (pde == XPINN_PDE_DIFFUSION) return 3;
  return net == 0 ? 3 : 0;
}

}  // namespace

struct Plan {
  std::vector<Item> items;       // [0, n_fwd): exchange items; then the main items
  int n_fwd = 0;
  int first_iface = 0;           // first item that reads the exchange buffer
  std::vector<int> q_items, q_item_begin;
  std::vector<int64_t> q_part_off;
  std::vector<int2> red_blocks;
  // per-subdomain ranges (loop schedule)
  std::vector<int> fwd_begin, main_begin;   // [n_sub + 1], relative to n_fwd for main
  int64_t partial_floats = 0;
  // residual items of the tensor-core kernel (step_tc.cu): the last n_tc
  // items; tc_begin [n_sub + 1] ranges per subdomain (loop schedule),
  // relative to the first of them
  int n_tc = 0;
  std::vector<int> tc_begin;
  int n_simt() const { return (int)items.size() - n_tc; }
  // threads that share one parameter's slice sum in the reduction (1-8): each
  // takes a contiguous run of at most about 8 of the subdomain's items
  int red_split = 1;
};

struct xpinn_ctx {
  // problem
  int pde = 0, flux_mode = 0;
  float nu = 0, re = 1, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  int n_sub = 0, n_iface = 0, spm = 0;
  std::vector<SubDev> subs;
  std::vector<IfaceDev> ifaces;
  // a fork (xpinn_fork_step) trains only some of its subdomains: the others
  // only provide their interface values; empty = every subdomain is trained
  std::vector<char> trained;
  // per-subdomain cap on the points of a sub-tile (0: none), chosen per shape
  // class by xpinn_autotune_shapes; empty = none
  std::vector<int> tile_cap;
  // per-subdomain choice of the tensor-core kernel for its residual items
  // (1 on, 0 off, -1 the default rule), chosen per shape class by
  // xpinn_autotune_shapes; empty = the default rule everywhere
  std::vector<int> tc_sel;
  int64_t n_params = 0, n_res_total = 0, n_pts_total = 0, n_if_pts = 0;
  int n_out_total = 0, n_eq = 1, d4_nv = 0;
  // device problem
  DevBuf<float> params, m, v, grads, res_f, tgt, d4, partials, scratch, loss_ring;
  DevBuf<float> jq;              // [n_sub + 1]: J(Theta_q) of the last step or grad, then their sum
  DevBuf<float2> pts, poly;
  int n_poly = 0;
  DevBuf<SubDev> subs_d;
  DevBuf<IfaceDev> ifaces_d;
  DevBuf<double> loss_part;
  DevBuf<Item> items_d;
  DevBuf<int> q_items_d, q_item_begin_d, counters, state_i, err_d;
  DevBuf<int64_t> q_part_off_d;
  DevBuf<int2> red_blocks_d;
  // weight images (see NetDev): rebuilt from params at the start of every
  // step and before an evaluation when params changed since the last build
  DevBuf<float> wimg;
  DevBuf<PackBlock> pack_d;
  std::vector<PackBlock> pack_h;
  int64_t n_img = 0;
  bool img_stale = true;
  // eval
  DevBuf<float2> e_pts;
  DevBuf<float> e_out;
  DevBuf<Item> e_items;
  DevBuf<char> e_ws;             // workspace of xpinn_eval (grown by that call only)
  // routed evaluation: per subdomain, how its bucket is cut into items, for
  // derivative orders 0, 1, 2 ([3][n_sub]); rebuilt with the plan
  DevBuf<EvalProto> e_proto;
  std::vector<int> e_min_chunk;  // [3][n_models]: smallest chunk of each model and order
  // tensor-core evaluation (eval_tc.cu, option eval_tensor_cores): per model
  // the hidden width its networks qualify with (0: the jet kernel evaluates
  // it), and the weight images, rebuilt from params like wimg
  std::vector<int> tc_w;         // [n_models], empty until first needed
  DevBuf<float> tc_img;
  DevBuf<int64_t> tc_off;        // [n_sub] first float of a subdomain's images, -1: none
  DevBuf<TcPack> tc_pack_d;
  int n_tc_pack = 0;
  bool tc_stale = true;
  // tensor-core training (step_tc.cu, option train_tensor_cores): weight
  // images of the qualifying subdomains (forward and reverse of every
  // hidden-to-hidden layer), rebuilt at the start of every step, and the
  // kernel's per-CTA scratch
  DevBuf<float> tct_img, tct_scratch;
  DevBuf<int64_t> tct_off;       // [n_sub] first float of a subdomain's images, -1: none
  DevBuf<TcTrainPack> tct_pack_d;
  int n_tct_pack = 0;
  int tct_grid = 0;
  int tct_gen = 0;               // 1: some of those networks need the general activation rules
  // device time of the evaluation kernel of the last routed evaluation
  // (profile_phases): events around its launch
  cudaEvent_t eval_ev[2] = {};
  bool eval_timed = false;
  // plan
  Plan plan;
  StepArgs base{};
  size_t smem = 0;
  int n_sm = 0, grid = 0;
  int ring_cap = 256;
  int host_t = 0, host_slot = 0;
  // train_tensor_cores 33: hidden widths 33..64 qualify (below 33 the zero-padding to 64 more than
  // quadruples the tensor work; the shape tuner decides per class above that)
  xpinn_options opt{0, 1, 4, 2, 0, 0, 256, 0, 1, 33};
  int device = 0;
  cudaEvent_t ev[6] = {};         // phase marks 0-4, and 5 after the tensor-core kernel
  bool tc_timed = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;        // one training step
  cudaGraphExec_t graph_multi = nullptr;  // GRAPH_STEPS training steps back to back
  int n_counters = 0;
  int p_cap = 256;
  bool step_open = false;        // xpinn_step_begin called, xpinn_step_end pending
  DevBuf<int> e_counter;

  ~xpinn_ctx() {
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_multi) cudaGraphExecDestroy(graph_multi);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : eval_ev)
      if (e) cudaEventDestroy(e);
  }

  int* step_t() { return state_i.p; }
  int* loss_slot() { return state_i.p + 1; }
  float* step_bc() { return reinterpret_cast<float*>(state_i.p + 2); }   // [2] bias corrections
};

// Facts of a handle for the request server.
namespace xp {
int ctx_out_total(xpinn_handle h) { return h->n_out_total; }
int ctx_n_sub(xpinn_handle h) { return h->n_sub; }
int ctx_n_copies(xpinn_handle h) { return h->n_sub / h->spm; }
int ctx_device(xpinn_handle h) { return h->device; }
int ctx_sub_params(xpinn_handle h, int q) { return h->subs[q].n_params; }
int* ctx_err_word(xpinn_handle h) { return h->err_d.p; }
}  // namespace xp

namespace {

// ---------------------------------------------------------------------------
// Validation and packing
// ---------------------------------------------------------------------------
void validate_net(const xpinn_net_desc& n, int pde, int net_idx, int q) {
  if (n.n_layers < 2 || n.n_layers > XPINN_MAX_LAYERS)
    fail(n.n_layers < 2 ? XPINN_ERR_INVALID : XPINN_ERR_UNSUPPORTED,
         "subdomain %d net %d: n_layers %d outside [2, %d]", q, net_idx, n.n_layers, XPINN_MAX_LAYERS);
  if (n.widths[0] != 2) fail(XPINN_ERR_INVALID, "subdomain %d net %d: widths[0] must be 2", q, net_idx);
  for (int k = 1; k < n.n_layers; ++k)
    if (n.widths[k] < 1 || n.widths[k] > XPINN_MAX_WIDTH)
      fail(n.widths[k] < 1 ? XPINN_ERR_INVALID : XPINN_ERR_UNSUPPORTED,
           "subdomain %d net %d: hidden width %d outside [1, %d]", q, net_idx, n.widths[k], XPINN_MAX_WIDTH);
  const int D = n.widths[n.n_layers];
  int want = 1;
  if (pde == XPINN_PDE_NS) want = 3;
  if (D != want) fail(XPINN_ERR_INVALID, "subdomain %d net %d: %d outputs, this PDE needs %d", q, net_idx, D, want);
  if (n.out_act != XPINN_ACT_IDENTITY && n.out_act != XPINN_ACT_SOFTPLUS)
    fail(XPINN_ERR_INVALID, "subdomain %d net %d: bad out_act %d", q, net_idx, n.out_act);
  if (n.act != XPINN_PHI_TANH && n.act != XPINN_PHI_SIN && n.act != XPINN_PHI_COS)
    fail(XPINN_ERR_INVALID, "subdomain %d net %d: bad act %d", q, net_idx, n.act);
  if (n.adaptive != 0 && n.adaptive != 1)
    fail(XPINN_ERR_INVALID, "subdomain %d net %d: adaptive must be 0 or 1", q, net_idx);
  if (n.adaptive && !(n.slope_scale > 0.f && n.slope_scale < 3.0e38f))
    fail(XPINN_ERR_INVALID, "subdomain %d net %d: slope_scale must be finite and > 0", q, net_idx);
}

void check_finite(const float* a, int64_t n, const char* what) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) fail(XPINN_ERR_INVALID, "%s[%lld] is not finite", what, (long long)i);
}

// ---------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------
int round_up(int x, int m) { return (x + m - 1) / m * m; }

int cta_threads(const xpinn_ctx* h) {
  const int t = h->opt.threads_per_cta;
  return (t == 128 || t == 512) ? t : 256;
}

size_t smem_of(const Limits& l, int gen) {
  StepArgs a{};
  a.gen = gen;
  a.szA = round_up(l.szA, 4);
  a.szW = round_up(l.szW, 4);
  a.szU = round_up(l.szU, 4);
  a.pmax = round_up(l.pmax, 4);
  return jet_step_smem_bytes(a);
}

// Fraction of the CTA's threads the weight-gradient tiles of an out_p x in_p
// layer keep busy: 8 x 4 tiles, the contraction split S ways (a power of two
// up to 16, S threads of a tile in one warp), as the kernel assigns them.
double dw_busy(int out_p, int in_p, int nt) {
  const int T = (in_p / 4) * (out_p / MT);
  if (T <= 0) return 1.0;
  int S = nt / T;
  S = S >= 16 ? 16 : (S >= 8 ? 8 : (S >= 4 ? 4 : (S >= 2 ? 2 : 1)));
  const int per_pass = (nt / 32) * (32 / S);
  const int passes = (T + per_pass - 1) / per_pass;
  return (double)T * S / ((double)passes * nt);
}

// Modelled time of an item (about ns on one SM): per point, the three
// contractions of every hidden layer with padded widths (the weight-gradient
// one divided by its thread occupancy), scaled by the jet components, plus a
// fixed cost per layer and sub-tile (barriers, activation passes, the first
// and output layers) spread over the sub-tile's P points, plus a fixed cost
// per item.  The coefficients were fitted to the measured time per point of
// sixteen shapes (widths 25-80, depths 4-6) run alone: within 20%, where a
// count of true-width multiply-adds was off by up to a factor of 2.3.
double item_cost(const SubDev& sd, const Item& it, int nt) {
  const bool fwd_only = it.kind == IT_IFACE_FWD || it.kind == IT_EVAL;
  double c = 0;
  for (int n = 0; n < sd.n_nets; ++n) {
    if (!it.K[n]) continue;
    const NetDev& nd = sd.net[n];
    double con = 0;
    for (int k = 2; k < nd.L; ++k) {
      con += (double)nd.wp[k] * nd.w[k - 1];
      if (!fwd_only)
        con += (double)nd.w[k] * nd.wp[k - 1] + (double)nd.wp[k] * nd.wp[k - 1] / dw_busy(nd.wp[k], nd.wp[k - 1], nt);
    }
    con += (double)nd.w[nd.L] * nd.w[nd.L - 1] * (fwd_only ? 1 : 3);
    c += 2.35e-4 * con * it.K[n] / 4.0 + 47.5 * nd.L / std::max(1, it.P) * (fwd_only ? 0.4 : 1.0);
  }
  return c * it.n_pts + 3000.0;
}

// Build items for the training step.  `schedule` 0 orders them by cost
// (largest first) for the grouped launch, 1 groups them by subdomain.
void build_plan(xpinn_ctx* h, int p_cap) {
  Plan pl;
  std::vector<Item> fwd, main_;
  auto mk = [&](int kind, int q, int edge, int side, int64_t off, int n, int K0, int K1) {
    Item it{};
    it.kind = kind;
    it.q = q;
    it.edge = edge;
    it.side = side;
    it.pt_off = off;
    it.n_pts = n;
    it.K[0] = K0;
    it.K[1] = K1;
    it.lap = lap_of(h->pde, K0);
    const int qcap = (h->tile_cap.empty() || h->tile_cap[q] <= 0) ? p_cap : std::min(p_cap, h->tile_cap[q]);
    it.P = choose_P(h->subs[q], it.K, qcap, h->opt.points_per_thread, cta_threads(h));
    it.part_off = -1;
    return it;
  };
  // subdomains whose residual items run on the tensor-core kernel
  std::vector<char> tcq(h->n_sub, 0);
  double tc_total = 0;
  bool any_tc = false;
  int64_t tc_pts = 0;
  for (int q = 0; q < h->n_sub; ++q) {
    const SubDev& sd = h->subs[q];
    const int sel = h->tc_sel.empty() ? -1 : h->tc_sel[q];
    if (sel != 0 && sd.n_res && step_tc_net_ok(sd.net[0], sd.n_nets, h->pde, h->opt.train_tensor_cores)) {
      tcq[q] = sel == 1 ? 2 : 1;   // 2: chosen for this subdomain, 1: by the default rule
      tc_pts += sd.n_res;
    }
  }
  // default rule: the tensor-core kernel runs before the jet kernel, so it
  // pays off only when it takes over most of the step, at least half of the
  // residual points; subdomains chosen explicitly keep it regardless
  if (2 * tc_pts < h->n_res_total)
    for (auto& t : tcq)
      if (t == 1) t = 0;
  for (int q = 0; q < h->n_sub; ++q)
    if (tcq[q]) {
      any_tc = true;
      tc_total += (double)h->subs[q].n_res * (h->subs[q].net[0].L - 1);
    }
  // first pass: one item per point set, to estimate the total cost (with
  // tensor-core residual items, of everything the jet kernel still runs)
  double total = 0;
  for (int q = 0; q < h->n_sub; ++q) {
    const SubDev& sd = h->subs[q];
    if (sd.n_res && !tcq[q]) {
      Item it = mk(IT_RES, q, -1, 0, sd.res_off, sd.n_res, k_res(h->pde, 0), sd.n_nets > 1 ? k_res(h->pde, 1) : 0);
      total += item_cost(sd, it, cta_threads(h));
    }
    if (any_tc)
      for (int n = 0; n < sd.n_nets; ++n)
        if (sd.n_data[n])
          total += item_cost(sd, mk(n == 0 ? IT_DATA0 : IT_DATA1, q, -1, 0, sd.data_off[n], sd.n_data[n],
                                    n == 0 ? 1 : 0, n == 1 ? 1 : 0),
                             cta_threads(h));
  }
  if (any_tc)
    for (int e = 0; e < h->n_iface; ++e) {
      const IfaceDev& f = h->ifaces[e];
      for (int side = 0; side < 2 && f.n_pts; ++side) {
        const int q = side ? f.qp : f.q;
        total += 2 * item_cost(h->subs[q],
                               mk(IT_IFACE, q, e, side, f.pt_off, f.n_pts, k_iface(h->pde, f.method, 0),
                                  h->subs[q].n_nets > 1 ? k_iface(h->pde, f.method, 1) : 0),
                               cta_threads(h));
      }
    }
  const double target = std::max(1.0, total / (double)(h->grid * std::max(1, h->opt.items_per_cta)));
  auto split = [&](Item proto, std::vector<Item>& out) {
    const SubDev& sd = h->subs[proto.q];
    const double c = item_cost(sd, proto, cta_threads(h));
    int chunks = std::max(1, (int)std::lround(c / target));
    int per = (proto.n_pts + chunks - 1) / chunks;
    per = std::max(proto.P, (per + proto.P - 1) / proto.P * proto.P);
    for (int s = 0; s < proto.n_pts; s += per) {
      Item it = proto;
      it.pt_off = proto.pt_off + s;
      it.n_pts = std::min(per, proto.n_pts - s);
      out.push_back(it);
    }
  };
  // tensor-core items: whole tiles of STC_PTS points, about tc_ipc items per
  // CTA of its launch (one CTA per SM), cost ~ points x layers
  std::vector<Item> tcv;
  constexpr int tc_ipc = 8;
  const double tc_target = tc_total / (double)(std::max(1, h->n_sm) * tc_ipc);
  for (int q = 0; q < h->n_sub; ++q) {
    const SubDev& sd = h->subs[q];
    const int K1 = sd.n_nets > 1 ? k_res(h->pde, 1) : 0;
    if (sd.n_res && tcq[q]) {
      Item proto = mk(IT_RES, q, -1, 0, sd.res_off, sd.n_res, 4, 0);
      proto.P = STC_PTS;
      // grouped: about tc_ipc items per CTA over the whole launch; loop
      // schedule: each subdomain's own launch gets two items per SM
      int per = h->opt.schedule == 1 ? (int)std::ceil(sd.n_res / (2.0 * std::max(1, h->n_sm)))
                                     : (int)std::ceil(tc_target / (sd.net[0].L - 1));
      per = std::max(4 * STC_PTS, (per + STC_PTS - 1) / STC_PTS * STC_PTS);
      const int chunks = (sd.n_res + per - 1) / per;
      per = ((sd.n_res + chunks - 1) / chunks + STC_PTS - 1) / STC_PTS * STC_PTS;
      for (int s0 = 0; s0 < sd.n_res; s0 += per) {
        Item it = proto;
        it.pt_off = proto.pt_off + s0;
        it.n_pts = std::min(per, sd.n_res - s0);
        tcv.push_back(it);
      }
    } else if (sd.n_res) {
      split(mk(IT_RES, q, -1, 0, sd.res_off, sd.n_res, k_res(h->pde, 0), K1), main_);
    }
    for (int n = 0; n < sd.n_nets; ++n)
      if (sd.n_data[n])
        split(mk(n == 0 ? IT_DATA0 : IT_DATA1, q, -1, 0, sd.data_off[n], sd.n_data[n], n == 0 ? 1 : 0,
                 n == 1 ? 1 : 0),
              main_);
  }
  auto is_trained = [&](int q) { return h->trained.empty() || h->trained[q] != 0; };
  for (int e = 0; e < h->n_iface; ++e) {
    const IfaceDev& f = h->ifaces[e];
    if (!f.n_pts) continue;
    for (int side = 0; side < 2; ++side) {
      const int q = side ? f.qp : f.q;
      const int K0 = k_iface(h->pde, f.method, 0);
      const int K1 = h->subs[q].n_nets > 1 ? k_iface(h->pde, f.method, 1) : 0;
      if (side == 1 && f.remote) continue;   // that side is computed by its own rank
      split(mk(IT_IFACE_FWD, q, e, side, f.pt_off, f.n_pts, K0, K1), fwd);
      if (is_trained(q)) split(mk(IT_IFACE, q, e, side, f.pt_off, f.n_pts, K0, K1), main_);
    }
  }
  // Grouped: largest first, but items that read the exchange buffer last (in
  // one launch they wait for the exchange items, which come first).  Loop:
  // by subdomain, then the same order.  Within a subdomain both orders agree,
  // so both schedules sum the gradient slices identically.
  auto order = [&](std::vector<Item>& v) {
    auto key = [&](const Item& a, const Item& b) {
      const bool ia = a.kind == IT_IFACE, ib = b.kind == IT_IFACE;
      if (ia != ib) return ib;
      return item_cost(h->subs[a.q], a, cta_threads(h)) > item_cost(h->subs[b.q], b, cta_threads(h));
    };
    if (h->opt.schedule == 0) {
      std::stable_sort(v.begin(), v.end(), key);
    } else {
      std::stable_sort(v.begin(), v.end(), [&](const Item& a, const Item& b) {
        if (a.q != b.q) return a.q < b.q;
        return key(a, b);
      });
    }
  };
  order(fwd);
  order(main_);
  {
    auto tc_cost = [&](const Item& a) { return (double)a.n_pts * (h->subs[a.q].net[0].L - 1); };
    std::stable_sort(tcv.begin(), tcv.end(), [&](const Item& a, const Item& b) {
      if (h->opt.schedule == 1 && a.q != b.q) return a.q < b.q;
      return tc_cost(a) > tc_cost(b);
    });
  }
  pl.n_fwd = (int)fwd.size();
  pl.first_iface = pl.n_fwd + (int)main_.size();
  for (size_t i = 0; i < main_.size(); ++i)
    if (main_[i].kind == IT_IFACE) {
      pl.first_iface = pl.n_fwd + (int)i;
      break;
    }
  pl.items = fwd;
  pl.items.insert(pl.items.end(), main_.begin(), main_.end());
  pl.items.insert(pl.items.end(), tcv.begin(), tcv.end());
  pl.n_tc = (int)tcv.size();
  // gradient slices and per-subdomain item lists (in item order: deterministic)
  std::vector<std::vector<int>> per_q(h->n_sub);
  for (size_t i = pl.n_fwd; i < pl.items.size(); ++i) {
    Item& it = pl.items[i];
    it.part_off = pl.partial_floats;
    pl.partial_floats += h->subs[it.q].n_params;
    per_q[it.q].push_back((int)i);
  }
  pl.q_item_begin.push_back(0);
  {
    size_t most = 1;
    for (const auto& v : per_q) most = std::max(most, v.size());
    int S = 1;
    while (S < 8 && (most + S - 1) / S > 8) S *= 2;
    pl.red_split = S;
  }
  for (int q = 0; q < h->n_sub; ++q) {
    for (int i : per_q[q]) {
      pl.q_items.push_back(i);
      pl.q_part_off.push_back(pl.items[i].part_off);
    }
    pl.q_item_begin.push_back((int)pl.q_items.size());
    if (is_trained(q))
      for (int e0 = 0; e0 < h->subs[q].n_params; e0 += 256 / pl.red_split) pl.red_blocks.push_back(make_int2(q, e0));
  }
  // per-subdomain ranges for the loop schedule
  pl.fwd_begin.assign(h->n_sub + 1, 0);
  pl.main_begin.assign(h->n_sub + 1, 0);
  pl.tc_begin.assign(h->n_sub + 1, 0);
  if (h->opt.schedule == 1) {
    for (int i = 0; i < pl.n_fwd; ++i) pl.fwd_begin[pl.items[i].q + 1]++;
    for (int i = pl.n_fwd; i < pl.n_simt(); ++i) pl.main_begin[pl.items[i].q + 1]++;
    for (int i = pl.n_simt(); i < (int)pl.items.size(); ++i) pl.tc_begin[pl.items[i].q + 1]++;
    for (int q = 0; q < h->n_sub; ++q) {
      pl.fwd_begin[q + 1] += pl.fwd_begin[q];
      pl.main_begin[q + 1] += pl.main_begin[q];
      pl.tc_begin[q + 1] += pl.tc_begin[q];
    }
  }
  h->plan = std::move(pl);
}

// Shared memory and scratch needs of the plan's items and of evaluation
// items (every network, order 2) under the same sub-tile cap.
Limits limits_of(xpinn_ctx* h, int cap) {
  Limits l;
  for (const Item& it : h->plan.items) item_needs(h->subs[it.q], it, l);
  for (int q = 0; q < h->n_sub; ++q) {
    const SubDev& sd = h->subs[q];
    for (int net = -1; net < sd.n_nets; ++net) {
      Item it{};
      it.kind = IT_EVAL;
      it.q = q;
      it.K[0] = (net <= 0) ? 5 : 0;
      it.K[1] = (net == 1 || (net < 0 && sd.n_nets > 1)) ? 5 : 0;
      it.P = choose_P(sd, it.K, cap, h->opt.points_per_thread, cta_threads(h));
      item_needs(sd, it, l);
    }
  }
  return l;
}

// Does some network need the general activation passes?
int any_general(const xpinn_ctx* h) {
  for (const SubDev& sd : h->subs)
    for (int n = 0; n < sd.n_nets; ++n)
      if (net_is_general(sd.net[n])) return 1;
  return 0;
}

// Weight images, pack list and scratch of the tensor-core residual items:
// per qualifying subdomain the forward images of layers 2..L-1, then their
// reverse images, STC_IMG floats each.
void plan_tc(xpinn_ctx* h) {
  const Plan& pl = h->plan;
  std::vector<int64_t> off(h->n_sub, -1);
  std::vector<TcTrainPack> pk;
  int64_t n = 0;
  int gen = 0;
  for (int i = pl.n_simt(); i < (int)pl.items.size(); ++i) {
    const int q = pl.items[i].q;
    if (off[q] >= 0) continue;
    const SubDev& sd = h->subs[q];
    const NetDev& nd = sd.net[0];
    off[q] = n;
    if (net_is_general(nd)) gen = 1;
    for (int k = 2; k < nd.L; ++k) {
      const int64_t src = sd.poff + nd.off[k];
      pk.push_back({src, n + (int64_t)(k - 2) * STC_IMG, nd.w[k], nd.w[k - 1], 0});
      pk.push_back({src, n + (int64_t)(nd.L - 2 + k - 2) * STC_IMG, nd.w[k], nd.w[k - 1], 1});
    }
    n += (int64_t)2 * (nd.L - 2) * STC_IMG;
  }
  h->n_tct_pack = pl.n_tc ? (int)pk.size() : 0;
  h->tct_gen = gen;
  h->tct_grid = 0;
  if (!pl.n_tc) {
    h->tct_img.release();
    h->tct_scratch.release();
    return;
  }
  h->tct_img.alloc((size_t)n);
  h->tct_off.upload(off.data(), off.size());
  h->tct_pack_d.upload(pk.data(), pk.size());
  h->tct_grid = std::min(h->n_sm, pl.n_tc);
  h->tct_scratch.alloc((size_t)h->tct_grid * STC_SCRATCH);
  ck(step_tc_configure(), "cudaFuncSetAttribute(step_tc smem)");
}

void size_and_upload_plan(xpinn_ctx* h) {
  const Plan& pl = h->plan;
  const Limits l = limits_of(h, h->p_cap);
  StepArgs& a = h->base;
  a.szA = round_up(l.szA, 4);
  a.szW = round_up(l.szW, 4);
  a.szU = round_up(l.szU, 4);
  a.pmax = round_up(l.pmax, 4);
  a.scratch_per_cta = round_up((int)std::min<int64_t>(l.scratch, 1 << 30), 4);
  a.pt = h->opt.points_per_thread;
  a.nt = cta_threads(h);
  a.gen = any_general(h);
  h->smem = jet_step_smem_bytes(a);
  h->items_d.upload(pl.items.data(), pl.items.size());
  h->q_items_d.upload(pl.q_items.data(), pl.q_items.size());
  h->q_item_begin_d.upload(pl.q_item_begin.data(), pl.q_item_begin.size());
  h->q_part_off_d.upload(pl.q_part_off.data(), pl.q_part_off.size());
  h->red_blocks_d.upload(pl.red_blocks.data(), pl.red_blocks.size());
  h->partials.alloc((size_t)pl.partial_floats);
  h->loss_part.alloc(2 * pl.items.size());
  h->scratch.alloc((size_t)h->grid * a.scratch_per_cta);
  // item prototypes of routed evaluations (all networks of a subdomain, K = 1, 3, 5)
  {
    const int n_models = h->n_sub / h->spm;
    std::vector<EvalProto> pr(3 * (size_t)h->n_sub);
    h->e_min_chunk.assign(3 * (size_t)n_models, 1 << 30);
    for (int o = 0; o < 3; ++o)
      for (int q = 0; q < h->n_sub; ++q) {
        const SubDev& sd = h->subs[q];
        const int K = o == 0 ? 1 : (o == 1 ? 3 : 5);
        int Ks[2] = {K, sd.n_nets > 1 ? K : 0};
        EvalProto e;
        e.K0 = Ks[0];
        e.K1 = Ks[1];
        e.P = choose_P(sd, Ks, h->p_cap, h->opt.points_per_thread, cta_threads(h));
        e.chunk = e.P * 16;
        pr[(size_t)o * h->n_sub + q] = e;
        int& mc = h->e_min_chunk[(size_t)o * n_models + q / h->spm];
        mc = std::min(mc, e.chunk);
      }
    h->e_proto.upload(pr.data(), pr.size());
  }
  // [0] main, [1] spare, [2] exchange done, [3, 3 + 2 n_sub) loop counters,
  // then the tensor-core launch's: grouped, and one per subdomain (loop)
  h->n_counters = 4 + 3 * h->n_sub;
  plan_tc(h);
  h->counters.alloc(h->n_counters);
  ck(cudaMemset(h->counters.p, 0, sizeof(int) * h->n_counters), "memset");
  // The limit is a property of the kernel, shared by every handle: raise it to
  // the device maximum (never to this handle's own need, which could lower it
  // below what another handle launches with).
  {
    int optin = 0;
    ck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device), "attr");
    ck(jet_step_configure((size_t)optin - 1024), "cudaFuncSetAttribute(smem)");
  }
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (h->graph_multi) {
    cudaGraphExecDestroy(h->graph_multi);
    h->graph_multi = nullptr;
  }
}

void plan(xpinn_ctx* h) {
  int optin = 0, per_sm = 0;
  ck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device), "attr");
  ck(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device), "attr");
  // one point per thread keeps registers <= 128: two 256-thread CTAs per SM;
  // 128-thread CTAs: twice as many
  const int pt = h->opt.points_per_thread;
  const int nt = cta_threads(h);
  const int per_sm_ctas = nt == 512 ? 1 : (pt == 1 ? 2 : 1) * (256 / nt);
  const size_t budget =
      per_sm_ctas == 1 ? (size_t)optin - 1024 : (size_t)per_sm / per_sm_ctas - 2048;
  int cap = h->opt.max_points_per_tile > 0 ? std::min(256, std::max(8, h->opt.max_points_per_tile)) : 256;
  for (;;) {
    h->grid = h->n_sm * per_sm_ctas;   // provisional, for item sizes
    build_plan(h, cap);
    if (smem_of(limits_of(h, cap), any_general(h)) <= budget || cap <= 8) break;
    cap -= 4;
  }
  h->p_cap = cap;
  size_and_upload_plan(h);
  if (h->smem + 1024 > (size_t)optin)
    fail(XPINN_ERR_UNSUPPORTED, "networks too wide for shared memory (%zu bytes)", h->smem);
  const int bps = jet_step_blocks_per_sm(pt, nt, any_general(h), h->smem);
  if (bps < 1) fail(XPINN_ERR_UNSUPPORTED, "jet kernel does not fit an SM (%zu bytes smem)", h->smem);
  if (h->n_sm * bps != h->grid) {
    // re-plan item sizes and scratch for the grid the occupancy allows
    h->grid = h->n_sm * bps;
    build_plan(h, cap);
    size_and_upload_plan(h);
  }
}

// ---------------------------------------------------------------------------
// Step launches
// ---------------------------------------------------------------------------
StepArgs args_for(xpinn_ctx* h, int begin, int count, int counter_idx) {
  StepArgs a = h->base;
  a.items = h->items_d.p + begin;
  a.n_items = count;
  a.item_base = begin;
  a.counter = h->counters.p + counter_idx;
  a.fwd_done = h->counters.p + 2;
  a.wait_from = 0;
  a.n_fwd_wait = 0;
  return a;
}

// Phase event i on s: an external event node while s is being captured into
// the step graph, a plain record otherwise (calls replayed outside a graph).
void mark(xpinn_ctx* h, int i, cudaStream_t s) {
  if (!h->opt.profile_phases) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ck(cudaStreamIsCapturing(s, &cs), "capture status");
  if (cs == cudaStreamCaptureStatusActive)
    ck(cudaEventRecordWithFlags(h->ev[i], s, cudaEventRecordExternal), "event");
  else
    ck(cudaEventRecord(h->ev[i], s), "event");
}

void pack_images(xpinn_ctx* h, cudaStream_t s) {
  launch_pack_weights(h->params.p, h->pack_d.p, (int)h->pack_h.size(), h->wimg.p, s);
}

// Start of a step and the weight images, one launch.
void step_start(xpinn_ctx* h, bool adam, cudaStream_t s) {
  StepStart a{};
  a.counters = h->counters.p;
  a.n_counters = h->n_counters;
  a.step_t = h->step_t();
  a.loss_slot = h->loss_slot();
  a.bc = h->step_bc();
  a.do_adam = adam ? 1 : 0;
  a.beta1 = h->beta1;
  a.beta2 = h->beta2;
  a.params = h->params.p;
  a.blocks = h->pack_d.p;
  a.n_blocks = (int)h->pack_h.size();
  a.wimg = h->wimg.p;
  launch_step_start(a, s);
}

constexpr int GRAPH_STEPS = 16;   // steps captured in the multi-step graph

// The tensor-core kernel over `count` of its items from plan item `begin`.
void launch_tc(xpinn_ctx* h, int begin, int count, int counter_idx, cudaStream_t s) {
  if (count <= 0) return;
  StepTcArgs a{};
  a.items = h->items_d.p + begin;
  a.n_items = count;
  a.item_base = begin;
  a.counter = h->counters.p + counter_idx;
  a.subs = h->subs_d.p;
  a.params = h->params.p;
  a.img = h->tct_img.p;
  a.img_off = h->tct_off.p;
  a.pts = h->pts.p;
  a.res_f = h->res_f.p;
  a.partials = h->partials.p;
  a.loss_part = h->loss_part.p;
  a.scratch = h->tct_scratch.p;
  a.pde = h->pde;
  a.nu = h->nu;
  a.re = h->re;
  a.gen = h->tct_gen;
  a.err = h->err_d.p;
  launch_step_tc(a, std::min(h->tct_grid, count), s);
}

// The weight images of the tensor-core kernel, from the current parameters.
void pack_tc_train(xpinn_ctx* h, cudaStream_t s) {
  launch_pack_tc_train(h->params.p, h->tct_pack_d.p, h->n_tct_pack, h->tct_img.p, s);
}

// part 0: the whole step.  Part 1: its start and the exchange items only
// (this handle's sides of every interface into the exchange buffer); part 2:
// the rest (residual, data and interface items, reduction and Adam) once the
// remote sides of the exchange buffer have been set (distributed training).
void enqueue_step(xpinn_ctx* h, cudaStream_t s, bool adam, float* grads, int part = 0) {
  const Plan& pl = h->plan;
  if (part == 1) {
    step_start(h, adam, s);
    if (pl.n_fwd) launch_jet_step(args_for(h, 0, pl.n_fwd, 0), std::min(h->grid, pl.n_fwd), h->smem, s);
    ck(cudaGetLastError(), "kernel launch");
    return;
  }
  if (part == 0) {
    mark(h, 0, s);
    step_start(h, adam, s);
  }
  ReduceArgs r{};
  r.blocks = h->red_blocks_d.p;
  r.n_blocks = (int)pl.red_blocks.size();
  r.split = pl.red_split;
  r.subs = h->subs_d.p;
  r.q_items = h->q_items_d.p;
  r.q_item_begin = h->q_item_begin_d.p;
  r.q_part_off = h->q_part_off_d.p;
  r.items = h->items_d.p;
  r.partials = h->partials.p;
  r.loss_part = h->loss_part.p;
  r.params = h->params.p;
  r.m = h->m.p;
  r.v = h->v.p;
  r.grads = grads;
  r.loss_ring = h->loss_ring.p;
  r.ring_cap = h->ring_cap;
  r.loss_slot = h->loss_slot();
  r.step_t = h->step_t();
  r.bc = h->step_bc();
  r.do_adam = adam ? 1 : 0;
  r.beta1 = h->beta1;
  r.beta2 = h->beta2;
  r.eps = h->eps;
  r.n_sub = h->n_sub;
  r.err = h->err_d.p;
  r.jq = h->jq.p;
  const int tc0 = pl.n_simt(), tc_ctr = 3 + 2 * h->n_sub;
  if (part == 2) {
    h->tc_timed = false;
    if (pl.n_tc) {
      pack_tc_train(h, s);
      launch_tc(h, tc0, pl.n_tc, tc_ctr, s);
    }
    const int n_rest = pl.n_simt() - pl.n_fwd;
    if (n_rest) launch_jet_step(args_for(h, pl.n_fwd, n_rest, 1), std::min(h->grid, n_rest), h->smem, s);
    launch_reduce_adam(r, s);
  } else if (h->opt.schedule == 0) {
    // one launch: exchange items first, interface items last (they wait)
    if (pl.n_tc) pack_tc_train(h, s);
    mark(h, 1, s);
    mark(h, 2, s);
    // residual items of the tensor-core kernel first, then the jet kernel's
    launch_tc(h, tc0, pl.n_tc, tc_ctr, s);
    if (pl.n_tc) mark(h, 5, s);
    h->tc_timed = pl.n_tc > 0 && h->opt.profile_phases;
    const int n_all = pl.n_simt();
    if (n_all) {
      StepArgs a = args_for(h, 0, n_all, 0);
      a.wait_from = pl.first_iface;
      a.n_fwd_wait = pl.n_fwd + (h->opt.inject_fault == 1 && pl.n_fwd ? 1 : 0);
      launch_jet_step(a, std::min(h->grid, n_all), h->smem, s);
    }
    mark(h, 3, s);
    launch_reduce_adam(r, s);
  } else {
    h->tc_timed = false;
    if (pl.n_tc) pack_tc_train(h, s);
    mark(h, 1, s);
    for (int q = 0; q < h->n_sub; ++q) {
      const int b = pl.fwd_begin[q], c = pl.fwd_begin[q + 1] - b;
      if (c) launch_jet_step(args_for(h, b, c, 2 + q), std::min(h->grid, c), h->smem, s);
    }
    mark(h, 2, s);
    for (int q = 0; q < h->n_sub; ++q) {
      launch_tc(h, tc0 + pl.tc_begin[q], pl.tc_begin[q + 1] - pl.tc_begin[q], tc_ctr + 1 + q, s);
      const int b = pl.n_fwd + pl.main_begin[q], c = pl.main_begin[q + 1] - pl.main_begin[q];
      if (c) launch_jet_step(args_for(h, b, c, 2 + h->n_sub + q), std::min(h->grid, c), h->smem, s);
    }
    mark(h, 3, s);
    // one reduce/Adam launch per subdomain
    int bi = 0;
    for (int q = 0; q < h->n_sub; ++q) {
      int nb = 0;
      while (bi + nb < (int)pl.red_blocks.size() && pl.red_blocks[bi + nb].x == q) ++nb;
      ReduceArgs rq = r;
      rq.blocks = h->red_blocks_d.p + bi;
      rq.n_blocks = nb;
      launch_reduce_adam(rq, s);
      bi += nb;
    }
  }
  mark(h, 4, s);
  ck(cudaGetLastError(), "kernel launch");
}

void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return;
  if (is_device_ptr(dst)) {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s), "copy out");
  } else {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s), "copy out");
    ck(cudaStreamSynchronize(s), "sync");
  }
}

void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return;
  if (is_device_ptr(src)) {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s), "copy in");
  } else {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), "copy in");
    ck(cudaStreamSynchronize(s), "sync");
  }
}

// Reads the handle's device status word after everything queued on `s`
// (synchronises `s`), clears it and turns a set word into an error.  Kernels
// only ever set the word (first code wins), so an error of an asynchronous
// call (xpinn_step without host losses) is reported by the next call that
// comes here: xpinn_sync, xpinn_grad, xpinn_step with host losses, eval.
void check_device_error(xpinn_ctx* h, cudaStream_t s) {
  int e = 0;
  ck(cudaMemcpyAsync(&e, h->err_d.p, sizeof(int), cudaMemcpyDeviceToHost, s), "read error flag");
  ck(cudaStreamSynchronize(s), "sync");
  if (e) {
    ck(cudaMemsetAsync(h->err_d.p, 0, sizeof(int), s), "reset error flag");
    ck(cudaStreamSynchronize(s), "sync");
    if (e == XPINN_ERR_TIMEOUT) fail(XPINN_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e == XPINN_ERR_NONFINITE) fail(XPINN_ERR_NONFINITE, "a loss became non-finite");
    fail(XPINN_ERR_INVALID, "device check failed (code %d)", e);
  }
}

// Jets of items over an evaluation buffer of points (already on the device).
void run_eval_items(xpinn_ctx* h, std::vector<Item>& items, const float2* pts, float* out, int dout,
                    const float* scale, cudaStream_t s) {
  if (items.empty()) return;
  h->e_items.ensure(items.size());
  ck(cudaMemcpyAsync(h->e_items.p, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice, s),
     "items");
  if (h->img_stale) {
    pack_images(h, s);
    h->img_stale = false;
  }
  StepArgs a = h->base;
  a.items = h->e_items.p;
  a.n_items = (int)items.size();
  a.item_base = 0;
  h->e_counter.ensure(1);
  a.counter = h->e_counter.p;
  a.eval_pts = pts;
  a.eval_out = out;
  a.eval_dout = dout;
  a.eval_scale = scale;
  ck(cudaMemsetAsync(a.counter, 0, sizeof(int), s), "memset");
  launch_jet_step(a, std::min<int>(h->grid, (int)items.size()), h->smem, s);
  ck(cudaGetLastError(), "eval launch");
  // keep the host copy alive until the copy has been consumed
  ck(cudaStreamSynchronize(s), "sync");
}

void eval_items_for(xpinn_ctx* h, int q, int net, int K, int64_t first, int64_t n, int64_t out_off,
                    int dout, std::vector<Item>& items) {
  const SubDev& sd = h->subs[q];
  Item proto{};
  proto.kind = IT_EVAL;
  proto.q = q;
  proto.K[0] = (net == 0 || net < 0) ? K : 0;
  proto.K[1] = (net == 1 || (net < 0 && sd.n_nets > 1)) ? K : 0;
  proto.P = choose_P(sd, proto.K, h->p_cap, h->opt.points_per_thread, cta_threads(h));
  proto.part_off = -1;
  const int64_t per = (int64_t)proto.P * 16;
  for (int64_t s = 0; s < n; s += per) {
    Item it = proto;
    it.pt_off = first + s;
    it.n_pts = (int)std::min<int64_t>(per, n - s);
    it.out_off = out_off + s * dout;
    items.push_back(it);
  }
}

// ---------------------------------------------------------------------------
// Routed evaluation (Eq. FSol) from a workspace, planned on the device:
// route (membership of every point) -> plan (bucket starts by a prefix sum
// of the counts, items cut from the buckets) -> bucket -> jet kernel (item
// count read on the device) -> gather (1/S sum per point).  No host round
// trip; every buffer is a slice of the workspace, sized for the worst case of
// MAXS = 4 memberships per point (a point at a corner of four boxes).
// ---------------------------------------------------------------------------
// Events around the evaluation kernel of a routed evaluation (profile_phases
// on, stream not being captured); `i` 0 before the launch, 1 after.
void eval_mark(xpinn_ctx* h, int i, cudaStream_t s) {
  if (!h->opt.profile_phases) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ck(cudaStreamIsCapturing(s, &cs), "capture status");
  if (cs != cudaStreamCaptureStatusNone) return;
  if (!h->eval_ev[i]) ck(cudaEventCreate(&h->eval_ev[i]), "cudaEventCreate");
  ck(cudaEventRecord(h->eval_ev[i], s), "event");
  h->eval_timed = i == 1;
}

// Hidden width W with which the networks of model `model` qualify for the
// tensor-core evaluation (eval_tc.h), or 0; on first use also the images'
// layout and pack list of every qualifying model.
int tc_width(xpinn_ctx* h, int model) {
  if (!h->opt.eval_tensor_cores) return 0;
  if (h->tc_w.empty()) {
    const int n_models = h->n_sub / h->spm;
    h->tc_w.assign(n_models, 0);
    std::vector<int64_t> off(h->n_sub, -1);
    std::vector<TcPack> pk;
    int64_t n_img = 0;
    for (int m = 0; m < n_models; ++m) {
      int W = -1;
      for (int q = m * h->spm; q < (m + 1) * h->spm && W != 0; ++q) {
        const SubDev& sd = h->subs[q];
        const NetDev& nd = sd.net[0];
        bool ok = sd.n_nets == 1 && nd.L >= 3 && nd.w[0] == 2 && nd.out_act == XPINN_ACT_IDENTITY &&
                  nd.w[nd.L] <= XPINN_MAX_OUT && eval_tc_width_ok(nd.w[1]) && (W < 0 || nd.w[1] == W);
        for (int k = 1; k < nd.L && ok; ++k) ok = nd.w[k] == nd.w[1];
        W = ok ? nd.w[1] : 0;
      }
      if (W <= 0) continue;
      h->tc_w[m] = W;
      for (int q = m * h->spm; q < (m + 1) * h->spm; ++q) {
        const SubDev& sd = h->subs[q];
        const NetDev& nd = sd.net[0];
        off[q] = n_img;
        for (int k = 2; k < nd.L; ++k) {
          pk.push_back(TcPack{sd.poff + nd.off[k], n_img, W, W});
          n_img += 2 * (int64_t)W * W;
        }
      }
    }
    h->tc_img.alloc((size_t)std::max<int64_t>(n_img, 4));
    h->tc_off.upload(off.data(), off.size());
    h->tc_pack_d.upload(pk.data(), pk.size());
    h->n_tc_pack = (int)pk.size();
    h->tc_stale = true;
    ck(eval_tc_configure(), "cudaFuncSetAttribute(tensor-core evaluation)");
  }
  return h->tc_w[model];
}

constexpr int EVAL_MAXS = 4;

struct EvalWs {
  size_t pts, S, memb, pos, counts, epts, escale, eout, out, items, n_items, counter, total;
  int max_items;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

EvalWs eval_ws_layout(const xpinn_ctx* h, int model, int64_t n, int order) {
  const int K = order == 0 ? 1 : (order == 1 ? 3 : 5);
  const int row = h->n_out_total * K;
  const int nq = h->spm;
  const int64_t ne = EVAL_MAXS * std::max<int64_t>(n, 1);
  const int chunk = h->e_min_chunk[(size_t)order * (h->n_sub / h->spm) + model];
  EvalWs w{};
  w.max_items = (int)std::min<int64_t>(nq + (ne + chunk - 1) / chunk, 1 << 30);
  size_t o = 0;
  auto take = [&](size_t& field, size_t bytes) { field = o; o = al256(o + bytes); };
  take(w.pts, sizeof(float2) * std::max<int64_t>(n, 1));
  take(w.S, sizeof(int) * std::max<int64_t>(n, 1));
  take(w.memb, sizeof(int) * ne);
  take(w.pos, sizeof(int) * ne);
  take(w.counts, sizeof(int) * 2 * nq);
  take(w.epts, sizeof(float2) * ne);
  take(w.escale, sizeof(float) * ne);
  take(w.eout, sizeof(float) * ne * row);
  take(w.out, sizeof(float) * std::max<int64_t>(n, 1) * row);
  take(w.items, sizeof(Item) * (size_t)w.max_items);
  take(w.n_items, sizeof(int));
  take(w.counter, sizeof(int));
  w.total = o;
  return w;
}

// Enqueues the routed evaluation of n points (device pointer pts) into out
// (device pointer, [n][row]); ws must hold eval_ws_layout(...).total bytes.
void eval_enqueue(xpinn_ctx* h, int model, const float2* pts, int64_t n, int order, float* out, char* ws,
                  const EvalWs& L, cudaStream_t s) {
  const int K = order == 0 ? 1 : (order == 1 ? 3 : 5);
  const int row = h->n_out_total * K;
  const int q0 = model * h->spm, nq = h->spm;
  int* S = reinterpret_cast<int*>(ws + L.S);
  int* memb = reinterpret_cast<int*>(ws + L.memb);
  int* pos = reinterpret_cast<int*>(ws + L.pos);
  int* counts = reinterpret_cast<int*>(ws + L.counts);
  float2* epts = reinterpret_cast<float2*>(ws + L.epts);
  float* escale = reinterpret_cast<float*>(ws + L.escale);
  float* eout = reinterpret_cast<float*>(ws + L.eout);
  Item* items = reinterpret_cast<Item*>(ws + L.items);
  int* n_items = reinterpret_cast<int*>(ws + L.n_items);
  int* counter = reinterpret_cast<int*>(ws + L.counter);
  ck(cudaMemsetAsync(counts, 0, sizeof(int) * 2 * nq, s), "memset");
  launch_route(pts, n, h->subs_d.p, q0, nq, S, memb, counts, h->err_d.p, h->poly.p, h->n_poly, s);
  launch_eval_plan(counts, nq, h->e_proto.p + (size_t)order * h->n_sub + q0, q0, row, counts + nq, items,
                   n_items, L.max_items, h->err_d.p, s);
  launch_bucket(pts, n, S, memb, counts + nq, pos, epts, escale, s);
  const int W = tc_width(h, model);
  if (W) {
    if (h->tc_stale) {
      launch_pack_tc(h->params.p, h->tc_pack_d.p, h->n_tc_pack, h->tc_img.p, s);
      h->tc_stale = false;
    }
    TcArgs t{};
    t.items = items;
    t.n_items = L.max_items;
    t.n_items_dev = n_items;
    t.counter = counter;
    t.subs = h->subs_d.p;
    t.params = h->params.p;
    t.img = h->tc_img.p;
    t.img_off = h->tc_off.p;
    t.pts = epts;
    t.scale = escale;
    t.out = eout;
    t.dout = row;
    t.err = h->err_d.p;
    const int per_sm = eval_tc_ctas_per_sm(W, K);
    ck(cudaMemsetAsync(t.counter, 0, sizeof(int), s), "memset");
    eval_mark(h, 0, s);
    launch_eval_tc(W, K, t, std::min<int>(h->n_sm * per_sm, L.max_items), s);
    eval_mark(h, 1, s);
    launch_gather(n, row, S, pos, eout, out, s);
    ck(cudaGetLastError(), "evaluation launches");
    return;
  }
  if (h->img_stale) {
    pack_images(h, s);
    h->img_stale = false;
  }
  StepArgs a = h->base;
  a.items = items;
  a.n_items = L.max_items;
  a.n_items_dev = n_items;
  a.item_base = 0;
  a.counter = counter;
  a.eval_pts = epts;
  a.eval_out = eout;
  a.eval_dout = row;
  a.eval_scale = escale;
  ck(cudaMemsetAsync(a.counter, 0, sizeof(int), s), "memset");
  eval_mark(h, 0, s);
  launch_jet_step(a, std::min<int>(h->grid, L.max_items), h->smem, s);
  eval_mark(h, 1, s);
  launch_gather(n, row, S, pos, eout, out, s);
  ck(cudaGetLastError(), "evaluation launches");
}

// The routed evaluation with caller-provided workspace: host or device xy
// and out (both on the same side); with device pointers nothing synchronises.
void eval_with_ws(xpinn_handle h, int32_t model, const float* xy, int64_t n, int32_t order, float* out,
                         char* ws, size_t ws_bytes, cudaStream_t s) {
  const EvalWs L = eval_ws_layout(h, model, n, order);
  if (ws_bytes < L.total) fail(XPINN_ERR_INVALID, "workspace of %zu bytes, %zu needed", ws_bytes, L.total);
  if (reinterpret_cast<uintptr_t>(ws) % 256) fail(XPINN_ERR_INVALID, "workspace must be 256-byte aligned");
  const int K = order == 0 ? 1 : (order == 1 ? 3 : 5);
  const int row = h->n_out_total * K;
  const bool dev_in = is_device_ptr(xy), dev_out = is_device_ptr(out);
  const float2* pts = reinterpret_cast<const float2*>(xy);
  if (!dev_in) {
    ck(cudaMemcpyAsync(ws + L.pts, xy, n * sizeof(float2), cudaMemcpyHostToDevice, s), "copy in");
    pts = reinterpret_cast<const float2*>(ws + L.pts);
  }
  float* o = dev_out ? out : reinterpret_cast<float*>(ws + L.out);
  eval_enqueue(h, model, pts, n, order, o, ws, L, s);
  if (!dev_out) {
    ck(cudaMemcpyAsync(out, o, sizeof(float) * n * row, cudaMemcpyDeviceToHost, s), "copy out");
    check_device_error(h, s);   // synchronises
  }
}


// ---------------------------------------------------------------------------
// Forks (xpinn_fork_step): a training request on a subset S of a handle's
// subdomains with its own residual points.  The fork is a second context
// whose device buffers are views into a caller-provided workspace: the
// parameters and Adam moments of S (copied from the handle), the parameters of
// S's interface neighbours N (copied; they only provide interface values and
// are not trained), S's data points and targets, the interface points, the
// request's residual points, the plan and the per-item gradient slices.  The
// handle's own parameters and Adam state are not touched.
// ---------------------------------------------------------------------------
struct ForkLayout {
  size_t subs, ifaces, items, q_items, q_item_begin, q_part_off, red_blocks, pack, params, m, v, wimg, pts,
      res_f, tgt, d4, partials, loss_part, counters, state, ring, total;
};

struct Fork {
  std::unique_ptr<xpinn_ctx> f;
  std::vector<int> T;                  // fork subdomain -> handle subdomain (S first, then N)
  int n_sel = 0;
  int64_t n_params_sel = 0;            // parameters of S: the first floats of the fork's vector
  std::vector<int64_t> src_poff;       // handle parameter offset of each fork subdomain
  struct Copy {
    int64_t dst, src, n;
  };
  std::vector<Copy> pt_copies, tgt_copies;   // (data and interface points, targets) from the handle
  std::vector<Copy> d4_copies;                // interfaces with a remote side: their exchange rows
  int64_t n_res_req = 0, n_data_pts = 0, n_tgt = 0;
  ForkLayout L{};
};

int img_floats_of(const SubDev& sd) {
  int ioff = 0;
  for (int n = 0; n < sd.n_nets; ++n) {
    NetDev nd = sd.net[n];
    ioff = assign_images(nd, ioff);
  }
  return ioff;
}

std::unique_ptr<Fork> make_fork(xpinn_ctx* h, const xpinn_fork_desc* d) {
  if (!d || d->n_sel < 1 || d->n_sel > h->n_sub || !d->sel || !d->n_pts || d->n_steps < 0)
    fail(XPINN_ERR_INVALID, "bad fork request");
  auto F = std::make_unique<Fork>();
  std::vector<int> idx(h->n_sub, -1);
  int64_t n_req = 0;
  for (int i = 0; i < d->n_sel; ++i) {
    const int q = d->sel[i];
    if (q < 0 || q >= h->n_sub || idx[q] >= 0) fail(XPINN_ERR_INVALID, "fork: bad or repeated subdomain %d", q);
    if (d->n_pts[i] < 0 || d->n_pts[i] > (1 << 30)) fail(XPINN_ERR_INVALID, "fork: bad point count");
    idx[q] = i;
    F->T.push_back(q);
    n_req += d->n_pts[i];
  }
  if (n_req > 0 && !d->xy) fail(XPINN_ERR_INVALID, "fork: NULL points");
  F->n_sel = d->n_sel;
  F->n_res_req = n_req;
  // interface neighbours of S outside S, ascending
  std::vector<int> nb;
  for (const IfaceDev& e : h->ifaces) {
    if (e.remote) continue;   // the remote side's values stay what the handle holds (see bind_fork)
    if (idx[e.q] >= 0 && idx[e.qp] < 0) nb.push_back(e.qp);
    if (idx[e.qp] >= 0 && idx[e.q] < 0) nb.push_back(e.q);
  }
  std::sort(nb.begin(), nb.end());
  nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
  for (int q : nb) {
    idx[q] = (int)F->T.size();
    F->T.push_back(q);
  }
  auto f = std::make_unique<xpinn_ctx>();
  f->pde = h->pde;
  f->flux_mode = h->flux_mode;
  f->nu = h->nu;
  f->re = h->re;
  f->beta1 = h->beta1;
  f->beta2 = h->beta2;
  f->eps = h->eps;
  f->n_sub = (int)F->T.size();
  f->spm = f->n_sub;
  f->n_out_total = h->n_out_total;
  f->n_eq = h->n_eq;
  f->d4_nv = h->d4_nv;
  f->opt = h->opt;
  f->opt.schedule = 0;
  f->opt.use_graph = 0;
  f->opt.profile_phases = 0;
  f->opt.inject_fault = 0;
  f->opt.train_tensor_cores = 0;   // forks train on the jet kernel
  f->grid = h->grid;
  f->n_sm = h->n_sm;
  f->device = h->device;
  f->p_cap = h->p_cap;
  f->ring_cap = std::max(1, (int)d->n_steps);
  f->trained.assign(f->n_sub, 0);
  for (int i = 0; i < d->n_sel; ++i) f->trained[i] = 1;
  if (!h->tile_cap.empty())
    for (int q : F->T) f->tile_cap.push_back(h->tile_cap[q]);
  // points: [request residual points][data points of S][interface points]
  int64_t n_data = 0;
  for (int i = 0; i < d->n_sel; ++i) {
    const SubDev& sd = h->subs[F->T[i]];
    for (int n = 0; n < sd.n_nets; ++n) n_data += sd.n_data[n];
  }
  int64_t poff = 0, img = 0, res = 0, dcur = n_req, tcur = 0;
  for (int i = 0; i < f->n_sub; ++i) {
    const int q = F->T[i];
    SubDev sd = h->subs[q];
    F->src_poff.push_back(sd.poff);
    sd.poff = poff;
    poff += sd.n_params;
    if (i < d->n_sel) F->n_params_sel = poff;
    sd.img_off = img;
    img += img_floats_of(sd);
    if (i < d->n_sel) {
      sd.n_res = (int)d->n_pts[i];
      sd.res_off = res;
      sd.inv_n_res = sd.n_res ? 1.f / (float)sd.n_res : 0.f;
      res += sd.n_res;
      for (int n = 0; n < sd.n_nets; ++n) {
        const SubDev& hs = h->subs[q];
        const int D = sd.net[n].w[sd.net[n].L];
        if (!hs.n_data[n]) continue;
        F->pt_copies.push_back({dcur, hs.data_off[n], hs.n_data[n]});
        F->tgt_copies.push_back({tcur, hs.tgt_off[n], (int64_t)hs.n_data[n] * D});
        sd.data_off[n] = dcur;
        sd.tgt_off[n] = tcur;
        dcur += hs.n_data[n];
        tcur += (int64_t)hs.n_data[n] * D;
      }
    } else {
      sd.n_res = 0;
      sd.inv_n_res = 0.f;
      sd.res_off = 0;
      for (int n = 0; n < sd.n_nets; ++n) {
        sd.n_data[n] = 0;
        sd.inv_n_data[n] = 0.f;
      }
    }
    f->subs.push_back(sd);
    for (int n = 0; n < sd.n_nets; ++n) {
      const NetDev& nd = sd.net[n];
      for (int k = 2; k < nd.L; ++k) {
        const int64_t src = sd.poff + nd.off[k];
        f->pack_h.push_back({src, sd.img_off + nd.imf[k], nd.w[k - 1], nd.w[k], nd.wp[k - 1], nd.wp[k], 1});
        f->pack_h.push_back({src, sd.img_off + nd.imb[k], nd.w[k - 1], nd.w[k], nd.wp[k - 1], nd.wp[k], 0});
      }
    }
  }
  F->n_data_pts = n_data;
  F->n_tgt = tcur;
  int64_t icur = 0;
  for (const IfaceDev& e : h->ifaces) {
    // interfaces with a trained side; the other side is in S or N
    const bool tq = idx[e.q] >= 0 && idx[e.q] < d->n_sel, tp = idx[e.qp] >= 0 && idx[e.qp] < d->n_sel;
    if (!tq && !tp) continue;
    IfaceDev fd = e;
    fd.q = idx[e.q];
    fd.qp = idx[e.qp];
    F->pt_copies.push_back({n_req + n_data + icur, e.pt_off, e.n_pts});
    if (e.remote)   // the remote side's values as the handle last received them
      F->d4_copies.push_back({icur * 2 * h->d4_nv, e.d4_pt * 2 * h->d4_nv, (int64_t)e.n_pts * 2 * h->d4_nv});
    fd.pt_off = n_req + n_data + icur;
    fd.d4_pt = icur;
    icur += e.n_pts;
    f->ifaces.push_back(fd);
  }
  f->n_iface = (int)f->ifaces.size();
  f->n_if_pts = icur;
  f->n_params = poff;
  f->n_img = img;
  f->n_res_total = n_req;
  f->n_pts_total = n_req + n_data + icur;
  f->n_counters = 3 + 2 * f->n_sub;
  build_plan(f.get(), h->p_cap);
  // workspace layout
  const Plan& pl = f->plan;
  ForkLayout& L = F->L;
  size_t o = 0;
  auto take = [&](size_t& field, size_t bytes) { field = o; o = al256(o + std::max<size_t>(bytes, 4)); };
  take(L.subs, sizeof(SubDev) * f->subs.size());
  take(L.ifaces, sizeof(IfaceDev) * f->ifaces.size());
  take(L.items, sizeof(Item) * pl.items.size());
  take(L.q_items, sizeof(int) * pl.q_items.size());
  take(L.q_item_begin, sizeof(int) * pl.q_item_begin.size());
  take(L.q_part_off, sizeof(int64_t) * pl.q_part_off.size());
  take(L.red_blocks, sizeof(int2) * pl.red_blocks.size());
  take(L.pack, sizeof(PackBlock) * f->pack_h.size());
  take(L.params, sizeof(float) * (size_t)f->n_params);
  take(L.m, sizeof(float) * (size_t)F->n_params_sel);
  take(L.v, sizeof(float) * (size_t)F->n_params_sel);
  take(L.wimg, sizeof(float) * (size_t)std::max<int64_t>(4, f->n_img));
  take(L.pts, sizeof(float2) * (size_t)f->n_pts_total);
  take(L.res_f, sizeof(float) * (size_t)n_req);
  take(L.tgt, sizeof(float) * (size_t)F->n_tgt);
  take(L.d4, sizeof(float) * (size_t)std::max<int64_t>(1, f->n_if_pts * 2 * f->d4_nv));
  take(L.partials, sizeof(float) * (size_t)pl.partial_floats);
  take(L.loss_part, sizeof(double) * 2 * pl.items.size());
  take(L.counters, sizeof(int) * f->n_counters);
  take(L.state, sizeof(int) * 4);
  take(L.ring, sizeof(float) * (size_t)f->ring_cap * f->n_sub * XPINN_N_TERMS);
  L.total = o;
  F->f = std::move(f);
  return F;
}

// Binds the fork's buffers to the workspace and fills it: tables from the
// host, parameters, moments, step count, data and interface points from the
// handle, the request's residual points and forcing from the caller.
// Bytes of the host tables a fork uploads (see bind_fork's `pinned`).
size_t fork_table_bytes(const Fork& F) {
  const xpinn_ctx* f = F.f.get();
  const Plan& pl = f->plan;
  size_t o = 0;
  for (size_t b : {sizeof(SubDev) * f->subs.size(), sizeof(IfaceDev) * f->ifaces.size(),
                   sizeof(Item) * pl.items.size(), sizeof(int) * pl.q_items.size(),
                   sizeof(int) * pl.q_item_begin.size(), sizeof(int64_t) * pl.q_part_off.size(),
                   sizeof(int2) * pl.red_blocks.size(), sizeof(PackBlock) * f->pack_h.size()})
    o = al256(o + b);
  return o;
}

// With `pinned` (host page-locked memory of fork_table_bytes), the tables are
// staged there and uploaded asynchronously; without it they are uploaded
// from pageable host memory, which waits for the work queued on `s`.
void bind_fork(xpinn_ctx* h, Fork& F, char* ws, const xpinn_fork_desc* d, cudaStream_t s,
               char* pinned = nullptr) {
  xpinn_ctx* f = F.f.get();
  const ForkLayout& L = F.L;
  const Plan& pl = f->plan;
  f->subs_d.view(ws + L.subs, f->subs.size());
  f->ifaces_d.view(ws + L.ifaces, f->ifaces.size());
  f->items_d.view(ws + L.items, pl.items.size());
  f->q_items_d.view(ws + L.q_items, pl.q_items.size());
  f->q_item_begin_d.view(ws + L.q_item_begin, pl.q_item_begin.size());
  f->q_part_off_d.view(ws + L.q_part_off, pl.q_part_off.size());
  f->red_blocks_d.view(ws + L.red_blocks, pl.red_blocks.size());
  f->pack_d.view(ws + L.pack, f->pack_h.size());
  f->params.view(ws + L.params, f->n_params);
  f->m.view(ws + L.m, F.n_params_sel);
  f->v.view(ws + L.v, F.n_params_sel);
  f->wimg.view(ws + L.wimg, std::max<int64_t>(4, f->n_img));
  f->pts.view(ws + L.pts, f->n_pts_total);
  f->res_f.view(ws + L.res_f, F.n_res_req);
  f->tgt.view(ws + L.tgt, F.n_tgt);
  f->d4.view(ws + L.d4, std::max<int64_t>(1, f->n_if_pts * 2 * f->d4_nv));
  f->partials.view(ws + L.partials, pl.partial_floats);
  f->loss_part.view(ws + L.loss_part, 2 * pl.items.size());
  f->counters.view(ws + L.counters, f->n_counters);
  f->state_i.view(ws + L.state, 4);
  f->loss_ring.view(ws + L.ring, (size_t)f->ring_cap * f->n_sub * XPINN_N_TERMS);
  f->err_d.view(h->err_d.p, 1);              // errors are the handle's (xpinn_sync reports them)
  f->scratch.view(h->scratch.p, h->scratch.n);
  size_t po = 0;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (!bytes) return;
    if (pinned) {
      memcpy(pinned + po, src, bytes);
      src = pinned + po;
      po = al256(po + bytes);
    }
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), "fork tables");
  };
  auto dd = [&](void* dst, const void* src, size_t bytes) {
    if (bytes) ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s), "fork copy");
  };
  up(f->subs_d.p, f->subs.data(), sizeof(SubDev) * f->subs.size());
  up(f->ifaces_d.p, f->ifaces.data(), sizeof(IfaceDev) * f->ifaces.size());
  up(f->items_d.p, pl.items.data(), sizeof(Item) * pl.items.size());
  up(f->q_items_d.p, pl.q_items.data(), sizeof(int) * pl.q_items.size());
  up(f->q_item_begin_d.p, pl.q_item_begin.data(), sizeof(int) * pl.q_item_begin.size());
  up(f->q_part_off_d.p, pl.q_part_off.data(), sizeof(int64_t) * pl.q_part_off.size());
  up(f->red_blocks_d.p, pl.red_blocks.data(), sizeof(int2) * pl.red_blocks.size());
  up(f->pack_d.p, f->pack_h.data(), sizeof(PackBlock) * f->pack_h.size());
  for (int i = 0; i < f->n_sub; ++i) {
    const SubDev& sd = f->subs[i];
    dd(f->params.p + sd.poff, h->params.p + F.src_poff[i], sizeof(float) * sd.n_params);
    if (i < F.n_sel) {
      dd(f->m.p + sd.poff, h->m.p + F.src_poff[i], sizeof(float) * sd.n_params);
      dd(f->v.p + sd.poff, h->v.p + F.src_poff[i], sizeof(float) * sd.n_params);
    }
  }
  for (const Fork::Copy& c : F.pt_copies) dd(f->pts.p + c.dst, h->pts.p + c.src, sizeof(float2) * c.n);
  for (const Fork::Copy& c : F.tgt_copies) dd(f->tgt.p + c.dst, h->tgt.p + c.src, sizeof(float) * c.n);
  if (F.n_res_req) {
    copy_in(f->pts.p, d->xy, sizeof(float2) * F.n_res_req, s);
    if (d->f)
      copy_in(f->res_f.p, d->f, sizeof(float) * F.n_res_req, s);
    else
      ck(cudaMemsetAsync(f->res_f.p, 0, sizeof(float) * F.n_res_req, s), "memset");
  }
  ck(cudaMemsetAsync(f->d4.p, 0, sizeof(float) * f->d4.n, s), "memset");
  for (const Fork::Copy& c : F.d4_copies) dd(f->d4.p + c.dst, h->d4.p + c.src, sizeof(float) * c.n);
  ck(cudaMemsetAsync(f->counters.p, 0, sizeof(int) * f->n_counters, s), "memset");
  ck(cudaMemsetAsync(f->state_i.p, 0, sizeof(int) * 4, s), "memset");
  dd(f->state_i.p, h->step_t(), sizeof(int));   // Adam continues from the handle's step count
  StepArgs& a = f->base;
  a = h->base;
  a.subs = f->subs_d.p;
  a.ifaces = f->ifaces_d.p;
  a.params = f->params.p;
  a.wimg = f->wimg.p;
  a.pts = f->pts.p;
  a.res_f = f->res_f.p;
  a.tgt = f->tgt.p;
  a.d4 = f->d4.p;
  a.partials = f->partials.p;
  a.loss_part = f->loss_part.p;
  a.scratch = h->scratch.p;
  a.err = h->err_d.p;
  a.n_items_dev = nullptr;
  f->smem = h->smem;
}

}  // namespace

// Makes the handle's device current for the duration of an API call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(const xpinn_ctx* h) {
    if (h && cudaGetDevice(&prev) == cudaSuccess && prev != h->device) {
      ck(cudaSetDevice(h->device), "cudaSetDevice");
    } else {
      prev = -1;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Re-plan the step for new options (items, shared memory, scratch).
void apply_options(xpinn_ctx* h, const xpinn_options& o) {
  h->opt = o;
  if (h->opt.profile_phases)
    for (auto& e : h->ev)
      if (!e) ck(cudaEventCreate(&e), "cudaEventCreate");
  plan(h);
  h->base.partials = h->partials.p;
  h->base.loss_part = h->loss_part.p;
  h->base.scratch = h->scratch.p;
}

// ===========================================================================
// C ABI
// ===========================================================================
#define API_BEGIN try {
#define API_END                                  \
  }                                              \
  catch (const Error& e) {                       \
    return e.code;                               \
  }                                              \
  catch (const std::bad_alloc&) {                \
    g_err = "host allocation failed";            \
    return XPINN_ERR_OOM;                        \
  }                                              \
  catch (...) {                                  \
    g_err = "unexpected host exception";         \
    return XPINN_ERR_INVALID;                    \
  }                                              \
  g_err.clear();                                 \
  return XPINN_OK;

extern "C" {

const char* xpinn_last_error(void) { return g_err.c_str(); }

int xpinn_create(const xpinn_problem_desc* d, xpinn_handle* out) {
  API_BEGIN
  if (!d || !out) fail(XPINN_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (d->pde < 0 || d->pde > 3) fail(XPINN_ERR_INVALID, "unknown pde %d", d->pde);
  if (d->n_sub < 1 || !d->subs) fail(XPINN_ERR_INVALID, "need at least one subdomain");
  if (d->n_iface < 0 || (d->n_iface > 0 && !d->ifaces)) fail(XPINN_ERR_INVALID, "bad interface list");
  if (!d->init_params) fail(XPINN_ERR_INVALID, "init_params is required");
  if (d->flux_mode != XPINN_FLUX_CONSERVATIVE && d->flux_mode != XPINN_FLUX_LITERAL)
    fail(XPINN_ERR_INVALID, "bad flux_mode");
  if (!(d->beta1 >= 0 && d->beta1 < 1 && d->beta2 >= 0 && d->beta2 < 1 && d->eps > 0))
    fail(XPINN_ERR_INVALID, "bad Adam constants");
  if (d->pde == XPINN_PDE_NS && !(d->re > 0)) fail(XPINN_ERR_INVALID, "Reynolds number must be > 0");
  const int spm = d->subs_per_model ? d->subs_per_model : d->n_sub;
  if (spm < 1 || d->n_sub % spm) fail(XPINN_ERR_INVALID, "subs_per_model must divide n_sub");
  auto h = std::make_unique<xpinn_ctx>();
  h->pde = d->pde;
  h->nu = d->nu;
  h->re = d->re;
  h->flux_mode = d->flux_mode;
  h->beta1 = d->beta1;
  h->beta2 = d->beta2;
  h->eps = d->eps;
  h->n_sub = d->n_sub;
  h->n_iface = d->n_iface;
  h->spm = spm;
  h->n_eq = d->pde == XPINN_PDE_NS ? 3 : 1;
  const int want_nets = d->pde == XPINN_PDE_DIFFUSION ? 2 : 1;
  // ---- subdomains
  std::vector<float2> pts_res, pts_data;
  std::vector<float> res_f, tgt;
  int64_t poff = 0;
  for (int q = 0; q < d->n_sub; ++q) {
    const xpinn_subdomain_desc& s = d->subs[q];
    if (s.n_nets != want_nets)
      fail(XPINN_ERR_INVALID, "subdomain %d: %d networks, this PDE needs %d", q, s.n_nets, want_nets);
    SubDev sd{};
    sd.n_nets = s.n_nets;
    sd.poff = poff;
    sd.img_off = h->n_img;
    int off = 0, ioff = 0;
    for (int n = 0; n < s.n_nets; ++n) {
      validate_net(s.nets[n], d->pde, n, q);
      off = fill_net_dev(sd.net[n], s.nets[n], off);
      NetDev& nd = sd.net[n];
      ioff = assign_images(nd, ioff);
      for (int k = 2; k < nd.L; ++k) {
        const int64_t src = sd.poff + nd.off[k];
        h->pack_h.push_back({src, sd.img_off + nd.imf[k], nd.w[k - 1], nd.w[k], nd.wp[k - 1], nd.wp[k], 1});
        h->pack_h.push_back({src, sd.img_off + nd.imb[k], nd.w[k - 1], nd.w[k], nd.wp[k - 1], nd.wp[k], 0});
      }
    }
    sd.n_params = off;
    poff += off;
    h->n_img += ioff;
    if (s.n_res < 0 || (s.n_res > 0 && !s.res_xy)) fail(XPINN_ERR_INVALID, "subdomain %d: bad residual points", q);
    if (s.n_res > (1 << 30)) fail(XPINN_ERR_UNSUPPORTED, "subdomain %d: too many residual points", q);
    sd.res_off = (int64_t)pts_res.size();
    sd.n_res = (int)s.n_res;
    sd.inv_n_res = s.n_res ? 1.f / (float)s.n_res : 0.f;
    check_finite(s.res_xy, 2 * s.n_res, "res_xy");
    for (int64_t i = 0; i < s.n_res; ++i) {
      pts_res.push_back(make_float2(s.res_xy[2 * i], s.res_xy[2 * i + 1]));
      res_f.push_back(s.res_f ? s.res_f[i] : 0.f);
    }
    if (s.res_f) check_finite(s.res_f, s.n_res, "res_f");
    for (int n = 0; n < s.n_nets; ++n) {
      const int D = sd.net[n].w[sd.net[n].L];
      if (s.n_data[n] < 0 || (s.n_data[n] > 0 && (!s.data_xy[n] || !s.data_val[n])))
        fail(XPINN_ERR_INVALID, "subdomain %d: bad data set %d", q, n);
      check_finite(s.data_xy[n], 2 * s.n_data[n], "data_xy");
      check_finite(s.data_val[n], D * s.n_data[n], "data_val");
      sd.data_off[n] = (int64_t)pts_data.size();   // rebased below
      sd.tgt_off[n] = (int64_t)tgt.size();
      sd.n_data[n] = (int)s.n_data[n];
      sd.inv_n_data[n] = s.n_data[n] ? 1.f / (float)s.n_data[n] : 0.f;
      sd.w_data[n] = s.w_data[n];
      for (int64_t i = 0; i < s.n_data[n]; ++i) {
        pts_data.push_back(make_float2(s.data_xy[n][2 * i], s.data_xy[n][2 * i + 1]));
        for (int o = 0; o < D; ++o) tgt.push_back(s.data_val[n][i * D + o]);
      }
    }
    sd.w_res = s.w_res;
    sd.w_avg = s.w_avg;
    sd.w_iface = s.w_iface;
    sd.lr = s.lr;
    if (!std::isfinite(s.lr) || !std::isfinite(s.w_res) || !std::isfinite(s.w_avg) || !std::isfinite(s.w_iface))
      fail(XPINN_ERR_INVALID, "subdomain %d: non-finite weight or learning rate", q);
    for (int i = 0; i < 4; ++i) sd.rect[i] = s.rect[i];
    if (s.region_kind != XPINN_REGION_BOX && s.region_kind != XPINN_REGION_VORONOI)
      fail(XPINN_ERR_INVALID, "subdomain %d: bad region_kind", q);
    sd.region_kind = s.region_kind;
    sd.site[0] = s.site[0];
    sd.site[1] = s.site[1];
    h->subs.push_back(sd);
  }
  h->n_params = poff;
  h->n_res_total = (int64_t)pts_res.size();
  h->n_out_total = 0;
  for (int n = 0; n < h->subs[0].n_nets; ++n) h->n_out_total += h->subs[0].net[n].w[h->subs[0].net[n].L];
  h->d4_nv = h->n_out_total + h->n_eq;
  for (auto& sd : h->subs)
    for (int n = 0; n < sd.n_nets; ++n) sd.data_off[n] += h->n_res_total;
  // ---- interfaces
  std::vector<float2> pts_if;
  for (int e = 0; e < d->n_iface; ++e) {
    const xpinn_interface_desc& f = d->ifaces[e];
    if (f.remote != 0 && f.remote != 1) fail(XPINN_ERR_INVALID, "interface %d: remote must be 0 or 1", e);
    if (f.q < 0 || f.q >= d->n_sub ||
        (!f.remote && (f.q_plus < 0 || f.q_plus >= d->n_sub || f.q == f.q_plus)))
      fail(XPINN_ERR_INVALID, "interface %d: bad subdomains (%d, %d)", e, f.q, f.q_plus);
    if (f.method != XPINN_CPINN && f.method != XPINN_XPINN) fail(XPINN_ERR_INVALID, "interface %d: bad method", e);
    if (f.n_pts < 0 || (f.n_pts > 0 && !f.xy)) fail(XPINN_ERR_INVALID, "interface %d: bad points", e);
    check_finite(f.xy, 2 * f.n_pts, "iface xy");
    IfaceDev fd{};
    fd.q = f.q;
    fd.qp = f.remote ? f.q : f.q_plus;   // a remote side has no subdomain in this handle
    fd.remote = f.remote;
    fd.method = f.method;
    fd.n_pts = (int)f.n_pts;
    fd.nx = f.normal[0];
    fd.ny = f.normal[1];
    fd.inv_n = f.n_pts ? 1.f / (float)f.n_pts : 0.f;
    fd.d4_pt = (int64_t)pts_if.size();
    for (int64_t i = 0; i < f.n_pts; ++i) pts_if.push_back(make_float2(f.xy[2 * i], f.xy[2 * i + 1]));
    h->ifaces.push_back(fd);
  }
  h->n_if_pts = (int64_t)pts_if.size();
  const int64_t if_base = h->n_res_total + (int64_t)pts_data.size();
  for (auto& f : h->ifaces) f.pt_off = if_base + f.d4_pt;
  check_finite(d->init_params, h->n_params, "init_params");
  if (d->n_poly < 0 || d->n_poly == 1 || d->n_poly == 2 || (d->n_poly > 0 && !d->poly))
    fail(XPINN_ERR_INVALID, "bad polygon");
  for (int q = 0; q < d->n_sub; q += spm)
    for (int l = 1; l < spm; ++l)
      if (d->subs[q + l].region_kind != d->subs[q].region_kind)
        fail(XPINN_ERR_INVALID, "copy %d mixes box and Voronoi regions", q / spm);
  if (d->subs[0].region_kind == XPINN_REGION_VORONOI && d->n_poly < 3)
    fail(XPINN_ERR_INVALID, "Voronoi regions need the polygon");
  std::vector<float2> poly_h;
  for (int v = 0; v < d->n_poly; ++v) poly_h.push_back(make_float2(d->poly[2 * v], d->poly[2 * v + 1]));
  check_finite(d->poly, 2 * (int64_t)d->n_poly, "poly");
  // ---- device
  ck(cudaFree(0), "CUDA init");
  ck(cudaGetDevice(&h->device), "cudaGetDevice");
  ck(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, 0), "attr");
  h->grid = h->n_sm;   // set by plan()
  std::vector<float2> all = pts_res;
  all.insert(all.end(), pts_data.begin(), pts_data.end());
  all.insert(all.end(), pts_if.begin(), pts_if.end());
  h->n_pts_total = (int64_t)all.size();
  h->pts.upload(all.data(), all.size());
  h->res_f.upload(res_f.data(), res_f.size());
  h->n_poly = (int)poly_h.size();
  h->poly.upload(poly_h.data(), poly_h.size());
  h->tgt.upload(tgt.data(), tgt.size());
  h->params.upload(d->init_params, (size_t)h->n_params);
  h->wimg.alloc((size_t)std::max<int64_t>(4, h->n_img));
  h->pack_d.upload(h->pack_h.data(), h->pack_h.size());
  h->m.alloc((size_t)h->n_params);
  h->v.alloc((size_t)h->n_params);
  h->grads.alloc((size_t)h->n_params);
  ck(cudaMemset(h->m.p, 0, h->n_params * sizeof(float)), "memset");
  ck(cudaMemset(h->v.p, 0, h->n_params * sizeof(float)), "memset");
  h->subs_d.upload(h->subs.data(), h->subs.size());
  h->ifaces_d.upload(h->ifaces.data(), h->ifaces.size());
  h->d4.alloc((size_t)std::max<int64_t>(1, h->n_if_pts * 2 * h->d4_nv));
  ck(cudaMemset(h->d4.p, 0, h->d4.n * sizeof(float)), "memset");
  h->state_i.alloc(4);   // step count, loss slot, two float bias corrections
  ck(cudaMemset(h->state_i.p, 0, 4 * sizeof(int)), "memset");
  h->err_d.alloc(1);
  ck(cudaMemset(h->err_d.p, 0, sizeof(int)), "memset");
  h->loss_ring.alloc((size_t)h->ring_cap * h->n_sub * XPINN_N_TERMS);
  h->jq.alloc((size_t)h->n_sub + 1);
  StepArgs& a = h->base;
  a.subs = h->subs_d.p;
  a.ifaces = h->ifaces_d.p;
  a.params = h->params.p;
  a.wimg = h->wimg.p;
  a.pts = h->pts.p;
  a.res_f = h->res_f.p;
  a.tgt = h->tgt.p;
  a.d4 = h->d4.p;
  a.d4_nv = h->d4_nv;
  a.pde = h->pde;
  a.nu = h->nu;
  a.re = h->re;
  a.flux_mode = h->flux_mode;
  a.n_out_total = h->n_out_total;
  a.n_eq = h->n_eq;
  a.err = h->err_d.p;
  plan(h.get());
  a.partials = h->partials.p;
  a.loss_part = h->loss_part.p;
  a.scratch = h->scratch.p;
  ck(cudaDeviceSynchronize(), "create");
  *out = h.release();
  API_END
}

int xpinn_destroy(xpinn_handle h) {
  API_BEGIN
  if (h) {
    cudaDeviceSynchronize();
    delete h;
  }
  API_END
}

int64_t xpinn_num_params(xpinn_handle h) { return h ? h->n_params : -1; }

int xpinn_get_params(xpinn_handle h, float* dst, int64_t n, void* stream) {
  API_BEGIN
  if (!h || !dst || n != h->n_params) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  copy_out(dst, h->params.p, n * sizeof(float), (cudaStream_t)stream);
  API_END
}

int xpinn_set_params(xpinn_handle h, const float* src, int64_t n, void* stream) {
  API_BEGIN
  if (!h || !src || n != h->n_params) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  copy_in(h->params.p, src, n * sizeof(float), (cudaStream_t)stream);
  h->img_stale = h->tc_stale = true;
  API_END
}

int xpinn_grad(xpinn_handle h, float* losses, float* grads, void* stream) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "NULL handle");
  DeviceGuard dg(h);
  cudaStream_t s = (cudaStream_t)stream;
  enqueue_step(h, s, false, h->grads.p);
  h->host_slot += 1;
  const int slot = h->host_slot % h->ring_cap;
  if (losses)
    copy_out(losses, h->loss_ring.p + (size_t)slot * h->n_sub * XPINN_N_TERMS,
             sizeof(float) * h->n_sub * XPINN_N_TERMS, s);
  if (grads) copy_out(grads, h->grads.p, sizeof(float) * h->n_params, s);
  check_device_error(h, s);
  API_END
}

int xpinn_step(xpinn_handle h, int32_t n_steps, float* losses, void* stream) {
  API_BEGIN
  if (!h || n_steps < 0) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t row = (size_t)h->n_sub * XPINN_N_TERMS;
  const bool dev_out = losses && is_device_ptr(losses);
  int done = 0;
  while (done < n_steps) {
    const int chunk = std::min(n_steps - done, h->ring_cap);
    const int first_slot = h->host_slot + 1;
    for (int i = 0; i < chunk;) {
      // runs of GRAPH_STEPS steps replay one graph that holds them all (a
      // launch-bound problem then pays the graph launch once per run); with
      // profile_phases the phase events must mark one step, so steps replay
      // one at a time
      const int g = (h->opt.use_graph && !h->opt.profile_phases && chunk - i >= GRAPH_STEPS) ? GRAPH_STEPS : 1;
      if (h->opt.use_graph) {
        cudaGraphExec_t& ge = g > 1 ? h->graph_multi : h->graph;
        if (!ge) {
          if (!h->cap_stream) ck(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "stream");
          cudaGraph_t gr;
          ck(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
          try {
            for (int k = 0; k < g; ++k) enqueue_step(h, h->cap_stream, true, nullptr);
          } catch (...) {
            cudaStreamEndCapture(h->cap_stream, &gr);
            throw;
          }
          ck(cudaStreamEndCapture(h->cap_stream, &gr), "end capture");
          ck(cudaGraphInstantiate(&ge, gr, 0), "instantiate");
          cudaGraphDestroy(gr);
        }
        ck(cudaGraphLaunch(ge, s), "graph launch");
      } else {
        enqueue_step(h, s, true, nullptr);
      }
      h->host_slot += g;
      h->host_t += g;
      i += g;
    }
    if (losses) {
      for (int i = 0; i < chunk; ++i) {
        const int slot = (first_slot + i) % h->ring_cap;
        float* dst = losses + (size_t)(done + i) * row;
        if (dev_out)
          ck(cudaMemcpyAsync(dst, h->loss_ring.p + slot * row, row * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy");
        else
          ck(cudaMemcpyAsync(dst, h->loss_ring.p + slot * row, row * sizeof(float), cudaMemcpyDeviceToHost, s), "copy");
      }
      if (!dev_out) ck(cudaStreamSynchronize(s), "sync");
    }
    done += chunk;
  }
  h->img_stale = h->tc_stale = true;
  ck(cudaGetLastError(), "step");
  // Host losses: the call has synchronised anyway, so the status word is
  // read now.  NULL or device losses: the call stays asynchronous and a
  // timeout or non-finite loss is reported by the next synchronising call
  // (xpinn_sync).
  if (losses && !dev_out) check_device_error(h, s);
  if (losses && !dev_out) {
    for (size_t i = 0; i < (size_t)n_steps * row; ++i)
      if (!std::isfinite(losses[i])) fail(XPINN_ERR_NONFINITE, "loss became non-finite");
  }
  API_END
}

int xpinn_objective(xpinn_handle h, float* J, float* J_sub, float* losses, float* grads, void* stream) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "NULL handle");
  DeviceGuard dg(h);
  cudaStream_t s = (cudaStream_t)stream;
  enqueue_step(h, s, false, h->grads.p);
  h->host_slot += 1;
  const int slot = h->host_slot % h->ring_cap;
  if (J) {
    launch_objective_sum(h->jq.p, h->n_sub, h->jq.p + h->n_sub, s);
    ck(cudaGetLastError(), "objective launch");
    copy_out(J, h->jq.p + h->n_sub, sizeof(float), s);
  }
  if (J_sub) copy_out(J_sub, h->jq.p, sizeof(float) * h->n_sub, s);
  if (losses)
    copy_out(losses, h->loss_ring.p + (size_t)slot * h->n_sub * XPINN_N_TERMS,
             sizeof(float) * h->n_sub * XPINN_N_TERMS, s);
  if (grads) copy_out(grads, h->grads.p, sizeof(float) * h->n_params, s);
  check_device_error(h, s);
  API_END
}

int xpinn_fork_workspace_size(xpinn_handle h, const xpinn_fork_desc* d, size_t* bytes) {
  API_BEGIN
  if (!h || !bytes) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  *bytes = make_fork(h, d)->L.total;
  API_END
}

}  // extern "C"

namespace xp {
// The request server's fork: sizes, then the enqueue with device outputs and
// the host tables staged in page-locked memory (nothing waits on the GPU).
int fork_sizes(xpinn_handle h, const xpinn_fork_desc* d, size_t* ws_bytes, size_t* table_bytes) {
  API_BEGIN
  DeviceGuard dg(h);
  auto F = make_fork(h, d);
  *ws_bytes = F->L.total;
  *table_bytes = fork_table_bytes(*F);
  API_END
}

int fork_enqueue(xpinn_handle h, const xpinn_fork_desc* d, void* workspace, size_t ws_bytes, float* dev_losses,
                 float* dev_params, char* pinned, cudaStream_t s) {
  API_BEGIN
  DeviceGuard dg(h);
  auto F = make_fork(h, d);
  if (ws_bytes < F->L.total) fail(XPINN_ERR_INVALID, "workspace of %zu bytes, %zu needed", ws_bytes, F->L.total);
  bind_fork(h, *F, static_cast<char*>(workspace), d, s, pinned);
  xpinn_ctx* f = F->f.get();
  for (int i = 0; i < d->n_steps; ++i) enqueue_step(f, s, true, nullptr);
  const size_t row = (size_t)F->n_sel * XPINN_N_TERMS;
  for (int i = 0; dev_losses && i < d->n_steps; ++i)
    ck(cudaMemcpyAsync(dev_losses + i * row, f->loss_ring.p + (size_t)((i + 1) % f->ring_cap) * f->n_sub * XPINN_N_TERMS,
                       sizeof(float) * row, cudaMemcpyDeviceToDevice, s),
       "fork losses");
  if (dev_params)
    ck(cudaMemcpyAsync(dev_params, f->params.p, sizeof(float) * F->n_params_sel, cudaMemcpyDeviceToDevice, s),
       "fork params");
  ck(cudaGetLastError(), "fork launches");
  API_END
}
}  // namespace xp

extern "C" {

int xpinn_fork_step(xpinn_handle h, const xpinn_fork_desc* d, void* workspace, size_t ws_bytes, float* losses,
                    float* params, void* stream) {
  API_BEGIN
  if (!h || !workspace) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  cudaStream_t s = (cudaStream_t)stream;
  auto F = make_fork(h, d);
  if (ws_bytes < F->L.total) fail(XPINN_ERR_INVALID, "workspace of %zu bytes, %zu needed", ws_bytes, F->L.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256) fail(XPINN_ERR_INVALID, "workspace must be 256-byte aligned");
  if (!is_device_ptr(workspace)) fail(XPINN_ERR_INVALID, "workspace must be device memory");
  bind_fork(h, *F, static_cast<char*>(workspace), d, s);
  xpinn_ctx* f = F->f.get();
  for (int i = 0; i < d->n_steps; ++i) enqueue_step(f, s, true, nullptr);
  bool host_out = false;
  if (losses && d->n_steps > 0) {
    const bool dev = is_device_ptr(losses);
    host_out = host_out || !dev;
    const size_t row = (size_t)F->n_sel * XPINN_N_TERMS;
    for (int i = 0; i < d->n_steps; ++i) {
      const int slot = (i + 1) % f->ring_cap;   // the loss slot advances once per step
      ck(cudaMemcpyAsync(losses + i * row, f->loss_ring.p + (size_t)slot * f->n_sub * XPINN_N_TERMS,
                         sizeof(float) * row, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
         "fork losses");
    }
  }
  if (params) {
    const bool dev = is_device_ptr(params);
    host_out = host_out || !dev;
    ck(cudaMemcpyAsync(params, f->params.p, sizeof(float) * F->n_params_sel,
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
       "fork params");
  }
  ck(cudaGetLastError(), "fork launches");
  if (host_out) check_device_error(h, s);   // synchronises
  API_END
}

int xpinn_step_begin(xpinn_handle h, void* stream) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "NULL handle");
  if (h->step_open) fail(XPINN_ERR_INVALID, "xpinn_step_begin called twice without xpinn_step_end");
  DeviceGuard dg(h);
  enqueue_step(h, (cudaStream_t)stream, true, nullptr, 1);
  h->step_open = true;
  API_END
}

int xpinn_step_end(xpinn_handle h, float* losses, void* stream) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "NULL handle");
  if (!h->step_open) fail(XPINN_ERR_INVALID, "xpinn_step_end without xpinn_step_begin");
  DeviceGuard dg(h);
  cudaStream_t s = (cudaStream_t)stream;
  h->step_open = false;
  enqueue_step(h, s, true, nullptr, 2);
  h->host_slot += 1;
  h->host_t += 1;
  h->img_stale = h->tc_stale = true;
  if (losses) {
    const size_t row = (size_t)h->n_sub * XPINN_N_TERMS;
    copy_out(losses, h->loss_ring.p + (size_t)(h->host_slot % h->ring_cap) * row, sizeof(float) * row, s);
    if (!is_device_ptr(losses)) check_device_error(h, s);
  }
  API_END
}

}  // extern "C"

namespace {
// Remote interfaces in interface order: (exchange-buffer row of the first
// point, points).
std::vector<std::pair<int64_t, int>> remote_ifaces(const xpinn_ctx* h) {
  std::vector<std::pair<int64_t, int>> r;
  for (const IfaceDev& f : h->ifaces)
    if (f.remote) r.emplace_back(f.d4_pt, f.n_pts);
  return r;
}
}  // namespace

extern "C" {

int xpinn_remote_values(xpinn_handle h, float* out, int64_t* n_floats, void* stream) {
  API_BEGIN
  if (!h || !n_floats) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  const auto rem = remote_ifaces(h);
  int64_t need = 0;
  for (const auto& e : rem) need += (int64_t)e.second * h->d4_nv;
  if (!out) {
    *n_floats = need;
    g_err.clear();
    return XPINN_OK;
  }
  if (*n_floats < need) fail(XPINN_ERR_INVALID, "buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nv = h->d4_nv;
  int64_t off = 0;
  for (const auto& e : rem) {
    if (e.second)
      ck(cudaMemcpy2DAsync(out + off, nv * sizeof(float), h->d4.p + (size_t)e.first * 2 * nv, 2 * nv * sizeof(float),
                           nv * sizeof(float), e.second, cudaMemcpyDefault, s),
         "remote values out");
    off += (int64_t)e.second * nv;
  }
  if (!is_device_ptr(out)) ck(cudaStreamSynchronize(s), "sync");
  *n_floats = need;
  API_END
}

int xpinn_set_remote_values(xpinn_handle h, const float* in, int64_t n_floats, void* stream) {
  API_BEGIN
  if (!h || (!in && n_floats)) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  const auto rem = remote_ifaces(h);
  int64_t need = 0;
  for (const auto& e : rem) need += (int64_t)e.second * h->d4_nv;
  if (n_floats != need) fail(XPINN_ERR_INVALID, "%lld floats given, %lld expected", (long long)n_floats, (long long)need);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nv = h->d4_nv;
  int64_t off = 0;
  for (const auto& e : rem) {
    if (e.second)
      ck(cudaMemcpy2DAsync(h->d4.p + ((size_t)e.first * 2 + 1) * nv, 2 * nv * sizeof(float), in + off,
                           nv * sizeof(float), nv * sizeof(float), e.second, cudaMemcpyDefault, s),
         "remote values in");
    off += (int64_t)e.second * nv;
  }
  if (need && !is_device_ptr(in)) ck(cudaStreamSynchronize(s), "sync");
  API_END
}

int xpinn_sync(xpinn_handle h, void* stream) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "NULL handle");
  DeviceGuard dg(h);
  check_device_error(h, (cudaStream_t)stream);
  API_END
}

int xpinn_net_jets(xpinn_handle h, int32_t q, int32_t net, const float* xy, int64_t n, int32_t order,
                   float* out, void* stream) {
  API_BEGIN
  if (!h || q < 0 || q >= h->n_sub || net < 0 || net >= h->subs[q].n_nets || order < 0 || order > 2 ||
      n < 0 || (n > 0 && (!xy || !out)))
    fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (n == 0) { g_err.clear(); return XPINN_OK; }
  cudaStream_t s = (cudaStream_t)stream;
  const int K = order == 0 ? 1 : (order == 1 ? 3 : 5);
  const NetDev& nd = h->subs[q].net[net];
  const int dout = nd.w[nd.L] * K;
  const bool dev = is_device_ptr(xy);
  const float2* pts;
  if (dev) {
    pts = reinterpret_cast<const float2*>(xy);
  } else {
    h->e_pts.ensure(n);
    copy_in(h->e_pts.p, xy, n * sizeof(float2), s);
    pts = h->e_pts.p;
  }
  float* o = out;
  if (!is_device_ptr(out)) {
    h->e_out.ensure((size_t)n * dout);
    o = h->e_out.p;
  }
  std::vector<Item> items;
  eval_items_for(h, q, net, K, 0, n, 0, dout, items);
  run_eval_items(h, items, pts, o, dout, nullptr, s);
  if (o != out) copy_out(out, o, sizeof(float) * n * dout, s);
  API_END
}

int xpinn_eval_workspace_size(xpinn_handle h, int32_t model, int64_t n, int32_t order, size_t* bytes) {
  API_BEGIN
  if (!h || !bytes || model < 0 || model >= h->n_sub / h->spm || order < 0 || order > 2 || n < 0)
    fail(XPINN_ERR_INVALID, "bad arguments");
  *bytes = eval_ws_layout(h, model, n, order).total;
  API_END
}

int xpinn_eval(xpinn_handle h, int32_t model, const float* xy, int64_t n, int32_t order, float* out,
               void* stream) {
  API_BEGIN
  if (!h || model < 0 || model >= h->n_sub / h->spm || order < 0 || order > 2 || n < 0 ||
      (n > 0 && (!xy || !out)))
    fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (n == 0) { g_err.clear(); return XPINN_OK; }
  const EvalWs L = eval_ws_layout(h, model, n, order);
  h->e_ws.ensure(L.total);
  eval_with_ws(h, model, xy, n, order, out, h->e_ws.p, h->e_ws.n, (cudaStream_t)stream);
  API_END
}

int xpinn_eval_ws(xpinn_handle h, int32_t model, const float* xy, int64_t n, int32_t order, float* out,
                  void* workspace, size_t ws_bytes, void* stream) {
  API_BEGIN
  if (!h || model < 0 || model >= h->n_sub / h->spm || order < 0 || order > 2 || n < 0 ||
      (n > 0 && (!xy || !out || !workspace)))
    fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (n == 0) { g_err.clear(); return XPINN_OK; }
  if (!is_device_ptr(workspace)) fail(XPINN_ERR_INVALID, "workspace must be device memory");
  eval_with_ws(h, model, xy, n, order, out, static_cast<char*>(workspace), ws_bytes, (cudaStream_t)stream);
  API_END
}

int xpinn_set_residual_points(xpinn_handle h, const float* xy, const float* f, int64_t n, void* stream) {
  API_BEGIN
  if (!h || !xy || n != h->n_res_total) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  cudaStream_t s = (cudaStream_t)stream;
  copy_in(h->pts.p, xy, n * sizeof(float2), s);
  if (f)
    copy_in(h->res_f.p, f, n * sizeof(float), s);
  else
    ck(cudaMemsetAsync(h->res_f.p, 0, n * sizeof(float), s), "memset");
  API_END
}

namespace {
struct StateHeader {
  char magic[8];
  int32_t version;
  int32_t step_t;
  int64_t n_params;
  int64_t n_sub;
};
}  // namespace

int xpinn_get_state(xpinn_handle h, void* blob, size_t* n) {
  API_BEGIN
  if (!h || !n) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  const size_t need = sizeof(StateHeader) + 3 * sizeof(float) * h->n_params;
  if (!blob) {
    *n = need;
    g_err.clear();
    return XPINN_OK;
  }
  if (*n < need) fail(XPINN_ERR_INVALID, "state buffer too small (%zu < %zu)", *n, need);
  StateHeader hd{};
  memcpy(hd.magic, "XPINNST1", 8);
  hd.version = 1;
  int t = 0;
  ck(cudaMemcpy(&t, h->step_t(), sizeof(int), cudaMemcpyDeviceToHost), "state");
  hd.step_t = t;
  hd.n_params = h->n_params;
  hd.n_sub = h->n_sub;
  char* b = static_cast<char*>(blob);
  memcpy(b, &hd, sizeof hd);
  float* p = reinterpret_cast<float*>(b + sizeof hd);
  ck(cudaMemcpy(p, h->params.p, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost), "state");
  ck(cudaMemcpy(p + h->n_params, h->m.p, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost), "state");
  ck(cudaMemcpy(p + 2 * h->n_params, h->v.p, sizeof(float) * h->n_params, cudaMemcpyDeviceToHost), "state");
  *n = need;
  API_END
}

int xpinn_set_state(xpinn_handle h, const void* blob, size_t n) {
  API_BEGIN
  if (!h || !blob) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  const size_t need = sizeof(StateHeader) + 3 * sizeof(float) * h->n_params;
  StateHeader hd;
  if (n < sizeof hd) fail(XPINN_ERR_INVALID, "state blob too small");
  memcpy(&hd, blob, sizeof hd);
  if (memcmp(hd.magic, "XPINNST1", 8) || hd.version != 1) fail(XPINN_ERR_INVALID, "not a state blob");
  if (hd.n_params != h->n_params || hd.n_sub != h->n_sub || n != need)
    fail(XPINN_ERR_INVALID, "state blob of another problem shape");
  const float* p = reinterpret_cast<const float*>(static_cast<const char*>(blob) + sizeof hd);
  ck(cudaDeviceSynchronize(), "sync");
  ck(cudaMemcpy(h->params.p, p, sizeof(float) * h->n_params, cudaMemcpyHostToDevice), "state");
  ck(cudaMemcpy(h->m.p, p + h->n_params, sizeof(float) * h->n_params, cudaMemcpyHostToDevice), "state");
  ck(cudaMemcpy(h->v.p, p + 2 * h->n_params, sizeof(float) * h->n_params, cudaMemcpyHostToDevice), "state");
  h->img_stale = h->tc_stale = true;
  ck(cudaMemcpy(h->step_t(), &hd.step_t, sizeof(int), cudaMemcpyHostToDevice), "state");
  h->host_t = hd.step_t;
  API_END
}

int xpinn_get_options(xpinn_handle h, xpinn_options* opt) {
  API_BEGIN
  if (!h || !opt) fail(XPINN_ERR_INVALID, "bad arguments");
  *opt = h->opt;
  API_END
}

int xpinn_set_options(xpinn_handle h, const xpinn_options* opt) {
  API_BEGIN
  if (!h || !opt) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (opt->schedule < 0 || opt->schedule > 1 || opt->items_per_cta < 1 || opt->items_per_cta > 64 ||
      opt->points_per_thread < 1 || opt->points_per_thread > 2 || opt->profile_phases < 0 ||
      opt->profile_phases > 1 || opt->max_points_per_tile < 0 ||
      (opt->threads_per_cta != 0 && opt->threads_per_cta != 128 && opt->threads_per_cta != 256 &&
       opt->threads_per_cta != 512) || opt->inject_fault < 0 || opt->inject_fault > 1 ||
      (opt->threads_per_cta == 512 && opt->points_per_thread != 1) || opt->eval_tensor_cores < 0 ||
      opt->eval_tensor_cores > 1 || opt->train_tensor_cores < 0 || opt->train_tensor_cores > STC_W)
    fail(XPINN_ERR_INVALID, "bad options");
  ck(cudaDeviceSynchronize(), "sync");
  apply_options(h, *opt);
  API_END
}

}  // extern "C"

namespace {
// Median device time (ms) of `steps` gradient passes after two warm-up passes.
float time_grads(xpinn_ctx* h, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int steps) {
  // warm-up: two passes, one when a pass takes more than 50 ms (long launches
  // are stable after one, and the tuners' time budget buys more candidates)
  for (int w = 0; w < 2; ++w) {
    ck(cudaEventRecord(e0, s), "event");
    enqueue_step(h, s, false, h->grads.p);
    h->host_slot += 1;
    ck(cudaEventRecord(e1, s), "event");
    ck(cudaEventSynchronize(e1), "event sync");
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    if (ms > 50.f) break;
  }
  std::vector<float> t;
  for (int i = 0; i < steps; ++i) {
    ck(cudaEventRecord(e0, s), "event");
    enqueue_step(h, s, false, h->grads.p);
    h->host_slot += 1;
    ck(cudaEventRecord(e1, s), "event");
    ck(cudaEventSynchronize(e1), "event sync");
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    t.push_back(ms);
  }
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Shape class of a subdomain: its networks' widths, activations, slopes and
// output activations (subdomains of one class run the same tile code).
std::string shape_key(const SubDev& sd) {
  std::string k;
  for (int n = 0; n < sd.n_nets; ++n) {
    const NetDev& nd = sd.net[n];
    for (int l = 0; l <= nd.L; ++l) k += std::to_string(nd.w[l]) + ",";
    k += "a" + std::to_string(nd.act) + (nd.aoff >= 0 ? "s" : "f") + "o" + std::to_string(nd.out_act) + "|";
  }
  return k;
}
}  // namespace

extern "C" {

int xpinn_get_tile_caps(xpinn_handle h, int32_t* caps) {
  API_BEGIN
  if (!h || !caps) fail(XPINN_ERR_INVALID, "bad arguments");
  for (int q = 0; q < h->n_sub; ++q) caps[q] = h->tile_cap.empty() ? 0 : h->tile_cap[q];
  API_END
}

int xpinn_set_tile_caps(xpinn_handle h, const int32_t* caps) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (caps)
    for (int q = 0; q < h->n_sub; ++q)
      if (caps[q] < 0 || (caps[q] > 0 && caps[q] < 8)) fail(XPINN_ERR_INVALID, "tile cap must be 0 or >= 8");
  ck(cudaDeviceSynchronize(), "sync");
  if (caps)
    h->tile_cap.assign(caps, caps + h->n_sub);
  else
    h->tile_cap.clear();
  apply_options(h, h->opt);
  API_END
}

int xpinn_get_tc_select(xpinn_handle h, int32_t* sel) {
  API_BEGIN
  if (!h || !sel) fail(XPINN_ERR_INVALID, "bad arguments");
  for (int q = 0; q < h->n_sub; ++q) sel[q] = h->tc_sel.empty() ? -1 : h->tc_sel[q];
  API_END
}

int xpinn_set_tc_select(xpinn_handle h, const int32_t* sel) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (sel)
    for (int q = 0; q < h->n_sub; ++q)
      if (sel[q] < -1 || sel[q] > 1) fail(XPINN_ERR_INVALID, "tensor-core selection must be -1, 0 or 1");
  ck(cudaDeviceSynchronize(), "sync");
  if (sel)
    h->tc_sel.assign(sel, sel + h->n_sub);
  else
    h->tc_sel.clear();
  apply_options(h, h->opt);
  API_END
}

int xpinn_autotune_shapes(xpinn_handle h, int32_t steps, float* best_ms) {
  API_BEGIN
  if (!h || steps < 1) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  ck(cudaDeviceSynchronize(), "sync");
  // classes, largest modelled share of the step first
  std::vector<std::string> keys;
  std::vector<double> share;
  std::vector<std::vector<int>> members;
  for (int q = 0; q < h->n_sub; ++q) {
    const std::string k = shape_key(h->subs[q]);
    size_t c = std::find(keys.begin(), keys.end(), k) - keys.begin();
    if (c == keys.size()) {
      keys.push_back(k);
      share.push_back(0);
      members.emplace_back();
    }
    members[c].push_back(q);
  }
  for (const Item& it : h->plan.items) {
    const size_t c = std::find(keys.begin(), keys.end(), shape_key(h->subs[it.q])) - keys.begin();
    share[c] += item_cost(h->subs[it.q], it, cta_threads(h));
  }
  std::vector<size_t> order(keys.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return share[a] > share[b]; });
  if (h->tile_cap.empty()) h->tile_cap.assign(h->n_sub, 0);
  const std::vector<int> orig = h->tile_cap;
  const std::vector<int> orig_sel = h->tc_sel;
  const xpinn_options orig_opt = h->opt;
  xpinn_options topt = h->opt;
  topt.profile_phases = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  const auto t_start = std::chrono::steady_clock::now();
  auto elapsed_s = [&] {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  };
  float best = 0;
  try {
    apply_options(h, topt);
    best = time_grads(h, s, e0, e1, steps);
    for (size_t c : order) {
      int keep = h->tile_cap[members[c][0]];
      for (int cap : {128, 96, 64, 48, 32, 160, 0}) {
        if (cap == keep || elapsed_s() > 20.0) continue;
        for (int q : members[c]) h->tile_cap[q] = cap;
        try {
          apply_options(h, topt);
        } catch (const Error&) {
          for (int q : members[c]) h->tile_cap[q] = keep;
          continue;
        }
        const float t = time_grads(h, s, e0, e1, steps);
        if (t < best * 0.995f) {   // keep a choice only for a clear gain
          best = t;
          keep = cap;
        }
      }
      for (int q : members[c]) h->tile_cap[q] = keep;
    }
    // then, for classes whose networks the tensor-core kernel takes, that
    // kernel on and off for their residual items
    if (h->tc_sel.empty()) h->tc_sel.assign(h->n_sub, -1);
    for (size_t c : order) {
      const SubDev& sd = h->subs[members[c][0]];
      if (!step_tc_net_ok(sd.net[0], sd.n_nets, h->pde, h->opt.train_tensor_cores)) continue;
      int keep = h->tc_sel[members[c][0]];
      for (int sel : {1, 0}) {
        if (sel == keep || elapsed_s() > 30.0) continue;
        for (int q : members[c]) h->tc_sel[q] = sel;
        apply_options(h, topt);
        const float t = time_grads(h, s, e0, e1, steps);
        if (t < best * 0.995f) {
          best = t;
          keep = sel;
        }
      }
      for (int q : members[c]) h->tc_sel[q] = keep;
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    h->tile_cap = orig;
    h->tc_sel = orig_sel;
    apply_options(h, orig_opt);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  apply_options(h, orig_opt);
  if (best_ms) *best_ms = best;
  API_END
}

int xpinn_autotune(xpinn_handle h, int32_t steps, xpinn_options* best, float* best_ms) {
  API_BEGIN
  if (!h || steps < 1 || !best) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  ck(cudaDeviceSynchronize(), "sync");
  const xpinn_options orig = h->opt;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  xpinn_options win = orig;
  float win_ms = 3.4e38f;
  const auto t_start = std::chrono::steady_clock::now();
  auto elapsed_s = [&] {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  };
  // The grid of CTA shapes (threads, points per thread) x items per CTA,
  // without a tile cap: the default first, then every change of one of the
  // two from it, then the remaining pairs; then the tile caps on the best
  // pair.  Passes longer than 200 ms are timed once per candidate (their
  // spread is small); the search stops after about 30 s, keeping the best.
  struct Cand {
    int nt, pt, ipc, cap;
  };
  const std::vector<std::pair<int, int>> shapes = {{256, 2}, {256, 1}, {512, 1}, {128, 2}, {128, 1}};
  const std::vector<int> ipcs = {4, 8, 16, 2, 32};
  std::vector<Cand> grid;
  for (size_t a = 0; a < shapes.size(); ++a)
    for (size_t b = 0; b < ipcs.size(); ++b)
      if (a == 0 || b == 0) grid.push_back({shapes[a].first, shapes[a].second, ipcs[b], 0});
  for (size_t a = 1; a < shapes.size(); ++a)
    for (size_t b = 1; b < ipcs.size(); ++b) grid.push_back({shapes[a].first, shapes[a].second, ipcs[b], 0});
  int n_steps = steps;
  Cand best_c = grid[0];
  float best_t = 3.4e38f;
  auto run = [&](const Cand& cd) {
    xpinn_options c = orig;
    c.schedule = 0;
    c.points_per_thread = cd.pt;
    c.items_per_cta = cd.ipc;
    c.max_points_per_tile = cd.cap;
    c.threads_per_cta = cd.nt;
    c.profile_phases = 0;
    try {
      apply_options(h, c);
    } catch (const Error&) {
      return;   // does not fit: skip
    }
    const float med = time_grads(h, s, e0, e1, n_steps);
    if (med > 200.f) n_steps = 1;
    if (med < win_ms) {
      win_ms = med;
      win = c;
    }
    if (med < best_t) {
      best_t = med;
      best_c = cd;
    }
  };
  try {
    for (const Cand& cd : grid) {
      if (elapsed_s() > 30.0) break;
      run(cd);
    }
    for (int cap : {64, 128, 32}) {
      if (elapsed_s() > 30.0) break;
      Cand cd = best_c;
      cd.cap = cap;
      run(cd);
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    apply_options(h, orig);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  win.schedule = orig.schedule;
  win.use_graph = orig.use_graph;
  win.profile_phases = orig.profile_phases;
  apply_options(h, win);
  *best = h->opt;
  if (best_ms) *best_ms = win_ms;
  API_END
}

int xpinn_phase_times(xpinn_handle h, float* ms) {
  API_BEGIN
  if (!h || !ms) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (!h->opt.profile_phases || !h->ev[0]) fail(XPINN_ERR_INVALID, "profile_phases is off");
  ck(cudaEventSynchronize(h->ev[4]), "event sync");
  for (int i = 0; i < 4; ++i) ck(cudaEventElapsedTime(ms + i, h->ev[i], h->ev[i + 1]), "elapsed");
  API_END
}

int xpinn_plan_counts(xpinn_handle h, int32_t* n_items, int32_t* n_tc, int32_t* n_tc_sub) {
  API_BEGIN
  if (!h) fail(XPINN_ERR_INVALID, "bad arguments");
  const Plan& pl = h->plan;
  if (n_items) *n_items = (int32_t)pl.items.size();
  if (n_tc) *n_tc = pl.n_tc;
  if (n_tc_sub) {
    std::vector<char> seen(h->n_sub, 0);
    int c = 0;
    for (int i = pl.n_simt(); i < (int)pl.items.size(); ++i)
      if (!seen[pl.items[i].q]) {
        seen[pl.items[i].q] = 1;
        ++c;
      }
    *n_tc_sub = c;
  }
  API_END
}

int xpinn_tc_subdomains(xpinn_handle h, int32_t* on) {
  API_BEGIN
  if (!h || !on) fail(XPINN_ERR_INVALID, "bad arguments");
  const Plan& pl = h->plan;
  for (int q = 0; q < h->n_sub; ++q) on[q] = 0;
  for (int i = pl.n_simt(); i < (int)pl.items.size(); ++i) on[pl.items[i].q] = 1;
  API_END
}

int xpinn_tc_kernel_time(xpinn_handle h, float* ms) {
  API_BEGIN
  if (!h || !ms) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (!h->tc_timed) fail(XPINN_ERR_INVALID, "no grouped step with tensor-core items timed (profile_phases off)");
  ck(cudaEventSynchronize(h->ev[5]), "event sync");
  ck(cudaEventElapsedTime(ms, h->ev[2], h->ev[5]), "elapsed");
  API_END
}

int xpinn_eval_kernel_time(xpinn_handle h, float* ms) {
  API_BEGIN
  if (!h || !ms) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  if (!h->eval_timed) fail(XPINN_ERR_INVALID, "no routed evaluation timed (profile_phases off)");
  ck(cudaEventSynchronize(h->eval_ev[1]), "event sync");
  ck(cudaEventElapsedTime(ms, h->eval_ev[0], h->eval_ev[1]), "elapsed");
  API_END
}

int xpinn_iface_values(xpinn_handle h, float* out, int64_t* n_floats, void* stream) {
  API_BEGIN
  if (!h || !n_floats) fail(XPINN_ERR_INVALID, "bad arguments");
  DeviceGuard dg(h);
  const int64_t need = h->n_if_pts * 2 * h->d4_nv;
  if (!out) {
    *n_floats = need;
    g_err.clear();
    return XPINN_OK;
  }
  if (*n_floats < need) fail(XPINN_ERR_INVALID, "buffer too small");
  copy_out(out, h->d4.p, sizeof(float) * need, (cudaStream_t)stream);
  *n_floats = need;
  API_END
}

}  // extern "C"
