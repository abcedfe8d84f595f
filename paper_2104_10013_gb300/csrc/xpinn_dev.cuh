// Device-side data layout shared by the kernels and the host planner.
//
// The whole problem lives in a handful of flat device arrays:
//   params / m / v / grads : the packed parameter vector (layout of xpinn.h)
//   pts                    : every training point as float2, grouped as
//                            [residual points of all subdomains]
//                            [data points of all subdomains and nets]
//                            [interface points of all interfaces]
//   res_f                  : forcing at residual points (indexed like pts)
//   tgt                    : data targets [point][D_out]
//   d4                     : interface exchange buffer
//                            [interface point][side][u..., exchanged qty...]
// A step is a list of work items (one subdomain, one point kind, one range of
// points).  Each item writes its gradient contribution to a private slice of
// `partials` and its loss sums to `loss_part`; a second kernel sums the slices
// of each subdomain in a fixed order, so results do not depend on which CTA
// ran which item.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "xpinn.h"

namespace xp {

constexpr int NT = 256;          // threads per CTA of the jet kernel (the largest; 128 also exists)
constexpr int MT = 8;            // neurons in a thread's register tile
constexpr int KMAX = 5;          // jet components (u, d0, d1, d00, d11)
constexpr int MAXL = XPINN_MAX_LAYERS;
constexpr int MAXNETS = XPINN_MAX_NETS;
constexpr int MAXW = XPINN_MAX_WIDTH;

enum ItemKind : int {
  IT_RES = 0,        // residual points: MSE_F
  IT_DATA0 = 1,      // data points of net 0: MSE_u
  IT_DATA1 = 2,      // data points of net 1: MSE_u
  IT_IFACE = 3,      // one side of an interface: MSE_uavg + MSE_flux / MSE_R
  IT_IFACE_FWD = 4,  // one side of an interface, forward only: writes d4
  IT_EVAL = 5,       // jets at caller points (xpinn_net_jets / xpinn_eval)
};

struct NetDev {
  int L;                 // weight layers
  int out_act;           // XPINN_ACT_*
  int w[MAXL + 1];       // widths N_0..N_L
  int wp[MAXL + 1];      // widths padded to a multiple of MT
  int off[MAXL + 1];     // offset of W^k inside the subdomain's parameters (k >= 1);
                         // b^k follows W^k
  int act;               // hidden activation XPINN_PHI_*
  int aoff;              // offset of the slopes a^1..a^{L-1}, or -1 (slopes fixed, n a^k = 1)
  float scale;           // n of n a^k
  int end;               // one past the network's last parameter
  // Weight images of the hidden-to-hidden layers k = 2..L-1 (offsets in
  // floats from the subdomain's image block), copied whole into shared
  // memory by the jet kernel:
  //   imf[k]: forward image, W^k transposed and zero-padded [wp[k-1]][wp[k]],
  //           then b^k zero-padded [wp[k]];
  //   imb[k]: reverse image, W^k zero-padded [wp[k]][wp[k-1]].
  int imf[MAXL + 1];
  int imb[MAXL + 1];
};

// Row stride (floats) of the adjoint rows [c][p] of one neuron in the
// reverse pass: K * P, padded by 4 when it is a multiple of 16, so that
// adjacent rows start in different shared-memory banks.
__host__ __device__ inline int adj_stride(int K, int P) {
  const int kp = K * P;
  return kp + ((kp & 15) == 0 ? 4 : 0);
}

// Floats of the forward image of layer k (the larger of the two).
__host__ __device__ inline int layer_img_floats(const NetDev& nd, int k) {
  return (nd.wp[k - 1] + 1) * nd.wp[k];
}

// Assigns the image offsets of a network starting at `ioff`; returns the end.
inline int assign_images(NetDev& nd, int ioff) {
  for (int k = 0; k <= MAXL; ++k) nd.imf[k] = nd.imb[k] = -1;
  for (int k = 2; k < nd.L; ++k) {
    nd.imf[k] = ioff;
    ioff += layer_img_floats(nd, k);
    nd.imb[k] = ioff;
    ioff += nd.wp[k] * nd.wp[k - 1];
  }
  return ioff;
}

// A network that is not tanh with fixed slopes needs the general passes.
__host__ __device__ inline bool net_is_general(const NetDev& nd) {
  return !(nd.act == XPINN_PHI_TANH && nd.aoff < 0);
}

// Fills the layout fields of a NetDev from a network description whose
// parameters start at `off` in the subdomain's block; returns the offset
// one past them.  Layout: W^1, b^1, ..., W^L, b^L, then the slopes.
inline int fill_net_dev(NetDev& nd, const xpinn_net_desc& n, int off) {
  nd.L = n.n_layers;
  nd.out_act = n.out_act;
  nd.act = n.act;
  for (int k = 0; k <= nd.L; ++k) {
    nd.w[k] = n.widths[k];
    nd.wp[k] = (nd.w[k] + MT - 1) / MT * MT;
  }
  for (int k = 1; k <= nd.L; ++k) {
    nd.off[k] = off;
    off += nd.w[k] * nd.w[k - 1] + nd.w[k];
  }
  nd.aoff = n.adaptive ? off : -1;
  nd.scale = n.adaptive ? n.slope_scale : 1.f;
  if (n.adaptive) off += nd.L - 1;
  nd.end = off;
  return off;
}

// ---------------------------------------------------------------------------
// Tile sizing shared by every planner of jet-kernel launches (the handle's
// step and evaluation plans and the allocation-free entry point), so that the
// shared memory and scratch a launch is given always match what the kernel
// addresses.
// ---------------------------------------------------------------------------
inline int max_hidden_wp(const NetDev& n) {
  int w = MT;
  for (int k = 1; k < n.L; ++k) w = w > n.wp[k] ? w : n.wp[k];
  return w;
}

struct SubDev {
  int n_nets;
  int n_params;
  int64_t poff;          // offset of the subdomain's parameters in the packed vector
  int64_t img_off;       // offset of the subdomain's weight images in wimg
  NetDev net[MAXNETS];
  float w_data[MAXNETS], w_res, w_avg, w_iface;
  float inv_n_res;
  float inv_n_data[MAXNETS];
  int64_t res_off;       // first residual point in pts
  int64_t data_off[MAXNETS];
  int64_t tgt_off[MAXNETS];   // first target float in tgt
  int n_res;
  int n_data[MAXNETS];
  float lr;
  float rect[4];
  int region_kind;       // XPINN_REGION_*
  float site[2];
};

struct IfaceDev {
  int q, qp, method;
  int n_pts;
  float nx, ny;
  float inv_n;
  int64_t pt_off;        // first point in pts
  int64_t d4_pt;         // first interface point index in d4
  int remote;            // 1: side 1 belongs to another rank; its d4 rows are set from outside
};

struct Item {
  int kind;
  int q;                 // subdomain
  int edge, side;        // interface items
  int n_pts;
  int P;                 // points per sub-tile
  int K[MAXNETS];        // jet components per net, 0 if the net is not evaluated
  int lap;               // 1: net 0 carries (u, d0 u, d1 u, d00 u + d11 u) in 4 components
  int64_t pt_off;        // first point (pts, or the eval point buffer)
  int64_t part_off;      // first float of this item's gradient slice (-1: none)
  int64_t out_off;       // eval: first output float; others unused
};

struct StepArgs {
  const Item* items;
  int n_items;
  int item_base;         // index of items[0] in the plan (loss_part slots)
  int* counter;          // work counter of this launch (reset before it)
  int* fwd_done;         // exchange items completed in this launch
  int wait_from;         // items from this index on read the exchange buffer:
  int n_fwd_wait;        // they wait until n_fwd_wait exchange items are done (0: no wait)
  const SubDev* subs;
  const IfaceDev* ifaces;
  const float* params;
  const float* wimg;     // weight images (see NetDev), rebuilt from params before each use
  const float2* pts;
  const float* res_f;
  const float* tgt;
  float* d4;
  int d4_nv;             // floats per (interface point, side)
  float* partials;
  double* loss_part;     // [n_items][2]
  float* scratch;        // per-CTA scratch for saved jets
  int64_t scratch_per_cta;
  int pde;
  float nu, re;
  int flux_mode;
  int n_out_total;       // outputs of all nets of a subdomain
  int n_eq;              // residual components
  // smem plan (floats)
  int szA, szW, szU;
  int pmax;              // largest sub-tile of any item
  int pt;                // points per thread in the register tile (1 or 2)
  int nt;                // threads per CTA (256, 128 or 512)
  int gen;               // 1: some network needs the general passes (general kernel)
  // eval
  const float2* eval_pts;
  float* eval_out;
  const float* eval_scale;   // per point weight (1/S) or NULL
  int eval_dout;             // output row stride in floats per point
  int* err;                  // device error flag (bounds checks)
  const int* n_items_dev;    // if not NULL: the number of items is min(n_items, *n_items_dev),
                             // written on the device by an earlier kernel (device-planned evaluation)
};

// Per subdomain of a model, how a routed evaluation cuts its bucket into
// items: the jet components of each network, the sub-tile and the entries
// per item.
struct EvalProto {
  int K0, K1, P, chunk;
};

// Points per sub-tile for an item evaluating the nets with K[n] > 0: enough
// (neuron group, point group) register tiles to occupy the CTA's nt threads
// at pt points per thread, at most 256 and `cap`, a multiple of 4 (>= 4).
inline int choose_P(const SubDev& sd, const int K[2], int cap, int pt, int nt) {
  int ng = 1, dk = 0;
  for (int n = 0; n < sd.n_nets; ++n)
    if (K[n]) {
      const int g = max_hidden_wp(sd.net[n]) / MT;
      ng = ng > g ? ng : g;
      dk += sd.net[n].w[sd.net[n].L] * K[n];
    }
  int P = (nt / ng) * pt;
  P = P < 256 ? P : 256;
  const int pd = 2048 / (dk > 1 ? dk : 1);
  P = P < (pd > 4 ? pd : 4) ? P : (pd > 4 ? pd : 4);
  P = P < cap ? P : cap;
  P = P / 4 * 4;
  return P > 4 ? P : 4;
}

// Shared-memory regions (floats) and per-CTA scratch (floats) a set of items
// needs; item_needs raises them to cover one item.
struct Limits {
  int szA = 4, szW = 4, szU = 4, pmax = 4;
  int64_t scratch = 4;
};

inline void item_needs(const SubDev& sd, const Item& it, Limits& l) {
  int u = 0;
  int64_t sc = 0;
  for (int n = 0; n < sd.n_nets; ++n) {
    const int K = it.K[n];
    if (!K) continue;
    const NetDev& nd = sd.net[n];
    int rows = 0;
    for (int k = 1; k < nd.L; ++k) {
      rows += nd.wp[k];
      const int a = nd.wp[k] * adj_stride(K, it.P);
      l.szA = l.szA > a ? l.szA : a;
    }
    for (int k = 2; k < nd.L; ++k) {
      const int w = layer_img_floats(nd, k);
      l.szW = l.szW > w ? l.szW : w;
    }
    u += nd.w[nd.L] * K * it.P;
    sc += (int64_t)(rows + nd.w[nd.L]) * K * it.P;
  }
  l.szU = l.szU > u ? l.szU : u;
  l.scratch = l.scratch > sc ? l.scratch : sc;
  l.pmax = l.pmax > it.P ? l.pmax : it.P;
}

inline int round_up4(int x) { return (x + 3) / 4 * 4; }

// Kernel entry points (defined in jet_step.cu / reduce_adam.cu / route.cu).
void launch_jet_step(const StepArgs& a, int grid, size_t smem, cudaStream_t s);
size_t jet_step_smem_bytes(const StepArgs& a);
cudaError_t jet_step_configure(size_t smem);
int jet_step_blocks_per_sm(int pt, int nt, bool gen, size_t smem);

struct ReduceArgs {
  const int2* blocks;        // (subdomain, first param) of each CTA: 256 / split params
  int n_blocks;
  int split;                 // threads per parameter (1, 2, 4 or 8), each summing a contiguous run of items
  const SubDev* subs;
  const int* q_items;        // CSR: items contributing to each subdomain
  const int* q_item_begin;   // [n_sub + 1]
  const Item* items;
  const float* partials;
  const double* loss_part;
  float* params;
  float* m;
  float* v;
  float* grads;              // NULL: not written
  float* loss_ring;          // [ring_cap][n_sub][5] loss rows, one slot per step
  int ring_cap;
  const int* loss_slot;      // device slot counter (already incremented)
  const int64_t* q_part_off; // CSR (like q_items): gradient slice offset of each item
  const int* step_t;         // device Adam step count (already incremented)
  const float* bc;           // [2] bias corrections 1 - beta1^t, 1 - beta2^t of this step
  int do_adam;
  float beta1, beta2, eps;
  int n_sub;
  int* err;                  // device status word: XPINN_ERR_NONFINITE is set here when a
                             // loss term is NaN or infinite (an earlier code is kept)
  float* jq;                 // [n_sub] J(Theta_q), the weighted loss of each subdomain, or NULL
};

void launch_reduce_adam(const ReduceArgs& a, cudaStream_t s);
// out[0] = sum_q jq[q] in a fixed order (one warp, double accumulation)
void launch_objective_sum(const float* jq, int n_sub, float* out, cudaStream_t s);

// One weight image to build from the packed parameters.
struct PackBlock {
  int64_t src;           // W^k in params (b^k follows)
  int64_t dst;           // image in wimg
  int in_w, out_w, in_p, out_p;
  int fwd;               // 1: forward image (transposed, with bias); 0: reverse image
};
void launch_pack_weights(const float* params, const PackBlock* blocks, int n_blocks, float* wimg,
                         cudaStream_t s);
// Start of a step (step_start_kernel): counters, step count, bias
// corrections, loss slot, weight images.
struct StepStart {
  int* counters;
  int n_counters;
  int* step_t;
  int* loss_slot;
  float* bc;                 // [2] out: 1 - beta1^t, 1 - beta2^t
  int do_adam;
  float beta1, beta2;
  const float* params;
  const PackBlock* blocks;
  int n_blocks;
  float* wimg;
};
void launch_step_start(const StepStart& a, cudaStream_t s);

}  // namespace xp
