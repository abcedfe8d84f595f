/*
 * xpinn.h — C ABI of the GB300 library for domain-decomposed physics-informed
 * neural networks (cPINN / XPINN), after "Parallel Physics-Informed Neural
 * Networks via Domain Decomposition" (Shukla, Jagtap, Karniadakis, 2021).
 *
 * One handle holds one problem: every subdomain Omega_q of a decomposed domain
 * (Sec. 4.2, Sec. 5.1), its network(s) (Sec. 3), its residual, data and
 * interface point sets, its loss weights (Eqs. cPINNLoss and XPINNLoss) and
 * its Adam state (Sec. 6).  Independent copies of a decomposition (for
 * hyper-parameter sweeps) are simply more subdomains in the same handle.
 *
 * Conventions, for every function below:
 *  - The return value is an xpinn_status; XPINN_OK (0) on success.  On error a
 *    message is available from xpinn_last_error() (thread-local).  No call
 *    aborts, throws across the ABI or traps on the device.
 *  - Pointers named "host" must be host memory.  Pointers documented as
 *    "host or device" may be either; the library asks the CUDA runtime which
 *    (cudaPointerGetAttributes).  With a device pointer the call is
 *    asynchronous in `stream`; with a host pointer it returns after the data
 *    has been copied, which synchronises `stream`.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls on one handle are stream-ordered and not thread-safe.
 *  - A handle belongs to the CUDA device that was current when it was
 *    created; every call makes that device current for its duration.
 *  - Jet components are ordered (u, d0 u, d1 u, d00 u, d11 u): value, first
 *    derivatives and diagonal second derivatives with respect to the two
 *    inputs z = (z0, z1), which are (x, t) for Burgers and (x, y) otherwise.
 *    A request of derivative order 0, 1 or 2 returns the first 1, 3 or 5.
 *  - The caller owns every buffer it passes; xpinn_create copies what it needs.
 */
#ifndef XPINN_H
#define XPINN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XPINN_MAX_NETS 2      /* networks per subdomain (inverse problems use 2) */
#define XPINN_MAX_LAYERS 12   /* weight layers L per network */
#define XPINN_MAX_WIDTH 112   /* neurons per hidden layer */
#define XPINN_MAX_OUT 3       /* outputs per network */
#define XPINN_N_TERMS 5       /* loss terms reported per subdomain, see below */
#define XPINN_NOALLOC_SCRATCH_BYTES (32 << 20)  /* see xpinn_residual_grad_noalloc */

typedef enum {
  XPINN_OK = 0,
  XPINN_ERR_INVALID = -1,     /* bad argument or inconsistent description */
  XPINN_ERR_OOM = -2,         /* device allocation failed */
  XPINN_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  XPINN_ERR_TIMEOUT = -4,     /* a bounded device wait gave up */
  XPINN_ERR_NONFINITE = -5,   /* a loss became NaN or infinite */
  XPINN_ERR_UNSUPPORTED = -6  /* valid, but outside what this build implements */
} xpinn_status;

/* PDEs (residual F(u) = L_x(u) - f, Sec. 2):
 *  BURGERS   u_t + u u_x - nu u_xx                     (Eq. BE), z = (x, t)
 *  POISSON   -(u_xx + u_yy) - f
 *  NS        steady incompressible Navier-Stokes, outputs (u, v, p),
 *            u.grad u + grad p - lap u / Re and div u  (Eq. NSEq)
 *  DIFFUSION div(K grad u) - f with two networks per subdomain, u and K
 *            (the inverse problem of Eq. heq)                                 */
enum { XPINN_PDE_BURGERS = 0, XPINN_PDE_POISSON = 1, XPINN_PDE_NS = 2, XPINN_PDE_DIFFUSION = 3 };
/* Interface conditions: cPINN (Eq. cPINNLoss: average solution + normal flux
 * continuity) or XPINN (Eq. XPINNLoss: average solution + residual continuity). */
enum { XPINN_CPINN = 0, XPINN_XPINN = 1 };
/* Output layer activation: identity (Sec. 3) or softplus (a positive field). */
enum { XPINN_ACT_IDENTITY = 0, XPINN_ACT_SOFTPLUS = 1 };
/* Routing of evaluation points (xpinn_eval): boxes, or Voronoi cells of sites
 * clipped to a polygon (irregular decompositions, Sec. 7.6). */
enum { XPINN_REGION_BOX = 0, XPINN_REGION_VORONOI = 1 };
/* Burgers flux for cPINN: conservative f = u^2/2 - nu u_x, or u u_x - nu u_x. */
enum { XPINN_FLUX_CONSERVATIVE = 0, XPINN_FLUX_LITERAL = 1 };

/* Loss terms, per subdomain, in this order (each is the MSE before weighting):
 *  0 MSE_u of the data set of network 0      1 MSE_u of the data set of network 1
 *  2 MSE_F (residual)                         3 MSE_uavg (sum over neighbours)
 *  4 MSE_flux (cPINN) or MSE_R (XPINN), summed over neighbours.
 * J(Theta_q) = w_data[0] T0 + w_data[1] T1 + w_res T2 + w_avg T3 + w_iface T4. */

/* Hidden activation Phi of a network (Sec. 3; Table Table_USmap uses tanh
 * and sin networks side by side). */
enum { XPINN_PHI_TANH = 0, XPINN_PHI_SIN = 1, XPINN_PHI_COS = 2 };

/* A fully connected network (Sec. 3): N^1 = W^1 z + b^1,
 * N^k = W^k Phi(n a^{k-1} N^{k-1}) + b^k for 2 <= k <= L; widths[0] = 2
 * (inputs), widths[L] = outputs.
 *
 * Parameter layout of one network inside its subdomain's block: for
 * k = 1..L, W^k row-major [widths[k]][widths[k-1]] then b^k [widths[k]];
 * then, if adaptive, the L-1 layer-wise slopes a^1..a^{L-1}.  Without
 * `adaptive` the slope n a^k is fixed at 1 and the network has no slope
 * parameters.  With it the slopes are trained like every other parameter
 * (same Adam, same learning rate); the paper's initialisation is
 * a^k = 1/n.  A zero-initialised descriptor (apart from n_layers, widths)
 * is a tanh network with fixed slopes. */
typedef struct {
  int32_t n_layers;                        /* L >= 2 */
  int32_t widths[XPINN_MAX_LAYERS + 1];
  int32_t out_act;                         /* XPINN_ACT_* */
  int32_t act;                             /* XPINN_PHI_* */
  int32_t adaptive;                        /* 0 or 1 */
  float slope_scale;                       /* n > 0 (read only when adaptive; 10 in Sec. 3) */
} xpinn_net_desc;

/* One subdomain Omega_q.  All arrays are host memory, float32, row-major. */
typedef struct {
  int32_t n_nets;                          /* 1, or 2 for XPINN_PDE_DIFFUSION (u, K) */
  xpinn_net_desc nets[XPINN_MAX_NETS];
  int64_t n_res;                           /* residual points x_F */
  const float* res_xy;                     /* [n_res][2] */
  const float* res_f;                      /* [n_res] forcing f, or NULL for f = 0 */
  int64_t n_data[XPINN_MAX_NETS];          /* data / boundary points of each net */
  const float* data_xy[XPINN_MAX_NETS];    /* [n_data][2] */
  const float* data_val[XPINN_MAX_NETS];   /* [n_data][D_out of that net] targets */
  float w_data[XPINN_MAX_NETS];            /* W_u */
  float w_res;                             /* W_F */
  float w_avg;                             /* W_I */
  float w_iface;                           /* W_I,flux (cPINN) or W_I,F (XPINN) */
  float lr;                                /* Adam learning rate of this subdomain */
  float rect[4];                           /* closed box x0, x1, y0, y1 used by xpinn_eval */
  int32_t region_kind;                     /* how xpinn_eval routes points to it:
                                              XPINN_REGION_BOX: the closed box `rect`;
                                              XPINN_REGION_VORONOI: the points of the
                                              problem's polygon nearest to `site` */
  float site[2];
} xpinn_subdomain_desc;

/* A common interface between subdomains q and q_plus with its own points
 * (one point set, evaluated by both networks).  Each side's loss treats the
 * other side's values as constants, as Algorithm 1 receives them. */
typedef struct {
  int32_t q, q_plus;
  int32_t method;                          /* XPINN_CPINN or XPINN_XPINN */
  float normal[2];                         /* n for the cPINN flux f . n */
  int64_t n_pts;
  const float* xy;                         /* [n_pts][2] */
  int32_t remote;                          /* 0: both sides are in this problem; 1: only
                                              side q is (distributed training: q_plus is
                                              another rank's, and that rank describes the
                                              same interface with the same points; its
                                              values come through xpinn_set_remote_values) */
} xpinn_interface_desc;

typedef struct {
  int32_t pde;                             /* XPINN_PDE_* */
  float nu;                                /* Burgers viscosity */
  float re;                                /* Navier-Stokes Reynolds number */
  int32_t flux_mode;                       /* XPINN_FLUX_* (Burgers cPINN only) */
  int32_t n_sub;
  const xpinn_subdomain_desc* subs;        /* [n_sub] */
  int32_t n_iface;
  const xpinn_interface_desc* ifaces;      /* [n_iface] */
  float beta1, beta2, eps;                 /* Adam constants shared by all subdomains */
  int32_t subs_per_model;                  /* subdomains per independent copy; 0 = n_sub */
  const float* init_params;                /* packed parameters (see xpinn_get_params) */
  int32_t n_poly;                          /* polygon (domain) for Voronoi regions, or 0 */
  const float* poly;                       /* [n_poly][2] vertices, host */
} xpinn_problem_desc;

typedef struct xpinn_ctx* xpinn_handle;

/* Create a handle: validates `desc`, copies every array to the device and
 * plans the grouped step.  Device memory is allocated here and freed by
 * xpinn_destroy.  Errors: INVALID (inconsistent description), UNSUPPORTED
 * (a width, depth or output count beyond the limits above), OOM, CUDA. */
int xpinn_create(const xpinn_problem_desc* desc, xpinn_handle* out);

/* Free all device and host memory of the handle.  NULL is accepted. */
int xpinn_destroy(xpinn_handle h);

/* Message of the last error on this thread ("" if none). */
const char* xpinn_last_error(void);

/* Number of floats in the packed parameter vector: subdomain by subdomain,
 * network by network, layer k = 1..L: W^k row-major [N_k][N_{k-1}], then b^k. */
int64_t xpinn_num_params(xpinn_handle h);

/* Copy the packed parameters out of / into the handle (host or device
 * pointer, n = xpinn_num_params).  set_params leaves Adam's moments and step
 * count unchanged. */
int xpinn_get_params(xpinn_handle h, float* dst, int64_t n, void* stream);
int xpinn_set_params(xpinn_handle h, const float* src, int64_t n, void* stream);

/* Loss terms and gradients at the current parameters, with no update:
 * losses [n_sub][XPINN_N_TERMS] (or NULL), grads packed like the parameters
 * (or NULL), dJ(Theta_q)/dTheta_q for every q with the neighbours' interface
 * values held constant (Algorithm 1).  Host or device pointers.  The call
 * synchronises `stream` and returns XPINN_ERR_NONFINITE (outputs written) if
 * a loss term is NaN or infinite, XPINN_ERR_TIMEOUT if a device wait gave up,
 * in this call or an earlier asynchronous one. */
int xpinn_grad(xpinn_handle h, float* losses, float* grads, void* stream);

/* The objective of the method and its gradient at the current parameters,
 * with no update: J (1 float, or NULL) = sum over q of J(Theta_q), where
 * J(Theta_q) = sum_t w_t MSE_t is the weighted loss of subdomain q (Eq.
 * cPINNLoss or Eq. XPINNLoss with the subdomain's weights, the terms as
 * listed above); J_sub [n_sub] (or NULL) the J(Theta_q); losses and grads
 * (or NULL) as xpinn_grad.  The gradient is that of each J(Theta_q) with
 * respect to its own Theta_q, the neighbours' interface values held
 * constant (Algorithm 1): the training direction of the method.  Sums are
 * taken in a fixed order (bitwise reproducible).  Host or device pointers;
 * synchronises `stream`; errors as xpinn_grad. */
int xpinn_objective(xpinn_handle h, float* J, float* J_sub, float* losses, float* grads, void* stream);

/* n_steps training steps of Algorithm 1, all subdomains in one grouped
 * launch per phase: interface values, jets + residual + interface terms +
 * reverse pass, then reduction and Adam (Sec. 6).  losses, if not NULL,
 * receives [n_steps][n_sub][XPINN_N_TERMS], each row measured before that
 * step's update.
 * Errors raised on the device (a bounded wait that gave up, a loss that
 * became NaN or infinite) are kept in the handle's device status word until
 * a synchronising call reads it.  With host `losses` this call synchronises
 * and returns XPINN_ERR_TIMEOUT or XPINN_ERR_NONFINITE itself (after
 * completing the steps).  With losses NULL or a device pointer it returns as
 * soon as the steps are queued, and the error is returned by the next
 * synchronising call on the handle: xpinn_sync, xpinn_grad, or xpinn_step
 * with host losses.  The steps after a non-finite loss still run. */
int xpinn_step(xpinn_handle h, int32_t n_steps, float* losses, void* stream);

/* ---------------------------------------------------------------------------
 * Distributed training (Algorithm 1 across ranks, one GPU each): a rank's
 * handle holds its own subdomains (xpinn_partition picks them), and every
 * interface it shares with another rank is described with remote = 1 and the
 * local subdomain as q.  A training step is then
 *   xpinn_step_begin   start of the step: this handle's side of every
 *                      interface into the exchange buffer (one launch);
 *   xpinn_remote_values / xpinn_set_remote_values
 *                      the host sends its sides of the remote interfaces and
 *                      writes the other ranks' sides (the paper's Isend /
 *                      Irecv; NCCL send/recv or any transport);
 *   xpinn_step_end     the residual, data and interface terms, the reverse
 *                      pass, the reduction and Adam; losses as one row of
 *                      xpinn_step (host or device, or NULL).
 * The remote values are the other side's solution vector and exchanged
 * quantity at the interface points, rows of [n_pts][nv] (nv = xpinn_iface_values'
 * floats per point and side), interface by interface in the order of the
 * description.  xpinn_step on such a handle uses the remote values last set.
 * ------------------------------------------------------------------------- */
int xpinn_step_begin(xpinn_handle h, void* stream);
int xpinn_step_end(xpinn_handle h, float* losses, void* stream);
/* out NULL: *n_floats receives the size.  Host or device pointer (host:
 * returns after the copy). */
int xpinn_remote_values(xpinn_handle h, float* out, int64_t* n_floats, void* stream);
int xpinn_set_remote_values(xpinn_handle h, const float* in, int64_t n_floats, void* stream);

/* Partition of n_sub subdomains over n_parts ranks (1 <= n_parts <= n_sub):
 * part[q] in [0, n_parts).  weight[q] is a subdomain's work (its points),
 * edges (eq[e], eqp[e]) its interfaces with edge_w[e] their points (the
 * exchanged rows).  Weighted graph growing from the lowest-numbered free
 * subdomain, then boundary refinement that moves subdomains to cut fewer
 * interface points while every part stays within 10% of an even share.
 * Deterministic; host only. */
int xpinn_partition(int32_t n_sub, const double* weight, int32_t n_edge, const int32_t* eq, const int32_t* eqp,
                    const double* edge_w, int32_t n_parts, int32_t* part);

/* Waits for everything queued on `stream`, then reads and clears the
 * handle's device status word: XPINN_OK, XPINN_ERR_TIMEOUT (a bounded device
 * wait of an earlier call gave up) or XPINN_ERR_NONFINITE (a loss of an
 * earlier step or grad was NaN or infinite).  Call it after asynchronous
 * steps (xpinn_step with losses NULL or on the device). */
int xpinn_sync(xpinn_handle h, void* stream);

/* Jets of network `net` of subdomain q at n points xy [n][2]:
 * out [n][D_out][1 + 2*(order>0) + 2*(order>1)], order 0..2.  Host or device
 * pointers (both on the same side). */
int xpinn_net_jets(xpinn_handle h, int32_t q, int32_t net, const float* xy, int64_t n,
                   int32_t order, float* out, void* stream);

/* The stitched solution of Eq. FSol for copy `model`: u(z) = sum_q u_q(z)
 * 1_{Omega_q}(z), with 1/S on an interface shared by S subdomains; points are
 * routed to subdomains on the device by their closed boxes (`rect`), or for
 * Voronoi regions by the even-odd polygon test and the nearest site (S sites
 * at exactly the same float32 distance (dx*dx + dy*dy, no fused multiply-add)
 * share the point).  out
 * [n][D_out_total][1 + 2*(order>0) + 2*(order>1)], where D_out_total counts
 * the outputs of all networks of a subdomain.  Points outside every box give
 * NaN.  Host or device pointers (both on the same side). */
int xpinn_eval(xpinn_handle h, int32_t model, const float* xy, int64_t n, int32_t order,
               float* out, void* stream);

/* xpinn_eval with caller-provided device workspace, for callers that keep a
 * memory pool (the request server): the routing, its prefix sums, the work
 * items and the stitching all run on the device from slices of `workspace`
 * (256-byte aligned, ws_bytes >= xpinn_eval_workspace_size), so the call
 * allocates nothing and, with device xy and out, does not synchronise (a
 * device error is then reported by the next synchronising call on the
 * handle, see xpinn_sync).  With host xy and out the points are staged in
 * the workspace and the call returns after the result has been copied.
 * xpinn_eval itself runs this path on a workspace the handle keeps.  The
 * size covers the worst case of a point shared by four subdomains. */
int xpinn_eval_workspace_size(xpinn_handle h, int32_t model, int64_t n, int32_t order, size_t* bytes);
int xpinn_eval_ws(xpinn_handle h, int32_t model, const float* xy, int64_t n, int32_t order, float* out,
                  void* workspace, size_t ws_bytes, void* stream);

/* Replace the residual points (and forcing) of every subdomain, keeping the
 * per-subdomain counts: xy [n_res_total][2], f [n_res_total] or NULL (f = 0),
 * subdomain by subdomain in order.  Host or device pointers.  Used to
 * resample residual points between steps. */
int xpinn_set_residual_points(xpinn_handle h, const float* xy, const float* f, int64_t n,
                              void* stream);

/* Training on a private fork (the request server's training-step requests):
 * n_steps steps of Algorithm 1 for the n_sel subdomains sel[] only, each with
 * the request's own residual points (n_pts[i] points for sel[i], given
 * subdomain by subdomain in xy [sum n_pts][2] with forcing f [sum n_pts], or
 * f NULL for f = 0) in place of its residual set; its data points and its
 * interfaces are the handle's.  The selected subdomains start from the
 * handle's current parameters, Adam moments and step count, on copies in
 * `workspace`; subdomains outside the selection that share an interface
 * with it provide their interface values from the handle's current
 * parameters (held constant, Algorithm 1) and are not trained.  The handle's
 * parameters and Adam state are not changed: the fork is independent of the
 * handle's own training and of other requests.
 *   losses [n_steps][n_sel][XPINN_N_TERMS] (or NULL): each step's loss terms
 *     of the selected subdomains, measured before that step's update;
 *   params (or NULL): the fork's parameters after the steps, the selected
 *     subdomains' blocks packed in the order of sel[].
 * workspace: device memory of at least xpinn_fork_workspace_size bytes,
 * 256-byte aligned; the call allocates nothing.  xy and f may be host or
 * device pointers, losses and params too; with device outputs the call does
 * not wait for the GPU (device errors: see xpinn_sync).  Errors: INVALID (a
 * subdomain out of range or repeated, a negative count, a small workspace). */
typedef struct {
  int32_t n_sel;
  const int32_t* sel;     /* [n_sel] distinct subdomain ids (host) */
  const int64_t* n_pts;   /* [n_sel] residual points of each (host) */
  const float* xy;        /* [sum n_pts][2] */
  const float* f;         /* [sum n_pts] or NULL */
  int32_t n_steps;
} xpinn_fork_desc;

int xpinn_fork_workspace_size(xpinn_handle h, const xpinn_fork_desc* d, size_t* bytes);
int xpinn_fork_step(xpinn_handle h, const xpinn_fork_desc* d, void* workspace, size_t ws_bytes, float* losses,
                    float* params, void* stream);

/* Checkpoint: the parameters, Adam moments m and v and the step count as one
 * versioned blob in host memory.  get_state with blob == NULL stores the
 * required size in *n.  set_state rejects a blob of another problem shape. */
int xpinn_get_state(xpinn_handle h, void* blob, size_t* n);
int xpinn_set_state(xpinn_handle h, const void* blob, size_t n);

/* Execution options (see xpinn_options). */
typedef struct {
  int32_t schedule;        /* 0 grouped (one launch per phase for all subdomains),
                              1 per-subdomain loop (the same kernels launched once
                              per subdomain per phase: the baseline) */
  int32_t use_graph;       /* 1: replay steps from captured CUDA graphs: one
                              graph of 16 steps for every run of 16 steps of a
                              call (without profile_phases), one of a single
                              step for the rest */
  int32_t items_per_cta;   /* work items per CTA the scheduler aims for (>= 1) */
  int32_t points_per_thread; /* points in a thread's register tile: 2 (default,
                              one CTA per SM) or 1 (two CTAs per SM) */
  int32_t profile_phases;  /* 1: record CUDA events between the phases of every
                              step (also inside the graph), see xpinn_phase_times */
  int32_t max_points_per_tile; /* cap on the points a CTA processes at once
                                  (0: as many as the register tiles allow) */
  int32_t threads_per_cta;  /* 256 (default); 128: smaller CTAs, more per SM;
                               512 (with points_per_thread = 1): more warps */
  int32_t inject_fault;     /* testing only: 1 makes the in-kernel wait for the
                               interface exchange wait for one item more than
                               exists, so it gives up after about 1 s and the
                               call returns XPINN_ERR_TIMEOUT; 0 (default) off */
  int32_t eval_tensor_cores; /* 1 (default): routed evaluations (xpinn_eval,
                               xpinn_eval_ws, the server's queries) of a model
                               whose subdomains each have one network with
                               input (x, y), identity output, at least two
                               hidden layers, all of one width 32, 64 or 80,
                               run the hidden-to-hidden contractions on the
                               tensor cores (tcgen05, three TF32 products over
                               a hi/lo split of both operands, FP32
                               accumulation); other models keep the FP32 jet
                               kernel.  0: the jet kernel for every model */
  int32_t train_tensor_cores; /* 0: the FP32 jet kernel trains every
                               subdomain.  N in [1, 64] (default 33): the
                               residual points of every subdomain with one
                               network of input (x, y), tanh, sin or cos
                               hidden layers (fixed or trained slopes),
                               identity output of at most 3 components, 3 to
                               8 weight layers and every hidden width within
                               [N, 64], under a PDE trained with Laplacian
                               jets (Poisson, Navier-Stokes), are trained by
                               the tensor-core kernel when those subdomains
                               hold at least half of the residual points (it
                               runs before the jet kernel, so it only pays off
                               when it takes over most of the step): the
                               forward, reverse and weight-gradient
                               contractions of the hidden-to-hidden layers as
                               tcgen05 MMAs (three TF32 products over hi/lo
                               splits of both operands, FP32 accumulation),
                               layers narrower than 64 zero-padded (the
                               default 33 admits the widths that fill more
                               than half of the 64-wide tile).  Their
                               data and interface points stay on the jet
                               kernel; forks (xpinn_fork_step) use the jet
                               kernel throughout */
} xpinn_options;

int xpinn_get_options(xpinn_handle h, xpinn_options* opt);
int xpinn_set_options(xpinn_handle h, const xpinn_options* opt);

/* Autotuner: times gradient passes (no parameter update, grouped schedule)
 * of candidate launch options and applies the fastest, returned in *best
 * (its median ms per pass in *best_ms).  Candidates: the grid of CTA shapes
 * (threads_per_cta x points_per_thread: 256x2, 256x1, 512x1, 128x2, 128x1)
 * x items_per_cta {4, 8, 16, 2, 32} without a tile cap, the default (256x2,
 * 4) first, then every change of one of the two, then the remaining pairs;
 * then max_points_per_tile {64, 128, 32} on the best pair.  Each candidate
 * takes the median of `steps` passes (one pass when a pass lasts more than
 * 200 ms); candidates that do not fit shared memory are skipped, and the
 * search stops after about 30 s, keeping the best so far.  Parameters,
 * Adam state and step count are unchanged.  Synchronises. */
int xpinn_autotune(xpinn_handle h, int32_t steps, xpinn_options* best, float* best_ms);

/* Per-shape tuning: subdomains whose networks have the same widths,
 * activations, slopes and output activation form a shape class; within one
 * grouped launch every item of a class is cut into sub-tiles of at most the
 * class's cap of points.  xpinn_autotune_shapes picks the caps by
 * coordinate descent over the classes (the classes with the largest modelled
 * share of the step first; candidates 128, 96, 64, 48, 32, 160 and none),
 * timing `steps` gradient passes of the grouped step for each and keeping a
 * choice only when it is clearly faster; about 20 s at most.  Then, for every
 * class whose networks the tensor-core kernel takes (see train_tensor_cores),
 * it times that kernel on and off for the class's residual items, keeping
 * the faster (about 30 s in all).  Parameters, Adam state and step count are
 * unchanged; synchronises.  *best_ms: the median ms per pass of the final
 * choice.  The caps and the tensor-core choices, one per subdomain, can be
 * read and set (for a cache of tuned choices); setting re-plans the step. */
int xpinn_autotune_shapes(xpinn_handle h, int32_t steps, float* best_ms);
int xpinn_get_tile_caps(xpinn_handle h, int32_t* caps);         /* caps [n_sub], host */
int xpinn_set_tile_caps(xpinn_handle h, const int32_t* caps);   /* [n_sub] (0 or >= 8), or NULL: none */
/* Tensor-core choice per subdomain, sel[n_sub] (host): 1 its residual items
 * run on the tensor-core kernel whenever its network qualifies (overriding
 * the rule that the qualifying subdomains must hold half of the residual
 * points), 0 never, -1 (the default; also sel = NULL) by that rule. */
int xpinn_get_tc_select(xpinn_handle h, int32_t* sel);
int xpinn_set_tc_select(xpinn_handle h, const int32_t* sel);

/* Device time in milliseconds of the four phases of the most recent step or
 * grad call, measured by CUDA events recorded on the call's stream:
 * ms[0] step start, ms[1] interface exchange launches (per-subdomain loop
 * schedule; 0 in the grouped schedule, whose single jet launch does the
 * exchange too), ms[2] jet kernel launch(es), ms[3] reduction and Adam.
 * Requires profile_phases = 1; waits for that step to finish. */
int xpinn_phase_times(xpinn_handle h, float* ms);

/* Work items of the current step plan (host tables, no device work):
 * *n_items all of them (exchange, residual, data and interface items),
 * *n_tc the residual items the tensor-core kernel runs (option
 * train_tensor_cores), *n_tc_sub the subdomains those belong to.  Any
 * output pointer may be NULL. */
int xpinn_plan_counts(xpinn_handle h, int32_t* n_items, int32_t* n_tc, int32_t* n_tc_sub);

/* on[n_sub] (host): 1 where the subdomain's residual items run on the
 * tensor-core kernel in the current plan (option train_tensor_cores, the
 * half-the-points rule, xpinn_set_tc_select), else 0.  No device work. */
int xpinn_tc_subdomains(xpinn_handle h, int32_t* on);

/* Device time in milliseconds of the evaluation kernel (the jet kernel, or
 * the tensor-core kernel under eval_tensor_cores) of the most recent routed
 * evaluation (xpinn_eval, xpinn_eval_ws) made with profile_phases = 1, from
 * CUDA events recorded around its launch on the call's stream (none while
 * the stream is being captured).  Waits for that kernel.  Errors: INVALID if
 * no evaluation has been timed. */
int xpinn_eval_kernel_time(xpinn_handle h, float* ms);

/* Device time in milliseconds of the tensor-core training kernel (option
 * train_tensor_cores) in the most recent grouped step or grad call made with
 * profile_phases = 1, from CUDA events recorded around its launch (inside
 * the step graph too).  Part of ms[2] of xpinn_phase_times.  Waits for that
 * kernel.  Errors: INVALID if no such step has been timed. */
int xpinn_tc_kernel_time(xpinn_handle h, float* ms);

/* Interface exchange buffer after the last grad/step: for every interface
 * (in order), every point, side 0 (q) then side 1 (q_plus): the solution
 * vector u (all outputs of all networks) followed by the exchanged quantity
 * (normal fluxes f . n for cPINN, residuals F for XPINN).  n_floats receives
 * the size when out is NULL.  Host or device pointer. */
int xpinn_iface_values(xpinn_handle h, float* out, int64_t* n_floats, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of evaluation and training requests over
 * several models (handles on one device).  At creation the server allocates
 * its two memory pools once: hbm_budget bytes of device memory and a staging
 * pool of page-locked host memory (hbm_budget, at most 1 GiB).  A scheduler
 * thread forms ticks: it admits submitted requests in arrival order while
 * each one's footprint (its device workspace and device copies of its inputs
 * and outputs; its staged host inputs and outputs) fits the free part of
 * both pools, so no request allocates and admission is by the memory the
 * request really holds.  In a tick:
 *   - the evaluation queries of one model, copy and derivative order are
 *     stitched (Eq. FSol) in one routed evaluation planned on the device
 *     (xpinn_eval_ws): one grouped launch over all their points;
 *   - XPINN_REQ_FORK requests train a subdomain subset on their own residual
 *     points on a private fork of the model (xpinn_fork_step): the model is
 *     not changed;
 *   - XPINN_REQ_STEP requests run xpinn_step on the model in place (on its
 *     resident buffers; only their loss rows count against the pools), in
 *     arrival order with that model's other requests.
 * The work of a model is queued on one CUDA stream, different models on
 * different streams, and a tick is queued while earlier ticks still run, so
 * work of different requests overlaps on the GPU.  A point's value does not
 * depend on the other points of a batch, and a fork depends only on its
 * request and the model, so a result is the same alone and in a mix
 * (bitwise).  All request buffers are host memory, owned by the caller until
 * the request completes.
 * ------------------------------------------------------------------------- */
enum { XPINN_REQ_EVAL = 0, XPINN_REQ_STEP = 1, XPINN_REQ_FORK = 2 };
enum { XPINN_PENDING = 1 };   /* xpinn_server_poll: not finished yet */

typedef struct {
  int32_t kind;       /* XPINN_REQ_EVAL, XPINN_REQ_STEP or XPINN_REQ_FORK */
  int32_t model;      /* index into the server's models */
  int32_t copy;       /* EVAL: copy (model) inside the handle, as xpinn_eval */
  int32_t order;      /* EVAL: derivative order 0..2 */
  int64_t n;          /* EVAL: points */
  const float* xy;    /* EVAL: [n][2]; FORK: [sum n_pts][2] residual points */
  float* out;         /* EVAL: [n][D_out_total][K], as xpinn_eval */
  int32_t n_steps;    /* STEP, FORK: training steps */
  float* losses;      /* STEP: [n_steps][n_sub][5]; FORK: [n_steps][n_sel][5]; or NULL */
  int32_t n_sel;      /* FORK: subdomains to train (see xpinn_fork_step) */
  const int32_t* sel; /* FORK: [n_sel] */
  const int64_t* n_pts; /* FORK: [n_sel] residual points of each */
  const float* f;     /* FORK: [sum n_pts] forcing, or NULL */
  float* params;      /* FORK: the fork's parameters of sel after the steps, or NULL */
} xpinn_request;

typedef struct {
  int32_t status;     /* xpinn_status of the request */
  double queue_ms;    /* submit -> admitted into a tick */
  double latency_ms;  /* submit -> completed */
  int32_t batch;      /* requests served in the same launch (stitched evaluations) */
  char error[160];    /* message when status != XPINN_OK */
  int32_t tick_requests;  /* requests admitted in the same tick */
} xpinn_result;

typedef struct xpinn_server xpinn_server;

/* models: handles that outlive the server (not owned), all on one device.
 * hbm_budget: bytes of the device pool (>= 4096).  Errors: INVALID,
 * UNSUPPORTED (models on different devices), OOM (the pools). */
int xpinn_server_create(const xpinn_handle* models, int32_t n_models, size_t hbm_budget,
                        xpinn_server** out);
/* Non-blocking.  *ticket identifies the request.  XPINN_ERR_OOM if the
 * request alone exceeds a pool (it could never be admitted), INVALID for a
 * malformed request. */
int xpinn_server_submit(xpinn_server* s, const xpinn_request* req, uint64_t* ticket);
/* XPINN_OK with *res filled once the request is finished (the ticket is then
 * released), XPINN_PENDING before, XPINN_ERR_INVALID for an unknown ticket. */
int xpinn_server_poll(xpinn_server* s, uint64_t ticket, xpinn_result* res);
/* Waits for every submitted request, stops the scheduler, frees the pools. */
int xpinn_server_destroy(xpinn_server* s);

/* Residual loss and its gradient for ONE network, allocating no device
 * memory.  (The paper has no counterpart: this is a deployment convenience.)
 *
 * For callers that cannot call cudaMalloc themselves or through this library
 * -- code that runs inside a host framework whose allocator owns the device,
 * a runtime with a fixed memory budget, or a region that must not allocate
 * while it is timed or replayed.  The caller passes device buffers it already
 * owns; the library's working memory comes from one built-in device array of
 * XPINN_NOALLOC_SCRATCH_BYTES (32 MiB), which every GPU that loads the
 * library holds until the library is unloaded.  When the working set of a
 * request does not fit, the call uses fewer CTAs; if it does not fit even
 * with one, it is rejected with XPINN_ERR_UNSUPPORTED and a message naming
 * the size.
 *
 * Computes, for pde BURGERS, POISSON or NS (single-network PDEs):
 *   loss[0]  = MSE_F = (1/n) sum_i |F(u)(xy_i)|^2              (device, 1 float)
 *   grads    = d (w_res * MSE_F) / d theta, packed like one net (device)
 * with the network `net` (host struct, any activation, slopes fixed or
 * adaptive) and parameters `params` (device, in the network's layout above:
 * layer by layer W^k row-major then b^k, then the slopes if adaptive),
 * points xy [n][2] and forcing f [n]
 * (device; pass zeros when f = 0: it is required).  It is the residual part
 * of xpinn_grad for one subdomain.  Asynchronous in `stream`.
 *
 * The first call on each device looks up the array's device address (and
 * raises the jet kernel's shared-memory limit); make that first call before
 * any stream capture.  Every call reuses the same array and leaves its
 * contents behind; each call clears what must start at zero itself.  Calls
 * that overlap on the GPU (other streams, other threads) race on the array:
 * order them on one stream.  The sub-tile of points is chosen as for a
 * handle (lowered in steps of 4 while the shared memory does not fit), and
 * the work is spread over at most one CTA per SM.  Errors: INVALID,
 * UNSUPPORTED (a network whose tiles do not fit shared memory even at 8
 * points, or a working set beyond the array), CUDA; the message is
 * available from xpinn_last_error().  An error on the device (a bounded wait
 * that gave up) cannot be returned by this asynchronous call: the loss and
 * every gradient element are then written as NaN. */
int xpinn_residual_grad_noalloc(int32_t pde, float nu, float re, const xpinn_net_desc* net,
                                const float* params, const float* xy, const float* f, int64_t n,
                                float w_res, float* loss, float* grads, void* stream);

/* Testing only: the next xpinn_residual_grad_noalloc call of this thread
 * starts with its device error word set to `code` (as if a wait had given up),
 * so that the NaN outputs of a failed call can be checked without making a
 * device wait fail.  0 (the default) leaves the word cleared. */
int xpinn_noalloc_debug_preset_error(int32_t code);

#ifdef __cplusplus
}
#endif

#endif /* XPINN_H */
