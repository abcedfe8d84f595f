"""Python binding of the C ABI in include/xpinn.h (ctypes, marshalling only).

Every computation runs in the CUDA library; this module only builds the
problem description, passes pointers and reshapes results.  Arrays may be
numpy arrays (host) or CUDA torch tensors (device); with device tensors the
calls are asynchronous on torch's current stream.

The library must have been built (paper_2104_10013_gb300.build.build()); if
it is missing, load() raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import problems as P

MAX_NETS, MAX_LAYERS, N_TERMS = 2, 12, 5

_STATUS = {0: "OK", -1: "INVALID", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "NONFINITE",
           -6: "UNSUPPORTED"}


class XpinnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"xpinn {_STATUS.get(code, code)}: {msg}")
        self.code = code


class NetDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.c_int32 * (MAX_LAYERS + 1)), ("out_act", C.c_int32),
                ("act", C.c_int32), ("adaptive", C.c_int32), ("slope_scale", C.c_float)]


class SubDesc(C.Structure):
    _fields_ = [("n_nets", C.c_int32), ("nets", NetDesc * MAX_NETS),
                ("n_res", C.c_int64), ("res_xy", C.c_void_p), ("res_f", C.c_void_p),
                ("n_data", C.c_int64 * MAX_NETS), ("data_xy", C.c_void_p * MAX_NETS),
                ("data_val", C.c_void_p * MAX_NETS), ("w_data", C.c_float * MAX_NETS),
                ("w_res", C.c_float), ("w_avg", C.c_float), ("w_iface", C.c_float),
                ("lr", C.c_float), ("rect", C.c_float * 4), ("region_kind", C.c_int32),
                ("site", C.c_float * 2)]


class IfaceDesc(C.Structure):
    _fields_ = [("q", C.c_int32), ("q_plus", C.c_int32), ("method", C.c_int32),
                ("normal", C.c_float * 2), ("n_pts", C.c_int64), ("xy", C.c_void_p), ("remote", C.c_int32)]


class ProblemDesc(C.Structure):
    _fields_ = [("pde", C.c_int32), ("nu", C.c_float), ("re", C.c_float), ("flux_mode", C.c_int32),
                ("n_sub", C.c_int32), ("subs", C.POINTER(SubDesc)),
                ("n_iface", C.c_int32), ("ifaces", C.POINTER(IfaceDesc)),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("subs_per_model", C.c_int32), ("init_params", C.c_void_p),
                ("n_poly", C.c_int32), ("poly", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("use_graph", C.c_int32), ("items_per_cta", C.c_int32),
                ("points_per_thread", C.c_int32), ("profile_phases", C.c_int32),
                ("max_points_per_tile", C.c_int32), ("threads_per_cta", C.c_int32),
                ("inject_fault", C.c_int32), ("eval_tensor_cores", C.c_int32),
                ("train_tensor_cores", C.c_int32)]


class ForkDesc(C.Structure):
    _fields_ = [("n_sel", C.c_int32), ("sel", C.c_void_p), ("n_pts", C.c_void_p), ("xy", C.c_void_p),
                ("f", C.c_void_p), ("n_steps", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("model", C.c_int32), ("copy", C.c_int32), ("order", C.c_int32),
                ("n", C.c_int64), ("xy", C.c_void_p), ("out", C.c_void_p), ("n_steps", C.c_int32),
                ("losses", C.c_void_p), ("n_sel", C.c_int32), ("sel", C.c_void_p), ("n_pts", C.c_void_p),
                ("f", C.c_void_p), ("params", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("batch", C.c_int32), ("error", C.c_char * 160), ("tick_requests", C.c_int32)]


_LIB = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libxpinn.so")


def load() -> C.CDLL:
    """Load lib/libxpinn.so (built in-tree).  Raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run paper_2104_10013_gb300.build.build())")
    L = C.CDLL(path)
    vp, i32, i64, fp = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        "xpinn_create": (C.c_int, [C.POINTER(ProblemDesc), C.POINTER(vp)]),
        "xpinn_destroy": (C.c_int, [vp]),
        "xpinn_last_error": (C.c_char_p, []),
        "xpinn_num_params": (i64, [vp]),
        "xpinn_get_params": (C.c_int, [vp, fp, i64, vp]),
        "xpinn_set_params": (C.c_int, [vp, fp, i64, vp]),
        "xpinn_grad": (C.c_int, [vp, fp, fp, vp]),
        "xpinn_step": (C.c_int, [vp, i32, fp, vp]),
        "xpinn_net_jets": (C.c_int, [vp, i32, i32, fp, i64, i32, fp, vp]),
        "xpinn_eval": (C.c_int, [vp, i32, fp, i64, i32, fp, vp]),
        "xpinn_set_residual_points": (C.c_int, [vp, fp, fp, i64, vp]),
        "xpinn_get_state": (C.c_int, [vp, vp, C.POINTER(C.c_size_t)]),
        "xpinn_set_state": (C.c_int, [vp, vp, C.c_size_t]),
        "xpinn_get_options": (C.c_int, [vp, C.POINTER(Options)]),
        "xpinn_set_options": (C.c_int, [vp, C.POINTER(Options)]),
        "xpinn_iface_values": (C.c_int, [vp, fp, C.POINTER(i64), vp]),
        "xpinn_phase_times": (C.c_int, [vp, fp]),
        "xpinn_plan_counts": (C.c_int, [vp, vp, vp, vp]),
        "xpinn_tc_subdomains": (C.c_int, [vp, vp]),
        "xpinn_eval_kernel_time": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "xpinn_tc_kernel_time": (C.c_int, [vp, C.POINTER(C.c_float)]),
        "xpinn_autotune": (C.c_int, [vp, i32, C.POINTER(Options), C.POINTER(C.c_float)]),
        "xpinn_autotune_shapes": (C.c_int, [vp, i32, C.POINTER(C.c_float)]),
        "xpinn_step_begin": (C.c_int, [vp, vp]),
        "xpinn_step_end": (C.c_int, [vp, fp, vp]),
        "xpinn_remote_values": (C.c_int, [vp, fp, C.POINTER(i64), vp]),
        "xpinn_set_remote_values": (C.c_int, [vp, fp, i64, vp]),
        "xpinn_partition": (C.c_int, [i32, vp, i32, vp, vp, vp, i32, vp]),
        "xpinn_get_tile_caps": (C.c_int, [vp, vp]),
        "xpinn_get_tc_select": (C.c_int, [vp, vp]),
        "xpinn_set_tc_select": (C.c_int, [vp, vp]),
        "xpinn_set_tile_caps": (C.c_int, [vp, vp]),
        "xpinn_server_create": (C.c_int, [C.POINTER(vp), i32, C.c_size_t, C.POINTER(vp)]),
        "xpinn_server_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "xpinn_server_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(Result)]),
        "xpinn_server_destroy": (C.c_int, [vp]),
        "xpinn_residual_grad_noalloc": (C.c_int, [i32, C.c_float, C.c_float, C.POINTER(NetDesc), fp, fp, fp,
                                                  i64, C.c_float, fp, fp, vp]),
        "xpinn_noalloc_debug_preset_error": (C.c_int, [i32]),
        "xpinn_sync": (C.c_int, [vp, vp]),
        "xpinn_objective": (C.c_int, [vp, fp, fp, fp, fp, vp]),
        "xpinn_eval_workspace_size": (C.c_int, [vp, i32, i64, i32, C.POINTER(C.c_size_t)]),
        "xpinn_fork_workspace_size": (C.c_int, [vp, C.POINTER(ForkDesc), C.POINTER(C.c_size_t)]),
        "xpinn_fork_step": (C.c_int, [vp, C.POINTER(ForkDesc), vp, C.c_size_t, fp, fp, vp]),
        "xpinn_eval_ws": (C.c_int, [vp, i32, fp, i64, i32, fp, vp, C.c_size_t, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _LIB = L
    return L


def _check(rc):
    if rc != 0:
        raise XpinnError(rc, load().xpinn_last_error().decode())


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _ptr(x):
    """(pointer, keepalive) of a numpy array or a CUDA torch tensor."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):          # torch tensor
        return x.data_ptr(), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, a


def _stream(x=None):
    if x is not None and hasattr(x, "is_cuda") and x.is_cuda:
        import torch
        return torch.cuda.current_stream(x.device).cuda_stream
    return None


class Solver:
    """One problem on the GPU: the grouped cPINN/XPINN training step, jets,
    stitched evaluation and checkpointing, through the C ABI."""

    def __init__(self, problem: P.Problem, init_params=None):
        self.lib = load()
        self.pb = problem
        keep = []

        def arr(a, dt=np.float32):
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            keep.append(a)
            return a.ctypes.data

        subs = (SubDesc * problem.n_sub)()
        for q, s in enumerate(problem.subs):
            d = subs[q]
            d.n_nets = len(s.nets)
            for n, net in enumerate(s.nets):
                d.nets[n].n_layers = len(net.widths) - 1
                for k, w in enumerate(net.widths):
                    d.nets[n].widths[k] = w
                d.nets[n].out_act = net.out_act
                d.nets[n].act = net.act
                d.nets[n].adaptive = int(net.adaptive)
                d.nets[n].slope_scale = net.slope_scale
            d.n_res = s.res_xy.shape[0]
            d.res_xy = arr(s.res_xy) if d.n_res else None
            d.res_f = arr(s.res_f) if d.n_res else None
            for n in range(len(s.nets)):
                ds = s.data[n] if n < len(s.data) else None
                if ds is not None and ds.xy.shape[0]:
                    d.n_data[n] = ds.xy.shape[0]
                    d.data_xy[n] = arr(ds.xy)
                    d.data_val[n] = arr(ds.val)
                d.w_data[n] = s.w_data[n] if n < len(s.w_data) else 0.0
            d.w_res, d.w_avg, d.w_iface, d.lr = s.w_res, s.w_avg, s.w_iface, s.lr
            for i, v in enumerate(s.rect if s.rect is not None else (0, 0, 0, 0)):
                d.rect[i] = v
            d.region_kind = s.region_kind
            if s.site is not None:
                d.site[0], d.site[1] = s.site
        ifs = (IfaceDesc * max(1, len(problem.ifaces)))()
        for e, it in enumerate(problem.ifaces):
            f = ifs[e]
            f.q, f.q_plus, f.method = it.q, it.qp, it.method
            f.normal[0], f.normal[1] = it.normal
            f.n_pts = it.xy.shape[0]
            f.xy = arr(it.xy) if f.n_pts else None
            f.remote = int(getattr(it, "remote", False))
        desc = ProblemDesc()
        desc.pde, desc.nu, desc.re, desc.flux_mode = problem.pde, problem.nu, problem.re, problem.flux_mode
        desc.n_sub, desc.subs = problem.n_sub, subs
        desc.n_iface, desc.ifaces = len(problem.ifaces), ifs
        desc.beta1, desc.beta2, desc.eps = problem.beta1, problem.beta2, problem.eps
        desc.subs_per_model = problem.subs_per_model
        if problem.polygon is not None:
            desc.n_poly = int(problem.polygon.shape[0])
            desc.poly = arr(problem.polygon)
        theta = problem.packed_params() if init_params is None else _f32(init_params)
        desc.init_params = arr(theta)
        h = C.c_void_p()
        _check(self.lib.xpinn_create(C.byref(desc), C.byref(h)))
        self.h = h
        self.n_params = int(self.lib.xpinn_num_params(h))
        self.n_sub = problem.n_sub

    # ---------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "h", None):
            self.lib.xpinn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- params
    def get_params(self, out=None):
        out = np.empty(self.n_params, np.float32) if out is None else out
        p, k = _ptr(out)
        _check(self.lib.xpinn_get_params(self.h, p, self.n_params, _stream(out)))
        return out

    def set_params(self, theta):
        p, k = _ptr(theta if hasattr(theta, "data_ptr") else _f32(theta))
        _check(self.lib.xpinn_set_params(self.h, p, self.n_params, _stream(theta)))

    # ---------------------------------------------------------------- step
    def grad(self, losses=None, grads=None):
        """(losses [n_sub, 5], grads [n_params]) at the current parameters."""
        losses = np.empty((self.n_sub, N_TERMS), np.float32) if losses is None else losses
        grads = np.empty(self.n_params, np.float32) if grads is None else grads
        lp, _ = _ptr(losses)
        gp, _ = _ptr(grads)
        _check(self.lib.xpinn_grad(self.h, lp, gp, _stream(grads)))
        return losses, grads

    def objective(self, J=None, J_sub=None, losses=None, grads=None):
        """The method's objective J = sum_q J(Theta_q) (Eqs. cPINNLoss /
        XPINNLoss, weighted in the library) and its gradient: returns
        (J [1], J_sub [n_sub], losses [n_sub, 5], grads [n_params]).  Buffers
        may be numpy arrays or CUDA tensors (all on the same side)."""
        J = np.empty(1, np.float32) if J is None else J
        J_sub = np.empty(self.n_sub, np.float32) if J_sub is None else J_sub
        losses = np.empty((self.n_sub, N_TERMS), np.float32) if losses is None else losses
        grads = np.empty(self.n_params, np.float32) if grads is None else grads
        ptrs = [_ptr(x)[0] for x in (J, J_sub, losses, grads)]
        _check(self.lib.xpinn_objective(self.h, *ptrs, _stream(grads)))
        return J, J_sub, losses, grads

    def step(self, n_steps=1, losses=True, stream=None):
        """Run n_steps training steps; returns losses [n_steps, n_sub, 5] (or None)."""
        if losses is True:
            losses = np.empty((n_steps, self.n_sub, N_TERMS), np.float32)
        lp, _ = _ptr(losses) if losses is not None and losses is not False else (None, None)
        st = stream if stream is not None else _stream(losses if hasattr(losses, "is_cuda") else None)
        _check(self.lib.xpinn_step(self.h, n_steps, lp, st))
        return losses if lp is not None else None

    def sync(self, stream=None):
        """Wait for the work queued on `stream` (a cudaStream_t handle or None)
        and raise XpinnError if a device error (a wait that gave up, a
        non-finite loss) was recorded by an earlier asynchronous call."""
        _check(self.lib.xpinn_sync(self.h, stream))

    def set_residual_points(self, xy, f=None):
        xp_, k1 = _ptr(xy if hasattr(xy, "data_ptr") else _f32(xy))
        fp_, k2 = _ptr(f if (f is None or hasattr(f, "data_ptr")) else _f32(f))
        _check(self.lib.xpinn_set_residual_points(self.h, xp_, fp_, self.pb.n_res, _stream(xy)))

    # ---------------------------------------------------------------- jets / eval
    @staticmethod
    def n_comp(order):
        return (1, 3, 5)[order]

    def net_jets(self, q, net, xy, order=2, out=None):
        """Jets [n, D_out, K] of network `net` of subdomain q at xy [n, 2]."""
        n = int(xy.shape[0])
        D = self.pb.subs[q].nets[net].widths[-1]
        K = self.n_comp(order)
        if out is None:
            out = np.empty((n, D, K), np.float32)
        src = xy if hasattr(xy, "data_ptr") else _f32(xy)
        xp_, _ = _ptr(src)
        op, _ = _ptr(out)
        _check(self.lib.xpinn_net_jets(self.h, q, net, xp_, n, order, op, _stream(xy)))
        return out

    def eval(self, model, xy, order=0, out=None):
        """Stitched solution of Eq. FSol: [n, D_out_total, K]."""
        n = int(xy.shape[0])
        D = sum(net.widths[-1] for net in self.pb.subs[0].nets)
        K = self.n_comp(order)
        if out is None:
            out = np.empty((n, D, K), np.float32)
        src = xy if hasattr(xy, "data_ptr") else _f32(xy)
        xp_, _ = _ptr(src)
        op, _ = _ptr(out)
        _check(self.lib.xpinn_eval(self.h, model, xp_, n, order, op, _stream(xy)))
        return out

    def eval_workspace_size(self, n, order=0, model=0) -> int:
        b = C.c_size_t(0)
        _check(self.lib.xpinn_eval_workspace_size(self.h, model, n, order, C.byref(b)))
        return b.value

    def eval_ws(self, model, xy, order, out, workspace):
        """xpinn_eval from a caller-provided device workspace (a uint8 CUDA
        tensor of at least eval_workspace_size bytes); xy, out on the same side."""
        xp_, _ = _ptr(xy)
        op, _ = _ptr(out)
        _check(self.lib.xpinn_eval_ws(self.h, model, xp_, int(xy.shape[0]), order, op, workspace.data_ptr(),
                                      workspace.numel(), _stream(xy)))
        return out

    def _fork_desc(self, sel, xy_list, f_list, n_steps):
        sel = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
        counts = np.ascontiguousarray(np.array([len(x) for x in xy_list], dtype=np.int64))
        xy = _f32(np.concatenate(xy_list)) if len(xy_list) else np.zeros((0, 2), np.float32)
        f = None if f_list is None else _f32(np.concatenate(f_list))
        d = ForkDesc(n_sel=len(sel), sel=sel.ctypes.data, n_pts=counts.ctypes.data,
                     xy=xy.ctypes.data if len(xy) else None,
                     f=f.ctypes.data if f is not None and len(f) else None, n_steps=n_steps)
        return d, (sel, counts, xy, f)

    def fork_workspace_size(self, sel, xy_list, f_list=None, n_steps=1) -> int:
        d, keep = self._fork_desc(sel, xy_list, f_list, n_steps)
        b = C.c_size_t(0)
        _check(self.lib.xpinn_fork_workspace_size(self.h, C.byref(d), C.byref(b)))
        return b.value

    def fork_step(self, sel, xy_list, f_list=None, n_steps=1, workspace=None):
        """Train the subdomains `sel` on their own residual points (xy_list[i]
        for sel[i], forcing f_list[i] or zero) for n_steps on a private fork
        (xpinn_fork_step); the handle is unchanged.  Returns (losses
        [n_steps, n_sel, 5], the fork's parameters of sel, packed)."""
        import torch
        d, keep = self._fork_desc(sel, xy_list, f_list, n_steps)
        if workspace is None:
            workspace = torch.empty(self.fork_workspace_size(sel, xy_list, f_list, n_steps), dtype=torch.uint8,
                                    device="cuda")
        n_par = sum(self.pb.subs[q].n_params for q in keep[0])
        losses = np.empty((n_steps, len(keep[0]), N_TERMS), np.float32)
        params = np.empty(n_par, np.float32)
        _check(self.lib.xpinn_fork_step(self.h, C.byref(d), workspace.data_ptr(), workspace.numel(),
                                        losses.ctypes.data, params.ctypes.data, None))
        return losses, params

    # ------------------------------------------------------------ distributed step
    def step_begin(self, stream=None):
        _check(self.lib.xpinn_step_begin(self.h, stream))

    def step_end(self, losses=None, stream=None):
        lp, _ = _ptr(losses)
        _check(self.lib.xpinn_step_end(self.h, lp, stream))
        return losses

    def remote_values(self, out=None, stream=None):
        """This handle's side of every remote interface, [sum n_pts * nv]."""
        n = C.c_int64(0)
        _check(self.lib.xpinn_remote_values(self.h, None, C.byref(n), None))
        if out is None:
            out = np.empty(n.value, np.float32)
        op, _ = _ptr(out)
        _check(self.lib.xpinn_remote_values(self.h, op, C.byref(n), stream))
        return out

    def set_remote_values(self, vals, stream=None):
        vp_, _ = _ptr(vals if hasattr(vals, "data_ptr") else _f32(vals))
        _check(self.lib.xpinn_set_remote_values(self.h, vp_, int(vals.shape[0]) if len(vals.shape) else 0, stream))

    def iface_values(self):
        n = C.c_int64(0)
        _check(self.lib.xpinn_iface_values(self.h, None, C.byref(n), None))
        out = np.empty(n.value, np.float32)
        _check(self.lib.xpinn_iface_values(self.h, out.ctypes.data, C.byref(n), None))
        return out

    # ---------------------------------------------------------------- state / options
    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(self.lib.xpinn_get_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self.lib.xpinn_get_state(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, blob: bytes):
        _check(self.lib.xpinn_set_state(self.h, blob, len(blob)))

    def options(self) -> dict:
        o = Options()
        _check(self.lib.xpinn_get_options(self.h, C.byref(o)))
        return {f: getattr(o, f) for f, _ in Options._fields_}

    def signature(self) -> str:
        """Key of the problem's shape for the autotuning cache: PDE, per
        subdomain the network widths and point counts, interface sizes."""
        import hashlib
        pb = self.pb
        parts = [str(pb.pde)]
        for sd in pb.subs:
            parts.append(";".join(",".join(map(str, n.widths)) for n in sd.nets))
            parts.append(str(sd.res_xy.shape[0]))
            parts.append(",".join(str(d.xy.shape[0]) if d is not None else "0" for d in sd.data))
        parts.append(",".join(f"{it.method}:{it.xy.shape[0]}" for it in pb.ifaces))
        return hashlib.sha256("|".join(parts).encode()).hexdigest()[:24]

    @staticmethod
    def shape_class(sd) -> str:
        """Key of a subdomain's shape class (its networks' widths, hidden and
        output activations, fixed or trained slopes)."""
        return "|".join(",".join(map(str, n.widths)) + f":a{n.act}{'s' if n.adaptive else 'f'}o{n.out_act}"
                        for n in sd.nets)

    def tile_caps(self):
        caps = np.zeros(self.n_sub, np.int32)
        _check(self.lib.xpinn_get_tile_caps(self.h, caps.ctypes.data))
        return caps

    def set_tile_caps(self, caps):
        caps = None if caps is None else np.ascontiguousarray(np.asarray(caps, np.int32))
        _check(self.lib.xpinn_set_tile_caps(self.h, None if caps is None else caps.ctypes.data))

    def tc_select(self):
        """Per subdomain: 1 tensor-core kernel, 0 jet kernel, -1 default rule."""
        sel = np.zeros(self.n_sub, np.int32)
        _check(self.lib.xpinn_get_tc_select(self.h, sel.ctypes.data))
        return sel

    def set_tc_select(self, sel):
        sel = None if sel is None else np.ascontiguousarray(np.asarray(sel, np.int32))
        _check(self.lib.xpinn_set_tc_select(self.h, None if sel is None else sel.ctypes.data))

    def autotune(self, steps=5, cache=None, shapes=True, write=True) -> dict:
        """Pick tile shapes by timing: the launch options (xpinn_autotune),
        then a sub-tile cap and the tensor-core choice per shape class
        (xpinn_autotune_shapes).  With
        `cache` (a JSON file path) reuse a recorded choice for this problem
        signature, else time and (with `write`) record it: the options per
        problem signature, the caps per shape class."""
        import json
        key = self.signature()
        db = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                db = json.load(f)
        if key in db:
            keep = {k: v for k, v in db[key]["options"].items()
                    if k in ("points_per_thread", "items_per_cta", "max_points_per_tile",
                             "threads_per_cta")}
            self.set_options(**keep)
            cc = db[key].get("class_caps")
            if cc:
                self.set_tile_caps([cc.get(self.shape_class(sd), 0) for sd in self.pb.subs])
            ct = db[key].get("class_tc")
            if ct:
                self.set_tc_select([ct.get(self.shape_class(sd), -1) for sd in self.pb.subs])
            return db[key]
        o = Options()
        ms = C.c_float(0)
        _check(self.lib.xpinn_autotune(self.h, steps, C.byref(o), C.byref(ms)))
        rec = {"options": {f: getattr(o, f) for f, _ in Options._fields_}, "ms": ms.value}
        if shapes:
            ms2 = C.c_float(0)
            _check(self.lib.xpinn_autotune_shapes(self.h, steps, C.byref(ms2)))
            caps = self.tile_caps()
            rec["class_caps"] = {self.shape_class(sd): int(c) for sd, c in zip(self.pb.subs, caps)}
            rec["class_tc"] = {self.shape_class(sd): int(c) for sd, c in zip(self.pb.subs, self.tc_select())}
            rec["ms_shapes"] = ms2.value
        if cache and write:
            db[key] = rec
            with open(cache, "w") as f:
                json.dump(db, f, indent=1)
        return rec

    def phase_times(self):
        """Device ms of (start, exchange, jet kernel, reduce+Adam) of the last step."""
        ms = np.zeros(4, np.float32)
        _check(self.lib.xpinn_phase_times(self.h, ms.ctypes.data))
        return ms

    def plan_counts(self):
        """(work items of the step plan, residual items on the tensor-core
        kernel, subdomains those belong to)."""
        v = (C.c_int32 * 3)()
        _check(self.lib.xpinn_plan_counts(self.h, C.byref(v, 0), C.byref(v, 4), C.byref(v, 8)))
        return int(v[0]), int(v[1]), int(v[2])

    def tc_subdomains(self):
        """Per subdomain, 1 where its residual items run on the tensor-core
        kernel in the current plan."""
        on = np.zeros(self.pb.n_sub, np.int32)
        _check(self.lib.xpinn_tc_subdomains(self.h, on.ctypes.data))
        return on

    def tc_kernel_ms(self) -> float:
        """Device ms of the tensor-core training kernel in the last grouped
        step or grad call made with profile_phases on."""
        ms = C.c_float(0)
        _check(self.lib.xpinn_tc_kernel_time(self.h, C.byref(ms)))
        return ms.value

    def eval_kernel_ms(self) -> float:
        """Device ms of the evaluation kernel of the last routed evaluation
        made with profile_phases on."""
        ms = C.c_float(0)
        _check(self.lib.xpinn_eval_kernel_time(self.h, C.byref(ms)))
        return ms.value

    def set_options(self, **kw):
        cur = self.options()
        cur.update(kw)
        o = Options(**cur)
        _check(self.lib.xpinn_set_options(self.h, C.byref(o)))


class Server:
    """Continuous-batching request server over several Solvers (xpinn_server_*).

    submit_eval / submit_step return a ticket; poll(ticket) returns None while
    the request is pending, else a dict with the status, queue and latency
    times (ms), the batch size it was served in and its output."""

    def __init__(self, solvers, hbm_budget=1 << 30):
        self.lib = load()
        self.solvers = list(solvers)
        hs = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        out = C.c_void_p()
        _check(self.lib.xpinn_server_create(hs, len(self.solvers), hbm_budget, C.byref(out)))
        self.s = out
        self._keep = {}

    def submit_eval(self, model, xy, order=0, copy=0):
        xy = _f32(xy)
        pb = self.solvers[model].pb
        D = sum(n.widths[-1] for n in pb.subs[0].nets)
        out = np.empty((xy.shape[0], D, Solver.n_comp(order)), np.float32)
        r = Request(kind=0, model=model, copy=copy, order=order, n=xy.shape[0], xy=xy.ctypes.data,
                    out=out.ctypes.data, n_steps=0, losses=None)
        t = C.c_uint64()
        _check(self.lib.xpinn_server_submit(self.s, C.byref(r), C.byref(t)))
        self._keep[t.value] = (xy, out)
        return t.value

    def submit_step(self, model, n_steps=1):
        """Train model `model` in place for n_steps (xpinn_step)."""
        sv = self.solvers[model]
        losses = np.empty((n_steps, sv.n_sub, N_TERMS), np.float32)
        r = Request(kind=1, model=model, copy=0, order=0, n=0, xy=None, out=None, n_steps=n_steps,
                    losses=losses.ctypes.data)
        t = C.c_uint64()
        _check(self.lib.xpinn_server_submit(self.s, C.byref(r), C.byref(t)))
        self._keep[t.value] = (None, losses)
        return t.value

    def submit_fork(self, model, sel, xy_list, f_list=None, n_steps=1):
        """Train subdomains `sel` of model `model` on their own residual points
        (xy_list[i] for sel[i]) on a private fork (xpinn_fork_step); the
        result's "out" is (losses [n_steps, n_sel, 5], fork parameters)."""
        sv = self.solvers[model]
        sel = np.ascontiguousarray(np.asarray(sel, np.int32))
        counts = np.ascontiguousarray(np.array([len(x) for x in xy_list], np.int64))
        xy = _f32(np.concatenate(xy_list))
        f = None if f_list is None else _f32(np.concatenate(f_list))
        losses = np.empty((n_steps, len(sel), N_TERMS), np.float32)
        params = np.empty(sum(sv.pb.subs[q].n_params for q in sel if 0 <= q < sv.n_sub), np.float32)
        r = Request(kind=2, model=model, n=0, xy=xy.ctypes.data, out=None, n_steps=n_steps,
                    losses=losses.ctypes.data, n_sel=len(sel), sel=sel.ctypes.data, n_pts=counts.ctypes.data,
                    f=f.ctypes.data if f is not None else None, params=params.ctypes.data)
        t = C.c_uint64()
        _check(self.lib.xpinn_server_submit(self.s, C.byref(r), C.byref(t)))
        self._keep[t.value] = ((sel, counts, xy, f), (losses, params))
        return t.value

    def poll(self, ticket):
        res = Result()
        rc = self.lib.xpinn_server_poll(self.s, ticket, C.byref(res))
        if rc == 1:
            return None
        _check(rc)
        _, out = self._keep.pop(ticket)
        return {"status": res.status, "queue_ms": res.queue_ms, "latency_ms": res.latency_ms,
                "batch": res.batch, "tick_requests": res.tick_requests, "error": res.error.decode(), "out": out}

    def wait(self, ticket, sleep=1e-4):
        import time
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            time.sleep(sleep)

    def close(self):
        if getattr(self, "s", None):
            self.lib.xpinn_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
