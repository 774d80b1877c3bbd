"""ctypes binding of ``libagents.so`` (declared in ``include/agents.h``).

Argument marshalling only: every function here forwards to the C entry point of the
same name, converting arrays to raw pointers and raising :class:`AgentsError` on a
non-zero status.  Arrays may be torch tensors (device or host) or numpy arrays (host);
they must be C-contiguous with the dtype the header states.  No computation happens in
Python, and there is no fallback: if the library is not built, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_double, c_float, c_int, c_int32, c_int64, c_void_p, POINTER

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libagents.so")

AGENTS_OK = 0
AGENTS_EINVAL = -1
AGENTS_ECUDA = -2
AGENTS_ENOMEM = -3
AGENTS_ETIMEOUT = -4
AGENTS_EDIVERGED = -5
AGENTS_ESTATE = -6

_NAMES = {0: "AGENTS_OK", -1: "AGENTS_EINVAL", -2: "AGENTS_ECUDA", -3: "AGENTS_ENOMEM",
          -4: "AGENTS_ETIMEOUT", -5: "AGENTS_EDIVERGED", -6: "AGENTS_ESTATE"}


class AgentsError(RuntimeError):
    def __init__(self, code: int, func: str, message: str):
        super().__init__(f"{func} -> {_NAMES.get(code, code)}: {message}")
        self.code = code


class agents_params(ctypes.Structure):
    _fields_ = [("height", c_int32), ("width", c_int32), ("channels", c_int32),
                ("radius", c_int32), ("nsteps", c_int32), ("dt", c_double),
                ("alpha", c_double), ("rho", c_double), ("gamma", c_double),
                ("eps_lo", c_double * 2), ("eps_hi", c_double * 2),
                ("norm_mode", c_int32), ("tv_mode", c_int32), ("traj_mode", c_int32)]


class agents_solve_opts(ctypes.Structure):
    _fields_ = [("k_out", c_int32), ("k_in", c_int32), ("max_ls", c_int32),
                ("sigma0", c_double), ("ls_b", c_double), ("ls_c", c_double), ("tol", c_double)]


class agents_solve_info(ctypes.Structure):
    _fields_ = [("outer_done", c_int32), ("inner_done", c_int32), ("trials", c_int32),
                ("stalls", c_int32), ("stationary", c_int32),
                ("forward_steps", c_int64), ("adjoint_steps", c_int64),
                ("tv_sweeps", c_int64), ("final_res", c_double), ("final_obj", c_double),
                ("final_gap", c_double), ("final_sigma", c_double), ("kernel_launches", c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class agents_iter_record(ctypes.Structure):
    _fields_ = [("outer", c_int32), ("trials", c_int32), ("status", c_int32),
                ("reserved", c_int32), ("L0", c_double), ("L", c_double),
                ("gnorm2", c_double), ("tau", c_double)]


class agents_outer_record(ctypes.Structure):
    _fields_ = [("outer", c_int32), ("inner_done", c_int32), ("L", c_double), ("K", c_double),
                ("r", c_double), ("s", c_double), ("gap", c_double), ("rel_dc", c_double),
                ("res", c_double), ("sigma", c_double)]


class ws_net_config(ctypes.Structure):
    _fields_ = [("in_ch", c_int32), ("out_ch", c_int32), ("base", c_int32),
                ("levels", c_int32), ("nsteps", c_int32), ("eps_lo", ctypes.c_float * 2),
                ("eps_hi", ctypes.c_float * 2)]


_lib = None

# name -> (restype, argtypes)
_SIGNATURES = {
    "agents_default_params": (None, [POINTER(agents_params), c_int32, c_int32, c_int32, c_int32, c_int32]),
    "agents_default_solve_opts": (None, [POINTER(agents_solve_opts)]),
    "agents_init": (c_int, [POINTER(agents_params), c_void_p, c_void_p, POINTER(c_void_p)]),
    "agents_set_image": (c_int, [c_void_p, c_void_p]),
    "agents_destroy": (c_int, [c_void_p]),
    "agents_set_memory_limit": (c_int, [ctypes.c_uint64]),
    "agents_memory_held": (ctypes.c_uint64, []),
    "agents_debug_set_label_loop_cap": (c_int, [c_int32]),
    "agents_debug_set_fused": (c_int, [c_int32, ctypes.c_int64, ctypes.c_uint32]),
    "agents_fp32_probe": (c_int, [c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                  POINTER(c_double)]),
    "agents_last_error": (ctypes.c_char_p, [c_void_p]),
    "agents_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "agents_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "agents_objective": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "agents_adjoint_from": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "agents_flow_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pd_tv_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "alm_update": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "agents_labels": (c_int, [c_void_p, c_void_p, c_float, c_void_p, c_void_p]),
    "agents_solve_log": (c_int, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "agents_solve_outer_log": (c_int, [c_void_p, c_void_p, c_int32, POINTER(c_int32)]),
    "agents_objective_noalloc": (c_int, [c_int32, c_int32, c_int32, c_double, c_double, c_int32,
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p, c_void_p]),
    "solve": (c_int, [c_void_p, POINTER(agents_solve_opts), c_void_p, c_void_p, c_void_p,
                      c_void_p, c_void_p, POINTER(agents_solve_info)]),
    "dal_solve": (c_int, [c_void_p, POINTER(agents_solve_opts), c_void_p, c_void_p,
                          POINTER(agents_solve_info)]),
    "agents_solve_batch": (c_int, [c_int32, POINTER(c_void_p), POINTER(agents_solve_opts),
                                   c_int32, c_int32, POINTER(c_void_p), POINTER(c_void_p),
                                   POINTER(c_void_p), POINTER(agents_solve_info)]),
    # warm-start network (include/warmstart.h)
    "ws_last_error": (ctypes.c_char_p, []),
    "ws_conv3x3_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                   c_int32, c_void_p]),
    "ws_conv3x3_backward_data": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                         c_int32, c_int32, c_int32, c_void_p]),
    "ws_conv3x3_backward_weight": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                           c_int32, c_int32, c_int32, c_int32, c_int32,
                                           c_void_p, ctypes.c_size_t, c_void_p]),
    "ws_conv3x3_backward_weight_workspace": (ctypes.c_size_t, [c_int32, c_int32, c_int32,
                                                               c_int32, c_int32]),
    "ws_transpose_weights": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "ws_tensor_core_fault_take": (c_int, []),
    "ws_net_create": (c_int, [POINTER(ws_net_config), c_void_p, POINTER(c_void_p)]),
    "ws_net_destroy": (None, [c_void_p]),
    "ws_net_num_params": (ctypes.c_int64, [c_void_p]),
    "ws_net_set_params": (c_int, [c_void_p, c_void_p]),
    "ws_net_get_params": (c_int, [c_void_p, c_void_p]),
    "ws_net_forward": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32,
                               c_void_p, c_void_p, c_void_p]),
    "ws_net_forward_lifted": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32,
                                      c_int32, c_void_p, c_void_p]),
    "ws_net_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32,
                                 c_int32, ctypes.c_float, POINTER(c_double), c_void_p]),
    "ws_net_adam_step": (c_int, [c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float]),
}


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2510_16154_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x, dtype=None):
    """Raw address of a torch tensor / numpy array / int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):          # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(x.dtype).split(".")[-1] != dtype:
            raise TypeError(f"expected {dtype}, got {x.dtype}")
        return x.data_ptr()
    if hasattr(x, "ctypes"):            # numpy.ndarray
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype.name != dtype:
            raise TypeError(f"expected {dtype}, got {x.dtype}")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x).__name__} as a pointer")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream           # torch.cuda.Stream


def _check(status: int, func: str, ctx=None):
    if status != AGENTS_OK:
        msg = load().agents_last_error(ctx)
        raise AgentsError(status, func, msg.decode() if msg else "")


# ---------------------------------------------------------------- entry points

def agents_default_params(height, width, channels, radius, nsteps) -> agents_params:
    p = agents_params()
    load().agents_default_params(ctypes.byref(p), height, width, channels, radius, nsteps)
    return p


def agents_default_solve_opts() -> agents_solve_opts:
    o = agents_solve_opts()
    load().agents_default_solve_opts(ctypes.byref(o))
    return o


def agents_init(params: agents_params, c0, stream=None) -> c_void_p:
    ctx = c_void_p()
    _check(load().agents_init(ctypes.byref(params), _ptr(c0, "float32"), _stream(stream),
                              ctypes.byref(ctx)), "agents_init")
    return ctx


def agents_set_image(ctx, c0):
    _check(load().agents_set_image(ctx, _ptr(c0, "float32")), "agents_set_image", ctx)


def agents_destroy(ctx):
    _check(load().agents_destroy(ctx), "agents_destroy")


def agents_set_memory_limit(nbytes: int):
    _check(load().agents_set_memory_limit(int(nbytes)), "agents_set_memory_limit")


def agents_memory_held() -> int:
    return int(load().agents_memory_held())


def agents_debug_set_label_loop_cap(cap: int):
    _check(load().agents_debug_set_label_loop_cap(int(cap)), "agents_debug_set_label_loop_cap")


def agents_debug_set_fused(mode: int = 1, wait_ns: int = 0, skew_once: int = 0):
    """Whole-sweep launches: mode 0 never, 1 where they measured faster (default), 2 for
    every tiled sweep; the time limit of one of their waits (0: the default); a one-shot
    offset of the next launch's wait targets (test hook)."""
    _check(load().agents_debug_set_fused(int(mode), int(wait_ns), int(skew_once)),
           "agents_debug_set_fused")


def agents_fp32_probe(packed: bool, blocks: int, iters: int, sink, stream=None) -> float:
    """Launch the FP32 FMA probe kernel; returns its flop count."""
    flops = c_double(0.0)
    _check(load().agents_fp32_probe(int(bool(packed)), int(blocks), int(iters),
                                    _ptr(sink, "float32"), _stream(stream),
                                    ctypes.byref(flops)), "agents_fp32_probe")
    return flops.value


def agents_last_error(ctx=None) -> str:
    msg = load().agents_last_error(ctx)
    return msg.decode() if msg else ""


def agents_forward(ctx, eps, cT=None, store=True):
    _check(load().agents_forward(ctx, _ptr(eps, "float64"), _ptr(cT, "float32"), int(bool(store))),
           "agents_forward", ctx)


def agents_adjoint(ctx, eps, v, mu, D_out, obj_out=None, lambda0=None):
    _check(load().agents_adjoint(ctx, _ptr(eps, "float64"), _ptr(v, "float32"),
                                 _ptr(mu, "float32"), _ptr(D_out, "float64"),
                                 _ptr(obj_out, "float64"), _ptr(lambda0, "float32")),
           "agents_adjoint", ctx)


def agents_adjoint_from(ctx, eps, lambdaT, D_out, lambda0=None):
    _check(load().agents_adjoint_from(ctx, _ptr(eps, "float64"), _ptr(lambdaT, "float32"),
                                      _ptr(D_out, "float64"), _ptr(lambda0, "float32")),
           "agents_adjoint_from", ctx)


def agents_flow_backward(ctx, eps, grad_cT, grad_eps=None, grad_c0=None):
    _check(load().agents_flow_backward(ctx, _ptr(eps, "float64"), _ptr(grad_cT, "float32"),
                                       _ptr(grad_eps, "float64"), _ptr(grad_c0, "float32")),
           "agents_flow_backward", ctx)


def agents_objective(ctx, c, v, mu, obj_out=None, lam=None):
    _check(load().agents_objective(ctx, _ptr(c, "float32"), _ptr(v, "float32"),
                                   _ptr(mu, "float32"), _ptr(obj_out, "float64"),
                                   _ptr(lam, "float32")), "agents_objective", ctx)


def pd_tv_step(ctx, c, mu, v):
    _check(load().pd_tv_step(ctx, _ptr(c, "float32"), _ptr(mu, "float32"), _ptr(v, "float32")),
           "pd_tv_step", ctx)


def alm_update(ctx, c, c_prev, v, v_prev, mu, stats=None):
    _check(load().alm_update(ctx, _ptr(c, "float32"), _ptr(c_prev, "float32"),
                             _ptr(v, "float32"), _ptr(v_prev, "float32"), _ptr(mu, "float32"),
                             _ptr(stats, "float64")), "alm_update", ctx)


def agents_labels(ctx, c, threshold, labels_out) -> int:
    count = c_int32(0)
    _check(load().agents_labels(ctx, _ptr(c, "float32"), c_float(threshold),
                                _ptr(labels_out, "int32"), ctypes.byref(count)),
           "agents_labels", ctx)
    return count.value


def solve(ctx, opts: agents_solve_opts, eps_io, mu_io, v_out=None, c_out=None,
          labels_out=None) -> agents_solve_info:
    info = agents_solve_info()
    _check(load().solve(ctx, ctypes.byref(opts), _ptr(eps_io, "float64"), _ptr(mu_io, "float32"),
                        _ptr(v_out, "float32"), _ptr(c_out, "float32"),
                        _ptr(labels_out, "int32"), ctypes.byref(info)), "solve", ctx)
    return info


def dal_solve(ctx, opts: agents_solve_opts, eps_io, c_out=None) -> agents_solve_info:
    info = agents_solve_info()
    _check(load().dal_solve(ctx, ctypes.byref(opts), _ptr(eps_io, "float64"),
                            _ptr(c_out, "float32"), ctypes.byref(info)), "dal_solve", ctx)
    return info


def agents_solve_batch(ctxs, opts: agents_solve_opts, eps_list, mu_list, c_out_list=None,
                       autotune=False, use_graph=True):
    """Batched solve of len(ctxs) contexts; returns a list of agents_solve_info."""
    n = len(ctxs)
    arr = (c_void_p * n)(*[c.value if isinstance(c, c_void_p) else c for c in ctxs])
    eps = (c_void_p * n)(*[_ptr(e, "float64") for e in eps_list])
    mus = (c_void_p * n)(*[_ptr(m, "float32") for m in mu_list])
    outs = None
    if c_out_list is not None:
        outs = (c_void_p * n)(*[_ptr(c, "float32") for c in c_out_list])
    infos = (agents_solve_info * n)()
    st = load().agents_solve_batch(n, arr, ctypes.byref(opts), int(bool(autotune)),
                                   int(bool(use_graph)), eps, mus, outs, infos)
    try:
        _check(st, "agents_solve_batch", ctxs[0])
    except AgentsError as err:
        # AGENTS_EDIVERGED still writes every image's outputs and record
        err.infos = list(infos) if st == AGENTS_EDIVERGED else None
        raise
    return list(infos)


def agents_solve_log(ctx):
    """Per-DAL-iteration records of the last solve() as a list of dicts."""
    n = c_int32(0)
    _check(load().agents_solve_log(ctx, None, 0, ctypes.byref(n)), "agents_solve_log", ctx)
    buf = (agents_iter_record * max(n.value, 1))()
    _check(load().agents_solve_log(ctx, buf, n.value, ctypes.byref(n)), "agents_solve_log", ctx)
    return [{f: getattr(buf[i], f) for f, _ in agents_iter_record._fields_ if f != "reserved"}
            for i in range(n.value)]


def agents_solve_outer_log(ctx):
    """Per-multiplier-step records of the last solve() as a list of dicts."""
    n = c_int32(0)
    _check(load().agents_solve_outer_log(ctx, None, 0, ctypes.byref(n)),
           "agents_solve_outer_log", ctx)
    buf = (agents_outer_record * max(n.value, 1))()
    _check(load().agents_solve_outer_log(ctx, buf, n.value, ctypes.byref(n)),
           "agents_solve_outer_log", ctx)
    return [{f: getattr(buf[i], f) for f, _ in agents_outer_record._fields_}
            for i in range(n.value)]


def write_solve_log_jsonl(ctx, path, info=None):
    """Write the last solve()'s logs as JSON lines: one {"kind": "dal", ...} line per DAL
    iteration, one {"kind": "outer", ...} line per multiplier step, and the solve_info."""
    import json
    with open(path, "w") as f:
        for rec in agents_solve_log(ctx):
            f.write(json.dumps({"kind": "dal", **rec}) + "\n")
        for rec in agents_solve_outer_log(ctx):
            f.write(json.dumps({"kind": "outer", **rec}) + "\n")
        if info is not None:
            f.write(json.dumps({"kind": "info", **info.as_dict()}) + "\n")


def _require_cuda(name, x, numel, dtype):
    if not (hasattr(x, "is_cuda") and x.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if str(x.dtype).split(".")[-1] != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {x.dtype}")
    if x.numel() < numel:
        raise ValueError(f"{name} holds {x.numel()} elements, needs at least {numel}")


def agents_objective_noalloc(height, width, channels, alpha, rho, tv_mode, c, c0, v, mu,
                             obj_out, lam=None, stream=None):
    """Objective and terminal adjoint with no device allocation (caller-owned inputs and
    outputs, a static device scratch array inside the library).  Every buffer must be a
    CUDA tensor holding at least its field's element count: the library cannot check
    sizes."""
    n = int(height) * int(width) * int(channels)
    for name, x, k in (("c", c, n), ("c0", c0, n), ("v", v, 2 * n), ("mu", mu, 2 * n)):
        _require_cuda(name, x, k, "float32")
    _require_cuda("obj_out", obj_out, 1, "float64")
    if lam is not None:
        _require_cuda("lam", lam, n, "float32")
    _check(load().agents_objective_noalloc(height, width, channels, alpha, rho, tv_mode,
                                           _ptr(c, "float32"), _ptr(c0, "float32"),
                                           _ptr(v, "float32"), _ptr(mu, "float32"),
                                           _ptr(obj_out, "float64"), _ptr(lam, "float32"),
                                           _stream(stream)), "agents_objective_noalloc")


class Context:
    """Owns one ``agents_ctx`` (destroyed on close / garbage collection)."""

    def __init__(self, params: agents_params, c0, stream=None):
        self.params = params
        self.handle = agents_init(params, c0, stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            agents_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- warm-start network
def _ws_check(status: int, func: str):
    if status != AGENTS_OK:
        msg = load().ws_last_error()
        raise AgentsError(status, func, msg.decode() if msg else "")


def ws_conv3x3_forward(x, w16, bias, y, N, H, W, Cin, Cout, relu=True, up=False, add=None,
                       y2=None, stream=None):
    _ws_check(load().ws_conv3x3_forward(_ptr(x, "float32"), _ptr(w16), _ptr(bias, "float32"),
                                        _ptr(y, "float32"), _ptr(add, "float32"),
                                        _ptr(y2, "float32"), N, H, W, Cin, Cout, int(relu),
                                        int(up), _stream(stream)), "ws_conv3x3_forward")


def ws_conv3x3_backward_data(dy, wt16, dx, N, H, W, Cin, Cout, stream=None):
    _ws_check(load().ws_conv3x3_backward_data(_ptr(dy, "float32"), _ptr(wt16), _ptr(dx, "float32"),
                                              N, H, W, Cin, Cout, _stream(stream)),
              "ws_conv3x3_backward_data")


def ws_conv3x3_backward_weight_workspace(N, H, W, Cin, Cout) -> int:
    return int(load().ws_conv3x3_backward_weight_workspace(N, H, W, Cin, Cout))


def ws_conv3x3_backward_weight(x, dy, dw, db, N, H, W, Cin, Cout, workspace, up=False,
                               stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _ws_check(load().ws_conv3x3_backward_weight(_ptr(x, "float32"), _ptr(dy, "float32"),
                                                _ptr(dw, "float32"), _ptr(db, "float32"), N, H,
                                                W, Cin, Cout, int(up), _ptr(workspace), nbytes,
                                                _stream(stream)),
              "ws_conv3x3_backward_weight")


def ws_transpose_weights(w, w16, wt16, Cin, Cout, stream=None):
    _ws_check(load().ws_transpose_weights(_ptr(w, "float32"), _ptr(w16), _ptr(wt16), Cin, Cout,
                                          _stream(stream)), "ws_transpose_weights")


def ws_tensor_core_fault_take() -> bool:
    """True if a tensor-core convolution gave up a bounded wait since the last call."""
    r = load().ws_tensor_core_fault_take()
    if r < 0:
        _ws_check(r, "ws_tensor_core_fault_take")
    return r == 1
