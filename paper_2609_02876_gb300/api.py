"""Python face of the C-ABI: the same entry points over torch CUDA tensors.

Argument marshalling only (shapes, dtypes, the current stream); every step of
the path runs in the library's kernels. Two layouts are accepted:
 - "aos" (default): the paper's shapes, params (n, P), y0 (n, d) (paper
   Sec. 3.4 interface); outputs in the same orientation.
 - "soa": the library's native structure-of-arrays layout, params [P][n],
   y0 [d][n], y_save [n_save][d][n]; no transposes.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N


def _pid(problem) -> int:
    return N.PROBLEMS[problem] if isinstance(problem, str) else int(problem)


def problem_info(problem):
    d, P, s, nw = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    rc = N.lib().gs_problem_info(_pid(problem), C.byref(d), C.byref(P), C.byref(s), C.byref(nw))
    if rc != N.GS_OK:
        raise N.GsError(rc, "gs_problem_info")
    return d.value, P.value, bool(s.value), nw.value


def _opts(precision="fp64", method=None, ckpt_k=0, max_steps=0, h0=0.0, step_counts=None,
          kernel_ms=None, timeout_ms=0.0, record_info=None, control="fast", record_stages=False) -> N.GsOptions:
    o = N.GsOptions()
    N.lib().gs_default_options(C.byref(o))
    o.precision = {"fp64": N.GS_FP64, "fp32_mixed": N.GS_FP32_MIXED}[precision]
    o.control = {"fast": N.GS_CONTROL_FAST, "fp64": N.GS_CONTROL_FP64}[control]
    o.record_stages = 1 if record_stages else 0
    o.method = {None: N.GS_METHOD_AUTO, "tsit5": N.GS_METHOD_TSIT5, "rodas5p": N.GS_METHOD_RODAS5P,
                "rosenbrock23": N.GS_METHOD_ROSENBROCK23, "verner7": N.GS_METHOD_VERNER7}[method]
    o.ckpt_k = int(ckpt_k)
    o.max_steps = int(max_steps)
    o.h0 = float(h0)
    o.timeout_ms = float(timeout_ms)
    o.step_counts = step_counts.data_ptr() if step_counts is not None else None
    if kernel_ms is not None:  # a (2,) float32 numpy array filled with the kernels' device times
        o.kernel_ms = kernel_ms.ctypes.data_as(C.POINTER(C.c_float))
    if record_info is not None:  # a (2,) int32 numpy array: checkpoint interval k, stored stages (0/1)
        o.record_info = record_info.ctypes.data_as(C.POINTER(C.c_int32))
    return o


def _dev(x: torch.Tensor, name: str, dtype=torch.float64) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return x.contiguous()


def _soa_in(x: torch.Tensor, width: int, layout: str, name: str) -> torch.Tensor:
    x = _dev(x, name)
    if layout == "aos":
        if x.dim() != 2 or x.shape[1] != width:
            raise ValueError(f"{name} must have shape (n, {width})")
        return x.t().contiguous()
    if x.dim() != 2 or x.shape[0] != width:
        raise ValueError(f"{name} must have shape ({width}, n)")
    return x


def _save_t(save_t):
    st = np.ascontiguousarray(np.asarray(save_t, dtype=np.float64).reshape(-1))
    return st, st.ctypes.data_as(C.POINTER(C.c_double))


def _ptr(x):
    return None if x is None else x.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Record:
    """A device-resident record (the accepted mesh + state checkpoints)."""

    def __init__(self, handle: int, problem: int, n: int, d: int, P: int, n_save: int):
        self._h = C.c_void_p(handle)
        self.problem, self.n, self.d, self.P, self.n_save = problem, n, d, P, n_save

    @property
    def handle(self):
        return self._h

    def bytes(self) -> int:
        b = C.c_size_t()
        rc = N.lib().gs_record_bytes(self._h, C.byref(b))
        if rc != N.GS_OK:
            raise N.GsError(rc, "gs_record_bytes")
        return b.value

    def stats(self):
        n, a, t = C.c_int64(), C.c_int64(), C.c_int64()
        rc = N.lib().gs_record_stats(self._h, C.byref(n), C.byref(a), C.byref(t))
        if rc != N.GS_OK:
            raise N.GsError(rc, "gs_record_stats")
        return {"n": n.value, "accepted": a.value, "attempted": t.value}

    def export_mesh(self):
        """(offsets [n+1], h [total]) as numpy arrays (host copy)."""
        off = np.zeros(self.n + 1, np.int64)
        rc = N.lib().gs_record_export_mesh(self._h, off.ctypes.data_as(C.POINTER(C.c_int64)), None)
        if rc != N.GS_OK:
            raise N.GsError(rc, "gs_record_export_mesh")
        h = np.zeros(max(int(off[-1]), 1))
        rc = N.lib().gs_record_export_mesh(self._h, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                           h.ctypes.data_as(C.POINTER(C.c_double)))
        if rc != N.GS_OK:
            raise N.GsError(rc, "gs_record_export_mesh")
        return off, h[: int(off[-1])]

    def free(self):
        if self._h and self._h.value:
            N.lib().gs_record_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def forward_record(problem, params, y0, t0, t1, save_t, rtol, atol, *, shared_w=None, layout="aos",
                   want_saves=True, check=True, **opts):
    """gs_forward_record. Returns (record, y_save, status)."""
    pid = _pid(problem)
    d, P, _, nw = problem_info(pid)
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    n = p.shape[1]
    st, stp = _save_t(save_t)
    ns = st.size
    ysv = torch.empty((ns, d, n), dtype=torch.float64, device=p.device) if want_saves else None
    status = torch.empty(n, dtype=torch.int32, device=p.device)
    w = _dev(shared_w, "shared_w", torch.float32) if nw else None
    counts = torch.empty((2, n), dtype=torch.int32, device=p.device) if opts.pop("step_counts", False) else None
    o = _opts(step_counts=counts, **opts)
    h = C.c_void_p()
    rc = N.lib().gs_forward_record(pid, n, p.data_ptr(), y.data_ptr(), _ptr(w), float(t0), float(t1), stp, ns,
                                   float(rtol), float(atol), C.byref(o), _stream(), _ptr(ysv), status.data_ptr(),
                                   C.byref(h))
    if rc not in (N.GS_OK, N.GS_ERR_TRAJ_FAILED) or (check and rc != N.GS_OK):
        if h.value:
            N.lib().gs_record_free(h)
        raise N.GsError(rc, "gs_forward_record")
    rec = Record(h.value, pid, n, d, P, ns)
    rec.step_counts = counts
    if ysv is not None and layout == "aos":
        ysv = ysv.permute(2, 0, 1)
    return rec, ysv, status


def reverse(record: Record, params, y0, y_save_bar=None, *, shared_w=None, layout="aos", want_loss=True):
    """gs_reverse. Returns dict(loss, params_bar, y0_bar[, shared_w_bar])."""
    d, P = record.d, record.P
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    n = p.shape[1]
    yb = None
    if y_save_bar is not None:
        yb = _dev(y_save_bar, "y_save_bar")
        if layout == "aos":
            yb = yb.permute(1, 2, 0).contiguous()
    pb = torch.empty((P, n), dtype=torch.float64, device=p.device)
    y0b = torch.empty((d, n), dtype=torch.float64, device=p.device)
    loss = torch.empty(n, dtype=torch.float64, device=p.device) if (want_loss and yb is None) else None
    nw = problem_info(record.problem)[3]
    w = _dev(shared_w, "shared_w", torch.float32) if nw else None
    wb = torch.zeros(nw, dtype=torch.float32, device=p.device) if nw else None
    rc = N.lib().gs_reverse(record.handle, p.data_ptr(), y.data_ptr(), _ptr(w), _ptr(yb), _ptr(loss),
                            pb.data_ptr(), y0b.data_ptr(), _ptr(wb), _stream())
    if rc != N.GS_OK:
        raise N.GsError(rc, "gs_reverse")
    if layout == "aos":
        pb, y0b = pb.t(), y0b.t()
    out = {"loss": loss, "params_bar": pb, "y0_bar": y0b}
    if nw:
        out["shared_w_bar"] = wb
    return out


def refresh(record: Record, params, y0, *, shared_w=None, layout="aos"):
    """gs_record_refresh: re-run the record's state chains on its frozen mesh with new
    (params, y0); a following reverse() at the same params gives the frozen-mesh gradient."""
    d, P = record.d, record.P
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    nw = problem_info(record.problem)[3]
    w = _dev(shared_w, "shared_w", torch.float32) if nw else None
    rc = N.lib().gs_record_refresh(record.handle, p.data_ptr(), y.data_ptr(), _ptr(w), _stream())
    if rc != N.GS_OK:
        raise N.GsError(rc, "gs_record_refresh")


def _dirs_in(x, width: int, layout: str, name: str):
    """Tangent directions: one (n, width) / (width, n) array or a stack (n_dir, ...). Returns [n_dir][width][n]."""
    if x is None:
        return None
    x = _dev(x, name)
    if x.dim() == 2:
        x = x.unsqueeze(0)
    if x.dim() != 3:
        raise ValueError(f"{name} must have 2 or 3 dimensions")
    if layout == "aos":
        if x.shape[2] != width:
            raise ValueError(f"{name} must have shape (n_dir, n, {width})")
        return x.permute(0, 2, 1).contiguous()
    if x.shape[1] != width:
        raise ValueError(f"{name} must have shape (n_dir, {width}, n)")
    return x.contiguous()


def replay_jvp(record: Record, params, y0, params_dot=None, y0_dot=None, *, layout="aos", want_y_save_dot=False):
    """gs_replay_jvp: forward mode of the replay on the record's mesh. Returns
    dict(loss, loss_dot (n_dir, n)[, y_save_dot]); y_save_dot is (n_dir, n, n_save, d)
    for layout "aos", [n_dir][n_save][d][n] for "soa"."""
    d, P = record.d, record.P
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    n = p.shape[1]
    pd = _dirs_in(params_dot, P, layout, "params_dot")
    yd = _dirs_in(y0_dot, d, layout, "y0_dot")
    if pd is None and yd is None:
        raise ValueError("at least one of params_dot and y0_dot is required")
    nd = (pd if pd is not None else yd).shape[0]
    if pd is not None and yd is not None and pd.shape[0] != yd.shape[0]:
        raise ValueError("params_dot and y0_dot must hold the same number of directions")
    loss = torch.empty(n, dtype=torch.float64, device=p.device)
    ldot = torch.empty((nd, n), dtype=torch.float64, device=p.device)
    ysd = torch.empty((nd, record.n_save, d, n), dtype=torch.float64, device=p.device) if want_y_save_dot else None
    rc = N.lib().gs_replay_jvp(record.handle, p.data_ptr(), y.data_ptr(), nd, _ptr(pd), _ptr(yd), loss.data_ptr(),
                               ldot.data_ptr(), _ptr(ysd), _stream())
    if rc != N.GS_OK:
        raise N.GsError(rc, "gs_replay_jvp")
    out = {"loss": loss, "loss_dot": ldot}
    if ysd is not None:
        out["y_save_dot"] = ysd.permute(0, 3, 1, 2) if layout == "aos" else ysd
    return out


def forward_grad(record: Record, params, y0, *, wrt=("params", "y0"), layout="aos"):
    """gs_forward_grad: the built-in loss's gradient by forward mode (one pass per input
    of a trajectory). Returns dict(loss, params_bar, y0_bar) (None for inputs not in wrt)."""
    d, P = record.d, record.P
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    n = p.shape[1]
    loss = torch.empty(n, dtype=torch.float64, device=p.device)
    pb = torch.empty((P, n), dtype=torch.float64, device=p.device) if "params" in wrt else None
    y0b = torch.empty((d, n), dtype=torch.float64, device=p.device) if "y0" in wrt else None
    rc = N.lib().gs_forward_grad(record.handle, p.data_ptr(), y.data_ptr(), loss.data_ptr(), _ptr(pb), _ptr(y0b),
                                 _stream())
    if rc != N.GS_OK:
        raise N.GsError(rc, "gs_forward_grad")
    if layout == "aos":
        pb = pb.t() if pb is not None else None
        y0b = y0b.t() if y0b is not None else None
    return {"loss": loss, "params_bar": pb, "y0_bar": y0b}


class Context:
    """A gs_context: its own device workspace, so solves on different contexts
    (and streams) run concurrently."""

    def __init__(self):
        h = C.c_void_p()
        rc = N.lib().gs_context_create(C.byref(h))
        if rc != N.GS_OK:
            raise N.GsError(rc, "gs_context_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def bytes(self) -> int:
        b = C.c_size_t()
        N.lib().gs_context_bytes(self._h, C.byref(b))
        return b.value

    def close(self):
        if self._h and self._h.value:
            N.lib().gs_context_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve_grad(self, problem, params, y0, t0, t1, save_t, rtol, atol, **kw):
        return solve_grad(problem, params, y0, t0, t1, save_t, rtol, atol, context=self, **kw)


def solve(problem, params, y0, t0, t1, save_t, rtol, atol, *, shared_w=None, layout="aos", want_saves=True,
          check=True, **opts):
    """gs_solve (forward only, nothing recorded). Returns dict(y_save, y_final, status, rc)."""
    pid = _pid(problem)
    d, P, _, nw = problem_info(pid)
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    n = p.shape[1]
    st, stp = _save_t(save_t)
    ns = st.size
    ysv = torch.empty((ns, d, n), dtype=torch.float64, device=p.device) if want_saves else None
    yf = torch.empty((d, n), dtype=torch.float64, device=p.device)
    status = torch.empty(n, dtype=torch.int32, device=p.device)
    w = _dev(shared_w, "shared_w", torch.float32) if nw else None
    counts = torch.empty((2, n), dtype=torch.int32, device=p.device) if opts.pop("step_counts", False) else None
    o = _opts(step_counts=counts, **opts)
    rc = N.lib().gs_solve(pid, n, p.data_ptr(), y.data_ptr(), _ptr(w), float(t0), float(t1), stp, ns, float(rtol),
                          float(atol), C.byref(o), _stream(), _ptr(ysv), yf.data_ptr(), status.data_ptr())
    if rc not in (N.GS_OK, N.GS_ERR_TRAJ_FAILED) or (check and rc != N.GS_OK):
        raise N.GsError(rc, "gs_solve")
    if layout == "aos":
        yf = yf.t()
        if ysv is not None:
            ysv = ysv.permute(2, 0, 1)
    res = {"y_save": ysv, "y_final": yf, "status": status, "rc": rc}
    if counts is not None:
        res["step_counts"] = counts
    return res


def solve_grad(problem, params, y0, t0, t1, save_t, rtol, atol, *, shared_w=None, layout="aos", check=True,
               out=None, context=None, **opts):
    """gs_solve_grad (record + reverse, built-in loss); with `context`, gs_solve_grad_ctx.
    Returns dict(loss, params_bar, y0_bar, status)."""
    pid = _pid(problem)
    d, P, _, nw = problem_info(pid)
    p = _soa_in(params, P, layout, "params")
    y = _soa_in(y0, d, layout, "y0")
    n = p.shape[1]
    st, stp = _save_t(save_t)
    if out is None:
        out = {"loss": torch.empty(n, dtype=torch.float64, device=p.device),
               "params_bar": torch.empty((P, n), dtype=torch.float64, device=p.device),
               "y0_bar": torch.empty((d, n), dtype=torch.float64, device=p.device),
               "status": torch.empty(n, dtype=torch.int32, device=p.device)}
    w = _dev(shared_w, "shared_w", torch.float32) if nw else None
    wb = torch.zeros(nw, dtype=torch.float32, device=p.device) if nw else None
    counts = torch.empty((2, n), dtype=torch.int32, device=p.device) if opts.pop("step_counts", False) else None
    o = _opts(step_counts=counts, **opts)
    args = (pid, n, p.data_ptr(), y.data_ptr(), _ptr(w), float(t0), float(t1), stp, st.size, float(rtol),
            float(atol), C.byref(o), _stream(), out["loss"].data_ptr(), out["params_bar"].data_ptr(),
            out["y0_bar"].data_ptr(), _ptr(wb), out["status"].data_ptr())
    if context is None:
        rc = N.lib().gs_solve_grad(*args)
    else:
        rc = N.lib().gs_solve_grad_ctx(context.handle, *args)
    if rc not in (N.GS_OK, N.GS_ERR_TRAJ_FAILED) or (check and rc != N.GS_OK):
        raise N.GsError(rc, "gs_solve_grad")
    res = dict(out)
    res["rc"] = rc
    if counts is not None:
        res["step_counts"] = counts
    if nw:
        res["shared_w_bar"] = wb
    if layout == "aos":
        res["params_bar"], res["y0_bar"] = res["params_bar"].t(), res["y0_bar"].t()
    return res


def solve_grad_host(problem, params, y0, t0, t1, save_t, rtol, atol, *, shared_w=None, chunk=0, check=True,
                    out=None, **opts):
    """gs_solve_grad_host: host (CPU) SoA tensors in and out, params [P][n], y0 [d][n]
    (pin them for overlapped copies); the library pipelines the copies with the
    solve in chunks. Returns dict(loss, params_bar [P][n], y0_bar [d][n], status) on
    the host (plus shared_w_bar on the device for shared-weight problems)."""
    pid = _pid(problem)
    d, P, _, nw = problem_info(pid)
    p = torch.as_tensor(params, dtype=torch.float64)
    y = torch.as_tensor(y0, dtype=torch.float64)
    if p.is_cuda or y.is_cuda or p.dim() != 2 or y.dim() != 2 or p.shape[0] != P or y.shape[0] != d:
        raise ValueError(f"params and y0 must be host tensors of shapes ({P}, n) and ({d}, n)")
    p, y = p.contiguous(), y.contiguous()
    n = p.shape[1]
    if y.shape[1] != n:
        raise ValueError("params and y0 hold different ensemble sizes")
    st, stp = _save_t(save_t)
    pin = p.is_pinned()
    if out is None:
        out = {"loss": torch.empty(n, dtype=torch.float64, pin_memory=pin),
               "params_bar": torch.empty((P, n), dtype=torch.float64, pin_memory=pin),
               "y0_bar": torch.empty((d, n), dtype=torch.float64, pin_memory=pin),
               "status": torch.empty(n, dtype=torch.int32, pin_memory=pin)}
    w = _dev(shared_w, "shared_w", torch.float32) if nw else None
    wb = torch.zeros(nw, dtype=torch.float32, device="cuda") if nw else None
    o = _opts(**opts)
    rc = N.lib().gs_solve_grad_host(pid, n, p.data_ptr(), y.data_ptr(), _ptr(w), float(t0), float(t1), stp, st.size,
                                    float(rtol), float(atol), C.byref(o), int(chunk), out["loss"].data_ptr(),
                                    out["params_bar"].data_ptr(), out["y0_bar"].data_ptr(), _ptr(wb),
                                    out["status"].data_ptr())
    if rc not in (N.GS_OK, N.GS_ERR_TRAJ_FAILED) or (check and rc != N.GS_OK):
        raise N.GsError(rc, "gs_solve_grad_host")
    res = dict(out)
    res["rc"] = rc
    if nw:
        res["shared_w_bar"] = wb
    return res


class GsFunction(torch.autograd.Function):
    """y_save = ODE ensemble solve at the save times; backward = the discrete adjoint
    on the recorded mesh (record in forward, replay sweep in backward). For the
    shared-weight problems (LV UDE, neural Robertson) the FP32 weight vector is an
    input too, and backward returns its gradient summed over the ensemble."""

    @staticmethod
    def forward(ctx, params, y0, shared_w, cfg):
        rec, ysv, status = forward_record(cfg["problem"], params, y0, cfg["t0"], cfg["t1"], cfg["save_t"],
                                          cfg["rtol"], cfg["atol"], shared_w=shared_w, **cfg.get("opts", {}))
        ctx.rec = rec
        if shared_w is None:
            ctx.save_for_backward(params, y0)
        else:
            ctx.save_for_backward(params, y0, shared_w)
        return ysv

    @staticmethod
    def backward(ctx, gy):
        saved = ctx.saved_tensors
        params, y0 = saved[0], saved[1]
        shared_w = saved[2] if len(saved) > 2 else None
        g = reverse(ctx.rec, params, y0, y_save_bar=gy.contiguous(), shared_w=shared_w)
        return g["params_bar"], g["y0_bar"], g.get("shared_w_bar"), None


def odeint_ensemble(problem, params, y0, t0, t1, save_t, rtol, atol, shared_w=None, **opts):
    """Differentiable ensemble solve: returns y_save (n, n_save, d). `shared_w`
    (FP32, the network weights of a shared-weight problem) may require grad.
    The record keeps every step's stage data when the method and memory allow
    (record_stages=True by default), so backward recomputes no stage."""
    opts.setdefault("record_stages", True)
    cfg = dict(problem=problem, t0=t0, t1=t1, save_t=save_t, rtol=rtol, atol=atol, opts=opts)
    return GsFunction.apply(params, y0, shared_w, cfg)
