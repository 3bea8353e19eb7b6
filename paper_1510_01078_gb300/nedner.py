"""Thin Python binding of the C-ABI in ``include/nedner.h`` (ctypes).

Argument marshalling only: every stage of the reconstruction runs in the CUDA
library ``_build/libnedner.so``.  Tensors are torch CUDA tensors (device
memory and streams come from PyTorch); there is no CPU fallback -- opening the
library fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnedner.so")

OK, EINVAL, ERANGE, ENOMEM, ECUDA, ENAN = range(6)
WINDOW_KB, WINDOW_GAUSS = 0, 1

_lib = None


class NednerError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _load().nedner_strerror(status).decode() if _lib is not None else str(status)
        super().__init__("%s: %s (status %d)" % (where, msg, status))


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class _Window(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("width", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("apply_weights", ctypes.c_int), ("band_mask", ctypes.c_int),
                ("max_workspace_bytes", ctypes.c_size_t), ("sensor_w", ctypes.c_void_p),
                ("precision", ctypes.c_int), ("ner_interp", ctypes.c_int)]


PRECISION_FP32_NUFFT, PRECISION_BF16_GEMM, PRECISION_FP16_GEMM = 0, 1, 2
# ned_mode names of the binding -> precision values of nedner_opts
NED_MODES = {"nufft": PRECISION_FP32_NUFFT, "tensor_bf16": PRECISION_BF16_GEMM, "tensor_fp16": PRECISION_FP16_GEMM}
# ner_interp names -> nedner_opts.ner_interp (the NER-NUFFT and the comparison methods of Sec. 5.1)
NER_MODES = {"nufft": 0, "linear2": 1, "linear1": 2, "direct": 3}


# symbol -> (restype, argtypes); mirrors include/nedner.h
_P = ctypes.c_void_p
SIGNATURES = {
    "nedner_plan": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(_Grid), _Window, ctypes.c_double, ctypes.POINTER(_Opts),
                                   _P, ctypes.POINTER(_P)]),
    "nedner_set_positions": (ctypes.c_int, [_P, _P]),
    "nedner_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner_grad_positions": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "nedner_ned_stage": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner_forward_profiled": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "nedner_adjoint_profiled": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "nedner_grad_positions_profiled": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "nedner_ned_stage_static": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner_workspace_bytes": (ctypes.c_size_t, [_P]),
    "nedner_plan_info": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "nedner_lowpass": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner_lowpass_bins": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "nedner_tenenbaum": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, _P]),
    "nedner_mip": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "nedner2d_plan": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double, _Window, ctypes.c_double, _P, _P,
                                     _P]),
    "nedner2d_set_positions": (ctypes.c_int, [_P, _P]),
    "nedner2d_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner2d_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner2d_destroy": (ctypes.c_int, [_P]),
    "nedner_work_split": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    "nedner_forward_host": (ctypes.c_int, [_P, _P, _P, _P]),
    "nedner_device_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "nedner_debug_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int]),
    "nedner_destroy": (ctypes.c_int, [_P]),
    "nedner_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def library():
    """The loaded ctypes library (raises if missing)."""
    return _load()


def _check(status: int, where: str):
    if status != OK:
        raise NednerError(status, where)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, shape: Sequence[int], name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor of shape %s (got %s %s)"
                         % (name, dtype, tuple(shape), t.dtype, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t, dtype, shape: Sequence[int], name: str):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s tensor of shape %s (got %s %s)"
                         % (name, dtype, tuple(shape), t.dtype, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A reconstruction plan (``nedner_plan``): geometry, tables, workspace.

    sensor_xy: (M, 2) positions in metres (array-like, float64 on the host).
    grid: (nx, ny, nz, dx, dy, dz).  window: ("kb"|"gauss", width).
    """

    def __init__(self, sensor_xy, Nt: int, dt: float, c: float, grid, window=("kb", 12), sigma: float = 2.0,
                 apply_weights: bool = True, band_mask: bool = False, sensor_w=None,
                 max_workspace_bytes: int = 0, stream=None, ned_mode: str = "nufft", ner_mode: str = "nufft"):
        lib = _load()
        self._xy = np.ascontiguousarray(np.asarray(sensor_xy, dtype=np.float64).reshape(-1, 2))
        self.M = int(self._xy.shape[0])
        self.Nt = int(Nt)
        self.nx, self.ny, self.nz = int(grid[0]), int(grid[1]), int(grid[2])
        self.grid = tuple(grid)
        g = _Grid(self.nx, self.ny, self.nz, float(grid[3]), float(grid[4]), float(grid[5]))
        kind = {"kb": WINDOW_KB, "gauss": WINDOW_GAUSS}[window[0]] if isinstance(window[0], str) else int(window[0])
        w = _Window(kind, int(window[1]))
        self._h = None if sensor_w is None else np.ascontiguousarray(np.asarray(sensor_w, dtype=np.float64))
        mode = NED_MODES[ned_mode]
        opts = _Opts(int(bool(apply_weights)), int(bool(band_mask)), int(max_workspace_bytes),
                     None if self._h is None else self._h.ctypes.data, mode, NER_MODES[ner_mode])
        handle = ctypes.c_void_p()
        st = lib.nedner_plan(self._xy.ctypes.data if self.M else None, self.M, self.Nt, float(dt), float(c),
                             ctypes.byref(g), w, float(sigma), ctypes.byref(opts), _stream_ptr(stream),
                             ctypes.byref(handle))
        _check(st, "nedner_plan")
        self._handle = handle

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            _load().nedner_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    STATUS_WAIT_TIMEOUT, STATUS_NONFINITE = 1, 2

    def device_status(self) -> int:
        """Device flags since the last call, read back and cleared (synchronous):
        STATUS_WAIT_TIMEOUT (a bounded wait of the tensor-core kernels ran out),
        STATUS_NONFINITE (an output kernel wrote a NaN or an infinity; the C call
        then returns NEDNER_ENAN, which is reported here as the flag)."""
        f = ctypes.c_int(0)
        st = _load().nedner_device_status(self._handle, ctypes.byref(f))
        if st != ENAN:
            _check(st, "nedner_device_status")
        return int(f.value)

    def debug_set_wait_limit(self, polls: int):
        """Test hook: the tensor-core kernels' pipeline waits give up after
        ``polls`` polls (0: at once); 1 << 26 restores the default."""
        _check(_load().nedner_debug_set_wait_limit(self._handle, int(polls)), "nedner_debug_set_wait_limit")

    @property
    def workspace_bytes(self) -> int:
        return int(_load().nedner_workspace_bytes(self._handle))

    def lowpass(self, g, out=None, stream=None):
        """Data low-pass of Sec. 8 (nedner_lowpass): each sensor's series cut at
        c / (2 x its nearest-neighbour distance); (M, Nt) float32 CUDA tensors."""
        import torch
        if out is None:
            out = torch.empty((self.M, self.Nt), dtype=torch.float32, device=g.device)
        st = _load().nedner_lowpass(self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
                                    _dev_ptr(out, torch.float32, (self.M, self.Nt), "out"), _stream_ptr(stream))
        _check(st, "nedner_lowpass")
        return out

    def lowpass_bins(self) -> np.ndarray:
        """Highest kept DFT bin of each sensor's low-pass (host)."""
        out = np.zeros(self.M, dtype=np.int32)
        if _load().nedner_lowpass_bins(self._handle, out.ctypes.data if self.M else None, self.M) != 0:
            raise NednerError(EINVAL, "nedner_lowpass_bins")
        return out

    PLAN_INFO_FIELDS = ("split", "tq", "tp_adj", "gsplit", "tp_g", "launches_forward", "launches_adjoint",
                        "launches_grad_positions")

    def info(self) -> dict:
        """The plan's passes over time and kernel launches per call (nedner_plan_info)."""
        out = (ctypes.c_int64 * len(self.PLAN_INFO_FIELDS))()
        n = _load().nedner_plan_info(self._handle, out, len(out))
        if n < 0:
            raise NednerError(EINVAL, "nedner_plan_info")
        return dict(zip(self.PLAN_INFO_FIELDS, [int(v) for v in out[:n]]))

    def set_positions(self, sensor_xy):
        xy = np.ascontiguousarray(np.asarray(sensor_xy, dtype=np.float64).reshape(self.M, 2))
        _check(_load().nedner_set_positions(self._handle, xy.ctypes.data if self.M else None),
               "nedner_set_positions")
        self._xy = xy

    # -- compute ----------------------------------------------------------
    def forward(self, g, out=None, stream=None):
        """p0 = R g.  g: (M, Nt) float32 CUDA tensor -> (nz, ny, nx)."""
        import torch
        if out is None:
            out = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float32, device=g.device)
        st = _load().nedner_forward(self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
                                    _dev_ptr(out, torch.float32, (self.nz, self.ny, self.nx), "p0"),
                                    _stream_ptr(stream))
        _check(st, "nedner_forward")
        return out

    def forward_host(self, g, out=None, stream=None):
        """p0 = R g with host tensors (``nedner_forward_host``): the uploads of g
        and downloads of p0 overlap the kernels.  g: (M, Nt) float32 CPU tensor
        (pinned for overlap) -> (nz, ny, nx) CPU tensor, valid once ``stream``
        has completed (the call returns before)."""
        import torch
        if out is None:
            out = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float32, pin_memory=True)
        st = _load().nedner_forward_host(self._handle, _host_ptr(g, torch.float32, (self.M, self.Nt), "g"),
                                         _host_ptr(out, torch.float32, (self.nz, self.ny, self.nx), "p0"),
                                         _stream_ptr(stream))
        _check(st, "nedner_forward_host")
        return out

    FORWARD_KERNELS = ("ned_spread", "ned_xfft", "ned_yfft", "ner_lines", "img_yifft", "img_xc2r")

    def forward_profiled(self, g, out, stream=None):
        """forward() that also returns each kernel's device time (ms), synchronously."""
        import torch
        ms = (ctypes.c_float * len(self.FORWARD_KERNELS))()
        st = _load().nedner_forward_profiled(self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
                                             _dev_ptr(out, torch.float32, (self.nz, self.ny, self.nx), "p0"),
                                             _stream_ptr(stream), ms)
        _check(st, "nedner_forward_profiled")
        return dict(zip(self.FORWARD_KERNELS, [float(v) for v in ms]))

    TRANSPOSED_KERNELS = ("img_xr2c_adj", "img_yfft_adj", "ner_lines_adj", "ned_yfft_adj", "ned_xfft_adj", "gather",
                          "entry_sum")

    def adjoint_profiled(self, p0, out, stream=None):
        """adjoint() that also returns each stage's device time (ms), synchronously."""
        import torch
        ms = (ctypes.c_float * len(self.TRANSPOSED_KERNELS))()
        st = _load().nedner_adjoint_profiled(self._handle,
                                             _dev_ptr(p0, torch.float32, (self.nz, self.ny, self.nx), "p0"),
                                             _dev_ptr(out, torch.float32, (self.M, self.Nt), "g"),
                                             _stream_ptr(stream), ms)
        _check(st, "nedner_adjoint_profiled")
        return dict(zip(self.TRANSPOSED_KERNELS, [float(v) for v in ms]))

    def grad_positions_profiled(self, g, dL_dp0, out, stream=None):
        """grad_positions() that also returns each stage's device time (ms), synchronously."""
        import torch
        ms = (ctypes.c_float * len(self.TRANSPOSED_KERNELS))()
        st = _load().nedner_grad_positions_profiled(
            self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
            _dev_ptr(dL_dp0, torch.float32, (self.nz, self.ny, self.nx), "dL_dp0"),
            _dev_ptr(out, torch.float32, (self.M, 2), "dL_dxy"), _stream_ptr(stream), ms)
        _check(st, "nedner_grad_positions_profiled")
        return dict(zip(self.TRANSPOSED_KERNELS, [float(v) for v in ms]))

    def adjoint(self, p0, out=None, stream=None):
        """g = R^T p0.  p0: (nz, ny, nx) -> (M, Nt)."""
        import torch
        if out is None:
            out = torch.empty((self.M, self.Nt), dtype=torch.float32, device=p0.device)
        st = _load().nedner_adjoint(self._handle, _dev_ptr(p0, torch.float32, (self.nz, self.ny, self.nx), "p0"),
                                    _dev_ptr(out, torch.float32, (self.M, self.Nt), "g"), _stream_ptr(stream))
        _check(st, "nedner_adjoint")
        return out

    def grad_positions(self, g, dL_dp0, out=None, stream=None):
        """dL/d(x_m, y_m): (M, 2)."""
        import torch
        if out is None:
            out = torch.empty((self.M, 2), dtype=torch.float32, device=g.device)
        st = _load().nedner_grad_positions(
            self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
            _dev_ptr(dL_dp0, torch.float32, (self.nz, self.ny, self.nx), "dL_dp0"),
            _dev_ptr(out, torch.float32, (self.M, 2), "dL_dxy"), _stream_ptr(stream))
        _check(st, "nedner_grad_positions")
        return out

    def ned_stage(self, g, stream=None):
        """Stage (a) output: complex64 (nx/2+1, ny+1, Nt), jx = 0..nx/2, jy = -ny/2..ny/2."""
        import torch
        out = torch.empty((self.nx // 2 + 1, self.ny + 1, self.Nt), dtype=torch.complex64, device=g.device)
        st = _load().nedner_ned_stage(self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
        _check(st, "nedner_ned_stage")
        return out


def ned_stage_static(plan: Plan, g, out=None, stream=None):
    """``nedner_ned_stage_static``: the NED stage of ``plan`` with its
    intermediate in the library's fixed 16 MiB device buffer instead of the
    plan's workspace; for callers that cannot allocate device memory when they
    run it.  The output ``out`` (complex64, (nx/2+1, ny+1, Nt)) is the caller's
    and must be passed in if no allocation may happen here.  Calls that overlap
    on the GPU race (one shared buffer)."""
    import torch
    if out is None:
        out = torch.empty((plan.nx // 2 + 1, plan.ny + 1, plan.Nt), dtype=torch.complex64, device=g.device)
    st = _load().nedner_ned_stage_static(plan._handle, _dev_ptr(g, torch.float32, (plan.M, plan.Nt), "g"),
                                         _dev_ptr(out, torch.complex64, (plan.nx // 2 + 1, plan.ny + 1, plan.Nt),
                                                  "Ghat"),
                                         _stream_ptr(stream))
    _check(st, "nedner_ned_stage_static")
    return out


def _autograd():
    import torch

    class ReconFunction(torch.autograd.Function):
        """p0 = R(x) g as a differentiable op: backward gives dL/dg = R^T dL/dp0
        (nedner_adjoint) and dL/d(sensor_xy) (nedner_grad_positions, areas
        held fixed).  The plan's sensor positions must equal sensor_xy."""

        @staticmethod
        def forward(ctx, g, sensor_xy, plan):
            ctx.plan = plan
            ctx.xy_like = (sensor_xy.device, sensor_xy.dtype)
            ctx.save_for_backward(g)
            return plan.forward(g.contiguous())

        @staticmethod
        def backward(ctx, dL_dp0):
            (g,) = ctx.saved_tensors
            plan = ctx.plan
            dL_dp0 = dL_dp0.contiguous()
            dg = plan.adjoint(dL_dp0) if ctx.needs_input_grad[0] else None
            dxy = None
            if ctx.needs_input_grad[1]:
                dxy = plan.grad_positions(g.contiguous(), dL_dp0).to(device=ctx.xy_like[0],
                                                                      dtype=ctx.xy_like[1])
            return dg, dxy, None

    return ReconFunction


_RECON = None
_MODEL = None


def _model_autograd():
    import torch

    class ModelFunction(torch.autograd.Function):
        """g = R^T p0 (nedner_adjoint) as a differentiable op; its backward is
        nedner_forward for p0 and, for the sensor positions,
        d/dx <dL/dg, R(x)^T p0> = d/dx <R(x) dL/dg, p0>, i.e.
        nedner_grad_positions with (g, dL/dp0) = (dL/dg, p0).  With an
        unweighted plan this is the physical forward model A (data from an
        initial pressure), A^T being the unweighted R."""

        @staticmethod
        def forward(ctx, p0, sensor_xy, plan):
            ctx.plan = plan
            ctx.xy_like = (sensor_xy.device, sensor_xy.dtype)
            ctx.save_for_backward(p0)
            return plan.adjoint(p0.contiguous())

        @staticmethod
        def backward(ctx, dL_dg):
            (p0,) = ctx.saved_tensors
            dL_dg = dL_dg.contiguous()
            dp0 = ctx.plan.forward(dL_dg) if ctx.needs_input_grad[0] else None
            dxy = None
            if ctx.needs_input_grad[1]:
                dxy = ctx.plan.grad_positions(dL_dg, p0.contiguous()).to(device=ctx.xy_like[0],
                                                                          dtype=ctx.xy_like[1])
            return dp0, dxy, None

    return ModelFunction


def _move(plan: Plan, sensor_xy):
    """The positions tensor to differentiate against; moves the plan there
    first (nedner_set_positions) when they differ from the plan's."""
    import torch
    if sensor_xy is None:
        return torch.as_tensor(plan._xy)
    xy = sensor_xy.detach().to("cpu", torch.float64).numpy()
    if not np.array_equal(xy, plan._xy):
        plan.set_positions(xy)
    return sensor_xy


def model(plan: Plan, p0, sensor_xy=None):
    """Differentiable g = R^T p0 (see ``ModelFunction``); ``sensor_xy`` as in
    ``reconstruct``."""
    global _MODEL
    if _MODEL is None:
        _MODEL = _model_autograd()
    return _MODEL.apply(p0, _move(plan, sensor_xy), plan)


def reconstruct(plan: Plan, g, sensor_xy=None):
    """Differentiable reconstruction.  ``sensor_xy``: optional (M, 2) float64
    tensor of positions (metres); if given and different from the plan's, the
    plan is moved there first (nedner_set_positions), and gradients with
    respect to it are available through autograd."""
    global _RECON
    if _RECON is None:
        _RECON = _autograd()
    return _RECON.apply(g, _move(plan, sensor_xy), plan)


WORK_SPLIT_FIELDS = ("c1", "c2f", "c4", "c5", "groups1", "threads1", "per1", "tpl1", "ca", "per_adj", "tpl_adj",
                     "threads_adj", "lpc", "threads3", "smem1", "smem2f", "smem3", "smem4", "smem5", "smem_adj",
                     "smem_grad", "split1", "tq", "wpc_s", "nbx", "thx", "perx", "smem_s", "smem_x", "smem3a",
                     "icap3a")


class Plan2D:
    """The two-dimensional variant (``nedner2d_plan``, Sec. 7): sensors at x_m
    on a line, an output image (nz, nx).  sensor_x: (M,) metres; grid: (nx, nz,
    dx, dz); sensor_w: lengths h_m (default X/M)."""

    def __init__(self, sensor_x, Nt: int, dt: float, c: float, grid, window=("kb", 12), sigma: float = 2.0,
                 apply_weights: bool = True, sensor_w=None, stream=None):
        lib = _load()
        self._x = np.ascontiguousarray(np.asarray(sensor_x, dtype=np.float64).reshape(-1))
        self.M = int(self._x.shape[0])
        self.Nt = int(Nt)
        self.nx, self.nz = int(grid[0]), int(grid[1])
        self.grid = tuple(grid)
        kind = {"kb": WINDOW_KB, "gauss": WINDOW_GAUSS}[window[0]] if isinstance(window[0], str) else int(window[0])
        self._h = None if sensor_w is None else np.ascontiguousarray(np.asarray(sensor_w, dtype=np.float64))
        opts = _Opts(int(bool(apply_weights)), 0, 0, None if self._h is None else self._h.ctypes.data,
                     PRECISION_FP32_NUFFT, 0)
        handle = ctypes.c_void_p()
        st = lib.nedner2d_plan(self._x.ctypes.data if self.M else None, self.M, self.Nt, float(dt), float(c),
                               self.nx, self.nz, float(grid[2]), float(grid[3]), _Window(kind, int(window[1])),
                               float(sigma), ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(handle))
        _check(st, "nedner2d_plan")
        self._handle = handle

    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            _load().nedner2d_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_positions(self, sensor_x):
        x = np.ascontiguousarray(np.asarray(sensor_x, dtype=np.float64).reshape(self.M))
        _check(_load().nedner2d_set_positions(self._handle, x.ctypes.data if self.M else None),
               "nedner2d_set_positions")
        self._x = x

    def forward(self, g, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.nz, self.nx), dtype=torch.float32, device=g.device)
        st = _load().nedner2d_forward(self._handle, _dev_ptr(g, torch.float32, (self.M, self.Nt), "g"),
                                      _dev_ptr(out, torch.float32, (self.nz, self.nx), "p2"), _stream_ptr(stream))
        _check(st, "nedner2d_forward")
        return out

    def adjoint(self, p2, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.M, self.Nt), dtype=torch.float32, device=p2.device)
        st = _load().nedner2d_adjoint(self._handle, _dev_ptr(p2, torch.float32, (self.nz, self.nx), "p2"),
                                      _dev_ptr(out, torch.float32, (self.M, self.Nt), "g"), _stream_ptr(stream))
        _check(st, "nedner2d_adjoint")
        return out


def tenenbaum(U, stream=None):
    """Tenenbaum sharpness (Appendix B) of an image (ny, nx) or a batch (B, ny,
    nx) of float32 CUDA images; returns a float64 CUDA tensor of B values
    (a 0-d tensor for one image)."""
    import torch
    one = U.dim() == 2
    U3 = U.unsqueeze(0) if one else U
    if U3.dim() != 3:
        raise ValueError("U must be (ny, nx) or (B, ny, nx)")
    B, ny, nx = (int(v) for v in U3.shape)
    F = torch.empty(B, dtype=torch.float64, device=U.device)
    st = _load().nedner_tenenbaum(_dev_ptr(U3, torch.float32, (B, ny, nx), "U"), B, ny, nx,
                                  _dev_ptr(F, torch.float64, (B,), "F"), _stream_ptr(stream))
    _check(st, "nedner_tenenbaum")
    return F[0] if one else F


def mip(vol, axis: int, stream=None):
    """Maximum intensity projection of a (nz, ny, nx) float32 CUDA volume along
    axis 0, 1 or 2 (nedner_mip)."""
    import torch
    nz, ny, nx = (int(v) for v in vol.shape)
    shape = {0: (ny, nx), 1: (nz, nx), 2: (nz, ny)}[axis]
    out = torch.empty(shape, dtype=torch.float32, device=vol.device)
    st = _load().nedner_mip(_dev_ptr(vol, torch.float32, (nz, ny, nx), "vol"), nz, ny, nx, axis,
                            _dev_ptr(out, torch.float32, shape, "out"), _stream_ptr(stream))
    _check(st, "nedner_mip")
    return out


def work_split(nx: int, ny: int, nz: int, Nt: int, w: int = 12) -> dict:
    """The per-stage work split a plan of this geometry uses (host only, no device)."""
    out = (ctypes.c_int64 * len(WORK_SPLIT_FIELDS))()
    n = _load().nedner_work_split(nx, ny, nz, Nt, w, out, len(out))
    if n < 0:
        raise NednerError(EINVAL, "nedner_work_split (%d x %d x %d, Nt %d, w %d)" % (nx, ny, nz, Nt, w))
    return dict(zip(WORK_SPLIT_FIELDS, [int(v) for v in out[:n]]))


def plan_from_config(cfg, **kw) -> Plan:
    """Plan for a workload dict as produced by ``inputs.make_config``/``small_case``."""
    return Plan(cfg["sensor_xy"], cfg["Nt"], cfg["dt"], cfg["c"],
                (cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"]),
                sensor_w=kw.pop("sensor_w", cfg.get("h")), **kw)


__all__ = ["Plan", "Plan2D", "plan_from_config", "work_split", "tenenbaum", "mip", "WORK_SPLIT_FIELDS", "ned_stage_static", "reconstruct", "model", "NednerError", "library", "LIB_PATH", "SIGNATURES",
           "WINDOW_KB", "WINDOW_GAUSS"]
