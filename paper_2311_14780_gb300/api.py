"""Python front end of the C ABI: argument marshalling only.

Every computation happens in the CUDA library; this module checks tensor dtypes,
shapes and devices, passes raw device pointers and the current torch stream, and turns
return codes into exceptions.  Names follow the C entry points (ptycho_forward,
ptycho_loss, ptycho_adjoint, ptycho_step).
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native

LOSS_CODES = {"amplitude": 0, "poisson": 1, "poisson_gaussian": 2}
# pipeline variants (PTYCHO_FLAG_* in include/ptycho.h, where each is described)
FLAG_RECOMPUTE_COLUMNS = 1
FLAG_OBJ_GRAD_ATOMIC = 2
FLAG_KEEP_PSI = 4
FLAG_NO_TMA = 8
FLAG_TMA = 16
FLAG_UNFUSED_ROW_ADJ = 32
FLAG_STAGED_COLUMNS = 64
FLAG_NARROW_COLUMNS = 128
FLAG_FUSED_ROW_FWD = 256
FLAG_NO_PDL = 512
FLAG_RESIDENT_FRAMES = 1024
FLAG_ROW_ADJ_PROBE_L2 = 2048
FLAG_ROW_ADJ_PROBE_SMEM = 4096
FLAG_UNFUSED_ROW_FWD = 8192
FLAG_ROWS_16_THREADS = 16384
FLAG_FWD_ROWS_WARP = 32768
FLAG_COLS_ONE_BLOCK = 65536
FLAG_FUSED_ROW_ADJ = 131072


class PtychoError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _native.lib().ptycho_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def _check(code: int, where: str):
    if code != 0:
        raise PtychoError(code, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def pack_objects(objs: Sequence, device="cuda") -> torch.Tensor:
    """Pack per-wavelength objects into the library's flat complex64 layout."""
    flat = [torch.as_tensor(np.asarray(o), dtype=torch.complex64).reshape(-1) for o in objs]
    return torch.cat(flat).to(device)


def unpack_objects(flat: torch.Tensor, shapes) -> list:
    out, off = [], 0
    for (h, w) in shapes:
        out.append(flat[off:off + h * w].reshape(h, w))
        off += h * w
    return out


def geom_struct(F: int, L: int, M: int, J: int, obj_shapes, pos, *, loss: str = "amplitude", eps: float = 0.0,
                remap: bool = False, z: float = 88e-3, det_pixel: float = 15e-6,
                tilt_rad: float = 1.2217304763960306, lambdas=None, scratch_bytes: int = 0, overlap: int = 0,
                flags: int = 0, col_groups: int = 0, read_noise_var: float = 0.0, zoom=None):
    """A ``ptycho_geom_t`` and the host arrays it points to (keep both alive while used)."""
    keep = {
        "h": np.ascontiguousarray([int(s_[0]) for s_ in obj_shapes], dtype=np.int32),
        "w": np.ascontiguousarray([int(s_[1]) for s_ in obj_shapes], dtype=np.int32),
        "pos": np.ascontiguousarray(np.asarray(pos, dtype=np.int32).reshape(L, J, 2)),
        "lam": None if lambdas is None else np.ascontiguousarray(lambdas, dtype=np.float64),
        "zoom": None if zoom is None else np.ascontiguousarray(zoom, dtype=np.float64).reshape(L),
    }
    g = _native.Geom()
    g.L, g.M, g.F, g.J = int(L), int(M), int(F), int(J)
    g.obj_h = keep["h"].ctypes.data_as(_native.c_int32_p)
    g.obj_w = keep["w"].ctypes.data_as(_native.c_int32_p)
    g.pos = keep["pos"].ctypes.data_as(_native.c_int32_p)
    g.lam = None if keep["lam"] is None else keep["lam"].ctypes.data_as(_native.c_double_p)
    g.z, g.det_pixel, g.tilt_rad = float(z), float(det_pixel), float(tilt_rad)
    g.remap = 1 if remap else 0
    g.loss = LOSS_CODES[loss]
    g.eps = float(eps)
    g.scratch_bytes = int(scratch_bytes)
    g.overlap = int(overlap)
    g.flags = int(flags)
    g.col_groups = int(col_groups)
    g.read_noise_var = float(read_noise_var)
    g.zoom = None if keep["zoom"] is None else keep["zoom"].ctypes.data_as(_native.c_double_p)
    return g, keep


class Plan:
    """A validated problem geometry with its device workspace (``ptycho_plan_t``)."""

    def __init__(self, F: int, L: int, M: int, J: int, obj_shapes, pos, *, loss: str = "amplitude",
                 eps: float = 0.0, remap: bool = False, z: float = 88e-3, det_pixel: float = 15e-6,
                 tilt_rad: float = 1.2217304763960306, lambdas=None, scratch_bytes: int = 0, overlap: int = 0,
                 flags: int = 0, col_groups: int = 0, read_noise_var: float = 0.0, zoom=None):
        self.F, self.L, self.M, self.J = int(F), int(L), int(M), int(J)
        self.remap = bool(remap)
        self.obj_shapes = [(int(h), int(w)) for (h, w) in obj_shapes]
        self.loss_kind = loss
        g, self._keep = geom_struct(F, L, M, J, obj_shapes, pos, loss=loss, eps=eps, remap=remap, z=z,
                                    det_pixel=det_pixel, tilt_rad=tilt_rad, lambdas=lambdas,
                                    scratch_bytes=scratch_bytes, overlap=overlap, flags=flags,
                                    col_groups=col_groups, read_noise_var=read_noise_var, zoom=zoom)
        self._geom = g
        h = ctypes.c_void_p()
        _check(_native.lib().ptycho_plan_create(ctypes.byref(g), ctypes.byref(h)), "ptycho_plan_create")
        self._h_plan = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    # -- properties ----------------------------------------------------------------
    @property
    def handle(self):
        return self._h_plan

    @property
    def numel_O(self) -> int:
        return int(_native.lib().ptycho_plan_numel_O(self._h_plan))

    @property
    def numel_P(self) -> int:
        return int(_native.lib().ptycho_plan_numel_P(self._h_plan))

    @property
    def workspace_bytes(self) -> int:
        return int(_native.lib().ptycho_plan_workspace_bytes(self._h_plan))

    @property
    def last_launches(self) -> int:
        return int(_native.lib().ptycho_plan_last_launches(self._h_plan))

    def profile(self, enable: bool = True):
        """Start (or stop) per-kernel event timing of this plan's launches."""
        _check(_native.lib().ptycho_plan_profile(self._h_plan, 1 if enable else 0), "ptycho_plan_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since profiling started or was last read."""
        ms = (ctypes.c_double * _native.NUM_KERNELS)()
        n = (ctypes.c_int64 * _native.NUM_KERNELS)()
        _check(_native.lib().ptycho_plan_profile_read(self._h_plan, ms, n), "ptycho_plan_profile_read")
        return {_native.lib().ptycho_kernel_name(k).decode(): (float(ms[k]), int(n[k]))
                for k in range(_native.NUM_KERNELS)}

    def regularise(self, O, mu_l1: float, mu_tv: float, eta: float, gO=None, loss_out=None, stream=None):
        """ptycho_regularise: adds the object regulariser's gradient to ``gO`` (zeros if None)
        and its value to ``loss_out`` (a float64 device scalar, zeros if None); returns both."""
        Or = self._c64(O, self.numel_O, "O")
        if gO is None:
            gO = torch.zeros_like(O)
        gr = self._c64(gO, self.numel_O, "gO")
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float64, device=O.device)
        rc = _native.lib().ptycho_regularise(self._h_plan, _ptr(Or), float(mu_l1), float(mu_tv), float(eta),
                                             _ptr(gr), _ptr(loss_out), _stream_handle(stream))
        _check(rc, "ptycho_regularise")
        return loss_out, gO

    def status(self) -> int:
        """Device status flags since the last query (synchronises; bit 0 = bad batch index,
        bit 1 = a column pass's bulk copy timed out)."""
        v = ctypes.c_int32(0)
        _check(_native.lib().ptycho_plan_status(self._h_plan, ctypes.byref(v)), "ptycho_plan_status")
        return int(v.value)

    def close(self):
        if getattr(self, "_h_plan", None) is not None and self._h_plan.value:
            _native.lib().ptycho_plan_destroy(self._h_plan)
            self._h_plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- argument checks -----------------------------------------------------------
    def _c64(self, t: torch.Tensor, n: int, name: str):
        if t.dtype != torch.complex64 or not t.is_contiguous() or t.device != self.device or t.numel() != n:
            raise ValueError(f"{name}: need a contiguous complex64 tensor of {n} elements on {self.device}")
        return torch.view_as_real(t)

    def _f32(self, t, n: int, name: str):
        if t is None:
            return None
        if t.dtype != torch.float32 or not t.is_contiguous() or t.device != self.device or t.numel() != n:
            raise ValueError(f"{name}: need a contiguous float32 tensor of {n} elements on {self.device}")
        return t

    def _mask(self, mask):
        FF = self.F * self.F
        if mask is None:
            return None, 0
        if mask.dtype != torch.uint8 or not mask.is_contiguous() or mask.device != self.device:
            raise ValueError("mask: need a contiguous uint8 tensor on the plan's device")
        if mask.numel() == FF:
            return mask, 0
        if mask.numel() == self.J * FF:
            return mask, 1
        raise ValueError("mask: need F*F or J*F*F elements")

    def _batch(self, batch):
        if batch is None:
            return None, 0
        if batch.dtype != torch.int32 or not batch.is_contiguous() or batch.device != self.device:
            raise ValueError("batch: need a contiguous int32 tensor on the plan's device")
        return batch, int(batch.numel())

    # -- compute calls ---------------------------------------------------------------
    def forward(self, O, P, sigma=None, bg=None, out=None, stream=None) -> torch.Tensor:
        """ptycho_forward: predicted camera-grid patterns [J, F, F] float32."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        if out is None:
            out = torch.empty((self.J, self.F, self.F), dtype=torch.float32, device=self.device)
        self._f32(out, self.J * FF, "out")
        rc = _native.lib().ptycho_forward(self._h_plan, _ptr(Or), _ptr(Pr), _ptr(self._f32(sigma, self.J, "sigma")),
                                          _ptr(self._f32(bg, FF, "bg")), _ptr(out), _stream_handle(stream))
        _check(rc, "ptycho_forward")
        return out

    def loss(self, O, P, Imeas, sigma=None, bg=None, mask=None, batch=None, out=None, stream=None):
        """ptycho_loss: FP64 loss (a 1-element device tensor)."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        m, mpf = self._mask(mask)
        bt, nb = self._batch(batch)
        if out is None:
            out = torch.zeros(1, dtype=torch.float64, device=self.device)
        rc = _native.lib().ptycho_loss(self._h_plan, _ptr(Or), _ptr(Pr), _ptr(self._f32(sigma, self.J, "sigma")),
                                       _ptr(self._f32(bg, FF, "bg")), _ptr(self._f32(Imeas, self.J * FF, "Imeas")),
                                       _ptr(m), mpf, _ptr(bt), nb, _ptr(out), _stream_handle(stream))
        _check(rc, "ptycho_loss")
        return out

    def adjoint(self, O, P, Imeas, sigma=None, bg=None, mask=None, batch=None, gO=None, gP=None, loss_out=None,
                stream=None):
        """ptycho_adjoint: (loss, grad O, grad P); gradients use dL/dRe + i dL/dIm."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        m, mpf = self._mask(mask)
        bt, nb = self._batch(batch)
        if gO is None:
            gO = torch.empty(self.numel_O, dtype=torch.complex64, device=self.device)
        if gP is None:
            gP = torch.empty(P.shape, dtype=torch.complex64, device=self.device)
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float64, device=self.device)
        gOr, gPr = self._c64(gO, self.numel_O, "gO"), self._c64(gP, self.numel_P, "gP")
        rc = _native.lib().ptycho_adjoint(self._h_plan, _ptr(Or), _ptr(Pr), _ptr(self._f32(sigma, self.J, "sigma")),
                                          _ptr(self._f32(bg, FF, "bg")),
                                          _ptr(self._f32(Imeas, self.J * FF, "Imeas")), _ptr(m), mpf, _ptr(bt), nb,
                                          _ptr(gOr), _ptr(gPr), _ptr(loss_out), _stream_handle(stream))
        _check(rc, "ptycho_adjoint")
        return loss_out, gO, gP

    def set_offsets(self, delta):
        """ptycho_plan_set_offsets: register fractional scan offsets (a contiguous float32
        device tensor of L*J*2 elements, [L, J, 2] rows then columns) or clear them (None).
        The plan keeps a reference to the tensor while it is registered."""
        if delta is not None:
            self._f32(delta, self.L * self.J * 2, "delta")
        _check(_native.lib().ptycho_plan_set_offsets(self._h_plan, _ptr(delta)), "ptycho_plan_set_offsets")
        self._delta = delta

    @property
    def offsets(self):
        return getattr(self, "_delta", None)

    def set_distance(self, z: float):
        """ptycho_plan_set_distance: rebuild the tilted-plane remap for propagation distance z."""
        _check(_native.lib().ptycho_plan_set_distance(self._h_plan, float(z)), "ptycho_plan_set_distance")

    def adjoint_ex(self, O, P, Imeas, sigma=None, bg=None, mask=None, batch=None, stream=None, want_z=None):
        """ptycho_adjoint_ex: (loss, grad O, grad P, grad sigma [J], grad bg [F, F],
        grad delta [L, J, 2] or None when no offsets are registered, dL/dz [1] FP64 or None
        without the remap; want_z=False skips it)."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        m, mpf = self._mask(mask)
        bt, nb = self._batch(batch)
        gO = torch.empty(self.numel_O, dtype=torch.complex64, device=self.device)
        gP = torch.empty(P.shape, dtype=torch.complex64, device=self.device)
        gs = torch.empty(self.J, dtype=torch.float32, device=self.device)
        gb = torch.empty(self.F, self.F, dtype=torch.float32, device=self.device)
        gd = torch.empty(self.L, self.J, 2, dtype=torch.float32, device=self.device) if self.offsets is not None \
            else None
        want_z = self.remap if want_z is None else (want_z and self.remap)
        gz = torch.zeros(1, dtype=torch.float64, device=self.device) if want_z else None
        loss_out = torch.zeros(1, dtype=torch.float64, device=self.device)
        rc = _native.lib().ptycho_adjoint_ex(self._h_plan, _ptr(Or), _ptr(Pr), _ptr(self._f32(sigma, self.J, "sigma")),
                                             _ptr(self._f32(bg, FF, "bg")),
                                             _ptr(self._f32(Imeas, self.J * FF, "Imeas")), _ptr(m), mpf, _ptr(bt), nb,
                                             _ptr(gO), _ptr(gP), _ptr(gs), _ptr(gb), _ptr(gd), _ptr(gz), _ptr(loss_out),
                                             _stream_handle(stream))
        _check(rc, "ptycho_adjoint_ex")
        return loss_out, gO, gP, gs, gb, gd, gz

    def step(self, state: "AdamState", O, P, Imeas, sigma=None, bg=None, mask=None, batch=None, loss_out=None,
             stream=None):
        """ptycho_step: adjoint + fused Adam on O and P in place (and on sigma / bg when the state
        has lr_sigma / lr_bg > 0); returns the FP64 loss tensor."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        m, mpf = self._mask(mask)
        bt, nb = self._batch(batch)
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float64, device=self.device)
        st = state.c_struct()
        rc = _native.lib().ptycho_step(self._h_plan, ctypes.byref(st), _ptr(Or), _ptr(Pr),
                                       _ptr(self._f32(sigma, self.J, "sigma")), _ptr(self._f32(bg, FF, "bg")),
                                       _ptr(self._f32(Imeas, self.J * FF, "Imeas")), _ptr(m), mpf, _ptr(bt), nb,
                                       _ptr(loss_out), _stream_handle(stream))
        _check(rc, "ptycho_step")
        state.t = int(st.t)
        return loss_out

    def step_host(self, state: "AdamState", O, P, Imeas_host, Imeas_dev, loss_dev, loss_host, sigma=None, bg=None,
                  mask=None, batch=None, stream=None):
        """ptycho_step_host: ``step`` with the measured patterns in host memory (``Imeas_host``,
        a contiguous float32 CPU tensor, pinned for an asynchronous copy) copied on the stream
        into ``Imeas_dev`` (device, float32), and the FP64 loss copied from ``loss_dev`` (device)
        into ``loss_host`` (a float64 CPU tensor, pinned for an asynchronous copy)."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        if Imeas_host.dtype != torch.float32 or Imeas_host.is_cuda or not Imeas_host.is_contiguous() or \
                Imeas_host.numel() != self.J * FF:
            raise ValueError(f"Imeas_host: need a contiguous float32 host tensor of {self.J * FF} elements")
        if loss_host.dtype != torch.float64 or loss_host.is_cuda or loss_host.numel() < 1:
            raise ValueError("loss_host: need a float64 host tensor")
        if loss_dev.dtype != torch.float64 or loss_dev.device != self.device:
            raise ValueError("loss_dev: need a float64 tensor on the plan's device")
        m, mpf = self._mask(mask)
        bt, nb = self._batch(batch)
        st = state.c_struct()
        rc = _native.lib().ptycho_step_host(self._h_plan, ctypes.byref(st), _ptr(Or), _ptr(Pr),
                                            _ptr(self._f32(sigma, self.J, "sigma")), _ptr(self._f32(bg, FF, "bg")),
                                            _ptr(Imeas_host), _ptr(self._f32(Imeas_dev, self.J * FF, "Imeas_dev")),
                                            _ptr(m), mpf, _ptr(bt), nb, _ptr(loss_dev), _ptr(loss_host),
                                            _stream_handle(stream))
        _check(rc, "ptycho_step_host")
        state.t = int(st.t)
        return loss_host

    def plain_step(self, state: "AdamState", O, P, Imeas, sigma=None, bg=None, mask=None, loss_out=None,
                   stream=None):
        """ptycho_plain_step: the unfused baseline of ``step`` over all positions."""
        FF = self.F * self.F
        Or, Pr = self._c64(O, self.numel_O, "O"), self._c64(P, self.numel_P, "P")
        m, mpf = self._mask(mask)
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float64, device=self.device)
        st = state.c_struct()
        rc = _native.lib().ptycho_plain_step(self._h_plan, ctypes.byref(st), _ptr(Or), _ptr(Pr),
                                             _ptr(self._f32(sigma, self.J, "sigma")), _ptr(self._f32(bg, FF, "bg")),
                                             _ptr(self._f32(Imeas, self.J * FF, "Imeas")), _ptr(m), mpf,
                                             _ptr(loss_out), _stream_handle(stream))
        _check(rc, "ptycho_plain_step")
        state.t = int(st.t)
        return loss_out


class AdamState:
    """Adam moments for O and P (device tensors, 2 floats per complex element)."""

    def __init__(self, plan: Plan, lr_O: float, lr_P: float, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, device_counter: bool = False, lr_sigma: float = 0.0, lr_bg: float = 0.0,
                 lr_delta: float = 0.0, with_z_gradient: bool = False, reg_l1: float = 0.0, reg_tv: float = 0.0,
                 reg_eta: float = 1e-3):
        dev = plan.device
        # optional object regularisation added by Plan.step (see Plan.regularise)
        self.reg_l1, self.reg_tv, self.reg_eta = reg_l1, reg_tv, reg_eta
        # optional: sigma [J] and the background [F, F] are optimised too (updated in place by
        # Plan.step, which then needs them as float32 device tensors)
        self.lr_sigma, self.lr_bg = lr_sigma, lr_bg
        self.m_sigma = torch.zeros(plan.J, dtype=torch.float32, device=dev) if lr_sigma > 0 else None
        self.v_sigma = torch.zeros_like(self.m_sigma) if lr_sigma > 0 else None
        self.m_bg = torch.zeros(plan.F * plan.F, dtype=torch.float32, device=dev) if lr_bg > 0 else None
        self.v_bg = torch.zeros_like(self.m_bg) if lr_bg > 0 else None
        # optional: the registered fractional scan offsets ([L, J, 2]) are optimised too
        self.lr_delta = lr_delta
        self.m_delta = torch.zeros(plan.L * plan.J * 2, dtype=torch.float32, device=dev) if lr_delta > 0 else None
        self.v_delta = torch.zeros_like(self.m_delta) if lr_delta > 0 else None
        # optional: each step also writes dL/dz here (FP64, device); z is updated by the caller
        self.g_z = torch.zeros(1, dtype=torch.float64, device=dev) if with_z_gradient else None
        # with a device step counter a captured CUDA graph of Plan.step can be replayed
        self.t_dev = torch.zeros(1, dtype=torch.int32, device=dev) if device_counter else None
        self.lr_O, self.lr_P, self.beta1, self.beta2, self.eps = lr_O, lr_P, beta1, beta2, eps
        self.t = 0
        self.mO = torch.zeros(2 * plan.numel_O, dtype=torch.float32, device=dev)
        self.vO = torch.zeros_like(self.mO)
        self.mP = torch.zeros(2 * plan.numel_P, dtype=torch.float32, device=dev)
        self.vP = torch.zeros_like(self.mP)

    def c_struct(self) -> _native.Adam:
        s = _native.Adam()
        s.lr_O, s.lr_P, s.beta1, s.beta2, s.eps, s.t = self.lr_O, self.lr_P, self.beta1, self.beta2, self.eps, self.t
        s.mO, s.vO = self.mO.data_ptr(), self.vO.data_ptr()
        s.mP, s.vP = self.mP.data_ptr(), self.vP.data_ptr()
        s.t_dev = None if self.t_dev is None else self.t_dev.data_ptr()
        s.lr_sigma, s.lr_bg, s.lr_delta = self.lr_sigma, self.lr_bg, self.lr_delta
        s.reg_l1, s.reg_tv, s.reg_eta = self.reg_l1, self.reg_tv, self.reg_eta
        for name in ("m_sigma", "v_sigma", "m_bg", "v_bg", "m_delta", "v_delta", "g_z"):
            t = getattr(self, name)
            setattr(s, name, None if t is None else t.data_ptr())
        return s


def tilt_correct(I_cam: torch.Tensor, z: float, det_pixel: float, tilt_rad: float, lo: float = -math.inf,
                 hi: float = math.inf, with_mask: bool = True, stream: Optional[torch.cuda.Stream] = None):
    """Data-side tilt correction (``ptycho_tilt_correct``): camera patterns [J][F][F] (or one
    [F][F]) float32 on the GPU -> (model-grid patterns, uint8 mask or None), ready for a plan
    built with ``remap=False`` and the mask passed per frame."""
    I_cam, out, mask = _tilt_io(I_cam, with_mask)
    rc = _native.lib().ptycho_tilt_correct(int(I_cam.shape[1]), int(I_cam.shape[0]), float(z), float(det_pixel),
                                           float(tilt_rad), _ptr(I_cam), float(lo), float(hi), _ptr(out),
                                           _ptr(mask), _stream_handle(stream))
    _check(rc, "ptycho_tilt_correct")
    return out, mask


def tilt_table(F: int, z: float, det_pixel: float, tilt_rad: float, device="cuda",
               stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """Camera positions of the model pixels for one geometry (``ptycho_tilt_table``): a device
    byte tensor to pass to :func:`tilt_apply` for every stack of patterns of that geometry."""
    n = int(_native.lib().ptycho_tilt_table_bytes(int(F)))
    if n < 0:
        raise ValueError("F must be in 2..8192")
    table = torch.empty(n, dtype=torch.uint8, device=device)
    _check(_native.lib().ptycho_tilt_table(int(F), float(z), float(det_pixel), float(tilt_rad), _ptr(table),
                                           _stream_handle(stream)), "ptycho_tilt_table")
    return table


def _tilt_io(I_cam: torch.Tensor, with_mask: bool):
    if I_cam.dim() == 2:
        I_cam = I_cam.unsqueeze(0)
    if I_cam.dim() != 3 or I_cam.shape[1] != I_cam.shape[2]:
        raise ValueError("I_cam must be [J][F][F]")
    if not I_cam.is_cuda or I_cam.dtype != torch.float32:
        raise ValueError("I_cam must be a float32 CUDA tensor")
    I_cam = I_cam.contiguous()
    out = torch.empty_like(I_cam)
    mask = torch.empty(I_cam.shape, dtype=torch.uint8, device=I_cam.device) if with_mask else None
    return I_cam, out, mask


def tilt_apply(table: torch.Tensor, I_cam: torch.Tensor, lo: float = -math.inf, hi: float = math.inf,
               with_mask: bool = True, stream: Optional[torch.cuda.Stream] = None):
    """``ptycho_tilt_apply``: the tilt correction of a stack with a table from :func:`tilt_table`."""
    I_cam, out, mask = _tilt_io(I_cam, with_mask)
    rc = _native.lib().ptycho_tilt_apply(int(I_cam.shape[1]), int(I_cam.shape[0]), _ptr(table), _ptr(I_cam),
                                         float(lo), float(hi), _ptr(out), _ptr(mask), _stream_handle(stream))
    _check(rc, "ptycho_tilt_apply")
    return out, mask


def plan_geometry_plan(r, **kw) -> Plan:
    """Plan for a serving request (``serve.Request``)."""
    return Plan(r.F, r.L, r.M, r.J, r.obj_shapes, r.pos, loss=r.loss, eps=r.eps, remap=r.remap, z=r.z,
                det_pixel=r.det_pixel, tilt_rad=r.tilt_rad, **kw)


def plan_for(w, **kw) -> Plan:
    """Plan for a :class:`synthetic.workloads.Workload`-like object (attribute access only)."""
    return Plan(w.F, w.L, w.M, w.J, w.obj_shapes, w.pos, loss=kw.pop("loss", w.loss),
                remap=kw.pop("remap", w.geom.remap), z=kw.pop("z", w.geom.z),
                det_pixel=kw.pop("det_pixel", w.geom.det_pixel), tilt_rad=kw.pop("tilt_rad", w.geom.tilt_rad),
                lambdas=w.geom.lambdas, **kw)
