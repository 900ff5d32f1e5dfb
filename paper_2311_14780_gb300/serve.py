"""Serving front end: many reconstructions resident on one GPU, continuous batching.

``Server`` wraps the C ABI (ptycho_server_*): sites are admitted while the HBM budget
allows, every ``tick`` runs one iteration of every active site as one graph launch, and
finished sites give their memory back.  ``serve_stream`` drives a stream of requests with
arrival times through it and records per-iteration and time-to-target latencies;
``plain_stream`` runs the same requests one site at a time with the unfused
``ptycho_plain_step``, the baseline.  Python here only schedules and marshals arguments;
every computation is in the CUDA library.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time
from typing import List, Optional

import numpy as np
import torch

from . import _native
from .api import AdamState, PtychoError, _check, _ptr, _stream_handle, geom_struct

EBUSY = -8


@dataclasses.dataclass
class Request:
    """One reconstruction job: geometry, resident device data, and its schedule."""
    name: str
    arrival_s: float
    F: int
    L: int
    M: int
    J: int
    obj_shapes: list
    pos: np.ndarray
    O: torch.Tensor                 # packed complex64, updated in place
    P: torch.Tensor                 # [L, M, F, F] complex64, updated in place
    I_meas: torch.Tensor            # [J, F, F] float32
    iterations: int = 20
    loss: str = "poisson"
    eps: float = 0.0
    remap: bool = True
    z: float = 88e-3
    det_pixel: float = 15e-6
    tilt_rad: float = 1.2217304763960306
    lr_O: float = 1e-3
    lr_P: float = 1e-3
    # filled in by the drivers
    admitted_s: Optional[float] = None
    done_s: Optional[float] = None
    final_loss: Optional[float] = None
    iter_ms: List[float] = dataclasses.field(default_factory=list)

    @property
    def evals(self) -> int:
        return self.J * self.L * self.M * self.iterations

    @property
    def evals_per_iteration(self) -> int:
        return self.J * self.L * self.M


class Server:
    """``ptycho_server_t``: resident sites, budgeted admission, one graph launch per tick."""

    SHARED_LAUNCHES = 0
    SITE_GRAPHS = 1

    def __init__(self, budget_bytes: int, max_sites: int = 128, mode: int = 1):
        h = ctypes.c_void_p()
        _check(_native.lib().ptycho_server_create(int(budget_bytes), int(max_sites), ctypes.byref(h)),
               "ptycho_server_create")
        self._h = h
        self._keep = {}
        _check(_native.lib().ptycho_server_set_mode(self._h, int(mode)), "ptycho_server_set_mode")

    def admit(self, r: Request) -> Optional[int]:
        """Slot of the admitted request, or None when it does not fit right now."""
        g, keep = geom_struct(r.F, r.L, r.M, r.J, r.obj_shapes, r.pos, loss=r.loss, eps=r.eps, remap=r.remap,
                              z=r.z, det_pixel=r.det_pixel, tilt_rad=r.tilt_rad)
        s = _native.Site()
        s.O = r.O.data_ptr()
        s.P = r.P.data_ptr()
        s.I_meas = r.I_meas.data_ptr()
        s.mask = None
        s.mask_per_frame = 0
        s.sigma = None
        s.bg = None
        s.lr_O, s.lr_P, s.beta1, s.beta2, s.eps = r.lr_O, r.lr_P, 0.9, 0.999, 1e-8
        s.iterations = int(r.iterations)
        slot = ctypes.c_int32(-1)
        rc = _native.lib().ptycho_server_admit(self._h, ctypes.byref(g), ctypes.byref(s), ctypes.byref(slot))
        if rc == EBUSY:
            return None
        _check(rc, "ptycho_server_admit")
        self._keep[slot.value] = (g, keep, r)
        return int(slot.value)

    def tick(self, stream=None) -> int:
        n = ctypes.c_int32(0)
        _check(_native.lib().ptycho_server_tick(self._h, _stream_handle(stream), ctypes.byref(n)),
               "ptycho_server_tick")
        return int(n.value)

    def status(self, slot: int):
        it = ctypes.c_int32(0)
        loss = ctypes.c_double(0.0)
        _check(_native.lib().ptycho_server_site_status(self._h, int(slot), ctypes.byref(it), ctypes.byref(loss)),
               "ptycho_server_site_status")
        return int(it.value), float(loss.value)

    def release(self, slot: int):
        _check(_native.lib().ptycho_server_release(self._h, int(slot)), "ptycho_server_release")
        self._keep.pop(slot, None)

    @property
    def used_bytes(self) -> int:
        return int(_native.lib().ptycho_server_used_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _native.lib().ptycho_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serve_stream(reqs: List[Request], budget_bytes: int, max_sites: int = 128, realtime: bool = True,
                 max_tick_evals: Optional[int] = None, mode: int = 1) -> dict:
    """Run the requests through a Server (``mode``: Server.SHARED_LAUNCHES or SITE_GRAPHS),
    admitting them as they arrive and fit.

    Requests are admitted in arrival order while the HBM budget allows and, if
    ``max_tick_evals`` is set, while the active sites' evaluations per tick stay within it
    (a request is always admitted when nothing is active).  With ``realtime`` the arrival
    times are honoured against the wall clock; otherwise all requests are present at time
    0.  Returns the latency and throughput summary.
    """
    sv = Server(budget_bytes, max_sites, mode)
    stream = torch.cuda.current_stream()
    pending = sorted(reqs, key=lambda r: r.arrival_s)
    active = {}
    t0 = time.perf_counter()
    ticks = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while pending or active:
        now = time.perf_counter() - t0
        while pending and (not realtime or pending[0].arrival_s <= now):
            r = pending[0]
            load = sum(a.evals_per_iteration for a in active.values())
            if active and max_tick_evals is not None and load + r.evals_per_iteration > max_tick_evals:
                break
            slot = sv.admit(r)
            if slot is None:
                if not active:
                    raise RuntimeError(f"request {r.name} does not fit the serving budget on its own")
                break
            r.admitted_s = time.perf_counter() - t0
            active[slot] = r
            pending.pop(0)
        if not active:
            time.sleep(max(0.0, pending[0].arrival_s - (time.perf_counter() - t0)))
            continue
        e0.record(stream)
        sv.tick(stream)
        e1.record(stream)
        e1.synchronize()
        ticks += 1
        ms = e0.elapsed_time(e1)
        for slot, r in list(active.items()):
            r.iter_ms.append(ms)
            it, loss = sv.status(slot)
            if it >= r.iterations:
                r.done_s = time.perf_counter() - t0
                r.final_loss = loss
                sv.release(slot)
                del active[slot]
    makespan = max(r.done_s for r in reqs) - min(r.arrival_s for r in reqs) if realtime else \
        max(r.done_s for r in reqs)
    sv.close()
    return summarize(reqs, makespan, ticks=ticks, max_tick_evals=max_tick_evals)


def plain_stream(reqs: List[Request], realtime: bool = True) -> dict:
    """The same requests one site at a time (FIFO) with the unfused plain step."""
    from .api import plan_geometry_plan
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    loss = torch.zeros(1, dtype=torch.float64, device=reqs[0].O.device)
    for r in sorted(reqs, key=lambda r: r.arrival_s):
        if realtime:
            wait = r.arrival_s - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        r.admitted_s = time.perf_counter() - t0
        plan = plan_geometry_plan(r)
        st = AdamState(plan, r.lr_O, r.lr_P)
        for _ in range(r.iterations):
            e0.record(stream)
            plan.plain_step(st, r.O, r.P, r.I_meas, loss_out=loss)
            e1.record(stream)
            e1.synchronize()
            r.iter_ms.append(e0.elapsed_time(e1))
        r.final_loss = float(loss.item())
        r.done_s = time.perf_counter() - t0
        plan.close()
    makespan = max(r.done_s for r in reqs) - min(r.arrival_s for r in reqs) if realtime else \
        max(r.done_s for r in reqs)
    return summarize(reqs, makespan)


def summarize(reqs: List[Request], makespan_s: float, **extra) -> dict:
    it = np.concatenate([np.asarray(r.iter_ms) for r in reqs])
    ttt = np.asarray([(r.done_s - r.arrival_s) * 1e3 for r in reqs])
    evals = sum(r.evals for r in reqs)
    out = {"requests": len(reqs), "evals": evals, "makespan_s": makespan_s, "evals_per_s": evals / makespan_s,
           "iter_ms_p50": float(np.percentile(it, 50)), "iter_ms_p99": float(np.percentile(it, 99)),
           "time_to_target_ms_p50": float(np.percentile(ttt, 50)),
           "time_to_target_ms_p99": float(np.percentile(ttt, 99))}
    out.update(extra)
    return out
