#!/usr/bin/env python
"""Throughput benchmark of the fused forward + adjoint + Adam step.

Headline workload (default): the ~200 M-parameter reconstruction on one GPU, the shape of
the paper's largest run (Discussion: 201 M parameters on one GPU): 6 wavelengths x 10
probe modes of 512 x 512, six 3584 x 3584 objects, a 30 x 30 jittered scan (900
positions), tilted-plane remap and Poisson loss.  One *step* is one ``ptycho_step`` over
all positions: forward model, loss, adjoint, object/probe gradients and Adam.  One
*evaluation* is the forward + adjoint of one (position, wavelength, mode) triple, so a
step is 900 * 6 * 10 = 54 000 evaluations.  A secondary block times the 3-wavelength x
4-mode 256 x 256 case (400 positions, 4800 evaluations per step) the same way.

Synthetic, seeded inputs stand in for the paper's EUV dataset.  ``--impl reference``
times the FP64 CPU oracle (the only reference available) on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint frame·mode·λ evals/s, % roofline; p50/p99 site-iteration latency"
UNIT = "evals/s"
L2_BYTES = 126 * 1024 * 1024
FP32_LANES_PER_SM = 128            # FP32 FMA lanes per SM (Blackwell)


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_peak(sms: int):
    """FP32 ALU peak from unit counts: SMs (read from the device) x 128 lanes x 2 flop per FMA
    x the maximum SM clock (the measured sm_max_mhz, else the part's 2070 MHz)."""
    pk = measured_peaks()
    mhz, src = (float(pk["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz") if "sm_max_mhz" in pk \
        else (2070.0, "GB300 maximum SM clock")
    tflops = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return tflops, (f"derived: {sms} SMs (device attribute) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                    f"{mhz:.0f} MHz ({src}); MEASURED_PEAKS.json has no FP32 figure")


def hbm_peak():
    pk = measured_peaks()
    if "hbm_gbs" in pk:
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: 20 at 512^2, 200 otherwise)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="config4", help="config1 | config2 | config4 | config3:F,M,L | config5")
    ap.add_argument("--secondary", default="config2",
                    help="workload of the secondary block of the default line ('none' to skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU work budget of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--scratch-mb", type=int, default=0, help="L2 scratch budget of the plan (0 = library default)")
    ap.add_argument("--overlap", type=int, default=0, help="position batches in flight (0 = library default)")
    ap.add_argument("--graph", action="store_true", help="replay one step captured as a CUDA graph")
    ap.add_argument("--flags", type=int, default=0, help="PTYCHO_FLAG_* pipeline variants")
    ap.add_argument("--col-groups", type=int, default=0, help="mode groups of the column passes (0 = default)")
    ap.add_argument("--requests", type=int, default=64, help="config5: number of serving requests")
    ap.add_argument("--iterations", type=int, default=20, help="config5: iterations per request")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="config5: HBM budget of the server")
    ap.add_argument("--no-plain", action="store_true", help="config5: skip the plain one-site-at-a-time run")
    ap.add_argument("--plain", action="store_true", help="time the plain unfused step instead of the fused one")
    ap.add_argument("--corrections-steps", type=int, default=None,
                    help="steps timed with position (and power/background) correction on "
                         "(default: 5 at 512^2, 20 otherwise; 0 = skip)")
    ap.add_argument("--serving-requests", type=int, default=16,
                    help="requests of the reduced serving stream appended to the default line (0 = none)")
    ap.add_argument("--serve-mode", type=int, default=1,
                    help="serving tick: 0 = one launch per pass over all sites, 1 = one child graph per site "
                         "(the library default); the default line also times the other form")
    ap.add_argument("--tick-evals", type=int, default=32768,
                    help="config5: admit while the active sites' evaluations per tick stay within this (0 = no cap)")
    return ap.parse_args()


def make_workload(name: str):
    from synthetic import workloads as syn
    if name == "config1":
        return syn.config1()
    if name == "config2":
        return syn.config2()
    if name == "config4":
        return syn.config4()
    if name.startswith("config3:"):
        F, M, L = (int(v) for v in name.split(":")[1].split(","))
        return syn.config3(F, M, L)
    raise SystemExit(f"unknown config {name}")


def input_bytes(w) -> int:
    """Bytes a step reads as its inputs: measured patterns, parameters and Adam moments."""
    n_o = sum(h * wd for h, wd in w.obj_shapes)
    n_p = w.L * w.M * w.F * w.F
    return 4 * w.J * w.F * w.F + 8 * (n_o + n_p) + 16 * (n_o + n_p)


def workload_config(w, name, world: int = 1):
    ib = input_bytes(w)
    return {"workload": f"{name}: {w.L} wavelengths x {w.M} probe modes, {w.F}x{w.F} frames, {w.J} positions, "
                        f"objects {w.obj_shapes[0][0]}x{w.obj_shapes[0][1]}, "
                        f"{'tilted-plane remap' if w.geom.remap else 'no remap'}, {w.loss} loss",
            "frames": w.F, "wavelengths": w.L, "modes": w.M, "positions": w.J,
            "evals_per_step": w.n_evals,
            "parallelism": f"replicas x{world}" if world > 1 else "one device",
            "l2": f"step inputs of {ib / 2**20:.0f} MiB (measured patterns, parameters, Adam moments) "
                  f"{'exceed' if ib > L2_BYTES else 'fit'} the 126 MiB L2"}


def default_steps(w) -> int:
    return 20 if w.F >= 512 else 200


# --------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[1].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + parts[1].split(".")[1]) if "." in parts[1] else 0.0
                    rows.append(dict(ts=ts, sm=float(parts[2]), smax=float(parts[3]),
                                     power=float(parts[4]) if parts[4] not in ("[N/A]", "N/A") else None,
                                     reasons={"hw_slowdown": parts[6], "hw_thermal_slowdown": parts[7],
                                              "sw_thermal_slowdown": parts[8], "sw_power_cap": parts[9]}))
                except Exception:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        win = [r for r in rows if self.t0 is not None and self.t0 - 0.05 <= r["ts"] <= self.t1 + 0.05]
        note = "samples inside the timed region"
        if len(win) < 3:
            win = [r for r in rows if self.t0 is not None and self.t0 - 1.0 <= r["ts"] <= self.t1 + 1.0] or rows
            note = "timed region shorter than the sampling interval: samples within 1 s of it"
        reasons = sorted({k for r in win for k, v in r["reasons"].items() if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r["sm"] for r in win), "sm_max_mhz": max(r["smax"] for r in win),
                "reasons": reasons, "samples": len(win),
                "power_w_max": max((r["power"] for r in win if r["power"] is not None), default=None), "note": note}


# --------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------------------


def oracle_evals_per_s(w, n_pos: int, repeat: int = 1, seed: int = 0):
    """Time the oracle's loss + gradient + Adam on n_pos positions; returns (evals/s, seconds, evals)."""
    from oracle import ptycho_oracle as orc
    from synthetic import workloads as syn
    taps = orc.remap_taps(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad) if w.geom.remap else None
    rng = np.random.default_rng(seed)
    frames = sorted(rng.choice(w.J, size=n_pos, replace=False).tolist())
    clean = np.zeros((w.J, w.F, w.F))
    clean[frames] = orc.predict(w.O_true, w.P_true, w.pos, None, None, taps, frames=frames)
    Ih = syn.poisson_measure(clean, 5)
    eps = 1e-9 * float(Ih[frames].mean())
    st = orc.AdamState([o.shape for o in w.O0], w.P0.shape)
    O, P = w.O0, w.P0
    t0 = time.perf_counter()
    for _ in range(repeat):
        _, O, P = orc.step(O, P, w.pos, Ih, w.loss, eps, st, 1e-3, 1e-3, taps=taps, frames=frames)
    dt = time.perf_counter() - t0
    ev = repeat * n_pos * w.L * w.M
    return ev / dt, dt, ev


def cpu_threads_used() -> int:
    # numpy's FFT (pocketfft) runs on one thread; the oracle makes no threaded calls
    return 1



def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    w = make_workload(args.config)
    steps = args.steps if args.steps is not None else default_steps(w)
    _, t1, _ = oracle_evals_per_s(w, 1)                         # calibration: one position
    budget = 150.0
    per_step = max(1, min(w.J, int(budget / max(1, steps + args.warmup) / max(t1, 1e-3))))
    for _ in range(args.warmup):
        oracle_evals_per_s(w, per_step, seed=1)
    tot_t, tot_e = 0.0, 0
    for k in range(steps):
        _, dt, ev = oracle_evals_per_s(w, per_step, seed=2 + k)
        tot_t += dt
        tot_e += ev
    v = tot_e / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args.config, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_threads_used(), "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{per_step} of {w.J} positions per step ({per_step * w.L * w.M} evals): "
                                       "FP64 NumPy loss + gradient + Adam"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------
def kernel_hash() -> str:
    """sha256 prefix of the library's kernel headers (every ``csrc/*.cuh``: the device code and its launches)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_14780_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith(".cuh"):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, units_per_launch: float):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernels and on launches of
    the same size (evaluations per launch within 5 %)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(f"{workload}:{kernel}")
    if not e or d.get("kernel_sha") != kernel_hash():
        return None
    ev = e.get("evaluations_per_launch")
    if not ev or abs(units_per_launch - ev) > 0.05 * ev:
        return None
    return e.get("dram_bytes_per_launch")


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (x itself without a process group)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: float, steps: int, world: int, t_ms_max: float) -> float:
    """Units all ranks processed (each rank runs the same workload) per second of the slowest rank."""
    return units_per_step * steps * world / (t_ms_max / 1e3)


def algorithmic_flops_per_eval(F: int) -> float:
    """Two orthonormal 2D DFTs (forward + adjoint) at 5 N log2 N flops each, N = F^2."""
    return 2 * 5.0 * F * F * math.log2(F * F)



def measured_data(w, dev, seed: int):
    """Measured patterns: our forward model on the ground truth plus Poisson noise drawn on the
    GPU (input synthesis outside every timing; not a parity claim)."""
    import torch
    from paper_2311_14780_gb300 import pack_objects, plan_for
    plan_true = plan_for(w, eps=0.0)
    Ot = pack_objects(w.O_true, dev)
    Pt = torch.as_tensor(w.P_true, dtype=torch.complex64, device=dev).contiguous()
    I_clean = plan_true.forward(Ot, Pt)
    torch.cuda.synchronize()
    plan_true.close()
    del Ot, Pt
    gen = torch.Generator(device=dev).manual_seed(seed)
    Im = torch.poisson(I_clean.clamp_min(0), generator=gen).contiguous()
    del I_clean
    eps = 1e-9 * max(float(Im.mean(dtype=torch.float64).item()), 1e-30)
    return Im, eps


def timed_steps(step, steps: int, flush, stream, dist, clocks=None):
    """Per-step CUDA events on the launch stream, L2 flushed before every step, barrier and
    synchronize on both sides; returns (per-step ms, total ms)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark_start()
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.mark_end()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return step_ms, float(sum(step_ms))


def kernel_profile(plan, step, evals: int, F: int, prof_steps: int, peak: float, peak_src: str, traffic_key: str):
    """Per-kernel CUDA-event times of the plan's launches over prof_steps steps (events on each
    launch's own stream); the roofline of the dominant kernel and every kernel's share."""
    import torch
    plan.profile(True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile(False)
    flops_eval = algorithmic_flops_per_eval(F)
    # each of the four DFT passes (row fwd, col fwd, col adj, row adj) carries a quarter of
    # the algorithmic flops of every evaluation it processes
    fft_kernels = ("row_fwd", "col_fwd", "col_adj", "row_adj")
    dom = max(prof, key=lambda k: prof[k][0])
    kern_ms, kern_n = prof[dom]
    roof = None
    if dom in fft_kernels and kern_n:
        units_per_launch = evals * prof_steps / kern_n
        per_launch_flops = 0.25 * flops_eval * units_per_launch
        achieved = per_launch_flops / (kern_ms / kern_n / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dom, traffic_key, units_per_launch), "peak_source": peak_src,
                "units_per_launch": units_per_launch, "flops_per_unit": 0.25 * flops_eval,
                "avg_launch_ms": kern_ms / kern_n,
                "note": "launch durations are CUDA events on the launch stream with three position batches in "
                        "flight, so each launch shares the GPU with the other streams' kernels"}
        tr = roof["traffic"]
        if tr:
            hbm, _ = hbm_peak()
            roof["traffic_gbs"] = tr / (kern_ms / kern_n / 1e3) / 1e9
            roof["traffic_frac_of_hbm"] = roof["traffic_gbs"] / hbm
    total = max(1e-9, sum(x[0] for x in prof.values()))
    kernels = {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps, "share": v[0] / total}
               for k, v in prof.items() if v[1]}
    return roof, kernels


def corrections_block(w, plan, st, O, P, Im, loss, eps, evals, dev, stream, flush, nsteps):
    """The step with correction of further variables (the paper's Fig. 3 comparison)."""
    import torch
    from paper_2311_14780_gb300 import AdamState
    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for k in range(n):
            flush.fill_(float(k))
            a0.record(stream)
            fn()
            a1.record(stream)
            a1.synchronize()
            tot += a0.elapsed_time(a1)
        return tot / n
    rng = np.random.default_rng(7)
    delta = torch.as_tensor(rng.uniform(-0.5, 0.5, size=(w.L, w.J, 2)).astype(np.float32), device=dev)
    sig = torch.ones(w.J, dtype=torch.float32, device=dev)
    bgt = torch.ones(w.F, w.F, dtype=torch.float32, device=dev)
    O2, P2 = O.clone(), P.clone()
    base_ms = timed(lambda: plan.step(st, O2, P2, Im, loss_out=loss), nsteps)
    st_reg = AdamState(plan, lr_O=1e-3, lr_P=1e-3, reg_l1=1e-2, reg_tv=1e-1, reg_eta=1e-3)
    reg_ms = timed(lambda: plan.step(st_reg, O2, P2, Im, loss_out=loss), nsteps)
    plan.set_offsets(delta)
    st_pos = AdamState(plan, lr_O=1e-3, lr_P=1e-3, lr_delta=1e-2)
    pos_ms = timed(lambda: plan.step(st_pos, O2, P2, Im, loss_out=loss), nsteps)
    st_all = AdamState(plan, lr_O=1e-3, lr_P=1e-3, lr_delta=1e-2, lr_sigma=1e-2, lr_bg=1e-2)
    all_ms = timed(lambda: plan.step(st_all, O2, P2, Im, sig, bgt, loss_out=loss), nsteps)
    z_ms = None
    if w.geom.remap:
        # + dL/dz from the same pass, then a host Adam step on z and the remap rebuilt for it
        st_z = AdamState(plan, lr_O=1e-3, lr_P=1e-3, lr_delta=1e-2, lr_sigma=1e-2, lr_bg=1e-2,
                         with_z_gradient=True)
        zs = {"z": float(w.geom.z), "m": 0.0, "v": 0.0, "t": 0}

        def z_step():
            plan.step(st_z, O2, P2, Im, sig, bgt, loss_out=loss)
            g = float(st_z.g_z.item())
            zs["t"] += 1
            zs["m"] = 0.9 * zs["m"] + 0.1 * g
            zs["v"] = 0.999 * zs["v"] + 0.001 * g * g
            mh, vh = zs["m"] / (1 - 0.9 ** zs["t"]), zs["v"] / (1 - 0.999 ** zs["t"])
            zs["z"] -= 1e-7 * mh / (math.sqrt(vh) + 1e-12)
            plan.set_distance(zs["z"])
        z_ms = timed(z_step, nsteps)
        plan.set_distance(float(w.geom.z))
    plan.set_offsets(None)
    tilt = None
    if w.geom.remap:
        # the data-side form of the remap: the step's camera patterns corrected onto the model
        # grid with the paper's thresholds.  The table of camera positions (FP64) is built once
        # per geometry; the apply pass is HBM-bound: 4 B read, 4 B + 1 B written per pixel.
        from paper_2311_14780_gb300 import _native, tilt_table
        Ic = torch.empty_like(Im)
        Mc = torch.empty(Im.shape, dtype=torch.uint8, device=dev)
        lib = _native.lib()
        table = tilt_table(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad, device=dev)

        def tilt_apply_call():
            rc = lib.ptycho_tilt_apply(w.F, w.J, table.data_ptr(), Im.data_ptr(), 4.0, 65535.0, Ic.data_ptr(),
                                       Mc.data_ptr(), stream.cuda_stream)
            assert rc == 0, rc

        def tilt_table_call():
            rc = lib.ptycho_tilt_table(w.F, float(w.geom.z), float(w.geom.det_pixel), float(w.geom.tilt_rad),
                                       table.data_ptr(), stream.cuda_stream)
            assert rc == 0, rc
        tilt_ms = timed(tilt_apply_call, nsteps)
        table_ms = timed(tilt_table_call, nsteps)
        tbytes = w.J * w.F * w.F * (4 + 4 + 1)
        peak_hbm, peak_src = hbm_peak()
        gbs = tbytes / (tilt_ms / 1e3) / 1e9
        tilt = {"apply_ms": tilt_ms, "frames": w.J, "algorithmic_bytes": tbytes, "GB_per_s": gbs,
                "hbm_frac": gbs / peak_hbm, "peak_gbs": peak_hbm, "peak_source": peak_src,
                "table_ms": table_ms,
                "note": "ptycho_tilt_apply of the step's camera patterns (thresholds 4 and 65535) with a table "
                        "built once per geometry (ptycho_tilt_table, FP64, timed separately); L2 flushed before "
                        "each call; frac of measured HBM copy bandwidth"}
    # the chirp-z propagator: every wavelength on the first one's object grid (zoom
    # lambda_1 / lambda_l, the first wavelength's positions for all)
    lam = np.asarray(w.geom.lambdas, dtype=np.float64)
    from paper_2311_14780_gb300.api import Plan
    pos_common = np.repeat(np.asarray(w.pos)[:1], w.L, axis=0)
    pz = Plan(w.F, w.L, w.M, w.J, w.obj_shapes, pos_common, loss=w.loss, eps=eps, remap=w.geom.remap,
              z=w.geom.z, det_pixel=w.geom.det_pixel, tilt_rad=w.geom.tilt_rad, zoom=lam[0] / lam)
    st_z2 = AdamState(pz, lr_O=1e-3, lr_P=1e-3)
    czt_ms = timed(lambda: pz.step(st_z2, O2, P2, Im, loss_out=loss), nsteps)
    pz.close()
    corrections = {
        "steps": nsteps,
        "object_probe": {"ms_per_step": base_ms, "evals_per_s": evals / (base_ms / 1e3)},
        "plus_regularisation": {"ms_per_step": reg_ms, "evals_per_s": evals / (reg_ms / 1e3),
                                "relative_time": reg_ms / base_ms,
                                "note": "L1 and TV of the object amplitude added in the step (ptycho_regularise)"},
        "plus_positions": {"ms_per_step": pos_ms, "evals_per_s": evals / (pos_ms / 1e3),
                           "relative_time": pos_ms / base_ms},
        "plus_positions_power_background": {"ms_per_step": all_ms, "evals_per_s": evals / (all_ms / 1e3),
                                            "relative_time": all_ms / base_ms},
        "plus_positions_power_background_distance": None if z_ms is None else
        {"ms_per_step": z_ms, "evals_per_s": evals / (z_ms / 1e3), "relative_time": z_ms / base_ms,
         "note": "dL/dz in the same pass; z updated by Adam on the host and the remap rebuilt every step"},
        "chirp_z_propagator": None if czt_ms is None else
        {"ms_per_step": czt_ms, "evals_per_s": evals / (czt_ms / 1e3), "relative_time": czt_ms / base_ms,
         "note": "zoom DFT (Bluestein, 2F-point transforms) with zoom lambda_1/lambda_l instead of the DFT"},
        "data_side_tilt_correction": tilt,
        "note": "fractional scan offsets (Fourier shift) optimised by Adam in the same step; uniform(-0.5, 0.5) px"}
    return corrections


def secondary_block(name, args, dev, flush, stream, peak, peak_src):
    """The fused step of a second workload, timed like the headline (no e2e, no corrections)."""
    import torch
    from paper_2311_14780_gb300 import AdamState, pack_objects, plan_for
    w = make_workload(name)
    Im, eps = measured_data(w, dev, 4321)
    plan = plan_for(w, eps=eps)
    O = pack_objects(w.O0, dev)
    P = torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous()
    st = AdamState(plan, lr_O=1e-3, lr_P=1e-3)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)

    def step():
        plan.step(st, O, P, Im, loss_out=loss)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    steps = default_steps(w)
    step_ms, t_ms = timed_steps(step, steps, flush, stream, None)
    roof, kernels = kernel_profile(plan, step, w.n_evals, w.F, min(steps, 50), peak, peak_src, name)
    plan.close()
    return {"config": workload_config(w, name), "value": w.n_evals * steps / (t_ms / 1e3), "unit": UNIT,
            "steps": steps, "ms_per_step": t_ms / steps, "step_ms_p50": statistics.median(step_ms),
            "step_flop_rate_tflops": algorithmic_flops_per_eval(w.F) * w.n_evals / (t_ms / steps / 1e3) / 1e12,
            "roofline": roof, "kernels": kernels}


def run_ours(args, rank: int, world: int):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2311_14780_gb300 import AdamState, pack_objects, plan_for

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_src = fp32_peak(sms)
    w = make_workload(args.config)
    steps = args.steps if args.steps is not None else default_steps(w)
    corr_steps = args.corrections_steps if args.corrections_steps is not None else (5 if w.F >= 512 else 20)
    Im, eps = measured_data(w, dev, 1234 + rank)
    plan = plan_for(w, eps=eps, scratch_bytes=args.scratch_mb << 20, overlap=args.overlap, flags=args.flags,
                    col_groups=args.col_groups)
    O = pack_objects(w.O0, dev)
    P = torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous()
    st = AdamState(plan, lr_O=1e-3, lr_P=1e-3, device_counter=args.graph)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(4 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    evals = w.n_evals

    def step():
        if args.plain:
            plan.plain_step(st, O, P, Im, loss_out=loss)
        else:
            plan.step(st, O, P, Im, loss_out=loss)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches_per_step = plan.last_launches
    eager_step = step
    if args.graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()

        def step():  # noqa: F811 - the timed step replays the captured one
            graph.replay()
        step()
        torch.cuda.synchronize()

    # ---- timed region: per-step events, L2 flushed between steps --------------------
    clocks = ClockSampler(local)
    time.sleep(0.2)
    step_ms, t_local = timed_steps(step, steps, flush, stream, dist, clocks)
    t_ms = max_over_ranks(t_local, dist, dev)
    clk = clocks.stop()
    value = whole_job_rate(evals, steps, world, t_ms)

    # ---- per-kernel event timing for the roofline (same workload, same streams) ----------
    roof, kernels = kernel_profile(plan, eager_step, evals, w.F, max(3, min(steps, 50)), peak, peak_src,
                                   args.config)
    step_flops = algorithmic_flops_per_eval(w.F) * evals

    # ---- end to end through the C ABI with host buffers ---------------------------------
    # ptycho_step_host: the measured patterns in pinned host memory are copied to the device on
    # the stream, the step runs, and the loss is copied back to pinned host memory, every step
    e2e = None
    if not args.no_e2e and not args.plain:
        Ih_pinned = Im.cpu().pin_memory()
        loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
        e_steps = max(3, min(steps, 50))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            plan.step_host(st, O, P, Ih_pinned, Im, loss, loss_host)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        e2e = {"value": whole_job_rate(evals, e_steps, world, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(Ih_pinned.numel() * 4), "d2h_bytes_per_step": 8,
               "steps": e_steps, "ms_per_step": e_ms / e_steps,
               "note": "ptycho_step_host (C ABI): I_meas in pinned host memory copied to the device with "
                       "cudaMemcpyAsync every step (batch by batch on a side stream that starts after the previous "
                       "step, each batch's loss waiting for its own frames), the step, and the FP64 loss copied back "
                       "to pinned host memory; CUDA events on the caller's stream around all of it"}
        del Ih_pinned

    corrections = None
    if corr_steps > 0 and not args.plain and not args.graph:
        corrections = corrections_block(w, plan, st, O, P, Im, loss, eps, evals, dev, stream, flush, corr_steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, t1, _ = oracle_evals_per_s(w, 1)
        n_pos = max(1, min(w.J, int(args.cpu_seconds / max(t1, 1e-3))))
        v_cpu, dt, ev = oracle_evals_per_s(w, n_pos, seed=3)
        cpu = {"value": v_cpu, "unit": UNIT, "cores": cpu_threads_used(), "host_cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{n_pos} of {w.J} positions ({ev} evals, {dt:.1f} s): FP64 NumPy loss + gradient + Adam "
                         f"on one of the host's {os.cpu_count()} cores"}
    plan.close()
    del O, P, Im, st

    secondary = None
    if world == 1 and args.secondary != "none" and args.secondary != args.config and not args.plain:
        secondary = secondary_block(args.secondary, args, dev, flush, stream, peak, peak_src)

    serving = None
    if world == 1 and args.serving_requests > 0 and not args.plain:
        from paper_2311_14780_gb300.serve import plain_stream, serve_stream
        import copy
        sargs = copy.copy(args)
        sargs.requests = args.serving_requests
        served, plain_reqs = serving_requests(sargs, dev)
        s_sum = serve_stream(served, int(args.budget_gb * (1 << 30)), max_tick_evals=args.tick_evals or None,
                             mode=args.serve_mode)
        p_sum = plain_stream(plain_reqs)
        p_sum["final_loss_rel_diff_max"] = max(abs(a.final_loss - b.final_loss) / max(abs(b.final_loss), 1e-300)
                                               for a, b in zip(served, plain_reqs))
        # the other tick form on a fresh copy of the same requests
        other = 1 - args.serve_mode
        served2, _ = serving_requests(sargs, dev)
        o_sum = serve_stream(served2, int(args.budget_gb * (1 << 30)), max_tick_evals=args.tick_evals or None,
                             mode=other)
        serving = {"stream": f"first {sargs.requests} requests of the config-5 stream (Poisson arrivals, mean 50 ms; "
                             f"F in {{128,256,512}}, J 100-900, L 1-5, M 1-8; {args.iterations} iterations each); "
                             "full stream: bench.py --config config5",
                   "mode": SERVE_MODES[args.serve_mode],
                   "served": s_sum, "plain_one_site_at_a_time": p_sum,
                   "served_over_plain": s_sum["evals_per_s"] / p_sum["evals_per_s"],
                   "site_iteration_ms_p50": s_sum["iter_ms_p50"], "site_iteration_ms_p99": s_sum["iter_ms_p99"],
                   "other_mode": {"mode": SERVE_MODES[other],
                                  **{k: o_sum[k] for k in ("evals_per_s", "iter_ms_p50", "iter_ms_p99",
                                                            "time_to_target_ms_p50", "time_to_target_ms_p99")}}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": max(3, args.warmup), "ms_per_step": t_ms / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64/f32 (loss sum f64)", "data": "synthetic",
                "config": workload_config(w, args.config, world),
                "l2_flush": "a 512 MiB buffer written before every timed step (outside the events)",
                "device": {"name": torch.cuda.get_device_name(dev), "sms": sms},
                "clocks": clk, "gpu_launches": int(launches_per_step * steps),
                "roofline": roof, "step_flop_rate_tflops": step_flops / (t_ms / steps / 1e3) / 1e12,
                "step_flop_frac_of_fp32_peak": step_flops / (t_ms / steps / 1e3) / 1e12 / peak,
                "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "step_ms_p50": statistics.median(step_ms), "step_ms_p99": float(np.percentile(step_ms, 99)),
                "secondary": secondary, "serving": serving, "corrections": corrections}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


SERVE_MODES = {0: "shared launches (one launch per pass over all sites)", 1: "one child graph per site"}


def serving_requests(args, dev):
    """Config 5: Poisson arrivals (mean 50 ms); F in {128, 256, 512}, J in [100, 900], L in 1..5,
    M in 1..8; flat-object / elliptical-aperture start.  Measured data: our forward model on
    the truth plus Poisson noise drawn on the GPU (input synthesis, outside every timing)."""
    import torch
    from paper_2311_14780_gb300 import pack_objects, plan_for
    from paper_2311_14780_gb300.serve import Request
    from synthetic import workloads as syn
    bank = syn.TextureBank()
    gen = torch.Generator(device=dev).manual_seed(5)
    served, plain = [], []
    for d in syn.config5_requests(n=args.requests):
        w = syn.serving_request_inputs(d, bank)
        pt = plan_for(w, eps=0.0)
        I = pt.forward(pack_objects(w.O_true, dev), torch.as_tensor(w.P_true, dtype=torch.complex64, device=dev))
        pt.close()
        Ih = torch.poisson(I.clamp_min(0), generator=gen).contiguous()
        eps = 1e-9 * float(Ih.mean().item())
        O0 = pack_objects(w.O0, dev)
        P0 = torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous()
        for out in (served, plain):
            out.append(Request(w.name, d["arrival_s"], w.F, w.L, w.M, w.J, w.obj_shapes, w.pos, O0.clone(),
                               P0.clone(), Ih, iterations=args.iterations, loss="poisson", eps=eps, remap=True,
                               lr_O=1e-2, lr_P=1e-2))
    torch.cuda.synchronize()
    return served, plain


def run_serving(args, rank: int, world: int):
    import torch
    from paper_2311_14780_gb300.serve import plain_stream, serve_stream
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    served, plain = serving_requests(args, dev)
    clocks = ClockSampler(local)
    time.sleep(0.2)
    clocks.mark_start()
    s_sum = serve_stream(served, int(args.budget_gb * (1 << 30)), max_tick_evals=args.tick_evals or None,
                             mode=args.serve_mode)
    clocks.mark_end()
    clk = clocks.stop()
    p_sum = None
    if not args.no_plain:
        p_sum = plain_stream(plain)
        rel = [abs(a.final_loss - b.final_loss) / max(abs(b.final_loss), 1e-300) for a, b in zip(served, plain)]
        p_sum["final_loss_rel_diff_max"] = max(rel)
    if rank == 0:
        line = {"metric": METRIC, "value": s_sum["evals_per_s"], "unit": UNIT, "n_gpus": world,
                "steps": args.iterations, "warmup": 0, "ms_per_step": s_sum["iter_ms_p50"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64/f32 (loss sum f64)", "data": "synthetic",
                "config": {"workload": f"config5: serving stream of {args.requests} requests, Poisson arrivals "
                                       f"(mean 50 ms), F in {{128,256,512}}, J in [100,900], L 1-5, M 1-8, "
                                       f"{args.iterations} iterations each, HBM budget {args.budget_gb} GB"},
                "clocks": clk, "mode": SERVE_MODES[args.serve_mode], "serving": s_sum, "plain": p_sum,
                "served_over_plain": (s_sum["evals_per_s"] / p_sum["evals_per_s"]) if p_sum else None}
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.config == "config5":
        return run_serving(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())

