#!/usr/bin/env python
"""Benchmark of the 2D TK-WFP per-step evaluation loop on GB300.

Default workload (the paper-scale case): 10^6 coincident sources/targets equispaced on 100
seeded random ellipses (semi-axes 10-40 wavelengths) in a 300x300-wavelength box, signals =
sums of three Gaussian-enveloped sinusoids (carrier 2 pi rad per unit time), dt = 0.1 (~10 steps
per period), N_t = 3000, tolerance 1e-6, mixed-precision path; the FP64 path runs beside it on
the same workload, and the 10^4-point workload (6 ellipses in a 30x30 box, N_t = 2000, timed in
its lagged / far-history regime) is reported as a sub-record on both paths.  A "step" is one pass
of the whole per-step loop (ingest, local part, self term, type-1 NUFFT(s), mode and far-history
updates, type-2 NUFFT).  The timed window ends at a step where the field is well developed.

Metric: target-updates/s = (targets x timed steps) / time.  `value` is device-timed with CUDA
events on the plan's stream, inputs resident in HBM; `e2e` is measured through the C ABI with
page-locked host buffers (host->device copy of sigma_n and device->host copy of u_n inside the
timed region).
Accuracy: relative L2 error against the FP64 CPU oracle (exact retarded field) on random targets
at two timed steps.  `--impl reference` times that oracle on the host cores on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M*N_t target-updates/s (targets x steps per second), mixed-precision path; FP64 path beside"
# unit counts x the maximum SM clock: the ALU roofline's peaks
FP64_PEAK_DERIVED = 152 * 2.07e9 * 4 / 1e12    # 2 FP64 FMA per clock per SM
FP32_PEAK_DERIVED = 152 * 2.07e9 * 256 / 1e12  # 128 FP32 FMA per clock per SM
# the step at which the timed window ends, per workload: one where the field is developed (the
# pulses start near t = 8); workloads with a lagged regime are timed after it instead
TIMED_END = {"cfg1": 90, "cfg4": 400}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg4")
    ap.add_argument("--nt", type=int, default=0, help="override the workload's N_t (e.g. to stay before the lag)")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-beside", action="store_true", help="skip the other path on the same workload")
    ap.add_argument("--sub", default="cfg2", help="workload of the sub-record ('' for none)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline and accuracy")
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--opt", action="append", default=[], help="plan option key=value (wfp_opts field)")
    ap.add_argument("--drive", type=int, default=0,
                    help="only step the workload this many times with graphs off and exit (profiler target)")
    ap.add_argument("--serve", type=int, default=0,
                    help="serving benchmark with this many requests (Poisson arrivals) instead of the step loop")
    ap.add_argument("--serve-load", type=float, default=0.8, help="offered load as a fraction of batch capacity")
    ap.add_argument("--serve-check", type=int, default=5, help="requests checked against the oracle (--serve)")
    ap.add_argument("--max-active", type=int, default=48)
    ap.add_argument("--accuracy-targets", type=int, default=100,
                    help="random targets compared with the oracle at two timed steps")
    a = ap.parse_args(argv)
    a.plan_opts = {}
    for kv in a.opt:
        k, v = kv.split("=")
        a.plan_opts[k] = float(v) if any(c in v for c in ".e") else int(v)
    return a


# ----------------------------------------------------------------------------- helpers
def dist_init():
    """One process per GPU under torchrun (NCCL), or gloo where no GPU is visible (CPU tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
        return dist, int(os.environ["RANK"]), ws
    return None, 0, 1


def max_over_ranks(dist, value: float, device=None) -> float:
    """The slowest rank's time (the job's time under weak scaling)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


_ALU = {}  # measured FMA-loop peaks of this GPU, filled once per run (TFLOP/s)


def measure_alu_peaks() -> None:
    """FP64 and FP32 FMA throughput of this GPU (wfp_debug_alu_peak: a timed loop of independent FMAs)."""
    from paper_2604_07170_gb300 import wfp
    for fp64 in (True, False):
        tf, _ = wfp.alu_peak(fp64)
        _ALU["fp64" if fp64 else "fp32"] = tf


def measured_peaks() -> dict:
    """HBM: the measured copy bandwidth.  ALU: derived from the unit counts and the maximum SM clock;
    the FMA loop measured on this GPU (wfp_debug_alu_peak) is reported beside it, and is a lower bound
    on the FP64 rate (the FP64 local-part kernel itself sustains more than the loop does)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "source": "fallback"}
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        out = {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    out.update(fp64_tflops=FP64_PEAK_DERIVED, fp32_tflops=FP32_PEAK_DERIVED,
               alu_source="derived: 152 SMs x 2070 MHz x FMA units per SM (2 FP64, 128 FP32 FMA/clk)")
    return out


def part_model(info: dict, M: int, Mt: int, fp64: bool) -> dict:
    """Algorithmic bytes and flops per launch of each part (the minimum the method moves)."""
    s = 8 if fp64 else 4          # reduced-precision word
    c = 2 * s                     # reduced-precision complex
    W = info["W"]
    NW = 32 if info["nmax"] <= 32 else 64
    npair, nm, nf_ = info["n_pairs"], info["n_modes"], info["n_far_modes"]
    nk, nl = info["n_kappa"], info["n_lambda"]
    nb, nfg, w = info["nb"], info["nf"], info["kernel_width"]
    nself, nsoe = info["n_self"], info["n_self_soe"]
    lag = 1 if info["lag_active"] else 0  # the timed window is in the lagged regime when there is one
    spreads = 1 + (lag and not info["lag_store"])  # a second (lagged) spread only without the stored S history
    # FIR taps per |k|: FP64 {p, q, pA, qA}; mixed, FP32 hi/lo pairs of all four, or FP32 {p, q} when
    # the lag never switches on
    tapw = 4 * W * s if fp64 else (8 * W * 4 if lag else 2 * W * 4)
    # the part of the [nb][nf] band that spreading writes and interpolation reads: its non-empty tiles,
    # all inside the nb x nb sub-box of columns lb0 .. lb0 + nb that the points map to (the whole sub-box
    # when the tile count is unknown)
    ts = info.get("spread_tile") or 0
    band = min(nb * nb, info["n_spread_tiles"] * ts * ts) if info.get("n_spread_tiles") and ts else nb * nb
    m = {}
    if info.get("local_form") == 2:
        # factored form: pair records (8 bytes, 16 in FP64), near pairs' stored rows, the per-step
        # contraction y written once and read once, the windows, row pointers and the output;
        # flops: the contraction (2 * 32 * NC per source and interval) and per table pair the
        # Chebyshev recurrence and dot product (2 * (2 NC - 2)), per near pair a 32-level dot product
        nc, nnear = info["local_nc"], info["n_near_pairs"]
        ntab = npair - nnear
        ybytes = (W - 1) * M * nc * s
        m["local"] = (ntab * 2 * s + nnear * (NW * s + 4) + 2 * ybytes + M * NW * s + Mt * (16 + 8),
                      2 * 32 * nc * (W - 1) * M + ntab * 2 * (2 * nc - 2) + nnear * 2 * NW)
    else:
        m["local"] = (npair * (NW * s + 4) + M * NW * s + Mt * (8 + 8), 2 * npair * info["nmax"])
    # shared window (W levels) + one-tap recurrences: Z_l read and written, FP64
    m["self"] = (nself * (nsoe * 16 + W * s + 12), nself * (nsoe * 4 + 2 * W))
    m["ingest"] = (M * (8 + 4 + 2 * s + (2 * NW * s if NW == 32 else 0)), 0)
    m["combine"] = (Mt * (4 + 4 * 8), Mt * 2)
    m["spread"] = (spreads * (band * s + M * (2 * w * s + 4 + s)), spreads * 2 * M * w * w)
    # S read and ring write, W ring levels (current and lagged), alpha/alphadot read+write, grid write
    m["modes"] = (nm * ((1 + lag) * W * c + 2 * c + 4 * 16 + 12 + c) + nk * tapw, nm * (8 * W * (1 + lag) + 16))
    # E_l read+write (FP64 complex) and H_l per term, W lagged levels, grid read+write
    m["far"] = (nf_ * (nl * (32 + 8) + W * c + 2 * c), nf_ * (nl * 8 + 4 * W))
    m["interp"] = (band * s + Mt * (2 * w * s + 4 + 8), 2 * Mt * w * w)
    # two-stage pruned FFTs: R2C over the nb band rows, C2C over the N_h + 1 kept columns (and back)
    nh2, nc1, lg = nfg // 2 + 1, info["Nh"] + 1, math.log2(nfg)
    fft_b = nb * nfg * s + nb * nh2 * c + 2 * nb * nc1 * c + 2 * nfg * nc1 * c  # rows, band transpose, columns
    fft_f = nb * 2.5 * nfg * lg + nc1 * 5 * nfg * lg
    m["fft_type1"] = (spreads * fft_b, spreads * fft_f)
    m["fft_type2"] = (fft_b, fft_f)
    return {k: {"bytes": int(b), "flops": int(f)} for k, (b, f) in m.items()}


# ----------------------------------------------------------------------------- our arm
def measure(wl, precision: str, K: int, Wm: int, e2e_steps: int, prof_steps: int, keep: int, dev, dist,
            plan_opts: dict, timed_end: int = 0) -> dict:
    """Plan the workload, step it to the timed window, time K steps (CUDA events on the plan's
    stream, inputs resident), keep the outputs of the last `keep` timed steps, then per-part event
    timing and the end-to-end rate through the C ABI with page-locked host buffers."""
    import torch
    from paper_2604_07170_gb300 import wfp
    M, Mt = wl.M, wl.M
    prec = 0 if precision == "fp64" else 1
    stream = torch.cuda.Stream(device=dev)
    p0 = wfp.select_params(wl.meta["box"] / 2, wl.dt, wl.n_steps, wl.band_limit, wl.tol, precision=prec)
    # every part the workload uses is active in the timed window: after the lag switches on when the
    # workload has a lagged regime (N_t > L), else once the local window is full and the field developed
    pre = p0["L"] + p0["W"] + 1 if p0["lag_active"] else p0["nmax"] + 1
    first = max(pre + Wm + 1, timed_end - K + 1)
    Nt = max(wl.n_steps, first + K - 1 + prof_steps + e2e_steps)
    t0 = time.perf_counter()
    plan = wfp.Plan(wl.src_xy, None, wl.dt, Nt, wl.band_limit, wl.tol, precision=prec, stream=stream.cuda_stream,
                    **plan_opts)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    out = torch.empty(Mt, dtype=torch.float64, device=dev)
    n = 0
    chunk = 256

    def run_device(nsteps):
        nonlocal n
        done = 0
        while done < nsteps:
            k = min(chunk, nsteps - done)
            sig = torch.from_numpy(wl.sigma(n + 1, n + 1 + k)).to(dev)
            torch.cuda.synchronize(dev)
            for i in range(k):
                plan.step(sig[i], out)
            n += k
            done += k

    run_device(first - 1)
    # timed region: inputs already resident in HBM; the last `keep` steps write their own buffers
    sig = torch.from_numpy(wl.sigma(n + 1, n + 1 + K)).to(dev)
    kept = torch.empty((keep, Mt), dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for i in range(K):
            plan.step(sig[i], kept[i - (K - keep)] if i >= K - keep else out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(dist, ms, dev)
    r = {"ms": ms, "K": K, "info": info, "plan_s": plan_s, "clocks": clk.summary(), "precision": precision,
         "kept": kept.cpu().numpy(), "kept_steps": list(range(n + K - keep + 1, n + K + 1)), "n_last": n + K,
         "workload": wl.name}
    n += K
    if prof_steps > 0:  # per-part timing with CUDA events on the plan's stream (parts in sequence)
        plan.profile(True)
        run_device(prof_steps)
        r["parts"] = plan.profile_read()
        r["prof_steps"] = prof_steps
        plan.profile(False)
    if e2e_steps > 0:  # end to end through the C ABI with page-locked host buffers
        sig_pin = torch.empty((e2e_steps, wl.M), dtype=torch.float64, pin_memory=True)
        u_pin = torch.empty(Mt, dtype=torch.float64, pin_memory=True)
        sig_h, u_h = sig_pin.numpy(), u_pin.numpy()
        sig_h[:] = wl.sigma(n + 1, n + 1 + e2e_steps)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            plan.step(sig_h[i], u_h)
        torch.cuda.synchronize(dev)
        r["e2e_s"] = time.perf_counter() - t0
        r["e2e_steps"] = e2e_steps
        n += e2e_steps
    plan.close()
    del plan
    torch.cuda.synchronize(dev)
    return r


def cpu_oracle_rate(wl, n_eval_hint: int, t_budget: float, step: int):
    """Oracle throughput (target-updates/s) on the host cores, on a bounded sample."""
    import oracle
    rng = np.random.default_rng(0)
    cores = oracle.num_threads()
    n = max(cores, 8)
    while True:
        idx = rng.choice(wl.M, n, replace=False)
        ev = np.column_stack([wl.src_xy[idx], np.full(n, step * wl.dt)])
        t0 = time.perf_counter()
        oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"])
        dt = time.perf_counter() - t0
        if dt > 0.25 * t_budget or n >= n_eval_hint:
            return n / dt, cores, n, dt
        n = int(min(n_eval_hint, max(2 * n, n * 0.5 * t_budget / max(dt, 1e-3))))


def oracle_reference(wl, steps, k: int, seed: int = 1):
    """The oracle's field at k random targets (seeded) at each of `steps`: (indices, array [steps][k])."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = rng.choice(wl.M, min(k, wl.M), replace=False)
    ev = np.array([[wl.src_xy[i, 0], wl.src_xy[i, 1], n * wl.dt] for n in steps for i in idx])
    ref = oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"]).reshape(len(steps), -1)
    return idx, ref


def accuracy(r: dict, idx, ref) -> dict:
    """Relative L2 error per kept step on the sampled targets, and the relative max-norm error."""
    got = r["kept"][:, idx]
    l2 = [float(np.linalg.norm(g - f) / np.linalg.norm(f)) for g, f in zip(got, ref)]
    mx = [float(np.max(np.abs(g - f)) / np.max(np.abs(f))) for g, f in zip(got, ref)]
    return {"rel_l2_vs_oracle": max(l2), "per_step": dict(zip(map(str, r["kept_steps"]), l2)),
            "rel_max_vs_oracle": max(mx), "targets": int(len(idx)), "steps": r["kept_steps"]}


def roofline(r: dict, M: int, Mt: int, fp64: bool) -> tuple[dict, dict]:
    peaks = measured_peaks()
    model = part_model(r["info"], M, Mt, fp64)
    alu_peak = peaks["fp64_tflops"] if fp64 else peaks["fp32_tflops"]
    parts = r.get("parts", {})
    per = {}
    for name, (ms, cnt) in parts.items():
        if cnt == 0:
            continue
        e = {"ms_per_launch": ms / cnt, "launches": cnt}
        if name in model:
            b, f = model[name]["bytes"], model[name]["flops"]
            t = ms / cnt * 1e-3
            e["GB/s"] = b / t / 1e9
            e["TFLOP/s"] = f / t / 1e12
            tb, tf = b / (peaks["hbm_gbs"] * 1e9), f / (alu_peak * 1e12)
            e["bound"] = "hbm" if tb >= tf else "alu"
        per[name] = e
    ours = {k: v for k, v in per.items() if k in model and not k.startswith("fft")}  # our kernels, not cuFFT's
    dom = max(ours, key=lambda k: ours[k]["ms_per_launch"] * ours[k]["launches"]) if ours else None
    roof = None
    if dom:
        e = ours[dom]
        traffic = None
        tj = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tj):
            with open(tj) as f:
                tr = json.load(f)
            key = f"{dom}:{'fp64' if fp64 else 'mixed'}:{r['workload']}"
            hkind = dom
            if dom == "local" and r["info"].get("local_form") == 2:
                key += ":factored"
                hkind = "local_factored"
            elif dom == "local":  # per variant (the autotuner may pick any of the bit-identical forms)
                key += f":v{r['info'].get('local_variant')}"
            ent = tr.get(key, {})
            if ent.get("source_hash") == source_hash(hkind):
                traffic = ent["bytes_per_launch"]
        if e["bound"] == "hbm":
            roof = {"kernel": dom, "bound": "hbm", "achieved": round(e["GB/s"], 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(e["GB/s"] / peaks["hbm_gbs"], 4), "traffic": traffic,
                    "peak_source": peaks["source"]}
        else:
            roof = {"kernel": dom, "bound": "alu", "achieved": round(e["TFLOP/s"], 4), "peak": round(alu_peak, 3),
                    "unit": "TFLOP/s", "frac": round(e["TFLOP/s"] / alu_peak, 4), "traffic": traffic,
                    "peak_source": peaks["alu_source"] + (" FP64" if fp64 else " FP32")}
    return roof, per


def parts_roofline(per: dict, fp64: bool) -> dict:
    """Each timed part against its own bound (algorithmic bytes / flops per launch over its
    event-timed launch, in sequence): HBM against the measured copy bandwidth, ALU against the
    FP64 (FP64 path) or FP32 FMA peak."""
    peaks = measured_peaks()
    alu = peaks["fp64_tflops"] if fp64 else peaks["fp32_tflops"]
    out = {}
    for k, e in per.items():
        if "bound" not in e:
            continue
        if e["bound"] == "hbm":
            out[k] = {"bound": "hbm", "GB/s": round(e["GB/s"], 1), "frac": round(e["GB/s"] / peaks["hbm_gbs"], 3)}
        else:
            out[k] = {"bound": "alu", "TFLOP/s": round(e["TFLOP/s"], 4), "frac": round(e["TFLOP/s"] / alu, 3)}
    return out


def source_hash(kernel: str = "local") -> str:
    """Hash of the code a kernel is built from, comments and blank lines left out (its counters go
    stale when the code changes)."""
    import hashlib
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2604_07170_gb300", "csrc")
    files = {"local": ("wfp_local_kernels.cuh", "wfp_ptx.h", "wfp_dev.h"),
             "local_factored": ("wfp_local_factored.cuh", "wfp_local_kernels.cuh", "wfp_dev.h", "wfp_local.cu")}.get(
        kernel, ("wfp_step.cu", "wfp_dev.h"))
    for fn in files:
        with open(os.path.join(d, fn)) as f:
            code = re.sub(r"//[^\n]*", "", f.read())
        h.update("\n".join(ln.strip() for ln in code.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def launches_per_step(info: dict, n_self: int) -> int:
    """Kernels of this library per step (cuFFT's own kernels not counted): ingest, local (two in the
    factored form), [self], combine, spread and the band-to-columns transpose (x2 when the lag is
    recomputed), modes, [far], the columns-to-band transpose, interp, tick."""
    lag = bool(info["lag_active"])
    spreads = 2 if (lag and not info["lag_store"]) else 1
    local = 2 if info.get("local_form") == 2 else 1
    far = 1 if (lag and info["far_active"]) else 0
    return 1 + local + (1 if n_self > 0 else 0) + 1 + 2 * spreads + 1 + far + 1 + 1 + 1


def footprint(info: dict) -> dict:
    return {"device_bytes": info["device_bytes"], "local_part": info["bytes_local"], "grid": info["bytes_grid"],
            "history_state": info["bytes_history"], "fft_work": info["bytes_fft_work"]}


def path_record(r: dict, wl, world: int, fp64: bool) -> dict:
    """The figures of one timed path: rate, step time, rooflines, part times, footprint, e2e."""
    roof, parts = roofline(r, wl.M, wl.M, fp64)
    fft_ms = sum(parts.get(k, {}).get("ms_per_launch", 0) * parts.get(k, {}).get("launches", 0)
                 for k in ("fft_type1", "fft_type2"))
    tot_ms = sum(v["ms_per_launch"] * v["launches"] for v in parts.values())
    info = r["info"]
    rec = {"value": world * wl.M * r["K"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / r["K"],
           "timed_steps": [r["n_last"] - r["K"] + 1, r["n_last"]], "roofline": roof,
           "fft_time_share": round(fft_ms / tot_ms, 4) if tot_ms else None,
           "parts_ms_per_step": {k: round(v["ms_per_launch"] * v["launches"] / r["prof_steps"], 5)
                                 for k, v in parts.items()} if "prof_steps" in r else {},
           "parts_roofline": parts_roofline(parts, fp64), "footprint": footprint(info),
           "plan_seconds": round(r["plan_s"], 3), "clocks": r["clocks"],
           "gpu_launches": r["K"] * launches_per_step(info, info["n_self"])}
    if "e2e_s" in r:
        rec["e2e"] = {"value": wl.M * r["e2e_steps"] / r["e2e_s"], "unit": "target-updates/s",
                      "h2d_bytes_per_step": wl.M * 8, "d2h_bytes_per_step": wl.M * 8, "steps": r["e2e_steps"]}
    return rec


def workload_label(wl, precision: str) -> str:
    return (f"{wl.name}: M={wl.M} coincident sources/targets on ellipses in a {wl.meta['box']:g}x"
            f"{wl.meta['box']:g}-wavelength box, dt={wl.dt}, N_t={wl.n_steps}, tol={wl.tol:g}, {precision}")


def drive(args):
    """Step the workload `args.drive` times through the C ABI with host buffers, graphs off, so that a
    profiler sees every kernel as its own launch.  Prints nothing but a completion line."""
    from paper_2604_07170_gb300 import inputs, wfp
    wl = inputs.make(args.config)
    if args.nt:
        wl.n_steps = args.nt
    opts = dict(args.plan_opts)
    opts.setdefault("use_graph", 0)
    plan = wfp.Plan(wl.src_xy, None, wl.dt, wl.n_steps if args.nt else max(wl.n_steps, args.drive), wl.band_limit, wl.tol,
                    precision=0 if args.precision == "fp64" else 1, **opts)
    u = np.empty(wl.M)
    for n0 in range(0, args.drive, 256):
        sig = wl.sigma(n0 + 1, min(args.drive, n0 + 256) + 1)
        for k in range(sig.shape[0]):
            plan.step(sig[k], u)
    plan.close()
    print(f"drove {args.drive} steps of {args.config} ({args.precision})")


def serve(args):
    """Request-server benchmark: a closed batch of all requests (capacity), then the same requests
    arriving as a Poisson stream at a fraction of that capacity (latency percentiles)."""
    import torch
    from paper_2604_07170_gb300 import inputs, wfp
    reqs = inputs.serve_requests(args.serve)
    work = np.array([w.M * w.n_steps for w in reqs], dtype=np.float64)
    torch.cuda.init()
    free_b, _ = torch.cuda.mem_get_info()
    budget = int(0.85 * free_b)
    prec = 0 if args.precision == "fp64" else 1

    def check_steps(w):  # outputs kept for the oracle check: mid-run steps and the last one
        return sorted({max(1, int(0.3 * w.n_steps)), max(1, int(0.6 * w.n_steps)), w.n_steps})

    rng_c = np.random.default_rng(inputs.SEED0 + 6)
    checked = sorted(rng_c.choice(len(reqs), min(args.serve_check, len(reqs)), replace=False).tolist())

    def run(arrivals, keep=()):
        sv = wfp.Server(budget, args.max_active, precision=prec, **args.plan_opts)
        ids = [None] * len(reqs)
        t0 = time.perf_counter()
        nxt = 0
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            while True:
                now = time.perf_counter() - t0
                while nxt < len(reqs) and arrivals[nxt] <= now:
                    w = reqs[nxt]
                    outs = check_steps(w) if nxt in keep else None
                    ids[nxt] = sv.submit(w.src_xy, w.params, w.dt, w.n_steps, w.band_limit, w.tol, out_steps=outs)
                    nxt += 1
                a, p = sv.tick()
                if a == 0 and p == 0:
                    if nxt == len(reqs):
                        break
                    time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
        st = [sv.query(i) for i in ids]
        kept = {k: sv.result(ids[k]) for k in keep if st[k]["state"] == wfp.REQ_DONE}
        sv.close()
        bad = [i for i, q in enumerate(st) if q["state"] != wfp.REQ_DONE]
        if bad:
            raise RuntimeError(f"requests failed: {bad}")
        lat = np.array([q["t_done"] - q["t_submit"] for q in st])
        wait = np.array([q["t_admit"] - q["t_submit"] for q in st])
        build = np.array([q["t_active"] - q["t_admit"] for q in st])
        span = max(q["t_done"] for q in st) - min(q["t_submit"] for q in st)
        return lat, wait, span, clk.summary(), build, kept

    lat_b, _, span_b, _, build_b, _ = run(np.zeros(len(reqs)))
    cap = work.sum() / span_b
    lam = args.serve_load * cap / work.mean()
    rng = np.random.default_rng(inputs.SEED0 + 5)
    arr = np.cumsum(rng.exponential(1.0 / lam, len(reqs)))
    arr -= arr[0]
    lat, wait, span, clocks, build, kept = run(arr, checked)
    # a few random requests against the oracle at three of their steps, on a bounded sample of targets;
    # error per step relative to max(|u_n|, f max_m |u_m|) as in the parity tests (f = 0.01 FP64, 0.1 mixed)
    checks = []
    if not args.no_cpu:
        import oracle
        floor_f = 1e-2 if prec == 0 else 1e-1
        for k in checked:
            w = reqs[k]
            steps = check_steps(w)
            rng_t = np.random.default_rng(inputs.SEED0 + 7 + k)
            order = rng_t.permutation(w.M)
            n_t = min(8, w.M)
            t0 = time.perf_counter()

            def ref_at(idx):
                ev = np.array([[w.src_xy[i, 0], w.src_xy[i, 1], n * w.dt] for n in steps for i in idx])
                return oracle.field(w.src_xy, w.params, ev, r_coinc=1e-12 * w.meta["box"]).reshape(len(steps), -1)

            ref = ref_at(order[:n_t])
            per = (time.perf_counter() - t0) / n_t
            more = int(min(100, w.M, 30.0 / max(per, 1e-6))) - n_t  # up to 100 targets, ~30 s a request
            if more > 0:
                ref = np.concatenate([ref, ref_at(order[n_t:n_t + more])], axis=1)
                n_t += min(more, w.M - n_t)
            idx = order[:n_t]
            got = kept[k][:, idx]
            norms = np.linalg.norm(ref, axis=1)
            e = np.linalg.norm(got - ref, axis=1) / np.maximum(norms, floor_f * norms.max())
            checks.append({"request": int(k), "M": w.M, "N_t": w.n_steps, "box": round(w.meta["box"], 2),
                           "targets": int(n_t), "steps": steps, "rel_l2_vs_oracle": [float(x) for x in e],
                           "field_norm_rel_to_peak": [float(x) for x in norms / norms.max()]})
    line = {
        "metric": "serving target-updates/s and request latency (Poisson arrivals)",
        "value": work.sum() / span, "unit": "target-updates/s", "n_gpus": 1, "steps": len(reqs), "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == 0 else "f64-state/f32",
        "data": "synthetic request mix (seeded ellipse geometry, Gaussian-sinusoid signals generated on the device)",
        "config": {"workload": f"{len(reqs)} requests: M log-uniform 1e3..1e5, N_t uniform 500..4000, box 10..100, "
                               f"tol 1e-6, {args.precision}",
                   "arrival_rate_per_s": lam, "offered_load": args.serve_load, "hbm_budget_bytes": budget,
                   "max_active": args.max_active},
        "batch_capacity": {"value": cap, "unit": "target-updates/s", "makespan_s": span_b},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "plan_build_s": {"p50": float(np.percentile(build, 50)), "max": float(build.max()), "sum": float(build.sum())},
        "makespan_s": span, "clocks": clocks,
        "oracle_checks": checks,
    }
    print(json.dumps(line))


def main(argv=None):
    args = parse(argv)
    if args.drive:
        return drive(args)
    if args.serve:
        return serve(args)
    dist, rank, world = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
        return
    import torch
    from paper_2604_07170_gb300 import inputs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    measure_alu_peaks()
    wl = inputs.make(args.config, seed_offset=rank)
    K, Wm = args.steps, args.warmup
    keep = min(2, K)
    tend = TIMED_END.get(args.config, 0)
    fp64 = args.precision == "fp64"
    r = measure(wl, args.precision, K, Wm, args.e2e_steps, args.profile_steps, keep, dev, dist, args.plan_opts, tend)
    other = "mixed" if fp64 else "fp64"
    rb = None
    if not args.no_beside:
        rb = measure(wl, other, K, Wm, min(args.e2e_steps, 20), min(args.profile_steps, 10), keep, dev, dist,
                     args.plan_opts, tend)
    subs = {}
    wl2 = None
    if args.sub and args.sub != args.config:
        wl2 = inputs.make(args.sub, seed_offset=rank)
        for prec in ("fp64", "mixed"):
            subs[prec] = measure(wl2, prec, max(K, 200), Wm, 0, 50, keep, dev, dist, args.plan_opts,
                                 TIMED_END.get(args.sub, 0))
    if rank != 0:
        return
    rec = path_record(r, wl, world, fp64)
    info = r["info"]
    line = {
        "metric": METRIC,
        "value": rec["value"],
        "unit": "target-updates/s",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": rec["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32+f64 (mixed)",
        "data": "synthetic (seeded ellipse geometry, Gaussian-sinusoid signals)",
        "config": {"workload": workload_label(wl, args.precision),
                   "timed_steps": rec["timed_steps"],
                   "l2": "inputs larger than L2 (%.2f GB of algorithmic bytes per step across the parts)" % (
                       sum(v["bytes"] for v in part_model(info, wl.M, wl.M, fp64).values()) / 1e9),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "W": info["W"], "p": info["p"], "L": info["L"], "N_modes_half": info["n_modes"],
                   "nf": info["nf"], "nb": info["nb"], "n_pairs": info["n_pairs"], "n_lambda": info["n_lambda"],
                   "plan_seconds": rec["plan_seconds"], "footprint": rec["footprint"],
                   "upsampfac": round(info["upsampfac"], 4), "kernel_width": info["kernel_width"],
                   "lag_active": info["lag_active"], "lag_store": info["lag_store"],
                   "local_form": info["local_form"], "local_nc": info["local_nc"],
                   "local_variant": info["local_variant"], "spread_tile": info["spread_tile"],
                   "spread_chunk": info["spread_chunk"], "n_self_soe": info["n_self_soe"],
                   "step_order": "serial" if info["step_order"] == 2 else "concurrent",
                   "plan_opts": args.plan_opts},
        "clocks": rec["clocks"],
        "gpu_launches": rec["gpu_launches"],
        "roofline": rec["roofline"],
        "fft_time_share": rec["fft_time_share"],
        "parts_ms_per_step": rec["parts_ms_per_step"],
        "parts_roofline": rec["parts_roofline"],
        "alu_peaks_tflops": {"fp64_derived": round(FP64_PEAK_DERIVED, 4), "fp32_derived": round(FP32_PEAK_DERIVED, 2),
                             "fp64_fma_loop": round(_ALU.get("fp64", 0.0), 4),
                             "fp32_fma_loop": round(_ALU.get("fp32", 0.0), 2),
                             "note": "roofline ALU peaks are the derived ones; the measured FMA loop is a lower bound"},
    }
    if "e2e" in rec:
        line["e2e"] = rec["e2e"]
    if rb is not None:
        line[other] = path_record(rb, wl, world, not fp64)
        line[other]["speedup_of_" + args.precision] = (line["value"] / line[other]["value"] if not fp64
                                                      else line[other]["value"] / line["value"])
    if subs:
        line["sub"] = {"workload": workload_label(wl2, "fp64 and mixed")}
        for prec, rs in subs.items():
            line["sub"][prec] = path_record(rs, wl2, world, prec == "fp64")
    if not args.no_cpu:
        try:
            rate, cores, n_ev, dt = cpu_oracle_rate(wl, 4096, 20.0, r["n_last"])
            line["cpu_baseline"] = {"value": rate, "unit": "target-updates/s", "cores": cores, "kind": "oracle",
                                    "sample": f"{n_ev} random targets of {args.config} at step {r['n_last']} "
                                              f"(exact retarded field by quadrature), {dt:.1f} s"}
            idx, ref = oracle_reference(wl, r["kept_steps"], args.accuracy_targets)
            line["accuracy"] = accuracy(r, idx, ref)
            if rb is not None:
                if rb["kept_steps"] != r["kept_steps"]:
                    idx, ref = oracle_reference(wl, rb["kept_steps"], args.accuracy_targets)
                line[other]["accuracy"] = accuracy(rb, idx, ref)
            for prec, rs in subs.items():
                i2, ref2 = oracle_reference(wl2, rs["kept_steps"], args.accuracy_targets)
                line["sub"][prec]["accuracy"] = accuracy(rs, i2, ref2)
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"error": str(e)}
    print(json.dumps(line))


def run_reference(args, rank, world, dist):
    """The FP64 CPU oracle as the reference arm, rank 0 only: the same workload, at the steps our
    arm times, on a bounded sample of targets per step."""
    if rank != 0:
        return
    import oracle
    from paper_2604_07170_gb300 import inputs
    wl = inputs.make(args.config)
    cores = oracle.num_threads()
    if args.config in TIMED_END:  # the window our arm times
        last = TIMED_END[args.config]
        steps = np.clip(np.arange(last - args.steps - args.warmup + 1, last + 1), 1, wl.n_steps)
    else:  # workloads timed in their lagged regime: steps spread over the second half of the run
        steps = np.linspace(wl.n_steps // 2, wl.n_steps, args.steps + args.warmup).astype(int)
    # size each step's sample so that warmup + steps stay within ~2 minutes
    rng = np.random.default_rng(0)
    probe = max(cores, 8)
    idx = rng.choice(wl.M, probe, replace=False)
    ev = np.column_stack([wl.src_xy[idx], np.full(probe, steps[-1] * wl.dt)])
    t0 = time.perf_counter()
    oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"])
    per_eval = (time.perf_counter() - t0) / probe
    S = int(max(1, min(wl.M, 120.0 / len(steps) / per_eval)))
    tot_t, tot_n = 0.0, 0
    for i, n in enumerate(steps):
        idx = rng.choice(wl.M, S, replace=False)
        ev = np.column_stack([wl.src_xy[idx], np.full(S, n * wl.dt)])
        t0 = time.perf_counter()
        oracle.field(wl.src_xy, wl.params, ev, r_coinc=1e-12 * wl.meta["box"])
        if i >= args.warmup:
            tot_t += time.perf_counter() - t0
            tot_n += S
    value = tot_n / tot_t
    sample = f"{S} random targets per step over steps {int(steps[args.warmup])}..{int(steps[-1])} of {args.config}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "target-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded ellipse geometry, Gaussian-sinusoid signals)",
            "config": {"workload": workload_label(wl, "fp64 (CPU oracle)")},
            "cpu_baseline": {"value": value, "unit": "target-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "target-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
