"""Benchmark: converged spectra/s of the grouped fit on one GB300 per rank.

One step = one pass of the whole hot path over one batch: lasp_fit_batch
(basis contraction, broadening, continuum WLS, loss, adjoint, grouped Adam
with per-spectrum stop rules) followed by lasp_errors (stage-9 covariance)
for 4096 LAMOST-like spectra x 3909 pixels, K = 26, Legendre degree 6,
SNR 5-100, 5% masked pixels, at most 500 Adam steps (paper defaults lr 0.1,
tol 1e-5, window 50).  value = spectra that stopped by rule 2 or 3 per
second.  Inputs (144 MB) exceed L2 and L2 is also flushed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU: replicas (each rank fits its own batch; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lasp_synth as S  # noqa: E402

WORKLOAD = "lamost4096x3909_k26_d6_snr5-100_mask5pct_max500"
METRIC = "converged spectra/s at fixed param tolerance, plain vs mixed; p50/p99 latency"
UNIT = "spectra/s"
N_SPEC, MAX_STEPS, DEG = 4096, 500, 6
TOL = np.array([1.0, 0.005, 0.005, 0.1])      # Teff K, log g, [Fe/H], RV km/s
FP32_LANES_PER_SM, N_SM = 128, 152
# The batch fit's main kernel on this workload (four spectra per CTA, after
# fit_prep_kernel) and the DRAM bytes of one launch, from one ncu capture of
# the current kernel source (reset to None whenever the kernel changes until it
# is captured again): it reads the prepared y, W rows (8 B a pixel) and the
# table, and writes the results.
FIT_KERNEL = "fit_multi_kernel<256,6,4,0>"
FIT_TRAFFIC_BYTES = 130_388_736 + 6_808_576


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 65536-spectra mixed-precision run")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision, curvature-aware and piecewise entries")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-only", action="store_true",
                    help="only the LAMOST-only served drain (burst, one-shot comparison and a "
                         "lasp_profile breakdown of its ticks), printed as one JSON line")
    ap.add_argument("--kernels-only", action="store_true",
                    help="only the per-kernel pass (lasp_profile) on the 4096-spectrum batch: one FP32 "
                         "fit, the stage-9 errors at both normal-equation levels, one curvature-aware "
                         "and one split-TF32 fit (for an ncu launch list of every kernel)")
    ap.add_argument("--cpu-sample", type=int, default=2048,
                    help="spectra in the oracle's timed CPU sample (about 16 s on 16 cores); "
                         "the reference arm times an eighth of it per step")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace('.', '').isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_flops(theta, steps, grid, K=26, D=DEG):
    """FLOPs of the fused step per spectrum, summed over the evaluations each
    spectrum ran (steps + 1), with its kernel width h = ceil(|mu| + 5 sigma)
    at the result.  Per spectrum-step: 2 K n_model (Eq. 1) + 2 T p (Eq. 5)
    + 4 T p (kernel-parameter adjoint) + 2 T n_model (transposed
    correlation) + 2 K n_model (basis adjoint) + p (2 (D+1)(D+2)/2 + 2 (D+1)
    + 4 D + 2 (D+1) + 8) (Legendre, normal equations, continuum, residual)."""
    p, nm = grid.n_pix, grid.n_model
    mu = np.abs(theta[:, 3]) / grid.kms_per_px
    sg = theta[:, 4] / grid.kms_per_px
    T = 2 * np.ceil(mu + 5 * sg) + 1
    nb = D + 1
    per_px = 2 * nb * (nb + 1) // 2 + 2 * nb + 4 * D + 2 * nb + 8
    per = 4 * K * nm + 6 * T * p + 2 * T * nm + per_px * p
    return float((per * (steps + 1)).sum())


def err_flops(theta, grid, K=26, D=DEG):
    """FLOPs of the stage-9 kernel per spectrum: F' and its three basis
    derivatives (4 contractions, 8 K n_model), six tap correlations (12 T p),
    and per pixel three Legendre evaluations, the normal equations, the five
    continuum sensitivities, the Jacobian row and J^T J."""
    p, nm = grid.n_pix, grid.n_model
    mu = np.abs(theta[:, 3]) / grid.kms_per_px
    sg = theta[:, 4] / grid.kms_per_px
    T = 2 * np.ceil(mu + 5 * sg) + 1
    nb = D + 1
    nv = nb * (nb + 1) // 2 + nb
    per_px = 3 * 4 * D + 2 * nv + 2 * (5 * nb + 1) + 5 * (2 * nb + 3) + 30 + 8
    return float((8 * K * nm + 12 * T * p + per_px * p).sum())


def lm_flops(theta, steps, grid, K=26, D=DEG):
    """Estimated FLOPs of the curvature-aware fit: per accepted step one full
    evaluation (F' and three basis derivatives, the tap correlations, the
    Jacobian and J^T J) and one S-only trial (one contraction, one correlation,
    normal equations and residual).  The kernel does not report its trial
    count, so this assumes one trial per accepted step."""
    p, nm = grid.n_pix, grid.n_model
    mu = np.abs(theta[:, 3]) / grid.kms_per_px
    sg = theta[:, 4] / grid.kms_per_px
    T = 2 * np.ceil(mu + 5 * sg) + 1
    nb = D + 1
    nv = nb * (nb + 1) // 2 + nb
    full = 8 * K * nm + 10 * T * p + 2 * T * nm + (3 * 4 * D + 2 * nv + 2 * (5 * nb + 1) + 5 * (2 * nb + 3) + 40) * p
    trial = 2 * K * nm + 2 * T * p + (4 * D + 2 * nv + 2 * nb + 8) * p
    return float(((full + trial) * (steps + 1)).sum())


def kernel_rooflines(torch, lasp, ip, g_in, grid, theta_np, steps_np, pk, alu_peak):
    """Each kernel's own device time (lasp_profile: CUDA events around the
    kernel on its stream, one untimed pass of each form after the timed
    region) against its algorithmic cost and its roof: FP32 ALU FLOPs for the
    per-spectrum kernels, bytes for the memory-bound ones."""
    hbm = pk["hbm_gbs"]
    p, nm = grid.n_pix, grid.n_model
    n = g_in[0].shape[0]
    ldp, ldf = (p + 15) & ~15, (nm + 15) & ~15
    rows = []

    def row(name, prof, bound, per_launch, unit_note):
        if name not in prof:
            return
        launches, ms = prof[name]
        t = ms / launches / 1e3
        if bound == "hbm":
            ach, peak, unit = per_launch / t / 1e9, hbm, "GB/s"
        else:
            ach, peak, unit = per_launch / t / 1e12, alu_peak, "TFLOP/s"
        rows.append({"kernel": name, "launches": launches, "ms_per_launch": ms / launches, "bound": bound,
                     "algorithmic_per_launch": per_launch, "achieved": ach, "peak": peak, "unit": unit,
                     "frac": ach / peak, "cost": unit_note})

    opts = dict(max_steps=MAX_STEPS, legendre_deg=DEG)
    lasp.profile(True)
    try:
        lasp.profile_read()
        o = ip.fit(*g_in, **opts)
        ip.errors(*g_in[:3], o["theta"], with_cov=False, **opts)
        ip.errors(*g_in[:3], o["theta"], with_cov=False, fp64_normal_eq=2, **opts)
        prof = lasp.profile_read()
        th = o["theta"].double().cpu().numpy()
        st = o["steps"].cpu().numpy()
        row("fit_prep_kernel", prof, "hbm", n * p * 9 + n * ldp * 8,
            "reads flux, ivar, mask (9 B/px), writes the y, W rows (8 B/px)")
        row("fit_multi_kernel", prof, "alu", algorithmic_flops(th, st, grid),
            "the fused step's FLOPs per spectrum-step x (steps + 1), summed")
        row("errors_kernel", prof, "alu", err_flops(th, grid), "stage-9 FLOPs per spectrum, summed")
        row("errors_kernel<fp64>", prof, "alu", err_flops(th, grid),
            "as errors_kernel; sums across the CTA and the 7x7 solves in FP64")
        # the Clean variant of the fused fit (the Clean update compiled in), Clean on
        oc = ip.fit(*g_in, clean=1, **opts)
        prof = lasp.profile_read()
        row("fit_multi_kernel<clean>", prof, "alu",
            algorithmic_flops(oc["theta"].double().cpu().numpy(), oc["steps"].cpu().numpy(), grid),
            "the fused step's FLOPs (Clean updates not counted), Clean on")
        lo = dict(max_steps=100, tol=1e-10, legendre_deg=DEG, optimizer="lm")
        ol = ip.fit(*g_in, **lo)
        prof = lasp.profile_read()
        row("lm_kernel", prof, "alu",
            lm_flops(ol["theta"].double().cpu().numpy(), ol["steps"].cpu().numpy(), grid),
            "estimated: one full evaluation and one damped trial per accepted step")
        om = ip.fit(*g_in, precision="tf32x3", fp64_normal_eq=1, **opts)
        prof = lasp.profile_read()
        thm = om["theta"].double().cpu().numpy()
        spec_steps = float((om["steps"].cpu().numpy() + 1).sum())
        if "k1_interp" in prof:
            L = prof["k1_interp"][0]
            per_step = algorithmic_flops(thm, om["steps"].cpu().numpy(), grid) / spec_steps
            row("k0_prep", prof, "hbm", n * p * 9 + n * ldp * 8, "reads the batch, writes y, W rows")
            row("k1_interp", prof, "hbm", spec_steps * 4 * ldf / L,
                "writes F' (4 B a model pixel) of every active spectrum")
            row("k2_rest", prof, "alu", spec_steps * (per_step - 2 * 26 * nm) / L,
                "the step's FLOPs without the forward contraction, per active spectrum")
            row("k3_back", prof, "hbm", spec_steps * 8 * ldf / L,
                "reads the dF' operand images (TF32 hi and lo, 8 B a model pixel)")
            row("k4_adam", prof, "hbm", spec_steps * (60 * 2 + 4 * 32 * 4 + 3 * 128 * 4 + 16) / L,
                "Adam state, split-K partials of dphi and the next step's taps")
    finally:
        lasp.profile(False)
    return rows


def aggregate(dist, torch, device, ms, conv):
    """Max step time and total converged count over ranks (replicas)."""
    if dist is None:
        return ms, conv
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([int(conv)], device=device, dtype=torch.int64)
    dist.all_reduce(c)
    return float(t.item()), int(c.item())


def served_stream(torch, lasp, grids, tables, seconds=2.0, loads=(0.5, 0.8, 0.95), burst=6144,
                  native=True, repeats=1, **fit_opts):
    """Continuous batching of a request mix over the given grids (equal
    shares; random masks 0-20%, SNR 5-100).  The saturated rate is the drain
    rate of a burst; then Poisson arrivals at fractions of it, `repeats`
    windows of `seconds` each per load.  Arrival times are drawn before the
    window; a producer thread submits every arrival that is due, per lane in
    one submit_many call of consecutive pool rows.  Latency: scheduled
    arrival -> result on host (the producer's lag behind the schedule plus
    the scheduler's submit -> result time).  With one grid, the one-shot batch
    fit of the same burst is timed too."""
    import threading
    from paper_2512_24840_gb300.server import Server
    from paper_2512_24840_gb300.server import DevicePool, NativeServer
    ips = {g.name: lasp.Interp.from_grid(g, tables[g.name], S.EXPS, S.BASIS_LO, S.BASIS_HI,
                                         S.BOX_LO, S.BOX_HI) for g in grids}
    pool = {}
    dev = torch.device("cuda")
    for k, g in enumerate(grids):
        d = S.draw_batch(g, 1024, S.SPECTRA_SEED + 5 + k, snr=(5, 100), mask_frac=0.0, mask_frac_max=0.2)
        model = ips[g.name].forward(torch.tensor(d["truth"], dtype=torch.float32, device=dev),
                                    torch.tensor(d["b_true"], dtype=torch.float32, device=dev))
        flux, ivar = S.finish_obs(model.double().cpu().numpy(), d)
        pool[g.name] = (np.ascontiguousarray(flux, np.float32), np.ascontiguousarray(ivar, np.float32),
                        np.ascontiguousarray(d["good"], np.uint8), np.asarray(d["theta0"], np.float32))
    prec = fit_opts.get("precision", "fp32")
    budget = 2 * burst * max(DevicePool.bytes_per_slot(g.n_pix, DEG, prec) for g in grids)
    cls = NativeServer if native else Server
    srv = cls.on_device(ips, hbm_budget_bytes=budget, chunk=25, max_steps=MAX_STEPS, **fit_opts)
    names = [g.name for g in grids]
    rng = np.random.default_rng(7)

    def submit(n):
        for _ in range(n):
            lane = names[rng.integers(len(names))]
            f, iv, gd, th = pool[lane]
            i = rng.integers(len(f))
            srv.submit(lane, f[i], iv[i], gd[i], th[i])

    # the native scheduler hands back each tick's finished fits as one array
    arrays = native
    drain = srv.run_until_idle_arrays if arrays else srv.run_until_idle
    tick = srv.tick_arrays if arrays else srv.tick

    submit(512)                                   # warm-up
    drain()
    sats = []
    for _ in range(3):                            # the median of three burst drains
        submit(burst)
        t0 = time.perf_counter()
        res = drain()
        sats.append(len(res) / (time.perf_counter() - t0))
    sat = statistics.median(sats)
    one_shot = tick_profile = None
    if len(grids) == 1:
        # the same kind of burst fitted in one batch call, inputs resident on the device
        g = grids[0]
        f, iv, gd, th = pool[g.name]
        idx = np.random.default_rng(8).integers(len(f), size=burst)
        args = [torch.tensor(f[idx], device=dev), torch.tensor(iv[idx], device=dev),
                torch.tensor(gd[idx], device=dev), torch.tensor(th[idx], device=dev)]
        o = ips[g.name].fit(*args, max_steps=MAX_STEPS, **fit_opts)
        torch.cuda.synchronize()
        shots = []
        for _ in range(3):
            t1 = time.perf_counter()
            o = ips[g.name].fit(*args, out=o, max_steps=MAX_STEPS, **fit_opts)
            torch.cuda.synchronize()
            shots.append(burst / (time.perf_counter() - t1))
        one_shot = statistics.median(shots)
        # where a tick's time goes: the same burst drained again with lasp_profile on
        # (each timed kernel and copy waits for its closing event, so this drain is slower)
        submit(burst)
        lasp.profile(True)
        lasp.profile_read()
        n_ticks, tp0 = 0, time.perf_counter()
        try:
            while srv.pending():
                tick()
                n_ticks += 1
        finally:
            prof = lasp.profile_read()
            lasp.profile(False)
        wall_p = (time.perf_counter() - tp0) * 1e3
        dev_ms = sum(v[1] for v in prof.values())
        tick_profile = {"ticks": n_ticks, "wall_ms": wall_p, "device_ms_total": dev_ms,
                        "device_frac_of_wall": dev_ms / wall_p,
                        "device_ms": {k: [v[0], round(v[1], 3)] for k, v in sorted(prof.items())}}
    levels = []
    for load in loads:
        rate = load * sat
        wins = []
        for rep in range(repeats):
            n_arr = int(rate * seconds * 1.2) + 64
            t_arr = np.cumsum(rng.exponential(1.0 / rate, size=n_arr))
            lane_arr = rng.integers(len(names), size=n_arr)
            stop = threading.Event()
            done, rid_parts, lag_parts = [], [], []
            cur = {nm: int(rng.integers(len(pool[nm][0]))) for nm in names}

            def producer():
                i = 0
                while not stop.is_set() and i < n_arr:
                    now = time.perf_counter() - t0
                    j = int(np.searchsorted(t_arr, now, side="right"))
                    if j <= i:
                        time.sleep(min(t_arr[i] - now, 0.001))
                        continue
                    for k, nm in enumerate(names):
                        due = np.nonzero(lane_arr[i:j] == k)[0] + i
                        f, iv, gd, th = pool[nm]
                        while len(due):
                            c = cur[nm]
                            m = min(len(due), len(f) - c)       # consecutive rows, split at the wrap
                            t_call = time.perf_counter() - t0
                            rid_parts.append(srv.submit_many(nm, f[c:c + m], iv[c:c + m], gd[c:c + m],
                                                             th[c:c + m]))
                            lag_parts.append(t_call - t_arr[due[:m]])
                            cur[nm] = (c + m) % len(f)
                            due = due[m:]
                    i = j

            prod = threading.Thread(target=producer, daemon=True)
            t0 = time.perf_counter()
            prod.start()
            while time.perf_counter() - t0 < seconds:
                done.append(tick()) if arrays else done.extend(tick())
                if not srv.pending():
                    time.sleep(0.0005)
            stop.set()
            prod.join()
            t_prod = time.perf_counter() - t0
            done.append(drain()) if arrays else done.extend(drain())
            elapsed = time.perf_counter() - t0
            rids = np.concatenate(rid_parts) if rid_parts else np.zeros(0, np.int64)
            lags = np.concatenate(lag_parts) if lag_parts else np.zeros(0)
            if arrays:
                a = np.concatenate(done)
                tags = a["tag"].astype(np.int64)
                conv = int(((a["status"] & 3) != 0).sum())
                in_sched = (a["t_done_ns"] - a["t_submit_ns"]) * 1e-9
            else:
                tags = np.array([r.rid for r in done], dtype=np.int64)
                conv = sum(1 for r in done if r.status & 3)
                in_sched = np.array([r.t_done - r.t_submit for r in done])
            n_done = len(tags)
            pos = np.searchsorted(rids, tags)
            assert n_done == len(rids) and np.array_equal(rids[np.minimum(pos, len(rids) - 1)], tags)
            lat = (lags[pos] + in_sched) * 1e3
            pct = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "submit_lag_p99_ms": float(np.percentile(lags, 99) * 1e3)} if n_done else {}
            wins.append({"served_per_s": n_done / elapsed, "converged_per_s": conv / elapsed,
                         "arrivals_per_s": len(rids) / t_prod, "n": n_done, **pct})
        lv = {"load": load, "offered_per_s": rate}
        for key in ("arrivals_per_s", "served_per_s", "converged_per_s", "p50_ms", "p99_ms",
                    "submit_lag_p99_ms"):
            vals = sorted(w[key] for w in wins if w.get(key) is not None)
            if vals:
                lv[key] = statistics.median(vals)
                if repeats > 1:
                    lv[key + "_min_max"] = [vals[0], vals[-1]]
        lv["n"] = sum(w["n"] for w in wins)
        lv["windows"] = f"{repeats} x {seconds:.0f} s"
        levels.append(lv)
    slots = srv.slots
    srv.close()
    out = {"scheduler": "native (lasp_server_*)" if native else "python (server.Server over lasp_slots_*)",
           "precision": prec + ("+float-float normal equations" if fit_opts.get("fp64_normal_eq") else ""),
           "saturated_per_s": sat, "saturated_per_s_runs": sats, "chunk_steps": 25, "lanes": names,
           "slots": slots, "levels": levels}
    if one_shot:
        out["one_shot_same_spectra_per_s"] = one_shot
        out["saturated_vs_one_shot"] = sat / one_shot
        out["tick_profile"] = tick_profile
    return out


def make_inputs(rank, torch, lasp, grid, C):
    """Batch of N_SPEC spectra; the noise-free model comes from the library's
    forward model, noise and masks from the generator."""
    d = S.draw_batch(grid, N_SPEC, S.SPECTRA_SEED + 1 + 1000 * rank, snr=(5, 100), mask_frac=0.05)
    ip = lasp.Interp.from_grid(grid, C, S.EXPS, S.BASIS_LO, S.BASIS_HI, S.BOX_LO, S.BOX_HI)
    dev = torch.device("cuda")
    model = ip.forward(torch.tensor(d["truth"], dtype=torch.float32, device=dev),
                       torch.tensor(d["b_true"], dtype=torch.float32, device=dev))
    flux, ivar = S.finish_obs(model.double().cpu().numpy(), d)
    return ip, d, flux, ivar


def run_ours(args):
    import torch
    from paper_2512_24840_gb300 import lasp

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lasp.load()
    grid = S.LAMOST
    C = S.make_table(grid)
    ip, d, flux, ivar = make_inputs(rank, torch, lasp, grid, C)
    dev = torch.device("cuda")
    g_flux = torch.tensor(flux, device=dev)
    g_ivar = torch.tensor(ivar, device=dev)
    g_good = torch.tensor(d["good"], device=dev)
    g_th0 = torch.tensor(d["theta0"], dtype=torch.float32, device=dev)
    opts = dict(max_steps=MAX_STEPS, legendre_deg=DEG)
    stream = torch.cuda.current_stream()
    if args.served_only:
        if rank == 0:
            r = served_stream(torch, lasp, [S.LAMOST], {S.LAMOST.name: C}, native=True, loads=())
            print(json.dumps({"workload": "served_lamost_only", **r}))
        return
    if args.kernels_only:
        pk, _ = peaks()
        mhz0 = pk.get("sm_max_mhz", 2070.0)
        rows = kernel_rooflines(torch, lasp, ip, [g_flux, g_ivar, g_good, g_th0], grid, None, None, pk,
                                N_SM * FP32_LANES_PER_SM * 2 * mhz0 * 1e6 / 1e12)
        if rank == 0:
            print(json.dumps({"workload": WORKLOAD, "kernels": rows}))
        return
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = None

    def step():
        nonlocal out
        out = ip.fit(g_flux, g_ivar, g_good, g_th0, out=out, **opts)
        e = ip.errors(g_flux, g_ivar, g_good, out["theta"], with_cov=False, **opts)
        return out, e

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    # per-kernel timing of the fit kernel on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    flush_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush_ev[k][0].record(stream)
            flush.fill_(float(k))
            flush_ev[k][1].record(stream)
            ev[k][0].record(stream)
            out = ip.fit(g_flux, g_ivar, g_good, g_th0, out=out, **opts)
            ev[k][1].record(stream)
            ip.errors(g_flux, g_ivar, g_good, out["theta"], with_cov=False, **opts)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    fit_ms = [a.elapsed_time(b) for a, b, c in ev]
    err_ms = [b.elapsed_time(c) for a, b, c in ev]
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    ms = sum(step_ms) / len(step_ms)
    status = out["status"].cpu().numpy()
    steps_np = out["steps"].cpu().numpy()
    theta_np = out["theta"].double().cpu().numpy()
    conv = int(((status & 3) != 0).sum())
    ms, conv_all = aggregate(dist, torch, dev, ms, conv)
    value = conv_all / (ms / 1e3)

    # ---- end to end through the public API from pinned host buffers
    h_flux = torch.tensor(flux).pin_memory()
    h_ivar = torch.tensor(ivar).pin_memory()
    h_good = torch.tensor(d["good"]).pin_memory()
    h_th0 = torch.tensor(d["theta0"], dtype=torch.float32).pin_memory()
    h_theta = torch.empty((N_SPEC, 5)).pin_memory()
    h_sig = torch.empty((N_SPEC, 5)).pin_memory()
    h_status = torch.empty(N_SPEC, dtype=torch.int32).pin_memory()
    bi = sum(t.numel() * t.element_size() for t in (h_flux, h_ivar, h_good, h_th0))
    bo = sum(t.numel() * t.element_size() for t in (h_theta, h_sig, h_status))
    e2e = []
    for k in range(args.warmup + args.steps):
        flush.fill_(0.5)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g_flux.copy_(h_flux, non_blocking=True)
        g_ivar.copy_(h_ivar, non_blocking=True)
        g_good.copy_(h_good, non_blocking=True)
        g_th0.copy_(h_th0, non_blocking=True)
        o2, e2 = step()
        h_theta.copy_(o2["theta"], non_blocking=True)
        h_sig.copy_(e2["sigma"], non_blocking=True)
        h_status.copy_(o2["status"], non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e.append(a.elapsed_time(b))
    e2e_ms = sum(e2e) / len(e2e)
    e2e_conv = int(((h_status.numpy() & 3) != 0).sum())
    e2e_ms, e2e_conv = aggregate(dist, torch, dev, e2e_ms, e2e_conv)

    # ---- mixed precision: grouped tensor-core pipeline (split TF32 and single-pass
    # TF32 contractions, FP64 normal equations), same batch, device-resident inputs
    mixed = {}
    try:
        if not args.no_mixed:
            for prec, ne in (("tf32x3", 1), ("tf32", 1), ("tf32x3", 2), ("fp32", 2)):
                mo = dict(opts, precision=prec, fp64_normal_eq=ne)
                mout = ip.fit(g_flux, g_ivar, g_good, g_th0, **mo)          # warm-up
                torch.cuda.synchronize()
                t_ms = []
                for k in range(max(1, args.steps)):
                    flush.fill_(float(k))
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    mout = ip.fit(g_flux, g_ivar, g_good, g_th0, out=mout, **mo)
                    b.record(stream)
                    torch.cuda.synchronize()
                    t_ms.append(a.elapsed_time(b))
                mst = mout["status"].cpu().numpy()
                mth = mout["theta"].double().cpu().numpy()
                mconv = int(((mst & 3) != 0).sum())
                agree = np.all(np.abs(mth - theta_np)[:, :4] <= np.array([1.0, 0.005, 0.005, 0.1]), axis=1)
                ne_name = {1: "float-float", 2: "fp64"}[ne]
                mixed[f"{prec}+{ne_name}_ne"] = {
                    "value": mconv / (sum(t_ms) / len(t_ms) / 1e3), "unit": UNIT,
                    "fit_ms": sum(t_ms) / len(t_ms), "converged": mconv,
                    "precision": f"{prec} contractions, {ne_name} normal equations",
                    "within_tol_of_fp32_fit_frac": float(agree.mean())}
    except Exception as e:       # a failed extra is reported; the headline still prints
        mixed = {"error": f"{type(e).__name__}: {e}"}

    # ---- the paper's joint loss (one RMS over the group, group stop rules), split TF32
    joint = {}
    try:
        if not args.no_mixed:
            jo = dict(opts, precision="tf32x3", fp64_normal_eq=1, loss_mode="joint")
            jout = ip.fit(g_flux, g_ivar, g_good, g_th0, **jo)
            torch.cuda.synchronize()
            t_ms = []
            for k in range(max(1, args.steps)):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                jout = ip.fit(g_flux, g_ivar, g_good, g_th0, out=jout, **jo)
                b.record(stream)
                torch.cuda.synchronize()
                t_ms.append(a.elapsed_time(b))
            jst = jout["status"].cpu().numpy()
            jconv = int(((jst & 3) != 0).sum())
            jth = jout["theta"].double().cpu().numpy()
            agree = np.all(np.abs(jth - theta_np)[:, :4] <= np.array([1.0, 0.005, 0.005, 0.1]), axis=1)
            joint = {"value": jconv / (sum(t_ms) / len(t_ms) / 1e3), "unit": UNIT,
                     "fit_ms": sum(t_ms) / len(t_ms), "converged": jconv,
                     "group_steps": int(jout["steps"].max().item()),
                     "within_tol_of_separable_fp32_fit_frac": float(agree.mean()),
                     "note": "Eq. 9 read literally: one RMS over the 4096-spectrum group, group stop rules"}
    except Exception as e:       # a failed extra is reported; the headline still prints
        joint = {"error": f"{type(e).__name__}: {e}"}

    # ---- mixed precision at the large configuration: 65536 LAMOST-like spectra,
    # split-TF32 contractions + float-float normal equations; parameter error
    # against the FP64 oracle on a sample of the batch
    mixed_large = {}
    try:
        if not args.no_mixed and not args.no_large:
            _, n_big, off, kw = S.workload("mixed65536")
            db = S.draw_batch(grid, n_big, S.SPECTRA_SEED + off + 1000 * rank, **kw)
            bmodel = torch.empty((n_big, grid.n_pix), device=dev)
            for c0 in range(0, n_big, 8192):
                bmodel[c0:c0 + 8192] = ip.forward(
                    torch.tensor(db["truth"][c0:c0 + 8192], dtype=torch.float32, device=dev),
                    torch.tensor(db["b_true"][c0:c0 + 8192], dtype=torch.float32, device=dev))
            bf, bv = S.finish_obs(bmodel.double().cpu().numpy(), db)
            del bmodel
            bin_ = [torch.tensor(bf, device=dev), torch.tensor(bv, device=dev),
                    torch.tensor(db["good"], device=dev),
                    torch.tensor(db["theta0"], dtype=torch.float32, device=dev)]
            mo = dict(opts, precision="tf32x3", fp64_normal_eq=1)
            bout = ip.fit(*bin_, **mo)
            torch.cuda.synchronize()
            t_ms = []
            for k in range(max(1, min(args.steps, 2))):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                bout = ip.fit(*bin_, out=bout, **mo)
                b.record(stream)
                torch.cuda.synchronize()
                t_ms.append(a.elapsed_time(b))
            bst = bout["status"].cpu().numpy()
            bconv = int(((bst & 3) != 0).sum())
            # the plain FP32 form on the same 65536 spectra
            fout = ip.fit(*bin_, **opts)
            torch.cuda.synchronize()
            f_ms = []
            for k in range(max(1, min(args.steps, 2))):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fout = ip.fit(*bin_, out=fout, **opts)
                b.record(stream)
                torch.cuda.synchronize()
                f_ms.append(a.elapsed_time(b))
            fconv = int(((fout["status"].cpu().numpy() & 3) != 0).sum())
            sample = np.arange(0, n_big, n_big // 512)[:512]
            within = within_fp32 = None
            if not args.no_cpu_baseline:
                from oracle import oracle as O
                M = O.Model(C, S.EXPS, grid.dln, grid.pad, grid.n_pix, DEG, S.BASIS_LO, S.BASIS_HI,
                            S.BOX_LO, S.BOX_HI)
                th0 = np.asarray(db["theta0"][sample], np.float32).astype(np.float64)
                ref = O.fit(M, bf[sample], bv[sample], db["good"][sample], th0,
                            threads=O.lib().orc_max_threads(), max_steps=MAX_STEPS)
                err = np.abs(bout["theta"].double().cpu().numpy()[sample] - ref["theta"])[:, :4]
                within = float(np.all(err <= TOL, axis=1).mean())
                err = np.abs(fout["theta"].double().cpu().numpy()[sample] - ref["theta"])[:, :4]
                within_fp32 = float(np.all(err <= TOL, axis=1).mean())
            mixed_large = {"value": bconv / (sum(t_ms) / len(t_ms) / 1e3), "unit": UNIT,
                           "fit_ms": sum(t_ms) / len(t_ms), "converged": bconv, "n_spectra": n_big,
                           "precision": "tf32x3+float-float normal equations",
                           "within_tol_of_oracle_frac": within,
                           "fp32": {"value": fconv / (sum(f_ms) / len(f_ms) / 1e3), "unit": UNIT,
                                    "fit_ms": sum(f_ms) / len(f_ms), "converged": fconv,
                                    "within_tol_of_oracle_frac": within_fp32},
                           "oracle_sample": f"{len(sample)} spectra (every {n_big // 512}th), FP64 oracle fit"}
            del bin_, bout, fout
    except Exception as e:       # a failed extra is reported; the headline still prints
        mixed_large = {"error": f"{type(e).__name__}: {e}"}

    # ---- curvature-aware step (Levenberg-Marquardt, the paper's outlook): same batch
    lm = {}
    try:
        if not args.no_mixed:
            lo = dict(max_steps=100, tol=1e-10, legendre_deg=DEG, optimizer="lm")
            lout = ip.fit(g_flux, g_ivar, g_good, g_th0, **lo)
            torch.cuda.synchronize()
            t_ms = []
            for k in range(max(1, args.steps)):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lout = ip.fit(g_flux, g_ivar, g_good, g_th0, out=lout, **lo)
                b.record(stream)
                torch.cuda.synchronize()
                t_ms.append(a.elapsed_time(b))
            lst = lout["status"].cpu().numpy()
            lconv = int(((lst & 3) != 0).sum())
            lm = {"value": lconv / (sum(t_ms) / len(t_ms) / 1e3), "unit": UNIT,
                  "fit_ms": sum(t_ms) / len(t_ms), "converged": lconv,
                  "mean_iterations": float(lout["steps"].float().mean()),
                  "loss_vs_adam_median_ratio": float(torch.median(lout["loss"] / out["loss"]).item()),
                  "note": "Levenberg-Marquardt to the least-squares minimum (Gauss-Newton predicted decrease <= 1e-10 S)"}
    except Exception as e:       # a failed extra is reported; the headline still prints
        lm = {"error": f"{type(e).__name__}: {e}"}

    # ---- Clean outlier masking (stage 6, Eq. 8): the same batch with eight
    # cosmic-ray-like three-pixel spikes added to every spectrum; mask updates
    # every 30 steps (at most 11), as the paper's Clean strategy
    clean = {}
    try:
        if not args.no_mixed:
            rs = np.random.default_rng(S.SPECTRA_SEED + 77 + 1000 * rank)
            n_sp = 8
            rows = np.repeat(np.arange(N_SPEC), n_sp)
            cols = rs.integers(0, grid.n_pix - 3, size=N_SPEC * n_sp)
            med = np.median(flux, axis=1)
            amp = (med[rows] * rs.uniform(0.5, 3.0, size=N_SPEC * n_sp)).astype(np.float32)
            spiky = flux.copy()
            for o, f in enumerate((1.0, 0.5, 0.2)):
                np.add.at(spiky, (rows, cols + o), amp * np.float32(f))
            c_flux = torch.tensor(spiky, device=dev)
            co = dict(opts, clean=1)
            cout = ip.fit(c_flux, g_ivar, g_good, g_th0, **co)          # warm-up
            torch.cuda.synchronize()
            t_ms = []
            for k in range(max(1, args.steps)):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                cout = ip.fit(c_flux, g_ivar, g_good, g_th0, out=cout, **co)
                b.record(stream)
                torch.cuda.synchronize()
                t_ms.append(a.elapsed_time(b))
            nout = ip.fit(c_flux, g_ivar, g_good, g_th0, **opts)         # same spiky data, no Clean
            torch.cuda.synchronize()
            cst = cout["status"].cpu().numpy()
            cconv = int(((cst & 3) != 0).sum())
            ref_t = out["theta"][:, 0].cpu().numpy()                       # spike-free fit
            dc = np.abs(cout["theta"][:, 0].cpu().numpy() - ref_t)
            dn = np.abs(nout["theta"][:, 0].cpu().numpy() - ref_t)
            clean = {"value": cconv / (sum(t_ms) / len(t_ms) / 1e3), "unit": UNIT,
                     "fit_ms": sum(t_ms) / len(t_ms), "converged": cconv, "n_spectra": N_SPEC,
                     "mean_steps": float(cout["steps"].float().mean()),
                     "median_abs_dteff_vs_spike_free_fit_K": {"clean": float(np.median(dc)),
                                                              "no_clean": float(np.median(dn))},
                     "workload": "lamost4096x3909 + 8 three-pixel spikes per spectrum, Clean every 30 steps"}
            del c_flux
    except Exception as e:       # a failed extra is reported; the headline still prints
        clean = {"error": f"{type(e).__name__}: {e}"}

    # ---- piecewise Teff-regime emulator (Eq. 1 with f1..f5; 25/26/19-term cold,
    # warm and hot regimes): its own 4096-spectrum batch over Teff 3300-11500 K
    piecewise = {}
    try:
        if not args.no_mixed:
            tabs = S.make_piecewise_tables(grid)
            ipw = lasp.Interp.piecewise(tabs, S.PW_EXPS, grid.n_pix, grid.pad, grid.dln, S.PW_BASIS_LO,
                                        S.PW_BASIS_HI, S.TEFF_BLEND, S.PW_BOX_LO, S.PW_BOX_HI)
            _, n_pw, off, kw = S.workload("piecewise4096")
            dp = S.draw_batch(grid, n_pw, S.SPECTRA_SEED + off + 1000 * rank, **kw)
            pmodel = ipw.forward(torch.tensor(dp["truth"], dtype=torch.float32, device=dev),
                                 torch.tensor(dp["b_true"], dtype=torch.float32, device=dev))
            pf, pv = S.finish_obs(pmodel.double().cpu().numpy(), dp)
            pin = [torch.tensor(pf, device=dev), torch.tensor(pv, device=dev),
                   torch.tensor(dp["good"], device=dev),
                   torch.tensor(dp["theta0"], dtype=torch.float32, device=dev)]
            pout = ipw.fit(*pin, **opts)
            torch.cuda.synchronize()
            t_ms = []
            for k in range(max(1, args.steps)):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pout = ipw.fit(*pin, out=pout, **opts)
                b.record(stream)
                torch.cuda.synchronize()
                t_ms.append(a.elapsed_time(b))
            pst = pout["status"].cpu().numpy()
            pconv = int(((pst & 3) != 0).sum())
            perr = np.abs(pout["theta"].double().cpu().numpy() - dp["truth"])
            # the same fit on the grouped tensor-core pipeline: the three regimes'
            # stacked rows in three K blocks (split TF32, float-float normal equations)
            po = dict(opts, precision="tf32x3", fp64_normal_eq=1)
            tout = ipw.fit(*pin, **po)
            torch.cuda.synchronize()
            tc_ms = []
            for k in range(max(1, args.steps)):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                tout = ipw.fit(*pin, out=tout, **po)
                b.record(stream)
                torch.cuda.synchronize()
                tc_ms.append(a.elapsed_time(b))
            tconv = int(((tout["status"].cpu().numpy() & 3) != 0).sum())
            tagree = np.all(np.abs(tout["theta"].double().cpu().numpy() - pout["theta"].double().cpu().numpy())[:, :4]
                            <= TOL, axis=1)
            piecewise = {"value": pconv / (sum(t_ms) / len(t_ms) / 1e3), "unit": UNIT,
                         "fit_ms": sum(t_ms) / len(t_ms), "converged": pconv,
                         "mean_steps": float(pout["steps"].float().mean()),
                         "median_abs_teff_err_vs_truth_K": float(np.median(perr[:, 0])),
                         "tf32x3": {"value": tconv / (sum(tc_ms) / len(tc_ms) / 1e3), "unit": UNIT,
                                    "fit_ms": sum(tc_ms) / len(tc_ms), "converged": tconv,
                                    "within_tol_of_fp32_fit_frac": float(tagree.mean())},
                         "workload": "piecewise4096x3909_k25+26+19_teff3300-11500_snr5-100"}
            ipw.close()
    except Exception as e:       # a failed extra is reported; the headline still prints
        piecewise = {"error": f"{type(e).__name__}: {e}"}

    pk, pk_kind = peaks()
    mhz0 = pk.get("sm_max_mhz", 2070.0)
    kernels = []
    try:
        kernels = kernel_rooflines(torch, lasp, ip, [g_flux, g_ivar, g_good, g_th0], grid, theta_np,
                                   steps_np, pk, N_SM * FP32_LANES_PER_SM * 2 * mhz0 * 1e6 / 1e12)
    except Exception as e:       # a failed extra is reported; the headline still prints
        kernels = [{"error": f"{type(e).__name__}: {e}"}]
    fit_avg = sum(fit_ms) / len(fit_ms)
    flops = algorithmic_flops(theta_np, steps_np, grid)
    clocks = clk.summary()
    mhz = pk.get("sm_max_mhz", 2070.0)
    alu_peak = N_SM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flops / (fit_avg / 1e3) / 1e12
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_spectra_per_gpu": N_SPEC, "n_pix": grid.n_pix,
                   "K": 26, "legendre_deg": DEG, "max_steps": MAX_STEPS, "lr": 0.1,
                   "tol": 1e-5, "precision": "fp32", "parallelism": f"replicas{world}",
                   "l2": "flushed (256 MB write) between steps; inputs 144 MB > L2"},
        "e2e": {"value": e2e_conv / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo},
        "gpu_launches": 3 * args.steps,
        "detail": {"fit_ms": fit_avg, "errors_ms": sum(err_ms) / len(err_ms),
                   "converged": conv, "n_spectra": N_SPEC,
                   "mean_steps": float(steps_np.mean()),
                   "steps_p50_p90_p99_max": [float(np.percentile(steps_np, q)) for q in (50, 90, 99)]
                                            + [int(steps_np.max())],
                   "spectrum_steps_per_s": float((steps_np + 1).sum() / (fit_avg / 1e3))},
        "roofline": {"kernel": FIT_KERNEL, "bound": "alu", "achieved": achieved,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                     "peak_source": f"derived, not measured: 152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz "
                                    f"(sm_max_mhz, {pk_kind})",
                     "traffic": FIT_TRAFFIC_BYTES,
                     "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one "
                                     f"{FIT_KERNEL} launch on this workload (ncu)"},
        "clocks": clocks,
        "kernels": kernels,
        "kernels_note": ("per-kernel device time from lasp_profile (CUDA events around each kernel on "
                         "its stream, one untimed pass after the timed region); alu peak derived: "
                         f"152 SMs x 128 FP32 lanes x 2 x {mhz0:.0f} MHz (not measured), hbm peak "
                         "measured (MEASURED_PEAKS.json hbm_gbs)"),
        "mixed": mixed,
        "mixed_65536": mixed_large,
        "joint_loss": joint,
        "lm": lm,
        "clean": clean,
        "piecewise": piecewise,
    }
    if rank == 0 and not args.no_served:
        tabs = {S.LAMOST.name: C, S.DESI.name: S.make_table(S.DESI)}
        for key, grids, kw in (
                ("served", [S.LAMOST, S.DESI], dict(native=True, seconds=10.0, repeats=3)),
                ("served_lamost_only", [S.LAMOST], dict(native=True, loads=())),
                ("served_python", [S.LAMOST, S.DESI], dict(native=False)),
                ("served_mixed", [S.LAMOST, S.DESI], dict(native=True, precision="tf32x3", fp64_normal_eq=1))):
            try:
                res[key] = served_stream(torch, lasp, grids, tabs, **kw)
            except Exception as e:   # a failed extra is reported; the headline still prints
                res[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_cpu_baseline:
        try:
            res["cpu_baseline"] = cpu_baseline(args.cpu_sample, grid, C, ip, torch, flux, ivar, d, theta_np)
            # the metric counts converged spectra at the parameter tolerance: scale the
            # converged count by the fraction within tolerance of the oracle, measured
            # on the first cpu_sample spectra of this timed batch
            frac = res["cpu_baseline"]["gpu_vs_oracle_within_tol_frac"]
            res["value"] = value * frac
            res["e2e"]["value"] *= frac
            res["detail"]["value_counting"] = (
                f"converged spectra x {frac:.4f}, the fraction of the first {args.cpu_sample} spectra of "
                "the timed batch whose GPU fit is within (1 K, 0.005, 0.005, 0.1 km/s) of the FP64 "
                "oracle's fit of the same spectrum")
            res["detail"]["converged_per_s_unchecked"] = value
        except Exception as e:
            res["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
    elif rank == 0:
        res["detail"]["value_counting"] = "converged spectra (no oracle sample: --no-cpu-baseline)"
    if rank == 0:
        print(json.dumps(res))
    if dist:
        dist.destroy_process_group()


def _oracle_sample(n, grid, C, seed):
    from oracle import oracle as O
    M = O.Model(C, S.EXPS, grid.dln, grid.pad, grid.n_pix, DEG, S.BASIS_LO, S.BASIS_HI,
                S.BOX_LO, S.BOX_HI)
    d = S.draw_batch(grid, n, seed, snr=(5, 100), mask_frac=0.05)
    flux, ivar = S.finish_obs(O.model_batch(M, d["truth"], d["b_true"]), d)
    return O, M, d, flux, ivar


def _oracle_step(O, M, d, flux, ivar, threads):
    r = O.fit(M, flux, ivar, d["good"], d["theta0"], threads=threads, max_steps=MAX_STEPS)
    for i in range(len(flux)):
        O.errors(M, flux[i], ivar[i], d["good"][i], r["theta"][i])
    return r


def cpu_baseline(n, grid, C, ip, torch, flux, ivar, d, gpu_theta):
    """The oracle (FP64 C, OpenMP over spectra) timed on this host's cores on
    the first n spectra of the timed batch itself (fit + stage-9 errors).  The
    same spectra give the GPU fit's agreement within the parameter tolerance
    (the headline counts converged spectra at that agreement) and the stage-9
    sigma error of both normal-equation levels, evaluated at the oracle's
    parameters."""
    from oracle import oracle as O
    M = O.Model(C, S.EXPS, grid.dln, grid.pad, grid.n_pix, DEG, S.BASIS_LO, S.BASIS_HI,
                S.BOX_LO, S.BOX_HI)
    sub = {k: (v[:n] if isinstance(v, np.ndarray) else v) for k, v in d.items()}
    f, iv = flux[:n], ivar[:n]
    threads = O.lib().orc_max_threads()
    t0 = time.perf_counter()
    r = O.fit(M, f, iv, sub["good"], sub["theta0"], threads=threads, max_steps=MAX_STEPS)
    sig_ref = np.stack([O.errors(M, f[i], iv[i], sub["good"][i], r["theta"][i])["sigma"] for i in range(n)])
    dt = time.perf_counter() - t0
    conv = int(((r["status"] & 3) != 0).sum())
    within = np.all(np.abs(gpu_theta[:n] - r["theta"])[:, :4] <= TOL, axis=1)
    # stage-9 sigma at the oracle's parameters, float-float and FP64 sums
    dev = torch.device("cuda")
    T = lambda a, dt_=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt_, device=dev)
    sig_err = {}
    for name, ne in (("float-float", 1), ("fp64", 2)):
        e = ip.errors(T(f), T(iv), T(sub["good"], torch.uint8), T(r["theta"]), with_cov=False,
                      legendre_deg=DEG, fp64_normal_eq=ne)
        rel = np.abs(e["sigma"].double().cpu().numpy() - sig_ref) / sig_ref
        ok = (r["status"] & 3) != 0
        sig_err[name] = {"median_rel": float(np.median(rel[ok])), "p99_rel": float(np.percentile(rel[ok], 99))}
    # one core, on the first 32 spectra of the sample
    n1 = min(32, n)
    t1 = time.perf_counter()
    r1 = O.fit(M, f[:n1], iv[:n1], sub["good"][:n1], sub["theta0"][:n1], threads=1, max_steps=MAX_STEPS)
    for i in range(n1):
        O.errors(M, f[i], iv[i], sub["good"][i], r1["theta"][i])
    dt1 = time.perf_counter() - t1
    conv1 = int(((r1["status"] & 3) != 0).sum())
    return {"value": conv / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {n} spectra of the timed batch (fit + errors), {dt:.1f} s",
            "value_1core": conv1 / dt1,
            "sample_1core": f"{n1} spectra on one core, {dt1:.1f} s",
            "gpu_vs_oracle_within_tol_frac": float(within.mean()),
            "sigma_rel_err_vs_oracle": sig_err}


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    grid = S.LAMOST
    C = S.make_table(grid)
    n = max(64, args.cpu_sample // 8)
    O, M, d, flux, ivar = _oracle_sample(n, grid, C, S.SPECTRA_SEED + 1)
    threads = O.lib().orc_max_threads()
    for _ in range(args.warmup):
        _oracle_step(O, M, {k: (v[:4] if isinstance(v, np.ndarray) else v) for k, v in d.items()},
                     flux[:4], ivar[:4], threads)
    times, conv = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = _oracle_step(O, M, d, flux, ivar, threads)
        times.append(time.perf_counter() - t0)
        conv = int(((r["status"] & 3) != 0).sum())
    dt = sum(times) / len(times)
    value = conv / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_spectra": n, "n_pix": grid.n_pix},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n} of the 4096 spectra per step (fit + errors)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
