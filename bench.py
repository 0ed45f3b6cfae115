#!/usr/bin/env python
"""Benchmark: batched AK log-likelihoods per second at 2^21 samples.

Workload (one "step"): one MCMC ensemble step of the 1024-walker ensemble
configuration -- 1024 walkers scattered N(0, 1e-4) about an injected
source, 2^21 samples at dt = 15 s (~1 yr), harmonics n <= 20, two channels,
seeded data at SNR 50 -- evaluated with emri_loglike_batch in FP64 end to
end.  The headline ``value`` is lnL/s of that FP64 step over all ranks; the
mixed-precision step on the same walkers is reported beside it, with its
largest |lnL_mixed - lnL_fp64|.

Inputs are resident in HBM when a timed step starts; between timed steps
a 512 MiB buffer is written to flush L2 (untimed).  ``e2e`` repeats the FP64
measurement through the C-ABI with host buffers: the walker parameters are
copied from pinned host memory and the lnL copied back inside the timed
region.  Multi-GPU (torchrun): every rank evaluates its own ensemble step on
its own GPU (walkers are independent units; no collective on the data path)
and the max time over ranks is used.

``--impl reference`` times the CPU oracle (the plain reference
implementation) on the same workload, a bounded sample of walkers per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AK log-likelihoods/sec at 2^21 samples (mixed vs FP64, same GPU); p50/p99 latency"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 / FP32 vector peaks of a GB300 derived from unit counts and clock:
# 152 SMs x 2 FP64 FMA/clk (resp. 128 FP32 FMA/clk) x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# walker groups whose orbits, waveforms and FFT passes overlap in the mixed
# step: 0 = the library's default for mixed precision (by size: two groups
# for the 1024-walker 2^21 step)
MIXED_GROUPS = 0


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--walkers", type=int, default=1024)
    ap.add_argument("--logn", type=int, default=21)
    ap.add_argument("--n-max", type=int, default=20)
    ap.add_argument("--cpu-walkers", type=int, default=0, help="oracle sample size (0: one per core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--mixed-groups", type=int, default=MIXED_GROUPS,
                    help="walker groups of the pipelined mixed schedule (emri_ctx_set_pipeline; 1: sequential, 0: by size)")
    ap.add_argument("--serve-seconds", type=float, default=6.0, help="serving measurement per precision (0: skip)")
    ap.add_argument("--multi-chains", type=int, default=64, help="uneven-batching leg: chains (0: skip)")
    ap.add_argument("--no-extra", action="store_true", help="skip the paper-workload and ensemble-step legs")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="serving at Poisson rates 10..2000 req/s (mixed) and 1..30 req/s (FP64), 4 s each, queue 64")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None,
                "reasons": reasons}


# ------------------------------------------------------------- workload
def build_workload(ctx, args, seed_offset=0):
    """Walkers, resident dataset and device buffers of the ensemble step."""
    from paper_2311_17174_gb300 import inputs as I

    wl = I.config_c2(walkers=args.walkers, n=1 << args.logn, n_max=args.n_max)
    ds, theta, z_inj = injected_dataset(ctx, wl, wl.noise_seed + seed_offset)
    return wl, ds, theta, z_inj


def injected_dataset(ctx, wl, noise_seed):
    """Resident dataset of one workload and its walkers at the injection's
    distance.  Data: the injection's unit-distance waveform and spectrum from
    the library's own waveform and FFT calls, scaled to the workload's SNR and
    added to the seeded noise; the injection's redshift is set from the target
    distance with the library's prologue (bisection)."""
    import torch
    from paper_2311_17174_gb300 import emri, inputs as I

    n = wl.n
    g = emri.grid(n, wl.dt)
    psd = I.psd_bc04(n, wl.dt)
    dev = f"cuda:{torch.cuda.current_device()}"
    inj = torch.tensor(wl.injection[:, None].copy(), dtype=torch.float64, device=dev)
    z = torch.zeros((1, n), dtype=torch.complex128, device=dev)
    o64 = emri.opts(precision=emri.FP64, n_max=wl.n_max)
    ctx.ak_waveform(g, inj, o64, z)
    ctx.fft_batch(z, n, 1, emri.FP64, -1)
    torch.cuda.synchronize()
    H = z[0].cpu().numpy()
    del z
    probe = ctx.dataset(g, H, psd, wl.fmin, 1.0 / (2 * wl.dt))
    rho_u = float(np.sqrt(probe.dd()))
    probe.close()
    target = rho_u / wl.snr
    out = torch.zeros((6, 1), dtype=torch.float64, device=dev)

    def dgw(zz):
        t = wl.injection.copy()
        t[I.I_Z] = zz
        ctx.prologue(g, torch.tensor(t[:, None].copy(), dtype=torch.float64, device=dev), o64, out)
        torch.cuda.synchronize()
        return float(out[2, 0])

    z_inj = I.solve_distance(target, dgw)
    data = H * (wl.snr / rho_u) + I.noise_spectrum(noise_seed, psd, n, wl.dt)
    ds = ctx.dataset(g, data, psd, wl.fmin, 1.0 / (2 * wl.dt))
    theta = wl.theta.copy()
    theta[:, I.I_Z] *= z_inj / wl.injection[I.I_Z]
    return ds, theta, z_inj


def multi_bench(ctx, chains: int, steps: int, warmup: int, flush):
    """Uneven batching: ``chains`` independent chains (32-512 walkers,
    2^16-2^22 samples, n_max 5-30, own injection and noise each), mixed
    precision, all chains in one emri_loglike_multi call (one captured CUDA
    graph, one branch per chain), with schedules from the autotuner (one
    tuning per length)."""
    import torch
    from paper_2311_17174_gb300 import emri, inputs as I

    wls = I.config_c4(chains)
    t_setup = time.perf_counter()
    tuned = {}
    for n in sorted({wl.n for wl in wls}):
        tuned[n] = ctx.autotune(emri.grid(n, I.DT), 20, emri.MIXED)
    items, dsets = [], []
    for wl in wls:
        ds, th, _ = injected_dataset(ctx, wl, wl.noise_seed)
        dsets.append(ds)
        w = th.shape[0]
        theta = torch.tensor(th.T.copy(), dtype=torch.float64, device="cuda")
        lnl = torch.zeros(w, dtype=torch.float64, device="cuda")
        items.append((ds, theta, emri.opts(precision=emri.MIXED, n_max=wl.n_max), lnl, None, None, None))
    t_setup = time.perf_counter() - t_setup
    for _ in range(warmup):
        ctx.loglike_multi(items)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.loglike_multi(items)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    walkers = sum(it[1].shape[1] for it in items)
    finite = all(bool(torch.isfinite(it[3]).all()) for it in items)
    for ds in dsets:
        ds.close()
    tot = float(sum(times))
    return {"value": walkers * steps / (tot / 1e3), "unit": "lnL/s", "ms_per_step": tot / steps,
            "chains": len(wls), "walkers": walkers,
            "samples_x_walkers": int(sum(wl.n * wl.theta.shape[0] for wl in wls)),
            "lengths": sorted({int(wl.n) for wl in wls}), "precision": "mixed",
            "launch": "one CUDA graph per call, one branch per chain",
            "autotuned": {str(k): v for k, v in tuned.items()}, "all_finite": finite,
            "setup_s": t_setup}


def time_steps(ctx, ds, theta_dev, o, lnl, steps, warmup, flush, barrier):
    import torch
    for _ in range(warmup):
        ctx.loglike_batch(ds, theta_dev, o, lnl)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.loglike_batch(ds, theta_dev, o, lnl)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def serve_datasets(ctx, count: int = 16):
    """The serving configuration's resident datasets: ``count`` seeded noise
    datasets spread over the lengths 2^16..2^22 (dataset i has length
    2^(16 + i mod 7)).  Returns {n: [datasets of that length]}."""
    from paper_2311_17174_gb300 import emri, inputs as I
    out = {}
    for i in range(count):
        n = 1 << (16 + i % 7)
        psd = I.psd_bc04(n)
        ds = ctx.dataset(emri.grid(n, I.DT), I.noise_spectrum(700 + i, psd, n), psd, 1e-4, 1 / (2 * I.DT))
        out.setdefault(n, []).append(ds)
    return out


def serve_bench(ctx, dsets, precision: int, rate: float, duration: float, n_max: int, seed: int = 5,
                queue_capacity: int = 4096):
    """Poisson-arriving requests (8-512 walkers, 2^16-2^22 samples; a request
    of length n uses the resident dataset of that length its dataset index
    selects) through the serving loop; latency is completion minus arrival as
    stamped by the library.  Served lnL/s counts the walkers of completed
    requests over the time from the first arrival to the last completion;
    requests refused by a full queue are counted apart."""
    import threading
    from paper_2311_17174_gb300 import emri, inputs as I
    sched = I.config_c5(rate, duration, seed=seed)
    src = I.draw_sources(seed, 1, 1 << 22)[0]
    pool = I.scatter_walkers(seed + 1, src, 512)
    o = emri.opts(precision=precision, n_max=n_max)
    ctx.serve_start(slots=4, queue_capacity=queue_capacity)
    lat, walkers, lock = [], [0], threading.Lock()
    tickets = []
    rejected = [0]

    def waiter():
        k = 0
        while True:
            with lock:
                if k >= len(tickets):
                    if done_submitting[0]:
                        return
                    t = None
                else:
                    t = tickets[k]
            if t is None:
                time.sleep(0.001)
                continue
            tk, w = t
            rc, _, _, st = ctx.serve_poll(tk, w, timeout_us=-1)
            lat.append((st.done_ns - st.arrival_ns) / 1e6)
            walkers[0] += w
            k += 1

    done_submitting = [False]
    th = threading.Thread(target=waiter)
    th.start()
    t0 = time.perf_counter()
    for (ta, dsi, w, n) in sched:
        dt_ = t0 + ta - time.perf_counter()
        if dt_ > 0:
            time.sleep(dt_)
        try:
            tk = ctx.serve_submit(dsets[n][dsi % len(dsets[n])], pool[:w].T.copy(), o)
        except emri.EmriError as exc:   # a full queue refuses the request (EAGAIN)
            if exc.code != emri.EAGAIN:
                raise
            rejected[0] += 1
            continue
        with lock:
            tickets.append((tk, w))
    with lock:
        done_submitting[0] = True
    th.join()
    elapsed = time.perf_counter() - t0
    ctx.serve_stop()
    lat = np.array(lat)
    return {"precision": "fp64" if precision == 0 else "mixed", "rate_per_s": rate, "requests": int(len(lat)),
            "rejected": rejected[0], "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "lnl_per_s": walkers[0] / elapsed, "seconds": elapsed, "slots": 4, "queue_capacity": queue_capacity,
            "resident_datasets": sum(len(v) for v in dsets.values())}


# DRAM bytes per sample of k2_wave_f64 from one ncu capture of the kernel
# (64 walkers x 2^20 samples, n_max 20: 69.54 MB read + 1013.18 MB written;
# profiles/ncu_k2_wave_f64_64w_2p20.md, the kernel with 1024-sample segments),
# scaled to a launch by the samples it processes (the kernel's traffic is its
# 16-byte output per sample plus the per-segment orbit records, both
# proportional to walkers x samples).
K2_F64_DRAM_BYTES_PER_SAMPLE = (69.544e6 + 1013.184e6) / (64 * 2 ** 20)


def paper_bench(ctx, steps: int, warmup: int):
    """The paper's own set-up (initial conditions at the LSO, e_LSO = 0.3,
    fixed geometry, M, mu, S/M^2, Xi_0 scattered; one year at 15 s; n_max 10;
    noise-free data at 1 Gpc): latency of an 8-walker likelihood batch (the
    paper's ensemble) and throughput at 1024 walkers, FP64 and mixed."""
    import torch
    from paper_2311_17174_gb300 import emri, inputs as I

    res = {}
    wl8 = I.config_paper(walkers=8)
    n, dt = wl8.n, wl8.dt
    g = emri.grid(n, dt)
    mode = emri.BACKWARD_FROM_LSO
    o64 = emri.opts(precision=emri.FP64, n_max=wl8.n_max, mode=mode)
    out = torch.zeros((6, 1), dtype=torch.float64, device="cuda")

    def dl(zz):
        t = wl8.injection.copy()
        t[I.I_Z] = zz
        ctx.prologue(g, torch.tensor(t[:, None].copy(), dtype=torch.float64, device="cuda"), o64, out)
        torch.cuda.synchronize()
        return float(out[2, 0])

    z = I.solve_distance(wl8.extra["d_gpc"] * 3.0856775814913673e27, dl)
    inj = wl8.injection.copy()
    inj[I.I_Z] = z
    zt = torch.zeros((1, n), dtype=torch.complex128, device="cuda")
    ctx.ak_waveform(g, torch.tensor(inj[:, None].copy(), device="cuda"), o64, zt)
    ctx.fft_batch(zt, n, 1, emri.FP64, -1)
    torch.cuda.synchronize()
    # the injection spectrum at its distance (Xi_0 = 1, GR speed: d_GW = d_L)
    data = zt[0].cpu().numpy() / dl(z)
    del zt
    psd = I.psd_bc04(n, dt)
    ds = ctx.dataset(g, data, psd, wl8.fmin, 1.0 / (2 * dt))
    for walkers in (8, 1024):
        wl = I.config_paper(walkers=walkers)
        th = wl.theta.copy()
        th[:, I.I_Z] = z
        theta = torch.tensor(th.T.copy(), device="cuda")
        lnl = torch.zeros(walkers, dtype=torch.float64, device="cuda")
        for prec, name in ((emri.FP64, "fp64"), (emri.MIXED, "mixed")):
            o = emri.opts(precision=prec, n_max=wl.n_max, mode=mode)
            for _ in range(warmup):
                ctx.loglike_batch(ds, theta, o, lnl)
            torch.cuda.synchronize()
            times = []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.loglike_batch(ds, theta, o, lnl)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            res[f"{name}_{walkers}w"] = {"ms_per_batch": ms, "lnl_per_s": walkers / (ms / 1e3),
                                         "lnl_walker0": float(lnl[0])}
    ds.close()
    return {"workload": "paper-lso-1yr-2^21-n10 (backward from the LSO, 1 Gpc, noise-free)", **res}


def stretch_bench(ctx, ds, theta_np, wl, steps: int, warmup: int, flush):
    """emri_stretch_step on the ensemble: proposals, the likelihood of the
    proposals and the acceptance on the device, the four free parameters of
    the paper (M, mu, S/M^2, Xi_0) in a box of +-1e-3 relative; uniforms drawn
    on the host and resident before the timed region."""
    import torch
    from paper_2311_17174_gb300 import emri, inputs as I

    w = theta_np.shape[0]
    free = [I.I_M, I.I_MU, I.I_SPIN, I.I_XI0]
    lo, hi = np.full(16, -np.inf), np.full(16, np.inf)
    for p_ in free:
        c = wl.injection[p_]
        lo[p_], hi[p_] = c * (1 - 1e-3), c * (1 + 1e-3)
    lo[I.I_SPIN], hi[I.I_SPIN] = 0.0, 1.0
    cfg = emri.stretch_cfg(free, lo, hi)
    res = {}
    g = np.random.default_rng(12)
    for prec, name in ((emri.FP64, "fp64"), (emri.MIXED, "mixed")):
        o = emri.opts(precision=prec, n_max=wl.n_max)
        theta = torch.tensor(theta_np.T.copy(), device="cuda")
        lnp = torch.zeros(w, dtype=torch.float64, device="cuda")
        acc = torch.zeros(w, dtype=torch.int32, device="cuda")
        ctx.loglike_batch(ds, theta, o, lnp)
        us = [torch.tensor(g.random((3, w)), device="cuda") for _ in range(warmup + steps)]
        for k in range(warmup):
            ctx.stretch_step(ds, theta, lnp, o, cfg, us[k], acc)
        torch.cuda.synchronize()
        times, accepted = [], 0
        for k in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.stretch_step(ds, theta, lnp, o, cfg, us[warmup + k], acc)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            accepted += int(acc.sum())
        tot = float(sum(times))
        res[name] = {"ms_per_step": tot / steps, "lnl_per_s": w * steps / (tot / 1e3),
                     "acceptance": accepted / (w * steps)}
    return {"walkers": w, "free_parameters": "M, mu, S/M^2, Xi_0", **res}


def sharded_bench(ctx, args, rank: int, world: int, steps: int, warmup: int, flush, barrier):
    """One ensemble of W x world walkers spread over the ranks (walker blocks
    of each half per GPU, an all-gather of the moved blocks after each
    half-step over NCCL): every rank builds the same seeded data and
    ensemble, moves its blocks with emri_stretch_half and holds the whole
    ensemble after each step.  lnL/s counts all ranks' proposals over the
    slowest rank's time (max over ranks)."""
    import torch
    import torch.distributed as dist
    from paper_2311_17174_gb300 import emri, ensemble as EN, inputs as I

    w = args.walkers * world
    wl = I.config_c2(walkers=w, n=1 << args.logn, n_max=args.n_max)
    ds, th, _ = injected_dataset(ctx, wl, wl.noise_seed)
    free = [I.I_M, I.I_MU, I.I_SPIN, I.I_XI0]
    lo, hi = np.full(16, -np.inf), np.full(16, np.inf)
    for p_ in free:
        c = wl.injection[p_]
        lo[p_], hi[p_] = c * (1 - 1e-3), c * (1 + 1e-3)
    lo[I.I_SPIN], hi[I.I_SPIN] = 0.0, 1.0
    cfg = emri.stretch_cfg(free, lo, hi)
    o = emri.opts(precision=emri.MIXED, n_max=wl.n_max)
    dev = f"cuda:{torch.cuda.current_device()}"
    theta = torch.tensor(th.T.copy(), device=dev)
    lnp = torch.zeros(w, dtype=torch.float64, device=dev)
    acc = torch.zeros(w, dtype=torch.int32, device=dev)
    ctx.loglike_batch(ds, theta, o, lnp)
    g = np.random.default_rng(13)
    us = [torch.tensor(g.random((3, w)), device=dev) for _ in range(warmup + steps)]
    ens = EN.ShardedEnsemble(ctx, ds, o, cfg, rank, world)
    for k in range(warmup):
        ens.step(theta, lnp, us[k], acc)
    torch.cuda.synchronize()
    times = []
    for k in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ens.step(theta, lnp, us[warmup + k], acc)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    tot = torch.tensor([float(sum(times))], device=dev)
    dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ds.close()
    return {"walkers": w, "ranks": world, "precision": "mixed", "ms_per_step": float(tot.item()) / steps,
            "lnl_per_s": w * steps / (float(tot.item()) / 1e3),
            "exchange": "all-gather of the moved walker blocks after each half-step (NCCL)"}


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json),
    else the recipe's fallback."""
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def mixed_roofline(kt, walkers: int, n: int, n_max: int, steps: int):
    """Roofline of each kernel of the mixed step from the live event times:
    the waveform kernel against the derived FP32 peak (algorithmic flops:
    the flop model per sample, in FP32), the two FFT passes against the
    measured HBM bandwidth (algorithmic bytes: pass 1 reads and writes the
    8-byte series, pass 2 reads it once; the dataset and delay tables it also
    reads are L2-resident and not counted)."""
    hbm, src = hbm_peak_gbs()
    out = {}
    samples = float(walkers) * n * steps
    if kt.get("wave", (0, 0))[1]:
        ms = kt["wave"][0]
        tf = flop_model(n_max) * samples / (ms / 1e3) / 1e12
        out["k2_wave_mixed"] = {"bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": tf / FP32_PEAK_TFLOPS, "ms_per_step": ms / steps,
                                "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 x 2.07 GHz"}
    for name, key, per_sample in (("k3_pass1<float2>", "fft_pass1", 16.0), ("k4_pass2_ip_r8", "fft_pass2_ip", 8.0)):
        if kt.get(key, (0, 0))[1]:
            ms = kt[key][0]
            gbs = per_sample * samples / (ms / 1e3) / 1e9
            out[name] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "ms_per_step": ms / steps, "peak_source": src}
    return out


def flop_model(n_max: int) -> float:
    """Algorithmic FP64 flops per sample of the factored harmonic sum and
    response (an FMA counts two): 24 per harmonic
    (rotation 6, three quadratic amplitudes 12, three accumulations 6) plus
    172 per sample (three phase cubics and x^(2/3) 28, three table sin/cos
    60, four antenna-pattern cubics 25, fixed-basis response and the two
    channels 57, fit time 2)."""
    return 24.0 * n_max + 172.0


# ------------------------------------------------------------ CPU oracle
def oracle_sample(theta, wl, data_fd, psd, walkers: int, threads: int):
    import oracle as O
    w = O.weights(psd, wl.n, wl.dt, wl.fmin, 1.0 / (2 * wl.dt))
    t0 = time.perf_counter()
    O.loglike(theta[:walkers], wl.n, wl.dt, data_fd, w, O.Opts(n_max=wl.n_max), nthreads=threads)
    return time.perf_counter() - t0


def cpu_baseline(args, wl, theta, data_fd, psd):
    cores = os.cpu_count() or 1
    walkers = args.cpu_walkers or cores
    threads = min(walkers, cores)
    secs = oracle_sample(theta, wl, data_fd, psd, walkers, threads)
    return {"value": walkers / secs, "unit": "lnL/s", "cores": threads, "kind": "oracle",
            "sample": f"{walkers} walkers of the ensemble step, full 2^{args.logn} samples, n<=20, FP64/long "
                      f"double oracle, OpenMP over walkers on {threads} host threads, {secs:.1f} s"}


def run_reference(args):
    """The reference arm: the CPU oracle on the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2311_17174_gb300 import inputs as I
    import oracle as O
    n = 1 << args.logn
    wl = I.config_c2(walkers=args.walkers, n=n, n_max=args.n_max)
    psd = I.psd_bc04(n, wl.dt)
    data = I.noise_spectrum(wl.noise_seed, psd, n, wl.dt)
    cores = os.cpu_count() or 1
    walkers = args.cpu_walkers or cores
    threads = min(walkers, cores)
    O.build()
    for _ in range(args.warmup):
        oracle_sample(wl.theta, wl, data, psd, min(walkers, threads), threads)
    secs = [oracle_sample(wl.theta, wl, data, psd, walkers, threads) for _ in range(args.steps)]
    tot = sum(secs)
    value = walkers * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": "lnL/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "walkers_per_step": walkers, "samples": n, "n_max": wl.n_max,
                       "note": "each step is a bounded sample of the ensemble step's walkers"},
            "cpu_baseline": {"value": value, "unit": "lnL/s", "cores": threads, "kind": "oracle",
                             "sample": f"{walkers} walkers per step, full length, {threads} threads"},
            "e2e": {"value": value, "unit": "lnL/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2311_17174_gb300 import emri

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    def barrier():
        if world > 1:
            dist.barrier()

    ctx = emri.Context(local)
    wl, ds, theta, z_inj = build_workload(ctx, args, seed_offset=rank)
    W = theta.shape[0]
    dev = f"cuda:{local}"
    theta_dev = torch.tensor(theta.T.copy(), dtype=torch.float64, device=dev)
    lnl = torch.zeros(W, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    o64 = emri.opts(precision=emri.FP64, n_max=wl.n_max)
    omix = emri.opts(precision=emri.MIXED, n_max=wl.n_max)

    # ---- FP64 headline
    clocks = ClockSampler(local)
    launches0 = ctx.launches()
    ctx.profile(True)
    for _ in range(args.warmup):
        ctx.loglike_batch(ds, theta_dev, o64, lnl)
    torch.cuda.synchronize()
    ctx.profile(True)   # reset: keep only the timed steps
    launches0 = ctx.launches()
    clocks.start()
    times = time_steps(ctx, ds, theta_dev, o64, lnl, args.steps, 0, flush, barrier)
    clk = clocks.stop()
    launches = ctx.launches() - launches0
    ktimes = ctx.kernel_times()
    ctx.profile(False)
    lnl64 = lnl.cpu().numpy().copy()
    tot_ms = float(sum(times))
    if world > 1:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = W * world * args.steps / (tot_ms / 1e3)

    # ---- mixed precision on the same walkers
    mixed = None
    if not args.no_mixed:
        ctx.set_pipeline(emri.MIXED, args.mixed_groups)
        for _ in range(args.warmup):
            ctx.loglike_batch(ds, theta_dev, omix, lnl)
        torch.cuda.synchronize()
        tm = time_steps(ctx, ds, theta_dev, omix, lnl, args.steps, 0, flush, barrier)
        lm = lnl.cpu().numpy()
        # per-kernel device times from the same step with its kernels in
        # sequence (in the pipelined schedule a launch's events would also
        # span the other streams' kernels running beside it)
        ctx.set_pipeline(emri.MIXED, 1)
        ctx.profile(True)
        tseq = time_steps(ctx, ds, theta_dev, omix, lnl, args.steps, 0, flush, barrier)
        kt_mix = ctx.kernel_times()
        ctx.profile(False)
        ctx.set_pipeline(emri.MIXED, args.mixed_groups)
        assert np.array_equal(lnl.cpu().numpy(), lm), "pipelined and sequential mixed steps differ"
        mt = float(sum(tm))
        if world > 1:
            t = torch.tensor([mt], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            mt = float(t.item())
        mixed = {"value": W * world * args.steps / (mt / 1e3), "unit": "lnL/s", "ms_per_step": mt / args.steps,
                 "pipeline_groups": args.mixed_groups or "by size (2 at 1024 walkers x 2^21)",
                 "ms_per_step_sequential": float(sum(tseq)) / args.steps,
                 "dlnl_max_vs_fp64": float(np.max(np.abs(lm - lnl64))),
                 "kernels_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in kt_mix.items() if v[1]},
                 "roofline": mixed_roofline(kt_mix, W, wl.n, wl.n_max, args.steps)}

    # ---- end to end through the C-ABI with host buffers (FP64)
    th_host = torch.tensor(theta.T.copy(), dtype=torch.float64).pin_memory()
    out_host = torch.zeros(W, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        theta_dev.copy_(th_host, non_blocking=True)
        ctx.loglike_batch(ds, theta_dev, o64, lnl)
        out_host.copy_(lnl, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_tot = float(sum(e2e_ms))
    if world > 1:
        t = torch.tensor([e2e_tot], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())

    # ---- serving: p50/p99 latency under Poisson arrivals (rank 0)
    # light load (the loop keeps up: latency) and a saturating rate per
    # precision (queue full: served lnL/s is the loop's capacity)
    serving = None
    if rank == 0 and (args.serve_seconds > 0 or args.serve_sweep):
        sdsets = serve_datasets(ctx)
        if args.serve_seconds > 0:
            serving = [serve_bench(ctx, sdsets, emri.MIXED, 20.0, args.serve_seconds, wl.n_max),
                       serve_bench(ctx, sdsets, emri.FP64, 1.5, args.serve_seconds, wl.n_max),
                       serve_bench(ctx, sdsets, emri.MIXED, 300.0, args.serve_seconds, wl.n_max, queue_capacity=32),
                       serve_bench(ctx, sdsets, emri.FP64, 10.0, args.serve_seconds, wl.n_max, queue_capacity=16)]
        if args.serve_sweep:
            serving = (serving or []) + \
                [serve_bench(ctx, sdsets, emri.MIXED, r, 4.0, wl.n_max, queue_capacity=64)
                 for r in (10, 30, 100, 300, 1000, 2000)] + \
                [serve_bench(ctx, sdsets, emri.FP64, r, 4.0, wl.n_max, queue_capacity=64) for r in (1, 3, 10, 30)]
        for v in sdsets.values():
            for d in v:
                d.close()

    # ---- the paper's own workload and the on-device ensemble step (rank 0)
    paper = stretch = None
    if rank == 0 and not args.no_extra:
        stretch = stretch_bench(ctx, ds, theta, wl, 3, 1, flush)
        paper = paper_bench(ctx, 5, 2)

    # ---- one ensemble spread over all ranks (N > 1 only)
    sharded = None
    if world > 1 and not args.no_extra:
        sharded = sharded_bench(ctx, args, rank, world, 3, 1, flush, barrier)

    # ---- uneven batching: many chains in one captured launch (rank 0)
    multi = None
    if rank == 0 and args.multi_chains > 0:
        multi = multi_bench(ctx, args.multi_chains, args.steps, 2, flush)

    # ---- roofline of the dominant kernel (FP64 step)
    per_step = {k: v[0] / args.steps for k, v in ktimes.items() if v[1]}
    dom = max(per_step, key=per_step.get)
    roof = None
    if dom == "wave":
        launches_wave = ktimes["wave"][1]
        avg_ms = ktimes["wave"][0] / launches_wave
        walkers_per_launch = W * args.steps / launches_wave
        flops = flop_model(wl.n_max) * wl.n * walkers_per_launch
        achieved = flops / (avg_ms / 1e3) / 1e12
        traffic = K2_F64_DRAM_BYTES_PER_SAMPLE * wl.n * walkers_per_launch if wl.n_max == 20 else None
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": "k2_wave_f64",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (FP64 vector unit)",
                "flops_per_launch": flops, "avg_launch_ms": avg_ms}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": dom}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            cpu = cpu_baseline(args, wl, theta, ds_data_host(ctx, wl, z_inj), psd_host(wl))
        except Exception as exc:  # the baseline is reported, not required
            cpu = {"value": None, "unit": "lnL/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {exc}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "lnL/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "walkers": W, "samples": wl.n, "dt": wl.dt, "n_max": wl.n_max,
                       "snr": wl.snr, "precision": "fp64 end to end", "l2": "flushed between timed steps",
                       "parallelism": f"replicas x{world} (walker blocks per GPU)"},
            "mixed": mixed,
            "e2e": {"value": W * world * args.steps / (e2e_tot / 1e3), "unit": "lnL/s",
                    "h2d_bytes_per_step": int(th_host.numel() * 8), "d2h_bytes_per_step": int(out_host.numel() * 8)},
            "serving": serving,
            "multi_chain": multi,
            "ensemble_step": stretch,
            "sharded_ensemble_step": sharded,
            "paper_workload": paper,
            "gpu_launches": int(launches),
            "kernels_ms_per_step": {k: round(v, 3) for k, v in per_step.items()},
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ds.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def psd_host(wl):
    from paper_2311_17174_gb300 import inputs as I
    return I.psd_bc04(wl.n, wl.dt)


def ds_data_host(ctx, wl, z_inj):
    """Data spectrum for the CPU baseline: the same seeded noise (the oracle's
    timing does not depend on the injection's amplitude)."""
    from paper_2311_17174_gb300 import inputs as I
    return I.noise_spectrum(wl.noise_seed, psd_host(wl), wl.n, wl.dt)


if __name__ == "__main__":
    main()
