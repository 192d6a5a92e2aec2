"""Benchmark of the metric-based importance-sampling hot path on GB300.

Workload (N = 1): the aligned-spin BNS population -- H1+L1, 20-1024 Hz at 1/128 Hz
(128,513 bins, complex64 data, FP64 PSD), coloured Gaussian noise, SNR 10-30; per event
2^20 proposal samples over (Mc, q, chi1, chi2, t_c) from a Gaussian in the Fisher metric
at the trigger; phase and distance marginalised.  One step = one event's batch:
draw (Philox) -> fused waveform/projection/inner-product/marginalisation -> two-pass
weight reduction.  Steps cycle over resident events; an L2 flush (256 MB write) runs
between steps inside the timed region.

JSON line (rank 0): value = likelihood evaluations / s over all ranks (weak scaling:
every rank runs its own events), e2e = the same through the C ABI from host buffers
(create + set_metric + draw + loglike + reduce + destroy per step, host->device data
and device->host summary inside the timed region), roofline of the fused likelihood
kernel against the SFU ceiling (two MUFU transcendentals per bin), cpu_baseline = the
FP64 oracle on the host cores on a bounded sample.

--impl reference times the FP64 CPU oracle on the same workload instead.
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

import workloads  # noqa: E402
from workloads import MC, Q, CHI1, CHI2, RA, DEC, PSI, IOTA, DL, TC, PHIC  # noqa: E402

METRIC = "likelihood evals/sec and seconds to 1e4 effective samples per event"
UNIT = "likelihood evals/s"
SFU_PER_SM_PER_CLK = 16        # MUFU results per SM per clock (Blackwell)
SFU_PER_BIN = 2                # one sine and one cosine per (sample, bin)
N_SM = 152
# dram__bytes_read.sum + dram__bytes_write.sum of one loglike_mixed_fold_kernel launch at this
# workload (2^20 samples), from a full ncu capture of the current kernel version (bench leg
# `--steps 1 --warmup 3`); not measured inside this run
FOLD_TRAFFIC_BYTES = 44_049_664 + 122_880
FOLD_TRAFFIC_SOURCE = ("ncu --set full capture of one launch of this kernel version at this workload "
                       "(dram__bytes_read.sum + dram__bytes_write.sum); not measured in this run")
SFU_PEAK_NOTE = ("peak = 152 SM x 16 MUFU results/clk (nominal; sine/cosine measured at 15.1 per SM per clock "
                 "on this part) x sm_max_mhz / 2 MUFU per (sample, bin)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------------- clock sampling
class ClockSampler:
    def __init__(self):
        self.samples, self.proc, self.thread = [], None, None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.proc = subprocess.Popen(["nvidia-smi", "-i", idx, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if not self.samples:
            return None
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------------- event set-up
def event_setup(m, w, spec, dets_np):
    """Synthetic data and proposal for one event through the library's own helpers:
    injection + noise (mbis_inject), Fisher-metric Gaussian proposal (mbis_fisher)."""
    n = w.n_bins
    psd1 = m.mbis_psd_aligo(w.f_lo, w.df, n)
    psd = np.tile(psd1, (w.n_det, 1))
    dets = m.make_detectors(*dets_np)
    th = np.zeros(11)
    mc = (spec.m1 * spec.m2) ** 0.6 / (spec.m1 + spec.m2) ** 0.2
    th[MC], th[Q] = mc, spec.m1 / spec.m2
    for k, v in spec.params.items():
        th[workloads.PARAM_NAMES.index(k)] = v
    th[DL] = 1.0
    _, snr2 = m.mbis_inject(w.f_lo, w.df, n, dets, psd, spec.gmst, th)
    th[DL] = math.sqrt(snr2) / spec.snr
    strain, _ = m.mbis_inject(w.f_lo, w.df, n, dets, psd, spec.gmst, th, spec.noise_seed or 0,
                              spec.noise_seed is not None)
    strain = strain.astype(np.complex64 if w.complex_dtype == "c64" else np.complex128)
    ctx = m.mbis_create(strain, psd, dets, w.f_lo, w.df, th, gmst=spec.gmst, precision=m.FP64, marg=w.marg,
                        dmin=w.dmin, dmax=w.dmax)
    try:
        prop = m.fisher_proposal(ctx, th, w.sampled, scale=w.scale, box_sigmas=w.box_sigmas, chi_max=w.chi_max,
                                 dmin=w.dmin, dmax=w.dmax, prior_flags=w.prior_flags)
    finally:
        m.mbis_destroy(ctx)
    return dict(spec=spec, th=th, strain=strain, psd=psd, dets=dets, prop=prop, w=w)


def make_ctx(m, w, ev, precision):
    ctx = m.mbis_create(ev["strain"], ev["psd"], ev["dets"], w.f_lo, w.df, ev["th"], gmst=ev["spec"].gmst,
                        precision=precision, marg=w.marg, n_tshift=w.n_tshift, dt_shift=w.dt_shift, dmin=w.dmin,
                        dmax=w.dmax)
    p = ev["prop"]
    m.mbis_set_metric(ctx, p["ids"], p["mean"], p["chol"], p["scale"], p["lo"], p["hi"], p["flags"])
    return ctx


# ------------------------------------------------------------------------- CPU oracle timing
class OracleLeg:
    """The FP64 oracle on the host cores, on events of the same workload that the oracle
    builds itself (injection, noise, Fisher proposal): no input comes from the GPU path."""

    def __init__(self, w, specs, threads=None):
        import oracle
        from oracle import events as oev
        oracle.build()
        self.oracle, self.w = oracle, w
        self.events = []
        for spec in specs:
            ev, th, _ = oev.make_event(w, spec)
            s = (ev.strain[..., 0] + 1j * ev.strain[..., 1]).astype(np.complex64)   # the data the GPU holds
            ev.set_strain(np.stack([s.real.astype(np.float64), s.imag.astype(np.float64)], axis=-1))
            self.events.append((spec, ev, th, oev.make_proposal(ev, w, th)))
        self.cores = threads or os.cpu_count() or 1

    def batch(self, i, n):
        """draw -> likelihood -> weights for n samples of event i; returns seconds."""
        o = self.oracle
        spec, ev, th, p = self.events[i % len(self.events)]
        t0 = time.perf_counter()
        theta, lq = o.draw(spec.draw_seed, (i // len(self.events)) * n, n, p["ids"], p["mean"], p["chol"],
                           p["scale"])
        ll = o.loglike_batch(ev, o.full_params(p["ids"], theta, th))
        lp = o.log_prior(p["ids"], p["lo"], p["hi"], p["flags"], theta)
        o.reduce(ll, lp, lq)
        return time.perf_counter() - t0

    def rate(self, budget_s):
        n = max(4, 2 * self.cores)
        evals, used, i = 0, 0.0, 0
        while used < budget_s:
            used += self.batch(i, n)
            evals += n
            i += 1
        return evals / used, evals, used


def oracle_one_core_rate(n_samples, budget_s):
    """The same oracle leg on one host core: a child process limited to one OpenMP thread
    (likelihoods / s of the first event of the workload)."""
    code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench, workloads; "
            f"w = workloads.bns_population(n_events=1, n_samples={int(n_samples)}); "
            f"leg = bench.OracleLeg(w, w.events[:1], threads=1); "
            f"print(json.dumps(leg.rate({float(budget_s)})))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        rate, evals, used = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": rate, "unit": UNIT, "cores": 1, "sample": f"{evals} likelihoods ({used:.1f} s)"}
    except (subprocess.SubprocessError, ValueError, IndexError, OSError) as e:
        return {"value": None, "error": str(e)[:200]}


# ------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import torch
    import paper_2410_05190_gb300 as m
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = workloads.bns_population(n_events=max(args.events * world, 1), n_samples=args.samples)
    from paper_2410_05190_gb300.dist import shard, max_over_ranks
    my_events = shard(w.events, rank, world)[: args.events]
    dets_np = workloads.network(w.detectors)
    t_setup = time.time()
    evs = [event_setup(m, w, spec, dets_np) for spec in my_events]
    ctxs = [make_ctx(m, w, ev, m.MIXED) for ev in evs]
    setup_s = time.time() - t_setup
    n, P = w.n_samples, len(w.sampled)
    stream = torch.cuda.current_stream()
    theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
    lq, lp, ll = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    launches_per_step = 4  # draw, fused likelihood, reduce max, reduce sums
    like_events = []

    def step(i, timed):
        ctx = ctxs[i % len(ctxs)]
        spec = evs[i % len(evs)]["spec"]
        flush.zero_()
        m.mbis_draw(ctx, spec.draw_seed, (i // len(ctxs)) * n, n, theta, lq, lp, stream)
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        m.mbis_loglike(ctx, n, theta, ll, stream)
        if timed:
            e1.record(stream)
            like_events.append((e0, e1))
        return m.mbis_reduce(ctx, n, ll, lp, lq, None, 0, stream)

    summaries = []
    for i in range(args.warmup):
        step(i, False)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler()
    clk.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        summaries.append(step(args.warmup + i, True))
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    like_ms = [a.elapsed_time(b) for a, b in like_events]
    elapsed = max_over_ranks(elapsed, device="cuda")
    evals = args.steps * n * world
    value = evals / elapsed

    # end to end through the C ABI from host buffers (create .. destroy per step)
    e2e = None
    if args.e2e_steps > 0:
        th_bytes = 0
        hbuf = torch.empty(4, dtype=torch.float64)
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        for i in range(args.e2e_steps):
            ev = evs[i % len(evs)]
            ctx = make_ctx(m, w, ev, m.MIXED)
            m.mbis_draw(ctx, ev["spec"].draw_seed, 0, n, theta, lq, lp, stream)
            m.mbis_loglike(ctx, n, theta, ll, stream)
            s = m.mbis_reduce(ctx, n, ll, lp, lq, None, 0, stream)
            m.mbis_destroy(ctx)
        torch.cuda.synchronize()
        te = time.perf_counter() - te0
        ev = evs[0]
        h2d = ev["strain"].nbytes + ev["psd"].nbytes + 8 * (ev["prop"]["chol"].size + 4 * P + 11)
        d2h = 4 * 8 + 4
        e2e = {"value": args.e2e_steps * n / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}

    out = None
    if rank == 0:
        pk = peaks()
        clock_mhz = pk.get("sm_max_mhz", 2070.0)
        bins_per_launch = n * w.n_bins
        avg_s = statistics.mean(like_ms) / 1e3
        achieved = bins_per_launch / avg_s / 1e9
        peak = N_SM * SFU_PER_SM_PER_CLK * clock_mhz * 1e6 / SFU_PER_BIN / 1e9
        ess = [s["ess"] for s in summaries]
        eff = [s["ess"] / n for s in summaries]
        per_event_s = [1e4 / max(e * value / world, 1e-30) for e in eff]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "bns_population: one event x 2^20 proposal samples per step, 128513 bins "
                                   "(20-1024 Hz, df=1/128), H1+L1, complex64 data, phase+distance marginalised",
                       "events_per_rank": len(evs), "n_samples": n, "n_bins": w.n_bins, "sampled": "Mc,q,chi1,chi2,tc",
                       "precision": "f32 per bin; f64 anchors, overlap sums, marginalisation, weights",
                       "l2": "flushed between steps (256 MB write inside the timed region)",
                       "parallelism": f"replicas x{world} (events sharded, no collective on the data path)",
                       "setup_s": round(setup_s, 2)},
            "fisher_proposal_efficiency": {"median": statistics.median(eff), "ess_median": statistics.median(ess),
                                           "seconds_to_1e4_at_this_efficiency_median": statistics.median(per_event_s)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gbin/s",
                         "frac": achieved / peak, "traffic": FOLD_TRAFFIC_BYTES, "traffic_unit": "bytes per launch",
                         "traffic_source": FOLD_TRAFFIC_SOURCE,
                         "kernel": "loglike_mixed_fold_kernel", "launch_ms": statistics.mean(like_ms),
                         "note": SFU_PEAK_NOTE},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        if e2e:
            out["e2e"] = e2e
    for c in ctxs:
        m.mbis_destroy(c)
    return out, w, evs


# ------------------------------------------------------------------------- further measurements (N = 1)
def ess_buffers(torch, P, batch):
    return [torch.empty((P, batch), dtype=torch.float64, device="cuda")] + \
           [torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(4)]


def seconds_to_ess(m, torch, evs, precision, target=1e4, batch=1 << 16, max_samples=1 << 26, refine=4, rb=None):
    """Wall time of mbis_run_to_ess (refit after each of the first `refine` batches) per event;
    rb = (n_sigma, eps_rad): the loop runs on the relative-binning likelihood (bins from
    mbis_rb_edges about the injection, set-up timed apart)."""
    out = []
    for ev in evs:
        w = ev["w"]
        ctx = make_ctx(m, w, ev, precision)
        try:
            bufs = ess_buffers(torch, len(ev["prop"]["ids"]), batch)
            extra = {}
            if rb is not None:
                t0 = time.perf_counter()
                edges = m.mbis_rb_edges(ctx, ev["th"], rb[0], rb[1])
                m.mbis_rb_setup(ctx, ev["th"], edges)
                m.mbis_rb_use(ctx, True)
                extra = dict(rb_setup_seconds=time.perf_counter() - t0, coarse_bins=int(len(edges) - 1))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s, nd, nu = m.mbis_run_to_ess(ctx, *bufs, ess_target=target, batch=batch, max_samples=max_samples,
                                          seed=ev["spec"].draw_seed, refine=refine, refine_scale=1.2)
            out.append(dict(seconds=time.perf_counter() - t0, ess=s["ess"], log_z=s["log_z"], drawn=nd, used=nu,
                            reached=bool(s["ess"] >= target), **extra))
        finally:
            m.mbis_destroy(ctx)
    return out


T_SUN = 4.925490947641267e-6


def live_bins(mc, q, f_lo, df, n_bins):
    """Bins f_lo + k df below the Schwarzschild ISCO of the total mass, per sample (the
    work a likelihood does; bins above the cut are not counted)."""
    m_sec = mc * T_SUN * (1.0 + q) ** 1.2 * q ** -0.6
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * m_sec)
    k = np.ceil((f_isco - f_lo) / df)
    return np.clip(np.nan_to_num(k, nan=0.0), 0, n_bins)


def sample_bins(theta, ids, fixed, w):
    """Sum over samples of the live bins (theta: host [P][n])."""
    ids = list(ids)
    mc = theta[ids.index(MC)] if MC in ids else np.full(theta.shape[1], fixed[MC])
    q = theta[ids.index(Q)] if Q in ids else np.full(theta.shape[1], fixed[Q])
    ok = (mc > 0) & (q > 0)
    return float(live_bins(np.where(ok, mc, 1.0), np.where(ok, q, 1.0), w.f_lo, w.df, w.n_bins)[ok].sum())


def likelihood_rate(m, torch, evs, precision, n, reps=3, units=None):
    """Likelihood evaluations / s of mbis_loglike on n proposal samples per event (CUDA
    events); units (list, optional) receives each event's live sample-bins."""
    times = []
    stream = torch.cuda.current_stream()
    for ev in evs:
        w = ev["w"]
        ctx = make_ctx(m, w, ev, precision)
        try:
            P = len(ev["prop"]["ids"])
            theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
            lq, lp, ll = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
            m.mbis_draw(ctx, ev["spec"].draw_seed, 0, n, theta, lq, lp, stream)
            if units is not None:
                units.append(sample_bins(theta.cpu().numpy(), ev["prop"]["ids"], ev["th"], w))
            m.mbis_loglike(ctx, n, theta, ll, stream)   # warm-up
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.mbis_loglike(ctx, n, theta, ll, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
        finally:
            m.mbis_destroy(ctx)
    return n / statistics.mean(times), statistics.mean(times)


def bbh_measurement(m, torch, n_events=2, n=1 << 18):
    w = workloads.bbh_population(n_events=n_events, n_samples=n)
    dn = workloads.network(w.detectors)
    evs = [event_setup(m, w, spec, dn) for spec in w.events]
    units = []
    mixed, t_mixed = likelihood_rate(m, torch, evs, m.MIXED, n, units=units)
    fp64, t_fp64 = likelihood_rate(m, torch, evs, m.FP64, n, reps=1)
    pk = peaks()
    peak = N_SM * SFU_PER_SM_PER_CLK * pk.get("sm_max_mhz", 2070.0) * 1e6 / SFU_PER_BIN / 1e9
    bin_det = statistics.mean(units) * w.n_det        # per launch: live (sample, bin, detector) triples
    achieved = bin_det / t_mixed / 1e9
    # tensor work of the time-shift contraction per likelihood: 3 split-TF32 products of
    # (2 K_eff) x 256 real MACs over the padded live bins of the tile
    return {"workload": "bbh_population: 2 events x 2^18 samples, H1+L1+V1, 8033 bins (df=1/8), 11 sampled "
                        "parameters, time marginalised over 128 shifts of 0.1 ms",
            "mixed_tcgen05": {"value": mixed, "unit": UNIT, "launch_ms": t_mixed * 1e3,
                              "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gbin/s",
                                           "frac": achieved / peak,
                                           "note": "live (sample, bin, detector) triples per launch / launch time "
                                                   "against 2 MUFU per triple"}},
            "fp64": {"value": fp64, "unit": UNIT, "launch_ms": t_fp64 * 1e3},
            "speedup_vs_fp64": mixed / fp64}


def batch_measurement(m, torch, steps=3, warmup=2):
    ws = workloads.uneven_batch()
    t0 = time.time()
    evs = [event_setup(m, w, w.events[0], workloads.network(w.detectors)) for w in ws]
    ctxs = [make_ctx(m, w, ev, m.MIXED) for w, ev in zip(ws, evs)]
    setup_s = time.time() - t0
    try:
        b = m.mbis_batch_create(ctxs, [w.n_samples for w in ws], [w.events[0].draw_seed for w in ws])
        try:
            grid, tune_ms = m.mbis_batch_autotune(b)
            tile, _ = m.mbis_batch_shape(b)
            for i in range(warmup):
                m.mbis_batch_step(b, i, len(ws))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(steps):
                m.mbis_batch_step(b, warmup + i, len(ws))
            dt = (time.perf_counter() - t0) / steps
            # the persistent likelihood launch alone (CUDA events on its stream), and its
            # live sample-bins from the samples of the last step
            units = sum(sample_bins(m.mbis_batch_copy_out(b, i, len(ev["prop"]["ids"]), w.n_samples)[0],
                                    ev["prop"]["ids"], ev["th"], w) for i, (w, ev) in enumerate(zip(ws, evs)))
            stream = torch.cuda.Stream()
            launch = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.mbis_batch_loglike(b, stream)
                e1.record(stream)
                stream.synchronize()
                launch.append(e0.elapsed_time(e1) / 1e3)
        finally:
            m.mbis_batch_destroy(b)
    finally:
        for c in ctxs:
            m.mbis_destroy(c)
    n = sum(w.n_samples for w in ws)
    out = {"workload": "uneven batch: 64 events (heavy and BNS families), 1969-128513 bins, 2-3 detectors, "
                        "2^14-2^20 samples each, one persistent likelihood launch per step, CUDA graph replay",
            "value": n / dt, "unit": UNIT, "ms_per_step": dt * 1e3, "samples_per_step": n, "grid": grid,
            "samples_per_cta": tile,
            "launch_ms": statistics.mean(launch) * 1e3,
            "roofline": {"bound": "alu", "achieved": units / statistics.mean(launch) / 1e9,
                         "peak": N_SM * SFU_PER_SM_PER_CLK * peaks().get("sm_max_mhz", 2070.0) * 1e6 / SFU_PER_BIN / 1e9,
                         "unit": "Gbin/s", "note": "live (sample, bin) pairs per persistent launch / launch time"},
            "autotune_launch_ms": tune_ms, "setup_s": round(setup_s, 2)}
    out["roofline"]["frac"] = out["roofline"]["achieved"] / out["roofline"]["peak"]
    return out




def tiled_measurement(m, torch, reps=3, target=1e4, batch=1 << 14):
    """The tiled proposal of the two-parameter demonstration: template placement, the
    tensor-core tile assignment of the 2^22-point prior pool (CUDA events; roofline in
    useful FP16 tensor flops), the pool's member lists, and the seconds from the template
    likelihoods to 1e4 effective samples."""
    d = workloads.tiled_demo()
    w = d.workload
    spec = w.events[0]
    ev = event_setup(m, w, spec, workloads.network(w.detectors))
    q_max = max(d.q_hi, 1.0 / d.q_lo)
    ev["prop"] = dict(ids=np.array([MC, Q], dtype=np.int32), mean=np.array([25.0, 3.5]), chol=np.diag([0.1, 0.1]),
                      scale=1.0, lo=np.array([d.mc_base, 1.0]), hi=np.array([d.mc_base + d.mc_period, q_max]), flags=0)
    t = m.mbis_tiling_create(w.f_lo, w.df, w.n_bins, ev["psd"][0], d.x_lo, d.x_hi, d.mc_period, d.mc_base, d.q_lo,
                             d.q_hi)
    ctx = make_ctx(m, w, ev, m.MIXED)
    try:
        cand = workloads.uniform_points(d.n_candidates, d.x_lo, d.x_hi, d.q_lo, d.q_hi, d.candidate_seed)
        t0 = time.perf_counter()
        T, used = m.mbis_tiling_bank(t, cand, d.min_match, d.stop_after, d.max_templates)
        bank_s = time.perf_counter() - t0
        _, phys, _ = m.mbis_tiling_templates(t)
        N = d.n_pool
        pool_h = workloads.uniform_points(N, d.x_lo, d.x_hi, d.q_lo, d.q_hi, d.pool_seed)
        pool = torch.tensor(pool_h, dtype=torch.float64, device="cuda")
        tile = torch.empty(N, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        m.mbis_tiling_assign(t, N, pool, tile, None, stream)       # warm-up
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.mbis_tiling_assign(t, N, pool, tile, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        t_assign = statistics.mean(times)
        # useful work: one complex multiply-add (8 flops) per (sample, live bin, template);
        # executed: samples sorted by live-bin count in CTAs of 128, templates sorted the
        # same way in passes of 256 (two MMA blocks of N = 256), each (CTA, pass) running
        # the 32-bin K-blocks that both reach
        mc_p = d.mc_base + np.mod(pool_h[0], d.mc_period)
        qp = np.maximum(pool_h[1], 1.0 / pool_h[1])
        live = live_bins(mc_p, qp, w.f_lo, w.df, w.n_bins)
        useful = 8.0 * float(live.sum()) * T
        srt = np.zeros(((N + 127) // 128) * 128)
        srt[:N] = np.sort(live)
        kb_cta = np.ceil(srt.reshape(-1, 128).max(axis=1) / 32)
        kc_t = np.sort(live_bins(phys[0], phys[1], w.f_lo, w.df, w.n_bins))[::-1]
        kb_pass = np.array([np.ceil(kc_t[i:i + 256].max() / 32) for i in range(0, T, 256)])
        kblocks = float(np.minimum(kb_cta[:, None], kb_pass[None, :]).sum())
        executed = kblocks * 128 * 64 * 512 * 2
        peak = peaks().get("bf16_tflops", 1900.0)   # dense FP16 runs at the BF16 rate
        achieved = useful / t_assign / 1e12
        t0 = time.perf_counter()
        m.mbis_tiling_set_pool(t, N, pool)
        pool_s = time.perf_counter() - t0
        # per event: template likelihoods -> mixture -> batches of draws, likelihoods, weights
        theta = torch.empty((2, batch), dtype=torch.float64, device="cuda")
        lq, lp, ll = (torch.empty(batch, dtype=torch.float64, device="cuda") for _ in range(3))
        th_t = torch.tensor(phys, dtype=torch.float64, device="cuda")
        ll_t = torch.empty(T, dtype=torch.float64, device="cuda")
        runs = []
        for r in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.mbis_loglike(ctx, T, th_t, ll_t)
            m.mbis_tiling_set_loglike(t, ll_t)
            m.mbis_reset_running(ctx)
            drawn = 0
            while True:
                m.mbis_tiling_draw(t, spec.draw_seed + r, drawn, batch, theta, lq, lp)
                m.mbis_loglike(ctx, batch, theta, ll)
                s = m.mbis_reduce(ctx, batch, ll, lp, lq, None, True)
                drawn += batch
                if s["ess"] >= target or drawn >= 1 << 22:
                    break
            runs.append(dict(seconds=time.perf_counter() - t0, ess=s["ess"], drawn=drawn, log_z=s["log_z"]))
    finally:
        m.mbis_destroy(ctx)
        m.mbis_tiling_destroy(t)
    return {"workload": "tiled proposal, two-parameter demonstration (App. A): cyclic chirp mass 24 + mod(x, 4) over "
                        "x in [20, 28), q in [1/6, 6], Mc = 25, q = 3.5 source at SNR 15, H1+L1, 20-128 Hz at 1/4 Hz; "
                        "bank at minimal match 0.996, prior pool of 2^22 points",
            "templates": T, "candidates_visited": used, "bank_seconds": bank_s,
            "assign": {"launch_ms": t_assign * 1e3, "samples_per_s": N / t_assign,
                       "sample_template_matches_per_s": N * T / t_assign,
                       "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                    "frac": achieved / peak,
                                    "note": "useful FP16 tensor flops (8 per sample x live bin x template) per "
                                            "launch / launch time, against the measured dense BF16 burst peak (FP16 "
                                            "runs at the BF16 rate)"},
                       "executed_tflops": executed / t_assign / 1e12, "useful_over_executed": useful / executed},
            "set_pool_seconds": pool_s,
            "seconds_to_1e4_ess": {"median": statistics.median(x["seconds"] for x in runs),
                                   "measured": "template likelihoods + mixture + batches of 2^14 draws, likelihoods "
                                               "and merged weights until ESS >= 1e4 (wall clock)",
                                   "runs": runs},
            "efficiency": statistics.mean(x["ess"] / x["drawn"] for x in runs)}


def pp_population(m, torch, wb, box, n_final=1 << 18, refine=4, refine_scale=1.2, batch=1 << 16,
                  max_samples=1 << 20, ess_ok=2000.0, refit_min_ess=0.0):
    """Credible levels of a population drawn from its analysis prior (box: the prior's
    (Mc, q, t_c) ranges): per source the ESS loop refits the Fisher Gaussian, then one batch
    of n_final draws gives the weighted posterior; KS p-values per parameter and combined,
    over all sources and over those whose final batch reached ESS >= ess_ok (the sources a
    user would accept; the others are proposal failures, counted)."""
    from paper_2410_05190_gb300 import pp
    dn = workloads.network(wb.detectors)
    lv, effs = [], []
    names = [workloads.PARAM_NAMES[i] for i in wb.sampled]
    t0 = time.perf_counter()
    for spec in wb.events:
        ev = event_setup(m, wb, spec, dn)
        for k, slot in enumerate(wb.sampled):   # the population's prior, not a box about the truth
            if slot in box:
                ev["prop"]["lo"][k], ev["prop"]["hi"][k] = box[slot]
        ctx = make_ctx(m, wb, ev, m.MIXED)
        try:
            P = len(ev["prop"]["ids"])
            bufs = ess_buffers(torch, P, batch)
            m.mbis_run_to_ess(ctx, *bufs, ess_target=ess_ok, batch=batch, max_samples=max_samples,
                              seed=spec.draw_seed, refine=refine, refine_scale=refine_scale,
                              refit_min_ess=refit_min_ess)
            th_s = torch.empty((P, n_final), dtype=torch.float64, device="cuda")
            lq, lp, ll, wt = (torch.empty(n_final, dtype=torch.float64, device="cuda") for _ in range(4))
            m.mbis_draw(ctx, spec.draw_seed ^ 0x5EED, 0, n_final, th_s, lq, lp)
            m.mbis_loglike(ctx, n_final, th_s, ll)
            summ = m.mbis_reduce(ctx, n_final, ll, lp, lq, wt)
            lv.append(pp.levels(m, torch, n_final, th_s, wt, [ev["th"][i] for i in wb.sampled]))
            effs.append(summ["ess"] / n_final)
        finally:
            m.mbis_destroy(ctx)
    secs = time.perf_counter() - t0
    lv, ok = np.array(lv), np.array(effs) * n_final >= ess_ok
    pv = {nm: pp.ks_pvalue(lv[:, k]) for k, nm in enumerate(names)}
    pv_ok = {nm: pp.ks_pvalue(lv[ok, k]) for k, nm in enumerate(names)}
    return {"events": len(wb.events), "samples_per_event": n_final, "ks_pvalue": pv,
            "combined_pvalue": pp.combined_pvalue(list(pv.values())),
            "converged": {"ess_at_least": ess_ok, "events": int(ok.sum()), "ks_pvalue": pv_ok,
                          "combined_pvalue": pp.combined_pvalue(list(pv_ok.values()))},
            "median_efficiency": float(np.median(effs)), "seconds": secs,
            "proposal": f"Fisher Gaussian refitted {refine} times (x{refine_scale}) by the ESS loop, "
                        f"batches of {batch}, at most {max_samples} draws"
                        + (f", refit batches pooled to ESS {refit_min_ess:g}" if refit_min_ess > 0 else ""),
            "population": wb.name, "detectors": wb.detectors, "n_bins": wb.n_bins}


def pp_measurement(m, torch, n_tiled=256, n_bns=512, n_bbh=512):
    """P-P self-consistency (Sec. III A): credible levels of the true parameters over
    simulated populations, KS p-value per parameter and Fisher's combination.
    (1) the tiled demonstration: sources drawn from the (x, q) prior, tiled proposal;
    (2) BNS sources drawn from the analysis prior (workloads.bns_pp_population) and (3) BBH
    sources (workloads.bbh_pp_population, intrinsic parameters sampled): the Fisher Gaussian
    refitted by the ESS loop, then one batch."""
    from paper_2410_05190_gb300 import pp
    out = {}
    # (1) tiled
    d = workloads.tiled_demo()
    w = d.workload
    spec = w.events[0]
    dn = workloads.network(w.detectors)
    dets = m.make_detectors(*dn)
    psd1 = m.mbis_psd_aligo(w.f_lo, w.df, w.n_bins)
    psd = np.tile(psd1, (w.n_det, 1))
    t = m.mbis_tiling_create(w.f_lo, w.df, w.n_bins, psd1, d.x_lo, d.x_hi, d.mc_period, d.mc_base, d.q_lo, d.q_hi)
    try:
        cand = workloads.uniform_points(d.n_candidates, d.x_lo, d.x_hi, d.q_lo, d.q_hi, d.candidate_seed)
        T, _ = m.mbis_tiling_bank(t, cand, d.min_match, d.stop_after, d.max_templates)
        _, phys, _ = m.mbis_tiling_templates(t)
        pool = workloads.uniform_points(d.n_pool, d.x_lo, d.x_hi, d.q_lo, d.q_hi, d.pool_seed)
        m.mbis_tiling_set_pool(t, d.n_pool, torch.tensor(pool, device="cuda"))
        an = pp.TiledAnalysis(m, torch, t, phys, (d.mc_base, d.mc_base + d.mc_period),
                              (1.0, max(d.q_hi, 1.0 / d.q_lo)), 1 << 16)
        th0 = np.zeros(11)
        mc0 = (spec.m1 * spec.m2) ** 0.6 / (spec.m1 + spec.m2) ** 0.2
        th0[MC], th0[Q] = mc0, spec.m1 / spec.m2
        for k, v in spec.params.items():
            th0[workloads.PARAM_NAMES.index(k)] = v
        th0[DL] = 1.0
        _, snr2 = m.mbis_inject(w.f_lo, w.df, w.n_bins, dets, psd, spec.gmst, th0)
        dl = math.sqrt(snr2) / spec.snr
        pop = workloads.tiled_population(d, n_tiled)
        lv, eff = [], []
        t0 = time.perf_counter()
        for src in pop:
            th = th0.copy()
            th[MC] = d.mc_base + math.fmod(src["x"], d.mc_period)
            th[Q] = max(src["q"], 1.0 / src["q"])
            th[PHIC] = src["phic"]
            th[DL] = dl
            strain, _ = m.mbis_inject(w.f_lo, w.df, w.n_bins, dets, psd, spec.gmst, th, src["noise_seed"], True)
            levels, summ = an.run(strain.astype(np.complex64), psd, dets, w.f_lo, w.df, th, spec.gmst,
                                  [src["x"], src["q"]], src["draw_seed"])
            lv.append(levels)
            eff.append(summ["ess"] / an.n)
        secs = time.perf_counter() - t0
        lv = np.array(lv)
        pv = {"x": pp.ks_pvalue(lv[:, 0]), "q": pp.ks_pvalue(lv[:, 1])}
        out["tiled_demo"] = {"sources": n_tiled, "samples_per_source": an.n, "ks_pvalue": pv,
                             "combined_pvalue": pp.combined_pvalue(list(pv.values())),
                             "median_efficiency": float(np.median(eff)), "seconds": secs,
                             "sources_per_s": n_tiled / secs}
    finally:
        m.mbis_tiling_destroy(t)
    # (2) BNS, and (3) BBH intrinsic parameters, drawn from their analysis priors, the
    # refitted Gaussian proposal
    out["bns_population"] = pp_population(m, torch, workloads.bns_pp_population(n_events=n_bns), workloads.PP_BOX)
    out["bbh_intrinsic_population"] = pp_population(m, torch, workloads.bbh_pp_population(n_events=n_bbh),
                                                    workloads.PP_BOX_BBH, n_final=1 << 21, refine=8,
                                                    refine_scale=1.5, batch=1 << 16, max_samples=1 << 22,
                                                    refit_min_ess=200.0)
    return out


def rb_measurement(m, torch, evs, n=1 << 20, n_sigma=5.0, eps=0.3, reps=3):
    """Relative binning on the BNS benchmark event: bins from mbis_rb_edges, likelihood rate
    (CUDA events) against the exact fused kernel on the same draws, and its error: per
    sample against the exact log L, and in ESS and log Z; then the ESS loop run on it
    (mbis_rb_use) against the exact loop on every resident event."""
    ev = evs[0]
    w = ev["w"]
    ctx = make_ctx(m, w, ev, m.MIXED)
    try:
        edges = m.mbis_rb_edges(ctx, ev["th"], n_sigma, eps)
        m.mbis_rb_setup(ctx, ev["th"], edges)
        P = len(ev["prop"]["ids"])
        theta = torch.empty((P, n), dtype=torch.float64, device="cuda")
        lq, lp, ll, lr = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4))
        stream = torch.cuda.current_stream()
        m.mbis_draw(ctx, ev["spec"].draw_seed, 0, n, theta, lq, lp, stream)
        m.mbis_loglike(ctx, n, theta, ll, stream)
        m.mbis_rb_loglike(ctx, n, theta, lr, stream)
        times = {"exact": [], "rb": []}
        for _ in range(reps):
            for key, fn in (("exact", lambda: m.mbis_loglike(ctx, n, theta, ll, stream)),
                            ("rb", lambda: m.mbis_rb_loglike(ctx, n, theta, lr, stream))):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                times[key].append(e0.elapsed_time(e1) / 1e3)
        se = m.mbis_reduce(ctx, n, ll, lp, lq)
        sr = m.mbis_reduce(ctx, n, lr, lp, lq)
        a, b, p = ll.cpu().numpy(), lr.cpu().numpy(), lp.cpu().numpy()
        ok = np.isfinite(p)
        lw = a[ok] + p[ok] - lq.cpu().numpy()[ok]
        heavy = lw > lw.max() - 10.0
        err = np.abs(b[ok] - a[ok])
        t_ex, t_rb = statistics.mean(times["exact"]), statistics.mean(times["rb"])
    finally:
        m.mbis_destroy(ctx)
    loops = {"exact": seconds_to_ess(m, torch, evs, m.MIXED), "rb": seconds_to_ess(m, torch, evs, m.MIXED, rb=(n_sigma, eps))}
    ess_loop = {k: {"median_s": statistics.median(x["seconds"] for x in v), "max_s": max(x["seconds"] for x in v),
                    "reached": sum(x["reached"] for x in v), "events": len(v)} for k, v in loops.items()}
    ess_loop["rb"]["rb_setup_s_median"] = statistics.median(x["rb_setup_seconds"] for x in loops["rb"])
    ess_loop["abs_dlogz"] = [abs(a["log_z"] - b["log_z"]) for a, b in zip(loops["rb"], loops["exact"])]
    ess_loop["measured"] = ("mbis_run_to_ess wall time per event to ESS 1e4 (batches of 2^16, 4 refits), exact "
                            "likelihood vs the relative-binning likelihood through mbis_rb_use")
    return {"workload": "bns_population event 0, 2^20 proposal samples, 128,513 bins, phase + distance marginalised",
            "coarse_bins": int(len(edges) - 1), "bins_rule": f"mbis_rb_edges: {n_sigma} proposal sigmas, {eps} rad per bin",
            "rb": {"value": n / t_rb, "unit": UNIT, "launch_ms": t_rb * 1e3},
            "exact": {"value": n / t_ex, "unit": UNIT, "launch_ms": t_ex * 1e3},
            "speedup": t_ex / t_rb,
            "abs_dlogl_posterior_samples": {"median": float(np.median(err[heavy])), "max": float(err[heavy].max()),
                                            "n": int(heavy.sum())},
            "abs_dlogl_all_in_prior": {"median": float(np.median(err)), "p99": float(np.quantile(err, 0.99))},
            "ess_exact": se["ess"], "ess_rb": sr["ess"], "dlogz": sr["log_z"] - se["log_z"],
            "seconds_to_1e4_ess": ess_loop}


SERVE_SEED = 0x5E12E


def serve_requests(m, n_req, rate_hz, seed=SERVE_SEED):
    """The served stream's requests: kind (0 plain-method tiny event, FP64; 1 BNS, mixed;
    2 BBH with full extrinsics, mixed), event set-up, ESS-loop options, Poisson arrival time."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, 3, size=n_req)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_req))
    tiny = workloads.tiny()
    bns = workloads.bns_population(n_events=8)
    bbh = workloads.bbh_population(n_events=8)
    cache, reqs = {}, []
    for i, k in enumerate(kinds):
        w = (tiny, bns, bbh)[k]
        e = 0 if k == 0 else int(rng.integers(0, len(w.events)))
        if (k, e) not in cache:
            cache[(k, e)] = event_setup(m, w, w.events[e], workloads.network(w.detectors))
        ev = cache[(k, e)]
        ess = dict(ess_target=1e4, batch=(1 << 20) if k == 2 else (1 << 16),
                   max_samples=(1 << 25) if k == 2 else (1 << 24), seed=ev["spec"].draw_seed + 1000 * i,
                   refine=4, refine_scale=1.2)
        reqs.append(dict(kind=int(k), ev=ev, w=w, ess=ess, arrival=float(arrivals[i]),
                         precision=m.FP64 if k == 0 else m.MIXED))
    return reqs


RB_RULE = (5.0, 0.3)  # relative-binning bins: proposal sigmas, radians per bin


def submit_request(m, srv, r, precision=None, tag=0, rb_bns=False):
    """rb_bns: a BNS request runs its ESS loop on relative binning about its injection."""
    ev, w, p = r["ev"], r["w"], r["ev"]["prop"]
    rb = dict(rb_fiducial=ev["th"], rb_n_sigma=RB_RULE[0], rb_eps_rad=RB_RULE[1]) if rb_bns and r["kind"] == 1 else {}
    return m.mbis_server_submit(srv, ev["strain"], ev["psd"], ev["dets"], w.f_lo, w.df, ev["th"], p["ids"], p["mean"],
                                p["chol"], p["scale"], p["lo"], p["hi"], prior_flags=p["flags"],
                                gmst=ev["spec"].gmst, precision=r["precision"] if precision is None else precision,
                                marg=w.marg, n_tshift=w.n_tshift, dt_shift=w.dt_shift, dmin=w.dmin, dmax=w.dmax,
                                tag=tag, **r["ess"], **rb)


def percentile(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def serve_measurement(m, torch, n_req=48, rate_hz=2.0, max_active=8, cap=150 * 10**9, rb_bns=False, reqs=None):
    reqs = serve_requests(m, n_req, rate_hz) if reqs is None else reqs
    srv = m.mbis_server_create(hbm_cap_bytes=cap, max_active=max_active)
    try:
        t0 = time.perf_counter()
        ids = []
        for k, r in enumerate(reqs):
            delay = r["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(submit_request(m, srv, r, tag=k, rb_bns=rb_bns)[0])
        res = [m.mbis_server_wait(srv, i, 600.0) for i in ids]
        wall = time.perf_counter() - t0
        st = m.mbis_server_stats_get(srv)
    finally:
        m.mbis_server_destroy(srv)
    ttr = [x["t_done"] - x["t_submit"] for x in res]
    names = ["plain_fp64", "bns_mixed", "bbh_mixed"]
    done = [i for i, x in enumerate(res) if x["summary"]["ess"] >= 1e4]
    by_kind = {}
    for k, name in enumerate(names):
        sel = [i for i, r in enumerate(reqs) if r["kind"] == k]
        if sel:
            by_kind[name] = {"n": len(sel), "p50_s": percentile([ttr[i] for i in sel], 50),
                             "p99_s": percentile([ttr[i] for i in sel], 99),
                             "reached_1e4": sum(res[i]["summary"]["ess"] >= 1e4 for i in sel)}
    return {"workload": f"{n_req} requests, Poisson arrivals at {rate_hz}/s, kinds drawn uniformly from the "
                        "plain-method tiny event (FP64), the BNS population and the BBH population (mixed), "
                        "each run to ESS >= 1e4 with 4 proposal refits (sample caps 2^24, BBH 2^25)" +
                        (f"; BNS requests on relative binning about their injection (bins: {RB_RULE[0]} proposal "
                         f"sigmas, {RB_RULE[1]} rad per bin)" if rb_bns else ""),
            "p50_s": percentile(ttr, 50), "p99_s": percentile(ttr, 99), "mean_s": statistics.mean(ttr),
            # time to result of the requests that reached their target (the others stop at
            # their sample cap: time to give up)
            "reached": {"n": len(done), "p50_s": percentile([ttr[i] for i in done], 50) if done else None,
                        "p99_s": percentile([ttr[i] for i in done], 99) if done else None},
            "throughput_req_s": n_req / wall, "evals_per_s": sum(x["n_drawn"] for x in res) / wall,
            "wall_s": wall, "failed": sum(x["status"] != 0 for x in res), "by_kind": by_kind,
            "max_active": max_active, "max_active_seen": st["max_active_seen"], "hbm_cap_bytes": cap,
            "bytes_peak": st["bytes_peak"]}, reqs, res


def serial_fp64(m, torch, reqs, n_first):
    """Serial FP64 processing of the stream's first n_first requests (each alone, in arrival
    order); time-to-result from the FIFO queue over the measured service times."""
    done, ttr = 0.0, []
    for r in reqs[:n_first]:
        ev, w = r["ev"], r["w"]
        ctx = make_ctx(m, w, ev, m.FP64)
        try:
            bufs = ess_buffers(torch, len(ev["prop"]["ids"]), r["ess"]["batch"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.mbis_run_to_ess(ctx, *bufs, **r["ess"])
            service = time.perf_counter() - t0
        finally:
            m.mbis_destroy(ctx)
        done = max(done, r["arrival"]) + service
        ttr.append(done - r["arrival"])
    return ttr


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--events", type=int, default=4, help="resident events per rank")
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--extras", default="ess,bbh,batch,serve,tiled,pp,rb",
                    help="comma list of further measurements at N=1 (ess, bbh, batch, serve, tiled, pp, rb) or "
                         "'none'")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-compare", type=int, default=3,
                    help="also process the stream's first K requests serially in FP64 (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args)
        return

    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
    out, w, evs = run_gpu(args, rank, world)
    extras = set(x for x in args.extras.split(",") if x and x != "none")
    if rank == 0 and world == 1 and extras:
        import torch
        import paper_2410_05190_gb300 as m
        if "ess" in extras:
            mixed = seconds_to_ess(m, torch, evs, m.MIXED)
            fp64 = seconds_to_ess(m, torch, evs[:2], m.FP64, max_samples=1 << 24)
            out["seconds_to_1e4_ess"] = {
                "measured": "mbis_run_to_ess wall time per event (batches of 2^16, proposal refit after each of "
                            "the first 4 batches, ESS target 1e4)",
                "mixed": {"median": statistics.median(x["seconds"] for x in mixed),
                          "max": max(x["seconds"] for x in mixed), "reached": sum(x["reached"] for x in mixed),
                          "events": len(mixed), "per_event": mixed},
                "fp64_gpu": {"median": statistics.median(x["seconds"] for x in fp64),
                             "max": max(x["seconds"] for x in fp64), "reached": sum(x["reached"] for x in fp64),
                             "events": len(fp64), "per_event": fp64}}
        if "bbh" in extras:
            out["bbh"] = bbh_measurement(m, torch)
        if "batch" in extras:
            out["uneven_batch"] = batch_measurement(m, torch)
        if "tiled" in extras:
            out["tiled_proposal"] = tiled_measurement(m, torch)
        if "pp" in extras:
            out["pp_self_consistency"] = pp_measurement(m, torch)
        if "rb" in extras:
            out["relative_binning"] = rb_measurement(m, torch, evs)
        if "serve" in extras:
            served, reqs, res = serve_measurement(m, torch, n_req=args.serve_requests)
            if args.serve_compare > 0:
                k = min(args.serve_compare, len(reqs))
                ser = serial_fp64(m, torch, reqs, k)
                mix = [res[i]["t_done"] - res[i]["t_submit"] for i in range(k)]
                served["vs_serial_fp64_first_k"] = {"k": k, "serial_fp64_p50_s": percentile(ser, 50),
                                                    "serial_fp64_p99_s": percentile(ser, 99),
                                                    "served_p50_s": percentile(mix, 50),
                                                    "served_p99_s": percentile(mix, 99)}
            out["served"] = served
            # the same stream with the BNS requests on relative binning (the faster likelihood
            # plugged into the served ESS loops)
            served_rb, _, _ = serve_measurement(m, torch, n_req=args.serve_requests, rb_bns=True, reqs=reqs)
            out["served_rb_bns"] = {k: served_rb[k] for k in ("workload", "p50_s", "p99_s", "mean_s", "reached",
                                                              "throughput_req_s", "failed", "by_kind")}
    if rank == 0:
        if world == 1 and args.cpu_budget > 0:
            leg = OracleLeg(w, w.events[:1])
            rate, evals, secs = leg.rate(args.cpu_budget)
            out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": leg.cores, "kind": "oracle",
                                   "sample": f"{evals} likelihoods of the first event ({secs:.1f} s of FP64 oracle "
                                             f"work, OpenMP over samples)",
                                   "one_core": oracle_one_core_rate(w.n_samples, max(2.0, args.cpu_budget / 4))}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle on the same workload, as the reference arm: each step a bounded
    sample of likelihoods of one event (draw -> likelihood -> weights)."""
    w = workloads.bns_population(n_events=max(args.events, 1), n_samples=args.samples)
    leg = OracleLeg(w, w.events[: min(args.events, 2)])
    pilot = leg.batch(0, max(4, leg.cores))
    per_step = max(leg.cores, int(4.0 * max(4, leg.cores) / max(pilot, 1e-3)))
    times = []
    for i in range(args.warmup + args.steps):
        t = leg.batch(i, per_step)
        if i >= args.warmup:
            times.append(t)
    tot_t, tot_n = sum(times), per_step * args.steps
    value = tot_n / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "bns_population: 128513 bins (20-1024 Hz, df=1/128), H1+L1, complex64 data, "
                               f"phase+distance marginalised; each step a bounded sample of {per_step} likelihoods",
                   "n_bins": w.n_bins},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": leg.cores, "kind": "oracle",
                         "sample": f"{tot_n} likelihoods over {args.steps} steps ({tot_t:.1f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
