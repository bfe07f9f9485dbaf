"""Benchmark: messenger-field Wiener-filter solves per second on a
WMAP-shaped problem (HEALPix Nside 512, lmax 1024, FP64, cooling of lambda,
stop at relative increment 1e-6), one JSON line on rank 0.

A step is one whole solve (every iteration of the cooled schedule until the
stop rule holds) of one synthetic data map already resident in HBM. Every N
ranks run their own independent solve (replicas: the problem does not shard),
so scaling is weak and value = solves of all ranks / max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded
sample of the same workload, projected over the same schedule).
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

METRIC = "WF solves/s @Nside512 to 1e-6 a_lm err, mixed vs FP64; SHT-pair ms; p99 latency"
NSIDE, LMAX, TOL = 512, 1024, 1e-6
WORKLOAD = "WMAP-shaped messenger-field Wiener filter, Nside 512 (3,145,728 px), lmax 1024, FP64, " \
           "cooling to relative increment 1e-6"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-mixed, constrained-realisation, Planck-shaped and serving measurements")
    ap.add_argument("--no-planck", action="store_true", help="skip the Planck-shaped (Nside 2048) measurement")
    ap.add_argument("--serving-only", action="store_true", help="run only the config-5 serving measurement")
    ap.add_argument("--planck-only", action="store_true", help="run only the Planck-shaped measurement")
    ap.add_argument("--polarisation-only", action="store_true",
                    help="run only the temperature-and-polarisation measurement (also a profiling target)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--fp64-form", choices=["table", "recurrence", "native"], default="table",
                    help="form of the FP64 solve: double-float kernels reading the precomputed lambda table "
                         "(the plan's default where it fits), the same running the recurrence, or native FP64")
    ap.add_argument("--profile-fp64", type=int, nargs=3, metavar=("NSIDE", "LMAX", "ITERS"), default=None,
                    help="profiling target: ITERS full-band FP64 iterations (wf_profile_iterations) of a "
                         "WMAP-shaped problem at NSIDE / LMAX, the plan's default Legendre form")
    ap.add_argument("--profile-shape", type=int, nargs=2, metavar=("NSIDE", "LMAX"), default=None,
                    help="shape of --profile-batch (default: the bench's Nside 512 / lmax 1024)")
    ap.add_argument("--alu-peaks", action="store_true", help="print the FP64 / FP32 FMA probe's JSON line and exit")
    ap.add_argument("--profile-batch", type=int, nargs=2, metavar=("NRHS", "ITERS"), default=None,
                    help="profiling target: ITERS full-band iterations of the batched engine on NRHS right-hand "
                         "sides of the WMAP-shaped problem (cooling off), one text line, no JSON")
    return ap.parse_args()


FP64_FORMS = {"table": {}, "recurrence": {"legendre_table_bytes": 0}, "native": {"precision": 2}}


class progress:
    """Start / end of a bench section on stderr, with its wall time."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        self.t0 = time.perf_counter()
        print(f"[bench] {self.name} ...", file=sys.stderr, flush=True)

    def __exit__(self, *exc):
        print(f"[bench] {self.name} done in {time.perf_counter() - self.t0:.1f} s", file=sys.stderr, flush=True)


def job_rate(local_seconds, steps, dist=None, device=None):
    """Whole-job rate of `steps` solves on every rank: the slowest rank's time
    (max over ranks) sets it, value = world * steps / that time; a barrier
    closes the timed region on every rank. Returns (value, max seconds)."""
    total = float(local_seconds)
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([total], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
        dist.barrier()
    return world * steps / total, total


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
            "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
            "clocks_event_reasons.sw_power_cap"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_problem(seed):
    from paper_1211_0585_gb300 import inputs as I
    return I.wmap_problem(seed=seed, nside=NSIDE, lmax=LMAX)


LEGENDRE_DF_INSTR = 90    # FP32 instructions per evaluated (l, m, ring pair) term, both passes
# DRAM bytes (read + write) per algorithmic byte of legendre_df_kernel<LEG_ITER, table>: 885.0 MB
# measured by ncu for one launch of `bench.py --profile-fp64 256 512 4` against 864.0 MB algorithmic;
# the full-size launch is scaled by it
TABLE_TRAFFIC_RATIO = 885.04e6 / 864049664


def run_ours(args):
    import torch
    from paper_1211_0585_gb300 import wf

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prob = make_problem(args.seed + rank)
    stream = torch.cuda.Stream()
    opts = wf.options(tol=TOL, max_iter=20000, stream=stream.cuda_stream, **FP64_FORMS[args.fp64_form])
    P = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask, opts)
    # synthetic data d = Y a + n, synthesised by the library itself (setup, untimed)
    a_true = torch.from_numpy(prob.alm_true.view(np.float64).copy()).cuda()
    dmap = torch.empty(prob.npix, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        P.alm2map(LMAX, a_true.data_ptr(), dmap.data_ptr())
    stream.synchronize()
    dmap += torch.from_numpy(prob.noise).cuda()
    torch.cuda.synchronize()
    out = torch.empty(2 * P.nalm, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_solve():
        _, st, status, _ = P.solve(dmap.data_ptr(), out.data_ptr(), on_device=True)
        return st, status

    for _ in range(args.warmup):
        st, status = one_solve()
    # timed region: K solves, events on the plan's stream, L2 flushed between solves
    times = []
    iters = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, status = one_solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(st["iters"])
    torch.cuda.synchronize()
    value, total = job_rate(sum(times), args.steps, dist, device="cuda")
    graph_iters = opts.graph_iters
    per_iter = P.kernels_per_iteration()
    # the iterations' graphs (controller-stopped launches return at once but count), then the posterior
    # gradient: one synthesis, the pixel kernel, two analyses, the norms (r = ring-stage launches)
    r = per_iter - 2
    posterior = (5 + 3 * r) if opts.posterior_grad else 0
    launches_per_solve = [math.ceil(i / graph_iters) * graph_iters * per_iter + posterior for i in iters]

    # SHT pair at full lmax (alm2map + map2alm), events on the stream
    m2 = torch.empty_like(dmap)
    a2 = torch.empty_like(out)
    with torch.cuda.stream(stream):
        for _ in range(2):
            P.alm2map(LMAX, out.data_ptr(), m2.data_ptr())
            P.map2alm(LMAX, m2.data_ptr(), a2.data_ptr())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            P.alm2map(LMAX, out.data_ptr(), m2.data_ptr())
            P.map2alm(LMAX, m2.data_ptr(), a2.data_ptr())
        e1.record(stream)
    e1.synchronize()
    sht_pair_ms = e0.elapsed_time(e1) / 5

    # per-kernel device times of a full-band iteration (the bench's dominant launches)
    s_prof = out.clone()
    prof = P.profile(dmap.data_ptr(), s_prof.data_ptr(), 1.0, LMAX, 10)
    evaluated, full = P.legendre_terms(LMAX)
    held, per_pass = P.legendre_table(LMAX)
    alu = {} if held else measure_alu_peaks()   # the ALU-bound forms' denominators
    fp32_peak = alu.get("fp32_tflops") or 75.3
    # the double-float Legendre kernel: per evaluated (l, m, ring pair) term, one
    # recurrence step (19 FP32 instructions) and two compensated multiply-adds
    # (13 each) in each of the analysis and synthesis passes = 90 FP32
    # instructions; each counted as 2 flops against the FP32 FMA peak
    t_leg = prof["legendre"] * 1e-3
    if held:
        # the table form reads lambda from HBM in both passes: algorithmic bytes
        # per launch = the table rows each pass needs, the ring-pair Fourier
        # coefficients in (analysis) and out (synthesis, every m), the start
        # rows read in both passes, and the a_lm state read and written
        rp = 2 * NSIDE
        nbytes = (2 * per_pass + (LMAX + 1) * rp * 32 * 2 + (LMAX + 1) * rp * 4 * 2 + P.nalm * 16 * 2)
        hbm_peak, src = hbm_peak_gbs()
        achieved = nbytes / t_leg / 1e9
        roofline = {"bound": "hbm", "kernel": "legendre_df_kernel<LEG_ITER, table> (double-float lambda table)",
                    "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(achieved / hbm_peak, 4), "traffic": int(TABLE_TRAFFIC_RATIO * nbytes),
                    "traffic_source": "ncu DRAM bytes of the same kernel at Nside 256 / lmax 512, scaled by "
                                      "the algorithmic bytes",
                    "per_launch_ms": round(prof["legendre"], 4), "algorithmic_bytes_per_launch": nbytes,
                    "table_bytes_held": held, "table_bytes_per_pass": per_pass,
                    "evaluated_terms": evaluated, "full_triangle_terms": full, "peak_source": src,
                    "kernel_ms": {k: round(v, 4) for k, v in prof.items()}}
    elif args.fp64_form == "native":
        # native FP64: per evaluated term and pass 8 flops of contraction + 3 of recurrence, two passes
        flops = 22.0 * evaluated
        fp64_peak = alu.get("fp64_tflops") or 1.25
        achieved = flops / t_leg / 1e12
        roofline = {"bound": "alu", "kernel": "legendre_kernel<LEG_ITER> (native FP64)",
                    "achieved": round(achieved, 4), "peak": round(fp64_peak, 3), "unit": "TFLOP/s",
                    "frac": round(achieved / fp64_peak, 4), "traffic": None,
                    "per_launch_ms": round(prof["legendre"], 4), "algorithmic_flops_per_launch": flops,
                    "evaluated_terms": evaluated, "full_triangle_terms": full,
                    "peak_source": "FP64 FMA rate measured by bench.py's ALU probe in this run"
                    if alu.get("fp64_tflops") else "recorded FP64 FMA probe value (probe unavailable)",
                    "kernel_ms": {k: round(v, 4) for k, v in prof.items()}}
    else:
        flops = 2.0 * LEGENDRE_DF_INSTR * evaluated
        achieved = flops / t_leg / 1e12
        roofline = {"bound": "alu", "kernel": "legendre_df_kernel<LEG_ITER> (double-float on the FP32 pipe)",
                    "achieved": round(achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                    "frac": round(achieved / fp32_peak, 4), "traffic": None,
                    "per_launch_ms": round(prof["legendre"], 4), "algorithmic_flops_per_launch": flops,
                    "evaluated_terms": evaluated, "full_triangle_terms": full,
                    "peak_source": "FP32 FMA rate measured by bench.py's ALU probe in this run"
                    if alu.get("fp32_tflops") else "recorded FP32 FMA probe value (probe unavailable)",
                    "fp64_pipe_tflops": alu.get("fp64_tflops"),
                    "kernel_ms": {k: round(v, 4) for k, v in prof.items()}}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    d_host = torch.empty(prob.npix, dtype=torch.float64).pin_memory()
    d_host.copy_(dmap.cpu())
    alm_host = torch.empty(2 * P.nalm, dtype=torch.float64).pin_memory()
    d_np, a_np = d_host.numpy(), alm_host.numpy().view(np.complex128)
    P.solve(d_np, alm_out=a_np)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.solve(d_np, alm_out=a_np)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": round(args.steps / sum(e2e_t), 6), "unit": "solves/s",
           "h2d_bytes_per_step": prob.npix * 8, "d2h_bytes_per_step": P.nalm * 16}

    # accuracy of the timed result (untimed): against the same solve on the native FP64 kernels, and
    # against the converged solution (the same solve to a relative increment of 1e-9)
    ours = out.cpu().numpy().view(np.complex128).copy()
    accuracy = {}
    if rank == 0 and not args.no_extras:
        Pn = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask,
                     wf.options(tol=TOL, max_iter=20000, precision=wf.WF_PREC_FP64_NATIVE))
        ref_n, st_n, _, _ = Pn.solve(dmap.cpu().numpy())
        Pn.close()
        P.set_options(wf.options(tol=1e-9, max_iter=20000, stream=stream.cuda_stream, **FP64_FORMS[args.fp64_form]))
        ref_c, st_c, _, _ = P.solve(dmap.cpu().numpy())
        P.set_options(opts)
        accuracy = {"rel_l2_vs_fp64_native": rel_l2_alm(ours, ref_n), "fp64_native_iterations": st_n["iters"],
                    "rel_l2_vs_converged_tol1e-9": rel_l2_alm(ours, ref_c), "converged_iterations": st_c["iters"],
                    "note": "a_lm relative L2 (m > 0 weighted x2) of the timed solve's result against the same "
                            "problem solved by the native FP64 kernels, and against the same form run to a "
                            "relative increment of 1e-9"}

    result = {
        "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.fp64_form == "native" else "f32x2+f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "nside": NSIDE, "lmax": LMAX, "npix": prob.npix, "tol": TOL,
                   "precision": ("fp64 native (every step on the FP64 pipe)" if args.fp64_form == "native" else
                                 "fp64 (double-float Legendre and ring FFTs, double updates and reductions)"
                                 + ("; Legendre stage reads a precomputed double-float lambda table" if held else "")),
                   "iterations_per_solve": iters, "parallelism": f"replicas{world}",
                   "stop_rule": "relative increment ||s_k - s_(k-1)|| / ||s_k|| <= 1e-6 at lambda = 1; the "
                                "relative residual of Eq. 2 at the stop is final.rel_posterior_grad, the distance "
                                "to the converged solution final.accuracy",
                   "l2": "flushed (512 MiB write) between timed solves", "seed": args.seed},
        "sht_pair_ms": round(sht_pair_ms, 4),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(sum(launches_per_solve)),
        "clocks": clk.summary(),
        "final": {"chi2_per_dof": st["chi2_per_dof"], "rel_increment": st["rel_increment"],
                  "rel_posterior_grad": st["rel_posterior_grad"],
                  "levels": st["levels"], "status": status, "accuracy": accuracy},
    }
    levels = schedule_levels(P, dmap.cpu().numpy()) if rank == 0 and world == 1 else None
    if rank == 0 and world == 1 and not args.no_extras:
        with progress("mixed_batched"):
            result["mixed_batched"] = mixed_batched(prob, dmap, P, out, flush, nrhs=64)
        with progress("fp64_batched"):
            result["fp64_batched"] = fp64_batched(prob, P, dmap)
        with progress("mixed_batched.roofline"):
            result["mixed_batched"]["roofline"] = batched_roofline(prob)
        with progress("constrained_realisations"):
            result["constrained_realisations"] = constrained_realisations_run(prob, dmap)
        P.close()
        torch.cuda.empty_cache()
        with progress("small"):
            result["small"] = small_run()
        with progress("multi"):
            result["multi"] = multi_run(prob)
        with progress("polarisation"):
            result["polarisation"] = polarisation_run()
        torch.cuda.empty_cache()
        if not args.no_planck:
            with progress("planck"):
                result["planck"] = planck_run()
            torch.cuda.empty_cache()
        with progress("serving"):
            result["serving"] = serving_run(weights=SERVING_BENCH_WEIGHTS)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(prob, dmap.cpu().numpy(), levels=levels, budget_s=25.0)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def mixed_batched(prob, dmap, P64, out64, flush, nrhs=64):
    """Config 4: nrhs constrained-realisation style right-hand sides
    d_i = Y (a + a_i) + n_i sharing the mask and noise, solved by the batched
    mixed-precision engine (FP32 Lambda table GEMMs, FP32 FFTs, double state
    and controller). Reports solves/s and the a_lm error of one right-hand
    side against the FP64 path."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    draws = I.fluctuation_draws(prob, nrhs, seed0=1)
    D = torch.empty((nrhs, prob.npix), dtype=torch.float64, device="cuda")
    a = torch.empty(2 * P64.nalm, dtype=torch.float64, device="cuda")
    for i, (a_i, n_i) in enumerate(draws):
        a.copy_(torch.from_numpy((prob.alm_true + a_i).view(np.float64)))
        P64.alm2map(LMAX, a.data_ptr(), D[i].data_ptr())
        torch.cuda.synchronize()
        D[i] += torch.from_numpy(n_i).cuda()
    Pm = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask,
                 wf.options(precision=wf.WF_PREC_MIXED, tol=TOL, max_iter=20000, batch_slots=min(nrhs, 64)))
    outm = torch.empty((nrhs, 2 * P64.nalm), dtype=torch.float64, device="cuda")
    # engine, tables and ring-stage autotuning for nrhs slots (as a server loads its model), then the timed run
    Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=outm.data_ptr(), nrhs=nrhs)
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, stats, status = Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=outm.data_ptr(), nrhs=nrhs)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # FP64 solves of the first n_err right-hand sides (spread over the engine's slots) for the error
    n_err = min(nrhs, 8)
    errs = []
    for i in range(n_err):
        P64.solve(D[i].data_ptr(), out64.data_ptr(), on_device=True)
        torch.cuda.synchronize()
        errs.append(rel_l2_alm(outm[i].cpu().numpy().view(np.complex128), out64.cpu().numpy().view(np.complex128)))
    iters = [s["iters"] for s in stats]
    Pm.close()
    return {"solves_per_s": round(nrhs / dt, 4), "nrhs": nrhs, "seconds": round(dt, 3), "status": status,
            "iterations_mean": round(float(np.mean(iters)), 1),
            "rel_l2_vs_fp64_max": max(errs), "rel_l2_vs_fp64_mean": float(np.mean(errs)),
            "rel_l2_vs_fp64_n": n_err,
            "precision": "FP32 ring FFTs (two slots per complex FFT); Legendre GEMMs on tcgen05 tensor cores "
                         "(kind::tf32, 22-bit tables, exact 3-way split of the FP32 data, five products, "
                         "double-float chunk sums); double-float state and Eq. 4; FP32 Eq. 3; double "
                         "reductions and controller",
            "timing": "host wall clock around wf_solve_batch with device-resident inputs"}


def serving_requests(n, rng, shapes, weights=None):
    """n requests of config 5: Nside uniform over `shapes`, lmax = 2 Nside, C_l amplitude x U[0.5, 2],
    per-request hit map and mask (10-30 % band cut plus 0-1000 discs of 0.5 deg), tol 1e-5 (mixed) or
    1e-8 (FP64) with equal odds. Pixel noise keeps the Nside 512 map's power per steradian."""
    from paper_1211_0585_gb300 import inputs as I
    geo = {}
    for ns, _ in shapes:
        z, phi = I.pixel_centres(ns)
        geo[ns] = (z, phi, np.abs(I.sin_ecliptic_latitude(z, phi)))
    out = []
    for _ in range(n):
        ns, lm = shapes[rng.choice(len(shapes), p=weights)]
        z, phi, sb = geo[ns]
        cut = rng.uniform(0.1, 0.3)
        mask = I.mask_discs(z, phi, I.mask_band(z, cut), int(rng.integers(0, 1001)), 0.5, rng)
        h = 1.0 + 7.0 * sb * rng.uniform(0.5, 1.5)
        var = 2200.0 ** 2 / h * (ns / 512.0) ** 2   # pixel area ~ 1 / Nside^2: same noise power per sr
        cl = I.cl_lcdm_like(lm, 13.0 * 512 / ns) * rng.uniform(0.5, 2.0)
        d = rng.standard_normal(len(z)) * np.sqrt(var) + rng.standard_normal(len(z)) * np.sqrt(cl[2:40].sum())
        out.append((ns, lm, cl, var, mask, d, 1e-8 if rng.random() < 0.5 else 1e-5))
    return out


SERVING_SHAPES = [(128, 256), (256, 512), (512, 1024), (1024, 2048)]
# the bench line's stream: Nside 1024 at a low share (its FP64 solves take ~16 s of a worker each, so at the
# uniform mix a 200-request window would take many minutes); --serving-only runs the uniform mix
SERVING_BENCH_WEIGHTS = [0.3, 0.3, 0.3, 0.1]


def serving_run(n_burst=24, n_stream=200, load=0.8, seed=3, max_batch=16, weights=None):
    """Config 5: requests of four shapes (Nside 128 / 256 / 512 / 1024, lmax = 2 Nside; drawn with
    `weights`, uniform when None) and two tolerances through wf_server. Capacity: a burst of n_burst
    requests submitted at once, completed solves / time (the throughput of the saturated server). Then a
    Poisson stream at `load` x that capacity for n_stream requests: p50 / p99 latency (submit to result on
    the host), solves/s, per shape and path."""
    from paper_1211_0585_gb300 import wf
    rng = np.random.default_rng(seed)
    shapes = SERVING_SHAPES
    t_gen = time.perf_counter()
    burst = serving_requests(n_burst, rng, shapes, weights)
    t_gen = time.perf_counter() - t_gen
    S = wf.Server(hbm_budget_bytes=0, max_batch=max_batch)
    t_warm = time.perf_counter()
    for ns, lm in shapes:  # the shapes are made resident before the requests, as a server loads its models
        S.warm(ns, lm, wf.WF_PREC_MIXED)
        S.warm(ns, lm, wf.WF_PREC_FP64)
    t_warm = time.perf_counter() - t_warm

    def collect(tickets):
        rows = []
        for t, ns, tol in tickets:
            res = S.poll(t)
            rows.append((ns, "fp64" if tol <= 1e-7 else "mixed", res[1]["ms_latency"], res[2]))
        return rows

    t0 = time.perf_counter()
    tk = [(S.submit(ns, lm, cl, var, mask, d, tol), ns, tol) for ns, lm, cl, var, mask, d, tol in burst]
    t1 = time.perf_counter()
    stream = serving_requests(n_stream, rng, shapes, weights)   # generated on the host while the burst is served
    t_gen += time.perf_counter() - t1
    print(f"[bench] serving: burst of {n_burst} submitted; stream inputs generated", file=sys.stderr, flush=True)
    S.drain(3600000)
    # all submitted at t0: the last completion (its latency) closes the burst, however long the host took
    # to generate the stream meanwhile
    t_burst = max(r[2] for r in collect(tk)) / 1e3 + (t1 - t0)
    capacity = n_burst / t_burst
    rate = load * capacity
    print(f"[bench] serving: capacity {capacity:.3f} / s, stream of {n_stream} at {rate:.3f} / s",
          file=sys.stderr, flush=True)
    gaps = rng.exponential(1.0 / rate, n_stream)
    t0 = time.perf_counter()
    tk = []
    for (ns, lm, cl, var, mask, d, tol), g in zip(stream, gaps):
        tk.append((S.submit(ns, lm, cl, var, mask, d, tol), ns, tol))
        time.sleep(g)
    t_sub = time.perf_counter() - t0
    S.drain(3600000)
    wall = time.perf_counter() - t0
    rows = collect(tk)
    S.close()
    lat = np.array([r[2] for r in rows])

    def summary(sel):
        v = lat[sel]
        return {"n": int(v.size), "p50_ms": round(float(np.percentile(v, 50)), 1),
                "p99_ms": round(float(np.percentile(v, 99)), 1)} if v.size else {"n": 0}

    per_shape = {f"nside{ns}": summary(np.array([r[0] == ns for r in rows])) for ns, _ in shapes}
    per_path = {k: summary(np.array([r[1] == k for r in rows])) for k in ("fp64", "mixed")}
    return {"saturation_rate_per_s": round(capacity, 3),
            "saturation": f"{n_burst} requests submitted at once, solves / time to drain ({t_burst:.1f} s)",
            "rate_per_s": round(rate, 3), "load_vs_saturation": load, "requests": n_stream,
            "arrival_s": round(t_sub, 1), "wall_s": round(wall, 1), "solves_per_s": round(n_stream / wall, 3),
            "p50_ms": round(float(np.percentile(lat, 50)), 1), "p99_ms": round(float(np.percentile(lat, 99)), 1),
            "statuses_ok": int(sum(r[3] == 0 for r in rows)), "per_shape": per_shape, "per_path": per_path,
            "max_batch": max_batch, "shapes": "Nside 128/256/512/1024, lmax = 2 Nside, drawn with weights "
                                              + ("uniform" if weights is None else str(weights)),
            "tol_mix": "1e-5 (mixed engine) / 1e-8 (FP64 pool), equal odds", "warm_s": round(t_warm, 1),
            "config5_rate_50_per_s": f"{50.0 / capacity:.1f} x the measured capacity: above saturation, the "
                                     "queue would grow without bound, so the stream runs at `load` x capacity",
            "note": f"inputs generated on the host ({t_gen:.0f} s; the stream's while the burst is served); the "
                    "four shapes made resident (wf_server_warm: mixed engine and one FP64 plan each) before "
                    "any request"}


def fp64_batched(prob, P64, dmap, nrhs=8):
    """FP64 solves of nrhs right-hand sides d + n_i through wf_solve_batch (pairs sharing the Legendre
    stage), against the single-solve rate of the same plan."""
    import torch
    D = torch.stack([dmap + torch.from_numpy(np.random.default_rng(50 + i).standard_normal(prob.npix)
                                             * np.sqrt(prob.noise_var)).cuda() for i in range(nrhs)])
    out = torch.empty((nrhs, 2 * P64.nalm), dtype=torch.float64, device="cuda")
    P64.solve_batch(D.data_ptr(), on_device=True, alm_out=out.data_ptr(), nrhs=nrhs)   # per-map buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, stats, status = P64.solve_batch(D.data_ptr(), on_device=True, alm_out=out.data_ptr(), nrhs=nrhs)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"solves_per_s": round(nrhs / dt, 4), "nrhs": nrhs, "seconds": round(dt, 3), "status": status,
            "iterations_mean": round(float(np.mean([s["iters"] for s in stats])), 1),
            "note": "pairs of right-hand sides share one Legendre launch per iteration (each lambda-table row "
                    "read once per group); every result equals its single FP64 solve bit for bit; host wall "
                    "clock, the posterior gradient of each result included"}


def batched_roofline(prob, nrhs=64, iters=12):
    """Full-band iterations of the 64-slot mixed engine (cooling off, lambda = 1): ms per iteration and
    its HBM roofline, the algorithmic bytes of one batched iteration being the FP32 Legendre tables read
    by the two GEMMs, the Fourier arrays written and read by the ring stage, the GEMM operands, and each
    slot's data and inverse noise."""
    import torch
    from paper_1211_0585_gb300 import wf
    Pm = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask,
                 wf.options(tol=0.0, max_iter=iters, cooling=0, precision=wf.WF_PREC_MIXED, batch_slots=nrhs))
    D = torch.from_numpy(np.stack([prob.noise] * nrhs)).cuda()
    out = torch.empty((nrhs, 2 * Pm.nalm), dtype=torch.float64, device="cuda")
    Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=out.data_ptr(), nrhs=nrhs)   # engine, autotune
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=out.data_ptr(), nrhs=nrhs)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / iters
    Pm.close()
    rp, npix = 2 * NSIDE, 12 * NSIDE * NSIDE
    nalm = (LMAX + 1) * (LMAX + 2) // 2
    rows = sum((LMAX - m + 2) // 2 for m in range(LMAX + 1))
    table = 2 * rows * 2 * rp * 4                       # two FP32 tables, rows of one parity, both parities
    fourier = 4 * (LMAX + 1) * rp * 16 * nrhs           # FS read + FT written (ring stage), XT, FS (GEMMs)
    data = npix * 8 * nrhs                              # (d, w) FP32 per slot
    state = 2 * nalm * 16 * nrhs                        # double-float state read and written
    nbytes = table + fourier + data + state
    peak, src = hbm_peak_gbs()
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "batched mixed engine, one full-band iteration (ring stage, XT, "
                                      "analysis and synthesis tcgen05 GEMMs, controller)",
            "ms_per_iteration": round(ms, 3), "nrhs": nrhs, "algorithmic_bytes_per_iteration": nbytes,
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "peak_source": src, "timing": f"host wall clock over {iters} full-band iterations of all slots"}


def planck_run(iters=8, slots=8, seed=1):
    """Config 3 (Planck-shaped, Nside 2048 / lmax 4096): the same data map through the FP64 path (double-
    float recurrence form: the lambda table would take 275 GB) and the mixed engine with one slot and with
    `slots` slots, `iters` fixed iterations at lambda = 1 (cooling off); ms per iteration per right-hand
    side and the mixed result's relative a_lm distance to the FP64 one."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    ns, lm = 2048, 4096
    t_gen = time.perf_counter()
    prob = I.planck_problem(seed=seed, nside=ns, lmax=lm)
    t_gen = time.perf_counter() - t_gen
    o = dict(tol=0.0, max_iter=iters, cooling=0, posterior_grad=0)
    P = wf.Plan(ns, lm, prob.cl, prob.noise_var, prob.mask, wf.options(**o))
    a = torch.from_numpy(prob.alm_true.view(np.float64).copy()).cuda()
    d = torch.empty(prob.npix, dtype=torch.float64, device="cuda")
    P.alm2map(lm, a.data_ptr(), d.data_ptr())
    torch.cuda.synchronize()
    d += torch.from_numpy(prob.noise).cuda()
    del a
    ref = torch.empty(2 * P.nalm, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st, _, _ = P.solve(d.data_ptr(), ref.data_ptr(), on_device=True)
    torch.cuda.synchronize()
    fp64_ms = 1e3 * (time.perf_counter() - t0) / iters
    P.close()
    out = {"workload": "Planck-shaped, Nside 2048 (50,331,648 px), lmax 4096, 5' beam, lognormal hits, 25 % cut",
           "iterations": iters, "fp64_ms_per_iteration": round(fp64_ms, 2)}
    for b in (1, slots):
        Pm = wf.Plan(ns, lm, prob.cl, prob.noise_var, prob.mask,
                     wf.options(precision=wf.WF_PREC_MIXED, batch_slots=b, **o))
        D = d.repeat(b)
        res = torch.empty(b * 2 * P.nalm, dtype=torch.float64, device="cuda")
        Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=res.data_ptr(), nrhs=b)   # engine and tables
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=res.data_ptr(), nrhs=b)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / iters
        err = rel_l2_alm(res[:2 * P.nalm].cpu().numpy().view(np.complex128), ref.cpu().numpy().view(np.complex128),
                         lm)
        out[f"mixed_{b}slot_ms_per_iteration"] = round(ms, 2)
        out[f"mixed_{b}slot_ms_per_rhs_iteration"] = round(ms / b, 2)
        out[f"mixed_{b}slot_rel_l2_vs_fp64"] = err
        Pm.close()
        del D, res
        torch.cuda.empty_cache()
    out["note"] = f"host generation of the inputs {t_gen:.0f} s; timing: host wall clock around solves of " \
                  f"{iters} iterations (FP64: one map; mixed: the same map in every slot)"
    return out


def polarisation_run(iters=10, seed=1):
    """Temperature and polarisation at the bench size (WMAP-shaped T + P, Nside 512 / lmax 1024): ms per
    full-band iteration of wf_pol_solve (fixed iterations, lambda = 1) and of its transform pair."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    pp = I.pol_wmap_problem(seed=seed, nside=NSIDE, lmax=LMAX)
    Q = wf.Pol(NSIDE, LMAX, pp.cls, pp.noise_cov, pp.mask_t, pp.mask_p,
               wf.options(tol=0.0, max_iter=iters, cooling=0))
    a = torch.from_numpy(pp.alm_true.view(np.float64).copy().reshape(-1)).cuda()
    m = torch.empty(3 * 12 * NSIDE * NSIDE, dtype=torch.float64, device="cuda")
    Q.alm2map(a.data_ptr(), m.data_ptr())
    torch.cuda.synchronize()
    d = m.cpu().numpy().reshape(3, -1) + pp.noise
    Q.solve(d)                                   # graph capture
    t0 = time.perf_counter()
    _, st, _, _ = Q.solve(d)
    ms_it = 1e3 * (time.perf_counter() - t0) / iters
    # the pair runs on the plan's own stream: a device-wide synchronize on both sides brackets it
    a2 = torch.empty_like(a)
    Q.alm2map(a.data_ptr(), m.data_ptr())
    Q.map2alm(m.data_ptr(), a2.data_ptr())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        Q.alm2map(a.data_ptr(), m.data_ptr())
        Q.map2alm(m.data_ptr(), a2.data_ptr())
    torch.cuda.synchronize()
    pair = 1e3 * (time.perf_counter() - t0) / 5
    Q.close()
    return {"workload": "WMAP-shaped T + P, Nside 512 / lmax 1024, 3x3 pixel noise, T and P masks",
            "ms_per_iteration": round(ms_it, 2), "iterations": iters, "transform_pair_ms": round(pair, 2),
            "chi2_per_dof_after": st["chi2_per_dof"],
            "timing": "host wall clock around wf_pol_solve of fixed full-band iterations, and around five "
                      "wf_pol_alm2map + wf_pol_map2alm pairs between device synchronizes"}


def small_run(iters=200, seed=1, reps=3):
    """The small configuration (Nside 16 / lmax 32, FP64, lambda = 1, no cooling): microseconds per
    iteration over a fixed 200-iteration solve, data resident on the device (host clock around
    wf_solve, the shortest of `reps` solves). At this size an iteration is a few launches of tiny
    kernels, so the number measures launch and graph overhead, not bandwidth."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    prob = I.small_problem(seed=seed)
    d = torch.from_numpy(prob.data(np.zeros(prob.npix))).cuda()
    P = wf.Plan(16, 32, prob.cl, prob.noise_var, prob.mask, wf.options(tol=0.0, max_iter=iters, cooling=0))
    out = torch.empty(2 * P.nalm, dtype=torch.float64, device="cuda")
    P.solve(d.data_ptr(), out.data_ptr(), on_device=True)   # graph capture
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st, _, _ = P.solve(d.data_ptr(), out.data_ptr(), on_device=True)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    P.close()
    return {"workload": "Nside 16 (3,072 px), lmax 32, FP64, 200 iterations at lambda = 1",
            "us_per_iteration": round(1e6 * best / iters, 2), "iterations": st["iters"],
            "chi2_per_dof": st["chi2_per_dof"],
            "timing": f"host wall clock around wf_solve (device-resident data), shortest of {reps}; the "
                      f"posterior gradient after the solve included"}


def multi_run(prob, iters=10):
    """Several messenger fields at the bench size: two maps of the WMAP-shaped sky (13' and 30' beams, the
    second with twice the noise and its own mask), ms per full-band iteration of wf_multi_solve."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    ell = np.arange(LMAX + 1)
    beams = [np.ones(LMAX + 1), np.exp(-0.5 * ell * (ell + 1) * (math.radians(30.0 / 60) / math.sqrt(8 * math.log(2))) ** 2)]
    cl = prob.cl
    z, phi = I.pixel_centres(NSIDE)
    mask2 = I.mask_band(z, 0.3)
    var2 = 2.0 * prob.noise_var
    rng = np.random.default_rng(9)
    M = wf.Multi(NSIDE, LMAX, cl, [prob.noise_var, var2], [prob.mask, mask2], beams,
                 wf.options(tol=0.0, max_iter=iters, cooling=0))
    d1 = prob.data(np.zeros(prob.npix))
    d2 = rng.standard_normal(prob.npix) * np.sqrt(var2)
    M.solve([d1, d2])                           # graph capture
    t0 = time.perf_counter()
    M.solve([d1, d2])
    ms_it = 1e3 * (time.perf_counter() - t0) / iters
    M.close()
    return {"workload": "two maps of the WMAP-shaped sky, Nside 512 / lmax 1024 (13' and 30' beams)",
            "ms_per_iteration": round(ms_it, 2), "iterations": iters,
            "timing": "host wall clock around wf_multi_solve of fixed full-band iterations"}


def constrained_realisations_run(prob, dmap, nreal=63):
    """Config 4's constrained realisations through wf_constrained_realisations on the mixed plan: nreal
    realisations and the Wiener filter of d in one 64-slot batch."""
    from paper_1211_0585_gb300 import wf
    Pm = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask,
                 wf.options(precision=wf.WF_PREC_MIXED, tol=TOL, max_iter=20000, batch_slots=nreal + 1))
    d = dmap.cpu().numpy()
    Pm.constrained_realisations(d, nreal, seed=7)           # engine and tables
    t0 = time.perf_counter()
    cr, wfd, stats, status = Pm.constrained_realisations(d, nreal, seed=8)
    dt = time.perf_counter() - t0
    Pm.close()
    return {"realisations_per_s": round(nreal / dt, 3), "nreal": nreal, "seconds": round(dt, 3),
            "status": status, "iterations_mean": round(float(np.mean([s["iters"] for s in stats])), 1),
            "timing": "host wall clock around wf_constrained_realisations (host data in, host results out; "
                      "draws, syntheses and the 64 Wiener filters on the device)"}


def rel_l2_alm(a, b, lmax=None):
    """Relative L2 distance of two a_lm vectors (lmax = LMAX by default), m > 0 weighted x2."""
    lmax = LMAX if lmax is None else lmax
    m = np.concatenate([np.full(lmax + 1 - mm, mm) for mm in range(lmax + 1)])
    wgt = np.where(m == 0, 1.0, 2.0)
    return float(np.sqrt(np.sum(wgt * np.abs(a - b) ** 2) / np.sum(wgt * np.abs(b) ** 2)))


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU type (MEASURED_PEAKS.json at the
    repository root), else the recorded fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured STREAM-style copy (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (no measured peak file)"


# FP64 / FP32 FMA throughput probe (the denominators of the ALU-bound kernels'
# rooflines): each thread runs 8 independent FMA chains; one JSON line.
ALU_PROBE_SRC = r"""
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_loop(T *out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T>
double tflops(int blocks, int threads, int iters) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_loop<T><<<blocks, threads>>>(out, 10, (T)0.999, (T)1e-3);
  cudaDeviceSynchronize();
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-3);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double f = 2.0 * 8 * 16 * (double)iters * blocks * threads / (ms * 1e9);
    if (f > best) best = f;
  }
  cudaFree(out);
  return best;
}
int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) { printf("{\"error\": \"no device\"}\n"); return 1; }
  const int sms = p.multiProcessorCount;
  const double f64 = tflops<double>(sms * 4, 256, 1000);
  const double f32 = tflops<float>(sms * 8, 256, 10000);
  printf("{\"device\": \"%s\", \"sms\": %d, \"fp64_tflops\": %.4f, \"fp32_tflops\": %.4f}\n",
         p.name, sms, f64, f32);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
"""


def measure_alu_peaks():
    """FP64 / FP32 FMA throughput of this GPU: the probe above, compiled for
    sm_103a into a temporary directory and run once."""
    import tempfile
    try:
        from paper_1211_0585_gb300 import build as B
        with tempfile.TemporaryDirectory() as tmp:
            src, exe = os.path.join(tmp, "alu_peak.cu"), os.path.join(tmp, "alu_peak")
            with open(src, "w") as f:
                f.write(ALU_PROBE_SRC)
            subprocess.run([B.nvcc(), *B.ARCH, "-O3", "-o", exe, src], check=True, capture_output=True, timeout=300)
            out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception:
        return {}


def schedule_levels(P, d):
    """The (lambda, lmax_SHT, n_iter) levels of one GPU solve of d."""
    _, st, _, recs = P.solve(d, history=20001)
    levels = []
    for r in recs:
        if levels and levels[-1][0] == r["lam"] and levels[-1][1] == r["lsht"]:
            levels[-1][2] += 1
        else:
            levels.append([r["lam"], r["lsht"], 1])
    return levels


def cpu_baseline(prob, d, P=None, budget_s=25.0, levels=None):
    """Time the FP64 oracle as it stands on the host cores: one oracle iteration
    at every band limit of the solve's schedule, projected over the schedule's
    iteration counts (solves/s)."""
    from oracle import oracle as O
    O.build_oracle()
    if levels is None:
        levels = schedule_levels(P, d)
    tau = O.messenger_tau(prob.noise_var, prob.mask)
    w = O.inverse_noise(prob.noise_var, prob.mask)
    omega = 4 * math.pi / prob.npix
    per = {}
    t_all = time.perf_counter()
    s = np.zeros(O.nalm_of(LMAX), dtype=np.complex128)
    for lam, lsht, n in sorted(levels, key=lambda x: x[1]):
        if lsht in per:
            continue
        t0 = time.perf_counter()
        O.messenger_step(NSIDE, LMAX, lsht, s, d, w, O.pixel_gain(lam, tau, w),
                         O.harmonic_filter(lam, tau, omega, prob.cl), prob.cl, lam, tau)
        per[lsht] = time.perf_counter() - t0
        if time.perf_counter() - t_all > budget_s:
            break
    missing = [l for _, l, _ in levels if l not in per]
    if missing:
        return {"value": None, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                "sample": f"over budget before band limits {sorted(set(missing))}"}
    t_solve = sum(n * per[l] for _, l, n in levels)
    n_it = sum(n for _, _, n in levels)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    return {"value": round(1.0 / t_solve, 8), "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": f"one oracle iteration at each band limit {sorted(per)} "
                      f"(s per iteration {[round(per[k], 2) for k in sorted(per)]}), projected over the "
                      f"{n_it}-iteration schedule of the GPU solve",
            "seconds_per_solve_projected": round(t_solve, 2),
            "one_core": oracle_one_core()}


def oracle_one_core(timeout_s=120):
    """The oracle on one host core (OMP_NUM_THREADS=1, a child process): seconds per iteration of the
    Nside 512 problem at band limit 120 (the schedule's first level), of the Nside 16 / lmax 32 problem,
    and the same two on all cores, for the speedup of the threaded oracle."""
    import subprocess
    code = ("import json, math, time, numpy as np, bench\n"
            "from oracle import oracle as O\n"
            "from paper_1211_0585_gb300 import inputs as I\n"
            "O.build_oracle()\n"
            "out = {}\n"
            "for tag, prob, ns, lm, lsht in (('nside512_lsht120', bench.make_problem(1), 512, 1024, 120),\n"
            "                                ('nside16_lmax32', I.small_problem(seed=1), 16, 32, 32)):\n"
            "    d = prob.data(O.alm2map(ns, lm, prob.alm_true))\n"
            "    tau = O.messenger_tau(prob.noise_var, prob.mask); w = O.inverse_noise(prob.noise_var, prob.mask)\n"
            "    s = np.zeros(O.nalm_of(lm), dtype=np.complex128); reps = 1 if ns > 16 else 20\n"
            "    t0 = time.perf_counter()\n"
            "    for _ in range(reps):\n"
            "        O.messenger_step(ns, lm, lsht, s, d, w, O.pixel_gain(1.0, tau, w),\n"
            "                         O.harmonic_filter(1.0, tau, 4 * math.pi / prob.npix, prob.cl), prob.cl, 1.0, tau)\n"
            "    out[tag] = (time.perf_counter() - t0) / reps\n"
            "print(json.dumps(out))\n")
    res = {}
    for cores in (1, os.cpu_count()):
        env = dict(os.environ, OMP_NUM_THREADS=str(cores))
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                               timeout=timeout_s, cwd=os.path.dirname(os.path.abspath(__file__)))
            vals = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            vals = None
        res[f"{cores}_cores"] = {k: round(v, 5) for k, v in vals.items()} if vals else None
    res["unit"] = "s per oracle iteration (lambda = 1)"
    return res


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    prob = make_problem(args.seed)
    from oracle import oracle as O
    # A whole oracle solve at this size takes tens of minutes, so the oracle is
    # timed for one iteration at each band limit of the solve's schedule and the
    # time is projected over that schedule's iteration counts (DEFAULT_LEVELS,
    # the levels of the seed-1 solve; WF_BENCH_LEVELS may override them).
    d = prob.data(O.alm2map(NSIDE, LMAX, prob.alm_true))
    levels = json.loads(os.environ.get("WF_BENCH_LEVELS", "[]")) or DEFAULT_LEVELS
    t0 = time.perf_counter()
    base = cpu_baseline(prob, d, levels=levels, budget_s=120.0)
    elapsed = time.perf_counter() - t0
    result = {"metric": METRIC, "value": base["value"], "unit": "solves/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": round(1e3 / base["value"], 1) if base["value"] else None,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
              "data": "synthetic", "impl": "reference",
              "config": {"workload": WORKLOAD, "nside": NSIDE, "lmax": LMAX, "tol": TOL, "precision": "fp64",
                         "parallelism": "host cores"},
              "cpu_baseline": {k: base[k] for k in ("kind", "cores", "sample")} | {"value": base["value"]},
              "e2e": {"value": base["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
              "wall_s": round(elapsed, 1)}
    print(json.dumps(result), flush=True)


# levels of the GPU solve of seed 1 (lambda, lmax_SHT, iterations)
DEFAULT_LEVELS = [[6.1793721184416155, 120, 5], [1.575, 140, 4], [1.0, 1024, 342]]


def profile_batch(nrhs, iters, seed, shape=None):
    """A fixed amount of full-band batched work for ncu captures: every
    iteration runs at lambda = 1 and lmax_SHT = lmax (cooling off)."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    NSIDE, LMAX = shape if shape else (globals()["NSIDE"], globals()["LMAX"])
    prob = I.wmap_problem(seed=seed, nside=NSIDE, lmax=LMAX)
    P64 = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask, wf.options(legendre_table_bytes=0))
    Pm = wf.Plan(NSIDE, LMAX, prob.cl, prob.noise_var, prob.mask,
                 wf.options(tol=0.0, max_iter=iters, cooling=0, precision=wf.WF_PREC_MIXED,
                            batch_slots=min(64, nrhs)))
    a = torch.from_numpy(prob.alm_true.view(np.float64).copy()).cuda()
    base = torch.empty(prob.npix, dtype=torch.float64, device="cuda")
    P64.alm2map(LMAX, a.data_ptr(), base.data_ptr())
    torch.cuda.synchronize()
    D = torch.stack([base + torch.from_numpy(np.random.default_rng(seed + i).standard_normal(prob.npix)
                                             * np.sqrt(prob.noise_var)).cuda() for i in range(nrhs)])
    out = torch.empty((nrhs, 2 * Pm.nalm), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, status = Pm.solve_batch(D.data_ptr(), on_device=True, alm_out=out.data_ptr(), nrhs=nrhs)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(f"full-band batched: {nrhs} right-hand sides x {iters} iterations in {dt:.3f} s "
          f"({1e3 * dt / iters:.2f} ms / iteration, status {status})", flush=True)


def profile_fp64(nside, lmax, iters, seed, form="table"):
    """A fixed amount of full-band FP64 work for ncu captures (lambda = 1,
    lmax_SHT = lmax): one synthesis launch, then per iteration the ring,
    Legendre and controller launches."""
    import torch
    from paper_1211_0585_gb300 import inputs as I
    from paper_1211_0585_gb300 import wf
    prob = I.wmap_problem(seed=seed, nside=nside, lmax=lmax)
    P = wf.Plan(nside, lmax, prob.cl, prob.noise_var, prob.mask, wf.options(**FP64_FORMS[form]))
    d = torch.from_numpy(prob.data(np.zeros(prob.npix))).cuda()
    s = torch.zeros(2 * P.nalm, dtype=torch.float64, device="cuda")
    held, per_pass = P.legendre_table(lmax)
    ms = P.profile(d.data_ptr(), s.data_ptr(), 1.0, lmax, iters)
    print(f"full-band FP64 at Nside {nside} / lmax {lmax}: {iters} iterations, ms per launch "
          f"{ {k: round(v, 4) for k, v in ms.items()} }, lambda table held {held} B, {per_pass} B per pass",
          flush=True)


def main():
    args = parse()
    if args.alu_peaks:
        print(json.dumps(measure_alu_peaks()), flush=True)
        return
    if args.profile_fp64:
        profile_fp64(*args.profile_fp64, args.seed, args.fp64_form)
        return
    if args.serving_only or args.planck_only or args.polarisation_only:
        import torch
        torch.cuda.set_device(0)
        run = serving_run if args.serving_only else planck_run if args.planck_only else polarisation_run
        print(json.dumps(run()), flush=True)
        return
    if args.profile_batch:
        profile_batch(args.profile_batch[0], args.profile_batch[1], args.seed, args.profile_shape)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
