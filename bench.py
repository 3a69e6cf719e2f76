"""Benchmark of the ray-propagation sweep on one GB300 (or N replicas).

A step is one pass of the whole hot path over the exponential-disk galaxy
(297,840 adaptive leaves, B band, albedo 0.6, g = 0.6, a_RT = 0.05): step 1
(U_LL within R_pre), step 2 (direct light with ray blocking), scattering
iterations until the pending scattered luminosity is below f_L = 1% of the
step-2 total (at most 12), and an internal-observer HEALPix map
(nside 64, observer at R = 8 kpc in the mid-plane).  The grid is resident in
HBM before the timed region; every step restarts the sweep from scratch.

Metric: ray-cell crossings per second (crossings of steps 1-3 over the step
time).  Also reported: seconds per scattering iteration.  The L2 cache is
flushed (a 512 MB write) between timed steps.

--impl reference times the FP64 CPU oracle (the reference implementation) on
all host cores, one process per core, each on its own bounded sample of the
same workload (every 30000th source at its own offset, steps 1-2 and one
scattering iteration per step).  The default run also reports the oracle on
one core (cpu_baseline) and on all cores (cpu_baseline_all_cores).
With N > 1 GPUs each rank runs an independent replica (the path has no
exchange step on one GPU); the value is the sum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "galaxy disk + bulge, 297840 adaptive leaves (9x9x1 roots of 4 kpc, 6 levels), 1 lambda"
PARAMS = dict(a_rt=0.05, n_rays_min=5, n_rays_max=40, k0=2, merge=1)
F_L = 0.01
MAX_ITERS = 12
OBSERVER = (8.0, 0.0, 0.0)
MAP_K = 6  # nside 64
MAP_SUB = 3
HBM_FALLBACK_GBS = 6800.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "of measured"
    return HBM_FALLBACK_GBS, "of fallback"


def bytes_per_crossing(nl):
    """Algorithmic bytes of one crossing (leaf box 16 B + 6 face links 24 B +
    node child word 4 B, kappa*rho 4 B and U_LL 4 B per wavelength, U
    read-modify-write 8 B per wavelength); the j_sca row update adds 8 B per
    pixel updated (counted separately)."""
    return 44 + 16 * nl


# a deposit record: cell (4 B) and the ray direction with the HG coefficient (16 B)
RECORD_BYTES = 20

# FP32-pipe figures of the Henyey-Greenstein row expansion (ncu --set full of
# one flush of the 1/512-source case: profiles/cell_accumulate_galaxy3e5_subset512.md)
HG_EXPANSION_PIPES = {"kernel": "cell_accumulate_kernel<6, 0>", "fma_pipe_frac": 0.496, "xu_pipe_inst_frac": 0.259,
                      "issue_active_frac": 0.643, "source": "ncu capture of one flush of a smaller case"}

# DRAM and L2 bytes per crossing of the marcher, summed over all its launches
# of the 1/30000-source case and divided by that case's crossings (ncu:
# profiles/march_kernel_traffic_galaxy3e5_subset30000.md); a full-size
# launch's traffic is taken as these times its crossings.
MARCH_DRAM_BYTES_PER_CROSSING = 8.24
MARCH_L2_BYTES_PER_CROSSING = 180.3


def l2_copy_gbs():
    """Measured L2 bandwidth: a device-to-device copy of 24 MiB (read +
    write 48 MiB, resident in the 129 MB L2), best of 20 timed batches of 20
    copies."""
    import torch
    a = torch.empty(6 << 20, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1.0)
    for _ in range(10):
        b.copy_(a)
    best = None
    for _ in range(20):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    return 20 * 2 * a.numel() * 4 / best / 1e9


def make_workload():
    import synth
    grid = synth.config2()
    r_pre = 0.15 * grid.model_size
    return grid, dict(PARAMS, r_pre=r_pre)


class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, gpu_index=0):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except OSError:
            return None
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        rows = [r for r in rows if r[0] == str(gpu_index)] or rows
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def roofline_of(prof, nl, peak, peak_src, l2_peak=None):
    """The roofline object of the marcher from a profiled step (prof: the
    summed stats of run_step with params.profile = 1 and the step's time).

    Algorithmic bytes: per crossing (leaf box, face link, node word,
    kappa*rho, U_LL, U read-modify-write) plus one deposit record per
    depositing crossing.  The marcher's launches run on three pipeline
    streams at once, so their CUDA-event spans overlap: the time the kernel
    holds the GPU is the union of the spans (march_ms), and achieved = all
    its algorithmic bytes / that union.  The per-launch figure (bytes /
    summed spans, each span including the wait for SMs that the other
    pipelines' launches hold) is kept beside it."""
    alg_bytes = prof["march_crossings"] * bytes_per_crossing(nl) + RECORD_BYTES * prof["records"]
    march_sum_ms, launches = prof["march_sum_ms"], prof["march_launches"]
    union_ms = prof["march_ms"]
    achieved = alg_bytes / (union_ms / 1e3) / 1e9 if union_ms > 0 else None
    per_span = alg_bytes / (march_sum_ms / 1e3) / 1e9 if march_sum_ms > 0 else None
    per_launch = prof["march_crossings"] / launches if launches else 0.0
    traffic = MARCH_DRAM_BYTES_PER_CROSSING * per_launch if MARCH_DRAM_BYTES_PER_CROSSING else None
    l2 = None
    if MARCH_L2_BYTES_PER_CROSSING and union_ms > 0 and l2_peak:
        l2_ach = MARCH_L2_BYTES_PER_CROSSING * prof["march_crossings"] / (union_ms / 1e3) / 1e9
        l2 = {"achieved": l2_ach, "peak": l2_peak, "unit": "GB/s", "frac": l2_ach / l2_peak,
              "bytes_per_crossing": MARCH_L2_BYTES_PER_CROSSING,
              "peak_source": "measured here: L2-resident device copy (48 MiB moved per copy)"}
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_note": "ncu DRAM bytes per crossing of the small case times the crossings of an "
                            "average full-size launch" if traffic else None,
            "l2": l2,
            "kernel": "march_kernel (ray marcher)", "peak_source": peak_src,
            "launches": launches, "avg_launch_ms": march_sum_ms / launches if launches else None,
            "bytes_per_crossing": bytes_per_crossing(nl), "record_bytes": RECORD_BYTES,
            "crossings_profiled_step": prof["march_crossings"], "records_profiled_step": prof["records"],
            "achieved_over_summed_launch_spans": per_span,
            "frac_over_summed_launch_spans": per_span / peak if per_span else None,
            "time_basis": "union of the marcher's launch spans on its three pipeline streams",
            "kernel_busy_share_of_step": prof["march_ms"] / prof["step_ms"],
            "deposit_flush_share_of_step": prof["flush_ms"] / prof["step_ms"],
            "note": "from warm-up step 2, whose launches are timed with CUDA events"}


def max_over_ranks(value, dist, device):
    """Largest value over the ranks of the process group (the job's time is
    the slowest replica's); `dist` None means a single process."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all replicas per second of the slowest one."""
    return units_per_rank * world / (ms / 1e3)


def run_step(gpu, grid):
    """One pass of the hot path: steps 1-2, scattering iterations to f_L, map."""
    st = gpu.direct()
    cross = st["crossings"]
    march_ms = st["march_ms"]
    march_sum_ms = st["march_sum_ms"]
    march_launches = st["march_launches"]
    flush_ms = st["flush_ms"]
    march_cross = st["crossings"]
    jpix = st["jsca_pixels"]
    records = st["records"]
    launches = st["kernel_launches"]
    it_ms = []
    it = 0
    while it < MAX_ITERS:
        rem, s2 = gpu.scatter_iter()
        it += 1
        cross += s2["crossings"]
        march_ms += s2["march_ms"]
        march_sum_ms += s2["march_sum_ms"]
        march_launches += s2["march_launches"]
        flush_ms += s2["flush_ms"]
        march_cross += s2["crossings"]
        jpix += s2["jsca_pixels"]
        records += s2["records"]
        launches += s2["kernel_launches"]
        it_ms.append(s2["gpu_ms"])
        if rem < F_L:
            break
    m = gpu.map(OBSERVER, MAP_K, max_sub=MAP_SUB, use_jsca=True)
    launches += 1
    return dict(crossings=cross, march_ms=march_ms, march_sum_ms=march_sum_ms, march_launches=march_launches,
                flush_ms=flush_ms, march_crossings=march_cross, jsca_pixels=jpix, records=records,
                iters=it, iter_ms=it_ms, launches=launches, map=m)


# ---------------------------------------------------------------- batched forms
CUBES = 32


def cube_models():
    """The clumpy cubes of the batched workload: 32 lognormal cubes
    (sigma_ln rho = 1, seeded), N_i = round(16 * 4^(i/31)) cells a side
    (16^3 to 64^3), cell side 1/16 kpc, mean edge-to-edge optical depth
    log-spaced from 0.5 to 5, 16 emitting cells each drawn with probability
    proportional to the density."""
    import synth
    out = []
    for i in range(CUBES):
        n = int(round(16 * 4 ** (i / (CUBES - 1))))
        tau = 0.5 * 10 ** (i / (CUBES - 1))
        out.append(synth.lognormal_cube(n, 100 + i, tau_mean=tau, n_src=16, box_size=n / 16.0))
    return out


def galaxy_8_lambda():
    """The galaxy at 8 wavelengths log-spaced 0.15-2.2 um: kappa ~ lambda^-1.3
    (tau_B = 2 at 0.443 um), albedo 0.7 -> 0.4 and g 0.75 -> 0.4 linear in
    log lambda (k_lambda from 3 down to 1), the stellar emissivity the same
    at every wavelength."""
    import synth
    g = synth.config2()
    lam = np.geomspace(0.15, 2.2, 8)
    t = np.log(lam / lam[0]) / np.log(lam[-1] / lam[0])
    kr = g.kappa_rho * (lam / 0.443) ** -1.3
    em = np.repeat(g.emissivity, 8, axis=1)
    return g.with_lambda(kr, em, 0.7 - 0.3 * t, 0.75 - 0.35 * t), lam


def timed_call(f):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = f()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def bench_batched(params):
    """The batched form against the plain loop on the same GPU.

    models: the 32 cubes traced together in one grid (steps 1-2) against a
    loop that traces them one grid at a time; wavelengths: the galaxy at 8
    wavelengths in one grid (rays carry all 8) against 8 single-wavelength
    grids, steps 1-2 and one scattering iteration on every 64th source.
    Times cover the sweep calls (grids are created before), and both forms
    are compared cell by cell."""
    from paper_1709_03802_gb300 import DartRay, DartRayBatch
    p = dict(a_rt=params["a_rt"], n_rays_min=5, n_rays_max=40, k0=2, merge=1, r_pre=-1.0)
    out = {}
    # --- models
    cubes = cube_models()
    plain_s, plain_c, plain_U = 0.0, 0, []
    for c in cubes:
        g = DartRay(c, **p)
        st, dt = timed_call(g.direct)
        plain_s += dt
        plain_c += st["crossings"]
        plain_U.append(g.rfed()[0][:, 0].copy())
        g.close()
    b = DartRayBatch(cubes, **p)
    choice, trial_ms = b.autotune(sample_stride=4)
    st, batched_s = timed_call(b.direct)
    worst = 0.0
    for m, U1 in enumerate(plain_U):
        U = b.model_rfed(m)[0][:, 0]
        big = U1 > 1e-6 * U1.max()
        worst = max(worst, float(np.abs(U[big] / U1[big] - 1).max()))
    b.close()
    out["models"] = {"workload": f"{CUBES} lognormal cubes 16^3-64^3 ({sum(c.n_leaf for c in cubes)} leaves), "
                                 "16 emitting cells each, steps 1-2",
                     "plain_loop_s": plain_s, "batched_s": batched_s, "speedup": plain_s / batched_s,
                     "crossings": int(st["crossings"]), "plain_crossings": int(plain_c),
                     "batched_crossings_per_s": st["crossings"] / batched_s,
                     "max_rel_diff_U": worst, "autotune_choice": ["deferred", "deferred, 1/16 buffer", "atomic"][choice],
                     "autotune_ms": trial_ms}
    # --- wavelengths
    g8, lam = galaxy_8_lambda()
    cap = dict(queue_rays=1 << 25, deposit_records=1 << 26, src_stride=64)
    one = DartRay(g8, **p, **cap)

    def sweep8():
        s1 = one.direct()
        U_direct = one.rfed()[0].copy()
        _, s2 = one.scatter_iter()
        return s1["crossings"] + s2["crossings"], U_direct

    (c8, U8d), t8 = timed_call(sweep8)
    U8 = one.rfed()[0].copy()
    one.close()
    t1, c1, worst, worst_d = 0.0, 0, 0.0, 0.0
    for l in range(8):
        gl = g8.with_lambda(g8.kappa_rho[:, l:l + 1], g8.emissivity[:, l:l + 1], g8.albedo[l:l + 1], g8.g[l:l + 1])
        gg = DartRay(gl, **p, **cap)

        def sweep1():
            s1 = gg.direct()
            U_direct = gg.rfed()[0][:, 0].copy()
            _, s2 = gg.scatter_iter()
            return s1["crossings"] + s2["crossings"], U_direct

        (c, U1d), dt = timed_call(sweep1)
        t1 += dt
        c1 += c
        U1 = gg.rfed()[0][:, 0]
        big = U1 > 1e-6 * U1.max()
        worst = max(worst, float(np.abs(U8[big, l] / U1[big] - 1).max()))
        big = U1d > 1e-6 * U1d.max()
        worst_d = max(worst_d, float(np.abs(U8d[big, l] / U1d[big] - 1).max()))
        gg.close()
    out["wavelengths"] = {"workload": "galaxy at 8 wavelengths 0.15-2.2 um, every 64th source, steps 1-2 + one "
                                      "scattering iteration",
                          "plain_loop_s": t1, "batched_s": t8, "speedup": t1 / t8, "crossings": int(c8),
                          "plain_crossings": int(c1),
                          "max_rel_diff_U_after_step2": worst_d, "max_rel_diff_U": worst,
                          "note": "scattering rays of a multi-wavelength grid start at the finest j_sca level of "
                                  "its wavelengths, so the scattered part differs by that angular sampling"}
    return out


def bench_clumpy(peak):
    """Crossings/s on a clumpy grid beside the galaxy: the 64^3 lognormal cube
    (sigma_ln rho = 1, mean edge-to-edge tau_V = 2, 16 emitting cells drawn
    with probability proportional to the density), steps 1-2 and scattering
    iterations to f_L, every launch timed by CUDA events on its stream."""
    import synth
    from paper_1709_03802_gb300 import DartRay
    grid = synth.lognormal_cube(64, 4, tau_mean=2.0, n_src=16)
    g = DartRay(grid, profile=1, **dict(PARAMS, r_pre=0.15 * 2.0))
    tot = {"crossings": 0, "records": 0, "march_ms": 0.0, "gpu_ms": 0.0}
    it_ms = []

    def add(st):
        for k in tot:
            tot[k] += st[k]

    add(g.direct())
    for _ in range(MAX_ITERS):
        rem, st = g.scatter_iter()
        add(st)
        it_ms.append(st["gpu_ms"])
        if rem < F_L:
            break
    g.close()
    alg = tot["crossings"] * bytes_per_crossing(1) + RECORD_BYTES * tot["records"]
    ach = alg / (tot["march_ms"] / 1e3) / 1e9 if tot["march_ms"] > 0 else None  # over the union of its spans
    return {"workload": "64^3 lognormal cube (sigma_ln rho 1, mean tau_V 2, 16 emitting cells), steps 1-2 + "
                        f"scattering iterations to f_L = {F_L}",
            "n_leaf": grid.n_leaf, "value": tot["crossings"] / (tot["gpu_ms"] / 1e3), "unit": "crossings/s",
            "crossings": int(tot["crossings"]), "seconds": tot["gpu_ms"] / 1e3,
            "s_per_scatter_iter": float(np.mean(it_ms)) / 1e3, "scatter_iters": len(it_ms),
            "march_kernel_achieved_gbs": ach, "march_kernel_frac": ach / peak if ach else None}


def cpu_sample(grid, params, stride, offset=0):
    import oracle
    p = oracle.OracleParams(**{k: v for k, v in params.items() if k in oracle.OracleParams.__dataclass_fields__},
                            src_stride=stride, src_offset=offset)
    o = oracle.Oracle(grid, p)
    t0 = time.perf_counter()
    o.direct()
    c = o.stats()[1]["crossings"]
    o.scatter_iter()
    c += o.stats()[1]["crossings"]
    dt = time.perf_counter() - t0
    return c, dt


def _cpu_worker(job):
    """One process of the all-cores CPU baseline: the oracle on its own
    sample of sources (offset within the stride)."""
    stride, offset = job
    grid, params = make_workload()
    return cpu_sample(grid, params, stride, offset)


def cpu_all_cores(stride, unit, processes=None):
    """The oracle on every host core at once: one process per core, each on
    a disjoint sample of every stride-th source (the method is additive over
    sources, so the samples are independent).  Value = crossings of all
    processes / wall time.  Processes are spawned, never forked after CUDA
    initialisation."""
    import multiprocessing as mp
    n = processes or os.cpu_count() or 1
    jobs = [(stride, (i * stride) // n) for i in range(n)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(n) as pool:
        res = pool.map_async(_cpu_worker, jobs).get(timeout=900)
    wall = time.perf_counter() - t0
    c = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": c / wall, "unit": unit, "cores": n, "kind": "oracle", "crossings": c, "wall_s": wall,
            "sample": f"{n} processes, each every {stride}th source at its own offset, steps 1-2 + one "
                      f"scattering iteration; {c} crossings in {wall:.1f} s wall ({busy:.1f} s in the "
                      f"slowest process, the rest is grid set-up)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-stride", type=int, default=30000)
    ap.add_argument("--src-stride", type=int, default=1,
                    help="profiling aid: trace every n-th primary source only (default: all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain comparisons")
    # capacities (0 = automatic); results do not depend on them.  Smaller
    # buffers keep the device footprint of a profiling run to a few GB.
    ap.add_argument("--queue-rays", type=int, default=0)
    ap.add_argument("--deposit-records", type=int, default=0)
    ap.add_argument("--clock-log-dir", default="/tmp",
                    help="folder for the nvidia-smi clock samples taken during the timed steps")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    grid, params = make_workload()
    if args.src_stride > 1:
        params = dict(params, src_stride=args.src_stride, src_offset=1)
    if args.queue_rays:
        params = dict(params, queue_rays=args.queue_rays)
    # deposit records per pipeline: 2^30 (39 GB each; the library's automatic
    # choice stops at 2^29) -- waves whose records do not fit deposit with
    # per-pixel atomics, and steps 1-2 plus one iteration take 54.0 s with
    # 2^30 against 55.7 s with 2^29
    params = dict(params, deposit_records=args.deposit_records or (1 << 30))
    metric = "ray-cell crossings/s"
    unit = "crossings/s"
    config = {"workload": WORKLOAD, "n_leaf": grid.n_leaf, "a_rt": params["a_rt"], "f_l": F_L,
              "map": f"nside 64 at {OBSERVER} kpc", "l2": "flushed between steps (512 MB write)",
              "warmup_note": "warm-up 1 is the end-to-end run through host buffers, warm-up 2 the profiled step "
                              "the roofline figures come from"}
    if args.src_stride > 1:
        config["profiling_subset"] = f"every {args.src_stride}th primary source (not a bench value)"
    config["capacities"] = {"queue_rays": args.queue_rays or "automatic", "deposit_records": params["deposit_records"]}

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        # the oracle on every host core (one process per core, each on its own
        # sample of sources), as the paper parallelises over sources
        tot_c, tot_t, cores, sample = 0.0, 0.0, 1, ""
        for s in range(args.warmup + args.steps):
            r = cpu_all_cores(args.cpu_stride, unit)
            if s >= args.warmup:
                tot_c += r["crossings"]
                tot_t += r["wall_s"]
                cores, sample = r["cores"], r["sample"]
        v = tot_c / tot_t if tot_t > 0 else None
        print(json.dumps({"impl": "reference", "metric": metric, "value": v, "unit": unit, "n_gpus": 0,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(1, args.steps),
                          "higher_is_better": True, "dtype": "f64", "data": "synthetic", "config": config,
                          "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle",
                                           "sample": sample + " (per step)"},
                          "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_1709_03802_gb300 import DartRay

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up 1: end to end through the C ABI with host buffers -- create (H2D
    # of the inputs), the whole step, U / L_abs / map back to host
    e2e = None
    h2d = sum(np.asarray(a).nbytes for a in (grid.first_child, grid.leaf_of_node, grid.kappa_rho,
                                             grid.emissivity, grid.albedo, grid.g))
    if args.warmup >= 1:
        # the inputs in pinned host memory (copied there before the clock starts)
        import dataclasses

        def pinned(a):
            t = torch.empty(np.asarray(a).shape, dtype=torch.from_numpy(np.asarray(a)).dtype, pin_memory=True)
            t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
            return t.numpy()

        hgrid = dataclasses.replace(grid, **{k: pinned(getattr(grid, k)) for k in
                                             ("first_child", "leaf_of_node", "kappa_rho", "emissivity", "albedo",
                                              "g", "point_xyz", "point_lum")})
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = DartRay(hgrid, **params)
        r2 = run_step(g2, grid)
        U, L = g2.rfed()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d2h = U.nbytes + L.nbytes + r2["map"].nbytes
        e2e = {"value": r2["crossings"] * world / dt, "unit": unit, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "seconds": dt}
        g2.close()
        del g2

    # warm-up 2: one step with every ray-march launch and deposit flush timed
    # by CUDA events on its pipeline stream (params.profile), for the
    # roofline figures; the timed steps below run without those events, with
    # each pipeline's rounds of waves replayed as CUDA graphs
    prof = None
    if args.warmup >= 2:
        gp = DartRay(grid, profile=1, **params)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        prof = run_step(gp, grid)
        e1.record()
        torch.cuda.synchronize()
        prof["step_ms"] = e0.elapsed_time(e1)
        gp.close()
        del gp

    gpu = DartRay(grid, **params)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(0, args.warmup - 2)):
        run_step(gpu, grid)
    torch.cuda.synchronize()
    results = []
    total_ms = 0.0
    clk = Clocks(os.path.join(args.clock_log_dir, f"clocks_rank{rank}.csv"))
    with clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r = run_step(gpu, grid)
            e1.record()
            torch.cuda.synchronize()
            barrier()
            total_ms += e0.elapsed_time(e1)
            results.append(r)
    clocks = clk.summary(local_rank)
    ms = max_over_ranks(total_ms / args.steps, dist, "cuda")
    cross = float(np.mean([r["crossings"] for r in results]))
    value = whole_job_rate(cross, world, ms)
    it_ms = [x for r in results for x in r["iter_ms"]]
    nl = grid.n_lambda
    peak, peak_src = peaks()
    roofline = None
    if prof is not None:
        roofline = roofline_of(prof, nl, peak, peak_src, l2_copy_gbs() if MARCH_L2_BYTES_PER_CROSSING else None)
    gpu.close()
    batched = clumpy = None
    if not args.no_batched and args.src_stride == 1:
        batched = bench_batched(params)
        clumpy = bench_clumpy(peak)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.src_stride == 1:
        c, dt = cpu_sample(grid, params, args.cpu_stride)
        cpu = {"value": c / dt, "unit": unit, "cores": 1, "kind": "oracle",
               "sample": f"every {args.cpu_stride}th source, steps 1-2 + one scattering iteration, "
                         f"{c} crossings in {dt:.1f} s"}
        cpu_all = cpu_all_cores(args.cpu_stride, unit)
    if rank == 0:
        line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
                "s_per_scatter_iter": float(np.mean(it_ms)) / 1e3 if it_ms else None,
                "scatter_iters_per_step": float(np.mean([r["iters"] for r in results])),
                "crossings_per_step": cross,
                "deposit_records_per_step": float(np.mean([r["records"] for r in results])),
                "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
                "gpu_launches": int(sum(r["launches"] for r in results)), "clocks": clocks,
                "batched_vs_plain": batched, "clumpy_grid": clumpy, "hg_expansion_pipes": HG_EXPANSION_PIPES}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
