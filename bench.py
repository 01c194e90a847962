"""Benchmark of the Gamma-point periodic J/K build on one GB300 (or N replicas).

One step = one J+K build (every row of the hot path: real-space quartets,
reciprocal structure factors and contractions, background, assembly) of the
water-box workload (64 H2O, 832 basis functions, omega = 0.4, thresholds
1e-14) with D already resident in HBM; the timed region covers exactly
--steps builds bracketed by a barrier and device synchronisation.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "JK builds/s & quartets/s, mixed vs FP64 same GB300, |ΔE|≤1µHa; p50/p99 latency"
WORKLOAD = "water64: 64 H2O, a=12.42 A, 832 bf (576 shells), omega=0.4, thresholds 1e-14"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


WORKLOADS = {
    "water64": (WORKLOAD, lambda sc: sc.config(2)),
    # same density and basis, 16 molecules: the small case for ncu captures
    "water16": ("water16: 16 H2O, a=7.82 A, 208 bf, omega=0.4, thresholds 1e-14",
                lambda sc: sc.water_cell(16, 12.42 / 4 ** (1.0 / 3.0), omega=0.4, n_occ=64, geo_purpose=3)),
    # the large single cell: 6x6x6 diamond, 1728 atoms, s(6) s(4) p(1), 8640 bf
    "large1728": ("large1728: diamond 6x6x6, 1728 atoms, a=21.40 A, 8640 bf, omega=0.4, Schwarz 1e-11",
                  lambda sc: sc.config(5)),
    # the diamond supercell: 3x3x3, 216 atoms, s(6) s(3) p(1) d(1), 2376 bf
    "diamond216": ("diamond216: diamond 3x3x3, 216 atoms, a=10.70 A, 2376 bf, omega=0.5", lambda sc: sc.config(3)),
}


def make_workload(name="water64"):
    import synthcells as sc

    return WORKLOADS[name][1](sc)


# ---------------------------------------------------------------------------------------------
def oracle_sample(cell, D, n_bra=40, n_g=2):
    """One bounded oracle sample: n_bra strided bra local pairs against every
    ket local pair (real space) and n_g reciprocal vectors (pair transforms,
    Coulomb and one exchange row), extrapolated to a full build."""
    from oracle import oracle as O

    nlp = O.pair_counts(cell)[2]
    full_s, det = O.jk_sample_seconds(cell, D, max(1, nlp // n_bra), n_g)
    return full_s, det


def run_reference(args):
    """The FP64 CPU oracle on the host cores (the reference arm of this
    build), each step a bounded sample of the same water-box build,
    extrapolated to builds/s."""
    from oracle import oracle as O

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cell = make_workload(args.workload)
    D = O.density(cell)
    fulls, samples = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        full_s, det = oracle_sample(cell, D, n_bra=32)
        if i >= args.warmup:
            fulls.append(full_s)
            samples.append(time.perf_counter() - t)
    full = statistics.mean(fulls)
    value = 1.0 / full
    out = {
        "metric": METRIC, "value": value, "unit": "builds/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": full * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "parallelism": "host cores (OpenMP)", "l2": "n/a"},
        "cpu_baseline": {"value": value, "unit": "builds/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": "per step: 32 strided bra local pairs of %d against all kets plus 2 of %d G vectors, "
                                   "extrapolated to a full build (%.1f s of CPU work per step)"
                                   % (det["local_pairs"], det["n_g"], statistics.mean(samples))},
        "e2e": {"value": value, "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def cpu_baseline_sample(cell, D):
    """The oracle timed on a bounded sample of the same build (about 10-30 s)."""
    from oracle import oracle as O

    t = time.perf_counter()
    full_s, det = oracle_sample(cell, D, n_bra=320)
    took = time.perf_counter() - t
    return {"value": 1.0 / full_s, "unit": "builds/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d strided bra local pairs of %d against all kets and 2 of %d G vectors (%.1f s), extrapolated to a "
                      "full J+K build (%.0f s)" % (det["bra_sampled"], det["local_pairs"], det["n_g"], took, full_s)}


def serve_stream(reqs, prec, slots, budget_bytes, iters, plan_precision_name):
    """Serve `reqs` (synthcells.Request, Poisson arrival times) through the
    library's request server: one client thread per request sleeps until its
    arrival, creates the request's plan (resident on the device), and submits
    its SCF iterations one after another (each a fresh density perturbation
    of norm 1e-3) while other requests' builds run.  Returns latency and
    throughput figures."""
    import threading

    import torch

    import synthcells as sc
    from paper_2410_22278_gb300 import jk

    dev = torch.device("cuda:0")
    srv = jk.Server(device=0, hbm_budget_bytes=int(budget_bytes), max_slots=slots)
    lat_build, lat_req, nbf = [], [], []
    lock = threading.Lock()
    errors = []
    t0 = time.perf_counter()

    def serve(r):
        try:
            arrive = t0 + (r.arrival_s - reqs[0].arrival_s)
            time.sleep(max(0.0, arrive - time.perf_counter()))
            t_arr = time.perf_counter()
            cell = r.cell
            plan = jk.plan_from_cell(cell, precision=prec)
            n = cell.nbf
            S = torch.empty((n, n), dtype=torch.float64, device=dev)
            plan.overlap(S.data_ptr(), 0)
            torch.cuda.synchronize()
            D0 = sc.density_from_overlap(cell.orbital_guess(), S.cpu().numpy())
            J = torch.empty((n, n), dtype=torch.float64, device=dev)
            K = torch.empty_like(J)
            for it in range(iters(r)):
                Dk = torch.from_numpy(D0 + sc.density_perturbation((r.rid << 8) + it, n)).to(dev)
                torch.cuda.synchronize()
                tk = srv.submit(plan, Dk.data_ptr(), J.data_ptr(), K.data_ptr())
                st, lat = srv.wait(tk)
                if st != 0:
                    raise RuntimeError("build status %d" % st)
                with lock:
                    lat_build.append(lat)
            with lock:
                lat_req.append(time.perf_counter() - t_arr)
                nbf.append(n)
            plan.close()
        except Exception as e:  # reported in the output
            with lock:
                errors.append(repr(e))

    threads = [threading.Thread(target=serve, args=(r,)) for r in reqs]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    wall = time.perf_counter() - t0
    srv.close()
    out = {"precision": plan_precision_name, "requests": len(reqs), "builds": len(lat_build),
           "builds_per_s": len(lat_build) / wall, "wall_s": wall,
           "nbf_range": [min(nbf), max(nbf)] if nbf else None, "slots": slots}
    if lat_build:
        out["build_latency_ms"] = {"p50": 1e3 * float(np.percentile(lat_build, 50)), "p99": 1e3 * float(np.percentile(lat_build, 99))}
    if lat_req:
        out["request_latency_s"] = {"p50": float(np.percentile(lat_req, 50)), "p99": float(np.percentile(lat_req, 99))}
    if errors:
        out["errors"] = errors[:3]
    return out


def serving_requests(args):
    import synthcells as sc

    return [r for r in sc.serving_requests(256) if r.natom_target <= args.max_atoms][: args.requests]


def run_serving(args):
    """The serving stream alone, both precisions; one JSON line."""
    from paper_2410_22278_gb300 import jk

    reqs = serving_requests(args)
    mixed = serve_stream(reqs, jk.JK_MIXED, args.slots, args.hbm_budget_gb * (1 << 30), lambda r: r.n_iter, "mixed")
    fp64 = serve_stream(reqs[: args.fp64_requests], jk.JK_FP64, args.slots, args.hbm_budget_gb * (1 << 30),
                        lambda r: min(3, r.n_iter), "fp64")
    out = {"metric": METRIC, "mode": "serving", "max_atoms": args.max_atoms, "arrival_rate_per_s": 50.0,
           "fp64_leg": "first %d requests, at most 3 iterations each" % args.fp64_requests,
           "data": "synthetic (serving stream: Poisson 50/s, diamond/water 50/50, 3-20 iterations, |E_k|_F = 1e-3; "
                   "requests above max_atoms skipped)", "mixed": mixed, "fp64": fp64}
    print(json.dumps(out))
    return 0


def aggregate(rank_times_ms, steps, world):
    """Whole-job throughput of N replicas: every rank builds `steps` times;
    the job time is the slowest rank's (max over ranks)."""
    t = max(rank_times_ms)
    return t / steps, world * steps / (t / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="water64", choices=sorted(WORKLOADS))
    ap.add_argument("--profile", action="store_true", help="mixed builds only (for ncu captures)")
    ap.add_argument("--coulomb-only", action="store_true", help="with --profile: time J-only builds (K = NULL)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default real-space schedule")
    ap.add_argument("--serving", action="store_true", help="run the serving stream instead of the single-cell build")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--max-atoms", type=int, default=64)
    ap.add_argument("--no-serving", action="store_true", help="leave the bounded serving stream out of the bench line")
    ap.add_argument("--fp64-requests", type=int, default=4)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--hbm-budget-gb", type=float, default=64.0)
    ap.add_argument("--autotune-cache", default=None)
    ap.add_argument("--no-cache", action="store_true", help="recompute the structure factors in every build")
    ap.add_argument("--mixed-switch", type=float, default=0.0, help="precision switch tau of the mixed path (0: library default)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)

    import torch

    from paper_2410_22278_gb300 import jk
    import synthcells as sc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    st = stream.cuda_stream

    cell = make_workload(args.workload)
    n = cell.nbf
    plan = jk.plan_from_cell(cell, precision=jk.JK_MIXED, device=local, mixed_switch=args.mixed_switch)
    plan64 = None if args.profile else jk.plan_from_cell(cell, precision=jk.JK_FP64, device=local)
    info = plan.info()
    S = torch.empty((n, n), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        plan.overlap(S.data_ptr(), st)
    stream.synchronize()
    Dh = sc.density_from_overlap(cell.orbital_guess(), S.cpu().numpy())
    D = torch.from_numpy(Dh).to(dev)
    J = torch.empty_like(D)
    K = torch.empty_like(D)

    def build(p):
        p.build(D.data_ptr(), J.data_ptr(), 0 if (args.profile and args.coulomb_only) else K.data_ptr(), st)

    # tile shapes of the real-space kernels chosen by the library's autotuner (outside the timed region)
    tiles = None if args.no_autotune else plan.autotune(D.data_ptr(), st, args.autotune_cache)
    for _ in range(args.warmup):
        build(plan)
    stream.synchronize()
    # the same build with every structure factor recomputed (no reciprocal
    # cache): its phase split, for reference beside the cached steady state
    phases_nocache = {k2: v[0] for k2, v in plan.build_times().items() if k2 != "mma_flops"}
    # steady state of an SCF loop on one geometry: the D-independent
    # reciprocal data stay resident (jk_plan_cache), filled by one untimed build
    cache_bytes = 0
    if not args.no_cache:
        free, _ = torch.cuda.mem_get_info(dev)
        try:
            cache_bytes = plan.cache(max(0, free - (24 << 30)))
        except jk.JkError as e:
            print("reciprocal cache not used: %s" % e, file=sys.stderr)
        for _ in range(2 if cache_bytes else 0):
            build(plan)
        stream.synchronize()

    # ---- timed region: exactly args.steps mixed builds
    clocks = Clocks(local)
    clocks.start()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase_sum = {}
    counts = (0, 0)
    for i in range(args.steps):
        ev[i][0].record(stream)
        build(plan)
        ev[i][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    cl = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    phases = plan.build_times()  # last build's phase split (library events on the same stream)
    counts = plan.build_counts()
    real_flops = plan.real_space_flops()
    if dist:
        t = torch.tensor([total_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step, value = aggregate([total_ms], args.steps, world)
    Jm, Km = J.cpu().numpy(), K.cpu().numpy()
    ej, ek = plan.energy(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
    if args.profile:
        print(json.dumps({"profile": args.workload, "coulomb_only": args.coulomb_only, "nbf": n, "plan": info,
                          "mixed_switch": args.mixed_switch, "ms_per_step": ms_per_step, "phases_ms": {k2: v for k2, v in phases.items()},
                          "counts": counts, "counters": plan.counters(), "schedule": tiles,
                          "phases_ms_without_cache": phases_nocache, "cache_bytes": cache_bytes}))
        return 0

    # ---- errors of this build against the oracle's J and K rows of the same
    # cell (tests/golden/water_rows_*.npz, written by tests/golden/make_rows.py
    # from the oracle alone; the oracle used its own overlap for D, equal to
    # the library's within 1e-14)
    def vs_oracle(Jx, Kx):
        import glob

        if args.workload != "water64":
            return None
        dj = dk = 0.0
        rows = 0
        for f in sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "water_rows_*.npz"))):
            g = np.load(f)
            r = g["rows"]
            dj = max(dj, float(np.abs(Jx[r] - g["J"]).max()))
            dk = max(dk, float(np.abs(Kx[r] - g["K"]).max()))
            rows += len(r)
        return {"max_abs_dJ": dj, "max_abs_dK": dk, "rows_compared": rows} if rows else None

    mixed_vs_oracle = vs_oracle(Jm, Km)

    # ---- Coulomb-only builds of the same plan (J alone, K = NULL): the
    # Hermite J-engine path
    def build_j(p):
        p.build(D.data_ptr(), J.data_ptr(), 0, st)

    build_j(plan)
    stream.synchronize()
    ej_only = []
    for _ in range(max(2, args.steps // 2)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        build_j(plan)
        b.record(stream)
        stream.synchronize()
        ej_only.append(a.elapsed_time(b))
    jonly_phases = {k2: v[0] for k2, v in plan.build_times().items() if k2 != "mma_flops"}
    Jonly = J.cpu().numpy()
    coulomb_only = {"ms_per_build": statistics.median(ej_only), "builds_per_s": 1e3 / statistics.median(ej_only),
                    "max_abs_dJ_vs_JK_build": float(np.abs(Jonly - Jm).max()), "phases_ms": jonly_phases,
                    "path": "Hermite J-engine (K = NULL)"}

    # ---- FP64 GPU form on the same GPU
    build(plan64)
    stream.synchronize()
    e64 = []
    for _ in range(args.fp64_steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        build(plan64)
        b.record(stream)
        stream.synchronize()
        e64.append(a.elapsed_time(b))
    phases64 = plan64.build_times()
    J64, K64 = J.cpu().numpy(), K.cpu().numpy()
    ej64, ek64 = plan64.energy(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
    fp64_vs_oracle = vs_oracle(J64, K64)
    # FMA peaks of this GPU (the ALU roofline denominators), measured by the
    # library's microbenchmark outside the timed region
    fma_peaks = {"fp32_tflops": statistics.median(jk.microbench_fma(False) for _ in range(3)),
                 "fp64_tflops": statistics.median(jk.microbench_fma(True) for _ in range(3)),
                 "sms": torch.cuda.get_device_properties(dev).multi_processor_count}

    # ---- end to end through the C ABI with pinned host buffers
    Dp = torch.from_numpy(Dh).pin_memory()
    Jp = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Kp = torch.empty((n, n), dtype=torch.float64).pin_memory()
    plan.build_host_into(Dp.numpy(), Jp.numpy(), Kp.numpy(), st)
    t0 = time.perf_counter()
    e2e_steps = max(2, args.steps // 2)
    for _ in range(e2e_steps):
        plan.build_host_into(Dp.numpy(), Jp.numpy(), Kp.numpy(), st)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    if rank != 0:
        if dist:
            tdist.destroy_process_group()
        return 0

    # ---- the serving stream, bounded (requests of at most --max-atoms atoms,
    # the first --requests of the 256-request stream), mixed precision
    serving = None
    if not args.no_serving:
        # every serving plan holds its own workspace: free the benchmark's
        # reciprocal cache and the FP64 plan first
        plan.cache(0)
        plan64.close()
        torch.cuda.empty_cache()
        reqs = serving_requests(args)
        serving = serve_stream(reqs, jk.JK_MIXED, args.slots, args.hbm_budget_gb * (1 << 30), lambda r: r.n_iter, "mixed")
        serving["stream"] = ("first %d of the 256-request stream with at most %d atoms; Poisson arrivals at 50/s, 3-20 SCF "
                             "iterations each, every iteration a fresh density" % (len(reqs), args.max_atoms))

    pk, pk_kind = peaks()
    launches = phases["total"][1]  # the library's own kernel launches per build (phases 0-5)
    nq = info["n_quartets_schwarz"]
    roof, roof_other = roofline(phases, real_flops, pk, pk_kind, fma_peaks)
    out = {
        "metric": METRIC, "value": value, "unit": "builds/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "precision": "mixed", "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush; each build streams the structure-factor slab (tens of GB, > L2)", "nbf": n,
                   "shell_pair_images": info["n_pair_images"], "n_g_half": info["n_g"],
                   "reciprocal_cache_bytes": cache_bytes,
                   "reciprocal_cache": ("D-independent structure factors and their exchange slices resident between builds "
                                        "(jk_plan_cache; an SCF loop on one geometry)") if cache_bytes else "off"},
        "phases_ms_without_cache": phases_nocache,
        "quartets_per_s": nq / (ms_per_step / 1e3),
        "image_quartets_evaluated_per_s": (counts[0] + counts[1]) / (ms_per_step / 1e3),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "fp64": {"builds_per_s": 1e3 / statistics.mean(e64), "ms_per_build": statistics.mean(e64),
                 "phases_ms": {k2: v[0] for k2, v in phases64.items() if k2 != "mma_flops"}},
        "mixed_vs_fp64": {"max_abs_dJ": float(np.abs(Jm - J64).max()), "max_abs_dK": float(np.abs(Km - K64).max()),
                          "dE_Ha": (ej + ek) - (ej64 + ek64), "E_J": ej64, "E_K": ek64},
        "mixed_vs_oracle_rows": mixed_vs_oracle,
        "fp64_vs_oracle_rows": fp64_vs_oracle,
        "fma_peaks_measured": fma_peaks,
        "phases_ms": {k2: v[0] for k2, v in phases.items() if k2 != "mma_flops"},
        "fp64_fraction": counts[0] / max(1, counts[0] + counts[1]),
        "autotuned_tiles": tiles,
        "gpu_launches": launches * args.steps,
        "roofline": roof,
        "roofline_other": roof_other,
        "clocks": cl,
        "e2e": {"value": 1.0 / e2e_s, "unit": "builds/s", "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": 2 * n * n * 8},
        "serving": serving,
        "coulomb_only": coulomb_only,
    }
    if not args.no_cpu_baseline and world == 1:
        from oracle import oracle as O

        # the oracle's inputs come from the oracle's own overlap metric
        out["cpu_baseline"] = cpu_baseline_sample(cell, O.density(cell))
    print(json.dumps(out))
    if dist:
        tdist.destroy_process_group()
    return 0


# DRAM traffic of k_real<0,0,0,0,float> per launch on the 64-water box, from
# ncu (dram__bytes_read.sum + dram__bytes_write.sum, one pass)
REAL_TILE_TRAFFIC = None


def roofline(phases, real_flops, pk, pk_kind, fma):
    """Roofline of each kernel family of a mixed build, from the library's
    CUDA events on the build stream (phase sums over one build) and the work
    the kernels tallied: real-space FP32 tile kernels and FP64 list kernels
    (algorithmic flops of the McMurchie-Davidson steps, against the FP32 /
    FP64 FMA rates measured on this GPU by jk_microbench_fma), split-precision
    GEMMs (BF16 MMA flops issued, against the measured BF16 peak).  Returns
    the family with the most device time first."""
    fl64, fl32 = real_flops
    list_ms, list_n = phases.get("real_fp64_list", (0.0, 0))
    tile_ms = max(phases["real_tiles"][0], 1e-9)
    mk = "measured on this GPU (jk_microbench_fma: independent FMA chains, %d SMs, CUDA events)" % fma["sms"]
    out = [
        {"bound": "alu", "kernel": "k_real<..., float> (FP32 real-space quartet tiles)", "achieved": fl32 / (tile_ms / 1e3) / 1e12,
         "peak": fma["fp32_tflops"], "unit": "TFLOP/s", "frac": fl32 / (tile_ms / 1e3) / 1e12 / fma["fp32_tflops"],
         "traffic": REAL_TILE_TRAFFIC, "ms": tile_ms, "launches": phases["real_tiles"][1],
         "peak_kind": "FP32 FMA rate " + mk,
         "work": "algorithmic flops of the MD steps (csrc/flops.h) tallied by the kernels"},
    ]
    if list_ms > 0:
        ach = fl64 / (list_ms / 1e3) / 1e12
        out.append({"bound": "alu", "kernel": "k_real_list (FP64 large quartets)", "achieved": ach, "peak": fma["fp64_tflops"],
                    "unit": "TFLOP/s", "frac": ach / fma["fp64_tflops"], "traffic": None, "ms": list_ms, "launches": list_n,
                    "peak_kind": "FP64 FMA rate " + mk, "work": "algorithmic flops of the MD steps (csrc/flops.h)"})
    gemm_ms, gemm_n = phases.get("tensor_gemm", (0.0, 0))
    if gemm_ms > 0:
        ach = phases["mma_flops"][0] / (gemm_ms / 1e3) / 1e12
        peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
        out.append({"bound": "tensor", "kernel": "k_ozaki_tc (split-precision BF16 tcgen05 GEMM)", "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": None, "ms": gemm_ms, "launches": gemm_n,
                    "peak_kind": "%s sustained bf16 (MEASURED_PEAKS.json)" % pk_kind, "work": "BF16 MMA flops issued"})
    out.sort(key=lambda r: -r["ms"])
    for r in out:
        r["ms_per_launch"] = r["ms"] / max(1, r["launches"])
    return out[0], out[1:]


if __name__ == "__main__":
    sys.exit(main())
