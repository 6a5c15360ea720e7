"""Benchmark of the particle time step (SDE + tracking + PIC statistics).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = pdf_step (coefficient rows + the fused particle kernel) followed by
pdf_estimate_stats (grouping, element and node statistics, derivatives): every
row a1-a12 of the hot path, on the channel workload of 200 x 400 nodes,
158,802 triangles and 100 particles per element (15,880,200 particles).
The particle state (1.02 GB) is larger than the 129 MB L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (a bounded sample of the same workload).
With --gpus N > 1 (under torchrun) each rank runs an independent replica.
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import inputs  # noqa: E402

WORKLOAD = "channel_200x400_ppe100"
METRIC = "particle-steps/s (SDE+search+PIC stats) at 16M particles; % HBM roofline"
UNIT = "particle-steps/s"
# Algorithmic DRAM bytes of the fused particle kernel per particle: read x, y,
# u, v, w, omega, psi (56) and elem (4); write the same (60).  Per element
# per launch: the coefficient row (256) and the tracking geometry (80).
K_STEP_BYTES_PER_PARTICLE = 120
K_STEP_BYTES_PER_ELEMENT = 336
# Algorithmic bytes of the whole step per particle (state read and written
# once, element and node tables amortised), the denominator of the
# whole-step roofline fraction.
STEP_BYTES_PER_PARTICLE = 134


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_sha():
    """Hash of the particle kernel's sources (step.cu, rng.cuh, common.cuh,
    fx.cuh) with comments and whitespace removed: a change of code, not of
    comments, makes the committed profile stale."""
    h = hashlib.sha256()
    for f in ("step.cu", "rng.cuh", "common.cuh", "fx.cuh"):
        with open(os.path.join(ROOT, "paper_1006_0720_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def _profile_numbers():
    """From the committed ncu summary of k_step, if it was taken on the
    current kernel source: DRAM bytes per launch at the benchmark size and
    warp instructions per particle; else an empty dict."""
    path = os.path.join(ROOT, "profiles", "k_step_fx_channel_200x400.md")
    try:
        text = open(path).read()
    except OSError:
        return {}
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m_sha or m_sha.group(1) != _kernel_sha():
        return {}
    out = {}
    for key in ("dram_bytes_per_launch", "warp_inst_per_particle"):
        m = re.search(key + r":\s*([0-9.eE+]+)", text)
        if m:
            out[key] = float(m.group(1))
    return out


def issue_peak(sm_mhz):
    """Warp instructions per second the SMs can issue: 152 SMs x 4
    schedulers x one instruction per clock."""
    return 152 * 4 * sm_mhz * 1e6


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "pdfgb_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _setup_dist(n_gpus, backend="nccl"):
    """Rank, world size, local rank and torch.distributed (None for one
    process) from the launcher's environment."""
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group(backend)
        dist = dist_mod
    return rank, world, local, dist


def max_over_ranks(dist, value, device):
    """The largest of the ranks' values, on every rank (the timing rule:
    the slowest replica sets the time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(seed, rank):
    """Independent replicas: rank r runs the workload with seed + r."""
    return seed + rank


def replica_value(world, n, steps, t_max_ms):
    """Whole-job throughput of `world` replicas of n particles each, `steps`
    steps in the slowest replica's t_max_ms."""
    return world * n * steps / (t_max_ms * 1e-3)


def cpu_baseline_measure(steps=1, warmup=0, ppe=None, threads=1):
    """The oracle as it stands on a bounded sample of the workload: the
    benchmark mesh with `ppe` particles per element (default: the
    workload's 100), initialised once (untimed), then `warmup` untimed and
    `steps` timed steps (coefficients + particle step + statistics); value =
    the median per-step throughput.  threads = 1: single-threaded on one host
    core; otherwise the particle loop runs over that many host threads (0:
    all; OpenMP, the paper's loop design (ii)) with the coefficients and
    statistics single-threaded, and `cores` reports the threads used."""
    import oracle
    cfg = inputs.workload(WORKLOAD)
    ppe = ppe or cfg["ppe"]
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], jitter=cfg["jitter"], seed=cfg["seed"])
    M = oracle.Mesh(m)
    counts = np.full(cfg["n_tri"], ppe, dtype=np.int32)
    st = oracle.init(M, counts, cfg["seed"], u_sigma=cfg["u_sigma"],
                     elem_psi0=inputs.scalar_slab(m, cfg["psi_slab_x"]))
    P = oracle.make_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"])
    es, ns, nd, _ = oracle.statistics(M, st)
    n = int(counts.sum())
    rates, total, used = [], 0.0, 1
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        rows = oracle.elem_coeff(M, ns, nd, P)
        if threads == 1:
            oracle.step(M, rows, P, cfg["seed"], s, st)
        else:
            _, _, used = oracle.step_threads(M, rows, P, cfg["seed"], s, st, threads=threads)
        es, ns, nd, _ = oracle.statistics(M, st, ns)
        dt = time.perf_counter() - t0
        if s >= warmup:
            rates.append(n / dt)
            total += dt
    kind = "oracle" if threads == 1 else ("oracle, particle loop over %d host threads (OpenMP, loop design (ii)); "
                                          "coefficients and statistics single-threaded" % used)
    return {"value": statistics.median(rates), "unit": UNIT, "cores": used, "kind": kind,
            "sample": "%d timed step(s) of the %d-triangle channel with %d particles per element (%d particles; "
                      "the workload has %d), %.1f s of stepping" % (steps, cfg["n_tri"], ppe, n, cfg["ppe"], total)}


def run_reference(args):
    rank, world, local, dist = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0, None
    if rank != 0:
        return 0
    cfg = inputs.workload(WORKLOAD)
    # bound the whole run to a few minutes of oracle work (all host cores on
    # the particle loop: ~1.5e7 particle-steps/s or more)
    per_step = 1.5e9 / max(1, args.steps + args.warmup)
    ppe = int(max(5, min(cfg["ppe"], per_step // cfg["n_tri"])))
    base = cpu_baseline_measure(args.steps, args.warmup, ppe=ppe, threads=0)
    value = base["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * cfg["n_particles"] / value if value else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_particles": cfg["n_particles"],
                                            "n_tri": cfg["n_tri"], "closure": cfg["closure"]},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import paper_1006_0720_gb300 as pg

    rank, world, local, dist = _setup_dist(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = inputs.workload(args.workload)
    m = inputs.channel_mesh(cfg["nx"], cfg["ny"], jitter=cfg["jitter"], seed=cfg["seed"])
    psi = inputs.scalar_slab(m, cfg["psi_slab_x"])
    gm = pg.Mesh(m)
    seed = replica_seed(cfg["seed"], rank)
    gp = pg.Particles(gm, seed, ppe=cfg["ppe"], u_sigma=cfg["u_sigma"], elem_psi0=psi)
    n = gp.n
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"])
    stream = torch.cuda.current_stream(dev)
    pg.pdf_estimate_stats(gp, gm)
    step_no = 0
    for _ in range(args.warmup):
        pg.pdf_step(gp, gm, p, step=step_no)
        pg.pdf_estimate_stats(gp, gm)
        step_no += 1
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (CUDA events around k_step only, for
    # its average launch duration)
    clocks = ClockSampler(local)
    pg.pdf_profile_reset()
    pg.pdf_profile_only("k_step")
    pg.pdf_profile_enable(True)
    launches0 = pg.pdf_kernel_launches()
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pg.pdf_step(gp, gm, p, step=step_no, stream=stream)
        pg.pdf_estimate_stats(gp, gm, stream=stream)
        step_no += 1
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = pg.pdf_kernel_launches() - launches0
    pg.pdf_profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    k_launch, k_ms = pg.pdf_profile_query("k_step")
    pg.pdf_profile_reset()
    # ---- a second pass of the same steps with every kernel timed, for the
    # per-kernel shares (events around every launch add a few us each)
    pg.pdf_profile_only(None)
    pg.pdf_profile_enable(True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        pg.pdf_step(gp, gm, p, step=step_no, stream=stream)
        pg.pdf_estimate_stats(gp, gm, stream=stream)
        step_no += 1
    ev1.record(stream)
    barrier()
    pg.pdf_profile_enable(False)
    ms_prof = ev0.elapsed_time(ev1)
    shares = {}
    for kname in ("k_step", "k_radix_scatter", "k_radix_hist", "k_elem_stats", "k_node_coeff",
                  "k_elem_rows", "k_seg_offsets", "k_node_stats", "k_scan_bins",
                  "k_elem_grad1", "k_node_grad1", "k_elem_grad2", "k_node_grad2", "k_reorder"):
        c, t = pg.pdf_profile_query(kname)
        shares[kname] = {"launches": c, "ms_per_launch": t / c if c else None,
                         "share": t / ms_prof if ms_prof else None}
    pg.pdf_profile_reset()
    t_max = max_over_ranks(dist, ms, dev)
    value = replica_value(world, n, args.steps, t_max)

    # ---- end-to-end through the public API with host-resident state
    keys = ("x", "y", "u", "v", "w", "om", "ps")
    host = {k: torch.empty(n, dtype=torch.float64, pin_memory=True) for k in keys}
    host["elem"] = torch.empty(n, dtype=torch.int32, pin_memory=True)
    host_ns = torch.empty((gm.n_nodes, 12), dtype=torch.float64, pin_memory=True)
    ptr = {k: v.data_ptr() for k, v in host.items()}
    import ctypes
    L = pg.lib()
    sp = ctypes.c_void_p(stream.cuda_stream)
    pg.capi.check(L.pdf_particles_get_state(gp.handle, *[ctypes.c_void_p(ptr[k]) for k in keys + ("elem",)], sp),
                  "get_state")
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 10))
    # untimed warm-up of the host path (its first call allocates the staging
    # buffers and creates the streams)
    for _ in range(2):
        pg.pdf_step_host_stats(gp, gm, p, host, node_stats=host_ns, step=step_no, stream=stream)
        step_no += 1
    stream.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        # the step reads the host state and writes the stepped state back
        # (chunks of loads, steps and stores overlapped), the statistics
        # running beside the last chunks' write-back, node statistics copied
        # to the host
        pg.pdf_step_host_stats(gp, gm, p, host, node_stats=host_ns, step=step_no, stream=stream)
        stream.synchronize()
        step_no += 1
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_max = max_over_ranks(dist, e2e_s, dev)
    state_bytes = n * (7 * 8 + 4)
    e2e = {"value": replica_value(world, n, e2e_steps, 1e3 * e2e_max), "unit": UNIT, "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes + gm.n_nodes * 12 * 8, "steps": e2e_steps,
           "what": "state in page-locked host memory: read, stepped and written back every step "
                   "(pdf_step_host_stats: chunks moved by the copy engines while the previous chunk is stepped, the "
                   "statistics beside the last chunks' write-back), node statistics copied out; after 2 untimed "
                   "warm-up steps"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    k_avg_ms = k_ms / k_launch if k_launch else float("nan")
    k_bytes = K_STEP_BYTES_PER_PARTICLE * n + K_STEP_BYTES_PER_ELEMENT * gm.n_tri
    achieved = k_bytes / (k_avg_ms * 1e-3) / 1e9
    prof = _profile_numbers()
    hbm = {"bound": "hbm", "kernel": "k_step", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": prof.get("dram_bytes_per_launch"), "peak_source": peak_kind,
           "bytes_per_launch_alg": k_bytes, "ms_per_launch": k_avg_ms,
           "roof_ms": k_bytes / (peak * 1e9) * 1e3}
    roofline = hbm
    if "warp_inst_per_particle" in prof and clk.get("sm_mhz"):
        # the instruction-issue roof: ncu's warp instructions per launch over
        # what 152 SMs x 4 schedulers issue at the sampled clock
        winst = prof["warp_inst_per_particle"] * n
        ipk = issue_peak(clk["sm_mhz"])
        issue = {"bound": "alu", "kernel": "k_step", "achieved": winst / (k_avg_ms * 1e-3), "peak": ipk,
                 "unit": "warp-inst/s", "frac": winst / (k_avg_ms * 1e-3) / ipk,
                 "traffic": prof.get("dram_bytes_per_launch"), "warp_inst_per_launch": winst,
                 "peak_source": "152 SMs x 4 schedulers x sampled SM clock", "ms_per_launch": k_avg_ms,
                 "roof_ms": winst / ipk * 1e3}
        if issue["roof_ms"] > hbm["roof_ms"]:
            roofline = dict(issue, hbm=hbm)
        else:
            roofline = dict(hbm, issue=issue)
    step_frac = STEP_BYTES_PER_PARTICLE * (n * args.steps / (ms * 1e-3)) / (peak * 1e9)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i64+f32x2", "data": "synthetic",
            "config": {"workload": args.workload, "n_particles": n, "n_tri": gm.n_tri, "n_nodes": gm.n_nodes,
                       "closure": cfg["closure"], "dt": cfg["dt"],
                       "arith": "FP64-accurate without FP64 instructions: positions 64-bit fixed point, "
                                "u, v, w, omega, psi double-float (FP32 pairs)",
                       "l2": "inputs larger than L2: particle state %.2f GB vs 129 MB L2" % (n * 64 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "hbm_frac_step": step_frac, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
            "roofline": roofline, "kernels": shares, "kernels_pass_ms_per_step": ms_prof / args.steps}
    def want(name):
        return not args.skip_extras and (args.extras == "all" or name in args.extras.split(","))

    # the complex-geometry workload (obstacles, FP32 state, 68.6M particles)
    if want("complex"):
        del gp
        torch.cuda.empty_cache()
        line["complex_geometry"] = run_obstacles(pg, torch, stream, steps=max(5, min(args.steps, 10)))
        torch.cuda.empty_cache()
        gp = None
    # the precision form (FP32 velocity/frequency/scalar state) on the same workload
    if want("fp32") or want("relax"):
        gq = pg.Particles(gm, seed, ppe=cfg["ppe"], u_sigma=cfg["u_sigma"], elem_psi0=psi,
                          precision=pg.capi.PDF_FP32_STATE)
        pg.pdf_estimate_stats(gq, gm)
        for s in range(3):
            pg.pdf_step(gq, gm, p, step=s)
            pg.pdf_estimate_stats(gq, gm)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if want("fp32"):
            e0.record(stream)
            ksteps = max(5, min(args.steps, 20))
            for s in range(ksteps):
                pg.pdf_step(gq, gm, p, step=3 + s, stream=stream)
                pg.pdf_estimate_stats(gq, gm, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms32 = e0.elapsed_time(e1) / ksteps
            line["precision_fp32_state"] = {"value": n / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
                                            "steps": ksteps,
                                            "what": "u, v, w, omega, psi stored and advanced in FP32; x, y 64-bit fixed point"}
        if want("relax"):
            # the elliptic-relaxation solve on this mesh: cold, and warm from the previous step
            wp = torch.zeros((9, gm.n_nodes), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it_cold, _ = pg.pdf_relax_solve_particles(gq, gm, p, wp, rtol=1e-10, max_it=20000)
            t_cold = time.perf_counter() - t0
            # the paper's Jacobi preconditioner on the same cold solve
            wj = torch.zeros_like(wp)
            pg.pdf_relax_set_solver(gq, False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it_jac, _ = pg.pdf_relax_solve_particles(gq, gm, p, wj, rtol=1e-10, max_it=20000)
            t_jac = time.perf_counter() - t0
            pg.pdf_relax_set_solver(gq, True)
            del wj
            pg.pdf_step(gq, gm, p, wp=wp, step=100)
            pg.pdf_estimate_stats(gq, gm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it_warm, _ = pg.pdf_relax_solve_particles(gq, gm, p, wp, rtol=1e-10, max_it=20000)
            t_warm = time.perf_counter() - t0
            # whole steps with the elliptic relaxation: step (drift from the
            # solved wp) + statistics + the solve warm-started from the previous
            # step's wp
            its = []
            ksteps_rx = 5
            torch.cuda.synchronize()
            e0.record(stream)
            for s in range(ksteps_rx):
                pg.pdf_step(gq, gm, p, wp=wp, step=200 + s, stream=stream)
                pg.pdf_estimate_stats(gq, gm, stream=stream)
                it_s, _ = pg.pdf_relax_solve_particles(gq, gm, p, wp, rtol=1e-8, max_it=20000, stream=stream)
                its.append(max(it_s))
            e1.record(stream)
            torch.cuda.synchronize()
            ms_rx = e0.elapsed_time(e1) / ksteps_rx
            line["relax_solve"] = {"rtol": 1e-10, "n_nodes": gm.n_nodes, "preconditioner": "multigrid",
                                   "cold": {"iterations_max": max(it_cold), "seconds": t_cold},
                                   "cold_jacobi": {"iterations_max": max(it_jac), "seconds": t_jac},
                                   "warm_previous_step": {"iterations_max": max(it_warm), "seconds": t_warm},
                                   "whole_step": {"value": n / (ms_rx * 1e-3), "unit": UNIT, "ms_per_step": ms_rx,
                                                  "steps": ksteps_rx, "rtol": 1e-8, "iterations": [min(its), max(its)],
                                                  "what": "step + statistics + elliptic-relaxation solve (FP32 state)"}}
        del gq
    if want("fp64"):
        line["native_fp64"] = run_native_fp64(pg, torch, stream, gm, cfg, seed, psi, p, max(3, min(args.steps, 10)))
    if want("hostlink"):
        line["host_link_copy_engines"] = measure_host_link(torch)
    if want("iecm"):
        line["iecm"] = run_iecm(pg, torch, stream, gm, cfg, seed, psi, p, max(5, min(args.steps, 20)))
    if want("projection"):
        line["pressure_projection"] = run_projection(pg, torch, stream, gm, cfg, seed, psi, p,
                                                     max(5, min(args.steps, 20)))
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline_measure(3)
        except Exception as exc:  # report, do not hide
            line["cpu_baseline"] = {"error": repr(exc)}
        try:
            line["cpu_baseline_all_cores"] = cpu_baseline_measure(3, threads=0)
        except Exception as exc:
            line["cpu_baseline_all_cores"] = {"error": repr(exc)}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_native_fp64(pg, torch, stream, gm, cfg, seed, psi, p, steps):
    """The benchmark workload with the particle kernel in native FP64
    instructions (PDF_ARITH_FP64: FP64 state arithmetic, the FP64 walk),
    the statistics as in the default path; time per step and of k_step."""
    g64 = pg.Particles(gm, seed, ppe=cfg["ppe"], u_sigma=cfg["u_sigma"], elem_psi0=psi)
    p64 = pg.model_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=cfg["closure"], arith="fp64")
    pg.pdf_estimate_stats(g64, gm)
    for s in range(2):
        pg.pdf_step(g64, gm, p64, step=s)
        pg.pdf_estimate_stats(g64, gm)
    torch.cuda.synchronize()
    pg.pdf_profile_reset()
    pg.pdf_profile_only("k_step")
    pg.pdf_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        pg.pdf_step(g64, gm, p64, step=2 + s, stream=stream)
        pg.pdf_estimate_stats(g64, gm, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    pg.pdf_profile_enable(False)
    c, t = pg.pdf_profile_query("k_step")
    pg.pdf_profile_reset()
    pg.pdf_profile_only(None)
    ms = e0.elapsed_time(e1) / steps
    del g64
    return {"value": gm_particles(cfg) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "k_step_ms": t / c if c else None, "dtype": "f64",
            "what": "native FP64 particle kernel (PDF_ARITH_FP64) + statistics, same workload"}


def measure_host_link(torch, nbytes=1 << 30, repeats=3):
    """The host link through the copy engines: cudaMemcpyAsync (torch
    non_blocking copies) of 1 GiB between page-locked host memory and the
    device, one call per direction on its own stream, each direction alone
    and both at once; best of `repeats`."""
    h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_in = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(ops):
        best = None
        for _ in range(repeats):
            torch.cuda.synchronize()
            start = torch.cuda.Event(enable_timing=True)
            start.record(torch.cuda.current_stream())
            ends = []
            for st, fn in ops:
                st.wait_event(start)
                with torch.cuda.stream(st):
                    fn()
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(st)
                ends.append(ev)
            torch.cuda.synchronize()
            ms = max(start.elapsed_time(ev) for ev in ends)
            best = ms if best is None else min(best, ms)
        return best

    h2d = (s_in, lambda: d_in.copy_(h_in, non_blocking=True))
    d2h = (s_out, lambda: h_out.copy_(d_out, non_blocking=True))
    t_in, t_out, t_both = timed([h2d]), timed([d2h]), timed([h2d, d2h])
    out = {"bytes_per_direction": nbytes, "h2d_gbs": nbytes / (t_in * 1e-3) / 1e9,
           "d2h_gbs": nbytes / (t_out * 1e-3) / 1e9, "both_gbs": 2 * nbytes / (t_both * 1e-3) / 1e9,
           "what": "cudaMemcpyAsync, page-locked host <-> device, one call per direction on separate streams"}
    del h_in, h_out, d_in, d_out
    return out


def run_iecm(pg, torch, stream, gm, cfg, seed, psi, p, steps, bins=(5, 5, 5)):
    """Steps of the benchmark workload with the IECM micromixing model: the
    velocity-conditioned scalar means (sort-and-divide binning) are computed
    at every statistics call; the time per step and of the conditioning
    kernel alone."""
    gi = pg.Particles(gm, seed, ppe=cfg["ppe"], u_sigma=cfg["u_sigma"], elem_psi0=psi)
    gi.set_iecm(bins, 2)
    pi = pg.model_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=cfg["closure"], mix="iecm")
    pg.pdf_estimate_stats(gi, gm)
    for s in range(3):
        pg.pdf_step(gi, gm, pi, step=s)
        pg.pdf_estimate_stats(gi, gm)
    torch.cuda.synchronize()
    pg.pdf_profile_reset()
    pg.pdf_profile_only("k_iecm_cond")
    pg.pdf_profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        pg.pdf_step(gi, gm, pi, step=3 + s, stream=stream)
        pg.pdf_estimate_stats(gi, gm, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    pg.pdf_profile_enable(False)
    c, t = pg.pdf_profile_query("k_iecm_cond")
    pg.pdf_profile_reset()
    pg.pdf_profile_only(None)
    ms = e0.elapsed_time(e1) / steps
    del gi
    return {"value": gm_particles(cfg) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "bins": list(bins), "m_min": 2, "k_iecm_cond_ms": t / c if c else None,
            "what": "IECM micromixing (eq. IECM) with sort-and-divide conditioning at every statistics call"}


def run_projection(pg, torch, stream, gm, cfg, seed, psi, p, steps, rtol=1e-8, Cp=5e-4):
    """Steps of the benchmark workload with the stabilised mean-pressure
    projection after every step (eqs. velocity-prediction, pressure-
    projection-smooth, velocity-correction): the drift sees Pi - grad <P'>,
    the Poisson system is solved to rtol, particles are corrected.  C_p =
    dt / 2 (C_p = dt lets the discrete pressure mode grow)."""
    gj = pg.Particles(gm, seed, ppe=cfg["ppe"], u_sigma=cfg["u_sigma"], elem_psi0=psi)
    pj = pg.model_params(dt=p.dt, nu=p.nu, Pi=p.Pi, closure=cfg["closure"], pressure="projection")
    pg.pdf_estimate_stats(gj, gm)
    t0 = time.perf_counter()
    pg.pdf_pressure_project(gj, gm, pj, Cp=Cp, rtol=rtol, max_it=2000)
    setup_s = time.perf_counter() - t0
    for s in range(3):
        pg.pdf_step(gj, gm, pj, step=s)
        pg.pdf_estimate_stats(gj, gm)
        pg.pdf_pressure_project(gj, gm, pj, Cp=Cp, rtol=rtol, max_it=2000)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    its = []
    proj_ms = 0.0
    e0.record(stream)
    for s in range(steps):
        pg.pdf_step(gj, gm, pj, step=3 + s, stream=stream)
        pg.pdf_estimate_stats(gj, gm, stream=stream)
        e1.record(stream)
        it, _ = pg.pdf_pressure_project(gj, gm, pj, Cp=Cp, rtol=rtol, max_it=2000, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        proj_ms += e1.elapsed_time(e2)
        its.append(it)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pres = pg.pdf_pressure_field(gj, gm)
    del gj
    return {"value": gm_particles(cfg) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "projection_ms": proj_ms / steps, "iterations": [min(its), max(its)], "rtol": rtol, "Cp": Cp,
            "n_unknowns": gm.n_nodes - int(cfg["ny"]), "setup_seconds_first_call": setup_s,
            "pressure_range": [float(pres.min()), float(pres.max())],
            "what": "step + statistics + pressure projection (multigrid-preconditioned CG, FP64) per step"}


def gm_particles(cfg):
    return cfg["n_tri"] * cfg["ppe"]


def run_obstacles(pg, torch, stream, steps=10, name="obstacles_20x5_mean128"):
    """Throughput of the complex-geometry workload: graded mesh around three
    obstacles, particles per element proportional to area (mean 128), point
    source, periodic inflow/outflow with re-injection, FP32 state."""
    cfg = inputs.OBSTACLES[name]
    t0 = time.perf_counter()
    m = inputs.obstacle_mesh(h_min=cfg["h_min"], ratio=cfg["ratio"], growth=cfg["growth"])
    counts = inputs.counts_by_area(m, cfg["mean_ppe"])
    gm = pg.Mesh(m)
    gp = pg.Particles(gm, cfg["seed"], count=counts, u_profile=cfg["u_profile"], u_sigma=cfg["u_sigma"],
                      precision=pg.capi.PDF_FP32_STATE)
    p = pg.model_params(dt=cfg["dt"], nu=cfg["nu"], Pi=cfg["Pi"], closure=cfg["closure"], tm_mode=cfg["tm_mode"],
                        src_x=cfg["src"][0], src_y=cfg["src"][1], src_r=cfg["src"][2])
    setup_s = time.perf_counter() - t0
    pg.pdf_estimate_stats(gp, gm)
    for s in range(3):
        pg.pdf_step(gp, gm, p, step=s)
        pg.pdf_estimate_stats(gp, gm)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(steps):
        pg.pdf_step(gp, gm, p, step=3 + s, stream=stream)
        pg.pdf_estimate_stats(gp, gm, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the same with the particle redistribution of App. D after every step
    # (at least min_npel particles per element, the cylinder case's 5)
    min_npel = 5
    moved = 0
    e0.record(stream)
    for s in range(steps):
        pg.pdf_step(gp, gm, p, step=3 + steps + s, stream=stream)
        moved += pg.pdf_redistribute(gp, gm, min_npel, cfg["seed"], 3 + steps + s, stream=stream)
        pg.pdf_estimate_stats(gp, gm, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_rd = e0.elapsed_time(e1) / steps
    info = pg.pdf_step(gp, gm, p, step=3 + 2 * steps, info=True)
    n = gp.n
    out = {"workload": name, "n_particles": n, "n_tri": gm.n_tri, "value": n / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms, "steps": steps, "setup_seconds": setup_s, "precision": "fp32_state",
           "with_redistribution": {"value": n / (ms_rd * 1e-3), "unit": UNIT, "ms_per_step": ms_rd,
                                   "min_npel": min_npel, "moved_per_step": moved / steps},
           "last_step_counters": info}
    del gp, gm
    return out


def run_warmstart(args):
    """Train the per-node MLP on elliptic-relaxation solves of the small
    channel (the library's kernels only), then on the 158,802-triangle mesh
    solve to rtol 1e-10 from zero, from the previous step's solution and from
    the network's guess."""
    import torch
    from paper_1006_0720_gb300 import experiments as E
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    X, Y = E.collect_solves(args.solves)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, losses = E.train(X, Y, steps=args.train_steps, batch=8192, lr=2e-3, log_every=max(1, args.train_steps // 10))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y
    cfg, gm, gp, p, wp = E.setup(WORKLOAD, seed=3)
    # the run on the benchmark mesh, its solves kept: a second network is
    # trained on them (the method's own solves on this mesh), then both are
    # judged on the state after the run (not in either training set)
    its, Xo, Yo = E.advance(gm, gp, p, wp, args.steps, collect=True)
    t0 = time.perf_counter()
    net_o, losses_o = E.train(Xo, Yo, steps=args.train_steps, batch=8192, lr=2e-3, seed=1,
                              log_every=max(1, args.train_steps // 10))
    torch.cuda.synchronize()
    t_train_o = time.perf_counter() - t0
    del Xo, Yo
    res = {"small_channel_net": {"jacobi": E.compare(gm, gp, p, wp, net, multigrid=False),
                                 "multigrid": E.compare(gm, gp, p, wp, net, multigrid=True)},
           "own_mesh_net": {"jacobi": E.compare(gm, gp, p, wp, net_o, multigrid=False),
                            "multigrid": E.compare(gm, gp, p, wp, net_o, multigrid=True)}}
    line = {"mode": "warmstart", "train_solves": args.solves, "train_samples": args.solves * 800,
            "train_steps": args.train_steps, "collect_seconds": t_collect, "train_seconds": t_train,
            "loss_log": losses, "eval_workload": WORKLOAD, "eval_after_steps": args.steps,
            "own_mesh_train_samples": args.steps * gm.n_nodes, "own_mesh_train_seconds": t_train_o,
            "own_mesh_loss_log": losses_o, "warm_iterations_during_run": its, "compare": res}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--solves", type=int, default=10000, help="warmstart: training solves of the small channel")
    ap.add_argument("--train-steps", type=int, default=4000, help="warmstart: Adam steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, help="a smaller workload for profiling runs")
    ap.add_argument("--skip-extras", action="store_true", help="only the main line (no FP32-state and solve figures)")
    ap.add_argument("--extras", default="all",
                    help="comma-separated subset of complex, fp32, relax, iecm, projection, fp64, hostlink "
                         "(for profiling runs)")
    ap.add_argument("--mode", default="step", choices=["step", "warmstart"],
                    help="warmstart: the learned warm start experiment instead of the step benchmark")
    args = ap.parse_args()
    if args.extras != "all":
        unknown = set(args.extras.split(",")) - {"complex", "fp32", "relax", "iecm", "projection", "fp64", "hostlink"}
        if unknown:
            ap.error("--extras: unknown %s" % ", ".join(sorted(unknown)))
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "warmstart":
        return run_warmstart(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
