"""Benchmark of the LLR hot path on GB300: window-restricted sweeps plus the
Robbins-Monro update for the whole batch of (interval, replica) lattices.

Workload: 4-D compact U(1), L=20, 256 intervals over E/6V in [0.62, 0.67]
x 8 replicas (2048 lattices, 5.2 GB of float32 link angles), dE = 12,
1 heat-bath : 4 overrelaxation.  One step = one Robbins-Monro iteration of
every lattice (n_therm + n_meas composite sweeps and the update of a).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "link updates/s"
SFU_OPS_PER_CLK_SM = 16          # special-function (MUFU) ops per SM per clock
MUFU_PER_UPDATE = 12             # algorithmic: sine and cosine of the 6 staple angles
BYTES_PER_UPDATE = 8             # algorithmic: read + write one float32 link
ISSUE_PER_CLK_SM = 4             # warp instructions issued per SM per clock (4 schedulers)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-therm", type=int, default=2)
    p.add_argument("--n-meas", type=int, default=8)
    p.add_argument("--threads", type=int, default=0,
                   help="threads per CTA (128/256/512); 0 = autotuned")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--intervals", type=int, default=256)
    p.add_argument("--converge", action="store_true",
                   help="learned warm start vs naive start vs plain form: RM-converged "
                        "intervals/s")
    p.add_argument("--no-converge", action="store_true",
                   help="skip the converged-intervals leg of the default run")
    p.add_argument("--train-replicas", type=int, default=2,
                   help="replicas per interval of the warm start's training runs (L = 8 ... 16)")
    p.add_argument("--train-rm", type=int, default=40,
                   help="Robbins-Monro steps of the warm start's training runs")
    p.add_argument("--c4", action="store_true",
                   help="learned warm start as configured: 128 intervals at L = 20 and 24")
    p.add_argument("--target-L", type=int, default=20)
    p.add_argument("--target-intervals", type=int, default=32)
    p.add_argument("--target-replicas", type=int, default=4)
    p.add_argument("--n-rm", type=int, default=150)
    p.add_argument("--no-configs", action="store_true",
                   help="skip the C0 / C1 / C3 intervals-per-second comparison with the oracle")
    p.add_argument("--physics", action="store_true",
                   help="the paper's volume study at one L (Table 1 parameters): "
                        "beta_c(L) and the specific-heat peak against Table 2 / Table 4")
    p.add_argument("--phys-L", type=int, default=8)
    p.add_argument("--phys-replicas", type=int, default=8)
    p.add_argument("--phys-therm", type=int, default=5)
    p.add_argument("--phys-meas", type=int, default=20)
    p.add_argument("--phys-rm", type=int, default=0, help="0 = the paper's N_RM")
    p.add_argument("--phys-start", choices=("hot", "cold", "mixed"), default="hot",
                   help="start of every chain: hot (uniform links, windows approached from "
                        "below), cold (all links 0, approached from above), or mixed (odd "
                        "replicas cold)")
    p.add_argument("--phys-intervals", default="512",
                   help="intervals over the E range; a comma-separated list runs the "
                        "discretisation study (C_V peak against dE^2, Sec. 3.5)")
    p.add_argument("--phys-save", default="", help="write the final slopes a[replica][interval] "
                                                    "to this .npy file")
    p.add_argument("--exchange", action="store_true",
                   help="replica exchange at the paper's L = 8 range (Sec. 2.5): half-overlapping "
                        "windows, one exchange round after every Robbins-Monro step; beta_c and "
                        "the C_V peak against the paper, exchange rates")
    p.add_argument("--canonical", action="store_true",
                   help="canonical <E>/6V in one pure phase (a heat-bath + overrelaxation run at "
                        "a = -beta in a window several fluctuation widths wide), against the "
                        "paper's L = 12 table beside Fig. 2")
    p.add_argument("--canon-L", type=int, default=12)
    p.add_argument("--canon-beta", type=float, default=1.014)
    p.add_argument("--canon-window", default="0.64,0.70",
                   help="E/6V bounds of the window (wide enough to hold the phase's peak)")
    p.add_argument("--canon-start", choices=("hot", "cold"), default="cold")
    p.add_argument("--canon-chains", type=int, default=2048)
    p.add_argument("--canon-therm", type=int, default=500)
    p.add_argument("--canon-blocks", type=int, default=40, help="measured blocks of 100 sweeps")
    p.add_argument("--muca", action="store_true",
                   help="multicanonical check of Sec. 2.6 at L = 8: LLR slopes of a coarse volume "
                        "study, then chains with the weight 1/rho~: histogram flatness, round "
                        "trips, reweighted <E> and C_V peak against the LLR reconstruction")
    p.add_argument("--muca-L", type=int, default=8)
    p.add_argument("--muca-slopes", default="",
                   help="take the LLR slopes from a --phys-save file (row 0 the interval "
                        "centres, then one row per replica) instead of a coarse LLR run")
    p.add_argument("--muca-chains", type=int, default=512)
    p.add_argument("--muca-sweeps", type=int, default=4000)
    p.add_argument("--muca-thin", type=int, default=1,
                   help="reweight every n-th sweep of each chain")
    p.add_argument("--uneven", action="store_true",
                   help="the uneven batch: L = 8, 12, 16 x 64 intervals, dE scaled with sqrt(V), "
                        "one persistent launch per Robbins-Monro step replayed from a CUDA graph, "
                        "autotuned launch shape")
    p.add_argument("--phases", action="store_true",
                   help="profiling driver: one overrelaxation pass, one heat-bath pass and one "
                        "composite sweep of 456 lattices of the workload (for ncu)")
    return p.parse_args()


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(args, rank):
    from paper_1509_08391_gb300 import workloads
    w = workloads.l20_critical(n_int=args.intervals)
    # weak scaling: each rank owns its own interval ids
    w.interval_id = [i + rank * 100000 for i in w.interval_id]
    w.n_therm, w.n_meas = args.n_therm, args.n_meas
    return w


def aggregate(units_per_rank, seconds, dist=None, device=None):
    """Whole-job throughput: units of all ranks over the slowest rank's time
    (max over ranks, the barrier-bracketed timing of the benchmark contract)."""
    total, t = float(units_per_rank), float(seconds)
    if dist is not None and dist.is_initialized():
        import torch
        v = torch.tensor([total, t], dtype=torch.float64, device=device)
        tot = v[:1].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        mx = v[1:].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        total, t = float(tot.item()), float(mx.item())
    return total / t, t


def config_dict(args, w, world):
    return {"workload": w.name, "L": 20, "lattices_per_gpu": w.n_lattices,
            "intervals": args.intervals, "replicas": 8, "dE": 12.0,
            "E_over_6V": [0.62, 0.67], "hb_or": "1:%d" % w.n_or,
            "sweeps_per_step": args.n_therm + args.n_meas, "n_therm": args.n_therm,
            "n_meas": args.n_meas, "accept_block": w.block,
            "parallelism": "dp%d (independent lattices, no collective)" % world,
            "threads_per_cta": getattr(args, "threads_used", args.threads),
            "launch_shape": getattr(args, "shape_used", None),
            "l2": "inputs larger than L2 (5.2 GB of links per GPU)"}


def cpu_baseline(w, n_sweeps=8, max_lat=None, threads=None):
    """The FP64 oracle on a bounded sample of the same workload (host cores):
    one lattice per core, n_sweeps composite sweeps (about 10 s on 16 cores);
    threads=1 gives the one-core figure."""
    import oracle
    cores = (os.cpu_count() or 1) if threads is None else threads
    n = min(cores, w.n_lattices) if max_lat is None else max_lat
    g = oracle.Geom([20] * 4)
    lats = [oracle.Lattice(g, w.seed, w.interval_id[i], w.replica_id[i], w.E_lo[i], w.dE[i],
                           n_or=w.n_or, block=w.block, beta_up=w.beta_up, beta_dn=w.beta_dn)
            for i in range(n)]
    for t in lats:
        t.hot_start()
    oracle.parallel_approach(lats, 200, cores)
    a = np.full(n, w.a0)
    t0 = time.perf_counter()
    oracle.parallel_sweeps(lats, a, n_sweeps, cores)
    dt = time.perf_counter() - t0
    upd = n * n_sweeps * (1 + w.n_or) * 4 * 20 ** 4
    return {"value": upd / dt, "unit": METRIC, "cores": min(cores, n), "kind": "oracle",
            "sample": "%d L=20 lattices of the workload x %d composite sweep(s) (%.3g link "
                      "updates, %.1f s), FP64 C, one host thread per lattice"
                      % (n, n_sweeps, upd, dt)}, lats


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle, as it stands, on the host cores."""
    w = workload(args, 0)
    if rank != 0:
        print(json.dumps({"impl": "reference", "rank": rank, "skipped": "rank 0 runs the oracle"}),
              file=sys.stderr)
        return
    import oracle
    cores = os.cpu_count() or 1
    n = min(cores, w.n_lattices)
    base, lats = cpu_baseline(w, n_sweeps=1, max_lat=n)
    a = np.full(n, w.a0)
    for _ in range(args.warmup):
        oracle.parallel_sweeps(lats, a, 1, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.parallel_sweeps(lats, a, 1, cores)
    dt = time.perf_counter() - t0
    upd = args.steps * n * (1 + w.n_or) * 4 * 20 ** 4
    v = upd / dt
    cfg = config_dict(args, w, 1)
    cfg["reference_sample"] = "%d lattices x 1 composite sweep per step" % n
    out = {"metric": METRIC, "value": v, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg, "impl": "reference",
           "cpu_baseline": {"value": v, "unit": METRIC, "cores": n, "kind": "oracle",
                            "sample": cfg["reference_sample"]},
           "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def kernel_profile():
    """The ncu record of the sweep kernel committed under profiles/ (DRAM bytes
    and warp instructions of one captured launch), or None when the kernel
    source has changed since the capture (SHA-256 check)."""
    import hashlib
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "llr_kernel_traffic.json")))
        src = open(os.path.join(ROOT, "paper_1509_08391_gb300", "csrc", "llr_chain.cu"), "rb").read()
    except (OSError, ValueError):
        return None
    if prof.get("source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return prof


def kernel_traffic(lattice_sweeps):
    """DRAM bytes (read + write) of one launch of the sweep kernel, from the ncu
    counters committed under profiles/: bytes per lattice-sweep of the captured
    case times the lattice-sweeps of this launch (the traffic grows in
    proportion to them).  None when the kernel source has changed since the
    capture."""
    prof = kernel_profile()
    if prof is None:
        return None
    return float(prof["dram_bytes_per_lattice_sweep"]) * lattice_sweeps


def issue_roofline(updates_per_s, n_sm, mhz):
    """The sweep kernel against the instruction-issue ceiling (4 schedulers per
    SM, one warp instruction each per clock): warp instructions per link
    update from the committed ncu capture times the measured update rate.
    None when the kernel source has changed since the capture."""
    prof = kernel_profile()
    if prof is None or "warp_instructions_per_update" not in prof:
        return None
    ipu = float(prof["warp_instructions_per_update"])
    achieved = updates_per_s * ipu / 1e9
    peak = ISSUE_PER_CLK_SM * n_sm * mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "G warp instructions/s", "frac": achieved / peak,
            "warp_instructions_per_update": ipu,
            "peak_source": "%d warp instructions/clk/SM x %d SMs x %.0f MHz (unit counts, the "
                           "queried SM count and the sampled max clock)"
                           % (ISSUE_PER_CLK_SM, n_sm, mhz),
            "instructions_source": "smsp__inst_executed.sum of the committed ncu capture"}


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import llr
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = workload(args, rank)
    from paper_1509_08391_gb300 import autotune
    if args.threads == 0:
        shape = autotune.tune(w)
    else:
        shape = dict(autotune.DEFAULT, threads=args.threads)
    stream = torch.cuda.Stream(device=dev)
    b = llr.Batch.from_workload(w, stream=stream.cuda_stream, max_approach=1000)
    autotune.apply(b, shape)
    b.stats(reset=True)
    args.threads_used = shape["threads"]
    args.shape_used = shape
    n = w.n_lattices
    upd_per_step = n * (args.n_therm + args.n_meas) * (1 + w.n_or) * 4 * 20 ** 4

    a_dev = torch.full((n,), w.a0, dtype=torch.float64, device=dev)
    mean_dev = torch.zeros(n, dtype=torch.float64, device=dev)
    rm = 0

    def step_dev():
        nonlocal rm
        b.rm_step_dev(a_dev, a_dev, args.n_therm, args.n_meas, rm, mean_dev)
        rm += 1

    for _ in range(args.warmup):
        step_dev()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        step_dev()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    value, secs = aggregate(upd_per_step * args.steps, ms / 1e3, dist, dev)
    per_launch_ms = 1e3 * secs / args.steps

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        a_host = torch.full((n,), w.a0, dtype=torch.float64).pin_memory()
        m_host = torch.zeros(n, dtype=torch.float64).pin_memory()
        import ctypes
        lib = llr.load()
        a_np = a_host.numpy()
        m_np = m_host.numpy()
        ke = max(1, args.steps // 2)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(ke):
            code = lib.llr_rm_step(b._h, args.n_therm, args.n_meas, rm,
                                   a_np.ctypes.data_as(ctypes.c_void_p),
                                   m_np.ctypes.data_as(ctypes.c_void_p))
            rm += 1
            if code != 0:
                raise RuntimeError(lib.llr_last_error().decode())
        dt = time.perf_counter() - t0
        e2e_value, _ = aggregate(upd_per_step * ke, dt, dist, dev)
        e2e = {"value": e2e_value, "unit": METRIC,
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 16 * n,
               "steps": ke}

    st = b.stats()
    hb = float(st["hb_acc"].sum() / max(st["hb_tot"].sum(), 1))
    orr = float(st["or_acc"].sum() / max(st["or_tot"].sum(), 1))
    drift = float(st["max_drift"].max())
    status_ok = bool(np.all(b.status() == 0))
    # heat-bath and overrelaxation passes of the whole batch, each timed as its
    # own launch (outside the timed region): link updates/s per pass kind
    a_pass = a_dev.cpu().numpy()
    pass_rates = {}
    for kind, name in ((0, "heat_bath"), (1, "overrelaxation")):
        b.single_pass(kind, a_pass)              # warm-up
        t_ms = []
        for _ in range(3):
            p0 = torch.cuda.Event(enable_timing=True)
            p1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            p0.record(stream)
            b.single_pass(kind, a_pass)
            p1.record(stream)
            p1.synchronize()
            t_ms.append(p0.elapsed_time(p1))
        pass_rates[name] = n * 4 * 20 ** 4 / (min(t_ms) / 1e3)
    b.close()
    if rank != 0:
        return

    # roofline of the dominant kernel (the batched sweep kernel, one launch per step)
    upd_per_launch = upd_per_step
    mhz = clk.get("sm_max_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_sfu = SFU_OPS_PER_CLK_SM * n_sm * mhz * 1e6 / 1e9              # G MUFU ops/s
    ach_sfu = MUFU_PER_UPDATE * upd_per_launch / (per_launch_ms / 1e3) / 1e9
    hbm_peak, hbm_src = 6800.0, "fallback (6.8 TB/s, no measured peaks file)"
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        hbm_src = "MEASURED_PEAKS.json"
    except Exception:
        pass
    ach_hbm = BYTES_PER_UPDATE * upd_per_launch / (per_launch_ms / 1e3) / 1e9
    traffic = kernel_traffic(n * (args.n_therm + args.n_meas))
    issue = issue_roofline(upd_per_launch / (per_launch_ms / 1e3), n_sm, mhz)
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_launch_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64",
        "data": "synthetic (hot start from Philox, seed %d)" % w.seed,
        "config": config_dict(args, w, world),
        "rm_lattice_steps_per_s": world * n / (per_launch_ms / 1e3),
        "rm_lattice_steps_note": "Robbins-Monro steps of (interval, replica) chains per second "
                                 "(one step = n_therm + n_meas composite sweeps and the update)",
        "link_updates_per_s_by_pass": pass_rates,
        "acceptance": {"heat_bath": hb, "overrelaxation": orr},
        "max_tracked_minus_fresh": drift, "status_ok": status_ok,
        "roofline": {"bound": "alu", "achieved": ach_sfu, "peak": peak_sfu,
                     "unit": "G MUFU ops/s (SFU pipe)", "frac": ach_sfu / peak_sfu,
                     "traffic": traffic,
                     "algorithmic": "12 MUFU ops per link update (sine and cosine of 6 staples)",
                     "peak_source": "16 MUFU ops/clk/SM x %d SMs x %.0f MHz (derived from "
                                    "unit counts, the queried SM count and the sampled max "
                                    "clock)" % (n_sm, mhz)},
        "roofline_hbm": {"bound": "hbm", "achieved": ach_hbm, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ach_hbm / hbm_peak, "peak_source": hbm_src},
        "roofline_issue": issue,
        "clocks": clk, "gpu_launches": args.steps,
        "e2e": e2e,
    }
    if not args.no_converge and world == 1:
        # second half of the benchmark metric: RM-converged intervals/s, three
        # arms on this GPU (a stated subset, see converge_leg)
        out["converged_intervals"] = converge_leg(args)
    if not args.no_cpu:
        try:
            out["cpu_baseline"], _ = cpu_baseline(w)
            out["cpu_baseline_1core"], _ = cpu_baseline(w, n_sweeps=1, max_lat=1, threads=1)
            if not args.no_configs and world == 1:
                out["cpu_baseline"]["config_rates"] = cpu_baseline_configs()
        except Exception as e:  # keep the GPU line even if the host baseline fails
            out["cpu_baseline"] = {"error": str(e)}
    if not args.no_configs and not args.no_cpu and world == 1:
        out["config_rates"] = config_rates_leg(args, w, value, out.get("cpu_baseline"))
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def config_rates_leg(args, w3, gpu_value, cpu_base):
    """Intervals per second for whole Robbins-Monro runs on this GPU (Algorithm
    1: hot start, approach, then the configuration's N_RM iterations of every
    (interval, replica) chain), set beside the oracle's figures for the same
    runs that the cpu_baseline leg measured (cpu_base["config_rates"]):
    - C0: L = 4, 8 intervals x 4 replicas, dE = 4, 50 + 100 sweeps per step,
      20 steps, run whole;
    - C1: L = 8, 32 intervals x 4 replicas, dE = 8, 50 + 100 sweeps per step,
      100 steps, run whole;
    - C3 (the benchmark, 256 intervals x 8 replicas at L = 20, 200 steps of the
      timed steps' sweeps): extrapolated from the timed link-update rate.
    An interval counts once all its replicas have finished."""
    import torch
    from paper_1509_08391_gb300 import llr
    res = {"unit": "intervals/s", "definition": "intervals x replicas whole Robbins-Monro runs "
           "(approach + N_RM steps); intervals / wall seconds"}
    cpu_rates = (cpu_base or {}).get("config_rates", {})

    def gpu_run(w):
        n = w.n_lattices
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with llr.Batch.from_workload(w, max_approach=w.max_approach) as b:
            a_dev = torch.full((n,), w.a0, dtype=torch.float64, device="cuda")
            b.rm_run(a_dev, w.n_therm, w.n_meas, 0, w.n_rm)
            torch.cuda.synchronize()
            ok = bool(np.all(b.status() == 0))
        return time.perf_counter() - t0, ok

    for name, w in config_workloads():
        n_int = len(set(w.interval_id))
        tg, okg = gpu_run(w)
        row = {"workload": w.name, "intervals": n_int, "lattices": w.n_lattices,
               "n_therm": w.n_therm, "n_meas": w.n_meas, "n_rm": w.n_rm,
               "gpu": {"intervals_per_s": n_int / tg, "seconds": tg, "status_ok": okg}}
        if name in cpu_rates and cpu_rates[name].get("intervals_per_s"):
            row["gpu_over_cpu_baseline"] = (row["gpu"]["intervals_per_s"]
                                            / cpu_rates[name]["intervals_per_s"])
        res[name] = row
    n3 = len(set(w3.interval_id))
    upd3 = w3.n_lattices * 200 * (args.n_therm + args.n_meas) * (1 + w3.n_or) * 4 * 20 ** 4
    c3 = {"workload": w3.name, "intervals": n3, "lattices": w3.n_lattices, "n_rm": 200,
          "sweeps_per_step": args.n_therm + args.n_meas,
          "gpu": {"intervals_per_s": n3 / (upd3 / gpu_value), "kind": "extrapolated",
                  "from": "the timed link-update rate of this line"}}
    if cpu_base and "value" in cpu_base:
        c3["cpu_baseline_intervals_per_s"] = n3 / (upd3 / cpu_base["value"])
        c3["cpu_baseline_kind"] = "extrapolated from cpu_baseline's link-update rate"
    res["C3"] = c3
    return res


def config_workloads():
    from paper_1509_08391_gb300 import workloads
    return (("C0", workloads.small_l4(replicas=4)), ("C1", workloads.l8_batch(replicas=4)))


def cpu_baseline_configs():
    """The oracle's intervals/s for the whole Robbins-Monro runs of C0 and C1
    (see config_rates_leg), on the host cores, one thread per lattice: C0 run
    whole; C1 from 1 and 2 steps of one lattice per core, extrapolated to 100
    steps and all lattices (labelled so)."""
    import oracle
    cores = os.cpu_count() or 1
    out = {}

    def oracle_run(w, idx, n_rm):
        g = oracle.Geom([w.L[idx[0]]] * 4)
        t0 = time.perf_counter()
        r = oracle.batch_run(g, w.seed, [w.interval_id[i] for i in idx],
                             [w.replica_id[i] for i in idx], [w.E_lo[i] for i in idx],
                             [w.dE[i] for i in idx], np.full(len(idx), w.a0), n_or=w.n_or,
                             block=w.block, n_therm=w.n_therm, n_meas=w.n_meas, n_rm=n_rm,
                             max_approach=w.max_approach, beta_up=w.beta_up,
                             beta_dn=w.beta_dn, n_threads=cores)
        return time.perf_counter() - t0, bool(np.all(r["status"] == 0))

    for name, w in config_workloads():
        n_int = len(set(w.interval_id))
        if name == "C0":
            t, ok = oracle_run(w, list(range(w.n_lattices)), w.n_rm)
            out[name] = {"intervals_per_s": n_int / t, "seconds": t, "cores": cores,
                         "status_ok": ok, "kind": "measured"}
        else:
            idx = list(range(min(cores, w.n_lattices)))
            t1, ok1 = oracle_run(w, idx, 1)
            t2, ok2 = oracle_run(w, idx, 2)
            step = max(t2 - t1, 1e-9)
            t_approach = max(t1 - step, 0.0)
            waves = -(-w.n_lattices // len(idx))
            t_all = waves * (t_approach + w.n_rm * step)
            out[name] = {"intervals_per_s": n_int / t_all, "seconds": t_all, "cores": cores,
                         "status_ok": ok1 and ok2, "kind": "extrapolated",
                         "sample": "%d lattices (one per core) for 1 and 2 Robbins-Monro steps: "
                                   "%.1f s per step, %.1f s approach; x %d steps x %d waves"
                                   % (len(idx), step, t_approach, w.n_rm, waves)}
    return out


def converge_leg(args, L=None, n_int=None, replicas=None, n_rm=None, plain=True):
    """RM-converged intervals/s at L = 20 in three arms on the same GPU:
    batched + learned warm start, batched + naive start, and the plain form
    (one lattice at a time, one launch per pass, no graph, naive start).
    Workload: intervals over E/6V in [0.58, 0.68] at dE = 8 (L/8)^2 (the
    learned-start targets; at the benchmark's dE = 12 the stopping rule would
    need ~700 steps), R replicas, 2 + 8 composite sweeps per step.  Stopping
    rule (Sec. 2.4): replica-mean |a(n+1) - a(n)| <= 1e-4 for 3 steps; the
    achieved |a - a_ref| at that step is reported beside it, a_ref being the
    naive run continued to twice the steps.  The plain arm runs, unextrapolated,
    the interval whose naive stopping step is the median, for exactly that many
    steps, and must end bit-identical to the batched naive chains."""
    import torch
    from paper_1509_08391_gb300 import warmstart, workloads
    L = L or args.target_L
    n_int = n_int or args.target_intervals
    R = replicas or args.target_replicas
    n_rm = n_rm or args.n_rm
    t_all = time.perf_counter()
    data = warmstart.training_set(n_int=24, replicas=args.train_replicas, n_rm=args.train_rm,
                                  n_therm=args.n_therm, n_meas=args.n_meas)
    net, eps, loss = warmstart.fit_network(data)
    target = workloads.warm_start_targets(L, replicas=R, n_int=n_int)
    warm, naive, ref_a, ref_err, n0 = warmstart.converge_arms(target, net, eps, n_rm,
                                                              args.n_therm, args.n_meas)
    net.close()

    def arm_dict(a):
        done = [k for k, s in enumerate(a.steps) if s is not None]
        return {"converged": len(done), "of": len(a.steps),
                "steps_to_all": max(a.converged()) if len(done) == len(a.steps) else None,
                "median_steps": float(np.median(a.converged())) if done else None,
                "seconds_per_step": a.seconds_per_step,
                "intervals_per_s": a.intervals_per_s(n_rm),
                "err_at_stop": {"mean": float(np.mean(a.err_at_stop[done])) if done else None,
                                "max": float(np.max(a.err_at_stop[done])) if done else None},
                "err_start": float(a.err_curve[0]),
                "err_after_10": float(a.err_curve[min(10, len(a.err_curve) - 1)])}

    out = {"metric": "RM-converged LLR intervals/s", "unit": "intervals/s",
           "workload": target.name, "L": L, "intervals": n_int, "replicas": R,
           "dE": float(target.dE[0]), "E_over_6V": [0.58, 0.68],
           "n_therm": args.n_therm, "n_meas": args.n_meas, "n_rm": n_rm,
           "stopping_rule": "replica-mean |a(n+1)-a(n)| <= 1e-4 for 3 consecutive steps",
           "reference": "naive batched run continued to %d steps; replica-mean stderr mean %.2g"
                        % (2 * n_rm, float(np.mean(ref_err))),
           "mlp": {"train_points": int(len(data["a"])), "train_seconds": data["seconds"],
                   "holdout_rms_L16": eps, "final_loss": loss, "gain_offset_n0": n0},
           "batched_learned": arm_dict(warm), "batched_naive": arm_dict(naive)}
    if plain:
        steps = naive.steps
        done = [(s, k) for k, s in enumerate(steps) if s is not None]
        if done:
            done.sort()
            s_med, k_med = done[len(done) // 2]
            a_plain, wall = warmstart.plain_arm(target, k_med, s_med, args.n_therm, args.n_meas)
            ids = np.asarray(target.interval_id)
            idx = np.nonzero(ids == np.unique(ids)[k_med])[0]
            same = bool(np.array_equal(a_plain, naive.hist[s_med - 1][idx]))
            out["plain_naive"] = {"interval": int(k_med), "steps": int(s_med),
                                  "lattices": int(idx.size), "wall_seconds": wall,
                                  "intervals_per_s": 1.0 / wall,
                                  "bit_identical_to_batched_naive": same,
                                  "timing": "measured (host wall clock), not extrapolated"}
            out["speedup_vs_plain"] = {
                "batched_learned": out["batched_learned"]["intervals_per_s"] * wall,
                "batched_naive": out["batched_naive"]["intervals_per_s"] * wall}
    out["wall_seconds"] = time.perf_counter() - t_all
    return out


def run_converge(args):
    """--converge: converge_leg with its full report."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    print(json.dumps(converge_leg(args)), flush=True)


def run_c4(args):
    """--c4: the learned warm start as configured: trained on the method's own
    slopes at L = 8 ... 16, predicting 128 intervals over E/6V in [0.58, 0.68]
    at L = 20 and L = 24 (R = 4); steps to the stopping rule and error after k
    steps with and without the network, per range of E/6V."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import warmstart, workloads
    t_all = time.perf_counter()
    data = warmstart.training_set(n_int=24, replicas=args.train_replicas, n_rm=args.train_rm,
                                  n_therm=args.n_therm, n_meas=args.n_meas)
    net, eps, loss = warmstart.fit_network(data)
    res = {"metric": "learned warm start vs naive start (C4)", "n_therm": args.n_therm,
           "n_meas": args.n_meas, "n_rm": args.n_rm, "replicas": 4,
           "stopping_rule": "replica-mean |a(n+1)-a(n)| <= 1e-4 for 3 consecutive steps",
           "mlp": {"train_points": int(len(data["a"])), "holdout_rms_L16": eps,
                   "train_replicas": args.train_replicas, "train_rm_steps": args.train_rm,
                   "final_loss": loss, "train_seconds": data["seconds"]}, "volumes": {}}
    bins = np.linspace(0.58, 0.68, 5)
    for L in (20, 24):
        target = workloads.warm_start_targets(L, replicas=4, n_int=128)
        t0 = time.perf_counter()
        warm, naive, ref_a, ref_err, n0 = warmstart.converge_arms(target, net, eps, args.n_rm,
                                                                  args.n_therm, args.n_meas)
        _, e6v, _ = warmstart.interval_features(target)
        iid = np.asarray(target.interval_id)
        e_int = np.array([e6v[np.nonzero(iid == k)[0][0]] for k in np.unique(iid)])
        rows = []
        for b0, b1 in zip(bins[:-1], bins[1:]):
            sel = np.nonzero((e_int >= b0) & (e_int < b1 + 1e-12))[0]

            def stat(a):
                st = [a.steps[k] for k in sel]
                ok = [s for s in st if s is not None]
                return {"converged": len(ok), "of": len(st),
                        "median_steps": float(np.median(ok)) if ok else None,
                        "err_at_stop_mean": float(np.mean([a.err_at_stop[k] for k in sel
                                                           if a.steps[k] is not None]))
                        if ok else None}
            rows.append({"E_over_6V": [float(b0), float(b1)], "intervals": int(sel.size),
                         "a_ref_mean": float(np.mean(ref_a[sel])),
                         "start_error": {"learned": float(np.mean(np.abs(
                             net_pred_cache(net, target)[sel] - ref_a[sel]))),
                                         "naive": float(np.mean(np.abs(target.a0 - ref_a[sel])))},
                         "learned": stat(warm), "naive": stat(naive)})
        res["volumes"][str(L)] = {
            "workload": target.name, "dE": float(target.dE[0]), "gain_offset_n0": n0,
            "seconds": time.perf_counter() - t0,
            "mean_err_after_k": {"k": [0, 5, 10, 20, 40],
                                 "learned": [float(warm.err_curve[k]) for k in (0, 5, 10, 20, 40)],
                                 "naive": [float(naive.err_curve[k]) for k in (0, 5, 10, 20, 40)]},
            "all": {"learned": {"converged": len(warm.converged()),
                                "median_steps": float(np.median(warm.converged()))
                                if warm.converged() else None},
                    "naive": {"converged": len(naive.converged()),
                              "median_steps": float(np.median(naive.converged()))
                              if naive.converged() else None}},
            "by_energy": rows, "ref_stderr_mean": float(np.mean(ref_err))}
    net.close()
    res["wall_seconds"] = time.perf_counter() - t_all
    print(json.dumps(res), flush=True)


def net_pred_cache(net, target, _cache={}):
    """The learned start a(L, E/6V, dE/6V) of each interval (one value per
    interval id, in ascending id order)."""
    from paper_1509_08391_gb300 import warmstart
    key = (target.name, target.n_lattices)
    if key not in _cache:
        L, e6v, d6v = warmstart.interval_features(target)
        a = net.predict(L, e6v, d6v)
        iid = np.asarray(target.interval_id)
        _cache[key] = np.array([a[np.nonzero(iid == k)[0][0]] for k in np.unique(iid)])
    return _cache[key]


# The paper's results for the volume study (Table 2, Table 4): beta_c(L)
# and the specific-heat peak, normalised as var(E/6V) (its "C_V/(6V)").
PAPER_BETA_C = {8: (1.00744, 2e-5), 10: (1.00939, 2e-5), 12: (1.010245, 1e-6),
                14: (1.010635, 5e-6), 16: (1.010833, 4e-6), 18: (1.010948, 2e-6),
                20: (1.011006, 2e-6)}
PAPER_CV_PEAK = {8: (0.000551, 2e-6), 10: (0.000384, 2e-6), 12: (0.0002971, 1.1e-6),
                 14: (0.0002537, 8e-7), 16: (0.0002272, 7e-7), 18: (0.0002097, 5e-7),
                 20: (0.0002007, 4e-7)}


def cold_replica(start, r):
    """Whether replica r starts cold under --phys-start (hot, cold, or mixed:
    odd replicas cold, even replicas hot)."""
    return start == "cold" or (start == "mixed" and r % 2 == 1)


def physics_study(L, replicas, n_therm, n_meas, n_rm, beta_window=(1.0, 1.016), n_int=512,
                  start="hot"):
    """The whole LLR path at the paper's volume-study parameters: start,
    approach, n_rm graph-replayed Robbins-Monro iterations of every
    (interval, replica) chain from a = -1, then per replica ln rho and the
    specific-heat peak; returns the per-replica beta_c and var(E/6V) peak.
    A hot start draws every link uniformly and approaches each window from
    below (a quench at beta_up); a cold start sets every link to 0 (E = 6V)
    and approaches from above (heating at beta_dn)."""
    import torch
    from paper_1509_08391_gb300 import llr, workloads
    w = workloads.paper_volume_study(L, replicas, n_therm, n_meas, n_rm, n_int=n_int)
    n = w.n_lattices
    stream = torch.cuda.Stream()
    t_all = time.perf_counter()
    cold = [cold_replica(start, r) for r in w.replica_id]
    with llr.Batch.from_workload(w, stream=stream.cuda_stream,
                                 max_approach=0 if any(cold) else 5000) as b:
        if any(cold):
            zeros = np.zeros(4 * L ** 4, dtype=np.float32)
            for i in np.nonzero(cold)[0]:
                b.set_links(int(i), zeros)
            b.approach(5000)
        a_dev = torch.full((n,), w.a0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.rm_run(a_dev, w.n_therm, w.n_meas, 0, w.n_rm)
        torch.cuda.synchronize()
        t_rm = time.perf_counter() - t0
        a = a_dev.cpu().numpy()
        ok = bool(np.all(b.status() == 0))
        st = b.stats()
    six_v = 6.0 * L ** 4
    lo = np.asarray(w.E_lo)
    rid = np.asarray(w.replica_id)
    iid = np.asarray(w.interval_id)
    dE = w.dE[0]
    bc, cv = [], []
    for r in range(replicas):
        idx = np.where(rid == r)[0]
        idx = idx[np.argsort(iid[idx])]
        c = lo[idx] + 0.5 * dE
        b_r, v_r = llr.cv_peak(c, a[idx], beta_window[0], beta_window[1], n_grid=1601, tol=1e-10)
        bc.append(b_r)
        cv.append(v_r / six_v ** 2)
    # the replica-mean slopes give one more estimate (averaging before the
    # non-linear peak search)
    a_rep = np.stack([a[np.where(rid == r)[0][np.argsort(iid[rid == r])]]
                      for r in range(replicas)])
    c_all = lo[np.where(rid == 0)[0][np.argsort(iid[rid == 0])]] + 0.5 * dE
    b_m, v_m = llr.cv_peak(c_all, a_rep.mean(axis=0), beta_window[0], beta_window[1],
                           n_grid=1601, tol=1e-10)
    upd = n * w.n_rm * (w.n_therm + w.n_meas) * (1 + w.n_or) * 4 * L ** 4
    return {"workload": w.name, "L": L, "intervals": n_int, "replicas": replicas, "dE": dE,
            "start": start, "cold_replicas": [r for r in range(replicas) if cold_replica(start, r)],
            "E_over_6V": [lo.min() / six_v, (lo.max() + dE) / six_v],
            "n_therm": w.n_therm, "n_meas": w.n_meas, "n_rm": w.n_rm, "a0": w.a0,
            "status_ok": ok, "heat_bath_acceptance": float(st["hb_acc"].sum() / st["hb_tot"].sum()),
            "beta_c_per_replica": bc, "cv_peak_per_replica": cv,
            "from_replica_mean_slopes": {"beta_c": b_m, "cv_peak": v_m / six_v ** 2},
            "slopes": a_rep, "centres": c_all,
            "rm_seconds": t_rm, "wall_seconds": time.perf_counter() - t_all,
            "link_updates_per_s": upd / t_rm}


def run_physics(args):
    """--physics: beta_c(L) and the specific-heat peak of the paper's volume
    study, computed end to end on the GPU, against the paper's tables."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    L = args.phys_L
    n_list = [int(x) for x in args.phys_intervals.split(",")]
    if len(n_list) > 1:
        run_discretisation(args, L, n_list)
        return
    res = physics_study(L, args.phys_replicas, args.phys_therm, args.phys_meas, args.phys_rm,
                        n_int=n_list[0], start=args.phys_start)
    a_rep, centres = res.pop("slopes"), res.pop("centres")
    if args.phys_save:
        np.save(args.phys_save, np.vstack([centres[None, :], a_rep]))
    R = len(res["beta_c_per_replica"])
    for key, paper in (("beta_c", PAPER_BETA_C), ("cv_peak", PAPER_CV_PEAK)):
        v = np.asarray(res[key + "_per_replica"])
        m, e = float(v.mean()), float(v.std(ddof=1) / np.sqrt(R)) if R > 1 else float("nan")
        res[key] = {"mean": m, "stderr": e}
        if L in paper:
            pv, pe = paper[L]
            res[key]["paper"] = pv
            res[key]["paper_err"] = pe
            res[key]["deviation_sigma"] = (m - pv) / float(np.hypot(e, pe))
    if args.phys_start == "mixed":
        # the same statistics per kind of start, and the slopes' difference
        cold = np.array([cold_replica("mixed", r) for r in range(R)])
        res["by_start"] = {}
        for name, sel in (("hot", ~cold), ("cold", cold)):
            bc = np.asarray(res["beta_c_per_replica"])[sel]
            cv = np.asarray(res["cv_peak_per_replica"])[sel]
            res["by_start"][name] = {
                "beta_c": float(bc.mean()), "beta_c_err": float(bc.std(ddof=1) / np.sqrt(bc.size)),
                "cv_peak": float(cv.mean()), "cv_peak_err": float(cv.std(ddof=1) / np.sqrt(cv.size))}
        da = a_rep[cold].mean(axis=0) - a_rep[~cold].mean(axis=0)
        err = np.sqrt(a_rep[cold].var(axis=0, ddof=1) / cold.sum()
                      + a_rep[~cold].var(axis=0, ddof=1) / (~cold).sum())
        six_v = 6.0 * L ** 4
        res["slopes_cold_minus_hot"] = {
            "E_over_6V": [float(x) for x in centres[::32] / six_v],
            "mean_diff_per_32": [float(x) for x in da.reshape(-1, 32).mean(axis=1)],
            "z_per_32": [float(x) for x in (da.reshape(-1, 32).sum(axis=1)
                                            / np.sqrt((err.reshape(-1, 32) ** 2).sum(axis=1)))]}
    res["metric"] = "beta_c(L) and C_V peak vs the paper (Table 2, Table 4)"
    print(json.dumps(res), flush=True)


def run_discretisation(args, L, n_list):
    """Sec. 3.5: the C_V peak against the interval width dE (the paper finds a
    quadratic law, C_V(dE) = C_V(0) + b dE^2); one volume-study run per number
    of intervals, then a weighted least-squares fit in dE^2."""
    rows = []
    for n_int in n_list:
        res = physics_study(L, args.phys_replicas, args.phys_therm, args.phys_meas,
                            args.phys_rm, n_int=n_int)
        res.pop("slopes")
        res.pop("centres")
        v = np.asarray(res["cv_peak_per_replica"])
        bc = np.asarray(res["beta_c_per_replica"])
        R = v.size
        rows.append({"intervals": n_int, "dE": res["dE"], "cv_peak": float(v.mean()),
                     "cv_err": float(v.std(ddof=1) / np.sqrt(R)), "beta_c": float(bc.mean()),
                     "beta_c_err": float(bc.std(ddof=1) / np.sqrt(R)),
                     "rm_seconds": res["rm_seconds"], "status_ok": res["status_ok"]})
    x = np.array([r["dE"] ** 2 for r in rows])
    y = np.array([r["cv_peak"] for r in rows])
    e = np.array([max(r["cv_err"], 1e-12) for r in rows])
    A = np.stack([np.ones_like(x), x], axis=1) / e[:, None]
    coef, *_ = np.linalg.lstsq(A, y / e, rcond=None)
    cov = np.linalg.inv(A.T @ A)
    chi2 = float(np.sum(((y - (coef[0] + coef[1] * x)) / e) ** 2))
    out = {"metric": "C_V peak against dE (Sec. 3.5)", "L": L, "replicas": args.phys_replicas,
           "n_therm": args.phys_therm, "n_meas": args.phys_meas, "rows": rows,
           "fit": {"cv_peak_dE0": float(coef[0]), "cv_peak_dE0_err": float(np.sqrt(cov[0, 0])),
                   "slope_per_dE2": float(coef[1]), "slope_err": float(np.sqrt(cov[1, 1])),
                   "chi2": chi2, "dof": len(rows) - 2},
           "paper_cv_peak_512": PAPER_CV_PEAK.get(L)}
    print(json.dumps(out), flush=True)


# <E>/6V at L = 12 from the paper's comparison of LLR and reweighting with
# rho~ (the table beside Fig. 2): beta -> (LLR, reweighting), errors.
PAPER_E_L12 = {1.006: ((0.60180, 6e-5), (0.601714, 8e-6)),
               1.008: ((0.60901, 8e-5), (0.60906, 1e-5)),
               1.010: ((0.6271, 4e-4), (0.6274, 1e-4)),
               1.01023: ((0.6349, 5e-4), (0.6352, 1e-4)),
               1.012: ((0.65685, 5e-5), (0.65687, 1e-5)),
               1.014: ((0.66018, 4e-5), (0.660230, 5e-6))}


def run_exchange(args):
    """--exchange: the LLR run of the paper's L = 8 range with overlapping
    intervals and replica exchange (Sec. 2.5): 511 windows of width 2 d,
    d = (E_max - E_min) / 512, lower edges d apart, 8 replicas; after every
    Robbins-Monro step one exchange round over the neighbouring windows of
    alternating parity (llr_replica_exchange).  Per replica the slopes at the
    window centres give ln rho~ and the C_V peak."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import llr, workloads
    L, R = 8, args.phys_replicas
    e_lo, e_hi, _, n_rm = workloads.PAPER_VOLUME_STUDY[L]
    six_v = 6.0 * L ** 4
    d = six_v * (e_hi - e_lo) / 512
    n_win = 511
    E = workloads.place_intervals(L, n_win, e_lo, e_hi, 2 * d)
    Ls, lo, de, iid, rid = [], [], [], [], []
    for k in range(n_win):
        for r in range(R):
            Ls.append(L)
            lo.append(float(E[k]))
            de.append(2 * d)
            iid.append(k)
            rid.append(r)
    w = workloads.Workload("u1_4d_L8_511win_overlap_x%d" % R, Ls, lo, de, iid, rid,
                           workloads.SEED_BASE + 30, n_therm=args.phys_therm,
                           n_meas=args.phys_meas, n_rm=n_rm)
    n = w.n_lattices
    t0 = time.perf_counter()
    tried = taken = 0
    with llr.Batch.from_workload(w, max_approach=5000) as b:
        a = np.full(n, w.a0)
        t_ex = 0.0
        for step in range(n_rm):
            a, _ = b.rm_step(a, w.n_therm, w.n_meas, step)
            te = time.perf_counter()
            acc = b.replica_exchange(workloads.exchange_pairs(w, step), a, step)
            t_ex += time.perf_counter() - te
            tried += acc.size
            taken += int(acc.sum())
        ok = bool(np.all(b.status() == 0))
    t_run = time.perf_counter() - t0
    rid = np.asarray(rid)
    bc, cv = [], []
    centres = E + d
    for r in range(R):
        idx = np.nonzero(rid == r)[0]
        b_r, v_r = llr.cv_peak(centres, a[idx], 1.0, 1.016, n_grid=1601, tol=1e-10)
        bc.append(b_r)
        cv.append(v_r / six_v ** 2)
    bc, cv = np.array(bc), np.array(cv)
    out = {"metric": "LLR with replica exchange (Sec. 2.5) at L = 8", "L": L, "windows": n_win,
           "window_width": 2 * d, "spacing": d, "replicas": R, "n_therm": w.n_therm,
           "n_meas": w.n_meas, "n_rm": n_rm, "status_ok": ok,
           "exchange": {"pairs_tried": tried, "exchanged": taken,
                        "rate": taken / max(tried, 1), "seconds": t_ex},
           "beta_c": {"mean": float(bc.mean()), "stderr": float(bc.std(ddof=1) / np.sqrt(R)),
                      "paper": PAPER_BETA_C[L]},
           "cv_peak": {"mean": float(cv.mean()), "stderr": float(cv.std(ddof=1) / np.sqrt(R)),
                       "paper": PAPER_CV_PEAK[L]},
           "beta_c_per_replica": bc.tolist(), "cv_peak_per_replica": cv.tolist(),
           "wall_seconds": t_run}
    print(json.dumps(out), flush=True)


def run_muca(args):
    """--muca: the ergodicity check of Sec. 2.6 at L = 8.  (1) LLR slopes of
    the paper's L = 8 range in 64 intervals (4 replicas, 300 Robbins-Monro
    steps); (2) independent multicanonical chains with W = 1/rho~ from the
    replica-mean slopes; (3) the energy histogram over the range, the
    tunnellings between its ends (llr_muca_tunnellings), and <E>, C_V(beta)
    reweighted from the multicanonical samples with W^-1 (eq. (2.56);
    llr_muca_reweight, llr_muca_cv_peak) against the LLR reconstruction of the
    same slopes (eqs. (2.46)/(2.47))."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import llr, workloads
    L, n_int = args.muca_L, 64
    six_v = 6.0 * L ** 4
    t_all = time.perf_counter()
    stream = torch.cuda.Stream()
    llr_info = {}
    if args.muca_slopes:
        tab = np.load(args.muca_slopes)
        centres, a_k = tab[0], tab[1:].mean(axis=0)
        n_int = centres.size
        dE = float(centres[1] - centres[0])
        llr_info = {"slopes_from": "file", "replicas": int(tab.shape[0] - 1)}
    else:
        w = workloads.paper_volume_study(L, replicas=4, n_therm=5, n_meas=20, n_rm=300,
                                         n_int=n_int)
        with llr.Batch.from_workload(w, stream=stream.cuda_stream, max_approach=5000) as b:
            a_dev = torch.full((w.n_lattices,), w.a0, dtype=torch.float64, device="cuda")
            b.rm_run(a_dev, w.n_therm, w.n_meas, 0, w.n_rm)
            torch.cuda.synchronize()
            a = a_dev.cpu().numpy()
        iid = np.asarray(w.interval_id)
        uniq = np.unique(iid)
        a_k = np.array([a[iid == k].mean() for k in uniq])
        lo = np.array([w.E_lo[np.nonzero(iid == k)[0][0]] for k in uniq])
        dE = w.dE[0]
        centres = lo + 0.5 * dE
        llr_info = {"replicas": 4, "n_rm": w.n_rm}
    e_min, e_max = centres[0] - 0.5 * dE, centres[-1] + 0.5 * dE
    # multicanonical chains: hot start, approach into [E_min, E_max], then W = 1/rho~
    nc = args.muca_chains
    # half the chains start at the bottom of the range, half at the top (the
    # approach stops where it enters its window: the first half approaches
    # the whole range and enters at its lower end, the second half a window
    # covering the top twentieth), so the bias of the starting point cancels
    span = e_max - e_min
    lo_start = [e_min if c < nc // 2 else e_max - 0.05 * span for c in range(nc)]
    de_start = [span if c < nc // 2 else 0.05 * span for c in range(nc)]
    wm = workloads.Workload("u1_4d_L%d_muca_x%d" % (L, nc), [L] * nc, lo_start, de_start,
                            list(range(nc)), [0] * nc, workloads.SEED_BASE + 40)
    a0 = float(a_k.mean())
    t0 = time.perf_counter()
    with llr.Batch.from_workload(wm, stream=stream.cuda_stream, max_approach=5000) as b:
        b.set_muca_weight(e_min, dE, a_k, a0)
        b.muca_sweep(200, history=False)
        E = b.muca_sweep(args.muca_sweeps)
        st = b.stats()
    t_muca = time.perf_counter() - t0
    # (3) flatness over the table's range
    h, _ = np.histogram(E.ravel(), bins=np.linspace(e_min, e_max, 17))
    frac = h / h.mean()
    # tunnellings between the lowest and the highest tenth of the range
    span = e_max - e_min
    trips = int(llr.muca_tunnellings(E, e_min + 0.1 * span, e_max - 0.1 * span).sum())
    # reweighting (eq. (2.56)) in the library: a sample at E carries
    # e^{beta E} / W(E) = e^{beta E + ln rho~(E)}; every muca_thin-th sweep
    # (successive sweeps of a chain are strongly correlated)
    Et = E[::max(1, args.muca_thin)]
    b_mu, cv_mu = llr.muca_cv_peak(Et, e_min, dE, a_k, 1.0, 1.016, n_grid=201, tol=1e-7)
    cv_mu /= six_v ** 2
    # spread of the reweighted peak over independent groups of chains
    groups = np.array_split(np.arange(nc), 8)
    grp = [llr.muca_cv_peak(Et[:, gidx], e_min, dE, a_k, 1.0, 1.016, n_grid=201, tol=1e-7)
           for gidx in groups]
    gb = np.array([g[0] for g in grp])
    gc = np.array([g[1] for g in grp]) / six_v ** 2
    b_llr, cv_llr = llr.cv_peak(centres, a_k, 1.0, 1.016, n_grid=1601, tol=1e-10)
    E_mu_c = llr.muca_reweight(Et, e_min, dE, a_k, [b_llr])[0][0] / six_v
    _, E1, _ = llr.observables(centres, a_k, [b_llr])
    out = {"metric": "multicanonical reweighting vs LLR reconstruction (Sec. 2.6)", "L": L,
           "starts": "half the chains at the bottom of the range, half at the top",
           "thin": max(1, args.muca_thin),
           "llr": dict(llr_info, intervals=int(n_int), dE=dE, beta_c=b_llr,
                       cv_peak=cv_llr / six_v ** 2),
           "muca": {"chains": nc, "sweeps": args.muca_sweeps, "a0": a0,
                    "heat_bath_acceptance": float(st["hb_acc"].sum() / st["hb_tot"].sum()),
                    "histogram_over_range": [float(f) for f in frac],
                    "histogram_max_dev": float(np.max(np.abs(frac - 1.0))),
                    "tunnellings": int(trips), "seconds": t_muca,
                    "beta_c": b_mu, "beta_c_err": float(gb.std(ddof=1) / np.sqrt(len(gb))),
                    "cv_peak": cv_mu, "cv_peak_err": float(gc.std(ddof=1) / np.sqrt(len(gc)))},
           "E_over_6V_at_llr_beta_c": {"muca": E_mu_c, "llr": float(E1[0] / six_v)},
           "paper": {"beta_c": PAPER_BETA_C[L], "cv_peak": PAPER_CV_PEAK[L]},
           "wall_seconds": time.perf_counter() - t_all}
    if L == 12:
        # the paper's table beside Fig. 2: <E>/6V at six couplings
        rows = []
        bl = sorted(PAPER_E_L12)
        _, E_llr, _ = llr.observables(centres, a_k, bl)
        E_all = llr.muca_reweight(Et, e_min, dE, a_k, bl)[0] / six_v
        E_grp = np.array([llr.muca_reweight(Et[:, gidx], e_min, dE, a_k, bl)[0] / six_v
                          for gidx in groups])
        for j, (bb, el) in enumerate(zip(bl, E_llr)):
            vals = E_grp[:, j]
            rows.append({"beta": bb, "muca": float(E_all[j]),
                         "muca_err": float(np.std(vals, ddof=1) / np.sqrt(len(vals))),
                         "llr_same_slopes": float(el / six_v),
                         "paper_llr": PAPER_E_L12[bb][0], "paper_reweighting": PAPER_E_L12[bb][1]})
        out["E_over_6V_table"] = rows
    print(json.dumps(out), flush=True)


def run_canonical(args):
    """--canonical: <E>/6V of one pure phase at coupling beta.  Every chain
    runs composite sweeps at a = -beta restricted to a window of E/6V several
    canonical fluctuation widths wide around the phase's peak (so the other
    phase, and the tunnelling between them, are cut away); a hot start draws
    every link uniformly and approaches the window from below (a quench at
    beta_up), a cold start sets every link to 0 and approaches from above.
    After n_therm sweeps, blocks of 100 measured sweeps (llr_sweep with
    measure); the error is the spread of the per-chain means over the
    independent chains; the block means of the first and second half show
    whether the chains still drift."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import llr, workloads
    L, nc, beta = args.canon_L, args.canon_chains, args.canon_beta
    e_lo, e_hi = (float(x) for x in args.canon_window.split(","))
    six_v = 6.0 * L ** 4
    lo, de = e_lo * six_v, (e_hi - e_lo) * six_v
    w = workloads.Workload("u1_4d_L%d_canonical_b%g_x%d" % (L, beta, nc), [L] * nc, [lo] * nc,
                           [de] * nc, list(range(nc)), [0] * nc, workloads.SEED_BASE + 77)
    cold = args.canon_start == "cold"
    t0 = time.perf_counter()
    with llr.Batch.from_workload(w, max_approach=0 if cold else 5000) as b:
        if cold:
            zeros = np.zeros(4 * L ** 4, dtype=np.float32)
            for i in range(nc):
                b.set_links(i, zeros)
            b.approach(5000)
        b.sweep(-beta, args.canon_therm)
        blocks = [b.sweep(-beta, 100, measure=True) / 100.0 + lo + 0.5 * de
                  for _ in range(args.canon_blocks)]
        ok = bool(np.all(b.status() == 0))
    e = np.array(blocks) / six_v                  # [block, chain]
    per_chain = e.mean(axis=0)
    half = args.canon_blocks // 2
    out = {"metric": "canonical <E>/6V in one pure phase", "L": L, "beta": beta,
           "window_E_over_6V": [e_lo, e_hi], "start": args.canon_start, "chains": nc,
           "n_therm": args.canon_therm, "measured_sweeps": 100 * args.canon_blocks,
           "status_ok": ok, "E_over_6V": float(per_chain.mean()),
           "err": float(per_chain.std(ddof=1) / np.sqrt(nc)),
           "first_half": float(e[:half].mean()), "second_half": float(e[half:].mean()),
           "block_range": [float(e.min()), float(e.max())],
           "seconds": time.perf_counter() - t0}
    if L == 12 and beta in PAPER_E_L12:
        out["paper_llr"], out["paper_reweighting"] = PAPER_E_L12[beta]
    print(json.dumps(out), flush=True)


def run_uneven(args):
    """--uneven: lattices of three sizes (L = 8, 12, 16, 64 intervals each over
    E/6V in [0.58, 0.68], dE = 8, 18, 32) in one persistent launch per
    Robbins-Monro step, the steps replayed from one captured CUDA graph
    (llr_rm_run), launch shape from the autotuner.  Each step is n_therm +
    n_meas composite sweeps of every lattice and the update of a."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import autotune, llr, workloads
    w = workloads.uneven_batch()
    t0 = time.perf_counter()
    shape = autotune.tune(w) if args.threads == 0 else dict(autotune.DEFAULT, threads=args.threads)
    t_tune = time.perf_counter() - t0
    n = w.n_lattices
    L = np.asarray(w.L)
    stream = torch.cuda.Stream()
    with llr.Batch.from_workload(w, stream=stream.cuda_stream, max_approach=5000) as b:
        autotune.apply(b, shape)
        a_dev = torch.full((n,), w.a0, dtype=torch.float64, device="cuda")
        b.rm_run(a_dev, args.n_therm, args.n_meas, 0, args.warmup)      # captures the graph
        torch.cuda.synchronize()
        clocks = Clocks(0)
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.rm_run(a_dev, args.n_therm, args.n_meas, 0, args.steps)       # graph replays
        e1.record(stream)
        e1.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
        last = b.last_launch()
        ok = bool(np.all(b.status() == 0))
    links = 4 * L.astype(np.float64) ** 4 * (args.n_therm + args.n_meas) * (1 + w.n_or)
    out = {"metric": "link updates/s (uneven batch, graph replays)", "unit": "link updates/s",
           "value": float(links.sum() / (ms / 1e3)), "ms_per_step": ms, "steps": args.steps,
           "warmup": args.warmup, "workload": w.name, "lattices": n,
           "L": {str(l): int((L == l).sum()) for l in sorted(set(w.L))},
           "dE": {str(l): float(w.dE[int(np.nonzero(L == l)[0][0])]) for l in sorted(set(w.L))},
           "link_update_share": {str(l): float(links[L == l].sum() / links.sum())
                                 for l in sorted(set(w.L))},
           "n_therm": args.n_therm, "n_meas": args.n_meas, "hb_or": "1:%d" % w.n_or,
           "launch_shape": shape, "last_launch": last, "tune_seconds": t_tune,
           "launches_per_step": 1, "status_ok": ok, "clocks": clk}
    print(json.dumps(out), flush=True)


def run_phases(args):
    """One launch per pass kind on 456 lattices of the benchmark workload (one
    full wave of 256-thread CTAs: 3 per SM on 152 SMs), so an ncu capture
    (-k regex:llr_kernel) sees: resync, approach, two composite sweeps (one
    launch), overrelaxation pass, heat-bath pass, composite sweep."""
    import torch
    torch.cuda.set_device(0)
    from paper_1509_08391_gb300 import build as bld
    bld.build()
    from paper_1509_08391_gb300 import llr, workloads
    w = workloads.subset(workloads.l20_critical(), range(456))
    with llr.Batch.from_workload(w, max_approach=1000) as b:
        b.set_kernel_config(args.threads or 256, True)
        a = np.full(w.n_lattices, -1.01)
        b.sweep(a, 2)           # leave the window edge the approach stops at
        b.single_pass(1, a)
        b.single_pass(0, a)
        b.sweep(a, 1)
        torch.cuda.synchronize()
    print(json.dumps({"phases": "done", "lattices": w.n_lattices}))


def main():
    args = parse()
    if args.phases:
        run_phases(args)
        return
    if args.converge:
        run_converge(args)
        return
    if args.uneven:
        run_uneven(args)
        return
    if args.c4:
        run_c4(args)
        return
    if args.physics:
        run_physics(args)
        return
    if args.muca:
        run_muca(args)
        return
    if args.canonical:
        run_canonical(args)
        return
    if args.exchange:
        run_exchange(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
