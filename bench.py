#!/usr/bin/env python
"""Benchmark of the D3Q27 high-order thread-safe LB step (arXiv 2401.17074) on one B300.

Workload: the turbulent channel, 512 x 130 x 256 lattice with halfway
bounce-back walls on the y = 0 and y = 129 layers, periodic in x and z,
tau = 0.503, constant body force g = u_tau^2 / H (u_tau = 0.0035, H = 64),
seeded laminar parabola + 2 % noise (synthetic; the paper's channel runs are
the model).  A "step" is one TSLB step over all 512*128*256 interior nodes.

Prints ONE JSON line (rank 0): MLUPS with inputs resident in HBM, the HBM
roofline of the step kernel, the 16-bit storage variants, an end-to-end
figure through the C ABI with host buffers, the FP64 oracle timed on the
host cores, and the SM clocks sampled during the timed region.

--impl reference times the FP64 CPU oracle (the only reference this method
has: the paper ships no code) on a bounded sample of the same workload.
"""
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

METRIC = "MLUPS and % of HBM roofline (D3Q27 TSLB step, 1 B300), FP32 vs BF16 storage"
BYTES_PER_NODE = {"fp32": 80, "bf16": 40, "fp16": 40}
PREC_CODE = {"fp32": 0, "bf16": 1, "fp16": 2}
FALLBACK_HBM_GBS = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="tslb", choices=["tslb", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "direct", "factored"])
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=130)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workload lines")
    ap.add_argument("--no-precision-study", action="store_true",
                    help="skip the time-averaged FP32 / BF16 / FP16 channel statistics")
    ap.add_argument("--warm", type=int, default=300000, help="precision-study: FP32 steps before the branch")
    ap.add_argument("--window", type=int, default=100000, help="precision-study: steps averaged per run")
    ap.add_argument("--only", default=None, choices=["d2q9", "adjoint", "precision-study"],
                    help="time one extra workload alone (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def profile_record(fname, kernel_name, precision, key):
    """`key` of a committed ncu record under profiles/, if the kernel sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        recs = json.load(f)
    for r in recs:
        if r.get("kernel") != kernel_name or r.get("precision") != precision:
            continue
        h = hashlib.sha256()
        for src in r["sources"]:
            path = os.path.join(ROOT, src)
            if not os.path.exists(path):
                return None
            h.update(open(path, "rb").read())
        if h.hexdigest() != r.get("sources_sha256"):
            return None
        return float(r[key])
    return None


def traffic_record(kernel_name, precision):
    """DRAM bytes per launch from a committed ncu capture."""
    return profile_record("traffic.json", kernel_name, precision, "bytes_per_launch_full")


FP32_LANES_PER_SM = 128
NOMINAL_SM_MHZ = 2032.0


def alu_entry(kernel_name, nodes, launch_s, sms, sm_mhz):
    """Executed FP32 FLOP/s of the step against the CUDA-core FP32 peak (SMs x 128 lanes x 2 FLOP x clock).
    FLOP per node come from committed ncu op counts (FFMA 2, packed FADD2/FMUL2 2, FFMA2 4); null when stale."""
    fpn = profile_record("fp32_ops.json", kernel_name, "fp32", "fp32_flop_per_node")
    if fpn is None:
        return None
    peak = sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    achieved = fpn * nodes / launch_s / 1e12
    return {"bound": "alu", "flop_per_node": fpn, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_basis": "%d SMs x %d FP32 lanes x 2 FLOP x %.0f MHz"
            % (sms, FP32_LANES_PER_SM, sm_mhz), "kernel": kernel_name}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def make_state(nx, ny, nz):
    from paper_2401_17074_b300 import workloads as W
    prm = W.channel_params(nx=nx, ny=ny, nz=nz)
    state = W.channel_state(prm, seed=1)
    return prm, state


def host_cpu():
    """The host CPU's model name (first processor entry of /proc/cpuinfo), or null."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(prm, seconds, nz_sample=None):
    """Time the FP64 oracle as it stands on a slab of the channel (periodic z) on all host cores."""
    import oracle
    from paper_2401_17074_b300 import workloads as W
    nx, ny, _ = prm["dims"]
    nz_s = nz_sample or 8
    sub = W.channel_params(nx=nx, ny=ny, nz=nz_s)
    state = W.channel_state(sub, seed=1)
    s = oracle.OracleSim(sub["dims"], sub["tau"], force=sub["force"], bc=sub["bc"])
    s.init_moments(*state)
    nodes = nx * (ny - 2) * nz_s
    t0 = time.perf_counter()
    steps = 0
    while True:
        s.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 1000:
            break
    # the oracle's step runs its (z, y) rows in parallel: every thread of the
    # team has work when there are at least as many rows as threads
    cores = min(oracle.threads(), nz_s * (ny - 2))
    return {"value": nodes * steps / el / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%dx%dx%d slab of the channel (periodic z), %d steps, FP64 populations, %.1f s"
                      % (nx, ny, nz_s, steps, el), "cpu": host_cpu(), "host_cpus": os.cpu_count()}


def cpu_other_configs(seconds):
    """The oracle, as it stands, on the other workloads' set-ups (all host cores,
    bounded samples): the 32^3 Taylor-Green vortex in full, and a 10-layer slab
    of the 256 x 256 x 640 jet (inflow and outflow faces, free-slip sides)."""
    import oracle
    from paper_2401_17074_b300 import workloads as W

    def timed(sim, nodes):
        t0 = time.perf_counter()
        steps = 0
        while True:
            sim.step(1)
            steps += 1
            el = time.perf_counter() - t0
            if el >= seconds or steps >= 200:
                return nodes * steps / el / 1e6, steps, el

    out = {}
    dims, state = W.taylor_green(n=32, u0=0.05, tau=0.6)
    s = oracle.OracleSim(dims, 0.6)
    s.init_moments(*state)
    v, n, el = timed(s, 32 ** 3)
    out["taylor_green_32"] = {"value": v, "unit": "MLUPS", "sample": "32^3, %d steps, %.1f s" % (n, el)}
    prm = W.jet_params(nz=10)
    s = oracle.OracleSim(prm["dims"], prm["tau"], bc=prm["bc"], inflow=prm["inflow"])
    s.init_moments(*W.rest_state(prm["dims"]))
    v, n, el = timed(s, 254 * 254 * 8)
    out["jet_slab"] = {"value": v, "unit": "MLUPS",
                       "sample": "256x256x10 slab of the jet (inflow, outflow, free-slip), %d steps, %.1f s" % (n, el)}
    return out


def cpu_single_core(prm, seconds):
    """The same oracle timing on one host core: a child process with
    OMP_NUM_THREADS=1 (a separate process, so the thread count is set before the
    OpenMP runtime starts), on a 3-plane slab."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline(%r, %r, nz_sample=3)))" % (ROOT, {"dims": prm["dims"]}, seconds))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=max(120, 10 * seconds))
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": d["unit"], "cores": 1, "sample": d["sample"]}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2401_17074_b300 import workloads as W
    nx, ny = args.nx, args.ny
    # Calibrate: one oracle step on a 3-layer slab, then size the per-step sample so
    # the whole warm-up + timed run stays within about two minutes.
    budget = 120.0
    nzs = 3
    probe = W.channel_params(nx=nx, ny=ny, nz=nzs)
    s = oracle.OracleSim(probe["dims"], probe["tau"], force=probe["force"], bc=probe["bc"])
    s.init_moments(*W.channel_state(probe, seed=1))
    t0 = time.perf_counter()
    s.step(1)
    rate = nx * (ny - 2) * nzs / (time.perf_counter() - t0)  # node updates / s
    per_step = budget / max(1, args.steps + args.warmup)
    sx = int(max(3, min(nx, per_step * rate / ((ny - 2) * nzs))))
    sub = W.channel_params(nx=sx, ny=ny, nz=nzs)
    s = oracle.OracleSim(sub["dims"], sub["tau"], force=sub["force"], bc=sub["bc"])
    s.init_moments(*W.channel_state(sub, seed=1))
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    el = time.perf_counter() - t0
    nodes = sx * (ny - 2) * nzs
    v = nodes * args.steps / el / 1e6
    cores = min(oracle.threads(), nzs * (ny - 2))
    sample = "%dx%dx%d sub-box of the channel (periodic x, z), FP64 populations, %d steps" % (sx, ny, nzs, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "turbulent channel %dx%dx%d (bounded sample per step)" % (nx, ny, args.nz),
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": host_cpu(), "host_cpus": os.cpu_count()},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(ms, dist, device="cuda"):
    """The slowest rank's timed region (every rank receives it); ms unchanged on one process."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank, world_size, steps, ms):
    """Whole-job throughput: node updates of all replicas over the slowest rank's time."""
    return nodes_per_rank * world_size * steps / (ms * 1e-3) / 1e6


def time_device(T, torch, prm, state, precision, kernel, steps, warmup, stream, dist, clocks=None, keep=False,
                rounding="nearest"):
    from paper_2401_17074_b300 import workloads as W
    s = T.Solver(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], precision=PREC_CODE[precision],
                 kernel=kernel, stream=stream.cuda_stream, u_ref=0.05, pi_ref=W.pi_reference(state),
                 rounding=rounding)
    s.init_moments(*state)
    s.step(warmup)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    if clocks:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ck = clocks.stop() if clocks else None
    if dist is not None:
        ms = max_over_ranks(ms, dist)
        dist.barrier()
    d, code = s.diagnostics()
    nodes = s.interior_nodes()
    final = s.get_moments() if keep else None
    s.close()
    return ms, nodes, d, code, ck, final


def precision_errors(prm, ref, got):
    """Relative L2 errors of a 16-bit run against the FP32 run: mean u_x(y) profile and u field."""
    nx, ny, nz = prm["dims"]
    prof = lambda u: u[0].reshape(nz, ny, nx)[:, 1:ny - 1, :].mean(axis=(0, 2))
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"mean_ux_profile": rel(prof(got[1]), prof(ref[1])), "u_field": rel(got[1], ref[1]),
            "pi_field": rel(got[2], ref[2])}


def precision_study(T, torch, stream, prm, state, warm=1000, window=5000, every=250):
    """The 16-bit storage study on the full channel: FP32, BF16 and FP16 runs from
    the same initial state; the mean velocity U(y) and the Reynolds stresses
    averaged over x, z and the samples of the last `window` of warm + window
    steps, each 16-bit run compared with the FP32 run."""
    from paper_2401_17074_b300 import workloads as W
    from paper_2401_17074_b300.channel_stats import ChannelStats, profile_errors
    dims = prm["dims"]
    u = torch.empty((3, dims[0] * dims[1] * dims[2]), dtype=torch.float64, device="cuda")
    runs = {}
    for run in ("fp32", "bf16", "fp16", "bf16_sr", "fp16_sr"):
        prec = run.split("_")[0]
        s = T.Solver(dims, prm["tau"], force=prm["force"], bc=prm["bc"], precision=PREC_CODE[prec],
                     stream=stream.cuda_stream, u_ref=0.05, pi_ref=W.pi_reference(state),
                     rounding="stochastic" if run.endswith("_sr") else "nearest", rounding_seed=1)
        s.init_moments(*state)
        s.step(warm)
        st = ChannelStats(dims)
        for k in range(window // every + 1):
            if k:
                s.step(every)
            T.tslb_get_moments(s.handle, None, u, None, T.DEVICE)
            st.add(u)
        _, code = s.diagnostics()
        s.close()
        runs[run] = (st.result(), code)
    del u
    torch.cuda.empty_cache()
    ref = runs["fp32"][0]
    out = {"workload": "channel %dx%dx%d from the bench's initial state, steps %d..%d, %d samples every %d steps"
                       % (dims + (warm, warm + window, window // every + 1, every)),
           "fp32_scale": {"U_max": float(ref["U"].max()), "uu_max": float(ref["uu"].max()),
                          "vv_max": float(ref["vv"].max()), "ww_max": float(ref["ww"].max()),
                          "uv_absmax": float(np.abs(ref["uv"]).max())},
           "status": {k: v[1] for k, v in runs.items()}}
    for run in ("bf16", "fp16", "bf16_sr", "fp16_sr"):
        out[run + "_vs_fp32"] = profile_errors(runs[run][0], ref)
    out["note"] = ("_sr: stochastic rounding of the stored rho - 1 and u; without it the per-step body-force "
                   "increment (%.3g) is below half a 16-bit spacing of u and is lost.  From the laminar start the "
                   "flow is still laminar in this window: the fluctuations are the decaying seeded noise (stress "
                   "scales in fp32_scale), so the stress errors compare noise, and U carries the result.  The "
                   "study on developed turbulence is bench.py --only precision-study" % prm["force"][0])
    return out


def turbulent_precision_study(T, torch, warm=300000, window=100000, every=1000, check=10000):
    """The 16-bit storage study on developed turbulence: the full channel from a disturbed state
    (workloads.channel_transition_state) run in FP32 for `warm` steps, its
    bulk velocity, wall shear and maximum speed recorded every `check` steps;
    then, from that state, runs of `window` steps in FP32, in FP32 from the
    same state with a 1e-3 relative perturbation of u (a trajectory that
    decorrelates within a few eddy times: the sampling noise of the
    statistics), and in BF16 / FP16 with rounding to nearest and with
    stochastic rounding.  Each run samples u every `every` steps and averages
    U(y) and the Reynolds stresses over x, z and the samples; each is compared
    with the FP32 run."""
    from paper_2401_17074_b300 import workloads as W
    from paper_2401_17074_b300.channel_stats import ChannelStats, profile_errors
    prm = W.channel_params()
    dims, tau = prm["dims"], prm["tau"]
    nx, ny, nz = dims
    N = nx * ny * nz
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    s = T.Solver(dims, tau, force=prm["force"], bc=prm["bc"], stream=stream.cuda_stream)
    s.init_moments(*W.channel_transition_state(prm, seed=2))
    history = []
    t = 0
    code = T.TSLB_OK
    while t < warm:
        s.step(check)
        t += check
        d, code = s.diagnostics()
        history.append({"step": t, "bulk_u": d["momentum"][0] / d["mass"], "wall_shear": d["wall_shear"],
                        "max_speed": d["max_speed"], "status": code})
        if code != T.TSLB_OK:
            break
    branch = s.get_moments()
    s.close()
    out = {"workload": "turbulent channel %dx%dx%d from a disturbed state, FP32 for %d steps, then runs of %d steps "
                       "sampled every %d" % (nx, ny, nz, warm, window, every),
           "u_tau": prm["u_tau"], "u_tau_sq": prm["u_tau"] ** 2, "history": history}
    if code != T.TSLB_OK:
        out["error"] = "the FP32 run became unstable"
        return out
    u_dev = torch.empty((3, N), dtype=torch.float64, device="cuda")
    pi_ref = W.pi_reference(branch)
    runs = {}
    for run in ("fp32", "fp32_perturbed", "bf16", "fp16", "bf16_sr", "fp16_sr"):
        prec = run.split("_")[0]
        s = T.Solver(dims, tau, force=prm["force"], bc=prm["bc"], precision=PREC_CODE[prec], stream=stream.cuda_stream,
                     u_ref=0.05, pi_ref=pi_ref, rounding="stochastic" if run.endswith("_sr") else "nearest",
                     rounding_seed=1)
        rho, u, pi = branch
        if run == "fp32_perturbed":
            u = u * (1.0 + 1e-3 * np.random.default_rng(9).uniform(-1.0, 1.0, u.shape))
        s.init_moments(rho, u, pi)
        st = ChannelStats(dims)
        for k in range(window // every):
            s.step(every)
            T.tslb_get_moments(s.handle, None, u_dev, None, T.DEVICE)
            st.add(u_dev)
        d, c = s.diagnostics()
        s.close()
        runs[run] = (st.result(), c, d["momentum"][0] / d["mass"])
    del u_dev
    torch.cuda.empty_cache()
    ref = runs["fp32"][0]
    yv = np.arange(1, ny - 1, dtype=np.float64)
    nu = (tau - 0.5) / 3.0
    # total shear stress of a stationary channel: -<u'v'> + nu dU/dy = u_tau^2 (y_c - y)/H
    dU = np.gradient(ref["U"], yv)
    total = -ref["uv"] + nu * dU
    yc, H = 0.5 * (ny - 1), prm["H"]
    linear = prm["u_tau"] ** 2 * (yc - yv) / H
    out.update({
        "fp32": {"U_max": float(ref["U"].max()), "uu_max": float(ref["uu"].max()), "vv_max": float(ref["vv"].max()),
                 "ww_max": float(ref["ww"].max()), "uv_absmax": float(np.abs(ref["uv"]).max()),
                 "bulk_u_end": runs["fp32"][2],
                 "total_stress_vs_linear_rel_l2": float(np.linalg.norm(total - linear) / np.linalg.norm(linear)),
                 "profiles": {k: [float(v) for v in ref[k]] for k in ("U", "uu", "vv", "ww", "uv")}},
        "status": {k: v[1] for k, v in runs.items()},
        "bulk_u_end": {k: v[2] for k, v in runs.items()},
        "seconds": time.perf_counter() - t0})
    for run in ("fp32_perturbed", "bf16", "fp16", "bf16_sr", "fp16_sr"):
        out[run + "_vs_fp32"] = profile_errors(runs[run][0], ref)
    return out


def time_jet(T, torch, stream, precision="fp32", steps=200, warmup=20):
    """The round jet of the benchmark set-up (256 x 256 x 640: NEE inflow with a
    D = 20 nozzle and 1 % uniform noise, zero-gradient outflow, free-slip sides),
    from rest, built on the device; the default kernel."""
    from paper_2401_17074_b300 import workloads as W
    prm = W.jet_params()
    dims = prm["dims"]
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, prm["tau"], force=prm["force"], bc=prm["bc"], inflow=prm["inflow"],
                 precision=PREC_CODE[precision], u_ref=0.05, pi_ref=1e-3, stream=stream.cuda_stream)
    rho = torch.ones(N, dtype=torch.float64, device="cuda")
    zeros = torch.zeros((9, N), dtype=torch.float64, device="cuda")
    s.init_moments(rho, zeros[0:3], zeros[3:9])
    del rho, zeros
    s.step(warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    d, code = s.diagnostics()
    nodes = s.interior_nodes()
    s.close()
    torch.cuda.empty_cache()
    return {"workload": "round jet %dx%dx%d: NEE inflow (D = 20, 1 %% uniform noise), outflow, free-slip sides; "
                        "%s storage" % (dims + (precision,)),
            "value": job_mlups(nodes, 1, steps, ms), "unit": "MLUPS", "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "interior_nodes": nodes, "max_speed": d["max_speed"], "status": code}


def time_jet_paper(T, torch, stream, steps=200, warmup=20):
    """The paper's jet set-up at its own size (440 x 440 x 600, periodic crossflow,
    Gaussian inflow noise, sponge layer), from the paper's initial state (fluid at
    rest), built on the device; FP32 storage, the default kernel."""
    from paper_2401_17074_b300 import workloads as W
    prm = W.jet_paper_params()
    dims = prm["dims"]
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, prm["tau"], force=prm["force"], bc=prm["bc"], inflow=prm["inflow"], sponge=prm["sponge"],
                 stream=stream.cuda_stream)
    rho = torch.ones(N, dtype=torch.float64, device="cuda")
    zeros = torch.zeros((9, N), dtype=torch.float64, device="cuda")
    s.init_moments(rho, zeros[0:3], zeros[3:9])
    del rho, zeros
    s.step(warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    d, code = s.diagnostics()
    nodes = s.interior_nodes()
    s.close()
    torch.cuda.empty_cache()
    return {"workload": "round jet %dx%dx%d (paper set-up): periodic x,y, NEE inflow with Gaussian noise, "
                        "outflow, sponge width %d K=%g; fp32 storage" % (dims + prm["sponge"]),
            "value": job_mlups(nodes, 1, steps, ms), "unit": "MLUPS", "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "interior_nodes": nodes, "max_speed": d["max_speed"], "status": code}


def time_channel2d(T, torch, stream, hbm, steps=500, warmup=20):
    """The D2Q9 variant on its channel (8192 x 2050, bounce-back walls, 16.78 M
    interior nodes); FP32 storage, 48 algorithmic bytes per node."""
    from paper_2401_17074_b300 import workloads as W
    prm = W.channel2d_params()
    state = W.channel2d_state(prm, seed=1)
    s = T.Solver(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], lattice=T.TSLB_D2Q9,
                 stream=stream.cuda_stream)
    s.init_moments(*state)
    s.step(warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    d, code = s.diagnostics()
    nodes = s.interior_nodes()
    s.close()
    achieved = 48.0 * nodes / (ms * 1e-3 / steps) / 1e9
    return {"workload": "D2Q9 channel %dx%d, bounce-back walls y=0,%d, tau=%.3f; fp32 storage"
                        % (prm["dims"][0], prm["dims"][1], prm["dims"][1] - 1, prm["tau"]),
            "value": job_mlups(nodes, 1, steps, ms), "unit": "MLUPS", "steps": steps, "ms_per_step": ms / steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "algorithmic_bytes_per_node": 48, "kernel": "tslb_step2d"},
            "alu": alu_entry("tslb_step2d", nodes, ms * 1e-3 / steps,
                             torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count,
                             NOMINAL_SM_MHZ),
            "status": code}


def time_pressure_driven(T, torch, stream, dims=(1024, 512, 576), steps=50, warmup=5):
    """The paper's performance benchmark, a pressure-driven flow on 3e8 nodes
    (Sec. 4): a periodic box driven by a uniform body force, FP32 storage, the
    state built on the device through the FP32 host interface."""
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, 0.6, force=(1e-7, 0.0, 0.0), stream=stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(1)
    drho = 0.002 * (torch.rand(N, device="cuda", dtype=torch.float32, generator=g) - 0.5)
    u = 0.02 * (torch.rand((3, N), device="cuda", dtype=torch.float32, generator=g) - 0.5)
    pi = torch.zeros((6, N), device="cuda", dtype=torch.float32)
    s.init_moments_f32(drho, u, pi)
    del drho, u, pi
    s.step(warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    _, code = s.diagnostics()
    nodes = s.interior_nodes()
    s.close()
    torch.cuda.empty_cache()
    return {"workload": "pressure-driven periodic flow %dx%dx%d (%.0f M nodes, the paper's benchmark size); fp32 storage"
                        % (dims + (nodes / 1e6,)),
            "value": job_mlups(nodes, 1, steps, ms), "unit": "MLUPS", "steps": steps, "ms_per_step": ms / steps,
            "paper_context": "about 3000 MLUPS on an A100 and 2000 on an RTX 3090 (other hardware)", "status": code}


def time_adjoint(T, torch, stream, n=128, nsteps=64, k=16, tau=0.52):
    """Forward (with checkpoints) and discrete adjoint of the force gradient on an n^3 periodic box."""
    from paper_2401_17074_b300 import workloads as W
    dims, state = W.divfree_random(n=n, u_rms=0.02, kmax=8, tau=tau, seed=5)
    s = T.Solver(dims, tau, checkpoint_every=k, stream=stream.cuda_stream)
    F = torch.zeros(3 * n ** 3, dtype=torch.float32, device="cuda")
    g = torch.empty(3 * n ** 3, dtype=torch.float32, device="cuda")
    s.init_moments(*state)
    s.set_force_field(F)
    s.step(nsteps)
    T.tslb_adjoint_force_gradient(s.handle, nsteps, g, T.DEVICE)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init_moments(*state)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s.step(nsteps)
    s.synchronize()
    t2 = time.perf_counter()
    T.tslb_adjoint_force_gradient(s.handle, nsteps, g, T.DEVICE)
    t3 = time.perf_counter()
    s.close()
    return {"workload": "%d^3 periodic, %d steps, checkpoint every %d" % (n, nsteps, k),
            "forward_ms": (t2 - t1) * 1e3, "adjoint_ms": (t3 - t2) * 1e3,
            "forward_mlups": n ** 3 * nsteps / (t2 - t1) / 1e6,
            "adjoint_mlups": n ** 3 * nsteps / (t3 - t2) / 1e6,
            "note": "wall clock; the adjoint recomputes each checkpoint segment"}


def time_adjoint_channel(T, torch, stream, prm, state, nsteps=64, k=16):
    """Forward (with checkpoints) and discrete adjoint on the full channel: the
    control is a force field equal to the channel's body force, J = 1/2 sum
    rho |u|^2 after nsteps; bounce-back y walls."""
    dims = prm["dims"]
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, prm["tau"], bc=prm["bc"], checkpoint_every=k, stream=stream.cuda_stream)
    F = torch.zeros((3, N), dtype=torch.float32, device="cuda")
    F[0] = prm["force"][0]
    g = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    s.set_force_field(F)
    s.init_moments(*state)
    s.step(nsteps)
    T.tslb_adjoint_force_gradient(s.handle, nsteps, g, T.DEVICE)  # warm-up: workspace allocation
    torch.cuda.synchronize()
    s.init_moments(*state)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s.step(nsteps)
    s.synchronize()
    t2 = time.perf_counter()
    T.tslb_adjoint_force_gradient(s.handle, nsteps, g, T.DEVICE)
    t3 = time.perf_counter()
    finite = bool(torch.isfinite(g).all().item())
    nodes = s.interior_nodes()
    s.close()
    del F, g
    torch.cuda.empty_cache()
    return {"workload": "turbulent channel %dx%dx%d, bounce-back walls, %d steps, checkpoint every %d"
                        % (tuple(dims) + (nsteps, k)),
            "forward_ms": (t2 - t1) * 1e3, "adjoint_ms": (t3 - t2) * 1e3,
            "adjoint_mlups": nodes * nsteps / (t3 - t2) / 1e6, "gradient_finite": finite,
            "note": "wall clock; the adjoint recomputes each checkpoint segment"}


def time_e2e(T, torch, prm, state, steps, stream, fp32_io=True):
    """End to end through the C ABI: moments in from pinned host memory, K steps,
    moments back to pinned host memory, wall clock.  fp32_io: the FP32 host
    interface (drho = rho - 1, u, Pi as FP32, tslb_init_moments_f32 /
    tslb_get_moments_f32: 40 B per node each way); else the FP64 one (80 B)."""
    rho, u, pi = state
    N = rho.size
    if fp32_io:
        dt, init, get = torch.float32, T.tslb_init_moments_f32, T.tslb_get_moments_f32
        first = (rho - 1.0).astype(np.float32)
        u_in, pi_in = u.astype(np.float32), pi.astype(np.float32)
    else:
        dt, init, get = torch.float64, T.tslb_init_moments, T.tslb_get_moments
        first, u_in, pi_in = rho, u, pi
    h_first = torch.from_numpy(first).pin_memory()
    h_u = torch.from_numpy(u_in.reshape(-1)).pin_memory()
    h_pi = torch.from_numpy(pi_in.reshape(-1)).pin_memory()
    o_first = torch.empty(N, dtype=dt).pin_memory()
    o_u = torch.empty(3 * N, dtype=dt).pin_memory()
    o_pi = torch.empty(6 * N, dtype=dt).pin_memory()
    s = T.Solver(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], stream=stream.cuda_stream)
    # one untimed pass to settle allocator pools
    init(s.handle, h_first, h_u, h_pi)
    s.step(2)
    get(s.handle, o_first, o_u, o_pi, T.HOST)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    init(s.handle, h_first, h_u, h_pi)
    s.step(steps)
    get(s.handle, o_first, o_u, o_pi, T.HOST)
    el = time.perf_counter() - t0
    nodes = s.interior_nodes()
    s.close()
    b = 4 if fp32_io else 8
    return {"value": nodes * steps / el / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": int(b * 10 * N / steps), "d2h_bytes_per_step": int(b * 10 * N / steps),
            "note": "init from pinned host %s moments + %d steps + moments back to pinned host, wall clock"
                    % ("FP32 (tslb_init_moments_f32 / tslb_get_moments_f32)" if fp32_io else "FP64", steps)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    else:
        torch.cuda.set_device(0)
    import paper_2401_17074_b300 as T
    T.load()
    if args.only == "adjoint":
        line = time_adjoint(T, torch, torch.cuda.Stream())
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.only == "precision-study":
        line = turbulent_precision_study(T, torch, warm=args.warm, window=args.window)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.only == "d2q9":
        hbm, hbm_src = measured_peaks()
        line = time_channel2d(T, torch, torch.cuda.Stream(), hbm, steps=args.steps, warmup=args.warmup)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    kernel = {"auto": T.KERNEL_AUTO, "direct": T.KERNEL_DIRECT, "factored": T.KERNEL_FACTORED}[args.kernel]
    prm, state = make_state(args.nx, args.ny, args.nz)
    stream = torch.cuda.Stream()
    hbm, hbm_src = measured_peaks()

    clocks = ClockSampler(local) if rank == 0 else None
    ms, nodes, diag, code, ck, ref_final = time_device(T, torch, prm, state, args.precision, kernel, args.steps,
                                                       args.warmup, stream, dist, clocks,
                                                       keep=not args.no_variants and rank == 0)
    value = job_mlups(nodes, ws, args.steps, ms)
    launch_s = ms * 1e-3 / args.steps
    bpn = BYTES_PER_NODE[args.precision]
    achieved = bpn * nodes / launch_s / 1e9
    from paper_2401_17074_b300 import build as B
    kname = "tslb_step_direct" if kernel == T.KERNEL_DIRECT else "tslb_step_factored"
    traffic = traffic_record(kname, args.precision)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu = alu_entry(kname, nodes, launch_s, sms, NOMINAL_SM_MHZ) if args.precision == "fp32" else None

    variants = {}
    if not args.no_variants:
        for prec in ("bf16", "fp16"):
            if prec == args.precision:
                continue
            msv, nv, dv, cv, _, fin = time_device(T, torch, prm, state, prec, kernel, args.steps, args.warmup,
                                                  stream, dist, keep=ref_final is not None)
            ls = msv * 1e-3 / args.steps
            variants[prec] = {"value": job_mlups(nv, ws, args.steps, msv), "unit": "MLUPS",
                              "roofline_frac": BYTES_PER_NODE[prec] * nv / ls / 1e9 / hbm,
                              "bytes_per_node": BYTES_PER_NODE[prec], "stable": cv == T.TSLB_OK}
            if fin is not None:
                variants[prec]["error_vs_fp32_after_%d_steps" % (args.steps + args.warmup)] = \
                    precision_errors(prm, ref_final, fin)
        msv, nv, dv, cv, _, _ = time_device(T, torch, prm, state, "bf16", kernel, args.steps, args.warmup, stream,
                                            dist, rounding="stochastic")
        variants["bf16_stochastic_rounding"] = {
            "value": job_mlups(nv, ws, args.steps, msv), "unit": "MLUPS",
            "roofline_frac": BYTES_PER_NODE["bf16"] * nv / (msv * 1e-3 / args.steps) / 1e9 / hbm,
            "bytes_per_node": BYTES_PER_NODE["bf16"], "stable": cv == T.TSLB_OK}
    e2e = e2e64 = None
    if not args.no_e2e and rank == 0:
        e2e = time_e2e(T, torch, prm, state, args.steps, stream, fp32_io=True)
        e2e64 = time_e2e(T, torch, prm, state, args.steps, stream, fp32_io=False)
    adj = None
    if not args.no_adjoint and rank == 0:
        adj = time_adjoint(T, torch, stream)
    extra = None
    if not args.no_extra and rank == 0:
        # the same channel with the paper's thread-safe NEE no-slip walls, and the paper's jet set-up
        prm_nee = dict(prm)
        prm_nee["bc"] = (0, 0, 5, 5, 0, 0)
        k_nee = min(args.steps, 500)
        msn, nn, dn, cn, _, _ = time_device(T, torch, prm_nee, state, args.precision, kernel, k_nee, args.warmup,
                                            stream, None)
        extra = {"channel_nee_walls": {
                     "workload": "turbulent channel %dx%dx%d with thread-safe NEE no-slip walls on y=0,%d "
                                 "(Eq. neq_final, u_B = 0); %s storage" % (args.nx, args.ny, args.nz, args.ny - 1,
                                                                           args.precision),
                     "value": job_mlups(nn, 1, k_nee, msn), "unit": "MLUPS", "steps": k_nee,
                     "ms_per_step": msn / k_nee, "status": cn},
                 "jet": time_jet(T, torch, stream),
                 "jet_bf16": time_jet(T, torch, stream, precision="bf16"),
                 "jet_paper": time_jet_paper(T, torch, stream),
                 "pressure_driven_300M": time_pressure_driven(T, torch, stream),
                 "d2q9_channel": time_channel2d(T, torch, stream, hbm)}
        if not args.no_adjoint:
            extra["adjoint_channel"] = time_adjoint_channel(T, torch, stream, prm, state)
    study = None
    if not args.no_precision_study and not args.no_variants and rank == 0:
        study = precision_study(T, torch, stream, prm, state)
    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        cpu = cpu_baseline(prm, args.cpu_seconds)
        cpu["single_core"] = cpu_single_core(prm, min(5.0, args.cpu_seconds))
        cpu["other_configs"] = cpu_other_configs(min(3.0, args.cpu_seconds))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded laminar parabola + 2% noise)",
            "config": {"workload": "turbulent channel %dx%dx%d, bounce-back walls y=0,%d, periodic x,z, tau=0.503, "
                                   "g=%.4g; %s moment storage" % (args.nx, args.ny, args.nz, args.ny - 1,
                                                                  prm["force"][0], args.precision),
                       "interior_nodes": nodes, "storage": args.precision,
                       "l2": "inputs larger than L2: two %.0f MB moment buffers" % (bpn / 2 * nodes / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single GPU", "kernel": kname,
                       "paper_form": "MLUPS = nx ny nz steps / (1e6 T) over interior nodes: %d x %d x %d x %d / "
                                     "(1e6 x %.4f s)" % (args.nx, prm["dims"][1] - 2, args.nz, args.steps,
                                                          ms * 1e-3)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic, "peak_source": hbm_src,
                         "algorithmic_bytes_per_node": bpn, "kernel": kname},
            "alu": alu,
            "variants": variants,
            "precision_study": study,
            "e2e": e2e,
            "e2e_fp64_io": e2e64,
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "adjoint": adj,
            "workloads": extra,
            "clocks": ck,
            "diagnostics_after_timed": {"mass": diag["mass"], "max_speed": diag["max_speed"], "status": code},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
