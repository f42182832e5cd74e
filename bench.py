#!/usr/bin/env python
"""Throughput of the THOR HE-VI dynamical core on GB300.

One step = one large step of the Held-Suarez workload (glevel 6, 40962
columns x 32 levels, dt = 600 s, 8 small steps: 13 small steps per large
step), i.e. three RK3 slow-term evaluations with hyperdiffusion, 13 acoustic
small steps (divergence damping, explicit horizontal momentum, tridiagonal
vertical solve, density, rho theta, pressure) and the Held-Suarez physics.

Metric: cell-substeps/s = columns x levels x small steps / wall time, plus
model days per hour. Default precision: mixed (float32 fields and stencils,
float64 vertical solve); a float64 leg is reported beside it.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank advances its own replica (the path needs no
exchange between replicas; scaling "weak"); rank 0 prints one JSON line.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

# the oracle legs time plain single-threaded numpy per process (their "cores"
# is the number of processes); set before numpy loads its BLAS
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wls  # noqa: E402

METRIC = "cell-substeps/s"

# The counting rule of the algorithmic roofline: unique field words a cell
# must read or write per pass that the method requires, times the word size
# (4 B in mixed precision); on-chip intermediates are not counted. Per large
# step at n small steps that is 3 x 13 (slow terms) + S_n x 27 (small steps)
# + 9 (physics) words, 399 at n = 8. The 27 words of a small step: the
# perturbations M* (3), W*, rho*, Theta, p* read and written (14), the slow
# tendencies S_M (3), S_W, S_rho, S_Theta (6) and the stage coefficients
# theta, Pi, M^(s) (3), W^(s), p (7).
SLOW_WORDS, SMALL_WORDS, PHYSICS_WORDS = 13, 27, 9


def step_method_words(n_small):
    return 3 * SLOW_WORDS + (1 + n_small // 2 + n_small) * SMALL_WORDS + PHYSICS_WORDS


# Per kernel: the method's words it reads or writes (those of the counting
# rule above that the kernel's part of the step consumes or produces,
# directly or through the kernel split's intermediates), and the words it
# actually moves, the split's intermediates included. The column solve's 15
# method words: W*, rho*, Theta and p* read and written (8; rho*, Theta, p*
# read through the flux kernel's a, b, c), S_W, S_rho, S_Theta (3; the
# latter two through a and b), theta at the interfaces, Pi, W^(s) and p (4).
# It moves 21: W*, S_W, a, b, c, theta_iface, p', Th^(s), D^(s), div_h M*
# read (10), the three float64 factor planes (6 words) and rho*, Theta, p*,
# W*, D written (5). The interface kernel also sets the stage's
# perturbations, and the last small step of a stage also ends it; the
# counts below are those of the other small steps.
KERNEL_WORDS = {        # name: (method words, moved words)
    "derived": (7, 16), "lap1": (6, 14), "slow": (13, 25), "slow_w": (4, 9),
    "ss_lapd": (1, 4), "ss_mom": (10, 13), "ss_flux": (10, 14), "ss_solve": (15, 21),
    "ss_factor": (2, 8), "physics": (9, 9), "stage_init": (7, 20),
}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def solve_source_sha1():
    """SHA-1 of the source the staged column solve compiles from: its section
    of csrc/thor_step.cu (from its banner to the ensemble kernels' banner),
    the stage-end helper it calls, and csrc/thor_kernels.cuh."""
    import hashlib
    d = os.path.join(ROOT, "paper_1607_05535_gb300", "csrc")
    src = open(os.path.join(d, "thor_step.cu")).read()
    a = src.index("// " + "-" * 64 + " staged column solve")
    b = src.index("// " + "-" * 64 + " kernels: ensemble")
    c0 = src.index("__device__ __forceinline__ void stage_end_cell")
    c1 = src.index("\n}\n", c0)
    text = src[a:b] + src[c0:c1] + open(os.path.join(d, "thor_kernels.cuh")).read()
    return hashlib.sha1(text.encode()).hexdigest()


def _traffic(kernel):
    """ncu DRAM bytes per launch of ``kernel`` from the committed profile, or
    None if that profile was taken of another version of the kernel source."""
    try:
        kv = dict(l.split(None, 1) for l in open(os.path.join(ROOT, "profiles", "traffic_hs_g6_L32_mixed.txt"))
                  if l.strip() and not l.startswith("#"))
        if kv["kernel"].strip() == kernel and kv["solve_source_sha1"].strip() == solve_source_sha1():
            return float(kv["bytes_per_launch"])
    except Exception:
        pass
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def workload_of(name):
    return {"hs_g6": wls.HS_G6.with_(spring_max_iter=100000, spring_tol=1e-5),
            "hs_g4": wls.HS_G4, "hj_g6": wls.HJ_G6}[name]


# ------------------------------------------------------------------ oracle

def oracle_sample(wl, n_small_steps=1):
    """Time the oracle on a bounded sample of the workload: one slow-term
    evaluation, ``n_small_steps`` small steps and one physics call, then
    scale to a large step (3 slow evaluations + S_n small steps + physics)."""
    from oracle import dycore as dc
    from oracle import operators as op
    from oracle import physics as ph
    from oracle.grid import build_grid
    P = wl.planet
    G = build_grid(wl.glevel, max_iter=10, tol=0.0)
    pl = dc.Planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref,
                   dc.diffusion_parameter(P.dt_paper, P.tau_d))
    m = dc.Model(G, op.VerticalGrid(wl.nv, wl.z_top, P.radius), pl, forcing=wl.forcing,
                 hj_dT=wl.hj_dT)
    u = wls.temperature_noise(wl, G.ncol)
    X = dc.initial_state(m, wl.T0, wl.p_surf, wl.noise_amp, u)
    Kd = m.Kd(wl.dt)
    t0 = time.perf_counter()
    co = dc.slow_terms(m, X, Kd)
    t_slow = time.perf_counter() - t0
    pert = dict(rho=np.zeros_like(X.rho), M=np.zeros_like(X.M), W=np.zeros_like(X.W),
                Th=X.Th.copy(), p=np.zeros_like(X.rho))
    t0 = time.perf_counter()
    for _ in range(n_small_steps):
        pert = dc.small_step(m, X, co, pert, wl.dt / wl.n_small, Kd)
    t_small = (time.perf_counter() - t0) / n_small_steps
    t0 = time.perf_counter()
    ph.apply_physics(m, X, wl.dt)
    t_phys = time.perf_counter() - t0
    return m, X, co, t_slow, t_small, t_phys


def _oracle_sample_times(name):
    """Worker of the oracle legs (a spawned process): the timed sample of
    oracle_sample for workload ``name``, as (slow, small, physics) seconds."""
    _, _, _, t_slow, t_small, t_phys = oracle_sample(workload_of(name))
    return t_slow, t_small, t_phys


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1048576.0
    except Exception:
        pass
    return 0.0


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def oracle_rates(wl, processes):
    """The oracle as it stands, timed on ``processes`` host processes at
    once (spawned, one thread each), every process running the bounded
    sample of oracle_sample on its own copy of the workload. Returns the
    whole host's cell-substeps/s (the sum over the processes) and the
    samples' times."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")          # never fork a process that holds a CUDA context
    with ctx.Pool(processes) as pool:
        times = pool.map(_oracle_sample_times, [args_name(wl)] * processes)
    sn = wl.substeps_per_large
    rate = sum(wl.cells * sn / (3 * a + sn * b + c) for a, b, c in times)
    return rate, times


def args_name(wl):
    for k in ("hs_g6", "hs_g4", "hj_g6"):
        if workload_of(k).name == wl.name:
            return k
    raise KeyError(wl.name)


def run_reference(args):
    """The oracle as it stands on the host cores (rank 0 only)."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    wl = workload_of(args.workload)
    from oracle import dycore as dc
    m, X, co, t_slow, t_small, t_phys = oracle_sample(wl)
    Kd = m.Kd(wl.dt)
    pert = dict(rho=np.zeros_like(X.rho), M=np.zeros_like(X.M), W=np.zeros_like(X.W),
                Th=X.Th.copy(), p=np.zeros_like(X.rho))
    dtau = wl.dt / wl.n_small
    for _ in range(args.warmup):
        pert = dc.small_step(m, X, co, pert, dtau, Kd)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pert = dc.small_step(m, X, co, pert, dtau, Kd)
    t = time.perf_counter() - t0
    sn = wl.substeps_per_large
    per_large = sn * t / args.steps + 3 * t_slow + t_phys
    value = wl.cells * sn / per_large
    sample = (f"each step = one oracle small step of {wl.name} ({wl.cells} cells); the value "
              f"scales it to a large step with the measured slow-term ({t_slow:.2f} s) and "
              f"physics ({t_phys:.2f} s) costs: 3 slow + {sn} small + physics")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(wl),
            "precision": "float64 (numpy), one thread",
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "host_cpus": os.cpu_count(), "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(wl):
    """The workload (the same for both arms; the precision is in dtype and
    precision)."""
    return {"workload": wl.name, "glevel": wl.glevel, "ncol": wl.ncol, "nv": wl.nv,
            "dt_s": wl.dt, "n_small": wl.n_small, "substeps_per_large_step": wl.substeps_per_large,
            "forcing": wl.forcing,
            "l2": "inputs larger than L2: state + stage work set at g6x32 exceed 129 MB"}


# ------------------------------------------------------------------ ranks

class Ranks:
    """The replicas of a multi-GPU run (one process per GPU under torchrun,
    RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* from the environment): every
    rank steps its own atmosphere (the path needs no exchange between
    replicas), and only the timing is combined: a barrier on both sides of
    a timed region and the maximum of the ranks' times. NCCL with CUDA,
    gloo without."""

    def __init__(self):
        import torch
        self.world = _env_int("WORLD_SIZE", 1)
        self.rank = _env_int("RANK", 0)
        self.local = _env_int("LOCAL_RANK", 0)
        self.dist = None
        self.cuda = torch.cuda.is_available()
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl" if self.cuda else "gloo")
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        """The largest x over the ranks (a float on every rank)."""
        if self.dist is None:
            return float(x)
        import torch
        dev = torch.device("cuda", self.local) if self.cuda else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(world, units_per_rank, seconds):
    """Units of all ranks per second of the slowest rank (weak scaling: every
    rank processes the same units)."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ GPU arm

def _lonlat_basis(points):
    """East and north unit vectors at unit positions (N, 3); zero at the
    poles, where they are undefined."""
    x, y, z = points[:, 0], points[:, 1], points[:, 2]
    rxy = np.hypot(x, y)
    ok = rxy > 1e-12
    east = np.zeros_like(points)
    north = np.zeros_like(points)
    east[ok] = np.stack([-y[ok] / rxy[ok], x[ok] / rxy[ok], np.zeros(ok.sum())], 1)
    north[ok] = np.stack([-z[ok] * x[ok] / rxy[ok], -z[ok] * y[ok] / rxy[ok], rxy[ok]], 1)
    return east, north


def physical_fields(thor, state, ncol, nv, east, north):
    """u, v (eastward, northward wind), w (vertical wind at the centres, the
    mean of the two interfaces), T and rho of a state, each (ncol, nv)."""
    rho = thor.thor_state_get(state, thor.THOR_FIELD_RHO, ncol, nv)
    M = thor.thor_state_get(state, thor.THOR_FIELD_MOM, ncol, nv)
    W = thor.thor_state_get(state, thor.THOR_FIELD_W, ncol, nv)
    T = thor.thor_state_get(state, thor.THOR_FIELD_TEMPERATURE, ncol, nv)
    v3 = M / rho[..., None]
    return {"u": np.einsum("ckj,cj->ck", v3, east), "v": np.einsum("ckj,cj->ck", v3, north),
            "w": 0.5 * (W[:, :-1] + W[:, 1:]) / rho, "T": T, "rho": rho}


def field_error_row(a, b):
    """Per field of the mixed run a against the float64 run b: relative L2
    and the largest absolute difference (m/s for the winds, K, kg/m^3)."""
    out = {}
    for k in ("u", "v", "w", "T", "rho"):
        d = a[k] - b[k]
        out[k] = {"rel_l2": float(np.linalg.norm(d) / max(np.linalg.norm(b[k]), 1e-300)),
                  "max_abs": float(np.max(np.abs(d)))}
    return out


def precision_error(thor, make_state, grid, wl, checkpoints, kc, bs, compensated=(False, True)):
    """The mixed path (launch shape kc, bs, graph replay), plain and with the
    compensated state, against the float64 path from the same start, per
    field after each large-step count in ``checkpoints``."""
    east, north = _lonlat_basis(thor.thor_grid_points(grid))
    ref = make_state(thor.THOR_FP64)
    runs = {}
    # the spread of the flow itself: a float64 run whose start differs from
    # the reference's only by the float32 rounding of the mixed start
    tmp = make_state(thor.THOR_MIXED)
    start = thor.thor_state_get_all(tmp, wl.ncol, wl.nv)
    thor.thor_state_destroy(tmp)
    floor = make_state(thor.THOR_FP64)
    thor.thor_state_set_all(floor, *start)
    runs["fp64_rounded_start"] = floor
    for cmp in compensated:
        a = make_state(thor.THOR_MIXED)
        thor.thor_tune(a, thor.THOR_TUNE_KCHUNK, kc)
        thor.thor_tune(a, thor.THOR_TUNE_BLOCK, bs)
        thor.thor_tune(a, thor.THOR_TUNE_COMPENSATED, 1 if cmp else 0)
        runs["compensated" if cmp else "plain"] = a
    rows = {k: {} for k in runs}
    mass = {}
    try:
        done = 0
        m0 = thor.thor_diag(ref)["mass"]
        for n in checkpoints:
            thor.thor_step(ref, n - done, wl.n_small, wl.dt)
            for a in runs.values():
                thor.thor_step(a, n - done, wl.n_small, wl.dt)
            done = n
            fb = physical_fields(thor, ref, wl.ncol, wl.nv, east, north)
            for k, a in runs.items():
                rows[k][str(n)] = field_error_row(physical_fields(thor, a, wl.ncol, wl.nv, east, north), fb)
        mass["fp64"] = abs(thor.thor_diag(ref)["mass"] - m0) / m0
        for k, a in runs.items():
            mass[k] = abs(thor.thor_diag(a)["mass"] - m0) / m0
    finally:
        thor.thor_state_destroy(ref)
        for a in runs.values():
            thor.thor_state_destroy(a)
    out = {"against": "the float64 path from the same start (which matches the float64 oracle to 1e-10)",
           "large_steps": rows.get("compensated", {}), "mass_drift_at_end": mass,
           "fp64_rounded_start_large_steps": rows["fp64_rounded_start"]}
    if "plain" in rows:
        out["plain_float_state_large_steps"] = rows["plain"]
    return out


def fp64_flops(kind):
    """Float64 operations per large step of the float64 path, from the
    committed ncu instruction counts, if they were taken of this source
    (thor_step.cu's SHA-1), else None."""
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_1607_05535_gb300", "csrc", "thor_step.cu")).read()
        kv = dict(l.split(None, 1) for l in open(os.path.join(ROOT, "profiles", "fp64_ops_hs_g6_L32.txt"))
                  if l.strip() and not l.startswith("#"))
        if kv["step_source_sha1"].strip() == hashlib.sha1(src.encode()).hexdigest():
            return float(kv[kind])
    except Exception:
        pass
    return None


def run_thor(args):
    import torch
    import paper_1607_05535_gb300 as thor

    ranks = Ranks()
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    def setup(wl):
        P = wl.planet
        forcing = {"none": 0, "held_suarez": 1, "hot_jupiter": 2}[wl.forcing]
        sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, wl.spring_tol, wl.spring_max_iter)
        grid = thor.thor_grid_create(wl.glevel, wl.nv, P.radius, wl.z_top, sp)
        planet = thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)

        def make_state(prec):
            init = thor.thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, forcing, wl.hj_dT, prec, 1, 1)
            return thor.thor_state_init(grid, planet, init, stream.cuda_stream)
        return grid, make_state

    def timed(state, wl, steps):
        """CUDA-event time (ms) of ``steps`` large steps on the state's stream."""
        barrier()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            thor.thor_step(state, 1, wl.n_small, wl.dt)
        b.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return a.elapsed_time(b)

    wl = workload_of(args.workload)
    grid, make_state = setup(wl)
    sn = wl.substeps_per_large
    cells = wl.cells
    peak, peak_kind = _peaks()

    # ---- mixed precision, the headline
    st = make_state(thor.THOR_MIXED)
    # clocks sampled over the whole GPU leg (autotuning, warm-up, timed steps,
    # profiled pass, end to end, float64 leg, ensemble, hot Jupiter, errors)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    # launch shape from the autotuner (state restored afterwards), unless given
    if args.kchunk:
        thor.thor_tune(st, thor.THOR_TUNE_KCHUNK, args.kchunk)
        thor.thor_tune(st, thor.THOR_TUNE_BLOCK, args.block)
        tuned_kc, tuned_bs, tuned_ms = args.kchunk, args.block, None
    else:
        tuned_kc, tuned_bs, tuned_ms = thor.thor_autotune(st, wl.n_small, wl.dt, steps=3)
    for _ in range(args.warmup):
        thor.thor_step(st, 1, wl.n_small, wl.dt)          # also captures the CUDA graph
    torch.cuda.synchronize(dev)
    l0 = thor.thor_launch_count(st)
    ms = timed(st, wl, args.steps)                          # graph replays, no per-kernel events
    launches = thor.thor_launch_count(st) - l0
    # per-kernel CUDA-event durations: the same steps launched kernel by kernel
    thor.thor_profile(st, 1)
    timed(st, wl, args.steps)
    prof = {}
    for kid, name in enumerate(thor.KERNELS):
        tot, n = thor.thor_profile_read(st, kid)
        if n:
            prof[name] = (tot, n)
    thor.thor_profile(st, 0)
    ms = max_over_ranks(ms)
    diag = thor.thor_diag(st)
    value = whole_job_rate(world, cells * sn * args.steps, ms / 1e3)
    days_per_hour = world * args.steps * wl.dt / 86400.0 / (ms / 1e3 / 3600.0)

    # dominant kernel and its roofline (method words of the counting rule)
    dom = max(prof, key=lambda k: prof[k][0])
    tot, n = prof[dom]
    nlev = wl.nv + 1 if dom in ("slow_w",) else wl.nv
    mw, moved = KERNEL_WORDS[dom]
    bytes_per_launch = mw * 4 * wl.ncol * nlev
    us = 1e3 * tot / n
    achieved = bytes_per_launch / (us / 1e6) / 1e9
    moved_bytes = moved * 4 * wl.ncol * nlev
    kernels = {}
    for k, v in prof.items():
        lev = wl.nv + 1 if k in ("slow_w",) else wl.nv
        kw = KERNEL_WORDS.get(k, (None, None))
        avg = 1e3 * v[0] / v[1]
        kernels[k] = {"ms_total": round(v[0], 4), "launches": v[1], "us_avg": round(avg, 2),
                      "share": round(v[0] / sum(x[0] for x in prof.values()), 4)}
        if kw[0] is not None:
            kernels[k]["method_words"] = kw[0]
            kernels[k]["moved_words"] = kw[1]
            kernels[k]["frac_method"] = round(kw[0] * 4 * wl.ncol * lev / (avg / 1e6) / 1e9 / peak, 4)
    step_bytes = step_method_words(wl.n_small) * 4 * cells
    whole = {"method_words_per_cell": step_method_words(wl.n_small), "bytes": step_bytes,
             "ms": ms / args.steps, "achieved": step_bytes / (ms / args.steps / 1e3) / 1e9,
             "unit": "GB/s", "peak": peak}
    whole["frac"] = whole["achieved"] / peak

    # ---- the same steps with a plain float32 state (THOR_TUNE_COMPENSATED 0)
    thor.thor_tune(st, thor.THOR_TUNE_COMPENSATED, 0)
    for _ in range(2):
        thor.thor_step(st, 1, wl.n_small, wl.dt)
    ms_plain = max_over_ranks(timed(st, wl, args.steps))
    thor.thor_tune(st, thor.THOR_TUNE_COMPENSATED, 1)
    plain = {"value": whole_job_rate(world, cells * sn * args.steps, ms_plain / 1e3), "unit": METRIC,
             "ms_per_step": ms_plain / args.steps, "steps": args.steps,
             "state": "float32 deviations without the compensating low parts"}

    # ---- end to end through the C ABI with pinned host buffers
    shapes = {thor.THOR_FIELD_RHO: (wl.ncol, wl.nv), thor.THOR_FIELD_MOM: (wl.ncol, wl.nv, 3),
              thor.THOR_FIELD_W: (wl.ncol, wl.nv + 1), thor.THOR_FIELD_RHOTHETA: (wl.ncol, wl.nv)}
    host = {f: torch.empty(s, dtype=torch.float64, pin_memory=True) for f, s in shapes.items()}
    bufs = [host[f] for f in thor.PROGNOSTIC]
    thor.thor_state_get_all(st, wl.ncol, wl.nv, out=bufs)
    e2e_steps = max(1, min(args.steps, 10))
    nbytes = sum(h.numel() * 8 for h in host.values())
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        thor.thor_state_set_all(st, *bufs)
        thor.thor_step(st, 1, wl.n_small, wl.dt)
        thor.thor_state_get_all(st, wl.ncol, wl.nv, out=bufs)
    torch.cuda.synchronize(dev)
    barrier()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    e2e = world * cells * sn * e2e_steps / t_e2e
    thor.thor_state_destroy(st)

    # ---- float64 leg and its bound: min of HBM (8-byte words) and the
    # float64 pipe (the float64 operations of a large step, counted by ncu,
    # at the GB300's nominal 1.25 TFLOP/s; 1.0 TFLOP/s measured)
    st64 = make_state(thor.THOR_FP64)
    for _ in range(min(args.warmup, 2)):
        thor.thor_step(st64, 1, wl.n_small, wl.dt)
    k64 = max(1, min(args.steps, 5))
    ms64 = max_over_ranks(timed(st64, wl, k64))
    thor.thor_state_destroy(st64)
    value64 = world * cells * sn * k64 / (ms64 / 1e3)
    t_hbm64 = 2 * step_bytes / (peak * 1e9)
    flops64 = fp64_flops("fp64_ops_per_large_step") if wl.name == wls.HS_G6.name else None
    fp64 = {"value": value64, "unit": METRIC, "steps": k64, "ms_per_step": ms64 / k64,
            "model_days_per_hour": world * k64 * wl.dt / 86400.0 / (ms64 / 1e3 / 3600.0),
            "bound": {"hbm_ms": 1e3 * t_hbm64, "hbm_frac": t_hbm64 / (ms64 / k64 / 1e3)}}
    inst64 = fp64_flops("fp64_instructions_per_large_step") if flops64 else None
    if flops64 and inst64:
        # each float64 add, multiply or FMA is one issue of the float64 pipe:
        # 0.625 T/s at the nominal 1.25 TFLOP/s
        t_alu = inst64 / 0.625e12
        fp64["bound"].update({"fp64_ops_per_step": flops64, "fp64_instructions_per_step": inst64,
                              "fp64_peak_tflops": 1.25, "fp64_peak_kind": "nominal",
                              "achieved_tflops": flops64 / (ms64 / k64 / 1e3) / 1e12,
                              "fp64_ms": 1e3 * t_alu, "fp64_frac": t_alu / (ms64 / k64 / 1e3),
                              "bound": "fp64" if t_alu > t_hbm64 else "hbm"})

    ens = run_ensemble(thor, torch, dev, stream, args, max_over_ranks) if not args.no_ensemble else None

    # ---- hot Jupiter (config 3), mixed precision in the same launch shape
    hj = None
    if not args.no_hot_jupiter and args.workload != "hj_g6":
        whj = workload_of("hj_g6")
        ghj, mk_hj = setup(whj)
        sh = mk_hj(thor.THOR_MIXED)
        thor.thor_tune(sh, thor.THOR_TUNE_KCHUNK, tuned_kc)
        thor.thor_tune(sh, thor.THOR_TUNE_BLOCK, tuned_bs)
        for _ in range(args.warmup):
            thor.thor_step(sh, 1, whj.n_small, whj.dt)
        khj = max(1, min(args.steps, 20))
        ms_hj = max_over_ranks(timed(sh, whj, khj))
        nf = thor.thor_diag(sh)["nonfinite"]
        thor.thor_state_destroy(sh)
        snj = whj.substeps_per_large
        hj = {"workload": whj.name, "value": world * whj.cells * snj * khj / (ms_hj / 1e3), "unit": METRIC,
              "steps": khj, "ms_per_step": ms_hj / khj, "substeps_per_large_step": snj, "dt_s": whj.dt,
              "model_days_per_hour": world * khj * whj.dt / 86400.0 / (ms_hj / 1e3 / 3600.0),
              "nonfinite": nf, "dtype": "f32"}
        hj_bytes = step_method_words(whj.n_small) * 4 * whj.cells
        hj["whole_step_frac"] = hj_bytes / (ms_hj / khj / 1e3) / 1e9 / peak
        if args.error_steps:
            hj["error"] = precision_error(thor, mk_hj, ghj, whj, args.error_steps, tuned_kc, tuned_bs)
        thor.thor_grid_destroy(ghj)

    # ---- per-field error of the headline number (mixed against float64)
    err = precision_error(thor, make_state, grid, wl, args.error_steps, tuned_kc, tuned_bs) \
        if args.error_steps else None
    thor.thor_grid_destroy(grid)
    clocks = sampler.stop() if sampler else None

    if rank != 0:
        ranks.close()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(wl),
        "precision": ("mixed: f32 stencils and tendencies, the state as compensated f32 pairs, double-float "
                      "vertical factorisation and elimination, f64 reductions"),
        "model_days_per_hour": days_per_hour,
        "error": err,
        "plain_float_state": plain,
        "fp64": fp64,
        "e2e": {"value": e2e, "unit": METRIC, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": e2e_steps},
        "gpu_launches": launches,
        "autotuned": {"kchunk": tuned_kc, "block": tuned_bs, "ms_per_step": tuned_ms},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": _traffic(dom), "algorithmic_bytes_per_launch": bytes_per_launch,
                     "method_words_per_cell": mw, "moved_words_per_cell": moved,
                     "moved_bytes_per_launch": moved_bytes,
                     "frac_moved": moved_bytes / (us / 1e6) / 1e9 / peak, "us_per_launch": us,
                     "whole_step": whole},
        "kernels": kernels,
        "clocks": clocks,
        "diag_after": {k: diag[k] for k in ("mass", "max_vh", "max_w", "mean_T", "nonfinite")},
    }
    if ens is not None:
        line["ensemble"] = ens
    if hj is not None:
        line["hot_jupiter"] = hj
    if world == 1 and not args.no_cpu_baseline:
        ncpu = os.cpu_count() or 1
        one, t1 = oracle_rates(wl, 1)
        # one process of the sample holds about 1.8 GB at glevel 6: keep
        # the leg well inside the memory the host has free
        procs = max(1, min(ncpu, args.cpu_processes, int(_mem_available_gb() // 4.0)))
        allc, tall = oracle_rates(wl, procs) if procs > 1 else (one, t1)
        a, b, c = t1[0]
        line["cpu_baseline"] = {
            "value": allc, "unit": METRIC, "cores": procs, "kind": "oracle",
            "single_core": one, "host_cpus": ncpu, "cpu_model": cpu_model(),
            "sample": (f"{wl.name}: one oracle slow-term evaluation ({a:.1f} s), one small step ({b:.1f} s) and "
                       f"one physics call ({c:.1f} s) per process, scaled to 3 slow + {sn} small + physics per "
                       f"large step; numpy float64, one thread per process; value = {procs} processes at once "
                       "(each its own copy of the workload), single_core = one process alone")}
    print(json.dumps(line), flush=True)
    ranks.close()
    return 0


def run_ensemble(thor, torch, dev, stream, args, max_over_ranks):
    """Batched ensemble: 64 Held-Suarez atmospheres (glevels 3-5 x 32 levels,
    radius and rotation log-uniform over [0.1, 10] x Earth, seeded), mixed
    precision. Launch shape from the autotuner, then K ensemble large steps
    timed with CUDA events; the same members stepped one after another (each
    with its own graph) for comparison."""
    members = wls.ensemble_members()
    sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, 10)
    grids, states = [], []
    for i, m in enumerate(members):
        P = m.planet
        g = thor.thor_grid_create(m.glevel, wls.ENSEMBLE_NV, P.radius, wls.ENSEMBLE_Z_TOP, sp)
        planet = thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
        init = thor.thor_init(300.0, 1.0e5, 0.1, wls.ENSEMBLE_SEED + i, 1, 300.0, thor.THOR_MIXED, 1, 1)
        grids.append(g)
        states.append(thor.thor_state_init(g, planet, init, stream.cuda_stream))
    n_small = [m.n_small for m in members]
    dts = [m.dt for m in members]
    cell_substeps = sum(m.ncol * wls.ENSEMBLE_NV * (1 + n // 2 + n) for m, n in zip(members, n_small))
    ens = thor.thor_ensemble_create(states, stream.cuda_stream)
    kc, bs, ms_tuned = thor.thor_ensemble_autotune(ens, n_small, dts, steps=2)
    for _ in range(args.warmup):
        thor.thor_ensemble_step(ens, 1, n_small, dts)
    torch.cuda.synchronize(dev)
    k = max(1, min(args.steps, 10))
    l0 = thor.thor_ensemble_info(ens)["launches"]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    thor.thor_ensemble_step(ens, k, n_small, dts)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(a.elapsed_time(b))
    launches = thor.thor_ensemble_info(ens)["launches"] - l0
    thor.thor_ensemble_destroy(ens)
    # the same members one after another, each replaying its own graph
    for s_, n_, d_ in zip(states, n_small, dts):
        thor.thor_tune(s_, thor.THOR_TUNE_KCHUNK, kc)
        thor.thor_tune(s_, thor.THOR_TUNE_BLOCK, bs)
        thor.thor_step(s_, 1, n_, d_)
    torch.cuda.synchronize(dev)
    seq_l0 = sum(thor.thor_launch_count(s_) for s_ in states)
    a.record(stream)
    for _ in range(k):
        for s_, n_, d_ in zip(states, n_small, dts):
            thor.thor_step(s_, 1, n_, d_)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = max_over_ranks(a.elapsed_time(b))
    nonfinite = sum(thor.thor_diag(s_)["nonfinite"] for s_ in states)
    seq_launches = sum(thor.thor_launch_count(s_) for s_ in states) - seq_l0
    for s_ in states:
        thor.thor_state_destroy(s_)
    for g in grids:
        thor.thor_grid_destroy(g)
    world = _env_int("WORLD_SIZE", 1)
    return {"workload": "held_suarez_ensemble_64_g3-5_L32", "members": len(members),
            "columns": sum(m.ncol for m in members), "levels": wls.ENSEMBLE_NV,
            "value": world * cell_substeps * k / (ms / 1e3), "unit": METRIC, "steps": k,
            "ms_per_step": ms / k, "gpu_launches": launches, "launches_per_step": launches / k,
            "autotuned": {"kchunk": kc, "block": bs, "ms_per_step": ms_tuned},
            "sequential": {"value": world * cell_substeps * k / (ms_seq / 1e3), "ms_per_step": ms_seq / k,
                           "launches_per_step": seq_launches / k},
            "speedup_vs_sequential": ms_seq / ms, "nonfinite": nonfinite, "dtype": "f32"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="thor", choices=["thor", "reference"])
    ap.add_argument("--workload", default="hs_g6", choices=["hs_g6", "hs_g4", "hj_g6"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--kchunk", type=int, default=0, help="levels per thread (skips the autotuner)")
    ap.add_argument("--block", type=int, default=128, help="block size with --kchunk")
    ap.add_argument("--no-hot-jupiter", action="store_true")
    ap.add_argument("--error-steps", default="10,100,1000",
                    help="large-step counts at which the mixed path is compared with float64 ('' skips)")
    ap.add_argument("--cpu-processes", type=int, default=16, help="processes of the all-cores oracle leg")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)      # at least 3 untimed warm-up steps
    args.error_steps = [int(x) for x in args.error_steps.split(",") if x.strip()]
    if args.impl == "reference":
        return run_reference(args)
    return run_thor(args)


if __name__ == "__main__":
    sys.exit(main())
