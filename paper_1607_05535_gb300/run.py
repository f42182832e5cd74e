"""Command-line runner: a few large steps of a named workload, or of the
64-member ensemble, through the C ABI; prints the diagnostics as JSON.

    python -m paper_1607_05535_gb300.run --workload hs_g6 --precision mixed --steps 3
    python -m paper_1607_05535_gb300.run --ensemble --steps 2
    python -m paper_1607_05535_gb300.run --mlp --steps 3

--mlp runs training steps of the closure-sized MLP (320-256-256-256-160,
batch --mlp-batch, default 1024) on seeded random data, on the GEMM path
--mlp-path; --mlp-timed N adds the mean time of N further training steps
and of N forwards.

Workloads (seeded, synthetic; module ``workloads`` at the repository root):
hs_g4 (Held-Suarez glevel 4 x 20), hs_g6 (glevel 6 x 32), hj_g6 (hot
Jupiter glevel 6 x 32). The grid uses --spring-iters spring-dynamics
iterations (default 10). Runs on the current CUDA device, default stream.
"""

import argparse
import json
import sys


def _workloads():
    import workloads as wls
    return wls, {"hs_g4": wls.HS_G4, "hs_g6": wls.HS_G6, "hj_g6": wls.HJ_G6}


def run_workload(thor, wl, precision, steps, spring_iters, kchunk, solve_tma=1):
    P = wl.planet
    forcing = {"none": 0, "held_suarez": 1, "hot_jupiter": 2}[wl.forcing]
    grid = thor.thor_grid_create(wl.glevel, wl.nv, P.radius, wl.z_top,
                                 thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, spring_iters))
    planet = thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
    init = thor.thor_init(wl.T0, wl.p_surf, wl.noise_amp, wl.seed, forcing, wl.hj_dT, precision, 1, 1)
    st = thor.thor_state_init(grid, planet, init, None)
    try:
        thor.thor_tune(st, thor.THOR_TUNE_KCHUNK, kchunk)
        thor.thor_tune(st, thor.THOR_TUNE_SOLVE_TMA, solve_tma)
        thor.thor_step(st, steps, wl.n_small, wl.dt)
        return {"workload": wl.name, "steps": steps, "diag": thor.thor_diag(st),
                "launches": thor.thor_launch_count(st)}
    finally:
        thor.thor_state_destroy(st)
        thor.thor_grid_destroy(grid)


def run_ensemble(thor, wls, steps, spring_iters):
    members = wls.ensemble_members()
    sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, spring_iters)
    grids, states = [], []
    try:
        for i, m in enumerate(members):
            P = m.planet
            g = thor.thor_grid_create(m.glevel, wls.ENSEMBLE_NV, P.radius, wls.ENSEMBLE_Z_TOP, sp)
            grids.append(g)
            planet = thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
            init = thor.thor_init(300.0, 1.0e5, 0.1, wls.ENSEMBLE_SEED + i, 1, 300.0, thor.THOR_MIXED, 1, 1)
            states.append(thor.thor_state_init(g, planet, init, None))
        ens = thor.thor_ensemble_create(states)
        try:
            thor.thor_ensemble_step(ens, steps, [m.n_small for m in members], [m.dt for m in members])
            info = thor.thor_ensemble_info(ens)
        finally:
            thor.thor_ensemble_destroy(ens)
        diags = [thor.thor_diag(s) for s in states]
        return {"workload": "held_suarez_ensemble_64_g3-5_L32", "steps": steps, "members": len(members),
                "launches": info["launches"], "nonfinite": sum(d["nonfinite"] for d in diags),
                "max_vh": max(d["max_vh"] for d in diags)}
    finally:
        for s in states:
            thor.thor_state_destroy(s)
        for g in grids:
            thor.thor_grid_destroy(g)


def run_mlp(thor, torch, steps, path=1, batch=1024, timed=0):
    """`steps` training steps of the closure-sized network on the default
    stream; with timed > 0, then the mean time of `timed` further training
    steps and of `timed` forwards (CUDA events on that stream)."""
    sizes = [320, 256, 256, 256, 160]
    net = thor.thor_mlp_create(sizes, batch, seed=1)
    try:
        thor.thor_mlp_tune(net, thor.THOR_MLP_TUNE_TCGEN05, path)
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        x = torch.randn(batch, sizes[0], device="cuda", generator=g)
        t = torch.randn(batch, sizes[-1], device="cuda", generator=g)
        y = torch.empty(batch, sizes[-1], device="cuda")
        loss = torch.zeros(1, device="cuda")
        for _ in range(steps):
            thor.thor_mlp_train_step(net, x, t, 1e-3, loss)
        thor.thor_mlp_get_params(net)
        out = {"mlp": sizes, "batch": batch, "path": path, "steps": steps, "loss": float(loss.item())}
        if timed > 0:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            ev[0].record()
            for _ in range(timed):
                thor.thor_mlp_train_step(net, x, t, 1e-3, loss)
            ev[1].record()
            for _ in range(timed):
                thor.thor_mlp_forward(net, x, y)
            ev[2].record()
            torch.cuda.synchronize()
            thor.thor_mlp_get_params(net)
            out["ms_train_step"] = ev[0].elapsed_time(ev[1]) / timed
            out["ms_forward"] = ev[1].elapsed_time(ev[2]) / timed
        return out
    finally:
        thor.thor_mlp_destroy(net)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="hs_g6", choices=["hs_g4", "hs_g6", "hj_g6"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--spring-iters", type=int, default=10)
    ap.add_argument("--kchunk", type=int, default=2)
    ap.add_argument("--solve-tma", type=int, default=1, choices=[0, 1])
    ap.add_argument("--ensemble", action="store_true")
    ap.add_argument("--mlp", action="store_true")
    ap.add_argument("--mlp-path", type=int, default=1, choices=[0, 1, 2],
                    help="GEMM path: 1 TMA-fed tcgen05, 2 thread-staged tcgen05, 0 mma.sync")
    ap.add_argument("--mlp-batch", type=int, default=1024)
    ap.add_argument("--mlp-timed", type=int, default=0)
    args = ap.parse_args(argv)
    import torch
    import paper_1607_05535_gb300 as thor
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    torch.cuda.set_device(0)
    wls, table = _workloads()
    if args.mlp:
        out = run_mlp(thor, torch, args.steps, args.mlp_path, args.mlp_batch, args.mlp_timed)
    elif args.ensemble:
        out = run_ensemble(thor, wls, args.steps, args.spring_iters)
    else:
        prec = thor.THOR_FP64 if args.precision == "fp64" else thor.THOR_MIXED
        out = run_workload(thor, table[args.workload], prec, args.steps, args.spring_iters, args.kchunk,
                           args.solve_tma)
    torch.cuda.synchronize()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
