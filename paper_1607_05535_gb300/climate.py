"""Long runs with zonal and time averages (Sec. 6): the Held-Suarez and
hot-Jupiter climates.

The library steps the state on the GPU and accumulates zonal band means of
the wind, temperature, pressure and eddy covariances on the device
(thor_zonal_accumulate). This module only drives those calls and turns the
accumulated band means (nv x nlat values) into the quantities Sec. 6.1
discusses: the position and speed of the jets, the mass stream function
Psi = (2 pi A cos(lat) / g) * integral from the top of the time- and zonal-mean
northward wind over pressure, and the eddy fluxes [u'v'] and [v'T']; the
same accumulation keeps the time mean [w] of every cell, from which the
grid-imprinting map [w*] = [w] - (zonal band mean of [w]) of Sec. 6.1
follows; zonal means go to pressure levels by linear interpolation in p
(Sec. 6: a post-processing step).

    python -m paper_1607_05535_gb300.climate --days 1200 --spinup 200 --out run.json

Default: the paper's Held-Suarez run (glevel 5, 37 levels to 32 km, dt
1000 s, 6 acoustic small steps, the planet of Table 1), from rest with the
equatorial T_eq in every column in hydrostatic balance (the start of Sec.
6.1; --isothermal starts from 300 K with 0.1 K of seeded noise instead),
mixed precision; --forcing hot_jupiter runs Sec. 6.2's
(37 levels to 4875 km, dt 600 s, isothermal 1600 K at rest without noise,
1 bar at the surface unless --p-surf says otherwise).
"""

import argparse
import json
import math
import sys
import time


def planet(forcing, table1=True):
    """The planet of a run: Table 1 of the paper (the Sec. 6 runs) or the
    benchmark workloads' values (which take c_p, R_d and the hot Jupiter's
    gravity from the benchmark configurations)."""
    import workloads as wls
    if forcing == "hot_jupiter":
        return wls.HOT_JUPITER_TABLE1 if table1 else wls.HOT_JUPITER
    return wls.EARTH_TABLE1 if table1 else wls.EARTH


def run(thor, glevel=5, nv=37, z_top=32.0e3, dt=1000.0, n_small=6, days=1200.0, spinup_days=200.0, nlat=36,
        sample_hours=24.0, forcing="held_suarez", precision="mixed", seed=1234, hj_dT=300.0, stream=None,
        table1=True, shallow=False, hydrostatic=False, extras=None, p_surf=1.0e5, profile=None, noise=0.1):
    """Steps the workload, accumulates one zonal sample every sample_hours
    after the spin-up, and returns (time means (nv, nlat, 9), samples,
    seconds of stepping, final diagnostics). shallow / hydrostatic: the
    approximation switches of Sec. 3. p_surf: the surface pressure of the
    resting start (1 bar for both planets: Sec. 6 gives none; p_ref is
    1 bar, and the hot Jupiter's jet is reported at 800 mbar). profile:
    "held_suarez" starts every column at the equatorial T_eq of Sec. 6.1 in
    hydrostatic balance (the paper's start), None isothermal; noise: the
    amplitude (K) of the seeded temperature noise. If extras is a dict it
    receives the
    time mean of w at every cell ("w_mean", (ncol, nv)), the unit position
    ("points") and the control-volume area ("areas") of every column."""
    P = planet(forcing, table1)
    fid = {"none": 0, "held_suarez": 1, "hot_jupiter": 2}[forcing]
    prec = thor.THOR_FP64 if precision == "fp64" else thor.THOR_MIXED
    grid = thor.thor_grid_create(glevel, nv, P.radius, z_top, thor.thor_spring(1.15, 1.0, 1.0, 0.01, 1e-5, 100000))
    pl = thor.thor_planet(P.radius, P.omega, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
    T0, ps = (300.0 if forcing != "hot_jupiter" else 1600.0), p_surf
    init = thor.thor_init(T0, ps, noise, seed, fid, hj_dT, prec, 1, 1, int(shallow), int(hydrostatic),
                          thor.THOR_PROFILE_HELD_SUAREZ if profile == "held_suarez" else thor.THOR_PROFILE_ISOTHERMAL)
    st = thor.thor_state_init(grid, pl, init, stream)
    try:
        per_sample = max(1, round(sample_hours * 3600.0 / dt))
        spin = round(spinup_days * 86400.0 / dt)
        total = round(days * 86400.0 / dt)
        t0 = time.perf_counter()
        done = 0
        while done < spin:
            n = min(per_sample * 10, spin - done)
            thor.thor_step(st, n, n_small, dt)
            done += n
        while done + per_sample <= total:
            thor.thor_step(st, per_sample, n_small, dt)
            done += per_sample
            thor.thor_zonal_accumulate(st, nlat)
        if extras is not None:
            ncol = thor.thor_grid_info(grid)["ncol"]
            extras["w_mean"] = thor.thor_zonal_read_w(st, nlat, ncol, nv)[0]
            extras["points"] = thor.thor_grid_points(grid)
            extras["areas"] = thor.thor_grid_areas(grid)
        sums, samples = thor.thor_zonal_read(st, nlat, nv)
        seconds = time.perf_counter() - t0
        diag = thor.thor_diag(st)
    finally:
        thor.thor_state_destroy(st)
        thor.thor_grid_destroy(grid)
    means = sums / max(samples, 1)
    return means, samples, seconds, diag


def bands(points, nlat):
    """Latitude band of every column: b = floor((lat + pi/2 + 1e-9) / pi *
    nlat), the north pole in the last band (the rule of the device
    accumulation)."""
    import numpy as np
    lat = np.arcsin(np.clip(points[:, 2], -1.0, 1.0))
    return np.minimum(np.floor((lat + 0.5 * math.pi + 1e-9) / math.pi * nlat).astype(np.int64), nlat - 1)


def w_star(w_mean, points, areas, nlat):
    """The grid-imprinting map of Sec. 6.1: [w*] = [w] minus its zonal band
    mean at every level, (ncol, nv). Within one level every cell's volume is
    its area times the same r^2 dz, so the volume-weighted band mean is the
    area-weighted one."""
    import numpy as np
    b = bands(points, nlat)
    out = np.empty_like(w_mean)
    wsum = np.bincount(b, weights=areas, minlength=nlat)
    for k in range(w_mean.shape[1]):
        m = np.bincount(b, weights=areas * w_mean[:, k], minlength=nlat) / np.where(wsum > 0, wsum, 1.0)
        out[:, k] = w_mean[:, k] - m[b]
    return out


def imprint_summary(ws, w_mean, points, areas, nlat, level=0):
    """Area-weighted RMS of [w*] and [w] at one level, the largest |[w*]|,
    and the share of [w*]'s variance in zonal wavenumber 5 (least squares
    on cos 5 lon, sin 5 lon within every band), the symmetry of the
    icosahedron's imprint."""
    import numpy as np
    a = areas / areas.sum()
    x, w = ws[:, level], w_mean[:, level]
    lon = np.arctan2(points[:, 1], points[:, 0])
    b = bands(points, nlat)
    fit = np.zeros_like(x)
    for j in range(nlat):
        sel = b == j
        if sel.sum() < 3:
            continue
        A = np.stack([np.cos(5 * lon[sel]), np.sin(5 * lon[sel])], axis=1) * np.sqrt(a[sel])[:, None]
        coef = np.linalg.lstsq(A, x[sel] * np.sqrt(a[sel]), rcond=None)[0]
        fit[sel] = coef[0] * np.cos(5 * lon[sel]) + coef[1] * np.sin(5 * lon[sel])
    var = float((a * x * x).sum())
    return {"level": level, "w_star_rms_ms": math.sqrt(var), "w_mean_rms_ms": math.sqrt(float((a * w * w).sum())),
            "w_star_max_ms": float(np.abs(x).max()),
            "w_star_wave5_share": float((a * fit * fit).sum() / var) if var > 0 else 0.0}


def to_pressure_levels(values, p_mean, p_levels):
    """Zonal-mean values on model levels (nv, nlat) to pressure levels
    (len(p_levels), nlat), linear in p between the two model levels whose
    band-mean pressures bracket the target; NaN outside a band's range."""
    import numpy as np
    nv, nlat = values.shape
    out = np.full((len(p_levels), nlat), np.nan)
    for j in range(nlat):
        p = p_mean[:, j]
        order = np.argsort(p)
        ps, vs = p[order], values[order, j]
        for i, pt in enumerate(p_levels):
            if not ps[0] <= pt <= ps[-1]:
                continue
            h = min(int(np.searchsorted(ps, pt, side="right")), nv - 1)
            lo = h - 1 if h > 0 else 0
            if ps[h] == ps[lo]:
                out[i, j] = vs[lo]
            else:
                t = (pt - ps[lo]) / (ps[h] - ps[lo])
                out[i, j] = (1.0 - t) * vs[lo] + t * vs[h]
    return out


def summarize(means, radius, gravity, p_levels=None):
    """The Sec. 6.1 quantities from time-mean band values (nv, nlat, 9)."""
    import numpy as np
    nv, nlat, _ = means.shape
    lat = (np.arange(nlat) + 0.5) * 180.0 / nlat - 90.0
    u, v, T, p = means[..., 1], means[..., 2], means[..., 3], means[..., 4]
    uv, vT = means[..., 5], means[..., 6]
    eke = 0.5 * (means[..., 7] + means[..., 8])
    out = {"lat": lat.tolist()}
    jets = {}
    for name, sel in (("north", lat > 0), ("south", lat < 0)):
        uu = np.where(sel[None, :], u, -np.inf)
        k, b = np.unravel_index(np.argmax(uu), uu.shape)
        jets[name] = {"u_ms": float(u[k, b]), "lat_deg": float(lat[b]), "p_hPa": float(p[k, b] / 100.0),
                      "level": int(k)}
    out["jets"] = jets
    eq = np.argsort(np.abs(lat))[:2]
    out["surface_u_equator_ms"] = float(u[0, eq].mean())
    out["surface_u_poleward_60_ms"] = float(u[0, np.abs(lat) > 60].mean())
    # mass stream function from the top down; the pressure thickness of a
    # level from the mean pressures of its neighbours (one spacing at the
    # lowest and highest level)
    dp = np.zeros_like(p)
    if nv > 1:
        dp[1:-1] = 0.5 * (p[:-2] - p[2:])
        dp[0] = p[0] - p[1]
        dp[-1] = p[-2] - p[-1]
    psi = np.cumsum((v * dp)[::-1], axis=0)[::-1] * (2 * math.pi * radius * np.cos(np.radians(lat))[None, :] /
                                                     gravity)
    out["psi_max_kg_s"] = float(psi.max())
    out["psi_min_kg_s"] = float(psi.min())
    out["psi_max_lat_deg"] = float(lat[np.unravel_index(np.argmax(psi), psi.shape)[1]])
    out["psi_min_lat_deg"] = float(lat[np.unravel_index(np.argmin(psi), psi.shape)[1]])
    mid_n, mid_s = (lat > 20) & (lat < 60), (lat < -20) & (lat > -60)
    out["eddy_uv_north_max"] = float(uv[:, mid_n].max())
    out["eddy_uv_south_min"] = float(uv[:, mid_s].min())
    low = p.mean(axis=1) > 6.0e4                      # levels below about 600 hPa
    out["eddy_vT_north_low_mean"] = float(vT[low][:, mid_n].mean())
    out["eddy_vT_south_low_mean"] = float(vT[low][:, mid_s].mean())
    out["eke_max"] = float(eke.max())
    out["u_zonal_mean"] = u.tolist()
    out["T_zonal_mean"] = T.tolist()
    out["p_zonal_mean"] = p.tolist()
    if p_levels is not None:
        out["p_levels_hPa"] = [float(x) / 100.0 for x in p_levels]
        for name, f in (("u", u), ("T", T), ("uv", uv), ("vT", vT)):
            q = to_pressure_levels(f, p, p_levels)
            out[name + "_p_levels"] = [[None if np.isnan(x) else float(x) for x in row] for row in q]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--forcing", default="held_suarez", choices=["held_suarez", "hot_jupiter"])
    ap.add_argument("--glevel", type=int, default=5)
    ap.add_argument("--nv", type=int, default=37)
    ap.add_argument("--z-top", type=float, default=None, help="default 32 km (Earth), 4875 km (hot Jupiter)")
    ap.add_argument("--dt", type=float, default=None, help="default 1000 s (Earth), 600 s (hot Jupiter)")
    ap.add_argument("--workload-planet", action="store_true",
                    help="the benchmark workloads' planet values instead of Table 1")
    ap.add_argument("--n-small", type=int, default=6)
    ap.add_argument("--days", type=float, default=1200.0)
    ap.add_argument("--spinup", type=float, default=200.0)
    ap.add_argument("--nlat", type=int, default=36)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--p-surf", type=float, default=1.0e5, help="surface pressure of the resting start (Pa)")
    ap.add_argument("--isothermal", action="store_true",
                    help="Held-Suarez from an isothermal 300 K start with 0.1 K of noise instead of the T_eq profile")
    ap.add_argument("--shallow", action="store_true", help="shallow-atmosphere approximation (Sec. 3)")
    ap.add_argument("--hydrostatic", action="store_true", help="hydrostatic approximation (Sec. 3)")
    ap.add_argument("--p-levels", type=int, default=20,
                    help="pressure levels (geometric spacing over the run's mean pressures) for the output")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    hj = args.forcing == "hot_jupiter"
    if args.z_top is None:
        args.z_top = 4.875e6 if hj else 32.0e3
    if args.dt is None:
        args.dt = 600.0 if hj else 1000.0
    import torch
    import paper_1607_05535_gb300 as thor
    import workloads as wls
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    torch.cuda.set_device(0)
    s = torch.cuda.Stream()
    extras = {}
    means, samples, seconds, diag = run(thor, args.glevel, args.nv, args.z_top, args.dt, args.n_small, args.days,
                                        args.spinup, args.nlat, forcing=args.forcing, precision=args.precision,
                                        stream=s.cuda_stream, table1=not args.workload_planet,
                                        shallow=args.shallow, hydrostatic=args.hydrostatic, extras=extras,
                                        p_surf=args.p_surf,
                                        profile=None if (hj or args.isothermal) else "held_suarez",
                                        noise=0.1 if (args.isothermal and not hj) else 0.0)
    P = planet(args.forcing, not args.workload_planet)
    import numpy as np
    pm = means[..., 4]
    p_levels = np.geomspace(pm.max(), pm[pm > 0].min(), args.p_levels) if args.p_levels > 1 else None
    summary = summarize(means, P.radius, P.gravity, p_levels)
    ws = w_star(extras["w_mean"], extras["points"], extras["areas"], args.nlat)
    summary["imprint"] = imprint_summary(ws, extras["w_mean"], extras["points"], extras["areas"], args.nlat)
    summary["w_star_level0"] = ws[:, 0].tolist()
    summary.update({"config": vars(args), "samples": samples, "seconds": seconds,
                    "large_steps": round(args.days * 86400.0 / args.dt),
                    "final_diag": {k: diag[k] for k in ("mass", "energy", "aam", "max_vh", "nonfinite")}})
    text = json.dumps(summary)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    short = {k: v for k, v in summary.items()
             if k not in ("u_zonal_mean", "T_zonal_mean", "p_zonal_mean", "lat", "w_star_level0", "p_levels_hPa")
             and not k.endswith("_p_levels")}
    print(json.dumps(short))
    return 0


if __name__ == "__main__":
    sys.exit(main())
