"""Ensemble stepping and the launch-shape autotuner: an ensemble of uneven
members (grid level, radius, rotation, time step, small-step count, forcing)
stepped in one launch per kernel reproduces every member stepped alone (one
member under the shallow-atmosphere approximation and one under the
hydrostatic one among nonhydrostatic deep ones), and
the autotuner leaves the state unchanged and changes no result.

The ensemble kernels inline the same device code as the single-state ones,
but the compiler may contract a product and a sum into one FMA differently
in the two kernels, so results agree to rounding (a unit in the last place
per operation, then carried by the dynamics), not bit for bit: 1e-12 of each
field's largest value in float64, 1e-5 in mixed precision (1e-4 for the
small vertical momentum)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1607_05535_gb300 as thor
import workloads as wls

FIELDS = (thor.THOR_FIELD_RHO, thor.THOR_FIELD_MOM, thor.THOR_FIELD_W, thor.THOR_FIELD_RHOTHETA)

# (glevel, radius factor, omega factor, dt, n_small, forcing)
MEMBERS = [
    (3, 1.0, 1.0, 1800.0, 6, thor.THOR_FORCING_HELD_SUAREZ),
    (2, 0.3, 4.0, 900.0, 8, thor.THOR_FORCING_HELD_SUAREZ),
    (4, 2.0, 0.5, 1200.0, 4, thor.THOR_FORCING_NONE),
    (3, 0.5, 2.0, 600.0, 8, thor.THOR_FORCING_HELD_SUAREZ),
    (2, 5.0, 0.2, 3600.0, 6, thor.THOR_FORCING_NONE),
]
SHALLOW = {3}                                    # members run with thor_init.shallow = 1
HYDROSTATIC = {1}                                # members run with thor_init.hydrostatic = 1


class Pool:
    """Two identical states per member: one for the ensemble, one stepped alone."""

    def __init__(self, precision, stream=None, nv=12):
        self.grids, self.a, self.b, self.n_small, self.dt, self.shape = [], [], [], [], [], []
        sp = thor.thor_spring(1.15, 1.0, 1.0, 0.01, 0.0, 10)
        for i, (g, rf, of, dt, ns, forcing) in enumerate(MEMBERS):
            P = wls.EARTH
            grid = thor.thor_grid_create(g, nv, P.radius * rf, 24.0e3, sp)
            planet = thor.thor_planet(P.radius * rf, P.omega * of, P.gravity, P.Rd, P.cp, P.p_ref, P.diff_D)
            init = thor.thor_init(300.0, 1.0e5, 0.5, 77 + i, forcing, 300.0, precision, 1, 1,
                                  int(i in SHALLOW), int(i in HYDROSTATIC))
            self.grids.append(grid)
            self.a.append(thor.thor_state_init(grid, planet, init, stream))
            self.b.append(thor.thor_state_init(grid, planet, init, stream))
            self.n_small.append(ns)
            self.dt.append(dt)
            self.shape.append((thor.thor_grid_info(grid)["ncol"], nv))

    def fields(self, st, i):
        ncol, nv = self.shape[i]
        return [thor.thor_state_get(st, f, ncol, nv) for f in FIELDS]

    def close(self):
        for s in self.a + self.b:
            thor.thor_state_destroy(s)
        for g in self.grids:
            thor.thor_grid_destroy(g)


def assert_same(pool, rtol, rtol_w=None):
    """Every field within rtol of its largest magnitude (rtol_w for W, a field
    three orders of magnitude below the others whose float32 rounding comes
    from the large vertical terms)."""
    for i in range(len(MEMBERS)):
        for f, fa, fb in zip(FIELDS, pool.fields(pool.a[i], i), pool.fields(pool.b[i], i)):
            tol = rtol_w if (f == thor.THOR_FIELD_W and rtol_w is not None) else rtol
            scale = np.max(np.abs(fb)) + 1e-300
            assert np.max(np.abs(fa - fb)) <= tol * scale, (i, f, np.max(np.abs(fa - fb)) / scale)


@pytest.mark.parametrize("precision", [thor.THOR_FP64, thor.THOR_MIXED])
@pytest.mark.parametrize("graph", [True, False])
def test_ensemble_matches_members_stepped_alone(precision, graph):
    torch.cuda.set_device(0)
    st = torch.cuda.Stream() if graph else None
    sp = st.cuda_stream if st is not None else None
    pool = Pool(precision, sp)
    ens = thor.thor_ensemble_create(pool.a, sp)
    try:
        for it in range(2):                      # second call replays the graph
            thor.thor_ensemble_step(ens, 2, pool.n_small, pool.dt)
            for i, s in enumerate(pool.b):
                thor.thor_step(s, 2, pool.n_small[i], pool.dt[i])
        info = thor.thor_ensemble_info(ens)
        assert info["members"] == len(MEMBERS) and info["launches"] > 0
        if precision == thor.THOR_FP64:
            assert_same(pool, 1e-12)
        else:
            assert_same(pool, 1e-5, rtol_w=1e-4)
        d = [thor.thor_diag(s)["nonfinite"] for s in pool.a]
        assert all(x == 0 for x in d)
    finally:
        thor.thor_ensemble_destroy(ens)
        pool.close()


# (glevel, radius factor, omega factor, dt, n_small, forcing, shallow, hydrostatic)
ORACLE_MEMBERS = [
    (3, 1.0, 1.0, 1800.0, 6, "held_suarez", 0, 0),
    (2, 0.3, 4.0, 900.0, 8, "held_suarez", 0, 1),
    (3, 0.5, 2.0, 600.0, 4, "none", 1, 0),
    (2, 2.0, 0.5, 2400.0, 6, "held_suarez", 0, 0),
]


def test_ensemble_members_match_the_oracle():
    """Four uneven members (grid level, radius, rotation, time step, small-step
    count, forcing; one under the hydrostatic and one under the shallow
    approximation) stepped together in float64, two large steps, against the
    oracle run of each member: every field within 1e-10 relative L2 and every
    element within 1e-8 of its field's largest change (W of the hydrostatic
    member, diagnosed from nearly cancelling terms, to 1e-12 g rho dtau)."""
    from dataclasses import replace
    from harness import Pair, change_errors, field_errors
    from oracle import dycore as dc
    torch.cuda.set_device(0)
    pairs, n_small, dts = [], [], []
    try:
        for i, (g, rf, of, dt, ns, forcing, sh, hy) in enumerate(ORACLE_MEMBERS):
            planet = replace(wls.EARTH, radius=wls.EARTH.radius * rf, omega=wls.EARTH.omega * of)
            wl = wls.Workload(f"member_{i}", glevel=g, nv=12, z_top=24.0e3, planet=planet, T0=300.0,
                              p_surf=1.0e5, noise_amp=0.5, seed=77 + i, forcing=forcing, dt=dt, n_small=ns,
                              n_large=2)
            pairs.append(Pair(wl, shallow=bool(sh), hydrostatic=bool(hy)))
            n_small.append(ns)
            dts.append(dt)
        X0 = [p.oracle_initial() for p in pairs]
        ens = thor.thor_ensemble_create([p.state for p in pairs], None)
        try:
            thor.thor_ensemble_step(ens, 2, n_small, dts)
        finally:
            thor.thor_ensemble_destroy(ens)
        for p, X, ns, dt in zip(pairs, X0, n_small, dts):
            ref = dc.run(p.model, X, 2, ns, dt)
            got = p.get()
            e = field_errors(got, ref)
            c = change_errors(got, ref, X)
            w_scale = p.wl.planet.gravity * float(np.max(ref.rho)) * dt / ns
            assert e["rho"] < 1e-10 and e["Th"] < 1e-10 and e["M"] < 1e-10, (p.wl.name, e)
            assert e["W"] < 1e-10 or e["W_maxabs"] < 1e-12 * w_scale, (p.wl.name, e)
            for k in ("rho", "Th", "M"):
                assert c[k] < 1e-8, (p.wl.name, k, c)
            assert c["W"] < 1e-8 or e["W_maxabs"] < 1e-12 * w_scale, (p.wl.name, c)
    finally:
        for p in pairs:
            p.close()


def test_ensemble_launch_count_is_independent_of_members():
    """One launch per kernel for the whole ensemble: the launch count of a
    large step does not grow with the member count."""
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    pool = Pool(thor.THOR_MIXED, st.cuda_stream)
    try:
        counts = []
        for n in (1, len(MEMBERS)):
            ens = thor.thor_ensemble_create(pool.a[:n], st.cuda_stream)
            ns = [8] * n
            thor.thor_ensemble_step(ens, 1, ns, pool.dt[:n])
            counts.append(thor.thor_ensemble_info(ens)["launches"])
            thor.thor_ensemble_destroy(ens)
        assert counts[0] == counts[1]
        # uneven n_small: the members still stepping form a prefix; launches follow the largest n_small
        ens = thor.thor_ensemble_create(pool.a, st.cuda_stream)
        thor.thor_ensemble_step(ens, 1, pool.n_small, pool.dt)
        ref = thor.thor_ensemble_info(ens)["launches"]
        thor.thor_ensemble_destroy(ens)
        ens = thor.thor_ensemble_create(pool.a[:1], st.cuda_stream)
        thor.thor_ensemble_step(ens, 1, [max(pool.n_small)], pool.dt[:1])
        assert thor.thor_ensemble_info(ens)["launches"] == ref
        thor.thor_ensemble_destroy(ens)
    finally:
        pool.close()


def test_autotune_keeps_the_state_and_the_results():
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    pool = Pool(thor.THOR_MIXED, st.cuda_stream, nv=20)
    try:
        i = 2
        before = pool.fields(pool.a[i], i)
        kc, bs, ms = thor.thor_autotune(pool.a[i], pool.n_small[i], pool.dt[i], steps=2)
        assert kc in (1, 2, 3, 4, 6, 8) and bs in (64, 96, 128, 192, 256) and ms > 0
        for x, y in zip(before, pool.fields(pool.a[i], i)):
            assert np.array_equal(x, y)
        thor.thor_step(pool.a[i], 3, pool.n_small[i], pool.dt[i])
        thor.thor_step(pool.b[i], 3, pool.n_small[i], pool.dt[i])
        for x, y in zip(pool.fields(pool.a[i], i), pool.fields(pool.b[i], i)):
            assert np.array_equal(x, y)
        # the ensemble autotuner restores every member
        ens = thor.thor_ensemble_create(pool.a, st.cuda_stream)
        before = [pool.fields(s, k) for k, s in enumerate(pool.a)]
        kc, bs, ms = thor.thor_ensemble_autotune(ens, pool.n_small, pool.dt, steps=1)
        assert kc in (1, 2, 3, 4, 6, 8) and bs in (64, 96, 128, 192, 256) and ms > 0
        for k, s in enumerate(pool.a):
            for x, y in zip(before[k], pool.fields(s, k)):
                assert np.array_equal(x, y)
        thor.thor_ensemble_destroy(ens)
    finally:
        pool.close()


def test_ensemble_rejects_bad_arguments():
    torch.cuda.set_device(0)
    pool = Pool(thor.THOR_MIXED)
    try:
        with pytest.raises(thor.ThorError):
            thor.thor_ensemble_create([pool.a[0], pool.a[0]])
        ens = thor.thor_ensemble_create(pool.a)
        with pytest.raises(thor.ThorError):
            thor.thor_ensemble_step(ens, 1, [7] + pool.n_small[1:], pool.dt)
        with pytest.raises(thor.ThorError):
            thor.thor_ensemble_step(ens, 1, pool.n_small, [0.0] + pool.dt[1:])
        with pytest.raises(thor.ThorError):
            thor.thor_ensemble_tune(ens, thor.THOR_TUNE_BLOCK, 96 + 1)
        thor.thor_ensemble_destroy(ens)
    finally:
        pool.close()
