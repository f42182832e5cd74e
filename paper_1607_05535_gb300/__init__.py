"""Python binding of libthor (include/thor.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
plain pointers and sizes through ctypes; all arithmetic of the method runs in
libthor's CUDA kernels (and its float64 host grid builder). Importing this
module fails loudly if the library has not been built
(``python paper_1607_05535_gb300/build.py`` or ``__graft_entry__.build()``).
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "libthor.so")

THOR_OK, THOR_EINVAL, THOR_ENOMEM, THOR_ECUDA, THOR_ENONFINITE, THOR_ETIMEOUT, THOR_ENOTCONV = \
    0, -1, -2, -3, -4, -5, -6
THOR_FP64, THOR_MIXED = 0, 1
THOR_FORCING_NONE, THOR_FORCING_HELD_SUAREZ, THOR_FORCING_HOT_JUPITER = 0, 1, 2
THOR_FIELD_RHO, THOR_FIELD_MOM, THOR_FIELD_W, THOR_FIELD_RHOTHETA, THOR_FIELD_PRESSURE, \
    THOR_FIELD_TEMPERATURE = range(6)
(THOR_TUNE_KCHUNK, THOR_TUNE_GRAPH, THOR_TUNE_CHECK_FINITE, THOR_TUNE_BLOCK, THOR_TUNE_SOLVE_TMA,
 THOR_TUNE_ENERGY_FIXER, THOR_TUNE_BUDGET, THOR_TUNE_RK_STAGES, THOR_TUNE_COMPENSATED,
 THOR_TUNE_L2_HINTS, THOR_TUNE_LEVEL_SPLIT) = range(11)
THOR_ENSEMBLE_MAX = 4096
THOR_MLP_TUNE_TCGEN05 = 0

EXPORTED = [
    "thor_strerror", "thor_grid_create", "thor_grid_info", "thor_grid_points",
    "thor_grid_neighbours", "thor_grid_areas", "thor_grid_coarse_map", "thor_grid_destroy", "thor_state_init",
    "thor_step", "thor_diag", "thor_state_get", "thor_state_set", "thor_state_get_all", "thor_state_set_all",
    "thor_launch_count",
    "thor_tune", "thor_profile", "thor_profile_read", "thor_state_destroy",
    "thor_mass_noalloc", "thor_mlp_create", "thor_mlp_info", "thor_mlp_get_params",
    "thor_mlp_set_params", "thor_mlp_forward", "thor_mlp_backward", "thor_mlp_train_step",
    "thor_mlp_destroy", "thor_closure_features", "thor_closure_attach", "thor_coarse_grain",
    "thor_autotune", "thor_ensemble_create", "thor_ensemble_step", "thor_ensemble_info",
    "thor_ensemble_tune", "thor_ensemble_autotune", "thor_ensemble_destroy", "thor_mlp_tune",
    "thor_checkpoint_bytes", "thor_checkpoint_save", "thor_checkpoint_load", "thor_wait_selftest",
    "thor_budget_read", "thor_zonal_accumulate", "thor_zonal_read",
    "thor_zonal_read_w",
]

# kernel ids of thor_profile_read
KERNELS = ["derived", "lap1", "slow", "slow_w", "stage_init", "ss_lapd", "ss_mom", "ss_solve",
           "physics", "ss_flux", "ss_factor"]


class thor_spring(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("alpha", ctypes.c_double), ("k", ctypes.c_double),
                ("dt", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class thor_planet(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("omega", ctypes.c_double),
                ("gravity", ctypes.c_double), ("Rd", ctypes.c_double), ("cp", ctypes.c_double),
                ("p_ref", ctypes.c_double), ("diff_D", ctypes.c_double)]


THOR_PROFILE_ISOTHERMAL, THOR_PROFILE_HELD_SUAREZ = 0, 1


class thor_init(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_double), ("p_surf", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("forcing", ctypes.c_int), ("hj_dT", ctypes.c_double),
                ("precision", ctypes.c_int), ("hyperdiffusion", ctypes.c_int),
                ("divergence_damping", ctypes.c_int), ("shallow", ctypes.c_int),
                ("hydrostatic", ctypes.c_int), ("profile", ctypes.c_int), ("vorder", ctypes.c_int),
                ("anelastic", ctypes.c_int)]


class thor_diag_t(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("energy", ctypes.c_double), ("aam", ctypes.c_double),
                ("max_vh", ctypes.c_double), ("max_w", ctypes.c_double),
                ("mean_T", ctypes.c_double), ("nonfinite", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ThorError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib.thor_strerror(status).decode()} ({status})")


def _load():
    if not os.path.exists(LIBRARY_PATH):
        raise ImportError(f"libthor is not built ({LIBRARY_PATH} missing); run "
                          "`python paper_1607_05535_gb300/build.py`")
    lib = ctypes.CDLL(LIBRARY_PATH)
    P, I, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    IP = ctypes.POINTER(ctypes.c_int)
    sig = {
        "thor_strerror": (ctypes.c_char_p, [I]),
        "thor_grid_create": (I, [I, I, D, D, ctypes.POINTER(thor_spring), ctypes.POINTER(P)]),
        "thor_grid_info": (I, [P, IP, IP, IP, IP, IP]),
        "thor_grid_points": (I, [P, P, Z]),
        "thor_grid_neighbours": (I, [P, P, Z]),
        "thor_grid_areas": (I, [P, P, Z]),
        "thor_grid_coarse_map": (I, [P, P, P, Z]),
        "thor_grid_destroy": (None, [P]),
        "thor_state_init": (I, [P, ctypes.POINTER(thor_planet), ctypes.POINTER(thor_init), P,
                                ctypes.POINTER(P)]),
        "thor_step": (I, [P, I, I, D]),
        "thor_diag": (I, [P, ctypes.POINTER(thor_diag_t)]),
        "thor_state_get": (I, [P, I, P, Z]),
        "thor_state_set": (I, [P, I, P, Z]),
        "thor_state_get_all": (I, [P, P, P, P, P, I, I]),
        "thor_state_set_all": (I, [P, P, P, P, P, I, I]),
        "thor_launch_count": (I, [P, ctypes.POINTER(ctypes.c_longlong)]),
        "thor_tune": (I, [P, I, I]),
        "thor_profile": (I, [P, I]),
        "thor_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_longlong)]),
        "thor_state_destroy": (None, [P]),
        "thor_mass_noalloc": (I, [P, P, Z, P, P]),
        "thor_mlp_create": (I, [P, I, I, ctypes.c_ulonglong, P, ctypes.POINTER(P)]),
        "thor_mlp_info": (I, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "thor_mlp_get_params": (I, [P, P, Z]),
        "thor_mlp_set_params": (I, [P, P, Z]),
        "thor_mlp_forward": (I, [P, P, I, P]),
        "thor_mlp_backward": (I, [P, P, I, P]),
        "thor_mlp_train_step": (I, [P, P, P, I, ctypes.c_float, P]),
        "thor_mlp_destroy": (None, [P]),
        "thor_closure_features": (I, [P, P, P, P]),
        "thor_closure_attach": (I, [P, P, P, P, P, P, I]),
        "thor_coarse_grain": (I, [P, P, P, Z]),
        "thor_autotune": (I, [P, I, D, I, IP, IP, ctypes.POINTER(D)]),
        "thor_ensemble_create": (I, [ctypes.POINTER(P), I, P, ctypes.POINTER(P)]),
        "thor_ensemble_step": (I, [P, I, IP, ctypes.POINTER(D)]),
        "thor_ensemble_info": (I, [P, IP, ctypes.POINTER(ctypes.c_longlong)]),
        "thor_ensemble_tune": (I, [P, I, I]),
        "thor_ensemble_autotune": (I, [P, IP, ctypes.POINTER(D), I, IP, IP, ctypes.POINTER(D)]),
        "thor_ensemble_destroy": (None, [P]),
        "thor_mlp_tune": (I, [P, I, I]),
        "thor_checkpoint_bytes": (I, [P, ctypes.POINTER(Z)]),
        "thor_checkpoint_save": (I, [P, P, Z]),
        "thor_checkpoint_load": (I, [P, P, Z]),
        "thor_wait_selftest": (I, [I, ctypes.c_uint, IP]),
        "thor_budget_read": (I, [P, ctypes.POINTER(D), I, IP]),
        "thor_zonal_accumulate": (I, [P, I]),
        "thor_zonal_read": (I, [P, I, ctypes.POINTER(D), Z, I, ctypes.POINTER(ctypes.c_longlong)]),
        "thor_zonal_read_w": (I, [P, I, ctypes.POINTER(D), Z, ctypes.POINTER(ctypes.c_longlong)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(status, where):
    if status != THOR_OK:
        raise ThorError(status, where)


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def thor_strerror(status):
    return _lib.thor_strerror(status).decode()


def thor_grid_create(glevel, nv, radius, z_top, spring=None):
    out = ctypes.c_void_p()
    sp = ctypes.byref(spring) if spring is not None else None
    _check(_lib.thor_grid_create(glevel, nv, radius, z_top, sp, ctypes.byref(out)), "thor_grid_create")
    return out


def thor_grid_info(grid):
    v = [ctypes.c_int() for _ in range(5)]
    _check(_lib.thor_grid_info(grid, *[ctypes.byref(x) for x in v]), "thor_grid_info")
    return dict(ncol=v[0].value, nv=v[1].value, npent=v[2].value, spring_iters=v[3].value,
                spring_converged=bool(v[4].value))


def thor_grid_points(grid):
    n = thor_grid_info(grid)["ncol"]
    out = np.empty((n, 3), dtype=np.float64)
    _check(_lib.thor_grid_points(grid, _ptr(out), out.size), "thor_grid_points")
    return out


def thor_grid_neighbours(grid):
    n = thor_grid_info(grid)["ncol"]
    out = np.empty((n, 6), dtype=np.int32)
    _check(_lib.thor_grid_neighbours(grid, _ptr(out), out.size), "thor_grid_neighbours")
    return out


def thor_grid_areas(grid):
    n = thor_grid_info(grid)["ncol"]
    out = np.empty(n, dtype=np.float64)
    _check(_lib.thor_grid_areas(grid, _ptr(out), out.size), "thor_grid_areas")
    return out


def thor_grid_coarse_map(fine, coarse):
    """Nearest coarse column of every fine column (int32, the fine grid's
    column count), the map thor_coarse_grain takes."""
    n = thor_grid_info(fine)["ncol"]
    out = np.empty(n, dtype=np.int32)
    _check(_lib.thor_grid_coarse_map(fine, coarse, _ptr(out), out.size), "thor_grid_coarse_map")
    return out


def thor_grid_destroy(grid):
    _lib.thor_grid_destroy(grid)


def thor_state_init(grid, planet, init, stream=None):
    out = ctypes.c_void_p()
    _check(_lib.thor_state_init(grid, ctypes.byref(planet), ctypes.byref(init),
                                ctypes.c_void_p(stream or 0), ctypes.byref(out)), "thor_state_init")
    return out


def thor_step(state, n_large, n_small, dt):
    _check(_lib.thor_step(state, n_large, n_small, dt), "thor_step")


def thor_diag(state):
    d = thor_diag_t()
    _check(_lib.thor_diag(state, ctypes.byref(d)), "thor_diag")
    return d.as_dict()


def _field_shape(field, ncol, nv):
    if field == THOR_FIELD_MOM:
        return (ncol, nv, 3)
    if field == THOR_FIELD_W:
        return (ncol, nv + 1)
    return (ncol, nv)


def thor_state_get(state, field, ncol, nv, out=None):
    shape = _field_shape(field, ncol, nv)
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    _check(_lib.thor_state_get(state, field, _ptr(out), int(np.prod(shape))), "thor_state_get")
    return out


def thor_state_set(state, field, host):
    a = host if hasattr(host, "data_ptr") else np.ascontiguousarray(host, dtype=np.float64)
    n = a.numel() if hasattr(a, "numel") else a.size
    _check(_lib.thor_state_set(state, field, _ptr(a), n), "thor_state_set")


PROGNOSTIC = (THOR_FIELD_RHO, THOR_FIELD_MOM, THOR_FIELD_W, THOR_FIELD_RHOTHETA)


def _checked(a, shape):
    """A float64 host buffer of the given shape (numpy array or CPU tensor),
    C-contiguous, without a copy."""
    if hasattr(a, "data_ptr"):
        if a.dtype != __import__("torch").float64 or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError("expected a contiguous float64 tensor of shape %s" % (shape,))
    elif a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != tuple(shape):
        raise ValueError("expected a C-contiguous float64 array of shape %s" % (shape,))
    return a


def thor_state_get_all(state, ncol, nv, out=None):
    """(rho, mom, w, rhotheta) in the layouts of thor_state_get, one
    synchronisation; out: four buffers to fill (e.g. page-locked tensors)."""
    shapes = [_field_shape(f, ncol, nv) for f in PROGNOSTIC]
    if out is None:
        out = [np.empty(s, dtype=np.float64) for s in shapes]
    bufs = [_checked(a, s) for a, s in zip(out, shapes)]
    _check(_lib.thor_state_get_all(state, *[_ptr(a) for a in bufs], int(ncol), int(nv)), "thor_state_get_all")
    return tuple(out)


def thor_state_set_all(state, rho, mom, w, rhotheta):
    """All four prognostic fields from host buffers (layouts of
    thor_state_get), one synchronisation."""
    ncol, nv = rho.shape
    bufs = [_checked(a, _field_shape(f, ncol, nv)) for a, f in zip((rho, mom, w, rhotheta), PROGNOSTIC)]
    _check(_lib.thor_state_set_all(state, *[_ptr(a) for a in bufs], int(ncol), int(nv)), "thor_state_set_all")


def thor_launch_count(state):
    c = ctypes.c_longlong()
    _check(_lib.thor_launch_count(state, ctypes.byref(c)), "thor_launch_count")
    return c.value


def thor_tune(state, knob, value):
    _check(_lib.thor_tune(state, knob, value), "thor_tune")


def thor_profile(state, enable):
    _check(_lib.thor_profile(state, int(bool(enable))), "thor_profile")


def thor_profile_read(state, kernel):
    """(total ms, launches) of kernel id ``kernel`` (an index of KERNELS)."""
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(_lib.thor_profile_read(state, kernel, ctypes.byref(ms), ctypes.byref(n)), "thor_profile_read")
    return ms.value, n.value


def thor_state_destroy(state):
    _lib.thor_state_destroy(state)


def thor_mass_noalloc(rho, volume, mass_out, stream=None):
    """sum(rho * volume) into the one-element device tensor ``mass_out``;
    ``rho`` and ``volume`` are float64 device tensors of the same size. For
    callers that must not allocate: the library allocates nothing here."""
    n = rho.numel()
    if volume.numel() != n:
        raise ValueError("rho and volume differ in size")
    _check(_lib.thor_mass_noalloc(_ptr(rho), _ptr(volume), n, _ptr(mass_out),
                                  ctypes.c_void_p(stream or 0)), "thor_mass_noalloc")


# ------------------------------------------------------------- learned closure

def thor_mlp_create(sizes, max_batch, seed=0, stream=None):
    arr = (ctypes.c_int * len(sizes))(*sizes)
    out = ctypes.c_void_p()
    _check(_lib.thor_mlp_create(arr, len(sizes), max_batch, seed, ctypes.c_void_p(stream or 0),
                                ctypes.byref(out)), "thor_mlp_create")
    return out


def thor_mlp_info(mlp):
    n = ctypes.c_size_t()
    _check(_lib.thor_mlp_info(mlp, ctypes.byref(n)), "thor_mlp_info")
    return n.value


def thor_mlp_get_params(mlp):
    out = np.empty(thor_mlp_info(mlp), dtype=np.float32)
    _check(_lib.thor_mlp_get_params(mlp, _ptr(out), out.size), "thor_mlp_get_params")
    return out


def thor_mlp_set_params(mlp, host):
    a = np.ascontiguousarray(host, dtype=np.float32)
    _check(_lib.thor_mlp_set_params(mlp, _ptr(a), a.size), "thor_mlp_set_params")


def thor_mlp_forward(mlp, x, y):
    """x, y: float32 device tensors [m][n_in], [m][n_out]."""
    _check(_lib.thor_mlp_forward(mlp, _ptr(x), x.shape[0], _ptr(y)), "thor_mlp_forward")


def thor_mlp_backward(mlp, dy, grad):
    _check(_lib.thor_mlp_backward(mlp, _ptr(dy), dy.shape[0], _ptr(grad)), "thor_mlp_backward")


def thor_mlp_train_step(mlp, x, target, lr, loss=None):
    _check(_lib.thor_mlp_train_step(mlp, _ptr(x), _ptr(target), x.shape[0], lr,
                                    _ptr(loss) if loss is not None else None), "thor_mlp_train_step")


def thor_mlp_tune(mlp, knob, value):
    _check(_lib.thor_mlp_tune(mlp, knob, value), "thor_mlp_tune")


def thor_mlp_destroy(mlp):
    _lib.thor_mlp_destroy(mlp)


def thor_closure_features(state, mean, std, x):
    _check(_lib.thor_closure_features(state, _ptr(mean), _ptr(std), _ptr(x)), "thor_closure_features")


def thor_closure_attach(state, mlp, in_mean=None, in_std=None, out_mean=None, out_std=None, period=1):
    p = lambda t: _ptr(t) if t is not None else None
    _check(_lib.thor_closure_attach(state, mlp, p(in_mean), p(in_std), p(out_mean), p(out_std), period),
           "thor_closure_attach")


def thor_coarse_grain(fine, coarse, fine_to_coarse):
    a = np.ascontiguousarray(fine_to_coarse, dtype=np.int32)
    _check(_lib.thor_coarse_grain(fine, coarse, _ptr(a), a.size), "thor_coarse_grain")


def thor_autotune(state, n_small, dt, steps=3):
    """Returns (kchunk, block, ms per large step) of the fastest launch shape,
    which is left set on the state."""
    kc, bs, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(_lib.thor_autotune(state, n_small, dt, steps, ctypes.byref(kc), ctypes.byref(bs), ctypes.byref(ms)),
           "thor_autotune")
    return kc.value, bs.value, ms.value


def _int_array(v):
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


def _double_array(v):
    return (ctypes.c_double * len(v))(*[float(x) for x in v])


def thor_ensemble_create(members, stream=None):
    arr = (ctypes.c_void_p * max(len(members), 1))(*[m.value if hasattr(m, "value") else m for m in members])
    out = ctypes.c_void_p()
    _check(_lib.thor_ensemble_create(arr, len(members), ctypes.c_void_p(stream or 0), ctypes.byref(out)),
           "thor_ensemble_create")
    return out


def thor_ensemble_step(ens, n_large, n_small, dt):
    _check(_lib.thor_ensemble_step(ens, n_large, _int_array(n_small), _double_array(dt)), "thor_ensemble_step")


def thor_ensemble_info(ens):
    n, l = ctypes.c_int(), ctypes.c_longlong()
    _check(_lib.thor_ensemble_info(ens, ctypes.byref(n), ctypes.byref(l)), "thor_ensemble_info")
    return {"members": n.value, "launches": l.value}


def thor_ensemble_tune(ens, knob, value):
    _check(_lib.thor_ensemble_tune(ens, knob, value), "thor_ensemble_tune")


def thor_ensemble_autotune(ens, n_small, dt, steps=3):
    kc, bs, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(_lib.thor_ensemble_autotune(ens, _int_array(n_small), _double_array(dt), steps, ctypes.byref(kc),
                                       ctypes.byref(bs), ctypes.byref(ms)), "thor_ensemble_autotune")
    return kc.value, bs.value, ms.value


def thor_ensemble_destroy(ens):
    _lib.thor_ensemble_destroy(ens)


def thor_checkpoint_bytes(state):
    n = ctypes.c_size_t()
    _check(_lib.thor_checkpoint_bytes(state, ctypes.byref(n)), "thor_checkpoint_bytes")
    return n.value


def thor_checkpoint_save(state, buf=None):
    """Raw checkpoint into `buf` (a numpy uint8 array or a torch uint8 tensor,
    host or device, of thor_checkpoint_bytes bytes); a new host array if None."""
    n = thor_checkpoint_bytes(state)
    if buf is None:
        buf = np.empty(n, dtype=np.uint8)
    _check(_lib.thor_checkpoint_save(state, _ptr(buf), n), "thor_checkpoint_save")
    return buf


def thor_checkpoint_load(state, buf):
    n = buf.numel() if hasattr(buf, "numel") else buf.size
    _check(_lib.thor_checkpoint_load(state, _ptr(buf), n), "thor_checkpoint_load")


def thor_wait_selftest(arrive, limit_us):
    """1 if a bounded device wait ran out, 0 if it completed."""
    g = ctypes.c_int()
    _check(_lib.thor_wait_selftest(int(arrive), int(limit_us), ctypes.byref(g)), "thor_wait_selftest")
    return g.value


def thor_budget_read(state, max_rows=1 << 16):
    """Budget rows recorded since thor_tune(THOR_TUNE_BUDGET, capacity), as a
    float64 array (n, 8): mass, energy, axial angular momentum at the start
    of each large step and after its dynamics, the energy fixer's dT, 0."""
    import numpy as np
    out = np.zeros((max_rows, 8))
    n = ctypes.c_int()
    _check(_lib.thor_budget_read(state, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(max_rows),
                                 ctypes.byref(n)), "thor_budget_read")
    return out[:n.value].copy()


ZONAL_QUANTITIES = ("weight", "u", "v", "T", "p", "uv", "vT", "uu", "vv")


def thor_zonal_accumulate(state, nlat):
    _check(_lib.thor_zonal_accumulate(state, int(nlat)), "thor_zonal_accumulate")


def thor_zonal_read(state, nlat, nv, reset=False):
    """(sums, samples): sums is a float64 array (nv, nlat, 9) of the
    accumulated band values ZONAL_QUANTITIES; divide by samples for time
    means."""
    import numpy as np
    out = np.zeros((nv, nlat, 9))
    n = ctypes.c_longlong()
    _check(_lib.thor_zonal_read(state, int(nlat), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size,
                                int(bool(reset)), ctypes.byref(n)), "thor_zonal_read")
    return out, n.value


def thor_zonal_read_w(state, nlat, ncol, nv):
    """(w_mean, samples): the time mean of w at every cell centre, float64
    (ncol, nv) in the column order of thor_state_get."""
    import numpy as np
    out = np.zeros((ncol, nv))
    n = ctypes.c_longlong()
    _check(_lib.thor_zonal_read_w(state, int(nlat), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size,
                                  ctypes.byref(n)), "thor_zonal_read_w")
    return out, n.value
