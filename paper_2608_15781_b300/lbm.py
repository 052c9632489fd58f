"""Thin ctypes binding of the C ABI in ``include/cglbm.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``libcglbm.so``; this module
only converts NumPy arrays and dataclasses to the C structures.  If the
library is missing or fails to load, the calls raise ``LbmError`` -- there is
no CPU fallback.

Functions carry the C names (``lbm_create``, ``lbm_step``, ``lbm_observables``,
...); ``Lattice`` bundles them for convenience.  Arrays use the library's
layout: lattice fields are (nz, ny, nx) with x fastest, populations are
(45, nz, ny, nx) ordered f^r_0..18, f^p_0..18, g_0..6.
"""
import ctypes
import dataclasses
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# the in-tree build; CGLBM_LIBRARY may name another build of the same C ABI
LIB_PATH = os.environ.get("CGLBM_LIBRARY", os.path.join(_PKG, "libcglbm.so"))
NPOP = 45

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENAN = 0, -1, -2, -3, -4
FIELD_RHON, FIELD_NORMAL, FIELD_GRADMAG, FIELD_NS, FIELD_NN, FIELD_CURV, FIELD_DELTA = range(7)
KERNEL_NAMES = ("density", "color_solid", "normal", "normal_solid", "main", "observables", "fields")

# exported symbols (kept in sync with include/cglbm.h; the CPU tests check both)
SYMBOLS = (
    "lbm_create", "lbm_step", "lbm_observables", "lbm_reaction", "lbm_init_fields", "lbm_get_state",
    "lbm_set_state", "lbm_get_field", "lbm_set_debug", "lbm_profile", "lbm_profile_read",
    "lbm_info", "lbm_destroy", "lbm_strerror", "lbm_step_static", "lbm_tune", "lbm_set_launch",
    "lbm_batch_create", "lbm_batch_step", "lbm_batch_observables", "lbm_batch_get_state",
    "lbm_batch_set_state", "lbm_batch_tune", "lbm_batch_set_launch", "lbm_batch_profile", "lbm_batch_profile_read",
    "lbm_batch_destroy", "lbm_reaction_async", "lbm_set_wetting", "lbm_set_inlet", "lbm_adjoint_forward", "lbm_adjoint_backward",
)
STATIC_MAX_NODES = 131072   # LBM_STATIC_MAX_NODES


class LbmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _strerror(code) if _lib is not None else f"error {code}"
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class _Geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("solid", ctypes.c_void_p), ("reactive", ctypes.c_void_p), ("bc_z", ctypes.c_int32),
                ("theta_deg", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("theta_deg", ctypes.c_double), ("accel", ctypes.c_double * 3),
                ("diffusivity", ctypes.c_double), ("k_rate", ctypes.c_double), ("c_init", ctypes.c_double),
                ("c_in", ctypes.c_double), ("u_in", ctypes.c_double), ("rho_out", ctypes.c_double),
                ("xi", ctypes.c_double), ("reaction_mode", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p)]


class _Obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("mass_r", "mass_p", "mass_c", "consumed", "rate", "conversion",
                                               "gas_saturation", "flux_in", "flux_out")] + \
               [(n, ctypes.c_int64) for n in ("step", "n_fluid", "n_bad")]


@dataclass
class Params:
    """Physical and numerical parameters (lattice units); mirrors ``lbm_params``."""
    tau: float = 1.0
    sigma: float = 0.01
    beta: float = 0.7
    theta_deg: float = 90.0
    accel: tuple = (0.0, 0.0, 0.0)
    diffusivity: float = 0.05
    k_rate: float = 1e-3
    c_init: float = 1.0
    c_in: float = 1.0
    u_in: float = 0.0
    rho_out: float = 1.0
    xi: float = 1.0
    reaction_mode: int = 0
    storage: int = 0

    def to_c(self, stream=None):
        p = _Params()
        for f in dataclasses.fields(self):
            if f.name == "accel":
                for a in range(3):
                    p.accel[a] = float(self.accel[a])
            else:
                setattr(p, f.name, getattr(self, f.name))
        p.cuda_stream = stream
        return p


_lib = None


def load_library(path=LIB_PATH):
    """Load ``libcglbm.so`` (once).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LbmError(LBM_EINVAL, f"CUDA library not built: {path} (run python -m paper_2608_15781_b300.build)")
    lib = ctypes.CDLL(path)
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(_Geometry), ctypes.POINTER(_Params), ctypes.POINTER(P)]),
        "lbm_step": (ctypes.c_int, [P, I64]),
        "lbm_observables": (ctypes.c_int, [P, ctypes.POINTER(_Obs)]),
        "lbm_reaction": (ctypes.c_int, [P, P, P]),
        "lbm_init_fields": (ctypes.c_int, [P, P, P, P, P]),
        "lbm_get_state": (ctypes.c_int, [P, P, SZ]),
        "lbm_set_state": (ctypes.c_int, [P, P, SZ]),
        "lbm_get_field": (ctypes.c_int, [P, I32, P, SZ]),
        "lbm_set_debug": (ctypes.c_int, [P, I32]),
        "lbm_profile": (ctypes.c_int, [P, I32]),
        "lbm_profile_read": (ctypes.c_int, [P, P, P, I32]),
        "lbm_info": (ctypes.c_int, [P, P, P, P, P]),
        "lbm_destroy": (None, [P]),
        "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_step_static": (ctypes.c_int, [I32, I32, I32, P, P, P, P, P, ctypes.POINTER(_Params)]),
        "lbm_tune": (ctypes.c_int, [P, P]),
        "lbm_set_launch": (ctypes.c_int, [P, P]),
        "lbm_batch_create": (ctypes.c_int, [I32, ctypes.POINTER(_Geometry), ctypes.POINTER(_Params), P,
                                            ctypes.POINTER(P)]),
        "lbm_batch_step": (ctypes.c_int, [P, I64]),
        "lbm_batch_observables": (ctypes.c_int, [P, ctypes.POINTER(_Obs), I32]),
        "lbm_batch_get_state": (ctypes.c_int, [P, I32, P, SZ]),
        "lbm_batch_set_state": (ctypes.c_int, [P, I32, P, SZ]),
        "lbm_batch_tune": (ctypes.c_int, [P, P]),
        "lbm_batch_set_launch": (ctypes.c_int, [P, P]),
        "lbm_batch_profile": (ctypes.c_int, [P, I32]),
        "lbm_batch_profile_read": (ctypes.c_int, [P, P, P, I32]),
        "lbm_batch_destroy": (None, [P]),
        "lbm_reaction_async": (ctypes.c_int, [P, P]),
        "lbm_set_wetting": (ctypes.c_int, [P, P]),
        "lbm_set_inlet": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_double]),
        "lbm_adjoint_forward": (ctypes.c_int, [P, I64, I64, P]),
        "lbm_adjoint_backward": (ctypes.c_int, [P, ctypes.c_double, P, P, P, SZ]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _strerror(code):
    return _lib.lbm_strerror(int(code)).decode()


def _check(rc, what):
    if rc != LBM_OK:
        raise LbmError(rc, what)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# --------------------------------------------------------------------------- C-named calls
def lbm_create(solid, params, reactive=None, bc_z=0, stream=None, theta=None):
    """Create a context for the (nz, ny, nx) mask ``solid``; returns the opaque handle.

    ``theta``: optional (nz, ny, nx) contact angles in degrees, read at solid nodes."""
    lib = load_library()
    g, _keep = _geometry(solid, reactive, bc_z, theta)
    p = params.to_c(stream)
    h = ctypes.c_void_p()
    _check(lib.lbm_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)), "lbm_create")
    return h


def lbm_step(ctx, nsteps):
    _check(load_library().lbm_step(ctx, int(nsteps)), "lbm_step")


def lbm_observables(ctx, allow_nan=False):
    o = _Obs()
    rc = load_library().lbm_observables(ctx, ctypes.byref(o))
    if rc != LBM_OK and not (allow_nan and rc == LBM_ENAN):
        _check(rc, "lbm_observables")
    return {n: getattr(o, n) for n, _ in _Obs._fields_}


def lbm_reaction(ctx):
    """(rate, consumed): the last step's and the cumulative sum of the reaction amounts."""
    r, c = ctypes.c_double(), ctypes.c_double()
    _check(load_library().lbm_reaction(ctx, ctypes.byref(r), ctypes.byref(c)), "lbm_reaction")
    return r.value, c.value


def lbm_reaction_async(ctx, dst_ptr):
    """Enqueue one 16-byte copy of (rate, consumed) into host memory at address ``dst_ptr`` (two
    doubles, page-locked), valid after the next synchronisation of the context's stream."""
    _check(load_library().lbm_reaction_async(ctx, dst_ptr), "lbm_reaction_async")


def lbm_init_fields(ctx, rho_r, rho_p, conc, u=None):
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (rho_r, rho_p, conc)]
    ua = None if u is None else np.ascontiguousarray(u, dtype=np.float32)
    _check(load_library().lbm_init_fields(ctx, *[_ptr(a) for a in arrs], _ptr(ua)), "lbm_init_fields")


def lbm_get_state(ctx, shape):
    nz, ny, nx = shape
    out = np.empty((NPOP, nz, ny, nx), dtype=np.float32)
    _check(load_library().lbm_get_state(ctx, _ptr(out), out.nbytes), "lbm_get_state")
    return out


def lbm_set_state(ctx, f):
    f = np.ascontiguousarray(f, dtype=np.float32)
    _check(load_library().lbm_set_state(ctx, _ptr(f), f.nbytes), "lbm_set_state")


def lbm_get_field(ctx, which, shape):
    nz, ny, nx = shape
    comps = 3 if which in (FIELD_NORMAL, FIELD_NS) else 1
    out = np.empty((comps, nz, ny, nx), dtype=np.float32)
    _check(load_library().lbm_get_field(ctx, int(which), _ptr(out), out.nbytes), "lbm_get_field")
    return out if comps == 3 else out[0]


def lbm_set_debug(ctx, enable):
    _check(load_library().lbm_set_debug(ctx, int(bool(enable))), "lbm_set_debug")


def lbm_profile(ctx, max_launches):
    _check(load_library().lbm_profile(ctx, int(max_launches)), "lbm_profile")


def lbm_profile_read(ctx):
    ms = np.zeros(len(KERNEL_NAMES), dtype=np.float64)
    n = np.zeros(len(KERNEL_NAMES), dtype=np.int64)
    _check(load_library().lbm_profile_read(ctx, _ptr(ms), _ptr(n), len(KERNEL_NAMES)), "lbm_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_NAMES)}


def lbm_info(ctx):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load_library().lbm_info(ctx, *[ctypes.byref(a) for a in v]), "lbm_info")
    return dict(n_fluid=v[0].value, n_wall=v[1].value, n_solid_bnd=v[2].value, device_bytes=v[3].value)


def _launch_dict(blocks):
    return dict(main=int(blocks[0]), density=int(blocks[1]), normal=int(blocks[2]), pdl=int(blocks[3]),
                fields=int(blocks[4]))


def _launch_array(launch):
    return np.array([launch["main"], launch["density"], launch["normal"], launch.get("pdl", 1),
                     launch.get("fields", 0)], dtype=np.int32)


def lbm_tune(ctx):
    """Time the candidate launch configurations on the current state and keep the fastest; returns it."""
    blocks = np.zeros(5, dtype=np.int32)
    _check(load_library().lbm_tune(ctx, _ptr(blocks)), "lbm_tune")
    return _launch_dict(blocks)


def lbm_set_launch(ctx, launch):
    """Set the launch configuration (a dict as returned by lbm_tune)."""
    _check(load_library().lbm_set_launch(ctx, _ptr(_launch_array(launch))), "lbm_set_launch")


def lbm_set_wetting(ctx, theta):
    """Replace the contact-angle field ((nz, ny, nx) degrees at solid nodes; None = uniform)."""
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
    _check(load_library().lbm_set_wetting(ctx, _ptr(th)), "lbm_set_wetting")


def lbm_set_inlet(ctx, u_in, c_in):
    _check(load_library().lbm_set_inlet(ctx, float(u_in), float(c_in)), "lbm_set_inlet")


def lbm_adjoint_forward(ctx, nsteps, checkpoint_every=0):
    """Advance nsteps storing checkpoints; returns the outlet conversion J."""
    j = ctypes.c_double()
    _check(load_library().lbm_adjoint_forward(ctx, int(nsteps), int(checkpoint_every), ctypes.byref(j)),
           "lbm_adjoint_forward")
    return j.value


def lbm_adjoint_backward(ctx, shape, seed=1.0, want_state=False):
    """(dJ/dtheta per node (degrees^-1, float64), dJ/du_in, dJ/df_0 or None), each times seed."""
    nz, ny, nx = shape
    dth = np.empty((nz, ny, nx), dtype=np.float64)
    du = ctypes.c_double()
    ds = np.empty((NPOP, nz, ny, nx), dtype=np.float32) if want_state else None
    _check(load_library().lbm_adjoint_backward(ctx, float(seed), _ptr(dth), ctypes.byref(du), _ptr(ds),
                                               ds.nbytes if ds is not None else 0), "lbm_adjoint_backward")
    return dth, du.value, ds


def lbm_destroy(ctx):
    if ctx is not None and ctx.value:
        load_library().lbm_destroy(ctx)


def lbm_step_static(shape, solid_dev, f_in_dev, f_out_dev, params, reactive_dev=None, delta_sum_dev=None,
                    stream=None):
    """One allocation-free step of a periodic box on caller-held device buffers.

    For callers that may not allocate device memory (pools or arenas that own
    every allocation, recorded streams): the intermediate fields live in a
    fixed scratch array inside the library, shared by all calls, so calls must
    not overlap on the GPU.  Pointers are raw device addresses (ints), e.g.
    ``tensor.data_ptr()``; f_in / f_out hold 45 * N floats in the
    ``lbm_get_state`` layout; nx * ny * nz must not exceed ``STATIC_MAX_NODES``.
    """
    nz, ny, nx = shape
    p = params.to_c(stream)
    _check(load_library().lbm_step_static(int(nx), int(ny), int(nz), solid_dev, reactive_dev, f_in_dev, f_out_dev,
                                           delta_sum_dev, ctypes.byref(p)), "lbm_step_static")


def _geometry(solid, reactive, bc_z, theta=None):
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    if solid.ndim != 3:
        raise LbmError(LBM_EINVAL, "solid must be a (nz, ny, nx) array")
    react = None if reactive is None else np.ascontiguousarray(reactive, dtype=np.uint8)
    if react is not None and react.shape != solid.shape:
        raise LbmError(LBM_EINVAL, "reactive mask shape")
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
    if th is not None and th.shape != solid.shape:
        raise LbmError(LBM_EINVAL, "theta field shape")
    nz, ny, nx = solid.shape
    g = _Geometry(nx, ny, nz, solid.ctypes.data, react.ctypes.data if react is not None else None, int(bc_z),
                  th.ctypes.data if th is not None else None)
    return g, (solid, react, th)


def lbm_batch_create(solids, params, reactives=None, bc_z=None, stream=None, thetas=None):
    """Create a batch of independent lattices (lists of masks, Params, optional r masks, bc_z,
    optional contact-angle fields)."""
    lib = load_library()
    n = len(solids)
    reactives = reactives or [None] * n
    thetas = thetas or [None] * n
    bc_z = bc_z if bc_z is not None else [0] * n
    geoms = (_Geometry * n)()
    keep = []
    for k in range(n):
        g, arrays = _geometry(solids[k], reactives[k], bc_z[k], thetas[k])
        geoms[k] = g
        keep.append(arrays)
    prms = (_Params * n)(*[p.to_c(stream) for p in params])
    h = ctypes.c_void_p()
    _check(lib.lbm_batch_create(n, geoms, prms, stream, ctypes.byref(h)), "lbm_batch_create")
    return h


# --------------------------------------------------------------------------- convenience
class Lattice:
    """One lattice on the current CUDA device, driven through the C ABI."""

    def __init__(self, solid, params, reactive=None, bc_z=0, stream=None, theta=None):
        self.shape = tuple(np.shape(solid))
        self.params = params
        self.bc_z = bc_z
        self.ctx = lbm_create(solid, params, reactive=reactive, bc_z=bc_z, stream=stream, theta=theta)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def observables(self, allow_nan=False):
        return lbm_observables(self.ctx, allow_nan=allow_nan)

    def reaction(self):
        return lbm_reaction(self.ctx)

    def reaction_async(self, dst_ptr):
        lbm_reaction_async(self.ctx, dst_ptr)

    def init_fields(self, rho_r, rho_p, conc, u=None):
        lbm_init_fields(self.ctx, rho_r, rho_p, conc, u)

    def get_state(self):
        return lbm_get_state(self.ctx, self.shape)

    def set_state(self, f):
        lbm_set_state(self.ctx, f)

    def field(self, which):
        return lbm_get_field(self.ctx, which, self.shape)

    def set_debug(self, enable=True):
        lbm_set_debug(self.ctx, enable)

    def profile(self, max_launches):
        lbm_profile(self.ctx, max_launches)

    def profile_read(self):
        return lbm_profile_read(self.ctx)

    def info(self):
        return lbm_info(self.ctx)

    def tune(self):
        return lbm_tune(self.ctx)

    def set_launch(self, launch):
        lbm_set_launch(self.ctx, launch)

    def set_wetting(self, theta):
        lbm_set_wetting(self.ctx, theta)

    def set_inlet(self, u_in, c_in=None):
        lbm_set_inlet(self.ctx, u_in, self.params.c_in if c_in is None else c_in)

    def adjoint_forward(self, nsteps, checkpoint_every=0):
        return lbm_adjoint_forward(self.ctx, nsteps, checkpoint_every)

    def adjoint_backward(self, seed=1.0, want_state=False):
        return lbm_adjoint_backward(self.ctx, self.shape, seed, want_state)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent lattices advanced together (one launch per kernel for all of them)."""

    def __init__(self, solids, params, reactives=None, bc_z=None, stream=None):
        self.shapes = [tuple(np.shape(s)) for s in solids]
        self.n = len(solids)
        self.handle = lbm_batch_create(solids, params, reactives, bc_z, stream)

    def step(self, n=1):
        _check(load_library().lbm_batch_step(self.handle, int(n)), "lbm_batch_step")

    def observables(self, allow_nan=False):
        obs = (_Obs * self.n)()
        rc = load_library().lbm_batch_observables(self.handle, obs, self.n)
        if rc != LBM_OK and not (allow_nan and rc == LBM_ENAN):
            _check(rc, "lbm_batch_observables")
        return [{nm: getattr(o, nm) for nm, _ in _Obs._fields_} for o in obs]

    def get_state(self, k):
        nz, ny, nx = self.shapes[k]
        out = np.empty((NPOP, nz, ny, nx), dtype=np.float32)
        _check(load_library().lbm_batch_get_state(self.handle, int(k), _ptr(out), out.nbytes), "lbm_batch_get_state")
        return out

    def set_state(self, k, f):
        f = np.ascontiguousarray(f, dtype=np.float32)
        _check(load_library().lbm_batch_set_state(self.handle, int(k), _ptr(f), f.nbytes), "lbm_batch_set_state")

    def tune(self):
        blocks = np.zeros(5, dtype=np.int32)
        _check(load_library().lbm_batch_tune(self.handle, _ptr(blocks)), "lbm_batch_tune")
        return _launch_dict(blocks)

    def set_launch(self, launch):
        _check(load_library().lbm_batch_set_launch(self.handle, _ptr(_launch_array(launch))), "lbm_batch_set_launch")

    def profile(self, max_launches):
        _check(load_library().lbm_batch_profile(self.handle, int(max_launches)), "lbm_batch_profile")

    def profile_read(self):
        ms = np.zeros(len(KERNEL_NAMES), dtype=np.float64)
        n = np.zeros(len(KERNEL_NAMES), dtype=np.int64)
        _check(load_library().lbm_batch_profile_read(self.handle, _ptr(ms), _ptr(n), len(KERNEL_NAMES)),
               "lbm_batch_profile_read")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_NAMES)}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load_library().lbm_batch_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
