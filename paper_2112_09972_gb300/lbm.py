"""Thin Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/liblbm_gb300.so``;
this module only converts arguments.  There is no CPU fallback: if the
library is missing or cannot be loaded, importing the functions raises.

The raw entry points keep the C names (``lbm_create``, ``lbm_set_gradient``,
``lbm_step``, ``lbm_deformation`` ...); ``DropletLBM`` wraps them with numpy
arrays and raises ``LBMError`` on a non-zero status.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm_gb300.so")

LBM_FP64, LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV = 0, 1, 2, 3
LBM_BC_GHOST_LINEAR, LBM_BC_PERIODIC_TEST = 0, 1
LBM_FRAME_DROPLET, LBM_FRAME_BOX = 0, 1
FRAMES = {"droplet": LBM_FRAME_DROPLET, "box": LBM_FRAME_BOX}
# "fp16dev" / "bf16dev": 16-bit deviation storage with float32 collision (lbm.h)
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16dev": LBM_FP16_DEV, "bf16dev": LBM_BF16_DEV}

# Every function the header declares, for the export check.
ABI_FUNCTIONS = [
    "lbm_opts_default", "lbm_create", "lbm_set_gradient", "lbm_set_gradient_table", "lbm_step", "lbm_sync",
    "lbm_deformation", "lbm_moments", "lbm_get_fields", "lbm_get_populations", "lbm_set_populations",
    "lbm_checksums", "lbm_get_step", "lbm_save", "lbm_load", "lbm_profile_enable", "lbm_profile_read",
    "lbm_launch_shape", "lbm_launch_variant", "lbm_destroy", "lbm_strerror", "lbm_moments_static",
    "lbm_batch_create", "lbm_batch_set_gradients", "lbm_batch_step", "lbm_batch_sync", "lbm_batch_deformation",
    "lbm_batch_get_populations", "lbm_batch_set_populations", "lbm_batch_autotune", "lbm_batch_shape",
    "lbm_batch_launch_kind",
    "lbm_batch_destroy", "lbm_batch_moments",
    "lbm_mlp_create", "lbm_mlp_set_normalisation", "lbm_mlp_param_count", "lbm_mlp_get_params",
    "lbm_mlp_set_params", "lbm_mlp_forward", "lbm_mlp_deformation", "lbm_mlp_gradients", "lbm_mlp_train_step",
    "lbm_mlp_sync", "lbm_mlp_destroy", "lbm_mlp_set_tensor_path", "lbm_mm_integrate", "lbm_components", "lbm_surface_deformation",
    "lbm_reinject_mass", "lbm_selftest_wait",
]


class lbm_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("rho_hi", ctypes.c_double),
        ("rho_lo", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("mach_limit", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("device", ctypes.c_int32),
        ("tile_y", ctypes.c_int32),
        ("z_chunk", ctypes.c_int32),
        ("frame", ctypes.c_int32),
        ("row_variant", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("mrt_rates", ctypes.c_double * 5),
    ]


class LBMError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)


def load_library(path=LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    sig = {
        "lbm_opts_default": (None, [ctypes.POINTER(lbm_opts)]),
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(vp), _I32P, ctypes.c_double, _DP, ctypes.c_double,
                                      ctypes.POINTER(lbm_opts)]),
        "lbm_set_gradient": (ctypes.c_int, [vp, _DP, ctypes.c_int64]),
        "lbm_set_gradient_table": (ctypes.c_int, [vp, _I64P, _DP, ctypes.c_int64]),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lbm_sync": (ctypes.c_int, [vp]),
        "lbm_deformation": (ctypes.c_int, [vp, _DP, _DP, _DP, _DP]),
        "lbm_moments": (ctypes.c_int, [vp, _DP]),
        "lbm_get_fields": (ctypes.c_int, [vp, _DP, _DP, _DP]),
        "lbm_get_populations": (ctypes.c_int, [vp, _DP]),
        "lbm_set_populations": (ctypes.c_int, [vp, _DP]),
        "lbm_checksums": (ctypes.c_int, [vp, _DP, _DP]),
        "lbm_get_step": (ctypes.c_int, [vp, _I64P]),
        "lbm_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "lbm_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "lbm_profile_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_profile_read": (ctypes.c_int, [vp, ctypes.c_int, _DP, _I64P]),
        "lbm_launch_shape": (ctypes.c_int, [vp, _I32P, _I32P, _I32P]),
        "lbm_launch_variant": (ctypes.c_int, [vp, _I32P]),
        "lbm_destroy": (None, [vp]),
        "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_moments_static": (ctypes.c_int, [vp, ctypes.c_int32, _I32P, vp, vp]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int32, _I32P, _DP, _DP, ctypes.c_double,
                                            ctypes.POINTER(lbm_opts)]),
        "lbm_batch_set_gradients": (ctypes.c_int, [vp, ctypes.c_int64, _DP]),
        "lbm_batch_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lbm_batch_sync": (ctypes.c_int, [vp]),
        "lbm_batch_deformation": (ctypes.c_int, [vp, _DP, _DP, _DP]),
        "lbm_batch_get_populations": (ctypes.c_int, [vp, ctypes.c_int32, _DP]),
        "lbm_batch_set_populations": (ctypes.c_int, [vp, ctypes.c_int32, _DP]),
        "lbm_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int32, _I32P, _I32P]),
        "lbm_batch_shape": (ctypes.c_int, [vp, _I32P, _I32P, _I32P]),
        "lbm_batch_launch_kind": (ctypes.c_int, [vp, _I32P]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_moments": (ctypes.c_int, [vp, _DP]),
        "lbm_mlp_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int32, _I32P, ctypes.c_int32, ctypes.c_uint64,
                                          vp, ctypes.c_int32]),
        "lbm_mlp_set_normalisation": (ctypes.c_int, [vp, _FP, _FP, _FP, _FP]),
        "lbm_mlp_param_count": (ctypes.c_int, [vp, _I64P]),
        "lbm_mlp_get_params": (ctypes.c_int, [vp, _FP]),
        "lbm_mlp_set_params": (ctypes.c_int, [vp, _FP]),
        "lbm_mlp_forward": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64]),
        "lbm_mlp_deformation": (ctypes.c_int, [vp, vp, ctypes.c_int64, vp, vp]),
        "lbm_mlp_gradients": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, _DP, _FP]),
        "lbm_mlp_train_step": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, ctypes.c_float, _DP]),
        "lbm_mlp_sync": (ctypes.c_int, [vp]),
        "lbm_mlp_destroy": (None, [vp]),
        "lbm_mlp_set_tensor_path": (ctypes.c_int, [vp, ctypes.c_int32]),
        "lbm_surface_deformation": (ctypes.c_int, [vp, _DP, _DP, _DP]),
        "lbm_reinject_mass": (ctypes.c_int, [vp, ctypes.c_double, _DP]),
        "lbm_selftest_wait": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
        "lbm_components": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int64, _I32P, _I64P, ctypes.c_int32]),
        "lbm_mm_integrate": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code):
    return load_library().lbm_strerror(int(code)).decode()


def _check(code, what):
    if code != 0:
        raise LBMError(code, what)


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def current_torch_stream():
    """The current torch CUDA stream handle, or None if torch has no CUDA."""
    try:
        import torch
    except ImportError:
        return None
    if not torch.cuda.is_available():
        return None
    return torch.cuda.current_stream().cuda_stream


def lbm_moments_static(f_dev_ptr, precision, box, out_dev_ptr, stream=None):
    """Allocation-free droplet moments of device-resident populations.

    For callers that cannot allocate device memory at that point (e.g. while a
    stream is being captured into a CUDA graph).  ``f_dev_ptr`` and
    ``out_dev_ptr`` are device addresses (ints) of the dense population array
    and of 26 doubles; ``precision`` is "fp64" or "fp32".  See ``lbm.h``.
    """
    lib = load_library()
    b = (ctypes.c_int32 * 3)(*[int(v) for v in box])
    _check(lib.lbm_moments_static(ctypes.c_void_p(int(f_dev_ptr)), PRECISIONS[precision], b,
                                  ctypes.c_void_p(int(out_dev_ptr)), None if stream is None else ctypes.c_void_p(stream)),
           "lbm_moments_static")


class DropletLBM:
    """A droplet box behind the C ABI.

    ``box`` is (Lx, Ly, Lz) or an int; ``visc`` (nu_A, nu_B) in lattice units;
    ``precision`` "fp32", "fp64", "fp16dev" or "bf16dev" (16-bit deviation
    storage, float32 collision); ``periodic`` selects the periodic test
    mode instead of the ghost-node boundary; ``frame`` "droplet" (the ghost
    flow is linear in the distance from the droplet's centre of mass) or "box".
    """

    def __init__(self, box, R, visc, G, precision="fp32", periodic=False, rho_hi=0.0, rho_lo=0.0, xi=0.0,
                 mach_limit=0.0, stream=None, device=-1, tile_y=0, z_chunk=0, frame="droplet", row_variant=0,
                 mrt=None):
        lib = load_library()
        self._lib = lib
        if isinstance(box, int):
            box = (box, box, box)
        self.box = tuple(int(v) for v in box)
        self.nodes = self.box[0] * self.box[1] * self.box[2]
        o = lbm_opts()
        lib.lbm_opts_default(ctypes.byref(o))
        o.precision = PRECISIONS[precision]
        o.bc = LBM_BC_PERIODIC_TEST if periodic else LBM_BC_GHOST_LINEAR
        o.rho_hi, o.rho_lo, o.xi, o.mach_limit = float(rho_hi), float(rho_lo), float(xi), float(mach_limit)
        if stream is None:
            stream = current_torch_stream()
        o.cuda_stream = stream
        o.device = int(device)
        o.tile_y, o.z_chunk = int(tile_y), int(z_chunk)
        o.row_variant = int(row_variant)
        # mrt: None (BGK), True (MRT, default free rates) or the rates (s_e, s_eps, s_q, s_pi, s_m)
        if mrt is not None and mrt is not False:
            o.collision = 1
            if mrt is not True:
                for k, v in enumerate(mrt):
                    o.mrt_rates[k] = float(v)
        o.frame = FRAMES[frame]
        b = (ctypes.c_int32 * 3)(*self.box)
        v = (ctypes.c_double * 2)(float(visc[0]), float(visc[1]))
        h = ctypes.c_void_p()
        _check(lib.lbm_create(ctypes.byref(h), b, float(R), v, float(G), ctypes.byref(o)), "lbm_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        Lx, Ly, Lz = self.box
        return (2, 19, Lz, Ly, Lx)

    def set_gradient(self, A, t):
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
        _check(self._lib.lbm_set_gradient(self._h, _dptr(A), int(t)), "lbm_set_gradient")

    def set_gradient_table(self, t, A):
        t = np.ascontiguousarray(np.asarray(t, dtype=np.int64).reshape(-1))
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1, 9))
        _check(self._lib.lbm_set_gradient_table(self._h, t.ctypes.data_as(_I64P), _dptr(A), int(t.size)),
               "lbm_set_gradient_table")

    def step(self, n=1):
        _check(self._lib.lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        _check(self._lib.lbm_sync(self._h), "lbm_sync")

    def deformation(self):
        """(D, axes[3,3] columns, lambda[3], centre[3])."""
        D = np.zeros(1)
        axes = np.zeros(9)
        lam = np.zeros(3)
        c = np.zeros(3)
        _check(self._lib.lbm_deformation(self._h, _dptr(D), _dptr(axes), _dptr(lam), _dptr(c)), "lbm_deformation")
        return float(D[0]), axes.reshape(3, 3), lam, c

    def moments(self):
        m = np.zeros(10)
        _check(self._lib.lbm_moments(self._h, _dptr(m)), "lbm_moments")
        return m

    def fields(self):
        Lx, Ly, Lz = self.box
        ra = np.zeros(self.nodes)
        rb = np.zeros(self.nodes)
        u = np.zeros(3 * self.nodes)
        _check(self._lib.lbm_get_fields(self._h, _dptr(ra), _dptr(rb), _dptr(u)), "lbm_get_fields")
        return ra.reshape(Lz, Ly, Lx), rb.reshape(Lz, Ly, Lx), u.reshape(Lz, Ly, Lx, 3)

    def populations(self):
        f = np.zeros(self.shape)
        _check(self._lib.lbm_get_populations(self._h, _dptr(f)), "lbm_get_populations")
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.shape))
        _check(self._lib.lbm_set_populations(self._h, _dptr(f)), "lbm_set_populations")

    def checksums(self):
        mass = np.zeros(2)
        mom = np.zeros(3)
        _check(self._lib.lbm_checksums(self._h, _dptr(mass), _dptr(mom)), "lbm_checksums")
        return mass, mom

    def components(self, threshold=0.0, min_nodes=1, max_sizes=8):
        """(count, sizes) of the droplet phase's connected components (lbm_components)."""
        cnt = ctypes.c_int32()
        sizes = np.zeros(max(int(max_sizes), 1), dtype=np.int64)
        _check(self._lib.lbm_components(self._h, float(threshold), int(min_nodes), ctypes.byref(cnt),
                                        sizes.ctypes.data_as(_I64P), int(max_sizes)), "lbm_components")
        return cnt.value, sizes[:max_sizes]

    def surface_deformation(self):
        """(D_LBM, area, volume) of Eq. 17 (lbm_surface_deformation)."""
        v = np.zeros(3)
        _check(self._lib.lbm_surface_deformation(self._h, _dptr(v[0:1]), _dptr(v[1:2]), _dptr(v[2:3])),
               "lbm_surface_deformation")
        return float(v[0]), float(v[1]), float(v[2])

    def reinject_mass(self, target):
        """Rescale the droplet component inside phi > 0 to total mass target; returns the factor."""
        k = np.zeros(1)
        _check(self._lib.lbm_reinject_mass(self._h, float(target), _dptr(k)), "lbm_reinject_mass")
        return float(k[0])

    def step_count(self):
        s = ctypes.c_int64()
        _check(self._lib.lbm_get_step(self._h, ctypes.byref(s)), "lbm_get_step")
        return s.value

    def save(self, path):
        _check(self._lib.lbm_save(self._h, str(path).encode()), "lbm_save")

    def load(self, path):
        _check(self._lib.lbm_load(self._h, str(path).encode()), "lbm_load")

    def profile(self, every=1):
        """Time the launches of every `every`-th step (0 or False: off)."""
        _check(self._lib.lbm_profile_enable(self._h, int(every)), "lbm_profile_enable")

    def profile_read(self, kernel=0):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self._lib.lbm_profile_read(self._h, int(kernel), ctypes.byref(ms), ctypes.byref(n)), "lbm_profile_read")
        return ms.value, n.value

    def launch_shape(self):
        ty, zc, ctas = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lbm_launch_shape(self._h, ctypes.byref(ty), ctypes.byref(zc), ctypes.byref(ctas)),
               "lbm_launch_shape")
        return ty.value, zc.value, ctas.value

    def launch_variant(self):
        """0: the generic tile kernel; 1, 2, 3: the row kernel's variant (lbm_opts.row_variant)."""
        v = ctypes.c_int32()
        _check(self._lib.lbm_launch_variant(self._h, ctypes.byref(v)), "lbm_launch_variant")
        return v.value


class BatchLBM:
    """An ensemble of independent droplet boxes behind the C ABI (fp32).

    ``boxes`` is a sequence of (Lx, Ly, Lz); ``R`` the droplet radius of each
    box; ``rho_lo`` the ghost density of the droplet component (required).
    """

    def __init__(self, boxes, R, visc, G, rho_lo, rho_hi=0.0, xi=0.0, mach_limit=0.0, stream=None, device=-1,
                 z_chunk=0, frame="droplet", tile_y=0):
        lib = load_library()
        self._lib = lib
        self.boxes = [tuple(int(v) for v in b) for b in boxes]
        self.nbox = len(self.boxes)
        o = lbm_opts()
        lib.lbm_opts_default(ctypes.byref(o))
        o.precision = LBM_FP32
        o.bc = LBM_BC_GHOST_LINEAR
        o.rho_hi, o.rho_lo, o.xi, o.mach_limit = float(rho_hi), float(rho_lo), float(xi), float(mach_limit)
        if stream is None:
            stream = current_torch_stream()
        o.cuda_stream = stream
        o.device = int(device)
        o.z_chunk = int(z_chunk)
        o.tile_y = int(tile_y)  # > 0: the generic tile march even where the row kernel applies
        o.frame = FRAMES[frame]
        flat = (ctypes.c_int32 * (3 * self.nbox))(*[v for b in self.boxes for v in b])
        r = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(self.nbox))
        v = (ctypes.c_double * 2)(float(visc[0]), float(visc[1]))
        h = ctypes.c_void_p()
        _check(lib.lbm_batch_create(ctypes.byref(h), self.nbox, flat, _dptr(r), v, float(G), ctypes.byref(o)),
               "lbm_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape_of(self, k):
        Lx, Ly, Lz = self.boxes[k]
        return (2, 19, Lz, Ly, Lx)

    def set_gradients(self, A):
        """A[t, k, 9]: gradient of box k at step t."""
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        assert A.ndim == 3 and A.shape[1] == self.nbox and A.shape[2] == 9
        _check(self._lib.lbm_batch_set_gradients(self._h, int(A.shape[0]), _dptr(A)), "lbm_batch_set_gradients")

    def step(self, n=1):
        _check(self._lib.lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def sync(self):
        _check(self._lib.lbm_batch_sync(self._h), "lbm_batch_sync")

    def deformation(self):
        D = np.zeros(self.nbox)
        axes = np.zeros(9 * self.nbox)
        c = np.zeros(3 * self.nbox)
        _check(self._lib.lbm_batch_deformation(self._h, _dptr(D), _dptr(axes), _dptr(c)), "lbm_batch_deformation")
        return D, axes.reshape(self.nbox, 3, 3), c.reshape(self.nbox, 3)

    def populations(self, k):
        f = np.zeros(self.shape_of(k))
        _check(self._lib.lbm_batch_get_populations(self._h, int(k), _dptr(f)), "lbm_batch_get_populations")
        return f

    def set_populations(self, k, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.shape_of(k)))
        _check(self._lib.lbm_batch_set_populations(self._h, int(k), _dptr(f)), "lbm_batch_set_populations")

    def moments(self):
        """The ten moments of every box, [nbox, 10] (see lbm_moments)."""
        m = np.zeros(10 * self.nbox)
        _check(self._lib.lbm_batch_moments(self._h, _dptr(m)), "lbm_batch_moments")
        return m.reshape(self.nbox, 10)

    def autotune(self, trial_steps=4):
        zc, per = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lbm_batch_autotune(self._h, int(trial_steps), ctypes.byref(zc), ctypes.byref(per)),
               "lbm_batch_autotune")
        return zc.value, per.value

    def shape(self):
        zc, ctas, items = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.lbm_batch_shape(self._h, ctypes.byref(zc), ctypes.byref(ctas), ctypes.byref(items)),
               "lbm_batch_shape")
        return zc.value, ctas.value, items.value

    def launch_kind(self):
        """0: the generic tile march, 1: the row kernel over padded rows."""
        k = ctypes.c_int32()
        _check(self._lib.lbm_batch_launch_kind(self._h, ctypes.byref(k)), "lbm_batch_launch_kind")
        return k.value


def _fptr(a):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_FP)


class MLP:
    """The surrogate's multilayer perceptron behind the C ABI (lbm_mlp_*).

    Device arrays are torch CUDA tensors (float32, contiguous) passed by
    address; host arrays are numpy.  ``sizes`` = (d0, hidden..., dL).  The
    network's kernels run on ``stream`` (a cudaStream_t handle; None: torch's
    current stream, and the library's own stream when that is the default
    stream): tensors passed in must be ready on that stream.
    """

    def __init__(self, sizes, max_batch=4096, seed=0, stream=None, device=-1):
        lib = load_library()
        self._lib = lib
        self.sizes = tuple(int(v) for v in sizes)
        if stream is None:
            stream = current_torch_stream()
        arr = (ctypes.c_int32 * len(self.sizes))(*self.sizes)
        h = ctypes.c_void_p()
        _check(lib.lbm_mlp_create(ctypes.byref(h), len(self.sizes) - 1, arr, int(max_batch), int(seed), stream,
                                  int(device)), "lbm_mlp_create")
        self._h = h
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_normalisation(self, x_mean, x_scale, y_mean, y_scale):
        a = [np.ascontiguousarray(np.asarray(v, dtype=np.float32)) for v in (x_mean, x_scale, y_mean, y_scale)]
        _check(self._lib.lbm_mlp_set_normalisation(self._h, *[_fptr(v) for v in a]), "lbm_mlp_set_normalisation")

    def param_count(self):
        n = ctypes.c_int64()
        _check(self._lib.lbm_mlp_param_count(self._h, ctypes.byref(n)), "lbm_mlp_param_count")
        return n.value

    def get_params(self):
        p = np.zeros(self.param_count(), dtype=np.float32)
        _check(self._lib.lbm_mlp_get_params(self._h, _fptr(p)), "lbm_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        _check(self._lib.lbm_mlp_set_params(self._h, _fptr(p)), "lbm_mlp_set_params")

    def forward(self, x, y):
        """y[n, dL] = network(x[n, d0]) (torch CUDA float32 tensors; async)."""
        _check(self._lib.lbm_mlp_forward(self._h, x.data_ptr(), y.data_ptr(), int(x.shape[0])), "lbm_mlp_forward")

    def deformation(self, x, m6, D):
        """m6[n, 6] and D[n] (float64) of predicted conformation tensors (async)."""
        _check(self._lib.lbm_mlp_deformation(self._h, x.data_ptr(), int(x.shape[0]), m6.data_ptr(), D.data_ptr()),
               "lbm_mlp_deformation")

    def gradients(self, x, t):
        """(loss, flat gradients) of a batch, without an update."""
        loss = np.zeros(1)
        g = np.zeros(self.param_count(), dtype=np.float32)
        _check(self._lib.lbm_mlp_gradients(self._h, x.data_ptr(), t.data_ptr(), int(x.shape[0]), _dptr(loss),
                                           _fptr(g)), "lbm_mlp_gradients")
        return float(loss[0]), g

    def train_step(self, x, t, lr, want_loss=False):
        loss = np.zeros(1) if want_loss else None
        _check(self._lib.lbm_mlp_train_step(self._h, x.data_ptr(), t.data_ptr(), int(x.shape[0]), ctypes.c_float(lr),
                                            _dptr(loss)), "lbm_mlp_train_step")
        return float(loss[0]) if want_loss else None

    def sync(self):
        _check(self._lib.lbm_mlp_sync(self._h), "lbm_mlp_sync")

    def set_tensor_path(self, path):
        """0: tcgen05 tensor cores where the shape allows (default); 1: mma.sync only."""
        _check(self._lib.lbm_mlp_set_tensor_path(self._h, int(path)), "lbm_mlp_set_tensor_path")


def selftest_wait(limit_ns, arrive=False, device=-1):
    """Status of lbm_selftest_wait: LBM_ETIMEOUT (-6) when nothing arrives and
    the bounded device-side wait gives up after limit_ns, 0 when it completes."""
    return int(load_library().lbm_selftest_wait(int(limit_ns), 1 if arrive else 0, int(device)))


def mm_integrate(A, tau_d, chi, substeps=10, record_every=1, precision="fp64", want_M=False, stream=None):
    """Maffettone-Minale D(t) of many trajectories on the GPU (lbm_mm_integrate).

    ``A`` is a torch CUDA float64 tensor [T, n, 9]; returns torch CUDA tensors
    D [floor((T-1)/record_every) + 1, n] and, if want_M, M [n, 6]."""
    import torch

    lib = load_library()
    T, n = int(A.shape[0]), int(A.shape[1])
    A = A.contiguous()
    D = torch.empty(((T - 1) // record_every + 1, n), dtype=torch.float64, device=A.device)
    M = torch.empty((n, 6), dtype=torch.float64, device=A.device) if want_M else None
    if stream is None:
        stream = torch.cuda.current_stream(A.device).cuda_stream
    _check(lib.lbm_mm_integrate(A.data_ptr(), T, n, float(tau_d), float(chi), int(substeps), int(record_every),
                                PRECISIONS[precision], D.data_ptr(), None if M is None else M.data_ptr(), stream),
           "lbm_mm_integrate")
    return (D, M) if want_M else D
