"""ctypes front end of the FP64 oracle (test infrastructure only).

Wraps ``lbm_oracle.cpp``: a plain CPU implementation of the two-component
Shan-Chen lattice Boltzmann step with exact-flow ghost boundaries (Sec. 2,
Eqs. 6-10; Sec. 3, Eq. 14).  Population arrays are float64 with layout
``[component][direction][z][y][x]``, component 0 = A (droplet), 1 = B
(solvent); the direction order is the D3Q19 order of ``lbm_oracle.cpp``.
"""

import ctypes

import numpy as np

from . import build as _build

_DP = ctypes.POINTER(ctypes.c_double)
_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 5
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_set_populations.argtypes = [ctypes.c_void_p, _DP]
        lib.orc_get_populations.argtypes = [ctypes.c_void_p, _DP]
        lib.orc_init_droplet.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 4 + [_DP]
        lib.orc_step.argtypes = [ctypes.c_void_p, _DP, _DP, _DP, _DP]
        lib.orc_fields.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
        lib.orc_checksums.argtypes = [ctypes.c_void_p, _DP, _DP]
        lib.orc_moments.argtypes = [ctypes.c_void_p, _DP]
        lib.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3 + [_DP]
        lib.orc_equilibrium.restype = ctypes.c_double
        lib.orc_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, _DP]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_storage.restype = ctypes.c_int
        lib.orc_set_storage.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_set_mrt.argtypes = [ctypes.c_void_p, ctypes.c_int, _DP]
        lib.orc_moment_basis.argtypes = [_DP]
        lib.orc_round.restype = ctypes.c_double
        lib.orc_round.argtypes = [ctypes.c_int, ctypes.c_double]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


STORAGE = {"exact": 0, "fp16dev": 1, "bf16dev": 2}
ROUND_FORMATS = {"float32": 0, "binary16": 1, "bfloat16": 2}


def round_to(fmt: str, x: float) -> float:
    """x rounded to nearest-even in ``fmt`` ("float32", "binary16", "bfloat16"):
    the rounding of the oracle's storage model."""
    return float(_load().orc_round(ROUND_FORMATS[fmt], float(x)))


# d'Humieres et al. (2002) rates for (s_e, s_eps, s_q, s_pi, s_m)
MRT_RATES = (1.19, 1.4, 1.2, 1.4, 1.98)


def moment_basis():
    """The oracle's D3Q19 moment basis M [19, 19] (row k, direction i)."""
    M = np.zeros(19 * 19)
    _load().orc_moment_basis(_ptr(M))
    return M.reshape(19, 19)


def set_threads(n: int) -> int:
    """Thread count of the oracle's OpenMP node loops (results do not depend on it).

    ``n <= 0`` leaves it unchanged; returns the count in effect."""
    return int(_load().orc_set_threads(int(n)))


def lattice():
    """The oracle's D3Q19 table: (c [19,3] int, w [19] float64)."""
    lib = _load()
    cx = (ctypes.c_int * 19)()
    cy = (ctypes.c_int * 19)()
    cz = (ctypes.c_int * 19)()
    w = np.zeros(19)
    lib.orc_lattice(cx, cy, cz, _ptr(w))
    c = np.stack([np.array(cx[:]), np.array(cy[:]), np.array(cz[:])], axis=1)
    return c, w


def equilibrium(i: int, rho: float, u) -> float:
    """Eq. 8 for one direction, as the oracle evaluates it."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    return _load().orc_equilibrium(int(i), float(rho), _ptr(uu))


def gradient_at(t: float, knots_t, knots_A) -> np.ndarray:
    """A(t) from a knot table: linear between knots, held constant outside.

    This is the reading adopted for the paper's gradient "sampling time"
    (Sec. 4): one sample of G_ij every Delta t steps, the boundary driven by
    the piecewise-linear signal through the samples.
    """
    kt = np.asarray(knots_t, dtype=np.float64)
    kA = np.asarray(knots_A, dtype=np.float64).reshape(-1, 9)
    if kt.size == 0:
        return np.zeros(9)
    return np.array([np.interp(t, kt, kA[:, j]) for j in range(9)])


class OracleLBM:
    """FP64 two-component Shan-Chen LBM on an Lx x Ly x Lz box.

    ``periodic=False`` is the paper's setup: ghost nodes one layer outside the
    box hold g^eq(rho_b, A(t) x) (Sec. 2, Eq. 8; Sec. 3, Eq. 14).
    ``periodic=True`` is a test mode with no boundary at all.

    ``frame="droplet"`` measures x in the ghost flow A(t) x from the droplet's
    centre of mass (the frame of Sec. 3, Eq. 14: "the droplet's centre of mass
    remains fixed ... linear in the distance from the droplet's centre of
    mass"), recomputed from the stored populations before every step;
    ``frame="box"`` measures it from the box centre.

    ``mrt`` (rates s_e, s_eps, s_q, s_pi, s_m, e.g. ``MRT_RATES``) selects
    the multi-relaxation-time collision of ``lbm_oracle.cpp`` instead of BGK.

    ``storage`` selects the storage model of ``lbm_oracle.cpp``: "exact"
    (full precision, the paper's method), or "fp16dev" / "bf16dev": after
    every state change the populations are replaced by the values 16-bit
    deviation storage holds (float32 densities, deviations from w_i rho* of
    the destination node rounded to binary16 / bfloat16, float32 rest
    population closing each node's mass).
    """

    def __init__(self, box, tau, G, rho_b, periodic=False, frame="droplet", storage="exact", mrt=None):
        self.box = tuple(int(v) for v in box)
        self.nodes = self.box[0] * self.box[1] * self.box[2]
        self.tau = (float(tau[0]), float(tau[1]))
        self.G = float(G)
        self.rho_b = (float(rho_b[0]), float(rho_b[1]))
        self.periodic = bool(periodic)
        if frame not in ("droplet", "box"):
            raise ValueError(frame)
        self.frame = frame
        self._lib = _load()
        self._h = self._lib.orc_create(
            self.box[0], self.box[1], self.box[2], int(self.periodic),
            self.tau[0], self.tau[1], self.G, self.rho_b[0], self.rho_b[1])
        self.storage = storage
        if self._lib.orc_set_storage(self._h, STORAGE[storage]) != 0:
            raise ValueError(storage)
        # mrt: None for BGK, or the rates (s_e, s_eps, s_q, s_pi, s_m) of the MRT operator
        self.mrt = None if mrt is None else tuple(float(v) for v in mrt)
        if self.mrt is not None:
            r = np.ascontiguousarray(self.mrt, dtype=np.float64)
            self._lib.orc_set_mrt(self._h, 1, _ptr(r))
        self.step_count = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def shape(self):
        Lx, Ly, Lz = self.box
        return (2, 19, Lz, Ly, Lx)

    def init_droplet(self, R, xi, rho_hi, rho_lo, A0=None):
        A = np.zeros(9) if A0 is None else np.ascontiguousarray(np.asarray(A0, dtype=np.float64).reshape(9))
        self._lib.orc_init_droplet(self._h, float(R), float(xi), float(rho_hi), float(rho_lo), _ptr(A))
        self.step_count = 0

    def set_populations(self, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.shape))
        self._lib.orc_set_populations(self._h, _ptr(f))

    def populations(self) -> np.ndarray:
        f = np.zeros(self.shape)
        self._lib.orc_get_populations(self._h, _ptr(f))
        return f

    def centre_of_mass(self):
        """Centre of mass of w = max(phi, 0) of the stored populations (box-centred
        coordinates); the box centre (0, 0, 0) when there is no droplet (sum w = 0)."""
        m = self.moments()
        if not m[0] > 0.0:
            return np.zeros(3)
        return m[1:4] / m[0]

    def step(self, A=None, fluxes=False):
        """One step with boundary gradient A (row-major A[a,b] = d_b u_a)."""
        A = np.zeros(9) if A is None else np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
        c = None
        if self.frame == "droplet" and not self.periodic:
            c = np.ascontiguousarray(self.centre_of_mass())
        cp = None if c is None else _ptr(c)
        if fluxes:
            fin = np.zeros(2)
            fout = np.zeros(2)
            self._lib.orc_step(self._h, _ptr(A), cp, _ptr(fin), _ptr(fout))
            self.step_count += 1
            return fin, fout
        self._lib.orc_step(self._h, _ptr(A), cp, None, None)
        self.step_count += 1
        return None

    def run(self, n, knots_t=(), knots_A=()):
        """n steps; step k uses A(t_k), t_k the running step counter."""
        for _ in range(int(n)):
            self.step(gradient_at(self.step_count, knots_t, knots_A))

    def fields(self):
        """(rho_A, rho_B, u[...,3]) of the stored populations (Eq. 6), shaped [z,y,x]."""
        Lx, Ly, Lz = self.box
        ra = np.zeros(self.nodes)
        rb = np.zeros(self.nodes)
        u = np.zeros(3 * self.nodes)
        self._lib.orc_fields(self._h, _ptr(ra), _ptr(rb), _ptr(u))
        return ra.reshape(Lz, Ly, Lx), rb.reshape(Lz, Ly, Lx), u.reshape(Lz, Ly, Lx, 3)

    def checksums(self):
        mass = np.zeros(2)
        mom = np.zeros(3)
        self._lib.orc_checksums(self._h, _ptr(mass), _ptr(mom))
        return mass, mom

    def moments(self) -> np.ndarray:
        out = np.zeros(10)
        self._lib.orc_moments(self._h, _ptr(out))
        return out
