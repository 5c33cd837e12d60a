"""FP64 CPU oracle of the planar WCSPH hydrodynamic-ram step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2609_05494_b300``) and never imports it; the two meet only in the
seeded inputs of ``casegen``.

The arithmetic lives in ``hram_oracle.c`` (plain C, double precision); this
module compiles it with gcc on first use and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hram_oracle.c")
_LIB = os.path.join(_HERE, "libhram_oracle.so")
_lock = threading.Lock()
_lib = None

N_PROBE_MAX = 16

MUT = dict(ghost_printed_sign=1, drop_pj=2, kernel_norm=4, av_sign=8, dt_no_ghosts=16,
           grad_sign=32, ghost_vel=64, energy_half=128, sum_no_self=256, xsph_gradw=512,
           xsph_rhoj=1024, lam_half=2048, av_const_c=4096)

DIAG_FIELDS = ("mass", "px", "py", "KE", "PE", "E_el", "rho_min", "rho_max", "p_min",
               "p_max", "vmax_fluid", "n_in", "penetrated", "t", "dt", "W_boundary",
               "wall_impulse", "dissipation", "step")
SCALAR_FIELDS = ("t", "dt", "step", "xc", "yc", "vproj", "aproj", "Fdisk_x", "Fdisk_y",
                 "Fwall", "W_boundary", "wall_impulse", "dissipation", "diss_rate")


class OracleParams(C.Structure):
    _fields_ = [
        ("dx", C.c_double), ("h_over_dx", C.c_double), ("Lx", C.c_double), ("W", C.c_double),
        ("wall_layers", C.c_int32), ("end_walls", C.c_int32),
        ("R_disk", C.c_double), ("v0", C.c_double), ("tau", C.c_double), ("t_ramp", C.c_double),
        ("x_c0", C.c_double), ("y_c0", C.c_double),
        ("Ng", C.c_int32), ("motion", C.c_int32),
        ("a_const", C.c_double), ("drag_M", C.c_double), ("drag_Cd", C.c_double),
        ("drag_R", C.c_double),
        ("rho0", C.c_double), ("c0", C.c_double), ("gamma", C.c_double), ("p_cav", C.c_double),
        ("alpha", C.c_double), ("eta2", C.c_double), ("eps_xsph", C.c_double),
        ("mu_lam", C.c_double), ("gx", C.c_double), ("gy", C.c_double), ("cfl", C.c_double),
        ("dt_mode", C.c_int32), ("n_probes", C.c_int32),
        ("rho_lo", C.c_double), ("rho_hi", C.c_double), ("box_pad", C.c_double),
        ("probe_xy", C.c_double * (2 * N_PROBE_MAX)),
        ("mutation", C.c_int32), ("brute", C.c_int32),
        ("disk_density", C.c_double),
        ("closure", C.c_int32),
        ("mg_S1", C.c_double), ("mg_gamma0", C.c_double), ("mg_a", C.c_double),
        ("mg_mu_max", C.c_double),
        ("wall_reflect", C.c_int32),
    ]


def _build() -> None:
    # a per-process temporary name: processes that build at the same time
    # each write their own file, and the rename is atomic
    tmp = "%s.%d.tmp" % (_LIB, os.getpid())
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)


def build() -> str:
    """Compile the oracle library if it is missing or older than its source."""
    with _lock:
        if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            _build()
    return _LIB


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        vp = C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [P(OracleParams), C.c_int64, vp, vp, vp]
        L.orc_destroy.argtypes = [vp]
        L.orc_prime.argtypes = [vp]
        L.orc_step.argtypes = [vp]
        L.orc_run.argtypes = [vp, C.c_int64]
        for f in ("orc_n_fluid", "orc_n_wall", "orc_n_disk"):
            getattr(L, f).restype = C.c_int64
            getattr(L, f).argtypes = [vp]
        L.orc_get_fluid.argtypes = [vp] + [vp] * 8
        L.orc_get_ghosts.argtypes = [vp] + [vp] * 7
        L.orc_get_scalars.argtypes = [vp, vp]
        L.orc_probe_history.restype = C.c_int64
        L.orc_probe_history.argtypes = [vp, vp, vp, C.c_int64]
        L.orc_neighbours.restype = C.c_int64
        L.orc_neighbours.argtypes = [vp, vp, vp, C.c_int64]
        L.orc_refresh_neighbours.argtypes = [vp]
        L.orc_diagnostics.argtypes = [vp, vp]
        L.orc_brute_neighbours.restype = C.c_int64
        L.orc_brute_neighbours.argtypes = [C.c_int64, vp, C.c_float, vp, vp, C.c_int64]
        L.orc_kernel_W.restype = C.c_double
        L.orc_kernel_W.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.orc_kernel_F.restype = C.c_double
        L.orc_kernel_F.argtypes = [C.c_double, C.c_double, C.c_int32]
        L.orc_predicate32.restype = C.c_int
        L.orc_predicate32.argtypes = [C.c_float] * 5
        L.orc_kinematics.argtypes = [P(OracleParams), C.c_double, vp, vp, vp]
        L.orc_cubic_W.restype = C.c_double
        L.orc_cubic_W.argtypes = [C.c_double, C.c_double]
        L.orc_cubic_F.restype = C.c_double
        L.orc_cubic_F.argtypes = [C.c_double, C.c_double]
        L.orc_mg_p.restype = C.c_double
        L.orc_mg_p.argtypes = [P(OracleParams), C.c_double, C.c_double]
        L.orc_get_energy.argtypes = [vp, vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(d: dict, mutation: int = 0, brute: bool = False) -> OracleParams:
    """Oracle parameter struct from a casegen parameter dict."""
    p = OracleParams()
    for name, ctype in OracleParams._fields_:
        if name in ("probe_xy", "n_probes", "mutation", "brute"):
            continue
        setattr(p, name, int(d[name]) if ctype is C.c_int32 else float(d[name]))
    probes = list(d.get("probes", []))
    if len(probes) > N_PROBE_MAX:
        raise ValueError("at most %d probes" % N_PROBE_MAX)
    p.n_probes = len(probes)
    for k, (x, y) in enumerate(probes):
        p.probe_xy[2 * k] = float(x)
        p.probe_xy[2 * k + 1] = float(y)
    p.mutation = int(mutation)
    p.brute = 1 if brute else 0
    return p


class OracleCase:
    """One simulated case held by the C oracle."""

    def __init__(self, params: dict, xy: np.ndarray, vel: np.ndarray | None = None,
                 rho: np.ndarray | None = None, mutation: int = 0, brute: bool = False,
                 prime: bool = True):
        self.params = dict(params)
        self._p = make_params(params, mutation, brute)
        self._xy = np.ascontiguousarray(xy, dtype=np.float64)
        vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
        rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        L = lib()
        self._h = L.orc_create(C.byref(self._p), int(self._xy.shape[0]), _ptr(self._xy),
                               _ptr(vel), _ptr(rho))
        self.nf = L.orc_n_fluid(self._h)
        self.nw = L.orc_n_wall(self._h)
        self.nd = L.orc_n_disk(self._h)
        self.ngh = self.nw + self.nd
        if prime:
            self.prime()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def prime(self) -> None:
        lib().orc_prime(self._h)

    def step(self) -> None:
        lib().orc_step(self._h)

    def run(self, n: int) -> None:
        lib().orc_run(self._h, int(n))

    def fluid(self) -> dict:
        n = self.nf
        out = dict(xy=np.empty((n, 2)), vel=np.empty((n, 2)), rho=np.empty(n), p=np.empty(n),
                   acc=np.empty((n, 2)), drho=np.empty(n), X=np.empty((n, 2)),
                   out=np.empty(n, dtype=np.uint8))
        lib().orc_get_fluid(self._h, *(_ptr(out[k]) for k in
                                       ("xy", "vel", "rho", "p", "acc", "drho", "X", "out")))
        return out

    def energy(self) -> dict:
        """Specific internal energy e and its rate De (closure 1)."""
        n = self.nf
        out = dict(e=np.empty(n), de=np.empty(n))
        lib().orc_get_energy(self._h, _ptr(out["e"]), _ptr(out["de"]))
        return out

    def ghosts(self) -> dict:
        n = self.ngh
        out = dict(xy=np.empty((n, 2)), p=np.empty(n), rho=np.empty(n), vel=np.empty((n, 2)),
                   mass=np.empty(n), kind=np.empty(n, dtype=np.int32),
                   out=np.empty(n, dtype=np.uint8))
        lib().orc_get_ghosts(self._h, *(_ptr(out[k]) for k in
                                        ("xy", "p", "rho", "vel", "mass", "kind", "out")))
        return out

    def scalars(self) -> dict:
        s = np.empty(len(SCALAR_FIELDS))
        lib().orc_get_scalars(self._h, _ptr(s))
        return dict(zip(SCALAR_FIELDS, s.tolist()))

    def probes(self) -> tuple[np.ndarray, np.ndarray]:
        L = lib()
        n = L.orc_probe_history(self._h, None, None, 0)
        npb = self._p.n_probes
        p = np.empty((n, max(npb, 1)))
        t = np.empty(n)
        L.orc_probe_history(self._h, _ptr(p), _ptr(t), n)
        return p[:, :npb], t

    def diagnostics(self) -> dict:
        d = np.empty(len(DIAG_FIELDS))
        lib().orc_diagnostics(self._h, _ptr(d))
        return dict(zip(DIAG_FIELDS, d.tolist()))

    def neighbours(self, refresh: bool = False) -> tuple[np.ndarray, np.ndarray]:
        """CSR (offsets, ids) over all points: fluid IDs 0..nf-1, then wall
        ghosts, then disk ghosts; ids ascending within each row."""
        L = lib()
        if refresh:
            L.orc_refresh_neighbours(self._h)
        npts = self.nf + self.ngh
        off = np.empty(npts + 1, dtype=np.int64)
        n = L.orc_neighbours(self._h, _ptr(off), None, 0)
        ids = np.empty(max(n, 1), dtype=np.int32)
        L.orc_neighbours(self._h, _ptr(off), _ptr(ids), n)
        return off, ids[:n]


def brute_neighbours(xy32: np.ndarray, s2: float) -> tuple[np.ndarray, np.ndarray]:
    """O(N^2) neighbour sets of a float32 point set under the float predicate."""
    xy32 = np.ascontiguousarray(xy32, dtype=np.float32)
    n = xy32.shape[0]
    off = np.empty(n + 1, dtype=np.int64)
    L = lib()
    k = L.orc_brute_neighbours(n, _ptr(xy32), float(np.float32(s2)), _ptr(off), None, 0)
    ids = np.empty(max(k, 1), dtype=np.int32)
    L.orc_brute_neighbours(n, _ptr(xy32), float(np.float32(s2)), _ptr(off), _ptr(ids), k)
    return off, ids[:k]


def kernel_W(r: float, h: float, mutation: int = 0) -> float:
    return lib().orc_kernel_W(float(r), float(h), int(mutation))


def kernel_F(r: float, h: float, mutation: int = 0) -> float:
    """F(r) with grad_i W_ij = F(r) (r_i - r_j)."""
    return lib().orc_kernel_F(float(r), float(h), int(mutation))


def cubic_W(r: float, h: float) -> float:
    """Cubic B-spline kernel of the paper (closure 1)."""
    return lib().orc_cubic_W(float(r), float(h))


def cubic_F(r: float, h: float) -> float:
    return lib().orc_cubic_F(float(r), float(h))


def mg_p(params: dict, rho: float, e: float) -> float:
    """Mie-Grueneisen pressure of the paper's closure (with the cutoff)."""
    p = make_params(params)
    return lib().orc_mg_p(C.byref(p), float(rho), float(e))


def predicate32(xi, yi, xj, yj, s2) -> bool:
    return bool(lib().orc_predicate32(xi, yi, xj, yj, s2))


def kinematics(params: dict, t: float) -> tuple[float, float, float]:
    p = make_params(params)
    x, v, a = C.c_double(), C.c_double(), C.c_double()
    lib().orc_kinematics(C.byref(p), float(t), C.byref(x), C.byref(v), C.byref(a))
    return x.value, v.value, a.value


def support_s2(params: dict) -> float:
    """fl32((2h)^2) with 2h = 2 * h_over_dx * dx evaluated in double."""
    s = 2.0 * params["h_over_dx"] * params["dx"]
    return float(np.float32(s * s))
