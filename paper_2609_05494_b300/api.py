"""Python interface of the B300 planar WCSPH hydrodynamic-ram library.

:class:`Case` wraps one ``hr_case`` of the C-ABI (include/hram.h).  PyTorch is
used only for device memory (the case's workspace) and the CUDA stream; all
arithmetic of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import HrDiag, HrParams, check, lib

DIAG_FIELDS = tuple(n for n, _ in HrDiag._fields_)
SCALAR_FIELDS = ("t", "dt", "step", "xc", "yc", "vproj", "aproj", "Fdisk_x", "Fdisk_y",
                 "Fwall", "W_boundary", "wall_impulse", "dissipation", "diss_rate")
KERNEL_GROUPS = ("drift", "sort", "ghost", "pass", "finalize")
TANGENT_PARAMS = ("alpha", "c0", "tau")


def make_params(d: dict, flags: int = 0, probe_capacity: int = 1 << 16,
                diag_every: int = 0) -> HrParams:
    """C parameter struct from a parameter dict (keys as in casegen)."""
    p = HrParams()
    skip = ("probe_xy", "n_probes", "probe_capacity", "diag_every", "flags")
    for name, ctype in HrParams._fields_:
        if name in skip:
            continue
        setattr(p, name, int(d[name]) if ctype in (C.c_int32, C.c_int64) else float(d[name]))
    probes = list(d.get("probes", []))
    if len(probes) > _lib.MAX_PROBES:
        raise ValueError("at most %d probes" % _lib.MAX_PROBES)
    p.n_probes = len(probes)
    for k, (x, y) in enumerate(probes):
        p.probe_xy[2 * k] = float(x)
        p.probe_xy[2 * k + 1] = float(y)
    p.probe_capacity = int(probe_capacity)
    p.diag_every = int(diag_every)
    p.flags = int(flags)
    return p


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Case:
    """One simulated case on the GPU.

    params: dict of parameters (see casegen.base_params); xy: (N, 2) initial
    positions in fluid-ID order; vel (N, 2) / rho (N,) optional.  The device
    workspace is a torch uint8 tensor unless ``torch_workspace`` is False, in
    which case the library allocates it.  ``stage`` picks the interaction
    pass variant: 0 reads candidates from global memory, 1 stages the
    candidates' positions in shared memory, 2 their whole records (the
    results are identical).  ``newton3`` evaluates every fluid pair once,
    ``lanes`` (2 or 4) splits each particle's pass work over that many lanes
    (results equal to rounding).  ``split`` runs the interaction pass as
    interior and boundary kernels beside the ghost pass (True), never
    (False), or by the library's size rule (None); results are identical.
    ``close_inline`` closes every step (partial sums, probes, FP64
    accumulators, CFL gate) inside its own step graph instead of beside the
    next step's drift; results are identical.
    """

    def __init__(self, params: dict, xy, vel=None, rho=None, stream=None, timing: bool = False,
                 probe_capacity: int = 1 << 16, diag_every: int = 0, torch_workspace: bool = True,
                 tangent: bool = False, stage: int = 0, newton3: bool = False,
                 lanes: int = 1, split: bool | None = None, close_inline: bool = False):
        L = lib()
        xy = _f32(xy)
        n = xy.shape[0]
        if xy.shape != (n, 2):
            raise ValueError("xy must be (N, 2)")
        self.n = n
        self.params = dict(params)
        flags = (_lib.HR_FLAG_TIMING if timing else 0) | (_lib.HR_FLAG_TANGENT if tangent else 0)
        if stage not in (0, 1, 2):
            raise ValueError("stage must be 0, 1 or 2")
        flags |= (0, _lib.HR_FLAG_STAGE_POS, _lib.HR_FLAG_STAGE_ALL)[stage]
        if newton3:
            flags |= _lib.HR_FLAG_NEWTON3
        if lanes not in (1, 2, 4):
            raise ValueError("lanes must be 1, 2 or 4")
        flags |= {1: 0, 2: _lib.HR_FLAG_PASS_LANES2, 4: _lib.HR_FLAG_PASS_LANES4}[lanes]
        if split is not None:
            flags |= _lib.HR_FLAG_PASS_SPLIT if split else _lib.HR_FLAG_PASS_FUSED
        if close_inline:
            flags |= _lib.HR_FLAG_CLOSE_INLINE
        self._p = make_params(params, flags, probe_capacity, diag_every)
        self.n_probes = self._p.n_probes
        nbytes = C.c_size_t(0)
        check(L.hr_workspace_bytes(C.byref(self._p), n, C.byref(nbytes)), "hr_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self._ws = None
        ws_ptr = None
        if torch_workspace:
            import torch
            self._ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
            ws_ptr = self._ws.data_ptr()
        self._stream = _stream_handle(stream)
        h = C.c_void_p()
        rc = L.hr_init_case(C.byref(self._p), _ptr(xy), n, _ptr(_f32(vel, (n, 2))),
                            _ptr(_f32(rho, (n,))), ws_ptr, nbytes.value, self._stream, C.byref(h))
        check(rc, "hr_init_case")
        self._h = h
        self.last_status = rc
        info = self.info()
        self.n_wall, self.n_disk = info["n_wall"], info["n_disk"]

    # -- lifecycle
    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h:
            lib().hr_destroy(h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping
    def step(self) -> int:
        self.last_status = check(lib().hr_step(self._h), "hr_step")
        return self.last_status

    def run(self, n_steps: int, t_end: float = 0.0) -> int:
        self.last_status = check(lib().hr_run(self._h, int(n_steps), float(t_end)), "hr_run")
        return self.last_status

    def sync(self) -> int:
        self.last_status = check(lib().hr_sync(self._h), "hr_sync")
        return self.last_status

    # -- outputs
    def probe_pressure(self, out: np.ndarray | None = None) -> np.ndarray:
        """Probe history [steps, n_probes] (float32).  ``out``: a caller-owned
        C-contiguous float32 buffer (for instance pinned) with room for at
        least the recorded rows; the filled rows are returned as a view."""
        L = lib()
        n = C.c_int64(0)
        check(L.hr_probe_pressure(self._h, None, 0, C.byref(n)), "hr_probe_pressure")
        width = max(self.n_probes, 1)
        if out is None:
            out = np.zeros((n.value, width), dtype=np.float32)
        elif (out.dtype != np.float32 or not out.flags.c_contiguous or out.ndim != 2
              or out.shape[1] != width or out.shape[0] < n.value):
            raise ValueError("out must be C-contiguous float32 of shape (>= %d, %d)"
                             % (n.value, width))
        check(L.hr_probe_pressure(self._h, _ptr(out), out.shape[0], C.byref(n)),
              "hr_probe_pressure")
        return out[:n.value, :self.n_probes]

    def probe_times(self) -> np.ndarray:
        L = lib()
        n = C.c_int64(0)
        check(L.hr_probe_times(self._h, None, 0, C.byref(n)), "hr_probe_times")
        out = np.zeros(n.value, dtype=np.float64)
        check(L.hr_probe_times(self._h, _ptr(out), n.value, C.byref(n)), "hr_probe_times")
        return out

    def diagnostics(self) -> dict:
        d = HrDiag()
        check(lib().hr_diagnostics(self._h, C.byref(d)), "hr_diagnostics")
        return {k: getattr(d, k) for k in DIAG_FIELDS}

    def diag_history(self) -> np.ndarray:
        L = lib()
        n = C.c_int64(0)
        check(L.hr_diag_history(self._h, None, 0, C.byref(n)), "hr_diag_history")
        out = np.zeros((n.value, len(DIAG_FIELDS)))
        check(L.hr_diag_history(self._h, _ptr(out), n.value, C.byref(n)), "hr_diag_history")
        return out

    def get_state(self, out: dict | None = None) -> dict:
        """Fluid state in ID order.  ``out``: caller-owned float32 arrays
        xy (N, 2), vel (N, 2), rho (N,), p (N,) (for instance pinned), filled
        in place."""
        n = self.n
        if out is None:
            out = dict(xy=np.empty((n, 2), np.float32), vel=np.empty((n, 2), np.float32),
                       rho=np.empty(n, np.float32), p=np.empty(n, np.float32))
        else:
            shapes = dict(xy=(n, 2), vel=(n, 2), rho=(n,), p=(n,))
            for k, shp in shapes.items():
                a = out[k]
                if a.dtype != np.float32 or a.shape != shp or not a.flags.c_contiguous:
                    raise ValueError("out[%r] must be C-contiguous float32 %s" % (k, shp))
        check(lib().hr_get_state(self._h, _ptr(out["xy"]), _ptr(out["vel"]), _ptr(out["rho"]),
                                 _ptr(out["p"]), n), "hr_get_state")
        return out

    def energy(self) -> dict:
        """Internal energy e and its rate De in ID order (closure 1)."""
        n = self.n
        out = dict(e=np.empty(n, np.float32), de=np.empty(n, np.float32))
        check(lib().hr_get_energy(self._h, _ptr(out["e"]), _ptr(out["de"]), n), "hr_get_energy")
        return out

    def set_state(self, xy, vel=None, rho=None) -> int:
        n = self.n
        self.last_status = check(lib().hr_set_state(self._h, _ptr(_f32(xy, (n, 2))),
                                                    _ptr(_f32(vel, (n, 2))),
                                                    _ptr(_f32(rho, (n,))), n), "hr_set_state")
        return self.last_status

    def ghosts(self) -> dict:
        g = self.n_wall + self.n_disk
        out = dict(xy=np.empty((g, 2), np.float32), p=np.empty(g, np.float32),
                   rho=np.empty(g, np.float32), vel=np.empty((g, 2), np.float32))
        check(lib().hr_get_ghosts(self._h, _ptr(out["xy"]), _ptr(out["p"]), _ptr(out["rho"]),
                                  _ptr(out["vel"]), g), "hr_get_ghosts")
        return out

    def scalars(self) -> dict:
        s = np.empty(len(SCALAR_FIELDS))
        check(lib().hr_get_scalars(self._h, _ptr(s), len(SCALAR_FIELDS)), "hr_get_scalars")
        return dict(zip(SCALAR_FIELDS, s.tolist()))

    def info(self) -> dict:
        v = np.empty(8, dtype=np.int64)
        check(lib().hr_case_info(self._h, _ptr(v), 8), "hr_case_info")
        return dict(zip(("n_fluid", "n_wall", "n_disk", "ncx", "ncy", "pass_blocks", "split",
                         "close_deferred"), (int(x) for x in v)))

    def neighbours(self) -> tuple[np.ndarray, np.ndarray]:
        """CSR over all points (fluid IDs, wall ghosts, disk ghosts), ids ascending."""
        L = lib()
        npts = self.n + self.n_wall + self.n_disk
        off = np.empty(npts + 1, dtype=np.int64)
        n = C.c_int64(0)
        check(L.hr_debug_neighbors(self._h, _ptr(off), None, 0, C.byref(n)), "hr_debug_neighbors")
        ids = np.empty(max(n.value, 1), dtype=np.int32)
        check(L.hr_debug_neighbors(self._h, _ptr(off), _ptr(ids), n.value, C.byref(n)),
              "hr_debug_neighbors")
        return off, ids[:n.value]

    def kernel_times(self) -> dict:
        ms = np.zeros(len(KERNEL_GROUPS), dtype=np.float32)
        check(lib().hr_kernel_times(self._h, _ptr(ms), len(KERNEL_GROUPS)), "hr_kernel_times")
        return dict(zip(KERNEL_GROUPS, ms.tolist()))

    def tangent_outputs(self) -> dict:
        """Peak probe-0 pressure and wall impulse with their derivatives along
        ln alpha, ln c0, ln tau (a case made with tangent=True)."""
        v = np.empty(9)
        self.last_status = check(lib().hr_tangent_outputs(self._h, _ptr(v), 9),
                                 "hr_tangent_outputs")
        return dict(peak=float(v[0]), dpeak=v[1:4].copy(), impulse=float(v[4]),
                    dimpulse=v[5:8].copy(), peak_row=int(v[8]))

    def adjoint_forward(self, n_steps: int, checkpoint_every: int = 20) -> dict:
        """Reverse mode, forward half: n_steps steps from the uploaded state
        with a checkpoint every checkpoint_every steps; the peak probe-0
        pressure, the wall impulse and the peak's history row."""
        v = np.empty(3)
        self.last_status = check(lib().hr_adjoint_forward(self._h, int(n_steps),
                                                          int(checkpoint_every), _ptr(v), 3),
                                 "hr_adjoint_forward")
        return dict(peak=float(v[0]), impulse=float(v[1]), peak_row=int(v[2]))

    def adjoint_backward(self) -> dict:
        """Reverse mode, backward half: the derivatives of the peak and the
        impulse along ln alpha, ln c0, ln tau by the reverse sweep with
        recomputation from the checkpoints."""
        v = np.empty(6)
        self.last_status = check(lib().hr_adjoint_backward(self._h, _ptr(v), 6),
                                 "hr_adjoint_backward")
        return dict(dpeak=v[0:3].copy(), dimpulse=v[3:6].copy())

    def save(self, path: str) -> None:
        check(lib().hr_save_state(self._h, str(path).encode()), "hr_save_state")

    def load(self, path: str) -> None:
        check(lib().hr_load_state(self._h, str(path).encode()), "hr_load_state")


class Batch:
    """Several cases advanced together up to simulated time t_end: one launch
    per kernel per step covers every case (each keeps its own grid, dt,
    probes and diagnostics).  The cases stay usable on their own."""

    SCHEDULES = ("case-major", "round-robin", "largest-first")

    def __init__(self, cases, t_end: float, stream=None, schedule: int = 0,
                 persistent: bool = False, case_blocks=None, spin_limit: int = 0):
        """persistent=True: the whole sweep as one persistent launch
        (hr_batch_create_persistent) with case_blocks[k] resident blocks for
        case k (None: in proportion to the particle counts) and barrier
        waits that give up after spin_limit polls (0: the library's default)."""
        L = lib()
        self.cases = list(cases)
        self.schedule = int(schedule)
        self.persistent = bool(persistent)
        arr = (C.c_void_p * len(self.cases))(*[c._h for c in self.cases])
        h = C.c_void_p()
        st = _stream_handle(stream) if stream is not None else self.cases[0]._stream
        if self.persistent:
            blocks = None
            if case_blocks is not None:
                cb = np.ascontiguousarray(case_blocks, dtype=np.int32)
                if cb.shape != (len(self.cases),):
                    raise ValueError("case_blocks needs one entry per case")
                blocks = cb
            check(L.hr_batch_create_persistent(arr, len(self.cases), float(t_end),
                                               None if blocks is None else _ptr(blocks),
                                               int(spin_limit), st, C.byref(h)),
                  "hr_batch_create_persistent")
        else:
            check(L.hr_batch_create(arr, len(self.cases), float(t_end), self.schedule, st,
                                    C.byref(h)), "hr_batch_create")
        self._h = h
        self.steps = 0

    @staticmethod
    def capacity(closure: int = 0) -> int:
        """Resident blocks a persistent batch may use on this device."""
        n = C.c_int32(0)
        check(lib().hr_persist_capacity(int(closure), C.byref(n)), "hr_persist_capacity")
        return n.value

    def step(self) -> None:
        check(lib().hr_batch_step(self._h), "hr_batch_step")

    def run(self, max_steps: int = 0) -> int:
        n = C.c_int64(0)
        st = check(lib().hr_batch_run(self._h, int(max_steps), C.byref(n)), "hr_batch_run")
        self.steps += n.value
        return st

    def n_done(self) -> int:
        n = C.c_int(0)
        check(lib().hr_batch_done(self._h, C.byref(n)), "hr_batch_done")
        return n.value

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h:
            lib().hr_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fp32_rate(packed: bool = False, stream=None) -> float:
    """Measured FP32 FMA rate of the current device, TFLOP/s (FMA = 2): the
    ALU roof of the interaction pass (scalar or packed f32x2 FMAs)."""
    out = C.c_double(0.0)
    check(lib().hr_fp32_rate(1 if packed else 0, _stream_handle(stream), C.byref(out)),
          "hr_fp32_rate")
    return out.value
