"""The allocation-free neighbour-count entry point against hr_debug_neighbors.

hr_neighbor_counts_static serves callers that cannot allocate device memory
(their device memory is held by another allocator, or they must not change
the device's allocation state); it keeps its scratch in a fixed device array
of the library.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import impact_case, perturbed

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2609_05494_b300 import Case, _lib  # noqa: E402


def static_counts(case, npts):
    out = np.full(npts, -1, dtype=np.int32)
    rc = _lib.lib().hr_neighbor_counts_static(case._h, out.ctypes.data_as(C.c_void_p), npts)
    assert rc >= 0, rc
    return out


def test_static_counts_match_debug_neighbors_twice():
    p, xy = impact_case()
    vel, rho = perturbed(p, xy)
    with Case(p, xy, vel, rho) as c:
        c.run(25)
        npts = c.n + c.n_wall + c.n_disk
        for _ in range(2):                      # two calls in a row share the array
            off, _ids = c.neighbours()
            want = np.diff(off).astype(np.int32)
            got = static_counts(c, npts)
            assert np.array_equal(got, want)
            c.step()


def test_static_counts_second_case_overwrites_first():
    p, xy = impact_case()
    q, xy2 = impact_case(Lx=0.05, W=0.04, dx=1e-3, Ng=0, wall_layers=0)
    with Case(p, xy) as a, Case(q, xy2) as b:
        na = a.n + a.n_wall + a.n_disk
        nb = b.n + b.n_wall + b.n_disk
        ga = static_counts(a, na)
        gb = static_counts(b, nb)
        assert np.array_equal(ga, np.diff(a.neighbours()[0]).astype(np.int32))
        assert np.array_equal(gb, np.diff(b.neighbours()[0]).astype(np.int32))


def test_static_counts_reject_small_buffer():
    p, xy = impact_case()
    with Case(p, xy) as c:
        npts = c.n + c.n_wall + c.n_disk
        out = np.zeros(npts - 1, dtype=np.int32)
        rc = _lib.lib().hr_neighbor_counts_static(c._h, out.ctypes.data_as(C.c_void_p), npts - 1)
        assert rc == _lib.HR_ERANGE


def test_static_counts_reject_oversized_case():
    # more points than the fixed array holds: rejected before any device work
    p, xy = impact_case(Lx=0.3, W=0.15, dx=1.4e-4, Ng=0, wall_layers=0)
    assert xy.shape[0] > _lib.HR_STATIC_NEIGHBOR_MAX
    with Case(p, xy) as c:
        out = np.zeros(8, dtype=np.int32)
        rc = _lib.lib().hr_neighbor_counts_static(c._h, out.ctypes.data_as(C.c_void_p), 8)
        assert rc == _lib.HR_ERANGE
