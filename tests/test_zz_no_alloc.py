"""The allocation-free lambda_k entry point, iblbm_dfc_lambda_noalloc.

Some callers cannot allocate device memory at the point where they need the
DFC factors (inside frameworks that own all device memory, solvers embedded in
another application's time loop, real-time loops).  The entry point keeps its
scratch in a library-wide device array instead.  These checks call it through
the C ABI on two marker sets in a row -- the second call reuses the array the
first left behind -- and compare each result with lambda_k as the regular path
computes it (a fixed DFC body on an FP64 lattice, read back after one step) and
with the FP64 oracle's Eq. 17, within the FP64 bar of the parity suite (1e-12).
This file is collected last."""
import ctypes as C

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_02298_b300 as L  # noqa: E402

TOL = 1e-12


def _regular_lambda(xy, ds, kernel, nx, ny, xc, yc, radius):
    lat = L.Lattice(nx, ny, collision=L.BGK, tau=0.8, storage=L.F64)
    b = lat.add_body(xy, ds, kernel, L.DFC, xc=xc, yc=yc, radius=radius)
    lat.step(1)
    lam = lat.marker_data(b)[:, 6].copy()
    lat.close()
    return lam


def _noalloc_lambda(xy, ds, kernel, nx, ny):
    xy_d = torch.tensor(np.ascontiguousarray(xy).ravel(), dtype=torch.float64, device="cuda")
    lam_d = torch.full((len(xy),), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.load_library().iblbm_dfc_lambda_noalloc(C.c_void_p(xy_d.data_ptr()), len(xy), ds, kernel, nx, ny,
                                                   C.c_void_p(lam_d.data_ptr()), C.c_void_p(stream))
    return rc, lam_d.cpu().numpy()


CASES = [  # (lattice, centre, diameter, markers, kernel): two different sets, called back to back
    ((64, 64), (32.0, 32.0), 20.0, 94, W.HAT),
    ((160, 120), (71.3, 58.6), 40.0, 188, W.PESKIN4),
]


def test_noalloc_lambda_matches_regular_path_on_consecutive_calls():
    ref = []
    for (nx, ny), (xc, yc), D, n, kernel in CASES:
        xy, ds = W.circle_markers(xc, yc, D, n)
        ref.append((xy, ds, kernel, nx, ny, _regular_lambda(xy, ds, kernel, nx, ny, xc, yc, 0.5 * D)))
    for xy, ds, kernel, nx, ny, lam_ref in ref:      # two calls in a row, sharing the scratch array
        rc, lam = _noalloc_lambda(xy, ds, kernel, nx, ny)
        assert rc == 0, L.strerror(rc)
        assert np.all(np.isfinite(lam))
        assert np.abs(lam - lam_ref).max() < TOL * np.abs(lam_ref).max()
        lam_orc = oracle.dfc_lambda(kernel, xy, ds, nx, ny)
        assert np.abs(lam - lam_orc).max() < TOL * np.abs(lam_orc).max()


def test_noalloc_lambda_skewed_box_matches_oracle():
    """A marker set whose bounding box is one stencil wide and thousands of nodes
    tall (a vertical line of markers), so the W_total pass walks many tiles."""
    n, nx, ny = 3000, 40, 3200
    xy = np.stack([np.full(n, 20.37), 50.0 + 1.01 * np.arange(n)], axis=1)
    for kernel in (W.HAT, W.PESKIN4):
        rc, lam = _noalloc_lambda(xy, 1.01, kernel, nx, ny)
        assert rc == 0, L.strerror(rc)
        lam_orc = oracle.dfc_lambda(kernel, xy, 1.01, nx, ny)
        assert np.abs(lam - lam_orc).max() < TOL * np.abs(lam_orc).max()


def test_noalloc_lambda_rejects_oversized_box():
    xy, ds = W.circle_markers(400.0, 400.0, 600.0, 1885)     # box about 604 x 604 > 512 x 512
    rc, lam = _noalloc_lambda(xy, ds, W.PESKIN4, 800, 800)
    assert rc == -11, L.strerror(rc)                          # IBLBM_ERR_CAPACITY
    rc, _ = _noalloc_lambda(xy[:10] - 399.5, ds, W.PESKIN4, 800, 800)
    assert rc == -4, L.strerror(rc)                           # footprint outside the lattice
    # and the entry point still works afterwards
    (nx, ny), (xc, yc), D, n, kernel = CASES[0]
    xy, ds = W.circle_markers(xc, yc, D, n)
    rc, lam = _noalloc_lambda(xy, ds, kernel, nx, ny)
    assert rc == 0
    np.testing.assert_allclose(lam, _regular_lambda(xy, ds, kernel, nx, ny, xc, yc, 0.5 * D), rtol=TOL, atol=0)
