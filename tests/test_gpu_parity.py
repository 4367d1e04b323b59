"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars: streaming permutations and stencil indices bit-exact; FP64 storage within
1e-12 relative L2 (populations and velocity); FP32 (shifted) storage within
1e-5 relative L2 on velocity and 1e-4 relative on drag and lift; FP16 shifted
storage within the bound derived from its unit round-off (see test)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from harness import (EX, EY, W9, channel_spec, cylinder_body, gpu_case, oracle_case, rel_l2,
                     velocity)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_02298_b300 as L  # noqa: E402

L.use_torch_allocator()

F64_TOL = 1e-12


def _dev(f, f0):
    """Deviation of populations from the rest weights (what carries the flow)."""
    return f - W9[:, None, None]


# ---------------------------------------------------------------- streaming, bit-exact
@pytest.mark.parametrize("storage,dt", [(W.F64, np.float64), (W.F32, np.float32), (W.F16S, np.float16)])
@pytest.mark.parametrize("nx,ny", [(7, 7), (37, 11), (300, 5)])
def test_streaming_bit_exact(storage, dt, nx, ny):
    f0 = W.random_populations(11, nx, ny)
    spec = W.CaseSpec(name="s", nx=nx, ny=ny, bc=(W.PERIODIC,) * 4, ubc=((0, 0),) * 4,
                      collision=W.STREAM_ONLY, tau=0.8, storage=storage)
    g = gpu_case(spec)
    g.set_populations(f0)
    stored0 = g.populations(shifted=True)
    np.testing.assert_array_equal(stored0, (f0 - W9[:, None, None]).astype(dt).astype(np.float64))
    c = oracle_case(spec)
    c.set_populations(stored0)   # the permutation is value-blind: feed it the stored values
    g.step(1)
    c.step(1)
    np.testing.assert_array_equal(g.populations(shifted=True), c.populations())
    g.step(math.lcm(nx, ny) - 1)          # every population back at its start
    np.testing.assert_array_equal(g.populations(shifted=True), stored0)


# ---------------------------------------------------------------- collision on periodic lattices
@pytest.mark.parametrize("collision", [W.BGK, W.TRT, W.CMMRT])
def test_periodic_collision_f64(collision):
    nx, ny = 70, 23
    f0 = W.random_populations(12, nx, ny, amp=0.05)
    spec = W.CaseSpec(name="p", nx=nx, ny=ny, bc=(W.PERIODIC,) * 4, ubc=((0, 0),) * 4,
                      collision=collision, tau=0.73, storage=W.F64, trt_lambda=3 / 16)
    g, c = gpu_case(spec), oracle_case(spec)
    g.set_populations(f0)
    c.set_populations(f0)
    g.step(25)
    c.step(25)
    fg, fc = g.populations(), c.populations()
    assert rel_l2(_dev(fg, f0), _dev(fc, f0)) < F64_TOL
    assert rel_l2(velocity(fg)[0], velocity(fc)[0]) < F64_TOL


@pytest.mark.parametrize("collision", [W.BGK, W.TRT, W.CMMRT])
def test_uniform_force_f64(collision):
    spec = W.CaseSpec(name="pf", nx=40, ny=21, bc=(W.PERIODIC, W.PERIODIC, W.VELOCITY, W.VELOCITY),
                      ubc=((0, 0),) * 4, collision=collision, tau=0.8, storage=W.F64, force=(2e-5, -1e-5))
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(300)
    c.step(300)
    assert rel_l2(velocity(g.populations())[0], velocity(c.populations())[0]) < F64_TOL
    rg, uxg, uyg = g.macro()
    rc, uxc, uyc = c.macro()
    assert rel_l2(uxg, uxc) < F64_TOL and rel_l2(rg, rc) < F64_TOL


# ---------------------------------------------------------------- domain conditions
BC_SETS = {
    "channel": ((W.VELOCITY, W.NEUMANN, W.VELOCITY, W.VELOCITY), ((0.05, 0), (0, 0), (0.05, 0), (0.05, 0))),
    "open": ((W.NEUMANN,) * 4, ((0, 0),) * 4),
    "walls": ((W.VELOCITY,) * 4, ((0, 0), (0, 0), (0, 0), (0.03, 0.0))),
    "periodic-y": ((W.VELOCITY, W.NEUMANN, W.PERIODIC, W.PERIODIC), ((0.04, 0), (0, 0), (0, 0), (0, 0))),
    "periodic-x": ((W.PERIODIC, W.PERIODIC, W.VELOCITY, W.NEUMANN), ((0, 0), (0, 0), (0.0, 0.0), (0, 0))),
}


@pytest.mark.parametrize("name", list(BC_SETS))
@pytest.mark.parametrize("nx,ny", [(150, 37), (129, 9), (5, 6)])
def test_domain_conditions_f64(name, nx, ny):
    bc, ubc = BC_SETS[name]
    f0 = W.random_populations(13, nx, ny, amp=0.02)
    spec = W.CaseSpec(name=name, nx=nx, ny=ny, bc=bc, ubc=ubc, collision=W.BGK, tau=0.7, storage=W.F64)
    g, c = gpu_case(spec), oracle_case(spec)
    g.set_populations(f0)
    c.set_populations(f0)
    for _ in range(3):
        g.step(7)
        c.step(7)
        fg, fc = g.populations(), c.populations()
        assert rel_l2(_dev(fg, f0), _dev(fc, f0)) < F64_TOL


# ---------------------------------------------------------------- immersed boundary, FP64
SCHEMES = [W.DF, W.MDF, W.DFC]
KERNELS = [W.HAT, W.PESKIN4]
COLLS = [W.BGK, W.TRT, W.CMMRT]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("collision", COLLS)
def test_ib_channel_f64(scheme, kernel, collision):
    body = cylinder_body(40.3, 31.7, 16.0, 47, kernel, scheme, mdf_nmin=2, mdf_nmax=12, mdf_tol=1e-4)
    spec = channel_spec(150, 64, collision=collision, tau=0.68, storage=W.F64, u=0.06, bodies=[body])
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(60)
    c.step(60)
    fg, fc = g.populations(), c.populations()
    assert rel_l2(_dev(fg, None), _dev(fc, None)) < F64_TOL
    ug, uc = velocity(fg), velocity(fc)
    assert rel_l2(ug[0] - 0.06, uc[0] - 0.06) < F64_TOL
    assert rel_l2(ug[1], uc[1]) < F64_TOL
    Fg, Fc = g.body_forces(0), c.body_forces(0)
    assert np.abs(Fg - Fc).max() < 1e-12 * np.abs(Fc[:2]).max()
    np.testing.assert_array_equal(g.marker_stencils(0), c.marker_stencils(0))
    mg, mc = g.marker_data(0), c.marker_data(0)
    assert rel_l2(mg[:, 4:6], mc[:, 4:6]) < F64_TOL
    if scheme == W.DFC:
        assert rel_l2(mg[:, 6], mc[:, 6]) < F64_TOL
    if scheme == W.MDF:
        it, res, om = g.mdf_info(0)
        assert it == c.mdf_iterations(0)
        assert om == pytest.approx(c.mdf_omega(0), rel=1e-13)
        assert res == pytest.approx(c.mdf_residual(0), rel=1e-9, abs=1e-15)
    hg, hc = g.force_history(0), c.force_history(0)
    assert hg.shape == hc.shape
    assert np.abs(hg - hc).max() < 1e-12 * np.abs(hc[:, :2]).max()


def test_cylinder_re20_2000_steps_f64():
    """200x100 lattice, D=20, 63 markers, DF + hat + BGK, U=0.05, tau=0.65, 2000 steps."""
    spec = W.fixed_cylinder_re20(storage=W.F64, steps=2000)
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(2000)
    c.step(2000)
    fg, fc = g.populations(), c.populations()
    ug, uc = velocity(fg), velocity(fc)
    assert rel_l2(ug[0], uc[0]) < F64_TOL and rel_l2(ug[1], uc[1]) < F64_TOL
    hg, hc = g.force_history(0), c.force_history(0)
    cd_g = hg[:, 0] / (0.5 * 0.05 ** 2 * 20.0)
    cd_c = hc[:, 0] / (0.5 * 0.05 ** 2 * 20.0)
    assert np.abs(cd_g - cd_c).max() < 1e-12 * np.abs(cd_c).max()


def test_cylinder_re20_2000_steps_f32():
    """Same case with FP32 shifted storage: velocity within 1e-5 relative L2 and
    drag/lift within 1e-4 relative to the FP64 oracle."""
    spec = W.fixed_cylinder_re20(storage=W.F32, steps=2000)
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(2000)
    c.step(2000)
    ug, uc = velocity(g.populations()), velocity(c.populations())
    assert rel_l2(np.stack(ug), np.stack(uc)) < 1e-5
    hg, hc = g.force_history(0), c.force_history(0)
    scale = 0.5 * 0.05 ** 2 * 20.0
    cd_g, cd_c = hg[:, 0] / scale, hc[:, 0] / scale
    cl_g, cl_c = hg[:, 1] / scale, hc[:, 1] / scale
    # drag and lift coefficients within 1e-4 relative to the drag over the whole history
    assert np.abs(cd_g - cd_c)[100:].max() < 1e-4 * np.abs(cd_c[-1])
    assert np.abs(cl_g - cl_c)[100:].max() < 1e-4 * np.abs(cd_c[-1])


# ---------------------------------------------------------------- moving bodies
def test_prescribed_oscillation_f64():
    spec = W.oscillating_cylinder(storage=W.F64, kernel=W.PESKIN4, scheme=W.DF, nx=128, ny=96,
                                  diameter=16.0, kc=5.0, u_max=0.05, re=60.0)
    spec.bodies[0].osc_period = 160.0
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(120)
    c.step(120)
    assert rel_l2(_dev(g.populations(), None), _dev(c.populations(), None)) < F64_TOL
    np.testing.assert_allclose(g.body_state(0), c.body_state(0), rtol=1e-13, atol=1e-15)
    mg, mc = g.marker_data(0), c.marker_data(0)
    np.testing.assert_allclose(mg[:, :4], mc[:, :4], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("internal_mass", [0, 1])
def test_free_body_f64(scheme, internal_mass):
    spec = W.sedimentation(two_particles=False, storage=W.F64, internal_mass=internal_mass,
                           kernel=W.PESKIN4, scheme=scheme, nx=64, ny=160, diameter=12.0, tau=0.7, g=4e-4)
    spec.bodies[0].mdf_nmin, spec.bodies[0].mdf_nmax = 3, 10
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(150)
    c.step(150)
    sg, sc = g.body_state(0), c.body_state(0)
    np.testing.assert_allclose(sg, sc, rtol=1e-11, atol=1e-14)
    assert sc[3] < 0.0                                     # settling down
    assert rel_l2(_dev(g.populations(), None), _dev(c.populations(), None)) < F64_TOL


def test_two_particle_dfc_f64():
    spec = W.sedimentation(two_particles=True, storage=W.F64, kernel=W.PESKIN4, scheme=W.DFC, nx=64,
                           ny=200, diameter=10.0, tau=0.7, g=4e-4)
    spec.bodies[0].xy, spec.bodies[0].ds = W.circle_markers(32.0, 120.0, 10.0, 31)
    spec.bodies[0].yc = 120.0
    spec.bodies[1].xy, spec.bodies[1].ds = W.circle_markers(32.0, 135.0, 10.0, 31)
    spec.bodies[1].yc = 135.0
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(80)
    c.step(80)
    for b in range(2):
        np.testing.assert_allclose(g.body_state(b), c.body_state(b), rtol=1e-11, atol=1e-14)
        assert rel_l2(g.marker_data(b)[:, 6], c.marker_data(b)[:, 6]) < F64_TOL
    assert rel_l2(_dev(g.populations(), None), _dev(c.populations(), None)) < F64_TOL


# ---------------------------------------------------------------- FP16 shifted storage
def test_f16_storage_within_roundoff_bound():
    """FP16 stores s = f - w with unit round-off u16 = 2^-11.  One rounding per
    population per step perturbs the velocity by at most ~ sum_i |e_i| |s_i| u16;
    over n steps of a stable (dissipative) flow the error stays within
    sqrt(n) times that.  Bound taken: 3 sqrt(n) u16 max|s| relative to |u|."""
    spec = W.fixed_cylinder_re20(storage=W.F16S, steps=300)
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(300)
    c.step(300)
    fc = c.populations()
    ug, uc = velocity(g.populations()), velocity(fc)
    smax = np.abs(fc - W9[:, None, None]).max()
    bound = 3.0 * math.sqrt(300) * 2.0 ** -11 * smax / 0.05
    assert rel_l2(ug[0], uc[0]) < bound


# ---------------------------------------------------------------- batching, checkpoints
def test_batch_equals_alone_bitwise():
    specs = [channel_spec(150, 64, collision=W.BGK, storage=W.F32, bodies=[cylinder_body(40.3, 31.7, 16.0, 47, W.PESKIN4, W.DF)]),
             channel_spec(96, 40, collision=W.TRT, storage=W.F32, bodies=[cylinder_body(30.0, 20.0, 10.0, 31, W.HAT, W.DFC)]),
             channel_spec(200, 50, collision=W.CMMRT, storage=W.F16S, bodies=[cylinder_body(50.0, 25.0, 12.0, 37, W.PESKIN4, W.MDF, mdf_nmin=5, mdf_nmax=5)]),
             channel_spec(64, 64, collision=W.BGK, storage=W.F64)]
    alone = [gpu_case(s) for s in specs]
    mixed = [gpu_case(s) for s in specs]
    for a in alone:
        a.step(37)
    L.step_batch(mixed, 37)
    for a, m in zip(alone, mixed):
        np.testing.assert_array_equal(a.populations(shifted=True), m.populations(shifted=True))
        if a.body_n:
            np.testing.assert_array_equal(a.force_history(0), m.force_history(0))


def test_snapshot_restore_continues_bitwise():
    spec = W.sedimentation(two_particles=False, storage=W.F32, kernel=W.PESKIN4, scheme=W.DFC, nx=64,
                           ny=160, diameter=12.0, tau=0.7, g=4e-4)
    a = gpu_case(spec)
    a.step(40)
    blob = a.snapshot()
    a.step(30)
    b = gpu_case(spec)
    b.restore(blob)
    b.step(30)
    np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))
    np.testing.assert_array_equal(a.body_state(0), b.body_state(0))


def test_graph_replay_equals_timed_launches():
    spec = channel_spec(150, 64, collision=W.BGK, storage=W.F32,
                        bodies=[cylinder_body(40.3, 31.7, 16.0, 47, W.PESKIN4, W.MDF, mdf_nmin=5, mdf_nmax=5)])
    a, b = gpu_case(spec), gpu_case(spec)
    a.step(33)
    b.set_timing(True)
    b.step(33)
    ms, n = b.kernel_timing()
    assert n == 33 and ms > 0
    np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))


def test_marker_out_of_domain_is_reported():
    spec = W.sedimentation(two_particles=False, storage=W.F32, kernel=W.PESKIN4, scheme=W.DF, nx=40,
                           ny=60, diameter=10.0, tau=0.7, g=5e-2)
    spec.bodies[0].xy, spec.bodies[0].ds = W.circle_markers(20.0, 12.0, 10.0, 31)
    spec.bodies[0].yc = 12.0
    g = gpu_case(spec)
    g.step(200)
    with pytest.raises(L.IblbmError) as e:
        g.sync()
    assert e.value.code == -4


# ---------------------------------------------------------------- full-size lattice, sampled
def test_full_size_2048x1024_f32_short_window():
    """2048x1024, D=64, 201 markers, Peskin DF, BGK, FP32, as benchmarked: five
    steps against the oracle over the whole field."""
    spec = W.fixed_cylinder_2048(re=100.0, storage=W.F32, collision=W.BGK, kernel=W.PESKIN4, scheme=W.DF)
    g, c = gpu_case(spec), oracle_case(spec)
    g.step(5)
    c.step(5)
    ug, uc = velocity(g.populations()), velocity(c.populations())
    assert rel_l2(np.stack(ug), np.stack(uc)) < 1e-5
    hg, hc = g.force_history(0), c.force_history(0)
    assert np.abs(hg[:, 0] - hc[:, 0]).max() < 1e-4 * np.abs(hc[:, 0]).max()
