"""Parity checks of the library (through its C ABI) against the FP64 CPU oracle,
written once and run twice: on the B300 by test_gpu_parity.py at full sizes,
and on the host-thread emulation of the same sources by test_emu_parity.py at
small sizes.

Bars: streaming permutations and stencil indices bit-exact; FP64 storage within
1e-12 relative L2 (populations' deviation from rest and velocity); FP32 shifted
storage within 1e-5 relative L2 on velocity and 1e-4 on drag and lift
(relative to the drag); FP16 shifted storage within the round-off bound derived
in check_f16_storage."""
import math

import numpy as np

import workloads as W
from harness import W9, channel_spec, cylinder_body, gpu_case, oracle_case, rel_l2, velocity

F64_TOL = 1e-12


def dev(f):
    """Deviation of populations from the rest weights (what carries the flow)."""
    return f - W9[:, None, None]


def stepped(g, c, n):
    g.step(n)
    c.step(n)
    assert g.sync() >= 0


def assert_f64_state(fg, fc, u_ref):
    """FP64 bar for flows that start from rest: populations within 1e-12 of the
    oracle's (max norm, relative to max|f|), and velocity within 1e-12 relative
    L2 with the norm floored at u_ref per node.  The floor is needed because the
    oracle keeps f unshifted (f ~ 0.44), so its own round-off (~1e-16 absolute)
    is ~1e-12 of the velocity while the flow is still ~1e-4."""
    assert np.abs(fg - fc).max() < F64_TOL * np.abs(fc).max()
    ug, uc = np.stack(velocity(fg)), np.stack(velocity(fc))
    den = max(np.sqrt((uc ** 2).sum()), u_ref * np.sqrt(uc[0].size))
    assert np.sqrt(((ug - uc) ** 2).sum()) / den < F64_TOL


# ---------------------------------------------------------------- streaming
def check_streaming_bit_exact(storage, dt, nx, ny, full_cycle=True):
    f0 = W.random_populations(11, nx, ny)
    spec = W.CaseSpec(name="s", nx=nx, ny=ny, bc=(W.PERIODIC,) * 4, ubc=((0, 0),) * 4,
                      collision=W.STREAM_ONLY, tau=0.8, storage=storage)
    g = gpu_case(spec)
    g.set_populations(f0)
    stored0 = g.populations(shifted=True)
    np.testing.assert_array_equal(stored0, (f0 - W9[:, None, None]).astype(dt).astype(np.float64))
    c = oracle_case(spec)
    c.set_populations(stored0)   # the permutation is value-blind: feed it the stored values
    stepped(g, c, 1)
    np.testing.assert_array_equal(g.populations(shifted=True), c.populations())
    if full_cycle:
        g.step(math.lcm(nx, ny) - 1)          # every population back at its start
        np.testing.assert_array_equal(g.populations(shifted=True), stored0)


# ---------------------------------------------------------------- collision
def check_periodic_collision_f64(collision, nx=70, ny=23, steps=25):
    f0 = W.random_populations(12, nx, ny, amp=0.05)
    spec = W.CaseSpec(name="p", nx=nx, ny=ny, bc=(W.PERIODIC,) * 4, ubc=((0, 0),) * 4,
                      collision=collision, tau=0.73, storage=W.F64, trt_lambda=3 / 16)
    g, c = gpu_case(spec), oracle_case(spec)
    g.set_populations(f0)
    c.set_populations(f0)
    stepped(g, c, steps)
    fg, fc = g.populations(), c.populations()
    assert rel_l2(dev(fg), dev(fc)) < F64_TOL
    assert rel_l2(np.stack(velocity(fg)), np.stack(velocity(fc))) < F64_TOL


def check_uniform_force_f64(collision, nx=40, ny=21, steps=300):
    spec = W.CaseSpec(name="pf", nx=nx, ny=ny, bc=(W.PERIODIC, W.PERIODIC, W.VELOCITY, W.VELOCITY),
                      ubc=((0, 0),) * 4, collision=collision, tau=0.8, storage=W.F64, force=(2e-5, -1e-5))
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    assert rel_l2(np.stack(velocity(g.populations())), np.stack(velocity(c.populations()))) < F64_TOL
    rg, uxg, uyg = g.macro()
    rc, uxc, uyc = c.macro()
    assert rel_l2(np.stack([uxg, uyg]), np.stack([uxc, uyc])) < F64_TOL and rel_l2(rg, rc) < F64_TOL


# ---------------------------------------------------------------- domain conditions
BC_SETS = {
    "channel": ((W.VELOCITY, W.NEUMANN, W.VELOCITY, W.VELOCITY), ((0.05, 0), (0, 0), (0.05, 0), (0.05, 0))),
    "open": ((W.NEUMANN,) * 4, ((0, 0),) * 4),
    "walls": ((W.VELOCITY,) * 4, ((0, 0), (0, 0), (0, 0), (0.03, 0.0))),
    "periodic-y": ((W.VELOCITY, W.NEUMANN, W.PERIODIC, W.PERIODIC), ((0.04, 0), (0, 0), (0, 0), (0, 0))),
    "periodic-x": ((W.PERIODIC, W.PERIODIC, W.VELOCITY, W.NEUMANN), ((0, 0), (0, 0), (0.0, 0.0), (0, 0))),
}


def check_domain_conditions_f64(name, nx, ny, storage=W.F64, rounds=3, steps=7, wall_closure=0):
    bc, ubc = BC_SETS[name]
    f0 = W.random_populations(13, nx, ny, amp=0.02)
    spec = W.CaseSpec(name=name, nx=nx, ny=ny, bc=bc, ubc=ubc, collision=W.BGK, tau=0.7, storage=storage,
                      wall_closure=wall_closure)
    g, c = gpu_case(spec), oracle_case(spec)
    g.set_populations(f0)
    c.set_populations(f0)
    for _ in range(rounds):
        stepped(g, c, steps)
        # the random perturbation decays towards rest, so the bar is floored (assert_f64_state)
        assert_f64_state(g.populations(), c.populations(), u_ref=0.02)


# ---------------------------------------------------------------- rows of many tiles
def check_wide_rows_f64(collision, scheme, kernel, nx=1600, ny=28, steps=3):
    """Rows spanning several tiles of every stream-collide variant (the bulk-staged
    variant's interior tiles need x0 > 0 and x0 + 512 < nx - 1), with a body whose
    footprint straddles the tile seam at x = 1024."""
    # fixed MDF iteration count: an adaptive stop near the tolerance could differ by one
    # iteration between two correct implementations on this noisy field
    body = cylinder_body(1024.3, 0.5 * ny + 0.2, 10.0, 31, kernel, scheme, mdf_nmin=5, mdf_nmax=5, mdf_tol=1e-4)
    spec = channel_spec(nx, ny, collision=collision, tau=0.7, storage=W.F64, u=0.05, bodies=[body])
    g, c = gpu_case(spec), oracle_case(spec)
    f0 = W.random_populations(17, nx, ny, amp=0.02)
    g.set_populations(f0)
    c.set_populations(f0)
    stepped(g, c, steps)
    assert_f64_state(g.populations(), c.populations(), u_ref=0.05)
    Fg, Fc = g.body_forces(0), c.body_forces(0)
    fscale = np.abs(Fc[:2]).max()
    assert np.abs(Fg[:2] - Fc[:2]).max() < 1e-12 * fscale
    # torque = sum of r x F (Sec. 2.7): its round-off scales with the lever arm times the force
    assert abs(Fg[2] - Fc[2]) < 1e-12 * (abs(Fc[2]) + body.radius * fscale)


def check_wide_rows_narrow(storage, nx=1600, ny=6):
    """One step of a wide channel in FP32 / FP16 storage from the stored state,
    within the storage round-off (as the narrow-type domain-condition check)."""
    bc, ubc = BC_SETS["channel"]
    f0 = W.random_populations(18, nx, ny, amp=0.02)
    spec = W.CaseSpec(name="wide", nx=nx, ny=ny, bc=bc, ubc=ubc, collision=W.TRT, tau=0.7, storage=storage,
                      trt_lambda=3.0 / 16.0)
    g, c = gpu_case(spec), oracle_case(spec)
    g.set_populations(f0)
    c.set_populations(g.populations())
    g.step(1)
    c.step(1)
    tol = 1e-6 if storage == W.F32 else 2e-3
    assert rel_l2(dev(g.populations()), dev(c.populations())) < tol


# ---------------------------------------------------------------- immersed boundary
def check_ib_channel_f64(scheme, kernel, collision, nx=150, ny=64, D=16.0, n=47, steps=60):
    body = cylinder_body(0.27 * nx, 0.495 * ny, D, n, kernel, scheme, mdf_nmin=2, mdf_nmax=12, mdf_tol=1e-4)
    spec = channel_spec(nx, ny, collision=collision, tau=0.68, storage=W.F64, u=0.06, bodies=[body])
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    fg, fc = g.populations(), c.populations()
    assert rel_l2(dev(fg), dev(fc)) < F64_TOL
    ug, uc = velocity(fg), velocity(fc)
    assert rel_l2(np.stack([ug[0] - 0.06, ug[1]]), np.stack([uc[0] - 0.06, uc[1]])) < F64_TOL
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
        assert abs(om - c.mdf_omega(0)) < 1e-13 * c.mdf_omega(0)
        assert abs(res - c.mdf_residual(0)) < 1e-9 * c.mdf_residual(0) + 1e-15
    hg, hc = g.force_history(0), c.force_history(0)
    assert hg.shape == hc.shape
    assert np.abs(hg - hc).max() < 1e-12 * np.abs(hc[:, :2]).max()


def check_cylinder_re20_f64(steps=2000, nx=200):
    """200x100 lattice, D=20, 63 markers, DF + hat + BGK, U=0.05, tau=0.65."""
    spec = W.fixed_cylinder_re20(storage=W.F64, steps=steps)
    spec.nx = nx
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    fg, fc = g.populations(), c.populations()
    assert rel_l2(np.stack(velocity(fg)), np.stack(velocity(fc))) < F64_TOL
    hg, hc = g.force_history(0), c.force_history(0)
    scale = 0.5 * 0.05 ** 2 * 20.0
    assert np.abs(hg[:, :2] - hc[:, :2]).max() / scale < 1e-12 * np.abs(hc[:, 0] / scale).max()


def check_cylinder_re20_f32(steps=2000, nx=200):
    """FP32 shifted storage: velocity within 1e-5 relative L2; drag and lift
    coefficients within 1e-4 (relative to the drag) of the FP64 oracle."""
    spec = W.fixed_cylinder_re20(storage=W.F32, steps=steps)
    spec.nx = nx
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    ug, uc = velocity(g.populations()), velocity(c.populations())
    assert rel_l2(np.stack(ug), np.stack(uc)) < 1e-5
    hg, hc = g.force_history(0), c.force_history(0)
    scale = 0.5 * 0.05 ** 2 * 20.0
    cd_c = hc[:, 0] / scale
    assert np.abs(hg[:, 0] - hc[:, 0]).max() / scale < 1e-4 * np.abs(cd_c).max()
    assert np.abs(hg[:, 1] - hc[:, 1]).max() / scale < 1e-4 * np.abs(cd_c).max()


_ORACLE_CACHE = {}


def check_cylinder_re20_f32_scheme(collision, kernel, scheme, steps=2000, nx=200):
    """The FP32 bar of check_cylinder_re20_f32 for another operator, kernel and
    scheme of the same 200x100 Re = 20 cylinder (MDF adaptive in [5, 20]).  The lift
    bar is taken relative to the drag: at Re = 20 the flow is steady and symmetric,
    so the lift itself is round-off and a bar relative to it would be meaningless."""
    spec = W.fixed_cylinder_re20(storage=W.F32, steps=steps, collision=collision, kernel=kernel,
                                 scheme=scheme)
    spec.nx = nx
    key = ("re20", collision, kernel, scheme, steps, nx)
    if key not in _ORACLE_CACHE:   # the oracle's result does not depend on the device variant
        c = oracle_case(spec)
        c.step(steps)
        _ORACLE_CACHE[key] = (np.stack(velocity(c.populations())), c.force_history(0))
    uc, hc = _ORACLE_CACHE[key]
    g = gpu_case(spec)
    g.step(steps)
    assert g.sync() >= 0
    ug = np.stack(velocity(g.populations()))
    assert rel_l2(ug, uc) < 1e-5
    hg = g.force_history(0)
    scale = 0.5 * 0.05 ** 2 * 20.0
    cd_max = np.abs(hc[:, 0]).max() / scale
    assert np.abs(hg[:, 0] - hc[:, 0]).max() / scale < 1e-4 * cd_max
    assert np.abs(hg[:, 1] - hc[:, 1]).max() / scale < 1e-4 * cd_max


def _full_size_oracle(args):
    """Worker of check_full_size_matrix (runs in a spawned process): the oracle's
    velocity field and force history after ``steps`` steps of one lattice."""
    spec, steps = args
    c = oracle_case(spec)
    c.step(steps)
    ux, uy = velocity(c.populations())
    return ux, uy, c.force_history(0)


_FULL_SIZE_CACHE = {}


def full_size_matrix_specs(re):
    """The 18 lattices of one Reynolds-number half of the 2048x1024 FP32 matrix:
    {DF, MDF(5), DFC} x {hat, Peskin} x {BGK, TRT, CM-MRT}."""
    return [W.fixed_cylinder_2048(re=re, storage=W.F32, collision=col, kernel=ker, scheme=sch)
            for sch in (W.DF, W.MDF, W.DFC) for ker in (W.HAT, W.PESKIN4) for col in (W.BGK, W.TRT, W.CMMRT)]


def full_size_oracle(re, steps):
    """Oracle results for full_size_matrix_specs(re), computed once per process in a
    pool of spawned workers (a fork after CUDA initialisation is unsafe)."""
    key = (re, steps)
    if key not in _FULL_SIZE_CACHE:
        import multiprocessing as mp
        import os
        specs = full_size_matrix_specs(re)
        workers = max(1, min(len(specs), (os.cpu_count() or 1), 9))
        with mp.get_context("spawn").Pool(workers) as pool:
            _FULL_SIZE_CACHE[key] = pool.map(_full_size_oracle, [(s, steps) for s in specs], chunksize=1)
    return _FULL_SIZE_CACHE[key]


def check_full_size_matrix(L, re, steps=5):
    """All 18 lattices of one Reynolds-number half of the benchmarked matrix
    (2048x1024, D = 64, 201 markers, FP32 shifted storage, MDF with 5 fixed
    iterations), stepped together in one batch as the benchmark steps them, each
    compared over the whole field with the FP64 oracle: velocity within 1e-5
    relative L2 and the force history within 1e-4 of the drag."""
    specs = full_size_matrix_specs(re)
    ref = full_size_oracle(re, steps)
    gs = [gpu_case(s) for s in specs]
    try:
        L.step_batch(gs, steps)
        for g, s, (ux, uy, hc) in zip(gs, specs, ref):
            assert g.sync() >= 0, s.name
            ug = velocity(g.populations())
            err = rel_l2(np.stack(ug), np.stack([ux, uy]))
            b = s.bodies[0]
            tag = "%s scheme %d kernel %d collision %d" % (s.name, b.scheme, b.kernel, s.collision)
            assert err < 1e-5, (tag, err)
            hg = g.force_history(0)
            assert hg.shape == hc.shape, tag
            drag = np.abs(hc[:, 0]).max()
            assert np.abs(hg[:, :2] - hc[:, :2]).max() < 1e-4 * drag, (tag, hg, hc)
    finally:
        for g in gs:
            g.close()


def check_f16_storage(steps=300, nx=200):
    """FP16 stores s = f - w with unit round-off u16 = 2^-11.  One rounding per
    stored population per step perturbs the velocity by at most about
    max|s| u16 / |u| relative; a dissipative flow accumulates these like a
    random walk, so the bound taken is 3 sqrt(n) u16 max|s| / |U|."""
    spec = W.fixed_cylinder_re20(storage=W.F16S, steps=steps)
    spec.nx = nx
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    fc = c.populations()
    ug, uc = velocity(g.populations()), velocity(fc)
    smax = np.abs(dev(fc)).max()
    bound = 3.0 * math.sqrt(steps) * 2.0 ** -11 * smax / 0.05
    assert rel_l2(np.stack(ug), np.stack(uc)) < bound


# ---------------------------------------------------------------- moving bodies
def check_mdf_large_body_f64(kernel, nx=260, ny=240, D=180.0, n=566, steps=3):
    """MDF body with more markers than the IB CTA's threads (and, for Peskin, more
    footprint nodes than its shared-memory iterate holds): the global-memory MDF path."""
    body = cylinder_body(0.5 * nx + 0.3, 0.5 * ny + 0.1, D, n, kernel, W.MDF, mdf_nmin=3, mdf_nmax=3)
    spec = channel_spec(nx, ny, collision=W.BGK, tau=0.8, storage=W.F64, u=0.03, bodies=[body])
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    assert_f64_state(g.populations(), c.populations(), u_ref=0.03)
    Fg, Fc = g.body_forces(0), c.body_forces(0)
    assert np.abs(Fg - Fc).max() < 1e-12 * np.abs(Fc[:2]).max()
    assert g.mdf_info(0)[0] == c.mdf_iterations(0) == 3


def check_prescribed_oscillation_f64(nx=128, ny=96, D=16.0, steps=120):
    spec = W.oscillating_cylinder(storage=W.F64, kernel=W.PESKIN4, scheme=W.DF, nx=nx, ny=ny, diameter=D,
                                  kc=5.0, u_max=0.05, re=60.0)
    spec.bodies[0].osc_amp = 0.2 * D
    spec.bodies[0].osc_period = 160.0
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    assert_f64_state(g.populations(), c.populations(), u_ref=0.05)
    np.testing.assert_allclose(g.body_state(0), c.body_state(0), rtol=1e-13, atol=1e-15)
    mg, mc = g.marker_data(0), c.marker_data(0)
    np.testing.assert_allclose(mg[:, :4], mc[:, :4], rtol=1e-13, atol=1e-13)


def check_free_body_f64(scheme, internal_mass, nx=64, ny=160, D=12.0, steps=150):
    """Settling disk, FP64.  MDF is checked over its first 8 steps only: with the
    explicit Velocity-Verlet coupling of Eq. 23 the converged MDF force makes a
    rho_s/rho_f = 1.5 disk diverge after some 20-40 steps, in the oracle exactly
    as on the device (DF and DFC stay stable)."""
    spec = W.sedimentation(two_particles=False, storage=W.F64, internal_mass=internal_mass,
                           kernel=W.PESKIN4, scheme=scheme, nx=nx, ny=ny, diameter=D, tau=0.7, g=1e-4)
    spec.bodies[0].mdf_nmin, spec.bodies[0].mdf_nmax = 3, 10
    if scheme == W.MDF:
        steps = min(steps, 8)
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    sg, sc = g.body_state(0), c.body_state(0)
    np.testing.assert_allclose(sg[:4], sc[:4], rtol=1e-11, atol=1e-14)
    # on the symmetry axis the rotation is round-off noise (|omega| ~ 1e-14 or below)
    np.testing.assert_allclose(sg[4:], sc[4:], rtol=1e-11, atol=1e-12)
    if scheme != W.MDF:
        assert sc[3] < 0.0                                 # settling down
    assert_f64_state(g.populations(), c.populations(), u_ref=0.01)
    np.testing.assert_array_equal(g.marker_stencils(0), c.marker_stencils(0))


def check_two_particle_dfc_f64(nx=100, ny=260, D=20.0, steps=100, spacing=1.5):
    """Two settling disks (rho_s/rho_f 1.5 below 1.01, ``spacing`` D apart centre to
    centre), DFC with a shared W_total, g and tau of the 400x1600 sedimentation
    workload.  At spacing 1.1 the disks' footprints share nodes, so each disk's
    lambda_k depends on where the other's markers are in the same step."""
    spec = W.sedimentation(two_particles=True, storage=W.F64, kernel=W.PESKIN4, scheme=W.DFC, nx=nx,
                           ny=ny, diameter=D, tau=0.65, g=8.33e-5)
    y0 = 0.5 * ny
    for b, yc in zip(spec.bodies, (y0, y0 + spacing * D)):
        b.xy, b.ds = W.circle_markers(b.xc, yc, D, 31)
        b.yc = yc
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    for b in range(2):
        np.testing.assert_allclose(g.body_state(b), c.body_state(b), rtol=1e-11, atol=1e-14)
        assert rel_l2(g.marker_data(b)[:, 6], c.marker_data(b)[:, 6]) < F64_TOL
    assert_f64_state(g.populations(), c.populations(), u_ref=0.01)


def check_coupled_mdf_f64(kernels, dsfac=1.0, nx=90, ny=64, D=14.0, n=44, steps=25, free=False,
                          rotation=True, rho=(1.5, 1.25), g=2e-4):
    """Two MDF disks 0.1 D apart at the surface (footprints sharing nodes) in the inflow
    channel: the coupled iteration of Sec. 2.5.2 on the device against the oracle --
    populations and velocity at the FP64 bar, marker forces, the trial-iteration count,
    the joint residual and the final relaxation of every step.  dsfac scales the arc
    lengths so that trials are rejected and omega halved; ``free`` releases both disks
    (density ratios 1.5 and 1.25, gravity across the stream), with their rotation held
    at rest when ``rotation`` is False."""
    kw = dict(mdf_nmin=5, mdf_nmax=20, mdf_omega=5.0 if dsfac != 1.0 else 0.0)
    if free:
        kw.update(motion=W.FREE if rotation else W.FREE_TRANSLATION, gx=0.0, gy=-g)
    xc0, yc0 = 0.3 * nx, 0.5 * ny
    b0 = cylinder_body(xc0, yc0 - 0.55 * D, D, n, kernels[0], W.MDF, rho_ratio=rho[0], **kw)
    b1 = cylinder_body(xc0 + 0.2 * D, yc0 + 0.55 * D, D, n, kernels[1], W.MDF, rho_ratio=rho[1], **kw)
    for b in (b0, b1):
        b.ds *= dsfac
    # free disks settle from rest in a quiescent channel (a stream hitting disks at rest
    # kicks them harder than the explicit MDF coupling tolerates at this size)
    spec = channel_spec(nx, ny, collision=W.BGK, tau=0.7, storage=W.F64, u=0.0 if free else 0.03, bodies=[b0, b1])
    g, c = gpu_case(spec), oracle_case(spec)
    for _ in range(steps):
        stepped(g, c, 1)
        it_g = [g.mdf_info(b)[0] for b in range(2)]
        assert it_g == [c.mdf_iterations(b) for b in range(2)]
        assert it_g[0] == it_g[1]
        for b in range(2):
            assert g.mdf_relaxation(b) == c.mdf_omega_end(b)
            np.testing.assert_allclose(g.mdf_info(b)[1], c.mdf_residual(b), rtol=1e-9, atol=1e-15)
            np.testing.assert_allclose(g.marker_data(b)[:, 4:6], c.marker_data(b)[:, 4:6], rtol=1e-10, atol=1e-14)
            np.testing.assert_allclose(g.body_state(b), c.body_state(b), rtol=1e-11, atol=1e-14)
    assert_f64_state(g.populations(), c.populations(), u_ref=0.01)
    g.close()


# ---------------------------------------------------------------- batching, checkpoints, errors
def batch_specs(scale=1.0):
    s = lambda v: max(8, int(v * scale))  # noqa: E731
    return [
        channel_spec(s(150), s(64), collision=W.BGK, storage=W.F32,
                     bodies=[cylinder_body(0.27 * s(150), 0.49 * s(64), 16.0 * scale, max(16, int(47 * scale)),
                                           W.PESKIN4, W.DF)]),
        channel_spec(s(96), s(40), collision=W.TRT, storage=W.F32,
                     bodies=[cylinder_body(0.31 * s(96), 0.5 * s(40), 10.0 * scale, max(12, int(31 * scale)),
                                           W.HAT, W.DFC)]),
        channel_spec(s(200), s(50), collision=W.CMMRT, storage=W.F16S,
                     bodies=[cylinder_body(0.25 * s(200), 0.5 * s(50), 12.0 * scale, max(12, int(37 * scale)),
                                           W.PESKIN4, W.MDF, mdf_nmin=5, mdf_nmax=5)]),
        channel_spec(s(64), s(64), collision=W.BGK, storage=W.F64),
    ]


def check_batch_equals_alone(L, specs, steps=37):
    alone = [gpu_case(s) for s in specs]
    mixed = [gpu_case(s) for s in specs]
    for a in alone:
        a.step(steps)
    L.step_batch(mixed, steps)
    for a, m in zip(alone, mixed):
        assert m.sync() >= 0
        np.testing.assert_array_equal(a.populations(shifted=True), m.populations(shifted=True))
        if a.body_n:
            np.testing.assert_array_equal(a.force_history(0), m.force_history(0))


def check_snapshot_restore(nx=64, ny=160, D=12.0, steps=(40, 30)):
    spec = W.sedimentation(two_particles=False, storage=W.F32, kernel=W.PESKIN4, scheme=W.DFC, nx=nx,
                           ny=ny, diameter=D, tau=0.7, g=4e-4)
    a = gpu_case(spec)
    a.step(steps[0])
    blob = a.snapshot()
    arr = a.snapshot(out=np.empty(a.snapshot_bytes(), dtype=np.uint8))   # caller-owned buffer
    assert arr.tobytes() == blob
    a.step(steps[1])
    for src in (blob, arr):
        b = gpu_case(spec)
        b.restore(src)
        b.step(steps[1])
        np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))
        np.testing.assert_array_equal(a.body_state(0), b.body_state(0))
        np.testing.assert_array_equal(a.force_history(0), b.force_history(0))
        b.close()


def check_graph_equals_direct(nx=150, ny=64, steps=33):
    spec = channel_spec(nx, ny, collision=W.BGK, storage=W.F32,
                        bodies=[cylinder_body(0.27 * nx, 0.49 * ny, 16.0, 47, W.PESKIN4, W.MDF,
                                              mdf_nmin=5, mdf_nmax=5)])
    a, b = gpu_case(spec), gpu_case(spec)
    a.step(steps)
    b.set_timing(True)
    b.step(steps)
    ms, n = b.kernel_timing()
    assert n == 2 * steps and ms >= 0   # stream-collide + lattice-edge launch per step
    np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))


def check_overlap_equals_serial(nx=1100, ny=960, steps=6):
    """A lattice of more than 2^20 nodes with two fixed bodies: the graph-replayed step runs
    the IB stage beside the sweep of everything outside the IB regions and sweeps those
    regions after it; the launch-by-launch (timed) step runs the IB stage, then the whole
    sweep.  Both must give the same populations and forces bit for bit."""
    bodies = [cylinder_body(0.3 * nx, 0.5 * ny, 40.0, 126, W.PESKIN4, W.DF),
              cylinder_body(0.6 * nx, 0.3 * ny, 30.0, 94, W.HAT, W.DFC)]
    spec = channel_spec(nx, ny, collision=W.TRT, storage=W.F32, bodies=bodies)
    a, b = gpu_case(spec), gpu_case(spec)
    a.step(steps)
    b.set_timing(True)
    b.step(steps)
    b.set_timing(False)
    assert a.sync() == 0 and b.sync() == 0
    np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))
    for k in range(2):
        np.testing.assert_array_equal(a.force_history(k), b.force_history(k))
    a.close()
    b.close()


def check_ib_fast_equals_general(L, storage=W.F32, nx=300, ny=120, steps=6):
    """Fixed DF and DFC bodies with cached footprints take the IB fast path (static data in
    registers and shared memory, gathered state in shared memory); the general path must
    give the same populations and force histories bit for bit.  One body's footprint
    reaches the bottom wall (its gather takes the domain conditions), one uses the hat
    kernel, one the Peskin kernel; an MDF body beside them always takes the general path."""
    bodies = [cylinder_body(0.25 * nx, 0.55 * ny, 20.0, 63, W.PESKIN4, W.DF),
              cylinder_body(0.55 * nx, 0.5 * ny, 16.0, 51, W.HAT, W.DFC),
              cylinder_body(0.8 * nx, 6.5, 10.0, 31, W.PESKIN4, W.DFC),
              cylinder_body(0.4 * nx, 0.2 * ny, 10.0, 31, W.HAT, W.MDF)]
    spec = channel_spec(nx, ny, collision=W.BGK, storage=storage, bodies=bodies)
    a, b = gpu_case(spec), gpu_case(spec)
    try:
        L.test_set_ib_fast(False)
        b.step(steps)
        sb = b.sync()
    finally:
        L.test_set_ib_fast(True)
    a.step(steps)
    assert a.sync() == sb >= 0   # (warning bits only: the MDF body may end on N_max)
    np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))
    for k in range(len(bodies)):
        np.testing.assert_array_equal(a.force_history(k), b.force_history(k))
    a.close()
    b.close()


def check_ib_fast_equals_general_moving(L, storage=W.F32, steps=6):
    """Moving bodies take the fast path after each step's footprint rebuild: a prescribed
    in-line oscillation (DFC, Peskin) and two settling disks (DF, hat; DFC, Peskin) against
    the general path, bit for bit."""
    specs = [W.oscillating_cylinder(storage=storage, kernel=W.PESKIN4, scheme=W.DFC, nx=160, ny=80, diameter=16.0),
             W.sedimentation(two_particles=True, storage=storage, kernel=W.HAT, scheme=W.DF, nx=80, ny=240,
                             diameter=12.0),
             W.sedimentation(two_particles=False, storage=storage, kernel=W.PESKIN4, scheme=W.DFC, nx=80, ny=240,
                             diameter=12.0)]
    for spec in specs:
        a, b = gpu_case(spec), gpu_case(spec)
        try:
            L.test_set_ib_fast(False)
            b.step(steps)
            sb = b.sync()
        finally:
            L.test_set_ib_fast(True)
        a.step(steps)
        assert a.sync() == sb >= 0
        np.testing.assert_array_equal(a.populations(shifted=True), b.populations(shifted=True))
        for k in range(len(spec.bodies)):
            np.testing.assert_array_equal(a.force_history(k), b.force_history(k))
            np.testing.assert_array_equal(a.body_state(k), b.body_state(k))
        a.close()
        b.close()


def check_marker_out_of_domain(L, steps=200):
    spec = W.sedimentation(two_particles=False, storage=W.F32, kernel=W.PESKIN4, scheme=W.DF, nx=40,
                           ny=60, diameter=10.0, tau=0.7, g=5e-2)
    spec.bodies[0].xy, spec.bodies[0].ds = W.circle_markers(20.0, 12.0, 10.0, 31)
    spec.bodies[0].yc = 12.0
    g = gpu_case(spec)
    g.step(steps)
    try:
        g.sync()
    except L.IblbmError as e:
        assert e.code == -4
    else:
        raise AssertionError("a marker left the lattice but no error was reported")


# ---------------------------------------------------------------- serving loop
def serving_specs(scale=1.0, n=6, steps=(24, 16, 40, 8, 30, 12)):
    """Mixed requests: sizes, schemes, kernels, collisions and storages differ."""
    s = lambda v: max(12, int(v * scale))  # noqa: E731
    combos = [(W.DF, W.HAT, W.BGK, W.F32), (W.MDF, W.PESKIN4, W.TRT, W.F32), (W.DFC, W.PESKIN4, W.CMMRT, W.F32),
              (W.DF, W.PESKIN4, W.CMMRT, W.F16S), (W.DFC, W.HAT, W.BGK, W.F64), (W.MDF, W.HAT, W.BGK, W.F32)]
    sizes = [(128, 64), (96, 48), (160, 64), (128, 48), (64, 40), (112, 56)]
    out = []
    for i in range(n):
        scheme, kernel, col, st = combos[i % len(combos)]
        nx, ny = sizes[i % len(sizes)]
        nx, ny = s(nx), s(ny)
        D = max(4.0, ny / 6.0)
        body = cylinder_body(0.3 * nx + 0.37, 0.5 * ny + 0.21, D, max(12, int(round(math.pi * D))), kernel, scheme,
                             mdf_nmin=5, mdf_nmax=5)
        sp = channel_spec(nx, ny, collision=col, tau=0.62 + 0.02 * i, storage=st, u=0.06, bodies=[body])
        out.append((sp, steps[i % len(steps)]))
    return out


def check_server_alone_vs_mix(L, cases, budget_lattices=2.5, max_steps=8):
    """Requests admitted under an HBM budget that holds about budget_lattices of
    them run in a continuous batch; each result equals the same case run alone
    (bitwise), and the budget is never exceeded."""
    alone = []
    for sp, n in cases:
        g = gpu_case(sp)
        g.step(n)
        assert g.sync() >= 0
        alone.append(g.force_history(0))
        g.close()
    sizes = []
    for sp, _ in cases:
        g = gpu_case(sp)
        sizes.append(g.device_bytes)
        g.close()
    budget = int(budget_lattices * max(sizes))
    srv = L.Server(budget, max_slots=8)
    ids = [srv.submit(sp, n) for sp, n in cases]
    done, peak_resident, ticks = 0, 0, 0
    while done < len(ids):
        k, res, que = srv.tick(max_steps)
        used, _, _ = srv.stats()
        assert used <= budget
        peak_resident = max(peak_resident, res)
        done += k
        ticks += 1
        assert ticks < 10000
    assert peak_resident >= 2                       # cases overlapped on the device
    for rid, ref in zip(ids, alone):
        hist, lat = srv.poll(rid)
        assert lat > 0
        np.testing.assert_array_equal(hist, ref)
    # a request that can never fit the budget is rejected, not queued forever
    big = channel_spec(1024, 1024, storage=W.F64)
    rid = srv.submit(big, 4)
    srv.tick(4)
    try:
        srv.poll(rid)
    except L.IblbmError as e:
        assert e.code == -7
    else:
        raise AssertionError("oversized request was not rejected")
    srv.close()


# ---------------------------------------------------------------- Sec. 2.8 diagnostics
def _assert_diagnostics(dg, dc, pg, pc, tol):
    """Slip, leakage and interior values are normalised by u_ref (O(1) at most);
    the interior count is decided in FP64 on both sides and must be equal."""
    assert dg[6] == dc[6] and dc[6] > 0
    np.testing.assert_allclose(dg[[0, 1, 2, 3, 4, 5]], dc[[0, 1, 2, 3, 4, 5]], rtol=tol, atol=tol * 1e-2)
    np.testing.assert_allclose(dg[7], dc[7], rtol=tol)
    np.testing.assert_allclose(pg[:, :3], pc[:, :3], rtol=tol, atol=tol * 1e-2)
    np.testing.assert_allclose(pg[:, 3], pc[:, 3], rtol=tol, atol=tol * 1e-4)
    np.testing.assert_allclose(pg[:, 4], pc[:, 4], rtol=tol, atol=tol * 1e-3 * pc[:, 4].max())


def check_local_diagnostics(scheme, kernel, storage=W.F64, nx=150, ny=64, D=16.0, n=47, steps=60):
    """Fixed cylinder in the channel: the device diagnostics of the device state
    against the oracle's diagnostics of its own state.  FP64: 1e-9 relative (the
    slip is a small difference of interpolated velocities, so it carries the
    state's 1e-12 at up to 1e3 times the weight); FP32 shifted storage 2e-3."""
    body = cylinder_body(0.27 * nx, 0.495 * ny, D, n, kernel, scheme, mdf_nmin=2, mdf_nmax=12, mdf_tol=1e-4)
    spec = channel_spec(nx, ny, collision=W.BGK, tau=0.68, storage=storage, u=0.06, bodies=[body])
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    dg, pg = g.local_diagnostics(0, 0.06, 2.0, per_marker=True)
    dc, pc = c.local_diagnostics(0, 0.06, 2.0, per_marker=True)
    _assert_diagnostics(dg, dc, pg, pc, 1e-9 if storage == W.F64 else 2e-3)
    # a wider buffer keeps fewer interior nodes
    assert g.local_diagnostics(0, 0.06, 4.0)[6] == c.local_diagnostics(0, 0.06, 4.0)[6] < dc[6]


def check_local_diagnostics_free_body(scheme=W.DF, steps=60):
    """Settling disk: the interior residual is taken against the rigid velocity of
    the moving body and the slip against the markers' desired velocity."""
    spec = W.sedimentation(two_particles=False, storage=W.F64, internal_mass=1, kernel=W.PESKIN4, scheme=scheme,
                           nx=64, ny=160, diameter=12.0, tau=0.7, g=1e-4)
    g, c = gpu_case(spec), oracle_case(spec)
    stepped(g, c, steps)
    dg, pg = g.local_diagnostics(0, 0.01, 2.0, per_marker=True)
    dc, pc = c.local_diagnostics(0, 0.01, 2.0, per_marker=True)
    assert abs(g.body_state(0)[3]) > 1e-5
    _assert_diagnostics(dg, dc, pg, pc, 1e-9)


# ---------------------------------------------------------------- App. D.1 Taylor-Green, IB mode
def check_taylor_green_ib(kernel, scheme, D=10, storage=W.F64):
    """Markers driven per step through iblbm_set_marker_velocity with the analytical
    field: device and oracle velocity fields and errors after t = D / u0.  FP64
    within 1e-12 (relative to the field); FP32 storage within 1e-5."""
    from harness import taylor_green_ib_run, taylor_green_ib_spec
    spec = taylor_green_ib_spec(D, kernel, scheme, storage=storage)
    g, c = gpu_case(spec), oracle_case(spec)
    eg = taylor_green_ib_run(g, spec, D)
    ec = taylor_green_ib_run(c, spec, D)
    assert g.sync() >= 0
    _, gx, gy = g.macro()
    _, cx, cy = c.macro()
    tol = F64_TOL if storage == W.F64 else 1e-5
    assert rel_l2(np.stack([gx, gy]), np.stack([cx, cy])) < tol
    # the error is a small difference of fields that agree to tol relative to |u|
    assert abs(eg - ec) < 10 * tol
    mg, mc = g.marker_data(0), c.marker_data(0)
    np.testing.assert_allclose(mg[:, 2:4], mc[:, 2:4], rtol=0, atol=1e-15)   # the U_d that was set
    return eg
