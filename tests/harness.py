"""Test helpers: build the same case on the oracle and on the CUDA library from
one seeded case description, and compare results."""
import math

import numpy as np

import oracle
import workloads as W

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def oracle_case(spec: W.CaseSpec) -> oracle.Case:
    p = oracle.lattice_params(spec.nx, spec.ny, bc=spec.bc, ubc=spec.ubc, collision=spec.collision,
                              tau=spec.tau, trt_lambda=spec.trt_lambda, cm_sq=spec.cm_sq,
                              cm_se=spec.cm_se, force=spec.force, wall_closure=spec.wall_closure)
    c = oracle.Case(p)
    c.set_uniform(1.0, *spec.init_u)
    for b in spec.bodies:
        bp = oracle.BodyParams()
        bp.xc, bp.yc, bp.radius, bp.rho_ratio = b.xc, b.yc, b.radius, b.rho_ratio
        bp.motion, bp.gx, bp.gy, bp.internal_mass = b.motion, b.gx, b.gy, b.internal_mass
        bp.mdf_nmin, bp.mdf_nmax, bp.mdf_tol, bp.mdf_omega = b.mdf_nmin, b.mdf_nmax, b.mdf_tol, b.mdf_omega
        bp.osc_amp, bp.osc_period = b.osc_amp, b.osc_period
        c.add_body(b.xy, b.ds, b.kernel, b.scheme, bp)
    return c


def gpu_case(spec: W.CaseSpec, storage=None):
    import paper_2609_02298_b300 as L
    return L.Lattice.from_spec(spec, storage=storage)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt((b * b).sum())
    return float(np.sqrt(((a - b) ** 2).sum()) / (den if den > 0 else 1.0))


def velocity(f):
    rho = f.sum(0)
    return (f * EX[:, None, None]).sum(0) / rho, (f * EY[:, None, None]).sum(0) / rho


def channel_spec(nx, ny, collision=W.BGK, tau=0.7, storage=W.F64, u=0.05, bodies=(), bc=None, ubc=None,
                 init_u=None):
    bc = bc or (W.VELOCITY, W.NEUMANN, W.VELOCITY, W.VELOCITY)
    ubc = ubc or ((u, 0.0), (0.0, 0.0), (u, 0.0), (u, 0.0))
    return W.CaseSpec(name="chan", nx=nx, ny=ny, bc=bc, ubc=ubc, collision=collision, tau=tau,
                      storage=storage, trt_lambda=3.0 / 16.0, init_u=init_u if init_u is not None else (u, 0.0),
                      bodies=list(bodies))


def cylinder_body(xc, yc, D, n, kernel, scheme, **kw):
    xy, ds = W.circle_markers(xc, yc, D, n)
    return W.BodySpec(xy=xy, ds=ds, kernel=kernel, scheme=scheme, xc=xc, yc=yc, radius=0.5 * D, **kw)


def taylor_green_fields(D, t, u0=0.04, re=10.0):
    """App. D Eq. D1 on the periodic 2D x 2D lattice (k = pi/D): (ux, uy, rho) at time t,
    rho from the pressure p = -u0^2 / 4 (cos 2kx + cos 2ky) e^{-4 nu k^2 t} / c_s^2."""
    nu = u0 * D / re
    k = math.pi / D
    n = 2 * D
    x = np.arange(n)[None, :] + 0.0
    y = np.arange(n)[:, None] + 0.0
    a = math.exp(-2.0 * nu * k * k * t)
    ux = -u0 * np.cos(k * x) * np.sin(k * y) * a
    uy = u0 * np.sin(k * x) * np.cos(k * y) * a
    rho = 1.0 - 3.0 * u0 * u0 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * a * a
    return ux, uy, rho


def taylor_green_ib_spec(D, kernel, scheme, storage=W.F64, u0=0.04, re=10.0):
    """App. D.1 IB-LBM mode.  Reading (the paper gives no marker layout): one fixed
    ring of markers of radius D/4 around the vortex centre (D/2, D/2), spacing ~1,
    whose desired velocity is the analytical field of Eq. D1 at each step."""
    nu = u0 * D / re
    r = 0.25 * D
    nm = max(8, int(round(2.0 * math.pi * r)))
    th = 2.0 * math.pi * np.arange(nm) / nm
    xy = np.stack([0.5 * D + r * np.cos(th), 0.5 * D + r * np.sin(th)], axis=1)
    body = W.BodySpec(xy=np.ascontiguousarray(xy), ds=2.0 * math.pi * r / nm, kernel=kernel, scheme=scheme,
                      xc=0.5 * D, yc=0.5 * D, radius=r, mdf_nmin=5, mdf_nmax=20, mdf_tol=1e-4)
    return W.CaseSpec(name="tg-ib-%d" % D, nx=2 * D, ny=2 * D, bc=(W.PERIODIC,) * 4, ubc=((0.0, 0.0),) * 4,
                      collision=W.BGK, tau=0.5 + 3.0 * nu, storage=storage, bodies=[body])


def taylor_green_ib_run(case, spec, D, u0=0.04, re=10.0, steps=None):
    """Runs App. D.1 on ``case`` (library lattice or oracle case built from ``spec``):
    equilibrium start from Eq. D1, before step s (0-based) the markers get the
    analytical velocity at t = s + 1 (the time the step's velocity stands for),
    measured at t = D / u0.  Returns the relative L2 error of u over the lattice."""
    nu = u0 * D / re
    k = math.pi / D
    steps = int(round(D / u0)) if steps is None else steps
    ux, uy, rho = taylor_green_fields(D, 0.0, u0, re)
    n = 2 * D
    f = np.zeros((9, n, n))
    for j in range(n):
        for i in range(n):
            f[:, j, i] = oracle.feq(rho[j, i], ux[j, i], uy[j, i])
    case.set_populations(f)
    xy = spec.bodies[0].xy
    X, Y = xy[:, 0], xy[:, 1]
    for s in range(steps):
        a = math.exp(-2.0 * nu * k * k * (s + 1))
        ud = np.stack([-u0 * np.cos(k * X) * np.sin(k * Y) * a, u0 * np.sin(k * X) * np.cos(k * Y) * a], axis=1)
        case.set_marker_velocity(0, ud)
        case.step(1)
    _, vx, vy = case.macro()
    ex_, ey_, _ = taylor_green_fields(D, float(steps), u0, re)
    return math.sqrt((((vx - ex_) ** 2 + (vy - ey_) ** 2).sum()) / ((ex_ ** 2 + ey_ ** 2).sum()))
