"""Test helpers: build the same case on the oracle and on the CUDA library from
one seeded case description, and compare results."""
import numpy as np

import oracle
import workloads as W

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def oracle_case(spec: W.CaseSpec) -> oracle.Case:
    p = oracle.lattice_params(spec.nx, spec.ny, bc=spec.bc, ubc=spec.ubc, collision=spec.collision,
                              tau=spec.tau, trt_lambda=spec.trt_lambda, cm_sq=spec.cm_sq,
                              cm_se=spec.cm_se, force=spec.force)
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
