"""Accuracy of the reduced-precision storage modes against the FP64 oracle on
shortened versions of the paper-shaped workloads: the drag history of the
in-line oscillating cylinder (FP32 and shifted FP16 storage) and the settling
velocity of a free disk (FP32 storage, FP64 rigid body).  Each test prints the
measured error; the bars are stated in the asserts."""
import math

import numpy as np
import pytest

import workloads as W
from harness import gpu_case, oracle_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2609_02298_b300 as L  # noqa: E402

L.use_torch_allocator()


def _osc_spec(storage):
    spec = W.oscillating_cylinder(storage=storage, kernel=W.PESKIN4, scheme=W.DF, nx=256, ny=128,
                                  diameter=20.0, kc=5.0, u_max=0.1, re=100.0)
    return spec


def test_oscillating_cylinder_drag_history_f32_f16():
    """One oscillation period (T = KC D / U_max = 1000 steps) on 256x128, D=20,
    Peskin DF, BGK.  Cd = F_x / (rho U_max^2 D / 2).  Bars: FP32 within 1e-4 of
    the oracle's drag (relative to max |Cd|); FP16 storage within 2e-2."""
    steps = 1000
    c = oracle_case(_osc_spec(W.F64))
    c.step(steps)
    ref = c.force_history(0)[:, 0] / (0.5 * 0.1 ** 2 * 20.0)
    out = {}
    for name, st in (("f32", W.F32), ("f16", W.F16S)):
        g = gpu_case(_osc_spec(st))
        g.step(steps)
        assert g.sync() >= 0
        cd = g.force_history(0)[:, 0] / (0.5 * 0.1 ** 2 * 20.0)
        out[name] = float(np.abs(cd - ref).max() / np.abs(ref).max())
        g.close()
    print("oscillating cylinder Cd history, max |dCd| / max |Cd|: f32 %.3e  f16 %.3e  (max |Cd| %.3f)"
          % (out["f32"], out["f16"], np.abs(ref).max()))
    assert out["f32"] < 1e-4
    assert out["f16"] < 2e-2


def test_settling_velocity_f32():
    """Free disk rho_s/rho_f = 1.5, D=20, DFC + Peskin, g = 8.33e-5 (the
    400x1600 workload's parameters) on a 100x260 channel for 600 steps.
    Bar: FP32 storage within 1e-4 relative of the oracle's settling velocity."""
    def spec(st):
        s = W.sedimentation(two_particles=False, storage=st, kernel=W.PESKIN4, scheme=W.DFC, nx=100, ny=260,
                            diameter=20.0, tau=0.65, g=8.33e-5)
        return s
    steps = 600
    c = oracle_case(spec(W.F64))
    c.step(steps)
    g = gpu_case(spec(W.F32))
    g.step(steps)
    assert g.sync() >= 0
    vc, vg = c.body_state(0)[3], g.body_state(0)[3]
    ug = math.sqrt(0.5 * 8.33e-5 * 20.0)
    err = abs(vg - vc) / abs(vc)
    print("settling velocity after %d steps: oracle %.6e, f32 %.6e, relative error %.3e (v*/u_g = %.4f)"
          % (steps, vc, vg, err, abs(vc) / ug))
    assert err < 1e-4
