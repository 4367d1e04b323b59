"""The parity checks of parity_cases.py run on CPU through the host-thread
emulation of the library's own CUDA sources (tests/emu): same kernels, same C
ABI, small lattices.  This exercises the kernel logic (streaming, domain
conditions, footprint CSR, DF/MDF/DFC, rigid bodies, batching, checkpoints)
without a GPU; the B300 run of test_gpu_parity.py is the parity claim."""
import os
import sys

import numpy as np
import pytest

import workloads as W
import parity_cases as P

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "emu"))


@pytest.fixture(scope="module", params=[1, 0, 2, 3], ids=["scalar", "vector", "scalar2", "bulk"])
def L(request):
    """The emulated library with the stream-collide variant fixed (both are checked)."""
    import build_emu
    import paper_2609_02298_b300 as lib
    path = build_emu.build()
    saved = lib._lib
    lib._lib = None
    lib.load_library(path)
    for st in (W.F64, W.F32, W.F16S):
        for col in (W.BGK, W.TRT, W.CMMRT, W.STREAM_ONLY):
            lib.set_kernel_variant(st, col, request.param)
    lib._test_variant = request.param
    yield lib
    lib._close_all()
    lib._lib = saved


def full_only(L):
    """Slow checks run for the one-node-per-lane variant only; the other
    variants get the streaming, boundary, a subset of the IB and batch checks."""
    if L._test_variant != 1:
        pytest.skip("checked with the one-node-per-lane variant")


def bulk_only(L):
    """Rows of several 512-node tiles matter to the bulk-staged variant (its
    interior-tile path); the other variants' segments are covered by the
    narrower lattices."""
    if L._test_variant != 3:
        pytest.skip("checked with the bulk-staged variant")


SCHEMES = [W.DF, W.MDF, W.DFC]
KERNELS = [W.HAT, W.PESKIN4]
COLLS = [W.BGK, W.TRT, W.CMMRT]


@pytest.mark.parametrize("storage,dt", [(W.F64, np.float64), (W.F32, np.float32), (W.F16S, np.float16)])
@pytest.mark.parametrize("nx,ny", [(7, 7), (37, 5)])
def test_streaming_bit_exact(L, storage, dt, nx, ny):
    P.check_streaming_bit_exact(storage, dt, nx, ny, full_cycle=(nx == 7))


@pytest.mark.parametrize("collision", COLLS)
def test_periodic_collision_f64(L, collision):
    full_only(L)
    P.check_periodic_collision_f64(collision, nx=20, ny=9, steps=4)


@pytest.mark.parametrize("collision", COLLS)
def test_uniform_force_f64(L, collision):
    full_only(L)
    P.check_uniform_force_f64(collision, nx=6, ny=9, steps=30)


@pytest.mark.parametrize("name", list(P.BC_SETS))
@pytest.mark.parametrize("nx,ny", [(37, 7), (65, 5), (5, 6)])
def test_domain_conditions_f64(L, name, nx, ny):
    P.check_domain_conditions_f64(name, nx, ny, rounds=2, steps=2)


@pytest.mark.parametrize("name", ["channel", "open"])
@pytest.mark.parametrize("storage", [W.F32, W.F16S])
def test_domain_conditions_narrow_types(L, name, storage):
    """FP32/FP16 vector paths (4 and 8 nodes per lane) against the FP64 oracle:
    one step, tolerance of the storage round-off."""
    bc, ubc = P.BC_SETS[name]
    from harness import gpu_case, oracle_case, rel_l2
    f0 = W.random_populations(13, 133, 6, amp=0.02)
    spec = W.CaseSpec(name=name, nx=133, ny=6, bc=bc, ubc=ubc, collision=W.BGK, tau=0.7, storage=storage)
    g, c = gpu_case(spec), oracle_case(spec)
    g.set_populations(f0)
    c.set_populations(g.populations())
    g.step(1)
    c.step(1)
    tol = 1e-6 if storage == W.F32 else 2e-3
    assert rel_l2(P.dev(g.populations()), P.dev(c.populations())) < tol


@pytest.mark.parametrize("storage,dt", [(W.F64, np.float64), (W.F32, np.float32), (W.F16S, np.float16)])
def test_wide_streaming_bit_exact(L, storage, dt):
    bulk_only(L)
    P.check_streaming_bit_exact(storage, dt, 1600, 3, full_cycle=False)


@pytest.mark.parametrize("scheme,kernel,collision", [(W.DFC, W.PESKIN4, W.CMMRT)])
def test_wide_rows_f64(L, scheme, kernel, collision):
    bulk_only(L)
    P.check_wide_rows_f64(collision, scheme, kernel, ny=24, steps=2)


@pytest.mark.parametrize("storage", [W.F32, W.F16S])
def test_wide_rows_narrow(L, storage):
    bulk_only(L)
    P.check_wide_rows_narrow(storage, ny=4)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("collision", COLLS)
def test_ib_channel_f64(L, scheme, kernel, collision):
    if L._test_variant != 1 and (kernel, collision) not in ((W.HAT, W.BGK), (W.PESKIN4, W.CMMRT)):
        pytest.skip("subset for this variant")
    P.check_ib_channel_f64(scheme, kernel, collision, nx=36, ny=24, D=8.0, n=23, steps=3)


@pytest.mark.parametrize("kernel", KERNELS)
def test_mdf_large_body_f64(L, kernel):
    full_only(L)
    P.check_mdf_large_body_f64(kernel, steps=1)


def test_prescribed_oscillation_f64(L):
    full_only(L)
    P.check_prescribed_oscillation_f64(nx=40, ny=24, D=8.0, steps=4)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_free_body_f64(L, scheme):
    full_only(L)
    P.check_free_body_f64(scheme, 1, nx=24, ny=64, D=6.0, steps=4)


@pytest.mark.parametrize("kernels,dsfac,free", [((W.HAT, W.PESKIN4), 1.0, False), ((W.PESKIN4, W.PESKIN4), 6.0, False),
                                                 ((W.PESKIN4, W.HAT), 1.0, True)])
def test_coupled_mdf_f64(L, kernels, dsfac, free):
    full_only(L)
    P.check_coupled_mdf_f64(kernels, dsfac=dsfac, nx=44, ny=34, D=8.0, n=26, steps=4, free=free)


def test_coupled_mdf_free_translation_f64(L):
    full_only(L)
    P.check_coupled_mdf_f64((W.PESKIN4, W.HAT), nx=44, ny=34, D=8.0, n=26, steps=4, free=True, rotation=False,
                            rho=(3.0, 2.5), g=5e-5)


def test_two_particle_dfc_f64(L):
    full_only(L)
    P.check_two_particle_dfc_f64(nx=24, ny=64, D=6.0, steps=3)


def test_two_particle_dfc_sharing_nodes_f64(L):
    full_only(L)
    P.check_two_particle_dfc_f64(nx=24, ny=64, D=6.0, steps=3, spacing=1.1)


def test_batch_equals_alone_bitwise(L):
    if L._test_variant not in (1, 3):
        pytest.skip("checked with the one-node-per-lane and bulk-staged variants")
    P.check_batch_equals_alone(L, P.batch_specs(scale=0.3), steps=3)


def test_snapshot_restore_continues_bitwise(L):
    full_only(L)
    P.check_snapshot_restore(nx=24, ny=64, D=6.0, steps=(2, 2))


def test_graph_replay_equals_timed_launches(L):
    full_only(L)
    P.check_graph_equals_direct(nx=40, ny=24, steps=3)


@pytest.mark.parametrize("storage", [W.F64, W.F32])
def test_ib_fast_path_equals_general_path(L, storage):
    full_only(L)
    P.check_ib_fast_equals_general(L, storage, nx=120, ny=60, steps=3)


def test_ib_fast_path_equals_general_path_moving(L):
    full_only(L)
    P.check_ib_fast_equals_general_moving(L, W.F64, steps=2)


def test_marker_out_of_domain_is_reported(L):
    full_only(L)
    P.check_marker_out_of_domain(L, steps=60)


def test_server_alone_vs_mix(L):
    full_only(L)
    P.check_server_alone_vs_mix(L, [(sp, 3) for sp, _ in P.serving_specs(scale=0.2)], max_steps=2)


def test_bulk_copy_that_never_lands_reports_timeout(L, monkeypatch):
    """Failure detection of the bulk-staged sweep, injected on the host: with the
    emulated bulk copies dropped, every mbarrier wait runs out its bounded poll
    count, the kernel returns with the timeout status instead of hanging, and the
    library stays usable once copies land again."""
    bulk_only(L)
    spec = W.CaseSpec(name="t", nx=1600, ny=5, bc=(W.PERIODIC,) * 4, ubc=((0, 0),) * 4,
                      collision=W.BGK, tau=0.8, storage=W.F32)
    monkeypatch.setenv("IBLBM_EMU_DROP_BULK_COPIES", "1")
    g = L.Lattice.from_spec(spec)
    g.step(1)
    with pytest.raises(L.IblbmError) as err:
        g.sync()
    assert err.value.code == -6   # IBLBM_ERR_TIMEOUT
    g.close()
    monkeypatch.delenv("IBLBM_EMU_DROP_BULK_COPIES")
    h = L.Lattice.from_spec(spec)
    h.step(2)
    assert h.sync() == 0
    h.close()


def test_bulk_consumer_poll_limit_gives_up(L):
    """The device-side give-up path as the GPU test drives it: consumers told to give up
    at their first wait, the launch reports the timeout status and returns, and with the
    default bound restored a fresh lattice steps to the same state as before."""
    bulk_only(L)
    spec = W.CaseSpec(name="t", nx=1600, ny=5, bc=(W.PERIODIC,) * 4, ubc=((0, 0),) * 4,
                      collision=W.BGK, tau=0.8, storage=W.F32)
    ref = L.Lattice.from_spec(spec)
    ref.step(2)
    assert ref.sync() == 0
    want = ref.populations(shifted=True)
    ref.close()
    try:
        L.test_set_consumer_poll_limit(0)
        g = L.Lattice.from_spec(spec)
        g.step(1)
        with pytest.raises(L.IblbmError) as err:
            g.sync()
        assert err.value.code == -6   # IBLBM_ERR_TIMEOUT
        g.close()
    finally:
        L.test_set_consumer_poll_limit(-1)
    h = L.Lattice.from_spec(spec)
    h.step(2)
    assert h.sync() == 0
    np.testing.assert_array_equal(h.populations(shifted=True), want)
    h.close()


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kernel", KERNELS)
def test_local_diagnostics(L, scheme, kernel):
    full_only(L)
    P.check_local_diagnostics(scheme, kernel, nx=70, ny=40, D=12.0, n=37, steps=12)


def test_local_diagnostics_free_body(L):
    full_only(L)
    P.check_local_diagnostics_free_body(steps=10)


@pytest.mark.parametrize("kernel,scheme", [(W.PESKIN4, W.DF), (W.HAT, W.DF), (W.PESKIN4, W.DFC)])
def test_taylor_green_ib(L, kernel, scheme):
    full_only(L)
    P.check_taylor_green_ib(kernel, scheme, D=8)


@pytest.mark.parametrize("name", ["walls", "periodic-x"])
def test_domain_conditions_bounce_back_walls(L, name):
    """wall_closure = 1: zero-velocity sides by on-node bounce-back, moving sides by Zou-He."""
    P.check_domain_conditions_f64(name, 33, 12, wall_closure=1)
