"""Failure reporting of the C interface, made to happen on the host side.

Each failure is produced by its input, never by a GPU fault: a state with a
NaN in it, element blocks made singular on the host and uploaded with
pmg_set_blocks, a pseudo-iteration budget of one V-cycle, and the diagnostic
copy_wait_s < 0 that makes every bounded wait for a bulk shared-memory copy
give up at once (the kernels then finish from global memory and the library
reports PMG_ETIMEOUT).
"""
import numpy as np
import pytest

from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TINF = W.freestream_T(0.005)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()


def _qc(q):
    rho = q[0] / q[3]
    return np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])


def _solver(**kw):
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(4, 4, Ng=1)
    args = dict(p_gauge=TINF, tol=1e-8, res_scale=W.freestream_scales(0.005))
    args.update(kw)
    s = pmgfr.Solver(nodes, nbr, [2, 1, 0], [2, 3, 4], **args)
    q = W.isentropic_vortex(s.coords(), center=(4.0, 6.0))
    omega_dt = 0.0436
    # a stage source whose solution is near q (the pattern of the parity tests)
    R = s.residual(q)
    s.set_stage(_qc(q) / omega_dt + 0.5 * R, omega_dt)
    return s, q


@pytest.mark.parametrize("device_loop", [0, 1])
def test_nan_state_gives_enonfinite(device_loop):
    from paper_1908_03972_gb300 import pmgfr
    s, q = _solver(device_loop=device_loop)
    try:
        q = q.copy()
        q[1, 5, 3] = np.nan
        s.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_stage_solve(s.h)
        assert ei.value.status == pmgfr.PMG_ENONFINITE
    finally:
        s.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("kind", ["zero_row", "zero_column"])
def test_singular_block_gives_esingular_with_element(prec, kind):
    """Blocks singular in exact arithmetic: every candidate pivot of one
    column is zero.  (A row that merely repeats another leaves a rounding
    residue as its pivot, which the growth of the elimination can lift above
    the n eps floor, so that case is not reliably caught.)"""
    from paper_1908_03972_gb300 import pmgfr
    s, q = _solver(block_prec=prec)
    try:
        D = s.blocks(q, 1.0)
        bad = 11
        if kind == "zero_row":
            D[bad, 7, :] = 0.0
        else:
            D[bad, :, 9] = 0.0
        pmgfr.pmg_set_blocks(s.h, 0, np.ascontiguousarray(D))
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_factor_blocks(s.h, 0)
        assert ei.value.status == pmgfr.PMG_ESINGULAR
        assert f"element block {bad} " in str(ei.value)
        # the regular blocks factor without complaint, and the flag was cleared
        pmgfr.pmg_set_blocks(s.h, 0, np.ascontiguousarray(s.blocks(q, 1.0)))
        pmgfr.pmg_factor_blocks(s.h, 0)
    finally:
        s.close()


def test_set_blocks_round_trip_and_factor_matches_assembled():
    """Blocks uploaded with pmg_set_blocks are the ones factored and applied."""
    from paper_1908_03972_gb300 import pmgfr
    s, q = _solver(block_prec=0)
    try:
        D = s.blocks(q, 1.0)
        pmgfr.pmg_set_blocks(s.h, 0, np.ascontiguousarray(2.0 * D))
        back = pmgfr.pmg_get_blocks(s.h, 0, np.zeros_like(D))
        assert np.array_equal(back, 2.0 * D)
        s.factor()
        rng = np.random.default_rng(5)
        r = rng.standard_normal(q.shape)
        x = s.apply(r)
        for e in range(s.E):
            xe = np.linalg.solve(2.0 * D[e], r[:, e].reshape(-1))
            assert np.linalg.norm(x[:, e].reshape(-1) - xe) <= 1e-11 * np.linalg.norm(xe)
    finally:
        s.close()


@pytest.mark.parametrize("device_loop", [0, 1])
def test_pseudo_iteration_budget_gives_enotconv(device_loop):
    from paper_1908_03972_gb300 import pmgfr
    s, q = _solver(max_pseudo=1, device_loop=device_loop)
    try:
        s.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_stage_solve(s.h)
        assert ei.value.status == pmgfr.PMG_ENOTCONV
        norms, _ = pmgfr.pmg_stage_history(s.h)
        assert len(norms) == 2   # the initial norm and the one after the single V-cycle
    finally:
        s.close()


@pytest.mark.parametrize("device_loop", [0, 1])
def test_stage_solve_with_waits_that_give_up_gives_etimeout(device_loop):
    from paper_1908_03972_gb300 import pmgfr
    s, q = _solver(copy_wait_s=-1.0, device_loop=device_loop)
    try:
        s.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_stage_solve(s.h)
        assert ei.value.status == pmgfr.PMG_ETIMEOUT
    finally:
        s.close()


@pytest.mark.parametrize("flux", ["fp64", "dw_smooth"])
@pytest.mark.parametrize("prec", [0, 1])
def test_copy_wait_that_gives_up_gives_etimeout_and_same_result(prec, flux):
    """Every sweep kernel's wait for its bulk copies gives up at once: the
    V-cycle reports PMG_ETIMEOUT, and its result, computed from global memory
    instead of the shared-memory copies, is the regular one bit for bit."""
    from paper_1908_03972_gb300 import pmgfr
    mode = pmgfr.PMG_FLUX_FP64 if flux == "fp64" else pmgfr.PMG_FLUX_DW_SMOOTH
    ref, q = _solver(block_prec=prec, flux_prec=mode)
    test, _ = _solver(block_prec=prec, flux_prec=mode, copy_wait_s=-1.0)
    try:
        q_ref, _ = ref.vcycle(q, 0.7, refresh=True)
        test.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_vcycle(test.h, 0.7, True)
        assert ei.value.status == pmgfr.PMG_ETIMEOUT
        assert np.array_equal(test.get_state(), q_ref)
        # the flag is cleared once reported: a residual call afterwards is fine
        R = test.residual(q)
        assert np.isfinite(R).all()
    finally:
        ref.close()
        test.close()


def test_newton_krylov_failure_restores_stage_source_and_iterate():
    """A Newton-Krylov stage whose preconditioner V-cycles report PMG_ETIMEOUT
    (every bulk-copy wait gives up at once): the call fails with that status,
    and the stage source it rewrites for the preconditioner and the finest
    state are those of before the call, so the stage residual is unchanged."""
    from paper_1908_03972_gb300 import pmgfr
    s, q = _solver(copy_wait_s=-1.0)
    try:
        F0 = s.stage_F(q)
        pmgfr.pmg_set_stage_solver(s.h, pmgfr.PMG_STAGE_NK, state_scale=(TINF, 1.0, 1.0, TINF))
        s.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_stage_solve(s.h)
        assert ei.value.status == pmgfr.PMG_ETIMEOUT
        assert np.array_equal(s.get_state(), q)
        assert np.array_equal(s.stage_F(q), F0)
    finally:
        s.close()
