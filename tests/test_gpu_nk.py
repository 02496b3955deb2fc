"""The Newton-Krylov stage solver (pmg_set_stage_solver / PMG_STAGE_NK)
against the oracle's (oracle/nk.py), on the vortex workload at its small size
(8 x 8, P{2-1-0}, I{5-10-20}).

- One Newton step with a fixed number of FGMRES iterations (no early stop,
  no backtracking) does the same arithmetic on both sides: the corrections
  agree to the rounding of the difference Jacobian.  Its products take
  (F(q + h z) - F(q)) / h; the truncation error of the difference is the
  same on both sides, its rounding is not: the oracle keeps the absolute
  pressure p ~ 1/(gamma Ma^2) ~ 3e4 in the momentum flux, which rounds at
  ~3e-12 and reaches the product divided by the relative step.  With the
  step delta0 = 1e-4 of the state scale that is ~1e-8 of the product, and k
  Krylov steps with a preconditioned condition number of ~10 give the 1e-6
  bound below (with the default 1e-7 step the corrections differ by 3e-5).
- Whole stages reach a 1e-8 drop in a handful of Newton steps and land on
  the oracle's converged state within the bounds of the pseudo-transient
  stage parity tests (1e-7 of rho |v|^2 and of |v|).
- An ESDIRK3 step with Newton-Krylov stages agrees with the pseudo-transient
  step (velocity 1e-7; pressure 1e-5 of rho |v|^2, the remainder the
  pseudo-transient stop leaves in the slow pressure mode), with far fewer
  V-cycles.
"""
import numpy as np
import pytest

import oracle as O
from oracle import nk
from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MA = 0.005
TINF = W.freestream_T(MA)
WT = 1.0 / np.array(W.freestream_scales(MA))
SC = (TINF, 1.0, 1.0, TINF)
KW = dict(tol=1e-8, res_scale=W.freestream_scales(MA))


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


def _pair(prec=1, gauge=TINF, n=8):
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(n, n, Ng=1)
    orc = O.Oracle(nodes, nbr, 1, [2, 1, 0], [5, 10, 20], Ma_inf=MA, **KW)
    gpu = pmgfr.Solver(nodes, nbr, [2, 1, 0], [5, 10, 20], Ma_inf=MA, block_prec=prec, p_gauge=gauge, **KW)
    q = W.isentropic_vortex(orc.coords())
    A, _, _ = O.esdirk3()
    odt = A[1, 1] * 0.1
    src = _qc(q) / odt + A[1, 0] / A[1, 1] * orc.residual(q)
    orc.set_stage(src, odt)
    gpu.set_stage(src, odt)
    return orc, gpu, q, src, odt


@pytest.mark.parametrize("precond", ["block", "vcycle"])
@pytest.mark.parametrize("k", [1, 4])
def test_one_newton_step_with_fixed_krylov_count_matches_oracle(precond, k):
    from paper_1908_03972_gb300 import pmgfr
    orc, gpu, q, src, odt = _pair(prec=0)
    try:
        pc = pmgfr.PMG_NK_PC_BLOCK if precond == "block" else pmgfr.PMG_NK_PC_VCYCLE
        pmgfr.pmg_set_stage_solver(gpu.h, pmgfr.PMG_STAGE_NK, max_newton=1, krylov_dim=k, max_krylov=k, eta=1e-30,
                                   precond=pc, dtau_pc=10.0, delta0=1e-4, state_scale=SC, max_backtrack=0)
        gpu.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_stage_solve(gpu.h)
        assert ei.value.status == pmgfr.PMG_ENOTCONV
        dg = gpu.get_state() - q
        out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond=precond, dtau_pc=10.0, max_newton=1, m=k,
                                max_krylov=k, eta=1e-30, max_backtrack=0, delta0=1e-4)
        do = out["q"] - q
        st = pmgfr.pmg_nk_stats_read(gpu.h, reset=True)
        assert st["newton"] == 1 and st["krylov"] == k
        assert st["vcycles"] == (k if precond == "vcycle" else 0)
        for v in range(4):
            scale = np.abs(do[v]).max()
            assert np.abs(dg[v] - do[v]).max() <= 1e-6 * scale, (v, np.abs(dg[v] - do[v]).max(), scale)
    finally:
        gpu.close()


@pytest.mark.parametrize("precond", ["block", "vcycle"])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_stage_converges_to_the_oracle_solution(precond, prec):
    from paper_1908_03972_gb300 import pmgfr
    orc, gpu, q, src, odt = _pair(prec=prec)
    try:
        pc = pmgfr.PMG_NK_PC_BLOCK if precond == "block" else pmgfr.PMG_NK_PC_VCYCLE
        pmgfr.pmg_set_stage_solver(gpu.h, pmgfr.PMG_STAGE_NK, krylov_dim=30, max_krylov=80, precond=pc,
                                   dtau_pc=10.0, state_scale=SC)
        qg, it, drop = gpu.stage_solve(q)
        assert drop <= 1e-8 and it <= 10
        out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond=precond, dtau_pc=10.0, m=30, max_krylov=80)
        assert out["status"] == 0
        if prec == 0:
            assert abs(it - out["newton"]) <= 1
        assert np.abs(qg[0] - out["q"][0]).max() / 2.0 <= 1e-7
        assert np.abs(qg[1:3] - out["q"][1:3]).max() <= 1e-7
        norms, dtau = pmgfr.pmg_stage_history(gpu.h)
        assert len(norms) == it + 1 and np.all(dtau == 0.0)
    finally:
        gpu.close()


@pytest.mark.parametrize("precond", ["block", "vcycle"])
def test_one_pseudo_transient_newton_step_matches_oracle(precond):
    """One pseudo-transient Newton step (dtau = 0.05, four FGMRES iterations,
    no early stop): the product carries Gamma(q) z / dtau, the preconditioner
    takes min(dtau, dtau_pc); the corrections agree to the bound of the plain
    Newton step."""
    from paper_1908_03972_gb300 import pmgfr
    orc, gpu, q, src, odt = _pair(prec=0)
    k = 4
    try:
        pc = pmgfr.PMG_NK_PC_BLOCK if precond == "block" else pmgfr.PMG_NK_PC_VCYCLE
        pmgfr.pmg_set_stage_solver(gpu.h, pmgfr.PMG_STAGE_NK, max_newton=1, krylov_dim=k, max_krylov=k, eta=1e-30,
                                   precond=pc, dtau_pc=10.0, delta0=1e-4, state_scale=SC, ptc_dtau=0.05)
        gpu.set_state(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_stage_solve(gpu.h)
        assert ei.value.status == pmgfr.PMG_ENOTCONV
        dg = gpu.get_state() - q
        out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond=precond, dtau_pc=10.0, max_newton=1, m=k,
                                max_krylov=k, eta=1e-30, delta0=1e-4, ptc_dtau=0.05)
        do = out["q"] - q
        for v in range(4):
            scale = np.abs(do[v]).max()
            assert np.abs(dg[v] - do[v]).max() <= 1e-6 * scale, (v, np.abs(dg[v] - do[v]).max(), scale)
        norms, dtau = pmgfr.pmg_stage_history(gpu.h)
        assert dtau[0] == 0.05 and dtau[1] == pytest.approx(0.05 * (norms[0] / norms[1]) ** 1.5, rel=1e-12)
    finally:
        gpu.close()


@pytest.mark.parametrize("precond", ["block", "vcycle"])
def test_pseudo_transient_newton_stage_converges_to_the_oracle_solution(precond):
    """From dtau = 0.1 the stage reaches a 1e-8 drop on the oracle's converged
    state, with the oracle's dtau sequence to the rounding of the norms it is
    formed from.  Velocity to the bound of the Newton stage test (1e-7);
    pressure to the bound of the Newton-against-pseudo-transient comparison
    (1e-5 of rho |v|^2): both sides stop at a 1e-8 drop, and what is left is
    a near-uniform pressure offset (measured 5e-7), the slow pressure mode
    that the pseudo-time term damps last."""
    from paper_1908_03972_gb300 import pmgfr
    orc, gpu, q, src, odt = _pair(prec=0)
    try:
        pc = pmgfr.PMG_NK_PC_BLOCK if precond == "block" else pmgfr.PMG_NK_PC_VCYCLE
        pmgfr.pmg_set_stage_solver(gpu.h, pmgfr.PMG_STAGE_NK, krylov_dim=30, max_krylov=80, precond=pc,
                                   dtau_pc=10.0, state_scale=SC, ptc_dtau=0.1)
        qg, it, drop = gpu.stage_solve(q)
        assert drop <= 1e-8 and it <= 10
        out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond=precond, dtau_pc=10.0, m=30, max_krylov=80,
                                ptc_dtau=0.1)
        assert out["status"] == 0 and abs(it - out["newton"]) <= 1
        assert np.abs(qg[1:3] - out["q"][1:3]).max() <= 1e-7
        assert np.abs(qg[0] - out["q"][0]).max() / 2.0 <= 1e-5
        norms, dtau = pmgfr.pmg_stage_history(gpu.h)
        assert len(norms) == it + 1
        n = min(3, len(out["dtaus"]))
        assert np.allclose(dtau[:n], out["dtaus"][:n], rtol=1e-3)
    finally:
        gpu.close()


def test_esdirk_step_with_newton_krylov_stages_matches_pseudo_transient():
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(8, 8, Ng=1)
    res = {}
    for solver in (pmgfr.PMG_STAGE_PTC, pmgfr.PMG_STAGE_NK):
        gpu = pmgfr.Solver(nodes, nbr, [2, 1, 0], [5, 10, 20], Ma_inf=MA, block_prec=1, p_gauge=TINF,
                           dtau_init=0.01, dtau_max=10.0, refresh_every=10, max_pseudo=4000, **KW)
        try:
            if solver == pmgfr.PMG_STAGE_NK:
                pmgfr.pmg_set_stage_solver(gpu.h, solver, krylov_dim=30, max_krylov=80, dtau_pc=10.0,
                                           state_scale=SC)
            q = W.isentropic_vortex(gpu.coords())
            qs, st = gpu.esdirk_step(q, 0.1)
            res[solver] = (qs, st.n_vcycles, list(st.pseudo_iters[:3]))
        finally:
            gpu.close()
    qp, vp, _ = res[pmgfr.PMG_STAGE_PTC]
    qn, vn, newton = res[pmgfr.PMG_STAGE_NK]
    assert all(1 <= k <= 10 for k in newton), newton
    assert vn < vp / 3, (vn, vp)
    # both stop at a 1e-8 drop of the scaled norm, which leaves different
    # remainders: pseudo-time marching leaves the slow pressure mode (its
    # decay per V-cycle is the slowest), Newton does not; the bounds are those
    # of the oracle's own Newton-against-pseudo-transient pin
    assert np.abs(qn[0] - qp[0]).max() / 2.0 <= 1e-5
    assert np.abs(qn[1:3] - qp[1:3]).max() <= 1e-7


def test_stage_solver_options_are_validated():
    from paper_1908_03972_gb300 import pmgfr
    orc, gpu, q, src, odt = _pair()
    try:
        for bad in (dict(krylov_dim=65), dict(precond=7), dict(eta=1.5), dict(delta0=2.0),
                    dict(ptc_dtau=float("inf"))):
            with pytest.raises(pmgfr.PmgError) as ei:
                pmgfr.pmg_set_stage_solver(gpu.h, pmgfr.PMG_STAGE_NK, **bad)
            assert ei.value.status == pmgfr.PMG_EINVAL
        with pytest.raises(pmgfr.PmgError):
            pmgfr.pmg_set_stage_solver(gpu.h, 5)
    finally:
        gpu.close()


@pytest.mark.parametrize("gauge,ptc", [(False, 0.0), (True, 0.0), (True, 0.2)])
def test_one_newton_step_on_hexahedra_matches_oracle(gauge, ptc):
    """The same fixed-count Newton step on the cubed-sphere shell (2 x 2 x 6
    elements per panel, Q2 hexahedra, slip wall, Ma = 0.001, P{2-1-0}) from
    the free stream with noise in v: five variables, the hexahedral residual
    and V-cycle as the preconditioner (measured differences 2e-9 with one
    Krylov step, 2e-7 with two); with ptc > 0 the pseudo-transient Newton
    step (Gamma/dtau added to the product, the V-cycle at min(dtau,
    dtau_pc))."""
    from paper_1908_03972_gb300 import pmgfr
    ma = 0.001
    T = W.freestream_T(ma, speed=1.0)
    nodes, nbr = W.cubed_sphere_shell(2, 6, 0.5, 20.0, Ng=2)
    kw = dict(Ma_inf=ma, cutoff=1, kappa=1.0)
    orc = O.Oracle3(nodes, nbr, 2, [2, 1, 0], [5, 10, 20], q_inf=(T, 1.0, 0.0, 0.0, T),
                    res_scale=W.freestream_scales3(ma, speed=1.0), **kw)
    gpu = pmgfr.Solver(nodes, nbr, [2, 1, 0], [5, 10, 20], block_prec=0, dim=3, q_inf3=(T, 1.0, 0.0, 0.0, T),
                       res_scale3=W.freestream_scales3(ma, speed=1.0), p_gauge=T if gauge else 0.0, **kw)
    try:
        E, N, _ = orc.coords().shape
        q = W.uniform_state3(E, N, T, 1.0, 0.0, 0.0, T)
        q[2] += 1e-3 * np.random.default_rng(7).standard_normal((E, N))
        A, _, _ = O.esdirk3()
        odt = A[1, 1] * 0.1
        rho = q[0] / q[4]
        qc = np.stack([rho, rho * q[1], rho * q[2], rho * q[3],
                       rho * (q[4] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2))])
        src = qc / odt + orc.residual(q)
        orc.set_stage(src, odt)
        gpu.set_stage(src, odt)
        sc = (T, 1.0, 1.0, 1.0, T)
        k = 2
        pmgfr.pmg_set_stage_solver(gpu.h, pmgfr.PMG_STAGE_NK, max_newton=1, krylov_dim=k, max_krylov=k, eta=1e-30,
                                   dtau_pc=1.0, delta0=1e-4, state_scale=sc, max_backtrack=0, ptc_dtau=ptc)
        gpu.set_state(q)
        with pytest.raises(pmgfr.PmgError):
            pmgfr.pmg_stage_solve(gpu.h)
        dg = gpu.get_state() - q
        out = nk.nk_stage_solve(orc, q, src, odt, 1.0 / np.array(W.freestream_scales3(ma, speed=1.0)), np.array(sc),
                                precond="vcycle", dtau_pc=1.0, max_newton=1, m=k, max_krylov=k, eta=1e-30,
                                max_backtrack=0, delta0=1e-4, ptc_dtau=ptc)
        do = out["q"] - q
        for v in range(5):
            assert np.abs(dg[v] - do[v]).max() <= 1e-6 * np.abs(do[v]).max(), v
    finally:
        gpu.close()
