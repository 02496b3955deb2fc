"""Pins of the oracle's Newton-Krylov stage solver (oracle/nk.py) against
facts that do not come from it: a dense solve for FGMRES, the oracle's
complex-step element blocks for the difference Jacobian, linearity for the
V-cycle preconditioner, and the pseudo-transient solver's converged stage for
the Newton iterate."""
import numpy as np
import pytest

import oracle as O
from oracle import nk
from paper_1908_03972_gb300 import workloads as W

MA = 0.005
TINF = W.freestream_T(MA)
WT = 1.0 / np.array(W.freestream_scales(MA))
SC = np.array([TINF, 1.0, 1.0, TINF])


def _qc(q):
    rho = q[0] / q[3]
    return np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])


@pytest.fixture(scope="module")
def c1():
    """The vortex workload at its small size (8 x 8, P{2-1-0}) and the system
    of its first implicit ESDIRK3 stage (dt = 0.1)."""
    nodes, nbr = W.periodic_box(8, 8, Ng=1)
    orc = O.Oracle(nodes, nbr, 1, [2, 1, 0], [5, 10, 20], Ma_inf=MA, res_scale=W.freestream_scales(MA))
    q = W.isentropic_vortex(orc.coords())
    A, _, _ = O.esdirk3()
    odt = A[1, 1] * 0.1
    src = _qc(q) / odt + A[1, 0] / A[1, 1] * orc.residual(q)
    orc.set_stage(src, odt)
    return orc, q, src, odt


# ------------------------------------------------------------------ FGMRES
def test_fgmres_full_dimension_is_the_dense_solve():
    rng = np.random.default_rng(3)
    n = 40
    A = rng.standard_normal((n, n)) + 8.0 * np.eye(n)
    b = rng.standard_normal(n)
    x, it, res, _ = nk.fgmres(lambda z: A @ z, lambda v: v, b, n, n, 1e-14)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10 * np.abs(x).max())
    assert it <= n


def test_fgmres_restarts_reach_the_tolerance_and_report_the_true_residual():
    rng = np.random.default_rng(4)
    n = 60
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 2.0 * np.eye(n)
    b = rng.standard_normal(n)
    x, it, res, beta0 = nk.fgmres(lambda z: A @ z, lambda v: v, b, 5, 500, 1e-10)
    true = np.linalg.norm(b - A @ x)
    assert true <= 1e-10 * beta0 * 1.001
    assert abs(res - true) <= 1e-6 * beta0
    assert it > 5                                     # it did restart


def test_fgmres_with_the_exact_inverse_takes_one_iteration():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((20, 20)) + 5.0 * np.eye(20)
    Ainv = np.linalg.inv(A)
    b = rng.standard_normal(20)
    x, it, res, _ = nk.fgmres(lambda z: A @ z, lambda v: Ainv @ v, b, 10, 10, 1e-12)
    assert it == 1 and np.allclose(A @ x, b, atol=1e-10)


# ---------------------------------------------------- difference Jacobian
def test_difference_jacobian_matches_the_element_blocks(c1):
    """For z on one element, the element's rows of A z = -(F(q + h z) - F(q))/h
    equal D_e z_e with the complex-step block D_e at dtau -> infinity
    (M/(omega dt) - dR_e/dq_e), to the differencing error."""
    orc, q, src, odt = c1
    E, N = q.shape[1], q.shape[2]
    D = orc.blocks(q, 1e300)
    F = orc.stage_F(q)
    rng = np.random.default_rng(6)
    for e in (0, 27, 63):
        z = np.zeros_like(q)
        z[:, e, :] = rng.standard_normal((4, N)) * SC[:, None]
        rms = np.sqrt(np.mean((z / SC[:, None, None]) ** 2))
        h = 1e-7 / rms
        Az = -(orc.stage_F(q + h * z) - F) / h
        ref = (D[e] @ z[:, e, :].reshape(-1)).reshape(4, N)
        assert np.abs(Az[:, e, :] - ref).max() <= 1e-5 * np.abs(ref).max()


# ------------------------------------------------------ V-cycle preconditioner
def _vcycle_pc(orc, q, src, odt, r, eps, refresh):
    F = orc.stage_F(q)
    orc.set_stage(src - F + eps * r, odt)
    qp = orc.vcycle(q, 10.0, refresh=refresh)
    orc.set_stage(src, odt)
    return (qp - q) / eps


def test_vcycle_preconditioner_acts_linearly(c1):
    """z = (V(q; src - F + eps r) - q)/eps is the V-cycle linearised at q up to
    terms of the size of the perturbation: its departure from additivity
    shrinks in proportion to eps."""
    orc, q, src, odt = c1
    F = orc.stage_F(q)
    eps0 = nk.wnorm(F, WT)
    rng = np.random.default_rng(7)
    r1 = rng.standard_normal(q.shape) / WT[:, None, None] * 1e-2
    r2 = rng.standard_normal(q.shape) / WT[:, None, None] * 1e-2
    _vcycle_pc(orc, q, src, odt, r1, eps0, True)          # build the smoother at q
    dev = []
    for eps in (eps0, 1e-2 * eps0):
        z1 = _vcycle_pc(orc, q, src, odt, r1, eps, False)
        z2 = _vcycle_pc(orc, q, src, odt, r2, eps, False)
        z12 = _vcycle_pc(orc, q, src, odt, r1 + r2, eps, False)
        scale = np.abs(z12).max(axis=(1, 2))[:, None, None]
        dev.append(float((np.abs(z12 - z1 - z2) / scale).max()))
    assert dev[0] <= 0.05
    assert dev[1] <= dev[0] / 20.0, dev


# ------------------------------------------------------------------ Newton
@pytest.mark.parametrize("precond", ["vcycle", "block"])
def test_newton_krylov_reaches_the_pseudo_transient_solution(c1, precond):
    orc, q, src, odt = c1
    out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond=precond, dtau_pc=10.0, max_newton=20, m=30,
                            max_krylov=80)
    assert out["status"] == 0
    norms = out["norms"]
    assert norms[-1] <= 1e-8 * norms[0]
    assert out["newton"] <= 8
    # the last two Newton steps reduce the norm by more than 10x each (inexact Newton)
    assert norms[-1] <= 0.1 * norms[-2] and norms[-2] <= 0.1 * norms[-3]
    orc.set_stage(src, odt)
    qp, it, drop, _, st = orc.stage_solve(q)
    assert st == 0 and drop <= 1e-8
    # both stop at a 1e-8 drop: the states differ by the remaining errors
    assert np.abs(out["q"][1:3] - qp[1:3]).max() <= 1e-7
    assert np.abs(out["q"][0] - qp[0]).max() / 2.0 <= 1e-5


# ------------------------------------------------- pseudo-transient Newton
def test_pseudo_transient_newton_small_dtau_is_the_explicit_pseudo_step(c1):
    """With dtau small, (Gamma/dtau + A) delta = F gives delta = dtau Gamma^-1 F
    to first order in dtau (the explicit pseudo-time step of eq.
    preconditioning): one step with dtau = 1e-8 matches the pointwise solve
    of the oracle's Gamma to 1e-5, and halving dtau halves the step (the
    step itself is compared: at this size it vanishes in q's rounding)."""
    orc, q, src, odt = c1
    F = orc.stage_F(q)
    G = nk.gamma_field(orc, q)
    ref = np.einsum("enij,jen->ien", np.linalg.inv(G), F)
    steps = []
    for dtau in (1e-8, 0.5e-8):
        out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond="block", dtau_pc=10.0, max_newton=1, m=30,
                                max_krylov=60, eta=1e-12, ptc_dtau=dtau, tol=0.0)
        d = out["step"]
        steps.append(d)
        scale = np.abs(dtau * ref).max(axis=(1, 2))[:, None, None]
        assert (np.abs(d - dtau * ref) / scale).max() <= 1e-5
    s0 = np.abs(steps[0]).max(axis=(1, 2))
    s1 = np.abs(steps[1]).max(axis=(1, 2))
    assert np.allclose(s1 / s0, 0.5, rtol=1e-5)


def test_pseudo_transient_newton_gamma_sign_and_scale(c1):
    """With an exact linear solve, delta satisfies Gamma delta / dtau + A delta
    = F: the Newton step of the pure system at the same state, A delta_N = F,
    differs from it by the pseudo-time term, so Gamma (delta - ...) checks the
    sign and the 1/dtau: F - A delta equals Gamma delta / dtau to the linear
    tolerance, with A delta from a difference of residuals."""
    orc, q, src, odt = c1
    dtau = 0.05
    out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond="block", dtau_pc=10.0, max_newton=1, m=60,
                            max_krylov=120, eta=1e-11, ptc_dtau=dtau, tol=0.0, max_update=1e9)
    d = out["step"]
    F = orc.stage_F(q)
    h = 1e-7 / np.sqrt(np.mean((d / SC[:, None, None]) ** 2))
    Ad = -(orc.stage_F(q + h * d) - F) / h
    G = nk.gamma_field(orc, q)
    Gd = np.einsum("enij,jen->ien", G, d) / dtau
    scale = np.abs(F).max(axis=(1, 2))[:, None, None]
    assert (np.abs(F - Ad - Gd) / scale).max() <= 1e-4
    assert (np.abs(Gd) / scale).max() >= 1e-2        # the pseudo-time term is not negligible here


def test_pseudo_transient_newton_reaches_the_stage_solution(c1):
    """From dtau = 0.1 the SER-grown dtau turns the iteration into Newton: it
    stops at the stage solution of the plain Newton solver, with dtau growing
    and the last steps converging faster than 10x each."""
    orc, q, src, odt = c1
    out = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond="block", dtau_pc=10.0, max_newton=30, m=30,
                            max_krylov=80, ptc_dtau=0.1)
    assert out["status"] == 0
    norms, dt = out["norms"], out["dtaus"]
    assert norms[-1] <= 1e-8 * norms[0]
    assert dt[-1] > 100.0 * dt[0]
    assert norms[-1] <= 0.1 * norms[-2]
    ref = nk.nk_stage_solve(orc, q, src, odt, WT, SC, precond="block", dtau_pc=10.0, max_newton=20, m=30,
                            max_krylov=80)
    assert np.abs(out["q"][1:3] - ref["q"][1:3]).max() <= 1e-7
    assert np.abs(out["q"][0] - ref["q"][0]).max() / 2.0 <= 1e-5
