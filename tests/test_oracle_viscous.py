"""Pins of the oracle's viscous terms (Section 2.1 fluxes, Section 2.3 common
viscous flux with the BR2 liftings, eqs. com_q and com_grad_q).

The discrete viscous operator is isolated as R(q; mu) - R(q; 0): the inviscid
part is computed identically in both, so the difference is the FR divergence of
the viscous flux alone.  It is checked against the divergence of the paper's
viscous flux derived symbolically (sympy, from the stress and heat-flux
definitions of Section 2.1) and against two hand-derived closed forms.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

L_BOX = 10.0
GAMMA, PR = 1.4, 0.72
CP = GAMMA / (GAMMA - 1.0)


def _viscous_pair(nodes, nbr, Ng, P, mu, Ma=0.5):
    o0 = O.Oracle(nodes, nbr, Ng, [P], [1], Ma_inf=Ma)
    o1 = O.Oracle(nodes, nbr, Ng, [P], [1], Ma_inf=Ma, mu=mu)
    return o0, o1


def _weights(orc, P):
    met, _ = orc.metrics()
    b = O.basis(P)
    w2 = np.outer(b["w"], b["w"]).reshape(-1)
    return w2[None, :] * met[:, :, 4]


def _manufactured(mu):
    """Smooth periodic (p, u, v, T) and the exact div f_vis, by sympy."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    k = 2 * sp.pi / L_BOX
    fields = (
        2.0 + 0.1 * sp.sin(k * x) * sp.cos(k * y),
        0.5 + 0.3 * sp.sin(k * x + 0.3) * sp.cos(k * y),
        -0.2 + 0.25 * sp.cos(k * x) * sp.sin(k * y + 0.7),
        2.0 + 0.2 * sp.cos(k * x - 0.4) * sp.sin(k * y + 0.5),
    )
    _, u, v, T = fields
    ux, uy, vx, vy = sp.diff(u, x), sp.diff(u, y), sp.diff(v, x), sp.diff(v, y)
    div = ux + vy
    # tau_ij = 2 mu (S_ij - div/3 delta_ij); -K_j = (mu Cp / Pr) dT/dx_j
    txx = 2 * mu * (ux - div / 3)
    tyy = 2 * mu * (vy - div / 3)
    txy = 2 * mu * (uy + vx) / 2
    kap = mu * CP / PR
    fx = (0, txx, txy, u * txx + v * txy + kap * sp.diff(T, x))
    fy = (0, txy, tyy, u * txy + v * tyy + kap * sp.diff(T, y))
    div_f = [sp.diff(a, x) + sp.diff(b, y) for a, b in zip(fx, fy)]
    qf = [sp.lambdify((x, y), e, "numpy") for e in fields]
    rf = [sp.lambdify((x, y), e, "numpy") for e in div_f]
    phi = sp.lambdify((x, y), sp.sin(k * x + 0.2) * sp.cos(k * y - 0.1), "numpy")

    def ev(fs, xy):
        return np.stack([np.broadcast_to(np.asarray(f(xy[..., 0], xy[..., 1]), float), xy.shape[:-1])
                         for f in fs])
    return (lambda xy: ev(qf, xy)), (lambda xy: ev(rf, xy)), (lambda xy: phi(xy[..., 0], xy[..., 1]))


@pytest.mark.parametrize("P", [2, 3])
def test_viscous_operator_weak_error_superconverges(P):
    # BR2 with the DG correction is adjoint consistent: tested against a smooth
    # function, the error of the discrete viscous divergence falls like h^(2P)
    # on curved meshes.  A dropped correction term or a lifting with the wrong
    # component lowers the rate.
    mu = 0.05
    qf, rf, phi = _manufactured(mu)
    errs = []
    for n in (8, 16):
        nodes, nbr = W.periodic_box(n, n, 0, L_BOX, 0, L_BOX, Ng=2, perturb=0.2)
        o0, o1 = _viscous_pair(nodes, nbr, 2, P, mu)
        xy = o0.coords()
        q = qf(xy)
        d = o1.residual(q) - o0.residual(q)
        ex = rf(xy)
        assert np.abs(d[0]).max() <= 1e-13
        wJ = _weights(o0, P)
        ph = phi(xy)
        errs.append([abs(((d[v] - ex[v]) * ph * wJ).sum()) for v in (1, 2, 3)])
    errs = np.array(errs)
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates >= 2 * P - 0.5), (errs, rates)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_viscous_operator_pointwise_truncation(P):
    # Pointwise (L2 over solution points) the truncation error of the DG
    # second-derivative operator falls like h^P for odd P and h^(P-1) for even P.
    mu = 0.05
    qf, rf, _ = _manufactured(mu)
    errs = []
    for n in (8, 16):
        nodes, nbr = W.periodic_box(n, n, 0, L_BOX, 0, L_BOX, Ng=2, perturb=0.2)
        o0, o1 = _viscous_pair(nodes, nbr, 2, P, mu)
        xy = o0.coords()
        q = qf(xy)
        d = o1.residual(q) - o0.residual(q)
        ex = rf(xy)
        wJ = _weights(o0, P)
        errs.append([math.sqrt(((d[v] - ex[v]) ** 2 * wJ).sum()) for v in (1, 2, 3)])
    errs = np.array(errs)
    rates = np.log2(errs[0] / errs[1])
    expect = P if P % 2 else P - 1
    assert np.all(rates >= expect - 0.4), (errs, rates)


def test_shear_layer_and_heat_conduction_closed_forms():
    # Hand-derived: u = U0 + A sin(k y), v = 0, p, T uniform gives
    # div f_vis = (0, mu u'', 0, mu (u'^2 + u u'')); u, v, p uniform,
    # T = T0 + B cos(k x) gives (0, 0, 0, (mu Cp / Pr) T'').  On the curved
    # mesh the zero components hold to truncation error, the mass row exactly.
    mu, P = 0.05, 3
    k = 2 * math.pi / L_BOX
    U0, A, T0, B = 0.4, 0.3, 2.0, 0.2
    errs = []
    for n in (8, 16):
        nodes, nbr = W.periodic_box(n, n, 0, L_BOX, 0, L_BOX, Ng=2, perturb=0.2)
        o0, o1 = _viscous_pair(nodes, nbr, 2, P, mu)
        xy = o0.coords()
        X, Y = xy[..., 0], xy[..., 1]
        wJ = _weights(o0, P)
        one = np.ones_like(X)
        u = U0 + A * np.sin(k * Y)
        du, d2u = A * k * np.cos(k * Y), -A * k * k * np.sin(k * Y)
        q = np.stack([T0 * one, u, 0 * one, T0 * one])
        d = o1.residual(q) - o0.residual(q)
        e_shear = [math.sqrt(((d[1] - mu * d2u) ** 2 * wJ).sum()),
                   math.sqrt((d[2] ** 2 * wJ).sum()),
                   math.sqrt(((d[3] - mu * (du * du + u * d2u)) ** 2 * wJ).sum())]
        assert np.abs(d[0]).max() <= 1e-13
        T = T0 + B * np.cos(k * X)
        q = np.stack([T0 * one, 0.3 * one, 0.2 * one, T])
        d = o1.residual(q) - o0.residual(q)
        e_heat = [math.sqrt(((d[3] - mu * CP / PR * (-B * k * k * np.cos(k * X))) ** 2 * wJ).sum())]
        # uniform velocity: the stress is zero to rounding
        assert np.abs(d[:3]).max() <= 1e-12
        errs.append(e_shear + e_heat)
    errs = np.array(errs)
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates >= P - 0.5), (errs, rates)
    # RMS error under 2 % of each term's amplitude on the 16 x 16 mesh
    amp = np.array([mu * A * k * k, mu * A * k * k, mu * A * k * k * (U0 + A), mu * CP / PR * B * k * k])
    assert np.all(errs[1] / L_BOX <= 0.02 * amp), (errs, amp)


@pytest.mark.parametrize("Ng,P", [(1, 1), (2, 2), (2, 3)])
def test_viscous_terms_vanish_on_uniform_flow(Ng, P):
    nodes, nbr = W.periodic_box(3, 3, Ng=Ng, perturb=0.3 if Ng > 1 else 0.0)
    o0, o1 = _viscous_pair(nodes, nbr, Ng, P, 0.1)
    T = W.freestream_T(0.5)
    q = W.uniform_state(o0.E, o0.N(), T, 1.0, 1.0, T)
    d = o1.residual(q) - o0.residual(q)
    assert np.abs(d).max() <= 1e-12 * CP * T


def test_viscous_discrete_conservation_periodic():
    # The common viscous flux is single-valued: both elements of a face form
    # the same q_com, the same broken-gradient average and the same liftings.
    P = 3
    nodes, nbr = W.periodic_box(4, 3, Ng=2, perturb=0.3)
    orc = O.Oracle(nodes, nbr, 2, [P], [1], mu=0.02)
    xy = orc.coords()
    q = W.isentropic_vortex(xy, center=(4.0, 6.0))
    R = orc.residual(q)
    total = (R * _weights(orc, P)[None]).sum(axis=(1, 2))
    TINF = W.freestream_T(0.005)
    scale = np.array([1.0, TINF, TINF, CP * TINF]) * orc.E * 4 * 4
    assert np.all(np.abs(total) <= 1e-14 * scale), (total, scale)


def test_viscous_orientation_flag_does_not_change_residual():
    nodes, nbr = W.periodic_box(3, 3, Ng=2, perturb=0.3)
    o1 = O.Oracle(nodes, nbr, 2, [2], [1], mu=0.05)
    nodes2, nbr2 = W.flip_elements(nodes, nbr, [1, 4, 5], Ng=2)
    o2 = O.Oracle(nodes2, nbr2, 2, [2], [1], mu=0.05)
    q = W.isentropic_vortex(o1.coords())
    R1 = o1.residual(q)
    q2 = q.copy()
    for e in (1, 4, 5):
        q2[:, e] = q[:, e, ::-1]
    R2 = o2.residual(q2)
    for e in (1, 4, 5):
        R2[:, e] = R2[:, e, ::-1]
    assert np.abs(R1 - R2).max() <= 1e-10 * np.abs(R1).max()


def test_viscous_block_matches_finite_differences():
    # The complex-step block carries the viscous Jacobian, including the BR2
    # lifting's dependence on the own element's traces.
    nodes, nbr = W.periodic_box(3, 3, Ng=2, perturb=0.3)
    orc = O.Oracle(nodes, nbr, 2, [2], [1], Ma_inf=0.3, mu=0.05)
    q = W.isentropic_vortex(orc.coords(), Ma_inf=0.3, center=(4.0, 5.0))
    e, N = 4, orc.N()
    n = 4 * N
    dtau, omega_dt = 0.37, 0.05
    orc.set_stage(np.zeros(orc.shape()), omega_dt)
    D = orc.blocks(q, 1e300)[e]
    J = np.zeros((n, n))
    for c in range(n):
        v, p = divmod(c, N)
        h = 1e-6 * max(abs(q[v, e, p]), 1.0)
        qp, qm = q.copy(), q.copy()
        qp[v, e, p] += h
        qm[v, e, p] -= h
        J[:, c] = ((orc.residual(qp) - orc.residual(qm))[:, e, :] / (2 * h)).reshape(-1)
    diag = np.zeros((n, n))
    for p in range(N):
        M, _, _ = O.point_matrices(q[:, e, p], Ma_inf=0.3)
        idx = np.arange(4) * N + p
        diag[np.ix_(idx, idx)] = M / omega_dt
    ref = diag - J
    assert np.linalg.norm(D - ref) <= 1e-6 * np.linalg.norm(ref)
    # and the viscous part of it is not negligible
    o0 = O.Oracle(nodes, nbr, 2, [2], [1], Ma_inf=0.3)
    o0.set_stage(np.zeros(o0.shape()), omega_dt)
    D0 = o0.blocks(q, 1e300)[e]
    assert np.linalg.norm(D - D0) >= 1e-3 * np.linalg.norm(D0)
