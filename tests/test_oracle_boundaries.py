"""Pins of the oracle's boundary faces (ghost states through the common
fluxes of Section 2.3; the paper states no boundary treatment).

Each check compares with a fact fixed independently of the oracle's formulas:
uniform flows that a boundary must leave at rest, conservation through an
adiabatic wall, the sign and viscosity scaling of wall drag, the symbolic
divergence of the viscous flux (sympy) for fields that satisfy the wall
conditions, and finite differences of the full residual.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

GAMMA, PR = 1.4, 0.72
CP = GAMMA / (GAMMA - 1.0)


def _weights(orc, P):
    met, _ = orc.metrics()
    b = O.basis(P)
    w2 = np.outer(b["w"], b["w"]).reshape(-1)
    return w2[None, :] * met[:, :, 4]


@pytest.mark.parametrize("P", [2, 3, 4])
def test_far_field_keeps_the_free_stream_on_a_curved_annulus(P):
    Ma = 0.5
    T = W.freestream_T(Ma, speed=1.0)
    nodes, nbr = W.cylinder_omesh(3, 12, r_in=0.5, r_out=5.0, Ng=2, wall=W.BC_FARFIELD, outer=W.BC_FARFIELD)
    orc = O.Oracle(nodes, nbr, 2, [P], [1], Ma_inf=Ma, q_inf=(T, 1.0, 0.0, T))
    R = orc.residual(W.uniform_state(orc.E, orc.N(), T, 1.0, 0.0, T))
    scale = np.array([1.0, T, T, CP * T])
    assert np.all(np.abs(R).max(axis=(1, 2)) <= 1e-12 * scale)


@pytest.mark.parametrize("Ng,P", [(1, 1), (2, 2), (2, 3)])
def test_slip_walls_keep_a_parallel_uniform_flow(Ng, P):
    Ma = 0.5
    T = W.freestream_T(Ma, speed=1.0)
    nodes, nbr = W.channel(4, 3, Ng=Ng, perturb=0.3 if Ng > 1 else 0.0,
                           bottom=W.BC_SLIP_WALL, top=W.BC_SLIP_WALL)
    orc = O.Oracle(nodes, nbr, Ng, [P], [1], Ma_inf=Ma)
    R = orc.residual(W.uniform_state(orc.E, orc.N(), T, 1.0, 0.0, T))
    scale = np.array([1.0, T, T, CP * T])
    assert np.all(np.abs(R).max(axis=(1, 2)) <= 1e-12 * scale)


def test_no_slip_walls_keep_a_fluid_at_rest():
    T = W.freestream_T(0.3, speed=1.0)
    nodes, nbr = W.channel(4, 3, Ng=2, perturb=0.3)
    orc = O.Oracle(nodes, nbr, 2, [3], [1], Ma_inf=0.3, cutoff=1, mu=0.05)
    R = orc.residual(W.uniform_state(orc.E, orc.N(), T, 0.0, 0.0, T))
    assert np.all(np.abs(R).max(axis=(1, 2)) <= 1e-12 * np.array([1.0, T, T, CP * T]))


def test_no_slip_wall_needs_the_eps_cut_off_and_slip_walls_no_viscosity():
    nodes, nbr = W.channel(4, 3, Ng=1)
    with pytest.raises(ValueError):
        O.Oracle(nodes, nbr, 1, [2], [1], cutoff=0)     # eps = Ma = 0 at the wall state
    nodes, nbr = W.channel(4, 3, Ng=1, bottom=W.BC_SLIP_WALL, top=W.BC_SLIP_WALL)
    with pytest.raises(ValueError):
        O.Oracle(nodes, nbr, 1, [2], [1], mu=0.1)


def test_adiabatic_walls_let_no_energy_through():
    # A fluid at rest, hottest at both walls: heat conducts inside, but
    # adiabatic walls supply none, so the total energy stays, and walls at rest
    # pass no mass.  (Heat flux through the walls would add energy at both.)
    T0 = W.freestream_T(0.3, speed=1.0)
    P = 3
    nodes, nbr = W.channel(6, 4, Ng=2, perturb=0.3)
    orc = O.Oracle(nodes, nbr, 2, [P], [1], Ma_inf=0.3, cutoff=1, mu=0.05)
    xy = orc.coords()
    T = T0 * (1.0 + 0.01 * (xy[..., 1] - 1.0) ** 2 + 0.005 * np.sin(2 * math.pi * xy[..., 0] / 10.0))
    q = np.stack([np.full_like(T, T0), np.zeros_like(T), np.zeros_like(T), T])
    R = orc.residual(q)
    tot = (R * _weights(orc, P)[None]).sum(axis=(1, 2))
    local = np.abs(R[3]).max()
    assert local > 1e-6                    # heat does flow inside
    assert abs(tot[0]) <= 1e-13 and abs(tot[3]) <= 1e-10 * local * orc.E


def test_no_slip_walls_drag_a_sliding_flow_in_proportion_to_mu():
    Ma = 0.3
    T = W.freestream_T(Ma, speed=1.0)
    P = 2
    nodes, nbr = W.channel(6, 4, Ng=2, perturb=0.3)
    kw = dict(Ma_inf=Ma, cutoff=1)
    for U in (0.3, -0.3):
        V = []
        for mu in (0.0, 0.02, 0.04):
            orc = O.Oracle(nodes, nbr, 2, [P], [1], mu=mu, **kw)
            q = W.uniform_state(orc.E, orc.N(), T, U, 0.0, T)
            wJ = _weights(orc, P)
            V.append((orc.residual(q) * wJ[None]).sum(axis=(1, 2)))
        drag1 = V[1][1] - V[0][1]
        drag2 = V[2][1] - V[0][1]
        assert np.sign(drag1) == -np.sign(U) and abs(drag1) > 1e-6      # the walls decelerate the flow
        assert abs(drag2 - 2 * drag1) <= 1e-9 * abs(drag1)              # the viscous part is linear in mu
    # slip walls exert no force on it
    nodes2, nbr2 = W.channel(6, 4, Ng=2, perturb=0.3, bottom=W.BC_SLIP_WALL, top=W.BC_SLIP_WALL)
    orc = O.Oracle(nodes2, nbr2, 2, [P], [1], **kw)
    R = orc.residual(W.uniform_state(orc.E, orc.N(), T, 0.3, 0.0, T))
    assert abs((R[1] * _weights(orc, P)).sum()) <= 1e-12 * T


def _wall_field(mu):
    """A field that meets no-slip adiabatic walls at y = 0 and y = 2 (nonzero
    wall shear), and the symbolic divergence of its viscous flux."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    k, eta, T0 = 2 * sp.pi / 10.0, y / 2.0, 2.0
    fields = (T0 + 0.1 * sp.cos(k * x) * sp.sin(sp.pi * eta),
              0.3 * sp.sin(sp.pi * eta) * (1 + 0.5 * sp.sin(k * x)),
              0.2 * sp.sin(sp.pi * eta) * sp.cos(k * x),
              T0 + 0.2 * sp.cos(sp.pi * eta) * sp.cos(k * x))
    _, u, v, T = fields
    ux, uy, vx, vy = sp.diff(u, x), sp.diff(u, y), sp.diff(v, x), sp.diff(v, y)
    div = ux + vy
    txx, tyy, txy = 2 * mu * (ux - div / 3), 2 * mu * (vy - div / 3), mu * (uy + vx)
    kap = mu * CP / PR
    fx = (0, txx, txy, u * txx + v * txy + kap * sp.diff(T, x))
    fy = (0, txy, tyy, u * txy + v * tyy + kap * sp.diff(T, y))
    lam = [sp.lambdify((x, y), e, "numpy") for e in fields]
    lamR = [sp.lambdify((x, y), sp.diff(a, x) + sp.diff(b, y), "numpy") for a, b in zip(fx, fy)]
    phis = [sp.lambdify((x, y), sp.cos(0.7 * sp.pi * eta + 0.2) * sp.cos(k * x + 0.3), "numpy"),
            sp.lambdify((x, y), sp.sin(sp.pi * eta) * sp.cos(k * x + 0.3), "numpy")]

    def ev(fs, xy):
        return np.stack([np.broadcast_to(np.asarray(f(xy[..., 0], xy[..., 1]), float), xy.shape[:-1])
                         for f in fs])
    return (lambda xy: ev(lam, xy)), (lambda xy: ev(lamR, xy)), phis


@pytest.mark.parametrize("P", [2, 3])
def test_viscous_operator_with_walls_converges(P):
    # Tested against a smooth function that does not vanish on the walls the
    # error falls like h^P in momentum (the wall shear stress) and h^4 in
    # energy; against one that vanishes there, like h^(2P) in momentum.  A
    # wall gradient without the element's own trace drops the first to ~0.
    mu = 0.05
    qf, rf, phis = _wall_field(mu)
    errs = [[], []]
    for n in (4, 8):
        nodes, nbr = W.channel(2 * n, n, 0, 10.0, 0, 2.0, Ng=2, perturb=0.2)
        kw = dict(Ma_inf=0.3, cutoff=1)
        o0 = O.Oracle(nodes, nbr, 2, [P], [1], **kw)
        o1 = O.Oracle(nodes, nbr, 2, [P], [1], mu=mu, **kw)
        xy = o0.coords()
        q = qf(xy)
        d = o1.residual(q) - o0.residual(q)
        ex = rf(xy)
        wJ = _weights(o0, P)
        for i, ph in enumerate(phis):
            pv = ph(xy[..., 0], xy[..., 1])
            errs[i].append([abs(((d[v] - ex[v]) * pv * wJ).sum()) for v in (1, 2, 3)])
    generic, vanishing = (np.log2(np.array(e)[0] / np.array(e)[1]) for e in errs)
    assert np.all(generic[:2] >= P - 0.5) and generic[2] >= 3.4, generic
    assert np.all(vanishing[:2] >= 2 * P - 0.5), vanishing


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_boundary_blocks_match_finite_differences(mu):
    # The complex-step blocks carry the ghost states' dependence on the own
    # trace (no-slip bottom wall, far-field top).
    Ma = 0.3
    T = W.freestream_T(Ma, speed=1.0)
    nodes, nbr = W.channel(3, 3, Ng=2, perturb=0.3, top=W.BC_FARFIELD)
    orc = O.Oracle(nodes, nbr, 2, [2], [1], Ma_inf=Ma, cutoff=1, mu=mu, q_inf=(T, 1.0, 0.0, T))
    xy = orc.coords()
    rng = np.random.default_rng(5)
    q = W.uniform_state(orc.E, orc.N(), T, 0.7, 0.1, T)
    q = q * (1 + 0.02 * rng.standard_normal(q.shape) * np.array([1e-3, 1, 1, 1e-3])[:, None, None])
    omega_dt = 0.05
    orc.set_stage(np.zeros(orc.shape()), omega_dt)
    N, n = orc.N(), 4 * orc.N()
    for e in (1, 7):                     # a wall element and a far-field element
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
            M, _, _ = O.point_matrices(q[:, e, p], Ma_inf=Ma, cutoff=1)
            idx = np.arange(4) * N + p
            diag[np.ix_(idx, idx)] = M / omega_dt
        ref = diag - J
        assert np.linalg.norm(D - ref) <= 1e-6 * np.linalg.norm(ref), e
