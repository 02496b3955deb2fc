"""Pins of the oracle's viscous terms on hexahedra (Section 2.1 viscous
fluxes, Section 2.3 eq. com_q and eq. com_grad_q with d = 3) against facts
that do not come from the three-dimensional code itself:

- reduction to the pinned two-dimensional viscous oracle: a quadrilateral
  mesh extruded along z (periodic box; the channel between no-slip walls; the
  cylinder O-mesh with its wall and far field) with a z-independent state,
  w = 0, gives the 2D residual layer by layer in mass, x- and y-momentum and
  energy.  (The z-momentum residual does not vanish: tau_zz = -2/3 mu div u
  is constant along z, but at the zeta faces the interface flux takes the
  broken gradient and the interior flux the corrected one, which differ where
  the state jumps across the x and y faces -- a property of the BR2 scheme,
  not of the reduction.);
- invariance under the renumbering of rotated elements' points (every
  reference direction and face orientation carries the same viscous terms);
- discrete conservation of mass, momentum and energy on a periodic mesh;
- a closed form: for the shear layer u = U sin(2 pi z / Lz) at constant p
  and T the residual is mu u'' in x-momentum and mu (u u')' in energy, to
  the discretisation error, which falls with P;
- the complex-step element blocks against central differences of the
  element's residual with its neighbours frozen.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

MU = 0.02
MAP = ((0, 0), (1, 1), (2, 2), (3, 4))   # 2D variable -> 3D variable


def _layers(q2, P):
    n1 = P + 1
    return [slice(kk * n1 * n1, (kk + 1) * n1 * n1) for kk in range(n1)]


def _lift(q2, shape3, P):
    q3 = np.zeros(shape3)
    for sl in _layers(q2, P):
        for v2, v3 in MAP:
            q3[v3, :, sl] = q2[v2]
    return q3


def _compare_2d(o2, o3, q2, P, tol=1e-11):
    q3 = _lift(q2, o3.shape(), P)
    R2, R3 = o2.residual(q2), o3.residual(q3)
    for sl in _layers(q2, P):
        for v2, v3 in MAP:
            assert np.abs(R3[v3, :, sl] - R2[v2]).max() <= tol * np.abs(R2[v2]).max(), v2
    return R2


@pytest.mark.parametrize("Ng,P,n2", [(1, 0, (4, 3)), (1, 2, (4, 3)), (1, 3, (3, 3)), (2, 2, (3, 3)), (2, 3, (3, 2))])
def test_viscous_residual_reduces_to_the_2d_residual(Ng, P, n2):
    nodes2, nbr2 = W.periodic_box(*n2, Ng=Ng, perturb=0.3 if Ng > 1 else 0.0)
    nodes3, nbr3 = W.extrude(nodes2, nbr2, Ng, nz=1, z0=0.0, z1=1.0)
    o2 = O.Oracle(nodes2, nbr2, Ng, [P], [1], Ma_inf=0.3, mu=MU)
    o3 = O.Oracle3(nodes3, nbr3, Ng, [P], [1], Ma_inf=0.3, mu=MU)
    q2 = W.isentropic_vortex(o2.coords(), Ma_inf=0.3, center=(4.3, 5.6))
    R2 = _compare_2d(o2, o3, q2, P)
    # the viscous terms are not negligible in this comparison
    o2i = O.Oracle(nodes2, nbr2, Ng, [P], [1], Ma_inf=0.3)
    assert np.abs(R2[1] - o2i.residual(q2)[1]).max() >= 1e-3 * np.abs(R2[1]).max()


@pytest.mark.parametrize("P", [1, 2])
def test_viscous_walls_reduce_to_the_2d_walls(P):
    """No-slip walls (the channel) and a wall plus far field (the cylinder
    O-mesh), extruded: the boundary ghost states, mirrored gradients and the
    missing viscous energy flux at walls match the 2D oracle's."""
    T = W.freestream_T(0.2, speed=1.0)
    for nodes2, nbr2, Ng in (W.channel(4, 3, Ng=1) + (1,), W.cylinder_omesh(3, 8, r_out=6.0, Ng=2) + (2,)):
        qinf = (T, 1.0, 0.0, T)
        kw = dict(Ma_inf=0.2, mu=MU, cutoff=1, kappa=1.0)
        o2 = O.Oracle(nodes2, nbr2, Ng, [P], [1], q_inf=qinf, **kw)
        nodes3, nbr3 = W.extrude(nodes2, nbr2, Ng, nz=1)
        o3 = O.Oracle3(nodes3, nbr3, Ng, [P], [1], q_inf=(T, 1.0, 0.0, 0.0, T), **kw)
        xy = o2.coords()
        rng = np.random.default_rng(4)
        q2 = np.stack([T * (1 + 0.01 * np.sin(xy[..., 0])), 0.5 + 0.3 * np.cos(xy[..., 1]) + 0.1 * xy[..., 0] / 10,
                       0.2 * np.sin(xy[..., 0] + xy[..., 1]), T * (1 + 0.02 * np.cos(xy[..., 0]))])
        q2 = q2 * (1 + 1e-3 * rng.standard_normal(q2.shape))
        _compare_2d(o2, o3, q2, P, tol=1e-10)


def _box(P, rot=None, mu=MU):
    nodes, nbr = W.periodic_box3d(3, 2, 2, Ng=2, perturb=0.3, rotations=rot or {})
    return O.Oracle3(nodes, nbr, 2, [P], [1], Ma_inf=0.3, mu=mu)


def test_viscous_residual_invariant_under_element_renumbering():
    P = 2
    rot = {0: 5, 3: 17, 5: 11, 8: 20, 10: 2}
    o0, o1 = _box(P), _box(P, rot)
    x0, x1 = o0.coords(), o1.coords()
    R0 = o0.residual(W.vortex3d(x0, Ma_inf=0.3, center=(4.3, 5.6)))
    R1 = o1.residual(W.vortex3d(x1, Ma_inf=0.3, center=(4.3, 5.6)))
    for e in range(o0.E):
        d = np.linalg.norm(x0[e][:, None, :] - x1[e][None, :, :], axis=2)
        perm = d.argmin(axis=1)
        for v in range(5):
            assert np.allclose(R1[v, e, perm], R0[v, e], rtol=0, atol=1e-11 * np.abs(R0[v]).max())


@pytest.mark.parametrize("P", [1, 2, 3])
def test_viscous_discrete_conservation_with_rotated_elements(P):
    orc = _box(P, {1: 3, 4: 13, 6: 22, 10: 8})
    _, J, _, xyz = orc.geometry()
    q = W.vortex3d(xyz, Ma_inf=0.3, center=(4.3, 5.6))
    R = orc.residual(q)
    w = np.polynomial.legendre.leggauss(P + 1)[1]
    wJ = np.einsum("k,j,i->kji", w, w, w).reshape(-1)[None, :] * J
    for v in range(5):
        assert abs((wJ * R[v]).sum()) <= 1e-11 * (wJ * np.abs(R[v])).sum(), v


def test_shear_layer_closed_form():
    """u = U sin(k z), p and T constant, v = w = 0 (eps cut-off on: u = 0 at
    some points): the inviscid fluxes are constant along their directions,
    and R = div f_vis gives mu u'' in x-momentum and mu (u u')' in energy;
    mass and y-momentum stay at rounding, and the error of x-momentum,
    energy and z-momentum (the BR2 interface/interior difference) falls with
    P on four elements per wavelength."""
    Lz, U = 10.0, 0.3
    k = 2 * math.pi / Lz
    T = W.freestream_T(0.3, speed=1.0)
    errs, rw = [], []
    for P in (3, 4, 5):
        nodes, nbr = W.periodic_box3d(2, 2, 4, Ng=1)
        orc = O.Oracle3(nodes, nbr, 1, [P], [1], Ma_inf=0.3, mu=MU, cutoff=1, kappa=1.0)
        xyz = orc.coords()
        z = xyz[..., 2]
        q = W.uniform_state3(orc.E, xyz.shape[1], T, 0.0, 0.0, 0.0, T)
        q[1] = U * np.sin(k * z)
        R = orc.residual(q)
        ux = -MU * U * k * k * np.sin(k * z)
        en = MU * U * U * k * k * np.cos(2 * k * z)
        e1 = np.abs(R[1] - ux).max() / np.abs(ux).max()
        e4 = np.abs(R[4] - en).max() / np.abs(en).max()
        assert np.abs(R[[0, 2]]).max() <= 1e-9 * np.abs(ux).max()
        errs.append(max(e1, e4))
        rw.append(np.abs(R[3]).max() / np.abs(ux).max())
    assert errs[-1] <= 2e-2, errs
    assert errs[2] < errs[1] < errs[0], errs
    assert rw[2] < rw[1] < rw[0] and rw[-1] <= 2e-3, rw


def test_viscous_blocks_match_central_differences():
    P = 1
    orc = _box(P, {1: 3, 4: 13})
    xyz = orc.coords()
    q = W.vortex3d(xyz, Ma_inf=0.3, center=(4.3, 5.6))
    orc.set_stage(np.zeros_like(q), 0.5)
    D = orc.blocks(q, 1e300)
    N = xyz.shape[1]
    h = 1e-6
    for e in (0, 5):
        for col in (1 * N + 2, 3 * N + 5, 4 * N + 0):
            v, p = divmod(col, N)
            dq = np.zeros_like(q)
            dq[v, e, p] = h * max(1.0, abs(q[v, e, p]))
            # element residual with neighbours frozen: differences of the
            # global residual restricted to element e change only through e
            Rp = orc.stage_F(q + dq)[:, e].reshape(-1)
            Rm = orc.stage_F(q - dq)[:, e].reshape(-1)
            fd = -(Rp - Rm) / (2 * dq[v, e, p])
            assert np.abs(D[e][:, col] - fd).max() <= 1e-6 * np.abs(D[e][:, col]).max(), (e, col)


def test_extruded_ellipse_mesh():
    """The extruded-ellipse mesh: wall nodes on the ellipse (chord 1,
    thickness 0.1), far-field nodes on the confocal ellipse through x = 20,
    positive Jacobians at every solution point, symmetric connectivity
    (periodic in z and around), and a P = 2 free stream kept steady by the
    oracle's conservative-curl metrics (P >= geometry order)."""
    nr, nt, nz = 4, 12, 3
    nodes, nbr = W.extruded_ellipse(nr, nt, nz, span=0.2, Ng=2)
    assert nodes.shape == (nr * nt * nz, 27, 3)
    n1 = 3
    for e in range(nodes.shape[0]):
        for f in range(6):
            en, fn, o = nbr[e, f]
            if en < 0:
                assert (f, fn) in ((0, 3), (1, 4)), (e, f, fn)
                pts = nodes[e].reshape(n1, n1, n1, 3)[:, :, 0 if f == 0 else -1, :2].reshape(-1, 2)
                if f == 0:
                    assert np.abs((pts[:, 0] / 0.5) ** 2 + (pts[:, 1] / 0.05) ** 2 - 1).max() < 1e-12
                else:
                    c = 0.5 / math.cosh(math.atanh(0.1))
                    m = np.arccosh(np.full(len(pts), 20.0 / c))
                    assert np.abs((pts[:, 0] / (c * np.cosh(m))) ** 2 + (pts[:, 1] / (c * np.sinh(m))) ** 2 - 1).max() < 1e-12
            else:
                assert tuple(nbr[en, fn][:2]) == (e, f)
    T = W.freestream_T(0.1, speed=1.0)
    a = math.radians(8.0)
    qinf = (T, math.cos(a), math.sin(a), 0.0, T)
    orc = O.Oracle3(nodes, nbr, 2, [2], [1], Ma_inf=0.1, mu=1.0 / 60000.0, cutoff=1, kappa=1.0, q_inf=qinf)
    _, J, _, xyz = orc.geometry()
    assert (J > 0).all()
    assert np.abs(xyz[..., 2]).max() <= 0.2 + 1e-12
    # a uniform state with zero velocity at rest is steady everywhere (walls included)
    q = W.uniform_state3(orc.E, xyz.shape[1], T, 0.0, 0.0, 0.0, T)
    orc2 = O.Oracle3(nodes, nbr, 2, [2], [1], Ma_inf=0.1, mu=1.0 / 60000.0, cutoff=1, kappa=1.0,
                     q_inf=(T, 0.0, 0.0, 0.0, T))
    R = orc2.residual(q)
    assert np.abs(R).max() <= 1e-9 * T
