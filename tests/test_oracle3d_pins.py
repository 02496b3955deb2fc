"""Pins of the oracle's three-dimensional discretisation (hexahedra, five
working variables) against facts that do not come from the oracle itself:
library routines, closed forms, the already pinned two-dimensional oracle,
invariants (free stream, conservation, invariance under element renumbering)
and finite differences.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W


# ---------------------------------------------------------------- Gauss-Lobatto points
@pytest.mark.parametrize("n", range(1, 7))
def test_gll_points_are_roots_of_legendre_derivative(n):
    x = O.gll(n)
    ref = np.sort(np.concatenate([[-1.0, 1.0], np.polynomial.legendre.Legendre.basis(n).deriv().roots()]))
    assert np.allclose(x, ref, atol=1e-14, rtol=0)


# ---------------------------------------------------------------- pointwise physics in 3D
def _states3(n, seed, Ma=0.005):
    rng = np.random.default_rng(seed)
    T0 = W.freestream_T(Ma)
    return [np.array([T0 * (1 + 0.01 * rng.standard_normal()), 1 + rng.standard_normal(), 1 + rng.standard_normal(),
                      0.5 * rng.standard_normal(), T0 * (1 + 1e-4 * rng.standard_normal())]) for _ in range(n)]


def test_M3_by_differences_and_gamma_equals_M_at_eps_one():
    for q in _states3(20, 1):
        M, G, eps = O.point_matrices3(q, Ma_inf=2.0, kappa=1.0, cutoff=1)
        assert eps == 1.0 and np.allclose(G, M, rtol=1e-13, atol=1e-13 * np.abs(M).max())
        Mfd = np.zeros((5, 5))
        for c in range(5):
            def cd(h):
                qp, qm = q.copy(), q.copy()
                qp[c] += h; qm[c] -= h
                return (O.cons_from_prim3(qp) - O.cons_from_prim3(qm)) / (2 * h)
            h = [1e-3 * q[0], 0.1, 0.1, 0.1, 1e-3 * q[4]][c]
            Mfd[:, c] = (4 * cd(h / 2) - cd(h)) / 3
        assert np.allclose(M, Mfd, rtol=1e-6, atol=1e-9 * np.abs(M).max())


@pytest.mark.parametrize("T,u,v,w,eps_ref", [(1 / 1.4, 0.2, 0.2, 0.1, 0.3),     # |v| = 0.3, c = 1
                                             (1e4 / 1.4, 2.0, 1.0, 2.0, 0.03),  # |v| = 3, c = 100
                                             (1 / 1.4, 2.0, 1.0, 2.0, 1.0)])    # Ma = 3: capped
def test_eps3_hand_values(T, u, v, w, eps_ref):
    _, _, eps = O.point_matrices3(np.array([T, u, v, w, T]), Ma_inf=0.005, cutoff=0)
    assert abs(eps - eps_ref) <= 1e-14


def test_preconditioned_eigenvalues_3d():
    # eq. eigenvalues_para in 3D: u_n three times, u_n' +- c'
    rng = np.random.default_rng(3)
    for q in _states3(30, 3):
        n = rng.standard_normal(3); n /= np.linalg.norm(n)
        _, G, _ = O.point_matrices3(q)
        _, A = O.flux3(q, n)
        lam = np.sort(np.linalg.eigvals(np.linalg.solve(G, A)).real)
        c = math.sqrt(1.4 * q[4]); Ur = min(1.0, np.linalg.norm(q[1:4]) / c) * c
        un = q[1:4] @ n
        alpha = (1 - Ur ** 2 / c ** 2) / 2
        cp = math.sqrt(alpha ** 2 * un ** 2 + Ur ** 2)
        ref = np.sort([un, un, un, un * (1 - alpha) + cp, un * (1 - alpha) - cp])
        assert np.allclose(lam, ref, rtol=1e-7, atol=1e-7)


def test_roe3_consistency_conservation_and_eigendecomposition():
    rng = np.random.default_rng(5)
    for qm in _states3(20, 5):
        qp = qm + np.array([rng.standard_normal(), 0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(),
                            0.1 * rng.standard_normal(), 1e-3 * rng.standard_normal()])
        S = rng.standard_normal(3)
        dS = np.linalg.norm(S); n = S / dS
        f, _ = O.flux3(qm, n)
        assert np.allclose(O.roe3(qm, qm, S), f * dS, rtol=1e-13, atol=1e-13 * np.abs(f).max())
        a, b = O.roe3(qm, qp, S), O.roe3(qp, qm, -S)
        assert np.allclose(a, -b, rtol=1e-10, atol=1e-10 * np.abs(a).max())
        # eq. invis_com literally, |Gamma^-1 A_n| by numpy's eigendecomposition
        qa = 0.5 * (qm + qp)
        _, G, _ = O.point_matrices3(qa)
        _, A = O.flux3(qa, n)
        lam, R = np.linalg.eig(np.linalg.solve(G, A))
        absM = (R @ np.diag(np.abs(lam)) @ np.linalg.inv(R)).real
        fm, _ = O.flux3(qm, n); fp, _ = O.flux3(qp, n)
        ref = (0.5 * (fm + fp) - 0.5 * G @ absM @ (qp - qm)) * dS
        assert np.allclose(a, ref, rtol=1e-8, atol=1e-8 * np.abs(ref).max())


def test_roe3_reduces_to_the_2d_flux():
    """w = 0 on both sides and a normal in the x-y plane: the 3D flux is the
    (pinned) 2D flux with a zero z-momentum component."""
    rng = np.random.default_rng(8)
    for qm in _states3(20, 8):
        qm[3] = 0.0
        qp = qm + np.array([rng.standard_normal(), 0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(), 0.0,
                            1e-3 * rng.standard_normal()])
        Sx, Sy = rng.standard_normal(2)
        f3 = O.roe3(qm, qp, np.array([Sx, Sy, 0.0]))
        f2 = O.roe(qm[[0, 1, 2, 4]], qp[[0, 1, 2, 4]], Sx, Sy)
        assert np.allclose(f3[[0, 1, 2, 4]], f2, rtol=1e-11, atol=1e-11 * np.abs(f2).max())
        assert abs(f3[3]) <= 1e-11 * np.abs(f2).max()


# ---------------------------------------------------------------- the discretisation
def _flux_scale(T):
    return np.array([1.0, T, T, T, 3.5 * T])


@pytest.mark.parametrize("Ng,P", [(1, 0), (1, 2), (2, 2), (2, 3), (2, 4)])
def test_free_stream_preserved_on_curved_hexahedra(Ng, P):
    """The conservative-curl metric terms keep a uniform flow exactly steady
    on straight elements at every P and on curved (Q2) elements from P = 2,
    with rotated elements too."""
    nodes, nbr = W.periodic_box3d(3, 2, 2, Ng=Ng, perturb=0.3 if Ng > 1 else 0.0,
                                  rotations={0: 5, 4: 17, 7: 11, 9: 20})
    orc = O.Oracle3(nodes, nbr, Ng, [P], [1], Ma_inf=0.5)
    T = W.freestream_T(0.5)
    q = W.uniform_state3(orc.E, orc.N(), T, 1.0, 0.7, -0.4, T)
    R = orc.residual(q)
    sc = _flux_scale(T) * (P + 1) ** 2 / 3.0
    for v in range(5):
        assert np.abs(R[v]).max() <= 1e-12 * sc[v], (v, np.abs(R[v]).max())


def test_metric_terms_are_exact_where_the_map_is_polynomial():
    """Straight (trilinear) elements of a sheared box: J a^i at the solution
    points equals the cofactor matrix of the map's Jacobian, and the face
    normals are the outward J a^d (both closed forms of the affine map)."""
    nodes, nbr = W.periodic_box3d(2, 2, 2, Ng=1)
    shear = np.array([[1.0, 0.3, 0.1], [0.0, 1.0, 0.2], [0.0, 0.0, 1.0]])
    nodes = nodes @ shear.T
    orc = O.Oracle3(nodes, nbr, 1, [2], [1])
    Ja, J, fS, _ = orc.geometry()
    Jm = shear * 2.5            # dX/dxi: element side 5 in every reference direction of length 2
    cof = np.linalg.det(Jm) * np.linalg.inv(Jm)   # rows: J grad(xi^i)
    assert np.allclose(Ja, cof[None, None], atol=1e-13)
    assert np.allclose(J, np.linalg.det(Jm), atol=1e-13)
    for f in range(6):
        sg = 1.0 if f % 2 else -1.0
        assert np.allclose(fS[:, f], sg * cof[f // 2][None, None], atol=1e-13)


def _extruded_pair(n2, Ng, perturb, P, Ma=0.3):
    nodes2, nbr2 = W.periodic_box(*n2, Ng=Ng, perturb=perturb)
    nodes3, nbr3 = W.extrude(nodes2, nbr2, Ng, nz=1, z0=0.0, z1=1.0)
    o2 = O.Oracle(nodes2, nbr2, Ng, [P], [1], Ma_inf=Ma)
    o3 = O.Oracle3(nodes3, nbr3, Ng, [P], [1], Ma_inf=Ma)
    return o2, o3


@pytest.mark.parametrize("Ng,P,n2", [(1, 0, (4, 3)), (1, 2, (4, 3)), (1, 3, (3, 3)), (2, 2, (3, 3)),
                                     (2, 3, (3, 2)), (2, 4, (2, 2))])
def test_residual_reduces_to_the_2d_residual(Ng, P, n2):
    """A quadrilateral mesh extruded one element along z (periodic), with a
    state independent of z and w = 0: the 3D residual is the 2D residual of
    the pinned 2D oracle, layer by layer, and the z-momentum residual vanishes.
    On curved meshes this holds from P >= geometry order, where the
    conservative-curl metrics equal the analytic ones."""
    o2, o3 = _extruded_pair(n2, Ng, 0.3 if Ng > 1 else 0.0, P)
    xy = o2.coords()
    q2 = W.isentropic_vortex(xy, Ma_inf=0.3, center=(4.3, 5.6))
    n1 = P + 1
    q3 = np.zeros(o3.shape())
    for kk in range(n1):
        sl = slice(kk * n1 * n1, (kk + 1) * n1 * n1)
        for v2, v3 in ((0, 0), (1, 1), (2, 2), (3, 4)):
            q3[v3, :, sl] = q2[v2]
    R2, R3 = o2.residual(q2), o3.residual(q3)
    for kk in range(n1):
        sl = slice(kk * n1 * n1, (kk + 1) * n1 * n1)
        for v2, v3 in ((0, 0), (1, 1), (2, 2), (3, 4)):
            assert np.abs(R3[v3, :, sl] - R2[v2]).max() <= 1e-11 * np.abs(R2[v2]).max(), (kk, v2)
        assert np.abs(R3[3, :, sl]).max() <= 1e-11 * np.abs(R2[1]).max()


def test_face_normals_agree_across_faces_at_every_level():
    """Both elements of a face, periodic images included, see opposite normals
    at every face point, also below the geometry order (P = 0, 1 on Q2)."""
    for P in (0, 1, 2, 3):
        nodes, nbr = W.periodic_box3d(3, 2, 2, Ng=2, perturb=0.3, rotations={1: 3, 4: 13, 6: 22, 10: 8})
        orc = O.Oracle3(nodes, nbr, 2, [P], [1])
        _, _, fS, _ = orc.geometry()
        n1 = P + 1
        worst = 0.0
        for e in range(orc.E):
            for f in range(6):
                e2, f2, o = nbr[e, f]
                for b in range(n1):
                    for a in range(n1):
                        s, t = (b, a) if o & 4 else (a, b)
                        a2, b2 = (P - s if o & 1 else s), (P - t if o & 2 else t)
                        worst = max(worst, np.abs(fS[e, f, b * n1 + a] + fS[e2, f2, b2 * n1 + a2]).max())
        assert worst <= 1e-12 * np.abs(fS).max(), (P, worst)


def _weights3(P):
    w = np.polynomial.legendre.leggauss(P + 1)[1]
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)


@pytest.mark.parametrize("P", [0, 1, 2, 3])
def test_discrete_conservation_with_rotated_elements(P):
    """sum_e sum_pts w |J| R = 0 on a periodic mesh: the common fluxes of the
    two sides of every face cancel, in every face orientation."""
    nodes, nbr = W.periodic_box3d(3, 2, 2, Ng=2, perturb=0.3, rotations={1: 3, 4: 13, 6: 22, 10: 8})
    orc = O.Oracle3(nodes, nbr, 2, [P], [1], Ma_inf=0.3)
    _, J, _, xyz = orc.geometry()
    q = W.vortex3d(xyz, Ma_inf=0.3, center=(4.3, 5.6))
    R = orc.residual(q)
    wJ = _weights3(P)[None, :] * J
    for v in range(5):
        tot = (wJ * R[v]).sum()
        assert abs(tot) <= 1e-11 * (wJ * np.abs(R[v])).sum(), (v, tot)


def test_residual_invariant_under_element_renumbering():
    """Rotating elements' local axes renumbers their points, not the physics:
    at every physical solution point the residual is unchanged."""
    P = 2
    rot = {0: 5, 3: 17, 5: 11, 8: 20, 10: 2}
    n0, b0 = W.periodic_box3d(3, 2, 2, Ng=2, perturb=0.3)
    n1_, b1 = W.periodic_box3d(3, 2, 2, Ng=2, perturb=0.3, rotations=rot)
    o0 = O.Oracle3(n0, b0, 2, [P], [1], Ma_inf=0.3)
    o1 = O.Oracle3(n1_, b1, 2, [P], [1], Ma_inf=0.3)
    x0, x1 = o0.coords(), o1.coords()
    R0 = o0.residual(W.vortex3d(x0, Ma_inf=0.3, center=(4.3, 5.6)))
    R1 = o1.residual(W.vortex3d(x1, Ma_inf=0.3, center=(4.3, 5.6)))
    for e in range(o0.E):
        d = np.linalg.norm(x0[e][:, None, :] - x1[e][None, :, :], axis=2)
        perm = d.argmin(axis=1)
        assert d[np.arange(len(perm)), perm].max() < 1e-12
        for v in range(5):
            assert np.allclose(R1[v, e, perm], R0[v, e], rtol=0, atol=1e-11 * np.abs(R0[v]).max())


def test_blocks_match_central_differences():
    nodes, nbr = W.periodic_box3d(2, 2, 2, Ng=2, perturb=0.3, rotations={3: 7})
    orc = O.Oracle3(nodes, nbr, 2, [1], [1], Ma_inf=0.3)
    q = W.vortex3d(orc.coords(), Ma_inf=0.3, center=(4.3, 5.6))
    odt, dtau = 0.05, 0.7
    orc.set_stage(np.zeros_like(q), odt)
    D = orc.blocks(q, dtau)
    N = orc.N()
    e = 5
    for col in (0, 7, N + 3, 3 * N + 1, 4 * N + 6):
        v, p = divmod(col, N)
        h = 1e-6 * max(abs(q[v, e, p]), 1.0)
        qp, qm = q.copy(), q.copy()
        qp[v, e, p] += h; qm[v, e, p] -= h
        # -dF/dq (the stage term and R) plus Gamma/dtau: F of the element only
        dF = (orc.stage_F(qp)[:, e].reshape(-1) - orc.stage_F(qm)[:, e].reshape(-1)) / (2 * h)
        _, G, _ = O.point_matrices3(q[:, e, p], Ma_inf=0.3)
        ref = -dF
        ref[np.arange(5) * N + p] += G[:, v] / dtau
        assert np.allclose(D[e][:, col], ref, rtol=1e-5, atol=1e-6 * np.abs(D[e]).max())


@pytest.mark.parametrize("Pf,Pc", [(1, 0), (2, 1), (3, 2), (2, 0)])
def test_transfers_3d(Pf, Pc):
    nodes, nbr = W.periodic_box3d(2, 1, 2, Ng=1)
    orc = O.Oracle3(nodes, nbr, 1, [Pf, Pc], [1, 1])
    rng = np.random.default_rng(2)
    qc = rng.standard_normal(orc.shape(1))
    assert np.allclose(orc.restrict(orc.prolong(qc, 0), 0), qc, atol=1e-14)


def test_vcycle_keeps_a_discrete_steady_state():
    """FAS consistency: for a state q* with F_0(q*) = 0 (the stage source set to
    cancel the residual) a V-cycle returns q* to rounding."""
    nodes, nbr = W.periodic_box3d(2, 2, 2, Ng=2, perturb=0.2)
    orc = O.Oracle3(nodes, nbr, 2, [2, 1, 0], [2, 2, 3], Ma_inf=0.3)
    q = W.vortex3d(orc.coords(), Ma_inf=0.3, center=(4.3, 5.6))
    odt = 0.05
    orc.set_stage(np.zeros_like(q), odt)
    F = orc.stage_F(q)
    orc.set_stage(-F, odt)
    q1 = orc.vcycle(q, 0.5, refresh=True)
    scale = np.abs(q).max(axis=(1, 2)) + 1.0
    assert (np.abs(q1 - q).max(axis=(1, 2)) / scale).max() <= 1e-12
