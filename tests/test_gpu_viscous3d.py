"""GPU parity of the viscous terms on hexahedra (dim = 3, mu > 0: Section 2.1
viscous fluxes, Section 2.3 eq. com_q and the BR2 common gradient of eq.
com_grad_q) against the FP64 oracle, with the bounds of the inviscid
hexahedral tests (residual 1e-10 of max|R_v| + 1e-4 S_v; blocks 1e-10
relative Frobenius; V-cycles 1e-8 of the change they make; converged stages
1e-7 of |v| and of rho |v|^2).

Meshes: the straight and the curved (Q2, rotated elements) triply periodic
boxes, and the channel between no-slip walls extruded along z (no-slip
ghost states, mirrored gradients, no viscous energy flux at the walls).
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MU = 0.02
ROT = {0: 5, 4: 17, 7: 11, 9: 20, 13: 3, 16: 22}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()
    O.set_threads(16)
    yield
    O.set_threads(1)


def _box(curved):
    if curved:
        return W.periodic_box3d(3, 3, 2, Ng=2, perturb=0.3, rotations=ROT), 2
    return W.periodic_box3d(3, 2, 3, Ng=1, rotations={1: 7, 8: 14}), 1


def _channel():
    nodes2, nbr2 = W.channel(4, 3, Ng=1)
    return W.extrude(nodes2, nbr2, 1, nz=2, z0=0.0, z1=2.0), 1


def _pair(nodes, nbr, Ng, levels, smooth, Ma=0.005, prec=0, p_gauge=0.0, **kw):
    from paper_1908_03972_gb300 import pmgfr
    orc = O.Oracle3(nodes, nbr, Ng, levels, smooth, Ma_inf=Ma, mu=MU, **kw)
    gkw = dict(kw)
    for name in ("res_scale", "q_inf"):
        if name in gkw:
            gkw[name + "3"] = gkw.pop(name)
    gpu = pmgfr.Solver(nodes, nbr, levels, smooth, Ma_inf=Ma, block_prec=prec, p_gauge=p_gauge, dim=3, mu=MU,
                       **gkw)
    return orc, gpu


def _scale(orc, level, Ma, speed=2 ** 0.5):
    _, J, _, _ = orc.geometry(level)
    h = 2.0 * float(J.min()) ** (1.0 / 3.0)
    p = W.freestream_T(Ma, speed=speed)
    return np.array([p / speed, p, p, p, (3.5 * p + 1.0) * p / speed]) * (orc.P[level] + 1) ** 2 / h


def _rel(a, b, S):
    return max(np.abs(a[v] - b[v]).max() / (np.abs(b[v]).max() + 1e-4 * S[v]) for v in range(5))


def _state(xyz, Ma, seed=1):
    q = W.vortex3d(xyz, Ma_inf=Ma, center=(4.3, 5.6))
    rng = np.random.default_rng(seed)
    return q * (1 + 1e-3 * rng.standard_normal(q.shape) * np.array([1e-3, 1, 1, 1, 1e-5])[:, None, None])


def _channel_state(xyz, Ma, seed=2):
    """A sheared channel flow with noise: u(y) parabolic-like, v, w small."""
    T = W.freestream_T(Ma, speed=1.0)
    E, N, _ = xyz.shape
    y = xyz[..., 1]
    q = W.uniform_state3(E, N, T, 0.0, 0.0, 0.0, T)
    rng = np.random.default_rng(seed)
    q[1] = y * (2.0 - y) + 0.05 * np.sin(xyz[..., 0])
    q[2] = 0.05 * np.sin(xyz[..., 0] + xyz[..., 2])
    q[3] = 0.05 * np.cos(xyz[..., 2])
    q[0] *= 1 + 1e-6 * rng.standard_normal((E, N))
    q[4] *= 1 + 1e-6 * rng.standard_normal((E, N))
    return q


def _qc(q):
    rho = q[0] / q[4]
    E = q[4] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2)
    return np.stack([rho, rho * q[1], rho * q[2], rho * q[3], rho * E])


def _stage(orc, gpu, q, dt=0.1):
    A, _, _ = O.esdirk3()
    odt = A[1, 1] * dt
    src = _qc(q) / odt + A[1, 0] / A[1, 1] * orc.residual(q)
    orc.set_stage(src, odt)
    gpu.set_stage(src, odt)


WALL = dict(cutoff=1, kappa=1.0)


# ---------------------------------------------------------------- residual
@pytest.mark.parametrize("gauge", [False, True])
@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("P", [0, 1, 2, 3])
def test_viscous_residual3_parity(P, curved, gauge):
    (nodes, nbr), Ng = _box(curved)
    if gauge and P < Ng:
        pytest.skip("gauge storage needs P >= geometry order")
    Ma = 0.005
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma=Ma, p_gauge=W.freestream_T(Ma) if gauge else 0.0)
    try:
        q = _state(orc.coords(), Ma)
        Ro, Rg = orc.residual(q), gpu.residual(q)
        assert _rel(Rg, Ro, _scale(orc, 0, Ma)) <= 1e-10
    finally:
        gpu.close()


@pytest.mark.parametrize("P", [1, 2, 3])
def test_viscous_residual3_walls_parity(P):
    (nodes, nbr), Ng = _channel()
    Ma = 0.2
    T = W.freestream_T(Ma, speed=1.0)
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma=Ma, q_inf=(T, 1.0, 0.0, 0.0, T), **WALL)
    try:
        q = _channel_state(orc.coords(), Ma)
        Ro, Rg = orc.residual(q), gpu.residual(q)
        assert _rel(Rg, Ro, _scale(orc, 0, Ma, speed=1.0)) <= 1e-10
    finally:
        gpu.close()


def test_viscous_terms_are_not_negligible_in_these_cases():
    """The comparisons above see the viscous terms: with mu = 0.02 they change
    the momentum residual of the curved box by more than 1e-3 of its size."""
    (nodes, nbr), Ng = _box(True)
    o1 = O.Oracle3(nodes, nbr, Ng, [2], [1], Ma_inf=0.005, mu=MU)
    o0 = O.Oracle3(nodes, nbr, Ng, [2], [1], Ma_inf=0.005)
    q = _state(o1.coords(), 0.005)
    R1, R0 = o1.residual(q), o0.residual(q)
    assert np.abs(R1[1] - R0[1]).max() >= 1e-3 * np.abs(R1[1]).max()


def test_slip_wall_with_viscosity_is_rejected():
    from paper_1908_03972_gb300 import pmgfr
    nodes2, nbr2 = W.channel(4, 3, Ng=1, bottom=W.BC_SLIP_WALL, top=W.BC_SLIP_WALL)
    nodes, nbr = W.extrude(nodes2, nbr2, 1, nz=1)
    with pytest.raises(pmgfr.PmgError) as ei:
        pmgfr.Solver(nodes, nbr, [1], [1], dim=3, mu=MU)
    assert ei.value.status == pmgfr.PMG_EINVAL


# ---------------------------------------------------------------- blocks
@pytest.mark.parametrize("case", ["straight", "curved", "walls"])
@pytest.mark.parametrize("P", [0, 1, 2])
def test_viscous_blocks3_parity(P, case):
    if case == "walls":
        (nodes, nbr), Ng = _channel()
        Ma = 0.2
        T = W.freestream_T(Ma, speed=1.0)
        kw = dict(q_inf=(T, 1.0, 0.0, 0.0, T), **WALL)
    else:
        (nodes, nbr), Ng = _box(case == "curved")
        Ma, kw = 0.005, {}
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma=Ma, **kw)
    try:
        q = _channel_state(orc.coords(), Ma) if case == "walls" else _state(orc.coords(), Ma)
        odt = 0.0436
        orc.set_stage(np.zeros_like(q), odt)
        gpu.set_stage(np.zeros_like(q), odt)
        for dtau in (0.01, 3.0):
            Do, Dg = orc.blocks(q, dtau), gpu.blocks(q, dtau)
            for e in range(orc.E):
                assert np.linalg.norm(Dg[e] - Do[e]) <= 1e-10 * np.linalg.norm(Do[e]), (e, dtau)
    finally:
        gpu.close()


def test_viscous_p3_blocks3_parity():
    """P = 3 (n = 320, the blocks the cluster kernel factors) on the straight box."""
    (nodes, nbr), Ng = _box(False)
    orc, gpu = _pair(nodes, nbr, Ng, [3], [1], Ma=0.005)
    try:
        q = _state(orc.coords(), 0.005)
        orc.set_stage(np.zeros_like(q), 0.0436)
        gpu.set_stage(np.zeros_like(q), 0.0436)
        Do, Dg = orc.blocks(q, 0.5), gpu.blocks(q, 0.5)
        for e in range(orc.E):
            assert np.linalg.norm(Dg[e] - Do[e]) <= 1e-10 * np.linalg.norm(Do[e]), e
    finally:
        gpu.close()


# ---------------------------------------------------------------- V-cycle and stage
@pytest.mark.parametrize("case", ["curved", "walls"])
def test_viscous_vcycle3_parity(case):
    """P{2-1-0}, I{2-3-4}: one V-cycle that builds the smoother and one with
    it frozen, FP64 blocks, 1e-8 of the change each makes."""
    if case == "walls":
        (nodes, nbr), Ng = _channel()
        Ma = 0.2
        T = W.freestream_T(Ma, speed=1.0)
        kw = dict(q_inf=(T, 1.0, 0.0, 0.0, T), **WALL)
    else:
        (nodes, nbr), Ng = _box(True)
        Ma, kw = 0.005, {}
    orc, gpu = _pair(nodes, nbr, Ng, [2, 1, 0], [2, 3, 4], Ma=Ma, **kw)
    try:
        q = _channel_state(orc.coords(), Ma) if case == "walls" else _state(orc.coords(), Ma)
        _stage(orc, gpu, q)
        qo = orc.vcycle(q, 0.7, refresh=True)
        qg, _ = gpu.vcycle(q, 0.7, refresh=True)
        dq = np.abs(qo - q).max(axis=(1, 2))
        assert (np.abs(qg - qo).max(axis=(1, 2)) / dq).max() <= 1e-8
        qo2 = orc.vcycle(qo, 5.0, refresh=False)
        qg2, _ = gpu.vcycle(qo, 5.0, refresh=False)
        dq2 = np.abs(qo2 - qo).max(axis=(1, 2))
        assert (np.abs(qg2 - qo2).max(axis=(1, 2)) / dq2).max() <= 1e-8
    finally:
        gpu.close()


def test_viscous_stage_solve3_parity():
    """One implicit ESDIRK3 stage of the viscous vortex on the straight box,
    solved to a 1e-8 drop by both (P{2-1-0}, I{2-3-4}, gauge storage)."""
    (nodes, nbr), Ng = _box(False)
    kw = dict(tol=1e-8, res_scale=W.freestream_scales3(0.005), max_pseudo=3000)
    orc, gpu = _pair(nodes, nbr, Ng, [2, 1, 0], [2, 3, 4], p_gauge=W.freestream_T(0.005), **kw)
    try:
        q = _state(orc.coords(), 0.005)
        _stage(orc, gpu, q)
        qo, it_o, drop_o, st = orc.stage_solve(q)
        assert st == 0
        qg, it_g, drop_g = gpu.stage_solve(q)
        assert drop_g <= 1e-8 and abs(it_g - it_o) <= 2, (it_o, it_g)
        assert np.abs(qg[0] - qo[0]).max() / 2.0 <= 1e-7 and np.abs(qg[1:4] - qo[1:4]).max() <= 1e-7
    finally:
        gpu.close()


# ---------------------------------------------------------------- the extruded ellipse
def _ellipse_state(xyz, T, qinf, seed=7):
    E, N, _ = xyz.shape
    q = W.uniform_state3(E, N, T, qinf[1], qinf[2], 0.0, T)
    q[2] += 1e-3 * np.random.default_rng(seed).standard_normal((E, N))
    return q


def test_extruded_ellipse_reduced_parity():
    """The extruded-ellipse workload at 6 x 16 x 2 elements (Q2, no-slip wall,
    far field, periodic span; 8 degrees incidence, Ma = 0.1, gauge storage)
    from the free stream with noise: the P = 3 residual, and P{2-1-0}
    V-cycles (the smoother built, then frozen) with FP64 blocks."""
    import math
    nodes, nbr = W.extruded_ellipse(6, 16, 2, span=0.2, Ng=2)
    Ma = 0.1
    T = W.freestream_T(Ma, speed=1.0)
    a = math.radians(8.0)
    qinf = (T, math.cos(a), math.sin(a), 0.0, T)
    kw = dict(q_inf=qinf, **WALL)
    orc, gpu = _pair(nodes, nbr, 2, [3], [1], Ma=Ma, p_gauge=T, **kw)
    try:
        q = _ellipse_state(orc.coords(), T, qinf)
        Ro, Rg = orc.residual(q), gpu.residual(q)
        assert _rel(Rg, Ro, _scale(orc, 0, Ma, speed=1.0)) <= 1e-10
    finally:
        gpu.close()
    orc, gpu = _pair(nodes, nbr, 2, [2, 1, 0], [2, 3, 4], Ma=Ma, p_gauge=T, **kw)
    try:
        q = _ellipse_state(orc.coords(), T, qinf)
        _stage(orc, gpu, q, dt=0.01)
        qo = orc.vcycle(q, 1e-3, refresh=True)
        qg, _ = gpu.vcycle(q, 1e-3, refresh=True)
        dq = np.abs(qo - q).max(axis=(1, 2))
        assert (np.abs(qg - qo).max(axis=(1, 2)) / dq).max() <= 1e-8
        qo2 = orc.vcycle(qo, 1e-2, refresh=False)
        qg2, _ = gpu.vcycle(qo, 1e-2, refresh=False)
        dq2 = np.abs(qo2 - qo).max(axis=(1, 2))
        assert (np.abs(qg2 - qo2).max(axis=(1, 2)) / dq2).max() <= 1e-8
    finally:
        gpu.close()
