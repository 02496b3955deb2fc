"""GPU parity of the hexahedral path (dim = 3) against the FP64 oracle.

Meshes: triply periodic boxes (straight, and curved Q2 with elements whose
local axes are rotated, so that faces meet in several orientations) and the
cubed-sphere shell of the sphere workload (6 x n x n x n_r Q2 hexahedra,
radii 0.5 40^(k/n_r), slip wall inside, far field at r = 20), at 1/16 of its
36,864 elements (n = 4, n_r = 24) and at full size for the residual.

Bounds are those of the quadrilateral tests: residual |R_gpu - R_orc| <=
1e-10 (max|R_orc,v| + 1e-4 S_v) per equation, S_v = (P+1)^2/h (p/|v|, p, p, p,
H p/|v|); blocks 1e-10 relative Frobenius; transfers 1e-13; V-cycles 1e-8 of
the change they make per sweep-count scaling (as in the full-size C2 test);
converged states 1e-7 (velocity) and 2e-6 rho|v|^2 (pressure).
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()
    O.set_threads(16)   # the oracle's element loops on the host cores (results do not depend on it)
    yield
    O.set_threads(1)


ROT = {0: 5, 4: 17, 7: 11, 9: 20, 13: 3, 16: 22}


def _box(curved):
    if curved:
        return W.periodic_box3d(3, 3, 2, Ng=2, perturb=0.3, rotations=ROT), 2
    return W.periodic_box3d(3, 2, 3, Ng=1, rotations={1: 7, 8: 14}), 1


def _pair(nodes, nbr, Ng, levels, smooth, Ma=0.005, prec=0, p_gauge=0.0, **kw):
    from paper_1908_03972_gb300 import pmgfr
    orc = O.Oracle3(nodes, nbr, Ng, levels, smooth, Ma_inf=Ma, **kw)
    gkw = dict(kw)
    for name in ("res_scale", "q_inf"):
        if name in gkw:
            gkw[name + "3"] = gkw.pop(name)
    gpu = pmgfr.Solver(nodes, nbr, levels, smooth, Ma_inf=Ma, block_prec=prec, p_gauge=p_gauge, dim=3, **gkw)
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


def _qc(q):
    rho = q[0] / q[4]
    E = q[4] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2)
    return np.stack([rho, rho * q[1], rho * q[2], rho * q[3], rho * E])


# ---------------------------------------------------------------- residual
@pytest.mark.parametrize("Ma", [0.3, 0.005])
@pytest.mark.parametrize("gauge", [False, True])
@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("P", [0, 1, 2, 3])
def test_residual3_parity(P, curved, gauge, Ma):
    (nodes, nbr), Ng = _box(curved)
    if gauge and P < Ng:
        pytest.skip("gauge storage needs P >= geometry order")
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma=Ma, p_gauge=W.freestream_T(Ma) if gauge else 0.0)
    try:
        q = _state(orc.coords(), Ma)
        Ro, Rg = orc.residual(q), gpu.residual(q)
        assert _rel(Rg, Ro, _scale(orc, 0, Ma)) <= 1e-10
        assert np.abs(gpu.coords() - orc.coords()).max() <= 1e-12
    finally:
        gpu.close()


def test_free_stream3_on_gpu():
    (nodes, nbr), Ng = _box(True)
    from paper_1908_03972_gb300 import pmgfr
    T = W.freestream_T(0.5)
    gpu = pmgfr.Solver(nodes, nbr, [3, 2], [1, 1], Ma_inf=0.5, dim=3)
    try:
        for l in range(2):
            q = W.uniform_state3(gpu.E, gpu.N(l), T, 1.0, 0.7, -0.4, T)
            R = gpu.residual(q, l)
            scale = np.array([1.0, T, T, T, 3.5 * T]) * 3.0
            assert all(np.abs(R[v]).max() <= 1e-12 * scale[v] for v in range(5))
    finally:
        gpu.close()


# ---------------------------------------------------------------- blocks, factor, transfers
@pytest.mark.parametrize("P", [0, 1, 2])
def test_blocks3_parity(P):
    (nodes, nbr), Ng = _box(P >= 2)
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma=0.005)
    try:
        q = _state(orc.coords(), 0.005)
        odt = 0.0436
        orc.set_stage(np.zeros_like(q), odt)
        gpu.set_stage(np.zeros_like(q), odt)
        for dtau in (0.01, 3.0):
            Do, Dg = orc.blocks(q, dtau), gpu.blocks(q, dtau)
            for e in range(orc.E):
                assert np.linalg.norm(Dg[e] - Do[e]) <= 1e-10 * np.linalg.norm(Do[e]), (e, dtau)
    finally:
        gpu.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4), (2, 5e-2)])
@pytest.mark.parametrize("P", [1, 2])
def test_factor_and_apply3(P, prec, tol):
    from paper_1908_03972_gb300 import pmgfr
    (nodes, nbr), Ng = _box(True)
    gpu = pmgfr.Solver(nodes, nbr, [P], [1], block_prec=prec, dim=3)
    try:
        q = _state(gpu.coords(), 0.005)
        gpu.set_stage(np.zeros_like(q), 0.0436)
        D = gpu.blocks(q, 1.0)
        gpu.factor()
        rng = np.random.default_rng(3)
        r = rng.standard_normal(q.shape) * np.array([1e-3, 1.0, 1.0, 1.0, 1e2])[:, None, None]
        x = gpu.apply(r)
        for e in range(gpu.E):
            xe = np.linalg.solve(D[e], r[:, e].reshape(-1))
            assert np.linalg.norm(x[:, e].reshape(-1) - xe) <= tol * np.linalg.norm(xe), e
    finally:
        gpu.close()


@pytest.mark.parametrize("levels", [[1, 0], [2, 1], [3, 2], [2, 0], [3, 1]])
def test_transfers3_parity(levels):
    (nodes, nbr), Ng = _box(True)
    orc, gpu = _pair(nodes, nbr, Ng, levels, [1, 1])
    try:
        rng = np.random.default_rng(11)
        qf, qc = rng.standard_normal(orc.shape(0)), rng.standard_normal(orc.shape(1))
        a, b = gpu.restrict(qf, 0), orc.restrict(qf, 0)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
        a, b = gpu.prolong(qc, 0), orc.prolong(qc, 0)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    finally:
        gpu.close()


# ---------------------------------------------------------------- V-cycles, stages, steps
def _stage(orc, gpu, q, odt=0.0436, scale=0.5):
    src = _qc(q) / odt + scale * orc.residual(q)
    orc.set_stage(src, odt)
    gpu.set_stage(src, odt)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("gauge", [False, True])
def test_vcycle3_parity(gauge, prec):
    """P{2-1-0}, I{2-3-4} (14 sweeps): one V-cycle that builds the smoother and
    one with it frozen.  FP64 blocks: 1e-8 of the change, as in 2D; FP32
    blocks: 5e-3."""
    (nodes, nbr), Ng = _box(not gauge)
    orc, gpu = _pair(nodes, nbr, Ng, [2, 1, 0], [2, 3, 4], prec=prec,
                     p_gauge=W.freestream_T(0.005) if gauge else 0.0)
    try:
        q = _state(orc.coords(), 0.005)
        _stage(orc, gpu, q)
        tol = 1e-8 if prec == 0 else 5e-3
        qo = orc.vcycle(q, 0.7, refresh=True)
        qg, _ = gpu.vcycle(q, 0.7, refresh=True)
        dq = np.abs(qo - q).max(axis=(1, 2))
        assert (np.abs(qg - qo).max(axis=(1, 2)) / dq).max() <= tol
        qo2 = orc.vcycle(qo, 5.0, refresh=False)
        qg2, _ = gpu.vcycle(qo, 5.0, refresh=False)
        dq2 = np.abs(qo2 - qo).max(axis=(1, 2))
        assert (np.abs(qg2 - qo2).max(axis=(1, 2)) / dq2).max() <= tol
    finally:
        gpu.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_stage_solve3_parity(prec):
    (nodes, nbr), Ng = _box(False)
    kw = dict(tol=1e-8, res_scale=W.freestream_scales3(0.005), max_pseudo=3000)
    orc, gpu = _pair(nodes, nbr, Ng, [2, 1, 0], [2, 3, 4], prec=prec, p_gauge=W.freestream_T(0.005), **kw)
    try:
        q = _state(orc.coords(), 0.005)
        _stage(orc, gpu, q)
        qo, it_o, drop_o, st = orc.stage_solve(q)
        assert st == 0
        qg, it_g, drop_g = gpu.stage_solve(q)
        assert drop_g <= 1e-8
        if prec == 0:
            assert abs(it_g - it_o) <= 2, (it_o, it_g)
        assert np.abs(qg[0] - qo[0]).max() / 2.0 <= 1e-7 and np.abs(qg[1:4] - qo[1:4]).max() <= 1e-7
    finally:
        gpu.close()


def test_esdirk3_step_3d_parity():
    """One ESDIRK3 step of a 3D vortex (dt = 0.1) from the same state."""
    (nodes, nbr), Ng = _box(False)
    kw = dict(tol=1e-8, res_scale=W.freestream_scales3(0.005), max_pseudo=3000, dtau_init=0.01, dtau_max=10.0)
    orc, gpu = _pair(nodes, nbr, Ng, [2, 1, 0], [2, 3, 4], prec=0, p_gauge=W.freestream_T(0.005), **kw)
    try:
        q = _state(orc.coords(), 0.005)
        qo, its_o, _ = orc.esdirk_step(q, 0.1)
        qg, st = gpu.esdirk_step(q, 0.1)
        its_g = list(st.pseudo_iters)[:3]
        assert max(st.res_drop[:3]) <= 1e-8
        assert all(b <= 1.1 * a + 5 and a <= 1.1 * b + 5 for a, b in zip(its_o[:3], its_g)), (its_o, its_g)
        assert np.abs(qg[0] - qo[0]).max() / 2.0 <= 2e-6 and np.abs(qg[1:4] - qo[1:4]).max() <= 1e-7
    finally:
        gpu.close()


# ---------------------------------------------------------------- the sphere workload
MA_S = 0.001
SPH_LEVELS, SPH_SMOOTH = [2, 1, 0], [5, 10, 20]


def _sphere_state(xyz, seed=7):
    """Free stream (rho = 1, u = 1 along x, Ma = 0.001) with a smooth seeded
    perturbation of the velocity and small ones of p and T."""
    T = W.freestream_T(MA_S, speed=1.0)
    E, N, _ = xyz.shape
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.2, 0.6, size=(3, 3))
    q = W.uniform_state3(E, N, T, 1.0, 0.0, 0.0, T)
    for c in range(3):
        q[1 + c] += 1e-2 * np.sin(xyz @ k[c])
    q[0] *= 1 + 1e-7 * np.cos(xyz[..., 0])
    q[4] *= 1 + 1e-7 * np.sin(xyz[..., 1])
    return q


def _sphere_pair(n, n_r, prec=0, levels=SPH_LEVELS, smooth=SPH_SMOOTH, p_gauge=0.0):
    T = W.freestream_T(MA_S, speed=1.0)
    nodes, nbr = W.cubed_sphere_shell(n, n_r, 0.5, 20.0, Ng=2)
    return _pair(nodes, nbr, 2, levels, smooth, Ma=MA_S, prec=prec, cutoff=1, kappa=1.0, p_gauge=p_gauge,
                 q_inf=(T, 1.0, 0.0, 0.0, T), res_scale=W.freestream_scales3(MA_S, speed=1.0))


def _free_stream_floor(orc_pair_nodes, level_P, n, n_r):
    """The oracle's residual of the uniform free stream on the same shell with
    far-field faces on both sides: the rounding of the discrete metric identity
    times p ~ 7e5, a floor under any residual comparison at Ma = 0.001."""
    T = W.freestream_T(MA_S, speed=1.0)
    nodes, nbr = W.cubed_sphere_shell(n, n_r, 0.5, 20.0, Ng=2, wall=W.BC_FARFIELD)
    o = O.Oracle3(nodes, nbr, 2, [level_P], [1], Ma_inf=MA_S, cutoff=1, kappa=1.0, q_inf=(T, 1.0, 0.0, 0.0, T))
    return np.abs(o.residual(W.uniform_state3(o.E, o.N(), T, 1.0, 0.0, 0.0, T))).max(axis=(1, 2))


def test_sphere_reduced_residual_parity_all_levels():
    orc, gpu = _sphere_pair(4, 24)
    try:
        assert orc.E == 2304
        for level in range(3):
            q = _sphere_state(orc.coords(level))
            Ro, Rg = orc.residual(q, level), gpu.residual(q, level)
            floor = _free_stream_floor(None, SPH_LEVELS[level], 4, 24)
            S = _scale(orc, level, MA_S, speed=1.0)
            for v in range(5):
                bound = 1e-10 * (np.abs(Ro[v]).max() + 1e-4 * S[v]) + 2.0 * floor[v]
                assert np.abs(Rg[v] - Ro[v]).max() <= bound, (level, v, np.abs(Rg[v] - Ro[v]).max(), bound)
    finally:
        gpu.close()


def test_sphere_reduced_p2_block_parity():
    orc, gpu = _sphere_pair(4, 24)
    try:
        q = _sphere_state(orc.coords())
        odt = 0.4358665215 * 0.1
        orc.set_stage(np.zeros_like(q), odt)
        gpu.set_stage(np.zeros_like(q), odt)
        Do, Dg = orc.blocks(q, 0.01), gpu.blocks(q, 0.01)
        assert Do.shape[1] == 135
        err = max(np.linalg.norm(Dg[e] - Do[e]) / np.linalg.norm(Do[e]) for e in range(orc.E))
        assert err <= 1e-10, err
    finally:
        gpu.close()


def test_sphere_reduced_vcycle_parity():
    """One V-cycle of I{5-10-20} (10 + 20 + 20 = 50 sweeps) that builds the
    smoother, at a small dtau: the 2D bound of 1e-8 per 13 sweeps scaled to 50."""
    orc, gpu = _sphere_pair(4, 24)
    try:
        q = _sphere_state(orc.coords())
        odt = 0.4358665215 * 0.1
        src = _qc(q) / odt + 0.2 * orc.residual(q)
        orc.set_stage(src, odt)
        gpu.set_stage(src, odt)
        qo = orc.vcycle(q, 1e-3, refresh=True)
        qg, _ = gpu.vcycle(q, 1e-3, refresh=True)
        dq = np.abs(qo - q).max(axis=(1, 2))
        err = (np.abs(qg - qo).max(axis=(1, 2)) / dq).max()
        print(f"sphere 1/16 V-cycle: max deviation / change = {err:.3e}")
        assert err <= 1e-8 / 13 * 50
    finally:
        gpu.close()


def test_sphere_full_size_residual_parity():
    """Full size (36,864 hexahedra, P = 2).  With p ~ 7e5 every code's own
    rounding of the discrete metric identity, times p, is a floor; the GPU
    stores the gauge pressure (one level, P = geometry order), which removes
    its floor from the momentum flux, and the bound adds twice the oracle's."""
    orc, gpu = _sphere_pair(16, 24, levels=[2], smooth=[1], p_gauge=W.freestream_T(MA_S, speed=1.0))
    try:
        assert orc.E == 36864
        q = _sphere_state(orc.coords())
        Ro, Rg = orc.residual(q), gpu.residual(q)
        floor = _free_stream_floor(None, 2, 16, 24)
        S = _scale(orc, 0, MA_S, speed=1.0)
        for v in range(5):
            bound = 1e-10 * (np.abs(Ro[v]).max() + 1e-4 * S[v]) + 2.0 * floor[v]
            assert np.abs(Rg[v] - Ro[v]).max() <= bound, (v, np.abs(Rg[v] - Ro[v]).max(), bound)
    finally:
        gpu.close()
