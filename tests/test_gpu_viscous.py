"""GPU parity of the viscous terms (Section 2.1 viscous fluxes, Section 2.3
common solution and BR2 common gradient) against the FP64 oracle, through the
C interface.

The viscous part is compared on its own, as R(q; mu) - R(q; 0) on both sides,
with a bound relative to its own size: |V_gpu - V_orc| <= 1e-10 (max|V_orc,v|
+ 1e-4 S_v) per equation, S_v the rounding scale of the inviscid residual
(the two inviscid evaluations that the difference cancels).  The full
residual, the element blocks and V-cycles use the bounds of the inviscid
parity tests.
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


def _h(orc):
    met, _ = orc.metrics()
    return 2.0 * float(np.sqrt(met[:, :, 4].min()))


def _scale(orc, Ma):
    p = W.freestream_T(Ma)
    vinf = 2 ** 0.5
    P = orc.P[0]
    return np.array([p / vinf, p, p, (3.5 * p + 1.0) * p / vinf]) * (P + 1) ** 2 / _h(orc)


def _rel(a, b, S):
    return max(np.abs(a[v] - b[v]).max() / (np.abs(b[v]).max() + 1e-4 * S[v]) for v in range(4))


def _solvers(nodes, nbr, Ng, levels, smooth, mu, Ma, p_gauge=0.0, **kw):
    from paper_1908_03972_gb300 import pmgfr
    orc = O.Oracle(nodes, nbr, Ng, levels, smooth, Ma_inf=Ma, mu=mu, **kw)
    gpu = pmgfr.Solver(nodes, nbr, levels, smooth, Ma_inf=Ma, mu=mu, p_gauge=p_gauge, **kw)
    return orc, gpu


MESHES = {
    "straight_6x6": dict(n=(6, 6), Ng=1, perturb=0.0),
    "curved_4x4": dict(n=(4, 4), Ng=2, perturb=0.3),
    "ragged_5x3": dict(n=(5, 3), Ng=2, perturb=0.25),
    "single_element": dict(n=(1, 1), Ng=1, perturb=0.0),
}


def _state(orc, Ma, seed):
    q = W.isentropic_vortex(orc.coords(), Ma_inf=Ma, center=(4.3, 5.6))
    rng = np.random.default_rng(seed)
    return q * (1 + 1e-3 * rng.standard_normal(q.shape) * np.array([1e-3, 1, 1, 1e-5])[:, None, None])


@pytest.mark.parametrize("Ma", [0.3, 0.005])
@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("P", [0, 1, 2, 3, 4])
def test_viscous_residual_parity(name, P, Ma):
    m = MESHES[name]
    nodes, nbr = W.periodic_box(*m["n"], Ng=m["Ng"], perturb=m["perturb"])
    Ng, mu = m["Ng"], 0.05
    orc, gpu = _solvers(nodes, nbr, Ng, [P], [1], mu, Ma)
    orc0, gpu0 = _solvers(nodes, nbr, Ng, [P], [1], 0.0, Ma)
    try:
        q = _state(orc, Ma, P)
        Ro, Rg = orc.residual(q), gpu.residual(q)
        S = _scale(orc, Ma)
        assert _rel(Rg, Ro, S) <= 1e-10
        Vo = Ro - orc0.residual(q)
        Vg = Rg - gpu0.residual(q)
        assert np.abs(Vo[1:]).max() > 0.0 or P == 0 and name == "single_element"
        assert _rel(Vg, Vo, S) <= 1e-10
    finally:
        gpu.close()
        gpu0.close()


@pytest.mark.parametrize("P", [1, 2, 3])
def test_viscous_residual_parity_gauge_and_reversed_faces(P):
    Ma, mu = 0.005, 0.02
    nodes, nbr = W.periodic_box(3, 3, Ng=2, perturb=0.3)
    nodes, nbr = W.flip_elements(nodes, nbr, [1, 4, 5], Ng=2)
    T = W.freestream_T(Ma)
    gauge = T if P >= 2 else 0.0
    orc, gpu = _solvers(nodes, nbr, 2, [P], [1], mu, Ma, p_gauge=gauge)
    try:
        q = _state(orc, Ma, 7)
        assert _rel(gpu.residual(q), orc.residual(q), _scale(orc, Ma)) <= 1e-10
    finally:
        gpu.close()


def test_viscous_static_residual_matches():
    torch = pytest.importorskip("torch")
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(4, 4, Ng=2, perturb=0.3)
    gpu = pmgfr.Solver(nodes, nbr, [3], [1], Ma_inf=0.3, mu=0.05)
    try:
        q = W.isentropic_vortex(gpu.coords(), Ma_inf=0.3)
        ref = gpu.residual(q)
        qd = torch.from_numpy(q).cuda()
        Rd = torch.empty_like(qd)
        pmgfr.pmg_residual_static(gpu.h, 0, qd, Rd)
        torch.cuda.synchronize()
        assert np.array_equal(Rd.cpu().numpy(), ref)
    finally:
        gpu.close()


@pytest.mark.parametrize("Ma", [0.3, 0.005])
@pytest.mark.parametrize("P", [0, 1, 2, 3, 4])
def test_viscous_block_assembly_parity(P, Ma):
    Ng = 2 if P >= 2 else 1
    nodes, nbr = W.periodic_box(3, 4, Ng=Ng, perturb=0.3 if Ng > 1 else 0.0)
    orc, gpu = _solvers(nodes, nbr, Ng, [P], [1], 0.05, Ma)
    try:
        q = W.isentropic_vortex(orc.coords(), Ma_inf=Ma, center=(4.0, 6.0))
        omega_dt = 0.0436
        src = np.zeros_like(q)
        orc.set_stage(src, omega_dt)
        gpu.set_stage(src, omega_dt)
        for dtau in (0.01, 3.0):
            Do = orc.blocks(q, dtau)
            Dg = gpu.blocks(q, dtau)
            for e in range(orc.E):
                assert np.linalg.norm(Dg[e] - Do[e]) <= 1e-10 * np.linalg.norm(Do[e]), (e, dtau)
    finally:
        gpu.close()


def _qc(q):
    rho = q[0] / q[3]
    E = q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2)
    return np.stack([rho, rho * q[1], rho * q[2], rho * E])


@pytest.mark.parametrize("levels,smooth", [([2, 1, 0], [2, 3, 4]), ([3, 2, 1], [1, 2, 3])])
def test_viscous_vcycle_parity(levels, smooth):
    Ma, mu = 0.005, 0.02
    nodes, nbr = W.periodic_box(4, 4, Ng=2, perturb=0.3)
    orc, gpu = _solvers(nodes, nbr, 2, levels, smooth, mu, Ma)
    try:
        q = W.isentropic_vortex(orc.coords(), center=(4.0, 6.0))
        omega_dt = 0.0436
        src = _qc(q) / omega_dt + 0.5 * orc.residual(q)
        orc.set_stage(src, omega_dt)
        gpu.set_stage(src, omega_dt)
        qo = orc.vcycle(q, 0.7, refresh=True)
        qg, nrm = gpu.vcycle(q, 0.7, refresh=True)
        dq = np.abs(qo - q).max(axis=(1, 2))
        assert (np.abs(qg - qo).max(axis=(1, 2)) / dq).max() <= 1e-8
        assert abs(nrm - np.linalg.norm(orc.stage_F(q))) <= 1e-10 * nrm
        qo2 = orc.vcycle(qo, 5.0, refresh=False)
        qg2, _ = gpu.vcycle(qg, 5.0, refresh=False)
        dq2 = np.abs(qo2 - qo).max(axis=(1, 2))
        assert (np.abs(qg2 - qo2).max(axis=(1, 2)) / dq2).max() <= 1e-7
    finally:
        gpu.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_viscous_stage_solve_parity(prec):
    Ma, mu = 0.005, 0.02
    nodes, nbr = W.periodic_box(4, 4, Ng=2, perturb=0.3)
    from paper_1908_03972_gb300 import pmgfr
    orc = O.Oracle(nodes, nbr, 2, [2, 1, 0], [2, 3, 4], Ma_inf=Ma, mu=mu, tol=1e-8)
    gpu = pmgfr.Solver(nodes, nbr, [2, 1, 0], [2, 3, 4], Ma_inf=Ma, mu=mu, tol=1e-8, block_prec=prec)
    try:
        q = W.isentropic_vortex(orc.coords(), center=(4.0, 6.0))
        omega_dt = 0.0436
        src = _qc(q) / omega_dt + 0.5 * orc.residual(q)
        orc.set_stage(src, omega_dt)
        gpu.set_stage(src, omega_dt)
        qo, it_o, drop_o, _, st = orc.stage_solve(q)
        assert st == 0
        qg, it_g, drop_g = gpu.stage_solve(q)
        assert drop_g <= 1e-8
        if prec == 0:
            assert abs(it_g - it_o) <= 2
        dp = np.abs(qg[0] - qo[0]).max() / 2.0
        du = np.abs(qg[1:3] - qo[1:3]).max()
        assert dp <= 1e-7 and du <= 1e-7, (dp, du, it_o, it_g)
    finally:
        gpu.close()


def test_viscosity_config_checked():
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(2, 2, Ng=1)
    with pytest.raises(pmgfr.PmgError):
        pmgfr.Solver(nodes, nbr, [1], [1], mu=-1.0)
    with pytest.raises(pmgfr.PmgError):
        pmgfr.Solver(nodes, nbr, [1], [1], mu=0.1, Pr=0.0)
