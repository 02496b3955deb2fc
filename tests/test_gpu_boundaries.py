"""GPU parity of boundary faces (ghost states: slip wall, no-slip adiabatic
wall, far field) against the FP64 oracle, through the C interface: residuals,
element blocks, a V-cycle and a stage solve on channels and on a small
cylinder O-mesh with curved (Q2) elements.  Bounds as in the inviscid and
viscous parity tests."""
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
    p = W.freestream_T(Ma, speed=1.0)
    P = orc.P[0]
    return np.array([p, p, p, (3.5 * p + 1.0) * p]) * (P + 1) ** 2 / _h(orc)


def _rel(a, b, S):
    return max(np.abs(a[v] - b[v]).max() / (np.abs(b[v]).max() + 1e-4 * S[v]) for v in range(4))


def _pair(nodes, nbr, Ng, levels, smooth, Ma, mu, **kw):
    from paper_1908_03972_gb300 import pmgfr
    T = W.freestream_T(Ma, speed=1.0)
    common = dict(Ma_inf=Ma, mu=mu, cutoff=1, kappa=1.0, q_inf=(T, 1.0, 0.0, T), **kw)
    orc = O.Oracle(nodes, nbr, Ng, levels, smooth, **common)
    gpu = pmgfr.Solver(nodes, nbr, levels, smooth, **common)
    return orc, gpu


def _state(orc, Ma, seed=3):
    xy = orc.coords()
    q = W.freestream_noise_state(xy, Ma, noise=0.05, seed=seed)
    q[1] += 0.2 * np.sin(0.7 * xy[..., 0]) * np.cos(0.9 * xy[..., 1])
    q[3] *= 1 + 1e-4 * np.cos(0.5 * xy[..., 0] + 0.3 * xy[..., 1])
    q[0] *= 1 + 1e-4 * np.sin(0.4 * xy[..., 1])
    return q


MESHES = {
    "channel_noslip": lambda: (W.channel(6, 3, Ng=2, perturb=0.3), 2),
    "channel_slip": lambda: (W.channel(6, 3, Ng=2, perturb=0.3, bottom=W.BC_SLIP_WALL, top=W.BC_SLIP_WALL), 2),
    "channel_wall_farfield": lambda: (W.channel(6, 3, Ng=1, top=W.BC_FARFIELD), 1),
    "cylinder": lambda: (W.cylinder_omesh(3, 12, r_in=0.5, r_out=8.0, Ng=2), 2),
    "cylinder_slip": lambda: (W.cylinder_omesh(3, 12, r_in=0.5, r_out=8.0, Ng=2, wall=W.BC_SLIP_WALL), 2),
}


@pytest.mark.parametrize("Ma", [0.1, 0.001])
@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("P", [0, 1, 2, 3, 4])
def test_boundary_residual_parity(name, P, Ma):
    (nodes, nbr), Ng = MESHES[name]()
    mu = 0.0 if "slip" in name else 0.02
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma, mu)
    try:
        q = _state(orc, Ma)
        assert _rel(gpu.residual(q), orc.residual(q), _scale(orc, Ma)) <= 1e-10
    finally:
        gpu.close()


@pytest.mark.parametrize("name", ["channel_noslip", "channel_wall_farfield", "cylinder", "cylinder_slip"])
@pytest.mark.parametrize("P", [1, 2, 3])
def test_boundary_block_parity(name, P):
    (nodes, nbr), Ng = MESHES[name]()
    mu = 0.0 if "slip" in name else 0.02
    Ma = 0.1
    orc, gpu = _pair(nodes, nbr, Ng, [P], [1], Ma, mu)
    try:
        q = _state(orc, Ma)
        orc.set_stage(np.zeros_like(q), 0.0436)
        gpu.set_stage(np.zeros_like(q), 0.0436)
        for dtau in (0.01, 3.0):
            Do, Dg = orc.blocks(q, dtau), gpu.blocks(q, dtau)
            for e in range(orc.E):
                assert np.linalg.norm(Dg[e] - Do[e]) <= 1e-10 * np.linalg.norm(Do[e]), (e, dtau)
    finally:
        gpu.close()


def _qc(q):
    rho = q[0] / q[3]
    E = q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2)
    return np.stack([rho, rho * q[1], rho * q[2], rho * E])


@pytest.mark.parametrize("prec", [0, 1])
def test_cylinder_vcycle_and_stage_parity(prec):
    Ma, mu = 0.1, 0.02
    nodes, nbr = W.cylinder_omesh(3, 12, r_in=0.5, r_out=8.0, Ng=2)
    scales = W.freestream_scales(Ma, speed=1.0)
    orc, gpu = _pair(nodes, nbr, 2, [3, 2, 1], [2, 3, 4], Ma, mu, tol=1e-6, max_pseudo=3000, res_scale=scales)
    from paper_1908_03972_gb300 import pmgfr
    gpu.close()
    T = W.freestream_T(Ma, speed=1.0)
    gpu = pmgfr.Solver(nodes, nbr, [3, 2, 1], [2, 3, 4], Ma_inf=Ma, mu=mu, cutoff=1, kappa=1.0,
                       q_inf=(T, 1.0, 0.0, T), tol=1e-6, max_pseudo=3000, res_scale=scales, block_prec=prec)
    try:
        q = W.freestream_noise_state(orc.coords(), Ma)
        omega_dt = 0.4358665215 * 0.05
        src = _qc(q) / omega_dt + 0.5 * orc.residual(q)
        orc.set_stage(src, omega_dt)
        gpu.set_stage(src, omega_dt)
        if prec == 0:
            qo = orc.vcycle(q, 0.01, refresh=True)
            qg, _ = gpu.vcycle(q, 0.01, refresh=True)
            dq = np.abs(qo - q).max(axis=(1, 2))
            assert (np.abs(qg - qo).max(axis=(1, 2)) / dq).max() <= 1e-8
        qo, it_o, drop_o, _, st = orc.stage_solve(q)
        assert st == 0
        qg, it_g, drop_g = gpu.stage_solve(q)
        assert drop_g <= 1e-6
        if prec == 0:
            assert abs(it_g - it_o) <= max(2, 0.05 * it_o), (it_o, it_g)
        du = np.abs(qg[1:3] - qo[1:3]).max()
        dp = np.abs(qg[0] - qo[0]).max()
        assert du <= 1e-5 and dp <= 1e-5 * T, (du, dp)
    finally:
        gpu.close()


def test_boundary_settings_checked():
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.channel(4, 3, Ng=1, bottom=W.BC_SLIP_WALL, top=W.BC_SLIP_WALL)
    with pytest.raises(pmgfr.PmgError):
        pmgfr.Solver(nodes, nbr, [1], [1], mu=0.1, cutoff=1)
    nodes, nbr = W.channel(4, 3, Ng=1)
    with pytest.raises(pmgfr.PmgError):
        pmgfr.Solver(nodes, nbr, [1], [1], cutoff=0)
    nodes, nbr = W.channel(4, 3, Ng=1, bottom=W.BC_FARFIELD, top=W.BC_FARFIELD)
    with pytest.raises(pmgfr.PmgError):
        pmgfr.Solver(nodes, nbr, [1], [1])          # far field without q_inf
    bad = nbr.copy()
    bad[0, 0] = (-1, 7, 0)
    with pytest.raises(pmgfr.PmgError):
        pmgfr.Solver(nodes, bad, [1], [1], q_inf=(1.0, 1.0, 0.0, 1.0))


def test_cfl_form_dtau_min_parity():
    from paper_1908_03972_gb300 import pmgfr
    for Ma, make in ((0.001, lambda: W.cylinder_omesh(16, 64, 0.5, 50.0, Ng=2)),
                     (0.005, lambda: W.periodic_box(8, 8, Ng=1))):
        nodes, nbr = make()
        Ng = 2 if nodes.shape[1] == 9 else 1
        T = W.freestream_T(Ma, speed=1.0)
        kw = dict(Ma_inf=Ma, mu=0.01, cutoff=1, kappa=1.0, q_inf=(T, 1.0, 0.0, T), cfl_mode=1)
        orc = O.Oracle(nodes, nbr, Ng, [4 if Ng == 2 else 2], [1], **kw)
        gpu = pmgfr.Solver(nodes, nbr, [4 if Ng == 2 else 2], [1], **kw)
        try:
            q = W.freestream_noise_state(orc.coords(), Ma, noise=0.05)
            gpu.set_state(q)
            a, b = pmgfr.pmg_dtau_min(gpu.h), orc.dtau_min(q)
            assert abs(a - b) <= 1e-12 * b, (a, b)
        finally:
            gpu.close()


def test_cfl_mode_stage_parity_on_the_cylinder():
    # the paper's wall-bounded setting: CFL_init = 1e2, CFL_max = 1e5
    from paper_1908_03972_gb300 import pmgfr
    Ma, mu = 0.1, 0.02
    nodes, nbr = W.cylinder_omesh(3, 12, r_in=0.5, r_out=8.0, Ng=2)
    T = W.freestream_T(Ma, speed=1.0)
    kw = dict(Ma_inf=Ma, mu=mu, cutoff=1, kappa=1.0, q_inf=(T, 1.0, 0.0, T), tol=1e-6, max_pseudo=3000,
              res_scale=W.freestream_scales(Ma, speed=1.0), cfl_mode=1, cfl_init=1e2, cfl_max=1e5)
    orc = O.Oracle(nodes, nbr, 2, [3, 2, 1], [2, 3, 4], **kw)
    gpu = pmgfr.Solver(nodes, nbr, [3, 2, 1], [2, 3, 4], **kw)
    try:
        q = W.freestream_noise_state(orc.coords(), Ma)
        omega_dt = 0.4358665215 * 0.05
        src = _qc(q) / omega_dt + 0.5 * orc.residual(q)
        orc.set_stage(src, omega_dt)
        gpu.set_stage(src, omega_dt)
        qo, it_o, _, _, st = orc.stage_solve(q)
        assert st == 0
        qg, it_g, drop_g = gpu.stage_solve(q)
        assert drop_g <= 1e-6 and abs(it_g - it_o) <= max(2, 0.05 * it_o), (it_o, it_g)
        assert np.abs(qg[1:3] - qo[1:3]).max() <= 1e-5 and np.abs(qg[0] - qo[0]).max() <= 1e-5 * T
    finally:
        gpu.close()
