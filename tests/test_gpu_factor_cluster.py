"""The element-block factorisation on a thread-block cluster
(k_factor_cluster.cu): blocks larger than one CTA's shared memory, the
hexahedral P = 3 blocks (n = 320) first, with their columns spread over 2, 4
or 8 CTAs.

- The cluster kernel performs the one-CTA kernel's operations on every entry
  in the same order, so with PMG_FACTOR_CLUSTER forcing it onto blocks that
  one CTA holds (2D P = 3, n = 64; hexahedra P = 2, n = 135), the factored
  blocks applied to the same vector give the same result bit for bit.
- At n = 320 (hexahedra, P = 3, where one CTA cannot hold the block) the
  applied inverse matches a dense solve of the library's own assembled block
  to the bounds of the P <= 2 test (FP64 1e-11, FP32 2e-4, BF16 5e-2), the
  assembled blocks match the oracle's complex-step blocks to 1e-10, and a
  P{3-2-1} V-cycle matches the oracle's to 1e-8 of the change it makes.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROT = {0: 5, 4: 11, 7: 17, 11: 3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()


def _state3(xyz, Ma=0.005, seed=1):
    q = W.vortex3d(xyz, Ma_inf=Ma, center=(4.3, 5.6))
    rng = np.random.default_rng(seed)
    return q * (1 + 1e-3 * rng.standard_normal(q.shape) * np.array([1e-3, 1, 1, 1, 1e-5])[:, None, None])


def _apply_after_factor(monkeypatch, force, make, q, r):
    from paper_1908_03972_gb300 import pmgfr
    monkeypatch.delenv("PMG_FACTOR_CLUSTER", raising=False)
    if force:
        monkeypatch.setenv("PMG_FACTOR_CLUSTER", str(force))
    s = make()
    try:
        s.set_stage(np.zeros_like(q), 0.0436)
        s.blocks(q, 1.0)
        pmgfr.pmg_factor_blocks(s.h, 0)
        return s.apply(r)
    finally:
        s.close()


@pytest.mark.parametrize("C", [2, 4, 8])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("case", ["quads_P3", "hexes_P2"])
def test_cluster_factor_is_bit_identical_to_one_cta(monkeypatch, case, prec, C):
    from paper_1908_03972_gb300 import pmgfr
    if case == "quads_P3":
        nodes, nbr = W.periodic_box(4, 4, Ng=2, perturb=0.3)
        make = lambda: pmgfr.Solver(nodes, nbr, [3], [1], block_prec=prec)
        probe = pmgfr.Solver(nodes, nbr, [3], [1])
        q = W.isentropic_vortex(probe.coords(), center=(4.0, 6.0))
        w = np.array([1e-3, 1.0, 1.0, 1e2])
    else:
        nodes, nbr = W.periodic_box3d(3, 3, 2, Ng=2, perturb=0.3, rotations=ROT)
        make = lambda: pmgfr.Solver(nodes, nbr, [2], [1], block_prec=prec, dim=3)
        probe = pmgfr.Solver(nodes, nbr, [2], [1], dim=3)
        q = _state3(probe.coords())
        w = np.array([1e-3, 1.0, 1.0, 1.0, 1e2])
    probe.close()
    r = np.random.default_rng(3).standard_normal(q.shape) * w[:, None, None]
    x1 = _apply_after_factor(monkeypatch, 0, make, q, r)
    xC = _apply_after_factor(monkeypatch, C, make, q, r)
    assert np.array_equal(x1, xC)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-4), (2, 5e-2)])
def test_p3_hexahedral_blocks_factor_and_apply(prec, tol):
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box3d(3, 3, 2, Ng=2, perturb=0.3, rotations=ROT)
    gpu = pmgfr.Solver(nodes, nbr, [3], [1], block_prec=prec, dim=3)
    try:
        q = _state3(gpu.coords())
        gpu.set_stage(np.zeros_like(q), 0.0436)
        D = gpu.blocks(q, 1.0)
        assert D.shape[1] == 320
        gpu.factor()
        r = np.random.default_rng(3).standard_normal(q.shape) * np.array([1e-3, 1.0, 1.0, 1.0, 1e2])[:, None, None]
        x = gpu.apply(r)
        for e in range(gpu.E):
            xe = np.linalg.solve(D[e], r[:, e].reshape(-1))
            assert np.linalg.norm(x[:, e].reshape(-1) - xe) <= tol * np.linalg.norm(xe), e
    finally:
        gpu.close()


def _pair3(nodes, nbr, Ng, levels, smooth, prec=0):
    from paper_1908_03972_gb300 import pmgfr
    orc = O.Oracle3(nodes, nbr, Ng, levels, smooth, Ma_inf=0.005)
    gpu = pmgfr.Solver(nodes, nbr, levels, smooth, Ma_inf=0.005, block_prec=prec, dim=3)
    return orc, gpu


def test_p3_hexahedral_blocks_match_oracle():
    nodes, nbr = W.periodic_box3d(3, 2, 3, Ng=1, rotations={1: 7, 8: 14})
    orc, gpu = _pair3(nodes, nbr, 1, [3], [1])
    try:
        q = _state3(orc.coords())
        orc.set_stage(np.zeros_like(q), 0.0436)
        gpu.set_stage(np.zeros_like(q), 0.0436)
        Do, Dg = orc.blocks(q, 0.5), gpu.blocks(q, 0.5)
        for e in range(orc.E):
            assert np.linalg.norm(Dg[e] - Do[e]) <= 1e-10 * np.linalg.norm(Do[e]), e
    finally:
        gpu.close()


def test_p3_vcycle3_parity():
    """P{3-2-1}, I{1-2-3} (9 sweeps) on the straight box: one V-cycle that
    builds the smoother (the P = 3 blocks on clusters) and one with it frozen,
    FP64 blocks, 1e-8 of the change each makes (the bound of the P{2-1-0}
    test)."""
    nodes, nbr = W.periodic_box3d(3, 2, 3, Ng=1, rotations={1: 7, 8: 14})
    orc, gpu = _pair3(nodes, nbr, 1, [3, 2, 1], [1, 2, 3])
    try:
        q = _state3(orc.coords())
        rho = q[0] / q[4]
        qc = np.stack([rho, rho * q[1], rho * q[2], rho * q[3],
                       rho * (q[4] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2 + q[3] ** 2))])
        src = qc / 0.0436 + 0.5 * orc.residual(q)
        orc.set_stage(src, 0.0436)
        gpu.set_stage(src, 0.0436)
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
