"""The allocation-free residual entry point (pmg_residual_static).

Some callers cannot allocate device memory once they run (a fixed device
budget, or all spare memory handed to their own pool), so the library offers
a residual call whose scratch lives in a static device array.  It must give
the same residual as the regular entry point, on repeated calls, and must
not change the device's free memory after its first call.  This file is
collected last on purpose: it also has to pass after every other GPU test.
"""
import numpy as np
import pytest

from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()
    return torch, pmgfr


# (p_gauge, mu, Ma_inf): absolute and gauge pressure storage of the Euler
# residual, and the viscous residual, whose broken gradients and face jumps
# also live in the static scratch
CASES = [(0.0, 0.0, 0.005), (W.freestream_T(0.005), 0.0, 0.005), (0.0, 0.02, 0.3)]


@pytest.mark.parametrize("gauge,mu,Ma", CASES)
def test_static_residual_matches_regular_entry_point(setup, gauge, mu, Ma):
    torch, pmgfr = setup
    nodes, nbr = W.periodic_box(24, 20, Ng=1)
    s = pmgfr.Solver(nodes, nbr, [3, 2, 1, 0], [1, 1, 1, 1], p_gauge=gauge, mu=mu, Ma_inf=Ma)
    try:
        dev = torch.device("cuda", torch.cuda.current_device())
        for level in range(4):
            q = W.isentropic_vortex(s.coords(level), center=(4.0, 6.0), Ma_inf=Ma)
            q_dev = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
            ref = torch.empty_like(q_dev)
            pmgfr.pmg_residual(s.h, level, q_dev, ref)
            out1 = torch.full_like(q_dev, float("nan"))
            out2 = torch.full_like(q_dev, float("nan"))
            pmgfr.pmg_residual_static(s.h, level, q_dev, out1)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            pmgfr.pmg_residual_static(s.h, level, q_dev, out2)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert free_after == free_before
            r = ref.cpu().numpy()
            for out in (out1, out2):
                o = out.cpu().numpy()
                assert np.isfinite(o).all()
                # same kernels, same inputs: identical up to the tolerance of the parity tests
                for v in range(4):
                    assert np.abs(o[v] - r[v]).max() <= 1e-10 * max(np.abs(r[v]).max(), 1e-300)
    finally:
        s.close()


def test_static_residual_rejects_oversized_levels(setup):
    torch, pmgfr = setup
    # 4 E N + 16 E (P+1) doubles must fit in 2^21 = 2.10e6: E = 36864 at P = 3
    # needs 2,359,296 + 2,359,296 = 4.72e6
    nodes, nbr = W.periodic_box(192, 192, Ng=1)
    s = pmgfr.Solver(nodes, nbr, [3], [1])
    try:
        dev = torch.device("cuda", torch.cuda.current_device())
        q = torch.zeros((4, s.E, 16), dtype=torch.float64, device=dev)
        out = torch.zeros_like(q)
        with pytest.raises(pmgfr.PmgError) as ei:
            pmgfr.pmg_residual_static(s.h, 0, q, out)
        assert "scratch" in str(ei.value)
    finally:
        s.close()


@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_static_residual_matches_on_hexahedra(setup, mu):
    """Hexahedra (five variables, 12 gradient planes and 24 E NF face jumps
    in the static scratch with mu > 0) on a curved box, every level."""
    torch, pmgfr = setup
    nodes, nbr = W.periodic_box3d(3, 3, 2, Ng=2, perturb=0.3, rotations={0: 5, 4: 17})
    s = pmgfr.Solver(nodes, nbr, [3, 2, 1, 0], [1, 1, 1, 1], mu=mu, Ma_inf=0.3, dim=3)
    try:
        dev = torch.device("cuda", torch.cuda.current_device())
        for level in range(4):
            q = W.vortex3d(s.coords(level), Ma_inf=0.3, center=(4.3, 5.6))
            q_dev = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
            ref = torch.empty_like(q_dev)
            pmgfr.pmg_residual(s.h, level, q_dev, ref)
            out = torch.full_like(q_dev, float("nan"))
            pmgfr.pmg_residual_static(s.h, level, q_dev, out)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            pmgfr.pmg_residual_static(s.h, level, q_dev, out)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free_before
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            for v in range(5):
                assert np.abs(o[v] - r[v]).max() <= 1e-10 * max(np.abs(r[v]).max(), 1e-300)
    finally:
        s.close()
