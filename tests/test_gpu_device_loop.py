"""The device-side stage loop (pmg_config.device_loop = 1): the
pseudo-iterations of each implicit stage (Section 2.4: SER growth of dtau by
eq. ser, smoother rebuild rule, stop at the relative drop tol) run as one CUDA
graph whose conditional WHILE node repeats a one-thread controller and the
V-cycle, instead of a host loop that reads the norm after every V-cycle.

Both loops apply the same rules; the device's pow may round dtau differently
in the last bit, so V-cycle counts may differ by one where a stage crosses
its tolerance, and converged states by the tolerance the stopping test allows
(the bounds of the oracle parity tests)."""
import numpy as np
import pytest

from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KW = dict(tol=1e-8, dtau_init=0.01, dtau_max=10.0, refresh_every=10, max_pseudo=4000,
          res_scale=W.freestream_scales(0.005), p_gauge=W.freestream_T(0.005))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_device_loop_steps_match_host_loop(prec):
    """Two consecutive ESDIRK3 steps of the C1 vortex (8x8, P{2-1-0},
    I{5-10-20}) with each loop."""
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(8, 8, Ng=1)
    runs = {}
    for dl in (0, 1):
        s = pmgfr.Solver(nodes, nbr, [2, 1, 0], [5, 10, 20], block_prec=prec, device_loop=dl, **KW)
        try:
            q = W.isentropic_vortex(s.coords())
            out = []
            for _ in range(2):
                q, st = s.esdirk_step(q, 0.1)
                norms, dtau = pmgfr.pmg_stage_history(s.h)
                out.append((q, list(st.pseudo_iters)[:3], st.n_refresh, max(st.res_drop[:3]), norms, dtau))
            runs[dl] = out
        finally:
            s.close()
    for (qh, ith, nrh, drh, nh, dh), (qd, itd, nrd, drd, nd, dd) in zip(runs[0], runs[1]):
        assert drd <= 1e-8 and drh <= 1e-8
        assert all(abs(a - b) <= 1 for a, b in zip(ith, itd)), (ith, itd)
        assert abs(nrh - nrd) <= 3, (nrh, nrd)
        # one history entry per pseudo-iteration and stage, plus the final norm
        assert len(nd) == sum(itd) + 3 and len(dd) == len(nd)
        assert np.abs(qd[0] - qh[0]).max() / 2.0 <= 2e-6 and np.abs(qd[1:3] - qh[1:3]).max() <= 1e-7
        k = min(len(nh), len(nd), 20)   # the first norms agree to rounding
        assert np.allclose(nd[:k], nh[:k], rtol=1e-9, atol=0.0)


def test_device_loop_graph_rebuilt_for_another_stage_form():
    """pmg_stage_solve after pmg_set_stage (full source) and pmg_esdirk_step
    (split source) use different V-cycle graphs; both converge."""
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(4, 4, Ng=1)
    s = pmgfr.Solver(nodes, nbr, [2, 1, 0], [2, 3, 4], device_loop=1, **KW)
    try:
        q = W.isentropic_vortex(s.coords(), center=(4.0, 6.0))
        rho = q[0] / q[3]
        qc = np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])
        odt = 0.0436
        s.set_stage(qc / odt + 0.5 * s.residual(q), odt)
        q1, it, drop = s.stage_solve(q)
        assert drop <= 1e-8 and it > 0
        q2, st = s.esdirk_step(q, 0.1)
        assert max(st.res_drop[:3]) <= 1e-8 and min(list(st.pseudo_iters)[:3]) > 0
    finally:
        s.close()
