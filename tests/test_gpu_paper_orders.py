"""The paper's order studies (Section 4.1, Tables 1 and 2) through the GPU
path, as accuracy pins of the whole solver.

Grid refinement (Table 2):

Setup of Section 4.1: the isentropic vortex of eq. VP_Solution (free stream
rho = u = v = 1, Ma_inf = 0.005, alpha = 5, phi = 1/2, centre at the origin)
on the periodic square [-10, 10]^2 with 12^2, 24^2 and 36^2 straight quads;
P^3 with the hierarchy P{3-2-1} and P^4 with P{4-2-1}; ESDIRK4 with
dt = t~/200 = 0.1 up to t_end = 2.  The paper does not give the smoothing
counts of this study; I{5-10-20} is used.  Every stage is solved to a 1e-8
drop of the free-stream-scaled norm: the paper's 1e-4 refers to its own
norm, and at a 1e-4 drop of the scaled norm the P^4 velocity error on the
finest mesh stops at the solver's accuracy (order 0.3), the effect the paper
reports for rho and p.

The velocity orders between consecutive meshes must reproduce the printed
ones (tests/golden/paper_orders.json, from Table 2) to 0.05: the paper prints
two decimals and does not define its error norm (here the discrete L2 norm
with the Gauss weights), which can move the third.  Measured: 4.369 / 3.913
(P^3) and 4.720 / 4.230 (P^4) against 4.37 / 3.91 and 4.72 / 4.23.

Time refinement (Table 1), reduced form run by default: ESDIRK3 alone, the
same P^5 50^2 mesh and P{5-3-1}, I{20-20-40}, stages to a 1e-6 drop, but over
a tenth of the period (t_end = 2) with dt = t~/100, t~/200, t~/400 (10, 20 and
40 steps).  Over the shorter interval the temporal error is a tenth of the
printed one and still far above the spatial error of P^5 on 50^2; the rates
must reproduce Table 1's ESDIRK3 velocity orders (2.73, 2.94) to 0.15, the
margin allowing for the shorter accumulation of the error.

Time refinement (Table 1), full form opt-in (about 15 GPU-minutes; set PMG_RUN_TABLE1=1):
P^5 on a 50^2 mesh of the same square, P{5-3-1}, I{20-20-40}, one period
t~ = 20 with ESDIRK2 and ESDIRK3 at dt = t~/100, t~/200, t~/400 and ESDIRK4 at
t~/40, t~/80, t~/120, stages to a 1e-6 drop of the scaled norm.  The velocity
orders must reproduce the printed ones to 0.05.  Measured: 1.98 / 2.00,
2.73 / 2.94 and 3.87 / 3.97 against 1.98 / 2.00, 2.73 / 2.94 and 3.87 / 4.00.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_orders.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()


def _velocity_error(P, levels, n):
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(n, n, -10.0, 10.0, -10.0, 10.0, Ng=1)
    gpu = pmgfr.Solver(nodes, nbr, levels, [5, 10, 20], Ma_inf=0.005, tol=1e-8, dtau_init=0.01, dtau_max=10.0,
                       refresh_every=10, max_pseudo=20000, p_gauge=W.freestream_T(0.005),
                       res_scale=W.freestream_scales(0.005), esdirk_order=4, block_prec=pmgfr.PMG_PREC_FP32)
    try:
        xy = gpu.coords()
        gpu.set_state(W.isentropic_vortex(xy, center=(0.0, 0.0), period=(20.0, 20.0)))
        for _ in range(20):
            pmgfr.pmg_esdirk_step(gpu.h, 0.1)
        q = gpu.get_state()
    finally:
        gpu.close()
    qe = W.isentropic_vortex(xy, t=2.0, center=(0.0, 0.0), period=(20.0, 20.0))
    _, w = np.polynomial.legendre.leggauss(P + 1)
    wJ = np.outer(w, w).reshape(-1) * (10.0 / n) ** 2     # Gauss weights x |J| of a square of side 20/n
    return math.sqrt(float((wJ[None, :] * (q[1] - qe[1]) ** 2).sum()))


@pytest.mark.parametrize("P,levels,key", [(3, [3, 2, 1], "fr_P3_velocity_orders"),
                                          (4, [4, 2, 1], "fr_P4_velocity_orders")])
def test_table2_velocity_orders(P, levels, key):
    paper = json.load(open(GOLDEN))[key]
    meshes = (12, 24, 36)
    err = [_velocity_error(P, levels, n) for n in meshes]
    orders = [math.log(err[i] / err[i + 1]) / math.log(meshes[i + 1] / meshes[i]) for i in range(2)]
    for ours, theirs in zip(orders, paper):
        assert abs(ours - theirs) <= 0.05, (orders, paper, err)


def _time_error(order, n_steps, t_end=20.0):
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(50, 50, -10.0, 10.0, -10.0, 10.0, Ng=1)
    gpu = pmgfr.Solver(nodes, nbr, [5, 3, 1], [20, 20, 40], Ma_inf=0.005, tol=1e-6, dtau_init=0.01, dtau_max=10.0,
                       refresh_every=10, max_pseudo=20000, p_gauge=W.freestream_T(0.005),
                       res_scale=W.freestream_scales(0.005), esdirk_order=order, block_prec=pmgfr.PMG_PREC_FP32)
    try:
        xy = gpu.coords()
        gpu.set_state(W.isentropic_vortex(xy, center=(0.0, 0.0), period=(20.0, 20.0)))
        for _ in range(n_steps):
            pmgfr.pmg_esdirk_step(gpu.h, t_end / n_steps)
        q = gpu.get_state()
    finally:
        gpu.close()
    qe = W.isentropic_vortex(xy, t=t_end, center=(0.0, 0.0), period=(20.0, 20.0))
    _, w = np.polynomial.legendre.leggauss(6)
    wJ = np.outer(w, w).reshape(-1) * (10.0 / 50) ** 2
    return math.sqrt(float((wJ[None, :] * (q[1] - qe[1]) ** 2).sum()))


@pytest.mark.skipif(os.environ.get("PMG_RUN_TABLE1") != "1", reason="about 15 GPU-minutes: set PMG_RUN_TABLE1=1")
@pytest.mark.parametrize("order,steps,key", [(2, (100, 200, 400), "esdirk2_time_orders"),
                                             (3, (100, 200, 400), "esdirk3_time_orders"),
                                             (4, (40, 80, 120), "esdirk4_time_orders")])
def test_table1_velocity_orders(order, steps, key):
    paper = json.load(open(GOLDEN))[key]["u"]
    err = [_time_error(order, n) for n in steps]
    orders = [math.log(err[i] / err[i + 1]) / math.log(steps[i + 1] / steps[i]) for i in range(2)]
    for ours, theirs in zip(orders, paper):
        assert abs(ours - theirs) <= 0.05, (orders, paper, err)


def test_table1_esdirk3_orders_reduced():
    paper = json.load(open(GOLDEN))["esdirk3_time_orders"]["u"]
    steps = (10, 20, 40)   # dt = 0.2, 0.1, 0.05 = t~/100, t~/200, t~/400 up to t = 2
    err = [_time_error(3, n, t_end=2.0) for n in steps]
    orders = [math.log(err[i] / err[i + 1]) / math.log(steps[i + 1] / steps[i]) for i in range(2)]
    print(f"Table 1 reduced (ESDIRK3, t = 2): errors {err}, orders {orders}, paper {paper}")
    for ours, theirs in zip(orders, paper):
        assert abs(ours - theirs) <= 0.15, (orders, paper, err)
