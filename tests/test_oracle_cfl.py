"""Pins of the CFL form of the pseudo time step (Section 2.4, eq. CFL):
element sizes, dtau_min, and the equivalence of CFL mode with dtau set to
CFL dtau_min."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W


def test_element_size_of_squares_and_rectangles():
    nodes, nbr = W.periodic_box(4, 5, 0, 10, 0, 6, Ng=1)
    o = O.Oracle(nodes, nbr, 1, [1], [1])
    # centroid to nearest face of a 2.5 x 1.2 rectangle is 0.6
    assert np.allclose(o.element_dx(), 1.2, rtol=1e-13)
    nodes, nbr = W.periodic_box(3, 3, Ng=2)          # quadratic nodes of straight squares
    o = O.Oracle(nodes, nbr, 2, [2], [1])
    assert np.allclose(o.element_dx(), 10.0 / 3, rtol=1e-13)


def test_element_size_of_annular_sectors():
    # Centroid of the sector r0 < r < r1, |theta - theta_c| < a/2 lies on the
    # bisector at r_c = (2/3) (r1^3 - r0^3)/(r1^2 - r0^2) sin(a/2)/(a/2); its
    # distances to the arcs and radial edges are r_c - r0, r1 - r_c and
    # r_c sin(a/2).  The quadratic map reproduces the arcs to ~1e-4 here.
    n_r, n_t = 8, 32
    nodes, nbr = W.cylinder_omesh(n_r, n_t, 0.5, 5.0, Ng=2)
    o = O.Oracle(nodes, nbr, 2, [2], [1], q_inf=(1, 1, 0, 1), cutoff=1)
    rk = 0.5 * (10.0) ** (np.arange(n_r + 1) / n_r)
    a = 2 * math.pi / n_t
    r0, r1 = rk[:-1], rk[1:]
    rc = (2.0 / 3.0) * (r1 ** 3 - r0 ** 3) / (r1 ** 2 - r0 ** 2) * math.sin(a / 2) / (a / 2)
    exact = 2 * np.minimum(np.minimum(rc - r0, r1 - rc), rc * math.sin(a / 2))
    dx = o.element_dx()[:n_r]                         # the first angular column
    assert np.allclose(dx, exact, rtol=2e-3), (dx, exact)


def test_dtau_min_closed_forms():
    nodes, nbr = W.periodic_box(4, 4, Ng=1)          # squares of side 2.5
    T = W.freestream_T(0.3)
    for P in (1, 3):
        o = O.Oracle(nodes, nbr, 1, [P], [1], Ma_inf=0.3)
        q = W.uniform_state(o.E, o.N(), T, 1.0, 1.0, T)
        inv = (2.5 / (P + 1)) / (math.sqrt(1.4 * T) + math.sqrt(2.0))
        assert abs(o.dtau_min(q) - inv) <= 1e-12 * inv
        mu = 50.0                                      # the viscous bound takes over
        ov = O.Oracle(nodes, nbr, 1, [P], [1], Ma_inf=0.3, mu=mu)
        vis = (2.5 / (P + 1)) ** 2 * 1.0 / mu
        assert abs(ov.dtau_min(q) - min(inv, vis)) <= 1e-12 * vis and vis < inv


def test_cfl_mode_is_dtau_mode_with_scaled_bounds():
    nodes, nbr = W.periodic_box(4, 4, Ng=1)
    kw = dict(tol=1e-6, max_pseudo=400, res_scale=W.freestream_scales(0.005))
    oc = O.Oracle(nodes, nbr, 1, [2, 1], [3, 6], cfl_mode=1, cfl_init=50.0, cfl_max=5e4, **kw)
    q = W.isentropic_vortex(oc.coords())
    dm = oc.dtau_min(q)
    od = O.Oracle(nodes, nbr, 1, [2, 1], [3, 6], dtau_init=50.0 * dm, dtau_max=5e4 * dm, **kw)
    rho = q[0] / q[3]
    qc = np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])
    for o in (oc, od):
        o.set_stage(qc / 0.0436 + 0.5 * o.residual(q), 0.0436)
    a = oc.stage_solve(q)
    b = od.stage_solve(q)
    assert a[4] == 0 and b[4] == 0 and a[1] == b[1]
    assert np.array_equal(a[0], b[0])
