"""The wall-ring instability of the cylinder workload's first stage, shown on
the FP64 oracle (the method's own steps, Sections 2.4 and 3).

Setting: the cylinder geometry at 1/16 of its size (16 x 64 Q2 quads, r from
0.5 to 50), Re = 100, Ma = 0.001, no-slip adiabatic wall, P{4-2-1},
I{5-10-20}, the first ESDIRK3 stage from the free stream with 1e-3 seeded
noise in v, and the configured Delta tau_max = 10 held fixed.

What the oracle shows:
- with the element blocks built at the start (the configured rebuild every 10
  pseudo-iterations), the residual first falls and then grows about threefold
  per V-cycle, and the growth sits in the two rings of elements nearest the
  wall (most of it in the first), in the streamwise velocity;
- rebuilding the blocks at the state where the growth starts restores the
  contraction.
The impulsive start puts u = 1 on the no-slip wall; within a few V-cycles the
wall ring's velocity drops, and blocks linearised at the free stream with a
pseudo-time term Gamma/Delta tau too small to dominate them overcorrect it.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1908_03972_gb300 import workloads as W

MA, MU = 0.001, 0.01
T = W.freestream_T(MA, speed=1.0)
NR, NT = 16, 64


def _setup():
    nodes, nbr = W.cylinder_omesh(NR, NT, 0.5, 50.0, Ng=2, wall=W.BC_NOSLIP_WALL)
    orc = O.Oracle(nodes, nbr, 2, [4, 2, 1], [5, 10, 20], Ma_inf=MA, cutoff=1, kappa=1.0,
                   q_inf=(T, 1.0, 0.0, T), mu=MU, res_scale=W.freestream_scales(MA, speed=1.0))
    q = W.freestream_noise_state(orc.coords(), MA)
    odt = 0.4358665215 * 0.05                       # ESDIRK3 diagonal x dt = 0.05
    rho = q[0] / q[3]
    qc = np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])
    orc.set_stage(qc / odt, odt)
    return orc, q


def _norm(orc, q):
    F = orc.stage_F(q)
    sc = W.freestream_scales(MA, speed=1.0)
    return float(np.sqrt(sum(((F[v] / sc[v]) ** 2).sum() for v in range(4))))


@pytest.fixture(scope="module")
def onset():
    O.set_threads(os.cpu_count() or 1)
    orc, q = _setup()
    norms = [_norm(orc, q)]
    for k in range(5):                              # blocks built at V-cycle 0 only
        q = orc.vcycle(q, 10.0, refresh=(k == 0))
        norms.append(_norm(orc, q))
    yield orc, q, norms
    O.set_threads(1)


def test_stale_blocks_grow_threefold_in_the_wall_ring(onset):
    orc, q5, norms = onset
    assert norms[5] < 0.05 * norms[0]                # the first V-cycles converge
    q = q5.copy()
    states = [q]
    for k in range(4):                              # still the blocks of V-cycle 0
        q = orc.vcycle(q, 10.0, refresh=False)
        states.append(q)
        norms.append(_norm(orc, q))
    growth = [norms[k + 1] / norms[k] for k in range(6, 9)]
    assert min(growth) > 2.0, norms
    d = (states[4] - states[3]) / np.array([T, 1.0, 1.0, T])[:, None, None]
    ring = np.arange(orc.E) % NR                    # element e = j NR + i, i = 0 at the wall
    energy = (d ** 2).sum(axis=(0, 2))
    assert energy[ring == 0].sum() > 0.5 * energy.sum()           # one ring of 16 elements deep
    assert energy[ring <= 1].sum() > 0.8 * energy.sum()
    by_var = (d ** 2).sum(axis=(1, 2))
    assert by_var[1] > 0.8 * by_var.sum()             # streamwise velocity


def test_blocks_rebuilt_at_the_onset_contract(onset):
    orc, q5, norms = onset
    q = orc.vcycle(q5.copy(), 10.0, refresh=True)    # blocks linearised at the onset state
    later = [_norm(orc, q)]
    for k in range(4):
        q = orc.vcycle(q, 10.0, refresh=False)
        later.append(_norm(orc, q))
    assert later[-1] < norms[5], (norms[5], later)
    assert all(b < a for a, b in zip(later, later[1:])), later
