"""The multi-sweep coarse-level smoother (k_tile.cu): several element-Jacobi
sweeps per launch on tiles that carry a halo of face neighbours.  Per element
and sweep it repeats the arithmetic of the one-sweep fused kernel operation for
operation, so V-cycles and stage solves with tiles must give the states of the
per-sweep path bit for bit, for any number of sweeps per launch (including a
last launch with fewer sweeps than the tile depth)."""
import numpy as np
import pytest

from paper_1908_03972_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TINF = W.freestream_T(0.005)
KW = dict(p_gauge=TINF, tol=1e-8, res_scale=W.freestream_scales(0.005), max_pseudo=4000)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03972_gb300 import build, pmgfr
    build.build()
    pmgfr.load()


def _qc(q):
    rho = q[0] / q[3]
    return np.stack([rho, rho * q[1], rho * q[2], rho * (q[3] / 0.4 + 0.5 * (q[1] ** 2 + q[2] ** 2))])


def _run(monkeypatch, env, prec, n=16, levels=(3, 2, 1, 0), smooth=(1, 2, 5, 9), stage=False):
    from paper_1908_03972_gb300 import pmgfr
    for k in ("PMG_TILE_DEPTH", "PMG_TILE_DEPTH1", "PMG_FUSE_MAX_P", "PMG_TILE_CORE", "PMG_TILE_CORE1"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, str(v))
    nodes, nbr = W.periodic_box(n, n, Ng=1)
    s = pmgfr.Solver(nodes, nbr, list(levels), list(smooth), block_prec=prec, **KW)
    try:
        q = W.isentropic_vortex(s.coords(), center=(4.0, 6.0))
        odt = 0.0436
        s.set_stage(_qc(q) / odt + 0.5 * s.residual(q), odt)
        if stage:
            qs, it, drop = s.stage_solve(q)
            return qs, it, drop
        q1, _ = s.vcycle(q, 0.01, refresh=True)
        q2, _ = s.vcycle(q1, 1.0, refresh=False)
        return q1, q2
    finally:
        s.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("depth", [2, 3, 4])
def test_tiled_p0_sweeps_are_bit_identical(monkeypatch, prec, depth):
    ref = _run(monkeypatch, {}, prec)
    # a CTA holds (tile elements) x (face points) <= 512 threads: cores of 32
    # elements take at most 3 halo layers at P = 0, cores of 16 take 4
    til = _run(monkeypatch, {"PMG_TILE_DEPTH": depth, "PMG_TILE_CORE": 32 if depth < 4 else 16}, prec)
    for a, b in zip(ref, til):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [1, 2])
def test_tiled_p1_sweeps_are_bit_identical_to_fused(monkeypatch, prec):
    ref = _run(monkeypatch, {"PMG_FUSE_MAX_P": 1}, prec)
    til = _run(monkeypatch, {"PMG_FUSE_MAX_P": 1, "PMG_TILE_DEPTH": 4, "PMG_TILE_CORE": 16, "PMG_TILE_DEPTH1": 2,
                             "PMG_TILE_CORE1": 16}, prec)
    for a, b in zip(ref, til):
        assert np.array_equal(a, b)


def test_tiled_stage_solve_is_bit_identical(monkeypatch):
    ref = _run(monkeypatch, {}, 1, n=12, levels=(2, 1, 0), smooth=(3, 5, 10), stage=True)
    til = _run(monkeypatch, {"PMG_TILE_DEPTH": 4, "PMG_TILE_CORE": 16}, 1, n=12, levels=(2, 1, 0), smooth=(3, 5, 10),
               stage=True)
    assert ref[1] == til[1] and ref[2] == til[2] and ref[2] <= 1e-8
    assert np.array_equal(ref[0], til[0])


def test_oversized_tile_is_refused(monkeypatch):
    """A tile whose elements x face points exceed one CTA's 512 threads is
    refused at upload with PMG_EINVAL, before any launch."""
    from paper_1908_03972_gb300 import pmgfr
    with pytest.raises(pmgfr.PmgError) as ei:
        _run(monkeypatch, {"PMG_TILE_DEPTH": 4, "PMG_TILE_CORE": 32}, 1)
    assert ei.value.status == pmgfr.PMG_EINVAL and "does not fit" in str(ei.value)


def test_autotune_reports_choices_and_keeps_convergence(monkeypatch, tmp_path):
    """pmg_autotune times the tunable coarse levels' schedules and keeps the
    fastest; a stage solve afterwards converges to the state of the untuned
    solver (within the stopping tolerance), and a second call with the cache
    file applies the recorded choice without timing the others."""
    from paper_1908_03972_gb300 import pmgfr
    for k in ("PMG_TILE_DEPTH", "PMG_TILE_DEPTH1", "PMG_FUSE_MAX_P"):
        monkeypatch.delenv(k, raising=False)
    nodes, nbr = W.periodic_box(16, 16, Ng=1)
    res = {}
    for tuned in (False, True):
        s = pmgfr.Solver(nodes, nbr, [3, 2, 1, 0], [1, 2, 5, 9], block_prec=1, **KW)
        try:
            q = W.isentropic_vortex(s.coords(), center=(4.0, 6.0))
            odt = 0.0436
            s.set_stage(_qc(q) / odt + 0.5 * s.residual(q), odt)
            s.vcycle(q, 0.01, refresh=True)
            if tuned:
                cache = str(tmp_path / "tune.txt")
                rep = pmgfr.pmg_autotune(s.h, reps=2, cache_path=cache)
                assert set(rep) == {2, 3}                      # the P = 1 and P = 0 levels
                assert rep[3]["candidates"] >= 2 and rep[2]["candidates"] >= 3
                assert all(v["us_per_sweep"] > 0 for v in rep.values())
                rep2 = pmgfr.pmg_autotune(s.h, reps=1, cache_path=cache)
                assert all(rep2[l]["candidates"] == 1 for l in rep2)
                assert all((rep2[l]["fused"], rep2[l]["tile_core"], rep2[l]["tile_depth"]) ==
                           (rep[l]["fused"], rep[l]["tile_core"], rep[l]["tile_depth"]) for l in rep)
            qs, it, drop = s.stage_solve(q)
            assert drop <= 1e-8
            res[tuned] = qs
        finally:
            s.close()
    assert np.abs(res[True][0] - res[False][0]).max() / 2.0 <= 2e-6
    assert np.abs(res[True][1:3] - res[False][1:3]).max() <= 1e-7
