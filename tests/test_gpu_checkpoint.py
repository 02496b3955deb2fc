"""Checkpoint and restore through the C interface: a restored context repeats
the next physical step bit for bit, and foreign files are rejected."""
import numpy as np
import pytest

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


KW = dict(tol=1e-8, dtau_init=0.01, dtau_max=10.0, refresh_every=10, max_pseudo=4000,
          res_scale=W.freestream_scales(0.005), p_gauge=W.freestream_T(0.005))


def _solver(n=8, prec=1, **extra):
    from paper_1908_03972_gb300 import pmgfr
    nodes, nbr = W.periodic_box(n, n, Ng=1)
    return pmgfr.Solver(nodes, nbr, [2, 1, 0], [5, 10, 20], block_prec=prec, **{**KW, **extra})


def test_restore_repeats_the_next_step_bit_for_bit(tmp_path):
    from paper_1908_03972_gb300 import pmgfr
    path = str(tmp_path / "c1.ckpt")
    a = _solver()
    try:
        a.set_state(W.isentropic_vortex(a.coords()))
        pmgfr.pmg_esdirk_step(a.h, 0.1)
        pmgfr.pmg_checkpoint(a.h, path)
        pmgfr.pmg_esdirk_step(a.h, 0.1)
        qa = a.get_state()
        # the same context, rolled back
        pmgfr.pmg_restore(a.h, path)
        pmgfr.pmg_esdirk_step(a.h, 0.1)
        assert np.array_equal(a.get_state(), qa)
    finally:
        a.close()
    b = _solver()   # a fresh context
    try:
        pmgfr.pmg_restore(b.h, path)
        pmgfr.pmg_esdirk_step(b.h, 0.1)
        assert np.array_equal(b.get_state(), qa)
    finally:
        b.close()


def test_restore_rejects_other_meshes_settings_and_bad_files(tmp_path):
    from paper_1908_03972_gb300 import pmgfr
    path = str(tmp_path / "c1.ckpt")
    a = _solver()
    try:
        a.set_state(W.isentropic_vortex(a.coords()))
        pmgfr.pmg_checkpoint(a.h, path)
    finally:
        a.close()
    for other in (dict(n=6), dict(mu=0.01), dict(p_gauge=0.0)):
        n = other.pop("n", 8)
        s = _solver(n=n, **other)
        try:
            with pytest.raises(pmgfr.PmgError):
                pmgfr.pmg_restore(s.h, path)
        finally:
            s.close()
    raw = open(path, "rb").read()
    s = _solver()
    try:
        for bad, name in ((raw[:-8], "short"), (raw + b"x", "long"), (b"XXXXXXXX" + raw[8:], "magic")):
            p = str(tmp_path / name)
            open(p, "wb").write(bad)
            with pytest.raises(pmgfr.PmgError):
                pmgfr.pmg_restore(s.h, p)
        with pytest.raises(pmgfr.PmgError):
            pmgfr.pmg_restore(s.h, str(tmp_path / "missing"))
    finally:
        s.close()
