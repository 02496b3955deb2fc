"""Python binding of libpmgfr (argument marshalling only).

Functions carry the names of the C interface in ``include/pmgfr.h``.  Arrays
may be NumPy arrays (host memory) or CUDA ``torch.Tensor`` objects (device
memory on the context's device); every computation runs in the library's
CUDA kernels.  There is no CPU fallback: if the library is missing the import
of this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpmgfr.so")

PMG_OK = 0
PMG_EINVAL, PMG_ENOMEM, PMG_ECUDA, PMG_ESINGULAR, PMG_ENONFINITE, PMG_ENOTCONV, PMG_ETIMEOUT, PMG_ESTATE = (
    -1, -2, -3, -4, -5, -6, -7, -8)
PMG_PREC_FP64, PMG_PREC_FP32, PMG_PREC_BF16R = 0, 1, 2
PMG_FLUX_FP64, PMG_FLUX_DW_SMOOTH, PMG_FLUX_DW = 0, 1, 2
PMG_STAGE_PTC, PMG_STAGE_NK = 0, 1
PMG_NK_PC_BLOCK, PMG_NK_PC_VCYCLE = 0, 1


class PmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libpmgfr status {status}: {msg}")
        self.status = status


class pmg_config(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("P", ctypes.c_int * 8),
        ("n_smooth", ctypes.c_int * 8),
        ("gamma", ctypes.c_double),
        ("Ma_inf", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("cutoff", ctypes.c_int),
        ("dtau_init", ctypes.c_double),
        ("dtau_max", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("refresh_every", ctypes.c_int),
        ("max_pseudo", ctypes.c_int),
        ("block_prec", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("p_gauge", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("res_scale", ctypes.c_double * 4),
        ("q_inf", ctypes.c_double * 4),
        ("cfl_mode", ctypes.c_int),
        ("cfl_init", ctypes.c_double),
        ("cfl_max", ctypes.c_double),
        ("esdirk_order", ctypes.c_int),
        ("refresh_always", ctypes.c_int),
        ("flux_prec", ctypes.c_int),
        ("copy_wait_s", ctypes.c_double),
        ("device_loop", ctypes.c_int),
        ("dim", ctypes.c_int),
        ("res_scale3", ctypes.c_double * 5),
        ("q_inf3", ctypes.c_double * 5),
    ]


class pmg_mesh(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int),
        ("geom_order", ctypes.c_int),
        ("nodes", ctypes.POINTER(ctypes.c_double)),
        ("nbr", ctypes.POINTER(ctypes.c_int)),
    ]


class pmg_step_stats(ctypes.Structure):
    _fields_ = [
        ("pseudo_iters", ctypes.c_int * 8),
        ("res_drop", ctypes.c_double * 8),
        ("ms_total", ctypes.c_double),
        ("n_vcycles", ctypes.c_int),
        ("n_refresh", ctypes.c_int),
    ]


class pmg_tune_report(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("fused", ctypes.c_int * 8),
        ("tile_core", ctypes.c_int * 8),
        ("tile_depth", ctypes.c_int * 8),
        ("candidates", ctypes.c_int * 8),
        ("us_per_sweep", ctypes.c_double * 8),
        ("us_per_sweep_before", ctypes.c_double * 8),
    ]


class pmg_nk_options(ctypes.Structure):
    _fields_ = [
        ("max_newton", ctypes.c_int),
        ("krylov_dim", ctypes.c_int),
        ("max_krylov", ctypes.c_int),
        ("eta", ctypes.c_double),
        ("precond", ctypes.c_int),
        ("dtau_pc", ctypes.c_double),
        ("pc_refresh", ctypes.c_int),
        ("delta0", ctypes.c_double),
        ("state_scale", ctypes.c_double * 5),
        ("max_backtrack", ctypes.c_int),
        ("max_update", ctypes.c_double),
        ("pc_eps", ctypes.c_double),
        ("ptc_dtau", ctypes.c_double),
    ]


class pmg_nk_stats(ctypes.Structure):
    _fields_ = [("newton", ctypes.c_longlong), ("krylov", ctypes.c_longlong), ("vcycles", ctypes.c_longlong),
                ("residuals", ctypes.c_longlong)]


_lib = None


def load():
    """Load libpmgfr.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpmgfr.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "pmg_create": ([ctypes.POINTER(pmg_config), vp, ctypes.POINTER(vp)], ci),
        "pmg_destroy": ([vp], None),
        "pmg_last_error": ([], ctypes.c_char_p),
        "pmg_upload_mesh": ([vp, ctypes.POINTER(pmg_mesh)], ci),
        "pmg_point_coords": ([vp, ci, pd], ci),
        "pmg_set_state": ([vp, ci, vp, ci], ci),
        "pmg_get_state": ([vp, ci, vp, ci], ci),
        "pmg_residual": ([vp, ci, vp, vp, ci], ci),
        "pmg_set_stage": ([vp, vp, cd, ci], ci),
        "pmg_stage_residual": ([vp, ci, vp, vp, ci], ci),
        "pmg_assemble_blocks": ([vp, ci, cd], ci),
        "pmg_get_blocks": ([vp, ci, vp, ci], ci),
        "pmg_set_blocks": ([vp, ci, vp, ci], ci),
        "pmg_factor_blocks": ([vp, ci], ci),
        "pmg_apply_blocks": ([vp, ci, vp, vp, ci], ci),
        "pmg_restrict": ([vp, ci, vp, vp, ci], ci),
        "pmg_prolong": ([vp, ci, vp, vp, ci], ci),
        "pmg_vcycle": ([vp, cd, ci, pd], ci),
        "pmg_stage_solve": ([vp, ctypes.POINTER(ci), pd], ci),
        "pmg_esdirk_step": ([vp, cd, ctypes.POINTER(pmg_step_stats)], ci),
        "pmg_stage_history": ([vp, pd, pd, ci, ctypes.POINTER(ci)], ci),
        "pmg_profile": ([vp, ci], ci),
        "pmg_residual_static": ([vp, ci, vp, vp], ci),
        "pmg_autotune": ([vp, ci, ctypes.c_char_p, ctypes.POINTER(pmg_tune_report)], ci),
        "pmg_checkpoint": ([vp, ctypes.c_char_p], ci),
        "pmg_dtau_min": ([vp, ctypes.POINTER(ctypes.c_double)], ci),
        "pmg_restore": ([vp, ctypes.c_char_p], ci),
        "pmg_profile_read": ([vp, pd, ctypes.POINTER(ctypes.c_longlong)], ci),
        "pmg_set_stage_solver": ([vp, ci, ctypes.POINTER(pmg_nk_options)], ci),
        "pmg_nk_stats_read": ([vp, ctypes.POINTER(pmg_nk_stats), ci], ci),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status):
    if status != PMG_OK:
        raise PmgError(status, load().pmg_last_error().decode())


def _ptr(x, writable=False):
    """(pointer, on_device) of a NumPy array or CUDA torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float64")
        if writable and not x.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        return ctypes.c_void_p(x.ctypes.data), 0
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    raise TypeError("expected numpy.ndarray or torch.Tensor")


def make_config(P_levels, n_smooth, *, gamma=1.4, Ma_inf=0.005, kappa=1.0, cutoff=0, dtau_init=0.01,
                dtau_max=10.0, tol=1e-8, refresh_every=10, max_pseudo=2000, block_prec=PMG_PREC_FP64,
                use_graph=1, p_gauge=0.0, mu=0.0, Pr=0.72, res_scale=(1.0, 1.0, 1.0, 1.0),
                q_inf=(0.0, 0.0, 0.0, 0.0), cfl_mode=0, cfl_init=1e2, cfl_max=1e5,
                esdirk_order=3, refresh_always=0, flux_prec=PMG_FLUX_DW_SMOOTH, copy_wait_s=0.0,
                device_loop=0, dim=2, res_scale3=(1.0,) * 5, q_inf3=(0.0,) * 5) -> pmg_config:
    cfg = pmg_config()
    cfg.n_levels = len(P_levels)
    for l, (P, n) in enumerate(zip(P_levels, n_smooth)):
        cfg.P[l] = P
        cfg.n_smooth[l] = n
    cfg.gamma, cfg.Ma_inf, cfg.kappa, cfg.cutoff = gamma, Ma_inf, kappa, cutoff
    cfg.dtau_init, cfg.dtau_max, cfg.tol = dtau_init, dtau_max, tol
    cfg.refresh_every, cfg.max_pseudo = refresh_every, max_pseudo
    cfg.block_prec, cfg.use_graph = block_prec, use_graph
    cfg.p_gauge = p_gauge
    cfg.mu, cfg.Pr = mu, Pr
    for v in range(4):
        cfg.res_scale[v] = res_scale[v]
        cfg.q_inf[v] = q_inf[v]
    cfg.cfl_mode, cfg.cfl_init, cfg.cfl_max = cfl_mode, cfl_init, cfl_max
    cfg.esdirk_order = esdirk_order
    cfg.refresh_always = refresh_always
    cfg.flux_prec = flux_prec
    cfg.copy_wait_s = copy_wait_s
    cfg.device_loop = device_loop
    cfg.dim = dim
    for v in range(5):
        cfg.res_scale3[v] = res_scale3[v]
        cfg.q_inf3[v] = q_inf3[v]
    return cfg


def pmg_create(cfg: pmg_config, stream=None):
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(stream) if stream else None
    _check(load().pmg_create(ctypes.byref(cfg), s, ctypes.byref(h)))
    return h


def pmg_destroy(h):
    if h:
        load().pmg_destroy(h)


def pmg_upload_mesh(h, nodes, nbr):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    nn, dim = nodes.shape[1], nodes.shape[2]
    Ng = int(round(nn ** (1.0 / dim))) - 1
    m = pmg_mesh(nodes.shape[0], Ng, nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    _check(load().pmg_upload_mesh(h, ctypes.byref(m)))


def pmg_point_coords(h, level, E, N, dim=2):
    xy = np.zeros((E, N, dim))
    _check(load().pmg_point_coords(h, level, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return xy


def pmg_set_state(h, level, q):
    p, dev = _ptr(q)
    _check(load().pmg_set_state(h, level, p, dev))


def pmg_get_state(h, level, out):
    p, dev = _ptr(out, True)
    _check(load().pmg_get_state(h, level, p, dev))
    return out


def pmg_residual(h, level, q, out):
    pq, d1 = _ptr(q)
    pr, d2 = _ptr(out, True)
    if d1 != d2:
        raise TypeError("q and R must both be host or both device arrays")
    _check(load().pmg_residual(h, level, pq, pr, d1))
    return out


def pmg_set_stage(h, src, omega_dt):
    p, dev = _ptr(src)
    _check(load().pmg_set_stage(h, p, float(omega_dt), dev))


def pmg_stage_residual(h, level, q, out):
    pq, d1 = _ptr(q)
    pr, d2 = _ptr(out, True)
    if d1 != d2:
        raise TypeError("q and F must both be host or both device arrays")
    _check(load().pmg_stage_residual(h, level, pq, pr, d1))
    return out


def pmg_assemble_blocks(h, level, dtau):
    _check(load().pmg_assemble_blocks(h, level, float(dtau)))


def pmg_get_blocks(h, level, out):
    p, dev = _ptr(out, True)
    _check(load().pmg_get_blocks(h, level, p, dev))
    return out


def pmg_set_blocks(h, level, D):
    p, dev = _ptr(D)
    _check(load().pmg_set_blocks(h, level, p, dev))


def pmg_factor_blocks(h, level):
    _check(load().pmg_factor_blocks(h, level))


def pmg_apply_blocks(h, level, r, out):
    pr, d1 = _ptr(r)
    px, d2 = _ptr(out, True)
    if d1 != d2:
        raise TypeError("r and x must both be host or both device arrays")
    _check(load().pmg_apply_blocks(h, level, pr, px, d1))
    return out


def pmg_restrict(h, lf, qf, out):
    pa, d1 = _ptr(qf)
    pb, d2 = _ptr(out, True)
    if d1 != d2:
        raise TypeError("mixed host/device arguments")
    _check(load().pmg_restrict(h, lf, pa, pb, d1))
    return out


def pmg_prolong(h, lf, qc, out):
    pa, d1 = _ptr(qc)
    pb, d2 = _ptr(out, True)
    if d1 != d2:
        raise TypeError("mixed host/device arguments")
    _check(load().pmg_prolong(h, lf, pa, pb, d1))
    return out


def pmg_vcycle(h, dtau, refresh=True):
    nm = ctypes.c_double()
    _check(load().pmg_vcycle(h, float(dtau), int(refresh), ctypes.byref(nm)))
    return nm.value


def pmg_stage_solve(h):
    it = ctypes.c_int()
    dr = ctypes.c_double()
    _check(load().pmg_stage_solve(h, ctypes.byref(it), ctypes.byref(dr)))
    return it.value, dr.value


def pmg_esdirk_step(h, dt, raise_on_error=True):
    st = pmg_step_stats()
    status = load().pmg_esdirk_step(h, float(dt), ctypes.byref(st))
    if raise_on_error:
        _check(status)
    return st if raise_on_error else (status, st)


def pmg_stage_history(h):
    n = ctypes.c_int()
    _check(load().pmg_stage_history(h, None, None, 0, ctypes.byref(n)))
    norms = np.zeros(max(n.value, 1))
    dtau = np.zeros(max(n.value, 1))
    pd = ctypes.POINTER(ctypes.c_double)
    _check(load().pmg_stage_history(h, norms.ctypes.data_as(pd), dtau.ctypes.data_as(pd), n.value, ctypes.byref(n)))
    return norms[: n.value], dtau[: n.value]


def pmg_set_stage_solver(h, solver, *, max_newton=0, krylov_dim=0, max_krylov=0, eta=0.0,
                         precond=PMG_NK_PC_VCYCLE, dtau_pc=0.0, pc_refresh=0, delta0=0.0, state_scale=(0.0,) * 5,
                         max_backtrack=-1, max_update=0.0, pc_eps=0.0, ptc_dtau=0.0):
    """PMG_STAGE_PTC, or PMG_STAGE_NK with its options (0 / negative: the defaults)."""
    o = pmg_nk_options()
    o.max_newton, o.krylov_dim, o.max_krylov, o.eta = max_newton, krylov_dim, max_krylov, eta
    o.precond, o.dtau_pc, o.pc_refresh, o.delta0 = precond, dtau_pc, pc_refresh, delta0
    for v in range(5):
        o.state_scale[v] = state_scale[v] if v < len(state_scale) else 0.0
    o.max_backtrack = max_backtrack
    o.max_update = max_update
    o.pc_eps = pc_eps
    o.ptc_dtau = ptc_dtau
    _check(load().pmg_set_stage_solver(h, int(solver), ctypes.byref(o)))


def pmg_nk_stats_read(h, reset=False):
    st = pmg_nk_stats()
    _check(load().pmg_nk_stats_read(h, ctypes.byref(st), int(reset)))
    return dict(newton=st.newton, krylov=st.krylov, vcycles=st.vcycles, residuals=st.residuals)


class Solver:
    """Owns one context: mesh, levels and stage data (convenience wrapper)."""

    def __init__(self, nodes, nbr, P_levels, n_smooth, stream=None, **cfg_kw):
        self.cfg = make_config(P_levels, n_smooth, **cfg_kw)
        self.dim = 3 if cfg_kw.get("dim", 2) == 3 else 2
        self.nv = self.dim + 2
        self.P = list(P_levels)
        self.E = int(np.asarray(nodes).shape[0])
        self.h = None
        self.h = pmg_create(self.cfg, stream)
        pmg_upload_mesh(self.h, nodes, nbr)

    def close(self):
        if self.h is not None:
            pmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def N(self, level=0):
        return (self.P[level] + 1) ** self.dim

    def shape(self, level=0):
        return (self.nv, self.E, self.N(level))

    def n(self, level=0):
        return self.nv * self.N(level)

    def coords(self, level=0):
        return pmg_point_coords(self.h, level, self.E, self.N(level), self.dim)

    def set_state(self, q, level=0):
        pmg_set_state(self.h, level, q)

    def get_state(self, level=0):
        return pmg_get_state(self.h, level, np.zeros(self.shape(level)))

    def residual(self, q, level=0):
        return pmg_residual(self.h, level, np.ascontiguousarray(q, dtype=np.float64), np.zeros(self.shape(level)))

    def set_stage(self, src, omega_dt):
        pmg_set_stage(self.h, np.ascontiguousarray(src, dtype=np.float64), omega_dt)

    def stage_F(self, q, level=0):
        return pmg_stage_residual(self.h, level, np.ascontiguousarray(q, dtype=np.float64),
                                  np.zeros(self.shape(level)))

    def blocks(self, q, dtau, level=0):
        self.set_state(np.ascontiguousarray(q, dtype=np.float64), level)
        pmg_assemble_blocks(self.h, level, dtau)
        n = self.n(level)
        return pmg_get_blocks(self.h, level, np.zeros((self.E, n, n)))

    def factor(self, level=0):
        pmg_factor_blocks(self.h, level)

    def apply(self, r, level=0):
        return pmg_apply_blocks(self.h, level, np.ascontiguousarray(r, dtype=np.float64),
                                np.zeros(self.shape(level)))

    def restrict(self, qf, lf):
        return pmg_restrict(self.h, lf, np.ascontiguousarray(qf, dtype=np.float64), np.zeros(self.shape(lf + 1)))

    def prolong(self, qc, lf):
        return pmg_prolong(self.h, lf, np.ascontiguousarray(qc, dtype=np.float64), np.zeros(self.shape(lf)))

    def vcycle(self, q, dtau, refresh=True):
        self.set_state(np.ascontiguousarray(q, dtype=np.float64))
        nm = pmg_vcycle(self.h, dtau, refresh)
        return self.get_state(), nm

    def stage_solve(self, q):
        self.set_state(np.ascontiguousarray(q, dtype=np.float64))
        it, dr = pmg_stage_solve(self.h)
        return self.get_state(), it, dr

    def esdirk_step(self, q, dt):
        self.set_state(np.ascontiguousarray(q, dtype=np.float64))
        st = pmg_esdirk_step(self.h, dt)
        return self.get_state(), st


def pmg_last_error() -> str:
    return load().pmg_last_error().decode()


PROF_CLASSES = ["face_flux", "volume", "apply", "assemble", "factor", "restrict", "prolong", "norm", "stage",
                "fused_sweep"]


def pmg_profile(h, enable=True):
    _check(load().pmg_profile(h, int(enable)))


def pmg_profile_read(h):
    """{(class, level): (ms, launches)} of the per-launch profiler."""
    ms = np.zeros(len(PROF_CLASSES) * 8)
    cnt = np.zeros(len(PROF_CLASSES) * 8, dtype=np.int64)
    _check(load().pmg_profile_read(h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))))
    out = {}
    for k, name in enumerate(PROF_CLASSES):
        for l in range(8):
            if cnt[k * 8 + l]:
                out[(name, l)] = (float(ms[k * 8 + l]), int(cnt[k * 8 + l]))
    return out


def pmg_residual_static(h, level, q, out):
    """Allocation-free residual: q and out must be CUDA float64 tensors."""
    pq, d1 = _ptr(q)
    pr, d2 = _ptr(out, True)
    if not (d1 and d2):
        raise TypeError("pmg_residual_static takes device tensors only")
    _check(load().pmg_residual_static(h, level, pq, pr))
    return out


def pmg_autotune(h, reps=3, cache_path=None):
    """Tune the coarse-level smoothing schedule; returns a dict per tuned level."""
    rep = pmg_tune_report()
    _check(load().pmg_autotune(h, int(reps), os.fsencode(cache_path) if cache_path else None, ctypes.byref(rep)))
    out = {}
    for l in range(rep.n_levels):
        if rep.candidates[l]:
            out[l] = dict(fused=rep.fused[l], tile_core=rep.tile_core[l], tile_depth=rep.tile_depth[l],
                          candidates=rep.candidates[l], us_per_sweep=rep.us_per_sweep[l],
                          us_per_sweep_before=rep.us_per_sweep_before[l])
    return out


def pmg_checkpoint(h, path):
    _check(load().pmg_checkpoint(h, os.fsencode(path)))


def pmg_restore(h, path):
    _check(load().pmg_restore(h, os.fsencode(path)))


def pmg_dtau_min(h):
    out = ctypes.c_double()
    _check(load().pmg_dtau_min(h, ctypes.byref(out)))
    return out.value
