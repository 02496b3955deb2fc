"""FP64 CPU oracle of the implicit P-multigrid FR solver -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``pmg_oracle.cpp`` (plain C++,
FP64, no shared code with the CUDA library) through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmg_oracle.cpp")
_LIB = os.path.join(_HERE, f"liboracle.{platform.machine()}.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no architecture-specific flags), with
    OpenMP element loops where the compiler offers it.  The loops run on one
    thread unless set_threads asks for more; results do not depend on it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        base = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
        _lib.orc_set_threads(1)
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's element loops; returns the number in use
    (1 when the library was built without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("P", ctypes.c_int * 8),
        ("n_smooth", ctypes.c_int * 8),
        ("gamma", ctypes.c_double),
        ("Ma_inf", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("cutoff", ctypes.c_int),
        ("esdirk_stages", ctypes.c_int),
        ("dtau_init", ctypes.c_double),
        ("dtau_max", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("refresh_every", ctypes.c_int),
        ("max_pseudo", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("res_scale", ctypes.c_double * 4),
        ("q_inf", ctypes.c_double * 4),
        ("cfl_mode", ctypes.c_int),
        ("cfl_init", ctypes.c_double),
        ("cfl_max", ctypes.c_double),
        ("refresh_always", ctypes.c_int),
    ]


def _declare(L):
    vp = ctypes.c_void_p
    ci, cd = ctypes.c_int, ctypes.c_double
    L.orc_basis.argtypes = [ci, _d, _d, _d, _d, _d, _d, _d]
    L.orc_transfer.argtypes = [ci, ci, _d, _d]
    L.orc_esdirk3.argtypes = [_d, _d, _d]
    L.orc_point_matrices.argtypes = [_d, cd, cd, cd, ci, _d, _d, _d]
    L.orc_flux.argtypes = [_d, cd, cd, cd, _d, _d]
    L.orc_flux_cs.argtypes = [_d, cd, cd, cd, _d]
    L.orc_roe.argtypes = [_d, _d, cd, cd, cd, cd, cd, ci, _d]
    L.orc_cons_from_prim.argtypes = [_d, cd, _d]
    L.orc_prim_from_cons.argtypes = [_d, cd, _d]
    L.orc_esdirk.argtypes = [ci, _d, _d, _d]
    L.orc_element_dx.argtypes = [vp, _d]
    L.orc_dtau_min.argtypes = [vp, _d]
    L.orc_dtau_min.restype = cd
    L.orc_create.argtypes = [ctypes.POINTER(OrcConfig), ci, ci, _d, _i]
    L.orc_create.restype = vp
    L.orc_destroy.argtypes = [vp]
    L.orc_metrics.argtypes = [vp, ci, _d, _d]
    L.orc_coords.argtypes = [vp, ci, _d]
    L.orc_residual.argtypes = [vp, ci, _d, _d]
    L.orc_set_stage.argtypes = [vp, _d, cd]
    L.orc_stage_F.argtypes = [vp, ci, _d, _d]
    L.orc_blocks.argtypes = [vp, ci, _d, cd, _d]
    L.orc_lu_solve.argtypes = [ci, _d, _d, _d]
    L.orc_restrict.argtypes = [vp, ci, _d, _d]
    L.orc_prolong.argtypes = [vp, ci, _d, _d]
    L.orc_vcycle.argtypes = [vp, _d, cd, ci]
    L.orc_stage_solve.argtypes = [vp, _d, _i, _d, _d, ci]
    L.orc_esdirk_step.argtypes = [vp, _d, cd, _i, _d]
    L.orc_ser_schedule.argtypes = [_d, ci, cd, cd, ci, _d, _i]
    L.orc_set_threads.argtypes = [ci]
    L.orc_set_threads.restype = ci


def _p(a):
    return a.ctypes.data_as(_d)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def basis(P: int):
    n = P + 1
    x, w, lm, lp, gL, gR = (np.zeros(n) for _ in range(6))
    D = np.zeros((n, n))
    lib().orc_basis(P, _p(x), _p(w), _p(D), _p(lm), _p(lp), _p(gL), _p(gR))
    return dict(x=x, w=w, D=D, lm=lm, lp=lp, gL=gL, gR=gR)


def transfer(Pf: int, Pc: int):
    R = np.zeros((Pc + 1, Pf + 1))
    I = np.zeros((Pf + 1, Pc + 1))
    lib().orc_transfer(Pf, Pc, _p(R), _p(I))
    return R, I


def esdirk(order):
    """ESDIRK tableau of the given order (2, 3 or 4): A (s x s), b, c."""
    stages = {2: 3, 3: 4, 4: 6}[order]
    A = np.zeros(stages * stages); b = np.zeros(stages); c = np.zeros(stages)
    s = lib().orc_esdirk(stages, _p(A), _p(b), _p(c))
    return A.reshape(s, s), b, c


def esdirk3():
    A = np.zeros((4, 4)); b = np.zeros(4); c = np.zeros(4)
    lib().orc_esdirk3(_p(A), _p(b), _p(c))
    return A, b, c


def point_matrices(q, gamma=1.4, Ma_inf=0.005, kappa=1.0, cutoff=0):
    q = _f64(q); M = np.zeros((4, 4)); G = np.zeros((4, 4)); eps = ctypes.c_double()
    lib().orc_point_matrices(_p(q), gamma, Ma_inf, kappa, cutoff, _p(M), _p(G), ctypes.byref(eps))
    return M, G, eps.value


def flux(q, nx, ny, gamma=1.4):
    q = _f64(q); f = np.zeros(4); A = np.zeros((4, 4))
    lib().orc_flux(_p(q), nx, ny, gamma, _p(f), _p(A))
    return f, A


def flux_jacobian_cs(q, nx, ny, gamma=1.4):
    q = _f64(q); A = np.zeros((4, 4))
    lib().orc_flux_cs(_p(q), nx, ny, gamma, _p(A))
    return A


def roe(qm, qp, Sx, Sy, gamma=1.4, Ma_inf=0.005, kappa=1.0, cutoff=0):
    qm = _f64(qm); qp = _f64(qp); out = np.zeros(4)
    lib().orc_roe(_p(qm), _p(qp), Sx, Sy, gamma, Ma_inf, kappa, cutoff, _p(out))
    return out


def cons_from_prim(q, gamma=1.4):
    q = _f64(q); qc = np.zeros(4)
    lib().orc_cons_from_prim(_p(q), gamma, _p(qc))
    return qc


def prim_from_cons(qc, gamma=1.4):
    qc = _f64(qc); q = np.zeros(4)
    lib().orc_prim_from_cons(_p(qc), gamma, _p(q))
    return q


class Oracle:
    """Stateful oracle solver on one mesh (levels, stage data, smoother)."""

    def __init__(self, nodes, nbr, Ng, P_levels, n_smooth, *, gamma=1.4, Ma_inf=0.005,
                 kappa=1.0, cutoff=0, dtau_init=0.01, dtau_max=10.0, tol=1e-8,
                 refresh_every=10, max_pseudo=2000, mu=0.0, Pr=0.72, res_scale=(1.0, 1.0, 1.0, 1.0),
                 q_inf=(0.0, 0.0, 0.0, 0.0), cfl_mode=0, cfl_init=1e2, cfl_max=1e5, esdirk_order=3,
                 refresh_always=0):
        cfg = OrcConfig()
        cfg.n_levels = len(P_levels)
        for l, P in enumerate(P_levels):
            cfg.P[l] = P
            cfg.n_smooth[l] = n_smooth[l]
        cfg.gamma, cfg.Ma_inf, cfg.kappa, cfg.cutoff = gamma, Ma_inf, kappa, cutoff
        cfg.esdirk_stages = {2: 3, 3: 4, 4: 6}[esdirk_order]
        cfg.dtau_init, cfg.dtau_max, cfg.tol = dtau_init, dtau_max, tol
        cfg.refresh_every, cfg.max_pseudo = refresh_every, max_pseudo
        cfg.mu, cfg.Pr = mu, Pr
        for v in range(4):
            cfg.res_scale[v] = res_scale[v]
            cfg.q_inf[v] = q_inf[v]
        cfg.cfl_mode, cfg.cfl_init, cfg.cfl_max = cfl_mode, cfl_init, cfl_max
        cfg.refresh_always = refresh_always
        self.cfg = cfg
        self.nodes = _f64(nodes)
        self.nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        self.E = self.nodes.shape[0]
        self.Ng = Ng
        self.P = list(P_levels)
        self.h = lib().orc_create(ctypes.byref(cfg), self.E, Ng, _p(self.nodes),
                                  self.nbr.ctypes.data_as(_i))
        if not self.h:
            raise ValueError("invalid neighbour table (or a slip wall with mu > 0, "
                             "or a no-slip wall without the eps cut-off)")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def N(self, level=0):
        return (self.P[level] + 1) ** 2

    def shape(self, level=0):
        return (4, self.E, self.N(level))

    def element_dx(self):
        dx = np.zeros(self.E)
        lib().orc_element_dx(self.h, _p(dx))
        return dx

    def dtau_min(self, q):
        return lib().orc_dtau_min(self.h, _p(_f64(q)))

    def coords(self, level=0):
        xy = np.zeros((self.E, self.N(level), 2))
        lib().orc_coords(self.h, level, _p(xy))
        return xy

    def metrics(self, level=0):
        n1 = self.P[level] + 1
        met = np.zeros((self.E, self.N(level), 5))
        fS = np.zeros((self.E, 4, n1, 2))
        lib().orc_metrics(self.h, level, _p(met), _p(fS))
        return met, fS

    def residual(self, q, level=0):
        q = _f64(q); R = np.zeros(self.shape(level))
        lib().orc_residual(self.h, level, _p(q), _p(R))
        return R

    def set_stage(self, src, omega_dt):
        self._src = _f64(src)
        lib().orc_set_stage(self.h, _p(self._src), omega_dt)

    def stage_F(self, q, level=0):
        q = _f64(q); F = np.zeros(self.shape(level))
        lib().orc_stage_F(self.h, level, _p(q), _p(F))
        return F

    def blocks(self, q, dtau, level=0):
        q = _f64(q); n = 4 * self.N(level)
        D = np.zeros((self.E, n, n))
        lib().orc_blocks(self.h, level, _p(q), dtau, _p(D))
        return D

    def restrict(self, qf, lf):
        qf = _f64(qf); qc = np.zeros(self.shape(lf + 1))
        lib().orc_restrict(self.h, lf, _p(qf), _p(qc))
        return qc

    def prolong(self, qc, lf):
        qc = _f64(qc); qf = np.zeros(self.shape(lf))
        lib().orc_prolong(self.h, lf, _p(qc), _p(qf))
        return qf

    def vcycle(self, q, dtau, refresh=True):
        q = _f64(q).copy()
        st = lib().orc_vcycle(self.h, _p(q), dtau, int(refresh))
        if st:
            raise RuntimeError(f"oracle vcycle status {st}")
        return q

    def stage_solve(self, q, max_norms=4096):
        q = _f64(q).copy()
        it = ctypes.c_int(); drop = ctypes.c_double(); norms = np.zeros(max_norms)
        st = lib().orc_stage_solve(self.h, _p(q), ctypes.byref(it), ctypes.byref(drop), _p(norms), max_norms)
        return q, it.value, drop.value, norms[: it.value + 1], st

    def esdirk_step(self, q, dt):
        q = _f64(q).copy()
        its = (ctypes.c_int * 8)(); drops = np.zeros(8)
        st = lib().orc_esdirk_step(self.h, _p(q), dt, its, _p(drops))
        if st:
            raise RuntimeError(f"oracle esdirk step status {st}")
        return q, list(its)[:3], drops[:3]


def ser_schedule(norms, dtau_init, dtau_max, k):
    norms = _f64(norms); n = len(norms)
    dt = np.zeros(n); rf = np.zeros(n, dtype=np.int32)
    lib().orc_ser_schedule(_p(norms), n, dtau_init, dtau_max, k, _p(dt), rf.ctypes.data_as(_i))
    return dt, rf.astype(bool)


def lu_solve(A, b):
    A = _f64(A); b = _f64(b); x = np.zeros_like(b)
    st = lib().orc_lu_solve(A.shape[0], _p(A), _p(b), _p(x))
    if st:
        raise RuntimeError("singular")
    return x


# ---------------------------------------------------------------------------
# Three dimensions: hexahedra, 5 working variables (p, u, v, w, T).
# ---------------------------------------------------------------------------
class OrcConfig3(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("P", ctypes.c_int * 8),
        ("n_smooth", ctypes.c_int * 8),
        ("gamma", ctypes.c_double),
        ("Ma_inf", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("cutoff", ctypes.c_int),
        ("esdirk_stages", ctypes.c_int),
        ("dtau_init", ctypes.c_double),
        ("dtau_max", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("refresh_every", ctypes.c_int),
        ("max_pseudo", ctypes.c_int),
        ("res_scale", ctypes.c_double * 5),
        ("q_inf", ctypes.c_double * 5),
        ("refresh_always", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
    ]


_declared3 = False


def _lib3():
    global _declared3
    L = lib()
    if not _declared3:
        vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.orc3_gll.argtypes = [ci, _d]
        L.orc3_point_matrices.argtypes = [_d, cd, cd, cd, ci, _d, _d, _d]
        L.orc3_flux.argtypes = [_d, _d, cd, _d, _d]
        L.orc3_roe.argtypes = [_d, _d, _d, cd, cd, cd, ci, _d]
        L.orc3_cons_from_prim.argtypes = [_d, cd, _d]
        L.orc3_create.argtypes = [ctypes.POINTER(OrcConfig3), ci, ci, _d, _i]
        L.orc3_create.restype = vp
        L.orc3_destroy.argtypes = [vp]
        L.orc3_geometry.argtypes = [vp, ci, _d, _d, _d, _d]
        L.orc3_residual.argtypes = [vp, ci, _d, _d]
        L.orc3_set_stage.argtypes = [vp, _d, cd]
        L.orc3_stage_F.argtypes = [vp, ci, _d, _d]
        L.orc3_blocks.argtypes = [vp, ci, _d, cd, _d]
        L.orc3_restrict.argtypes = [vp, ci, _d, _d]
        L.orc3_prolong.argtypes = [vp, ci, _d, _d]
        L.orc3_vcycle.argtypes = [vp, _d, cd, ci]
        L.orc3_stage_solve.argtypes = [vp, _d, _i, _d]
        L.orc3_esdirk_step.argtypes = [vp, _d, cd, _i, _d]
        _declared3 = True
    return L


def gll(n: int):
    """Gauss-Lobatto points of degree n (n + 1 points)."""
    x = np.zeros(n + 1)
    _lib3().orc3_gll(n, _p(x))
    return x


def point_matrices3(q, gamma=1.4, Ma_inf=0.005, kappa=1.0, cutoff=0):
    q = _f64(q); M = np.zeros((5, 5)); G = np.zeros((5, 5)); eps = ctypes.c_double()
    _lib3().orc3_point_matrices(_p(q), gamma, Ma_inf, kappa, cutoff, _p(M), _p(G), ctypes.byref(eps))
    return M, G, eps.value


def flux3(q, n, gamma=1.4):
    q = _f64(q); n = _f64(n); f = np.zeros(5); A = np.zeros((5, 5))
    _lib3().orc3_flux(_p(q), _p(n), gamma, _p(f), _p(A))
    return f, A


def roe3(qm, qp, S, gamma=1.4, Ma_inf=0.005, kappa=1.0, cutoff=0):
    qm = _f64(qm); qp = _f64(qp); S = _f64(S); out = np.zeros(5)
    _lib3().orc3_roe(_p(qm), _p(qp), _p(S), gamma, Ma_inf, kappa, cutoff, _p(out))
    return out


def cons_from_prim3(q, gamma=1.4):
    q = _f64(q); qc = np.zeros(5)
    _lib3().orc3_cons_from_prim(_p(q), gamma, _p(qc))
    return qc


class Oracle3:
    """Stateful 3D oracle solver on one hexahedral mesh."""

    def __init__(self, nodes, nbr, Ng, P_levels, n_smooth, *, gamma=1.4, Ma_inf=0.005, kappa=1.0, cutoff=0,
                 dtau_init=0.01, dtau_max=10.0, tol=1e-8, refresh_every=10, max_pseudo=2000,
                 res_scale=(1.0,) * 5, q_inf=(0.0,) * 5, esdirk_order=3, refresh_always=0, mu=0.0, Pr=0.72):
        cfg = OrcConfig3()
        cfg.n_levels = len(P_levels)
        for l, P in enumerate(P_levels):
            cfg.P[l] = P
            cfg.n_smooth[l] = n_smooth[l]
        cfg.gamma, cfg.Ma_inf, cfg.kappa, cfg.cutoff = gamma, Ma_inf, kappa, cutoff
        cfg.esdirk_stages = {2: 3, 3: 4, 4: 6}[esdirk_order]
        cfg.dtau_init, cfg.dtau_max, cfg.tol = dtau_init, dtau_max, tol
        cfg.refresh_every, cfg.max_pseudo = refresh_every, max_pseudo
        for v in range(5):
            cfg.res_scale[v] = res_scale[v]
            cfg.q_inf[v] = q_inf[v]
        cfg.refresh_always = refresh_always
        cfg.mu, cfg.Pr = mu, Pr
        self.cfg = cfg
        self.nodes = _f64(nodes)
        self.nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        self.E = self.nodes.shape[0]
        self.Ng = Ng
        self.P = list(P_levels)
        self.h = _lib3().orc3_create(ctypes.byref(cfg), self.E, Ng, _p(self.nodes), self.nbr.ctypes.data_as(_i))
        if not self.h:
            raise ValueError("invalid neighbour table (or a slip wall with mu > 0, "
                             "or a no-slip wall without the eps cut-off)")

    def __del__(self):
        try:
            if self.h:
                _lib3().orc3_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def N(self, level=0):
        return (self.P[level] + 1) ** 3

    def shape(self, level=0):
        return (5, self.E, self.N(level))

    def geometry(self, level=0):
        """(Ja (E, N, 3, 3), J (E, N), face normals (E, 6, NF, 3), coordinates (E, N, 3))."""
        N, NF = self.N(level), (self.P[level] + 1) ** 2
        Ja = np.zeros((self.E, N, 3, 3)); J = np.zeros((self.E, N))
        fS = np.zeros((self.E, 6, NF, 3)); xyz = np.zeros((self.E, N, 3))
        _lib3().orc3_geometry(self.h, level, _p(Ja), _p(J), _p(fS), _p(xyz))
        return Ja, J, fS, xyz

    def coords(self, level=0):
        return self.geometry(level)[3]

    def residual(self, q, level=0):
        q = _f64(q); R = np.zeros(self.shape(level))
        _lib3().orc3_residual(self.h, level, _p(q), _p(R))
        return R

    def set_stage(self, src, omega_dt):
        src = _f64(src)
        _lib3().orc3_set_stage(self.h, _p(src), omega_dt)

    def stage_F(self, q, level=0):
        q = _f64(q); F = np.zeros(self.shape(level))
        _lib3().orc3_stage_F(self.h, level, _p(q), _p(F))
        return F

    def blocks(self, q, dtau, level=0):
        q = _f64(q); n = 5 * self.N(level)
        D = np.zeros((self.E, n, n))
        _lib3().orc3_blocks(self.h, level, _p(q), dtau, _p(D))
        return D

    def restrict(self, qf, lf):
        qf = _f64(qf); qc = np.zeros(self.shape(lf + 1))
        _lib3().orc3_restrict(self.h, lf, _p(qf), _p(qc))
        return qc

    def prolong(self, qc, lf):
        qc = _f64(qc); qf = np.zeros(self.shape(lf))
        _lib3().orc3_prolong(self.h, lf, _p(qc), _p(qf))
        return qf

    def vcycle(self, q, dtau, refresh=True):
        q = _f64(q).copy()
        st = _lib3().orc3_vcycle(self.h, _p(q), dtau, int(refresh))
        if st:
            raise RuntimeError(f"oracle V-cycle failed ({st})")
        return q

    def stage_solve(self, q):
        q = _f64(q).copy(); it = ctypes.c_int(); dr = ctypes.c_double()
        st = _lib3().orc3_stage_solve(self.h, _p(q), ctypes.byref(it), ctypes.byref(dr))
        return q, it.value, dr.value, st

    def esdirk_step(self, q, dt):
        q = _f64(q).copy(); its = np.zeros(6, dtype=np.int32); drops = np.zeros(6)
        st = _lib3().orc3_esdirk_step(self.h, _p(q), dt, its.ctypes.data_as(_i), _p(drops))
        if st:
            raise RuntimeError(f"oracle step failed ({st})")
        return q, its, drops
