"""Newton-Krylov solve of one implicit stage -- TEST INFRASTRUCTURE (oracle).

Only the tests may import this module.  It is plain numpy on top of the FP64
oracle (``oracle.Oracle``): the stage residual F, the element blocks and the
FAS V-cycle come from ``pmg_oracle.cpp``; nothing here is shared with the CUDA
library.

The paper solves each implicit stage (Section 2.4) by pseudo-transient
continuation with a P-multigrid V-cycle (Section 3).  Its introduction
describes the matrix-free Newton-Krylov alternative, in which the Krylov
method needs the Jacobian only as a product with a vector, approximated by a
difference of residuals (Knoll & Keyes, J. Comput. Phys. 193, 2004), and its
concluding section names Newton-Krylov with the P-multigrid method as the
preconditioner as future work.  This module writes that variant out:

- Newton on the stage system F(q) = R(q) - q_c(q)/(omega dt) + src = 0
  (F as the oracle's stage_F; the element-Jacobi smoother of eq.
  smoothing_element_jacobi updates q += D^-1 F, so D approximates
  A = -dF/dq): solve A delta = F(q) inexactly, then q <- q + lam delta with
  lam starting at min(1, max_update / r), r the largest relative change
  |dp|/p, |dT|/T of any point under the full step, and halved until ||F||_W
  falls by the factor (1 - 1e-4 lam) (at most max_backtrack halvings; the
  last trial is taken regardless).
- Pseudo-transient Newton (ptc_dtau > 0; Kelley & Keyes, SIAM J. Numer.
  Anal. 35, 1998): every Newton step is the backward-Euler step of the
  paper's pseudo-time system Gamma dq/dtau = F (Section 2.4, eq.
  preconditioning), linearised: (Gamma(q)/dtau + A) delta = F(q), Gamma
  pointwise at q.  dtau starts at ptc_dtau and follows the SER rule of eq.
  ser with exponent 1.5 and no upper bound, dtau <- dtau (||F_old|| /
  ||F_new||)^1.5; the step lam delta takes lam from the max_update limit
  alone (no backtracking: a step that raises ||F|| shrinks dtau instead).  The
  preconditioners take dtau_pc' = min(dtau, dtau_pc): the element blocks are
  then the block diagonal of Gamma/dtau + A itself.
- ||.||_W: each equation divided by its residual scale (the stage norm of the
  pseudo-transient solver).
- Krylov: restarted FGMRES(m), right-preconditioned (Saad, SIAM J. Sci.
  Comput. 14, 1993), in the W-weighted space, with classical Gram-Schmidt
  done twice and the small least-squares problem solved by numpy; it stops
  when the weighted linear residual is at most eta times its initial value,
  or after max_krylov iterations.
- A z = -(F(q + h z) - F(q)) / h with h = delta0 / rms(z / s), s the state
  scales (p, u, v, T).
- Preconditioners (z = M^-1 r for r in the F space):
  * "block": element-block Jacobi, z = D^-1 r with the finest level's blocks
    D at q and dtau_pc (Section 2.4: Gamma/dtau + M/(omega dt) - dR_e/dq_e);
  * "vcycle": one FAS V-cycle (Section 3) on G(q') = F(q') - F(q) + eps r
    from q' = q, i.e. the stage system with source src - F(q) + eps r, and
    z = (q' - q) / eps with eps = pc_eps ||F(q)||_W (pc_eps = 0.1: the
    V-cycle sees a tenth of the Newton defect, within its linear range); the
    blocks of every level are rebuilt in
    the first application of each Newton step whose index is a multiple of
    pc_refresh.
"""
from __future__ import annotations

import numpy as np


def wnorm(F, W):
    """sqrt(sum_v sum (F_v / scale_v)^2), W = 1 / scale."""
    return float(np.sqrt(sum(((F[v] * W[v]) ** 2).sum() for v in range(F.shape[0]))))


def gamma_field(orc, q):
    """Gamma of eq. preconditioning at every point of q (nv, E, N), as an
    (E, N, nv, nv) array, from the oracle's point matrices (absolute pressure)
    with the oracle's gamma, Mach number and cut-off."""
    import oracle as O
    nv, E, N = q.shape
    pm = O.point_matrices if nv == 4 else O.point_matrices3
    cf = orc.cfg
    G = np.empty((E, N, nv, nv))
    for e in range(E):
        for i in range(N):
            G[e, i] = pm(q[:, e, i], gamma=cf.gamma, Ma_inf=cf.Ma_inf, kappa=cf.kappa, cutoff=cf.cutoff)[1]
    return G


def fgmres(apply_A, apply_M, b, m, max_it, rtol):
    """Right-preconditioned restarted FGMRES(m) for A x = b from x = 0.

    apply_A(z) -> A z and apply_M(v) -> z (the preconditioned direction) act on
    flat vectors.  Returns (x, iterations, final residual norm, initial norm)."""
    x = np.zeros_like(b)
    beta0 = float(np.linalg.norm(b))
    target = rtol * beta0
    it = 0
    res = beta0
    r = b.copy()
    while it < max_it and res > target:
        beta = float(np.linalg.norm(r))
        if beta == 0.0:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        y = np.zeros(0)
        for j in range(m):
            z = apply_M(V[j])
            Z.append(z)
            w = apply_A(z)
            h = np.array([V[i] @ w for i in range(j + 1)])
            w = w - sum(h[i] * V[i] for i in range(j + 1))
            h2 = np.array([V[i] @ w for i in range(j + 1)])
            w = w - sum(h2[i] * V[i] for i in range(j + 1))
            H[: j + 1, j] = h + h2
            H[j + 1, j] = float(np.linalg.norm(w))
            it += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
            res = float(np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y))
            if H[j + 1, j] == 0.0 or res <= target or it >= max_it:
                break
            V.append(w / H[j + 1, j])
        x = x + sum(y[i] * Z[i] for i in range(len(y)))
        if res > target and it < max_it:
            r = b - apply_A(x)
    return x, it, res, beta0


def nk_stage_solve(orc, q, src, odt, W, s, *, tol=1e-8, max_newton=30, m=20, max_krylov=40, eta=1e-2,
                   precond="vcycle", dtau_pc=10.0, pc_refresh=1, delta0=1e-7, max_backtrack=6, norm0=None,
                   pc_eps=0.1, max_update=0.2, ptc_dtau=0.0):
    """Newton-Krylov solve of the stage system with source src and omega dt =
    odt on the oracle `orc`, from q.  W: 1 / residual scale per equation; s:
    state scale per variable.  Stops when ||F||_W <= tol * ||F(q_start)||_W
    (or tol * norm0 if given).  Returns dict(q, newton, krylov, vcycles,
    residuals, norms, dtaus, step, status): dtaus the pseudo-time step of each
    Newton step (ptc_dtau > 0), step the last accepted lam delta, status 0
    converged, 1 not converged within max_newton, 2 non-finite."""
    W = np.asarray(W, dtype=float)
    s = np.asarray(s, dtype=float)
    shape = q.shape
    nv = shape[0]
    Wb = W.reshape(nv, 1, 1)
    sb = s.reshape(nv, 1, 1)
    q = np.array(q, dtype=float, copy=True)
    orc.set_stage(src, odt)
    F = orc.stage_F(q)
    n_res = 1
    nrm = wnorm(F, W)
    n0 = nrm if norm0 is None else norm0
    norms = [nrm]
    stats = dict(newton=0, krylov=0, vcycles=0, step=None)
    D = None
    ptc = ptc_dtau > 0.0
    dtau = ptc_dtau
    dtaus = []
    for k in range(max_newton):
        if nrm <= tol * n0 or n0 == 0.0:
            return dict(q=q, residuals=n_res, norms=norms, status=0, dtaus=dtaus, **stats)
        eps = pc_eps * nrm
        refresh = [k % pc_refresh == 0]
        dpc = min(dtau, dtau_pc) if ptc else dtau_pc
        if precond == "block" and refresh[0]:
            D = orc.blocks(q, dpc)
        G = gamma_field(orc, q) if ptc else None
        dtaus.append(dtau)

        def apply_A(z, q=q, F=F):
            nonlocal n_res
            zz = z.reshape(shape)
            rms = float(np.sqrt(np.mean((zz / sb) ** 2)))
            if rms == 0.0:
                return np.zeros_like(z)
            h = delta0 / rms
            Fh = orc.stage_F(q + h * zz)
            n_res += 1
            Az = -(Fh - F) / h
            if ptc:
                Az = Az + np.einsum("enij,jen->ien", G, zz) / dtau
            return (Az * Wb).reshape(-1)

        def apply_M(v, q=q, F=F):
            r = v.reshape(shape) / Wb
            if precond == "block":
                E, N = shape[1], shape[2]
                z = np.empty(shape)
                for e in range(E):
                    x = np.linalg.solve(D[e], r[:, e, :].reshape(-1))
                    z[:, e, :] = x.reshape(nv, N)
                return z.reshape(-1)
            orc.set_stage(src - F + eps * r, odt)
            qp = orc.vcycle(q, dpc, refresh=refresh[0])
            refresh[0] = False
            orc.set_stage(src, odt)
            stats["vcycles"] += 1
            return ((qp - q) / eps).reshape(-1)

        b = (F * Wb).reshape(-1)
        delta, its, _, _ = fgmres(apply_A, apply_M, b, m, max_krylov, eta)
        stats["krylov"] += its
        stats["newton"] += 1
        delta = delta.reshape(shape)
        # the largest relative change of p (absolute) and T under the full step
        rel = max(float(np.max(np.abs(delta[0]) / np.abs(q[0]))), float(np.max(np.abs(delta[-1]) / np.abs(q[-1]))))
        lam = max_update / rel if rel > max_update else 1.0
        for t in range(0 if ptc else max_backtrack + 1):
            qn = q + lam * delta
            Fn = orc.stage_F(qn)
            n_res += 1
            nn = wnorm(Fn, W)
            if np.isfinite(nn) and nn <= (1.0 - 1e-4 * lam) * nrm:
                break
            if t < max_backtrack:
                lam *= 0.5
        if ptc:
            qn = q + lam * delta
            Fn = orc.stage_F(qn)
            n_res += 1
            nn = wnorm(Fn, W)
        if not np.isfinite(nn):
            return dict(q=qn, residuals=n_res, norms=norms + [nn], status=2, dtaus=dtaus, **stats)
        if ptc:
            dtau = dtau * (nrm / nn) ** 1.5
        stats["step"] = lam * delta
        q, F, nrm = qn, Fn, nn
        norms.append(nrm)
    status = 0 if nrm <= tol * n0 else 1
    return dict(q=q, residuals=n_res, norms=norms, status=status, dtaus=dtaus, **stats)
