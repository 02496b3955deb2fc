"""Seeded synthetic inputs: meshes and initial states.

This module holds no arithmetic of the solver.  It builds the geometry and
connectivity arrays that the library (and the test oracle) take as input, and
evaluates analytic flow fields at point coordinates supplied by the caller.

Mesh conventions (the library's C interface documents the same layout):

* ``nodes``: float64 ``(E, (Ng+1)**2, 2)``: Lagrange geometry nodes of each
  element at equispaced reference positions, node index ``b*(Ng+1)+a`` with
  ``a`` along the first reference direction xi.
* ``nbr``: int32 ``(E, 4, 3)``: for each local face (0: eta=-1, 1: xi=+1,
  2: eta=+1, 3: xi=-1) the neighbour element, its local face and a flag that
  is 1 when the two faces number their points in opposite order.  A boundary
  face has neighbour element -1 and its boundary type in the second slot
  (``BC_SLIP_WALL``, ``BC_NOSLIP_WALL`` adiabatic, ``BC_FARFIELD``).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4
BC_SLIP_WALL, BC_NOSLIP_WALL, BC_FARFIELD = 2, 3, 4


def periodic_box(nx: int, ny: int, x0: float = 0.0, x1: float = 10.0,
                 y0: float = 0.0, y1: float = 10.0, Ng: int = 1,
                 perturb: float = 0.0, seed: int = 1234):
    """Doubly periodic ``nx`` x ``ny`` quadrilateral mesh of a rectangle.

    With ``perturb > 0`` every node is moved by a smooth periodic displacement
    made of a few seeded Fourier modes, so that ``Ng >= 2`` elements are
    genuinely curved while periodic faces still match.  Element ``e = jy*nx+ix``.
    """
    Lx, Ly = x1 - x0, y1 - y0
    rng = np.random.default_rng(seed)
    modes = []
    if perturb > 0.0:
        for _ in range(3):
            kx, ky = rng.integers(1, 3, size=2)
            ax, ay = rng.uniform(-1.0, 1.0, size=2)
            ph = rng.uniform(0.0, 2 * math.pi, size=2)
            modes.append((kx, ky, ax, ay, ph))
    hx, hy = Lx / nx, Ly / ny

    def disp(X, Y):
        dx = np.zeros_like(X)
        dy = np.zeros_like(Y)
        for kx, ky, ax, ay, ph in modes:
            arg = 2 * math.pi * (kx * (X - x0) / Lx + ky * (Y - y0) / Ly)
            dx += ax * np.sin(arg + ph[0])
            dy += ay * np.sin(arg + ph[1])
        scale = perturb * min(hx, hy) / max(1, len(modes))
        return dx * scale, dy * scale

    r = np.linspace(0.0, 1.0, Ng + 1)
    E = nx * ny
    nodes = np.zeros((E, (Ng + 1) ** 2, 2))
    for jy in range(ny):
        for ix in range(nx):
            e = jy * nx + ix
            A, B = np.meshgrid(r, r, indexing="xy")   # A along xi (columns)
            X = x0 + (ix + A) * hx
            Y = y0 + (jy + B) * hy
            dX, dY = disp(X, Y)
            nodes[e, :, 0] = (X + dX).reshape(-1)
            nodes[e, :, 1] = (Y + dY).reshape(-1)
    nbr = np.zeros((E, 4, 3), dtype=np.int32)
    for jy in range(ny):
        for ix in range(nx):
            e = jy * nx + ix
            nbr[e, 0] = (((jy - 1) % ny) * nx + ix, 2, 0)
            nbr[e, 1] = (jy * nx + (ix + 1) % nx, 3, 0)
            nbr[e, 2] = (((jy + 1) % ny) * nx + ix, 0, 0)
            nbr[e, 3] = (jy * nx + (ix - 1) % nx, 1, 0)
    return nodes, nbr


def channel(nx: int, ny: int, x0: float = 0.0, x1: float = 10.0, y0: float = 0.0, y1: float = 2.0,
            Ng: int = 1, perturb: float = 0.0, seed: int = 1234,
            bottom: int = BC_NOSLIP_WALL, top: int = BC_NOSLIP_WALL):
    """``nx`` x ``ny`` quadrilaterals of a rectangle, periodic in x, with
    boundary faces of type ``bottom`` at y0 and ``top`` at y1.

    With ``perturb > 0`` interior nodes move by seeded smooth modes that are
    periodic in x and vanish in y at both walls, so the walls stay straight.
    """
    Lx, Ly = x1 - x0, y1 - y0
    rng = np.random.default_rng(seed)
    modes = []
    if perturb > 0.0:
        for _ in range(3):
            kx = int(rng.integers(1, 3))
            ax, ay = rng.uniform(-1.0, 1.0, size=2)
            ph = rng.uniform(0.0, 2 * math.pi, size=2)
            modes.append((kx, ax, ay, ph))
    hx, hy = Lx / nx, Ly / ny
    r = np.linspace(0.0, 1.0, Ng + 1)
    E = nx * ny
    nodes = np.zeros((E, (Ng + 1) ** 2, 2))
    for jy in range(ny):
        for ix in range(nx):
            e = jy * nx + ix
            A, B = np.meshgrid(r, r, indexing="xy")
            X = x0 + (ix + A) * hx
            Y = y0 + (jy + B) * hy
            eta = (Y - y0) / Ly
            dX = np.zeros_like(X)
            dY = np.zeros_like(Y)
            for kx, ax, ay, ph in modes:
                arg = 2 * math.pi * kx * (X - x0) / Lx
                dX += ax * np.sin(arg + ph[0]) * np.sin(math.pi * eta)
                dY += ay * np.sin(arg + ph[1]) * np.sin(math.pi * eta)
            sc = perturb * min(hx, hy) / max(1, len(modes))
            nodes[e, :, 0] = (X + sc * dX).reshape(-1)
            nodes[e, :, 1] = (Y + sc * dY).reshape(-1)
    nbr = np.zeros((E, 4, 3), dtype=np.int32)
    for jy in range(ny):
        for ix in range(nx):
            e = jy * nx + ix
            nbr[e, 0] = ((jy - 1) * nx + ix, 2, 0) if jy > 0 else (-1, bottom, 0)
            nbr[e, 1] = (jy * nx + (ix + 1) % nx, 3, 0)
            nbr[e, 2] = ((jy + 1) * nx + ix, 0, 0) if jy < ny - 1 else (-1, top, 0)
            nbr[e, 3] = (jy * nx + (ix - 1) % nx, 1, 0)
    return nodes, nbr


def cylinder_omesh(n_r: int, n_theta: int, r_in: float = 0.5, r_out: float = 50.0, Ng: int = 2,
                   wall: int = BC_NOSLIP_WALL, outer: int = BC_FARFIELD):
    """O-mesh around a circular cylinder centred at the origin.

    Radii r_k = r_in (r_out/r_in)^(k/n_r), k = 0..n_r; angles 2 pi j/n_theta.
    Element e = j*n_r + i spans [r_i, r_i+1] x [theta_j, theta_j+1], xi along
    r and eta along theta; its Lagrange nodes sit at equispaced radius and
    angle, so every node lies exactly on its circle.  Faces at r_in carry
    ``wall``, faces at r_out ``outer``; the angular direction is periodic.
    """
    rk = r_in * (r_out / r_in) ** (np.arange(n_r + 1) / n_r)
    dth = 2 * math.pi / n_theta
    t = np.linspace(0.0, 1.0, Ng + 1)
    E = n_r * n_theta
    nodes = np.zeros((E, (Ng + 1) ** 2, 2))
    for j in range(n_theta):
        for i in range(n_r):
            e = j * n_r + i
            A, B = np.meshgrid(t, t, indexing="xy")   # A along xi = r, B along eta = theta
            R = rk[i] + A * (rk[i + 1] - rk[i])
            TH = (j + B) * dth
            nodes[e, :, 0] = (R * np.cos(TH)).reshape(-1)
            nodes[e, :, 1] = (R * np.sin(TH)).reshape(-1)
    nbr = np.zeros((E, 4, 3), dtype=np.int32)
    for j in range(n_theta):
        for i in range(n_r):
            e = j * n_r + i
            nbr[e, 0] = (((j - 1) % n_theta) * n_r + i, 2, 0)
            nbr[e, 1] = (j * n_r + i + 1, 3, 0) if i < n_r - 1 else (-1, outer, 0)
            nbr[e, 2] = (((j + 1) % n_theta) * n_r + i, 0, 0)
            nbr[e, 3] = (j * n_r + i - 1, 1, 0) if i > 0 else (-1, wall, 0)
    return nodes, nbr


def ellipse_omesh(n_r: int, n_theta: int, chord: float = 1.0, thickness: float = 0.1, r_out: float = 20.0,
                  Ng: int = 2, wall: int = BC_NOSLIP_WALL, outer: int = BC_FARFIELD):
    """O-mesh around an ellipse of the given chord and thickness centred at
    the origin, major axis along x, in elliptic coordinates x = c cosh(m)
    cos(t), y = c sinh(m) sin(t) (c the focal distance): the ellipse is
    m = m0 with tanh(m0) = thickness / chord, the outer boundary m1 with
    c cosh(m1) = r_out.  Element e = j*n_r + i spans [m_i, m_i+1] x
    [t_j, t_j+1] with m equispaced (radii growing geometrically away from the
    body) and t equispaced (points clustered at the leading and trailing
    edges); xi along m, eta along t.  Its Lagrange nodes sit at equispaced m
    and t, so the wall nodes lie exactly on the ellipse.  Faces at m0 carry
    ``wall``, faces at m1 ``outer``; the angular direction is periodic.
    """
    a, b = 0.5 * chord, 0.5 * thickness
    m0 = math.atanh(b / a)
    c = a / math.cosh(m0)
    m1 = math.acosh(r_out / c)
    mk = m0 + (m1 - m0) * np.arange(n_r + 1) / n_r
    dth = 2 * math.pi / n_theta
    t = np.linspace(0.0, 1.0, Ng + 1)
    E = n_r * n_theta
    nodes = np.zeros((E, (Ng + 1) ** 2, 2))
    for j in range(n_theta):
        for i in range(n_r):
            e = j * n_r + i
            A, B = np.meshgrid(t, t, indexing="xy")   # A along xi = m, B along eta = t
            M = mk[i] + A * (mk[i + 1] - mk[i])
            TH = (j + B) * dth
            nodes[e, :, 0] = (c * np.cosh(M) * np.cos(TH)).reshape(-1)
            nodes[e, :, 1] = (c * np.sinh(M) * np.sin(TH)).reshape(-1)
    nbr = np.zeros((E, 4, 3), dtype=np.int32)
    for j in range(n_theta):
        for i in range(n_r):
            e = j * n_r + i
            nbr[e, 0] = (((j - 1) % n_theta) * n_r + i, 2, 0)
            nbr[e, 1] = (j * n_r + i + 1, 3, 0) if i < n_r - 1 else (-1, outer, 0)
            nbr[e, 2] = (((j + 1) % n_theta) * n_r + i, 0, 0)
            nbr[e, 3] = (j * n_r + i - 1, 1, 0) if i > 0 else (-1, wall, 0)
    return nodes, nbr


def extruded_ellipse(n_r: int, n_theta: int, n_z: int, span: float = 0.2, Ng: int = 2, **kw):
    """The ellipse O-mesh extruded along z over ``span`` with ``n_z`` layers,
    periodic in z (the extruded-ellipse workload: 48 x 64 x 20 = 61,440
    hexahedra at full size)."""
    nodes2, nbr2 = ellipse_omesh(n_r, n_theta, Ng=Ng, **kw)
    return extrude(nodes2, nbr2, Ng, nz=n_z, z0=0.0, z1=span)


def flip_elements(nodes: np.ndarray, nbr: np.ndarray, which, Ng: int):
    """Rotate the local numbering of the listed elements by 180 degrees.

    The mesh is unchanged geometrically, but the rotated elements meet their
    neighbours with reversed face-point order, which exercises the
    orientation flag of the connectivity table.
    """
    nodes = nodes.copy()
    nbr = nbr.copy()
    n1 = Ng + 1
    which = set(int(e) for e in which)
    for e in which:
        nodes[e] = nodes[e].reshape(n1, n1, 2)[::-1, ::-1].reshape(-1, 2)
    # local face f of a rotated element is old face (f+2)%4
    old = nbr.copy()
    for e in range(nbr.shape[0]):
        for f in range(4):
            of = (f + 2) % 4 if e in which else f
            en, fn, _ = old[e, of]
            fn_new = (fn + 2) % 4 if en in which else fn
            # both elements sharing the face agree on orientation unless exactly one is rotated
            rev = 1 if ((e in which) != (int(en) in which)) else 0
            nbr[e, f] = (en, fn_new, rev)
    return nodes, nbr


def freestream_T(Ma_inf: float, speed: float = math.sqrt(2.0), gamma: float = GAMMA) -> float:
    """Free-stream temperature for a Mach number defined with |v_inf| (R = 1)."""
    c = speed / Ma_inf
    return c * c / gamma


def freestream_scales(Ma_inf: float, rho: float = 1.0, speed: float = math.sqrt(2.0),
                      gamma: float = GAMMA) -> tuple:
    """Convective flux scales (rho U, rho U^2, rho U^2, rho U H) of the free
    stream, one per equation: the reference scales of the residual norm."""
    T = freestream_T(Ma_inf, speed, gamma)
    H = gamma / (gamma - 1.0) * T + 0.5 * speed * speed
    return (rho * speed, rho * speed * speed, rho * speed * speed, rho * speed * H)


def isentropic_vortex(xy: np.ndarray, t: float = 0.0, Ma_inf: float = 0.005,
                      strength: float = 5.0, phi: float = 0.5,
                      center=(5.0, 5.0), period=(10.0, 10.0),
                      gamma: float = GAMMA) -> np.ndarray:
    """Isentropic vortex of eq. VP_Solution advected by (u, v) = (1, 1).

    ``xy`` has shape ``(..., 2)``.  Returns primitive variables (p, u, v, T)
    in an array of shape ``(4,) + xy.shape[:-1]``.  r is the Euclidean
    distance to the (periodically nearest) vortex centre; the free stream is
    rho = u = v = 1 with Ma_inf = |v_inf| / c_inf and R = 1.
    """
    Tinf = freestream_T(Ma_inf, gamma=gamma)
    xc = center[0] + t
    yc = center[1] + t
    dx = xy[..., 0] - xc
    dy = xy[..., 1] - yc
    if period is not None:
        dx = dx - period[0] * np.round(dx / period[0])
        dy = dy - period[1] * np.round(dy / period[1])
    r2 = dx * dx + dy * dy
    ex = np.exp(phi * (1.0 - r2))
    du = -strength / (2 * math.pi) * dy * ex
    dv = strength / (2 * math.pi) * dx * ex
    dT = -strength ** 2 * (gamma - 1.0) / (16.0 * phi * gamma * math.pi ** 2) * ex * ex
    T = Tinf + dT
    rho = (T / Tinf) ** (1.0 / (gamma - 1.0))
    p = rho * T
    return np.stack([p, 1.0 + du, 1.0 + dv, T])


def to_soa(field: np.ndarray) -> np.ndarray:
    """(4, E, N) field -> contiguous float64 state array, variable-major."""
    return np.ascontiguousarray(field, dtype=np.float64)


def freestream_noise_state(xy: np.ndarray, Ma_inf: float, speed: float = 1.0, noise: float = 1e-3,
                           seed: int = 7, gamma: float = GAMMA) -> np.ndarray:
    """Free stream (rho = 1, u = speed, v = 0) with seeded Gaussian noise of
    relative size ``noise`` in v: the start of the cylinder case."""
    T = freestream_T(Ma_inf, speed, gamma)
    rng = np.random.default_rng(seed)
    shape = xy.shape[:-1]
    return np.stack([np.full(shape, T), np.full(shape, speed),
                     noise * speed * rng.standard_normal(shape), np.full(shape, T)])


def uniform_state(E: int, N: int, p: float, u: float, v: float, T: float) -> np.ndarray:
    q = np.empty((4, E, N))
    q[0], q[1], q[2], q[3] = p, u, v, T
    return q


def random_perturbed_state(E: int, N: int, Ma_inf: float = 0.005, amp: float = 0.05,
                           seed: int = 7) -> np.ndarray:
    """Free stream (rho = u = v = 1) plus seeded noise, for parity tests."""
    rng = np.random.default_rng(seed)
    Tinf = freestream_T(Ma_inf)
    q = uniform_state(E, N, Tinf, 1.0, 1.0, Tinf)
    q[0] += amp * rng.standard_normal((E, N))
    q[1] += amp * rng.standard_normal((E, N))
    q[2] += amp * rng.standard_normal((E, N))
    q[3] += 1e-3 * amp * rng.standard_normal((E, N))
    return q


# ---------------------------------------------------------------------------
# Three dimensions: hexahedral meshes and 5-variable states (p, u, v, w, T).
#
# * ``nodes``: float64 ``(E, (Ng+1)**3, 3)``, node ``(c*(Ng+1)+b)*(Ng+1)+a``
#   with ``a`` along xi, ``b`` along eta, ``c`` along zeta.
# * ``nbr``: int32 ``(E, 6, 3)``: for each local face ``f = 2*d + s`` (d = 0
#   xi, 1 eta, 2 zeta; s = 0 the -1 side, 1 the +1 side) the neighbour
#   element, its local face and an orientation code ``o`` (0..7): a face point
#   ``(a, b)`` (a along the first, b along the second of the face's two
#   reference directions in increasing order) is the neighbour's point
#   ``(a', b')`` with ``(s, t) = (b, a) if o & 4 else (a, b)``,
#   ``a' = P - s if o & 1 else s``, ``b' = P - t if o & 2 else t``.  A boundary
#   face has neighbour -1 and its boundary type in the second slot.
# ---------------------------------------------------------------------------
def _face_local_nodes(f: int, Ng: int):
    """Element-local node indices of face f, ordered (b, a) row-major."""
    d, s = f // 2, f % 2
    t1, t2 = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
    out = np.zeros((Ng + 1, Ng + 1), dtype=np.int64)
    for b in range(Ng + 1):
        for a in range(Ng + 1):
            idx = [0, 0, 0]
            idx[d] = s * Ng
            idx[t1] = a
            idx[t2] = b
            out[b, a] = (idx[2] * (Ng + 1) + idx[1]) * (Ng + 1) + idx[0]
    return out


def _orient_map(o: int, P: int, a, b):
    s, t = (b, a) if o & 4 else (a, b)
    return (P - s if o & 1 else s), (P - t if o & 2 else t)


def hex_connectivity(nodes: np.ndarray, Ng: int, period=(None, None, None), boundary=None, tol: float = 1e-9):
    """Face neighbours and orientation codes of hexahedra from their geometry.

    Faces are paired by their centroids (coordinates taken modulo
    ``period[d]`` in periodic directions); the orientation code of a pair is
    the one under which every face node of one face lies on the matching node
    of the other.  Faces left unmatched get ``boundary(e, f)`` as their type."""
    from scipy.spatial import cKDTree
    E = nodes.shape[0]
    fl = [_face_local_nodes(f, Ng) for f in range(6)]
    ext = np.ptp(nodes.reshape(-1, 3), axis=0).max() + 1.0
    lo = nodes.reshape(-1, 3).min(axis=0)
    box = np.array([period[d] if period[d] else 1e6 * ext for d in range(3)])
    cent = np.zeros((E * 6, 3))
    for e in range(E):
        for f in range(6):
            cent[e * 6 + f] = nodes[e][fl[f].reshape(-1)].mean(axis=0)
    cw = np.mod(cent - lo, box)
    tree = cKDTree(cw, boxsize=box)
    scale = tol * ext
    A, B = np.meshgrid(np.arange(Ng + 1), np.arange(Ng + 1), indexing="xy")

    def wrapped(d):
        for k in range(3):
            if period[k]:
                d[..., k] -= period[k] * np.round(d[..., k] / period[k])
        return d

    nbr = np.zeros((E, 6, 3), dtype=np.int32)
    for e in range(E):
        for f in range(6):
            cand = [c for c in tree.query_ball_point(cw[e * 6 + f], scale) if c != e * 6 + f]
            if not cand:
                if boundary is None:
                    raise ValueError(f"unmatched face {f} of element {e}")
                nbr[e, f] = (-1, boundary(e, f), 0)
                continue
            if len(cand) != 1:
                raise ValueError(f"face {f} of element {e} matches {len(cand)} faces")
            e2, f2 = divmod(cand[0], 6)
            mine = nodes[e][fl[f]]
            theirs = nodes[e2][fl[f2]]
            for o in range(8):
                a2, b2 = _orient_map(o, Ng, A, B)
                if np.abs(wrapped(mine - theirs[b2, a2])).max() <= scale:
                    nbr[e, f] = (e2, f2, o)
                    break
            else:
                raise ValueError(f"faces ({e},{f}) and ({e2},{f2}) meet but no orientation matches")
    return nbr


def _box3d(nx, ny, nz, lo, hi, Ng, perturb, seed, periodic=(True, True, True)):
    L = [hi[i] - lo[i] for i in range(3)]
    h = [L[0] / nx, L[1] / ny, L[2] / nz]
    rng = np.random.default_rng(seed)
    modes = []
    if perturb > 0.0:
        for _ in range(3):
            k = rng.integers(1, 3, size=3)
            amp = rng.uniform(-1.0, 1.0, size=3)
            ph = rng.uniform(0.0, 2 * math.pi, size=3)
            modes.append((k, amp, ph))
    r = np.linspace(0.0, 1.0, Ng + 1)
    C, B, A = np.meshgrid(r, r, r, indexing="ij")   # node (c, b, a): A along xi
    E = nx * ny * nz
    n1 = Ng + 1
    nodes = np.zeros((E, n1 ** 3, 3))
    for kz in range(nz):
        for jy in range(ny):
            for ix in range(nx):
                e = (kz * ny + jy) * nx + ix
                X = lo[0] + (ix + A) * h[0]
                Y = lo[1] + (jy + B) * h[1]
                Z = lo[2] + (kz + C) * h[2]
                dX, dY, dZ = np.zeros_like(X), np.zeros_like(X), np.zeros_like(X)
                for k, amp, ph in modes:
                    arg = 2 * math.pi * (k[0] * (X - lo[0]) / L[0] + k[1] * (Y - lo[1]) / L[1] +
                                         k[2] * (Z - lo[2]) / L[2])
                    # vanish on non-periodic sides so that walls stay flat
                    damp = np.ones_like(X)
                    for dd, (Q, per) in enumerate(zip((X, Y, Z), periodic)):
                        if not per:
                            damp *= np.sin(math.pi * (Q - lo[dd]) / L[dd])
                    dX += amp[0] * np.sin(arg + ph[0]) * damp
                    dY += amp[1] * np.sin(arg + ph[1]) * damp
                    dZ += amp[2] * np.sin(arg + ph[2]) * damp
                sc = perturb * min(h) / max(1, len(modes))
                nodes[e, :, 0] = (X + sc * dX).reshape(-1)
                nodes[e, :, 1] = (Y + sc * dY).reshape(-1)
                nodes[e, :, 2] = (Z + sc * dZ).reshape(-1)
    return nodes


# the 24 proper rotations of the reference cube (signed permutation matrices, det +1)
def _cube_rotations():
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for i in range(3):
                R[i, perm[i]] = signs[i]
            if round(np.linalg.det(R)) == 1:
                out.append(R)
    return out


CUBE_ROTATIONS = _cube_rotations()


def rotate_hex_elements(nodes, Ng: int, rotations: dict):
    """Renumber the local nodes of the listed elements ({element: rotation
    index into CUBE_ROTATIONS}); the geometry is unchanged."""
    nodes = nodes.copy()
    n1 = Ng + 1
    for e, ri in rotations.items():
        R = CUBE_ROTATIONS[ri]
        old_n = nodes[e].copy()
        for c in range(n1):
            for b in range(n1):
                for a in range(n1):
                    rn = np.array([2 * a - Ng, 2 * b - Ng, 2 * c - Ng])   # new reference coords x Ng
                    ro = R.T @ rn
                    ao, bo, co = ((ro + Ng) // 2).tolist()
                    nodes[e, (c * n1 + b) * n1 + a] = old_n[(co * n1 + bo) * n1 + ao]
    return nodes


def periodic_box3d(nx: int, ny: int, nz: int, lo=(0.0, 0.0, 0.0), hi=(10.0, 10.0, 10.0), Ng: int = 1,
                   perturb: float = 0.0, seed: int = 1234, rotations=None):
    """Triply periodic ``nx`` x ``ny`` x ``nz`` hexahedral mesh of a box,
    element ``e = (kz*ny + jy)*nx + ix``.  With ``perturb > 0`` the nodes move
    by a smooth periodic displacement of a few seeded Fourier modes (curved
    elements for ``Ng >= 2``); ``rotations`` {element: index into
    CUBE_ROTATIONS} renumbers elements' local axes, so that faces meet in
    other orientations."""
    nodes = _box3d(nx, ny, nz, lo, hi, Ng, perturb, seed)
    if rotations:
        nodes = rotate_hex_elements(nodes, Ng, rotations)
    period = tuple(hi[d] - lo[d] for d in range(3))
    return nodes, hex_connectivity(nodes, Ng, period=period)


def extrude(nodes2d, nbr2d, Ng: int, nz: int = 1, z0: float = 0.0, z1: float = 1.0):
    """Hexahedra extruded from a quadrilateral mesh along z (periodic in z):
    element ``e3 = kz*E2 + e2`` with xi, eta of the quadrilateral and zeta along
    z.  Quadrilateral faces (0 eta-, 1 xi+, 2 eta+, 3 xi-) become hexahedral
    faces 2, 1, 3, 0; a reversed quadrilateral face becomes orientation 1."""
    E2 = nodes2d.shape[0]
    n1 = Ng + 1
    hz = (z1 - z0) / nz
    E = E2 * nz
    nodes = np.zeros((E, n1 ** 3, 3))
    nbr = np.zeros((E, 6, 3), dtype=np.int32)
    f3 = {0: 2, 1: 1, 2: 3, 3: 0}
    for kz in range(nz):
        for e2 in range(E2):
            e = kz * E2 + e2
            for c in range(n1):
                z = z0 + (kz + c / Ng) * hz
                for b in range(n1):
                    for a in range(n1):
                        nodes[e, (c * n1 + b) * n1 + a, :2] = nodes2d[e2, b * n1 + a]
                        nodes[e, (c * n1 + b) * n1 + a, 2] = z
            for f in range(4):
                en, fn, rev = nbr2d[e2, f]
                if en < 0:
                    nbr[e, f3[f]] = (-1, fn, 0)
                else:
                    nbr[e, f3[f]] = (kz * E2 + en, f3[int(fn)], 1 if rev else 0)
            nbr[e, 4] = (((kz - 1) % nz) * E2 + e2, 5, 0)
            nbr[e, 5] = (((kz + 1) % nz) * E2 + e2, 4, 0)
    return nodes, nbr


def uniform_state3(E: int, N: int, p: float, u: float, v: float, w: float, T: float) -> np.ndarray:
    q = np.empty((5, E, N))
    for k, val in enumerate((p, u, v, w, T)):
        q[k] = val
    return q


def vortex3d(xyz: np.ndarray, Ma_inf: float = 0.005, center=(5.0, 5.0), period=(10.0, 10.0),
             Lz: float = 10.0, w_amp: float = 0.1, gamma: float = GAMMA) -> np.ndarray:
    """The isentropic vortex of eq. VP_Solution in (x, y), uniform in z, plus
    a divergence-free w = w_amp sin(2 pi x / Lx) sin(2 pi y / Ly) shear that
    makes the state genuinely three-dimensional: (5, E, N) primitive state."""
    E, N, _ = xyz.shape
    q2 = isentropic_vortex(xyz[:, :, :2], Ma_inf=Ma_inf, center=center, period=period, gamma=gamma)
    q = np.zeros((5, E, N))
    q[0], q[1], q[2], q[4] = q2[0], q2[1], q2[2], q2[3]
    q[3] = w_amp * np.sin(2 * math.pi * xyz[:, :, 0] / period[0]) * np.sin(2 * math.pi * xyz[:, :, 1] / period[1])
    return q


def freestream_scales3(Ma_inf: float, rho: float = 1.0, speed: float = math.sqrt(2.0),
                       gamma: float = GAMMA) -> tuple:
    """Convective flux scales of the five equations (rho U, rho U^2 x 3, rho U H)."""
    m, mx, my, e = freestream_scales(Ma_inf, rho, speed, gamma)
    return (m, mx, my, mx, e)


def cubed_sphere_shell(n: int, n_r: int, r_in: float = 0.5, r_out: float = 20.0, Ng: int = 2,
                       wall: int = BC_SLIP_WALL, outer: int = BC_FARFIELD):
    """Spherical shell of 6 n n n_r hexahedra: the six faces of a cube, each
    cut into n x n cells of equal angle (equiangular gnomonic map), times n_r
    radial layers r_k = r_in (r_out/r_in)^(k/n_r).  Element
    e = ((face*n_r + k)*n + j)*n + i; xi and eta follow the face's two angles
    and zeta the radius, so every geometry node lies exactly on its sphere.
    Faces at r_in carry ``wall``, faces at r_out ``outer``; the patches meet
    along their edges in the orientations that the face matching finds."""
    axes = [((0, 1, 0), (0, 0, 1), (1, 0, 0)), ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),
            ((0, 0, 1), (1, 0, 0), (0, 1, 0)), ((1, 0, 0), (0, 0, 1), (0, -1, 0)),
            ((1, 0, 0), (0, 1, 0), (0, 0, 1)), ((0, 1, 0), (1, 0, 0), (0, 0, -1))]
    rk = r_in * (r_out / r_in) ** (np.arange(n_r + 1) / n_r)
    da = 0.5 * math.pi / n
    t = np.linspace(0.0, 1.0, Ng + 1)
    n1 = Ng + 1
    E = 6 * n * n * n_r
    nodes = np.zeros((E, n1 ** 3, 3))
    for fc, (u, v, c0) in enumerate(axes):
        u, v, c0 = np.array(u, float), np.array(v, float), np.array(c0, float)
        for k in range(n_r):
            for j in range(n):
                for i in range(n):
                    e = ((fc * n_r + k) * n + j) * n + i
                    for cc in range(n1):
                        r = rk[k] + t[cc] * (rk[k + 1] - rk[k])
                        for b in range(n1):
                            beta = -0.25 * math.pi + (j + t[b]) * da
                            for a in range(n1):
                                alpha = -0.25 * math.pi + (i + t[a]) * da
                                d = c0 + math.tan(alpha) * u + math.tan(beta) * v
                                nodes[e, (cc * n1 + b) * n1 + a] = r * d / np.linalg.norm(d)

    def bc(e, f):
        if f == 4:
            return wall
        if f == 5:
            return outer
        raise ValueError(f"unmatched side face {f} of element {e}")

    return nodes, hex_connectivity(nodes, Ng, boundary=bc)
