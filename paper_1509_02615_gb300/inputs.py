"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module builds node sets (Cartesian, hexagonal and Poisson-disk scattered
layouts with their ghost or mirror layers, Sec. 5.1-5.2), the closed-form
initial states of the test cases (Sec. 6) and the analytic velocity field of
the scalar-advection case.  It holds none of the RBF-FD arithmetic: no stencil
selection, no weights, no right-hand side.  Both the CUDA path and the oracle
import it; neither imports the other.

Node ordering convention (every node set):
  * prognostic nodes ``[0, n_prog)`` come first (interior and boundary nodes,
    Sec. 5.2: the PDE is enforced on the boundary, so boundary nodes are
    stepped), then ghost or mirror nodes ``[n_prog, n_all)``;
  * ``kind[i]`` for prognostic node i: 0 interior, 1 bottom wall, 2 top wall,
    3 left wall, 4 right wall;
  * ``ghost_owner[g]`` is the prognostic boundary node served by ghost
    ``n_prog + g`` (one ghost per boundary node, Sec. 5.2);
  * ``src[j]`` maps every node to the prognostic node whose value it carries:
    the identity on prognostic nodes, the reflected source on mirror nodes
    (reflection boundary of the advection case, Sec. 6.1); -1 on ghosts, whose
    values are solved for.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KIND_INTERIOR, KIND_BOTTOM, KIND_TOP, KIND_LEFT, KIND_RIGHT = 0, 1, 2, 3, 4

# Physical constants of the Navier-Stokes test cases (Sec. 6.2).
CP, CV, RD, G = 1004.0, 717.0, 287.0, 9.81
THETA_BAR = 300.0


@dataclasses.dataclass
class NodeSet:
    x: np.ndarray            # float64 [n_all]
    z: np.ndarray            # float64 [n_all]  (y for the unit-square case)
    n_prog: int
    kind: np.ndarray         # int32 [n_prog]
    ghost_owner: np.ndarray  # int32 [n_all - n_prog]; -1 for mirror nodes
    src: np.ndarray          # int32 [n_all]
    period_x: float          # > 0: periodic in x with this period
    h: float                 # nominal node spacing
    layout: str
    domain: tuple            # (x0, x1, z0, z1)

    @property
    def n_all(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_ghost(self) -> int:
        return self.n_all - self.n_prog


def _lattice_rows(layout, x0, x1, z0, z1, h, periodic_x, rows=None):
    """Row positions and per-row x coordinates of a lattice covering the box.

    Hexagonal rows are fitted to the domain height: R = round(H / (h*sqrt(3)/2))
    intervals of dz = H / R, odd rows shifted by half a column (Sec. 5.1).
    ``rows`` overrides R (nested lattices).
    """
    W, H = x1 - x0, z1 - z0
    if rows is not None:
        nint = int(rows)
    elif layout == "hex":
        nint = max(1, int(round(H / (h * math.sqrt(3.0) / 2.0))))
    elif layout == "cart":
        nint = max(1, int(round(H / h)))
    else:
        raise ValueError(layout)
    dz = H / nint
    if periodic_x:
        ncol = int(round(W / h))
        dx = W / ncol
    else:
        ncol = int(round(W / h)) + 1
        dx = W / (ncol - 1)
    return nint, dz, ncol, dx


def _row_x(layout, r, x0, ncol, dx, periodic_x):
    c = np.arange(ncol, dtype=np.float64)
    if layout == "hex" and (r % 2) == 1:
        if periodic_x:
            return x0 + (c + 0.5) * dx
        # walls: odd rows keep the wall nodes and sit half a column inside
        inner = x0 + (np.arange(ncol - 1) + 0.5) * dx
        return np.concatenate([[x0], inner, [x0 + (ncol - 1) * dx]])
    return x0 + c * dx


def lattice_nodes(layout: str, x0: float, x1: float, z0: float, z1: float, h: float,
                  periodic_x: bool = True, rows: int = None) -> NodeSet:
    """Cartesian or hexagonal lattice with one ghost row below and above.

    Each top and bottom wall node gets one ghost one row spacing outside it,
    straight along the wall normal (Sec. 5.2).  With ``periodic_x`` false the left and right columns are
    walls as well and get one ghost column outside, continuing the row.  Corner
    nodes belong to the top or bottom wall.
    """
    nint, dz, ncol, dx = _lattice_rows(layout, x0, x1, z0, z1, h, periodic_x, rows)
    xs, zs, kinds = [], [], []
    gx, gz, gown = [], [], []
    for r in range(nint + 1):
        xr = _row_x(layout, r, x0, ncol, dx, periodic_x)
        k = np.zeros(xr.shape[0], np.int32)
        if not periodic_x:
            k[0], k[-1] = KIND_LEFT, KIND_RIGHT
        if r == 0:
            k[:] = KIND_BOTTOM
        elif r == nint:
            k[:] = KIND_TOP
        xs.append(xr)
        zs.append(np.full(xr.shape[0], z0 + r * dz))
        kinds.append(k)
    x = np.concatenate(xs)
    z = np.concatenate(zs)
    kind = np.concatenate(kinds)
    n_prog = x.shape[0]
    # ghosts: one per wall node, one row spacing outside along the outward
    # normal.  (Continuing the hexagonal offset instead would make the
    # periodic ghost system circulant with a zero at the checkerboard mode.)
    row_start = np.cumsum([0] + [a.shape[0] for a in xs])
    for r_own, zg in ((0, z0 - dz), (nint, z1 + dz)):
        own_idx = np.arange(row_start[r_own], row_start[r_own + 1])
        gx.append(x[own_idx].copy())
        gz.append(np.full(own_idx.shape[0], zg))
        gown.append(own_idx)
    if not periodic_x:
        for side, kk in ((0, KIND_LEFT), (1, KIND_RIGHT)):
            own_idx = np.nonzero(kind == kk)[0]
            xg = x[own_idx] + (-dx if side == 0 else dx)
            gx.append(xg)
            gz.append(z[own_idx].copy())
            gown.append(own_idx)
    x = np.concatenate([x] + gx)
    z = np.concatenate([z] + gz)
    ghost_owner = np.concatenate(gown).astype(np.int32)
    src = np.concatenate([np.arange(n_prog), -np.ones(x.shape[0] - n_prog, np.int64)]).astype(np.int32)
    return NodeSet(x=x, z=z, n_prog=n_prog, kind=kind.astype(np.int32), ghost_owner=ghost_owner,
                   src=src, period_x=(x1 - x0) if periodic_x else 0.0, h=h, layout=layout,
                   domain=(x0, x1, z0, z1))


def density_current_nodes(h: float = 100.0, layout: str = "hex", periodic_x: bool = True) -> NodeSet:
    """Straka density-current domain [-25.6, 25.6] x [0, 6.4] km (Sec. 6.3)."""
    return lattice_nodes(layout, -25600.0, 25600.0, 0.0, 6400.0, h, periodic_x)


def translating_current_nodes(h: float = 100.0, layout: str = "hex") -> NodeSet:
    """Translating density-current domain [0, 36] x [0, 6.4] km, periodic in x
    (Sec. 6.3.2, Wicker-Skamarock set-up)."""
    return lattice_nodes(layout, 0.0, 36000.0, 0.0, 6400.0, h, periodic_x=True)


def rising_bubble_nodes(h: float = 100.0, layout: str = "hex", seed: int = 1) -> NodeSet:
    """Rising-bubble box [0, 10] x [0, 10] km with walls on all four sides
    (Sec. 6.4): Cartesian or hexagonal lattice, or seeded Poisson-disk nodes."""
    if layout == "scattered":
        return poisson_disk_nodes(0.0, 10000.0, 0.0, 10000.0, h, seed=seed)
    return lattice_nodes(layout, 0.0, 10000.0, 0.0, 10000.0, h, periodic_x=False)


def unit_square_mirrored(m: int = 64, layers: int = 4) -> NodeSet:
    """Cartesian m x m nodes on [0,1]^2 (boundary nodes included, h = 1/(m-1))
    plus ``layers`` rows of nodes reflected across each wall and doubly
    reflected across each corner (Sec. 6.1: reflected nodes carry the values of
    their interior sources, so no boundary condition is needed)."""
    h = 1.0 / (m - 1)
    c = np.arange(m) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    x = X.ravel().copy()
    y = Y.ravel().copy()
    n_prog = x.shape[0]
    gi, gj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    gi, gj = gi.ravel(), gj.ravel()
    mx, my, msrc = [], [], []

    def refl(k):
        # index k in [-layers, m-1+layers] -> source index and coordinate
        if k < 0:
            return -k, k * h
        if k > m - 1:
            return 2 * (m - 1) - k, k * h
        return k, k * h

    for jj in range(-layers, m + layers):
        for ii in range(-layers, m + layers):
            if 0 <= ii < m and 0 <= jj < m:
                continue
            si, xc = refl(ii)
            sj, yc = refl(jj)
            mx.append(xc)
            my.append(yc)
            msrc.append(sj * m + si)
    x = np.concatenate([x, np.array(mx)])
    y = np.concatenate([y, np.array(my)])
    src = np.concatenate([np.arange(n_prog), np.array(msrc)]).astype(np.int32)
    kind = np.zeros(n_prog, np.int32)
    return NodeSet(x=x, z=y, n_prog=n_prog, kind=kind,
                   ghost_owner=-np.ones(x.shape[0] - n_prog, np.int32), src=src, period_x=0.0,
                   h=h, layout="cart-mirror", domain=(0.0, 1.0, 0.0, 1.0))


def unit_square_hex_mirrored(h: float = 0.005, layers: int = 5) -> NodeSet:
    """Hexagonal lattice on [0,1]^2 with reflected layers (Sec. 6.1).

    Rows are fitted to the height like the density-current lattice:
    R = round(1 / (h sqrt(3)/2)) intervals of dy = 1/R; M = round(1/h) column
    intervals of dx = 1/M; even rows hold x = c dx (c = 0..M, wall nodes
    included), odd rows x = (c + 1/2) dx (c = 0..M-1).  The reflection of a
    lattice node across any wall is a lattice node (row r -> -r or 2R - r keeps
    its parity; an odd row's offsets map onto themselves), so the reflected
    nodes continue the lattice: every lattice node within ``layers`` row or
    column spacings outside the square is added, carrying the value of its
    reflected source (corners reflected twice).
    """
    R = max(1, int(round(1.0 / (h * math.sqrt(3.0) / 2.0))))
    M = max(1, int(round(1.0 / h)))
    dx, dy = 1.0 / M, 1.0 / R

    def row_cols(r, lo, hi):
        # column numbers c of row r with lattice x in [lo*dx, hi*dx]
        if r % 2 == 0:
            return np.arange(lo, hi + 1)
        return np.arange(lo, hi)   # x = (c + 1/2) dx

    def xpos(r, c):
        return (c + (0.5 if r % 2 else 0.0)) * dx

    key = {}
    xs, ys = [], []
    for r in range(R + 1):
        for c in row_cols(r, 0, M):
            key[(r, int(c))] = len(xs)
            xs.append(xpos(r, c))
            ys.append(r * dy)
    n_prog = len(xs)
    mx, my, msrc = [], [], []
    for r in range(-layers, R + layers + 1):
        for c in row_cols(r, -layers, M + layers):
            c = int(c)
            inside_r = 0 <= r <= R
            inside_c = (0 <= c <= M) if r % 2 == 0 else (0 <= c <= M - 1)
            if inside_r and inside_c:
                continue
            sr = -r if r < 0 else (2 * R - r if r > R else r)
            if r % 2 == 0:
                sc = -c if c < 0 else (2 * M - c if c > M else c)
            else:
                sc = -c - 1 if c < 0 else (2 * M - c - 1 if c > M - 1 else c)
            mx.append(xpos(r, c))
            my.append(r * dy)
            msrc.append(key[(sr, sc)])
    x = np.concatenate([np.array(xs), np.array(mx)])
    y = np.concatenate([np.array(ys), np.array(my)])
    src = np.concatenate([np.arange(n_prog), np.array(msrc, np.int64)]).astype(np.int32)
    return NodeSet(x=x, z=y, n_prog=n_prog, kind=np.zeros(n_prog, np.int32),
                   ghost_owner=-np.ones(x.shape[0] - n_prog, np.int32), src=src, period_x=0.0,
                   h=h, layout="hex-mirror", domain=(0.0, 1.0, 0.0, 1.0))


def hilbert_order(x: np.ndarray, z: np.ndarray, bits: int = 16) -> np.ndarray:
    """Permutation sorting points along a Hilbert curve (locality for gathers)."""
    xs = (x - x.min()) / max(x.max() - x.min(), 1e-300)
    zs = (z - z.min()) / max(z.max() - z.min(), 1e-300)
    n = 1 << bits
    X = np.minimum((xs * (n - 1)).astype(np.int64), n - 1)
    Y = np.minimum((zs * (n - 1)).astype(np.int64), n - 1)
    d = np.zeros_like(X)
    s = n >> 1
    while s > 0:
        rx = ((X & s) > 0).astype(np.int64)
        ry = ((Y & s) > 0).astype(np.int64)
        d += s * s * ((3 * rx) ^ ry)
        # rotate
        flip = ry == 0
        sw = flip & (rx == 1)
        X = np.where(sw, s - 1 - X, X)
        Y = np.where(sw, s - 1 - Y, Y)
        Xn = np.where(flip, Y, X)
        Yn = np.where(flip, X, Y)
        X, Y = Xn, Yn
        s >>= 1
    return np.argsort(d, kind="stable")


def _poisson_disk_points(x0, W, z0, H, r, rng, periodic_x=False, rounds=60):
    """Near-maximal Poisson-disk sample with minimum distance r in the box
    [x0, x0+W) x [z0, z0+H], by parallel dart throwing on a background grid
    of cells of size about r/sqrt(2) (at most one point per cell).  Cells are
    processed in 9 colour classes (i mod 3, j mod 3): proposals of one class
    are at least two cells apart and cannot conflict with each other, so a
    whole class is tested against the accepted points at once.  With a
    periodic x the column count is a multiple of 3, so the classes also stay
    apart across the seam."""
    cs = r / math.sqrt(2.0)
    if periodic_x:
        ncx = max(3, 3 * int(math.floor(W / cs) // 3))
    else:
        ncx = max(1, int(math.ceil(W / cs)))
    ncz = max(1, int(math.ceil(H / cs)))
    cw, ch = W / ncx, H / ncz
    px = np.full((ncz, ncx), np.nan)
    pz = np.full((ncz, ncx), np.nan)
    offs = [(dj, di) for dj in range(-2, 3) for di in range(-2, 3) if (dj, di) != (0, 0)]
    total = 0
    for _ in range(rounds):
        added = 0
        for cj in range(3):
            for ci in range(3):
                sub_x = px[cj::3, ci::3]
                if sub_x.size == 0:
                    continue
                empty = np.isnan(sub_x)
                if not empty.any():
                    continue
                # neighbours through a 2-cell NaN (or periodic) border
                Px = np.pad(px, 2, constant_values=np.nan)
                Pz = np.pad(pz, 2, constant_values=np.nan)
                if periodic_x:
                    Px[2:-2, :2] = px[:, -2:] - W
                    Px[2:-2, -2:] = px[:, :2] + W
                    Pz[2:-2, :2] = pz[:, -2:]
                    Pz[2:-2, -2:] = pz[:, :2]
                nr, nc = sub_x.shape
                jj = (cj + 3 * np.arange(nr))[:, None]
                ii = (ci + 3 * np.arange(nc))[None, :]
                cx = x0 + (ii + rng.uniform(size=(nr, nc))) * cw
                cz = z0 + (jj + rng.uniform(size=(nr, nc))) * ch
                ok = empty.copy()
                for dj, di in offs:
                    qx = Px[2 + cj + dj::3, 2 + ci + di::3][:nr, :nc]
                    qz = Pz[2 + cj + dj::3, 2 + ci + di::3][:nr, :nc]
                    ok &= ~((cx - qx) ** 2 + (cz - qz) ** 2 < r * r)   # NaN compares False
                px[cj::3, ci::3] = np.where(ok, cx, sub_x)
                pz[cj::3, ci::3] = np.where(ok, cz, pz[cj::3, ci::3])
                added += int(ok.sum())
        total += added
        if added <= max(1, total // 500):   # saturated: further darts rarely land
            break
    m = ~np.isnan(px)
    return px[m], pz[m]


def poisson_disk_nodes(x0: float, x1: float, z0: float, z1: float, h: float, seed: int = 1,
                       periodic_x: bool = False) -> NodeSet:
    """Quasi-uniformly scattered nodes (Sec. 5.1) by seeded Poisson-disk sampling.

    Walls carry evenly spaced boundary nodes (spacing h): top and bottom, and
    left and right unless ``periodic_x``.  Interior samples keep a minimum
    distance r_min = 0.83 h from each other (so that sqrt(area / N) is close to
    h) and at least h/2 from the walls.  Each wall node gets one ghost at
    distance h outside along the wall normal; corner nodes belong to the
    bottom/top walls.  Nodes are ordered along a Hilbert curve.
    """
    rng = np.random.default_rng(seed)
    W, H = x1 - x0, z1 - z0
    nbx = int(round(W / h))
    nbz = int(round(H / h))
    if periodic_x:
        bx = x0 + np.arange(nbx) * (W / nbx)
        wall_x = np.concatenate([bx, bx])
        wall_z = np.concatenate([np.full(bx.shape, z0), np.full(bx.shape, z1)])
        wall_k = np.concatenate([np.full(bx.shape, KIND_BOTTOM), np.full(bx.shape, KIND_TOP)])
        ix, iz = _poisson_disk_points(x0, W, z0 + 0.5 * h, H - h, 0.83 * h, rng, periodic_x=True)
    else:
        bx = x0 + np.arange(nbx + 1) * (W / nbx)
        bz = z0 + np.arange(1, nbz) * (H / nbz)
        wall_x = np.concatenate([bx, bx, np.full(bz.shape, x0), np.full(bz.shape, x1)])
        wall_z = np.concatenate([np.full(bx.shape, z0), np.full(bx.shape, z1), bz, bz])
        wall_k = np.concatenate([np.full(bx.shape, KIND_BOTTOM), np.full(bx.shape, KIND_TOP),
                                 np.full(bz.shape, KIND_LEFT), np.full(bz.shape, KIND_RIGHT)])
        ix, iz = _poisson_disk_points(x0 + 0.5 * h, W - h, z0 + 0.5 * h, H - h, 0.83 * h, rng)
    x = np.concatenate([ix, wall_x])
    z = np.concatenate([iz, wall_z])
    kind = np.concatenate([np.zeros(ix.shape[0], np.int32), wall_k.astype(np.int32)])
    perm = hilbert_order(x, z)
    x, z, kind = x[perm], z[perm], kind[perm]
    n_prog = x.shape[0]
    bidx = np.nonzero(kind != KIND_INTERIOR)[0]
    nx = np.select([kind[bidx] == KIND_LEFT, kind[bidx] == KIND_RIGHT], [-1.0, 1.0], 0.0)
    nz = np.select([kind[bidx] == KIND_BOTTOM, kind[bidx] == KIND_TOP], [-1.0, 1.0], 0.0)
    gx = x[bidx] + h * nx
    gz = z[bidx] + h * nz
    return NodeSet(x=np.concatenate([x, gx]), z=np.concatenate([z, gz]), n_prog=n_prog, kind=kind,
                   ghost_owner=bidx.astype(np.int32),
                   src=np.concatenate([np.arange(n_prog), -np.ones(bidx.shape[0], np.int64)]).astype(np.int32),
                   period_x=W if periodic_x else 0.0, h=h, layout="scattered", domain=(x0, x1, z0, z1))


# ----------------------------------------------------------------------------
# Initial states (closed forms of Sec. 6).  Fields are stacked [u, w, theta', pi'].
# ----------------------------------------------------------------------------

def pibar(z):
    """Hydrostatic background Exner pressure, 1 - g z / (c_p T_s) (Sec. 6.3)."""
    return 1.0 - G * np.asarray(z) / (CP * THETA_BAR)


def density_current_state(nodes: NodeSet, amp: float = -15.0, xc: float = 0.0, zc: float = 3000.0,
                          xr: float = 4000.0, zr: float = 2000.0) -> np.ndarray:
    """Straka cold bubble: T' = amp/2 (1 + cos(pi r)) for r <= 1, theta' = T'/pibar
    (Sec. 6.3); u = w = pi' = 0.  Returns float64 [4, n_all] (ghosts 0)."""
    x, z = nodes.x, nodes.z
    r = np.sqrt(((x - xc) / xr) ** 2 + ((z - zc) / zr) ** 2)
    tp = np.where(r <= 1.0, 0.5 * amp * (1.0 + np.cos(np.pi * r)), 0.0)
    U = np.zeros((4, nodes.n_all))
    U[2] = tp / pibar(z)
    U[:, nodes.n_prog:] = 0.0
    return U


def warm_bubble_state(nodes: NodeSet, amp: float = 2.0, xc: float = 10000.0, zc: float = 2000.0,
                      R: float = 2000.0) -> np.ndarray:
    """Warm bubble theta' = amp cos^2(pi r / (2R)) for r <= R; u = w = pi' = 0."""
    r = np.hypot(nodes.x - xc, nodes.z - zc)
    U = np.zeros((4, nodes.n_all))
    U[2] = np.where(r <= R, amp * np.cos(np.pi * r / (2.0 * R)) ** 2, 0.0)
    U[:, nodes.n_prog:] = 0.0
    return U


def translating_current_state(nodes: NodeSet, ubar: float = 20.0, xc: float = 18000.0) -> np.ndarray:
    """Translating density current (Sec. 6.3.2): the cold bubble of Sec. 6.3
    centred at x = 18 km in the 36 km periodic domain, carried by a uniform
    background wind ubar = 20 m/s held in u (a uniform u is a steady solution of
    the unforced equations, so u keeps the full velocity).  After 900 s the
    current has moved 18 km and its two fronts face each other about x = 18 km."""
    U = density_current_state(nodes, xc=xc)
    U[0, :nodes.n_prog] = ubar
    return U


def cone_bubble_state(nodes: NodeSet, amp: float = 2.0, xc: float = 5000.0, zc: float = 3000.0,
                      R: float = 1500.0) -> np.ndarray:
    """Rising thermal bubble of Sec. 6.4: the C0 cone theta' = amp max(0, 1 - r/R),
    R = 1.5 km at (5, 3) km; u = w = pi' = 0."""
    r = np.hypot(nodes.x - xc, nodes.z - zc)
    U = np.zeros((4, nodes.n_all))
    U[2] = amp * np.maximum(0.0, 1.0 - r / R)
    U[:, nodes.n_prog:] = 0.0
    return U


def cosine_bell(x, y, xc=0.25, yc=0.25, radius=0.15):
    """Cosine bell (1 + cos(pi rt))/2 for rt = dist / radius <= 1 (Sec. 6.1)."""
    rt = np.hypot(np.asarray(x) - xc, np.asarray(y) - yc) / radius
    return np.where(rt <= 1.0, 0.5 * (1.0 + np.cos(np.pi * rt)), 0.0)


def deformational_velocity(x, y):
    """Spatial factors of the deformational shear flow
    u = sin^2(pi x) sin(2 pi y) c(t), v = -sin^2(pi y) sin(2 pi x) c(t),
    c(t) = cos(pi t / T)."""
    x = np.asarray(x)
    y = np.asarray(y)
    return (np.sin(np.pi * x) ** 2 * np.sin(2 * np.pi * y),
            -np.sin(np.pi * y) ** 2 * np.sin(2 * np.pi * x))


def vortex_flow_parts(x, y, T=1.0):
    """The vortex flow of Sec. 6.1 split into time-separable parts.

    u_theta(r, t) = (4 pi r / T) [1 - cos(2 pi t / T) q(r)] with
    q = (1 - (4r)^6) / (1 + (4r)^6), u = u_theta sin(theta),
    v = -u_theta cos(theta), r sin(theta) = y - 1/2, r cos(theta) = x - 1/2
    (theta taken in the quadrant of (x - 1/2, y - 1/2)).  Hence
    (u, v) = c_1(t) (U_1, V_1) + c_2(t) (U_2, V_2) with the solid-body rotation
    U_1 = 4 pi (y - 1/2) / T, V_1 = -4 pi (x - 1/2) / T, c_1 = 1, and
    (U_2, V_2) = q (U_1, V_1), c_2 = -cos(2 pi t / T).
    Returns ([(U_1, V_1), (U_2, V_2)], [(a, b, m)] per part) with
    c_k(t) = a + b cos(m pi t / T)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    r = np.hypot(x - 0.5, y - 0.5)
    s6 = (4.0 * r) ** 6
    q = (1.0 - s6) / (1.0 + s6)
    U1 = 4.0 * np.pi * (y - 0.5) / T
    V1 = -4.0 * np.pi * (x - 0.5) / T
    return [(U1, V1), (q * U1, q * V1)], [(1.0, 0.0, 0.0), (0.0, -1.0, 2.0)]


def vortex_bell(x, y):
    """Initial scalar of the vortex-flow test (Sec. 6.1): the cosine bell
    (1 + cos(pi rt))/2 with rt = 5 |(x, y) - (0.3, 0.5)|, i.e. radius 0.2."""
    return cosine_bell(x, y, xc=0.3, yc=0.5, radius=0.2)


def perturbed_density_current(nodes: NodeSet, seed: int) -> np.ndarray:
    """Density current with seeded +/-10% amplitude and centre perturbations."""
    rng = np.random.default_rng(seed)
    a = -15.0 * (1.0 + rng.uniform(-0.1, 0.1))
    xc = 0.0 + 4000.0 * rng.uniform(-0.1, 0.1)
    zc = 3000.0 * (1.0 + rng.uniform(-0.1, 0.1))
    return density_current_state(nodes, amp=a, xc=xc, zc=zc)


# ----------------------------------------------------------------------------
# Batched ensembles of density-current runs of uneven size
# ----------------------------------------------------------------------------

# (stencil size, polynomial degree) choices of ensemble members, with the
# hyperviscosity of Sec. 5.3 and dt = h/400 (n = 21 is left out: the RK4
# amplification of its worst linear mode exceeds 1.09 at 800 m)
ENSEMBLE_STENCILS = ((31, 3), (37, 4), (45, 4), (56, 5), (75, 5))

# (layout, n, l) pairs the draw skips because those runs blow up before 900 s:
# on the Cartesian lattice n = 75 with l = 5 has a real growing mode of the
# operator linearised about rest at 400 m (RK4 amplification 1.17 per step)
# and goes non-finite at every spacing from 100 to 400 m with every
# hyperviscosity constant from 2^-6 to 2^-3 and with dt = h/500.
ENSEMBLE_UNSTABLE = (("cart", 75, 5),)

# Hyperviscosity constant of Sec. 5.3 per (layout, n, l); 2^-6 elsewhere.  The
# Cartesian n = 31, l = 3 member goes non-finite near t = 630 s at 50 m with
# 2^-6 (and with dt = h/500) and runs to 900 s with 2^-5 or 2^-4.
ENSEMBLE_GAMMA_C = {("cart", 31, 3): 2.0 ** -5}
ENSEMBLE_DEFAULT_GAMMA_C = 2.0 ** -6


@dataclasses.dataclass
class EnsembleMember:
    nodes: NodeSet
    n: int          # stencil size
    l: int          # polynomial degree
    dt: float
    n_steps: int
    U0: np.ndarray  # float64 [4, n_all] initial state
    seed: int
    gamma_c: float = ENSEMBLE_DEFAULT_GAMMA_C   # hyperviscosity constant (Sec. 5.3)


def density_current_member(h, layout, n, l, seed, t_end=900.0):
    """One ensemble member: the density current at spacing h on a Cartesian,
    hexagonal or scattered layout, with the seeded +/-10% perturbation of its
    amplitude and centre, stepped with dt = h/400 (Sec. 6.3 table) to t_end,
    with the hyperviscosity constant of its (layout, n, l) (ENSEMBLE_GAMMA_C)."""
    if layout == "scattered":
        nodes = poisson_disk_nodes(-25600.0, 25600.0, 0.0, 6400.0, h, seed=seed, periodic_x=True)
    else:
        nodes = density_current_nodes(h, layout=layout)
    dt = h / 400.0
    return EnsembleMember(nodes=nodes, n=n, l=l, dt=dt, n_steps=int(round(t_end / dt)),
                          U0=perturbed_density_current(nodes, seed), seed=seed,
                          gamma_c=ENSEMBLE_GAMMA_C.get((layout, n, l), ENSEMBLE_DEFAULT_GAMMA_C))


def ensemble_members(n_runs=256, seed=0, spacings=(50.0, 100.0, 200.0, 400.0),
                     layouts=("cart", "hex", "scattered"), stencils=ENSEMBLE_STENCILS, t_end=900.0):
    """Seeded draw of ensemble members: spacing, layout, stencil size and
    perturbation of each run.  The stencil is drawn among the choices that
    are stable on the drawn layout (ENSEMBLE_UNSTABLE)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_runs):
        h = float(spacings[rng.integers(len(spacings))])
        layout = str(layouts[rng.integers(len(layouts))])
        ok = [s for s in stencils if (layout,) + tuple(s) not in ENSEMBLE_UNSTABLE]
        n, l = ok[rng.integers(len(ok))]
        out.append(density_current_member(h, layout, n, l, seed=seed * 100003 + r, t_end=t_end))
    return out


# ----------------------------------------------------------------------------
# Nested lattices for the learned coarse-grid correction
# ----------------------------------------------------------------------------

def nested_density_current(h_coarse: float, ratio: int):
    """Coarse and fine hexagonal density-current lattices with every coarse node
    on a fine node: the coarse lattice keeps its fitted row count R_c, the
    fine one uses ratio * R_c rows and ratio times the columns (an odd coarse
    row's half-column shift is ratio/2 fine columns, so ratio is even).
    Returns (coarse, fine, restrict) with restrict[i] the fine node of coarse
    prognostic node i (restriction by injection)."""
    if ratio % 2:
        raise ValueError("the nesting ratio must be even")
    coarse = density_current_nodes(h_coarse)
    Rc = len(np.unique(coarse.z[:coarse.n_prog])) - 1   # coarse row intervals
    fine = lattice_nodes("hex", -25600.0, 25600.0, 0.0, 6400.0, h_coarse / ratio, True, rows=ratio * Rc)
    key = {(round(a, 6), round(b, 6)): j for j, (a, b) in enumerate(zip(fine.x[:fine.n_prog], fine.z[:fine.n_prog]))}
    restrict = np.array([key[(round(a, 6), round(b, 6))]
                         for a, b in zip(coarse.x[:coarse.n_prog], coarse.z[:coarse.n_prog])], np.int64)
    return coarse, fine, restrict


def restriction_average(coarse: NodeSet, fine: NodeSet, inject: np.ndarray, radius: float, sigma: float):
    """Low-pass restriction from fine to coarse prognostic nodes: a Gaussian
    average (width sigma) over the fine prognostic nodes within ``radius`` of
    each coarse node (minimum image in periodic x), weights normalised to 1.
    Returns (idx [n_c, m], w [n_c, m]) padded with zero weights."""
    P = fine.period_x
    xf, zf = fine.x[:fine.n_prog], fine.z[:fine.n_prog]
    rows_i, rows_w = [], []
    for c in range(coarse.n_prog):
        dx = xf - coarse.x[c]
        if P > 0:
            dx = np.where(dx > 0.5 * P, dx - P, np.where(dx < -0.5 * P, dx + P, dx))
        d2 = dx * dx + (zf - coarse.z[c]) ** 2
        sel = np.nonzero(d2 <= radius * radius)[0]
        w = np.exp(-0.5 * d2[sel] / (sigma * sigma))
        rows_i.append(sel)
        rows_w.append(w / w.sum())
    m = max(len(r) for r in rows_i)
    idx = np.zeros((coarse.n_prog, m), np.int64)
    wt = np.zeros((coarse.n_prog, m))
    for c, (ii, ww) in enumerate(zip(rows_i, rows_w)):
        idx[c, :len(ii)] = ii
        idx[c, len(ii):] = inject[c]
        wt[c, :len(ii)] = ww
    return idx, wt


def learned_correction_seeds(n_seeds=64, seed=5):
    """Seeds of the perturbed density currents of the learned-correction data
    set; the last eighth are held out for testing."""
    return [int(seed * 1000 + s) for s in range(n_seeds)]
