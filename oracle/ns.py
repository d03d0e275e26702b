"""2D compressible Navier-Stokes in perturbation form (oracle; test
infrastructure).

Sec. 6.2, Eqs. uEq-piEq, fields U = [u, w, theta', pi'] about the hydrostatic
base theta_bar = T_s, pibar(z) = 1 - g z / (c_p T_s) (Sec. 6.3):

  u_t  = -u u_x - w u_z - c_p (theta_bar + theta') pi'_x + mu Lap u
  w_t  = -u w_x - w w_z - c_p (theta_bar + theta') pi'_z + g theta'/theta_bar + mu Lap w
  th_t = -u th_x - w th_z + mu Lap theta'
  pi_t = -u pi_x - w (dpibar/dz + pi_z) - (R_d/c_v)(pibar + pi')(u_x + w_z)

plus hyperviscosity (-1)^(k+1) gamma Delta^k on every field (Sec. 5.3; the
sign makes it damp).  Boundary treatment (Sec. 5.2, Eq. bcEqn): one ghost per
boundary node; the ghost values solve W_G u_G = b - W_I u_I - W_B u_B, the
rows being the boundary condition's operator at the boundary nodes:

  top/bottom (Sec. 6.3):  u_z = 0, w_zz = 0 (w = 0 held), theta'_z = 0,
                          pi'_z = g theta' / (c_p theta_bar (theta_bar + theta'))
  left/right (Sec. 6.4):  u_xx = 0 (u = 0 held), w_x = 0, theta'_x = 0, pi'_x = 0

The right-hand side uses the plain DM product sum_j w_ij f_j.  Time stepping
is classical RK4 (Sec. 6, method of lines).
"""
import numpy as np
import scipy.sparse.linalg as spla

from paper_1509_02615_gb300 import inputs as inp

from .operators import Discretisation

# operator of the boundary condition per field for (bottom/top, left/right)
BC_OPS = {"tb": ("dz", "dzz", "dz", "dz"), "lr": ("dxx", "dx", "dx", "dx")}


class NSOracle:
    def __init__(self, nodes, n=37, p=7, l=4, hv_k=3, hv_p=None, mu=75.0, gamma_c=2.0 ** -6,
                 gamma=None, theta_bar=inp.THETA_BAR, stencil_order="nearest", workers=1):
        """``stencil_order`` "reversed" lists each stencil's neighbours
        farthest first (the same method up to rounding: the oracle's own
        spread); ``workers`` > 1 solves the weights in that many processes."""
        self.nodes = nodes
        self.n_prog = nodes.n_prog
        self.disc = Discretisation(nodes, n, p, l, ops=("dx", "dz", "lap", "dxx", "dzz"), hv_k=hv_k, hv_p=hv_p,
                                   stencil_order=stencil_order, workers=workers)
        self.D = self.disc.D
        self.mu = mu
        self.hv_k = hv_k
        if gamma is None:
            gamma = gamma_c * nodes.h ** (2 * hv_k - 1)
        self.gamma = gamma
        self.hv_coef = (-1.0) ** (hv_k + 1) * gamma if hv_k > 0 else 0.0
        self.theta_bar = theta_bar
        zp = nodes.z[:self.n_prog]
        self.pibar = 1.0 - inp.G * zp / (inp.CP * theta_bar)
        self.dpibar = -inp.G / (inp.CP * theta_bar)
        kind = nodes.kind
        self.w_dirichlet = (kind == inp.KIND_BOTTOM) | (kind == inp.KIND_TOP)
        self.u_dirichlet = (kind == inp.KIND_LEFT) | (kind == inp.KIND_RIGHT)
        self._build_ghost_systems()

    # -- Sec. 5.2: ghost systems -------------------------------------------------
    def _build_ghost_systems(self):
        nodes = self.nodes
        self.owner = nodes.ghost_owner.astype(np.int64)
        ng = self.owner.shape[0]
        self.ghost_sys = []
        if ng == 0:
            return
        wall = np.where(np.isin(nodes.kind[self.owner], (inp.KIND_LEFT, inp.KIND_RIGHT)), "lr", "tb")
        for f in range(4):
            rows = []
            for r in range(ng):
                op = BC_OPS[wall[r]][f]
                rows.append(self.D[op][self.owner[r]])
            import scipy.sparse as sp
            W = sp.vstack(rows).tocsc()
            WG = W[:, self.n_prog:]
            WP = W[:, :self.n_prog]
            self.ghost_sys.append((spla.splu(WG.tocsc()), WP.tocsr(), W.tocsr()))
        self.ghost_wall = wall

    def ghost_rhs(self, U):
        """Right-hand side b of the boundary conditions per field [4, N_G]."""
        ng = self.owner.shape[0]
        b = np.zeros((4, ng))
        tb = self.ghost_wall == "tb"
        th = U[2, self.owner]
        b[3] = np.where(tb, inp.G * th / (inp.CP * self.theta_bar * (self.theta_bar + th)), 0.0)
        return b

    def fill_ghosts(self, U):
        """Solve W_G u_G = b - W_I u_I - W_B u_B for every field; writes U's
        ghost entries in place."""
        if not self.ghost_sys:
            return U
        b = self.ghost_rhs(U)
        for f in range(4):
            lu, WP, _ = self.ghost_sys[f]
            r = b[f] - WP @ U[f, :self.n_prog]
            U[f, self.n_prog:] = lu.solve(r)
        return U

    def bc_residual(self, U):
        """W u - b at the boundary rows, per field [4, N_G] (zero after fill)."""
        b = self.ghost_rhs(U)
        return np.stack([self.ghost_sys[f][2] @ U[f] - b[f] for f in range(4)])

    # -- Eqs. uEq-piEq ------------------------------------------------------------
    def rhs(self, t, U):
        """Tendencies [4, n_prog] of the state U [4, n_all] (ghosts refilled)."""
        U = np.array(U, dtype=np.float64, copy=True)
        self.fill_ghosts(U)
        D = self.D
        u, w, th, pi = U
        up, wp, thp, pip = U[:, :self.n_prog]
        ux, uz = D["dx"] @ u, D["dz"] @ u
        wx, wz = D["dx"] @ w, D["dz"] @ w
        tx, tz = D["dx"] @ th, D["dz"] @ th
        px, pz = D["dx"] @ pi, D["dz"] @ pi
        cpth = inp.CP * (self.theta_bar + thp)
        du = -up * ux - wp * uz - cpth * px
        dw = -up * wx - wp * wz - cpth * pz + inp.G * thp / self.theta_bar
        dth = -up * tx - wp * tz
        dpi = -up * px - wp * (self.dpibar + pz) - (inp.RD / inp.CV) * (self.pibar + pip) * (ux + wz)
        if self.mu != 0.0:
            du = du + self.mu * (D["lap"] @ u)
            dw = dw + self.mu * (D["lap"] @ w)
            dth = dth + self.mu * (D["lap"] @ th)
        if self.hv_coef != 0.0:
            H = D["hv"]
            du = du + self.hv_coef * (H @ u)
            dw = dw + self.hv_coef * (H @ w)
            dth = dth + self.hv_coef * (H @ th)
            dpi = dpi + self.hv_coef * (H @ pi)
        dw = np.where(self.w_dirichlet, 0.0, dw)
        du = np.where(self.u_dirichlet, 0.0, du)
        return np.stack([du, dw, dth, dpi])

    def rk4_step(self, t, dt, U):
        """One classical RK4 step of the prognostic values; returns the new
        state [4, n_all] with ghosts filled for the new values."""
        return rk4_step(self.rhs, t, dt, U, self.n_prog, self.fill_ghosts)

    def run(self, U, t0, dt, n_steps):
        U = np.array(U, dtype=np.float64, copy=True)
        t = t0
        for _ in range(n_steps):
            U = self.rk4_step(t, dt, U)
            t += dt
        return U


def rk4_step(rhs, t, dt, U, n_prog, fill=None):
    """Classical fourth-order Runge-Kutta for dU/dt = rhs(t, U) on the first
    n_prog columns of U (the remaining columns are refilled by ``fill``)."""
    U = np.array(U, dtype=np.float64, copy=True)
    y0 = U[:, :n_prog].copy()

    def at(y):
        V = U.copy()
        V[:, :n_prog] = y
        return V

    k1 = rhs(t, at(y0))
    k2 = rhs(t + 0.5 * dt, at(y0 + 0.5 * dt * k1))
    k3 = rhs(t + 0.5 * dt, at(y0 + 0.5 * dt * k2))
    k4 = rhs(t + dt, at(y0 + dt * k3))
    V = at(y0 + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))
    if fill is not None:
        fill(V)
    return V


# -- diagnostics (Sec. 6.3 table) ---------------------------------------------------

def front_location(nodes, theta, level=-0.5):
    """Largest x >= 0 on the ground (z = 0 nodes) where theta' crosses ``level``,
    by linear interpolation between neighbouring ground nodes."""
    g = np.nonzero((nodes.z[:nodes.n_prog] == nodes.domain[2]))[0]
    order = np.argsort(nodes.x[g])
    xs, ts = nodes.x[g][order], theta[g][order]
    keep = xs >= 0.0
    xs, ts = xs[keep], ts[keep]
    below = np.nonzero(ts <= level)[0]
    if below.size == 0:
        return float("nan")
    i = below[-1]
    if i + 1 >= xs.shape[0]:
        return float(xs[i])
    t0, t1 = ts[i], ts[i + 1]
    return float(xs[i] + (level - t0) / (t1 - t0) * (xs[i + 1] - xs[i]))


def facing_fronts(nodes, theta, x_mid, level=-0.5):
    """Distances from x_mid to the nearest ground crossings of ``level`` on
    either side (Sec. 6.3.2 table: the two fronts of the translating current
    face each other about x = 18 km).  Returns (left, right) in metres, each by
    linear interpolation between neighbouring ground nodes."""
    g = np.nonzero(nodes.z[:nodes.n_prog] == nodes.domain[2])[0]
    order = np.argsort(nodes.x[g])
    xs, ts = nodes.x[g][order], theta[g][order]
    cold = ts <= level
    left = np.nonzero(cold & (xs < x_mid))[0]
    right = np.nonzero(cold & (xs > x_mid))[0]
    out = []
    for idx, step in ((left, 1), (right, -1)):
        if idx.size == 0:
            out.append(float("nan"))
            continue
        i = idx[-1] if step == 1 else idx[0]
        j = i + step                      # first warm node towards x_mid
        t0, t1 = ts[i], ts[j]
        xc = xs[i] + (level - t0) / (t1 - t0) * (xs[j] - xs[i])
        out.append(float(abs(x_mid - xc)))
    return tuple(out)


def bubble_height(nodes, theta, x_line, level=0.1, dz=1.0):
    """Height of the rising bubble (Sec. 6.4 table): the highest point of the
    ``level`` contour on the vertical line x = x_line.  theta' is interpolated
    to the line piecewise linearly on the Delaunay triangulation of the
    prognostic nodes, sampled every dz metres, and the top crossing refined by
    linear interpolation between samples."""
    from scipy.interpolate import LinearNDInterpolator
    n = nodes.n_prog
    f = LinearNDInterpolator(np.c_[nodes.x[:n], nodes.z[:n]], theta[:n])
    z0, z1 = nodes.domain[2], nodes.domain[3]
    zs = np.arange(z0, z1 + 0.5 * dz, dz)
    vals = f(np.full(zs.shape, x_line), zs)
    vals = np.where(np.isnan(vals), -np.inf, vals)
    above = np.nonzero(vals >= level)[0]
    if above.size == 0:
        return float("nan")
    i = above[-1]
    if i + 1 >= zs.shape[0]:
        return float(zs[i])
    return float(zs[i] + (vals[i] - level) / (vals[i] - vals[i + 1]) * dz)
