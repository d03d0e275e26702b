"""Flux-form scalar advection on reflected nodes (oracle; test infrastructure).

Sec. 6.1: psi_t = -(u psi)_x - (v psi)_y on the unit square.  Nodes near the
walls are reflected outside together with their values, so every boundary
stencil is symmetric and no boundary condition is needed; the boundary nodes
are stepped with the interior.  The velocity is evaluated at each stencil
node's own (possibly reflected) position:

  * deformational flow: u = U(x, y) c(t), v = V(x, y) c(t),
    c(t) = cos(pi t / T);
  * vortex flow (Sec. 6.1): u = u_theta(r, t) sin(theta),
    v = -u_theta(r, t) cos(theta),
    u_theta = (4 pi r / T) [1 - cos(2 pi t / T) (1 - (4r)^6) / (1 + (4r)^6)],
    r, theta the polar coordinates about (1/2, 1/2), written out here at
    every evaluation (not split into parts).

Hyperviscosity (-1)^(k+1) gamma Delta^k (Sec. 5.3) uses its own PHS exponent.

  psi_t(x_i) = -sum_j [Dx_ij u(x_j, t) + Dy_ij v(x_j, t)] psi(src(j))
               + (-1)^(k+1) gamma sum_j H_ij psi(src(j))
"""
import numpy as np

from paper_1509_02615_gb300 import inputs as inp

from .operators import Discretisation
from .ns import rk4_step


def vortex_velocity(x, y, t, T):
    """u, v of the vortex flow of Sec. 6.1 at time t (theta in the quadrant
    of (x - 1/2, y - 1/2); at r = 0 u_theta = 0)."""
    dx, dy = np.asarray(x) - 0.5, np.asarray(y) - 0.5
    r = np.hypot(dx, dy)
    theta = np.arctan2(dy, dx)
    ut = 4.0 * np.pi * r / T * (1.0 - np.cos(2.0 * np.pi * t / T) * (1.0 - (4.0 * r) ** 6) / (1.0 + (4.0 * r) ** 6))
    return ut * np.sin(theta), -ut * np.cos(theta)


class AdvectionOracle:
    def __init__(self, nodes, n=37, p=7, l=4, hv_k=4, hv_p=9, gamma_c=2.0 ** -14, gamma=None, T=5.0,
                 flow="deformational", stencil_order="nearest"):
        """``stencil_order`` "reversed" lists each stencil's neighbours
        farthest first (the same method up to rounding)."""
        self.nodes = nodes
        self.n_prog = nodes.n_prog
        self.T = T
        self.flow = flow
        self.disc = Discretisation(nodes, n, p, l, ops=("dx", "dz"), hv_k=hv_k, hv_p=hv_p,
                                   stencil_order=stencil_order)
        if gamma is None:
            gamma = gamma_c * nodes.h ** (2 * hv_k - 1)
        self.gamma = gamma
        self.hv_coef = (-1.0) ** (hv_k + 1) * gamma if hv_k > 0 else 0.0
        idx = self.disc.idx
        self.idx = idx
        if flow == "deformational":
            Uv, Vv = inp.deformational_velocity(nodes.x, nodes.z)
            # flux-form weights: -(Dx_ij U(x_j) + Dy_ij V(x_j)), columns at stencil nodes
            self.Wadv = -(self.disc.W["dx"] * Uv[idx] + self.disc.W["dz"] * Vv[idx])
        elif flow != "vortex":
            raise ValueError(flow)
        self.Whv = self.hv_coef * self.disc.W["hv"] if hv_k > 0 else np.zeros_like(self.disc.W["dx"])
        self.cols = nodes.src[idx]

    def velocity_factor(self, t):
        return np.cos(np.pi * t / self.T)

    def advection_weights(self, t):
        """-(Dx_ij u(x_j, t) + Dy_ij v(x_j, t)) for every stencil slot."""
        if self.flow == "deformational":
            return self.velocity_factor(t) * self.Wadv
        u, v = vortex_velocity(self.nodes.x, self.nodes.z, t, self.T)
        return -(self.disc.W["dx"] * u[self.idx] + self.disc.W["dz"] * v[self.idx])

    def rhs(self, t, psi):
        """psi_t at the prognostic nodes; psi is [1, n_prog] or [n_prog]."""
        y = np.asarray(psi, np.float64).reshape(-1)[:self.n_prog]
        g = y[self.cols]
        out = np.sum(self.advection_weights(t) * g, axis=1) + np.sum(self.Whv * g, axis=1)
        return out[None, :]

    def rk4_step(self, t, dt, psi):
        return rk4_step(self.rhs, t, dt, np.asarray(psi, np.float64).reshape(1, -1), self.n_prog)

    def run(self, psi, t0, dt, n_steps):
        y = np.asarray(psi, np.float64).reshape(1, -1)
        t = t0
        for _ in range(n_steps):
            y = self.rk4_step(t, dt, y)
            t += dt
        return y
