"""Flux-form scalar advection on reflected nodes (oracle; test infrastructure).

Sec. 6.1: psi_t = -(u psi)_x - (v psi)_y on the unit square.  Nodes near the
walls are reflected outside together with their values, so every boundary
stencil is symmetric and no boundary condition is needed; the boundary nodes
are stepped with the interior.  The velocity of the deformational flow is
u = U(x, y) c(t), v = V(x, y) c(t), c(t) = cos(pi t / T), evaluated at each
stencil node's own (possibly reflected) position.  Hyperviscosity
(-1)^(k+1) gamma Delta^k (Sec. 5.3) uses its own PHS exponent.

  psi_t(x_i) = -c(t) sum_j [Dx_ij U(x_j) + Dy_ij V(x_j)] psi(src(j))
               + (-1)^(k+1) gamma sum_j H_ij psi(src(j))
"""
import numpy as np

from paper_1509_02615_gb300 import inputs as inp

from .operators import Discretisation
from .ns import rk4_step


class AdvectionOracle:
    def __init__(self, nodes, n=37, p=7, l=4, hv_k=4, hv_p=9, gamma_c=2.0 ** -14, gamma=None, T=5.0):
        self.nodes = nodes
        self.n_prog = nodes.n_prog
        self.T = T
        self.disc = Discretisation(nodes, n, p, l, ops=("dx", "dz"), hv_k=hv_k, hv_p=hv_p)
        if gamma is None:
            gamma = gamma_c * nodes.h ** (2 * hv_k - 1)
        self.gamma = gamma
        self.hv_coef = (-1.0) ** (hv_k + 1) * gamma if hv_k > 0 else 0.0
        Uv, Vv = inp.deformational_velocity(nodes.x, nodes.z)
        idx = self.disc.idx
        # flux-form weights: -(Dx_ij U(x_j) + Dy_ij V(x_j)), columns at stencil nodes
        self.Wadv = -(self.disc.W["dx"] * Uv[idx] + self.disc.W["dz"] * Vv[idx])
        self.Whv = self.hv_coef * self.disc.W["hv"] if hv_k > 0 else np.zeros_like(self.Wadv)
        self.cols = nodes.src[idx]

    def velocity_factor(self, t):
        return np.cos(np.pi * t / self.T)

    def rhs(self, t, psi):
        """psi_t at the prognostic nodes; psi is [1, n_prog] or [n_prog]."""
        y = np.asarray(psi, np.float64).reshape(-1)[:self.n_prog]
        g = y[self.cols]
        out = self.velocity_factor(t) * np.sum(self.Wadv * g, axis=1) + np.sum(self.Whv * g, axis=1)
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
