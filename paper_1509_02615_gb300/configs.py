"""The five workloads of this package: node sets, method parameters, initial
states, time steps and end times (synthetic, seeded; the paper's cases are
closed-form, so no data set is involved).

  advection        scalar transport in the deformational shear flow on the
                   unit square (Sec. 6.1 method; flow, bell and T = 5 of the
                   task), Cartesian 64 x 64 + 4 reflected layers, r^7 + deg 4,
                   n = 37, -gamma Delta^4 from r^9, dt = T/1000, FP64
  density_current  Sec. 6.3 at hexagonal 100 m, r^7 + deg 4, n = 37, Delta^3,
                   mu = 75, dt = 0.25 s to 900 s
  bubble           warm bubble (+2 K cos^2, R = 2 km at (10, 2) km) in a
                   walled [0, 20] x [0, 10] km box, Poisson-disk nodes at 25 m,
                   r^9 + deg 5, n = 56, Delta^3 from r^9, mu = 10,
                   dt = 1/16 s to 1000 s, FP64 weights in FP32
  vortex           Sec. 6.1's own test: the cosine bell (radius 0.2 at
                   (0.3, 0.5)) in the reversing vortex flow, T = 1, on reflected
                   Cartesian or hexagonal nodes, dt = h/15 to t = T; "paper":
                   r^9 + deg 4 with -gamma Delta^4; "r3": r^3 + deg 5 with
                   -gamma Delta^3 from r^7 (the convergence study)
  translating      Sec. 6.3.2: the density current in a periodic [0, 36] km
                   domain carried by a 20 m/s background wind, r^7 + deg 4,
                   n = 37, Delta^3, mu = 75, dt = h/400 to 900 s
  rising_bubble    Sec. 6.4: C0 cone bubble (2 K, R = 1.5 km at (5, 3) km) in
                   a walled [0, 10]^2 km box, Cartesian, hexagonal or
                   scattered nodes, r^7 + deg 4, n = 37, Delta^3, mu = 10,
                   dt = h/400 to 1100 s
  ensemble         256 density-current members (inputs.ensemble_members)
  learned          400 m coarse runs corrected by an MLP trained on fine runs
                   (learned.py)
"""
from __future__ import annotations

import dataclasses

from . import inputs as inp


@dataclasses.dataclass
class Workload:
    name: str
    nodes: inp.NodeSet
    params: dict          # keyword arguments of rbffd.ns_problem / advection_problem
    U0: object            # float64 [F, n_all] (advection: [n_prog])
    dt: float
    n_steps: int


def advection(m: int = 64) -> Workload:
    nodes = inp.unit_square_mirrored(m)
    U0 = inp.cosine_bell(nodes.x[:nodes.n_prog], nodes.z[:nodes.n_prog])
    return Workload("advection", nodes, dict(n=37, p=7, l=4, hv_k=4, hv_p=9, gamma_c=2.0 ** -14, T=5.0), U0,
                    5.0 / 1000.0, 1000)


def density_current(h: float = 100.0, layout: str = "hex") -> Workload:
    nodes = inp.density_current_nodes(h, layout=layout)
    return Workload("density_current", nodes, dict(n=37, p=7, l=4, hv_k=3, mu=75.0, gamma_c=2.0 ** -6),
                    inp.density_current_state(nodes), h / 400.0, int(round(900.0 * 400.0 / h)))


# Hyperviscosity constant of the bubble: with c = 2^-6 a corner of the
# scattered walled node set has a linear mode outside RK4's stability region
# (|R| = 1.009 per step at 500 m); c = 2^-4 damps it (|R| <= 1.00003).
BUBBLE_GAMMA_C = 2.0 ** -4
BUBBLE_METHOD = dict(n=56, p=9, l=5, hv_k=3, hv_p=9, mu=10.0, gamma_c=BUBBLE_GAMMA_C)


def bubble(h: float = 25.0, seed: int = 1, t_end: float = 1000.0) -> Workload:
    nodes = inp.poisson_disk_nodes(0.0, 20000.0, 0.0, 10000.0, h, seed=seed)
    return Workload("bubble", nodes, dict(BUBBLE_METHOD), inp.warm_bubble_state(nodes), h / 400.0,
                    int(round(t_end * 400.0 / h)))


# Hyperviscosity constant of the translating current on Cartesian nodes at
# 50 m and finer: with c = 2^-6 and dt = h/400 the FP64 run goes non-finite
# near t = 540 s (the resolved current's outflow reaches 56 m/s, and the
# acoustic modes carried by it leave RK4's stability region); c = 2^-5 runs to
# 900 s, as does c = 2^-6 with dt = h/500.  Hexagonal nodes and coarser
# Cartesian nodes keep c = 2^-6.
TRANSLATING_CART_FINE_GAMMA_C = 2.0 ** -5


def translating(h: float = 100.0, layout: str = "hex") -> Workload:
    nodes = inp.translating_current_nodes(h, layout)
    c = TRANSLATING_CART_FINE_GAMMA_C if (layout == "cart" and h <= 50.0) else 2.0 ** -6
    return Workload("translating", nodes, dict(n=37, p=7, l=4, hv_k=3, mu=75.0, gamma_c=c),
                    inp.translating_current_state(nodes), h / 400.0, int(round(900.0 * 400.0 / h)))


def rising_bubble(h: float = 100.0, layout: str = "hex", seed: int = 1) -> Workload:
    nodes = inp.rising_bubble_nodes(h, layout, seed=seed)
    return Workload("rising_bubble", nodes, dict(n=37, p=7, l=4, hv_k=3, mu=10.0, gamma_c=2.0 ** -6),
                    inp.cone_bubble_state(nodes), h / 400.0, int(round(1100.0 * 400.0 / h)))


# "paper": the Sec. 6.1 figure's r^9 + deg 4 with the printed -2^-14 Delta^4.
# "r3": the convergence study's r^3 + deg 5 with Delta^3 (from r^7, since
# Delta^3 r^3 is singular); c = 2^-10 puts gamma = c h^5 at 3e-12 (h = 0.02) to
# 3e-15 (h = 0.005), near the O(1e-12..1e-14) the paper states, and damps the
# modes that the walls' inflow stretches (with 2^-14 they grow at 13-26 per
# unit time, rising as h shrinks; with 2^-10 at most 0.9).
VORTEX_METHODS = {
    "paper": dict(n=37, p=9, l=4, hv_k=4, hv_p=9, gamma_c=2.0 ** -14),
    "r3": dict(n=37, p=3, l=5, hv_k=3, hv_p=7, gamma_c=2.0 ** -10),
}


def vortex(h: float = 0.005, layout: str = "hex", method: str = "paper") -> Workload:
    nodes = inp.unit_square_hex_mirrored(h) if layout == "hex" else inp.unit_square_mirrored(int(round(1.0 / h)) + 1)
    U0 = inp.vortex_bell(nodes.x[:nodes.n_prog], nodes.z[:nodes.n_prog])
    dt = h / 15.0
    return Workload("vortex", nodes, dict(VORTEX_METHODS[method], T=1.0, flow="vortex"), U0, dt,
                    int(round(1.0 / dt)))
