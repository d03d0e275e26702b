"""RBF-FD weights from the augmented PHS + polynomial system (oracle; test
infrastructure).

Sec. 3, Eq. (weights): for a stencil x_1..x_n around the centre x_c, solve

    [ A   P ] [ w      ]   [ L phi(||x - x_j||) at x_c ]
    [ P^T 0 ] [ lambda ] = [ L p_k(x) at x_c           ]

with A_ij = ||x_i - x_j||^p (odd PHS, p = 2m + 1) and P_jk = p_k(x_j) over all
2D monomials of degree <= l.  w_1..w_n is one row of the differentiation
matrix; lambda is discarded.

The system is written in shifted and scaled coordinates xi = (x - x_c)/s with
s = max_j ||x_j - x_c|| and the weights are rescaled by s^-order afterwards
(exact in real arithmetic; it keeps the matrix well scaled).  Operators:

  dx, dz     first derivatives               L r^p = p r^(p-2) (x_c - x_j)
  dxx, dzz   second derivatives              p r^(p-2) + p(p-2) r^(p-4) dx^2
  lap        Laplacian, Eq. (laplacian)      p (p + d - 2) r^(p-2), d = 2
  hv         Delta^k by repeating Eq. (laplacian) k times (Sec. 5.3)

Each function restates the operator's definition; the solve is one library
call (numpy.linalg.solve, LAPACK partial-pivoting LU) per stencil.
"""
import math

import numpy as np

from .stencils import min_image

OPS = ("dx", "dz", "lap", "hv", "dxx", "dzz")


def monomials(l):
    """All 2D monomial exponents (a, b) with a + b <= l, by degree."""
    return [(d - b, b) for d in range(l + 1) for b in range(d + 1)]


def op_order(op, k):
    return {"dx": 1, "dz": 1, "lap": 2, "dxx": 2, "dzz": 2, "hv": 2 * k}[op]


def phs_applied(op, p, k, dx, dz):
    """L applied to phi(||x - x_j||) = ||x - x_j||^p and evaluated at x = x_c,
    with (dx, dz) = x_c - x_j.  p odd, p >= 2k + 1 for hv (Sec. 5.3)."""
    r = np.hypot(dx, dz)
    with np.errstate(divide="ignore", invalid="ignore"):
        if op == "dx":
            v = p * r ** (p - 2) * dx
        elif op == "dz":
            v = p * r ** (p - 2) * dz
        elif op == "lap":
            v = p * p * r ** (p - 2)
        elif op == "dxx":
            v = p * r ** (p - 2) + p * (p - 2) * r ** (p - 4) * dx * dx
        elif op == "dzz":
            v = p * r ** (p - 2) + p * (p - 2) * r ** (p - 4) * dz * dz
        elif op == "hv":
            c = 1.0
            q = p
            for _ in range(k):  # Delta r^q = q^2 r^(q-2) in 2D
                c *= q * q
                q -= 2
            v = c * r ** q
        else:
            raise ValueError(op)
    return np.where(r == 0.0, 0.0, v)


def poly_applied(op, k, a, b):
    """L applied to xi^a eta^b, evaluated at the origin."""
    if op == "dx":
        return 1.0 if (a, b) == (1, 0) else 0.0
    if op == "dz":
        return 1.0 if (a, b) == (0, 1) else 0.0
    if op == "lap":
        return 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0
    if op == "dxx":
        return 2.0 if (a, b) == (2, 0) else 0.0
    if op == "dzz":
        return 2.0 if (a, b) == (0, 2) else 0.0
    if op == "hv":
        # Delta^k = sum_i C(k,i) d^{2i}/dxi^{2i} d^{2(k-i)}/deta^{2(k-i)}
        if a % 2 or b % 2 or a + b != 2 * k:
            return 0.0
        i = a // 2
        return float(math.comb(k, i) * math.factorial(a) * math.factorial(b))
    raise ValueError(op)


def _systems(x, z, idx, p, l, period_x):
    """Scaled augmented matrices [B, S, S] of the stencils ``idx`` [B, n]
    (centre first), with the scaled offsets and the scales s."""
    idx = np.asarray(idx)
    xc, zc = x[idx[:, :1]], z[idx[:, :1]]
    ex = min_image(x[idx] - xc, period_x)
    ez = z[idx] - zc
    s = np.max(np.hypot(ex, ez), axis=1)
    xi, eta = ex / s[:, None], ez / s[:, None]
    B, n = idx.shape
    mono = monomials(l)
    S = n + len(mono)
    A = np.zeros((B, S, S))
    A[:, :n, :n] = np.hypot(xi[:, :, None] - xi[:, None, :], eta[:, :, None] - eta[:, None, :]) ** p
    for c, (a, b) in enumerate(mono):
        A[:, :n, n + c] = xi ** a * eta ** b
        A[:, n + c, :n] = xi ** a * eta ** b
    return A, xi, eta, s


def all_weights(x, z, idx, p, l, ops, k=0, period_x=0.0, batch=2048):
    """Weights [len(ops), N, n] for every stencil row of ``idx`` [N, n]
    (centre first): one augmented solve per stencil, Eq. (weights)."""
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    idx = np.asarray(idx)
    N, n = idx.shape
    mono = monomials(l)
    out = np.empty((len(ops), N, n))
    for b0 in range(0, N, batch):
        A, xi, eta, s = _systems(x, z, idx[b0:b0 + batch], p, l, period_x)
        B = A.shape[0]
        rhs = np.zeros((B, A.shape[1], len(ops)))
        for o, op in enumerate(ops):
            rhs[:, :n, o] = phs_applied(op, p, k, 0.0 - xi, 0.0 - eta)
            for c, (a, bb) in enumerate(mono):
                rhs[:, n + c, o] = poly_applied(op, k, a, bb)
        sol = np.linalg.solve(A, rhs)
        for o, op in enumerate(ops):
            out[o, b0:b0 + B] = sol[:, :n, o] / s[:, None] ** op_order(op, k)
    return out


def stencil_weights(x, z, sten, p, l, ops, k=0, period_x=0.0):
    """Weights [len(ops), n] of one stencil (centre first)."""
    return all_weights(x, z, np.asarray(sten)[None, :], p, l, ops, k, period_x)[:, 0, :]


def condition_number(x, z, sten, p, l, period_x=0.0):
    """2-norm condition number of the scaled augmented matrix of one stencil."""
    A = _systems(np.asarray(x, np.float64), np.asarray(z, np.float64), np.asarray(sten)[None, :], p, l, period_x)[0]
    return float(np.linalg.cond(A[0]))


def _weights_block(args):
    return all_weights(*args)


def all_weights_pool(x, z, idx, p, l, ops, k=0, period_x=0.0, workers=1):
    """``all_weights`` over contiguous blocks of stencil rows, one block at a
    time per worker process (spawned, so that a parent holding a CUDA context
    is safe).  Every stencil is solved on its own, so the result is the
    serial one, bit for bit; only the wall time changes."""
    idx = np.asarray(idx)
    if workers <= 1 or idx.shape[0] < 4096:
        return all_weights(x, z, idx, p, l, ops, k, period_x)
    import multiprocessing as mp
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    cuts = np.linspace(0, idx.shape[0], 4 * workers + 1).astype(np.int64)
    jobs = [(x, z, idx[a:b], p, l, list(ops), k, period_x) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_weights_block, jobs)
    return np.concatenate(parts, axis=1)
