"""Pins of the oracle's stencils and weights against what the paper and the
mathematics fix (no GPU).

* Appendix A: 37-node stencils are complete rings on Cartesian and hexagonal
  lattices (ring radii and multiplicities checked here).
* Eq. (weights) constraint rows: exact reproduction of every polynomial of
  degree <= l by every operator (to 1e-11 relative), checked against
  derivatives of polynomials computed by exact polynomial arithmetic.
* Brute force: on 10-node sets the weights equal L applied to the global
  PHS + polynomial interpolant, whose derivative is taken by complex-step
  differentiation (dx, dz) or a 4th-order difference (Laplacian).
* Sec. 4, Fig. r3_vs_r7_poly: the error of d/dx of 1 + sin 4x + cos 3x + sin 2y
  on a 37-node hexagonal stencil falls as h^l for r^3 and r^7.
"""
import math

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from oracle import stencils as st
from oracle import weights as wt
from paper_1509_02615_gb300 import inputs as inp


def _torus(layout, h=1.0, n=16):
    return inp.lattice_nodes(layout, 0.0, n * h, 0.0, n * h, h, True)


@pytest.mark.parametrize("layout,rings", [
    ("hex", [(0.0, 1), (1.0, 6), (3.0, 6), (4.0, 6), (7.0, 12), (9.0, 6)]),
    ("cart", [(0.0, 1), (1.0, 4), (2.0, 4), (4.0, 4), (5.0, 8), (8.0, 4), (9.0, 4), (10.0, 8)]),
])
def test_37_node_stencils_are_complete_rings(layout, rings):
    nodes = inp.lattice_nodes(layout, 0.0, 20.0, 0.0, 20.0 * (math.sqrt(3) / 2 if layout == "hex" else 1.0),
                              1.0, True)
    c = nodes.n_prog // 2 + 3
    idx = st.knn(nodes.x, nodes.z, [c], 37, nodes.period_x)[0]
    d2 = st.sq_dist(nodes.x[c], nodes.z[c], nodes.x[idx], nodes.z[idx], nodes.period_x)
    got = np.round(d2, 6)
    vals, counts = np.unique(got, return_counts=True)
    assert [(float(v), int(k)) for v, k in zip(vals, counts)] == rings
    assert idx[0] == c


def test_knn_matches_full_sort_on_random_points():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 10, 60)
    z = rng.uniform(0, 3, 60)
    for period in (0.0, 10.0):
        idx = st.knn(x, z, np.arange(20), 9, period)
        for c in range(20):
            keys = []
            for j in range(60):
                dx = x[j] - x[c]
                if period > 0:
                    if dx > period / 2:
                        dx -= period
                    elif dx < -period / 2:
                        dx += period
                dz = z[j] - z[c]
                keys.append((dx * dx + dz * dz, j))
            assert [j for _, j in sorted(keys)[:9]] == list(idx[c])


# ---- exact polynomial arithmetic for L q --------------------------------------

def _poly_coeffs(a, b):
    C = np.zeros((a + 1, b + 1))
    C[a, b] = 1.0
    return C


def _apply(op, C, k):
    """Coefficients of L q for q given by 2D coefficient array C[i, j] of x^i z^j."""
    dx = lambda M: P.polyder(M, axis=0) if M.shape[0] > 1 else np.zeros((1, M.shape[1]))
    dz = lambda M: P.polyder(M, axis=1) if M.shape[1] > 1 else np.zeros((M.shape[0], 1))

    def lap(M):
        A, B = dx(dx(M)), dz(dz(M))
        out = np.zeros((max(A.shape[0], B.shape[0]), max(A.shape[1], B.shape[1])))
        out[:A.shape[0], :A.shape[1]] += A
        out[:B.shape[0], :B.shape[1]] += B
        return out

    if op == "dx":
        return dx(C)
    if op == "dz":
        return dz(C)
    if op == "dxx":
        return dx(dx(C))
    if op == "dzz":
        return dz(dz(C))
    if op == "lap":
        return lap(C)
    if op == "hv":
        for _ in range(k):
            C = lap(C)
        return C
    raise ValueError(op)


def _eval(C, x, z):
    return P.polyval2d(x, z, C)


@pytest.mark.parametrize("layout,p,l,ops,k", [
    ("hex", 7, 4, ["dx", "dz", "lap", "dxx", "dzz", "hv"], 3),
    ("cart", 7, 4, ["dx", "dz", "lap", "dxx", "dzz", "hv"], 3),
    ("hex", 9, 5, ["dx", "dz", "lap", "hv"], 3),
    ("hex", 7, 6, ["dx", "dz", "lap", "hv"], 2),
    ("cart", 3, 5, ["dx", "dz", "lap", "dzz"], 0),
    ("scattered", 9, 5, ["dx", "dz", "lap", "dxx", "hv"], 3),
])
def test_polynomial_reproduction(layout, p, l, ops, k):
    if layout == "scattered":
        nodes = inp.poisson_disk_nodes(0.0, 12.0, 0.0, 8.0, 1.0, seed=5)
        n = 56
    else:
        nodes = _torus(layout)
        n = 37
    rng = np.random.default_rng(1)
    if layout == "scattered":
        centers = rng.choice(nodes.n_prog, 12, replace=False)
    else:
        # interior stencils (degree 6 is unisolvent only on complete rings)
        zmid = 0.5 * (nodes.z.min() + nodes.z.max())
        pool = np.nonzero(np.abs(nodes.z[:nodes.n_prog] - zmid) < 3.0)[0]
        centers = rng.choice(pool, 12, replace=False)
    idx = st.knn(nodes.x, nodes.z, centers, n, nodes.period_x)
    W = wt.all_weights(nodes.x, nodes.z, idx, p, l, ops, k, nodes.period_x)
    for r, c in enumerate(centers):
        xc, zc = nodes.x[c], nodes.z[c]
        ex = st.min_image(nodes.x[idx[r]] - xc, nodes.period_x)
        ez = nodes.z[idx[r]] - zc
        s = np.max(np.hypot(ex, ez))
        # polynomials about an off-centre origin, scaled by the stencil size
        ox, oz = 0.3 * s, -0.2 * s
        X, Z = (ex - ox) / s, (ez - oz) / s
        for a in range(l + 1):
            for b in range(l + 1 - a):
                C = _poly_coeffs(a, b)
                vals = _eval(C, X, Z)
                for o, op in enumerate(ops):
                    order = wt.op_order(op, k)
                    exact = _eval(_apply(op, C, k), -ox / s, -oz / s) / s ** order
                    got = np.dot(W[o, r], vals)
                    scale = np.sum(np.abs(W[o, r] * vals)) + abs(exact) + 1e-300
                    assert abs(got - exact) <= 1e-11 * scale, (op, a, b, got, exact)


def _global_interpolant_derivative(xs, zs, f, p, l, xc, zc):
    """Global PHS + degree-l interpolant of f on the nodes, and its x-, z-
    derivatives and Laplacian at (xc, zc): complex step for the first
    derivatives, a fourth-order central difference for the Laplacian."""
    n = xs.shape[0]
    mono = [(d - b, b) for d in range(l + 1) for b in range(d + 1)]
    A = np.zeros((n + len(mono),) * 2)
    A[:n, :n] = np.hypot(xs[:, None] - xs[None, :], zs[:, None] - zs[None, :]) ** p
    for c, (a, b) in enumerate(mono):
        A[:n, n + c] = xs ** a * zs ** b
        A[n + c, :n] = xs ** a * zs ** b
    coef = np.linalg.solve(A, np.concatenate([f, np.zeros(len(mono))]))
    lam, cp = coef[:n], coef[n:]

    def s(x, z):
        r2 = (x - xs) ** 2 + (z - zs) ** 2
        val = np.sum(lam * np.where(r2 == 0, 0.0, r2) ** (p / 2.0))
        return val + sum(cp[c] * x ** a * z ** b for c, (a, b) in enumerate(mono))

    eps = 1e-30
    sx = s(xc + 1j * eps, zc + 0j).imag / eps
    sz = s(xc + 0j, zc + 1j * eps).imag / eps
    hh = 1e-3
    lap = 0.0
    for dxh, dzh in ((1, 0), (0, 1)):
        fm2 = s(xc - 2 * hh * dxh, zc - 2 * hh * dzh)
        fm1 = s(xc - hh * dxh, zc - hh * dzh)
        f0 = s(xc, zc)
        fp1 = s(xc + hh * dxh, zc + hh * dzh)
        fp2 = s(xc + 2 * hh * dxh, zc + 2 * hh * dzh)
        lap += (-fp2 + 16 * fp1 - 30 * f0 + 16 * fm1 - fm2) / (12 * hh * hh)
    return sx.real, sz.real, lap.real


@pytest.mark.parametrize("p,l", [(3, 1), (5, 2), (7, 2)])
def test_weights_equal_global_interpolant_derivative(p, l):
    rng = np.random.default_rng(10 + p)
    for trial in range(5):
        xs = rng.uniform(-1, 1, 10)
        zs = rng.uniform(-1, 1, 10)
        f = rng.normal(size=10)
        idx = np.arange(10)[None, :]
        W = wt.all_weights(xs, zs, idx, p, l, ["dx", "dz", "lap"], 0, 0.0)[:, 0, :]
        sx, sz, lap = _global_interpolant_derivative(xs, zs, f, p, l, xs[0], zs[0])
        assert abs(W[0] @ f - sx) <= 1e-12 * (np.abs(W[0] * f).sum())
        assert abs(W[1] @ f - sz) <= 1e-12 * (np.abs(W[1] * f).sum())
        # the difference quotient carries ~1e-9 truncation and rounding error;
        # it needs r^p to be C^4 at the centre node, so p >= 5
        if p >= 5:
            assert abs(W[2] @ f - lap) <= 1e-7 * (np.abs(W[2] * f).sum())


@pytest.mark.parametrize("p", [3, 7])
def test_ddx_convergence_order_is_l(p):
    """Fig. r3_vs_r7_poly: the slope of the d/dx error is the polynomial degree."""
    f = lambda x, y: 1 + np.sin(4 * x) + np.cos(3 * x) + np.sin(2 * y)
    fx = lambda x, y: 4 * np.cos(4 * x) - 3 * np.sin(3 * x)
    base = _torus("hex", 1.0, 16)
    c = base.n_prog // 2 + 5
    idx = st.knn(base.x, base.z, [c], 37, base.period_x)[0]
    ex = st.min_image(base.x[idx] - base.x[c], base.period_x)
    ez = base.z[idx] - base.z[c]
    # a fixed small jitter of the non-centre nodes breaks the lattice symmetry
    # that would cancel the leading error term for odd l
    jit = np.random.default_rng(7).uniform(-0.15, 0.15, (2, 37))
    jit[:, 0] = 0.0
    ex, ez = ex + jit[0], ez + jit[1]
    pts = np.random.default_rng(8).uniform(-1.5, 1.5, (12, 2))
    for l in (2, 3, 4, 5):
        hs = np.array([0.16, 0.08, 0.04, 0.02, 0.01]) if l < 5 else np.array([0.2, 0.1, 0.05, 0.025])
        errs = []
        for h in hs:
            e = 0.0
            for x0, y0 in pts:  # max error over several stencil positions
                xs, ys = x0 + h * ex, y0 + h * ez
                w = wt.all_weights(xs, ys, np.arange(37)[None, :], p, l, ["dx"], 0, 0.0)[0, 0]
                e = max(e, abs(w @ f(xs, ys) - fx(x0, y0)))
            errs.append(e)
        # asymptotic slope from the three finest spacings
        slope = np.polyfit(np.log(hs[-3:]), np.log(errs[-3:]), 1)[0]
        assert abs(slope - l) < 0.5, (l, slope, errs)


def test_hv_recursion_matches_repeated_laplacian_of_phs():
    """Eq. (laplacian): Delta r^p = p (p + d - 2) r^(p-2) in d = 2, checked by
    a centred difference of r^p itself away from r = 0."""
    for p in (5, 7, 9):
        x, z, h = 0.7, -0.4, 1e-4
        f = lambda a, b: np.hypot(a, b) ** p
        lap = (f(x + h, z) + f(x - h, z) + f(x, z + h) + f(x, z - h) - 4 * f(x, z)) / h ** 2
        r = np.hypot(x, z)
        assert abs(lap - p * p * r ** (p - 2)) < 1e-6 * p * p
        got = wt.phs_applied("hv", p, 1, np.array([x]), np.array([z]))[0]
        assert abs(got - p * p * r ** (p - 2)) < 1e-13 * p * p
        got3 = wt.phs_applied("hv", p, 2, np.array([x]), np.array([z]))[0]
        assert abs(got3 - p * p * (p - 2) ** 2 * r ** (p - 4)) < 1e-12 * p ** 4


def _mp_global_interpolant(xs, zs, f, p, l, mp):
    """The global PHS + degree-l interpolant of f on the nodes, solved and
    evaluated in 60-digit arithmetic (mpmath); returns s(x, z) and the
    centre node (the first node)."""
    n = len(xs)
    mono = [(d - b, b) for d in range(l + 1) for b in range(d + 1)]
    X = [mp.mpf(float(v)) for v in xs]
    Z = [mp.mpf(float(v)) for v in zs]
    A = mp.matrix(n + len(mono), n + len(mono))
    for i in range(n):
        for j in range(n):
            A[i, j] = mp.sqrt((X[i] - X[j]) ** 2 + (Z[i] - Z[j]) ** 2) ** p
        for c, (a, b) in enumerate(mono):
            A[i, n + c] = A[n + c, i] = X[i] ** a * Z[i] ** b
    coef = mp.lu_solve(A, mp.matrix([mp.mpf(float(v)) for v in f] + [0] * len(mono)))

    def s(x, z):
        v = sum(coef[j] * mp.sqrt((x - X[j]) ** 2 + (z - Z[j]) ** 2) ** p for j in range(n))
        return v + sum(coef[n + c] * x ** a * z ** b for c, (a, b) in enumerate(mono))

    return s, X[0], Z[0]


@pytest.mark.parametrize("p,l,n_nodes", [(3, 1, 10), (5, 2, 10), (7, 2, 10), (7, 3, 20), (9, 4, 20)])
def test_every_operator_equals_the_global_interpolants_derivative(p, l, n_nodes):
    """Brute force for every operator of Eq. (weights), including the second
    derivatives behind the wall conditions and Delta^k (Sec. 5.3): on small
    node sets the stencil is the whole set, so w . f must equal L applied to
    the global interpolant of f at the centre.  The interpolant is solved in
    60-digit arithmetic and differentiated by central differences of step
    1e-15 there (the PHS term of the centre node is C^(p-1), so the
    differences stay exact to far below FP64); Delta^k is the sum of
    C(k, i) d^2i/dx^2i d^2(k-i)/dz^2(k-i)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    rng = np.random.default_rng(100 * p + l)
    xs, zs, f = rng.uniform(-1, 1, n_nodes), rng.uniform(-1, 1, n_nodes), rng.normal(size=n_nodes)
    s, xc, zc = _mp_global_interpolant(xs, zs, f, p, l, mp)
    step = mp.mpf(10) ** -15
    dd = lambda a, b: float(mp.diff(s, (xc, zc), (a, b), h=step))
    exact = {"dx": dd(1, 0), "dz": dd(0, 1), "dxx": dd(2, 0), "dzz": dd(0, 2)}
    exact["lap"] = exact["dxx"] + exact["dzz"]
    idx = np.arange(n_nodes)[None, :]
    ops = ["dx", "dz", "dxx", "dzz", "lap"]
    W = wt.all_weights(xs, zs, idx, p, l, ops, 0, 0.0)[:, 0, :]
    for o, op in enumerate(ops):
        assert abs(W[o] @ f - exact[op]) <= 1e-10 * np.abs(W[o] * f).sum(), (op, W[o] @ f, exact[op])
    for k in (1, 2, 3):
        if p < 2 * k + 1:       # Delta^k r^p is singular at the centre (Sec. 5.3: p >= 2k + 1)
            continue
        lapk = sum(math.comb(k, i) * dd(2 * i, 2 * (k - i)) for i in range(k + 1))
        Wh = wt.all_weights(xs, zs, idx, p, l, ["hv"], k, 0.0)[0, 0]
        assert abs(Wh @ f - lapk) <= 1e-10 * np.abs(Wh * f).sum(), (k, Wh @ f, lapk)
