"""Brute-force stencil selection (oracle; test infrastructure).

Sec. 6 uses the n = 37 nearest nodes of each node (complete rings on Cartesian
and hexagonal lattices, Appendix A).  Ordering key: squared distance in FP64,
then the global node index.  Squared distance is dx*dx + dz*dz rounded after
each operation; with a period L in x, dx is first brought to the minimum image
(dx > L/2 -> dx - L, dx < -L/2 -> dx + L).
"""
import numpy as np


def min_image(dx, period_x):
    if period_x > 0.0:
        dx = np.where(dx > 0.5 * period_x, dx - period_x, dx)
        dx = np.where(dx < -0.5 * period_x, dx + period_x, dx)
    return dx


def sq_dist(xc, zc, x, z, period_x):
    dx = min_image(x - xc, period_x)
    dz = z - zc
    return dx * dx + dz * dz


def knn(x, z, centers, n, period_x=0.0, chunk=256):
    """Indices [len(centers), n] of the n nearest nodes of each center, sorted
    by (squared distance, index).  ``centers`` are node indices into x, z."""
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    centers = np.asarray(centers, np.int64)
    out = np.empty((centers.shape[0], n), np.int64)
    idx_all = np.arange(x.shape[0])
    for s in range(0, centers.shape[0], chunk):
        c = centers[s:s + chunk]
        d2 = sq_dist(x[c][:, None], z[c][:, None], x[None, :], z[None, :], period_x)
        # n-th smallest squared distance of every row; every node at or below
        # it is a candidate, and the candidates are ordered by (d2, index)
        kth = np.partition(d2, n - 1, axis=1)[:, n - 1]
        for r in range(c.shape[0]):
            cand = np.nonzero(d2[r] <= kth[r])[0]
            order = cand[np.lexsort((idx_all[cand], d2[r, cand]))][:n]
            out[s + r] = order
    return out
