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


def knn_tree(x, z, centers, n, period_x=0.0, extra=16):
    """The same stencils as ``knn`` for large node sets, without its O(N^2)
    scan.  A k-d tree (scipy.spatial.cKDTree, a library nearest-neighbour
    search) proposes the n + extra nearest nodes of each centre -- with a
    period, among the nodes and their copies shifted by +-L -- and the
    proposals are ranked by the same key as ``knn``: the squared distance
    rounded as in ``sq_dist``, then the node index.  The proposal list is
    complete when the tree's farthest proposal lies beyond the n-th ranked
    distance by more than the tree's own rounding (a relative 1e-9 here);
    rows where it does not are asked again with twice as many proposals."""
    from scipy.spatial import cKDTree
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    centers = np.asarray(centers, np.int64)
    N = x.shape[0]
    pts = np.c_[x, z]
    orig = np.arange(N)
    if period_x > 0.0:
        pts = np.concatenate([pts, pts + [period_x, 0.0], pts - [period_x, 0.0]])
        orig = np.tile(orig, 3)
    tree = cKDTree(pts)
    out = np.empty((centers.shape[0], n), np.int64)
    todo = np.arange(centers.shape[0])
    k = n + extra
    while todo.size:
        k = min(k, pts.shape[0])
        c = centers[todo]
        dist, j = tree.query(np.c_[x[c], z[c]], k=k)
        cand = orig[j]
        d2 = sq_dist(x[c][:, None], z[c][:, None], x[cand], z[cand], period_x)
        order = np.lexsort((cand, d2), axis=-1)
        cand = np.take_along_axis(cand, order, axis=1)
        d2s = np.take_along_axis(d2, order, axis=1)
        # a node proposed twice (itself and a periodic copy) appears in
        # adjacent positions after ranking; such rows are redone one by one
        dup = np.any(cand[:, 1:] == cand[:, :-1], axis=1)
        complete = dist[:, -1] ** 2 > d2s[:, n - 1] * (1.0 + 1e-9) + 1e-300
        if k >= pts.shape[0]:
            complete[:] = True
        ok = complete & ~dup
        out[todo[ok]] = cand[ok, :n]
        for r in np.nonzero(complete & dup)[0]:
            _, first = np.unique(cand[r], return_index=True)
            keep = cand[r, np.sort(first)]
            if keep.shape[0] >= n:
                out[todo[r]] = keep[:n]
            else:
                complete[r] = False
        todo = todo[~complete]
        k *= 2
    return out


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
