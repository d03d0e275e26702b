"""Sparse differentiation matrices (oracle; test infrastructure).

Sec. 3: each stencil solve gives one row of a differentiation matrix (DM); the
DM is more than 99% empty, so only its nonzeros are kept.  Here a DM is a
scipy CSR matrix of shape [rows, n_all]; row i holds the weights of stencil i
at the columns of its nodes.  On reflected (mirror) nodes the column is folded
onto the source node (Sec. 6.1): a mirror carries its source's value.
"""
import numpy as np
import scipy.sparse as sp

from . import stencils as st
from . import weights as wt


BRUTE_FORCE_MAX = 10000


def stencil_permutation(order, n):
    """Column order of an n-node stencil (centre first): "nearest" keeps the
    ranked order, "reversed" lists the neighbours farthest first, "shuffled"
    in a fixed seeded order."""
    if order == "nearest":
        return np.arange(n)
    if order == "reversed":
        return np.concatenate([[0], np.arange(n - 1, 0, -1)])
    if order == "shuffled":
        return np.concatenate([[0], 1 + np.random.default_rng(1509).permutation(n - 1)])
    raise ValueError(order)


def dm(w, idx, n_cols):
    """CSR matrix from weights [N, n] at columns idx [N, n]; duplicate columns
    (a node reached directly and through its mirror) are summed."""
    N, n = idx.shape
    rows = np.repeat(np.arange(N), n)
    return sp.csr_matrix((w.ravel(), (rows, idx.ravel())), shape=(N, n_cols))


class Discretisation:
    """Stencils, weights and DMs of one node set.

    ``ops`` is the operator list built from PHS r^p with degree-l polynomials;
    ``hv`` (optional) adds Delta^k from PHS r^hv_p (Sec. 5.3: the PHS used for
    hyperviscosity need not be the one used for the other operators)."""

    def __init__(self, nodes, n, p, l, ops=("dx", "dz", "lap"), hv_k=0, hv_p=None, fold_mirrors=False,
                 stencil_order="nearest", workers=1):
        self.nodes = nodes
        self.n, self.p, self.l = n, p, l
        centers = np.arange(nodes.n_prog)
        # the brute-force search is the definition; above BRUTE_FORCE_MAX nodes
        # the k-d tree search, which the tests pin to it, gives the same lists
        find = st.knn if nodes.n_all <= BRUTE_FORCE_MAX else st.knn_tree
        self.idx = find(nodes.x, nodes.z, centers, n, nodes.period_x)
        # "reversed" / "shuffled": the same stencils with the neighbours listed
        # farthest first or in a fixed shuffled order.  The augmented systems
        # are permuted, so the weights differ only by rounding: the oracle's
        # own spread between two orders of the same solve.
        self.idx = self.idx[:, stencil_permutation(stencil_order, n)]
        self.W = {}
        w = wt.all_weights_pool(nodes.x, nodes.z, self.idx, p, l, list(ops), 0, nodes.period_x, workers)
        for o, op in enumerate(ops):
            self.W[op] = w[o]
        if hv_k > 0:
            hp = p if hv_p is None else hv_p
            self.W["hv"] = wt.all_weights_pool(nodes.x, nodes.z, self.idx, hp, l, ["hv"], hv_k, nodes.period_x,
                                               workers)[0]
        self.hv_k = hv_k
        cols = nodes.src[self.idx] if fold_mirrors else self.idx
        self.cols = cols
        n_cols = nodes.n_prog if fold_mirrors else nodes.n_all
        self.D = {op: dm(self.W[op], cols, n_cols) for op in self.W}
