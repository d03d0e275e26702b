"""FP64 parity bound of the GPU tests.

The GPU path and the oracle compute the same method with different LU pivot
sequences and summation orders, so in FP64 they agree only up to the rounding
those orders leave, amplified by the conditioning of the augmented systems
(kappa ~1e6 for r^7 + degree 4 on 37 nodes, ~1e9 for r^9 + degree 5 on 56).
Every FP64 comparison with the oracle is bounded per output field by

    max(1e-12, 10 s)

where s is the oracle's own spread for that case: the largest relative l2
gap, over the same outputs, between the oracle as written and the same oracle
with every stencil's neighbours listed in another order ("reversed",
"shuffled").  Permuting a stencil changes nothing but the rounding of its
augmented solve, so s measures how far rounding alone moves the answer; the
GPU is a third such order.
"""
import numpy as np

ORDERS = ("reversed", "shuffled")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def with_spread(make, compute):
    """(reference, spread): ``compute(make("nearest"))`` -- outputs [F, ...]
    of the oracle as written -- and, per output field, the largest relative l2
    gap to ``compute(make(order))`` over the other stencil orders."""
    ref = np.asarray(compute(make("nearest")))
    s = np.zeros(ref.shape[0])
    for order in ORDERS:
        alt = np.asarray(compute(make(order)))
        s = np.maximum(s, [rel(alt[f], ref[f]) for f in range(ref.shape[0])])
    return ref, s


def bound(spread):
    """The per-field FP64 bound max(1e-12, 10 s)."""
    return np.maximum(1e-12, 10.0 * np.asarray(spread, dtype=np.float64))


def check(got, ref, spread, label=""):
    """Asserts rel(got[f], ref[f]) < bound(spread[f]) for every field f and
    prints the gaps and bounds."""
    errs = np.array([rel(got[f], ref[f]) for f in range(len(spread))])
    b = bound(spread)
    print(f"{label} FP64 vs oracle {['%.2e' % e for e in errs]}, spread {['%.1e' % v for v in spread]}, "
          f"bound {['%.1e' % v for v in b]}")
    assert np.all(errs < b), (label, errs.tolist(), b.tolist())
    return errs
