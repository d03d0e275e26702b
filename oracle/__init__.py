"""FP64 CPU oracle of the PHS RBF-FD method (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The CUDA library never calls it and shares no code with it: the only
module both sides import is ``paper_1509_02615_gb300.inputs`` (seeded node sets
and closed-form initial states, none of the method's arithmetic).

Every function follows the paper's definitions in plain, unblocked numpy/scipy:

* ``stencils``   n nearest nodes by brute force (Sec. 6, n = 37; Appendix A)
* ``weights``    the augmented PHS + polynomial system of Eq. (weights), Sec. 3,
                 with the Laplacian recursion of Eq. (laplacian), Sec. 5.3
* ``operators``  sparse differentiation matrices (Sec. 3: only nonzeros kept)
* ``ns``         ghost-node solve (Sec. 5.2, Eq. bcEqn), the perturbation
                 equations uEq-piEq (Sec. 6.2) and classical RK4 (Sec. 6.3)
* ``advection``  flux-form scalar transport with reflected nodes (Sec. 6.1)
* ``mlp``        the learned tendency correction (no counterpart in the paper)
"""
