"""Learned coarse-grid correction workflow (a9).

The training data are fine runs of the method, restricted (a Gaussian average
over one coarse spacing by default, or injection) to
the nodes of a nested coarse lattice.  Each training sample pairs a coarse
state with the tendency that one coarse RK4 step misses:
    target = (R u_fine(t + dt_c) - step_c(R u_fine(t))) / dt_c.
A corrected coarse run then adds dt_c * MLP(state) after each coarse step.

This module only orders the library calls (control flow and argument
marshalling); every step runs in librbffd: the fine ensemble, restriction,
ghost solves, targets, feature scales, training, corrected runs.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs as inp
from . import rbffd


@dataclasses.dataclass
class Dataset:
    coarse_nodes: inp.NodeSet
    coarse: rbffd.Problem          # FP32 coarse problem (stencils shared with the MLP)
    states: object                 # torch float32 [R, n_snap, n_all_c, 4], ghosts filled
    targets: object                # torch float32 [R, n_snap - 1, n_prog_c, 4]
    seeds: list
    dt_c: float
    n_snap: int
    fine_node_updates: float
    fine_seconds: float


def build_dataset(h_coarse: float, ratio: int, seeds, t_end: float, fine_precision: int = 64,
                  average: bool = True) -> Dataset:
    """Fine runs (spacing h_coarse / ratio) of every seed in one batched
    ensemble, restricted to the coarse nodes after every coarse step, by a
    Gaussian average over one coarse spacing (average=True) or injection."""
    import torch
    coarse_nodes, fine_nodes, rmap = inp.nested_density_current(h_coarse, ratio)
    coarse = rbffd.ns_problem(coarse_nodes, precision=32)
    dt_c = h_coarse / 400.0
    dt_f = dt_c / ratio
    n_snap = int(round(t_end / dt_c)) + 1
    members = [inp.EnsembleMember(nodes=fine_nodes, n=37, l=4, dt=dt_f, n_steps=(n_snap - 1) * ratio,
                                  U0=inp.perturbed_density_current(fine_nodes, s), seed=s) for s in seeds]
    ens = rbffd.ensemble_problem(members, precision=fine_precision)
    R = len(seeds)
    n_all_c, n_prog_c = coarse_nodes.n_all, coarse_nodes.n_prog
    states = torch.zeros((R, n_snap, n_all_c, 4), dtype=torch.float32, device="cuda")
    index = torch.as_tensor(np.concatenate([ens.rec0[r] + rmap for r in range(R)]), dtype=torch.int64,
                            device="cuda")
    if average:
        aidx, aw = inp.restriction_average(coarse_nodes, fine_nodes, rmap, radius=h_coarse, sigma=0.5 * h_coarse)
        aidx = torch.as_tensor(np.concatenate([ens.rec0[r] + aidx for r in range(R)]), device="cuda")
        aw = torch.as_tensor(np.concatenate([aw] * R), device="cuda")
    U = ens.state()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fine_ms = 0.0
    for k in range(n_snap):
        if average:
            rbffd.restrict_weighted(U, fine_precision, aidx, aw, states[:, k], n_prog_c, n_snap * n_all_c)
        else:
            rbffd.restrict(U, fine_precision, index, states[:, k], 32, n_prog_c, n_snap * n_all_c)
        if k + 1 < n_snap:
            e0.record()
            ens.run(ratio, U)
            e1.record()
            e1.synchronize()
            fine_ms += e0.elapsed_time(e1)
    for r in range(R):
        for k in range(n_snap):
            rbffd.fill_ghosts(coarse, states[r, k])
    targets = torch.empty((R, n_snap - 1, n_prog_c, 4), dtype=torch.float32, device="cuda")
    rbffd.mlp_targets(coarse, states, R, n_snap, dt_c, targets)
    torch.cuda.synchronize()
    upd = ens.node_updates(-1)
    ens.close()
    return Dataset(coarse_nodes, coarse, states, targets, list(seeds), dt_c, n_snap, upd, fine_ms / 1e3)


def init_params(n_in: int, width: int = 64, seed: int = 0) -> np.ndarray:
    """Seeded Glorot-uniform weights, zero biases, small output layer."""
    rng = np.random.default_rng(seed)

    def glorot(a, b, gain=1.0):
        lim = gain * np.sqrt(6.0 / (a + b))
        return rng.uniform(-lim, lim, size=(a, b))

    return np.concatenate([glorot(n_in, width).ravel(), np.zeros(width), glorot(width, width).ravel(),
                           np.zeros(width), glorot(width, 4, 0.1).ravel(), np.zeros(4)]).astype(np.float32)


def train(ds: Dataset, n_train: int, iters: int = 2000, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Fits feature scales on the training runs, trains the MLP and chooses
    the coarse problem's persistent plan for corrected runs."""
    mlp = rbffd.Mlp(ds.coarse)
    n_in = 4 * (ds.coarse.info()["n_sten"] - 1) + 4   # differences, then own values
    mlp.set_params(init_params(n_in, seed=seed))
    S, T = ds.states[:n_train], ds.targets[:n_train]
    mlp.fit_scales(S, T, n_train, ds.n_snap)
    loss = mlp.train(S, T, n_train, ds.n_snap, iters, batch=batch, lr=lr, seed=seed)
    mlp.tune_run()   # the coarse problem's persistent plan, timed for corrected runs
    return mlp, loss


def rel_l2(a, b):
    """Per-field relative l2 difference of node-major tensors [n, 4]."""
    import torch
    d = torch.linalg.vector_norm((a - b).double(), dim=0)
    return (d / torch.clamp(torch.linalg.vector_norm(b.double(), dim=0), min=1e-300)).cpu().numpy()


# per-field correction strengths tried on the validation runs; all-zero is the
# uncorrected solver, the fallback when no strength helps
ALPHA_CANDIDATES = ((0.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.125, 0.0), (0.0, 0.0, 0.25, 0.0), (0.0, 0.0, 0.375, 0.0),
                    (0.0, 0.0, 0.5, 0.0), (0.0, 0.0, 0.75, 0.0), (0.0, 0.0, 1.0, 0.0), (0.25, 0.25, 0.25, 0.0),
                    (0.5, 0.5, 0.5, 0.0))


def run_errors(ds: Dataset, mlp, runs, alpha):
    """Per-field relative l2 errors at the final time of corrected coarse runs
    (alpha all zero: uncorrected) against the restricted fine reference."""
    n = ds.coarse_nodes.n_prog
    errs = []
    for r in runs:
        V = ds.states[r, 0].clone()
        if any(a > 0 for a in alpha):
            mlp.run(0.0, ds.dt_c, ds.n_snap - 1, V, alpha=alpha)
        else:
            ds.coarse.run(0.0, ds.dt_c, ds.n_snap - 1, V)
            ds.coarse.sync()
        errs.append(rel_l2(V[:n], ds.states[r, -1, :n]))
    return np.mean(errs, axis=0)


def select_alpha(ds: Dataset, mlp, val_runs, candidates=ALPHA_CANDIDATES):
    """Strength with the smallest mean validation error (the uncorrected
    solver is the reference for the correction: it is one of the candidates)."""
    scores = [(float(np.mean(run_errors(ds, mlp, val_runs, a))), a) for a in candidates]
    return min(scores)[1], scores


def prediction_skill(ds: Dataset, mlp, runs):
    """Per field, the fraction of the one-step defect's variance that the
    network predicts on the given runs' samples: 1 - sum (f(x) - f(0) - d)^2 /
    sum (d - mean d)^2 over every snapshot and prognostic node (rbf_mlp_forward
    per snapshot; the sums are a diagnostic, not part of the corrected run)."""
    import torch
    n = ds.coarse_nodes.n_prog
    se = torch.zeros(4, dtype=torch.float64, device="cuda")
    s1 = torch.zeros(4, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(4, dtype=torch.float64, device="cuda")
    cnt = 0
    for r in runs:
        for k in range(ds.n_snap - 1):
            d = mlp.forward(ds.states[r, k]).double()
            y = ds.targets[r, k].double()
            se += ((d - y) ** 2).sum(dim=0)
            s1 += y.sum(dim=0)
            s2 += (y ** 2).sum(dim=0)
            cnt += n
    var = s2 - s1 ** 2 / cnt
    return (1.0 - se / torch.clamp(var, min=1e-300)).cpu().numpy()
