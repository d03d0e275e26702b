"""Throughput of the PHS RBF-FD hot path on one GB300 (or N replicas).

Workload (default): the density current of Sec. 6.3 on hexagonal nodes at
100 m -- 38,400 prognostic nodes + 1,024 ghosts, PHS r^7 + degree-4
polynomials, n = 37, Delta^3 hyperviscosity, mu = 75 m^2/s, dt = 0.25 s --
stepped in FP32 (FP64-built weights stored in FP32).  One step = one
classical RK4 step: four stages, each a ghost solve (Sec. 5.2) and one fused
right-hand-side + RK4-update kernel.  Setup (stencils, weights, packing,
ghost inverses) is timed separately and reported under "setup".

Metric: node-RHS evaluations per second (4 per node per RK4 step).  The
working set (~31 MB) fits in L2, so L2 is flushed (a 512 MB write) between
timed steps; each step is timed alone with CUDA events on the problem's
stream.  The FP64 form of the same workload is reported under "fp64".

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on a bounded sample of the same workload: one 1/8-width strip
per host core.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-RHS evals/s (RK4)"
UNIT = "node-RHS/s"
WORKLOAD = "density current (Sec. 6.3), hexagonal 100 m, 38400 nodes + 1024 ghosts, r^7 + deg 4, n=37, Delta^3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--h", type=float, default=100.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--threads-per-node", type=int, default=0, help="0 = autotuned")
    ap.add_argument("--run-mode", default="auto", choices=["auto", "graph", "persistent"],
                    help="headline run mode (auto: timed at creation); fixing it makes profiled runs reproducible")
    ap.add_argument("--persistent-lanes", type=int, default=1, help="lanes per node with --run-mode persistent")
    ap.add_argument("--persistent-ctas", type=int, default=0, help="CTAs with --run-mode persistent (0: one per SM)")
    ap.add_argument("--ens-runs", type=int, default=256, help="ensemble members (0 = skip the batched case)")
    ap.add_argument("--ens-steps", type=int, default=40, help="timed global RK4 steps of the ensemble")
    ap.add_argument("--ens-threads", type=int, default=0, choices=(0, 1, 2, 4),
                    help="lanes per node of the batched ensembles (0 = autotuned)")
    ap.add_argument("--learned", type=int, default=1, help="1 = measure the learned coarse-grid correction")
    ap.add_argument("--learned-coarse", type=float, default=400.0)
    ap.add_argument("--learned-ratio", type=int, default=4)
    ap.add_argument("--learned-seeds", type=int, default=16)
    ap.add_argument("--large-h", type=float, default=25.0,
                    help="spacing of the HBM-roofline case (0 = skip); its working set exceeds L2")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world):
    """Maximum of a per-rank float over all ranks (the whole job's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks divided by the (max-over-ranks) time."""
    return units_per_rank * world / seconds


def sum_over_ranks(value, world):
    """Sum of a per-rank float over all ranks."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_members(members, rank, world):
    """This rank's share of the ensemble's members: every world-th member
    from its rank (round robin over the seeded draw, so the spacings, layouts
    and stencil sizes spread evenly); the members are independent runs, so
    the ranks exchange nothing but the final timing."""
    return list(members[rank::world])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash(key=""):
    """Hash of the source files holding the device code of the kernel a
    profile key names: its translation unit and the device headers it uses."""
    h = hashlib.sha256()
    unit = ("persistent.cu" if key.startswith("persistent") else
            "ensemble.cu" if key.startswith("ens_stage") else "ns.cu")
    for fn in (unit, "records.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1509_02615_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def profiled_traffic(key, nodes=None, algorithmic=None, **launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source and the same launch shape (the ``launch``
    keywords, e.g. threads_per_node, that the summary records); else None."""
    try:
        with open(TRAFFIC_JSON) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(key)
    if not e or e.get("source_hash") != kernel_source_hash(key):
        return None
    if any(k in e and e[k] != v for k, v in launch.items()):
        return None
    if nodes is not None and "dram_bytes_per_node" in e:
        return e["dram_bytes_per_node"] * nodes   # captured on a smaller launch of the same kernel
    if algorithmic is not None and "dram_per_algorithmic_byte" in e:
        # captured on another mix of the same kernel's units: scaled by its
        # traffic per algorithmic byte
        return e["dram_per_algorithmic_byte"] * algorithmic
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.path = f"/tmp/rbffd_clocks_{os.getpid()}.csv"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except OSError:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(h, precision, tpn=0, run_mode="auto", lanes=1, ctas=0):
    from paper_1509_02615_gb300 import inputs as inp
    from paper_1509_02615_gb300 import rbffd
    nodes = inp.density_current_nodes(h)
    if run_mode == "auto":
        pb = rbffd.ns_problem(nodes, precision=precision, threads_per_node=tpn)
    else:
        pb = rbffd.ns_problem(nodes, precision=precision, threads_per_node=tpn or 2)
        pb.set_run_mode(run_mode, lanes=lanes if run_mode == "persistent" else 0, ctas=ctas)
    U0 = inp.density_current_state(nodes)
    return nodes, pb, U0


def time_steps(torch, pb, U, dt, steps, warmup, flush, stage_timing):
    """Per-step device times (ms) and summed stage-kernel times (ms)."""
    stream = torch.cuda.current_stream()
    pb.set_stage_timing(stage_timing)
    t = 0.0
    for _ in range(warmup):
        flush.zero_()
        pb.run(t, dt, 1, U)
        t += dt
    torch.cuda.synchronize()
    step_ms, stage_ms = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        flush.zero_()                    # evict the 31 MB working set from L2
        e0.record(stream)
        pb.run(t, dt, 1, U)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if stage_timing:
            stage_ms.append(pb.stage_kernel_ms())
        t += dt
    pb.set_stage_timing(False)
    return step_ms, stage_ms


def fp64_peak_tflops(torch, n=4096, reps=5):
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul) of two
    n x n matrices, best of reps, 2 n^3 flops each (CUDA events)."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        a @ b
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a @ b
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def weights_case(torch, h, peak_tflops):
    """a2 alone: the FP64 weight build of the headline node set through the C
    ABI (rbf_build_weights: d/dx, d/dz, Lap, d2/dx2, d2/dz2 and Delta^3, all
    from r^7 with degree 4 and n = 37, so one augmented system per node with
    K = 6 right-hand sides, as rbf_ns_create builds them), timed with CUDA
    events after a warm-up build.  Algorithmic flops per node:
    (2/3) S^3 + 2 K S^2 (LU of the S x S system and its K right-hand sides)."""
    from paper_1509_02615_gb300 import inputs as inp
    from paper_1509_02615_gb300 import rbffd
    nodes = inp.density_current_nodes(h)
    x = torch.as_tensor(nodes.x, device="cuda")
    z = torch.as_tensor(nodes.z, device="cuda")
    idx = rbffd.build_stencils(x, z, nodes.n_prog, 37, nodes.period_x)
    ops = ("dx", "dz", "lap", "dxx", "dzz", "hv")
    stream = torch.cuda.current_stream()

    def build():
        rbffd.build_weights(x, z, idx, 7, 4, ops, 3, nodes.period_x)

    build()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    build()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    S = 37 + 15
    flops = nodes.n_prog * ((2.0 / 3.0) * S ** 3 + 2.0 * len(ops) * S ** 2)
    ach = flops / (ms / 1e3) / 1e12
    return {"workload": f"FP64 weights of the {nodes.n_prog} prognostic nodes at {h:g} m (6 operators from r^7, "
                        f"one augmented system of size S = {S} per node)",
            "ms": ms, "nodes_per_s": nodes.n_prog / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": ach / peak_tflops, "algorithmic_flops": flops,
                         "peak_source": "measured cuBLAS DGEMM 4096^3 in this run"}}


def large_case(torch, args, flush):
    """The same density current at a finer spacing, whose FP32 working set is
    several times larger than L2: the stage kernel's HBM roofline."""
    from paper_1509_02615_gb300 import rbffd
    pk, pk_kind = peaks()
    nodes, pb, U0 = make_problem(args.large_h, 32)
    info = pb.info()
    U = rbffd.state_tensor(U0, 32)
    dt = args.large_h / 400.0
    steps = 10
    step_ms, _ = time_steps(torch, pb, U, dt, steps, 3, flush, False)
    _, stage_ms = time_steps(torch, pb, U, dt, steps, 1, flush, True)
    avg = float(np.mean(stage_ms)) / 4.0
    bpl = info["rhs_bytes_per_node"] * nodes.n_prog
    ach = bpl / (avg / 1e3) / 1e9
    out = {"workload": f"density current, hexagonal {args.large_h:g} m, {nodes.n_prog} nodes + {nodes.n_ghost} ghosts, FP32",
           "node_rhs_per_s": 4.0 * nodes.n_prog * steps / (float(sum(step_ms)) / 1e3),
           "ms_per_step": float(sum(step_ms)) / steps,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / pk["hbm_gbs"], "traffic": profiled_traffic(f"ns_stage_fp32_hex{int(args.large_h)}",
                                                                   threads_per_node=info["threads_per_node"]),
                        "algorithmic_bytes_per_launch": bpl, "avg_launch_ms": avg,
                        "peak_source": f"{pk_kind} hbm_gbs"},
           "threads_per_node": info["threads_per_node"], "prefetch": info["prefetch"],
           "setup": {"weight_build_ms": info["weight_build_ms"], "ghost_setup_ms": info["ghost_setup_ms"]}}
    # f4: the same steps with lattice operator storage (one operator row per
    # class of translated stencils); its bytes per node-RHS follow the storage
    Ur = U.clone()
    t0 = time.perf_counter()
    cn, nc = pb.set_operator_storage("lattice")
    lat_setup_s = time.perf_counter() - t0
    li = pb.info()
    Ul = rbffd.state_tensor(U0, 32)
    lstep, _ = time_steps(torch, pb, Ul, dt, steps, 3, flush, False)
    _, lstage = time_steps(torch, pb, Ul, dt, steps, 1, flush, True)
    lavg = float(np.mean(lstage)) / 4.0
    lbpl = li["rhs_bytes_per_node"] * nodes.n_prog
    lach = lbpl / (lavg / 1e3) / 1e9
    # same number of steps from the same state as the per-node run above
    fl, fp = rbffd.fields(Ul)[:, :nodes.n_prog], rbffd.fields(Ur)[:, :nodes.n_prog]
    out["lattice"] = {
        "node_rhs_per_s": 4.0 * nodes.n_prog * steps / (float(sum(lstep)) / 1e3),
        "ms_per_step": float(sum(lstep)) / steps, "avg_stage_kernel_ms": lavg,
        "speedup_vs_per_node": float(sum(step_ms)) / float(sum(lstep)),
        "classes": nc, "class_nodes": cn, "class_fraction": cn / nodes.n_prog,
        "rhs_bytes_per_node": li["rhs_bytes_per_node"], "threads_per_node": li["threads_per_node"],
        "roofline": {"bound": "hbm", "achieved": lach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": lach / pk["hbm_gbs"], "traffic": profiled_traffic(f"ns_stage_lattice_fp32_hex{int(args.large_h)}",
                                                                threads_per_node=li["threads_per_node"]),
                     "algorithmic_bytes_per_launch": lbpl, "avg_launch_ms": lavg,
                     "peak_source": f"{pk_kind} hbm_gbs",
                     "note": "algorithmic bytes of the lattice storage: class id + records, no per-node operators"},
        "rel_l2_vs_per_node_after_%d_steps" % (2 * steps + 4): [
            float(np.linalg.norm(fl[f] - fp[f]) / max(np.linalg.norm(fp[f]), 1e-30)) for f in range(4)],
        "setup_s": lat_setup_s}
    pb.close()
    return out


def _time_ensemble(torch, ens, K):
    """Node-updates/s of K global RK4 steps (after 3 untimed) and the median
    stage-kernel time of 3 more, for an ensemble's initial state."""
    U = ens.state()
    stream = torch.cuda.current_stream()
    ens.run(3, U)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.run(K, U)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ens.set_stage_timing(True)
    stage = []
    for _ in range(3):
        ens.run(1, U)
        stage.append(ens.stage_kernel_ms() / 4.0)
    ens.set_stage_timing(False)
    mm = ens.minmax(U)
    return ms, float(np.median(stage)), bool(np.all(np.isfinite(mm))), U


def ensemble_case(torch, args):
    """Batched ensemble (FP32): 256 seeded density-current members of uneven
    size (spacings 50-400 m, Cartesian/hexagonal/scattered, stencils 31-75),
    stepped together; the timed region is the first ens_steps global RK4
    steps (every member active), inputs ~8 GB (larger than L2).  Measured with
    per-node operator storage (the headline form) and with lattice storage
    (f4: the lattice members keep one operator row per stencil class)."""
    from paper_1509_02615_gb300 import inputs as inp
    from paper_1509_02615_gb300 import rbffd
    pk, pk_kind = peaks()
    rank, world, _ = dist_env()
    t0 = time.perf_counter()
    every = inp.ensemble_members(args.ens_runs, seed=0)
    members = shard_members(every, rank, world)
    t_gen = time.perf_counter() - t0
    ens = rbffd.ensemble_problem(members, precision=32, threads_per_node=args.ens_threads)
    info = ens.info()
    K = args.ens_steps
    ms, avg, finite, U = _time_ensemble(torch, ens, K)
    upd = sum_over_ranks(ens.node_updates(K), world)
    ms = max_over_ranks(ms, world)
    bpl = info["rhs_bytes_per_node"] * ens.n_prog
    ach = bpl / (avg / 1e3) / 1e9
    out = {"workload": f"{len(every)} density-current members, {ens.n_prog} nodes + {ens.n_all - ens.n_prog} ghosts "
                       f"on this rank ({len(members)} members), h in 50-400 m, cart/hex/scattered, n 31-75 "
                       f"(Cartesian without n=31 l=3 and n=75 l=5), FP32",
           "value": upd / (ms / 1e3), "unit": "node-updates/s", "node_rhs_per_s": 4.0 * upd / (ms / 1e3),
           "scaling": "strong", "ranks": world, "members_per_rank": len(members),
           "timed_global_steps": K, "ms": ms, "node_updates_to_900s": sum_over_ranks(ens.node_updates(-1), world),
           "threads_per_node": info["threads_per_node"],
           "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / pk["hbm_gbs"], "traffic": profiled_traffic("ens_stage_fp32", algorithmic=bpl,
                                                                   threads_per_node=info["threads_per_node"]),
                        "kernel": "ens_stage_kernel",
                        "algorithmic_bytes_per_launch": bpl, "avg_launch_ms": avg,
                        "peak_source": f"{pk_kind} hbm_gbs"},
           "setup": {"host_node_generation_s": t_gen, "gpu_build_ms": info["weight_build_ms"]},
           "finite": finite}
    Ur = U.cpu()
    ens.close()
    del U
    # the same members in FP64 (per-node storage): the plain-FP64 form the
    # FP32 batched form is compared with, and the FP32 error after the same steps
    e64 = rbffd.ensemble_problem(members, precision=64, threads_per_node=args.ens_threads)
    ms64, _, fin64, U64 = _time_ensemble(torch, e64, K)
    upd64 = sum_over_ranks(e64.node_updates(K), world)
    ms64 = max_over_ranks(ms64, world)
    f32, f64 = Ur.double(), U64.cpu()
    out["fp64"] = {"value": upd64 / (ms64 / 1e3), "unit": "node-updates/s", "ms": ms64, "finite": fin64,
                   "fp32_speedup": (upd / (ms / 1e3)) / (upd64 / (ms64 / 1e3)),
                   "fp32_rel_l2_vs_fp64_same_steps": [
                       float(torch.linalg.vector_norm(f32[:, f] - f64[:, f]) / torch.linalg.vector_norm(f64[:, f]))
                       for f in range(4)]}
    e64.close()
    del U64, f64
    t0 = time.perf_counter()
    lens = rbffd.ensemble_problem(members, precision=32, storage="lattice", threads_per_node=args.ens_threads)
    build_s = time.perf_counter() - t0
    li = lens.info()
    lms, lavg, lfin, LU = _time_ensemble(torch, lens, K)
    lupd = sum_over_ranks(lens.node_updates(K), world)
    lms = max_over_ranks(lms, world)
    lbpl = li["rhs_bytes_per_node"] * lens.n_prog
    diff = float(torch.linalg.vector_norm((LU.cpu() - Ur).double()) / torch.linalg.vector_norm(Ur.double()))
    out["lattice"] = {
        "value": lupd / (lms / 1e3), "unit": "node-updates/s", "node_rhs_per_s": 4.0 * lupd / (lms / 1e3),
        "ms": lms, "avg_stage_kernel_ms": lavg, "speedup_vs_per_node": ms / lms,
        "rhs_bytes_per_node": li["rhs_bytes_per_node"], "threads_per_node": li["threads_per_node"],
        "roofline": {"bound": "hbm", "achieved": lbpl / (lavg / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": lbpl / (lavg / 1e3) / 1e9 / pk["hbm_gbs"],
                     "traffic": profiled_traffic("ens_stage_lattice_fp32", algorithmic=lbpl,
                                                 threads_per_node=li["threads_per_node"]),
                     "algorithmic_bytes_per_launch": lbpl, "avg_launch_ms": lavg,
                     "peak_source": f"{pk_kind} hbm_gbs"},
        "rel_l2_vs_per_node_same_steps": diff, "finite": lfin, "build_s": build_s}
    lens.close()
    return out


def learned_case(torch, args):
    """Learned coarse-grid correction: coarse hexagonal runs corrected by the MLP,
    against the restricted fine FP64 reference at 900 s (held-out seeds), with
    the uncorrected coarse and 2x-finer runs beside it."""
    from paper_1509_02615_gb300 import inputs as inp
    from paper_1509_02615_gb300 import learned
    from paper_1509_02615_gb300 import rbffd
    hc, ratio, ns = args.learned_coarse, args.learned_ratio, args.learned_seeds
    n_train, n_val = int(round(ns * 0.625)), int(round(ns * 0.1875))
    seeds = inp.learned_correction_seeds(ns, seed=1)
    t0 = time.perf_counter()
    ds = learned.build_dataset(hc, ratio, seeds, 900.0)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    mlp, loss = learned.train(ds, n_train, iters=30000, batch=4096, lr=2e-3)
    t_train = time.perf_counter() - t0
    alpha, scores = learned.select_alpha(ds, mlp, range(n_train, n_train + n_val))
    test = list(range(n_train + n_val, ns))
    err_plain = learned.run_errors(ds, mlp, test, (0.0, 0.0, 0.0, 0.0))
    err_learned = learned.run_errors(ds, mlp, test, alpha)
    steps = ds.n_snap - 1
    nc = ds.coarse_nodes.n_prog
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    V = ds.states[test[0], 0].clone()
    mlp.run(0.0, ds.dt_c, steps, V, alpha=alpha)   # warm-up
    V = ds.states[test[0], 0].clone()
    e0.record()
    mlp.run(0.0, ds.dt_c, steps, V, alpha=alpha)
    e1.record()
    e1.synchronize()
    ms_learned = e0.elapsed_time(e1)
    V = ds.states[test[0], 0].clone()
    ds.coarse.run(0.0, ds.dt_c, steps, V)
    e0.record()
    ds.coarse.run(0.0, ds.dt_c, steps, V)
    e1.record()
    e1.synchronize()
    ms_plain = e0.elapsed_time(e1)
    # uncorrected runs at half the coarse spacing (FP64), restricted the same way
    coarse_nodes, mid, rmap = inp.nested_density_current(hc, 2)
    aidx, aw = inp.restriction_average(coarse_nodes, mid, rmap, radius=hc, sigma=0.5 * hc)
    aidx_t = torch.as_tensor(aidx, device="cuda")
    aw_t = torch.as_tensor(aw, device="cuda")
    pb_mid = rbffd.ns_problem(mid, precision=64)
    err_mid = []
    ms_mid = 0.0
    for r in test:
        U = rbffd.state_tensor(inp.perturbed_density_current(mid, seeds[r]), 64)
        e0.record()
        pb_mid.run(0.0, hc / 800.0, 2 * steps, U)
        e1.record()
        e1.synchronize()
        ms_mid += e0.elapsed_time(e1)
        out = torch.zeros((coarse_nodes.n_all, 4), dtype=torch.float32, device="cuda")
        rbffd.restrict_weighted(U, 64, aidx_t, aw_t, out, nc, coarse_nodes.n_all)
        err_mid.append(learned.rel_l2(out[:nc], ds.states[r, -1, :nc]))
    pb_mid.close()
    out = {"workload": f"density current, hexagonal {hc:g} m coarse ({nc} nodes), MLP trained on {hc / ratio:g} m FP64 "
                       f"runs restricted to the coarse nodes ({n_train} train / {n_val} validation / {len(test)} test "
                       f"seeds), t = 900 s",
           "selected_alpha": alpha, "validation_scores": [[sc, list(a)] for sc, a in scores],
           "rel_l2_test": {"fields": ["u", "w", "theta'", "pi'"],
                           "uncorrected_coarse_fp32": [float(v) for v in err_plain],
                           "learned_coarse_fp32": [float(v) for v in err_learned],
                           f"uncorrected_{hc / 2:g}m_fp64": [float(v) for v in np.mean(err_mid, axis=0)]},
           "node_updates_per_s": {"learned_coarse_fp32": nc * steps / (ms_learned / 1e3),
                                  "uncorrected_coarse_fp32": nc * steps / (ms_plain / 1e3),
                                  f"uncorrected_{hc / 2:g}m_fp64": mid.n_prog * 2 * steps * len(test) / (ms_mid / 1e3),
                                  "fine_reference_fp64_batched": ds.fine_node_updates / ds.fine_seconds},
           # GPU time of one run to t = 900 s, and the stated-error comparison:
           # the cheapest run whose mean test error is at most the learned one's
           "ms_to_900s": {"learned_coarse_fp32": ms_learned, "uncorrected_coarse_fp32": ms_plain,
                          f"uncorrected_{hc / 2:g}m_fp64": ms_mid / len(test)},
           "stated_error": {"metric": "mean over fields and test seeds of the relative l2 error at 900 s",
                            "learned_coarse_fp32": float(np.mean(err_learned)),
                            "uncorrected_coarse_fp32": float(np.mean(err_plain)),
                            f"uncorrected_{hc / 2:g}m_fp64": float(np.mean(err_mid))},
           "final_training_loss": float(np.mean(loss[-50:])),
           "seconds": {"data": t_data, "train": t_train}}
    mlp.close()
    return out


def _oracle_strip(h):
    """The FP64 oracle on a 1/8-width periodic strip of the workload (same
    spacing, stencils, operators and boundary treatment), its setup time
    (stencils, weights, ghost factorisations) and a state one step in."""
    from oracle.ns import NSOracle
    from paper_1509_02615_gb300 import inputs as inp
    width = 25600.0 / 8.0
    nodes = inp.lattice_nodes("hex", -width, width, 0.0, 6400.0, h, True)
    t0 = time.perf_counter()
    o = NSOracle(nodes)
    setup_s = time.perf_counter() - t0
    U = inp.density_current_state(nodes)
    U = o.rk4_step(0.0, h / 400.0, U)
    return nodes, o, U, setup_s


def _oracle_rhs_rate(args):
    """RHS evaluations of one strip for budget_s seconds: (evaluations,
    nodes, seconds, setup seconds).  Runs in a spawned worker process."""
    h, budget_s = args
    nodes, o, U, setup_s = _oracle_strip(h)
    t0 = time.perf_counter()
    n_eval = 0
    while time.perf_counter() - t0 < budget_s:
        o.rhs(0.0, U)
        n_eval += 1
    return n_eval, nodes.n_prog, time.perf_counter() - t0, setup_s


def cpu_baseline(h, budget_s=12.0):
    """FP64 oracle node-RHS/s on the host cores: one strip per core in spawned
    single-threaded processes (the headline figure), and one core alone."""
    import multiprocessing as mp
    n_eval, n_prog, el, setup_s = _oracle_rhs_rate((h, budget_s))
    single = n_eval * n_prog / el
    cores = os.cpu_count() or 1
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"          # the spawned workers' BLAS stays single-threaded
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_rhs_rate, [(h, budget_s)] * cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    value = sum(ne * npg / t for ne, npg, t, _ in res)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle RHS (ghost solve + sparse DM products) on periodic strips of the workload, 1/8 of "
                      f"its width ({n_prog} of 38400 nodes, same h, stencils and walls): one strip per core in "
                      f"{cores} spawned single-threaded processes, {sum(r[0] for r in res)} evaluations in "
                      f"{budget_s:.0f} s each",
            "single_core": {"value": single, "cores": 1, "evaluations": n_eval, "seconds": el},
            "oracle_setup_s": setup_s}


def _oracle_rk4_steps(args):
    """W untimed and K timed oracle RK4 steps on one strip: (nodes, seconds).
    Runs in a spawned worker process."""
    h, warmup, steps = args
    nodes, o, U, _ = _oracle_strip(h)
    dt = h / 400.0
    for s in range(warmup):
        U = o.rk4_step((1 + s) * dt, dt, U)
    t0 = time.perf_counter()
    for s in range(steps):
        U = o.rk4_step((1 + warmup + s) * dt, dt, U)
    return nodes.n_prog, time.perf_counter() - t0


def run_reference(args, rank, world):
    """The oracle arm: W untimed and K timed RK4 steps of the FP64 oracle on
    1/8-width strips of the workload (same spacing, stencils, walls), one
    strip per host core in spawned single-threaded processes; one step is four
    right-hand sides with their ghost solves.  The rate sums the strips'
    node-RHS/s."""
    if rank != 0:
        return
    import multiprocessing as mp
    t_start = time.perf_counter()
    cores = os.cpu_count() or 1
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_rk4_steps, [(args.h, args.warmup, args.steps)] * cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    value = sum(4.0 * n * args.steps / el for n, el in res)
    ms_step = 1e3 * float(np.mean([el for _, el in res])) / max(args.steps, 1)
    n_strip = res[0][0]
    sample = (f"FP64 oracle RK4 steps (ghost solves + sparse DM products) on periodic strips of the workload, 1/8 of "
              f"its width ({n_strip} of 38400 nodes, same h, stencils and walls), one strip per core in {cores} "
              f"spawned single-threaded processes: {args.warmup} untimed + {args.steps} timed steps each, "
              f"{ms_step:.1f} ms per step per strip")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 oracle", "l2": "n/a (CPU)",
                       "sample_nodes": n_strip * cores},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1509_02615_gb300 import _build
    if rank == 0:
        _build.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
        if rank != 0:
            _build.build()   # no-op once rank 0 has built
    torch.cuda.set_device(local)
    from paper_1509_02615_gb300 import rbffd
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pk, pk_kind = peaks()

    nodes, pb, U0 = make_problem(args.h, args.precision, args.threads_per_node, args.run_mode,
                                 args.persistent_lanes, args.persistent_ctas)
    info = pb.info()
    dt = args.h / 400.0
    U = rbffd.state_tensor(U0, args.precision)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    persistent = info["run_mode"] == 2
    with ClockSampler(local) as clk:
        step_ms, _ = time_steps(torch, pb, U, dt, args.steps, args.warmup, flush, False)
        torch.cuda.synchronize()
        stage_ms = []
        if not persistent:
            # same steps again with timing events around the four stage kernels
            # (the events also break the programmatic overlap of the launches)
            _, stage_ms = time_steps(torch, pb, U, dt, args.steps, 1, flush, True)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(step_ms), world)
    value = whole_job_rate(4.0 * nodes.n_prog * args.steps, world, total_ms / 1e3)
    mm = pb.minmax(U)   # fails loudly on NaN/Inf

    # roofline of the dominant kernel: the persistent kernel (one launch per
    # step: 4 stages of algorithmic bytes) or the fused RHS + RK4 stage kernel
    if persistent:
        avg_ms = float(np.mean(step_ms))
        bytes_per_launch = 4.0 * info["rhs_bytes_per_node"] * nodes.n_prog
        kernel = "rk4_persistent"
        share = 1.0
    else:
        avg_ms = float(np.mean(stage_ms)) / 4.0
        bytes_per_launch = info["rhs_bytes_per_node"] * nodes.n_prog
        kernel = "ns_stage_kernel"
        share = float(np.sum(stage_ms) / np.sum(step_ms))
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    key = f"{'persistent' if persistent else 'ns_stage'}_fp{args.precision}_hex{int(args.h)}"
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": profiled_traffic(key, **({"persistent_lanes": info["persist_lanes"],
                                                  "persistent_ctas": info["persist_ctas"]} if persistent else
                                                 {"threads_per_node": info["threads_per_node"]})),
            "kernel": kernel,
            "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
            "kernel_share_of_step": share, "peak_source": f"{pk_kind} hbm_gbs"}

    # context: a sustained run (one rbf_run of many steps, L2 flushed once
    # before it) -- the way a simulation uses the library; not the headline
    sus_steps = 400
    flush.zero_()
    Us = rbffd.state_tensor(U0, args.precision)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pb.run(0.0, dt, sus_steps, Us)
    e1.record(stream)
    e1.synchronize()
    pb.sync()
    sus_ms = e0.elapsed_time(e1)
    sustained = {"value": 4.0 * nodes.n_prog * sus_steps / (sus_ms / 1e3), "unit": UNIT, "steps": sus_steps,
                 "ms_per_step": sus_ms / sus_steps,
                 "note": "one rbf_run of 400 steps, L2 flushed once before it (context only)"}

    # end to end through the C ABI on a pinned host state, copies included
    Uh = rbffd.state_tensor(U0, args.precision, device="cpu").pin_memory()
    e2e_steps = max(10, args.steps // 4)
    pb.run_host(0.0, dt, 1, Uh)
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        pb.run_host(s * dt, dt, 1, Uh)
    e2e_s = time.perf_counter() - t0
    state_bytes = Uh.numel() * Uh.element_size()
    e2e = {"value": 4.0 * nodes.n_prog * e2e_steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
           "note": "rbf_run_host per RK4 step: pinned host state -> device, one RK4 step, device -> host"}

    fp64 = None
    weights = None
    if not args.no_fp64 and args.precision == 32:
        n64, pb64, _ = make_problem(args.h, 64)
        U64 = rbffd.state_tensor(U0, 64)
        i64 = pb64.info()
        n_t = max(20, args.steps // 4)
        s64, _ = time_steps(torch, pb64, U64, dt, n_t, args.warmup, flush, False)
        t64 = float(sum(s64))
        if i64["run_mode"] == 2:      # one persistent launch per step
            avg64 = t64 / len(s64)
            flops = 4.0 * i64["rhs_flops_per_node"] * n64.n_prog
        else:
            _, k64 = time_steps(torch, pb64, U64, dt, n_t, 1, flush, True)
            avg64 = float(np.mean(k64)) / 4.0
            flops = i64["rhs_flops_per_node"] * n64.n_prog
        p64 = fp64_peak_tflops(torch)
        weights = weights_case(torch, args.h, p64)
        fp64 = {"value": 4.0 * n64.n_prog * len(s64) / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / len(s64),
                "roofline": {"bound": "alu", "achieved": flops / (avg64 / 1e3) / 1e12, "peak": p64,
                             "unit": "TFLOP/s", "frac": flops / (avg64 / 1e3) / 1e12 / p64,
                             "peak_source": "measured cuBLAS DGEMM 4096^3 in this run (nominal GB300 FP64: 1.25)",
                             "frac_of_nominal": flops / (avg64 / 1e3) / 1e12 / 1.25, "avg_launch_ms": avg64,
                             "hbm_GBps": i64["rhs_bytes_per_node"] * n64.n_prog / (avg64 / 1e3) / 1e9},
                "threads_per_node": i64["threads_per_node"],
                "run_mode": "persistent" if i64["run_mode"] == 2 else "graph",
                "persistent_lanes": i64["persist_lanes"], "persistent_ctas": i64["persist_ctas"]}
        # accuracy of the FP32 form: the whole run to 900 s in both precisions
        # (the FP64 path matches the FP64 oracle to ~1e-12), per-field
        # relative l2 of FP32 against FP64 at t_final
        n_end = int(round(900.0 / dt))
        A64 = rbffd.state_tensor(U0, 64)
        pb64.run(0.0, dt, n_end, A64)
        pb64.sync()
        A32 = rbffd.state_tensor(U0, 32)
        pb.run(0.0, dt, n_end, A32)
        pb.sync()
        f64 = rbffd.fields(A64)[:, :nodes.n_prog]
        f32 = rbffd.fields(A32)[:, :nodes.n_prog]
        fp64["fp32_error_at_900s"] = {
            "fields": ["u", "w", "theta'", "pi'"],
            "rel_l2_vs_fp64": [float(np.linalg.norm(f32[f] - f64[f]) / np.linalg.norm(f64[f])) for f in range(4)],
            "steps": n_end}
        pb64.close()

    large = None
    if args.large_h > 0:
        large = large_case(torch, args, flush)
    batched = None
    if args.ens_runs > 0:
        batched = ensemble_case(torch, args)
    learned_form = None
    if args.learned:
        learned_form = learned_case(torch, args)

    base = None
    if rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(args.h)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n_prog": nodes.n_prog, "n_ghost": nodes.n_ghost,
                           "dt_s": dt, "precision": f"fp{args.precision}",
                           "l2": "flushed between timed steps (512 MB write); working set ~31 MB",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "threads_per_node": info["threads_per_node"], "prefetch": info["prefetch"],
                           "run_mode": "persistent" if persistent else "graph",
                           "persistent_lanes": info["persist_lanes"], "persistent_chunk": info["persist_chunk"]},
                "roofline": roof, "clocks": clk.summary(), "e2e": e2e,
                "gpu_launches": (1 if persistent else info["launches_per_step"]) * args.steps,
                "setup": {"weight_build_ms": info["weight_build_ms"], "ghost_setup_ms": info["ghost_setup_ms"]},
                "sustained_run": sustained,
                "fp64": fp64, "weights": weights, "roofline_large": large, "batched": batched,
                "learned": learned_form,
                "cpu_baseline": base,
                "state_minmax": {"theta_min": mm[2, 0], "w_min": mm[1, 0], "w_max": mm[1, 1]}}
        print(json.dumps(line), flush=True)
    pb.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
