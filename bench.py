"""Throughput of the PHS RBF-FD hot path on one GB300 (or N replicas).

Headline workload: the warm rising bubble in a walled [0, 20] x [0, 10] km box
-- a +2 K cos^2 bubble of radius 2 km at (10, 2) km on a neutral 300 K base
state, 308,097 quasi-uniform Poisson-disk nodes at 25 m (seed 1) + 2,400
ghosts, PHS r^9 + degree-5 polynomials, n = 56, Delta^3 hyperviscosity from
r^9, mu = 10 m^2/s, dt = 1/16 s -- stepped in FP64, the paper's precision.
One step = one classical RK4 step: four stages, each a ghost solve (Sec. 5.2)
and one fused right-hand-side + RK4-update kernel, replayed from a CUDA graph.
Setup (stencils, weights, packing, ghost inverses) is timed separately.

Metric: node-RHS evaluations per second (4 per node per RK4 step).  The
headline's working set (operators, records, RK4 buffers: ~0.7 GB in FP64) is
several times larger than L2, so steps are timed back to back without an L2
flush, each with CUDA events on the problem's stream.  The dominant kernel is
the FP64 stage kernel, bound by the FP64 pipe: its roofline is in TFLOP/s
against a DGEMM measured in the same run.

Beside the headline, in the same JSON line:
  bubble_fp32      the same workload with FP64-built weights stored in FP32
                   and FP32 stages (HBM roofline), and its per-field error at
                   t = 1000 s against the FP64 run
  density_current  Sec. 6.3 at hexagonal 100 m (38,400 nodes, n = 37, r^7 +
                   deg 4): FP32 in one persistent launch per step (L2
                   flushed between steps), FP64, and FP32's error at 900 s
  advection        the deformational-flow scalar on 64 x 64 nodes, one period
  weights          the FP64 weight build of the headline node set
  roofline_large   the density current at 25 m (608k nodes): the FP32 stage
                   kernel against HBM, per-node and lattice operator storage
  batched          256 uneven density-current members in FP32 and FP64, and
                   the FP32 error at 900 s on a subset
  learned          the coarse-grid correction against plain runs at a stated
                   error

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on a bounded sample of the headline workload: one 1/16-width
strip of the walled box per host core.
"""
import argparse
import hashlib
import json
import math
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
LEGS = ("headline", "bubble_fp32", "density_current", "advection", "weights", "large", "batched", "learned")
STRIPS = 16          # the CPU sample: 1/16-width strips of the walled box


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--legs", default="all",
                    help="comma list of " + ",".join(LEGS) + " (default all); the headline always runs")
    ap.add_argument("--bubble-h", type=float, default=25.0, help="node spacing of the headline bubble (m)")
    ap.add_argument("--bubble-threads", type=int, default=0, choices=(0, 1, 2, 4, 8),
                    help="lanes per node of the bubble legs (0 = autotuned at creation; fixing it makes profiled "
                         "runs reproducible)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-final-error", action="store_true",
                    help="skip the whole runs to t_final that state the FP32 forms' errors")
    ap.add_argument("--h", type=float, default=100.0, help="density-current spacing (m)")
    ap.add_argument("--threads-per-node", type=int, default=0, help="density current: 0 = autotuned")
    ap.add_argument("--run-mode", default="auto", choices=["auto", "graph", "persistent"],
                    help="density current FP32 run mode (auto: timed at creation)")
    ap.add_argument("--persistent-lanes", type=int, default=1, help="lanes per node with --run-mode persistent")
    ap.add_argument("--persistent-ctas", type=int, default=0, help="CTAs with --run-mode persistent (0: one per SM)")
    ap.add_argument("--ens-runs", type=int, default=256, help="ensemble members (0 = skip the batched case)")
    ap.add_argument("--ens-steps", type=int, default=40, help="timed global RK4 steps of the ensemble")
    ap.add_argument("--ens-final-members", type=int, default=32,
                    help="members run to 900 s in FP32 and FP64 for the batched error at t_final")
    ap.add_argument("--ens-threads", type=int, default=0, choices=(0, 1, 2, 4),
                    help="lanes per node of the batched ensembles (0 = autotuned)")
    ap.add_argument("--learned-coarse", type=float, default=400.0)
    ap.add_argument("--learned-ratio", type=int, default=4)
    ap.add_argument("--learned-seeds", type=int, default=16)
    ap.add_argument("--learned-iters", type=int, default=30000)
    ap.add_argument("--large-h", type=float, default=25.0,
                    help="spacing of the HBM-roofline density current; its working set exceeds L2")
    a = ap.parse_args()
    a.legs = set(LEGS) if a.legs == "all" else {"headline"} | {s.strip() for s in a.legs.split(",") if s.strip()}
    unknown = a.legs - set(LEGS)
    if unknown:
        ap.error(f"unknown legs {sorted(unknown)}")
    return a


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


def bubble_workload(h):
    from paper_1509_02615_gb300 import configs
    return configs.bubble(h=h, seed=1, t_end=1000.0)


def headline_config(wl, world):
    """The headline's config object (the same in both arms)."""
    nd = wl.nodes
    return {"workload": f"warm bubble in a walled [0,20]x[0,10] km box, Poisson-disk nodes at {nd.h:g} m "
                        f"({nd.n_prog} + {nd.n_ghost} ghosts), r^9 + deg 5, n=56, Delta^3 from r^9, mu=10, "
                        f"dt={wl.dt:g} s",
            "n_prog": nd.n_prog, "n_ghost": nd.n_ghost, "dt_s": wl.dt, "precision": "fp64",
            "l2": "not flushed: inputs larger than L2 (~0.7 GB of FP64 operators, records and RK4 buffers)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def time_run(torch, pb, U, t0, dt, n_steps):
    """Device time (ms) of one rbf_run of n_steps on the current stream."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pb.run(t0, dt, n_steps, U)
    e1.record(stream)
    e1.synchronize()
    pb.sync()
    return e0.elapsed_time(e1)


def rel_fields(a, b):
    """Per-field relative l2 of field-major arrays [4, n]."""
    return [float(np.linalg.norm(a[f] - b[f]) / max(np.linalg.norm(b[f]), 1e-300)) for f in range(a.shape[0])]


def headline_case(torch, args, wl, world, local, p64):
    """The headline: FP64 RK4 steps of the bubble, each timed with CUDA
    events; then the same steps with events around the four stage kernels
    (the dominant kernel's average launch time); then the end-to-end form on
    a pinned host state."""
    from paper_1509_02615_gb300 import rbffd
    nodes = wl.nodes
    t0 = time.perf_counter()
    pb = rbffd.ns_problem(nodes, precision=64, threads_per_node=args.bubble_threads, **wl.params)
    create_s = time.perf_counter() - t0
    info = pb.info()
    U = rbffd.state_tensor(wl.U0, 64)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms, _ = time_steps(torch, pb, U, wl.dt, args.steps, args.warmup, None, False, nvtx="timed")
        torch.cuda.synchronize()
    _, stage_ms = time_steps(torch, pb, U, wl.dt, args.steps, 1, None, True)
    mm = pb.minmax(U)   # fails loudly on NaN/Inf
    total_ms = max_over_ranks(sum(step_ms), world)
    value = whole_job_rate(4.0 * nodes.n_prog * args.steps, world, total_ms / 1e3)
    persistent = info["run_mode"] == 2
    if persistent:
        avg_ms = float(np.mean(step_ms))
        flops = 4.0 * info["rhs_flops_per_node"] * nodes.n_prog
        kernel, share = "rk4_persistent", 1.0
    else:
        avg_ms = float(np.mean(stage_ms)) / 4.0
        flops = info["rhs_flops_per_node"] * nodes.n_prog
        kernel, share = "ns_stage_kernel<double>", float(np.sum(stage_ms) / np.sum(step_ms))
    ach = flops / (avg_ms / 1e3) / 1e12
    key = f"ns_stage_fp64_bubble{int(nodes.h)}"
    roof = {"bound": "alu", "achieved": ach, "peak": p64, "unit": "TFLOP/s", "frac": ach / p64,
            "traffic": None if persistent else profiled_traffic(key, threads_per_node=info["threads_per_node"]),
            "kernel": kernel, "algorithmic_flops_per_launch": flops,
            "algorithmic_bytes_per_launch": info["rhs_bytes_per_node"] * nodes.n_prog * (4 if persistent else 1),
            "avg_launch_ms": avg_ms, "kernel_share_of_step": share,
            "peak_source": "FP64 DGEMM (cuBLAS via torch.matmul, 4096^3) measured in this run; GB300 nominal FP64 "
                           "1.25 TFLOP/s", "frac_of_nominal": ach / 1.25,
            "hbm_GBps": info["rhs_bytes_per_node"] * nodes.n_prog * (4 if persistent else 1) / (avg_ms / 1e3) / 1e9}
    # end to end through the C ABI: pinned host state -> device, one RK4 step, device -> host
    Uh = rbffd.state_tensor(wl.U0, 64, device="cpu").pin_memory()
    n_e2e = max(5, args.steps // 4)
    pb.run_host(0.0, wl.dt, 1, Uh)
    t0 = time.perf_counter()
    for s in range(n_e2e):
        pb.run_host(s * wl.dt, wl.dt, 1, Uh)
    e2e_s = time.perf_counter() - t0
    state_bytes = Uh.numel() * Uh.element_size()
    e2e = {"value": 4.0 * nodes.n_prog * n_e2e * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
           "note": "rbf_run_host per RK4 step: pinned host state -> device, one RK4 step, device -> host"}
    out = {"value": value, "ms_per_step": total_ms / args.steps, "roofline": roof, "clocks": clk.summary(),
           "e2e": e2e, "gpu_launches": (1 if persistent else info["launches_per_step"]) * args.steps,
           "launch": {"run_mode": "persistent" if persistent else "graph",
                      "threads_per_node": info["threads_per_node"], "prefetch": info["prefetch"],
                      "stage_split": info["stage_split"], "launches_per_step": info["launches_per_step"]},
           "setup": {"create_s": create_s, "weight_build_ms": info["weight_build_ms"],
                     "ghost_setup_ms": info["ghost_setup_ms"]},
           "state_minmax": {"theta_max": float(mm[2, 1]), "w_min": float(mm[1, 0]), "w_max": float(mm[1, 1])}}
    return pb, out


def bubble_fp32_case(torch, args, wl, pb64, pk, pk_kind):
    """The headline workload in FP32 (FP64-built weights stored in FP32): its
    throughput, the stage kernel's HBM roofline, and both precisions run to
    t = 1000 s: FP32's per-field error against FP64 there, and the time of
    each whole run."""
    from paper_1509_02615_gb300 import rbffd
    nodes = wl.nodes
    pb = rbffd.ns_problem(nodes, precision=32, threads_per_node=args.bubble_threads, **wl.params)
    info = pb.info()
    U = rbffd.state_tensor(wl.U0, 32)
    step_ms, _ = time_steps(torch, pb, U, wl.dt, args.steps, args.warmup, None, False, nvtx="timed_fp32")
    _, stage_ms = time_steps(torch, pb, U, wl.dt, args.steps, 1, None, True)
    avg = float(np.mean(stage_ms)) / 4.0
    bpl = info["rhs_bytes_per_node"] * nodes.n_prog
    ach = bpl / (avg / 1e3) / 1e9
    out = {"workload": "the headline workload, FP64-built weights stored in FP32, FP32 stages",
           "value": 4.0 * nodes.n_prog * args.steps / (float(sum(step_ms)) / 1e3), "unit": UNIT,
           "ms_per_step": float(sum(step_ms)) / args.steps, "dtype": "f32",
           "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / pk["hbm_gbs"], "kernel": "ns_stage_kernel<float>",
                        "traffic": profiled_traffic(f"ns_stage_fp32_bubble{int(nodes.h)}",
                                                    threads_per_node=info["threads_per_node"]),
                        "algorithmic_bytes_per_launch": bpl, "avg_launch_ms": avg,
                        "kernel_share_of_step": float(np.sum(stage_ms) / np.sum(step_ms)),
                        "peak_source": f"{pk_kind} hbm_gbs"},
           "threads_per_node": info["threads_per_node"], "stage_split": info["stage_split"],
           "launches_per_step": info["launches_per_step"]}
    if not args.no_final_error:
        A32 = rbffd.state_tensor(wl.U0, 32)
        ms32 = time_run(torch, pb, A32, 0.0, wl.dt, wl.n_steps)
        A64 = rbffd.state_tensor(wl.U0, 64)
        ms64 = time_run(torch, pb64, A64, 0.0, wl.dt, wl.n_steps)
        f32 = rbffd.fields(A32)[:, :nodes.n_prog]
        f64 = rbffd.fields(A64)[:, :nodes.n_prog]
        out["error_at_1000s"] = {"fields": ["u", "w", "theta'", "pi'"], "rel_l2_fp32_vs_fp64": rel_fields(f32, f64),
                                 "steps": wl.n_steps,
                                 "note": "the FP64 run matches the FP64 oracle (tests); FP32 against it at t_final"}
        out["time_to_1000s_s"] = {"fp32": ms32 / 1e3, "fp64": ms64 / 1e3, "fp32_speedup": ms64 / ms32}
    pb.close()
    return out


def make_dc_problem(h, precision, tpn=0, run_mode="auto", lanes=1, ctas=0):
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


def density_current_case(torch, args, pk, pk_kind, p64, flush):
    """Sec. 6.3 at hexagonal 100 m: FP32 (each RK4 step one persistent
    launch when that is faster, L2 flushed between steps: the working set is
    ~31 MB), a sustained 400-step run, FP64, and FP32's error at 900 s."""
    from paper_1509_02615_gb300 import rbffd
    nodes, pb, U0 = make_dc_problem(args.h, 32, args.threads_per_node, args.run_mode, args.persistent_lanes,
                                    args.persistent_ctas)
    info = pb.info()
    dt = args.h / 400.0
    U = rbffd.state_tensor(U0, 32)
    persistent = info["run_mode"] == 2
    step_ms, _ = time_steps(torch, pb, U, dt, args.steps, args.warmup, flush, False, nvtx="dc_timed")
    stage_ms = [] if persistent else time_steps(torch, pb, U, dt, args.steps, 1, flush, True)[1]
    if persistent:
        avg_ms, bpl, kernel, share = float(np.mean(step_ms)), 4.0 * info["rhs_bytes_per_node"] * nodes.n_prog, \
            "rk4_persistent", 1.0
    else:
        avg_ms, bpl, kernel = float(np.mean(stage_ms)) / 4.0, info["rhs_bytes_per_node"] * nodes.n_prog, \
            "ns_stage_kernel<float>"
        share = float(np.sum(stage_ms) / np.sum(step_ms))
    ach = bpl / (avg_ms / 1e3) / 1e9
    key = f"{'persistent' if persistent else 'ns_stage'}_fp32_hex{int(args.h)}"
    launch = ({"persistent_lanes": info["persist_lanes"], "persistent_ctas": info["persist_ctas"]} if persistent
              else {"threads_per_node": info["threads_per_node"]})
    out = {"workload": f"density current (Sec. 6.3), hexagonal {args.h:g} m, {nodes.n_prog} nodes + "
                       f"{nodes.n_ghost} ghosts, r^7 + deg 4, n=37, Delta^3, mu=75, dt={dt:g} s",
           "value": 4.0 * nodes.n_prog * args.steps / (float(sum(step_ms)) / 1e3), "unit": UNIT, "dtype": "f32",
           "ms_per_step": float(sum(step_ms)) / args.steps,
           "l2": "flushed between timed steps (512 MB write); working set ~31 MB",
           "run_mode": "persistent" if persistent else "graph", "threads_per_node": info["threads_per_node"],
           "persistent_lanes": info["persist_lanes"], "persistent_chunk": info["persist_chunk"],
           "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / pk["hbm_gbs"], "traffic": profiled_traffic(key, **launch), "kernel": kernel,
                        "algorithmic_bytes_per_launch": bpl, "avg_launch_ms": avg_ms, "kernel_share_of_step": share,
                        "peak_source": f"{pk_kind} hbm_gbs",
                        "note": "the working set fits in L2: latency-bound, reported against HBM for reference"}}
    # a sustained run (one rbf_run of many steps, L2 flushed once before it)
    sus = 400
    flush.zero_()
    Us = rbffd.state_tensor(U0, 32)
    sus_ms = time_run(torch, pb, Us, 0.0, dt, sus)
    out["sustained_run"] = {"value": 4.0 * nodes.n_prog * sus / (sus_ms / 1e3), "unit": UNIT, "steps": sus,
                            "ms_per_step": sus_ms / sus}
    n64, pb64, _ = make_dc_problem(args.h, 64)
    i64 = pb64.info()
    U64 = rbffd.state_tensor(U0, 64)
    s64, _ = time_steps(torch, pb64, U64, dt, args.steps, args.warmup, flush, False)
    t64 = float(sum(s64))
    if i64["run_mode"] == 2:
        avg64, flops = t64 / len(s64), 4.0 * i64["rhs_flops_per_node"] * n64.n_prog
    else:
        _, k64 = time_steps(torch, pb64, U64, dt, args.steps, 1, flush, True)
        avg64, flops = float(np.mean(k64)) / 4.0, i64["rhs_flops_per_node"] * n64.n_prog
    out["fp64"] = {"value": 4.0 * n64.n_prog * len(s64) / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / len(s64),
                   "run_mode": "persistent" if i64["run_mode"] == 2 else "graph",
                   "roofline": {"bound": "alu", "achieved": flops / (avg64 / 1e3) / 1e12, "peak": p64,
                                "unit": "TFLOP/s", "frac": flops / (avg64 / 1e3) / 1e12 / p64,
                                "peak_source": "measured FP64 DGEMM in this run", "avg_launch_ms": avg64}}
    if not args.no_final_error:
        n_end = int(round(900.0 / dt))
        A64 = rbffd.state_tensor(U0, 64)
        ms64 = time_run(torch, pb64, A64, 0.0, dt, n_end)
        A32 = rbffd.state_tensor(U0, 32)
        ms32 = time_run(torch, pb, A32, 0.0, dt, n_end)
        f64 = rbffd.fields(A64)[:, :nodes.n_prog]
        f32 = rbffd.fields(A32)[:, :nodes.n_prog]
        out["error_at_900s"] = {"fields": ["u", "w", "theta'", "pi'"], "rel_l2_fp32_vs_fp64": rel_fields(f32, f64),
                                "steps": n_end}
        out["time_to_900s_s"] = {"fp32": ms32 / 1e3, "fp64": ms64 / 1e3, "fp32_speedup": ms64 / ms32}
    pb64.close()
    pb.close()
    return out


def advection_case(torch):
    """The deformational-flow scalar (64 x 64 nodes, r^7 + deg 4, n = 37,
    Delta^4 from r^9): one whole period T = 5 (1000 RK4 steps) in FP64 and
    FP32, after a warm-up period."""
    from paper_1509_02615_gb300 import configs
    from paper_1509_02615_gb300 import rbffd
    wl = configs.advection(64)
    n = wl.nodes.n_prog
    out = {"workload": f"scalar advection in the deformational flow, Cartesian 64 x 64 ({n} nodes + reflected "
                       f"layers), r^7 + deg 4, n=37, Delta^4 from r^9, {wl.n_steps} RK4 steps to t = T"}
    for prec in (64, 32):
        pb = rbffd.advection_problem(wl.nodes, precision=prec, **wl.params)
        P = rbffd.state_tensor(wl.U0, prec)
        time_run(torch, pb, P, 0.0, wl.dt, wl.n_steps)
        P = rbffd.state_tensor(wl.U0, prec)
        ms = time_run(torch, pb, P, 0.0, wl.dt, wl.n_steps)
        psi = rbffd.fields(P)[0]
        info = pb.info()
        persistent = info["run_mode"] == 2
        out[f"fp{prec}"] = {"value": 4.0 * n * wl.n_steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / wl.n_steps,
                            "return_error_rel_l2": float(np.linalg.norm(psi - wl.U0) / np.linalg.norm(wl.U0)),
                            "run_mode": "persistent" if persistent else "graph",
                            "threads_per_node": info["threads_per_node"],
                            "launches_per_run": 1 if persistent else info["launches_per_step"] * wl.n_steps}
        if persistent:
            out[f"fp{prec}"]["persistent_ctas"] = info["persist_ctas"]
        pb.close()
    return out


def weights_case(torch, nodes, n, p, l, hv_k, peak_tflops, label):
    """a2 alone: the FP64 weight build of a node set through the C ABI
    (rbf_build_weights: d/dx, d/dz, Lap, d2/dx2, d2/dz2 and Delta^k, all from
    r^p with degree l, so one augmented system of size S = n + M per node with
    K = 6 right-hand sides), timed with CUDA events after a warm-up build.
    Algorithmic flops per node: (2/3) S^3 + 2 K S^2."""
    from paper_1509_02615_gb300 import rbffd
    x = torch.as_tensor(nodes.x, device="cuda")
    z = torch.as_tensor(nodes.z, device="cuda")
    idx = rbffd.build_stencils(x, z, nodes.n_prog, n, nodes.period_x)
    ops = ("dx", "dz", "lap", "dxx", "dzz", "hv")
    stream = torch.cuda.current_stream()

    def build():
        rbffd.build_weights(x, z, idx, p, l, ops, hv_k, nodes.period_x)

    build()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(f"weights_S{n + (l + 1) * (l + 2) // 2}")
    e0.record(stream)
    build()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    S = n + (l + 1) * (l + 2) // 2
    flops = nodes.n_prog * ((2.0 / 3.0) * S ** 3 + 2.0 * len(ops) * S ** 2)
    ach = flops / (ms / 1e3) / 1e12
    return {"workload": f"FP64 weights of the {nodes.n_prog} prognostic nodes of {label} (6 operators from r^{p}, "
                        f"degree {l}, n = {n}: one augmented system of size S = {S} per node)",
            "ms": ms, "nodes_per_s": nodes.n_prog / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": ach / peak_tflops, "algorithmic_flops": flops,
                         "peak_source": "measured FP64 DGEMM in this run"}}


def time_steps(torch, pb, U, dt, steps, warmup, flush, stage_timing, nvtx=None):
    """Per-step device times (ms) and summed stage-kernel times (ms).  With a
    ``flush`` buffer, L2 is evicted before every step (for working sets that
    fit in L2) and each step is timed on its own; without one (and without
    stage timing) the timed steps are enqueued back to back between one pair
    of events (one ``run`` call per step, as in the warm-up, so the host's
    launch latency overlaps the device work) and each step gets the mean.
    ``nvtx`` names an NVTX range around the timed steps (for a profiler's
    launch filter)."""
    stream = torch.cuda.current_stream()
    pb.set_stage_timing(stage_timing)
    t = 0.0
    for _ in range(warmup):
        if flush is not None:
            flush.zero_()
        pb.run(t, dt, 1, U)
        t += dt
    torch.cuda.synchronize()
    step_ms, stage_ms = [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    if flush is None and not stage_timing:
        e0.record(stream)
        for _ in range(steps):
            pb.run(t, dt, 1, U)
            t += dt
        e1.record(stream)
        e1.synchronize()
        step_ms = [e0.elapsed_time(e1) / steps] * steps
    else:
        for _ in range(steps):
            if flush is not None:
                flush.zero_()
            e0.record(stream)
            pb.run(t, dt, 1, U)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            if stage_timing:
                stage_ms.append(pb.stage_kernel_ms())
            t += dt
    if nvtx:
        torch.cuda.nvtx.range_pop()
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


def large_case(torch, args, flush):
    """The same density current at a finer spacing, whose FP32 working set is
    several times larger than L2: the stage kernel's HBM roofline."""
    from paper_1509_02615_gb300 import rbffd
    pk, pk_kind = peaks()
    nodes, pb, U0 = make_dc_problem(args.large_h, 32, tpn=args.threads_per_node)
    info = pb.info()
    U = rbffd.state_tensor(U0, 32)
    dt = args.large_h / 400.0
    steps = 10
    step_ms, _ = time_steps(torch, pb, U, dt, steps, 3, flush, False, nvtx="large_timed")
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
           "stage_split": info["stage_split"],
           "setup": {"weight_build_ms": info["weight_build_ms"], "ghost_setup_ms": info["ghost_setup_ms"]}}
    # f4: the same steps with lattice operator storage (one operator row per
    # class of translated stencils); its bytes per node-RHS follow the storage
    Ur = U.clone()
    t0 = time.perf_counter()
    cn, nc = pb.set_operator_storage("lattice", args.threads_per_node)
    lat_setup_s = time.perf_counter() - t0
    li = pb.info()
    Ul = rbffd.state_tensor(U0, 32)
    lstep, _ = time_steps(torch, pb, Ul, dt, steps, 3, flush, False, nvtx="large_lattice_timed")
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


def _time_ensemble(torch, ens, K, nvtx):
    """Node-updates/s of K global RK4 steps (after K untimed ones, which also
    build the run's graph) and the median stage-kernel time of 3 more, for an
    ensemble's initial state; ``nvtx`` names an NVTX range around the K timed
    steps and ``nvtx + "_stages"`` one around the 3 stage-timed steps (plain
    kernel launches, which an ncu capture can select)."""
    U = ens.state()
    stream = torch.cuda.current_stream()
    ens.run(K, U)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(nvtx)
    e0.record(stream)
    ens.run(K, U)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    ens.set_stage_timing(True)
    stage = []
    torch.cuda.nvtx.range_push(nvtx + "_stages")
    for _ in range(3):
        ens.run(1, U)
        stage.append(ens.stage_kernel_ms() / 4.0)
    torch.cuda.nvtx.range_pop()
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
    ms, avg, finite, U = _time_ensemble(torch, ens, K, "ens_per_node")
    upd = sum_over_ranks(ens.node_updates(K), world)
    ms = max_over_ranks(ms, world)
    bpl = info["rhs_bytes_per_node"] * ens.n_prog
    ach = bpl / (avg / 1e3) / 1e9
    out = {"workload": f"{len(every)} density-current members, {ens.n_prog} nodes + {ens.n_all - ens.n_prog} ghosts "
                       f"on this rank ({len(members)} members), h in 50-400 m, cart/hex/scattered, n 31-75 "
                       f"(Cartesian without n=75 l=5; Cartesian n=31 l=3 with hyperviscosity constant 2^-5), FP32",
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
    ms64, _, fin64, U64 = _time_ensemble(torch, e64, K, "ens_fp64")
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
    if not args.no_final_error and args.ens_final_members > 0:
        out["error_at_900s"] = ensemble_final_error(torch, members[:args.ens_final_members], args.ens_threads)
    t0 = time.perf_counter()
    lens = rbffd.ensemble_problem(members, precision=32, storage="lattice", threads_per_node=args.ens_threads)
    build_s = time.perf_counter() - t0
    li = lens.info()
    lms, lavg, lfin, LU = _time_ensemble(torch, lens, K, "ens_lattice")
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


def ensemble_final_error(torch, members, threads):
    """The first members of this rank's share run to t = 900 s (each member
    to its own step count) in FP32 and in FP64: per-field relative l2 of the
    concatenated FP32 states against FP64 at t_final, and both run times."""
    from paper_1509_02615_gb300 import rbffd
    res = {}
    for prec in (32, 64):
        ens = rbffd.ensemble_problem(members, precision=prec, threads_per_node=threads)
        U = ens.state()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.run(-1, U)
        e1.record(stream)
        e1.synchronize()
        res[prec] = (U.cpu().double(), e0.elapsed_time(e1), ens.node_updates(-1))
        ens.close()
        del U
    (a, ms32, upd), (b, ms64, _) = res[32], res[64]
    prog = np.concatenate([np.arange(r0, r0 + m.nodes.n_prog) for r0, m in
                           zip(np.cumsum([0] + [m.nodes.n_all for m in members])[:-1], members)])
    a, b = a[prog], b[prog]
    return {"members": len(members), "node_updates": upd,
            "fields": ["u", "w", "theta'", "pi'"],
            "rel_l2_fp32_vs_fp64": [float(torch.linalg.vector_norm(a[:, f] - b[:, f]) /
                                          torch.linalg.vector_norm(b[:, f])) for f in range(4)],
            "seconds_to_900s": {"fp32": ms32 / 1e3, "fp64": ms64 / 1e3, "fp32_speedup": ms64 / ms32},
            "finite": bool(torch.isfinite(a).all() and torch.isfinite(b).all())}


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
    mlp, loss = learned.train(ds, n_train, iters=args.learned_iters, batch=4096, lr=2e-3)
    t_train = time.perf_counter() - t0
    alpha, scores = learned.select_alpha(ds, mlp, range(n_train, n_train + n_val))
    test = list(range(n_train + n_val, ns))
    err_plain = learned.run_errors(ds, mlp, test, (0.0, 0.0, 0.0, 0.0))
    err_learned = learned.run_errors(ds, mlp, test, alpha)
    skill = learned.prediction_skill(ds, mlp, range(n_train, n_train + n_val))
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
    # error against cost: plain runs at the coarse spacing, 1/sqrt(2) of it and
    # half of it, in FP64 and FP32, restricted to the coarse nodes the same way
    # as the reference; the learned point is placed on that curve
    coarse_nodes = ds.coarse_nodes
    curve = []
    for h in (hc, hc / math.sqrt(2.0), hc / 2.0):
        nodes_h = inp.density_current_nodes(h)
        aidx, aw = inp.restriction_average(coarse_nodes, nodes_h, np.zeros(nc, np.int64), radius=hc,
                                           sigma=0.5 * hc)
        aidx_t = torch.as_tensor(aidx, device="cuda")
        aw_t = torch.as_tensor(aw, device="cuda")
        if h == hc:
            # the learned run through the same restriction as the plain runs
            errs_r = []
            for r in test:
                V = ds.states[r, 0].clone()
                mlp.run(0.0, ds.dt_c, steps, V, alpha=alpha)
                res = torch.zeros((coarse_nodes.n_all, 4), dtype=torch.float32, device="cuda")
                rbffd.restrict_weighted(V, 32, aidx_t, aw_t, res, nc, coarse_nodes.n_all)
                errs_r.append(learned.rel_l2(res[:nc], ds.states[r, -1, :nc]))
            err_learned_r = np.mean(errs_r, axis=0)
        n_steps = int(math.ceil(900.0 * 400.0 / h - 1e-9))
        dt_h = 900.0 / n_steps
        for prec in (64, 32):
            pb_h = rbffd.ns_problem(nodes_h, precision=prec)
            errs, ms = [], 0.0
            for r in test:
                U = rbffd.state_tensor(inp.perturbed_density_current(nodes_h, seeds[r]), prec)
                ms += time_run(torch, pb_h, U, 0.0, dt_h, n_steps)
                res = torch.zeros((coarse_nodes.n_all, 4), dtype=torch.float32, device="cuda")
                rbffd.restrict_weighted(U, prec, aidx_t, aw_t, res, nc, coarse_nodes.n_all)
                errs.append(learned.rel_l2(res[:nc], ds.states[r, -1, :nc]))
            pb_h.close()
            curve.append({"h_m": h, "precision": prec, "nodes": nodes_h.n_prog, "steps": n_steps,
                          "ms_to_900s": ms / len(test), "rel_l2": [float(v) for v in np.mean(errs, axis=0)],
                          "rel_l2_mean": float(np.mean(errs)),
                          "node_updates_per_s": nodes_h.n_prog * n_steps * len(test) / (ms / 1e3)})
    e_l = float(np.mean(err_learned_r))
    def cost_at(prec, e):
        """GPU time to 900 s of the plain runs in one precision at error e:
        log-log interpolation between the curve points that bracket it
        (None outside the curve)."""
        pts = sorted((c for c in curve if c["precision"] == prec), key=lambda c: c["rel_l2_mean"])
        for lo, hi in zip(pts[:-1], pts[1:]):
            if lo["rel_l2_mean"] <= e <= hi["rel_l2_mean"]:
                w = (math.log(e) - math.log(hi["rel_l2_mean"])) / (math.log(lo["rel_l2_mean"]) -
                                                                   math.log(hi["rel_l2_mean"]))
                return math.exp(math.log(hi["ms_to_900s"]) +
                                w * (math.log(lo["ms_to_900s"]) - math.log(hi["ms_to_900s"])))
        return None
    dominated = any(c["ms_to_900s"] <= ms_learned and c["rel_l2_mean"] <= e_l
                    for c in curve if c["precision"] == 64)
    t64 = cost_at(64, e_l)
    t32 = cost_at(32, e_l)

    def speedup_floor(prec):
        """Learned error below every plain run of a precision: the most
        accurate plain run's time over the learned time, a lower bound on the
        speedup at equal error (a plain run as accurate would be finer still)."""
        pts = [c for c in curve if c["precision"] == prec]
        best = min(pts, key=lambda c: c["rel_l2_mean"])
        return best["ms_to_900s"] / ms_learned if e_l <= best["rel_l2_mean"] else None
    mid = [c for c in curve if c["precision"] == 64 and abs(c["h_m"] - hc / 2.0) < 1e-6][0]
    out = {"workload": f"density current, hexagonal {hc:g} m coarse ({nc} nodes), MLP trained on {hc / ratio:g} m FP64 "
                       f"runs restricted to the coarse nodes ({n_train} train / {n_val} validation / {len(test)} test "
                       f"seeds), t = 900 s; the task's set-up uses 50 m runs of 64 seeds, this default is that "
                       f"set-up scaled down to {hc / ratio:g} m and {ns} seeds (--learned-ratio 8 --learned-seeds 64 "
                       f"runs the full one)",
           "selected_alpha": alpha, "validation_scores": [[sc, list(a)] for sc, a in scores],
           "validation_skill": {"fields": ["u", "w", "theta'", "pi'"],
                                "fraction_of_defect_variance_predicted": [float(v) for v in skill]},
           "rel_l2_test": {"fields": ["u", "w", "theta'", "pi'"],
                           "uncorrected_coarse_fp32": [float(v) for v in err_plain],
                           "learned_coarse_fp32": [float(v) for v in err_learned],
                           "learned_coarse_fp32_restricted_as_the_curve": [float(v) for v in err_learned_r],
                           f"uncorrected_{hc / 2:g}m_fp64": mid["rel_l2"]},
           "node_updates_per_s": {"learned_coarse_fp32": nc * steps / (ms_learned / 1e3),
                                  "uncorrected_coarse_fp32": nc * steps / (ms_plain / 1e3),
                                  f"uncorrected_{hc / 2:g}m_fp64": mid["node_updates_per_s"],
                                  "fine_reference_fp64_batched": ds.fine_node_updates / ds.fine_seconds},
           "ms_to_900s": {"learned_coarse_fp32": ms_learned, "uncorrected_coarse_fp32": ms_plain,
                          f"uncorrected_{hc / 2:g}m_fp64": mid["ms_to_900s"]},
           "error_cost_curve": curve,
           "stated_error": {"metric": "mean over fields and test seeds of the relative l2 error at 900 s against "
                                      "the restricted fine FP64 reference",
                            "learned_coarse_fp32": float(np.mean(err_learned)),
                            "learned_coarse_fp32_restricted_as_the_curve": e_l,
                            "uncorrected_coarse_fp32": float(np.mean(err_plain)),
                            f"uncorrected_{hc / 2:g}m_fp64": mid["rel_l2_mean"],
                            "fp64_run_faster_and_as_accurate_exists": dominated,
                            "fp64_ms_at_learned_error": t64,
                            "speedup_vs_fp64_at_learned_error": None if t64 is None else t64 / ms_learned,
                            "fp32_ms_at_learned_error": t32,
                            "speedup_vs_fp32_at_learned_error": None if t32 is None else t32 / ms_learned,
                            "learned_error_below_every_plain_run": speedup_floor(64) is not None,
                            "speedup_vs_fp64_at_least": speedup_floor(64),
                            "speedup_vs_fp32_at_least": speedup_floor(32)},
           "final_training_loss": float(np.mean(loss[-50:])),
           "seconds": {"data": t_data, "train": t_train}}
    mlp.close()
    return out


def _strip_nodes(h, k):
    """Strip k of the headline's walled box: 1/STRIPS of its width, the same
    spacing, stencils, operators and walls (Poisson-disk nodes, seed 1 + k),
    with the warm bubble centred in the strip."""
    from paper_1509_02615_gb300 import inputs as inp
    width = 20000.0 / STRIPS
    nodes = inp.poisson_disk_nodes(0.0, width, 0.0, 10000.0, h, seed=1 + k)
    U = inp.warm_bubble_state(nodes, xc=0.5 * width, R=min(2000.0, 0.4 * width))
    return nodes, U


def _oracle_strip(h, k):
    """The FP64 oracle on strip k, its setup time (stencils, weights, ghost
    factorisations) and a state one step in."""
    from oracle.ns import NSOracle
    from paper_1509_02615_gb300 import configs
    nodes, U = _strip_nodes(h, k)
    t0 = time.perf_counter()
    o = NSOracle(nodes, **configs.BUBBLE_METHOD)
    setup_s = time.perf_counter() - t0
    U = o.rk4_step(0.0, h / 400.0, U)
    return nodes, o, U, setup_s


def _oracle_rhs_rate(args):
    """RHS evaluations of one strip for budget_s seconds: (evaluations,
    nodes, seconds, setup seconds).  Runs in a spawned worker process."""
    h, k, budget_s = args
    nodes, o, U, setup_s = _oracle_strip(h, k)
    t0 = time.perf_counter()
    n_eval = 0
    while time.perf_counter() - t0 < budget_s:
        o.rhs(0.0, U)
        n_eval += 1
    return n_eval, nodes.n_prog, time.perf_counter() - t0, setup_s


def _spawn_pool_map(fn, jobs):
    """Map fn over jobs in spawned single-threaded worker processes, one per
    job, at most one per host core."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"          # the workers' BLAS stays single-threaded
    try:
        with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
            return pool.map(fn, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_baseline(h, budget_s=10.0):
    """FP64 oracle node-RHS/s on the host cores: one strip per core (up to
    STRIPS strips) in spawned single-threaded processes."""
    cores = min(os.cpu_count() or 1, STRIPS)
    res = _spawn_pool_map(_oracle_rhs_rate, [(h, k, budget_s) for k in range(cores)])
    value = sum(ne * npg / t for ne, npg, t, _ in res)
    n0, npg0, t_0, setup0 = res[0]
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle RHS (ghost solves + sparse DM products) on {cores} strips of the workload, each "
                      f"1/{STRIPS} of its width ({npg0} nodes; same spacing, stencils, operators and walls), one strip "
                      f"per core in spawned single-threaded processes, {sum(r[0] for r in res)} evaluations in "
                      f"{budget_s:.0f} s each",
            "single_strip": {"value": n0 * npg0 / t_0, "cores": 1, "evaluations": n0, "seconds": t_0},
            "oracle_setup_s": setup0}


def _oracle_rk4_steps(args):
    """W untimed and K timed oracle RK4 steps on one strip: (nodes, seconds).
    Runs in a spawned worker process."""
    h, k, warmup, steps = args
    nodes, o, U, _ = _oracle_strip(h, k)
    dt = h / 400.0
    for s in range(warmup):
        U = o.rk4_step((1 + s) * dt, dt, U)
    t0 = time.perf_counter()
    for s in range(steps):
        U = o.rk4_step((1 + warmup + s) * dt, dt, U)
    return nodes.n_prog, time.perf_counter() - t0


def run_reference(args, rank, world):
    """The oracle arm: W untimed and K timed RK4 steps of the FP64 oracle on
    strips of the headline workload, one strip per host core in spawned
    single-threaded processes; one step is four right-hand sides with their
    ghost solves.  The rate sums the strips' node-RHS/s."""
    if rank != 0:
        return
    from paper_1509_02615_gb300 import configs
    t_start = time.perf_counter()
    cores = min(os.cpu_count() or 1, STRIPS)
    res = _spawn_pool_map(_oracle_rk4_steps, [(args.bubble_h, k, args.warmup, args.steps) for k in range(cores)])
    value = sum(4.0 * n * args.steps / el for n, el in res)
    ms_step = 1e3 * float(np.mean([el for _, el in res])) / max(args.steps, 1)
    n_strip = res[0][0]
    sample = (f"FP64 oracle RK4 steps (ghost solves + sparse DM products) on {cores} strips of the workload, each "
              f"1/{STRIPS} of its width ({n_strip} nodes; same spacing, stencils, operators and walls), one strip per "
              f"core in spawned single-threaded processes: {args.warmup} untimed + {args.steps} timed steps each, "
              f"{ms_step:.1f} ms per step per strip")
    # the config object of the headline (the node set is generated, not solved)
    wl = configs.bubble(h=args.bubble_h, seed=1, t_end=1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(wl, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_nodes": n_strip * cores, "wall_s": time.perf_counter() - t_start}
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
    from paper_1509_02615_gb300 import inputs as inp
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    pk, pk_kind = peaks()
    p64 = fp64_peak_tflops(torch)

    wl = bubble_workload(args.bubble_h)
    pb64, head = headline_case(torch, args, wl, world, local, p64)
    legs = {}
    if "bubble_fp32" in args.legs:
        legs["bubble_fp32"] = bubble_fp32_case(torch, args, wl, pb64, pk, pk_kind)
    pb64.close()
    if "weights" in args.legs:
        legs["weights"] = weights_case(torch, wl.nodes, 56, 9, 5, 3, p64, "the headline bubble")
        legs["weights"]["density_current_100m"] = weights_case(
            torch, inp.density_current_nodes(100.0), 37, 7, 4, 3, p64, "the density current at 100 m")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if "density_current" in args.legs:
        legs["density_current"] = density_current_case(torch, args, pk, pk_kind, p64, flush)
    if "advection" in args.legs:
        legs["advection"] = advection_case(torch)
    if "large" in args.legs and args.large_h > 0:
        legs["roofline_large"] = large_case(torch, args, flush)
    del flush
    if "batched" in args.legs and args.ens_runs > 0:
        legs["batched"] = ensemble_case(torch, args)
    if "learned" in args.legs:
        legs["learned"] = learned_case(torch, args)

    base = None
    if rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(args.bubble_h)

    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": headline_config(wl, world),
                "roofline": head["roofline"], "clocks": head["clocks"], "e2e": head["e2e"],
                "gpu_launches": head["gpu_launches"], "launch": head["launch"], "setup": head["setup"],
                "state_minmax": head["state_minmax"], "fp64_dgemm_tflops": p64,
                "cpu_baseline": base}
        line.update(legs)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
