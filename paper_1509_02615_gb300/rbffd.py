"""Python binding of librbffd (ctypes): argument marshalling only.

Every step of the method runs in the CUDA library; this module turns torch
tensors into device pointers and the library's status codes into exceptions.
There is no CPU fallback: if librbffd.so is missing or no GPU is present,
every call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import inputs as inp

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librbffd.so")

RBF_OK, RBF_E_ARG, RBF_E_SINGULAR, RBF_E_NONFINITE, RBF_E_TIMEOUT, RBF_E_CUDA, RBF_E_OOM = range(7)
OP = {"dx": 0, "dz": 1, "lap": 2, "hv": 3, "dxx": 4, "dzz": 5}


class RBFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"librbffd error {code}: {msg}")
        self.code = code


class NSParams(C.Structure):
    _fields_ = [("n_sten", C.c_int32), ("phs_p", C.c_int32), ("poly_l", C.c_int32), ("hv_k", C.c_int32),
                ("hv_p", C.c_int32), ("precision", C.c_int32), ("threads_per_node", C.c_int32),
                ("storage", C.c_int32), ("period_x", C.c_double), ("mu", C.c_double), ("gamma", C.c_double),
                ("theta_bar", C.c_double), ("g", C.c_double), ("cp", C.c_double), ("cv", C.c_double),
                ("rd", C.c_double), ("gamma_c", C.c_double), ("spacing", C.c_double)]


class AdvParams(C.Structure):
    _fields_ = [("n_sten", C.c_int32), ("phs_p", C.c_int32), ("poly_l", C.c_int32), ("hv_k", C.c_int32),
                ("hv_p", C.c_int32), ("precision", C.c_int32), ("gamma", C.c_double), ("period_T", C.c_double),
                ("gamma_c", C.c_double), ("spacing", C.c_double)]


class EnsMember(C.Structure):
    _fields_ = [("n_prog", C.c_int64), ("n_all", C.c_int64), ("n_sten", C.c_int32), ("poly_l", C.c_int32),
                ("period_x", C.c_double), ("gamma", C.c_double), ("dt", C.c_double), ("n_steps", C.c_int64),
                ("spacing", C.c_double), ("gamma_c", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n_prog", C.c_int64), ("n_all", C.c_int64), ("n_ghost", C.c_int64), ("n_fields", C.c_int32),
                ("precision", C.c_int32), ("n_sten", C.c_int32), ("threads_per_node", C.c_int32),
                ("slots", C.c_int32), ("launches_per_step", C.c_int32), ("n_components", C.c_int32),
                ("n_ghost_classes", C.c_int32), ("prefetch", C.c_int32), ("run_mode", C.c_int32),
                ("weight_build_ms", C.c_double), ("ghost_setup_ms", C.c_double),
                ("rhs_bytes_per_node", C.c_double), ("rhs_flops_per_node", C.c_double),
                ("persist_lanes", C.c_int32), ("persist_regs", C.c_int32), ("persist_chunk", C.c_int32),
                ("persist_halo_max", C.c_int32), ("persist_ctas", C.c_int32), ("stage_split", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) of every entry point declared in include/rbffd.h
_P, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
SIGNATURES = [
    ("rbf_last_error", C.c_char_p, []),
    ("rbf_hyperviscosity_gamma", C.c_int, [_D, _D, _I32, C.POINTER(C.c_double)]),
    ("rbf_build_stencils", C.c_int, [_P, _P, _I64, _I64, _I32, _D, _P, _P]),
    ("rbf_build_stencils_static", C.c_int, [_P, _P, _I64, _I64, _I32, _D, _P, _P]),
    ("rbf_build_weights", C.c_int, [_P, _P, _I64, _P, _I64, _I32, _D, _I32, _I32, _I32, _P, _I32, _P, _P]),
    ("rbf_ns_create", C.c_int, [C.POINTER(_P), C.POINTER(NSParams), _P, _P, _I64, _I64, _P, _P, _P]),
    ("rbf_adv_create", C.c_int, [C.POINTER(_P), C.POINTER(AdvParams), _P, _P, _I64, _I64, _P, _P, _P, _P]),
    ("rbf_adv_create_flow", C.c_int, [C.POINTER(_P), C.POINTER(AdvParams), _P, _P, _I64, _I64, _P, _I32, _P, _P,
                                      _P, _P]),
    ("rbf_ens_create", C.c_int, [C.POINTER(_P), C.POINTER(NSParams), _I32, C.POINTER(EnsMember), _P, _P, _P, _P,
                                 _P]),
    ("rbf_ens_run", C.c_int, [_P, _I64, _P]),
    ("rbf_ens_node_updates", C.c_int, [_P, _I64, C.POINTER(C.c_double)]),
    ("rbf_mlp_create", C.c_int, [C.POINTER(_P), _P, _P]),
    ("rbf_mlp_n_params", C.c_int, [_P, C.POINTER(C.c_int64)]),
    ("rbf_mlp_set_params", C.c_int, [_P, _P]),
    ("rbf_mlp_get_params", C.c_int, [_P, _P]),
    ("rbf_mlp_set_scales", C.c_int, [_P, _P]),
    ("rbf_mlp_get_scales", C.c_int, [_P, _P]),
    ("rbf_mlp_fit_scales", C.c_int, [_P, _P, _P, _I64, _I64]),
    ("rbf_mlp_grad", C.c_int, [_P, _P, _P, _I64, _I64, _P, _I32, _P, _P]),
    ("rbf_mlp_train", C.c_int, [_P, _P, _P, _I64, _I64, _I64, _I32, C.c_float, C.c_uint64, _P]),
    ("rbf_mlp_forward", C.c_int, [_P, _P, _P]),
    ("rbf_learned_run", C.c_int, [_P, _D, _D, _I64, _P, _P, C.POINTER(C.c_int64)]),
    ("rbf_mlp_tune_run", C.c_int, [_P]),
    ("rbf_mlp_destroy", C.c_int, [_P]),
    ("rbf_restrict", C.c_int, [_P, _I32, _P, _I64, _P, _I32, _I64, _I64, _P]),
    ("rbf_restrict_weighted", C.c_int, [_P, _I32, _P, _P, _I32, _I64, _P, _I64, _I64, _P]),
    ("rbf_fill_ghosts", C.c_int, [_P, _P]),
    ("rbf_mlp_targets", C.c_int, [_P, _P, _I64, _I64, _D, _P]),
    ("rbf_rhs", C.c_int, [_P, _D, _P, _P]),
    ("rbf_rk4_step", C.c_int, [_P, _D, _D, _P]),
    ("rbf_run", C.c_int, [_P, _D, _D, _I64, _P]),
    ("rbf_run_host", C.c_int, [_P, _D, _D, _I64, _P]),
    ("rbf_set_run_mode", C.c_int, [_P, _I32, _I32, _I32]),
    ("rbf_set_stage_split", C.c_int, [_P, _I32]),
    ("rbf_set_spin_limit", C.c_int, [_P, _I64]),
    ("rbf_set_operator_storage", C.c_int, [_P, _I32, _I32, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    ("rbf_lattice_classes", C.c_int, [_P, _P, _P, _I64, _I64, _I32, _D, _D, _I32, _P, C.POINTER(C.c_int32)]),
    ("rbf_partition_blocks", C.c_int, [_P, _P, _I64, _I32, _P]),
    ("rbf_sync", C.c_int, [_P]),
    ("rbf_minmax", C.c_int, [_P, _P, _P]),
    ("rbf_get_info", C.c_int, [_P, C.POINTER(Info)]),
    ("rbf_get_weights", C.c_int, [_P, _I32, _P, _P]),
    ("rbf_set_stage_timing", C.c_int, [_P, _I32]),
    ("rbf_stage_kernel_ms", C.c_int, [_P, C.POINTER(C.c_double)]),
    ("rbf_destroy", C.c_int, [_P]),
]


def lib():
    """The loaded librbffd (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1509_02615_gb300._build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != RBF_OK:
        raise RBFError(code, lib().rbf_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("librbffd needs a CUDA GPU; none is available")
    return torch


def _stream():
    return C.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _host_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ---- a1, a2: stateless builders ---------------------------------------------------

def build_stencils(x, z, n_centers, n, period_x=0.0):
    """n nearest nodes of nodes 0..n_centers-1 among all nodes (device tensors)."""
    torch = _torch()
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    z = z.to(device="cuda", dtype=torch.float64).contiguous()
    idx = torch.empty((n_centers, n), dtype=torch.int32, device="cuda")
    _check(lib().rbf_build_stencils(_ptr(x), _ptr(z), x.numel(), n_centers, n, float(period_x), _ptr(idx), _stream()))
    return idx


def build_weights(x, z, idx, p, l, ops, hv_k=0, period_x=0.0):
    """Weights [len(ops), N, n] (float64, device) of the stencils idx [N, n]."""
    torch = _torch()
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    z = z.to(device="cuda", dtype=torch.float64).contiguous()
    idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
    N, n = idx.shape
    codes = np.array([OP[o] if isinstance(o, str) else int(o) for o in ops], np.int32)
    w = torch.empty((len(codes), N, n), dtype=torch.float64, device="cuda")
    _check(lib().rbf_build_weights(_ptr(x), _ptr(z), x.numel(), _ptr(idx), N, n, float(period_x), p, l, hv_k,
                                   _host_ptr(codes), len(codes), _ptr(w), _stream()))
    return w


# ---- problems ---------------------------------------------------------------------

class Problem:
    """A stepping context owned by librbffd (Navier-Stokes or advection)."""

    def __init__(self, handle, n_fields, n_prog, n_all, precision, kind):
        self._h = handle
        self.n_fields = n_fields
        self.n_prog = n_prog
        self.n_all = n_all
        self.precision = precision
        self.kind = kind

    @property
    def dtype(self):
        torch = _torch()
        return torch.float64 if self.precision == 64 else torch.float32

    @property
    def state_shape(self):
        """Node-major records: row i holds the fields of node i."""
        return (self.n_all if self.kind == "ns" else self.n_prog, self.n_fields)

    def _state(self, U):
        torch = _torch()
        if not (U.is_cuda and U.dtype == self.dtype and U.is_contiguous() and tuple(U.shape) == self.state_shape):
            raise ValueError(f"state must be a contiguous CUDA {self.dtype} tensor of shape {self.state_shape}")
        return U

    def rhs(self, t, U, dUdt=None):
        U = self._state(U)
        if dUdt is None:
            dUdt = _torch().empty((self.n_prog, self.n_fields), dtype=self.dtype, device="cuda")
        _check(lib().rbf_rhs(self._h, float(t), _ptr(U), _ptr(dUdt)))
        return dUdt

    def rk4_step(self, t, dt, U):
        _check(lib().rbf_rk4_step(self._h, float(t), float(dt), _ptr(self._state(U))))
        return U

    def run(self, t0, dt, n_steps, U):
        _check(lib().rbf_run(self._h, float(t0), float(dt), int(n_steps), _ptr(self._state(U))))
        return U

    def run_host(self, t0, dt, n_steps, U_host):
        """End-to-end run on a host (ideally pinned) tensor, copies included."""
        if U_host.is_cuda or U_host.dtype != self.dtype or tuple(U_host.shape) != self.state_shape:
            raise ValueError("run_host takes a CPU tensor of the state's dtype and shape")
        _check(lib().rbf_run_host(self._h, float(t0), float(dt), int(n_steps), C.c_void_p(U_host.data_ptr())))
        return U_host

    def sync(self):
        _check(lib().rbf_sync(self._h))

    RUN_MODES = {"auto": 0, "graph": 1, "persistent": 2}

    def set_run_mode(self, mode, lanes=0, ctas=0):
        """'graph', 'persistent' or 'auto' (see rbf_set_run_mode)."""
        _check(lib().rbf_set_run_mode(self._h, self.RUN_MODES[mode], int(lanes), int(ctas)))

    def set_stage_split(self, enable):
        """Split each stage into a wall-set launch and the rest, so that the
        next stage's ghost fill overlaps the rest (see rbf_set_stage_split)."""
        _check(lib().rbf_set_stage_split(self._h, int(bool(enable))))

    def set_operator_storage(self, mode, threads_per_node=0):
        """'per-node' (Sec. 3's rows) or 'lattice' (one row per class of
        translated stencils); returns (nodes in classes, classes)."""
        cn, nc = C.c_int64(0), C.c_int32(0)
        code = STORAGE[mode]
        _check(lib().rbf_set_operator_storage(self._h, code, threads_per_node, C.byref(cn), C.byref(nc)))
        return cn.value, nc.value

    def set_spin_limit(self, polls):
        _check(lib().rbf_set_spin_limit(self._h, int(polls)))

    def minmax(self, U):
        out = np.zeros((self.n_fields, 2))
        _check(lib().rbf_minmax(self._h, _ptr(self._state(U)), _host_ptr(out)))
        return out

    def info(self):
        i = Info()
        _check(lib().rbf_get_info(self._h, C.byref(i)))
        return i.as_dict()

    def weights(self, op):
        n = self.info()["n_sten"]
        w = np.zeros((self.n_prog, n))
        idx = np.zeros((self.n_prog, n), np.int32)
        _check(lib().rbf_get_weights(self._h, OP[op] if isinstance(op, str) else int(op), _host_ptr(w), _host_ptr(idx)))
        return w, idx

    def set_stage_timing(self, enable):
        _check(lib().rbf_set_stage_timing(self._h, 1 if enable else 0))

    def stage_kernel_ms(self):
        v = C.c_double()
        _check(lib().rbf_stage_kernel_ms(self._h, C.byref(v)))
        return v.value

    def close(self):
        if self._h:
            _check(lib().rbf_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def partition_blocks(x, z, parts):
    """Block of every point under the persistent mode's recursive coordinate
    bisection (host-only; see rbf_partition_blocks)."""
    x = np.ascontiguousarray(x, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    out = np.zeros(x.shape[0], np.int32)
    _check(lib().rbf_partition_blocks(_host_ptr(x), _host_ptr(z), x.shape[0], int(parts), _host_ptr(out)))
    return out


def lattice_classes(idx, x, z, n_prog, period_x, h, min_members=32):
    """Host-only lattice classes of given stencils (rbf_lattice_classes):
    per node its class id (-1: irregular) and the class count."""
    idx = np.ascontiguousarray(idx, np.int32)
    x = np.ascontiguousarray(x, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    cls = np.zeros(n_prog, np.int32)
    nc = C.c_int32(0)
    _check(lib().rbf_lattice_classes(_host_ptr(idx), _host_ptr(x), _host_ptr(z), n_prog, x.shape[0], idx.shape[1],
                                     period_x, h, min_members, _host_ptr(cls), C.byref(nc)))
    return cls, nc.value


def hyperviscosity_gamma(c, h, k):
    """The library's gamma of Sec. 5.3 for constant c, spacing h and power k
    (rbf_hyperviscosity_gamma; host only)."""
    v = C.c_double()
    _check(lib().rbf_hyperviscosity_gamma(float(c), float(h), int(k), C.byref(v)))
    return v.value


STORAGE = {"per-node": 0, "lattice": 1}


def ns_problem(nodes: inp.NodeSet, precision=64, n=37, p=7, l=4, hv_k=3, hv_p=None, mu=75.0, gamma=None,
               gamma_c=2.0 ** -6, threads_per_node=0, theta_bar=inp.THETA_BAR, storage="per-node"):
    """Navier-Stokes problem on a node set (Sec. 6.2-6.3 defaults)."""
    prm = NSParams(n_sten=n, phs_p=p, poly_l=l, hv_k=hv_k, hv_p=hv_p if hv_p else p, precision=precision,
                   threads_per_node=threads_per_node, storage=STORAGE[storage], period_x=nodes.period_x, mu=mu,
                   gamma=0.0 if gamma is None else gamma, gamma_c=gamma_c if gamma is None else 0.0,
                   spacing=nodes.h, theta_bar=theta_bar, g=inp.G, cp=inp.CP, cv=inp.CV, rd=inp.RD)
    _torch()
    h = C.c_void_p()
    x = np.ascontiguousarray(nodes.x, np.float64)
    z = np.ascontiguousarray(nodes.z, np.float64)
    kind = np.ascontiguousarray(nodes.kind, np.int32)
    owner = np.ascontiguousarray(nodes.ghost_owner, np.int32)
    _check(lib().rbf_ns_create(C.byref(h), C.byref(prm), _host_ptr(x), _host_ptr(z), nodes.n_prog, nodes.n_all,
                               _host_ptr(kind), _host_ptr(owner) if owner.size else None, _stream()))
    pb = Problem(h, 4, nodes.n_prog, nodes.n_all, precision, "ns")
    pb.params = prm
    return pb


def advection_problem(nodes: inp.NodeSet, precision=64, n=37, p=7, l=4, hv_k=4, hv_p=9, gamma=None,
                      gamma_c=2.0 ** -14, T=5.0, flow="deformational"):
    """Scalar advection on reflected nodes (Sec. 6.1) in the deformational
    flow (one separable part, rbf_adv_create) or the paper's vortex flow (two
    parts, rbf_adv_create_flow)."""
    prm = AdvParams(n_sten=n, phs_p=p, poly_l=l, hv_k=hv_k, hv_p=hv_p, precision=precision,
                    gamma=0.0 if gamma is None else gamma, gamma_c=gamma_c if gamma is None else 0.0,
                    spacing=nodes.h, period_T=T)
    _torch()
    x = np.ascontiguousarray(nodes.x, np.float64)
    z = np.ascontiguousarray(nodes.z, np.float64)
    src = np.ascontiguousarray(nodes.src, np.int32)
    h = C.c_void_p()
    if flow == "deformational":
        Uv, Vv = inp.deformational_velocity(nodes.x, nodes.z)
        Uv = np.ascontiguousarray(Uv, np.float64)
        Vv = np.ascontiguousarray(Vv, np.float64)
        _check(lib().rbf_adv_create(C.byref(h), C.byref(prm), _host_ptr(x), _host_ptr(z), nodes.n_prog, nodes.n_all,
                                    _host_ptr(src), _host_ptr(Uv), _host_ptr(Vv), _stream()))
    elif flow == "vortex":
        parts, coef = inp.vortex_flow_parts(nodes.x, nodes.z, T)
        Uv = np.ascontiguousarray(np.stack([pu for pu, _ in parts]), np.float64)
        Vv = np.ascontiguousarray(np.stack([pv for _, pv in parts]), np.float64)
        cf = np.ascontiguousarray(np.asarray(coef, np.float64).reshape(-1))
        _check(lib().rbf_adv_create_flow(C.byref(h), C.byref(prm), _host_ptr(x), _host_ptr(z), nodes.n_prog,
                                         nodes.n_all, _host_ptr(src), len(parts), _host_ptr(Uv), _host_ptr(Vv),
                                         _host_ptr(cf), _stream()))
    else:
        raise ValueError(f"unknown flow {flow!r}")
    pb = Problem(h, 1, nodes.n_prog, nodes.n_all, precision, "advection")
    pb.params = prm
    return pb


def state_tensor(U, precision, device="cuda"):
    """Field-major float64 numpy state [F, n] -> node-major tensor [n, F] of the
    problem's precision (the layout the library steps)."""
    import torch
    U = np.asarray(U, dtype=np.float64)
    if U.ndim == 1:
        U = U[None, :]
    return torch.as_tensor(np.ascontiguousarray(U.T), dtype=torch.float64 if precision == 64 else torch.float32,
                           device=device).contiguous()


def fields(t):
    """Node-major tensor [n, F] -> field-major float64 numpy array [F, n]."""
    return t.detach().cpu().double().numpy().T.copy()


class Ensemble(Problem):
    """A batched ensemble (a8): members' node-major records concatenated."""

    def __init__(self, handle, members, precision):
        n_all = sum(m.nodes.n_all for m in members)
        n_prog = sum(m.nodes.n_prog for m in members)
        super().__init__(handle, 4, n_prog, n_all, precision, "ensemble")
        self.members = members
        self.rec0 = np.cumsum([0] + [m.nodes.n_all for m in members])[:-1]

    @property
    def state_shape(self):
        return (self.n_all, 4)

    def state(self, device="cuda"):
        """Initial state of every member, node-major, concatenated."""
        return state_tensor(np.concatenate([m.U0 for m in self.members], axis=1), self.precision, device)

    def member_fields(self, U, r):
        """Field-major float64 [4, n_all] of member r."""
        m = self.members[r]
        return fields(U[self.rec0[r]:self.rec0[r] + m.nodes.n_all])

    def run(self, max_steps, U):
        _check(lib().rbf_ens_run(self._h, int(max_steps), _ptr(self._state(U))))
        return U

    def node_updates(self, max_steps=-1):
        v = C.c_double()
        _check(lib().rbf_ens_node_updates(self._h, int(max_steps), C.byref(v)))
        return v.value


def ensemble_problem(members, precision=32, p=7, hv_k=3, mu=75.0, gamma_c=2.0 ** -6, theta_bar=inp.THETA_BAR,
                     storage="per-node", threads_per_node=0):
    """Batched ensemble of density-current members (inputs.EnsembleMember);
    threads_per_node 0 autotunes the lanes per node."""
    _torch()
    common = NSParams(n_sten=37, phs_p=p, poly_l=4, hv_k=hv_k, hv_p=p, precision=precision,
                      threads_per_node=threads_per_node,
                      storage=STORAGE[storage], period_x=0.0, mu=mu, gamma=0.0, theta_bar=theta_bar, g=inp.G, cp=inp.CP,
                      cv=inp.CV, rd=inp.RD, gamma_c=gamma_c)
    arr = (EnsMember * len(members))()
    for r, m in enumerate(members):
        arr[r] = EnsMember(n_prog=m.nodes.n_prog, n_all=m.nodes.n_all, n_sten=m.n, poly_l=m.l,
                           period_x=m.nodes.period_x, gamma=0.0, dt=m.dt, n_steps=m.n_steps,
                           spacing=m.nodes.h, gamma_c=getattr(m, "gamma_c", 0.0) or 0.0)
    x = np.ascontiguousarray(np.concatenate([m.nodes.x for m in members]), np.float64)
    z = np.ascontiguousarray(np.concatenate([m.nodes.z for m in members]), np.float64)
    kind = np.ascontiguousarray(np.concatenate([m.nodes.kind for m in members]), np.int32)
    owner = np.ascontiguousarray(np.concatenate([m.nodes.ghost_owner for m in members]), np.int32)
    h = C.c_void_p()
    _check(lib().rbf_ens_create(C.byref(h), C.byref(common), len(members), arr, _host_ptr(x), _host_ptr(z),
                                _host_ptr(kind), _host_ptr(owner), _stream()))
    return Ensemble(h, members, precision)


# ---- a9: learned tendency correction ----------------------------------------------

class Mlp:
    """The learned correction's network, bound to a coarse NS problem."""

    def __init__(self, coarse: Problem):
        _torch()
        self.coarse = coarse
        h = C.c_void_p()
        _check(lib().rbf_mlp_create(C.byref(h), coarse._h, _stream()))
        self._h = h
        n = C.c_int64()
        _check(lib().rbf_mlp_n_params(self._h, C.byref(n)))
        self.n_params = n.value

    def set_params(self, params):
        a = np.ascontiguousarray(params, np.float32)
        assert a.size == self.n_params
        _check(lib().rbf_mlp_set_params(self._h, _host_ptr(a)))

    def params(self):
        a = np.zeros(self.n_params, np.float32)
        _check(lib().rbf_mlp_get_params(self._h, _host_ptr(a)))
        return a

    def set_scales(self, scales):
        a = np.ascontiguousarray(scales, np.float32)
        _check(lib().rbf_mlp_set_scales(self._h, _host_ptr(a)))

    def scales(self):
        a = np.zeros(12, np.float32)
        _check(lib().rbf_mlp_get_scales(self._h, _host_ptr(a)))
        return a

    def fit_scales(self, states, targets, n_runs, n_snap):
        _check(lib().rbf_mlp_fit_scales(self._h, _ptr(states), _ptr(targets), n_runs, n_snap))

    def grad(self, states, targets, n_runs, n_snap, samples):
        g = np.zeros(self.n_params, np.float32)
        loss = np.zeros(1, np.float32)
        _check(lib().rbf_mlp_grad(self._h, _ptr(states), _ptr(targets), n_runs, n_snap, _ptr(samples),
                                  samples.shape[0], _host_ptr(g), _host_ptr(loss)))
        return float(loss[0]), g

    def train(self, states, targets, n_runs, n_snap, iters, batch=4096, lr=2e-3, seed=0):
        loss = np.zeros(max(iters, 1), np.float32)
        _check(lib().rbf_mlp_train(self._h, _ptr(states), _ptr(targets), n_runs, n_snap, iters, batch, float(lr),
                                   int(seed), _host_ptr(loss)))
        return loss[:iters]

    def forward(self, U, delta=None):
        if delta is None:
            delta = _torch().empty((self.coarse.n_prog, 4), dtype=U.dtype, device="cuda")
        _check(lib().rbf_mlp_forward(self._h, _ptr(U), _ptr(delta)))
        return delta

    def tune_run(self):
        """Persistent plan of the coarse problem chosen for corrected runs
        (rbf_mlp_tune_run); returns (lanes per node, CTAs)."""
        _check(lib().rbf_mlp_tune_run(self._h))
        i = self.coarse.info()
        return i["persist_lanes"], i["persist_ctas"]

    def run(self, t0, dt, n_steps, U, alpha=(1.0, 1.0, 1.0, 1.0)):
        """Corrected coarse run (U_f += alpha_f dt delta_f after each step);
        returns the number of skipped (non-finite) corrections."""
        nf = C.c_int64()
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float64), (4,)))
        _check(lib().rbf_learned_run(self._h, float(t0), float(dt), int(n_steps), _host_ptr(a), _ptr(U),
                                     C.byref(nf)))
        return nf.value

    def close(self):
        if self._h:
            _check(lib().rbf_mlp_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fill_ghosts(pb: Problem, U):
    _check(lib().rbf_fill_ghosts(pb._h, _ptr(U)))
    return U


def restrict(src, src_precision, index_map, dst, dst_precision, block_records, block_stride):
    _check(lib().rbf_restrict(_ptr(src), src_precision, _ptr(index_map), index_map.numel(), _ptr(dst),
                              dst_precision, int(block_records), int(block_stride), _stream()))


def restrict_weighted(src, src_precision, idx, w, dst, block_records, block_stride):
    _check(lib().rbf_restrict_weighted(_ptr(src), src_precision, _ptr(idx), _ptr(w), idx.shape[1], idx.shape[0],
                                       _ptr(dst), int(block_records), int(block_stride), _stream()))


def mlp_targets(pb: Problem, states, n_runs, n_snap, dt, targets):
    _check(lib().rbf_mlp_targets(pb._h, _ptr(states), int(n_runs), int(n_snap), float(dt), _ptr(targets)))
    return targets
