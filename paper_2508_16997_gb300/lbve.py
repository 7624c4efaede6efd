"""Thin ctypes binding of ``liblbve.so`` (declared in ``include/lbve.h``).

The functions below carry the C names and only marshal arguments; every
step of the computation runs in the library's CUDA kernels.  Device memory
and the stream come from PyTorch.  There is no CPU fallback: if the library
is missing, the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbve.so")

LBVE_OK = 0
LBVE_ERR_ARG = -1
LBVE_ERR_CUDA = -2
LBVE_ERR_NONFINITE = -3
LBVE_ERR_TIMEOUT = -4
LBVE_ERR_GEOMETRY = -5
LBVE_ERR_WORKSPACE = -6
LBVE_ERR_STATE = -7
LBVE_FP64 = 0
LBVE_FP32_DEV = 1
LBVE_DF32 = 2
LBVE_NTOTALS = 14

EXPORTED = ["lbve_workspace_bytes", "lbve_create", "lbve_set_geometry", "lbve_step",
            "lbve_status", "lbve_fields", "lbve_totals", "lbve_residual", "lbve_time",
            "lbve_destroy", "lbve_error_string", "lbve_last_error", "lbve_field_totals_noalloc",
            "lbve_adjoint_workspace_bytes", "lbve_adjoint_step", "lbve_state_bytes", "lbve_save",
            "lbve_load", "lbve_autotune", "lbve_set_wall_distances", "lbve_set_inlet",
            "lbve_adjoint_step_ex", "lbve_adjoint_workspace_bytes_interval", "lbve_profile",
            "lbve_profile_read", "lbve_set_geometry_many", "lbve_fields_many"]


class lbve_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("beta", ctypes.c_double), ("Wi", ctypes.c_double),
                ("Re", ctypes.c_double), ("Sc", ctypes.c_double), ("Ma", ctypes.c_double),
                ("Lc", ctypes.c_double), ("Lambda_s", ctypes.c_double),
                ("Lambda_p", ctypes.c_double), ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
                ("tile_tx", ctypes.c_int32), ("max_wall_nodes", ctypes.c_int32),
                ("open_x", ctypes.c_int32), ("model", ctypes.c_int32), ("gtilde", ctypes.c_int32),
                ("L2", ctypes.c_double)]


class LbveError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        L = _lib
        name = L.lbve_error_string(code).decode() if L else str(code)
        detail = L.lbve_last_error().decode() if L else ""
        super().__init__(f"{where}: {name} ({code}): {detail}")


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2508_16997_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(lbve_params)
        L.lbve_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        L.lbve_create.argtypes = [P, ctypes.c_int32, _vp, ctypes.c_size_t, _vp,
                                  ctypes.POINTER(_vp)]
        L.lbve_set_geometry.argtypes = [_vp, ctypes.c_int32, _vp, _dp, _dp]
        L.lbve_set_geometry_many.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                             _vp, _vp, _vp]
        L.lbve_fields_many.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _vp,
                                       ctypes.c_int32]
        L.lbve_step.argtypes = [_vp, ctypes.c_int64]
        L.lbve_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
        L.lbve_fields.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int32]
        L.lbve_totals.argtypes = [_vp, ctypes.c_int32, _dp]
        L.lbve_residual.argtypes = [_vp, ctypes.c_int32, _dp]
        L.lbve_time.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
        L.lbve_field_totals_noalloc.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
        L.lbve_adjoint_workspace_bytes.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64,
                                                    ctypes.POINTER(ctypes.c_size_t)]
        L.lbve_adjoint_workspace_bytes_interval.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64,
                                                            ctypes.c_int64,
                                                            ctypes.POINTER(ctypes.c_size_t)]
        L.lbve_adjoint_step.argtypes = [_vp, ctypes.c_int32, _dp, _vp, ctypes.c_int64, _vp,
                                        ctypes.c_size_t, _vp]
        L.lbve_adjoint_step_ex.argtypes = [_vp, ctypes.c_int32, _dp, _vp, _dp, ctypes.c_int64,
                                           _vp, ctypes.c_size_t, _vp, _vp]
        L.lbve_state_bytes.argtypes = [_vp, ctypes.POINTER(ctypes.c_size_t)]
        L.lbve_save.argtypes = [_vp, _vp, ctypes.c_size_t]
        L.lbve_load.argtypes = [_vp, _vp, ctypes.c_size_t]
        L.lbve_autotune.argtypes = [P, ctypes.c_int32, _vp, ctypes.c_size_t, _vp, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]
        L.lbve_set_inlet.argtypes = [_vp, ctypes.c_int32, _dp]
        L.lbve_set_wall_distances.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32), _dp]
        L.lbve_profile.argtypes = [_vp, ctypes.c_int32]
        L.lbve_profile_read.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32), _dp, _dp, _dp]
        L.lbve_destroy.argtypes = [_vp]
        L.lbve_destroy.restype = None
        L.lbve_error_string.argtypes = [ctypes.c_int]
        L.lbve_error_string.restype = ctypes.c_char_p
        L.lbve_last_error.argtypes = []
        L.lbve_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("lbve_destroy", "lbve_error_string", "lbve_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != LBVE_OK:
        raise LbveError(rc, where)


def _params_array(params) -> ctypes.Array:
    arr = (lbve_params * len(params))()
    for i, p in enumerate(params):
        arr[i] = p
    return arr


def _f64(a, n):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} float64 values, got {a.size}")
    return a, a.ctypes.data_as(_dp)


# ---- the C entry points, same names -----------------------------------------

def lbve_workspace_bytes(params) -> int:
    arr = _params_array(params)
    out = ctypes.c_size_t()
    _check(load().lbve_workspace_bytes(arr, len(params), ctypes.byref(out)),
           "lbve_workspace_bytes")
    return out.value


def lbve_create(params, d_workspace: int, nbytes: int, stream: int) -> ctypes.c_void_p:
    arr = _params_array(params)
    h = _vp()
    _check(load().lbve_create(arr, len(params), _vp(d_workspace), nbytes, _vp(stream),
                              ctypes.byref(h)), "lbve_create")
    return h


def lbve_set_geometry(h, inst: int, solid_mask=None, body_force=None, init_fields=None,
                      n_nodes: int | None = None) -> None:
    mask_ptr = None
    if solid_mask is not None:
        m = np.ascontiguousarray(solid_mask, dtype=np.uint8)
        mask_ptr = m.ctypes.data
    bf, bf_ptr = _f64(body_force, 2 * n_nodes) if body_force is not None else (None, None)
    ini, ini_ptr = _f64(init_fields, 6 * n_nodes) if init_fields is not None else (None, None)
    _check(load().lbve_set_geometry(h, inst, mask_ptr, bf_ptr, ini_ptr), "lbve_set_geometry")


def _ptr_list(arrays):
    """A C array of pointers (NULL for None) to the arrays' data, or None if
    every entry is None."""
    if all(a is None for a in arrays):
        return None
    return (_vp * len(arrays))(*[None if a is None else a.ctypes.data for a in arrays])


def lbve_set_geometry_many(h, insts, solid_masks=None, body_forces=None, init_fields=None,
                           n_nodes=None) -> None:
    """lbve_set_geometry for several instances with one synchronisation.
    The lists (None = all None) are indexed like ``insts``; ``n_nodes[j]``
    (nx * ny of insts[j]) sizes the checks of the float64 arrays."""
    n = len(insts)
    ids = np.ascontiguousarray(insts, dtype=np.int32)
    masks = [None] * n if solid_masks is None else list(solid_masks)
    forces = [None] * n if body_forces is None else list(body_forces)
    inits = [None] * n if init_fields is None else list(init_fields)
    if not (len(masks) == len(forces) == len(inits) == n):
        raise ValueError("the lists must have one entry per instance")
    masks = [None if m is None else np.ascontiguousarray(m, dtype=np.uint8) for m in masks]

    def planes(a, j, k):  # float64, contiguous, k planes of n_nodes[j] values (if given)
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a if n_nodes is None else _f64(a, k * n_nodes[j])[0]
    forces = [None if f is None else planes(f, j, 2) for j, f in enumerate(forces)]
    inits = [None if a is None else planes(a, j, 6) for j, a in enumerate(inits)]
    pm, pf, pi = _ptr_list(masks), _ptr_list(forces), _ptr_list(inits)
    _check(load().lbve_set_geometry_many(h, n, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         pm, pf, pi), "lbve_set_geometry_many")


def lbve_set_inlet(h, inst: int, inlet) -> None:
    """Inlet profile [5][ny] = u_x, u_y, A_xx, A_xy, A_yy of an open channel."""
    a = np.ascontiguousarray(inlet, dtype=np.float64)
    _check(load().lbve_set_inlet(h, inst, a.ctypes.data_as(_dp)), "lbve_set_inlet")


def lbve_set_wall_distances(h, inst: int, node, direction, q) -> None:
    """Wall fractions q of wall links (node = y nx + x, direction 1..8)."""
    node = np.ascontiguousarray(node, dtype=np.int32)
    direction = np.ascontiguousarray(direction, dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if not (node.size == direction.size == q.size):
        raise ValueError("node, direction and q must have the same length")
    ip = ctypes.POINTER(ctypes.c_int32)
    _check(load().lbve_set_wall_distances(h, inst, int(node.size), node.ctypes.data_as(ip),
                                          direction.ctypes.data_as(ip), q.ctypes.data_as(_dp)),
           "lbve_set_wall_distances")


def lbve_step(h, n_steps: int) -> None:
    _check(load().lbve_step(h, int(n_steps)), "lbve_step")


def lbve_profile(h, max_launches: int) -> None:
    _check(load().lbve_profile(h, int(max_launches)), "lbve_profile")


def lbve_profile_read(h, precision: int, final_step: bool = False):
    """(launches, total ms, shortest ms, longest ms) of the timed step-kernel
    launches of one precision: the ordinary steps, or the final step of
    each lbve_step call."""
    n = ctypes.c_int32()
    tot, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().lbve_profile_read(h, int(precision), 1 if final_step else 0, ctypes.byref(n),
                                    ctypes.byref(tot), ctypes.byref(lo), ctypes.byref(hi)),
           "lbve_profile_read")
    return n.value, tot.value, lo.value, hi.value


def lbve_status(h, n_instances: int) -> np.ndarray:
    flags = np.zeros(n_instances, dtype=np.int32)
    rc = load().lbve_status(h, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc not in (LBVE_OK, LBVE_ERR_NONFINITE):
        _check(rc, "lbve_status")
    return flags


def lbve_fields(h, inst: int, out_ptr: int, on_device: bool) -> None:
    _check(load().lbve_fields(h, inst, _vp(out_ptr), 1 if on_device else 0), "lbve_fields")


def lbve_fields_many(h, insts, out_ptrs, on_device: bool) -> None:
    """lbve_fields for several instances; out_ptrs[j] receives insts[j]."""
    n = len(insts)
    if len(out_ptrs) != n:
        raise ValueError("one output per instance")
    ids = np.ascontiguousarray(insts, dtype=np.int32)
    outs = (_vp * n)(*[int(p) for p in out_ptrs])
    _check(load().lbve_fields_many(h, n, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), outs,
                                   1 if on_device else 0), "lbve_fields_many")


def lbve_totals(h, inst: int) -> np.ndarray:
    out = np.empty(LBVE_NTOTALS)
    _check(load().lbve_totals(h, inst, out.ctypes.data_as(_dp)), "lbve_totals")
    return out


def lbve_residual(h, inst: int) -> float:
    out = ctypes.c_double()
    _check(load().lbve_residual(h, inst, ctypes.byref(out)), "lbve_residual")
    return out.value


def lbve_time(h, inst: int) -> int:
    out = ctypes.c_int64()
    _check(load().lbve_time(h, inst, ctypes.byref(out)), "lbve_time")
    return out.value


def lbve_field_totals_noalloc(d_fields: int, nx: int, ny: int, d_out: int, stream: int) -> None:
    """Sums of a device field array [6][ny][nx] into a device array of 6
    doubles, using only the library's static scratch (no allocation)."""
    _check(load().lbve_field_totals_noalloc(_vp(d_fields), nx, ny, _vp(d_out), _vp(stream)),
           "lbve_field_totals_noalloc")


def lbve_adjoint_workspace_bytes(h, inst: int, n_steps: int) -> int:
    out = ctypes.c_size_t()
    _check(load().lbve_adjoint_workspace_bytes(h, inst, int(n_steps), ctypes.byref(out)),
           "lbve_adjoint_workspace_bytes")
    return out.value


def lbve_adjoint_workspace_bytes_interval(h, inst: int, n_steps: int, interval: int) -> int:
    out = ctypes.c_size_t()
    _check(load().lbve_adjoint_workspace_bytes_interval(h, inst, int(n_steps), int(interval),
                                                        ctypes.byref(out)),
           "lbve_adjoint_workspace_bytes_interval")
    return out.value


def lbve_adjoint_step(h, inst: int, init_fields, d_dL_dfields: int, n_steps: int, d_ws: int,
                      nbytes: int, d_dL_dforce: int, n_nodes: int) -> None:
    ini, ini_ptr = _f64(init_fields, 6 * n_nodes) if init_fields is not None else (None, None)
    _check(load().lbve_adjoint_step(h, inst, ini_ptr, _vp(d_dL_dfields), int(n_steps), _vp(d_ws),
                                    nbytes, _vp(d_dL_dforce)), "lbve_adjoint_step")


def lbve_adjoint_step_ex(h, inst: int, init_fields, d_dL_dfields: int | None, dL_ddrag,
                         n_steps: int, d_ws: int, nbytes: int, d_dL_dforce: int,
                         d_dL_dq: int | None, n_nodes: int) -> None:
    """Adjoint with an optional field loss (device pointer or None), drag loss
    weights (2 floats or None) and an optional dL/dq output [8][ny][nx]."""
    ini, ini_ptr = _f64(init_fields, 6 * n_nodes) if init_fields is not None else (None, None)
    dr, dr_ptr = _f64(dL_ddrag, 2) if dL_ddrag is not None else (None, None)
    _check(load().lbve_adjoint_step_ex(h, inst, ini_ptr, _vp(d_dL_dfields or 0), dr_ptr,
                                       int(n_steps), _vp(d_ws), nbytes, _vp(d_dL_dforce),
                                       _vp(d_dL_dq or 0)), "lbve_adjoint_step_ex")


def lbve_state_bytes(h) -> int:
    out = ctypes.c_size_t()
    _check(load().lbve_state_bytes(h, ctypes.byref(out)), "lbve_state_bytes")
    return out.value


def lbve_save(h) -> bytes:
    n = lbve_state_bytes(h)
    buf = ctypes.create_string_buffer(n)
    _check(load().lbve_save(h, buf, n), "lbve_save")
    return buf.raw


def lbve_load(h, state: bytes) -> None:
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load().lbve_load(h, buf, len(state)), "lbve_load")


def lbve_autotune(params, d_workspace: int, nbytes: int, stream: int,
                  trial_steps: int = 64) -> list:
    """Fastest tile width per instance (list of ints); the workspace is scratch."""
    arr = _params_array(params)
    out = (ctypes.c_int32 * len(params))()
    _check(load().lbve_autotune(arr, len(params), _vp(d_workspace), nbytes, _vp(stream),
                                int(trial_steps), out), "lbve_autotune")
    return list(out)


def lbve_destroy(h) -> None:
    if h:
        load().lbve_destroy(h)


# ---- convenience wrapper ----------------------------------------------------

def params_from(inst, precision: int = LBVE_FP64, tile_tx: int = 0) -> lbve_params:
    """lbve_params of a :class:`workloads.Instance` (room for its mask's wall
    nodes when it has a solid mask)."""
    walls = 0
    if getattr(inst, "solid", None) is not None:
        walls = len({k for k, _, _ in inst.wall_links()})
    return lbve_params(inst.nx, inst.ny, 1 if inst.periodic_y else 0, precision, inst.beta,
                       inst.Wi, inst.Re, inst.Sc, inst.Ma, inst.Lc, inst.Lambda_s, inst.Lambda_p,
                       inst.Fx, inst.Fy, tile_tx, walls,
                       1 if getattr(inst, "open_x", False) else 0, getattr(inst, "model", 0),
                       getattr(inst, "gtilde", 0), getattr(inst, "L2", 0.0))


class Simulation:
    """A batch of instances advanced together on the current CUDA device.

    The workspace is one torch uint8 tensor; the library runs on torch's
    current stream.  ``tile_tx`` is an int or per-instance list of tile
    widths (0 = default); ``autotune`` (a trial step count, or True for 64)
    picks them with lbve_autotune on the workspace before the handle is made.
    """

    def __init__(self, instances, precision=LBVE_FP64, init_fields=None, device=None,
                 tile_tx=0, autotune=False):
        import torch
        self.torch = torch
        self.instances = list(instances)
        if isinstance(precision, int):
            precision = [precision] * len(self.instances)
        if isinstance(tile_tx, int):
            tile_tx = [tile_tx] * len(self.instances)
        self.params = [params_from(inst, pr, tx)
                       for inst, pr, tx in zip(self.instances, precision, tile_tx)]
        self.device = torch.device(device or "cuda")
        self.nbytes = lbve_workspace_bytes(self.params)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device)
        if autotune:
            steps = 64 if autotune is True else int(autotune)
            widths = lbve_autotune(self.params, self.workspace.data_ptr(), self.nbytes,
                                   self.stream.cuda_stream, steps)
            for p, tx in zip(self.params, widths):
                p.tile_tx = tx
        self.tile_tx = [p.tile_tx for p in self.params]
        self.h = lbve_create(self.params, self.workspace.data_ptr(), self.nbytes,
                             self.stream.cuda_stream)
        n = len(self.instances)
        lbve_set_geometry_many(self.h, list(range(n)),
                               [getattr(inst, "solid", None) for inst in self.instances],
                               [inst.force_field for inst in self.instances],
                               None if init_fields is None else list(init_fields),
                               n_nodes=[inst.n_nodes for inst in self.instances])
        for i, inst in enumerate(self.instances):
            solid = getattr(inst, "solid", None)
            if getattr(inst, "open_x", False) and getattr(inst, "inlet", None) is not None:
                lbve_set_inlet(self.h, i, inst.inlet)
            if solid is not None and getattr(inst, "wall_q", None) is not None:
                links = inst.wall_links()
                lbve_set_wall_distances(self.h, i, [k for k, _, _ in links],
                                        [d for _, d, _ in links], [q for _, _, q in links])

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lbve_destroy(h)
            self.h = None

    def step(self, n: int) -> None:
        lbve_step(self.h, n)

    def fields(self, i: int) -> np.ndarray:
        inst = self.instances[i]
        out = np.empty((6, inst.ny, inst.nx))
        lbve_fields(self.h, i, out.ctypes.data, False)
        return out

    def fields_device(self, i: int):
        inst = self.instances[i]
        out = self.torch.empty((6, inst.ny, inst.nx), dtype=self.torch.float64,
                               device=self.device)
        lbve_fields(self.h, i, out.data_ptr(), True)
        return out

    def totals(self, i: int) -> np.ndarray:
        return lbve_totals(self.h, i)

    def residual(self, i: int) -> float:
        return lbve_residual(self.h, i)

    def status(self) -> np.ndarray:
        return lbve_status(self.h, len(self.instances))

    def time(self, i: int = 0) -> int:
        return lbve_time(self.h, i)


def force_to_fields(sim: "Simulation", inst: int, force, n_steps: int, init_fields=None):
    """Differentiable map per-node body force -> fields after n_steps steps.

    ``force`` is a float64 torch tensor [2, ny, nx] (requires_grad allowed);
    the result is the float64 device tensor [6, ny, nx] of (rho, ux, uy, Axx,
    Axy, Ayy).  The backward pass calls lbve_adjoint_step (hand-written
    adjoint with sqrt(T) checkpointing)."""
    import torch

    class _ForceToFields(torch.autograd.Function):
        @staticmethod
        def forward(ctx, f):
            ctx.in_device = f.device
            inst_obj = sim.instances[inst]
            host = f.detach().to("cpu", torch.float64).contiguous().numpy()
            lbve_set_geometry(sim.h, inst, None, host, init_fields, n_nodes=inst_obj.n_nodes)
            sim.step(n_steps)
            return sim.fields_device(inst)

        @staticmethod
        def backward(ctx, grad_fields):
            inst_obj = sim.instances[inst]
            g = grad_fields.to(sim.device, torch.float64).contiguous()
            nbytes = lbve_adjoint_workspace_bytes(sim.h, inst, n_steps)
            ws = torch.empty(nbytes, dtype=torch.uint8, device=sim.device)
            out = torch.empty((2, inst_obj.ny, inst_obj.nx), dtype=torch.float64,
                              device=sim.device)
            lbve_adjoint_step(sim.h, inst, init_fields, g.data_ptr(), n_steps, ws.data_ptr(),
                              nbytes, out.data_ptr(), inst_obj.n_nodes)
            return out.to(ctx.in_device)

    return _ForceToFields.apply(force)
