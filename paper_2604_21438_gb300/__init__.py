"""Python binding of libsfchem (GB300 / sm_103a): the per-cell thermochemical
update of SFUMATO# (arXiv 2604.21438, Sec. 2.2.8 and Appendices A-C).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of ``libsfchem.so``.  PyTorch supplies device memory and streams.  There is no
CPU fallback: importing the binding on a machine without the library raises.

Low level: the ctypes structures and functions carry the C names of
``include/sfchem.h`` (``sfchem_init``, ``sfchem_step``, ...).  High level:
``Solver`` wraps a context and takes dicts of CUDA float64 tensors
(``Solver.step_host``: CPU tensors).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = [
    "lib", "sfchem_config_t", "sfchem_state_t", "sfchem_fields_t", "sfchem_stats_t", "sfchem_launch_t",
    "Solver", "SfchemError", "FP64", "MIXED", "STATE_FIELDS", "INPUT_FIELDS", "OUTPUT_FIELDS",
]

FP64, MIXED = 0, 1
OK, EINVAL, ENOTINIT, ECUDA, ETIMEOUT, ENOMEM = 0, 1, 2, 3, 4, 5
CELL_CAP, CELL_BADINPUT, CELL_NOCONV, CELL_TIGHT, CELL_BADSTEP = 1, 2, 4, 8, 16
P_ALL = (1 << 17) - 1
F_FREEZE_TG, F_FREEZE_TD, F_FREEZE_EIR, F_FREEZE_YH2, F_FREEZE_YE, F_SPLIT, F_REFINE_FF = 1, 2, 4, 8, 16, 32, 64
F_NO_REJECT = 128

STATE_FIELDS = ("T_g", "T_d", "E_IR", "y_H2", "y_e")            # evolved in place
INPUT_FIELDS = ("n_H", "G0", "n_EUV", "N_H2")                      # read only
OUTPUT_FIELDS = ("y_H", "y_Hp", "y_Hm", "status", "n_sub", "n_itr")  # written when present


class SfchemError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().sfchem_strerror(code).decode()
        if code == ECUDA:
            msg += ": " + lib().sfchem_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class sfchem_config_t(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("n_cyc", ctypes.c_int32), ("n_sub_max", ctypes.c_int32),
        ("nr_itr_limit", ctypes.c_int32), ("f_chem", ctypes.c_double), ("Z", ctypes.c_double),
        ("gamma_ad", ctypes.c_double), ("y_floor", ctypes.c_double), ("nr_tol", ctypes.c_double),
        ("reaction_mask", ctypes.c_uint32), ("process_mask", ctypes.c_uint32), ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class sfchem_state_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("n_H", "T_gas", "T_dust", "E_IR", "y_H2", "y_e", "y_H", "y_Hp", "y_Hm", "status", "n_sub",
                 "n_itr")]


class sfchem_fields_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("G0_fuv", "n_euv", "N_H2")]


class sfchem_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("calls", "cells", "substeps", "newton_iters", "tight_cells", "capped_cells",
                 "noconv_cells", "badinput_cells", "badstep_cells", "rejected_substeps", "step_halvings")] + [
        ("max_substeps", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("last_kernel_ms", ctypes.c_double)]


class sfchem_launch_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("threads_per_cta", "ctas_per_sm", "chunk", "reserved")]


_lib = None

# every entry point declared in include/sfchem.h
EXPORTS = ("sfchem_config_default", "sfchem_config_validate", "sfchem_init", "sfchem_set_config",
           "sfchem_step", "sfchem_step_nr", "sfchem_step_batched", "sfchem_set_launch", "sfchem_get_launch",
           "sfchem_autotune", "sfchem_stats", "sfchem_stats_reset", "sfchem_finalize",
           "sfchem_strerror", "sfchem_last_cuda_error", "sfchem_version", "sfchem_step_batched_noalloc",
           "sfchem_step_host", "sfchem_partition", "sfchem_block_costs", "sfchem_photon_update")
# scratch limits of sfchem_step_batched_noalloc (include/sfchem.h)
NOALLOC_MAX_BLOCKS, NOALLOC_MAX_CHUNKS = 4096, 65536


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libsfchem.so (building it in-tree when stale and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    try:
        _build.build()
    except RuntimeError:
        if not os.path.exists(_build.LIB):
            raise
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libsfchem is not built ({_build.LIB}); run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.sfchem_config_default.argtypes = [P(sfchem_config_t)]
    L.sfchem_config_default.restype = None
    L.sfchem_config_validate.argtypes = [P(sfchem_config_t)]
    L.sfchem_init.argtypes = [P(sfchem_config_t), P(vp)]
    L.sfchem_set_config.argtypes = [vp, P(sfchem_config_t)]
    L.sfchem_step.argtypes = [vp, P(sfchem_state_t), P(sfchem_fields_t), i64, dbl, dbl, vp]
    L.sfchem_step_nr.argtypes = [vp, P(sfchem_state_t), P(sfchem_fields_t), i64, dbl, dbl, vp]
    L.sfchem_step_batched.argtypes = [vp, P(sfchem_state_t), P(sfchem_fields_t), P(ctypes.c_int64),
                                      P(ctypes.c_double), i32, dbl, vp]
    L.sfchem_set_launch.argtypes = [vp, P(sfchem_launch_t)]
    L.sfchem_get_launch.argtypes = [vp, P(sfchem_launch_t)]
    L.sfchem_autotune.argtypes = [vp, P(sfchem_state_t), P(sfchem_fields_t), P(ctypes.c_int64),
                                  P(ctypes.c_double), i32, dbl, vp]
    L.sfchem_step_batched_noalloc.argtypes = [P(sfchem_config_t), P(sfchem_state_t), P(sfchem_fields_t),
                                              P(ctypes.c_int64), P(ctypes.c_double), i32, dbl, vp]
    L.sfchem_step_host.argtypes = [vp, P(sfchem_state_t), P(sfchem_fields_t), P(ctypes.c_int64),
                                   P(ctypes.c_double), i32, dbl, i64, vp]
    L.sfchem_partition.argtypes = [P(ctypes.c_int64), P(ctypes.c_double), i32, i32, P(ctypes.c_int32)]
    L.sfchem_photon_update.argtypes = [P(sfchem_state_t), P(sfchem_fields_t), i64, dbl, vp, vp, vp, vp]
    L.sfchem_block_costs.argtypes = [vp, P(ctypes.c_float), i32]
    L.sfchem_stats.argtypes = [vp, P(sfchem_stats_t)]
    L.sfchem_stats_reset.argtypes = [vp]
    L.sfchem_finalize.argtypes = [vp]
    L.sfchem_strerror.argtypes = [ctypes.c_int]
    L.sfchem_strerror.restype = ctypes.c_char_p
    L.sfchem_last_cuda_error.argtypes = []
    L.sfchem_last_cuda_error.restype = ctypes.c_char_p
    L.sfchem_version.argtypes = []
    L.sfchem_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("sfchem_config_default", "sfchem_strerror", "sfchem_last_cuda_error",
                        "sfchem_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != OK:
        raise SfchemError(rc, where)


def default_config(**kw) -> sfchem_config_t:
    c = sfchem_config_t()
    lib().sfchem_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED}[v]
        setattr(c, k, v)
    return c


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_tensor(name, t, n, dtype, cuda=True):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda != cuda:
        raise TypeError(f"{name} must be a {'CUDA' if cuda else 'CPU'} tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {n} elements")


def make_structs(cells: dict, n: int, cuda: bool = True):
    """Build (sfchem_state_t, sfchem_fields_t) from a dict of CUDA tensors
    (cuda=False: CPU tensors, for sfchem_step_host)."""
    import torch
    for k in STATE_FIELDS + INPUT_FIELDS:
        _check_tensor(k, cells[k], n, torch.float64, cuda)
    for k in ("y_H", "y_Hp", "y_Hm"):
        if cells.get(k) is not None:
            _check_tensor(k, cells[k], n, torch.float64, cuda)
    if cells.get("status") is not None:
        _check_tensor("status", cells["status"], n, torch.uint8, cuda)
    for k in ("n_sub", "n_itr"):
        if cells.get(k) is not None:
            _check_tensor(k, cells[k], n, torch.int32, cuda)
    st = sfchem_state_t(
        _ptr(cells["n_H"]), _ptr(cells["T_g"]), _ptr(cells["T_d"]), _ptr(cells["E_IR"]),
        _ptr(cells["y_H2"]), _ptr(cells["y_e"]), _ptr(cells.get("y_H")), _ptr(cells.get("y_Hp")),
        _ptr(cells.get("y_Hm")), _ptr(cells.get("status")), _ptr(cells.get("n_sub")), _ptr(cells.get("n_itr")))
    fl = sfchem_fields_t(_ptr(cells["G0"]), _ptr(cells["n_EUV"]), _ptr(cells["N_H2"]))
    return st, fl


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Solver:
    """One libsfchem context on the current CUDA device."""

    def __init__(self, precision="fp64", **cfg):
        self.cfg = default_config(precision=precision, **cfg)
        h = ctypes.c_void_p()
        _check(lib().sfchem_init(ctypes.byref(self.cfg), ctypes.byref(h)), "sfchem_init")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().sfchem_finalize(self.handle), "sfchem_finalize")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, **kw):
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = {"fp64": FP64, "mixed": MIXED}[v]
            setattr(self.cfg, k, v)
        _check(lib().sfchem_set_config(self.handle, ctypes.byref(self.cfg)), "sfchem_set_config")

    def step(self, cells: dict, dt: float, cd_factor: float = 1.0, stream=None):
        n = cells["n_H"].numel()
        st, fl = make_structs(cells, n)
        _check(lib().sfchem_step(self.handle, ctypes.byref(st), ctypes.byref(fl), n, float(dt),
                                 float(cd_factor), _stream_handle(stream)), "sfchem_step")

    def step_nr(self, cells: dict, dt: float, cd_factor: float = 1.0, stream=None):
        """The Newton-Raphson reference solver (FP64) on the same arrays."""
        n = cells["n_H"].numel()
        st, fl = make_structs(cells, n)
        _check(lib().sfchem_step_nr(self.handle, ctypes.byref(st), ctypes.byref(fl), n, float(dt),
                                    float(cd_factor), _stream_handle(stream)), "sfchem_step_nr")

    def step_batched(self, cells: dict, block_offset, block_dt, cd_factor: float = 1.0, stream=None):
        import numpy as np
        n = cells["n_H"].numel()
        st, fl = make_structs(cells, n)
        off = np.ascontiguousarray(block_offset, dtype=np.int64)
        bdt = np.ascontiguousarray(block_dt, dtype=np.float64)
        nb = len(bdt)
        if len(off) != nb + 1 or off[-1] != n:
            raise ValueError("block_offset must have n_blocks + 1 entries ending at n_cells")
        _check(lib().sfchem_step_batched(
            self.handle, ctypes.byref(st), ctypes.byref(fl),
            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            bdt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nb, float(cd_factor),
            _stream_handle(stream)), "sfchem_step_batched")

    def step_host(self, cells: dict, block_offset, block_dt, cd_factor: float = 1.0, slice_cells: int = 0,
                  stream=None):
        """sfchem_step_host: `cells` holds CPU tensors (pinned for overlapped
        copies); returns when the results are in them."""
        import numpy as np
        n = cells["n_H"].numel()
        st, fl = make_structs(cells, n, cuda=False)
        off = np.ascontiguousarray(block_offset, dtype=np.int64)
        bdt = np.ascontiguousarray(block_dt, dtype=np.float64)
        nb = len(bdt)
        if len(off) != nb + 1 or off[-1] != n:
            raise ValueError("block_offset must have n_blocks + 1 entries ending at n_cells")
        _check(lib().sfchem_step_host(
            self.handle, ctypes.byref(st), ctypes.byref(fl),
            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            bdt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nb, float(cd_factor), int(slice_cells),
            _stream_handle(stream)), "sfchem_step_host")

    def autotune(self, cells: dict, block_offset, block_dt, cd_factor: float = 1.0, stream=None):
        import numpy as np
        n = cells["n_H"].numel()
        st, fl = make_structs(cells, n)
        off = np.ascontiguousarray(block_offset, dtype=np.int64)
        bdt = np.ascontiguousarray(block_dt, dtype=np.float64)
        _check(lib().sfchem_autotune(
            self.handle, ctypes.byref(st), ctypes.byref(fl),
            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            bdt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(bdt), float(cd_factor),
            _stream_handle(stream)), "sfchem_autotune")
        return self.get_launch()

    def set_launch(self, threads_per_cta=0, ctas_per_sm=0, chunk=0):
        l = sfchem_launch_t(threads_per_cta, ctas_per_sm, chunk, 0)
        _check(lib().sfchem_set_launch(self.handle, ctypes.byref(l)), "sfchem_set_launch")

    def get_launch(self) -> dict:
        l = sfchem_launch_t()
        _check(lib().sfchem_get_launch(self.handle, ctypes.byref(l)), "sfchem_get_launch")
        return {"threads_per_cta": l.threads_per_cta, "ctas_per_sm": l.ctas_per_sm, "chunk": l.chunk}

    def block_costs(self, n_blocks: int):
        """Per-block substep sums of the last batched call (numpy float32)."""
        import numpy as np
        out = np.zeros(n_blocks, np.float32)
        _check(lib().sfchem_block_costs(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        int(n_blocks)), "sfchem_block_costs")
        return out

    def stats(self) -> dict:
        s = sfchem_stats_t()
        _check(lib().sfchem_stats(self.handle, ctypes.byref(s)), "sfchem_stats")
        return {k: getattr(s, k) for k, _ in sfchem_stats_t._fields_ if k != "reserved"}

    def stats_reset(self):
        _check(lib().sfchem_stats_reset(self.handle), "sfchem_stats_reset")


def photon_update(cells: dict, dt: float, G0_out=None, n_euv_out=None, absorbed=None, stream=None):
    """sfchem_photon_update on a dict of CUDA tensors (after a step on the same
    dict): writes the absorbed bands into G0_out / n_euv_out (new tensors when
    None; pass cells["G0"] / cells["n_EUV"] for an in-place update) and,
    when given, the (n, 4) absorbed photon counts; returns (G0_out, n_euv_out)."""
    import torch
    n = cells["n_H"].numel()
    st, fl = make_structs(cells, n)
    G0_out = torch.empty_like(cells["G0"]) if G0_out is None else G0_out
    n_euv_out = torch.empty_like(cells["n_EUV"]) if n_euv_out is None else n_euv_out
    for name, t, m in (("G0_out", G0_out, n), ("n_euv_out", n_euv_out, n)):
        _check_tensor(name, t, m, torch.float64)
    if absorbed is not None:
        _check_tensor("absorbed", absorbed, 4 * n, torch.float64)
    _check(lib().sfchem_photon_update(ctypes.byref(st), ctypes.byref(fl), n, float(dt), _ptr(G0_out),
                                      _ptr(n_euv_out), _ptr(absorbed), _stream_handle(stream)),
           "sfchem_photon_update")
    return G0_out, n_euv_out


def partition(block_offset, n_parts: int, block_cost=None):
    """sfchem_partition: cut the blocks into n_parts contiguous, cost-balanced
    ranges; returns the n_parts + 1 block indices of the cuts (host only)."""
    import numpy as np
    off = np.ascontiguousarray(block_offset, dtype=np.int64)
    nb = len(off) - 1
    cost = None if block_cost is None else np.ascontiguousarray(block_cost, dtype=np.float64)
    if cost is not None and len(cost) != nb:
        raise ValueError("block_cost must have one entry per block")
    cut = np.zeros(n_parts + 1, np.int32)
    _check(lib().sfchem_partition(
        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        None if cost is None else cost.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nb, int(n_parts),
        cut.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "sfchem_partition")
    return cut


def to_device(cells: dict, device="cuda", outputs: bool = True) -> dict:
    """Copy a dict of numpy float64 arrays to CUDA tensors (plus output buffers)."""
    import torch
    out = {k: torch.as_tensor(cells[k], dtype=torch.float64).to(device).contiguous()
           for k in STATE_FIELDS + INPUT_FIELDS}
    n = out["n_H"].numel()
    if outputs:
        for k in ("y_H", "y_Hp", "y_Hm"):
            out[k] = torch.empty(n, dtype=torch.float64, device=device)
        out["status"] = torch.empty(n, dtype=torch.uint8, device=device)
        out["n_sub"] = torch.empty(n, dtype=torch.int32, device=device)
        out["n_itr"] = torch.empty(n, dtype=torch.int32, device=device)
    return out


def to_host(cells: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in cells.items() if v is not None}
