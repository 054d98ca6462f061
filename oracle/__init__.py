"""Python access to the plain FP64 CPU oracle (``oracle/sfchem_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path (``libsfchem`` and
its binding) never imports this package, and this package imports nothing
from the product path.

The oracle implements the linearized-implicit (LI) thermochemical step of
SFUMATO# (arXiv 2604.21438, Sec. 2.2.8 with Appendices A-C) and the
Newton-Raphson backward-Euler reference solver of Sec. 2.2.8.  Parity of the
stand-in physics (the rates and processes the paper only cites: k_H4, k_H9,
k_H10, k_H11, photo-heating, photoelectric heating, line cooling and the dust
opacity) is unpinned against nature: those functions are pinned only through
closed forms and invariants (the line cooling's LTE limit excepted, which is
pinned to atomic data).  Parity unpinned as well: the critical densities
of k_H7 and of Gamma_1 (their limits are pinned) and the prefactor and He+
abundance of Lambda_10.

SFCHEM_ORACLE_LIB, when set, names a build of a modified copy of the oracle
that lib() loads instead of this one (the mutation check of the pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfchem_oracle.cpp")
_HDR = os.path.join(_HERE, "sfchem_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
# A second build of the same source with floating-point contraction allowed
# (-ffp-contract=fast): on a machine with fused multiply-add (aarch64) it is
# the oracle with another, equally valid FP64 rounding sequence.  The tests
# use it to measure how much a cell's result depends on FP64 rounding at all.
_LIB_FMA = os.path.join(_HERE, "liboracle_fma.so")
_lock = threading.RLock()
_lib = None
_lib_fma = None

# process_mask bits (Table 4 rows and the Appendix C dust terms)
P_G1_H2FORM, P_G2_PHOTOION, P_G3_PHOTODISS, P_G4_PHOTOELEC = 1 << 0, 1 << 1, 1 << 2, 1 << 3
P_L5_HION, P_L6_H2DISS, P_L7_HREC, P_L8_HMFB = 1 << 4, 1 << 5, 1 << 6, 1 << 7
P_L9_HEXC, P_L10_HEPEXC, P_L11_FF, P_L12_COMPTON = 1 << 8, 1 << 9, 1 << 10, 1 << 11
P_L13_LINE, P_GASGRAIN, P_DUST_UV, P_DUST_EMIT, P_DUST_IRABS = 1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16
P_ALL = (1 << 17) - 1
P_GAS_ONLY = P_ALL & ~(P_GASGRAIN | P_DUST_UV | P_DUST_EMIT | P_DUST_IRABS)
# flags
F_FREEZE_TG, F_FREEZE_TD, F_FREEZE_EIR, F_FREEZE_YH2, F_FREEZE_YE, F_SPLIT = 1, 2, 4, 8, 16, 32
F_NO_REJECT = 64   # paper-literal controller (no step rejection)
F_FREEZE_THERMAL = F_FREEZE_TG | F_FREEZE_TD | F_FREEZE_EIR
# status bits
ST_CAP, ST_BADINPUT, ST_NOCONV, ST_TIGHT, ST_BADSTEP = 1, 2, 4, 8, 16


class OracleConfig(ctypes.Structure):
    _fields_ = [
        ("f_chem", ctypes.c_double),
        ("n_cyc", ctypes.c_int32),
        ("n_sub_max", ctypes.c_int32),
        ("Z", ctypes.c_double),
        ("gamma_ad", ctypes.c_double),
        ("y_floor", ctypes.c_double),
        ("reaction_mask", ctypes.c_uint32),
        ("process_mask", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("nr_itr_limit", ctypes.c_int32),
        ("nr_tol", ctypes.c_double),
    ]


def build(force: bool = False, fma: bool = False) -> str:
    """Compile liboracle.so (plain g++, OpenMP) if missing or stale
    (fma=True: liboracle_fma.so, the same source with contraction allowed)."""
    out = _LIB_FMA if fma else _LIB
    with _lock:
        stale = (not os.path.exists(out)) or any(
            os.path.getmtime(p) > os.path.getmtime(out) for p in (_SRC, _HDR))
        if force or stale:
            # -ffp-contract=off: no fused multiply-adds the source does not ask
            # for, so the oracle gives the same numbers on x86-64 and aarch64
            contract = "-ffp-contract=fast" if fma else "-ffp-contract=off"
            cmd = ["g++", "-O3", contract, "-fopenmp", "-fPIC", "-shared", "-std=c++17",
                   "-o", out + ".tmp", _SRC]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(out + ".tmp", out)
    return out


_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "liboracle_opcount.so")
_opc = None
OPCOUNT_SECTIONS = ("system", "solve", "newton", "control")
OPCOUNT_OPS = ("add", "mul", "div", "fma", "sqrt", "exp", "log", "pow", "cmp")


def build_opcount(force: bool = False) -> str:
    """Compile the op-counting build of the oracle (opcount.cpp) if stale."""
    with _lock:
        srcs = (_OPC_SRC, _SRC, _HDR)
        stale = (not os.path.exists(_OPC_LIB)) or any(os.path.getmtime(p) > os.path.getmtime(_OPC_LIB) for p in srcs)
        if force or stale:
            cmd = ["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17", "-o", _OPC_LIB + ".tmp",
                   _OPC_SRC]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(_OPC_LIB + ".tmp", _OPC_LIB)
    return _OPC_LIB


def opcount(cells: dict, dt, cd_factor: float = 1.0, cfg: OracleConfig | None = None, method: str = "li") -> dict:
    """Floating-point operations of the oracle's LI step (method "li") or
    Newton-Raphson step ("nr") on these cells, counted by type and section
    (single thread).  Returns {"substeps": N, "cells": valid cells,
    "counts": {section: {op: count}}, "per_substep": {...}, "per_cell": {...}}
    where flops count add/sub, mul and div as 1 and fma as 2, and sqrt /
    exp / log / pow are reported apart."""
    global _opc
    if _opc is None:
        build_opcount()
        L = ctypes.CDLL(_OPC_LIB)
        L.oracle_opcount_li.restype = ctypes.c_int64
        L.oracle_opcount_nr.restype = ctypes.c_int64
        _opc = L
    fn = {"li": _opc.oracle_opcount_li, "nr": _opc.oracle_opcount_nr}[method]
    cfg = cfg or default_config()
    n = len(cells["n_H"])
    a = {k: np.ascontiguousarray(cells[k], dtype=np.float64) for k in FIELDS_IN + FIELDS_STATE}
    dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
    counts = np.zeros((len(OPCOUNT_SECTIONS), len(OPCOUNT_OPS)), np.uint64)
    nsub = fn(
        ctypes.c_int64(n), _p(a["n_H"]), _p(a["T_g"]), _p(a["T_d"]), _p(a["E_IR"]), _p(a["y_H2"]), _p(a["y_e"]),
        _p(a["G0"]), _p(a["n_EUV"]), _p(a["N_H2"]), _p(dtv), ctypes.c_double(cd_factor), ctypes.byref(cfg),
        _p(counts))
    if nsub < 0:
        raise ValueError(f"oracle_opcount_{method} rejected its arguments")
    out = {"substeps": int(nsub), "cells": int(n), "counts": {}, "per_substep": {}, "per_cell": {}}
    tot = np.zeros(len(OPCOUNT_OPS))
    for i, sec in enumerate(OPCOUNT_SECTIONS):
        out["counts"][sec] = {op: int(counts[i, j]) for j, op in enumerate(OPCOUNT_OPS)}
        tot += counts[i]
    for key, den in (("per_substep", max(nsub, 1)), ("per_cell", max(n, 1))):
        d = dict(zip(OPCOUNT_OPS, tot / den))
        out[key] = {op: float(v) for op, v in d.items()}
        out[key]["flops"] = float(d["add"] + d["mul"] + d["div"] + 2 * d["fma"])
        out[key]["transcendentals"] = float(d["sqrt"] + d["exp"] + d["log"] + d["pow"])
    return out


def lib(fma: bool = False):
    global _lib, _lib_fma
    if fma:
        if _lib_fma is None:
            build(fma=True)
            _lib_fma = _setup(ctypes.CDLL(_LIB_FMA))
        return _lib_fma
    if _lib is None:
        # SFCHEM_ORACLE_LIB: a build of a modified copy of the oracle, loaded
        # in place of this one (tests/test_oracle_mutations.py plants a
        # mistake in such a copy and checks that a pin fails)
        alt = os.environ.get("SFCHEM_ORACLE_LIB")
        if alt:
            _lib = _setup(ctypes.CDLL(os.path.abspath(alt)))
        else:
            build()
            _lib = _setup(ctypes.CDLL(_LIB))
    return _lib


def _setup(L):
    """Argument and result types of the oracle's C functions."""
    dp = ctypes.POINTER(ctypes.c_double)
    L.oracle_default_config.argtypes = [ctypes.POINTER(OracleConfig)]
    L.oracle_li_cells.restype = ctypes.c_int
    L.oracle_nr_cells.restype = ctypes.c_int
    L.oracle_li_trace.restype = ctypes.c_int
    L.oracle_li_trace.argtypes = [ctypes.c_double] * 11 + [
        ctypes.POINTER(OracleConfig), ctypes.c_int, dp, ctypes.POINTER(ctypes.c_uint8)]
    L.oracle_rates.argtypes = [ctypes.c_double] * 6 + [ctypes.POINTER(OracleConfig), dp]
    L.oracle_system.argtypes = [ctypes.c_double, dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(OracleConfig), dp, dp, dp, dp, dp, dp]
    L.oracle_rhs.argtypes = [ctypes.c_double, dp, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_double, ctypes.POINTER(OracleConfig), dp]
    L.oracle_photon_update.restype = ctypes.c_int
    L.oracle_set_perturbation.argtypes = [ctypes.c_double]
    L.oracle_set_perturbation.restype = None
    L.oracle_solve5.argtypes = [dp, dp, dp]
    L.oracle_solve5.restype = ctypes.c_int
    return L


def default_config(**kw) -> OracleConfig:
    c = OracleConfig()
    lib().oracle_default_config(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


FIELDS_IN = ("n_H", "G0", "n_EUV", "N_H2")
FIELDS_STATE = ("T_g", "T_d", "E_IR", "y_H2", "y_e")


def li_step(cells: dict, dt, cd_factor: float = 1.0, cfg: OracleConfig | None = None,
            n_threads: int = 0, fma: bool = False, perturb: float = 0.0) -> dict:
    """LI step (Sec. 2.2.8) on a dict of 1-D float64 arrays; returns a new dict.

    ``dt`` is a scalar (seconds) or one value per cell; fma=True runs the
    build with floating-point contraction allowed; perturb != 0 multiplies
    every entry of each substep's linear system by 1 +- perturb (a test of
    the result's sensitivity to rounding-level changes)."""
    if perturb:
        with _lock:
            L = lib(fma)
            L.oracle_set_perturbation(ctypes.c_double(perturb))
            try:
                return _li_step(cells, dt, cd_factor, cfg, n_threads, fma)
            finally:
                L.oracle_set_perturbation(ctypes.c_double(0.0))
    return _li_step(cells, dt, cd_factor, cfg, n_threads, fma)


def _li_step(cells, dt, cd_factor, cfg, n_threads, fma):
    cfg = cfg or default_config()
    n = len(cells["n_H"])
    st = {k: np.array(cells[k], dtype=np.float64, copy=True) for k in FIELDS_STATE}
    ins = {k: np.ascontiguousarray(cells[k], dtype=np.float64) for k in FIELDS_IN}
    dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
    out = {k: np.empty(n) for k in ("y_H", "y_Hp", "y_Hm")}
    status = np.zeros(n, np.uint8)
    n_sub = np.zeros(n, np.int32)
    n_itr = np.zeros(n, np.int32)
    n_rej = np.zeros((n, 2), np.int32)
    rc = lib(fma).oracle_li_cells(
        ctypes.c_int64(n), _p(ins["n_H"]), _p(st["T_g"]), _p(st["T_d"]), _p(st["E_IR"]),
        _p(st["y_H2"]), _p(st["y_e"]), _p(out["y_H"]), _p(out["y_Hp"]), _p(out["y_Hm"]),
        _p(status), _p(n_sub), _p(n_itr), _p(n_rej), _p(ins["G0"]), _p(ins["n_EUV"]), _p(ins["N_H2"]),
        _p(dtv), ctypes.c_double(cd_factor), ctypes.byref(cfg), ctypes.c_int(n_threads))
    if rc != 0:
        raise ValueError("oracle_li_cells rejected its arguments")
    st.update(out)
    st.update(status=status, n_sub=n_sub, n_itr=n_itr, n_rej=n_rej[:, 0].copy(), n_halv=n_rej[:, 1].copy())
    return st


HNU_FUV = 12.4 * 1.602176634e-12    # erg: mean FUV photon energy (stand-in)
U_HABING = 5.29e-14                 # erg cm^-3 per Habing unit (stand-in)


def photon_update(cells: dict, dt) -> dict:
    """Photon consumption after the update (oracle_photon_update): returns
    {"G0", "n_EUV", "absorbed"} with absorbed[:, 0..3] = EUV by H, EUV by
    dust, FUV by H2, FUV by dust (photons cm^-3)."""
    n = len(cells["n_H"])
    a = {k: np.ascontiguousarray(cells[k], dtype=np.float64) for k in ("n_H", "y_H2", "y_e", "G0", "n_EUV", "N_H2")}
    dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
    G0, nE, ab = np.empty(n), np.empty(n), np.empty((n, 4))
    rc = lib().oracle_photon_update(ctypes.c_int64(n), _p(a["n_H"]), _p(a["y_H2"]), _p(a["y_e"]), _p(a["G0"]),
                                    _p(a["n_EUV"]), _p(a["N_H2"]), _p(dtv), _p(G0), _p(nE), _p(ab))
    if rc != 0:
        raise ValueError("oracle_photon_update rejected its arguments")
    return {"G0": G0, "n_EUV": nE, "absorbed": ab}


def nr_step(cells: dict, dt, cd_factor: float = 1.0, cfg: OracleConfig | None = None,
            n_threads: int = 0) -> dict:
    """Newton-Raphson backward-Euler reference step (Sec. 2.2.8)."""
    cfg = cfg or default_config()
    n = len(cells["n_H"])
    st = {k: np.array(cells[k], dtype=np.float64, copy=True) for k in FIELDS_STATE}
    ins = {k: np.ascontiguousarray(cells[k], dtype=np.float64) for k in FIELDS_IN}
    dtv = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (n,)))
    status = np.zeros(n, np.uint8)
    n_sub = np.zeros(n, np.int32)
    n_itr = np.zeros(n, np.int32)
    rc = lib().oracle_nr_cells(
        ctypes.c_int64(n), _p(ins["n_H"]), _p(st["T_g"]), _p(st["T_d"]), _p(st["E_IR"]),
        _p(st["y_H2"]), _p(st["y_e"]), _p(status), _p(n_sub), _p(n_itr), _p(ins["G0"]),
        _p(ins["n_EUV"]), _p(ins["N_H2"]), _p(dtv), ctypes.c_double(cd_factor),
        ctypes.byref(cfg), ctypes.c_int(n_threads))
    if rc != 0:
        raise ValueError("oracle_nr_cells rejected its arguments")
    st.update(status=status, n_sub=n_sub, n_itr=n_itr)
    return st


def li_trace(cell: dict, dt: float, cd_factor: float = 1.0, cfg: OracleConfig | None = None,
             max_rec: int = 200000):
    """One cell's LI step with every substep recorded.

    Returns (rec, status): rec[k] = (t_end, dt_s, y_H2, y_e, T_g, T_d, E_IR)."""
    cfg = cfg or default_config()
    rec = np.zeros((max_rec, 7))
    st = ctypes.c_uint8(0)
    dp = ctypes.POINTER(ctypes.c_double)
    ns = lib().oracle_li_trace(
        *(ctypes.c_double(float(cell[k])) for k in ("n_H", "T_g", "T_d", "E_IR", "y_H2", "y_e",
                                                      "G0", "n_EUV", "N_H2")),
        ctypes.c_double(dt), ctypes.c_double(cd_factor), ctypes.byref(cfg), max_rec,
        rec.ctypes.data_as(dp), ctypes.byref(st))
    return rec[:min(ns, max_rec)], st.value


def rates(T_g, T_d, n_H, G0=0.0, n_EUV=0.0, N_H2=0.0, cfg: OracleConfig | None = None):
    cfg = cfg or default_config()
    k = np.zeros(12)
    lib().oracle_rates(T_g, T_d, n_H, G0, n_EUV, N_H2, ctypes.byref(cfg),
                       k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return k


def system(n_H, u, G0, n_EUV, N_H2, dt, cd_factor=1.0, cfg: OracleConfig | None = None):
    """(A, b, F, Mdiag, ts, aux) of one LI substep at state u."""
    cfg = cfg or default_config()
    dp = ctypes.POINTER(ctypes.c_double)
    u = np.ascontiguousarray(u, dtype=np.float64)
    A, b, F, M, ts, aux = np.zeros(25), np.zeros(5), np.zeros(5), np.zeros(5), np.zeros(3), np.zeros(5)
    lib().oracle_system(n_H, u.ctypes.data_as(dp), G0, n_EUV, N_H2, dt, cd_factor,
                        ctypes.byref(cfg), *(a.ctypes.data_as(dp) for a in (A, b, F, M, ts, aux)))
    return A.reshape(5, 5), b, F, M, ts, aux


def rhs(n_H, u, G0, n_EUV, N_H2, cd_factor=1.0, cfg: OracleConfig | None = None):
    cfg = cfg or default_config()
    dp = ctypes.POINTER(ctypes.c_double)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(5)
    lib().oracle_rhs(n_H, u.ctypes.data_as(dp), G0, n_EUV, N_H2, cd_factor, ctypes.byref(cfg),
                     out.ctypes.data_as(dp))
    return out


def solve5(A, b):
    dp = ctypes.POINTER(ctypes.c_double)
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(25)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(5)
    rc = lib().oracle_solve5(A.ctypes.data_as(dp), b.ctypes.data_as(dp), x.ctypes.data_as(dp))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x
