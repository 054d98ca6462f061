"""Host-side checks of the C ABI: the library loads, exports every entry point
that include/sfchem.h declares, and rejects bad arguments on the host before
touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2604_21438_gb300 as sf

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sfchem.h")


def declared_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sfchem_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(sf.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = sf.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_default_config_and_validation():
    L = sf.lib()
    c = sf.default_config()
    assert c.f_chem == 0.03 and c.n_cyc == 300 and c.nr_itr_limit == 20 and c.nr_tol == 1e-5
    assert c.reaction_mask == 0xFFF and c.process_mask == sf.P_ALL and c.flags == 0
    assert L.sfchem_config_validate(ctypes.byref(c)) == sf.OK
    bad = [dict(f_chem=0.0), dict(f_chem=1.5), dict(n_cyc=0), dict(gamma_ad=1.0), dict(y_floor=0.0),
           dict(precision=2), dict(reaction_mask=1 << 12), dict(process_mask=1 << 17), dict(flags=1 << 8),
           dict(nr_tol=-1.0), dict(Z=float("nan")), dict(reserved=1), dict(n_sub_max=0)]
    for kw in bad:
        c = sf.default_config(**kw)
        assert L.sfchem_config_validate(ctypes.byref(c)) == sf.EINVAL, kw
    assert L.sfchem_config_validate(None) == sf.EINVAL


def test_host_rejections_before_any_launch():
    L = sf.lib()
    h = ctypes.c_void_p()
    bad = sf.default_config(f_chem=-1.0)
    assert L.sfchem_init(ctypes.byref(bad), ctypes.byref(h)) == sf.EINVAL
    assert L.sfchem_init(None, None) == sf.EINVAL
    st, fl = sf.sfchem_state_t(), sf.sfchem_fields_t()
    assert L.sfchem_step(None, ctypes.byref(st), ctypes.byref(fl), 10, 1.0, 1.0, None) == sf.ENOTINIT
    assert L.sfchem_stats(None, None) == sf.ENOTINIT
    assert L.sfchem_finalize(None) == sf.ENOTINIT
    assert L.sfchem_step_batched(None, None, None, None, None, 0, 1.0, None) == sf.ENOTINIT
    assert L.sfchem_step_host(None, None, None, None, None, 0, 1.0, 0, None) == sf.ENOTINIT
    assert L.sfchem_step_nr(None, ctypes.byref(st), ctypes.byref(fl), 10, 1.0, 1.0, None) == sf.ENOTINIT


def test_strerror_and_version():
    L = sf.lib()
    for code in range(6):
        assert L.sfchem_strerror(code)
    assert L.sfchem_strerror(99) == b"unknown status"
    assert re.match(rb"\d+\.\d+\.\d+", L.sfchem_version())


def _header_constants():
    """Integer constants of the header's enums and #defines (1u << k and
    (1u << k) - 1u forms), by name."""
    txt = re.sub(r"/\*.*?\*/", "", open(HDR).read(), flags=re.S)
    out = {}
    for name, expr in re.findall(r"\b(SFCHEM_[A-Z0-9_]+)\s*=\s*([^,}\n]+)", txt):
        expr = expr.strip()
        m = re.fullmatch(r"\(1u << (\d+)\) - 1u", expr)
        if m:
            out[name] = (1 << int(m.group(1))) - 1
            continue
        m = re.fullmatch(r"1u << (\d+)", expr)
        out[name] = (1 << int(m.group(1))) if m else int(expr)
    for name, val in re.findall(r"#define\s+(SFCHEM_[A-Z0-9_]+)\s+(\d+)", txt):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    h = _header_constants()
    assert (h["SFCHEM_FP64"], h["SFCHEM_MIXED"]) == (sf.FP64, sf.MIXED)
    for k in ("OK", "EINVAL", "ENOTINIT", "ECUDA", "ETIMEOUT", "ENOMEM"):
        assert h["SFCHEM_" + k] == getattr(sf, k), k
    for k in ("CAP", "BADINPUT", "NOCONV", "TIGHT", "BADSTEP"):
        assert h["SFCHEM_CELL_" + k] == getattr(sf, "CELL_" + k), k
    for k in ("FREEZE_TG", "FREEZE_TD", "FREEZE_EIR", "FREEZE_YH2", "FREEZE_YE", "SPLIT", "REFINE_FF"):
        assert h["SFCHEM_F_" + k] == getattr(sf, "F_" + k), k
    assert h["SFCHEM_P_ALL"] == sf.P_ALL
    assert h["SFCHEM_HOST_SLICE_DEFAULT"] > 0
    # the process bits are the 17 distinct bits under P_ALL
    bits = [v for k, v in h.items() if k.startswith("SFCHEM_P_") and k != "SFCHEM_P_ALL"]
    assert len(bits) == 17 and sum(bits) == sf.P_ALL


def _device_constants():
    """constexpr integer constants of the kernels' header (csrc/li_device.cuh)."""
    path = os.path.join(os.path.dirname(HDR), "..", "paper_2604_21438_gb300", "csrc", "li_device.cuh")
    txt = re.sub(r"//.*", "", open(path).read())
    out = {}
    for decl in re.findall(r"constexpr\s+uint(?:8|32)_t\s+([^;]+);", txt):
        for name, expr in re.findall(r"([A-Z][A-Z0-9_]*)\s*=\s*([^,]+)", decl):
            expr = expr.strip()
            m = re.fullmatch(r"\(1u << (\d+)\) - 1u", expr)
            if m:
                out[name] = (1 << int(m.group(1))) - 1
                continue
            m = re.fullmatch(r"1u << (\d+)", expr)
            out[name] = (1 << int(m.group(1))) if m else int(expr)
    return out


def test_kernel_constants_match_the_header():
    """The kernels keep their own copies of the status, flag and mask bits;
    they must equal the public header's."""
    h, d = _header_constants(), _device_constants()
    pairs = dict(ST_CAP="CELL_CAP", ST_BAD="CELL_BADINPUT", ST_NOCONV="CELL_NOCONV", ST_TIGHT="CELL_TIGHT",
                 ST_BADSTEP="CELL_BADSTEP", F_FTG="F_FREEZE_TG", F_FTD="F_FREEZE_TD", F_FE="F_FREEZE_EIR",
                 F_FY2="F_FREEZE_YH2", F_FYE="F_FREEZE_YE", F_SPLIT="F_SPLIT", F_REFINE_FF="F_REFINE_FF",
                 P_ALL="P_ALL")
    for dev, pub in pairs.items():
        assert d[dev] == h["SFCHEM_" + pub], dev
    dev_p = sorted(v for k, v in d.items() if k.startswith("P_") and k != "P_ALL")
    pub_p = sorted(v for k, v in h.items() if k.startswith("SFCHEM_P_") and k != "SFCHEM_P_ALL")
    assert dev_p == pub_p
    assert d["R_ALL"] == (1 << 12) - 1        # reactions H0 ... H11 of Table 3
