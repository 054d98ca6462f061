"""Shared helpers of the GPU parity tests (run the CUDA path, compare with the
oracle).  Imported by the tests only."""
import numpy as np

import inputs

FIELDS_CMP = ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H")

# The FP64 bar (the thresholds of the mixed-precision workload description:
# relative above 1e-8, absolute below): 1e-9 relative on T_g, T_d, E_IR and
# on abundances above 1e-8, 1e-17 absolute below.  y_H = 1 - 2 y_H2 - y_e is
# formed by subtraction from 1, so its absolute rounding is that of numbers
# near 1: its bar is max(1e-9 |y_H|, 2^-52).
Y_SMALL = 1e-8
FP64_REL, FP64_ABS, ULP1 = 1e-9, 1e-17, 2.0 ** -52


def fp64_score(got, ref, idx=None):
    """Per cell, the largest error over FIELDS_CMP in units of its FP64 bar
    (a cell meets the bar when the score is <= 1)."""
    worst = None
    for k in FIELDS_CMP:
        a, b = got[k], ref[k]
        if idx is not None:
            a = a[idx]
        d = np.abs(a - b)
        if k == "y_H":
            bar = np.maximum(FP64_REL * np.abs(b), ULP1)
        elif k.startswith("y_"):
            bar = np.where(np.abs(b) > Y_SMALL, FP64_REL * np.abs(b), FP64_ABS)
        else:
            bar = FP64_REL * np.abs(b)
        e = d / bar
        worst = e if worst is None else np.maximum(worst, e)
    return worst


def mixed_errors(got, ref, idx=None):
    """Per field, per cell: the relative error where |ref| > 1e-8 (NaN below)
    and the absolute error where |ref| <= 1e-8 (NaN above)."""
    out = {}
    for k in FIELDS_CMP:
        a, b = got[k], ref[k]
        if idx is not None:
            a = a[idx]
        big = np.abs(b) > Y_SMALL
        d = np.abs(a - b)
        out[k] = (np.where(big, d / np.where(big, np.abs(b), 1.0), np.nan), np.where(big, np.nan, d))
    return out


def run_gpu(cells, dt, cd_factor=1.0, precision="fp64", batched=None, **cfg):
    import torch
    import paper_2604_21438_gb300 as sf
    s = sf.Solver(precision, **cfg)
    d = sf.to_device(cells)
    if batched is None:
        s.step(d, dt, cd_factor)
    else:
        off, bdt = batched
        s.step_batched(d, off, bdt, cd_factor)
    torch.cuda.synchronize()
    out = sf.to_host(d)
    out["_stats"] = s.stats()
    s.close()
    return out


def errors(got, ref, small=1e-8, idx=None):
    """Per field: max relative error where |ref| > small, and max absolute
    error where |ref| <= small."""
    out = {}
    for k in FIELDS_CMP:
        a, b = got[k], ref[k]
        if idx is not None:
            a = a[idx]
        big = np.abs(b) > small
        rel = np.abs(a - b)[big] / np.abs(b)[big]
        ab = np.abs(a - b)[~big]
        out[k] = (float(rel.max()) if rel.size else 0.0, float(ab.max()) if ab.size else 0.0)
    return out


def err_summary(got, ref, small=1e-8, idx=None):
    """max / p99 / median of the relative error (abundances below `small`
    measured in units of `small`)."""
    res = {}
    for k in FIELDS_CMP:
        a, b = got[k], ref[k]
        if idx is not None:
            a = a[idx]
        e = np.where(np.abs(b) > small, np.abs(a - b) / np.maximum(np.abs(b), 1e-300), np.abs(a - b) / small)
        res[k] = dict(max=float(e.max()), p99=float(np.percentile(e, 99)), median=float(np.median(e)))
    return res


# status bits that flag a cell (not the tight-coupling mode bit)
FLAGGED = 1 | 2 | 4 | 16


def sample_with_flagged(got, n_cells, n, seed):
    """Sorted indices of a seeded sample of n cells plus every cell whose
    GPU status carries a flag (substep cap, bad input, Newton limit, bad
    step)."""
    idx = np.random.default_rng(seed).choice(n_cells, min(n, n_cells), replace=False)
    flagged = np.nonzero(got["status"] & FLAGGED)[0]
    return np.unique(np.concatenate([idx, flagged]))
