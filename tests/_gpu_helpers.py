"""Shared helpers of the GPU parity tests (run the CUDA path, compare with the
oracle).  Imported by the tests only."""
import numpy as np

import inputs

FIELDS_CMP = ("T_g", "T_d", "E_IR", "y_H2", "y_e", "y_H")
# An abundance carries an absolute rounding error of about eps times the
# largest value it held along the trajectory (up to 1), so relative errors are
# taken only above 1e-6; below, the error is measured in units of 1e-6
# (1e-9 of relative error at the threshold = 1e-15 absolute).
Y_FLOOR = 1e-6


def cell_errors(got, ref, idx=None, y_floor=Y_FLOOR):
    """Per cell, the largest normalised error over FIELDS_CMP."""
    worst = None
    for k in FIELDS_CMP:
        a, b = got[k], ref[k]
        if idx is not None:
            a = a[idx]
        floor = y_floor if k.startswith("y_") else 1e-300
        e = np.abs(a - b) / np.maximum(np.abs(b), floor)
        worst = e if worst is None else np.maximum(worst, e)
    return worst


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
