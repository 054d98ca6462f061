"""Metallicity sweep on the initial Bonnor-Ebert sphere (Sec. 4.3, Table
BEsphere seeds): the CUDA path against the oracle at Z = 1, 1e-2 and 1e-4
Z_sun, where the dust abundance f_d = Z / Z_sun scales the IR row and the
gas-dust coupling of Appendix C, H2 formation on grains and the metal lines.
C_d = 1e7 erg g^-1 K^-1 (the paper's choice for the low-metallicity runs).

Bars as in the other workloads' tests: the FP64 parity bar of
tests/test_gpu_fp64.py (every cell, or an oracle that is itself that
sensitive) and the stated mixed-precision bound of the AMR workload
(tests/test_gpu_mixed_batched.py)."""
import numpy as np
import pytest

import inputs
import oracle
from _gpu_helpers import fp64_score, run_gpu
from test_gpu_fp64 import assert_parity
from test_gpu_mixed_batched import BOUND_AMR, check_mixed

pytestmark = pytest.mark.gpu
CD = 1e3   # C_d = 1e7


def _sample(Z, n=3000, seed=5):
    cells, off, lev = inputs.cells_be(Z)
    idx = np.sort(np.random.default_rng(seed).choice(len(cells["n_H"]), n, replace=False))
    return cells, off, idx


def _ocfg(Z):
    c = oracle.default_config()
    c.Z = Z
    return c


@pytest.mark.parametrize("Z", [1.0, 1e-2, 1e-4])
def test_fp64_matches_oracle(Z):
    cells, _, idx = _sample(Z)
    sub = inputs.subset(cells, idx)
    dt = inputs.be_dt()
    ref = oracle.li_step(sub, dt, CD, _ocfg(Z))
    got = run_gpu(sub, dt, CD, Z=Z)
    assert_parity(got, ref, cells=sub, dt=dt, cd=CD, cfg=_ocfg(Z))


@pytest.mark.parametrize("Z", [1e-2, 1e-4])
def test_mixed_batched_full_sphere_sampled(Z):
    """The whole sphere (720,896 cells in 1408 blocks) through the batched
    mixed path; sampled cells against the oracle."""
    cells, off, idx = _sample(Z)
    dt = inputs.be_dt()
    bdt = np.full(len(off) - 1, dt)
    got = run_gpu(cells, None, CD, precision="mixed", batched=(off, bdt), Z=Z)
    ref = oracle.li_step(inputs.subset(cells, idx), dt, CD, _ocfg(Z))
    check_mixed(got, ref, idx=idx, bound=BOUND_AMR, cells=cells, dt=dt, cd=CD, cfg=_ocfg(Z))
    assert got["_stats"]["cells"] == len(cells["n_H"])


def test_metallicity_changes_the_result():
    """f_d reaches the kernels: the same cells at Z = 1 and Z = 1e-2 (with the
    Z = 1 seeds) end in different states."""
    cells, _, idx = _sample(1.0, n=256)
    sub = inputs.subset(cells, idx)
    dt = inputs.be_dt()
    a = run_gpu(sub, dt, CD, Z=1.0)
    b = run_gpu(sub, dt, CD, Z=1e-2)
    ref = oracle.li_step(sub, dt, CD, _ocfg(1e-2))
    assert np.max(np.abs(a["y_H2"] - b["y_H2"])) > 1e-6
    assert np.percentile(fp64_score(b, ref), 99) <= 1.0
