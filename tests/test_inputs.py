"""The seeded workload generators draw what their recipes state: ranges,
marginals, block layouts and the time steps of the AMR hierarchy."""
import numpy as np
from scipy import stats

import inputs

TCMB = 2.725


def _valid(c):
    assert set(inputs.FIELDS) <= set(c)
    n = len(c["n_H"])
    for k in inputs.FIELDS:
        assert c[k].dtype == np.float64 and c[k].shape == (n,) and np.all(np.isfinite(c[k])), k
    assert np.all(c["y_e"] >= 0) and np.all(c["y_H2"] >= 0)
    assert np.all(2 * c["y_H2"] + c["y_e"] <= 1 + 1e-12)
    # IR radiation in equilibrium with the dust: a T_IR^4 = (c~/c) E_IR = a T_d^4
    np.testing.assert_allclose(c["E_IR"], 1e4 * 7.565733250e-15 * c["T_d"] ** 4, rtol=1e-12)


def test_uniform_marginals():
    c = inputs.cells_uniform(4096, seed=1001)
    _valid(c)
    for k, lo, hi in (("n_H", 0, 6), ("T_g", 1, 4), ("G0", -2, 4), ("n_EUV", -6, 2), ("N_H2", 14, 22)):
        v = (np.log10(c[k]) - lo) / (hi - lo)
        assert v.min() >= 0 and v.max() <= 1
        assert stats.kstest(v, "uniform").pvalue > 1e-3, k
    assert stats.kstest((c["T_d"] - 8) / 22, "uniform").pvalue > 1e-3
    assert stats.kstest((np.log10(c["y_e"]) + 8) / 7, "uniform").pvalue > 1e-3
    assert stats.kstest(c["y_H2"] / ((1 - c["y_e"]) / 2), "uniform").pvalue > 1e-3
    # the same seed draws the same cells
    d = inputs.cells_uniform(4096, seed=1001)
    assert all(np.array_equal(c[k], d[k]) for k in inputs.FIELDS)


def test_grf_marginals_and_correlation_length():
    c = inputs.cells_grf(32, seed=1002)
    _valid(c)
    v = np.log10(c["n_H"]) / 6
    assert v.min() >= 0 and v.max() <= 1
    # a Gaussian random field smoothed over 8 cells: neighbours are strongly
    # correlated, cells 16 apart much less
    g = np.log10(c["n_H"]).reshape(32, 32, 32)
    near = np.corrcoef(g.ravel(), np.roll(g, 1, axis=2).ravel())[0, 1]
    far = np.corrcoef(g.ravel(), np.roll(g, 16, axis=2).ravel())[0, 1]
    assert near > 0.95 and far < near - 0.3


def test_amr_hierarchy():
    c, off, bdt, lvl = inputs.cells_amr(seed=1004)
    _valid(c)
    assert len(bdt) == 3000 and len(off) == 3001 and off[-1] == 3000 * 512
    assert lvl.min() == 0 and lvl.max() == 6
    np.testing.assert_allclose(bdt, 1e3 * inputs.YR / 2.0 ** lvl, rtol=1e-15)
    assert c["n_H"].min() >= 1e2 * (1 - 1e-12) and c["n_H"].max() <= 1e8 * (1 + 1e-12)
    assert c["T_g"].min() >= 10 - 1e-9 and c["T_g"].max() <= 1e4 + 1e-9


def test_gmc_lognormal_density():
    c = inputs.cells_gmc(64, seed=1005)
    _valid(c)
    ln = np.log(c["n_H"])
    # ln n ~ N(ln 100 - 1.125, 1.5^2): mean density 100 cm^-3
    assert abs(ln.std() - 1.5) < 0.15
    assert abs(ln.mean() - (np.log(100.0) - 1.125)) < 0.3
    assert c["T_g"].min() >= 10 - 1e-9 and c["T_g"].max() <= 1e4 + 1e-9
    # temperature anti-correlated with density
    assert np.corrcoef(ln, np.log(c["T_g"]))[0, 1] < -0.9


def test_block_major_is_a_permutation():
    c = inputs.cells_grf(32, seed=3)
    b, off = inputs.block_major(c, 32, 16)
    assert len(off) == 9 and off[-1] == 32 ** 3
    for k in inputs.FIELDS:
        assert np.array_equal(np.sort(b[k]), np.sort(c[k]))
    # the first block holds the x-fastest 16^3 corner of the grid
    g = c["T_g"].reshape(32, 32, 32)
    assert np.array_equal(b["T_g"][:4096], g[:16, :16, :16].ravel())
