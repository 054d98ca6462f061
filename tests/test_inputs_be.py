"""The Bonnor-Ebert sphere workload against what the paper and the textbook
fix: Table BEsphere's seeds and the critical isothermal sphere."""
import numpy as np
import pytest

import inputs

# Table BEsphere as printed: Z, T_g, y_H2, y_H, y_H+
TABLE = [(1.0, 5.0, 4.98e-1, 4.40e-3, 1.27e-7),
         (1e-2, 21.0, 3.47e-2, 9.30e-1, 1.99e-7),
         (1e-4, 190.0, 1.18e-3, 9.98e-1, 8.29e-7)]


@pytest.mark.parametrize("Z,T,y2,yH,yp", TABLE)
def test_seeds_follow_table(Z, T, y2, yH, yp):
    cells, off, lev = inputs.cells_be(Z)
    assert np.all(cells["T_g"] == T) and np.all(cells["y_H2"] == y2) and np.all(cells["y_e"] == yp)
    y_H = 1.0 - 2.0 * cells["y_H2"] - cells["y_e"]
    # the printed y_H agrees with H-nuclei conservation to the rounding of
    # the printed values (three significant digits)
    tol = 2 * 0.5 * 10.0 ** (np.floor(np.log10(y2)) - 2) + 0.5 * 10.0 ** (np.floor(np.log10(yH)) - 2)
    assert np.all(np.abs(y_H - yH) <= tol)
    assert np.all(cells["G0"] == 0.0) and np.all(cells["n_EUV"] == 0.0)


def test_critical_sphere_and_grid():
    cells, off, lev = inputs.cells_be(1.0)
    n = cells["n_H"]
    assert len(n) == 720896 and len(off) == 1409 and off[-1] == len(n)
    assert np.bincount(lev).tolist() == [448, 448, 512]
    # critical Bonnor-Ebert sphere: centre-to-edge density contrast 14.04
    # at xi = 6.451 (Bonnor 1956; Ebert 1955)
    assert abs(n.max() / n.min() / 14.04 - 1.0) < 0.01
    assert abs(n.max() / 1.2e4 - 1.0) < 0.01
    # density falls monotonically with radius inside the sphere: the finest
    # level holds the densest cells
    assert n[off[896 * 1]:].mean() > n[off[448]:off[896]].mean() > n[:off[448]].mean()


def test_step_is_half_the_finest_sound_crossing():
    # dx_f / c_s = (6.45 / 128) L_BE / c_s = (6.45 / 128) / sqrt(4 pi G rho_c)
    G, mH = 6.674e-8, 1.6726e-24
    t = 0.5 * (6.45 / 128.0) / np.sqrt(4 * np.pi * G * 1.4 * mH * 1.2e4)
    assert abs(inputs.be_dt() / t - 1.0) < 1e-12
    assert 4e3 < inputs.be_dt() / inputs.YR < 7e3
