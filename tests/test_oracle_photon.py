"""Pins of the oracle's photon consumption after the update (reading of Sec.
2.2.8, "Radiation components"; oracle_photon_update): photon-number
conservation, its limits, and consistency with the chemistry and dust rows
it follows -- in an optically thin step the photons absorbed by H are the
ions the LI step made (photoionization only), those absorbed by H2 the
molecules it dissociated (photodissociation only), and the photons absorbed
by dust carry the UV energy the dust row of Appendix C received."""
import numpy as np
import pytest

import inputs
import oracle

YR = inputs.YR
A_RAD = 7.565733250e-15
EV = 1.602176634e-12
HNU_EUV = 18.0 * EV        # the stand-in mean EUV photon energy of the dust UV term


def _cells(n=512, seed=3):
    c = inputs.cells_uniform(n, seed=seed)
    return c


def test_photon_number_is_conserved():
    c = _cells()
    for dt in (1.0, 1e3 * YR, 1e6 * YR):
        r = oracle.photon_update(c, dt)
        ab = r["absorbed"]
        assert np.all(r["n_EUV"] >= 0) and np.all(r["G0"] >= 0) and np.all(ab >= 0)
        np.testing.assert_allclose(r["n_EUV"] + ab[:, 0] + ab[:, 1], c["n_EUV"], rtol=1e-13)
        nF_in = c["G0"] * oracle.U_HABING / oracle.HNU_FUV
        nF_out = r["G0"] * oracle.U_HABING / oracle.HNU_FUV
        np.testing.assert_allclose(nF_out + ab[:, 2] + ab[:, 3], nF_in, rtol=1e-13)


def test_limits():
    c = _cells(64)
    r = oracle.photon_update(c, 0.0)
    assert np.array_equal(r["n_EUV"], c["n_EUV"]) and np.array_equal(r["G0"], c["G0"])
    r = oracle.photon_update(c, 1e30)                        # opaque: everything absorbed
    assert np.all(r["n_EUV"] < 1e-15 * c["n_EUV"]) and np.all(r["G0"] < 1e-15 * c["G0"])
    # fully molecular gas: no EUV photon goes to H
    c2 = dict(c)
    c2["y_e"] = np.zeros(64)
    c2["y_H2"] = np.full(64, 0.5)
    r = oracle.photon_update(c2, 1e3 * YR)
    assert np.all(r["absorbed"][:, 0] == 0.0) and np.all(r["absorbed"][:, 1] > 0.0)


def _thin_cell(**kw):
    c = dict(n_H=1.0, T_g=1e4, T_d=20.0, y_H2=0.2, y_e=0.01, G0=1.0, n_EUV=1e-3, N_H2=1e14)
    c.update(kw)
    c["E_IR"] = 1e4 * A_RAD * c["T_d"] ** 4
    return c


def test_photons_absorbed_by_H_are_the_ions_the_chemistry_made():
    """Only photoionization (H9) in the LI step, temperatures and H2 frozen,
    a short step (lam dt ~ 1e-4): the EUV photons the update absorbs by H
    (with the updated y_H) equal n_H dy_e of the chemistry to first order in
    lam dt -- the same cross-section enters k_H9 and the photon update."""
    cell = _thin_cell()
    dt = 1.0e3
    cfg = oracle.default_config(reaction_mask=1 << 9, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YH2)
    one = {k: np.array([v]) for k, v in cell.items()}
    o = oracle.li_step(one, dt, 1.0, cfg)
    ions = cell["n_H"] * (o["y_e"][0] - cell["y_e"])
    upd = dict(one, y_H2=o["y_H2"], y_e=o["y_e"])
    r = oracle.photon_update(upd, dt)
    absorbed_H = r["absorbed"][0, 0]
    lam_dt = 1.0 - r["n_EUV"][0] / cell["n_EUV"]
    assert 1e-6 < lam_dt < 1e-3
    assert absorbed_H == pytest.approx(ions, rel=5 * lam_dt + 1e-9, abs=0)


def test_photons_absorbed_by_H2_are_the_molecules_the_chemistry_dissociated():
    """Only photodissociation (H10), T and electrons frozen, a short step: the
    FUV photons the update absorbs by H2 equal n_H (y_H2 - y_H2') to first
    order in lam dt (one photon per photodissociation)."""
    cell = _thin_cell(G0=3.0, N_H2=1e15)
    dt = 1.0e6
    cfg = oracle.default_config(reaction_mask=1 << 10, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YE)
    one = {k: np.array([v]) for k, v in cell.items()}
    o = oracle.li_step(one, dt, 1.0, cfg)
    dissociated = cell["n_H"] * (cell["y_H2"] - o["y_H2"][0])
    upd = dict(one, y_H2=o["y_H2"], y_e=o["y_e"])
    r = oracle.photon_update(upd, dt)
    lam_dt = 1.0 - r["G0"][0] / cell["G0"]
    assert 1e-7 < lam_dt < 1e-2
    assert r["absorbed"][0, 2] == pytest.approx(dissociated, rel=5 * lam_dt + 1e-6, abs=0)


def test_photons_absorbed_by_dust_carry_the_dust_row_uv_energy():
    """The dust row of Appendix C receives E_UV per unit gas mass (oracle
    aux[2]); in a thin step the photons the update absorbs by dust, times
    their mean energies (18 eV EUV, h nu_F FUV), carry rho E_UV dt."""
    cell = _thin_cell(y_e=1.0 - 1e-12, y_H2=0.0, G0=10.0, n_EUV=1e-4)   # ionized: EUV goes to dust only
    dt = 1.0e6
    u = np.array([cell[k] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
    aux = oracle.system(cell["n_H"], u, cell["G0"], cell["n_EUV"], cell["N_H2"], 1.0, 1.0)[5]
    rho, EUV = aux[0], aux[2]
    r = oracle.photon_update({k: np.array([v]) for k, v in cell.items()}, dt)
    energy = r["absorbed"][0, 1] * HNU_EUV + r["absorbed"][0, 3] * oracle.HNU_FUV
    lam_dt = 1.0 - r["G0"][0] / cell["G0"]
    assert energy == pytest.approx(rho * EUV * dt, rel=5 * lam_dt + 1e-9, abs=0)


def test_each_band_decays_implicitly_at_its_thin_limit_rate():
    """Reading R32: over a step each band keeps n / (1 + lam dt) of its
    photons (the implicit update of dn/dt = -lam n), on both sides of
    lam dt = 1 (the thin and opaque formulas).  lam is measured from the
    oracle itself in the thin limit (photons removed / (n dt), per cell at
    lam dt ~ 1e-7, where the form of the update changes it by ~1e-7), so the
    pin fixes the form of the update, not its stand-in constants: an
    explicit thin-side update (n (1 - lam dt)) or a mismatch between the two
    branches fails it."""
    c = _cells(64, seed=5)

    def thin_rate(key):
        dt = np.full(len(c["n_H"]), 1e-3)
        for _ in range(2):           # a rough rate, then dt = 1e-7 / rate per cell
            r = oracle.photon_update(c, dt)
            lam = (c[key] - r[key]) / (c[key] * dt)
            dt = 1e-7 / lam
        return lam

    lam_E, lam_F = thin_rate("n_EUV"), thin_rate("G0")
    assert np.all(lam_E > 0) and np.all(lam_F > 0)
    for x in (0.3, 0.999, 1.001, 4.0):
        rE = oracle.photon_update(c, x / lam_E)
        np.testing.assert_allclose(rE["n_EUV"], c["n_EUV"] / (1.0 + x), rtol=1e-6)
        rF = oracle.photon_update(c, x / lam_F)
        np.testing.assert_allclose(rF["G0"], c["G0"] / (1.0 + x), rtol=1e-6)
