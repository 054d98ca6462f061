"""Pins of the oracle's heating/cooling rows (Table 4), of rates of Table 3
and of its substep controller (Sec. 2.2.8) against physics that does not come
from the paper's formulas: energies, coefficients and equilibrium constants
derived from physical constants (tests/golden/physical_constants.txt),
independent published fits, and closed forms of the LI update.

Each test names the oracle function it pins and the mistake it would catch.
No GPU is needed.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def golden_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line and line.split()[0][0].isdigit():
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


C = golden("physical_constants.txt")
HBAR = C["h"] / (2 * np.pi)
EV, KB = C["eV"], C["k_B"]
# ionization energy of H(1s): the Rydberg energy m_e c^2 alpha^2 / 2 with the
# reduced-mass correction
RY_INF = C["m_e"] * C["c"] ** 2 * C["alpha_fs"] ** 2 / 2.0
CHI_H = RY_INF / (1.0 + C["m_e"] / C["m_p"])
D0_H2 = C["D0_H2_cm"] * C["h"] * C["c"]                  # erg
T_CMB_READING = 2.725                                    # reading (z = 0)
Y_HE = 0.0833                                            # reading: He per H nucleus


def gas_rate(pmask, T, n=1.0, y2=0.0, ye=0.1, Td=20.0, G0=0.0, nE=0.0, NH2=0.0, rmask=0xFFF):
    """Volumetric Gamma - Lambda [erg cm^-3 s^-1] of the oracle with only the
    processes in pmask switched on (the aux[4] output of oracle.system)."""
    cfg = oracle.default_config(process_mask=pmask, reaction_mask=rmask)
    u = np.array([y2, ye, T, Td, 1e4 * C["a_rad"] * Td ** 4])
    return oracle.system(n, u, G0, nE, NH2, 1.0, 1.0, cfg)[5][4]


# ------------------------------------------------------------- energies per event
def test_reading_of_T_CMB_is_the_measured_value():
    assert abs(T_CMB_READING / C["T_CMB"] - 1.0) < 1e-3


def test_L5_ionization_cooling_removes_the_ionization_energy_of_H():
    """Lambda_5 = 13.6 eV k_H0 n(H) n(e) (Table 4): each collisional
    ionization costs the ionization energy of H(1s), the reduced-mass
    Rydberg energy from CODATA constants.  Catches a wrong energy (13.6 -> 1.36)."""
    for T in (2e4, 5e4, 1e5):
        n, ye = 10.0, 0.2
        yH = 1.0 - ye
        L5 = -gas_rate(oracle.P_L5_HION, T, n, 0.0, ye)
        k0 = oracle.rates(T, 20.0, n)[0]
        per_event = L5 / (k0 * n * n * yH * ye)
        assert per_event == pytest.approx(CHI_H, rel=1e-3, abs=0), (T, per_event / EV)


def test_L6_and_G1_formation_heat_obey_the_H2_binding_energy():
    """Lambda_6 = 4.48 eV [k_H4 n(H2) n(H) + k_H7 n(H2)^2]: each collisional
    dissociation costs D_0(H2).  Gamma_1: at densities far above n_cr (f = 1)
    the H- channel (H- + H -> H2 + e) releases D_0 - EA(H) and three-body
    formation releases D_0; formation on grains deposits at most D_0 (energy
    conservation) and, at f = 1, nearly all of it."""
    T, n = 1000.0, 1e3
    y2, ye = 0.2, 1e-3
    yH = 1.0 - 2 * y2 - ye
    k = oracle.rates(T, 20.0, n)
    L6 = -gas_rate(oracle.P_L6_H2DISS, T, n, y2, ye)
    assert L6 / (n * n * (k[4] * y2 * yH + k[7] * y2 * y2)) == pytest.approx(D0_H2, rel=1e-3, abs=0)
    # Gamma_1 at f -> 1 (n >> n_cr ~ 1e4 cm^-3 here), one channel at a time
    nn = 1e14
    y2, ye = 0.0, 1e-4
    yH = 1.0 - ye
    k = oracle.rates(T, 20.0, nn)
    g_hm = gas_rate(oracle.P_G1_H2FORM, T, nn, y2, ye, rmask=(1 << 2) | (1 << 3))
    assert g_hm / (k[2] * nn * nn * yH * ye) == pytest.approx(D0_H2 - C["EA_H_eV"] * EV, rel=3e-3, abs=0)
    g_3b = gas_rate(oracle.P_G1_H2FORM, T, nn, y2, ye, rmask=1 << 5)
    assert g_3b / (k[5] * nn ** 3 * yH ** 3) == pytest.approx(D0_H2, rel=1e-3, abs=0)
    g_gr = gas_rate(oracle.P_G1_H2FORM, T, nn, y2, ye, rmask=1 << 8)
    per = g_gr / (k[8] * nn * nn * yH)
    assert 0.97 * D0_H2 < per <= D0_H2


# ----------------------------------------------------------- recombination, excitation
def test_L7_matches_the_hui_gnedin_case_b_cooling_fit():
    """Lambda_7 (Table 4, a polynomial in log10 T) against the independent case-B
    recombination-cooling fit of Hui & Gnedin (1997), 3e3-1e6 K, 2 per cent
    (golden).  Catches a wrong coefficient (-25.87 -> -25.57 doubles it)."""
    g = golden("hui_gnedin_1997.txt")
    for T in (3e3, 5e3, 1e4, 2e4, 5e4, 1e5, 3e5, 1e6):
        ye = 0.5
        L7 = -gas_rate(oracle.P_L7_HREC, T, 1.0, 0.0, ye) / (ye * ye)
        lam = 2.0 * g["T_HI"] / T
        fit = g["A"] * T * lam ** g["p1"] / (1.0 + (lam / g["l0"]) ** g["p2"]) ** g["p3"]
        assert abs(L7 / fit - 1.0) < g["tol"], (T, L7, fit)


def _boltzmann_energy(pbit, T, **kw):
    """-k_B d ln Lambda / d(1/T) at T (central difference in 1/T)."""
    h = 1e-4
    up, dn = T / (1 - h), T / (1 + h)
    Lp, Lm = -gas_rate(pbit, up, **kw), -gas_rate(pbit, dn, **kw)
    return -KB * (np.log(Lp) - np.log(Lm)) / (1.0 / up - 1.0 / dn)


def test_L9_excitation_energy_and_collision_strength():
    """Lambda_9 (H excitation, Cen 1992): its Boltzmann factor is the Ly-alpha
    excitation energy 3/4 chi_H (slope of ln Lambda in 1/T at low T), and the
    effective collision strength it implies,
    Upsilon = Lambda / (n_e n_H E q0 g^-1 T^-1/2 e^{-E/kT}) with
    q0 = hbar^2 (2 pi / (k m_e^3))^{1/2} and g = 2, lies within a factor 2
    of the published e + H(1s) -> n = 2 values (golden).  Catches a prefactor
    off by an order of magnitude and a wrong exponent."""
    E = 0.75 * CHI_H
    assert _boltzmann_energy(oracle.P_L9_HEXC, 3000.0, ye=1e-3) == pytest.approx(E, rel=5e-3, abs=0)
    q0 = HBAR ** 2 * np.sqrt(2 * np.pi / (KB * C["m_e"] ** 3))
    tab = golden_rows("h_collision_strength.txt")
    fac = golden("h_collision_strength.txt")["factor"]
    for T, ups_ref in tab:
        ye = 1e-3
        L9 = -gas_rate(oracle.P_L9_HEXC, T, 1.0, 0.0, ye) / (ye * (1.0 - ye))
        ups = L9 * 2.0 * np.sqrt(T) / (q0 * E * np.exp(-E / (KB * T)))
        assert ups_ref / fac < ups < ups_ref * fac, (T, ups)


def test_L10_excitation_energy_is_the_HeII_lyman_alpha():
    """Lambda_10 (He+ excitation): Boltzmann factor at the He+ Ly-alpha energy,
    Z^2 x 3/4 of the He+ Rydberg (Z = 2), up to the slope of its T^-0.397
    prefactor (0.397 T, 0.3 per cent at 3000 K)."""
    E = 4 * 0.75 * RY_INF / (1.0 + C["m_e"] / C["m_He"])
    got = _boltzmann_energy(oracle.P_L10_HEPEXC, 3000.0, ye=0.5)
    assert got == pytest.approx(E, rel=5e-3, abs=0)


def test_L11_free_free_is_the_bremsstrahlung_of_a_maxwellian_plasma():
    """Lambda_11 = 1.426e-27 T^1/2 g_ff n(H+) n(e): the classical
    thermal-bremsstrahlung emissivity of a Z = 1 plasma,
    2^5 pi e^6 / (3 h m_e c^3) (2 pi k / (3 m_e))^{1/2} T^1/2 g_B
    (Rybicki & Lightman 1979, Eq. 5.14b), computed here from constants, with
    the frequency-averaged Gaunt factor g_B between 1.1 and 1.5 (ibid.)."""
    coef = (2 ** 5 * np.pi * C["e_esu"] ** 6 / (3 * C["h"] * C["m_e"] * C["c"] ** 3)
            * np.sqrt(2 * np.pi * KB / (3 * C["m_e"])))
    for T in (3e3, 1e4, 1e5, 1e6, 1e7):
        ye = 0.5
        L11 = -gas_rate(oracle.P_L11_FF, T, 1.0, 0.0, ye) / (ye * ye)
        g_B = L11 / (coef * np.sqrt(T))
        assert 1.1 <= g_B <= 1.5, (T, g_B)
    # the two branches of the printed g_ff meet at 3.2e5 K to 2.1 per cent
    # (a sign or coefficient slip in either branch would open a wide gap)
    lo = -gas_rate(oracle.P_L11_FF, 3.2e5 * (1 - 1e-9), 1.0, 0.0, 0.5)
    hi = -gas_rate(oracle.P_L11_FF, 3.2e5 * (1 + 1e-9), 1.0, 0.0, 0.5)
    assert abs(lo / hi - 1.0) < 0.03


def test_L12_compton_coefficient_from_thomson_scattering():
    """Lambda_12 = 1.017e-37 T_CMB^4 (T - T_CMB) n(e): the Compton energy
    exchange 4 sigma_T a k_B / (m_e c) T_CMB^4 (T - T_CMB) n_e, from constants."""
    coef = 4 * C["sigma_T"] * C["a_rad"] * KB / (C["m_e"] * C["c"])
    for T in (10.0, 1e3, 1e5):
        ye = 0.3
        L12 = -gas_rate(oracle.P_L12_COMPTON, T, 2.0, 0.0, ye)
        assert L12 == pytest.approx(coef * T_CMB_READING ** 4 * (T - T_CMB_READING) * 2.0 * ye, rel=2e-3, abs=0)


# ---------------------------------------------------------------------- rates
def test_k_H3_is_of_the_order_of_the_langevin_capture_rate():
    """k_H3 (associative detachment H- + H, Kreckel et al. 2010 fit) against the
    ion - induced-dipole (Langevin) capture rate 2 pi e (alpha_pol / mu)^{1/2}
    with the exact polarizability of H(1s), 4.5 a_0^3: within a factor 2 over
    10-3000 K.  Catches a coefficient off by an order of magnitude."""
    a0 = HBAR ** 2 / (C["m_e"] * C["e_esu"] ** 2)
    mu = C["m_Hatom"] / 2.0
    kL = 2 * np.pi * C["e_esu"] * np.sqrt(C["alpha_pol_H"] * a0 ** 3 / mu)
    for T in (10.0, 30.0, 100.0, 300.0, 1000.0, 3000.0):
        k3 = oracle.rates(T, 20.0, 1.0)[3]
        assert 0.5 < k3 / kL < 2.0, (T, k3, kL)


def _K_eq_H2(T):
    """n(H)^2 / n(H2) in chemical equilibrium (statistical mechanics): the
    translational factor of the reduced mass m_H / 2, the internal partition
    functions (H: electron x nuclear spin = 4 states; H2: rigid rotor with
    ortho/para nuclear-spin weights 3/1 and a harmonic vibration at the
    fundamental), and the binding energy D_0."""
    J = np.arange(0, 80)
    th_r = C["B_H2_cm"] * C["h"] * C["c"] / KB
    th_v = C["we_H2_cm"] * C["h"] * C["c"] / KB
    Q_rot = np.sum(np.where(J % 2 == 0, 1.0, 3.0) * (2 * J + 1) * np.exp(-th_r * J * (J + 1) / T))
    Q_vib = 1.0 / (1.0 - np.exp(-th_v / T))
    trans = (2 * np.pi * (C["m_Hatom"] / 2) * KB * T / C["h"] ** 2) ** 1.5
    return trans * 16.0 / (Q_rot * Q_vib) * np.exp(-D0_H2 / (KB * T))


def test_k_H7_and_k_H6_obey_detailed_balance_at_high_density():
    """H7 (2 H2 -> 2 H + H2) and H6 (2 H + H2 -> 2 H2) are a forward/reverse
    pair.  Where n >> n_cr the level populations are thermal and
    k_H7 / k_H6 must approach the equilibrium constant n(H)^2 / n(H2) of
    statistical mechanics (D_0, the H2 rotational and vibrational constants).
    The published fits (Table 3) meet it within a factor 3 at 1000-3000 K.
    Catches a factor 10 in k_H5 (hence k_H6 = k_H5 / 8) or in k_high."""
    for T in (1000.0, 1500.0, 2000.0, 3000.0):
        k = oracle.rates(T, 20.0, 1e20)
        r = (k[7] / k[6]) / _K_eq_H2(T)
        assert 1.0 / 3.0 < r < 3.0, (T, r)
    # the ratio H6 / H5 is the printed 1/8 at every temperature
    for T in (10.0, 1e3, 1e4):
        k = oracle.rates(T, 20.0, 1.0)
        assert k[6] == pytest.approx(k[5] / 8.0, rel=1e-15, abs=0)


def test_k_H7_does_not_fall_with_density():
    """H7 interpolates between a low-density limit (upper vibrational levels
    drained below their thermal populations) and the high-density limit
    (thermal populations).  Depleted upper levels cannot dissociate faster
    than thermal ones, so at fixed T the rate coefficient must not fall as the
    density rises: k_low <= k_high, up to 2e4 K, where H2 is already
    collisionally destroyed (the printed fits give k_low / k_high = 0.33
    there).  Catches a low-density coefficient too large by a factor >~ 3."""
    for T in (1e3, 3e3, 5e3, 1e4, 1.5e4, 2e4):
        ks = [oracle.rates(T, 20.0, n)[7] for n in (1e-6, 1e0, 1e3, 1e6, 1e12)]
        assert all(b >= a * (1 - 1e-12) for a, b in zip(ks, ks[1:])), (T, ks)


# ------------------------------------------------------- gas-grain transfer
def test_gas_grain_term_equals_table_4_lambda_cool():
    """The gas-grain transfer of the gas energy equation (App. C, Eq.
    ap_eq:Tg, with R_g, T_high and T_low of App. C), times rho, equals the
    separately printed Table 4 row Lambda_COOL = 5.83e-8 n_H rho
    (T_g / 1e3)^{1/2} [1 - 0.8 exp(-75 / T_g)] (T_g - T_d) (Z / Z_sun), on both
    sides of T_low and at Z != Z_sun; the dust equation (Eq. ap_eq:dust_temp)
    carries the same coupling without f_d.  Catches a wrong R_g, T_high or
    T_low in either equation."""
    for Z in (1.0, 0.01):
        cfg = oracle.default_config(process_mask=oracle.P_GASGRAIN, reaction_mask=0)
        cfg.Z = Z
        for T, Td, n in ((30.0, 12.0, 1e4), (300.0, 20.0, 1e5), (3000.0, 40.0, 1e2), (50.0, 80.0, 1e6)):
            u = np.array([0.3, 1e-6, T, Td, 1e4 * C["a_rad"] * Td ** 4])
            A, b, F, M, ts, aux = oracle.system(n, u, 0.0, 0.0, 0.0, 1.0, 1.0, cfg)
            rho = aux[0]
            lam_cool = 5.83e-8 * n * rho * (T / 1e3) ** 0.5 * (1 - 0.8 * np.exp(-75.0 / T)) * (T - Td) * Z
            assert aux[4] == pytest.approx(-lam_cool, rel=1e-12, abs=0), (Z, T, Td)
            # dust row: C_d dT_d/dt = -R_g n sqrt(T/T_high) gamma_d (T_d - T_g)
            assert F[3] == pytest.approx(lam_cool / (rho * Z), rel=1e-12, abs=0)


# ------------------------------------------------------- substep controller
def test_energy_timescale_and_LI_update_on_compton_cooling():
    """Compton cooling alone (chemistry, T_d and E_IR frozen) makes the gas row
    linear in T_g: dT/dt = -lambda (T - T_CMB) with
    lambda = c_C T_CMB^4 n_e (gamma - 1) / (k_B n_tot)  (alpha_g of Eq.
    ap_eq:alpha_g times rho is k_B n_tot / (gamma - 1)).  Then
    (1) each substep is dt_s = f_chem P / ((gamma - 1) |Gamma - Lambda|)
        (Eqs. timescale_energy, timestep_subcycle), which with the Compton
        coefficient c_C from Thomson scattering is
        f_chem n_tot k_B T / ((gamma - 1) c_C T_CMB^4 (T - T_CMB) n_e);
    (2) each LI update is exactly T' - T_CMB = (T - T_CMB) / (1 + lambda dt_s),
        and lambda dt_s = f_chem T / (T - T_CMB) whatever gamma and c_C are.
    Catches a dropped (gamma - 1) in dt_energy or alpha_g, a wrong pressure,
    and a wrong Compton coefficient."""
    cC = 4 * C["sigma_T"] * C["a_rad"] * KB / (C["m_e"] * C["c"])
    fl = oracle.F_FREEZE_YH2 | oracle.F_FREEZE_YE | oracle.F_FREEZE_TD | oracle.F_FREEZE_EIR
    for gamma, (n, T0, y2, ye) in ((5.0 / 3.0, (1.0, 1e4, 0.1, 0.5)), (1.4, (30.0, 300.0, 0.45, 1e-3))):
        cfg = oracle.default_config(process_mask=oracle.P_L12_COMPTON, reaction_mask=0, flags=fl)
        cfg.gamma_ad = gamma
        cell = dict(n_H=n, T_g=T0, T_d=15.0, E_IR=1e4 * C["a_rad"] * 15.0 ** 4, y_H2=y2, y_e=ye,
                    G0=0.0, n_EUV=0.0, N_H2=0.0)
        lam_tcool = cC * T_CMB_READING ** 4 * n * ye * (gamma - 1.0) / (KB * n * (1 - y2 + ye + Y_HE))
        t_end = 40.0 / lam_tcool
        rec, st = oracle.li_trace(cell, t_end, 1.0, cfg)
        assert st == 0 and 50 < len(rec) < 5000
        n_tot = n * (1.0 - y2 + ye + Y_HE)
        T = T0
        for t, dts, *u in rec:
            Tn = u[2]
            if t < t_end:
                expect = 0.03 * n_tot * KB * T / ((gamma - 1.0) * cC * T_CMB_READING ** 4 * (T - T_CMB_READING) * n * ye)
                assert dts == pytest.approx(expect, rel=2e-3, abs=0), (gamma, t, dts, expect)
                x = 0.03 * T / (T - T_CMB_READING)
                assert Tn - T_CMB_READING == pytest.approx((T - T_CMB_READING) / (1.0 + x), rel=1e-12, abs=0)
            T = Tn


def test_n_cyc_switch_at_300_estimated_subcycles():
    """Mode choice (Sec. 2.2.8): with N_req = dt_hydro / (f_chem dt_dust)
    below N_cyc = 300 the cell subcycles on the dust timescale; at or above it
    the dust timescale is dropped (tight coupling).  Dust cooling by emission
    alone: dt_dust = C_d T_d / |kappa a c T_d^4 - E_UV| (Eq.
    timescale_of_dust).  A cell at N_req = 299 subcycles (first substep
    dt_hydro / 299), one at 301 runs in the tight-coupling mode (here one
    substep covers dt_hydro: nothing else limits it).  Catches a wrong N_cyc."""
    cfg = oracle.default_config(process_mask=oracle.P_DUST_EMIT, reaction_mask=0,
                                flags=oracle.F_FREEZE_TG | oracle.F_FREEZE_EIR | oracle.F_FREEZE_YH2
                                | oracle.F_FREEZE_YE)
    Td, n, cd = 40.0, 1e3, 10.0
    cell = dict(n_H=n, T_g=50.0, T_d=Td, E_IR=1e4 * C["a_rad"] * Td ** 4, y_H2=0.3, y_e=1e-6,
                G0=0.0, n_EUV=0.0, N_H2=0.0)
    u = np.array([cell[k] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
    ts = oracle.system(n, u, 0.0, 0.0, 0.0, 1.0, cd, cfg)[4]
    dt_dust = ts[0]
    assert np.isinf(ts[1]) and np.isinf(ts[2])
    for N_req, tight in ((299.0, False), (301.0, True)):
        dt_h = N_req * 0.03 * dt_dust
        rec, st = oracle.li_trace(cell, dt_h, cd, cfg)
        assert bool(st & oracle.ST_TIGHT) == tight, (N_req, st)
        if tight:
            assert len(rec) == 1 and rec[0][1] == dt_h
        else:
            assert rec[0][1] == pytest.approx(dt_h / N_req, rel=1e-13, abs=0)


def test_cosmic_ray_ionization_balanced_by_recombination():
    """Table 3 H11 and H1 in R_e (Eq. eq_chemq): with only cosmic-ray
    ionization and radiative recombination, y_e relaxes to the root of
    k_H11 y_H = k_H1 n_H y_e^2 with y_H = 1 - 2 y_H2 - y_e (y_H2 held), from
    above and from below.  Catches an ionization or recombination term
    missing from the electron row, or one with the wrong abundance."""
    import inputs
    cfg = oracle.default_config(reaction_mask=(1 << 11) | (1 << 1),
                                flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YH2)
    n, y2 = 1e4, 0.2
    k = oracle.rates(100.0, 20.0, n, cfg=cfg)
    a, b, c0 = k[1] * n, k[11], -k[11] * (1.0 - 2.0 * y2)
    ye_eq = (-b + np.sqrt(b * b - 4.0 * a * c0)) / (2.0 * a)
    for ye0 in (1e-4, 1e-6):
        cell = dict(n_H=n, T_g=100.0, T_d=20.0, E_IR=1e4 * C["a_rad"] * 20.0 ** 4, y_H2=y2, y_e=ye0,
                    G0=0.0, n_EUV=0.0, N_H2=0.0)
        o = oracle.li_step({kk: np.array([v]) for kk, v in cell.items()}, 1e6 * inputs.YR, 1.0, cfg)
        assert float(o["y_e"][0]) == pytest.approx(ye_eq, rel=1e-4, abs=0), ye0


def test_three_body_formation_against_the_analytic_solution():
    """Table 3 H5 in R_H2 (Eq. eq_chemq): three-body formation alone,
    3H -> H2 + H at k_H5 n(H)^3 per volume, gives dy_H/dt = -2 k_H5 n_H^2
    y_H^3, solved by 1/y_H^2 = 1/y_H0^2 + 4 k_H5 n_H^2 t.  The LI step, first
    order in f_chem, approaches it: within 2e-3 at f_chem = 3e-3 (measured
    6.4e-4), with the error falling about tenfold from f_chem = 3e-2.  k_H5
    is the printed fit, evaluated here; the powers of n_H and y_H are what
    is pinned."""
    import inputs
    n, T, t = 1e11, 1000.0, 100.0 * inputs.YR
    k5 = 6e-32 * T ** -0.25 + 2e-31 * T ** -0.5
    yH_exact = 1.0 / np.sqrt(1.0 + 4.0 * k5 * n * n * t)
    cell = dict(n_H=n, T_g=T, T_d=T, E_IR=1e4 * C["a_rad"] * T ** 4, y_H2=0.0, y_e=0.0,
                G0=0.0, n_EUV=0.0, N_H2=0.0)
    err = {}
    for fc in (3e-2, 3e-3):
        cfg = oracle.default_config(reaction_mask=1 << 5, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YE,
                                    f_chem=fc)
        o = oracle.li_step({kk: np.array([v]) for kk, v in cell.items()}, t, 1.0, cfg)
        err[fc] = abs(float(o["y_H"][0]) / yH_exact - 1.0)
    assert err[3e-3] < 2e-3
    assert 5.0 < err[3e-2] / err[3e-3] < 20.0


def test_mass_density_per_h_nucleus_carries_the_helium_mass():
    """rho = n_H m_H (1 + (m_He/m_H) y_He) (App. C's rho, per H nucleus):
    y_He is read off the oracle's particle count of neutral atomic gas
    (n_tot/n_H - 1 from its pressure P = n_tot k_B T) and the helium mass
    from CODATA (m_He/m_p = 3.97; the oracle's 4 m_H is within 0.2 % in
    rho).  The helium mass fraction that y_He implies lies in the range of
    the primordial and protosolar values, Y = 0.24-0.28.  Catches a wrong
    helium mass or abundance in rho."""
    n, T = 100.0, 100.0
    A, b, F, M, ts, aux = oracle.system(n, np.array([0.0, 0.0, T, 20.0, 1e-3]), 0.0, 0.0, 0.0, 1.0, 1.0)
    rho, P = aux[0], aux[3]
    y_He = P / (n * C["k_B"] * T) - 1.0
    mass_ratio = C["m_He"] / C["m_p"]
    assert rho / (n * C["m_p"]) == pytest.approx(1.0 + mass_ratio * y_He, rel=5e-3, abs=0)
    Y = mass_ratio * y_He / (1.0 + mass_ratio * y_He)
    assert 0.24 <= Y <= 0.28


def _three_body_cell(n, T):
    return dict(n_H=n, T_g=T, T_d=T, E_IR=1e4 * C["a_rad"] * T ** 4, y_H2=0.0, y_e=0.0,
                G0=0.0, n_EUV=0.0, N_H2=0.0)


def test_nr_step_is_the_backward_euler_root():
    """The Newton-Raphson reference of Sec. 2.2.8 solves the backward-Euler
    equations of the step: with three-body formation alone (Table 3 H5;
    temperatures and electrons held), y_H' + 2 dt k_H5 n_H^2 y_H'^3 = y_H0,
    a cubic with one positive root (numpy).  One Newton-Raphson step over
    dt_hydro lands on it to 1e-10 (the 1e-5 stopping test and quadratic
    convergence).  Catches a wrong residual or a wrong dt in it."""
    n, T = 1e11, 1000.0
    k5 = 6e-32 * T ** -0.25 + 2e-31 * T ** -0.5
    cfg = oracle.default_config(reaction_mask=1 << 5, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YE)
    one = {k: np.array([v]) for k, v in _three_body_cell(n, T).items()}
    import inputs
    for dt_yr in (10.0, 100.0, 1000.0):
        dt = dt_yr * inputs.YR
        o = oracle.nr_step(one, dt, 1.0, cfg)
        assert o["n_sub"][0] == 1 and o["status"][0] == 0
        yH = 1.0 - 2.0 * o["y_H2"][0] - o["y_e"][0]
        r = np.roots([2.0 * dt * k5 * n * n, 0.0, 1.0, -1.0])
        r = r[np.abs(r.imag) < 1e-12].real
        root = r[r > 0][0]
        assert yH == pytest.approx(root, rel=1e-10, abs=0), dt_yr


def test_nr_substeps_cover_the_hydro_step():
    """Sec. 2.2.8's substepping of the Newton-Raphson reference: when an
    attempt fails, dt_sub = (dt_hydro - t_sub) / 2^i, and the accepted
    substeps must add up to dt_hydro.  With the iteration limit at 2 the
    100-yr step of three-body formation cannot be taken at once (its one
    backward-Euler step would be 19 % off the analytic y_H): the reference
    subdivides and, being first order in the substep, ends within 1 % of the
    analytic solution 1/y_H^2 = 1 + 4 k_H5 n_H^2 t (measured 0.4 %).  Time
    lost or double-counted between substeps fails it."""
    import inputs
    n, T = 1e11, 1000.0
    k5 = 6e-32 * T ** -0.25 + 2e-31 * T ** -0.5
    dt = 100.0 * inputs.YR
    cfg = oracle.default_config(reaction_mask=1 << 5, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YE,
                                nr_itr_limit=2)
    o = oracle.nr_step({k: np.array([v]) for k, v in _three_body_cell(n, T).items()}, dt, 1.0, cfg)
    assert o["status"][0] == 0 and o["n_sub"][0] > 10
    yH = 1.0 - 2.0 * o["y_H2"][0] - o["y_e"][0]
    assert yH == pytest.approx(1.0 / np.sqrt(1.0 + 4.0 * k5 * n * n * dt), rel=1e-2, abs=0)


def test_line_cooling_stand_in_at_lte():
    """Reading R23 (line cooling, a stand-in for the cited models): two-level
    [C II] 158 um and [O I] 63 um emitters at fixed abundances.  Above their
    critical densities the level populations are Boltzmann, and each line
    cools at x f_d n_H h nu A g e^{-h nu / k T} / (1 + g e^{-h nu / k T}),
    whatever the collision rates.  The oracle's line cooling at n_H = 1e10
    (three decades above either critical density) matches that sum built
    from laboratory wavelengths, NIST A values, statistical weights and
    diffuse-cloud gas-phase abundances (tests/golden/fine_structure_lines.txt)
    within 2 %, at 30, 100 and 1000 K and at Z = Z_sun and 0.1 Z_sun."""
    g = golden("fine_structure_lines.txt")
    h, c, kB = C["h"], C["c"], C["k_B"]
    n = 1e10
    for Z in (1.0, 0.1):
        cfg = oracle.default_config(process_mask=oracle.P_L13_LINE, reaction_mask=0)
        cfg.Z = Z
        for T in (30.0, 100.0, 1000.0):
            u = np.array([0.3, 1e-6, T, 20.0, 1e4 * C["a_rad"] * 20.0 ** 4])
            A, b, F, M, ts, aux = oracle.system(n, u, 0.0, 0.0, 0.0, 1.0, 1.0, cfg)
            lte = 0.0
            for ion in ("CII", "OI"):
                hnu = h * c / (g[f"lambda_{ion}_um"] * 1e-4)
                e = g[f"g_{ion}"] * np.exp(-hnu / (kB * T))
                lte += g[f"x_{ion}"] * Z * n * hnu * g[f"A_{ion}"] * e / (1.0 + e)
            assert -aux[4] == pytest.approx(lte, rel=2e-2, abs=0), (Z, T, -aux[4] / lte)


def test_k_H9_cross_section_is_the_hydrogenic_threshold_value():
    """Reading R19 (stand-in for the cited photoionization rate): k_H9 =
    c sigma n_EUV with sigma the photoionization cross-section of H(1s) at
    threshold, which for a hydrogenic ground state is
    sigma_0 = (2^9 pi^2 / (3 e^4)) alpha a_0^2 = 6.30e-18 cm^2 (e = exp(1);
    Bethe & Salpeter's closed form, CODATA alpha and a_0), to the 3 digits the
    stand-in carries.  Catches a wrong cross-section or a missing c."""
    sigma0 = 2.0 ** 9 * np.pi ** 2 / (3.0 * np.e ** 4) * C["alpha_fs"] * C["a0_cm"] ** 2
    for n_euv in (1e-3, 1.0):
        k9 = oracle.rates(1e4, 20.0, 1.0, 0.0, n_euv, 0.0)[9]
        assert k9 / (C["c"] * n_euv) == pytest.approx(sigma0, rel=1e-3, abs=0)
