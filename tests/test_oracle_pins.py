"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test states which part of the oracle it pins and what it is pinned to
(a value the paper prints, a textbook value, a closed form, an invariant, a
library routine, or brute-force convergence).  No GPU is needed.
"""
import os

import numpy as np
import pytest

import inputs
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
YR = inputs.YR


def golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            out[parts[0]] = float(parts[1])
    return out


def golden_table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def one_cell(**kw):
    c = dict(n_H=1.0, T_g=100.0, T_d=20.0, y_H2=0.1, y_e=1e-4, G0=1.0, n_EUV=0.0, N_H2=1e14)
    c.update(kw)
    if "E_IR" not in c:
        c["E_IR"] = 1e4 * 7.565733250e-15 * c["T_d"] ** 4
    return c


# ----------------------------------------------------------- rate coefficients
def test_k_H1_matches_case_B_textbook():
    """k_H1 (Table 3, H1) against the textbook case-B coefficient (golden)."""
    tab = golden_table("case_b_recombination.txt")
    for T, alpha in tab:
        k = oracle.rates(T, 20.0, 1.0)
        assert abs(k[1] / alpha - 1.0) < 0.01, (T, k[1], alpha)


def test_k_H0_matches_cen_fit_near_threshold():
    """k_H0 (Table 3, H0; Abel et al. 1997 fit) against the independent Cen (1992)
    collisional-ionization fit 5.85e-11 T^0.5 exp(-157809/T) / (1 + (T/1e5)^0.5),
    where the two published fits agree (1.5e4-2e4 K)."""
    for T in (1.5e4, 1.75e4, 2e4):
        k = oracle.rates(T, 20.0, 1.0)[0]
        cen = 5.85e-11 * T ** 0.5 * np.exp(-157809.1 / T) / (1.0 + (T / 1e5) ** 0.5)
        assert abs(k / cen - 1.0) < 0.08, (T, k, cen)
    # and it vanishes at molecular-cloud temperatures
    assert oracle.rates(10.0, 10.0, 1.0)[0] == 0.0


def test_k_H2_matches_abel_fit():
    """k_H2 (Table 3, H2; Galli & Palla 1998) against the independent H- formation
    fit of Abel et al. (1997), 6.77e-15 T_eV^0.8779."""
    for T in (100.0, 300.0, 1000.0, 3000.0):
        k = oracle.rates(T, 20.0, 1.0)[2]
        abel = 6.77e-15 * (T / 11604.5) ** 0.8779
        assert abs(k / abel - 1.0) < 0.06, (T, k, abel)


def test_masks_switch_rates_off():
    cfg = oracle.default_config(reaction_mask=0)
    assert np.all(oracle.rates(1e4, 20.0, 1e3, 1.0, 1.0, 1e15, cfg) == 0.0)
    cfg = oracle.default_config(reaction_mask=1 << 8)
    k = oracle.rates(10.0, 10.0, 1e5, cfg=cfg)
    assert k[8] > 0 and np.count_nonzero(k) == 1


# ------------------------------------------------- Sec. 3.5 case 1 (H2 formation)
def _case_cell(case):
    c = inputs.paper_case(case)
    return {k: float(v[0]) for k, v in c.items()}


def test_case1_discrete_closed_form():
    """P1: with only H8 and frozen temperatures, R_H2 = k8 n (1 - 2 y - y_e) is
    linear, so each LI substep is exactly y' - y_eq = (y - y_eq) / (1 + 2 k8 n dt_s)
    (Eqs. eq_chem2-eq_deq).  The closed-form product over the oracle's own
    substep sequence must match its trajectory; the substep sequence itself must
    follow Eq. timestep_subcycle with dt_chem = y_H2 / R_H2."""
    g = golden("paper_sec3_5_chemistry_tests.txt")
    cell = _case_cell(1)
    cfg = oracle.default_config(reaction_mask=1 << 8, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YE)
    rec, st = oracle.li_trace(cell, 2e5 * YR, 1.0, cfg)
    assert st == 0 and len(rec) > 10
    k8 = oracle.rates(g["case1_T_g"], g["case1_T_d"], g["case1_n_H"], cfg=cfg)[8]
    lam = 2.0 * k8 * g["case1_n_H"]
    yeq = (1.0 - cell["y_e"]) / 2.0
    y = cell["y_H2"]          # closed-form product over the whole sequence
    prev = cell["y_H2"]       # the oracle's own previous value
    for t_end, dts, yH2, ye, Tg, Td, E in rec:
        # controller: dt_s = f_chem * y / R (except the truncated last substep)
        R = k8 * g["case1_n_H"] * (1.0 - 2.0 * prev - cell["y_e"])
        if t_end < 2e5 * YR:
            assert dts == pytest.approx(0.03 * prev / R, rel=1e-13, abs=0)
        # the same update written as an increment, (y_eq - y) x / (1 + x): the
        # form y_eq + (y - y_eq) / (1 + x) cancels from ~0.5 down to y ~ 1e-5
        # and would carry 5e-12 of its own rounding
        x = lam * dts
        assert yH2 == pytest.approx(prev + (yeq - prev) * (x / (1.0 + x)), rel=1e-14, abs=0)
        y = y + (yeq - y) * (x / (1.0 + x))
        assert yH2 == pytest.approx(y, rel=1e-11, abs=0)
        assert ye == cell["y_e"] and Tg == cell["T_g"] and Td == cell["T_d"]
        prev = yH2


def _rel_err_vs_analytic_case1(f_chem, t_max):
    g = golden("paper_sec3_5_chemistry_tests.txt")
    cell = _case_cell(1)
    # the paper evolves the network with every other variable fixed
    cfg = oracle.default_config(f_chem=f_chem, flags=oracle.F_FREEZE_THERMAL)
    rec, st = oracle.li_trace(cell, t_max, 1.0, cfg)
    k8 = oracle.rates(g["case1_T_g"], g["case1_T_d"], g["case1_n_H"])[8]
    t = rec[:, 0]
    exact = 0.5 + (g["case1_y_H2"] - 0.5) * np.exp(-2.0 * k8 * g["case1_n_H"] * t)   # Eq. H2form2
    return t, rec[:, 2], np.abs(rec[:, 2] / exact - 1.0)


def test_case1_against_analytic_solution():
    """P1 (paper): relative error of y_H2 vs Eq. H2form2 is below 1e-3 for
    t >~ 1e5 yr and below 1 per cent shortly after 1e4 yr at f_chem = 0.03; the
    gas is almost fully molecular at t ~ 4e4 yr (Sec. 3.5.1, golden)."""
    g = golden("paper_sec3_5_chemistry_tests.txt")
    t, y, err = _rel_err_vs_analytic_case1(0.03, 3e5 * YR)
    late = t >= g["case1_err_below_1e-3_after_yr"] * YR
    assert late.any() and err[late].max() < 1e-3
    mid = t >= 2.0 * g["case1_err_below_1pc_after_yr"] * YR
    assert err[mid].max() < 1e-2
    i = np.searchsorted(t, g["case1_almost_molecular_yr"] * YR)
    assert 0.4 < y[i] < 0.5
    assert y[np.searchsorted(t, 0.25 * g["case1_almost_molecular_yr"] * YR)] < 0.3
    # smaller f_chem is never worse (Fig. of Sec. 3.5.1: error ordered by f_chem)
    e = [np.interp(2e4 * YR, *_rel_err_vs_analytic_case1(f, 3e4 * YR)[::2]) for f in (0.1, 0.03, 0.01)]
    assert e[0] > e[1] > e[2]


# ---------------------------------------------- Sec. 3.5 case 2 (photoionization)
def _n_euv_for(R_ph):
    # the photoionization stand-in is k_H9 = c sigma_EUV n_EUV
    return R_ph / (2.99792458e10 * 6.3e-18)


def test_case2_discrete_closed_form_and_analytic():
    """P2: only H9 (R_ph = 1.1e-6 s^-1), H2 and temperatures frozen: each LI
    substep is exactly y_e' - y_eq = (y_e - y_eq) / (1 + R dt_s); the result
    tracks Eq. HIIform2 and the gas is fully ionized at ~0.1 yr (golden)."""
    g = golden("paper_sec3_5_chemistry_tests.txt")
    cell = _case_cell(2)
    cell["n_EUV"] = _n_euv_for(g["case2_R_ph"])
    cfg = oracle.default_config(reaction_mask=1 << 9,
                                flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YH2)
    rec, st = oracle.li_trace(cell, 1.0 * YR, 1.0, cfg)
    R = oracle.rates(12000.0, 75.0, 100.0, 0.0, cell["n_EUV"], 0.0, cfg)[9]
    assert R == pytest.approx(g["case2_R_ph"], rel=1e-12, abs=0)
    yeq = 1.0 - 2.0 * cell["y_H2"]
    y = cell["y_e"]
    prev = cell["y_e"]
    for t_end, dts, yH2, ye, *_ in rec:
        x = R * dts            # the update as an increment (see P1)
        assert ye == pytest.approx(prev + (yeq - prev) * (x / (1.0 + x)), rel=1e-14, abs=0)
        y = y + (yeq - y) * (x / (1.0 + x))
        assert ye == pytest.approx(y, rel=1e-11, abs=0)
        prev = ye
    t = rec[:, 0]
    exact = 1.0 + (g["case2_y_Hp"] - 1.0) * np.exp(-R * t)           # Eq. HIIform2
    err = np.abs(rec[:, 3] / exact - 1.0)
    assert err.max() < 0.03                                            # of order f_chem or less
    yi = np.interp(g["case2_fully_ionized_yr"] * YR, t, rec[:, 3])
    assert yi > 0.95
    assert np.interp(0.01 * YR, t, rec[:, 3]) < 0.5
    late = t > 0.3 * YR
    assert err[late].max() < 1e-3


def test_case2_ionization_recombination_equilibrium():
    """P3: photoionization balanced by recombination (H9 + H1 at T_g = 12000 K,
    n_H = 100) drives y_H to alpha_rec n_H / R_ph ~ 2e-5 (Eqs. HIIeq, yelinHII;
    the paper prints 2e-5, golden).  Also the exact root of the balance
    R (1 - 2 y_H2 - y_e) = k_H1 n y_e^2."""
    g = golden("paper_sec3_5_chemistry_tests.txt")
    cell = _case_cell(2)
    cell["n_EUV"] = _n_euv_for(g["case2_R_ph"])
    cfg = oracle.default_config(reaction_mask=(1 << 9) | (1 << 1),
                                flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YH2)
    o = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, 10.0 * YR, 1.0, cfg)
    yH = float(o["y_H"][0])
    assert abs(yH / g["case2_y_H_equilibrium"] - 1.0) < 0.05
    k1 = oracle.rates(12000.0, 75.0, 100.0, cfg=cfg)[1]
    a, b, c0 = k1 * 100.0, g["case2_R_ph"], -g["case2_R_ph"] * (1.0 - 2.0 * cell["y_H2"])
    ye = (-b + np.sqrt(b * b - 4 * a * c0)) / (2 * a)
    # the LI step ends with one linearized step toward the balance, so the
    # neutral fraction agrees with the exact root to a fraction of a per cent
    assert float(o["y_H"][0]) == pytest.approx(1.0 - 2.0 * cell["y_H2"] - ye, rel=5e-3, abs=0)


def test_h2_formation_dissociation_equilibrium():
    """P4: with only H8 and H10, y_H2 relaxes to k8 n (1 - y_e) / (2 k8 n + k10)."""
    cell = one_cell(n_H=300.0, T_g=50.0, T_d=15.0, y_H2=0.2, y_e=1e-4, G0=3.0, N_H2=1e15)
    cfg = oracle.default_config(reaction_mask=(1 << 8) | (1 << 10),
                                flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YE)
    o = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, 1e7 * YR, 1.0, cfg)
    k = oracle.rates(50.0, 15.0, 300.0, 3.0, 0.0, 1e15, cfg)
    yeq = k[8] * 300.0 * (1.0 - 1e-4) / (2.0 * k[8] * 300.0 + k[10])
    assert float(o["y_H2"][0]) == pytest.approx(yeq, rel=1e-10, abs=0)


def test_radiative_balance_dust_temperature():
    """P5: with only UV absorption and thermal emission in Eq. ap_eq:dust_temp,
    T_d relaxes to the radiative balance kappa(T_d) a c T_d^4 = E_UV, i.e.
    T_d^6 = E_UV T0^2 / (kappa0 a c) on the T^2 branch of the opacity."""
    cell = one_cell(n_H=10.0, T_g=50.0, T_d=12.0, G0=30.0)
    cfg = oracle.default_config(reaction_mask=0,
                                process_mask=oracle.P_DUST_UV | oracle.P_DUST_EMIT,
                                flags=oracle.F_FREEZE_TG | oracle.F_FREEZE_EIR)
    st = {k: np.array([v]) for k, v in cell.items()}
    for _ in range(3):   # a backward-Euler step lands C_d dT/dt away from balance
        o = oracle.li_step(st, 1e3 * YR, 1.0, cfg)
        st["T_d"] = o["T_d"]
    u = np.array([cell[k] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
    EUV = oracle.system(10.0, u, 30.0, 0.0, 1e14, 1.0, 1.0, cfg)[5][2]
    Teq = (EUV * 10.0 ** 2 / (0.1 * 7.565733250e-15 * 2.99792458e10)) ** (1.0 / 6.0)
    assert Teq < 200.0
    assert float(o["T_d"][0]) == pytest.approx(Teq, rel=1e-10, abs=0)


def test_conservation_and_bounds():
    """P6: H-nuclei conservation y_H + 2 y_H2 + y_H+ = 1 and charge neutrality
    y_H+ = y_e (Sec. 2.2.8) hold after the step; abundances stay in [0, 1];
    temperatures stay above the CMB floor."""
    c = inputs.cells_uniform(512, seed=7)
    o = oracle.li_step(c, 1e3 * YR, 1.0)
    assert np.all(o["status"] & oracle.ST_BADINPUT == 0)
    np.testing.assert_allclose(o["y_H"] + 2 * o["y_H2"] + o["y_Hp"], 1.0, rtol=0, atol=1e-15)
    assert np.array_equal(o["y_Hp"], o["y_e"])
    for k in ("y_H", "y_H2", "y_e"):
        assert np.all((o[k] >= 0) & (o[k] <= 1))
    assert np.all(o["T_g"] >= 2.725) and np.all(o["T_d"] >= 2.725)


@pytest.mark.parametrize("Z", [1.0, 1e-2, 1e-4])
def test_energy_invariant_of_appendix_c(Z):
    """P7: with the gas heating/cooling of Table 4 switched off, the LI rows of
    Appendix C conserve rho f_d C_d dT_d + dE_IR + rho alpha_g dT_g =
    rho f_d dt E_UV in every substep (their column sums cancel once the dust
    row, which is written per unit of solar-metallicity dust, is weighted by
    the dust abundance f_d = Z / Z_sun; Eqs. ap_eq:Td2, ap_eq:Tg_2 and the IR
    row).  A misplaced or missing f_d breaks it at Z != Z_sun."""
    cell = one_cell(n_H=1e4, T_g=40.0, T_d=15.0, G0=100.0, E_IR=1e-6)
    cfg = oracle.default_config(reaction_mask=0,
                                process_mask=oracle.P_GASGRAIN | oracle.P_DUST_UV | oracle.P_DUST_EMIT
                                | oracle.P_DUST_IRABS)
    cfg.Z = Z
    cd = 1000.0
    dt = 1e6
    rec, st = oracle.li_trace(cell, dt, cd, cfg)
    assert st & oracle.ST_TIGHT == 0 and len(rec) > 5
    u0 = np.array([cell[k] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
    _, _, _, M, _, aux = oracle.system(cell["n_H"], u0, cell["G0"], 0.0, cell["N_H2"], 1.0, cd, cfg)
    rho, alpha_g, EUV = aux[0], aux[1], aux[2]
    wd = rho * Z * cd * 1e4
    prev = u0
    for t_end, dts, *u in rec:
        u = np.array(u)
        lhs = wd * (u[3] - prev[3]) + (u[4] - prev[4]) + rho * alpha_g * (u[2] - prev[2])
        scale = wd * abs(u[3] - prev[3]) + abs(u[4] - prev[4]) + rho * alpha_g * abs(u[2] - prev[2])
        src = rho * Z * dts * EUV
        # plus the rounding of the recorded states the differences are taken
        # from (E_IR changes by ~1e-11 of itself per substep here)
        ulp = 4 * np.finfo(float).eps * (wd * (abs(u[3]) + abs(prev[3])) + abs(u[4]) + abs(prev[4]) +
                                         rho * alpha_g * (abs(u[2]) + abs(prev[2])))
        assert abs(lhs - src) <= 1e-9 * max(scale, src) + ulp
        prev = u


# ------------------------------------------------------------ Jacobian and solve
def _fd_jacobian(n_H, u, G0, nE, NH2, cd, cfg):
    """Central differences with one Richardson extrapolation step."""
    J = np.zeros((5, 5))
    for j in range(5):
        def F_at(h):
            up, um = u.copy(), u.copy()
            up[j] += h
            um[j] -= h
            Fp = oracle.system(n_H, up, G0, nE, NH2, 1.0, cd, cfg)[2]
            Fm = oracle.system(n_H, um, G0, nE, NH2, 1.0, cd, cfg)[2]
            return (Fp - Fm) / (2 * h)
        h = 1e-4 * abs(u[j])
        J[:, j] = (4.0 * F_at(h / 2) - F_at(h)) / 3.0
    return J


def test_jacobian_matches_finite_differences():
    """P9: the exact Jacobian in A = M - dt J (dual numbers for the chemistry and
    heating/cooling, Appendix C's beta_d, beta_IR, zeta for the dust rows)
    equals Richardson-extrapolated central differences of F."""
    c = inputs.cells_uniform(64, seed=11)
    cfg = oracle.default_config()
    checked = 0
    for i in range(64):
        u = np.array([c[k][i] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
        if not (5.0 < u[3] < 150.0) or abs(u[2] - 3.2e5) < 1e4:
            continue   # stay off the opacity kink at 200 K and the g_ff switch
        args = (c["n_H"][i], u, c["G0"][i], c["n_EUV"][i], c["N_H2"][i])
        big = 1e40   # A = M - dt J with a huge dt leaves J without cancellation
        A, b, F, M, ts, aux = oracle.system(*args, big, 1.0, cfg)
        J = (np.diag(M) - A) / big
        Jfd = _fd_jacobian(*args, 1.0, cfg)
        # effect of a relative change of u_j on F_r, against the row's scale
        w = np.abs(u)[None, :]
        rowscale = np.maximum((np.abs(J) * w).max(axis=1, keepdims=True), np.abs(F)[:, None]) + 1e-300
        err = np.abs(J - Jfd) * w / rowscale
        assert err.max() < 1e-6, (i, err.max())
        checked += 1
    assert checked > 30


def test_solve5_matches_library_and_pivots():
    """P10: the oracle's Gaussian elimination equals numpy.linalg.solve on
    well-conditioned systems, including ones whose leading pivot is zero."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        A = rng.standard_normal((5, 5)) + 5 * np.eye(5)
        b = rng.standard_normal(5)
        np.testing.assert_allclose(oracle.solve5(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)
    A = rng.standard_normal((5, 5))
    A[0, 0] = 0.0
    b = rng.standard_normal(5)
    np.testing.assert_allclose(oracle.solve5(A, b), np.linalg.solve(A, b), rtol=1e-10)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.solve5(np.zeros((5, 5)), b)


# ------------------------------------------------- brute-force convergence (P8)
def _ode_reference(cell, dt, cd, cfg):
    from scipy.integrate import solve_ivp
    u0 = np.array([cell[k] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])

    def f(t, u):
        return oracle.rhs(cell["n_H"], u, cell["G0"], cell["n_EUV"], cell["N_H2"], cd, cfg)
    sol = solve_ivp(f, (0.0, dt), u0, method="Radau", rtol=1e-10,
                    atol=np.maximum(np.abs(u0) * 1e-14, 1e-22))
    assert sol.success
    return sol.y[:, -1]


def _rel(a, b):
    d = np.abs(a - b) / np.maximum(np.abs(b), 1e-6 * np.array([1, 1, 0, 0, 0]) + 1e-300)
    return d.max()


@pytest.mark.slow
def test_li_converges_first_order_to_the_ode():
    """P8: as f_chem -> 0 the LI result converges at first order to the exact
    solution of the ODE it discretises (Radau, rtol 1e-10); the error is of
    order f_chem (Sec. 3.5)."""
    c = inputs.cells_uniform(256, seed=21)
    base = oracle.li_step(c, 1e2 * YR, 100.0)
    picks = [i for i in np.argsort(base["n_sub"]) if 20 < base["n_sub"][i] < 200][:4]
    assert len(picks) == 4
    for i in picks:
        cell = {k: float(c[k][i]) for k in inputs.FIELDS}
        cfg = oracle.default_config()
        ref = _ode_reference(cell, 1e2 * YR, 100.0, cfg)
        errs = []
        for f in (0.03, 0.01, 0.003):
            o = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, 1e2 * YR, 100.0,
                               oracle.default_config(f_chem=f))
            got = np.array([o[k][0] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
            errs.append(_rel(got, ref))
        assert errs[2] < 3e-3, (i, errs)
        assert errs[2] < 0.5 * errs[0] + 1e-9, (i, errs)


def test_nr_reference_converges_to_the_ode():
    """The Newton-Raphson backward-Euler reference (Sec. 2.2.8) solves the same
    ODE: split into M equal hydro steps it approaches the Radau solution at first
    order (quiet molecular cell, C_d = 1e6)."""
    cell = one_cell(n_H=1e3, T_g=60.0, T_d=15.0, y_H2=0.3, y_e=1e-5, G0=10.0, N_H2=1e20)
    cd = 100.0
    dt = 100.0 * YR
    cfg = oracle.default_config()
    ref = _ode_reference(cell, dt, cd, cfg)
    errs = []
    for M in (10, 100):
        st = {k: np.array([v]) for k, v in cell.items()}
        for _ in range(M):
            o = oracle.nr_step(st, dt / M, cd, cfg)
            assert o["status"][0] & oracle.ST_NOCONV == 0
            for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR"):
                st[k] = o[k]
        got = np.array([st[k][0] for k in ("y_H2", "y_e", "T_g", "T_d", "E_IR")])
        errs.append(_rel(got, ref))
    assert errs[1] < 0.2 * errs[0], errs
    assert errs[1] < 1e-4, errs


def test_nr_and_li_agree_on_quiet_cells():
    """LI vs NR on cells near thermal balance: the paper finds agreement at the
    NR tolerance level for C_d = 1e4 in the Bonnor-Ebert collapse (Sec. 3.6)."""
    cell = one_cell(n_H=1e4, T_g=10.0, T_d=10.0, y_H2=0.499, y_e=1e-7, G0=1e-2, N_H2=1e21)
    c = {k: np.array([v]) for k, v in cell.items()}
    li = oracle.li_step(c, 10.0 * YR, 1.0)
    nr = oracle.nr_step(c, 10.0 * YR, 1.0)
    for k in ("T_g", "T_d"):
        assert abs(li[k][0] / nr[k][0] - 1.0) < 1e-3, (k, li[k][0], nr[k][0])


# ---------------------------------------------------------------- host logic
def test_invalid_inputs_are_flagged_and_left_alone():
    c = inputs.cells_uniform(8, seed=2)
    c["n_H"][1] = -1.0
    c["T_g"][2] = np.nan
    c["y_H2"][3] = 0.6
    o = oracle.li_step(c, 1e3 * YR, 1.0)
    for i in (1, 2, 3):
        assert o["status"][i] == oracle.ST_BADINPUT and o["n_sub"][i] == 0
    assert o["T_d"][1] == c["T_d"][1]
    assert np.all(o["status"][[0, 4, 5, 6, 7]] & oracle.ST_BADINPUT == 0)


def test_substep_cap_sets_status():
    c = inputs.cells_uniform(16, seed=2)
    o = oracle.li_step(c, 1e3 * YR, 1.0, oracle.default_config(n_sub_max=3))
    assert np.all(o["n_sub"] <= 3)
    assert np.any(o["status"] & oracle.ST_CAP)


def test_zero_dt_is_identity():
    c = inputs.cells_uniform(8, seed=2)
    o = oracle.li_step(c, 0.0, 1.0)
    assert np.all(o["n_sub"] == 0)
    np.testing.assert_array_equal(o["T_g"], c["T_g"])


def test_solve5_is_exact_on_badly_scaled_systems():
    """P10b: the LI systems mix units spanning ~30 decades (condition numbers
    near 1e16 before scaling).  A = D1 B D2 with B well conditioned and
    diagonal D1, D2 over 1e-20..1e10: the oracle must recover the known x."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        B = rng.standard_normal((5, 5)) + 4 * np.eye(5)
        d1 = 10.0 ** rng.uniform(-20, 10, 5)
        d2 = 10.0 ** rng.uniform(-20, 10, 5)
        A = d1[:, None] * B * d2[None, :]
        x = rng.standard_normal(5) / d2
        b = d1 * (B @ (d2 * x))
        np.testing.assert_allclose(oracle.solve5(A, b), x, rtol=1e-10)


# ------------------------------------------------------------ reading R30
def test_step_rejection_keeps_updates_small():
    """Reading of the small-change assumption behind Eq. eq_deq: an update
    that would move y_H2 or y_e by more than half of max(y, y_floor), or T_g
    by more than a factor 2, is redone with half the step.  On the GRF cell
    that sits at an unstable thermal balance (the single LI update threw it
    to T_CMB or 1.4e5 K depending on C_d), every recorded substep stays
    inside those bounds and the result is the same physical state for
    C_d = 1e4 and 1e7."""
    g = inputs.cells_grf(128, seed=1002)
    cell = {k: float(g[k][1024557]) for k in inputs.FIELDS}
    cfg = oracle.default_config()
    finals = []
    for cd in (1.0, 1000.0):
        rec, st = oracle.li_trace(cell, 1e3 * inputs.YR, cd, cfg)
        u = np.array([[cell["y_H2"], cell["y_e"], cell["T_g"]]] + [r[2:5] for r in rec])
        dy = np.abs(np.diff(u[:, :2], axis=0))
        assert np.all(dy <= 0.5 * np.maximum(u[:-1, :2], cfg.y_floor) * (1 + 1e-12))
        ratio = u[1:, 2] / u[:-1, 2]
        assert np.all((ratio <= 2.0 + 1e-12) & (ratio >= 0.5 - 1e-12))
        finals.append(rec[-1][4])
        assert 10.0 < rec[-1][4] < 2e4
    assert abs(finals[0] / finals[1] - 1.0) < 1e-3


def test_step_rejection_bounds_on_wide_range_cells():
    """The same reading on the wide-range cells, where it fires (about 7 %
    of them take at least one halving): on every cell that had a substep
    redone, every accepted update keeps |dy_H2|, |dy_e| <= max(y, y_floor)/2
    and T_g within a factor 2, and the controller as printed
    (ORACLE_F_NO_REJECT) takes updates outside those bounds on the same
    cells, so the bounds are what the halving enforces."""
    c = inputs.cells_extreme(4096, seed=3)
    o = oracle.li_step(c, 1e3 * YR, 1.0)
    picks = np.nonzero(o["n_rej"] > 0)[0][:24]
    assert len(picks) == 24
    cfg = oracle.default_config()
    lit = oracle.default_config(flags=oracle.F_NO_REJECT)
    outside = 0
    for i in picks:
        cell = {k: float(c[k][i]) for k in inputs.FIELDS}
        for conf, bounded in ((cfg, True), (lit, False)):
            rec, st = oracle.li_trace(cell, 1e3 * YR, 1.0, conf)
            u = np.array([[cell["y_H2"], cell["y_e"], cell["T_g"]]] + [r[2:5] for r in rec])
            dy = np.abs(np.diff(u[:, :2], axis=0))
            ok_y = dy <= 0.5 * np.maximum(u[:-1, :2], conf.y_floor) * (1 + 1e-12)
            ratio = u[1:, 2] / u[:-1, 2]
            ok_T = (ratio <= 2.0 + 1e-12) & (ratio >= 0.5 - 1e-12)
            if bounded:
                assert np.all(ok_y) and np.all(ok_T), i
            else:
                outside += int(not (np.all(ok_y) and np.all(ok_T)))
    assert outside >= len(picks) // 2


def test_conservation_and_bounds_on_wide_range_cells():
    """P6 where the bounds bind: on the wide-range cells (y_e within 1e-8 of 1
    for a fifth of them, y_H2 within 1e-8 of (1 - y_e)/2 for 30 %), after the
    step y_H + 2 y_H2 + y_H+ = 1 with every abundance in [0, 1], both
    temperatures at least T_CMB (Fixsen 2009) and E_IR at least the CMB's
    energy density seen through the reduced light speed, (c / c~) a T_CMB^4
    with c~ = 1e-4 c (Sec. 2) and a from CODATA."""
    g = golden("physical_constants.txt")
    c = inputs.cells_extreme(4096, seed=3)
    o = oracle.li_step(c, 1e3 * YR, 1.0)
    ok = (o["status"] & oracle.ST_BADINPUT) == 0
    assert ok.mean() > 0.99
    np.testing.assert_allclose((o["y_H"] + 2 * o["y_H2"] + o["y_Hp"])[ok], 1.0, rtol=0, atol=1e-15)
    for k in ("y_H", "y_H2", "y_e"):
        assert np.all((o[k][ok] >= 0) & (o[k][ok] <= 1)), k
    T_cmb = g["T_CMB"]
    assert np.all(o["T_g"][ok] >= T_cmb * (1 - 1e-4)) and np.all(o["T_d"][ok] >= T_cmb * (1 - 1e-4))
    E_floor = 1e4 * g["a_rad"] * T_cmb ** 4
    assert np.all(o["E_IR"][ok] >= E_floor * (1 - 1e-3))
    # where it binds: an E_IR below the floor, drained further by dust held at
    # 10 K that absorbs IR and does not emit, ends at the floor
    cfg = oracle.default_config(process_mask=oracle.P_DUST_IRABS, reaction_mask=0,
                                flags=oracle.F_FREEZE_TG | oracle.F_FREEZE_TD | oracle.F_FREEZE_YH2
                                | oracle.F_FREEZE_YE)
    cell = one_cell(n_H=1e4, T_g=10.0, T_d=10.0, E_IR=1e-12)
    r = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, 1.0 * YR, 1.0, cfg)
    assert float(r["E_IR"][0]) == pytest.approx(E_floor, rel=1e-3, abs=0)


def test_projection_of_inputs_at_the_budget_tolerance():
    """The projection of Sec. 2.2.8 (H-nuclei conservation, y_H >= 0) applies
    to the inputs: a state with 2 y_H2 + y_e = 1 + 5e-10 (accepted: the
    input check allows 1e-9) leaves the call with y_H2 = (1 - y_e)/2, y_H = 0
    and y_H + 2 y_H2 + y_H+ = 1, also with nothing to integrate."""
    ye = 0.25
    cell = one_cell(y_e=ye, y_H2=(1.0 - ye) / 2.0 + 2.5e-10)
    for dt in (0.0, 1.0 * YR):
        o = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, dt, 1.0,
                           oracle.default_config(reaction_mask=0, flags=oracle.F_FREEZE_THERMAL))
        assert o["status"][0] & oracle.ST_BADINPUT == 0
        assert o["y_H2"][0] == (1.0 - ye) / 2.0 and o["y_H"][0] == 0.0
        assert o["y_H"][0] + 2.0 * o["y_H2"][0] + o["y_Hp"][0] == 1.0


def test_projection_bounds_a_linearized_overshoot():
    """The LI update is linear in the change: collisional ionization (Table 3
    H0) at y_e = 0.8, T_g = 1e5 K has dR_e/dy_e = k_H0 n (y_H - y_e) < 0, and
    one long substep (f_chem = 10) carries y_e to 0.8 + 0.16/0.6 = 1.07 > 1
    (within the step-rejection bound of 0.4).  The projection keeps y_e <= 1
    and y_H >= 0."""
    cfg = oracle.default_config(reaction_mask=1 << 0, flags=oracle.F_FREEZE_THERMAL | oracle.F_FREEZE_YH2,
                                f_chem=10.0)
    cell = one_cell(n_H=1.0, T_g=1e5, y_H2=0.0, y_e=0.8, G0=0.0)
    rec, st = oracle.li_trace(cell, 1e10, 1.0, cfg)
    assert len(rec) == 1 and rec[0][3] == 1.0
    o = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, 1e10, 1.0, cfg)
    assert o["y_e"][0] == 1.0 and o["y_H"][0] == 0.0


def test_step_rejection_bounds_the_gas_temperature():
    """The T_g bound of the step-rejection reading: photoelectric heating
    alone (independent of T_g) with f_chem = 10 would multiply T_g by ~11 in
    one substep; every recorded substep stays within a factor 2 (measured
    1.71), after halvings."""
    cfg = oracle.default_config(reaction_mask=0, process_mask=oracle.P_G4_PHOTOELEC,
                                flags=oracle.F_FREEZE_TD | oracle.F_FREEZE_EIR | oracle.F_FREEZE_YH2
                                | oracle.F_FREEZE_YE, f_chem=10.0)
    cell = one_cell(n_H=1.0, T_g=100.0, y_H2=0.0, y_e=1e-4, G0=10.0)
    rec, st = oracle.li_trace(cell, 1e5 * YR, 1.0, cfg)
    T = np.array([cell["T_g"]] + [r[4] for r in rec])
    assert np.all(T[1:] / T[:-1] <= 2.0 + 1e-12)
    o = oracle.li_step({k: np.array([v]) for k, v in cell.items()}, 1e5 * YR, 1.0, cfg)
    assert o["n_halv"][0] > 0
