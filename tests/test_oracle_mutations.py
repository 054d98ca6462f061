"""Mutation check of the oracle's pins: each case plants one plausible
transcription mistake in the printed physics (a coefficient off by a decade,
an activation temperature or an exponent changed, a factor dropped) in a
copy of oracle/sfchem_oracle.cpp, builds the copy with the oracle's own
flags, and runs the pin suites against it (SFCHEM_ORACLE_LIB): at least one
pin must fail.  The unmodified copy, built and run the same way, must pass
every pin, so a failure is the mutation's and not the procedure's.

Covered: the printed rows of Table 3 (k_H0-k_H3, k_H5/k_H6, both limits of
k_H7, k_H8) and Table 4 (Gamma_1, Lambda_5-Lambda_12), the rate equations
(Eq. eq_chemq: signs, dropped terms, wrong abundances, H-nuclei
conservation), the dust, IR and gas-grain terms of App. C with their
Jacobian entries (R_g, T_low, gamma_d, zeta, beta_d, beta_IR, kappa, the
emission law), the gas state (particle count, helium mass in rho,
Eq. ap_eq:alpha_g), the controller and update of Sec. 2.2.8 (f_chem,
y_floor, N_cyc, the (gamma - 1) and the gas-grain term of Eq.
timescale_energy, C_d in the dust timescale, the dust timescale dropped in
tight coupling, the truncation of the last substep, the time accounting,
M - dt J and its heat capacities, the step-rejection bounds, the projection
and the E_IR floor); and, against
its own pin file, the photon consumption after the update (reading R32:
absorbers, shielding, unit conversions, the implicit decay on both sides of
lam dt = 1, the split of the removed photons).

The Newton-Raphson reference is covered too: its residuals, its stopping
tolerance, the coverage of dt_hydro by its substeps and its outer T_g step.

Not covered, because nothing independent of the printed formula pins them
(parity unpinned): the critical densities n_cr of k_H7 and of Gamma_1 (only
their limits are pinned), the prefactor and He+ abundance of Lambda_10, and
the stand-ins for the rates and processes the paper only cites -- except
the line cooling, whose LTE limit is pinned to atomic data.  Not
covered either: an error in a Newton matrix (it changes the iterations, not
the root they converge to) and the tolerance relaxed to 1e-3 after
N_itr,limit/2 outer iterations (no pin's cell takes that many)."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sfchem_oracle.cpp")
HDR = os.path.join(ROOT, "oracle", "sfchem_oracle.h")
# (the physics pins first: a mutant that slows the LI step down fails one of
# them before the longer integrations of the other file run)
PINS = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins_physics.py", "test_oracle_pins.py")]
PHOTON_PINS = [os.path.join(ROOT, "tests", "test_oracle_photon.py")]

# (name, text of the oracle, replacement): one change each
MUTATIONS = [
    ("Lambda5 /10 (13.6 eV per ionization)", "net - 13.6 * eV * k[0]", "net - 1.36 * eV * k[0]"),
    ("Lambda6 /10 (4.48 eV per dissociation)", "net - 4.48 * eV * (k[4]", "net - 0.448 * eV * (k[4]"),
    ("Lambda7 x2 (-25.87 -> -25.57)", "Dual p = -25.87 +", "Dual p = -25.57 +"),
    ("Lambda9 x10 (7.50e-19)", "net - 7.50e-19 /", "net - 7.50e-18 /"),
    ("Lambda9 activation /10 (118348 K)", "dexp(-118348.0 / T)", "dexp(-11834.8 / T)"),
    ("Lambda10 activation /10 (473638 K)", "dexp(-473638.0 / T)", "dexp(-47363.8 / T)"),
    ("Lambda11 x10 (1.426e-27)", "net - 1.426e-27 *", "net - 1.426e-26 *"),
    ("Lambda12 x10 (1.017e-37)", "net - 1.017e-37 *", "net - 1.017e-36 *"),
    ("Lambda12 T_CMB^4 -> T_CMB^3", "std::pow(T_CMB, 4) * (T - T_CMB)", "std::pow(T_CMB, 3) * (T - T_CMB)"),
    ("Gamma1 H- channel 3.73 eV /10", "eV * (3.73 * f * via_Hm", "eV * (0.373 * f * via_Hm"),
    ("k_H3 x10 (1.35e-9)", "k[3] = 1.35e-9 *", "k[3] = 1.35e-8 *"),
    ("k_H5 x10", "Dual k5 = 6e-32 * dpow(T, -0.25) + 2e-31 * dpow(T, -0.5);",
     "Dual k5 = 6e-31 * dpow(T, -0.25) + 2e-30 * dpow(T, -0.5);"),
    ("k_H7 low-density limit x10", "std::log(1.18e-10) - 6.95e4 / T", "std::log(1.18e-9) - 6.95e4 / T"),
    ("k_H7 high-density limit x10", "std::log(8.125e-8) -", "std::log(8.125e-7) -"),
    ("R_g x10", "const double R_g = 5.83e-8;", "const double R_g = 5.83e-7;"),
    ("T_low /10", "const double T_low = 75.0;", "const double T_low = 7.5;"),
    ("(gamma - 1) dropped from dt_energy", "gs.P / ((c.gamma_ad - 1.0) * std::fabs(GmL))", "gs.P / (std::fabs(GmL))"),
    ("(gamma - 1) dropped from alpha_g", "kB / ((c.gamma_ad - 1.0) * s.mu * mH)", "kB / (s.mu * mH)"),
    ("N_cyc /10", "c->n_cyc = 300;", "c->n_cyc = 30;"),
    # the line-cooling stand-in (reading R23), pinned at LTE to atomic data
    ("[C II] excitation temperature 91.2 K -> 9.12 K", "TC_star = 91.2,", "TC_star = 9.12,"),
    ("[O I] A x10", "A_O = 8.9e-5,", "A_O = 8.9e-4,"),
    ("[O I] statistical weight ratio 3/5 -> 5/3", "g_O = 0.6,", "g_O = 1.6667,"),
    ("[C II] abundance x10", "const double x_C = 1.4e-4,", "const double x_C = 1.4e-3,"),
    ("k_H9 cross-section x10 (stand-in R19)", "const double sigma_EUV = 6.3e-18;", "const double sigma_EUV = 6.3e-17;"),
    # other printed rates
    ("k_H0 slope 13.536556 -> 13.636556", "-32.71396786, 13.536556,", "-32.71396786, 13.636556,"),
    ("k_H1 x10", "k[1] = 2.753e-14", "k[1] = 2.753e-13"),
    ("k_H1 exponent 1.5 -> 1", "dpow(315614.0 / T, 1.5)", "dpow(315614.0 / T, 1.0)"),
    ("k_H2 x10", "k[2] = 1.4e-18", "k[2] = 1.4e-17"),
    ("k_H2 cutoff 16200 K /10", "dexp(-T / 16200.0)", "dexp(-T / 1620.0)"),
    ("k_H6 = k_H5 / 0.8", "k[6] = k5 / 8.0;", "k[6] = k5 / 0.8;"),
    ("k_H8 x10", "k[8] = 6.0e-17", "k[8] = 6.0e-16"),
    ("k_H8 sqrt(T/300) -> T/300", "6.0e-17 * dsqrt(T / 300.0)", "6.0e-17 * (T / 300.0)"),
    # rate equations (Eq. eq_chemq): signs, dropped terms, wrong abundances
    ("R_H2: sign of the k_H7 term", "- k[7] * n * yH2 * yH2 - k[10] * yH2", "+ k[7] * n * yH2 * yH2 - k[10] * yH2"),
    ("R_H2: grain formation dropped", "k[6] * n * n * yH * yH * yH2 + k[8] * n * yH -",
     "k[6] * n * n * yH * yH * yH2 -"),
    ("R_H2: one n of three-body formation dropped", "k[5] * n * n * yH * yH * yH + k[6]",
     "k[5] * n * yH * yH * yH + k[6]"),
    ("R_e: recombination on y_H instead of y_H+", "- k[1] * n * yHp * ye;", "- k[1] * n * yH * ye;"),
    ("R_e: cosmic-ray ionization dropped", "+ k[9] * yH + k[11] * yH -", "+ k[9] * yH -"),
    ("H-nuclei conservation: y_H = 1 - y_H2 - y_e", "Dual yH = 1.0 - 2.0 * yH2 - ye;   // H-nuclei",
     "Dual yH = 1.0 - yH2 - ye;   // H-nuclei"),
    # heating and cooling (Table 4)
    ("Gamma1 grain channel 4.2 -> 0.42", "(0.2 + 4.2 * f) * k[8]", "(0.2 + 0.42 * f) * k[8]"),
    ("Lambda6 on y_H2^2 instead of y_H2 y_H", "k[4] * n2 * yH2 * yH +", "k[4] * n2 * yH2 * yH2 +"),
    ("Lambda8 without T", "net - kB * T * k[2]", "net - kB * k[2]"),
    ("Lambda11 Gaunt slope sign", "0.79464 + 0.1243 * dlog10(T)", "0.79464 - 0.1243 * dlog10(T)"),
    ("Lambda12 (T + T_CMB)", "std::pow(T_CMB, 4) * (T - T_CMB)", "std::pow(T_CMB, 4) * (T + T_CMB)"),
    # dust, IR and gas-grain terms (App. C) and their Jacobian entries
    ("kappa quadratic -> linear", "T < kap_Tc ? kap0 * (T / kap_T0) * (T / kap_T0) :", "T < kap_Tc ? kap0 * (T / kap_T0) :"),
    ("dust emission T_d^4 -> T_d^3", "std::pow(Td, 4) : 0.0", "std::pow(Td, 3) : 0.0"),
    ("beta_d 4 kappa -> 3 kappa", "4.0 * kappa(Td) + dkappa(Td) * Td", "3.0 * kappa(Td) + dkappa(Td) * Td"),
    ("beta_IR T kappa'/4 -> /2", "dkappa(d.T_IR) * d.T_IR / 4.0", "dkappa(d.T_IR) * d.T_IR / 2.0"),
    ("gamma_d 0.8 -> 0.08", "d.gam = 1.0 - 0.8 *", "d.gam = 1.0 - 0.08 *"),
    ("zeta: gamma_d/2 -> gamma_d", "d.zeta = d.gam / 2.0 * (Td / Tg - 1.0)", "d.zeta = d.gam * (Td / Tg - 1.0)"),
    ("IR row without f_d", "d.I = ci.rho * ci.fd * (d.emit - d.irabs);", "d.I = ci.rho * (d.emit - d.irabs);"),
    ("gas-grain sign", "d.Qgg = ci.fd * d.G * d.gam * (Td - Tg);", "d.Qgg = ci.fd * d.G * d.gam * (Tg - Td);"),
    ("J[2][2] zeta term sign", "s.J[2][2] += ci.fd * d.G * d.zeta;", "s.J[2][2] -= ci.fd * d.G * d.zeta;"),
    ("J[3][3] without beta_d", "s.J[3][3] = -(d.G * d.gam + acTd3 * d.beta_d);", "s.J[3][3] = -(d.G * d.gam);"),
    ("J[3][4] sign", "s.J[3][4] = c_red * d.beta_IR;", "s.J[3][4] = -c_red * d.beta_IR;"),
    ("J[4][3] without f_d", "s.J[4][3] = ci.rho * acTd3 * ci.fd * d.beta_d;", "s.J[4][3] = ci.rho * acTd3 * d.beta_d;"),
    # gas state and controller
    ("particle count without electrons", "(yH + yH2 + ye + ye + y_He)", "(yH + yH2 + ye + y_He)"),
    ("rho: helium mass 4 m_H -> m_H", "ci.rho = (1.0 + 4.0 * y_He) * mH * n;", "ci.rho = (1.0 + y_He) * mH * n;"),
    ("f_chem 0.03 -> 0.3", "c->f_chem = 0.03;", "c->f_chem = 0.3;"),
    ("dust timescale without C_d", "ratio_ts(u[3], d.D / Cd)", "ratio_ts(u[3], d.D)"),
    ("energy timescale without the gas-grain term", "real GmL = ci.rho * (q.v + d.Qgg);", "real GmL = ci.rho * (q.v);"),
    ("step rejection: y_H2 bound 0.5 -> 5", "bool small = std::fabs(du[0]) <= 0.5 * std::max(u0[0], c.y_floor) &&",
     "bool small = std::fabs(du[0]) <= 5.0 * std::max(u0[0], c.y_floor) &&"),
    ("step rejection: y_e bound 0.5 -> 5", "std::fabs(du[1]) <= 0.5 * std::max(u0[1], c.y_floor) &&",
     "std::fabs(du[1]) <= 5.0 * std::max(u0[1], c.y_floor) &&"),
    ("step rejection: T_g factor 2 -> 10", "du[2] <= u0[2] && du[2] >= -0.5 * u0[2];", "du[2] <= 9.0 * u0[2] && du[2] >= -0.9 * u0[2];"),
    ("projection y_H2 <= 1 - y_e", "u[0] = std::min(std::max(u[0], 0.0), (1.0 - u[1]) / 2.0);",
     "u[0] = std::min(std::max(u[0], 0.0), (1.0 - u[1]));"),
    ("projection without y_e <= 1", "u[1] = std::min(std::max(u[1], 0.0), 1.0);", "u[1] = std::max(u[1], 0.0);"),
    ("E_IR floor from T_CMB^3", "real E_floor_of() { return (c_light / c_red) * a_rad * std::pow(T_CMB, 4); }",
     "real E_floor_of() { return (c_light / c_red) * a_rad * std::pow(T_CMB, 3); }"),
    ("last substep not truncated to the time left", "if (dtc >= rem || rem - dtc <= 1e-12 * dt_h) { dts = rem; last = true; }",
     "if (dtc >= rem || rem - dtc <= 1e-12 * dt_h) { dts = dtc; last = true; }"),
    ("time advanced by 2 dt_s", "t = last ? dt_h : t + dts;", "t = last ? dt_h : t + 2.0 * dts;"),
    ("tight mode keeps the dust timescale", "if (!tight) tmin = std::min(tmin, s.ts[0]);", "tmin = std::min(tmin, s.ts[0]);"),
    ("update u += 2 du", "for (int j = 0; j < 5; ++j) u[j] += du[j];", "for (int j = 0; j < 5; ++j) u[j] += 2.0 * du[j];"),
    ("heat capacity alpha_g missing from M", "s.M[2] = gs.alpha_g;", "s.M[2] = 1.0;"),
    ("C_d missing from M", "s.M[3] = Cd;", "s.M[3] = 1.0;"),
    ("A = M + dt J", "A[r * 5 + j] = (r == j ? s.M[r] : 0.0) - dt * s.J[r][j];",
     "A[r * 5 + j] = (r == j ? s.M[r] : 0.0) + dt * s.J[r][j];"),
    ("y_floor 1e-8 -> 1e-4", "c->y_floor = 1e-8;", "c->y_floor = 1e-4;"),
    # the Newton-Raphson reference (Sec. 2.2.8)
    ("NR species residual with dt/2", "real G[2] = {u[0] - u0[0] - dt * RH2.v, u[1] - u0[1] - dt * Re.v};",
     "real G[2] = {u[0] - u0[0] - 0.5 * dt * RH2.v, u[1] - u0[1] - dt * Re.v};"),
    ("NR energy residual without gas-grain", "g = gs0.alpha_g * (Tg - u0[2]) - dt * (net.v / ci.rho + d.Qgg);",
     "g = gs0.alpha_g * (Tg - u0[2]) - dt * (net.v / ci.rho);"),
    ("NR energy residual with 2 dt", "g = gs0.alpha_g * (Tg - u0[2]) - dt * (net.v / ci.rho + d.Qgg);",
     "g = gs0.alpha_g * (Tg - u0[2]) - 2.0 * dt * (net.v / ci.rho + d.Qgg);"),
    ("NR tolerance 1e-5 -> 1e-2", "c->nr_tol = 1e-5;", "c->nr_tol = 1e-2;"),
    ("NR substeps: time double-counted", "t = (i == 0) ? dt_h : t + dts;", "t = (i == 0) ? dt_h : t + 2.0 * dts;"),
    ("NR outer step sign and length", "real Tn = std::max(Tg - g / dg, T_CMB);", "real Tn = std::max(Tg + 0.5 * g / dg, T_CMB);"),
]


# the photon consumption after the update (reading R32 of Sec. 2.2.8)
PHOTON_MUTATIONS = [
    ("EUV absorption by H without y_H", "c_light * nh * sigma_EUV * yH;", "c_light * nh * sigma_EUV;"),
    ("EUV dust absorption dropped", "const double xE = (lam_H + lam_dE) * dt[i];", "const double xE = (lam_H) * dt[i];"),
    ("EUV opaque branch n/(1 + 2x)", "const double nE = xE < 1.0 ? n_EUV[i] - takeE : n_EUV[i] / (1.0 + xE);",
     "const double nE = xE < 1.0 ? n_EUV[i] - takeE : n_EUV[i] / (1.0 + 2.0 * xE);"),
    ("EUV thin branch explicit (n x instead of n x/(1+x))", "n_EUV[i] * (xE / (1.0 + xE))", "n_EUV[i] * (xE)"),
    ("FUV self-shielding dropped", "const double lam_2 = k_LW * fsh * nh", "const double lam_2 = k_LW * nh"),
    ("FUV photon energy ratio inverted", "y_H2[i] * hnu_FUV / u_Habing;", "y_H2[i] * u_Habing / hnu_FUV;"),
    ("FUV absorbed by y_H instead of y_H2", "nh * y_H2[i] * hnu_FUV", "nh * yH * hnu_FUV"),
    ("FUV opaque branch G0/x", "const double g = xF < 1.0 ? G0[i] - takeF : G0[i] / (1.0 + xF);",
     "const double g = xF < 1.0 ? G0[i] - takeF : G0[i] / (xF);"),
    ("EUV split between H and dust swapped", "absorbed[4 * i + 0] = sE > 0.0 ? dE * lam_H / sE : 0.0;",
     "absorbed[4 * i + 0] = sE > 0.0 ? dE * lam_dE / sE : 0.0;"),
    ("FUV photons removed not converted from G0 units", "const double dF = takeF * u_Habing / hnu_FUV;",
     "const double dF = takeF;"),
    ("y_H without y_e", "std::max(1.0 - 2.0 * y_H2[i] - y_e[i], 0.0);", "std::max(1.0 - 2.0 * y_H2[i], 0.0);"),
]


def _build_and_run(work, name, old, new, pins=PINS):
    """Build the (mutated) copy in `work` and run the pins against it;
    returns (pins passed?, pytest's last line)."""
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"{name}: the oracle text to mutate is not unique or is missing"
        src = src.replace(old, new)
    d = os.path.join(work, str(abs(hash(name))))
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(d, "sfchem_oracle.cpp"), "w") as f:
        f.write(src)
    with open(os.path.join(d, "sfchem_oracle.h"), "w") as f:
        f.write(open(HDR).read())
    so = os.path.join(d, "liboracle_mut.so")
    subprocess.run(["g++", "-O3", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", so,
                    "sfchem_oracle.cpp"], cwd=d, check=True, capture_output=True)
    env = dict(os.environ, SFCHEM_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    return r.returncode == 0, (lines[-1] if lines else r.stderr[-300:])


def _check(mutations, pins):
    cases = [("unmodified", None, None)] + mutations
    with tempfile.TemporaryDirectory() as work, cf.ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        res = dict(zip([c[0] for c in cases], ex.map(lambda c: _build_and_run(work, *c, pins=pins), cases)))
    ok, last = res.pop("unmodified")
    assert ok, f"the unmodified oracle copy fails its pins: {last}"
    survivors = {name: last for name, (passed, last) in res.items() if passed}
    for name, (passed, last) in res.items():
        print(f"{name}: {'SURVIVED' if passed else 'caught'} ({last})")
    assert not survivors, f"mutations that no pin catches: {survivors}"


def test_every_mutation_of_the_printed_physics_fails_a_pin():
    _check(MUTATIONS, PINS)


def test_every_mutation_of_the_photon_update_fails_a_pin():
    _check(PHOTON_MUTATIONS, PHOTON_PINS)
