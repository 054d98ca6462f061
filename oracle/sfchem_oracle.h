/*
 * sfchem_oracle.h -- plain FP64 CPU oracle for the per-cell thermochemical
 * update of SFUMATO# (arXiv 2604.21438).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (libsfchem, its kernels and its Python binding) never calls it, and this
 * oracle includes nothing from the product path.
 *
 * What it computes (see sfchem_oracle.cpp for the per-function citations):
 *   - the linearized-implicit (LI) thermochemical step of Sec. 2.2.8
 *     (Eqs. eq_chem2..eq_deq, Eqs. timescale_of_dust..timestep_subcycle)
 *     coupled with the dust / IR / gas-grain update of Appendix C
 *     (Eqs. ap_eq:dust_temp..ap_eq:zeta);
 *   - the Newton-Raphson backward-Euler reference solver of Sec. 2.2.8
 *     (Eq. substep_NRchem) that the paper validates the LI solver against;
 *   - the pieces the pins need: rate coefficients (Table 3), the 5x5 linear
 *     system of one LI substep, the ODE right-hand side, the 5x5 solve.
 *
 * Every state array is a host pointer, structure-of-arrays, FP64, one entry
 * per cell; CGS units; temperatures in K; times in seconds.
 */
#ifndef SFCHEM_ORACLE_H
#define SFCHEM_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Parameters of one call.  Defaults (oracle_default_config): f_chem 0.03
 * (Sec. 2.2.8), N_cyc 300 (Sec. 2.2.8), n_sub_max 100000, Z/Zsun 1,
 * gamma_ad 5/3, y_floor 1e-8, all reactions and processes on, flags 0,
 * NR iteration limit 20 and tolerance 1e-5 (Sec. 2.2.8). */
typedef struct {
  double f_chem;
  int32_t n_cyc;
  int32_t n_sub_max;
  double Z;            /* metallicity in solar units: f_d = Z */
  double gamma_ad;
  double y_floor;
  uint32_t reaction_mask; /* bit i enables reaction H<i>, i = 0..11 (Table 3) */
  uint32_t process_mask;  /* bit layout: see ORACLE_P_* below */
  uint32_t flags;         /* ORACLE_F_* */
  int32_t nr_itr_limit;
  double nr_tol;
} oracle_config;

/* process_mask bits (Table 4 rows and the Appendix C dust terms) */
enum {
  ORACLE_P_G1_H2FORM = 1u << 0,
  ORACLE_P_G2_PHOTOION = 1u << 1,
  ORACLE_P_G3_PHOTODISS = 1u << 2,
  ORACLE_P_G4_PHOTOELEC = 1u << 3,
  ORACLE_P_L5_HION = 1u << 4,
  ORACLE_P_L6_H2DISS = 1u << 5,
  ORACLE_P_L7_HREC = 1u << 6,
  ORACLE_P_L8_HMFB = 1u << 7,
  ORACLE_P_L9_HEXC = 1u << 8,
  ORACLE_P_L10_HEPEXC = 1u << 9,
  ORACLE_P_L11_FF = 1u << 10,
  ORACLE_P_L12_COMPTON = 1u << 11,
  ORACLE_P_L13_LINE = 1u << 12,
  ORACLE_P_GASGRAIN = 1u << 13,
  ORACLE_P_DUST_UV = 1u << 14,
  ORACLE_P_DUST_EMIT = 1u << 15,
  ORACLE_P_DUST_IRABS = 1u << 16
};

/* flags */
enum {
  ORACLE_F_FREEZE_TG = 1u << 0,
  ORACLE_F_FREEZE_TD = 1u << 1,
  ORACLE_F_FREEZE_EIR = 1u << 2,
  ORACLE_F_FREEZE_YH2 = 1u << 3,
  ORACLE_F_FREEZE_YE = 1u << 4,
  ORACLE_F_SPLIT = 1u << 5,
  ORACLE_F_NO_REJECT = 1u << 6   /* paper-literal controller: no step rejection (reading R30 off) */
};

/* per-cell status bits */
enum {
  ORACLE_ST_CAP = 1u << 0,       /* n_sub_max reached before dt_hydro */
  ORACLE_ST_BADINPUT = 1u << 1,  /* invalid input: cell left unchanged */
  ORACLE_ST_NOCONV = 1u << 2,    /* a tight-coupling Newton loop hit its limit */
  ORACLE_ST_TIGHT = 1u << 3,     /* cell ran in the tight-coupling mode */
  ORACLE_ST_BADSTEP = 1u << 4    /* non-finite or non-positive substep */
};

void oracle_default_config(oracle_config *cfg);

/* LI step of n cells over dt[i] seconds each (in place on T_g, T_d, E_IR,
 * y_H2, y_e).  y_H, y_Hp, y_Hm, status, n_sub, n_itr, n_rej may be NULL.
 * n_rej[2*i] counts the substeps of cell i that the step-rejection reading
 * redid with a smaller step, n_rej[2*i+1] the halvings they took.
 * n_threads <= 0 uses OpenMP's default.  Returns 0, or -1 on a bad argument. */
int oracle_li_cells(int64_t n, const double *n_H, double *T_g, double *T_d,
                    double *E_IR, double *y_H2, double *y_e, double *y_H,
                    double *y_Hp, double *y_Hm, uint8_t *status,
                    int32_t *n_sub, int32_t *n_itr, int32_t *n_rej, const double *G0,
                    const double *n_EUV, const double *N_H2, const double *dt,
                    double cd_factor, const oracle_config *cfg, int n_threads);

/* LI step of one cell that records every substep: rec[7*k + 0..6] =
 * (t_end, dt_s, y_H2, y_e, T_g, T_d, E_IR) after substep k.  Returns the
 * number of substeps (records beyond max_rec are dropped). */
int oracle_li_trace(double n_H, double T_g, double T_d, double E_IR,
                    double y_H2, double y_e, double G0, double n_EUV,
                    double N_H2, double dt, double cd_factor,
                    const oracle_config *cfg, int max_rec, double *rec,
                    uint8_t *status);

/* Newton-Raphson backward-Euler reference (Sec. 2.2.8) on n cells. */
int oracle_nr_cells(int64_t n, const double *n_H, double *T_g, double *T_d,
                    double *E_IR, double *y_H2, double *y_e, uint8_t *status,
                    int32_t *n_sub, int32_t *n_itr, const double *G0,
                    const double *n_EUV, const double *N_H2, const double *dt,
                    double cd_factor, const oracle_config *cfg, int n_threads);

/* Rate coefficients k_H0..k_H11 (Table 3, masked by reaction_mask). */
void oracle_rates(double T_g, double T_d, double n_H, double G0, double n_EUV,
                  double N_H2, const oracle_config *cfg, double k[12]);

/* The linear system of one LI substep at state u = (y_H2, y_e, T_g, T_d,
 * E_IR): A du = b.  Also returns F (the right-hand sides), Mdiag (the
 * diagonal "mass" factors 1, 1, alpha_g, C_d, 1), the timescales
 * ts = (dt_dust, dt_chem, dt_energy) and aux = (rho, alpha_g, E_UV, P,
 * Gamma-Lambda volumetric incl. gas-grain). */
void oracle_system(double n_H, const double u[5], double G0, double n_EUV,
                   double N_H2, double dt, double cd_factor,
                   const oracle_config *cfg, double A[25], double b[5],
                   double F[5], double Mdiag[5], double ts[3], double aux[5]);

/* du/dt = F(u) / Mdiag(u) (the ODE that the LI scheme discretises). */
void oracle_rhs(double n_H, const double u[5], double G0, double n_EUV,
                double N_H2, double cd_factor, const oracle_config *cfg,
                double dudt[5]);

/* Photon consumption after the thermochemical update (Sec. 2.2.8,
 * "Radiation components"; reading: the absorption of the step's EUV and FUV
 * photons by the updated gas and dust, implicit over dt).  Per cell, with
 * y_H = 1 - 2 y_H2 - y_e of the updated state:
 *   EUV: loss rate per photon lam_E = c n_H (sigma_H y_H + sigma_d);
 *        n_EUV' = n_EUV / (1 + lam_E dt) (of n photons n x/(1+x) are
 *        absorbed, x = lam dt; the smaller share is formed from its own
 *        formula, the other as the rest);
 *   FUV: photon density N_F = G0 u_Habing / h nu_F; loss rate per photon
 *        lam_F = k_LW f_sh(N_H2) n_H y_H2 h nu_F / u_Habing + c n_H sigma_d
 *        (one photon per photodissociation); G0' = G0 / (1 + lam_F dt).
 * The photons removed (n_EUV - n_EUV', N_F - N_F') are split between gas and
 * dust in proportion to their loss rates: absorbed[4*i + 0..3] = (EUV by H,
 * EUV by dust, FUV by H2, FUV by dust) in photons cm^-3 (may be NULL).  The
 * stand-in constants are those of the rates (sigma_H, k_LW, f_sh) and of the
 * dust UV absorption (sigma_d, u_Habing), with h nu_F = 12.4 eV. */
int oracle_photon_update(int64_t n, const double *n_H, const double *y_H2, const double *y_e,
                         const double *G0, const double *n_EUV, const double *N_H2, const double *dt,
                         double *G0_out, double *n_EUV_out, double *absorbed);

/* Test hook, 0 (off) by default: multiply every entry of each LI substep's
 * linear system by 1 +- eps in a fixed sign pattern (a rounding-level change
 * of the system), to measure how much a result depends on such changes.
 * Global: set it before a call, not during one. */
void oracle_set_perturbation(double eps);

/* Solve a row-major 5x5 system: power-of-two row/column equilibration,
 * Gaussian elimination with partial pivoting, two refinement steps with
 * double-word residuals.  Returns -1 when singular. */
int oracle_solve5(const double A[25], const double b[5], double x[5]);

#ifdef __cplusplus
}
#endif
#endif
