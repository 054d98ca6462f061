// nr_device.cuh -- the Newton-Raphson backward-Euler thermochemical solver
// of Sec. 2.2.8 (the reference the paper validates the LI method against),
// on the GPU in FP64, one thread per cell.
//
// Each attempt solves the backward-Euler equations of a substep
//   y - y^t = dt R(y, T_g, T_d),  C_d (T_d - T_d^t) = dt D,  E - E^t = dt I,
//   alpha_g^t (T_g - T_g^t) = dt (Gamma - Lambda)/rho
// by three nested Newton groups: the outer iteration on T_g with a
// central-difference derivative; for each trial T_g the dust/IR group
// (T_d, E_IR) and then the species group (y_H2, y_e).  Convergence: relative
// change below 1e-5 (relaxed to 1e-3 after N_itr,limit/2 outer iterations).
// The hydro step is tried first; on failure it is subdivided as
// dt_sub = (dt_hydro - t_sub) / 2^i, i = 1 first, i-1 after a success and
// i+1 after a failure (Eq. substep_NRchem).
#pragma once
#include "li_kernels.cuh"

namespace sfc {

// Group (iii): species at fixed (T_g, T_d).  Returns iterations, < 0 on failure.
__device__ __forceinline__ int newton_species(double u[5], const double u0[5], double dt, const CellK<double> &k,
                                              const DevCfg &cfg, double tol) {
  const bool fr0 = cfg.flags & F_FY2, fr1 = cfg.flags & F_FYE;
  if (fr0 && fr1) return 0;
  Pre<double> q;
  const double T = u[2], Td = u[3];
  make_pre<double>(T, Td, q);
  Rates<double> r;
  eval_rates<double>(T, Td, q, k, cfg.rmask, r);
  const bool via_on = ((cfg.rmask >> 2) & 1u) && ((cfg.rmask >> 3) & 1u);
  for (int it = 1; it <= cfg.nr_itr_limit; ++it) {
    const double yH = 1.0 - 2.0 * u[0] - u[1];
    double F0, F1, J0[4], J1[4];
    chem_rows<double>(r, k.n, u[0], u[1], yH, via_on, F0, F1, J0, J1, false);
    double g0 = -(u[0] - u0[0] - dt * F0), g1 = -(u[1] - u0[1] - dt * F1);
    double a00 = 1.0 - dt * J0[0], a01 = -dt * J0[1], a10 = -dt * J1[0], a11 = 1.0 - dt * J1[1];
    if (fr0) { a00 = 1.0; a01 = 0.0; g0 = 0.0; }
    if (fr1) { a10 = 0.0; a11 = 1.0; g1 = 0.0; }
    const double det = a00 * a11 - a01 * a10;
    if (!(fabs(det) > 0.0)) return -it;
    const double d0 = (g0 * a11 - a01 * g1) / det, d1 = (a00 * g1 - a10 * g0) / det;
    u[0] += d0;
    u[1] += d1;
    project(u);
    if (fabs(d0) <= tol * fmax(u[0], cfg.y_floor) && fabs(d1) <= tol * fmax(u[1], cfg.y_floor)) return it;
  }
  return -cfg.nr_itr_limit;
}

// Inner groups at a trial T_g, then the gas-energy residual in units of
// k_B / (mu_H m_H): g = (n_tot/n_H)^t (T_g - T_g^t)/(gamma_ad - 1) - dt H.
__device__ __forceinline__ bool nr_inner(double Tg, const double u0[5], double dt, double tol,
                                         const CellK<double> &k, const DevCfg &cfg, const CfgW<double> &cw,
                                         double uo[5], double &g) {
#pragma unroll
  for (int i = 0; i < 5; ++i) uo[i] = u0[i];
  uo[2] = Tg;
  if (newton_dust(uo, u0, dt, k, cfg, tol) < 0) return false;
  if (newton_species(uo, u0, dt, k, cfg, tol) < 0) return false;
  Sys<double> S;
  eval_system<double>(uo, 1.0 - 2.0 * uo[0] - uo[1], k, cfg, cw, S);
  const double ytot0 = 1.0 - u0[0] + u0[1] + YHE;
  g = ytot0 * (Tg - u0[2]) / (cfg.gamma_ad - 1.0) - dt * S.H;
  return true;
}

// One backward-Euler step by nested Newton-Raphson; > 0 (outer iterations)
// on convergence, 0 on failure.
__device__ __forceinline__ int nr_be_step(double u[5], double dt, const CellK<double> &k, const DevCfg &cfg,
                                          const CfgW<double> &cw) {
  double u0[5], uo[5], g;
#pragma unroll
  for (int i = 0; i < 5; ++i) u0[i] = u[i];
  const int limit = cfg.nr_itr_limit;
  if (cfg.flags & F_FTG) {
    if (!nr_inner(u0[2], u0, dt, cfg.nr_tol, k, cfg, cw, uo, g)) return 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) u[i] = uo[i];
    return 1;
  }
  double Tg = u0[2];
  for (int it = 1; it <= limit; ++it) {
    const double tol = (it > limit / 2) ? 1e-3 : cfg.nr_tol;
    const double h = 1e-4 * Tg;
    double up[5], gp, gm;
    if (!nr_inner(Tg, u0, dt, tol, k, cfg, cw, uo, g)) return 0;
    if (!nr_inner(Tg + h, u0, dt, tol, k, cfg, cw, up, gp)) return 0;
    if (!nr_inner(Tg - h, u0, dt, tol, k, cfg, cw, up, gm)) return 0;
    const double dg = (gp - gm) / (2.0 * h);
    if (dg == 0.0 || !isfinite(dg)) return 0;
    const double Tn = fmax(Tg - g / dg, TCMB);
    const bool conv = fabs(Tn - Tg) <= tol * Tn;
    Tg = Tn;
    if (conv) {
      if (!nr_inner(Tg, u0, dt, tol, k, cfg, cw, uo, g)) return 0;
#pragma unroll
      for (int i = 0; i < 5; ++i) u[i] = uo[i];
      return it;
    }
  }
  return 0;
}

// One attempt of the substepping procedure; true when the cell is finished.
__device__ __forceinline__ bool nr_attempt(CellRun<double> &c, const DevCfg &cfg, const CfgW<double> &cw) {
  const double dt_h = c.k.dt_h;
  if (!(c.t < dt_h)) return true;
  const double dts = ldexp(dt_h - c.t, -c.nri);
  double uu[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) uu[i] = c.u[i];
  const int it = nr_be_step(uu, dts, c.k, cfg, cw);
  c.ntries++;
  if (it > 0) {
#pragma unroll
    for (int i = 0; i < 5; ++i) c.u[i] = uu[i];
    c.t = (c.nri == 0) ? dt_h : c.t + dts;
    c.nsub++;
    c.nitr += it;
    c.nri = max(c.nri - 1, 0);
  } else {
    c.nri++;
    if (c.nri > 60 || c.ntries > cfg.n_sub_max) { c.st |= ST_NOCONV; return true; }
  }
  return !(c.t < dt_h);
}

}  // namespace sfc
