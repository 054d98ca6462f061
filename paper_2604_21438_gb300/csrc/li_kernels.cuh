// li_kernels.cuh -- per-cell substep driver, 5x5 LU, tight-coupling Newton
// iteration and the persistent lane-refill kernel of libsfchem.
//
// Execution model: one thread per cell.  A persistent grid of warps pulls
// chunks of cells from a global counter (one atomic per chunk).  Inside a
// warp every lane owns one cell and advances it one LI substep per loop
// trip; a lane whose cell has reached dt_hydro stores it and is refilled from
// the warp's chunk (warp-vote refill; the mixed kernel waits until a few
// lanes are idle and serves them together), so lanes with long substep
// sequences do not hold idle lanes hostage.  There are no waits
// on other threads anywhere, so the kernel always terminates: every cell
// loop is bounded by n_sub_max, every Newton loop by nr_itr_limit.
#pragma once
#include "li_device.cuh"

namespace sfc {

// ------------------------------------------------------------------- 5x5 LU
// Gaussian elimination with scaled partial pivoting on the fixed structure of
// A = I - dt J: rows 0-2 (y_H2, y_e, T_g) have non-zeros in columns 0-3, row
// 3 (T_d) in columns 2-4, row 4 (E_IR) in columns 3-4.  The pivot of a
// column is the candidate with the largest |a| after each row of A is scaled
// by the power of two that brings its diagonal entry into [1, 2) (the first
// such row on ties); the arithmetic stays on the unscaled rows.  Plain
// partial pivoting lets a row dominated by its own diagonal win a column it
// barely depends on -- the T_g row (entries ~1e2 in the abundance columns of
// hot ionized gas) or the T_d row (diagonal ~1e5, T_g entry ~3 in tight
// coupling) -- and the unknown of that column is then recovered from it by a
// cancellation of up to ~1e11.  Scaling by the diagonal measures each entry
// against the row's own unknown.  Measured on the mixed path (65,536 cells
// per workload): y_H errors 4-10x smaller than with plain pivoting (max and
// p99, uniform and GRF cells; max on the GMC-like grid), the same as scaling
// by the row's largest entry, for 2 % of the kernel's time instead of 4 %.
// A structural zero never wins a pivot search and eliminating against it
// changes nothing, so only the candidate rows and the non-zero columns are
// visited: the factors are those of the dense elimination.  Row exchanges
// touch only the active columns, and the multipliers stay where they were
// computed, so a second right-hand side is solved by replaying the same
// exchanges (bits of sw) and eliminations.
template <typename W> struct LU5 {
  W a[5][5];
  W inv[5];
  uint32_t sw;
};

// The biased exponent field of |x| (integer instructions, sign dropped) and
// the power of two 2^-e for an entry in [2^e, 2^(e+1)): exact scalings that
// never overflow.  A zero or subnormal diagonal gets the largest factor; one
// with the top finite exponent gets 0, an infinite or NaN one -inf, so that
// such a row wins no pivot over a finite one (such a system ends as a bad
// substep at its pivot test or in the non-finite update anyway).
__device__ __forceinline__ int expo_field(float x) { return __float_as_int(x) & 0x7f800000; }
__device__ __forceinline__ int expo_field(double x) { return __double2hiint(x) & 0x7ff00000; }
__device__ __forceinline__ void row_scale(int e, float &s) { s = __int_as_float(0x7f000000 - e); }
__device__ __forceinline__ void row_scale(int e, double &s) { s = __hiloint2double(0x7fe00000 - e, 0); }

template <typename W>
__device__ __forceinline__ W lu5_row_scale(const LU5<W> &L, int r) {
  W s;
  row_scale(expo_field(L.a[r][r]), s);
  return s;
}

template <typename W>
__device__ __forceinline__ void lu5_swap(LU5<W> &L, W rs[5], int p, int r, int j0, int j1, int bit) {
  const bool ex = M<W>::abs(L.a[r][p]) * rs[r] > M<W>::abs(L.a[p][p]) * rs[p];
  L.sw |= (ex ? 1u : 0u) << bit;
#pragma unroll
  for (int j = j0; j < j1; ++j) {
    const W x = L.a[p][j], y = L.a[r][j];
    L.a[p][j] = ex ? y : x;
    L.a[r][j] = ex ? x : y;
  }
  const W sp = rs[p], sr = rs[r];
  rs[p] = ex ? sr : sp;
  rs[r] = ex ? sp : sr;
}

template <typename W>
__device__ __forceinline__ bool lu5_pivot(LU5<W> &L, int p) {
  const W piv = L.a[p][p];
  if (!(M<W>::abs(piv) > W(0))) return false;
  L.inv[p] = M<W>::rcp(piv);
  return true;
}

template <typename W>
__device__ __forceinline__ void lu5_elim(LU5<W> &L, int p, int r, int j1) {
  const W f = L.a[r][p] * L.inv[p];
  L.a[r][p] = f;
#pragma unroll
  for (int j = p + 1; j < j1; ++j) L.a[r][j] -= f * L.a[p][j];
}

template <typename W>
__device__ __forceinline__ bool lu5_factor(LU5<W> &L) {
  L.sw = 0u;
  W rs[5] = {lu5_row_scale(L, 0), lu5_row_scale(L, 1), lu5_row_scale(L, 2), lu5_row_scale(L, 3),
             lu5_row_scale(L, 4)};
  // column 0: candidates rows 1, 2 (columns 0-3)
  lu5_swap(L, rs, 0, 1, 0, 4, 0);
  lu5_swap(L, rs, 0, 2, 0, 4, 1);
  if (!lu5_pivot(L, 0)) return false;
  lu5_elim(L, 0, 1, 4);
  lu5_elim(L, 0, 2, 4);
  // column 1: candidate row 2 (columns 1-3)
  lu5_swap(L, rs, 1, 2, 1, 4, 2);
  if (!lu5_pivot(L, 1)) return false;
  lu5_elim(L, 1, 2, 4);
  // column 2: candidate row 3 (columns 2-4; row 2 is zero in column 4)
  lu5_swap(L, rs, 2, 3, 2, 5, 3);
  if (!lu5_pivot(L, 2)) return false;
  lu5_elim(L, 2, 3, 5);
  // column 3: candidate row 4 (columns 3-4)
  lu5_swap(L, rs, 3, 4, 3, 5, 4);
  if (!lu5_pivot(L, 3)) return false;
  lu5_elim(L, 3, 4, 5);
  return lu5_pivot(L, 4);
}

template <typename V>
__device__ __forceinline__ void lu5_xchg(uint32_t sw, int bit, V &x, V &y) {
  const bool ex = (sw >> bit) & 1u;
  const V p = x, q = y;
  x = ex ? q : p;
  y = ex ? p : q;
}

template <typename W, typename V>
__device__ __forceinline__ void lu5_solve(const LU5<W> &L, V b[5]) {
  // forward: the exchanges and eliminations of the factor, column by column
  lu5_xchg(L.sw, 0, b[0], b[1]);
  lu5_xchg(L.sw, 1, b[0], b[2]);
  b[1] -= V(L.a[1][0]) * b[0];
  b[2] -= V(L.a[2][0]) * b[0];
  lu5_xchg(L.sw, 2, b[1], b[2]);
  b[2] -= V(L.a[2][1]) * b[1];
  lu5_xchg(L.sw, 3, b[2], b[3]);
  b[3] -= V(L.a[3][2]) * b[2];
  lu5_xchg(L.sw, 4, b[3], b[4]);
  b[4] -= V(L.a[4][3]) * b[3];
  // back substitution over the non-zeros of U
  b[4] = b[4] * V(L.inv[4]);
  b[3] = (b[3] - V(L.a[3][4]) * b[4]) * V(L.inv[3]);
  b[2] = (b[2] - V(L.a[2][3]) * b[3] - V(L.a[2][4]) * b[4]) * V(L.inv[2]);
  b[1] = (b[1] - V(L.a[1][2]) * b[2] - V(L.a[1][3]) * b[3]) * V(L.inv[1]);
  b[0] = (b[0] - V(L.a[0][1]) * b[1] - V(L.a[0][2]) * b[2] - V(L.a[0][3]) * b[3]) * V(L.inv[0]);
}

template <typename W> __device__ __forceinline__ W m_abs(W x) { return M<W>::abs(x); }

// ----------------------------------------------------------- projection
// max(x, lo) and min(x, hi) of FP64 values against bounds lo >= +0 and
// hi > 0 on the bit patterns: a non-negative double orders like its bits read
// as a signed 64-bit integer, and a negative one (sign bit set) below every
// non-negative bound.  Integer instructions only; equal to fmax / fmin for
// every value but NaN, which they pass through.
__device__ __forceinline__ double max_bits(double x, double lo) {
  return __double_as_longlong(x) < __double_as_longlong(lo) ? lo : x;
}
__device__ __forceinline__ double min_bits(double x, double hi) {
  return __double_as_longlong(x) > __double_as_longlong(hi) ? hi : x;
}

// project() with the constant bounds applied on the bit patterns: FP64
// arithmetic only for the bound (1 - y_e)/2 of y_H2.
__device__ __forceinline__ void project_bits(double u[5]) {
  u[1] = min_bits(max_bits(u[1], 0.0), 1.0);
  u[0] = fmin(max_bits(u[0], 0.0), (1.0 - u[1]) * 0.5);
  u[2] = max_bits(u[2], TCMB);
  u[3] = max_bits(u[3], TCMB);
  u[4] = max_bits(u[4], EFLOOR);
}

// Positivity and conservation after an update: 0 <= y_e <= 1,
// 0 <= y_H2 <= (1 - y_e)/2 (so y_H = 1 - 2 y_H2 - y_e >= 0), temperatures at
// least T_CMB, E_IR at least the CMB-equivalent energy density.  FP64.
__device__ __forceinline__ void project(double u[5]) {
  u[1] = fmin(fmax(u[1], 0.0), 1.0);
  u[0] = fmin(fmax(u[0], 0.0), (1.0 - u[1]) * 0.5);
  u[2] = fmax(u[2], TCMB);
  u[3] = fmax(u[3], TCMB);
  u[4] = fmax(u[4], EFLOOR);
}

// A Newton correction of the tight-coupling iteration is scaled by one
// factor so that T_d changes by at most 2x and E_IR by at most 16x.
template <typename W>
__device__ __forceinline__ W damp_factor(W Td, W E, W dTd, W dE) {
  W lam = W(1);
  // (each division runs only where its condition holds, so its divisor is
  // non-zero there)
  if (Td + dTd > W(2) * Td) lam = min(lam, div_w(Td, dTd));
  if (Td + dTd < W(0.5) * Td) lam = min(lam, div_w(W(-0.5) * Td, dTd));
  if (E + dE > W(16) * E) lam = min(lam, div_w(W(15) * E, dE));
  if (E + dE < E * W(0.0625)) lam = min(lam, div_w(W(-15.0 / 16.0) * E, dE));
  return lam;
}

// Tight coupling (Sec. 2.2.8): Newton iteration of the backward-Euler
// residual of the dust row (Eq. ap_eq:dust_temp) and the IR row
// (Eq. ap_eq:Eir) at the substep's new T_g and abundances.  The iterate is
// the starting point plus corrections accumulated in W, so the loop itself
// runs in W; the corrections come back in a3 / a4 (T_d, E_IR) and the caller
// adds them to its FP64 state once.  Returns the iteration count, negative
// when nr_itr_limit was reached.  Inputs in W: T (= T_g, fixed), Tb / Eb
// (the starting point), g3 / g4 (the starting point minus the substep's
// start), dTg (T_d - T_g at the starting point) and dtw (the substep).  The
// FP64 path forms them exactly from the FP64 state; the mixed path from its
// W-precision view of the state and the LI increments.
// POLISH: once the stopping test holds, one more full Newton step (not
// counted) makes the FP64 result independent of the iteration at which the
// test happened to pass (reading R11 of the oracle).  The mixed path stops at
// the test: after a correction below 1e-5 of T_d, the iterate is within
// ~1e-10 of the root, under its FP32 resolution, and the step costs 4.5 % of
// the mixed kernel's time (measured T_d error on the GMC-like grid: p99
// 1.06e-7 -> 1.32e-7, max 1.8e-7 -> 2.1e-7; the Newton counts are the same).
template <typename W, bool POLISH>
__device__ __forceinline__ int newton_dust_w(W &a3, W &a4, W T, W Tb, W Eb, W g3, W g4, W dTg, W dtw,
                                             const CellK<W> &c, const DevCfg &cfg, W tol) {
  typedef M<W> m;
  const bool frTd = cfg.flags & F_FTD, frE = cfg.flags & F_FE;
  a3 = W(0);                                    // accumulated corrections
  a4 = W(0);
  if (frTd && frE) return 0;
  const uint32_t pm = cfg.pmask;
  const W G = c.Gpre * m::sqrt(T);
  const W gam = W(1) - W(0.8) * m::exp(W(-TLOW) * m::rcp(T));
  const W rho = c.rho, fd = c.fd;
  int result = -cfg.nr_itr_limit;
  bool polish = false;
  for (int it = 1; it <= cfg.nr_itr_limit + 1; ++it) {
    if (it > cfg.nr_itr_limit && !polish) break;
    const W Td = Tb + a3, E = Eb + a4;
    W be_d, ba_d, be_i, ba_i;
    const W kd = kappa_w<W>(Td, be_d, ba_d);
    const W TIR = m::sqrt(m::sqrt(W(1e-4 / ARAD) * E));
    const W ki = kappa_w<W>(TIR, be_i, ba_i);
    const W acTd3 = W(ARAD * CLIGHT) * Td * Td * Td;
    const W emit = (pm & P_EMIT) ? kd * acTd3 * Td : W(0);
    const W irabs = (pm & P_IRABS) ? ki * W(CRED) * E : W(0);
    const W beta_d = (pm & P_EMIT) ? be_d : W(0);
    const W beta_IR = (pm & P_IRABS) ? ba_i : W(0);
    const W D = irabs + c.EUV - emit - G * gam * (dTg + a3);
    const W I = rho * fd * (emit - irabs);
    // Newton system in the corrections (dT_d, dE_IR) themselves, the dust
    // row divided by C_d: J00 and J11 are the diagonals of the relative
    // system, K01 = J01 T_d / E_IR and K10 = J10 E_IR / T_d its off-diagonals
    // with the scalings cancelled, so that no reciprocal of T_d or E_IR is
    // needed (the same determinant; Cramer's rule is scale-invariant)
    W R0 = -(g3 + a3) + dtw * D * c.rCd;
    W R1 = -(g4 + a4) + dtw * I;
    W J00 = W(1) + dtw * (G * gam + acTd3 * beta_d) * c.rCd;
    W K01 = -dtw * W(CRED) * beta_IR * c.rCd;
    W K10 = -dtw * rho * fd * acTd3 * beta_d;
    W J11 = W(1) + dtw * rho * W(CRED) * fd * beta_IR;
    if (frTd) { J00 = W(1); K01 = W(0); R0 = W(0); }
    if (frE) { K10 = W(0); J11 = W(1); R1 = W(0); }
    const W det = J00 * J11 - K01 * K10;
    if (!(m::abs(det) > W(0))) { result = -it; break; }
    const W rdet = m::rcp(det);
    const W d0 = (R0 * J11 - K01 * R1) * rdet;
    const W d1 = (J00 * R1 - K10 * R0) * rdet;
    const W lam = polish ? W(1) : damp_factor<W>(Td, E, d0, d1);
    a3 = fmax_w(Tb + (a3 + lam * d0), W(TCMB)) - Tb;
    a4 = fmax_w(Eb + (a4 + lam * d1), W(EFLOOR)) - Eb;
    // with POLISH, after the stopping test holds, one more full step (not
    // counted) makes the result independent of where the test happened to
    // pass; without it the iteration ends at the test
    if (polish) { result = it - 1; break; }
    if (lam == W(1) && m::abs(d0) <= tol * (Tb + a3) && m::abs(d1) <= tol * (Eb + a4)) {
      if constexpr (!POLISH) {
        result = it;
        break;
      }
      polish = true;
    }
  }
  return result;
}

// FP64 entry: the starting point is the FP64 state u, the substep's start u0;
// the corrections are added to u.
__device__ __forceinline__ int newton_dust(double u[5], const double u0[5], double dt, const CellK<double> &c,
                                           const DevCfg &cfg, double tol) {
  double a3, a4;
  const int it =
      newton_dust_w<double, true>(a3, a4, u[2], u[3], u[4], u[3] - u0[3], u[4] - u0[4], u[3] - u[2], dt, c, cfg, tol);
  u[3] = fmax(u[3] + a3, TCMB);
  u[4] = fmax(u[4] + a4, EFLOOR);
  return it;
}

// Per-launch statistics (device), reduced per warp except the rare
// step-rejection counts, which are added where they happen.
struct DevStats {
  unsigned long long cells, substeps, newton, tight, cap, noconv, bad, badstep, rejected, halvings;
  unsigned int max_sub, pad;
};

// ------------------------------------------------------------- one cell
template <typename W> struct CellRun {
  double u[5];   // y_H2, y_e, T_g, T_d, E_IR
  double t;      // time advanced so far in this call (mixed LI path: time left)
  CellK<W> k;
  int32_t nsub, nitr;
  int32_t nri, ntries;   // halving exponent of the step (both methods); NR attempts
  uint8_t st;
  int8_t mode;   // -1 undecided, 0 subcycling, 1 tight coupling
};

// Input checks on the bit patterns (integer instructions; a lane runs them
// alone when its warp refills it): finite, n_H, T_g, T_d > 0, the others >= 0
// (-0 included), y_e <= 1; only the H-nuclei budget 2 y_H2 + y_e <= 1 + 1e-9
// takes FP64 arithmetic.
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool positive_bits(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool nonneg_bits(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool valid_input(double n, double Tg, double Td, double E, double y2,
                                            double ye, double G0, double nE, double NH2, double dt) {
  const double v[10] = {n, Tg, Td, E, y2, ye, G0, nE, NH2, dt};
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 10; ++i) ok = ok && finite_bits(v[i]);
  ok = ok && positive_bits(n) && positive_bits(Tg) && positive_bits(Td);
  ok = ok && nonneg_bits(E) && nonneg_bits(y2) && nonneg_bits(ye) && nonneg_bits(G0) && nonneg_bits(nE) &&
       nonneg_bits(NH2) && nonneg_bits(dt);
  ok = ok && __double_as_longlong(ye) <= __double_as_longlong(1.0);
  return ok && 2.0 * y2 + ye <= 1.0 + 1e-9;
}

// Residual of the factored FP32 system, r = b - A x, formed to about twice
// the FP32 precision with error-free transformations (TwoProduct by fma,
// TwoSum) and rounded once.  Only the structural non-zeros of A are visited.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ float residual_ff(float b, const float *a, const float *x, int j0, int j1) {
  float s = b, c = 0.0f;
  for (int j = j0; j < j1; ++j) {
    const float p = -a[j] * x[j];
    const float pe = fmaf(-a[j], x[j], -p);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    c += pe + te;
  }
  return s + c;
}

// Abundance rows of the mixed path in FP64, for the lanes whose update
// cancels an abundance.  The substep's rate coefficients are evaluated again
// (the same FP32 operations on the same inputs give the same values); the
// chemistry rows -- R_H2, R_e and their partials in y_H2 and y_e (Eq. eq_deq)
// -- are formed from them in FP64, with y_H = 1 - 2 y_H2 - y_e from the FP64
// state.  The residual of those two rows, r = dt F - A x (their temperature
// columns as in the FP32 system), is solved with the FP32 factors for a
// correction d; with rows 2-4 left at their (refined) residual, x + d solves
// the system whose chemistry rows are the FP64 ones.  Out of line, and every
// argument by value: a reference would give the caller's registers an
// address and move them to local memory for the whole loop.
struct F5 { float v[5]; };
struct PreciseOut { double inc0, inc1; float d2, d3, d4; };
static __device__ __noinline__ PreciseOut precise_abundance_rows(
    double y2, double ye, double yH64, float T, float Td, float n, float fd, float lnn, float k9, float k10,
    float k11, uint32_t rmask, uint32_t flags, float dw, LU5<float> L, F5 x, F5 dx, float J02, float J03,
    float J12, float J13) {
  CellK<float> ck;
  ck.n = n; ck.fd = fd; ck.lnn = lnn; ck.k9 = k9; ck.k10 = k10; ck.k11 = k11;
  Pre<float> q;
  make_pre<float>(T, Td, q);
  Rates<float> r;
  eval_rates<float>(T, Td, q, ck, rmask, r);
  Rates<double> r64;
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    r64.k[i] = f2d_int(r.k[i]);
    r64.kT[i] = 0.0;
  }
  r64.k8d = 0.0;
  const bool via_on = ((rmask >> 2) & 1u) && ((rmask >> 3) & 1u);
  double F[2], Jr[2][4];
  chem_rows<double>(r64, f2d_int(n), y2, ye, yH64, via_on, F[0], F[1], Jr[0], Jr[1], false);
  const double dt = f2d_int(dw);
  double X[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) X[j] = f2d_int(x.v[j]) + f2d_int(dx.v[j]);
  const float Jt[2][2] = {{J02, J03}, {J12, J13}};
  const uint32_t frozen[2] = {F_FY2, F_FYE};
  float rr[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (flags & frozen[i]) continue;          // a frozen row is the identity: x_i = 0
    double acc = dt * F[i];
#pragma unroll
    for (int j = 0; j < 2; ++j) acc = fma(-((i == j ? 1.0 : 0.0) - dt * Jr[i][j]), X[j], acc);
#pragma unroll
    for (int j = 2; j < 4; ++j) acc = fma(-f2d_int(-dw * Jt[i][j - 2]), X[j], acc);
    rr[i] = d2f_int(acc);
  }
  lu5_solve<float, float>(L, rr);
  PreciseOut o;
  o.inc0 = X[0] + f2d_int(rr[0]);
  o.inc1 = X[1] + f2d_int(rr[1]);
  o.d2 = rr[2]; o.d3 = rr[3]; o.d4 = rr[4];
  return o;
}

// One LI substep of Sec. 2.2.8; returns true when the cell is finished.
// MIXED: W = float for rates, Jacobian and LU, followed by one residual
// refinement of the 5x5 solve (residual in FP64, or with error-free FP32
// transformations when F_REFINE_FF is set); the update, the projection and the
// time accounting stay FP64.
// RF: how the mixed path forms its refinement residual -- -1 at run time
// from SFCHEM_F_REFINE_FF, 0 the default (FP64 abundance rows), 1 every row
// with error-free FP32 (a compile-time choice keeps one variant in the loop).
template <typename W, bool MIXED, int RF = -1>
__device__ __forceinline__ bool li_substep(CellRun<W> &c, const DevCfg &cfg, const CfgW<W> &cw,
                                           DevStats *stats) {
  Sys<W> S;
  double yH;
  if constexpr (MIXED) {
    // The projection's bound y_H2 <= (1 - y_e)/2 is applied here, at the
    // next use of the state, where y_H = 1 - 2 y_H2 - y_e is formed anyway: a
    // negative y_H (sign bit) is the violated bound.  The FP64 arithmetic of
    // the bound then runs only in the lanes where it binds.
    yH = fma(-2.0, c.u[0], 1.0) - c.u[1];
    if (__double_as_longlong(yH) < 0) {
      c.u[0] = (1.0 - c.u[1]) * 0.5;
      yH = max_bits(fma(-2.0, c.u[0], 1.0) - c.u[1], 0.0);
    }
  } else {
    yH = 1.0 - 2.0 * c.u[0] - c.u[1];
  }
  eval_system<W>(c.u, yH, c.k, cfg, cw, S);
  const double dt_h = c.k.dt_h;
  if (c.mode < 0) {
    // estimated subcycles dt_hydro / (f_chem dt_dust) against N_cyc, from the start state
    const bool tight = !(to_w<W>(dt_h) * S.rate_dust < cw.ncyc_fchem);
    c.mode = tight ? 1 : 0;
    if (tight) c.st |= ST_TIGHT;
  }
  W inv = fmax_w(S.rate_chem, S.rate_energy);
  if (c.mode == 0) inv = fmax_w(inv, S.rate_dust);
  // +inf when every rate vanishes; NaN rates give NaN (a bad substep below)
  const W dtcw = inv == W(0) ? W(INFINITY) : div_w(cw.f_chem, inv);
  const double dtc = to_f64(dtcw);
  // time left: the FP64 path keeps the elapsed time (the oracle's order of
  // operations), the mixed path the time left itself (one FP64 add less)
  const double rem = MIXED ? c.t : dt_h - c.t;
  // c.nri > 0: the update of this substep was rejected c.nri times (below)
  // and is redone with the step halved as often (exact powers of two)
  bool fits;
  double dts;
  W dw;
  if constexpr (MIXED) {
    // W-precision control (the FP64 pipe is the scarce one): the substep
    // takes the time left once dt_c reaches it to W rounding.  dt_c is
    // finite when it falls short of the time left, so only its sign and
    // NaN need a test.
    const W remw = to_w<W>(rem);
    fits = dtcw >= remw;
    if (!(fits || dtcw > W(0))) { c.st |= ST_BADSTEP; return true; }
    dts = fits ? rem : dtc;
    dw = fits ? remw : dtcw;
    if (c.nri != 0) {
      dts = scale_pow2_neg(dts, c.nri);
      dw *= pow2_neg<W>(c.nri);
    }
  } else {
    fits = (dtc >= rem) || (rem - dtc <= 1e-12 * dt_h);
    dts = (fits ? rem : dtc) * pow2_neg<double>(c.nri);
    if (!(dts > 0.0) || !isfinite(dts)) { c.st |= ST_BADSTEP; return true; }
    dw = (fits ? to_w<W>(rem) : dtcw) * pow2_neg<W>(c.nri);
  }
  const bool last = fits && c.nri == 0;
  // A = I - dt J, b = dt F (scaled rows and columns)
  LU5<W> L;
  W x[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#pragma unroll
    for (int j = 0; j < 5; ++j) L.a[i][j] = (i == j ? W(1) : W(0)) - dw * S.J[i][j];
    x[i] = dw * S.F[i];
  }
  W b[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) b[i] = x[i];
  if (!lu5_factor<W>(L)) { c.st |= ST_BADSTEP; return true; }
  lu5_solve<W, W>(L, x);
  W dx[5];
  {
    // One refinement pass against the factored system (A, b): non-zeros of
    // A are rows 0-2 x columns 0-3, row 3 x columns 2-4, row 4 x columns 3-4
    // (A is re-formed from J: the same operations give the same entries).
    // FP64 path: the residual in FP64 (fixed-precision refinement, which
    // makes the solution componentwise accurate: an unknown that the pivot
    // order recovers through a cancellation -- an abundance under a
    // dominant T_g row, T_g under the T_d row in tight coupling -- comes back
    // to rounding level, whichever valid pivot order was taken).
    // Mixed path: the residual of the two abundance rows is formed in FP64
    // (they feed y_H = 1 - 2 y_H2 - y_e, which cancels as the gas turns
    // fully molecular or ionized); the three thermal rows, whose unknowns are
    // relative changes, take the error-free FP32 residual (TwoProduct by
    // fma, TwoSum: about 48 bits, the FP64 pipe being this kernel's scarce
    // unit).  F_REFINE_FF forms every row's residual the error-free FP32 way.
    const int j0[5] = {0, 0, 0, 2, 3}, j1[5] = {4, 4, 4, 5, 5};
    const bool ff_all = RF < 0 ? (cfg.flags & F_REFINE_FF) != 0u : RF == 1;
    W r[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      W Ai[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) Ai[j] = (i == j ? W(1) : W(0)) - dw * S.J[i][j];
      double acc = to_f64(b[i]);
      if constexpr (!MIXED) {
#pragma unroll
        for (int j = j0[i]; j < j1[i]; ++j) acc = fma(-Ai[j], x[j], acc);
        r[i] = acc;
      } else if (i < 2 && !ff_all) {
#pragma unroll
        for (int j = j0[i]; j < j1[i]; ++j) acc = fma(-to_f64(Ai[j]), to_f64(x[j]), acc);
        r[i] = to_w<W>(acc);
      } else {
        r[i] = residual_ff(float(b[i]), (const float *)Ai, (const float *)x, j0[i], j1[i]);
      }
    }
    lu5_solve<W, W>(L, r);
#pragma unroll
    for (int i = 0; i < 5; ++i) dx[i] = r[i];
  }
  double inc0 = to_f64(x[0]) + to_f64(dx[0]), inc1 = to_f64(x[1]) + to_f64(dx[1]);
  if constexpr (MIXED) {
    // The increments come from FP32 rows and carry an absolute error of
    // ~1e-7 of themselves.  Where an abundance's increment (for y_H, the two
    // increments it is formed from) exceeds 64x the abundance's new value,
    // that error is a relative one of up to ~4e-6 and more: a species driven
    // towards 0, or y_H kept small while H2 and electrons trade places.
    // Those lanes form the abundance rows again in FP64
    // (precise_abundance_rows above).  Measured: about 1 lane-substep in 1e4
    // on the GMC-like grid, 1 in 80 on uniform random cells; 8x instead of
    // 64x triggers 15x more often for the same error.
    const W e0 = x[0] + dx[0], e1 = x[1] + dx[1];
    const W a0 = m_abs(e0), a1 = m_abs(e1);
    const bool cancel = (W(2) * a0 + a1 > W(64) * (S.uyH - W(2) * e0 - e1)) || (a0 > W(64) * (S.uf[0] + e0)) ||
                        (a1 > W(64) * (S.uf[1] + e1));
    if (cancel) {
      F5 xv, dxv;
#pragma unroll
      for (int i = 0; i < 5; ++i) { xv.v[i] = x[i]; dxv.v[i] = dx[i]; }
      const PreciseOut o = precise_abundance_rows(
          c.u[0], c.u[1], yH, S.uf[2], S.uf[3], c.k.n, c.k.fd, c.k.lnn, c.k.k9, c.k.k10, c.k.k11, cfg.rmask,
          cfg.flags, dw, L, xv, dxv, S.J[0][2], S.J[0][3], S.J[1][2], S.J[1][3]);
      inc0 = o.inc0;
      inc1 = o.inc1;
      x[2] += o.d2;
      x[3] += o.d3;
      x[4] += o.d4;
    }
  }
  {
    // The LI step rests on small changes (Delta y << y in the derivation of
    // Eq. eq_deq).  An update that moves y_H2 or y_e by more than half of
    // max(y, y_floor), or T_g by more than a factor 2, is outside that regime
    // (a nearly singular I - dt J): the substep is taken again with half the
    // step, at most 30 times.  The retry is a trip of the caller's loop, so
    // nothing of this system stays live across it; the system is evaluated
    // again from the same state.
    // (the FP32 increments: a precise-pass correction is ~1e-7 of them)
    const W e0 = x[0] + dx[0], e1 = x[1] + dx[1], e2 = x[2] + dx[2];
    bool small = m_abs(e0) <= W(0.5) * fmax_w(S.uf[0], cw.y_floor) &&
                 m_abs(e1) <= W(0.5) * fmax_w(S.uf[1], cw.y_floor) && e2 <= W(1) && e2 >= W(-0.5);
    if constexpr (MIXED) {
      // The conversions to FP64 below take finite values (to_f64).  e0-e2
      // pass the tests above only when x and dx are finite in those rows;
      // the T_d and E_IR rows are tested here, so a solution that is not
      // finite (a NaN or an infinity from a singular or overflowing system)
      // always reaches the rare branch below.
      small = small && m_abs(x[3] + dx[3]) + m_abs(x[4] + dx[4]) < W(INFINITY);
    }
    if (!small) {
      if constexpr (MIXED) {
        // a solution that is not finite ends the cell as a bad substep, with
        // its state as it was before the substep
        W sa = W(0);
#pragma unroll
        for (int i = 0; i < 5; ++i) sa += m_abs(x[i]) + m_abs(dx[i]);
        if (!(sa < W(INFINITY))) { c.st |= ST_BADSTEP; return true; }
      }
      if (c.nri < 30 && !(cfg.flags & F_NO_REJECT)) {
        // rare: counted straight into the statistics (no per-lane registers)
        if (c.nri == 0) atomicAdd(&stats->rejected, 1ull);
        atomicAdd(&stats->halvings, 1ull);
        c.nri++;
        return false;
      }
    }
    c.nri = 0;
  }
  double u0[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) u0[i] = c.u[i];
  // FP64 update: x holds dy_H2, dy_e, dT_g/T_g, dT_d/T_d, dE/E.  The
  // abundance increments keep the refinement as a separate FP64 term (they
  // feed y_H = 1 - 2 y_H2 - y_e, which cancels as the gas turns fully
  // molecular or ionized); the relative thermal increments are combined in W.
  c.u[0] += inc0;
  c.u[1] += inc1;
#pragma unroll
  for (int i = 2; i < 5; ++i) x[i] += dx[i];
  c.u[2] = fma(c.u[2], to_f64(x[2]), c.u[2]);
  // (the mixed path's tight-coupling lanes add the LI increments of T_d and
  // E_IR together with the Newton corrections, below)
  if (!MIXED || c.mode != 1) {
    c.u[3] = fma(c.u[3], to_f64(x[3]), c.u[3]);
    c.u[4] = fma(c.u[4], to_f64(x[4]), c.u[4]);
  }
  if constexpr (MIXED) {
    // The projection of project() without the FP64 pipe where the bound is
    // a constant (integer clamps on the bit patterns, the same values); the
    // bound y_H2 <= (1 - y_e)/2 is applied where y_H is next formed (the
    // next substep, or the store of the finished cell).  An FP64 warp
    // instruction occupies the pipe whatever its number of active lanes, so
    // FP64 code that a few lanes need is kept out of the common path.
    c.u[1] = min_bits(max_bits(c.u[1], 0.0), 1.0);
    c.u[0] = max_bits(c.u[0], 0.0);
    c.u[2] = max_bits(c.u[2], TCMB);
    c.u[3] = max_bits(c.u[3], TCMB);
    c.u[4] = max_bits(c.u[4], EFLOOR);
  } else {
    project(c.u);
  }
  if (c.mode == 1) {
    // the iteration starts from the LI update of (T_d, E_IR), limited like a Newton correction
    int it;
    if constexpr (MIXED) {
      // W-precision view of the updated state: the start values plus the
      // (limited) LI increments; the state takes the LI increment and the
      // Newton corrections in one FP64 add each
      const W lam = damp_factor<W>(S.uf[3], S.uf[4], S.uf[3] * x[3], S.uf[4] * x[4]);
      const W d3 = lam * (S.uf[3] * x[3]), d4 = lam * (S.uf[4] * x[4]);
      const W d2 = S.uf[2] * x[2];
      W a3, a4;
      it = newton_dust_w<W, !MIXED>(a3, a4, S.uf[2] + d2, S.uf[3] + d3, S.uf[4] + d4, d3, d4, S.dTdg + (d3 - d2), dw,
                            c.k, cfg, cw.nr_tol);
      // Newton corrections that are not finite end the cell as a bad
      // substep, with the substep's (limited) LI update of T_d and E_IR in
      // place of the iteration's (the conversions take finite values)
      const bool fin = m_abs(a3) + m_abs(a4) < W(INFINITY);
      c.u[3] = max_bits(u0[3] + to_f64(fin ? d3 + a3 : d3), TCMB);
      c.u[4] = max_bits(u0[4] + to_f64(fin ? d4 + a4 : d4), EFLOOR);
      if (!fin) { c.st |= ST_BADSTEP; return true; }
    } else {
      const double lam = damp_factor<double>(u0[3], u0[4], c.u[3] - u0[3], c.u[4] - u0[4]);
      if (lam < 1.0) {
        c.u[3] = fmax(u0[3] + lam * (c.u[3] - u0[3]), TCMB);
        c.u[4] = fmax(u0[4] + lam * (c.u[4] - u0[4]), EFLOOR);
      }
      it = newton_dust(c.u, u0, dts, c.k, cfg, cw.nr_tol);
    }
    if (it < 0) { c.st |= ST_NOCONV; it = -it; }
    c.nitr += it;
  }
  if constexpr (MIXED) c.t = last ? 0.0 : rem - dts;
  else c.t = last ? dt_h : c.t + dts;
  c.nsub++;
  if (last) return true;
  if (c.nsub >= cfg.n_sub_max) { c.st |= ST_CAP; return true; }
  return false;
}

// H- abundance from the equilibrium of reactions H2 and H3 (unmasked rates)
// at the gas temperature: y_H- = k_H2 y_e / k_H3.  Formed for every finished
// cell by a separate elementwise kernel after the solver (derived.cu): in the
// solver it ran once per finished cell with a few lanes of the warp active,
// code outside the substep loop that also evicted the loop from the
// instruction cache (4 % of the mixed kernel's time, 7 % of the FP64 one's).
template <typename W>
__device__ __forceinline__ double y_hminus(double Tg, double ye) {
  typedef M<W> m;
  const W T = to_w<W>(Tg);
  const W lnT = m::log(T);
  const W k2 = m::exp(W(-41.11005943727161) + W(0.928) * lnT - T * W(1.0 / 16200.0));
  const W N = m::exp(W(0.098493) * lnT) + W(0.32852) * m::exp(W(0.5561) * lnT) +
              W(2.771e-7) * m::exp(W(2.1826) * lnT);
  const W D = W(1) + W(6.191e-3) * m::exp(W(1.0461) * lnT) + W(8.9712e-11) * m::exp(W(3.0424) * lnT) +
              W(3.2576e-14) * m::exp(W(3.7741) * lnT);
  const W k3 = W(1.35e-9) * N / D;
  return to_f64(k2 / k3) * ye;
}

// ------------------------------------------------------------ the kernel

struct KArgs {
  // state (device pointers)
  const double *nH;
  double *Tg, *Td, *E, *y2, *ye, *yH, *yHp, *yHm;
  uint8_t *status;
  int32_t *nsub, *niter;
  const double *G0, *nEUV, *NH2;
  // work: flat (ch_start == nullptr) or a chunk table
  int64_t n_cells;
  double dt;
  int32_t chunk;
  int32_t n_chunks;
  const int64_t *ch_start;
  const int32_t *ch_count;
  const int32_t *ch_block;
  const double *block_dt;
  float *block_cost;
  double cd_factor;
  unsigned long long *counter;
  DevStats *stats;
  DevCfg cfg;
};

// Newton-Raphson attempt (nr_device.cuh), used by the NR instantiation.
__device__ __forceinline__ bool nr_attempt(CellRun<double> &c, const DevCfg &cfg, const CfgW<double> &cw);

// The persistent body.  NR = false: the LI method (Sec. 2.2.8, one substep
// per loop trip); NR = true: the Newton-Raphson reference (one backward-Euler
// attempt per loop trip, FP64).  ALL_ON: an instance for the configuration
// of every production call -- all reactions and processes on, no freeze or
// split flags -- where the mask tests of the rates and the heating and
// cooling terms fold away at compile time (fewer instructions per substep,
// a smaller loop for the instruction cache); RF fixes the refinement variant
// at compile time as well (see li_substep).
template <typename W, bool MIXED, bool NR = false, bool ALL_ON = false, int RF = -1>
__device__ __forceinline__ void li_persistent_body(const KArgs &a) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  DevCfg cfg = a.cfg;
  if constexpr (ALL_ON) {
    cfg.rmask = R_ALL;
    cfg.pmask = P_ALL;
    cfg.flags &= F_REFINE_FF | F_NO_REJECT;
  }
  const CfgW<W> cw = make_cfgw<W>(cfg);
  // warp-uniform chunk cursor
  int64_t cpos = 0, cend = 0;
  int32_t cblock = -1;
  double cdt = a.dt;
  bool exhausted = false;
  // lane state
  bool have = false;
  CellRun<W> c;
  int64_t idx = 0;
  int32_t blk = -1;
  // lane statistics
  unsigned long long s_cells = 0, s_sub = 0, s_newton = 0, s_tight = 0, s_cap = 0, s_noconv = 0,
                     s_bad = 0, s_badstep = 0;
  unsigned int s_max = 0;

  // A lane whose cell is finished stores it and takes a new one in the
  // warp's refill phase; that code runs with only the idle lanes active and
  // lies outside the substep loop, so each pass costs about as much as a
  // substep of the whole warp and evicts the loop from the instruction cache.
  // The mixed kernel therefore lets finished lanes wait (pend) until
  // REFILL_MIN lanes are idle and serves them in one pass.  Measured on the
  // GMC-like grid (the same results bit for bit): with y_H- still formed in
  // the store, waiting for 3 / 4 / 6 / 8 / 12 idle lanes took 5.5 / 7.0 /
  // 7.6 / 6.6 / 1.2 % off the kernel's time; with y_H- formed after the
  // solver (derived.cu), 3 / 4 / 5 / 6 / 8 lanes gave 73.7 / 73.1 / 72.9 /
  // 73.1 / 74.1 ms.  The FP64 kernels spend ~40x longer per substep, so a
  // pass is cheap for them and waiting is not: they refill at once.  All
  // lanes idle always makes a pass, so every finished cell is stored before
  // the warp leaves the loop.
  constexpr int REFILL_MIN = (MIXED && !NR) ? 4 : 1;
  bool pend = false;
  while (true) {
    unsigned need = __ballot_sync(FULL, !have);
    if (__popc(need) < REFILL_MIN && need != FULL) need = 0u;
    if (need != 0u && pend) {
      if constexpr (MIXED && !NR) {
        // the bound y_H2 <= (1 - y_e)/2 not yet applied to the last update
        if (__double_as_longlong(fma(-2.0, c.u[0], 1.0) - c.u[1]) < 0) c.u[0] = (1.0 - c.u[1]) * 0.5;
      }
      a.y2[idx] = c.u[0]; a.ye[idx] = c.u[1]; a.Tg[idx] = c.u[2]; a.Td[idx] = c.u[3]; a.E[idx] = c.u[4];
      if (a.yH) a.yH[idx] = 1.0 - 2.0 * c.u[0] - c.u[1];
      if (a.yHp) a.yHp[idx] = c.u[1];
      if (a.yHm) a.yHm[idx] = 0.0;   // marks a valid cell: y_H- is formed after the solver
      if (a.status) a.status[idx] = c.st;
      if (a.nsub) a.nsub[idx] = c.nsub;
      if (a.niter) a.niter[idx] = c.nitr;
      s_sub += (unsigned long long)c.nsub;
      s_newton += (unsigned long long)c.nitr;
      s_max = max(s_max, (unsigned int)c.nsub);
      if (c.st & ST_TIGHT) s_tight++;
      if (c.st & ST_CAP) s_cap++;
      if (c.st & ST_NOCONV) s_noconv++;
      if (c.st & ST_BADSTEP) s_badstep++;
      if (a.block_cost && blk >= 0) atomicAdd(a.block_cost + blk, (float)c.nsub);
      pend = false;
    }
    while (need != 0u && !exhausted) {
      if (cpos >= cend) {
        unsigned long long ci = 0;
        if (lane == 0) ci = atomicAdd(a.counter, 1ull);
        ci = __shfl_sync(FULL, ci, 0);
        if (ci >= (unsigned long long)a.n_chunks) { exhausted = true; break; }
        if (a.ch_start) {
          cpos = a.ch_start[ci];
          cend = cpos + a.ch_count[ci];
          cblock = a.ch_block[ci];
          cdt = a.block_dt[cblock];
        } else {
          cpos = (int64_t)ci * a.chunk;
          cend = min(cpos + (int64_t)a.chunk, a.n_cells);
        }
        continue;
      }
      const int avail = (int)(cend - cpos);
      const int k = __popc(need);
      const int take = min(k, avail);
      const int rank = __popc(need & lt_mask);
      if (((need >> lane) & 1u) && rank < take) {
        idx = cpos + rank;
        blk = cblock;
        const double n = __ldg(a.nH + idx), G0 = __ldg(a.G0 + idx), nE = __ldg(a.nEUV + idx),
                     NH2 = __ldg(a.NH2 + idx);
        c.u[0] = a.y2[idx]; c.u[1] = a.ye[idx]; c.u[2] = a.Tg[idx]; c.u[3] = a.Td[idx]; c.u[4] = a.E[idx];
        c.t = (MIXED && !NR) ? cdt : 0.0; c.nsub = 0; c.nitr = 0; c.nri = 0; c.ntries = 0; c.st = 0; c.mode = -1;
        s_cells++;
        if (!valid_input(n, c.u[2], c.u[3], c.u[4], c.u[0], c.u[1], G0, nE, NH2, cdt)) {
          c.st = ST_BAD;
          s_bad++;
          if (a.yH) a.yH[idx] = __longlong_as_double(0x7ff8000000000000LL);
          if (a.yHp) a.yHp[idx] = __longlong_as_double(0x7ff8000000000000LL);
          if (a.yHm) a.yHm[idx] = __longlong_as_double(0x7ff8000000000000LL);
          if (a.status) a.status[idx] = ST_BAD;
          if (a.nsub) a.nsub[idx] = 0;
          if (a.niter) a.niter[idx] = 0;
        } else {
          make_cellk<W>(c.k, n, G0, nE, NH2, a.cd_factor, cdt, cfg);
          if constexpr (MIXED) project_bits(c.u);
          else project(c.u);
          have = true;
          if (cdt == 0.0) have = false;   // nothing to integrate: store the projected state
          if (!have) {
            a.y2[idx] = c.u[0]; a.ye[idx] = c.u[1]; a.Tg[idx] = c.u[2]; a.Td[idx] = c.u[3]; a.E[idx] = c.u[4];
            if (a.yH) a.yH[idx] = 1.0 - 2.0 * c.u[0] - c.u[1];
            if (a.yHp) a.yHp[idx] = c.u[1];
            if (a.yHm) a.yHm[idx] = 0.0;   // formed after the solver (derived.cu)
            if (a.status) a.status[idx] = 0;
            if (a.nsub) a.nsub[idx] = 0;
            if (a.niter) a.niter[idx] = 0;
          }
        }
      }
      cpos += take;
      need = __ballot_sync(FULL, !have);
    }
    if (!__any_sync(FULL, have)) break;
    if (have) {
      bool done;
      if constexpr (NR) done = nr_attempt(c, cfg, cw);
      else done = li_substep<W, MIXED, RF>(c, cfg, cw, a.stats);
      if (done) {
        have = false;
        pend = true;
      }
    }
  }
  // statistics: warp reduction, one set of atomics per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s_cells += __shfl_down_sync(FULL, s_cells, o);
    s_sub += __shfl_down_sync(FULL, s_sub, o);
    s_newton += __shfl_down_sync(FULL, s_newton, o);
    s_tight += __shfl_down_sync(FULL, s_tight, o);
    s_cap += __shfl_down_sync(FULL, s_cap, o);
    s_noconv += __shfl_down_sync(FULL, s_noconv, o);
    s_bad += __shfl_down_sync(FULL, s_bad, o);
    s_badstep += __shfl_down_sync(FULL, s_badstep, o);
    s_max = max(s_max, __shfl_down_sync(FULL, s_max, o));
  }
  if (lane == 0 && s_cells) {
    atomicAdd(&a.stats->cells, s_cells);
    atomicAdd(&a.stats->substeps, s_sub);
    if (s_newton) atomicAdd(&a.stats->newton, s_newton);
    if (s_tight) atomicAdd(&a.stats->tight, s_tight);
    if (s_cap) atomicAdd(&a.stats->cap, s_cap);
    if (s_noconv) atomicAdd(&a.stats->noconv, s_noconv);
    if (s_bad) atomicAdd(&a.stats->bad, s_bad);
    if (s_badstep) atomicAdd(&a.stats->badstep, s_badstep);
    atomicMax(&a.stats->max_sub, s_max);
  }
}

}  // namespace sfc
