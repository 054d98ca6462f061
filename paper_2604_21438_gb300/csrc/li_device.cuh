// li_device.cuh -- device-side physics of the linearized-implicit (LI)
// thermochemical update of SFUMATO# (arXiv 2604.21438, Sec. 2.2.8 and
// Appendices A-C), written for one thread per cell with all state in
// registers.
//
// The arithmetic type W of the rates, Jacobian and 5x5 solve is a template
// parameter (double for the FP64 path, float for the mixed path); the cell
// state, the time accounting, the update and the conservation projection are
// always FP64.
//
// Formulation.  With u = (y_H2, y_e, T_g, T_d, E_IR), F the right-hand sides
// and M = diag(1, 1, alpha_g, C_d, 1), one LI substep solves
// (M - dt J) du = dt F (Eq. eq_deq for the two species, Eq. ap_eq:Tg_2 for
// the gas, Eq. ap_eq:Td2 and the IR row of Appendix C for the dust and the
// radiation).  The system is solved in scaled form: unknowns
// x = (dy_H2, dy_e, dT_g/T_g, dT_d/T_d, dE_IR/E_IR) and rows divided by
// (1, 1, alpha_g T_g, C_d T_d, E_IR), so that every diagonal of M becomes 1,
// every entry is a rate in s^-1 and FP32 neither underflows nor loses the
// pivots.  The scaled gas row is (gamma_ad - 1)(Gamma - Lambda)/P, i.e. each
// volumetric heating or cooling term divided by n_H k_B and multiplied by
// hs = (gamma_ad - 1) / (n_tot/n_H T_g).  Derivatives are analytic, written
// by hand term by term (T-derivatives as T dX/dT).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sfc {

// ------------------------------------------------------------------ constants
constexpr double KB = 1.380649e-16;          // erg / K
constexpr double MH = 1.67262192e-24;        // g, hydrogen nucleus
constexpr double EV = 1.602176634e-12;       // erg
constexpr double CLIGHT = 2.99792458e10;     // cm / s
constexpr double CRED = 2.99792458e6;        // reduced light speed 1e-4 c (Sec. 2.1)
constexpr double ARAD = 7.565733250e-15;     // erg cm^-3 K^-4
constexpr double TCMB = 2.725;               // K (z = 0)
constexpr double YHE = 0.0833;               // He per H nucleus
constexpr double MUH = 1.0 + 4.0 * YHE;      // mass per H nucleus in m_H
constexpr double RG = 5.83e-8;               // gas-grain coefficient (App. C)
constexpr double THIGH = 1000.0, TLOW = 75.0;
constexpr double CD_UNIT = 1.0e4;            // C_d = cd_factor * 1e4 erg g^-1 K^-1
constexpr double EFLOOR = 1.0e4 * ARAD * TCMB * TCMB * TCMB * TCMB;  // E_IR with T_IR = T_CMB
// stand-ins for the physics the paper cites without printing it
constexpr double SIG_EUV = 6.3e-18;          // H photoionization cross-section
constexpr double K_LW = 3.3e-11;             // H2 photodissociation per Habing unit
constexpr double NSH0 = 1.0e14, SH_POW = 0.75;
constexpr double ZETA_CR = 1.0e-17;
constexpr double EPI_K = 2.0 * EV / KB;      // photoionization heat per event / k_B
constexpr double EPD_K = 0.4 * EV / KB;      // photodissociation heat per event / k_B
constexpr double EV_K = EV / KB;
constexpr double PE_K = 1.0e-24 * 0.03 / KB; // photoelectric: 1e-24 eps G0 n f_d, eps = 0.03
constexpr double XC = 1.4e-4, TC_S = 91.2, AC = 2.3e-6, GC = 2.0, NCRC = 2.3e-6 / 8.0e-10;
constexpr double XO = 3.2e-4, TO_S = 228.0, AO = 8.9e-5, GO = 0.6, NCRO = 8.9e-5 / 5.0e-10;
constexpr double KAP0 = 0.1, KAPT0 = 10.0, KAPTC = 200.0;
constexpr double SIG_DUV = 1.0e-21, U_HAB = 5.29e-14, HNU_EUV = 18.0 * EV;
constexpr double KGG = MUH * MH / KB;        // rho / (n_H k_B)

// process / reaction / flag bits (same values as the public header)
constexpr uint32_t P_G1 = 1u << 0, P_G2 = 1u << 1, P_G3 = 1u << 2, P_G4 = 1u << 3;
constexpr uint32_t P_L5 = 1u << 4, P_L6 = 1u << 5, P_L7 = 1u << 6, P_L8 = 1u << 7;
constexpr uint32_t P_L9 = 1u << 8, P_L10 = 1u << 9, P_L11 = 1u << 10, P_L12 = 1u << 11;
constexpr uint32_t P_L13 = 1u << 12, P_GG = 1u << 13, P_UV = 1u << 14, P_EMIT = 1u << 15,
                   P_IRABS = 1u << 16;
constexpr uint32_t F_FTG = 1u << 0, F_FTD = 1u << 1, F_FE = 1u << 2, F_FY2 = 1u << 3,
                   F_FYE = 1u << 4, F_SPLIT = 1u << 5, F_REFINE_FF = 1u << 6, F_NO_REJECT = 1u << 7;
constexpr uint32_t R_ALL = (1u << 12) - 1u, P_ALL = (1u << 17) - 1u;   // every reaction / process
constexpr uint8_t ST_CAP = 1, ST_BAD = 2, ST_NOCONV = 4, ST_TIGHT = 8, ST_BADSTEP = 16;

// Solver parameters as the kernels see them.
struct DevCfg {
  double f_chem, Z, gamma_ad, y_floor, nr_tol;
  int32_t n_cyc, n_sub_max, nr_itr_limit;
  uint32_t rmask, pmask, flags;
};

// ------------------------------------------------------- precision wrappers
// FP64 reciprocal estimate of the PTX ISA (rcp.approx.ftz.f64); the FP64
// reciprocal below refines it by Newton-Raphson.
__device__ __forceinline__ double ptx_rcp64(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
template <typename W> struct M;
template <> struct M<double> {
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  // 1/x for finite non-zero x: two Newton-Raphson steps r' = r + r (1 - x r)
  // on the hardware estimate (each squares the relative error), within 1 ulp
  // of the IEEE quotient (tests/test_gpu_math.py), in fewer FP64 pipe slots
  // than the IEEE division: the FP64 kernels are bound by that pipe and take
  // ~30 reciprocals per substep.  0 and infinities are not handled.
  static __device__ __forceinline__ double rcp(double x) {
    double r = ptx_rcp64(x);
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
  }
  static __device__ __forceinline__ double abs(double x) { return ::fabs(x); }
};
// FP32 (mixed path): the hardware approximations of the PTX ISA (ex2, lg2,
// rcp, sqrt .approx.ftz) with the corrections below, instead of the IEEE
// division and the full-range libm sequences, whose code more than tripled
// the kernel's size and left a third of its instruction fetches missing the
// instruction cache.  Accuracy, checked against CUDA's expf, logf, 1/x and
// sqrtf by tests/test_gpu_math.py: exp within 4 ulp on [-87, 88]; log within
// 4 ulp for x >= 2.7 (it is only taken of temperatures >= T_CMB, where
// ln x >= 1 and the absolute error bound of lg2.approx is also a relative
// one); rcp and sqrt within 1 ulp.  Results below the FP32 normal range
// flush to zero.
__device__ __forceinline__ float ptx_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ptx_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ptx_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ptx_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <> struct M<float> {
  // exp(x) = 2^h 2^e with h = fl(x log2 e) and e its error: the rounding
  // error of the product, exact by one FMA (the FMA form of Dekker's exact
  // product), plus x times the part of log2 e that a float drops.  2^e is
  // taken to first order (|e| < 2^-17); e is clamped so that x = -inf gives
  // 0, and an overflowed 2^h is returned as it is.
  static __device__ __forceinline__ float exp(float x) {
    const float L2E = 1.44269502f, L2E_TAIL = 1.92596299e-8f;   // log2 e = L2E + L2E_TAIL
    const float h = x * L2E;
    const float e = fmaf(x, L2E, -h) + x * L2E_TAIL;
    const float p = ptx_ex2(h);
    const float q = fmaf(p, fminf(fmaxf(e, -1.0f), 1.0f) * 0.693147181f, p);
    return p < __int_as_float(0x7f800000) ? q : p;
  }
  static __device__ __forceinline__ float log(float x) { return ptx_lg2(x) * 0.693147181f; }
  static __device__ __forceinline__ float log1p(float x) { return ::log1pf(x); }
  static __device__ __forceinline__ float sqrt(float x) { return ptx_sqrt(x); }
  // one Newton-Raphson step r' = r + r (1 - x r) on the hardware estimate
  static __device__ __forceinline__ float rcp(float x) {
    const float r = ptx_rcp(x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
  }
  static __device__ __forceinline__ float abs(float x) { return ::fabsf(x); }
};

// ------------------------------------------------ FP32 <-> FP64 conversions
// On GB300 the FP64 pipe issues 2 instructions per clock per SM against 128
// FP32/INT lanes, and hardware float<->double conversions run on the FP64
// pipe.  The mixed path converts often (state in, increments and residuals
// out), so it converts with integer operations on the exponent and mantissa
// bits instead.  f2d: exact for normal numbers and zeros; FP32 subnormals
// (|x| < 1.2e-38) become signed zeros; inf and NaN are kept.  d2f: rounds to
// nearest (ties away from zero); results below the FP32 normal range become
// signed zeros, above it signed infinities; NaN stays NaN.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t u = __float_as_uint(f), a = u & 0x7fffffffu;
  const bool tiny = a < 0x00800000u;                                // zero or subnormal
  // exponent and mantissa shifted into place, the exponent rebiased 127 -> 1023
  // (255 -> 2047 for inf and NaN)
  uint32_t hi = (a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u);
  hi = (tiny ? 0u : hi) | (u & 0x80000000u);
  const uint32_t lo = tiny ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_int(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t a = hi & 0x7fffffffu;
  // exponent and the top 23 mantissa bits, rebiased 1023 -> 127 modulo 2^32
  // (exact inside the FP32 normal range), plus the rounding bit; a carry
  // rounds into the exponent
  uint32_t bits = ((a << 3) | (lo >> 29)) + 0x40000000u + ((lo >> 28) & 1u);
  bits = (a < 0x38100000u) ? 0u : bits;                             // below the normal range
  bits = (a >= 0x47f00000u) ? 0x7f800000u : bits;                   // above it (and inf, NaN)
  bits |= hi & 0x80000000u;
  bits = (a > 0x7ff00000u || (a == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : bits;
  return __uint_as_float(bits);
}
// The same conversions for finite values: no infinity or NaN case (an
// infinity or NaN converts to a finite or infinite value of no meaning).  The
// substep loop converts only finite values -- a solve or Newton correction
// that is not finite ends the cell as a bad substep before it reaches the
// state -- and with the two cases gone the hot loop runs 9 % faster (about 36
// conversions per substep, each on a dependency chain).  f2d_fin shifts the
// sign, exponent and mantissa together (an arithmetic shift keeps the sign
// bit in place once the three copies of it below are masked off) and rebiases
// the exponent only when it is non-zero: exact for normal numbers and signed
// zeros; an FP32 subnormal m 2^-149 becomes the FP64 subnormal m 2^-1045 of
// the same sign (below 2^-1022: zero for every use here).  Four integer
// instructions fewer than f2d_int, 1.5 % of the mixed kernel's time.
__device__ __forceinline__ double f2d_fin(float f) {
  const uint32_t u = __float_as_uint(f);
  const bool tiny = (u & 0x7fffffffu) < 0x00800000u;                // zero or subnormal
  const uint32_t hi = (uint32_t)(((int32_t)u >> 3) & (int32_t)0x8fffffff) + (tiny ? 0u : 0x38000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ float d2f_fin(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t a = hi & 0x7fffffffu;
  uint32_t bits = ((a << 3) | (lo >> 29)) + 0x40000000u + ((lo >> 28) & 1u);
  bits = (a < 0x38100000u) ? 0u : bits;                             // below the normal range
  bits = (a >= 0x47f00000u) ? 0x7f800000u : bits;                   // above it
  return __uint_as_float(bits | (hi & 0x80000000u));
}
// W-precision views of FP64 values and FP64 views of W values in the
// substep loop (finite values; FP64 path: identity)
template <typename W> __device__ __forceinline__ W to_w(double d);
template <> __device__ __forceinline__ double to_w<double>(double d) { return d; }
template <> __device__ __forceinline__ float to_w<float>(double d) { return d2f_fin(d); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_fin(x); }

// a / b as a times the refined reciprocal in both precisions (within 2 ulp
// of the IEEE quotient, and a fraction of the instructions of an IEEE
// division), for b > 0 finite
__device__ __forceinline__ double div_w(double a, double b) { return a * M<double>::rcp(b); }
__device__ __forceinline__ float div_w(float a, float b) { return a * M<float>::rcp(b); }

__device__ __forceinline__ double fmax_w(double a, double b) { return ::fmax(a, b); }
__device__ __forceinline__ float fmax_w(float a, float b) { return ::fmaxf(a, b); }
// 2^-n for 0 <= n <= 126, built from the exponent field (exact)
template <typename W> __device__ __forceinline__ W pow2_neg(int n);
template <> __device__ __forceinline__ double pow2_neg<double>(int n) {
  return __longlong_as_double((long long)(1023 - n) << 52);
}
template <> __device__ __forceinline__ float pow2_neg<float>(int n) { return __int_as_float((127 - n) << 23); }
// x 2^-n for a positive double whose exponent field exceeds n (a substep
// length: at least the smallest FP32 subnormal, with n <= 30), by taking n
// from the exponent field: exact, and integer instructions only.
__device__ __forceinline__ double scale_pow2_neg(double x, int n) {
  return __longlong_as_double(__double_as_longlong(x) - ((long long)n << 52));
}

// ----------------------------------------------------------- per-cell inputs
// Quantities a cell keeps over one call, computed once in FP64 and held in
// the arithmetic type W of the rates (so the substep loop converts nothing).
template <typename W> struct CellK {
  W n, rho, fd, Cd, EUV, k9, k10, k11, Gpre, pe;
  W lnn, rn, rCd;    // ln n_H, 1/n_H, 1/C_d
  double dt_h;
};

template <typename W>
__device__ __forceinline__ void make_cellk(CellK<W> &c, double n, double G0, double nEUV, double NH2,
                                           double cd_factor, double dt_h, const DevCfg &cfg) {
  if constexpr (sizeof(W) == sizeof(float)) {
    // Mixed path: the same constants in FP32 from the rounded inputs.  A lane
    // computes them alone when its warp refills it with a new cell, and an
    // FP64 warp instruction occupies the FP64 pipe whatever its number of
    // active lanes: in FP64 these ~160 instructions per cell cost more pipe
    // time than the substeps of a cell that needs a few dozen.
    typedef M<float> m;
    const float nf = d2f_int(n), G0f = d2f_int(G0), nEf = d2f_int(nEUV), NH2f = d2f_int(NH2);
    const float Z = d2f_int(cfg.Z), Cd = d2f_int(cd_factor) * float(CD_UNIT);
    c.n = nf;
    c.rho = nf * float(MUH * MH);
    c.fd = Z;
    c.Cd = Cd;
    c.EUV = (cfg.pmask & P_UV) ? float(CLIGHT * (SIG_DUV / (MUH * MH))) * (G0f * float(U_HAB) + nEf * float(HNU_EUV))
                               : 0.0f;
    c.k9 = ((cfg.rmask >> 9) & 1u) ? float(CLIGHT * SIG_EUV) * nEf : 0.0f;
    // (N_H2 / N_0)^-3/4 as 1 / (sqrt(x) sqrt(sqrt(x))): a few ulp, where
    // exp(-0.75 ln x) would carry the rounding of ln x (up to 5e-7)
    static_assert(SH_POW == 0.75, "the FP32 shielding factor assumes the exponent 3/4");
    const float xs = NH2f * float(1.0 / NSH0), sq = m::sqrt(xs);
    const float fsh = NH2f > float(NSH0) ? m::rcp(sq * m::sqrt(sq)) : 1.0f;
    c.k10 = ((cfg.rmask >> 10) & 1u) ? float(K_LW) * G0f * fsh : 0.0f;
    c.k11 = ((cfg.rmask >> 11) & 1u) ? float(ZETA_CR) : 0.0f;
    c.Gpre = (cfg.pmask & P_GG) ? nf * float(RG * 0.031622776601683794) : 0.0f;   // RG n / sqrt(T_high)
    c.pe = (cfg.pmask & P_G4) ? float(PE_K) * G0f * Z : 0.0f;
    c.lnn = m::log(nf);
    c.rn = m::rcp(nf);
    c.rCd = m::rcp(Cd);
    c.dt_h = dt_h;
    return;
  }
  c.n = W(n);
  c.rho = W(MUH * MH * n);
  c.fd = W(cfg.Z);
  c.Cd = W(cd_factor * CD_UNIT);
  c.EUV = (cfg.pmask & P_UV) ? W(CLIGHT * (SIG_DUV / (MUH * MH)) * (G0 * U_HAB + nEUV * HNU_EUV)) : W(0);
  c.k9 = ((cfg.rmask >> 9) & 1u) ? W(CLIGHT * SIG_EUV * nEUV) : W(0);
  const double fsh = NH2 > NSH0 ? ::exp(-SH_POW * ::log(NH2 / NSH0)) : 1.0;
  c.k10 = ((cfg.rmask >> 10) & 1u) ? W(K_LW * G0 * fsh) : W(0);
  c.k11 = ((cfg.rmask >> 11) & 1u) ? W(ZETA_CR) : W(0);
  c.Gpre = (cfg.pmask & P_GG) ? W(RG * n / ::sqrt(THIGH)) : W(0);
  c.pe = (cfg.pmask & P_G4) ? W(PE_K * G0 * cfg.Z) : W(0);
  c.lnn = W(::log(n));
  c.rn = W(1.0 / n);
  c.rCd = W(1.0 / (cd_factor * CD_UNIT));
  c.dt_h = dt_h;
}

// Solver parameters in the arithmetic type W.
template <typename W> struct CfgW {
  W f_chem, y_floor, gm1, nr_tol, ncyc_fchem;
};
template <typename W> __device__ __forceinline__ CfgW<W> make_cfgw(const DevCfg &d) {
  CfgW<W> w;
  w.f_chem = W(d.f_chem);
  w.y_floor = W(d.y_floor);
  w.gm1 = W(d.gamma_ad - 1.0);
  w.nr_tol = W(d.nr_tol);
  w.ncyc_fchem = W(double(d.n_cyc) * d.f_chem);
  return w;
}

// ------------------------------------------------- Table 3 rate coefficients
// k[i] = k_H<i>, kT[i] = T_g dk_H<i>/dT_g; k8d = T_d dk_H8/dT_d.
template <typename W> struct Rates {
  W k[12], kT[12], k8d;
};

// Powers and reciprocals of T_g and T_d shared by the rate and cooling terms.
template <typename W> struct Pre {
  W lnT, lnT4, rT, sqT, rsqT, rTd;   // lnT4 = ln(T / 1e4), accurate near 1e4 K
};

// FP32: ln T is taken relative to 1e4 K, through log1p near it: the rates
// that matter in ionized gas (H0, H1) are steep in T, and the absolute
// rounding of ln T ~ 9.5 (half an ulp is 4.8e-7 in FP32) would move them by
// up to |d ln k / d ln T| x 4.8e-7 (13.5 x for collisional ionization near
// its threshold).  FP64 has the digits to spare and takes ln T directly.
template <typename W>
__device__ __forceinline__ void make_pre(W T, W Td, Pre<W> &q) {
  typedef M<W> m;
  if constexpr (sizeof(W) == sizeof(double)) {
    q.lnT = m::log(T);
    q.lnT4 = q.lnT - W(9.210340371976184);
  } else {
    const W t = T * W(1e-4);
    q.lnT4 = (t > W(0.5) && t < W(2)) ? m::log1p(t - W(1)) : m::log(t);
    q.lnT = q.lnT4 + W(9.210340371976184);
  }
  q.rT = m::rcp(T);
  q.sqT = m::sqrt(T);
  q.rsqT = m::rcp(q.sqT);
  q.rTd = m::rcp(Td);
}

template <typename W>
__device__ __forceinline__ void eval_rates(W T, W Td, const Pre<W> &q, const CellK<W> &c, uint32_t rmask,
                                           Rates<W> &r) {
  typedef M<W> m;
  const W lnT = q.lnT, lnT4 = q.lnT4, rT = q.rT;
  // H0: Abel et al. fit in ln T(eV)
  {
    const W x = lnT4 - W(0.14880786093196532);  // ln(T / 11604.5)
    // a0 = -32.71396786 enters as exp(a0), outside the exponential below
    const W a1 = W(13.536556), a2 = W(-5.73932875), a3 = W(1.563154998),
            a4 = W(-0.2877056), a5 = W(3.48255977e-2), a6 = W(-2.63197617e-3),
            a7 = W(1.11954395e-4), a8 = W(-2.03914985e-6);
    W p = a8;
    p = p * x + a7; p = p * x + a6; p = p * x + a5; p = p * x + a4;
    p = p * x + a3; p = p * x + a2; p = p * x + a1; p = p * x;   // minus a0
    W dp = W(8) * a8;
    dp = dp * x + W(7) * a7; dp = dp * x + W(6) * a6; dp = dp * x + W(5) * a5;
    dp = dp * x + W(4) * a4; dp = dp * x + W(3) * a3; dp = dp * x + W(2) * a2; dp = dp * x + a1;
    r.k[0] = W(6.201607514089056e-15) * m::exp(p);   // exp(a0) exp(p - a0): p - a0 is small near 1e4 K
    r.kT[0] = r.k[0] * dp;
  }
  // H1: case-B recombination
  {
    const W X = m::exp(W(0.407) * (W(2.4439804831753538) - lnT4));      // (115188/T)^0.407
    // the constant part of ln k taken out of the exponential (e^-26.0456)
    r.k[1] = W(4.881357330013074e-12) * m::exp(W(-1.5) * lnT4 - W(2.242) * m::log1p(X));
    r.kT[1] = r.k[1] * (W(-1.5) + W(2.242 * 0.407) * X * m::rcp(W(1) + X));
  }
  // H2: H- formation
  {
    r.k[2] = m::exp(W(-41.11005943727161) + W(0.928) * lnT - T * W(1.0 / 16200.0));
    r.kT[2] = r.k[2] * (W(0.928) - T * W(1.0 / 16200.0));
  }
  // H3: associative detachment
  {
    const W e1 = m::exp(W(0.098493) * lnT), e2 = m::exp(W(0.5561) * lnT), e3 = m::exp(W(2.1826) * lnT);
    const W e4 = m::exp(W(1.0461) * lnT), e5 = m::exp(W(3.0424) * lnT), e6 = m::exp(W(3.7741) * lnT);
    const W N = e1 + W(0.32852) * e2 + W(2.771e-7) * e3;
    const W NT = W(0.098493) * e1 + W(0.32852 * 0.5561) * e2 + W(2.771e-7 * 2.1826) * e3;
    const W D = W(1) + W(6.191e-3) * e4 + W(8.9712e-11) * e5 + W(3.2576e-14) * e6;
    const W DT = W(6.191e-3 * 1.0461) * e4 + W(8.9712e-11 * 3.0424) * e5 + W(3.2576e-14 * 3.7741) * e6;
    const W rD = m::rcp(D);
    r.k[3] = W(1.35e-9) * N * rD;
    r.kT[3] = r.k[3] * (NT * m::rcp(N) - DT * rD);
  }
  // H5: three-body formation (T^-1/4 = sqrt(T^-1/2)); H6 = H5 / 8
  {
    const W eb = q.rsqT, ea = m::sqrt(q.rsqT);
    r.k[5] = W(6e-32) * ea + W(2e-31) * eb;
    r.kT[5] = W(-0.25 * 6e-32) * ea - W(0.5 * 2e-31) * eb;
    r.k[6] = r.k[5] * W(0.125);
    r.kT[6] = r.kT[5] * W(0.125);
  }
  // H7: k_high^(1-a) k_low^a with a = 1/(1 + n/n_cr); H4 stand-in: the same function
  {
    const W L = (lnT - W(9.210340371976184)) * W(0.4342944819032518);     // log10(T/1e4)
    const W lnncr = W(2.302585092994046) * (W(4.845) - W(1.3) * L + W(1.62) * L * L);
    const W a = m::rcp(W(1) + m::exp(c.lnn - lnncr));
    const W ln_klow = W(-22.860336491462885) - W(6.95e4) * rT;  // ln 1.18e-10
    const W x = W(6000.0) * rT;
    const W em = m::exp(-x);
    const W ln_khigh = W(-16.325735015736566) - W(0.5) * lnT - W(5.2e4) * rT + m::log1p(-em);  // ln 8.125e-8
    const W lnk = (W(1) - a) * ln_khigh + a * ln_klow;
    const W k7 = m::exp(lnk);
    const W dkh = W(-0.5) + W(5.2e4) * rT - x * em * m::rcp(W(1) - em);
    const W dkl = W(6.95e4) * rT;
    const W da = a * (W(1) - a) * (W(-1.3) + W(3.24) * L);
    const W kT7 = k7 * ((W(1) - a) * dkh + a * dkl + (ln_klow - ln_khigh) * da);
    r.k[7] = k7; r.kT[7] = kT7;
    r.k[4] = k7; r.kT[4] = kT7;
  }
  // H8: grain-surface formation
  {
    const W s = m::sqrt(T + Td);
    const W rs = m::rcp(s);
    const W B = W(1) + W(4e-2) * s + W(2e-3) * T + W(8e-6) * T * T;
    const W rB = m::rcp(B);
    const W ez = m::exp(W(750.0) * (W(1.0 / 75.0) - q.rTd));
    const W fa = m::rcp(W(1) + ez);
    const W om = ez * fa;                                         // 1 - f_a
    const W k8 = W(6e-17 * 0.057735026918962584) * q.sqT * fa * c.fd * rB;   // sqrt(T/300)
    r.k[8] = k8;
    r.kT[8] = k8 * (W(0.5) - T * (W(0.02) * rs + W(2e-3) + W(1.6e-5) * T) * rB);
    r.k8d = k8 * (-om * W(750.0) * q.rTd - Td * W(0.02) * rs * rB);
  }
  r.k[9] = c.k9; r.kT[9] = W(0);
  r.k[10] = c.k10; r.kT[10] = W(0);
  r.k[11] = c.k11; r.kT[11] = W(0);
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (!((rmask >> i) & 1u)) { r.k[i] = W(0); r.kT[i] = W(0); }
  if (!((rmask >> 8) & 1u)) r.k8d = W(0);
}

// ----------------------------------------- reaction rates R_i (Eq. eq_chemq)
// R_H2 = k2 n yH ye + k5 n^2 yH^3 + k6 n^2 yH^2 y2 + k8 n yH - k4 n yH y2 - k7 n y2^2 - k10 y2
// R_e  = k0 n yH ye + (k9 + k11) yH - k1 n ye^2
// (H- in equilibrium between reactions H2 and H3: the H- channel forms H2 at
// k2 n yH ye and returns the electron; yH = 1 - 2 y2 - ye, y_H+ = ye.)
// J0/J1: d/dy2, d/dye, T d/dT, Td d/dTd (the last two only when withT).
template <typename W>
__device__ __forceinline__ void chem_rows(const Rates<W> &r, W n, W y2, W ye, W yH, bool via_on, W &F0, W &F1,
                                          W J0[4], W J1[4], bool withT) {
  const W k2v = via_on ? r.k[2] : W(0), k2Tv = via_on ? r.kT[2] : W(0);
  const W n2 = n * n;
  const W yH2sq = yH * yH;
  const W g1 = k2v * n, g5 = r.k[5] * n2, g6 = r.k[6] * n2, g8 = r.k[8] * n, g4 = r.k[4] * n,
          g7 = r.k[7] * n;
  F0 = g1 * yH * ye + g5 * yH2sq * yH + g6 * yH2sq * y2 + g8 * yH - g4 * yH * y2 - g7 * y2 * y2 - r.k[10] * y2;
  // d/dy2 (dyH/dy2 = -2)
  J0[0] = W(-2) * g1 * ye - W(6) * g5 * yH2sq + g6 * (yH2sq - W(4) * yH * y2) - W(2) * g8 -
          g4 * (yH - W(2) * y2) - W(2) * g7 * y2 - r.k[10];
  // d/dye (dyH/dye = -1)
  J0[1] = g1 * (yH - ye) - W(3) * g5 * yH2sq - W(2) * g6 * yH * y2 - g8 + g4 * y2;
  const W g0 = r.k[0] * n, g1r = r.k[1] * n, gp = r.k[9] + r.k[11];
  F1 = g0 * yH * ye + gp * yH - g1r * ye * ye;
  J1[0] = W(-2) * (g0 * ye + gp);
  J1[1] = g0 * (yH - ye) - gp - W(2) * g1r * ye;
  if (withT) {
    J0[2] = (k2Tv * n) * yH * ye + (r.kT[5] * n2) * yH2sq * yH + (r.kT[6] * n2) * yH2sq * y2 +
            (r.kT[8] * n) * yH - (r.kT[4] * n) * yH * y2 - (r.kT[7] * n) * y2 * y2;
    J0[3] = (r.k8d * n) * yH;
    J1[2] = (r.kT[0] * n) * yH * ye - (r.kT[1] * n) * ye * ye;
    J1[3] = W(0);
  }
}

// --------------------------------------------------------- scaled system
// F[i]: scaled right-hand side (s^-1); J[i][j]: scaled Jacobian (s^-1),
// entry (i, j) = (dF_i/du_j) c_j / r_i.  rate_dust / rate_chem / rate_energy:
// inverse timescales of Eqs. timescale_of_dust, timescale_chemi,
// timescale_energy (zero when the quantity is frozen or inert).
template <typename W> struct Sys {
  W J[5][5];
  W F[5];
  W rate_dust, rate_chem, rate_energy;
  W H;   // (Gamma - Lambda) / (n_H k_B), gas-grain transfer included, unscaled
  W uf[5];   // the state as seen by this evaluation (rounded to W)
  W uyH;     // y_H = 1 - 2 y_H2 - y_e, formed in FP64 and rounded to W
  W dTdg;    // T_d - T_g, formed in FP64 and rounded to W
};

__device__ __forceinline__ double kappa_d(double T) {
  return T < KAPTC ? KAP0 * (T / KAPT0) * (T / KAPT0) : KAP0 * (KAPTC / KAPT0) * (KAPTC / KAPT0);
}

template <typename W>
__device__ __forceinline__ W kappa_w(W T, W &beta_emit, W &beta_abs) {
  // kappa_d^0(T) = kappa0 (T/T0)^2 below 200 K, constant above (stand-in);
  // beta_emit = 4 kappa + T kappa' (Eq. ap_eq:beta_d),
  // beta_abs = kappa + T kappa' / 4 (Eq. ap_eq:beta_IR)
  W k;
  if (T < W(KAPTC)) {
    const W q = T * W(1.0 / KAPT0);
    k = W(KAP0) * q * q;
    beta_emit = W(6) * k;
    beta_abs = W(1.5) * k;
  } else {
    k = W(KAP0 * (KAPTC / KAPT0) * (KAPTC / KAPT0));
    beta_emit = W(4) * k;
    beta_abs = k;
  }
  return k;
}

template <typename W>
__device__ __forceinline__ void eval_system(const double u[5], double yH64, const CellK<W> &c, const DevCfg &cfg,
                                            const CfgW<W> &cw, Sys<W> &S) {
  typedef M<W> m;
  const W y2 = to_w<W>(u[0]), ye = to_w<W>(u[1]), T = to_w<W>(u[2]), Td = to_w<W>(u[3]), E = to_w<W>(u[4]);
  S.uf[0] = y2; S.uf[1] = ye; S.uf[2] = T; S.uf[3] = Td; S.uf[4] = E;
  const W n = c.n;
  const uint32_t pm = cfg.pmask, fl = cfg.flags;
  Pre<W> q;
  make_pre<W>(T, Td, q);
  const W rT = q.rT;
  Rates<W> r;
  eval_rates<W>(T, Td, q, c, cfg.rmask, r);
  // differences that cancel are taken in FP64 and rounded once: y_H near 0
  // (fully molecular or ionized gas; yH64 = 1 - 2 y_H2 - y_e, formed by the
  // caller) and T_d - T_g in tight gas-dust coupling
  const W yH = to_w<W>(yH64);
  S.uyH = yH;
  const W dTdg = to_w<W>(u[3] - u[2]);
  S.dTdg = dTdg;
  const bool via_on = ((cfg.rmask >> 2) & 1u) && ((cfg.rmask >> 3) & 1u);

  // ---- chemistry rows (Eq. eq_deq): R and partials
  const W k2v = via_on ? r.k[2] : W(0), k2Tv = via_on ? r.kT[2] : W(0);
  const W n2 = n * n;
  const W yH2sq = yH * yH;
  {
    W F0, F1, J0[4], J1[4];
    chem_rows<W>(r, n, y2, ye, yH, via_on, F0, F1, J0, J1, true);
    S.F[0] = F0;
    S.F[1] = F1;
#pragma unroll
    for (int j = 0; j < 4; ++j) { S.J[0][j] = J0[j]; S.J[1][j] = J1[j]; }
    S.J[0][4] = W(0);
    S.J[1][4] = W(0);
  }

  // ---- gas row: H = (Gamma - Lambda) / (n k_B), then scaled by hs
  W H = W(0), H0 = W(0), H1 = W(0), H2 = W(0), H3h = W(0);  // value, d/dy2, d/dye, T d/dT, Td d/dTd
  // generic term C(T) P(y): add value, C P_y2, C P_ye, C_T P
#define SFC_TERM(C, CT, P, Py2, Pye) \
  { const W c_ = (C), p_ = (P); H += c_ * p_; H0 += c_ * (Py2); H1 += c_ * (Pye); H2 += (CT) * p_; }
  if (pm & P_G1) {
    const W q1 = W(400) * rT;
    const W e1 = m::exp(-q1 * q1);
    const W r12 = m::rcp(T + W(1200));
    const W e2 = m::exp(W(-12000) * r12);
    const W Dn = W(1.6) * yH * e1 + W(1.4) * y2 * e2;
    const W Dy2 = W(-3.2) * e1 + W(1.4) * e2, Dye = W(-1.6) * e1;
    const W DT = W(1.6) * yH * e1 * (W(2) * q1 * q1) + W(1.4) * y2 * e2 * (W(12000) * T * r12 * r12);
    const W qq = W(1e6) * q.rsqT;
    const W rden = m::rcp(n * Dn + qq);
    const W f = n * Dn * rden;
    const W fD = n * qq * rden * rden;                          // df/dDn
    const W fy2 = fD * Dy2, fye = fD * Dye;
    const W fT = (n * qq * DT + W(0.5) * n * Dn * qq) * rden * rden;  // T df/dT
    const W gA = k2v * n * yH * ye;                              // H- channel per n
    const W gAy2 = k2v * n * (W(-2) * ye), gAye = k2v * n * (yH - ye), gAT = k2Tv * n * yH * ye;
    const W gB = r.k[5] * n2 * yH2sq * yH;
    const W gBy2 = r.k[5] * n2 * W(-6) * yH2sq, gBye = r.k[5] * n2 * W(-3) * yH2sq,
            gBT = r.kT[5] * n2 * yH2sq * yH;
    const W gC = r.k[8] * n * yH;
    const W gCy2 = r.k[8] * n * W(-2), gCye = -r.k[8] * n, gCT = r.kT[8] * n * yH, gCd = r.k8d * n * yH;
    const W ce = W(EV_K);
    H += ce * (W(3.73) * f * gA + W(4.48) * f * gB + (W(0.2) + W(4.2) * f) * gC);
    H0 += ce * (W(3.73) * (fy2 * gA + f * gAy2) + W(4.48) * (fy2 * gB + f * gBy2) + W(4.2) * fy2 * gC +
                (W(0.2) + W(4.2) * f) * gCy2);
    H1 += ce * (W(3.73) * (fye * gA + f * gAye) + W(4.48) * (fye * gB + f * gBye) + W(4.2) * fye * gC +
                (W(0.2) + W(4.2) * f) * gCye);
    H2 += ce * (W(3.73) * (fT * gA + f * gAT) + W(4.48) * (fT * gB + f * gBT) + W(4.2) * fT * gC +
                (W(0.2) + W(4.2) * f) * gCT);
    H3h += ce * (W(0.2) + W(4.2) * f) * gCd;
  }
  if (pm & P_G2) SFC_TERM(W(EPI_K) * r.k[9], W(0), yH, W(-2), W(-1));
  if (pm & P_G3) SFC_TERM(W(EPD_K) * r.k[10], W(0), y2, W(1), W(0));
  if (pm & P_G4) { H += c.pe; }
  if (pm & P_L5) SFC_TERM(W(-13.6 * EV_K) * r.k[0] * n, W(-13.6 * EV_K) * r.kT[0] * n, yH * ye,
                          W(-2) * ye, yH - ye);
  if (pm & P_L6) {
    SFC_TERM(W(-4.48 * EV_K) * r.k[4] * n, W(-4.48 * EV_K) * r.kT[4] * n, y2 * yH, yH - W(2) * y2, -y2);
    SFC_TERM(W(-4.48 * EV_K) * r.k[7] * n, W(-4.48 * EV_K) * r.kT[7] * n, y2 * y2, W(2) * y2, W(0));
  }
  const W lnT = q.lnT;
  const W L10 = lnT * W(0.4342944819032518);
  if (pm & P_L7) {
    W p = W(5.491e-4);
    p = p * L10 + W(-9.165e-3); p = p * L10 + W(0.04264); p = p * L10 + W(-0.1052);
    p = p * L10 + W(0.4958); p = p * L10 + W(-25.87);
    W dp = W(5 * 5.491e-4);
    dp = dp * L10 + W(4 * -9.165e-3); dp = dp * L10 + W(3 * 0.04264); dp = dp * L10 + W(2 * -0.1052);
    dp = dp * L10 + W(0.4958);
    const W C = -m::exp(W(2.302585092994046) * p + W(36.51880780943216)) * n;  // 10^p / k_B
    SFC_TERM(C, C * dp, ye * ye, W(0), W(2) * ye);
  }
  if (pm & P_L8) SFC_TERM(-T * k2v * n, -T * (k2v + k2Tv) * n, yH * ye, W(-2) * ye, yH - ye);
  const W sq5 = q.sqT * W(0.0031622776601683794);               // sqrt(T / 1e5)
  const W r1s = m::rcp(W(1) + sq5);
  if (pm & P_L9) {
    const W C = W(-7.50e-19 / KB) * n * m::exp(W(-118348) * rT) * r1s;
    SFC_TERM(C, C * (W(118348) * rT - W(0.5) * sq5 * r1s), ye * yH, W(-2) * ye, yH - ye);
  }
  if (pm & P_L10) {
    const W C = W(-5.54e-17 / KB * YHE) * n * m::exp(W(-0.397) * lnT - W(473638) * rT) * r1s;
    SFC_TERM(C, C * (W(-0.397) + W(473638) * rT - W(0.5) * sq5 * r1s), ye, W(0), W(1));
  }
  if (pm & P_L11) {
    const bool lo = T < W(3.2e5);
    const W gff = lo ? W(0.79464) + W(0.1243) * L10 : W(2.13164) - W(0.1240) * L10;
    const W gT = lo ? W(0.1243 * 0.4342944819032518) : W(-0.1240 * 0.4342944819032518);
    const W b = W(-1.426e-27 / KB) * n * q.sqT;
    SFC_TERM(b * gff, b * (W(0.5) * gff + gT), ye * ye, W(0), W(2) * ye);
  }
  if (pm & P_L12) {
    const W b = W(-1.017e-37 * TCMB * TCMB * TCMB * TCMB / KB);
    SFC_TERM(b * (T - W(TCMB)), b * T, ye, W(0), W(1));
  }
  if (pm & P_L13) {
    const W fd = c.fd;
    const W wC = W(GC) * m::exp(W(-TC_S) * rT), cC = W(NCRC) * c.rn;
    const W wO = W(GO) * m::exp(W(-TO_S) * rT), cO = W(NCRO) * c.rn;
    const W KC = W(XC * TC_S * AC) * fd, KO = W(XO * TO_S * AO) * fd;
    const W rC = m::rcp(W(1) + wC + cC), rO = m::rcp(W(1) + wO + cO);
    const W val = -(KC * wC * rC + KO * wO * rO);
    const W valT = -(KC * wC * (W(TC_S) * rT) * (W(1) + cC) * rC * rC +
                     KO * wO * (W(TO_S) * rT) * (W(1) + cO) * rO * rO);
    H += val; H2 += valT;
  }
#undef SFC_TERM
  // dust-side quantities (Appendix C)
  W be_d, ba_d, be_i, ba_i;
  const W kd = kappa_w<W>(Td, be_d, ba_d);
  const W TIR = m::sqrt(m::sqrt(W(1e-4 / ARAD) * E));          // a T_IR^4 = (c~/c) E_IR
  const W ki = kappa_w<W>(TIR, be_i, ba_i);
  const W acTd3 = W(ARAD * CLIGHT) * Td * Td * Td;
  const bool on_emit = pm & P_EMIT, on_abs = pm & P_IRABS;
  const W emit = on_emit ? kd * acTd3 * Td : W(0);
  const W irabs = on_abs ? ki * W(CRED) * E : W(0);
  const W beta_d = on_emit ? be_d : W(0);
  const W beta_IR = on_abs ? ba_i : W(0);
  const W G = c.Gpre * q.sqT;
  const W gam = W(1) - W(0.8) * m::exp(W(-TLOW) * rT);
  const W rr = dTdg * rT;                                        // T_d/T_g - 1
  const W zeta = gam * W(0.5) * rr + (gam - W(1)) * W(TLOW) * rT * rr - gam;
  const W gg = G * gam * dTdg;                                   // R_g n sqrt(T/T_high) gamma_d (T_d - T_g)
  const W fd = c.fd;
  // gas-grain transfer in the gas row (Eq. ap_eq:Tg, the gamma_d and zeta terms of Eq. ap_eq:Tg_2)
  const W Hgg = W(KGG) * fd * gg;
  H += Hgg;
  H2 += W(KGG) * fd * G * zeta * T;
  const W Hgg_d = W(KGG) * fd * G * gam * Td;
  // scale of the gas row: hs = (gamma_ad - 1) / (ntot/n_H T_g), fixed over the substep
  const W ytot = W(1) - y2 + ye + W(YHE);
  const W hs = cw.gm1 * rT * m::rcp(ytot);
  S.F[2] = hs * H;
  S.H = H;
  S.J[2][0] = hs * H0;
  S.J[2][1] = hs * H1;
  S.J[2][2] = hs * H2;
  S.J[2][3] = hs * (H3h + Hgg_d);
  S.J[2][4] = W(0);
  // dust row (Eq. ap_eq:Td2) scaled by C_d T_d
  const W Cd = c.Cd;
  const W inv_cdtd = c.rCd * q.rTd;
  S.F[3] = (irabs + c.EUV - emit - gg) * inv_cdtd;
  S.J[3][0] = W(0);
  S.J[3][1] = W(0);
  S.J[3][2] = -G * zeta * T * inv_cdtd;
  S.J[3][3] = -(G * gam + acTd3 * beta_d) * c.rCd;
  S.J[3][4] = W(CRED) * beta_IR * E * inv_cdtd;
  // IR row (Appendix C) scaled by E_IR
  const W rho = c.rho;
  const W invE = m::rcp(E);
  S.F[4] = rho * fd * (emit - irabs) * invE;
  S.J[4][0] = W(0);
  S.J[4][1] = W(0);
  S.J[4][2] = W(0);
  S.J[4][3] = rho * fd * acTd3 * beta_d * Td * invE;
  S.J[4][4] = -rho * W(CRED) * fd * beta_IR;
  // the split variant keeps only the blocks printed in Eq. eq_deq and Appendix C
  if (fl & F_SPLIT) {
    S.J[0][2] = S.J[0][3] = S.J[1][2] = S.J[1][3] = W(0);
    S.J[2][0] = S.J[2][1] = W(0);
    S.J[2][3] = hs * Hgg_d;
  }
  // inverse timescales
  W rd = W(0);
  if (!(fl & F_FTD)) rd = m::abs(S.F[3]);
  if (!(fl & F_FTG)) rd = fmax_w(rd, m::abs(hs * Hgg));
  if (!(fl & F_FE)) rd = fmax_w(rd, m::abs(S.F[4]));
  W rc = W(0);
  if (!(fl & F_FY2)) rc = div_w(m::abs(S.F[0]), fmax_w(y2, cw.y_floor));
  if (!(fl & F_FYE)) rc = fmax_w(rc, div_w(m::abs(S.F[1]), fmax_w(ye, cw.y_floor)));
  S.rate_dust = rd;
  S.rate_chem = rc;
  S.rate_energy = (fl & F_FTG) ? W(0) : m::abs(S.F[2]);
  // frozen variables: their rows vanish (du_j = 0)
  const uint32_t fr[5] = {F_FY2, F_FYE, F_FTG, F_FTD, F_FE};
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (fl & fr[i]) {
      S.F[i] = W(0);
#pragma unroll
      for (int j = 0; j < 5; ++j) S.J[i][j] = W(0);
    }
}

}  // namespace sfc
