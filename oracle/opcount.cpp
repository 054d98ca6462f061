// opcount.cpp -- the oracle's LI step (sfchem_oracle.cpp) compiled with an
// op-counting scalar type in place of double, to measure the floating-point
// work of the method per substep: additions, multiplications, divisions,
// fused multiply-adds, square roots and the transcendental functions (exp,
// log, pow) are counted separately, in four sections of the step (the
// substep's system: rates, heating/cooling, dust terms and their exact
// derivatives; the linear solves; the tight-coupling Newton iteration; the
// controller, update and projection).
//
// TEST INFRASTRUCTURE ONLY, like the oracle it includes: the benchmark uses
// the counts as the algorithmic work of its roofline; the product path never
// loads it.  Every value is computed in double exactly as in the oracle, so
// the counted run takes the oracle's own substep sequence.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <limits>

#include "sfchem_oracle.h"

namespace ocount {

enum Op { ADD, MUL, DIV, FMA, SQRT, EXP, LOG, POW, CMP, NOPS };
constexpr int NSEC = 4;
thread_local uint64_t g_count[NSEC][NOPS];
thread_local int g_sec = 3;

inline void tick(Op o) { ++g_count[g_sec][o]; }

struct Section {
  int prev;
  explicit Section(int k) : prev(g_sec) { g_sec = k; }
  ~Section() { g_sec = prev; }
};

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}   // NOLINT: implicit, so that constants mix in
  explicit operator double() const { return v; }
};

inline Cnt operator+(Cnt a, Cnt b) { tick(ADD); return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { tick(ADD); return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { tick(MUL); return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { tick(DIV); return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt &operator+=(Cnt &a, Cnt b) { a = a + b; return a; }
inline Cnt &operator-=(Cnt &a, Cnt b) { a = a - b; return a; }
inline Cnt &operator*=(Cnt &a, Cnt b) { a = a * b; return a; }
inline Cnt &operator/=(Cnt &a, Cnt b) { a = a / b; return a; }
inline bool operator<(Cnt a, Cnt b) { tick(CMP); return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { tick(CMP); return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { tick(CMP); return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { tick(CMP); return a.v >= b.v; }
inline bool operator==(Cnt a, Cnt b) { tick(CMP); return a.v == b.v; }
inline bool operator!=(Cnt a, Cnt b) { tick(CMP); return a.v != b.v; }

}  // namespace ocount

// The math functions the oracle calls as std::..., for the counting type.
namespace std {
inline ocount::Cnt exp(ocount::Cnt a) { ocount::tick(ocount::EXP); return ocount::Cnt(std::exp(a.v)); }
inline ocount::Cnt log(ocount::Cnt a) { ocount::tick(ocount::LOG); return ocount::Cnt(std::log(a.v)); }
inline ocount::Cnt sqrt(ocount::Cnt a) { ocount::tick(ocount::SQRT); return ocount::Cnt(std::sqrt(a.v)); }
inline ocount::Cnt pow(ocount::Cnt a, double p) { ocount::tick(ocount::POW); return ocount::Cnt(std::pow(a.v, p)); }
inline ocount::Cnt pow(ocount::Cnt a, int p) { ocount::tick(ocount::POW); return ocount::Cnt(std::pow(a.v, p)); }
inline ocount::Cnt fabs(ocount::Cnt a) { return ocount::Cnt(std::fabs(a.v)); }
inline ocount::Cnt fma(ocount::Cnt a, ocount::Cnt b, ocount::Cnt c) {
  ocount::tick(ocount::FMA);
  return ocount::Cnt(std::fma(a.v, b.v, c.v));
}
inline ocount::Cnt frexp(ocount::Cnt a, int *e) { return ocount::Cnt(std::frexp(a.v, e)); }
inline bool isfinite(ocount::Cnt a) { return std::isfinite(a.v); }
inline ocount::Cnt max(ocount::Cnt a, ocount::Cnt b) { ocount::tick(ocount::CMP); return a.v < b.v ? b : a; }
inline ocount::Cnt min(ocount::Cnt a, ocount::Cnt b) { ocount::tick(ocount::CMP); return b.v < a.v ? b : a; }
inline ocount::Cnt max(ocount::Cnt a, double b) { return std::max(a, ocount::Cnt(b)); }
inline ocount::Cnt max(double a, ocount::Cnt b) { return std::max(ocount::Cnt(a), b); }
inline ocount::Cnt min(ocount::Cnt a, double b) { return std::min(a, ocount::Cnt(b)); }
inline ocount::Cnt min(double a, ocount::Cnt b) { return std::min(ocount::Cnt(a), b); }
}  // namespace std

#define SFCHEM_ORACLE_REAL ocount::Cnt
#define SFCHEM_ORACLE_OPCOUNT 1
#define ORACLE_SECTION(k) ocount::Section oracle_section_guard_(k)
#include "sfchem_oracle.cpp"

extern "C" {

// Counted LI step of n cells, one after another (single thread).  counts
// receives NSEC x NOPS totals (sections: system, solve, Newton, control; ops:
// add/sub, mul, div, fma, sqrt, exp, log, pow, compare); returns the total
// number of substeps, or -1 on a bad argument.
int64_t oracle_opcount_li(int64_t n, const double *n_H, const double *T_g, const double *T_d, const double *E_IR,
                          const double *y_H2, const double *y_e, const double *G0, const double *n_EUV,
                          const double *N_H2, const double *dt, double cd_factor, const oracle_config *cfg,
                          uint64_t *counts) {
  if (n < 0 || !counts || !(cd_factor > 0.0)) return -1;
  oracle_config c = checked(cfg);
  std::memset(ocount::g_count, 0, sizeof(ocount::g_count));
  int64_t nsub = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!valid_input(n_H[i], T_g[i], T_d[i], E_IR[i], y_H2[i], y_e[i], G0[i], n_EUV[i], N_H2[i], dt[i])) continue;
    CellIn ci = make_cell(n_H[i], G0[i], n_EUV[i], N_H2[i], cd_factor, c);
    real u[5] = {y_H2[i], y_e[i], T_g[i], T_d[i], E_IR[i]};
    LIOut o = li_cell(u, ci, dt[i], c, 0, nullptr);
    nsub += o.nsub;
  }
  std::memcpy(counts, ocount::g_count, sizeof(ocount::g_count));
  return nsub;
}

// Counted Newton-Raphson backward-Euler step (the paper's reference solver,
// nr_cell) of n cells, one after another (single thread); counts as above,
// by the section of the oracle function that runs each operation; returns
// the total number of accepted steps, or -1 on a bad argument.
int64_t oracle_opcount_nr(int64_t n, const double *n_H, const double *T_g, const double *T_d, const double *E_IR,
                          const double *y_H2, const double *y_e, const double *G0, const double *n_EUV,
                          const double *N_H2, const double *dt, double cd_factor, const oracle_config *cfg,
                          uint64_t *counts) {
  if (n < 0 || !counts || !(cd_factor > 0.0)) return -1;
  oracle_config c = checked(cfg);
  std::memset(ocount::g_count, 0, sizeof(ocount::g_count));
  int64_t nsub = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!valid_input(n_H[i], T_g[i], T_d[i], E_IR[i], y_H2[i], y_e[i], G0[i], n_EUV[i], N_H2[i], dt[i])) continue;
    CellIn ci = make_cell(n_H[i], G0[i], n_EUV[i], N_H2[i], cd_factor, c);
    real u[5] = {y_H2[i], y_e[i], T_g[i], T_d[i], E_IR[i]};
    LIOut o = nr_cell(u, ci, dt[i], c);
    nsub += o.nsub;
  }
  std::memcpy(counts, ocount::g_count, sizeof(ocount::g_count));
  return nsub;
}

}  // extern "C"
