// photon.cu -- photon consumption after the thermochemical update (Sec.
// 2.2.8, "Radiation components": the EUV and FUV photons of the step are
// absorbed once the abundances and temperatures have been updated).
//
// Reading (the paper defers the details to another paper): per cell, with
// y_H = 1 - 2 y_H2 - y_e of the updated state, each band loses photons at a
// rate per photon lam = (gas) + (dust), taken implicitly over dt, so that
// n' = n / (1 + lam dt) never goes negative and the photons removed equal
// those absorbed:
//   EUV: lam_E = c n_H (sigma_H y_H + sigma_d)      (photoionization of H with
//        the cross-section of k_H9, and dust)
//   FUV: lam_F = k_LW f_sh(N_H2) n_H y_H2 h nu_F / u_Habing + c n_H sigma_d
//        (one photon per photodissociation of H2 at the rate of k_H10, and dust)
// The photons removed are split between gas and dust in proportion to
// their rates.  The constants are those of the rates and of the dust UV
// absorption (stand-ins), with h nu_F = 12.4 eV.
//
// Elementwise and HBM-bound: grid-stride, two cells per thread and trip,
// coalesced FP64 loads of 6 fields (48 B) and stores of 2 (16 B; 48 B with
// the absorbed photon counts).  The rate factors (the shielding power,
// lam dt and the band's surviving fraction 1 / (1 + lam dt)) are taken in
// FP32 -- like the per-cell constants of the mixed solver, ~1e-7 relative --
// and the photon bookkeeping in FP64: n', the photons removed and their
// split, so that n' + absorbed = n holds to FP64 rounding.  GB300's FP64
// pipe (2 instructions per clock per SM) is the kernel's other limit: in
// FP64 the shielding power and two divisions cost ~100 FP64 instructions
// per cell and held it at 4 % of the HBM bandwidth; with the FP32 factors
// and 4 FP64 instructions per cell (y_H, one fma per band) it runs at about
// 95 % of the measured copy bandwidth.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sfchem.h"
#include "li_device.cuh"

namespace {

constexpr double HNU_FUV = 12.4 * sfc::EV;

// One cell: the photon update from the six inputs, stores of the two
// outputs (and the absorbed counts when abs4 is given).
__device__ __forceinline__ void photon_cell(int64_t i, double nh, double h2, double e, double g0, double ne,
                                            double col, float dtf, double *__restrict__ G0o,
                                            double *__restrict__ nEo, double *__restrict__ abs4) {
  using namespace sfc;
  typedef M<float> m;
  // y_H = 1 - 2 y_H2 - y_e cancels in molecular or ionized gas: formed in FP64
  const float yH = fmaxf(d2f_int(fma(-2.0, h2, 1.0) - e), 0.0f);
  const float nf = d2f_int(nh), h2f = d2f_int(h2);
  const float lam_H = float(CLIGHT * SIG_EUV) * nf * yH;
  const float lam_d = float(CLIGHT * SIG_DUV) * nf;
  // (N_H2 / N_0)^-3/4 as 1 / (sqrt(x) sqrt(sqrt(x))), above N_0 (the factor
  // is continuous there, so the test is taken on the rounded x)
  static_assert(SH_POW == 0.75, "the shielding factor assumes the exponent 3/4");
  const float xs = d2f_int(col) * float(1.0 / NSH0), sq = m::sqrt(xs);
  const float fsh = xs > 1.0f ? m::rcp(sq * m::sqrt(sq)) : 1.0f;
  const float lam_2 = float(K_LW * (HNU_FUV / U_HAB)) * fsh * nf * h2f;
  const float sE = lam_H + lam_d, sF = lam_2 + lam_d;
  // of n photons, n x / (1 + x) are absorbed and n / (1 + x) survive
  // (x = lam dt); the smaller of the two is formed from its own formula and
  // the other as n minus it, so both keep FP32 relative accuracy from
  // optically thin (x << 1) to opaque (x >> 1) cells.  Each band's new count
  // is one FP64 fma: n - n take (thin) or n keep + 0 (opaque).
  const float xE = fminf(sE * dtf, 1e37f), xF = fminf(sF * dtf, 1e37f);
  const float rE1 = m::rcp(1.0f + xE), rF1 = m::rcp(1.0f + xF);
  const bool thinE = xE < 1.0f, thinF = xF < 1.0f;
  const double cE = f2d_int(thinE ? -(xE * rE1) : rE1), cF = f2d_int(thinF ? -(xF * rF1) : rF1);
  const double ne_new = fma(ne, cE, thinE ? ne : 0.0);
  const double g_new = fma(g0, cF, thinF ? g0 : 0.0);
  nEo[i] = ne_new;
  G0o[i] = g_new;
  if (abs4) {
    const double dE = thinE ? -(ne * cE) : ne - ne_new;
    const double dF = (thinF ? -(g0 * cF) : g0 - g_new) * (U_HAB / HNU_FUV);
    // the split between gas and dust in proportion to the rates, again
    // with the smaller share from its own fraction and the larger as the
    // rest (dE (1 - w) with an FP32 w near 1 would lose the dust share)
    const float rE = sE > 0.0f ? m::rcp(sE) : 0.0f, rF = sF > 0.0f ? m::rcp(sF) : 0.0f;
    const bool gE = lam_H <= lam_d, gF = lam_2 <= lam_d;
    const double sE_small = dE * f2d_int((gE ? lam_H : lam_d) * rE);
    const double sF_small = dF * f2d_int((gF ? lam_2 : lam_d) * rF);
    abs4[4 * i + 0] = gE ? sE_small : dE - sE_small;
    abs4[4 * i + 1] = gE ? dE - sE_small : sE_small;
    abs4[4 * i + 2] = gF ? sF_small : dF - sF_small;
    abs4[4 * i + 3] = gF ? dF - sF_small : sF_small;
  }
}

// Grid-stride over the cells, two cells per trip: both cells' twelve loads
// are issued before either is computed, to keep more bytes in flight.  Each
// element is read and then written by one thread only, so the in-place
// update (G0_out == G0_fuv, n_euv_out == n_euv) is safe.
__global__ void __launch_bounds__(256) sfchem_photon_kernel(int64_t n, const double *__restrict__ nH,
                                                            const double *__restrict__ y2,
                                                            const double *__restrict__ ye,
                                                            const double *__restrict__ G0,
                                                            const double *__restrict__ nE,
                                                            const double *__restrict__ NH2, double dt,
                                                            double *__restrict__ G0o, double *__restrict__ nEo,
                                                            double *__restrict__ abs4) {
  const float dtf = sfc::d2f_int(dt);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    const int64_t j = i + stride;
    const bool two = j < n;
    const double nh = __ldg(nH + i), h2 = __ldg(y2 + i), e = __ldg(ye + i);
    const double g0 = __ldg(G0 + i), ne = __ldg(nE + i), col = __ldg(NH2 + i);
    double nh2 = 1.0, h22 = 0.0, e2 = 0.0, g02 = 0.0, ne2 = 0.0, col2 = 0.0;
    if (two) {
      nh2 = __ldg(nH + j); h22 = __ldg(y2 + j); e2 = __ldg(ye + j);
      g02 = __ldg(G0 + j); ne2 = __ldg(nE + j); col2 = __ldg(NH2 + j);
    }
    photon_cell(i, nh, h2, e, g0, ne, col, dtf, G0o, nEo, abs4);
    if (two) photon_cell(j, nh2, h22, e2, g02, ne2, col2, dtf, G0o, nEo, abs4);
  }
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

}  // namespace

extern "C" int sfchem_photon_update(const sfchem_state_t *state, const sfchem_fields_t *fields, int64_t n_cells,
                                    double dt_seconds, double *G0_out, double *n_euv_out, double *absorbed,
                                    void *stream) {
  if (n_cells < 0 || !(std::isfinite(dt_seconds) && dt_seconds >= 0.0)) return SFCHEM_EINVAL;
  if (n_cells == 0) return SFCHEM_OK;
  if (!state || !fields || !G0_out || !n_euv_out) return SFCHEM_EINVAL;
  const void *req[8] = {state->n_H, state->y_H2, state->y_e, fields->G0_fuv, fields->n_euv, fields->N_H2,
                        G0_out, n_euv_out};
  for (const void *p : req)
    if (!p || !aligned8(p)) return SFCHEM_EINVAL;
  if (absorbed && !aligned8(absorbed)) return SFCHEM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return SFCHEM_ECUDA;
  // a grid of 8 CTAs of 256 threads per SM, grid-stride over the cells
  const int64_t want = (n_cells + 255) / 256;
  const int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  sfchem_photon_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n_cells, state->n_H, state->y_H2, state->y_e, fields->G0_fuv, fields->n_euv, fields->N_H2, dt_seconds, G0_out,
      n_euv_out, absorbed);
  return cudaGetLastError() == cudaSuccess ? SFCHEM_OK : SFCHEM_ECUDA;
}
