// noalloc.cu -- sfchem_step_batched_noalloc: the batched thermochemical step
// for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host-side memory budget managed by someone else (a simulation framework
// that owns every device allocation), in a callback or a signal-safe path,
// or in a process that must not grow its device footprint after start-up.
// sfchem_init allocates the context (counters, statistics, schedule tables),
// so such callers get this one entry point instead: its scratch lives in a
// file-scope __device__ array.  CUDA loads the library's device code, and
// with it the array, on a GPU the first time the library uses that GPU (by
// default lazily, at the first call that needs it), and keeps it until the
// process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "sfchem.h"
#include "launch.h"

using namespace sfc;

namespace {

constexpr int NA_MAX_BLOCKS = SFCHEM_NOALLOC_MAX_BLOCKS;   // include/sfchem.h
constexpr int NA_MAX_CHUNKS = SFCHEM_NOALLOC_MAX_CHUNKS;
constexpr int NA_CHUNK = 64;      // cells per chunk (the library default)
constexpr int NA_TPB = 128;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// layout of the scratch array (bytes)
constexpr size_t NA_COUNTER = 0;
constexpr size_t NA_STATS = 256;
constexpr size_t NA_BOFF = NA_STATS + align256(sizeof(DevStats));
constexpr size_t NA_BDT = NA_BOFF + align256(sizeof(int64_t) * (NA_MAX_BLOCKS + 1));
constexpr size_t NA_COST = NA_BDT + align256(sizeof(double) * NA_MAX_BLOCKS);
constexpr size_t NA_CHSTART = NA_COST + align256(sizeof(float) * NA_MAX_BLOCKS);
constexpr size_t NA_CHCOUNT = NA_CHSTART + align256(sizeof(int64_t) * NA_MAX_CHUNKS);
constexpr size_t NA_CHBLOCK = NA_CHCOUNT + align256(sizeof(int32_t) * NA_MAX_CHUNKS);
constexpr size_t NA_BYTES = NA_CHBLOCK + align256(sizeof(int32_t) * NA_MAX_CHUNKS);
static_assert(NA_BYTES == 1131264, "the scratch size stated in include/sfchem.h");

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEVICES] = {};

}  // namespace

// The scratch: work counter, statistics, block tables and the chunk table.
static __device__ __align__(256) unsigned char g_sfchem_noalloc_scratch[NA_BYTES];

namespace {

// Device address of the scratch on the current device (looked up once per
// device; in host code the array's name is only a host-side stand-in).
int scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return SFCHEM_ECUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return SFCHEM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sfchem_noalloc_scratch);
    if (e != cudaSuccess || !p) return SFCHEM_ECUDA;
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return SFCHEM_OK;
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

}  // namespace

extern "C" int sfchem_step_batched_noalloc(const sfchem_config_t *cfg, const sfchem_state_t *state,
                                           const sfchem_fields_t *fields, const int64_t *block_offset,
                                           const double *block_dt, int32_t n_blocks, double cd_factor,
                                           void *stream) {
  sfchem_config_t c;
  if (cfg) c = *cfg; else sfchem_config_default(&c);
  if (sfchem_config_validate(&c) != SFCHEM_OK) return SFCHEM_EINVAL;
  if (!(std::isfinite(cd_factor) && cd_factor > 0.0)) return SFCHEM_EINVAL;
  if (!state || !fields || !block_offset || !block_dt) return SFCHEM_EINVAL;
  if (n_blocks < 0 || n_blocks > NA_MAX_BLOCKS) return SFCHEM_EINVAL;   // beyond the scratch: refused
  if (n_blocks == 0) return SFCHEM_OK;
  const void *req[9] = {state->n_H, state->T_gas, state->T_dust, state->E_IR, state->y_H2, state->y_e,
                        fields->G0_fuv, fields->n_euv, fields->N_H2};
  for (const void *p : req)
    if (!p || !aligned8(p)) return SFCHEM_EINVAL;
  if ((state->y_H && !aligned8(state->y_H)) || (state->y_Hp && !aligned8(state->y_Hp)) ||
      (state->y_Hm && !aligned8(state->y_Hm)) ||
      (state->n_sub && (reinterpret_cast<uintptr_t>(state->n_sub) & 3u)) ||
      (state->n_itr && (reinterpret_cast<uintptr_t>(state->n_itr) & 3u)))
    return SFCHEM_EINVAL;
  if (block_offset[0] != 0) return SFCHEM_EINVAL;
  int64_t chunks = 0;
  for (int32_t b = 0; b < n_blocks; ++b) {
    const int64_t sz = block_offset[b + 1] - block_offset[b];
    if (sz < 0 || !(std::isfinite(block_dt[b]) && block_dt[b] >= 0.0)) return SFCHEM_EINVAL;
    chunks += (sz + NA_CHUNK - 1) / NA_CHUNK;
  }
  if (chunks > NA_MAX_CHUNKS) return SFCHEM_EINVAL;                    // beyond the scratch: refused
  if (chunks == 0) return SFCHEM_OK;

  unsigned char *base = nullptr;
  if (int rc = scratch_address(&base)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto *counter = reinterpret_cast<unsigned long long *>(base + NA_COUNTER);
  auto *stats = reinterpret_cast<DevStats *>(base + NA_STATS);
  auto *boff = reinterpret_cast<int64_t *>(base + NA_BOFF);
  auto *bdt = reinterpret_cast<double *>(base + NA_BDT);
  auto *cost = reinterpret_cast<float *>(base + NA_COST);
  auto *chs = reinterpret_cast<int64_t *>(base + NA_CHSTART);
  auto *chc = reinterpret_cast<int32_t *>(base + NA_CHCOUNT);
  auto *chb = reinterpret_cast<int32_t *>(base + NA_CHBLOCK);
  // the scratch keeps the previous call's contents: reset what must start at zero
  if (cudaMemsetAsync(base, 0, NA_BOFF, s) != cudaSuccess) return SFCHEM_ECUDA;
  if (cudaMemsetAsync(cost, 0, sizeof(float) * n_blocks, s) != cudaSuccess) return SFCHEM_ECUDA;
  if (cudaMemcpyAsync(boff, block_offset, sizeof(int64_t) * (n_blocks + 1), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return SFCHEM_ECUDA;
  if (cudaMemcpyAsync(bdt, block_dt, sizeof(double) * n_blocks, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SFCHEM_ECUDA;
  // the caller may reuse or free its (possibly pinned) host arrays as soon as
  // this call returns: wait until the stream has read them
  if (cudaStreamSynchronize(s) != cudaSuccess) return SFCHEM_ECUDA;
  if (launch_schedule(boff, cost, n_blocks, NA_CHUNK, chs, chc, chb, s) != cudaSuccess) return SFCHEM_ECUDA;

  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nH = state->n_H; a.Tg = state->T_gas; a.Td = state->T_dust; a.E = state->E_IR;
  a.y2 = state->y_H2; a.ye = state->y_e; a.yH = state->y_H; a.yHp = state->y_Hp; a.yHm = state->y_Hm;
  a.status = state->status; a.nsub = state->n_sub; a.niter = state->n_itr;
  a.G0 = fields->G0_fuv; a.nEUV = fields->n_euv; a.NH2 = fields->N_H2;
  a.n_cells = block_offset[n_blocks];
  a.chunk = NA_CHUNK;
  a.n_chunks = (int32_t)chunks;
  a.ch_start = chs; a.ch_count = chc; a.ch_block = chb;
  a.block_dt = bdt; a.block_cost = cost;
  a.cd_factor = cd_factor;
  a.counter = counter;
  a.stats = stats;
  a.cfg.f_chem = c.f_chem; a.cfg.Z = c.Z; a.cfg.gamma_ad = c.gamma_ad; a.cfg.y_floor = c.y_floor;
  a.cfg.nr_tol = c.nr_tol; a.cfg.n_cyc = c.n_cyc; a.cfg.n_sub_max = c.n_sub_max;
  a.cfg.nr_itr_limit = c.nr_itr_limit; a.cfg.rmask = c.reaction_mask; a.cfg.pmask = c.process_mask;
  a.cfg.flags = c.flags;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SFCHEM_ECUDA;
  const bool mixed = c.precision == SFCHEM_MIXED;
  if ((mixed ? occupancy_li_mixed(NA_TPB, &occ) : occupancy_li_fp64(NA_TPB, &occ)) != cudaSuccess)
    return SFCHEM_ECUDA;
  const int grid = sms * (occ > 0 ? occ : 1);
  cudaError_t e = mixed ? launch_li_mixed(a, grid, NA_TPB, s) : launch_li_fp64(a, grid, NA_TPB, s);
  return e == cudaSuccess ? SFCHEM_OK : SFCHEM_ECUDA;
}
