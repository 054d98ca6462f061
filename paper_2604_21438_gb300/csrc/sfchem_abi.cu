// sfchem_abi.cu -- the C ABI of libsfchem (see include/sfchem.h): argument
// checks, context and scratch management, the batched schedule (cost-sorted
// chunk table built on the device), CUDA-graph capture and replay of the
// batched launch sequence, the autotuner and the statistics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sfchem.h"
#include "launch.h"

using namespace sfc;

namespace {

const uint64_t CTX_MAGIC = 0x53464348454d3031ull;  // "SFCHEM01"
const int SCHED_THREADS = 1024;
const int SCHED_SORT_MAX = 8192;                   // blocks sorted by cost in shared memory

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char *where) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
  return SFCHEM_ECUDA;
}
#define SFC_CUDA(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct GraphKey {
  const void *ptrs[15];
  int32_t n_blocks, n_chunks, chunk, tpb, grid;
  double cd_factor;
  sfchem_config_t cfg;
  uint64_t sched_version;
  bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

}  // namespace

struct sfchem_ctx {
  uint64_t magic;
  sfchem_config_t cfg;
  int device, num_sms;
  unsigned long long *d_counter;
  DevStats *d_stats;
  cudaEvent_t ev0, ev1;
  bool timed;
  uint64_t calls;
  sfchem_launch_t launch;     // zero fields: defaults
  // batched schedule
  std::vector<int64_t> h_block_offset;
  std::vector<double> h_block_dt;
  int64_t *d_block_offset;
  double *d_block_dt;
  float *d_block_cost;
  int32_t cap_blocks;
  int64_t *d_ch_start;
  int32_t *d_ch_count, *d_ch_block;
  int32_t cap_chunks;
  int32_t sched_chunk;
  int32_t n_chunks;
  uint64_t sched_version;
  // graph cache for the batched launch sequence
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  GraphKey gkey;
  bool have_graph;
  // host-buffer pipeline: a copy-in and a copy-out stream, and per staging
  // slot a compute stream, a work counter and a chunk table, so that the
  // solver of one slice runs while the previous one drains its last cells
  bool have_pipe;
  cudaStream_t s_in, s_out, s_comp[2];
  cudaEvent_t ev_start, ev_end, ev_in[2], ev_comp[2], ev_free[2];
  void *stage_mem;
  int64_t stage_cap;            // cells per slot
  double *stage_f[2][12];       // n_H, T_g, T_d, E_IR, y_H2, y_e, G0, n_EUV, N_H2, y_H, y_H+, y_H-
  int32_t *stage_nsub[2];
  uint8_t *stage_status[2];
  void *pipe_tab;
  int64_t pipe_tab_cap;         // chunks per slot
  unsigned long long *pipe_counter[2];
  int64_t *pipe_ch_start[2];
  int32_t *pipe_ch_count[2], *pipe_ch_block[2];
};

// ------------------------------------------------------------- schedule
// One CTA: sort the blocks by the previous call's cost (descending, index
// ascending on ties), zero the cost accumulators, and write the chunk table
// (chunks never cross a block; `chunk` cells each, the last one ragged).
__global__ void __launch_bounds__(SCHED_THREADS)
sfchem_schedule(const int64_t *block_offset, float *block_cost, int32_t n_blocks, int32_t chunk,
                int64_t *ch_start, int32_t *ch_count, int32_t *ch_block) {
  extern __shared__ unsigned char smem[];
  const bool sort = n_blocks <= SCHED_SORT_MAX;
  float *key = reinterpret_cast<float *>(smem);
  int32_t *val = reinterpret_cast<int32_t *>(smem + sizeof(float) * SCHED_SORT_MAX);
  __shared__ int32_t scan[SCHED_THREADS];
  __shared__ int32_t running;
  int P = 1;
  while (P < n_blocks) P <<= 1;
  if (sort) {
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      key[i] = i < n_blocks ? block_cost[i] : -1.0f;
      val[i] = i;
    }
    __syncthreads();
    // bitonic sort: "before" = larger cost, or equal cost and smaller index
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) {
            const bool up = (i & k) == 0;
            const float ki = key[i], kl = key[l];
            const int vi = val[i], vl = val[l];
            const bool l_before_i = (kl > ki) || (kl == ki && vl < vi);
            if (up ? l_before_i : !l_before_i) {
              key[i] = kl; key[l] = ki; val[i] = vl; val[l] = vi;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) block_cost[i] = 0.0f;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  for (int base = 0; base < n_blocks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int b = -1, cnt = 0;
    if (i < n_blocks) {
      b = sort ? val[i] : i;
      const int64_t sz = block_offset[b + 1] - block_offset[b];
      cnt = (int)((sz + chunk - 1) / chunk);
    }
    scan[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      const int v = threadIdx.x >= (unsigned)o ? scan[threadIdx.x - o] : 0;
      __syncthreads();
      scan[threadIdx.x] += v;
      __syncthreads();
    }
    const int first = running + scan[threadIdx.x] - cnt;
    if (i < n_blocks) {
      // cell index relative to the first block passed (0 for a whole layout)
      const int64_t s0 = block_offset[b] - block_offset[0], sz = block_offset[b + 1] - block_offset[b];
      for (int c = 0; c < cnt; ++c) {
        ch_start[first + c] = s0 + (int64_t)c * chunk;
        ch_count[first + c] = (int32_t)min((int64_t)chunk, sz - (int64_t)c * chunk);
        ch_block[first + c] = b;
      }
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) running += scan[threadIdx.x];
    __syncthreads();
  }
}

namespace sfc {
cudaError_t launch_schedule(const int64_t *block_offset, float *block_cost, int32_t n_blocks, int32_t chunk,
                            int64_t *ch_start, int32_t *ch_count, int32_t *ch_block, cudaStream_t s) {
  const size_t smem = n_blocks <= SCHED_SORT_MAX ? (sizeof(float) + sizeof(int32_t)) * SCHED_SORT_MAX : 0;
  cudaError_t e = cudaFuncSetAttribute(sfchem_schedule, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((sizeof(float) + sizeof(int32_t)) * SCHED_SORT_MAX));
  if (e != cudaSuccess) return e;
  sfchem_schedule<<<1, SCHED_THREADS, smem, s>>>(block_offset, block_cost, n_blocks, chunk, ch_start, ch_count,
                                                 ch_block);
  return cudaGetLastError();
}
}  // namespace sfc

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_ctx(const sfchem_ctx *c) {
  if (!c || c->magic != CTX_MAGIC) return SFCHEM_ENOTINIT;
  return SFCHEM_OK;
}

int check_arrays(const sfchem_state_t *s, const sfchem_fields_t *f) {
  if (!s || !f) return SFCHEM_EINVAL;
  const void *req[9] = {s->n_H, s->T_gas, s->T_dust, s->E_IR, s->y_H2, s->y_e, f->G0_fuv, f->n_euv, f->N_H2};
  for (const void *p : req)
    if (!p || !aligned(p, 8)) return SFCHEM_EINVAL;
  const void *opt[3] = {s->y_H, s->y_Hp, s->y_Hm};
  for (const void *p : opt)
    if (p && !aligned(p, 8)) return SFCHEM_EINVAL;
  if (s->n_sub && !aligned(s->n_sub, 4)) return SFCHEM_EINVAL;
  if (s->n_itr && !aligned(s->n_itr, 4)) return SFCHEM_EINVAL;
  return SFCHEM_OK;
}

DevCfg dev_cfg(const sfchem_config_t &c) {
  DevCfg d;
  d.f_chem = c.f_chem; d.Z = c.Z; d.gamma_ad = c.gamma_ad; d.y_floor = c.y_floor; d.nr_tol = c.nr_tol;
  d.n_cyc = c.n_cyc; d.n_sub_max = c.n_sub_max; d.nr_itr_limit = c.nr_itr_limit;
  d.rmask = c.reaction_mask; d.pmask = c.process_mask; d.flags = c.flags;
  return d;
}

KArgs base_args(sfchem_ctx *ctx, const sfchem_state_t *s, const sfchem_fields_t *f, double cd_factor) {
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nH = s->n_H; a.Tg = s->T_gas; a.Td = s->T_dust; a.E = s->E_IR; a.y2 = s->y_H2; a.ye = s->y_e;
  a.yH = s->y_H; a.yHp = s->y_Hp; a.yHm = s->y_Hm; a.status = s->status; a.nsub = s->n_sub; a.niter = s->n_itr;
  a.G0 = f->G0_fuv; a.nEUV = f->n_euv; a.NH2 = f->N_H2;
  a.cd_factor = cd_factor;
  a.counter = ctx->d_counter;
  a.stats = ctx->d_stats;
  a.cfg = dev_cfg(ctx->cfg);
  return a;
}

struct Shape { int tpb, ctas_per_sm, chunk, grid; };

int resolve_shape(sfchem_ctx *ctx, Shape &sh) {
  sh.tpb = ctx->launch.threads_per_cta ? ctx->launch.threads_per_cta : 128;
  int occ = 0;
  cudaError_t e = ctx->cfg.precision == SFCHEM_MIXED ? occupancy_li_mixed(sh.tpb, &occ)
                                                      : occupancy_li_fp64(sh.tpb, &occ);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ < 1) occ = 1;
  sh.ctas_per_sm = ctx->launch.ctas_per_sm ? std::min(ctx->launch.ctas_per_sm, occ) : occ;
  sh.chunk = ctx->launch.chunk ? ctx->launch.chunk : 64;
  sh.grid = ctx->num_sms * sh.ctas_per_sm;
  return SFCHEM_OK;
}

cudaError_t launch_solver(sfchem_ctx *ctx, const KArgs &a, const Shape &sh, cudaStream_t s) {
  return ctx->cfg.precision == SFCHEM_MIXED ? launch_li_mixed(a, sh.grid, sh.tpb, s)
                                             : launch_li_fp64(a, sh.grid, sh.tpb, s);
}

int validate_cfg(const sfchem_config_t *c) {
  if (!c) return SFCHEM_EINVAL;
  if (c->precision != SFCHEM_FP64 && c->precision != SFCHEM_MIXED) return SFCHEM_EINVAL;
  if (c->n_cyc < 1 || c->n_sub_max < 1 || c->nr_itr_limit < 1) return SFCHEM_EINVAL;
  if (!(c->f_chem > 0.0 && c->f_chem <= 1.0)) return SFCHEM_EINVAL;
  if (!(std::isfinite(c->Z) && c->Z >= 0.0)) return SFCHEM_EINVAL;
  if (!(std::isfinite(c->gamma_ad) && c->gamma_ad > 1.0)) return SFCHEM_EINVAL;
  if (!(std::isfinite(c->y_floor) && c->y_floor > 0.0)) return SFCHEM_EINVAL;
  if (!(std::isfinite(c->nr_tol) && c->nr_tol > 0.0)) return SFCHEM_EINVAL;
  if (c->reaction_mask >> 12 || c->process_mask >> 17 || c->flags >> 8 || c->reserved) return SFCHEM_EINVAL;
  return SFCHEM_OK;
}

int ensure_schedule_capacity(sfchem_ctx *ctx, int32_t n_blocks, int32_t n_chunks) {
  if (n_blocks > ctx->cap_blocks) {
    cudaFree(ctx->d_block_offset); cudaFree(ctx->d_block_dt); cudaFree(ctx->d_block_cost);
    ctx->d_block_offset = nullptr; ctx->d_block_dt = nullptr; ctx->d_block_cost = nullptr;
    ctx->cap_blocks = 0;
    SFC_CUDA(cudaMalloc(&ctx->d_block_offset, sizeof(int64_t) * (n_blocks + 1)));
    SFC_CUDA(cudaMalloc(&ctx->d_block_dt, sizeof(double) * n_blocks));
    SFC_CUDA(cudaMalloc(&ctx->d_block_cost, sizeof(float) * n_blocks));
    SFC_CUDA(cudaMemset(ctx->d_block_cost, 0, sizeof(float) * n_blocks));
    ctx->cap_blocks = n_blocks;
  }
  if (n_chunks > ctx->cap_chunks) {
    cudaFree(ctx->d_ch_start); cudaFree(ctx->d_ch_count); cudaFree(ctx->d_ch_block);
    ctx->d_ch_start = nullptr; ctx->d_ch_count = nullptr; ctx->d_ch_block = nullptr;
    ctx->cap_chunks = 0;
    SFC_CUDA(cudaMalloc(&ctx->d_ch_start, sizeof(int64_t) * n_chunks));
    SFC_CUDA(cudaMalloc(&ctx->d_ch_count, sizeof(int32_t) * n_chunks));
    SFC_CUDA(cudaMalloc(&ctx->d_ch_block, sizeof(int32_t) * n_chunks));
    ctx->cap_chunks = n_chunks;
  }
  return SFCHEM_OK;
}

void drop_graph(sfchem_ctx *ctx) {
  if (ctx->have_graph) {
    cudaGraphExecDestroy(ctx->gexec);
    cudaGraphDestroy(ctx->graph);
    ctx->have_graph = false;
  }
}

// Host checks of a batched schedule; returns the chunk count through *nch.
int check_blocks(const int64_t *off, const double *bdt, int32_t n_blocks, int32_t chunk, int64_t *ncells,
                 int64_t *nch) {
  if (!off || !bdt || n_blocks < 0 || chunk < 1) return SFCHEM_EINVAL;
  if (off[0] != 0) return SFCHEM_EINVAL;
  int64_t chunks = 0;
  for (int32_t b = 0; b < n_blocks; ++b) {
    const int64_t sz = off[b + 1] - off[b];
    if (sz < 0) return SFCHEM_EINVAL;
    if (!(std::isfinite(bdt[b]) && bdt[b] >= 0.0)) return SFCHEM_EINVAL;
    chunks += (sz + chunk - 1) / chunk;
  }
  if (chunks > INT32_MAX) return SFCHEM_EINVAL;
  *ncells = off[n_blocks];
  *nch = chunks;
  return SFCHEM_OK;
}

// Upload the schedule arrays when they changed since the last call.
int sync_schedule(sfchem_ctx *ctx, const int64_t *off, const double *bdt, int32_t n_blocks, int32_t chunk,
                  int32_t n_chunks, cudaStream_t s) {
  bool same = chunk == ctx->sched_chunk && (int64_t)ctx->h_block_dt.size() == n_blocks &&
              std::equal(off, off + n_blocks + 1, ctx->h_block_offset.begin()) &&
              std::equal(bdt, bdt + n_blocks, ctx->h_block_dt.begin());
  if (same) return SFCHEM_OK;
  int rc = ensure_schedule_capacity(ctx, n_blocks, n_chunks);
  if (rc) return rc;
  // a new layout invalidates the previous costs
  SFC_CUDA(cudaMemcpyAsync(ctx->d_block_offset, off, sizeof(int64_t) * (n_blocks + 1), cudaMemcpyHostToDevice, s));
  SFC_CUDA(cudaMemcpyAsync(ctx->d_block_dt, bdt, sizeof(double) * n_blocks, cudaMemcpyHostToDevice, s));
  SFC_CUDA(cudaMemsetAsync(ctx->d_block_cost, 0, sizeof(float) * n_blocks, s));
  SFC_CUDA(cudaStreamSynchronize(s));   // the host arrays may change after we return
  ctx->h_block_offset.assign(off, off + n_blocks + 1);
  ctx->h_block_dt.assign(bdt, bdt + n_blocks);
  ctx->sched_chunk = chunk;
  ctx->n_chunks = n_chunks;
  ctx->sched_version++;
  return SFCHEM_OK;
}

int record_batched(sfchem_ctx *ctx, const KArgs &a, const Shape &sh, int32_t n_blocks, cudaStream_t s) {
  SFC_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), s));
  const size_t smem = n_blocks <= SCHED_SORT_MAX ? (sizeof(float) + sizeof(int32_t)) * SCHED_SORT_MAX : 0;
  sfchem_schedule<<<1, SCHED_THREADS, smem, s>>>(ctx->d_block_offset, ctx->d_block_cost, n_blocks,
                                                 sh.chunk, ctx->d_ch_start, ctx->d_ch_count, ctx->d_ch_block);
  SFC_CUDA(cudaGetLastError());
  SFC_CUDA(launch_solver(ctx, a, sh, s));
  return SFCHEM_OK;
}

int batched_launch(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                   int32_t n_blocks, double cd_factor, const Shape &sh, cudaStream_t s, bool use_graph) {
  KArgs a = base_args(ctx, state, fields, cd_factor);
  a.n_cells = ctx->h_block_offset[n_blocks];
  a.chunk = sh.chunk;
  a.n_chunks = ctx->n_chunks;
  a.ch_start = ctx->d_ch_start; a.ch_count = ctx->d_ch_count; a.ch_block = ctx->d_ch_block;
  a.block_dt = ctx->d_block_dt; a.block_cost = ctx->d_block_cost;
  if (!use_graph) return record_batched(ctx, a, sh, n_blocks, s);
  GraphKey k;
  std::memset(&k, 0, sizeof(k));
  const void *p[15] = {a.nH, a.Tg, a.Td, a.E, a.y2, a.ye, a.yH, a.yHp, a.yHm, a.status, a.nsub, a.niter,
                       a.G0, a.nEUV, a.NH2};
  std::memcpy(k.ptrs, p, sizeof(p));
  k.n_blocks = n_blocks; k.n_chunks = a.n_chunks; k.chunk = sh.chunk; k.tpb = sh.tpb; k.grid = sh.grid;
  k.cd_factor = cd_factor; k.cfg = ctx->cfg; k.sched_version = ctx->sched_version;
  if (!(ctx->have_graph && k == ctx->gkey)) {
    drop_graph(ctx);
    SFC_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = record_batched(ctx, a, sh, n_blocks, ctx->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaGraphInstantiate"); }
    ctx->graph = g;
    ctx->gkey = k;
    ctx->have_graph = true;
  }
  SFC_CUDA(cudaGraphLaunch(ctx->gexec, s));
  return SFCHEM_OK;
}

// Streams, events and staging slots of the host-buffer pipeline (created on
// first use, slots grown to `cells` cells each).
int ensure_pipeline(sfchem_ctx *ctx, int64_t cells, int64_t chunks) {
  if (!ctx->have_pipe) {
    SFC_CUDA(cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking));
    SFC_CUDA(cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
    SFC_CUDA(cudaStreamCreateWithFlags(&ctx->s_comp[0], cudaStreamNonBlocking));
    SFC_CUDA(cudaStreamCreateWithFlags(&ctx->s_comp[1], cudaStreamNonBlocking));
    cudaEvent_t *evs[8] = {&ctx->ev_start, &ctx->ev_end, &ctx->ev_in[0], &ctx->ev_in[1], &ctx->ev_comp[0],
                           &ctx->ev_comp[1], &ctx->ev_free[0], &ctx->ev_free[1]};
    for (cudaEvent_t *e : evs) SFC_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    ctx->have_pipe = true;
  }
  if (cells > ctx->stage_cap) {
    cudaFree(ctx->stage_mem);
    ctx->stage_mem = nullptr;
    ctx->stage_cap = 0;
    // per slot: 12 double arrays, one int32 and one uint8 array, each start
    // rounded up to 256 bytes
    const size_t nd = ((size_t)cells * 8 + 255) / 256 * 256, ni = ((size_t)cells * 4 + 255) / 256 * 256,
                 nb = ((size_t)cells + 255) / 256 * 256;
    const size_t slot = 12 * nd + ni + nb;
    SFC_CUDA(cudaMalloc(&ctx->stage_mem, 2 * slot));
    for (int k = 0; k < 2; ++k) {
      char *base = static_cast<char *>(ctx->stage_mem) + k * slot;
      for (int j = 0; j < 12; ++j) ctx->stage_f[k][j] = reinterpret_cast<double *>(base + j * nd);
      ctx->stage_nsub[k] = reinterpret_cast<int32_t *>(base + 12 * nd);
      ctx->stage_status[k] = reinterpret_cast<uint8_t *>(base + 12 * nd + ni);
    }
    ctx->stage_cap = cells;
  }
  if (chunks > ctx->pipe_tab_cap) {
    cudaFree(ctx->pipe_tab);
    ctx->pipe_tab = nullptr;
    ctx->pipe_tab_cap = 0;
    // per slot: counter, chunk starts (int64), counts and blocks (int32)
    const size_t n8 = ((size_t)chunks * 8 + 255) / 256 * 256, n4 = ((size_t)chunks * 4 + 255) / 256 * 256;
    const size_t slot = 256 + n8 + 2 * n4;
    SFC_CUDA(cudaMalloc(&ctx->pipe_tab, 2 * slot));
    for (int k = 0; k < 2; ++k) {
      char *base = static_cast<char *>(ctx->pipe_tab) + k * slot;
      ctx->pipe_counter[k] = reinterpret_cast<unsigned long long *>(base);
      ctx->pipe_ch_start[k] = reinterpret_cast<int64_t *>(base + 256);
      ctx->pipe_ch_count[k] = reinterpret_cast<int32_t *>(base + 256 + n8);
      ctx->pipe_ch_block[k] = reinterpret_cast<int32_t *>(base + 256 + n8 + n4);
    }
    ctx->pipe_tab_cap = chunks;
  }
  return SFCHEM_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

void sfchem_config_default(sfchem_config_t *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->precision = SFCHEM_FP64;
  c->n_cyc = 300;
  c->n_sub_max = 100000;
  c->nr_itr_limit = 20;
  c->f_chem = 0.03;
  c->Z = 1.0;
  c->gamma_ad = 5.0 / 3.0;
  c->y_floor = 1e-8;
  c->nr_tol = 1e-5;
  c->reaction_mask = 0xFFFu;
  c->process_mask = SFCHEM_P_ALL;
  c->flags = 0u;
}

int sfchem_config_validate(const sfchem_config_t *cfg) { return validate_cfg(cfg); }

int sfchem_init(const sfchem_config_t *cfg, sfchem_ctx **out) {
  if (!out) return SFCHEM_EINVAL;
  *out = nullptr;
  sfchem_config_t c;
  if (cfg) c = *cfg; else sfchem_config_default(&c);
  if (validate_cfg(&c)) return SFCHEM_EINVAL;
  sfchem_ctx *ctx = new (std::nothrow) sfchem_ctx();
  if (!ctx) return SFCHEM_ENOMEM;
  ctx->cfg = c;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counter, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stats, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sfchem_schedule, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((sizeof(float) + sizeof(int32_t)) * SCHED_SORT_MAX));
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "sfchem_init");
    cudaFree(ctx->d_counter);
    cudaFree(ctx->d_stats);
    delete ctx;
    return rc == SFCHEM_ECUDA && e == cudaErrorMemoryAllocation ? SFCHEM_ENOMEM : rc;
  }
  ctx->sched_chunk = -1;
  ctx->magic = CTX_MAGIC;
  *out = ctx;
  return SFCHEM_OK;
}

int sfchem_set_config(sfchem_ctx *ctx, const sfchem_config_t *cfg) {
  if (int rc = check_ctx(ctx)) return rc;
  if (validate_cfg(cfg)) return SFCHEM_EINVAL;
  ctx->cfg = *cfg;
  return SFCHEM_OK;
}

int sfchem_step(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields, int64_t n_cells,
                double dt_seconds, double cd_factor, void *stream) {
  if (int rc = check_ctx(ctx)) return rc;
  if (n_cells < 0 || !(std::isfinite(dt_seconds) && dt_seconds >= 0.0) ||
      !(std::isfinite(cd_factor) && cd_factor > 0.0))
    return SFCHEM_EINVAL;
  if (n_cells == 0) return SFCHEM_OK;   // nothing is read: empty arrays may be NULL
  if (int rc = check_arrays(state, fields)) return rc;
  Shape sh;
  if (int rc = resolve_shape(ctx, sh)) return rc;
  const int64_t n_chunks = (n_cells + sh.chunk - 1) / sh.chunk;
  if (n_chunks > INT32_MAX) return SFCHEM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  KArgs a = base_args(ctx, state, fields, cd_factor);
  a.n_cells = n_cells;
  a.dt = dt_seconds;
  a.chunk = sh.chunk;
  a.n_chunks = (int32_t)n_chunks;
  SFC_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), s));
  SFC_CUDA(cudaEventRecord(ctx->ev0, s));
  SFC_CUDA(launch_solver(ctx, a, sh, s));
  SFC_CUDA(cudaEventRecord(ctx->ev1, s));
  ctx->timed = true;
  ctx->calls++;
  return SFCHEM_OK;
}

int sfchem_step_nr(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields, int64_t n_cells,
                   double dt_seconds, double cd_factor, void *stream) {
  if (int rc = check_ctx(ctx)) return rc;
  if (n_cells < 0 || !(std::isfinite(dt_seconds) && dt_seconds >= 0.0) ||
      !(std::isfinite(cd_factor) && cd_factor > 0.0))
    return SFCHEM_EINVAL;
  if (n_cells == 0) return SFCHEM_OK;
  if (int rc = check_arrays(state, fields)) return rc;
  const int tpb = 128;
  int occ = 0;
  SFC_CUDA(occupancy_nr_fp64(tpb, &occ));
  Shape sh;
  sh.tpb = tpb;
  sh.ctas_per_sm = occ > 0 ? occ : 1;
  sh.chunk = 32;
  sh.grid = ctx->num_sms * sh.ctas_per_sm;
  const int64_t n_chunks = (n_cells + sh.chunk - 1) / sh.chunk;
  if (n_chunks > INT32_MAX) return SFCHEM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  KArgs a = base_args(ctx, state, fields, cd_factor);
  a.n_cells = n_cells;
  a.dt = dt_seconds;
  a.chunk = sh.chunk;
  a.n_chunks = (int32_t)n_chunks;
  SFC_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(unsigned long long), s));
  SFC_CUDA(cudaEventRecord(ctx->ev0, s));
  SFC_CUDA(launch_nr_fp64(a, sh.grid, sh.tpb, s));
  SFC_CUDA(cudaEventRecord(ctx->ev1, s));
  ctx->timed = true;
  ctx->calls++;
  return SFCHEM_OK;
}

int sfchem_step_batched(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                        const int64_t *block_offset, const double *block_dt, int32_t n_blocks, double cd_factor,
                        void *stream) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!(std::isfinite(cd_factor) && cd_factor > 0.0)) return SFCHEM_EINVAL;
  if (int rc = check_arrays(state, fields)) return rc;
  Shape sh;
  if (int rc = resolve_shape(ctx, sh)) return rc;
  int64_t ncells = 0, nch = 0;
  if (int rc = check_blocks(block_offset, block_dt, n_blocks, sh.chunk, &ncells, &nch)) return rc;
  if (n_blocks == 0 || ncells == 0) return SFCHEM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = sync_schedule(ctx, block_offset, block_dt, n_blocks, sh.chunk, (int32_t)nch, s)) return rc;
  SFC_CUDA(cudaEventRecord(ctx->ev0, s));
  if (int rc = batched_launch(ctx, state, fields, n_blocks, cd_factor, sh, s, true)) return rc;
  SFC_CUDA(cudaEventRecord(ctx->ev1, s));
  ctx->timed = true;
  ctx->calls++;
  return SFCHEM_OK;
}

int sfchem_step_host(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                     const int64_t *block_offset, const double *block_dt, int32_t n_blocks, double cd_factor,
                     int64_t slice_cells, void *stream) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!(std::isfinite(cd_factor) && cd_factor > 0.0) || slice_cells < 0) return SFCHEM_EINVAL;
  if (int rc = check_arrays(state, fields)) return rc;
  Shape sh;
  if (int rc = resolve_shape(ctx, sh)) return rc;
  int64_t ncells = 0, nch = 0;
  if (int rc = check_blocks(block_offset, block_dt, n_blocks, sh.chunk, &ncells, &nch)) return rc;
  if (n_blocks == 0 || ncells == 0) return SFCHEM_OK;
  if (slice_cells == 0) slice_cells = SFCHEM_HOST_SLICE_DEFAULT;
  // slices: runs of whole consecutive blocks of at most slice_cells cells
  // (a larger block is a slice of its own).  The copy-in of the first slice
  // and the copy-out of the last one overlap no solver work, so those two
  // slices take a quarter of slice_cells.
  std::vector<int32_t> cut(1, 0);
  int64_t max_slice = 0, max_chunks = 0;
  const int64_t total = block_offset[n_blocks], quarter = std::max<int64_t>(slice_cells / 4, 1);
  for (int32_t b = 0; b < n_blocks;) {
    const int64_t left = total - block_offset[b];
    int64_t target = slice_cells;
    if (b == 0) target = quarter;
    else if (left > quarter && left <= slice_cells + quarter) target = left - quarter;
    int32_t e = b + 1;
    while (e < n_blocks && block_offset[e + 1] - block_offset[b] <= target) ++e;
    max_slice = std::max(max_slice, block_offset[e] - block_offset[b]);
    int64_t chunks = 0;
    for (int32_t q = b; q < e; ++q) chunks += (block_offset[q + 1] - block_offset[q] + sh.chunk - 1) / sh.chunk;
    max_chunks = std::max(max_chunks, chunks);
    cut.push_back(e);
    b = e;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = sync_schedule(ctx, block_offset, block_dt, n_blocks, sh.chunk, (int32_t)nch, s)) return rc;
  if (int rc = ensure_pipeline(ctx, max_slice, max_chunks)) return rc;
  const double *in_h[9] = {state->n_H, state->T_gas, state->T_dust, state->E_IR, state->y_H2, state->y_e,
                           fields->G0_fuv, fields->n_euv, fields->N_H2};
  double *out_h[8] = {state->T_gas, state->T_dust, state->E_IR, state->y_H2, state->y_e,
                      state->y_H, state->y_Hp, state->y_Hm};
  const int out_j[8] = {1, 2, 3, 4, 5, 9, 10, 11};
  // the copies are ordered after the work already queued on `stream`
  SFC_CUDA(cudaEventRecord(ctx->ev_start, s));
  cudaStream_t deps[4] = {ctx->s_in, ctx->s_out, ctx->s_comp[0], ctx->s_comp[1]};
  for (cudaStream_t d : deps) SFC_CUDA(cudaStreamWaitEvent(d, ctx->ev_start, 0));
  const size_t smem = (sizeof(float) + sizeof(int32_t)) * SCHED_SORT_MAX;
  for (size_t i = 0; i + 1 < cut.size(); ++i) {
    const int k = (int)(i & 1);
    const int32_t b0 = cut[i], b1 = cut[i + 1], nb = b1 - b0;
    const int64_t c0 = block_offset[b0], nc = block_offset[b1] - c0;
    int64_t chunks = 0;
    for (int32_t b = b0; b < b1; ++b) chunks += (block_offset[b + 1] - block_offset[b] + sh.chunk - 1) / sh.chunk;
    // in: wait until slot k's previous results are home, then copy the inputs
    if (i >= 2) SFC_CUDA(cudaStreamWaitEvent(ctx->s_in, ctx->ev_free[k], 0));
    for (int j = 0; j < 9; ++j)
      SFC_CUDA(cudaMemcpyAsync(ctx->stage_f[k][j], in_h[j] + c0, sizeof(double) * nc, cudaMemcpyHostToDevice,
                               ctx->s_in));
    SFC_CUDA(cudaEventRecord(ctx->ev_in[k], ctx->s_in));
    // compute on slot k's stream: the slice's chunk table, then the solver
    // (it overlaps the end of the previous slice's solver on the other one)
    cudaStream_t sc = ctx->s_comp[k];
    SFC_CUDA(cudaStreamWaitEvent(sc, ctx->ev_in[k], 0));
    sfchem_state_t st;
    std::memset(&st, 0, sizeof(st));
    double *const *f = ctx->stage_f[k];
    st.n_H = f[0]; st.T_gas = f[1]; st.T_dust = f[2]; st.E_IR = f[3]; st.y_H2 = f[4]; st.y_e = f[5];
    st.y_H = state->y_H ? f[9] : nullptr;
    st.y_Hp = state->y_Hp ? f[10] : nullptr;
    st.y_Hm = state->y_Hm ? f[11] : nullptr;
    st.status = state->status ? ctx->stage_status[k] : nullptr;
    st.n_sub = state->n_sub ? ctx->stage_nsub[k] : nullptr;
    st.n_itr = nullptr;   // not staged: sfchem_step_host does not write n_itr
    sfchem_fields_t fl;
    fl.G0_fuv = f[6]; fl.n_euv = f[7]; fl.N_H2 = f[8];
    KArgs a = base_args(ctx, &st, &fl, cd_factor);
    a.n_cells = nc;
    a.chunk = sh.chunk;
    a.n_chunks = (int32_t)chunks;
    a.ch_start = ctx->pipe_ch_start[k]; a.ch_count = ctx->pipe_ch_count[k]; a.ch_block = ctx->pipe_ch_block[k];
    a.counter = ctx->pipe_counter[k];
    a.block_dt = ctx->d_block_dt + b0;
    a.block_cost = ctx->d_block_cost + b0;
    if (i == 0) SFC_CUDA(cudaEventRecord(ctx->ev0, sc));
    SFC_CUDA(cudaMemsetAsync(ctx->pipe_counter[k], 0, sizeof(unsigned long long), sc));
    sfchem_schedule<<<1, SCHED_THREADS, nb <= SCHED_SORT_MAX ? smem : 0, sc>>>(
        ctx->d_block_offset + b0, ctx->d_block_cost + b0, nb, sh.chunk, ctx->pipe_ch_start[k],
        ctx->pipe_ch_count[k], ctx->pipe_ch_block[k]);
    SFC_CUDA(cudaGetLastError());
    SFC_CUDA(launch_solver(ctx, a, sh, sc));
    SFC_CUDA(cudaEventRecord(ctx->ev_comp[k], sc));
    // out: copy the results home, then free slot k
    SFC_CUDA(cudaStreamWaitEvent(ctx->s_out, ctx->ev_comp[k], 0));
    for (int j = 0; j < 8; ++j)
      if (out_h[j])
        SFC_CUDA(cudaMemcpyAsync(out_h[j] + c0, f[out_j[j]], sizeof(double) * nc, cudaMemcpyDeviceToHost,
                                 ctx->s_out));
    if (state->status)
      SFC_CUDA(cudaMemcpyAsync(state->status + c0, ctx->stage_status[k], nc, cudaMemcpyDeviceToHost, ctx->s_out));
    if (state->n_sub)
      SFC_CUDA(cudaMemcpyAsync(state->n_sub + c0, ctx->stage_nsub[k], sizeof(int32_t) * nc,
                               cudaMemcpyDeviceToHost, ctx->s_out));
    SFC_CUDA(cudaEventRecord(ctx->ev_free[k], ctx->s_out));
  }
  SFC_CUDA(cudaEventRecord(ctx->ev_end, ctx->s_out));
  SFC_CUDA(cudaStreamWaitEvent(s, ctx->ev_end, 0));
  SFC_CUDA(cudaEventRecord(ctx->ev1, s));
  SFC_CUDA(cudaStreamSynchronize(s));
  ctx->timed = true;
  ctx->calls++;
  return SFCHEM_OK;
}

int sfchem_set_launch(sfchem_ctx *ctx, const sfchem_launch_t *launch) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!launch) { std::memset(&ctx->launch, 0, sizeof(ctx->launch)); return SFCHEM_OK; }
  const int t = launch->threads_per_cta;
  if (!(t == 0 || t == 64 || t == 128)) return SFCHEM_EINVAL;
  if (launch->ctas_per_sm < 0 || launch->chunk < 0 || (launch->chunk % 32) != 0 || launch->chunk > 4096 ||
      launch->reserved)
    return SFCHEM_EINVAL;
  ctx->launch = *launch;
  return SFCHEM_OK;
}

int sfchem_get_launch(sfchem_ctx *ctx, sfchem_launch_t *launch) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!launch) return SFCHEM_EINVAL;
  Shape sh;
  if (int rc = resolve_shape(ctx, sh)) return rc;
  launch->threads_per_cta = sh.tpb;
  launch->ctas_per_sm = sh.ctas_per_sm;
  launch->chunk = sh.chunk;
  launch->reserved = 0;
  return SFCHEM_OK;
}

int sfchem_autotune(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                    const int64_t *block_offset, const double *block_dt, int32_t n_blocks, double cd_factor,
                    void *stream) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!(std::isfinite(cd_factor) && cd_factor > 0.0)) return SFCHEM_EINVAL;
  if (int rc = check_arrays(state, fields)) return rc;
  int64_t ncells = 0, nch = 0;
  if (int rc = check_blocks(block_offset, block_dt, n_blocks, 32, &ncells, &nch)) return rc;
  if (n_blocks == 0 || ncells == 0) return SFCHEM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // library-owned copies of the evolved arrays
  double *buf = nullptr;
  SFC_CUDA(cudaMalloc(&buf, sizeof(double) * 5 * ncells));
  sfchem_state_t w = *state;
  w.T_gas = buf; w.T_dust = buf + ncells; w.E_IR = buf + 2 * ncells; w.y_H2 = buf + 3 * ncells;
  w.y_e = buf + 4 * ncells;
  w.y_H = w.y_Hp = w.y_Hm = nullptr;
  w.status = nullptr;
  w.n_sub = nullptr;
  const double *src[5] = {state->T_gas, state->T_dust, state->E_IR, state->y_H2, state->y_e};
  const sfchem_launch_t saved = ctx->launch;
  DevStats saved_stats;
  cudaError_t e = cudaMemcpyAsync(&saved_stats, ctx->d_stats, sizeof(DevStats), cudaMemcpyDeviceToHost, s);
  float best_ms = 1e30f;
  sfchem_launch_t best = saved;
  const int tpbs[2] = {64, 128};
  const int chunks[3] = {32, 64, 128};
  int rc = SFCHEM_OK;
  for (int ti = 0; ti < 2 && e == cudaSuccess && !rc; ++ti) {
    int occ = 0;
    e = ctx->cfg.precision == SFCHEM_MIXED ? occupancy_li_mixed(tpbs[ti], &occ) : occupancy_li_fp64(tpbs[ti], &occ);
    if (e != cudaSuccess) break;
    std::vector<int> cands;
    for (int cps = 1; cps < occ; cps *= 2) cands.push_back(cps);
    cands.push_back(std::max(occ, 1));
    for (int cps : cands) {
      if (rc) break;
      for (int ci = 0; ci < 3 && !rc; ++ci) {
        sfchem_launch_t l = {tpbs[ti], cps, chunks[ci], 0};
        ctx->launch = l;
        Shape sh;
        if ((rc = resolve_shape(ctx, sh))) break;
        int64_t nc2 = 0, nch2 = 0;
        if ((rc = check_blocks(block_offset, block_dt, n_blocks, sh.chunk, &nc2, &nch2))) break;
        if ((rc = sync_schedule(ctx, block_offset, block_dt, n_blocks, sh.chunk, (int32_t)nch2, s))) break;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && !rc; ++rep) {   // the second run uses the cost order of the first
          for (int k = 0; k < 5; ++k)
            if ((e = cudaMemcpyAsync(buf + k * ncells, src[k], sizeof(double) * ncells,
                                     cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
          if (e != cudaSuccess) break;
          cudaEventRecord(ctx->ev0, s);
          rc = batched_launch(ctx, &w, fields, n_blocks, cd_factor, sh, s, false);
          cudaEventRecord(ctx->ev1, s);
          if ((e = cudaEventSynchronize(ctx->ev1)) != cudaSuccess) break;
          cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        }
        if (e != cudaSuccess) break;
        if (!rc && ms < best_ms) { best_ms = ms; best = l; }
      }
    }
  }
  ctx->launch = (rc || e != cudaSuccess) ? saved : best;
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_stats, &saved_stats, sizeof(DevStats), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  ctx->timed = false;
  drop_graph(ctx);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "sfchem_autotune");
  return SFCHEM_OK;
}

// Greedy test of a bottleneck: can blocks [0, n) be cut into at most
// n_parts contiguous ranges whose costs stay <= cap?  Writes the cut when
// `cut` is not NULL (ranges left over at the end are empty).
static bool partition_fits(const double *cost, int32_t n, int32_t n_parts, double cap, int32_t *cut) {
  int32_t part = 0;
  double acc = 0.0;
  if (cut) cut[0] = 0;
  for (int32_t b = 0; b < n; ++b) {
    if (acc > 0.0 && acc + cost[b] > cap) {
      if (++part >= n_parts) return false;
      if (cut) cut[part] = b;
      acc = 0.0;
    }
    acc += cost[b];
  }
  if (cut)
    for (int32_t k = part + 1; k <= n_parts; ++k) cut[k] = n;
  return true;
}

int sfchem_partition(const int64_t *block_offset, const double *block_cost, int32_t n_blocks, int32_t n_parts,
                     int32_t *cut) {
  if (!block_offset || !cut || n_blocks < 0 || n_parts < 1) return SFCHEM_EINVAL;
  if (block_offset[0] != 0) return SFCHEM_EINVAL;
  std::vector<double> cost(n_blocks);
  double total = 0.0, big = 0.0;
  for (int32_t b = 0; b < n_blocks; ++b) {
    const int64_t cells = block_offset[b + 1] - block_offset[b];
    if (cells < 0) return SFCHEM_EINVAL;
    double c = block_cost ? block_cost[b] : (double)cells;
    if (!(std::isfinite(c) && c >= 0.0)) return SFCHEM_EINVAL;
    // a block that costs nothing measurable still takes time to load and store
    if (block_cost && c == 0.0) c = (double)cells;
    cost[b] = c;
    total += c;
    big = std::max(big, c);
  }
  if (n_blocks == 0 || total == 0.0) {
    for (int32_t k = 0; k <= n_parts; ++k) cut[k] = k == 0 ? 0 : n_blocks;
    return SFCHEM_OK;
  }
  // bisection on the largest part cost between its lower bound
  // max(total / n_parts, largest block) and the greedy bound lo + largest
  // block, to a relative width of 1e-12
  double lo = std::max(total / n_parts, big), hi = lo + big;
  while (!partition_fits(cost.data(), n_blocks, n_parts, hi, nullptr)) hi *= 2.0;   // rounding safety
  for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (partition_fits(cost.data(), n_blocks, n_parts, mid, nullptr)) hi = mid;
    else lo = mid;
  }
  partition_fits(cost.data(), n_blocks, n_parts, hi, cut);
  return SFCHEM_OK;
}

int sfchem_block_costs(sfchem_ctx *ctx, float *cost, int32_t n_blocks) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!cost || n_blocks < 0 || n_blocks > ctx->cap_blocks ||
      (int64_t)ctx->h_block_dt.size() != n_blocks)
    return SFCHEM_EINVAL;
  if (n_blocks == 0) return SFCHEM_OK;
  SFC_CUDA(cudaDeviceSynchronize());
  SFC_CUDA(cudaMemcpy(cost, ctx->d_block_cost, sizeof(float) * n_blocks, cudaMemcpyDeviceToHost));
  return SFCHEM_OK;
}

int sfchem_stats(sfchem_ctx *ctx, sfchem_stats_t *out) {
  if (int rc = check_ctx(ctx)) return rc;
  if (!out) return SFCHEM_EINVAL;
  DevStats d;
  SFC_CUDA(cudaDeviceSynchronize());
  SFC_CUDA(cudaMemcpy(&d, ctx->d_stats, sizeof(d), cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof(*out));
  out->calls = ctx->calls;
  out->cells = d.cells;
  out->substeps = d.substeps;
  out->newton_iters = d.newton;
  out->tight_cells = d.tight;
  out->capped_cells = d.cap;
  out->noconv_cells = d.noconv;
  out->badinput_cells = d.bad;
  out->badstep_cells = d.badstep;
  out->rejected_substeps = d.rejected;
  out->step_halvings = d.halvings;
  out->max_substeps = d.max_sub;
  float ms = 0.0f;
  if (ctx->timed && cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) out->last_kernel_ms = ms;
  return SFCHEM_OK;
}

int sfchem_stats_reset(sfchem_ctx *ctx) {
  if (int rc = check_ctx(ctx)) return rc;
  SFC_CUDA(cudaMemset(ctx->d_stats, 0, sizeof(DevStats)));
  ctx->calls = 0;
  return SFCHEM_OK;
}

int sfchem_finalize(sfchem_ctx *ctx) {
  if (int rc = check_ctx(ctx)) return rc;
  cudaDeviceSynchronize();
  drop_graph(ctx);
  cudaFree(ctx->d_counter);
  cudaFree(ctx->d_stats);
  cudaFree(ctx->d_block_offset);
  cudaFree(ctx->d_block_dt);
  cudaFree(ctx->d_block_cost);
  cudaFree(ctx->d_ch_start);
  cudaFree(ctx->d_ch_count);
  cudaFree(ctx->d_ch_block);
  cudaEventDestroy(ctx->ev0);
  cudaEventDestroy(ctx->ev1);
  cudaStreamDestroy(ctx->cap_stream);
  if (ctx->have_pipe) {
    cudaStreamDestroy(ctx->s_in);
    cudaStreamDestroy(ctx->s_out);
    cudaStreamDestroy(ctx->s_comp[0]);
    cudaStreamDestroy(ctx->s_comp[1]);
    cudaEvent_t evs[8] = {ctx->ev_start, ctx->ev_end, ctx->ev_in[0], ctx->ev_in[1], ctx->ev_comp[0],
                          ctx->ev_comp[1], ctx->ev_free[0], ctx->ev_free[1]};
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
  }
  cudaFree(ctx->stage_mem);
  cudaFree(ctx->pipe_tab);
  ctx->magic = 0;
  delete ctx;
  return SFCHEM_OK;
}

const char *sfchem_strerror(int status) {
  switch (status) {
    case SFCHEM_OK: return "success";
    case SFCHEM_EINVAL: return "invalid argument";
    case SFCHEM_ENOTINIT: return "context not initialized";
    case SFCHEM_ECUDA: return "CUDA error";
    case SFCHEM_ETIMEOUT: return "bounded device wait timed out";
    case SFCHEM_ENOMEM: return "out of memory";
    default: return "unknown status";
  }
}

const char *sfchem_last_cuda_error(void) { return g_cuda_err; }

const char *sfchem_version(void) { return "0.1.0"; }

}  // extern "C"
