/*
 * sfchem.h -- C ABI of libsfchem, the GB300 (sm_103a) per-cell thermochemical
 * update of SFUMATO# (Fukushima & Matsumoto, arXiv 2604.21438).
 *
 * One call advances every cell by its hydro time step dt with the paper's
 * linearized-implicit (LI) solver (Sec. 2.2.8, Eqs. eq_chem2..eq_deq): the
 * hydrogen network of Table 3 (H, H2, H+, e; H- in equilibrium), the heating
 * and cooling of Table 4, and the dust-temperature / IR-energy / gas-grain
 * update of Appendix C (Eqs. ap_eq:dust_temp..ap_eq:zeta) with the pseudo dust
 * heat capacity C_d = cd_factor * 1e4 erg g^-1 K^-1.  Each cell subcycles with
 * dt_s = f_chem * min(dt_dust, dt_chem, dt_energy) (Eqs. timescale_of_dust,
 * timescale_chemi, timescale_energy, timestep_subcycle); when the estimated
 * number of subcycles reaches N_cyc the dust timescale is dropped and the
 * dust and IR rows are iterated to the backward-Euler solution instead (the
 * tight-coupling mode of Sec. 2.2.8).  The five unknowns (y_H2, y_e, T_g, T_d,
 * E_IR) are solved together as one 5x5 linear system per substep.
 *
 * Memory: every array is a caller-owned DEVICE pointer to contiguous FP64
 * (uint8 / int32 for status and n_sub), one entry per cell, structure of
 * arrays -- except for sfchem_step_host, which takes HOST arrays.  Units are
 * CGS; temperatures in K; dt in seconds.  Calls are asynchronous on the
 * caller's stream (sfchem_step_host returns when its results are home); the
 * arrays must stay valid until the stream reaches the call.  The library owns
 * only its context (work counters, statistics, schedule tables, captured CUDA
 * graphs, and the staging slots and streams of sfchem_step_host).
 *
 * Precision: SFCHEM_FP64 runs every step in FP64 (the paper's arithmetic).
 * SFCHEM_MIXED evaluates the rates, heating/cooling, Jacobian and the 5x5
 * factorization in FP32, and keeps the state, its update and projection, the
 * time left and one residual-refinement pass of each solve in FP64 (the
 * residual in FP32 error-free arithmetic with SFCHEM_F_REFINE_FF); its error
 * against FP64 is stated by the library's tests (median <= 2e-6, p99 <= 1e-3
 * relative on every field).
 *
 * Errors: every entry point returns an sfchem_status code.  Argument errors
 * are detected on the host before anything is launched.  Problems of single
 * cells are not call errors: they set bits of status[i] and count in the
 * statistics (see SFCHEM_CELL_*).
 *
 * Threading: a context serves one stream at a time; use one context per
 * concurrent stream.
 */
#ifndef SFCHEM_H
#define SFCHEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
typedef enum {
  SFCHEM_OK = 0,
  SFCHEM_EINVAL = 1,    /* bad argument (NULL or misaligned pointer, n < 0, dt < 0, ...) */
  SFCHEM_ENOTINIT = 2,  /* NULL or finalized context */
  SFCHEM_ECUDA = 3,     /* a CUDA call failed; sfchem_last_cuda_error() has the text */
  SFCHEM_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  SFCHEM_ENOMEM = 5     /* a library allocation failed */
} sfchem_status;

/* precision of the rate / Jacobian / LU arithmetic */
enum { SFCHEM_FP64 = 0, SFCHEM_MIXED = 1 };

/* per-cell status bits (status[i]) */
enum {
  SFCHEM_CELL_CAP = 1u << 0,      /* stopped at n_sub_max substeps before dt */
  SFCHEM_CELL_BADINPUT = 1u << 1, /* invalid input; the cell is left unchanged */
  SFCHEM_CELL_NOCONV = 1u << 2,   /* a tight-coupling Newton loop hit nr_itr_limit */
  SFCHEM_CELL_TIGHT = 1u << 3,    /* cell ran in the tight-coupling mode */
  SFCHEM_CELL_BADSTEP = 1u << 4   /* non-finite substep or singular system; stopped */
};

/* process_mask bits: rows of Table 4 and the Appendix C dust terms */
enum {
  SFCHEM_P_G1_H2FORM = 1u << 0,    /* H2 formation heating */
  SFCHEM_P_G2_PHOTOION = 1u << 1,  /* H photoionization heating */
  SFCHEM_P_G3_PHOTODISS = 1u << 2, /* H2 photodissociation heating */
  SFCHEM_P_G4_PHOTOELEC = 1u << 3, /* photoelectric heating */
  SFCHEM_P_L5_HION = 1u << 4,      /* H collisional ionization cooling */
  SFCHEM_P_L6_H2DISS = 1u << 5,    /* H2 dissociation cooling */
  SFCHEM_P_L7_HREC = 1u << 6,      /* H recombination cooling */
  SFCHEM_P_L8_HMFB = 1u << 7,      /* H- free-bound cooling */
  SFCHEM_P_L9_HEXC = 1u << 8,      /* H excitation cooling */
  SFCHEM_P_L10_HEPEXC = 1u << 9,   /* He+ excitation cooling */
  SFCHEM_P_L11_FF = 1u << 10,      /* free-free cooling */
  SFCHEM_P_L12_COMPTON = 1u << 11, /* Compton cooling */
  SFCHEM_P_L13_LINE = 1u << 12,    /* metal line cooling */
  SFCHEM_P_GASGRAIN = 1u << 13,    /* gas-grain energy transfer */
  SFCHEM_P_DUST_UV = 1u << 14,     /* dust absorption of EUV/FUV */
  SFCHEM_P_DUST_EMIT = 1u << 15,   /* dust thermal emission */
  SFCHEM_P_DUST_IRABS = 1u << 16,  /* dust absorption of IR */
  SFCHEM_P_ALL = (1u << 17) - 1u
};

/* flags */
enum {
  SFCHEM_F_FREEZE_TG = 1u << 0,  /* hold T_gas fixed */
  SFCHEM_F_FREEZE_TD = 1u << 1,  /* hold T_dust fixed */
  SFCHEM_F_FREEZE_EIR = 1u << 2, /* hold E_IR fixed */
  SFCHEM_F_FREEZE_YH2 = 1u << 3, /* hold y_H2 fixed */
  SFCHEM_F_FREEZE_YE = 1u << 4,  /* hold y_e fixed */
  SFCHEM_F_SPLIT = 1u << 5,      /* drop the chemistry <-> energy cross-derivatives */
  SFCHEM_F_REFINE_FF = 1u << 6,  /* mixed precision: form the refinement residual with error-free
                                    FP32 transformations (about 48 bits) instead of FP64 */
  SFCHEM_F_NO_REJECT = 1u << 7   /* the substep controller exactly as Eq. timestep_subcycle prints
                                    it: no step rejection (see sfchem_stats_t.rejected_substeps) */
};

/* ------------------------------------------------------------------ types */
typedef struct sfchem_ctx sfchem_ctx; /* opaque */

/* Cell state.  n_H is read; T_gas, T_dust, E_IR, y_H2, y_e are read and
 * overwritten; y_H, y_Hp, y_Hm, status, n_sub, n_itr are written when
 * non-NULL.
 * y_H = 1 - 2 y_H2 - y_e and y_Hp = y_e (H-nuclei conservation and charge
 * neutrality, Sec. 2.2.8); y_Hm = k_H2 y_e / k_H3 (H- equilibrium, Table 3,
 * at the final T_gas), formed by a second kernel that each step call queues
 * on its stream after the solver.  Cells with invalid inputs get NaN in y_H,
 * y_Hp and y_Hm. */
typedef struct {
  const double *n_H;   /* H-nuclei number density [cm^-3], > 0 */
  double *T_gas;       /* gas temperature [K] */
  double *T_dust;      /* dust temperature [K] */
  double *E_IR;        /* IR radiation energy density [erg cm^-3], >= 0 */
  double *y_H2;        /* H2 abundance per H nucleus */
  double *y_e;         /* electron abundance per H nucleus (= y_H+) */
  double *y_H;         /* out: atomic H abundance (may be NULL) */
  double *y_Hp;        /* out: H+ abundance (may be NULL) */
  double *y_Hm;        /* out: H- abundance (may be NULL) */
  uint8_t *status;     /* out: SFCHEM_CELL_* bits (may be NULL) */
  int32_t *n_sub;      /* out: substeps taken (may be NULL) */
  int32_t *n_itr;      /* out: Newton iterations of the cell (may be NULL): the tight-coupling
                          iterations of the LI method, the outer T_gas iterations of
                          sfchem_step_nr; sfchem_step_host does not write it */
} sfchem_state_t;

/* Radiation inputs per cell (read only). */
typedef struct {
  const double *G0_fuv; /* FUV field in Habing units */
  const double *n_euv;  /* EUV photon number density [cm^-3] */
  const double *N_H2;   /* H2 column density for self-shielding [cm^-2] */
} sfchem_fields_t;

/* Solver parameters.  sfchem_config_default() fills the paper's values:
 * f_chem = 0.03 and N_cyc = 300 (Sec. 2.2.8), Newton limit 20 and tolerance
 * 1e-5 (Sec. 2.2.8), Z = 1, gamma_ad = 5/3, y_floor = 1e-8,
 * n_sub_max = 100000, every reaction and process on, no flags. */
typedef struct {
  int32_t precision;      /* SFCHEM_FP64 or SFCHEM_MIXED */
  int32_t n_cyc;          /* subcycle limit N_cyc */
  int32_t n_sub_max;      /* substep cap per cell and call */
  int32_t nr_itr_limit;   /* tight-coupling Newton iteration limit */
  double f_chem;          /* substep factor, 0 < f_chem <= 1 */
  double Z;               /* metallicity / Z_sun; dust abundance f_d = Z */
  double gamma_ad;        /* adiabatic exponent, > 1 */
  double y_floor;         /* abundance floor in dt_chem, > 0 */
  double nr_tol;          /* tight-coupling Newton tolerance, > 0 */
  uint32_t reaction_mask; /* bit i enables reaction H<i> of Table 3 (i = 0..11) */
  uint32_t process_mask;  /* SFCHEM_P_* */
  uint32_t flags;         /* SFCHEM_F_* */
  uint32_t reserved;      /* must be 0 */
} sfchem_config_t;

/* Per-context statistics, accumulated over calls since the last reset. */
typedef struct {
  uint64_t calls;
  uint64_t cells;           /* cells processed */
  uint64_t substeps;        /* sum of n_sub */
  uint64_t newton_iters;    /* tight-coupling Newton iterations */
  uint64_t tight_cells;     /* cells in the tight-coupling mode */
  uint64_t capped_cells;    /* SFCHEM_CELL_CAP */
  uint64_t noconv_cells;    /* SFCHEM_CELL_NOCONV */
  uint64_t badinput_cells;  /* SFCHEM_CELL_BADINPUT */
  uint64_t badstep_cells;   /* SFCHEM_CELL_BADSTEP */
  /* Step rejection (a reading of the small-change assumption behind Eq.
   * eq_deq; the paper's controller has no such step): an update that moves
   * y_H2 or y_e by more than half of max(y, y_floor), or T_gas by more than
   * a factor 2, is redone with half the step, at most 30 times.
   * rejected_substeps counts the substeps that were redone at least once,
   * step_halvings the halvings they took (both 0 under SFCHEM_F_NO_REJECT). */
  uint64_t rejected_substeps;
  uint64_t step_halvings;
  uint32_t max_substeps;    /* largest n_sub of a cell */
  uint32_t reserved;
  double last_kernel_ms;    /* device time of the last call's solver kernel */
} sfchem_stats_t;

/* Launch shape of the persistent kernels; zero fields mean "library
 * default / autotuned". */
typedef struct {
  int32_t threads_per_cta;  /* 64 or 128 */
  int32_t ctas_per_sm;      /* resident CTAs per SM, >= 1 */
  int32_t chunk;            /* cells claimed per warp refill (multiple of 32) */
  int32_t reserved;
} sfchem_launch_t;

/* --------------------------------------------------------------- functions */

/* Fill *cfg with the defaults listed above.  cfg must not be NULL. */
void sfchem_config_default(sfchem_config_t *cfg);

/* Check a configuration on the host.  Returns SFCHEM_OK or SFCHEM_EINVAL. */
int sfchem_config_validate(const sfchem_config_t *cfg);

/* Create a context on the current CUDA device (allocates the library-owned
 * scratch: work counters and statistics, a few hundred bytes).  cfg may be
 * NULL for the defaults; *out receives the context.  SFCHEM_EINVAL on a bad
 * config, SFCHEM_ECUDA / SFCHEM_ENOMEM when the device allocation fails. */
int sfchem_init(const sfchem_config_t *cfg, sfchem_ctx **out);

/* Replace the context's configuration (host-side check first). */
int sfchem_set_config(sfchem_ctx *ctx, const sfchem_config_t *cfg);

/* Advance n_cells cells by dt_seconds each (Sec. 2.2.8) on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  cd_factor sets
 * C_d = cd_factor * 1e4 erg g^-1 K^-1 (> 0).  n_cells == 0 is a no-op (the
 * arrays are not read and may be NULL).
 * Pointers must be 8-byte aligned device pointers (state and fields arrays
 * of n_cells entries).  Asynchronous: returns once its kernels are queued. */
int sfchem_step(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                int64_t n_cells, double dt_seconds, double cd_factor, void *stream);

/* Batched AMR form: cells are grouped in n_blocks contiguous blocks; block b
 * holds cells [block_offset[b], block_offset[b+1]) and advances by
 * block_dt[b] seconds (per-level time steps, Eqs. timestep, timestep2).
 * block_offset (int64, n_blocks + 1 entries, non-decreasing, starting at 0)
 * and block_dt (n_blocks entries, >= 0) are HOST arrays, read during the
 * call.  One persistent work-stealing kernel processes all blocks, most
 * expensive first (by the previous call's substep counts of the same
 * schedule); the launch sequence is captured once in a CUDA graph per
 * (schedule, arrays, stream) and replayed.  Asynchronous like sfchem_step. */
int sfchem_step_batched(sfchem_ctx *ctx, const sfchem_state_t *state,
                        const sfchem_fields_t *fields, const int64_t *block_offset,
                        const double *block_dt, int32_t n_blocks, double cd_factor,
                        void *stream);

/* sfchem_step_batched on state and fields in HOST memory (no counterpart in
 * the paper, whose solver runs on device-resident hydro data; this is the
 * call for a caller whose cells live on the host).  The blocks are cut into
 * slices of consecutive whole blocks of at most slice_cells cells (0: the
 * default below; a larger block is a slice of its own; the first and the
 * last slice take a quarter of it, since their copies overlap no solver
 * work).  While slice i is solved, the inputs of slice i+1 are copied to the
 * device and the results of slice i-1 back to the host; the solvers of
 * consecutive slices overlap.  The library owns the streams (copy-in,
 * copy-out, one compute stream per slot) and two device staging slots (each
 * grown on demand to the largest slice: 101 bytes per cell, plus its chunk
 * table).  All arrays of state and fields are host arrays of
 * block_offset[n_blocks] entries (pinned memory gives asynchronous copies;
 * pageable memory works, copied synchronously by the driver); optional
 * outputs (y_H, y_Hp, y_Hm, status, n_sub) may be NULL and are then neither
 * computed into nor copied.  The work is ordered after the work already
 * queued on `stream`, and the call returns when every result is in host
 * memory (it synchronizes `stream`).  Errors as sfchem_step_batched;
 * slice_cells < 0 is SFCHEM_EINVAL. */
#define SFCHEM_HOST_SLICE_DEFAULT 16777216
int sfchem_step_host(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                     const int64_t *block_offset, const double *block_dt, int32_t n_blocks,
                     double cd_factor, int64_t slice_cells, void *stream);

/* The Newton-Raphson reference solver of Sec. 2.2.8 (FP64), which the paper
 * validates the LI method against: backward Euler over dt_seconds by three
 * nested Newton groups -- T_gas outer with a central-difference derivative,
 * (T_dust, E_IR), species -- to a relative change of nr_tol (relaxed to 1e-3
 * after nr_itr_limit/2 outer iterations), with substeps
 * dt_sub = (dt - t_sub)/2^i on failure (Eq. substep_NRchem).  Same arrays,
 * masks and flags as sfchem_step (precision is ignored); n_sub counts the
 * accepted substeps and the statistics' newton_iters the outer iterations.
 * SFCHEM_CELL_NOCONV marks a cell that gave up.  Asynchronous. */
int sfchem_step_nr(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                   int64_t n_cells, double dt_seconds, double cd_factor, void *stream);

/* Force a launch shape (NULL restores the default / autotuned one). */
int sfchem_set_launch(sfchem_ctx *ctx, const sfchem_launch_t *launch);

/* Read the launch shape in use (after autotuning, the chosen one). */
int sfchem_get_launch(sfchem_ctx *ctx, sfchem_launch_t *launch);

/* Autotune the batched kernel's launch shape on this workload: runs each
 * candidate (threads per CTA x CTAs per SM x chunk) on library-owned copies
 * of the state (the caller's arrays are not modified), times it with CUDA
 * events and keeps the fastest for this context.  Synchronizes `stream`. */
int sfchem_autotune(sfchem_ctx *ctx, const sfchem_state_t *state, const sfchem_fields_t *fields,
                    const int64_t *block_offset, const double *block_dt, int32_t n_blocks,
                    double cd_factor, void *stream);

/* Photon consumption after the thermochemical update (Sec. 2.2.8,
 * "Radiation components": the EUV and FUV photons of the step are absorbed
 * once the abundances and temperatures have been updated; the paper gives
 * the details in another paper, so this is a reading with stand-in
 * constants).  Per cell, with y_H = 1 - 2 y_H2 - y_e of the UPDATED state
 * (call it after sfchem_step on the same arrays): each band loses photons at
 * a rate per photon lam, taken implicitly over dt_seconds,
 *   EUV: lam = c n_H (sigma_H y_H + sigma_d),   n_euv_out = n_euv / (1 + lam dt)
 *   FUV: lam = k_LW f_sh(N_H2) n_H y_H2 h nu_F / u_Habing + c n_H sigma_d,
 *        G0_out = G0 / (1 + lam dt)
 * (sigma_H: the cross-section of k_H9; k_LW f_sh: k_H10 per Habing unit, one
 * photon per photodissociation; sigma_d, u_Habing: the dust UV absorption of
 * Appendix C's E_UV; h nu_F = 12.4 eV), so that no band goes negative and
 * the photons removed are the photons absorbed.  Reads state->n_H, y_H2,
 * y_e and fields->G0_fuv, n_euv, N_H2 (device arrays of n_cells); writes
 * G0_out and n_euv_out (device arrays of n_cells; they may be the fields'
 * own arrays, for an in-place update) and, when not NULL, absorbed (4
 * n_cells doubles: per cell the EUV photons absorbed by H and by dust and
 * the FUV photons absorbed by H2 and by dust, photons cm^-3, split in
 * proportion to the rates).  Asynchronous on `stream`; n_cells == 0 is a
 * no-op; SFCHEM_EINVAL on a NULL or misaligned pointer, n_cells < 0 or
 * dt_seconds < 0. */
int sfchem_photon_update(const sfchem_state_t *state, const sfchem_fields_t *fields, int64_t n_cells,
                         double dt_seconds, double *G0_out, double *n_euv_out, double *absorbed, void *stream);

/* Cost-balanced partition of a block list across devices (Sec. 4: the
 * thermochemical update runs independently on each device; the cells are
 * independent, so a rank may take any contiguous range of blocks).  Splits
 * the blocks [0, n_blocks) (block b holds cells [block_offset[b],
 * block_offset[b+1]), a HOST array of n_blocks + 1 entries starting at 0)
 * into n_parts contiguous ranges: part k takes blocks [cut[k], cut[k+1]),
 * with cut[0] = 0 <= cut[1] <= ... <= cut[n_parts] = n_blocks (n_parts + 1
 * entries, written by the call).  The largest part's cost is minimal among
 * contiguous cuts (to a relative 1e-12), and so at most
 * total / n_parts + the largest block's cost.  block_cost (n_blocks HOST
 * doubles, >= 0; e.g. the previous call's substeps per block from
 * sfchem_block_costs) gives the cost of each block; NULL weighs blocks by
 * their cell counts, and a block of cost 0 by its cell count.  Host only,
 * no device needed; SFCHEM_EINVAL on bad arguments. */
int sfchem_partition(const int64_t *block_offset, const double *block_cost, int32_t n_blocks, int32_t n_parts,
                     int32_t *cut);

/* The per-block cost of the context's last batched call (sfchem_step_batched,
 * sfchem_step_host or sfchem_autotune): the sum of n_sub over each block's
 * cells, as float, into the HOST array cost (n_blocks entries, n_blocks being
 * that schedule's block count; otherwise SFCHEM_EINVAL).  Synchronizes the
 * device. */
int sfchem_block_costs(sfchem_ctx *ctx, float *cost, int32_t n_blocks);

/* Copy the accumulated statistics to *out (synchronizes the stream of the
 * last call). */
int sfchem_stats(sfchem_ctx *ctx, sfchem_stats_t *out);

/* Zero the statistics (asynchronous on the stream of the last call). */
int sfchem_stats_reset(sfchem_ctx *ctx);

/* Destroy the context and release its scratch and graphs. */
int sfchem_finalize(sfchem_ctx *ctx);

/* Static text for a status code. */
const char *sfchem_strerror(int status);

/* Text of the last CUDA error seen by the library on this thread. */
const char *sfchem_last_cuda_error(void);

/* Allocation-free batched step (the paper has no counterpart: it is an
 * interface for embedding).  For callers that cannot call cudaMalloc -- a
 * host framework that owns every device allocation and forbids others, or
 * code that must not grow its device footprint once it is running -- and so
 * cannot create a context.  Same arguments and results as
 * sfchem_step_batched with a configuration instead of a context (cfg may be
 * NULL for the defaults).  It allocates nothing: its scratch (work counter,
 * statistics, the block tables and the chunk table) is one file-scope
 * __device__ array of 1,131,264 bytes.  CUDA places the library's device
 * code and this array on a GPU when the library first uses that GPU (with
 * CUDA's default lazy loading, inside the first call that needs them) and
 * keeps them until the process exits: the first call on a device may
 * therefore grow the device footprint by the array and the kernels' code,
 * and belongs in start-up; later calls do not.
 * Limits: at most SFCHEM_NOALLOC_MAX_BLOCKS blocks and at most
 * SFCHEM_NOALLOC_MAX_CHUNKS chunks of 64 cells (a block of s cells takes
 * ceil(s/64) chunks); larger schedules are refused with SFCHEM_EINVAL before
 * anything is launched.  The first call on a device looks up the array's
 * device address (once per device, with that device current) and should come
 * before any stream capture.  All calls share the one array, which keeps the
 * previous call's contents (each call clears what must start at zero):
 * calls whose work overlaps on the GPU race on it, so issue them one after
 * another (one stream, or synchronised).  block_offset and block_dt are
 * read during the call: it waits until `stream` has copied them to the
 * device (and so for the work queued on `stream` before it), after which
 * the caller may reuse or free them.  Statistics are not reported and the
 * blocks run in index order (no cost ordering across calls). */
#define SFCHEM_NOALLOC_MAX_BLOCKS 4096
#define SFCHEM_NOALLOC_MAX_CHUNKS 65536
int sfchem_step_batched_noalloc(const sfchem_config_t *cfg, const sfchem_state_t *state,
                                const sfchem_fields_t *fields, const int64_t *block_offset,
                                const double *block_dt, int32_t n_blocks, double cd_factor, void *stream);

/* Library version as "major.minor.patch". */
const char *sfchem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SFCHEM_H */
