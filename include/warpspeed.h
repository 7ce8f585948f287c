/*
 * warpspeed.h -- C ABI of libwarpspeed, a GB300 (sm_103a) implementation of the
 * data-volume hot path of the Warpspeed metric estimator (Ernst et al., "Analytical
 * Performance Estimation during Code Generation on Modern GPUs").
 *
 * For every code-generation candidate the library evaluates the address expression
 * of every thread of a representative thread block and of a wave of co-resident
 * blocks (Sec. 4.2-4.4), collapses the addresses to unique 32 B sectors and 128 B
 * lines, derives bank-conflict cycles (Sec. 4.2), L1/L2/DRAM volumes per lattice
 * update with layer-condition reuse (Sec. 4.4.2) and capacity misses (Sec. 4.5), and
 * combines them in the four-limiter performance model (Sec. 2) into a predicted time
 * and a ranking (Sec. 5.8).
 *
 * Conventions
 *   - All structs are plain C with natural alignment; sizes are fixed (see the
 *     static asserts in the implementation).
 *   - Unless stated otherwise pointers are HOST pointers owned by the caller; the
 *     library copies what it needs before returning and never keeps them.
 *   - Every call returns a status: WS_OK (0) or a negative WS_E* code.  Per-candidate
 *     problems are reported in ws_result.status and do not fail the call.
 *   - A ws_ctx binds one CUDA device.  It is not thread safe, except that one
 *     ws_server may run on it while the owner thread makes no other call.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     context's own stream).
 *   - Address expressions are affine (Sec. 1.2): for a thread whose grid point is p,
 *     access (o, dc) of field f touches the byte
 *         align + elem_bytes * (stride . (p + o) + const_off + dc)
 *     i.e. the unknown base pointer is replaced by the field alignment (Sec. 4.3).
 */
#ifndef WARPSPEED_H
#define WARPSPEED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WS_VERSION 1

/* ---- status codes --------------------------------------------------------------- */
#define WS_OK 0
#define WS_EINVAL (-1)     /* malformed argument or descriptor                           */
#define WS_ENOMEM (-2)     /* does not fit the context's device-memory budget            */
#define WS_EAGAIN (-3)     /* server: request not finished yet                           */
#define WS_ETIMEDOUT (-4)  /* a bounded wait (host or device) ran out                    */
#define WS_EOVERFLOW (-5)  /* a counting structure overflowed (never silent)             */
#define WS_ECUDA (-6)      /* a CUDA runtime call failed                                 */
#define WS_ENOTFOUND (-7)  /* unknown request id                                         */
#define WS_ECANCELED (-8)  /* server: request withdrawn, or shut down before it ran       */

/* ---- modes of ws_plan_execute / ws_estimate_batch ---------------------------------- */
#define WS_MODE_PLAIN 0    /* one synchronous launch sequence per candidate               */
#define WS_MODE_BATCHED 1  /* one persistent launch over all candidates, CUDA graph replay */
#define WS_MODE_DIRECT 2   /* the batched kernels launched directly (no graph)            */

/* ---- limiters (ws_result.limiter, Sec. 2) ------------------------------------------ */
#define WS_LIMITER_L1 0    /* L1 <-> register cycles (bank conflicts)                     */
#define WS_LIMITER_L2 1    /* L2 <-> L1 bandwidth                                         */
#define WS_LIMITER_DRAM 2  /* DRAM <-> L2 bandwidth                                       */
#define WS_LIMITER_FP 3    /* floating-point throughput                                   */

/* One relative access of a field (Sec. 1.2, 4.3): grid offset (dx, dy, dz) from the
 * updated point, plus an extra element offset dc (components of AoS layouts).
 * is_store: 0 = load, 1 = store.  |dx|,|dy|,|dz| <= 65535, |dc| < 2^40. */
typedef struct ws_access {
  int32_t dx, dy, dz;
  int32_t is_store;
  int64_t dc;
} ws_access; /* 24 bytes */

/* One array.  Fields never alias (Sec. 4.3): sectors are counted per field and then
 * summed.  elem_bytes in 1..64; stride[d] in elements (|stride| < 2^40, any sign);
 * align_bytes replaces the base pointer (|align| < 2^50, any value, negative allowed);
 * the field's accesses are acc[access_off .. access_off + n_access). */
typedef struct ws_field {
  int32_t elem_bytes;
  int32_t n_access;
  int64_t align_bytes;
  int64_t stride[3];
  int64_t const_off;
  int64_t access_off;
} ws_field; /* 56 bytes */

/* One candidate (Sec. 5.1, 5.2): domain N (points), thread-block shape B, thread folding
 * (fold_axis 0 = none, 1 = y, 2 = z; each thread updates `fold` consecutive points
 * along that axis, fold in 1..16, fold == 1 when fold_axis == 0), its fields
 * fld[field_off .. field_off + n_field), flops per lattice update (0 = no FP limiter),
 * registers per thread (0 = not limiting; Sec. 5.1 LBM remark), and an optional wave
 * size in blocks (0 = SMs x resident blocks per SM).  Limits: 1 <= N[d] <= 2^20,
 * B[0]*B[1]*B[2] <= 1024, B[2] <= 64, grid blocks < 2^31. */
typedef struct ws_config {
  int32_t N[3];
  int32_t B[3];
  int32_t fold_axis;
  int32_t fold;
  int32_t n_field;
  int32_t regs_per_thread;
  int64_t field_off;
  double flops_per_lup;
  int32_t wave_blocks_override;
  int32_t address_mode; /* WS_ADDR_LINEAR: linear byte addresses everywhere.
                           WS_ADDR_MULTIDIM: the wave and the y / z layer sets count in the
                           multi-dimensional address space of Sec. 4.4.1 -- a sector is
                           (innermost coordinate in bytes / 32, y, z), the base alignment is
                           ignored and a line wrapping to the next row counts at both ends;
                           the representative block keeps linear addresses.               */
} ws_config; /* 64 bytes */

enum { WS_ADDR_LINEAR = 0, WS_ADDR_MULTIDIM = 1 };

/* Modelled GPU (Table 1 of the paper; the A100-SXM4-40G column with a 20 MB effective
 * L2 is the reference setting).  Rates in bytes/s, flop/s and Hz; sizes in bytes.
 * hit[i] = (a, b, c) of the capacity hit-rate fit R(O) = a*exp(-b*exp(-c*O))
 * (Sec. 4.5) for i = 0 L1 redundant loads, 1 L2 y-layer overlap, 2 L2 z-layer
 * overlap, 3 L2 redundant stores.  capacity_model = 0 sets every R to 1. */
typedef struct ws_hw {
  int32_t sms, max_threads_sm, max_blocks_sm, regs_sm;
  double clock_hz, l1_bytes, l2_bytes, bw_l2, bw_dram, fp_peak;
  int32_t banks, bank_bytes, pair_dist_bytes, capacity_model;
  double hit[4][3];
} ws_hw; /* 176 bytes */

/* Result of one candidate.  The int64 part is exact (it is what the parity tests
 * compare bit for bit); volumes are bytes per lattice update (LUP), o_* are
 * oversubscription factors, t_* are seconds per LUP for the whole GPU. */
typedef struct ws_result {
  int64_t lups_block, lups_wave;              /* valid lattice updates of block / wave   */
  int64_t l1_req_sectors;                     /* sum over warp x load instr of unique sectors */
  int64_t l1_bank_cycles;                     /* sum over half-warp x instr of wavefronts */
  int64_t l1_store_sectors;                   /* sum over warp x store instr of unique sectors */
  int64_t blk_load_sectors, blk_load_lines;   /* unique in the representative block     */
  int64_t blk_store_sectors, blk_store_lines;
  int64_t wave_load_sectors, wave_load_lines; /* unique in the representative wave      */
  int64_t wave_store_sectors, wave_store_lines;
  int64_t wave_store_req_sectors;             /* sum over wave warps x store instr       */
  int64_t ov_y, ov_z;                         /* wave footprint shared with the y / z sets */
  int64_t y_lines, z_lines;                   /* footprint lines of the y / z sets        */
  int64_t wave_blocks, wave_first_block;      /* representative wave [first, first+blocks) */
  int64_t y_dist_blocks, z_dist_blocks;       /* blocks scheduled since the y / z set start */
  int64_t blocks_per_sm;
  double v_l1, v_l2_load, v_l2_store, v_dram_load, v_dram_store;
  double o_l1, o_y, o_z, o_st;
  double t_l1, t_l2, t_dram, t_fp, t_pred, glups;
  int32_t limiter;                            /* WS_LIMITER_*                            */
  int32_t status;                             /* WS_OK or WS_E*                          */
} ws_result; /* 312 bytes */

/* Tuning of the batched kernels (picked by ws_autotune; zeros = defaults). */
typedef struct ws_tuning {
  int32_t chunk_warps;     /* modelled warps per enumeration work item                   */
  int32_t enum_threads;    /* threads per CTA of the enumeration kernel (64..512, x32)   */
  int32_t count_words;     /* bitmap words per counting work item                        */
  int32_t ctas_per_sm;     /* persistent CTAs per SM (0 = occupancy limit)               */
  int32_t pass_mb;         /* bitmap scratch per pass in MiB, e.g. sized to stay in L2 (0 or
                              < 0 = as large as the arena allows); never below one field   */
  int32_t walk;            /* How the wave and the y / z layer sets are enumerated; all give
                              identical counts.  WS_WALK_INTERVAL (0): closed-form interval
                              counting (Sec. 4.4) wherever it is exact -- whole grid rows of
                              a level as sector ranges, per-warp store sectors by floor sums,
                              else row segments of each warp; WS_WALK_SEGMENT (2): intervals
                              per row segment of each modelled warp only; WS_WALK_ADDRESS
                              (1): every address evaluated.                                */
} ws_tuning; /* 24 bytes */

enum { WS_WALK_INTERVAL = 0, WS_WALK_ADDRESS = 1, WS_WALK_SEGMENT = 2 };

/* Per-kernel device time of one profiled step (CUDA events on the launch stream). */
typedef struct ws_profile {
  float ms_total, ms_enum, ms_count, ms_model, ms_rank;
  float ms_rows;             /* row-walk kernel (levels 1-3 of row-walk groups)            */
  int32_t launches;          /* kernels launched by the step                             */
  int64_t enum_items, count_items;
  int64_t warp_instr;        /* modelled (warp, access) pairs evaluated                  */
  int64_t addresses;         /* valid (thread, access) address evaluations               */
  int64_t bitmap_bytes;      /* bitmap and page-flag bytes the plan's fields occupy        */
  int64_t passes;            /* scratch passes the plan needed                            */
  int64_t upload_bytes;      /* descriptor bytes the plan copied host -> device           */
  int64_t row_reds;          /* 64-bit red.or issued by the row walk                      */
  int64_t block_addresses;   /* (thread, access) address evaluations of the representative
                                blocks (the exact per-address path)                        */
  float ms_create_host;      /* wall time of the plan's creation on the host: descriptor
                                compilation, list sharing, grouping, pass layout           */
  float ms_create_device;    /* wall time of the rest of the creation: device memory,
                                descriptor upload, scratch zeroing, stream synchronisation */
  int64_t count_bytes;       /* bitmap bytes the counting kernel read: the pages the row walk
                                flagged as written (every word for the other walks)        */
} ws_profile; /* 120 bytes */

typedef struct ws_ctx ws_ctx;
typedef struct ws_plan ws_plan;
typedef struct ws_server ws_server;

int ws_version(void);
const char *ws_status_string(int status);
/* Text of the last CUDA or allocation failure seen by the calling thread. */
const char *ws_last_error(void);

/* Default modelled hardware: A100-SXM4-40G (Table 1, 20 MB effective L2, Sec. 3),
 * illustrative hit-rate coefficients (the paper prints none). */
void ws_hw_a100(ws_hw *hw);

/* Binds `device`.  arena / arena_bytes: a caller-owned DEVICE buffer used for all
 * device memory of the context (descriptors, bitmaps, results); arena == NULL makes
 * the library allocate arena_bytes itself.  The arena is the memory budget. */
int ws_create(ws_ctx **ctx, int device, void *arena, size_t arena_bytes);
int ws_destroy(ws_ctx *ctx);

/* Compiles n_cfg candidates into device-resident descriptors (host descriptor
 * compiler: grid, representative block and wave, y/z sets, folded access lists,
 * bitmap ranges; Sec. 4.2-4.4) and reserves their scratch.  cfgs[i].field_off indexes
 * fld[0..n_fld), fld[j].access_off indexes acc[0..n_acc).  seg_begin (n_seg + 1
 * entries, ascending, seg_begin[0] = 0, seg_begin[n_seg] = n_cfg) splits the
 * candidates into independently ranked lists; NULL = one list.  tuning may be NULL.
 * Malformed candidates get status WS_EINVAL in their result; the call still
 * succeeds.  WS_ENOMEM if one field's scratch alone exceeds the arena. */
int ws_plan_create(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                   const ws_access *acc, int n_acc, const ws_hw *hw, const int32_t *seg_begin,
                   int n_seg, const ws_tuning *tuning, ws_plan **plan);
/* Runs one full estimation step on the device (enumeration, counting, model,
 * ranking) in `mode`; results stay on the device.  Asynchronous except in
 * WS_MODE_PLAIN, which synchronises after every candidate. */
int ws_plan_execute(ws_plan *plan, int mode, void *stream);
/* Copies results (n_cfg) and ranking (n_cfg indices; per segment, ascending predicted
 * time, ties by index) to host arrays and synchronises `stream`.  Either may be NULL. */
int ws_plan_results(ws_plan *plan, ws_result *out, int32_t *order, void *stream);
/* Device pointers of the plan's result and order arrays (valid until destroy). */
int ws_plan_device_results(ws_plan *plan, ws_result **results, int32_t **order);
/* Runs one direct step with CUDA events around each kernel and synchronises. */
int ws_plan_profile(ws_plan *plan, void *stream, ws_profile *out);
/* Tries a small grid of tunings (chunk, CTA size, pass size) on this plan and keeps the
 * fastest (also returned); with WS_TUNE_CACHE set, the choice is appended to that file
 * and later plans of the same size class start from it. */
int ws_autotune(ws_plan *plan, void *stream, ws_tuning *best);
int ws_plan_destroy(ws_plan *plan);

/* ---- host-only introspection of the descriptor compiler (no GPU needed) ------------ */
typedef struct ws_cfg_info {
  int32_t status;                 /* WS_OK or the candidate's WS_E* status               */
  int32_t grid[3];                /* thread-block grid (after folding)                   */
  int32_t threads, warps_per_block, blocks_per_sm, n_field;
  int64_t total_blocks, rep_block;            /* representative block: grid middle      */
  int64_t wave_first, wave_blocks;            /* representative wave (Sec. 4.4)         */
  int64_t y_lo, y_hi, z_lo, z_hi;             /* y / z layer-set candidate block ranges */
  int64_t y_dist, z_dist;                     /* blocks since the first y / z set block */
  int64_t modelled_warps;                     /* warps enumerated per loaded field      */
  int64_t folded_loads, folded_stores;        /* folded instructions, summed over fields */
  int64_t scratch_bytes;                      /* bitmap bytes of the candidate          */
} ws_cfg_info; /* 144 bytes */

typedef struct ws_field_info {
  int64_t lo_sector[2];     /* first sector of the block [0] and wave/y/z [1] bitmaps    */
  int64_t words[2];         /* 32-bit words of each of those bitmaps                     */
  int32_t n_load, n_store;  /* folded load / store instructions                          */
} ws_field_info; /* 40 bytes */

/* Compiles candidates on the host only and reports what the device would run
 * (Sec. 4.3-4.4 thread groups).  out: n_cfg entries.  Returns WS_EINVAL on a bad
 * argument; per-candidate problems go to out[i].status. */
int ws_describe(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld, const ws_access *acc, int n_acc,
                const ws_hw *hw, ws_cfg_info *out);
/* Per-field bitmap ranges of one candidate; out holds cfg->n_field entries (for
 * WS_ADDR_MULTIDIM the wave range is the one of the virtual row-slab layout). */
int ws_describe_fields(const ws_config *cfg, const ws_field *fld, int n_fld, const ws_access *acc, int n_acc,
                       const ws_hw *hw, ws_field_info *out);

/* Sizes of the plan a batch would make (host only, no device needed): the descriptor
 * compiler, the sharing of access lists, field groups, scratch passes and work items run
 * exactly as in ws_plan_create, with `scratch_bytes` of bitmap scratch available. */
typedef struct ws_plan_summary {
  int64_t candidates_ok;      /* candidates that compiled (the others get an error status) */
  int64_t fields;             /* field descriptors (a multi-dimensional candidate has two per field) */
  int64_t groups;             /* field groups */
  int64_t passes;             /* scratch passes */
  int64_t enum_items, row_items, count_items;   /* work items of the three kernels */
  int64_t access_entries;     /* folded access list entries after sharing */
  int64_t interval_entries;   /* merged load run entries after sharing */
  int64_t descriptor_bytes;   /* device bytes of descriptors, counters and results */
  int64_t scratch_bytes;      /* bitmap scratch the plan takes */
  int64_t bitmap_bytes;       /* bitmap bytes of all fields (what one pass would need) */
} ws_plan_summary; /* 96 bytes */
int ws_plan_dry_run(const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld, const ws_access *acc,
                    int n_acc, const ws_hw *hw, const ws_tuning *tuning, size_t scratch_bytes,
                    ws_plan_summary *out);

/* One-shot estimate from host buffers: plan_create + execute + results + destroy.
 * out: n_cfg results; order_out (may be NULL): ranking of the whole batch.  In
 * WS_MODE_BATCHED the batched kernels are launched directly (a graph of a one-shot
 * plan would be replayed only once); results are identical in every mode.  The bitmap
 * scratch stays in the context's arena between calls (kept zeroed, so later calls skip
 * the clearing); ws_plan_create and ws_server_create take that room back when they run.
 * Batches of 4096 or more candidates (not WS_MODE_PLAIN) run as up to six parts whose
 * descriptors compile and upload while earlier parts execute, alternately on `stream` and
 * on a second stream of the context (joined back into `stream`); results and ranking are
 * those of one plan.  Blocks until the results are on the host. */
int ws_estimate_batch(ws_ctx *ctx, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                      const ws_access *acc, int n_acc, const ws_hw *hw, ws_result *out,
                      int32_t *order_out, int mode, void *stream);

/* ---- estimation without device allocation ------------------------------------------ */
/* Size of the fixed device scratch of ws_estimate_batch_noalloc: 32 MiB, reserved on
 * every GPU that loads this library's device code, for as long as the process lives. */
#define WS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The paper has no counterpart: this is a deployment variant of ws_estimate_batch for
 * callers that must not allocate device memory (a code generator running inside an
 * application whose device memory is owned by another runtime or a fixed pool, or
 * whose steady state forbids allocation).  Same inputs and outputs as
 * ws_estimate_batch (host buffers; results and ranking of the whole batch), same
 * kernels launched directly on `stream` (NULL = legacy default stream), but every
 * device buffer comes from one fixed array of WS_NOALLOC_SCRATCH_BYTES inside the
 * library, and the call creates no CUDA resource: no cudaMalloc, cudaFree,
 * cudaHostAlloc, stream or event (ws_resource_counts_get does not move).  Its host
 * memory is plain heap memory (descriptor compilation and pageable upload arrays).
 *   - The first call on a device looks up the array's device address there with
 *     cudaGetSymbolAddress; make that first call before any stream capture.  The
 *     caller's current device is restored before the call returns.
 *   - A batch whose descriptors plus its largest field's bitmaps plus 8 MiB of
 *     headroom exceed the array returns WS_ENOMEM (ws_last_error says so) before any
 *     kernel runs; larger batches otherwise run in several bitmap passes.
 *   - Every call on a device uses the same array and clears the bitmaps it uses first.
 *     Two calls whose device work overlapped would race on it, so calls on one device
 *     are serialised in this process: each holds a per-device lock for its whole
 *     duration and returns only after its device work has finished.  Work the caller
 *     enqueues on other streams never touches the array.  Each process has its own. */
int ws_estimate_batch_noalloc(int device, const ws_config *cfgs, int n_cfg, const ws_field *fld, int n_fld,
                              const ws_access *acc, int n_acc, const ws_hw *hw, ws_result *out,
                              int32_t *order_out, void *stream);

/* Stable ranking on the device (Sec. 5.8): ascending t_pred rounded to 40
 * significant bits, ties by index; NaN ranks as +inf.  res: n host results. */
int ws_rank(ws_ctx *ctx, const ws_result *res, int n, int32_t *order_out, void *stream);
/* The rank key: t rounded to 40 significant mantissa bits, half to even. */
double ws_rank_key(double t);

/* Measures, on the context's GPU, the two rates that bound the enumeration kernel:
 * 32-bit integer adds per second (8 independent add chains per thread, all SMs) and
 * L2 red.or operations per second on distinct words of a 64 MiB buffer.  Used as the
 * roofline denominators of the benchmark. */
int ws_measure_peaks(ws_ctx *ctx, double *int_ops_per_s, double *l2_red_per_s);

/* The same two rates plus the rate of the row walk's own access pattern: every thread
 * sets runs of three consecutive 64-bit words (one sector range) with 64-bit red.or, at
 * far-apart places of a 64 MiB buffer (L2 resident). */
typedef struct ws_peaks {
  double int_ops_per_s;        /* 32-bit integer adds per second                          */
  double l2_red_per_s;         /* 32-bit red.or per second on distinct random words        */
  double l2_red64_run_per_s;   /* 64-bit red.or per second in runs of 3 adjacent words    */
  double reserved;
} ws_peaks; /* 32 bytes */
int ws_measure_peaks2(ws_ctx *ctx, ws_peaks *out);

/* CUDA resources this library has created in this process so far, for callers that must
 * check that a code path creates none (see ws_estimate_batch_noalloc). */
typedef struct ws_resource_counts {
  int64_t device_allocs;       /* cudaMalloc (context arenas the library allocates)       */
  int64_t pinned_host_allocs;  /* cudaHostAlloc (upload staging, server result buffers)   */
  int64_t streams;             /* cudaStreamCreate* (contexts, server slots)              */
  int64_t events;              /* cudaEventCreate* (plan readiness, profiling, parts)     */
} ws_resource_counts; /* 32 bytes */
int ws_resource_counts_get(ws_resource_counts *out);

/* ---- continuous-batching server ---------------------------------------------------- */
typedef struct ws_server_opts {
  size_t mem_budget;        /* bytes of the arena the server may hold (0 = whole arena)  */
  int32_t max_inflight;     /* concurrent device steps (streams), 1..8                   */
  int32_t max_step_cfgs;    /* candidates admitted into one step (and per request)       */
  int32_t max_queue;        /* pending requests before submit fails with WS_EAGAIN       */
  int32_t reserved;
} ws_server_opts;

/* One estimation request: a candidate list of one stencil (same layout rules as
 * ws_plan_create); the whole list is ranked as one segment. */
typedef struct ws_request {
  const ws_config *cfgs;
  int32_t n_cfg;
  int32_t n_fld;
  const ws_field *fld;
  const ws_access *acc;
  int32_t n_acc;
  int32_t reserved;
} ws_request;

typedef struct ws_server_stats {
  int64_t submitted, completed, rejected, steps, configs_done;
  int64_t bytes_in_use, peak_bytes;
  int32_t inflight_steps, queued;
  int64_t canceled;           /* requests withdrawn by ws_server_cancel                    */
} ws_server_stats; /* 72 bytes */

int ws_server_create(ws_ctx *ctx, const ws_server_opts *opts, const ws_hw *hw, ws_server **srv);
/* Copies the request and queues it; returns at once.  A request whose scratch exceeds
 * the free budget runs in several scratch passes; WS_ENOMEM only if one of its fields
 * alone can never fit the budget.  WS_EAGAIN if the queue is full. */
int ws_server_submit(ws_server *srv, const ws_request *req, uint64_t *req_id);
/* Waits up to timeout_us (0 = just test) for the request; on WS_OK copies its n_cfg
 * results (and ranking, may be NULL) and forgets it.  WS_EAGAIN if not finished. */
int ws_server_poll(ws_server *srv, uint64_t req_id, ws_result *out, int32_t *order, int64_t timeout_us);
int ws_server_stats_get(ws_server *srv, ws_server_stats *out);
/* paused != 0: admit no new device steps (steps already admitted run to the end);
 * requests keep queueing until the queue is full.  paused == 0: resume admission.
 * Lets a host drain the GPU for other work, or gather a burst of requests into fewer,
 * larger steps, without losing queued requests. */
int ws_server_pause(ws_server *srv, int paused);
/* Withdraws a request that is still queued: WS_OK, and its next poll returns
 * WS_ECANCELED (and forgets it).  WS_EAGAIN if it was already admitted into a step
 * (poll for its result), WS_ENOTFOUND for an unknown or already collected id. */
int ws_server_cancel(ws_server *srv, uint64_t req_id);
/* Finishes every admitted step, cancels queued requests, joins the worker. */
int ws_server_destroy(ws_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* WARPSPEED_H */
