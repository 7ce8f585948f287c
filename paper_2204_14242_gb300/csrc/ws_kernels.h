// Kernel argument blocks and launchers (implemented in ws_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "ws_internal.h"

namespace ws {

struct EnumArgs {
  const DCfg *cfg;
  const DField *fld;
  const DGroup *grp;
  const DAcc *acc;
  const DIv *iv;                   // merged load intervals
  int32_t iv_cap;                  // dynamic shared memory holds this many staged intervals
  uint32_t *scratch;               // bitmaps of the pass
  int64_t *counters;               // [n_cfg][N_COUNTERS]
  unsigned long long *grab;        // work-stealing counter (zeroed before the launch)
  unsigned long long *rgrab;       //   of the row kernel
  const int32_t *own_enum;         // field group of every enumeration item (global numbering)
  const int32_t *own_rows;         // field group of every row-walk item
  int64_t item_lo, item_hi;        // enumeration items of the pass
  int64_t ritem_lo, ritem_hi;      // row-walk items of the pass
  int32_t chunk;                   // modelled warps per item
  int32_t chunk_rows;              // row slots per item (row walk)
  int32_t banks, bank_bytes, pair_dist;
  int32_t bank_shift;              // log2(bank_bytes) when banks x bank_bytes is a power of two <= 1024, else -1
  int32_t block_pairs;             // (modelled warp, instruction) pairs per representative-block item
};

struct CountArgs {
  const DField *fld;
  const int32_t *item_unit;        // first counting unit of every counting item, then the end
  const int32_t *units;            // counting units: (field, chunk) pairs; chunks of the block
                                   // bitmaps' words first, then of the wave bitmaps' words
  uint32_t *scratch;
  int64_t *counters;
  unsigned long long *grab;
  int64_t citem_lo, citem_hi;
  int32_t chunk_words;             // a multiple of kPageWords, at most kCountMaxWords
};

struct ModelArgs {
  const DCfg *cfg;
  const int64_t *counters;
  ws_result *results;
  double *keys;                    // rank keys (t_pred rounded to 40 bits)
  int32_t n;
  DHw hw;
};

struct RankArgs {
  const double *keys;
  const int32_t *seg;              // n_seg + 1 segment starts
  int32_t *order;
  int32_t *rank;                   // n scratch counters
  int32_t n, n_seg;
};

cudaError_t launch_enum(const EnumArgs &args, int grid, int threads, cudaStream_t st);
cudaError_t launch_rows(const EnumArgs &args, int grid, cudaStream_t st);
cudaError_t launch_count(const CountArgs &args, int grid, cudaStream_t st);
cudaError_t launch_model(const ModelArgs &args, cudaStream_t st);
cudaError_t launch_rank(const RankArgs &args, cudaStream_t st);
cudaError_t launch_keys(const ws_result *res, int n, double *keys, cudaStream_t st);
cudaError_t enum_occupancy(int threads, int iv_cap, int *blocks_per_sm);
size_t enum_dyn_smem(int iv_cap);
cudaError_t rows_occupancy(int iv_cap, int *blocks_per_sm);
constexpr int kRowsThreads = 256;
constexpr int kCountThreads = 256;   // counting kernel: threads per CTA
constexpr int kCountMaxWords = 65536;   // most bitmap words of one counting unit of a field without page flags
constexpr int kPagedChunkWords = 262144;   // bitmap words of one counting unit of a field with page flags (1024 pages)
constexpr int kCountMaxPages = 1024;   // most pages of one counting item (one unit or several packed)
constexpr int kCountItemUnits = 64;    // most counting units packed into one counting item
constexpr int kPlainBlockPairs = 128;   // the same in the plain form (one candidate per launch)
constexpr int kBlockPairs = 512;   // (modelled warp, instruction) pairs per representative-block item (mixed set: 4.4 ms of enumeration against 5.5 with 128)
cudaError_t count_occupancy(int *blocks_per_sm);

}  // namespace ws
