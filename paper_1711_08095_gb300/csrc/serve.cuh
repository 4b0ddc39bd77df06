// Fold-in / top-k launch shapes and launchers (serve.cu).
#pragma once

#include "common.cuh"

namespace snect {

constexpr int kFoldThreads = 256;                                       // threads per CTA
constexpr int kFoldTile = 256;                                          // cells staged at once
constexpr int kFoldPerThread = (kMaxRank * kMaxRank + kFoldThreads - 1) / kFoldThreads;
constexpr int64_t kFoldChunk = 256;                                     // cells per CTA (one tile)

// number of per-CTA partials of a query with n cells
int64_t foldin_parts(int64_t n);
cudaError_t launch_wtable(Ctx *c, float *table);
// fold-in of one query: partials, then the solve.  Bad cells OR into *flag (1: a cell outside
// the tensor, 2: a value that is not finite); with flag_out the solve moves *flag there and
// zeroes it, else *flag keeps the bits (the caller zeroes it before the next query)
cudaError_t launch_foldin(Ctx *c, cudaStream_t st, const int2 *jk, const float *val, int64_t n,
                          const float *table, float *part, float *u_out, int32_t *status, int32_t *flag,
                          int32_t *flag_out);
cudaError_t launch_topk(Ctx *c, cudaStream_t st, const float *u, int32_t k, float *score,
                        uint8_t *taken, int32_t *idx_out, float *score_out);

}  // namespace snect
