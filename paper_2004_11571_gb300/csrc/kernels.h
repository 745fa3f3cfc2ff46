// Host-side launchers of the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include "common.h"

namespace pe {

constexpr int kMaxStepBWarps = 4;   // warps per block of the plain Step B kernel

cudaError_t launch_powtab(const BetaArg &beta, uint32_t E, uint32_t dp1, const ModCtx &mc, uint64_t *ptab,
                          cudaStream_t st);
cudaError_t launch_stepA(const void *exps, uint32_t exp_bytes, uint64_t s, uint32_t E, const uint64_t *ptab,
                         uint32_t dp1, const ModCtx &mc, uint64_t *mR, int num_sms, cudaStream_t st);
cudaError_t launch_stepA_starts(const void *exps, uint32_t exp_bytes, const uint64_t *coeffs, uint64_t s, uint32_t E,
                               const uint64_t *ptab, uint32_t dp1, const ModCtx &mc, uint64_t t0, const StartRows &sr,
                               uint64_t *mR, uint64_t *vstart, int num_sms, cudaStream_t st);
// Chunk tables of a plan (cs: NC+1 chunk starts, cg: NC group ids) from the
// group offsets and each group's first chunk.
cudaError_t launch_chunk_tables(const uint32_t *goff, const uint32_t *gfirst, uint64_t G, uint32_t K, uint64_t s,
                                uint32_t NC, uint32_t *cs, uint32_t *cg, cudaStream_t st);
cudaError_t launch_stepB(int K, int var, const StepBJob &J0, uint32_t n0, const StepBJob &J1, uint32_t n1, int wpb,
                         cudaStream_t st);
cudaError_t stepB_occupancy(int K, int var, int wpb, int *blocks_per_sm);

// Exclusive scan of n counts into out[0..n] (out[n] = total), one block.
cudaError_t launch_scan_counts(const uint64_t *counts, uint64_t n, uint64_t *out, cudaStream_t st);

// Device side of poly_eval_create (create.cu).
struct CreateInfo {
    unsigned long long bad;   // lowest index of a coefficient >= p, or ~0
    uint32_t dmax;            // largest exponent of x3..xn
    uint32_t unsorted;        // nonzero if some (d, e) key exceeds the previous one
};
cudaError_t launch_term_scan(const uint64_t *coeffs, const void *exps, uint32_t width, uint64_t s, uint32_t n,
                             uint64_t p, uint64_t *keys, CreateInfo *info, uint64_t *counts, uint64_t *base,
                             uint64_t *goff, uint32_t *gkeys, cudaStream_t st);
cudaError_t launch_pack_exps(const void *exps, uint32_t width, uint64_t s, uint32_t n, uint32_t out_bytes,
                             void *out, cudaStream_t st);

}  // namespace pe
