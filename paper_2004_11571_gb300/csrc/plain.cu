// Plain (one polynomial per call) kernels: power tables, Step A, Step B.
#include <algorithm>
#include <cstdio>
#include "common.h"
#include "modarith.cuh"
#include "stepb.cuh"
#include "kernels.h"

namespace pe {

// ------------------------------------------------------------------ Step A0
// Power tables [beta_k^e, 0 <= e <= d] in Montgomery form (Sect. 2.3); one
// thread per entry, by square-and-multiply from beta_k * 2^64 mod p.
__global__ void k_powtab(BetaArg beta, uint32_t E, uint32_t dp1, ModCtx mc, uint64_t *__restrict__ ptab)
{
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * dp1) return;
    const uint32_t j = idx / dp1, e = idx - j * dp1;
    const uint64_t bR = canon(mont_mul(beta.b[j], mc.r2, mc), mc.p);
    ptab[idx] = mont_pow(bR, e, mc);
}

// ------------------------------------------------------------------- Step A
// m_i = M_i(beta) in Montgomery form for every term (n-3 products each).
template <typename ExpT>
__global__ void k_stepA(const ExpT *__restrict__ exps, uint64_t s, uint32_t E, const uint64_t *__restrict__ ptab,
                        uint32_t dp1, ModCtx mc, uint64_t *__restrict__ mR)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (uint64_t)gridDim.x * blockDim.x)
        mR[i] = monomial_mont(exps, s, i, E, ptab, dp1, mc);
}

// Step A with starting values: besides m_i, every term's value a_i * m_i^t
// at each work-item start row t = t0 + row[k], so that Step B items start
// with one load.  Consecutive rows are reached by multiplying by m_i^gap; the
// powers for the (at most kMaxGaps) distinct gaps come from one chain of
// squarings m_i^(2^b), b <= the highest gap bit, shared by all of them (the
// gaps are the same for every term, so the branches are uniform).
template <typename ExpT>
__global__ void k_stepA_starts(const ExpT *__restrict__ exps, const uint64_t *__restrict__ coeffs, uint64_t s,
                               uint32_t E, const uint64_t *__restrict__ ptab, uint32_t dp1, ModCtx mc, uint64_t t0,
                               StartRows sr, uint64_t *__restrict__ mR_out, uint64_t *__restrict__ vstart)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t mR = monomial_mont(exps, s, i, E, ptab, dp1, mc);
        mR_out[i] = mR;
        uint64_t cur = canon(mont_mul(coeffs[i], mont_pow(mR, t0 + sr.row[0], mc), mc), mc.p);
        vstart[i] = cur;
        uint64_t gp[kMaxGaps];
#pragma unroll
        for (int j = 0; j < kMaxGaps; ++j) gp[j] = 0;
        uint64_t sq = mR;
        for (uint32_t b = 0; b <= sr.gap_hb; ++b) {
#pragma unroll
            for (int j = 0; j < kMaxGaps; ++j)
                if ((sr.gap[j] >> b) & 1)   // the lowest set bit starts the product, later ones multiply
                    gp[j] = (sr.gap[j] & ((1u << b) - 1)) ? mont_mul(gp[j], sq, mc) : sq;
            if (b < sr.gap_hb) sq = mont_mul(sq, sq, mc);
        }
        for (uint32_t k = 1; k < sr.n; ++k) {
            const uint32_t gi = sr.gidx[k];
            const uint64_t g = gi == 0 ? gp[0] : gi == 1 ? gp[1] : gi == 2 ? gp[2] : gp[3];
            cur = canon(mont_mul(cur, g, mc), mc.p);
            vstart[(uint64_t)k * s + i] = cur;
        }
    }
}

// ------------------------------------------------------------ chunk tables
// Lane chunks of a plan: chunk c belongs to the group g with
// gfirst[g] <= c < gfirst[g+1] and starts at term goff[g] + (c - gfirst[g]) K.
__global__ void k_chunk_tables(const uint32_t *__restrict__ goff, const uint32_t *__restrict__ gfirst, uint32_t G,
                               uint32_t K, uint32_t s, uint32_t NC, uint32_t *__restrict__ cs, uint32_t *__restrict__ cg)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= NC; c += gridDim.x * blockDim.x) {
        if (c == NC) {
            cs[NC] = s;
            continue;
        }
        uint32_t lo = 0, hi = G;   // largest g with gfirst[g] <= c
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (gfirst[mid] <= c) lo = mid;
            else hi = mid;
        }
        cs[c] = goff[lo] + (c - gfirst[lo]) * K;
        cg[c] = lo;
    }
}

cudaError_t launch_chunk_tables(const uint32_t *goff, const uint32_t *gfirst, uint64_t G, uint32_t K, uint64_t s,
                                uint32_t NC, uint32_t *cs, uint32_t *cg, cudaStream_t st)
{
    if (G == 0) return cudaSuccess;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(((uint64_t)NC + 256) / 256, 4096);
    k_chunk_tables<<<grid, 256, 0, st>>>(goff, gfirst, (uint32_t)G, K, (uint32_t)s, NC, cs, cg);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- Step B
// Two bands of work items: J0 covers the first rows with large items, J1 the
// last rows with small ones.  Blocks are issued in index order, so the small
// items run last and fill the SMs that finish their large items early.
// At most 4 warps per block, 5 blocks per SM: 20 warps fit the register file
// (<= 96 registers) and shared memory (9.6 KB per warp).
template <int K, int VAR>
__global__ void __launch_bounds__(128, (K >= 16 ? 3 : K >= 12 ? 4 : 5)) k_stepB(StepBJob J0, uint32_t n0, StepBJob J1, uint32_t n1)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem *sm = reinterpret_cast<WarpSmem *>(smem_raw);
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + warp;
    if (item < n0)
        stepb_item<K, VAR>(J0, J0.item0 + item, sm[warp]);
    else if (item - n0 < n1)
        stepb_item<K, VAR>(J1, J1.item0 + (item - n0), sm[warp]);
}

cudaError_t launch_powtab(const BetaArg &beta, uint32_t E, uint32_t dp1, const ModCtx &mc, uint64_t *ptab,
                          cudaStream_t st)
{
    const uint32_t n = E * dp1;
    if (n == 0) return cudaSuccess;
    k_powtab<<<(n + 127) / 128, 128, 0, st>>>(beta, E, dp1, mc, ptab);
    return cudaGetLastError();
}

cudaError_t launch_stepA(const void *exps, uint32_t exp_bytes, uint64_t s, uint32_t E, const uint64_t *ptab,
                         uint32_t dp1, const ModCtx &mc, uint64_t *mR, int num_sms, cudaStream_t st)
{
    if (s == 0) return cudaSuccess;
    const uint64_t want = (s + 255) / 256;
    const uint32_t grid = (uint32_t)(want < (uint64_t)num_sms * 16 ? want : (uint64_t)num_sms * 16);
    if (exp_bytes == 1)
        k_stepA<uint8_t><<<grid, 256, 0, st>>>((const uint8_t *)exps, s, E, ptab, dp1, mc, mR);
    else
        k_stepA<uint16_t><<<grid, 256, 0, st>>>((const uint16_t *)exps, s, E, ptab, dp1, mc, mR);
    return cudaGetLastError();
}

cudaError_t launch_stepA_starts(const void *exps, uint32_t exp_bytes, const uint64_t *coeffs, uint64_t s, uint32_t E,
                               const uint64_t *ptab, uint32_t dp1, const ModCtx &mc, uint64_t t0, const StartRows &sr,
                               uint64_t *mR, uint64_t *vstart, int num_sms, cudaStream_t st)
{
    if (s == 0) return cudaSuccess;
    const uint64_t want = (s + 255) / 256;
    const uint32_t grid = (uint32_t)(want < (uint64_t)num_sms * 16 ? want : (uint64_t)num_sms * 16);
    if (exp_bytes == 1)
        k_stepA_starts<uint8_t><<<grid, 256, 0, st>>>((const uint8_t *)exps, coeffs, s, E, ptab, dp1, mc, t0, sr,
                                                      mR, vstart);
    else
        k_stepA_starts<uint16_t><<<grid, 256, 0, st>>>((const uint16_t *)exps, coeffs, s, E, ptab, dp1, mc, t0, sr,
                                                       mR, vstart);
    return cudaGetLastError();
}

template <int K, int VAR>
static cudaError_t launch_b(const StepBJob &J, uint32_t nitems, const StepBJob &J1, uint32_t n1, int wpb,
                           cudaStream_t st, int *occ)
{
    const size_t smem = (size_t)wpb * sizeof(WarpSmem);
    // once per device, at the largest block (8 warps)
    cudaError_t e = smem_limit_once((const void *)k_stepB<K, VAR>, (int)(kMaxStepBWarps * sizeof(WarpSmem)));
    if (e != cudaSuccess) return e;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_stepB<K, VAR>, wpb * 32, smem);
    if (nitems + n1 == 0) return cudaSuccess;
    const uint32_t grid = (nitems + n1 + wpb - 1) / wpb;
    k_stepB<K, VAR><<<grid, wpb * 32, smem, st>>>(J, nitems, J1, n1);
    return cudaGetLastError();
}

template <int VAR>
static cudaError_t dispatch_k(int K, const StepBJob &J, uint32_t n0, const StepBJob &J1, uint32_t n1, int wpb,
                              cudaStream_t st, int *occ)
{
    switch (K) {
    case 1: return launch_b<1, VAR>(J, n0, J1, n1, wpb, st, occ);
    case 2: return launch_b<2, VAR>(J, n0, J1, n1, wpb, st, occ);
    case 4: return launch_b<4, VAR>(J, n0, J1, n1, wpb, st, occ);
    case 8: return launch_b<8, VAR>(J, n0, J1, n1, wpb, st, occ);
    case 12: return launch_b<12, VAR>(J, n0, J1, n1, wpb, st, occ);
    case 16: return launch_b<16, VAR>(J, n0, J1, n1, wpb, st, occ);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t dispatch(int K, int var, const StepBJob &J, uint32_t n0, const StepBJob &J1, uint32_t n1, int wpb,
                            cudaStream_t st, int *occ)
{
    if (wpb < 1 || wpb > kMaxStepBWarps) return cudaErrorInvalidValue;
    switch (var) {
    case VAR_BARRETT: return dispatch_k<VAR_BARRETT>(K, J, n0, J1, n1, wpb, st, occ);
    case VAR_MONT: return dispatch_k<VAR_MONT>(K, J, n0, J1, n1, wpb, st, occ);
    case VAR_FP64: return dispatch_k<VAR_FP64>(K, J, n0, J1, n1, wpb, st, occ);
    case VAR_BARRETT32: return dispatch_k<VAR_BARRETT32>(K, J, n0, J1, n1, wpb, st, occ);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stepB(int K, int var, const StepBJob &J0, uint32_t n0, const StepBJob &J1, uint32_t n1, int wpb,
                         cudaStream_t st)
{
    return dispatch(K, var, J0, n0, J1, n1, wpb, st, nullptr);
}

cudaError_t stepB_occupancy(int K, int var, int wpb, int *blocks_per_sm)
{
    StepBJob dummy{};
    return dispatch(K, var, dummy, 0, dummy, 0, wpb, nullptr, blocks_per_sm);
}

}  // namespace pe
