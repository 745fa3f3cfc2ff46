// Plain (one polynomial per call) kernels: power tables, Step A, Step B.
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

// ------------------------------------------------------------------- Step B
template <int K, int VAR>
__global__ void __launch_bounds__(256) k_stepB(StepBJob J, uint32_t nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem *sm = reinterpret_cast<WarpSmem *>(smem_raw);
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t item = blockIdx.x * (blockDim.x >> 5) + warp;
    if (item >= nitems) return;
    stepb_item<K, VAR>(J, item, sm[warp]);
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

template <int K, int VAR>
static cudaError_t launch_b(const StepBJob &J, uint32_t nitems, int wpb, cudaStream_t st, int *occ)
{
    const size_t smem = (size_t)wpb * sizeof(WarpSmem);
    static bool attr_set = false;   // once, at the largest block (8 warps)
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_stepB<K, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(8 * sizeof(WarpSmem)));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_stepB<K, VAR>, wpb * 32, smem);
    if (nitems == 0) return cudaSuccess;
    const uint32_t grid = (nitems + wpb - 1) / wpb;
    k_stepB<K, VAR><<<grid, wpb * 32, smem, st>>>(J, nitems);
    return cudaGetLastError();
}

template <int VAR>
static cudaError_t dispatch_k(int K, const StepBJob &J, uint32_t nitems, int wpb, cudaStream_t st, int *occ)
{
    switch (K) {
    case 1: return launch_b<1, VAR>(J, nitems, wpb, st, occ);
    case 2: return launch_b<2, VAR>(J, nitems, wpb, st, occ);
    case 4: return launch_b<4, VAR>(J, nitems, wpb, st, occ);
    case 8: return launch_b<8, VAR>(J, nitems, wpb, st, occ);
    case 16: return launch_b<16, VAR>(J, nitems, wpb, st, occ);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t dispatch(int K, int var, const StepBJob &J, uint32_t nitems, int wpb, cudaStream_t st, int *occ)
{
    if (wpb < 1 || wpb > 8) return cudaErrorInvalidValue;
    switch (var) {
    case VAR_BARRETT: return dispatch_k<VAR_BARRETT>(K, J, nitems, wpb, st, occ);
    case VAR_MONT: return dispatch_k<VAR_MONT>(K, J, nitems, wpb, st, occ);
    case VAR_FP64: return dispatch_k<VAR_FP64>(K, J, nitems, wpb, st, occ);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stepB(int K, int var, const StepBJob &J, uint32_t nitems, int wpb, cudaStream_t st)
{
    return dispatch(K, var, J, nitems, wpb, st, nullptr);
}

cudaError_t stepB_occupancy(int K, int var, int wpb, int *blocks_per_sm)
{
    StepBJob dummy{};
    return dispatch(K, var, dummy, 0, wpb, nullptr, blocks_per_sm);
}

}  // namespace pe
