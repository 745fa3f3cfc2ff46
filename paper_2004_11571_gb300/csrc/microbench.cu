// Roofline calibration: the Step B inner operation alone, from registers.
//
// Each thread advances 16 independent (v, m) chains through the same
// lane_point() the kernels use (one modular product and one lazy sum per
// term-point, Algorithm 1), with no memory traffic, at full occupancy.  The
// measured rate is the ceiling for Step B with the same modular product.
#include "internal.h"
#include "stepb.cuh"

namespace pe {

template <int VAR>
__global__ void __launch_bounds__(256) k_modmul_peak(uint64_t *sink, ModCtx mc, uint32_t iters,
                                                     unsigned long long *clk)
{
    constexpr int C = 16;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Lane<VAR> st[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        uint64_t x = (tid * 0x9E3779B97F4A7C15ull) ^ (0xD1B54A32D192ED03ull * (k + 1));
        x ^= x >> 29;
        const uint64_t v0 = x % mc.p;
        const uint64_t mR = (x * 0xBF58476D1CE4E5B9ull) % mc.p;
        st[k].init(v0, mR, mc);
    }
    unsigned long long c0 = 0, g0 = 0;
    if (tid == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    }
    uint64_t alo = 0;
    uint32_t ahi = 0;
    for (uint32_t it = 0; it < iters; ++it) {
        uint64_t lo;
        uint32_t hi;
        lane_point<C, VAR>(st, mc, lo, hi);
        add96(alo, ahi, lo, hi);
    }
    if (tid == 0) {
        unsigned long long g1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
        clk[0] = clock64() - c0;
        clk[1] = g1 - g0;
    }
    sink[tid] = alo ^ ((uint64_t)ahi << 32);
}

template <int VAR>
static pe_status run_peak(const ModCtx &mc, double *tps, double *mhz)
{
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_modmul_peak<VAR>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (bps < 1) bps = 1;
    const uint32_t grid = (uint32_t)(bps * num_sms());
    const uint64_t threads = (uint64_t)grid * 256;
    DevBuf sink, clk;
    if ((e = sink.ensure(threads * 8)) != cudaSuccess || (e = clk.ensure(16)) != cudaSuccess)
        return cuda_fail(e, "alloc");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    uint32_t iters = 256;
    float ms = 0.f;
    for (int rep = 0; rep < 8; ++rep) {  // grow until the kernel runs ~50 ms
        cudaEventRecord(a);
        k_modmul_peak<VAR><<<grid, 256>>>(sink.as<uint64_t>(), mc, iters, clk.as<unsigned long long>());
        cudaEventRecord(b);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
        cudaEventElapsedTime(&ms, a, b);
        if (ms > 40.f) break;
        iters = (uint32_t)std::min<double>(1u << 22, iters * std::min(16.0, std::max(2.0, 50.0 / std::max(ms, 0.01f))));
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    unsigned long long hc[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(hc, clk.p, 16, cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "modmul peak");
    *tps = (double)threads * iters * 16.0 / (ms * 1e-3);
    if (mhz) *mhz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;
    return PE_OK;
}

}  // namespace pe

using namespace pe;

extern "C" pe_status poly_eval_modmul_peak(pe_variant variant, uint64_t p, double *tps, double *mhz)
{
    if (!tps) {
        set_error("NULL output");
        return PE_ERR_ARG;
    }
    if (p < 3 || !(p & 1) || p >= (1ull << 62) || (variant == PE_MODMUL_FP64 && p >= (1ull << 50)) ||
        (variant == PE_MODMUL_BARRETT32 && p >= (1ull << 30))) {
        set_error("p out of range for the variant");
        return PE_ERR_PRIME;
    }
    const ModCtx mc = make_modctx(p);
    switch (variant) {
    case PE_MODMUL_MONT64: return run_peak<VAR_MONT>(mc, tps, mhz);
    case PE_MODMUL_FP64: return run_peak<VAR_FP64>(mc, tps, mhz);
    case PE_MODMUL_BARRETT32: return run_peak<VAR_BARRETT32>(mc, tps, mhz);
    case PE_MODMUL_AUTO:
    case PE_MODMUL_BARRETT64: return run_peak<VAR_BARRETT>(mc, tps, mhz);
    default: set_error("unknown variant"); return PE_ERR_ARG;
    }
}
