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

// Integer pipe rates: 8 independent dependency chains per thread of one
// instruction kind (PTX mad.lo.u32, mad.hi.u32, mad.wide.u32, add.u32).
template <int KIND>
__global__ void __launch_bounds__(256) k_int_rate(uint32_t *sink, uint32_t iters, unsigned long long *clk)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[8];
    uint64_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = tid * 2654435761u + k * 40503u + 1u;
        w[k] = x[k];
    }
    const uint32_t y = 0x9E3779B1u ^ (tid >> 5), c = 12345u + (tid & 7);
    unsigned long long c0 = 0, g0 = 0;
    if (tid == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(y), "r"(c));
                if constexpr (KIND == 1) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(y), "r"(c));
                if constexpr (KIND == 2) {
                    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[k]) : "r"((uint32_t)w[k]), "r"(y));
                }
                if constexpr (KIND == 3) asm volatile("add.u32 %0, %0, %1;" : "+r"(x[k]) : "r"(y));
            }
        }
    }
    if (tid == 0) {
        unsigned long long g1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
        clk[0] = clock64() - c0;
        clk[1] = g1 - g0;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= x[k] ^ (uint32_t)w[k] ^ (uint32_t)(w[k] >> 32);
    sink[tid] = acc;
}

template <int KIND>
static pe_status int_rate(double *per_sm_clk)
{
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_int_rate<KIND>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    bps = std::max(1, bps);
    const uint32_t grid = (uint32_t)(bps * num_sms());
    const uint64_t threads = (uint64_t)grid * 256;
    DevBuf sink, clk;
    if ((e = sink.ensure(threads * 4)) != cudaSuccess || (e = clk.ensure(16)) != cudaSuccess)
        return cuda_fail(e, "alloc");
    const uint32_t iters = 1u << 14;
    k_int_rate<KIND><<<grid, 256>>>(sink.as<uint32_t>(), iters / 16, clk.as<unsigned long long>());  // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    k_int_rate<KIND><<<grid, 256>>>(sink.as<uint32_t>(), iters, clk.as<unsigned long long>());
    cudaEventRecord(b);
    unsigned long long hc[2] = {0, 0};
    float ms = 0.f;
    if ((e = cudaEventSynchronize(b)) == cudaSuccess && (e = cudaGetLastError()) == cudaSuccess)
        e = cudaMemcpy(hc, clk.p, 16, cudaMemcpyDeviceToHost);
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "int rate");
    // Kernel time from events; the SM clock from thread 0's cycle and nanosecond
    // counters (warps are not scheduled evenly, so its cycle count is not the duration).
    const double hz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e9 : 1.9e9;
    *per_sm_clk = (double)threads * iters * 32.0 / ((double)num_sms() * (ms * 1e-3) * hz);
    return PE_OK;
}

// FP64 pipe rates: 8 independent dependency chains per thread of fma.rn.f64
// (x <- x*y + c, y just below 1, so x stays bounded) or add.rn.f64.
template <int KIND>
__global__ void __launch_bounds__(256) k_fp64_rate(double *sink, uint32_t iters, unsigned long long *clk)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1.0 + (double)((tid * 2654435761u + k * 40503u) & 1023) * 1e-4;
    const double y = 0.9999995 - (double)(tid & 7) * 1e-9, c = 1e-3 + (double)(tid >> 5 & 15) * 1e-7;
    unsigned long long c0 = 0, g0 = 0;
    if (tid == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    }
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 0) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[k]) : "d"(y), "d"(c));
                if constexpr (KIND == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(x[k]) : "d"(c));
            }
        }
    }
    if (tid == 0) {
        unsigned long long g1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
        clk[0] = clock64() - c0;
        clk[1] = g1 - g0;
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += x[k];
    sink[tid] = acc;
}

template <int KIND>
static pe_status fp64_rate(double *per_sm_clk)
{
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_fp64_rate<KIND>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    bps = std::max(1, bps);
    const uint32_t grid = (uint32_t)(bps * num_sms());
    const uint64_t threads = (uint64_t)grid * 256;
    DevBuf sink, clk;
    if ((e = sink.ensure(threads * 8)) != cudaSuccess || (e = clk.ensure(16)) != cudaSuccess)
        return cuda_fail(e, "alloc");
    const uint32_t iters = 1u << 10;
    k_fp64_rate<KIND><<<grid, 256>>>(sink.as<double>(), iters / 16, clk.as<unsigned long long>());  // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    k_fp64_rate<KIND><<<grid, 256>>>(sink.as<double>(), iters, clk.as<unsigned long long>());
    cudaEventRecord(b);
    unsigned long long hc[2] = {0, 0};
    float ms = 0.f;
    if ((e = cudaEventSynchronize(b)) == cudaSuccess && (e = cudaGetLastError()) == cudaSuccess)
        e = cudaMemcpy(hc, clk.p, 16, cudaMemcpyDeviceToHost);
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 rate");
    const double hz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e9 : 1.9e9;
    *per_sm_clk = (double)threads * iters * 32.0 / ((double)num_sms() * (ms * 1e-3) * hz);
    return PE_OK;
}

}  // namespace pe

using namespace pe;

extern "C" pe_status poly_eval_fp64_pipe_rates(double rates[2])
{
    if (!rates) {
        set_error("NULL output");
        return PE_ERR_ARG;
    }
    pe_status st;
    if ((st = fp64_rate<0>(&rates[0])) != PE_OK || (st = fp64_rate<1>(&rates[1])) != PE_OK) return st;
    return PE_OK;
}

extern "C" pe_status poly_eval_int_pipe_rates(double rates[4])
{
    if (!rates) {
        set_error("NULL output");
        return PE_ERR_ARG;
    }
    pe_status st;
    if ((st = int_rate<0>(&rates[0])) != PE_OK || (st = int_rate<1>(&rates[1])) != PE_OK ||
        (st = int_rate<2>(&rates[2])) != PE_OK || (st = int_rate<3>(&rates[3])) != PE_OK)
        return st;
    return PE_OK;
}

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

extern "C" pe_status poly_eval_num_sms(uint32_t *sms)
{
    if (!sms) {
        set_error("NULL output");
        return PE_ERR_ARG;
    }
    int dev = 0, n = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "SM count");
    *sms = (uint32_t)n;
    return PE_OK;
}
