// Sparse images: keep only the nonzero coefficients of each image, as
// Algorithm 1 does when it adds c x1^d x2^e to b_t only if c != 0.
//
// Dense T x G images become a CSR structure: row r (image b_{t0+r}) holds the
// columns g with out[r][g] != 0 in ascending order and their values.  Three
// kernels: count the nonzeros of every row (one block per row), an exclusive
// scan of the counts (one block), then each row's block writes its entries in
// column order using a block-wide prefix of per-warp ballots.  The work is a
// streaming read of the dense images: HBM-bound.
#include "internal.h"
#include "kernels.h"

namespace pe {

constexpr int kCompactThreads = 256;

__global__ void __launch_bounds__(kCompactThreads) k_count_rows(const uint64_t *__restrict__ dense, uint64_t G,
                                                               uint64_t *__restrict__ counts)
{
    const uint64_t *row = dense + (uint64_t)blockIdx.x * G;
    uint32_t c = 0;
    for (uint64_t g = threadIdx.x; g < G; g += kCompactThreads) c += row[g] != 0;
    __shared__ uint32_t red[kCompactThreads / 32];
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}

// Exclusive scan of T counts in one block of 1024 threads: every thread owns a
// contiguous run of rows.  row_ptr has T+1 entries; row_ptr[T] is the total.
__global__ void __launch_bounds__(1024) k_scan_rows(const uint64_t *__restrict__ counts, uint64_t T,
                                                   uint64_t *__restrict__ row_ptr)
{
    __shared__ uint64_t part[1024];
    const uint64_t per = (T + 1023) / 1024;
    const uint64_t r0 = threadIdx.x * per, r1 = min(T, r0 + per);
    uint64_t s = 0;
    for (uint64_t r = r0; r < r1; ++r) s += counts[r];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // Hillis-Steele inclusive scan
        const uint64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t acc = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (uint64_t r = r0; r < r1; ++r) {
        row_ptr[r] = acc;
        acc += counts[r];
    }
    if (threadIdx.x == 1023) row_ptr[T] = part[1023];
}

__global__ void __launch_bounds__(kCompactThreads) k_write_rows(const uint64_t *__restrict__ dense, uint64_t G,
                                                               const uint64_t *__restrict__ row_ptr,
                                                               uint32_t *__restrict__ cols,
                                                               uint64_t *__restrict__ vals)
{
    const uint64_t *row = dense + (uint64_t)blockIdx.x * G;
    uint64_t base = row_ptr[blockIdx.x];
    __shared__ uint32_t wsum[kCompactThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t g0 = 0; g0 < G; g0 += kCompactThreads) {
        const uint64_t g = g0 + threadIdx.x;
        const uint64_t v = g < G ? row[g] : 0;
        const unsigned ball = __ballot_sync(0xffffffffu, v != 0);
        if (lane == 0) wsum[warp] = __popc(ball);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) {
            before += w < warp ? wsum[w] : 0;
            total += wsum[w];
        }
        if (v) {
            const uint64_t at = base + before + __popc(ball & ((1u << lane) - 1));
            cols[at] = (uint32_t)g;
            vals[at] = v;
        }
        base += total;
        __syncthreads();
    }
}

cudaError_t launch_scan_counts(const uint64_t *counts, uint64_t n, uint64_t *out, cudaStream_t st)
{
    k_scan_rows<<<1, 1024, 0, st>>>(counts, n, out);
    return cudaGetLastError();
}

}  // namespace pe

using namespace pe;

extern "C" pe_status poly_eval_compact(const uint64_t *dense, uint64_t T, uint64_t G, uint64_t *row_ptr,
                                       uint32_t *cols, uint64_t *vals, uint64_t capacity, uint64_t *nnz,
                                       void *stream)
{
    if (!nnz || (T && !row_ptr) || (T && G && !dense) || T > 0x7fffffffull || G > 0xffffffffull) {
        set_error("bad arguments (device dense and row_ptr, host nnz; T < 2^31, G < 2^32)");
        return PE_ERR_ARG;
    }
    *nnz = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (T == 0) return PE_OK;
    if (G == 0) {
        if ((e = cudaMemsetAsync(row_ptr, 0, (T + 1) * 8, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "compact");
        return PE_OK;
    }
    // Row counts go to scratch; the scan writes row_ptr from them.
    DevBuf counts;
    if ((e = counts.ensure(T * 8, st)) != cudaSuccess) return cuda_fail(e, "compact scratch");
    k_count_rows<<<(unsigned)T, kCompactThreads, 0, st>>>(dense, G, counts.as<uint64_t>());
    k_scan_rows<<<1, 1024, 0, st>>>(counts.as<uint64_t>(), T, row_ptr);
    uint64_t total = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&total, row_ptr + T, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "compact count");
    *nnz = total;
    if (total > capacity) {
        set_error("%llu nonzero coefficients exceed the capacity %llu", (unsigned long long)total,
                  (unsigned long long)capacity);
        return PE_ERR_ARG;
    }
    if (total && (!cols || !vals)) {
        set_error("cols or vals is NULL");
        return PE_ERR_ARG;
    }
    if (total) k_write_rows<<<(unsigned)T, kCompactThreads, 0, st>>>(dense, G, row_ptr, cols, vals);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "compact write");
    return PE_OK;
}
