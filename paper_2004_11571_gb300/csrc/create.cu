// Device side of poly_eval_create for terms already in group order: the raw
// term arrays are copied to the device as given, and these kernels check
// them, find the (x1, x2) groups and pack the exponents of x3..xn into the
// structure-of-arrays layout that Step A reads (Sect. 2.3: terms sorted in
// lex order, so like monomials in (x1, x2) are adjacent).
//
//   k_term_scan   : coefficient range (a_i < p), (d, e) keys, largest evaluated
//                   exponent, and whether the keys are nonincreasing
//   k_group_count : group starts per block of 1024 terms
//   k_group_write : start offset and (d, e) of every group, in order
//   k_pack_exps   : exponents of x3..xn as E rows of s values (u8 or u16)
// Memory-bound passes over the input; the host reads back only the flags,
// the group count and the group table.
#include "internal.h"
#include "kernels.h"

namespace pe {

constexpr int kCreateBlock = 1024;

template <typename W>
__global__ void k_term_scan(const uint64_t *__restrict__ coeffs, const W *__restrict__ exps, uint64_t s, uint32_t n,
                            uint64_t p, uint64_t *__restrict__ keys, CreateInfo *__restrict__ info)
{
    uint32_t dm = 0;
    bool unsorted = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (uint64_t)gridDim.x * blockDim.x) {
        if (coeffs[i] >= p) atomicMin((unsigned long long *)&info->bad, (unsigned long long)i);
        const W *row = exps + i * n;
        const uint64_t key = ((uint64_t)row[0] << 32) | (uint64_t)row[1];
        keys[i] = key;
        for (uint32_t j = 2; j < n; ++j) dm = max(dm, (uint32_t)row[j]);
        if (i > 0) {
            const W *prev = row - n;
            const uint64_t pk = ((uint64_t)prev[0] << 32) | (uint64_t)prev[1];
            unsorted |= key > pk;
        }
    }
    for (int o = 16; o; o >>= 1) dm = max(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    const bool any_unsorted = __any_sync(0xffffffffu, unsorted);
    if ((threadIdx.x & 31) == 0) {
        if (dm) atomicMax(&info->dmax, dm);
        if (any_unsorted) atomicOr(&info->unsorted, 1u);
    }
}

__device__ __forceinline__ bool group_start(const uint64_t *keys, uint64_t i)
{
    return i == 0 || keys[i] != keys[i - 1];
}

__global__ void __launch_bounds__(kCreateBlock) k_group_count(const uint64_t *__restrict__ keys, uint64_t s,
                                                             uint64_t *__restrict__ counts)
{
    const uint64_t i = (uint64_t)blockIdx.x * kCreateBlock + threadIdx.x;
    const int c = __syncthreads_count(i < s && group_start(keys, i));
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint64_t)c;
}

// Block b writes its groups at base[b] + (starts before them in the block).
__global__ void __launch_bounds__(kCreateBlock) k_group_write(const uint64_t *__restrict__ keys, uint64_t s,
                                                             const uint64_t *__restrict__ base,
                                                             uint64_t *__restrict__ goff, uint32_t *__restrict__ gkeys)
{
    __shared__ uint32_t wsum[kCreateBlock / 32];
    const uint64_t i = (uint64_t)blockIdx.x * kCreateBlock + threadIdx.x;
    const bool st = i < s && group_start(keys, i);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ball = __ballot_sync(0xffffffffu, st);
    if (lane == 0) wsum[warp] = __popc(ball);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (st) {
        const uint64_t at = base[blockIdx.x] + before + __popc(ball & ((1u << lane) - 1u));
        const uint64_t key = keys[i];
        goff[at] = i;
        gkeys[2 * at] = (uint32_t)(key >> 32);
        gkeys[2 * at + 1] = (uint32_t)key;
    }
}

template <typename W, typename OutT>
__global__ void k_pack_exps(const W *__restrict__ exps, uint64_t s, uint32_t n, uint32_t E, OutT *__restrict__ out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (uint64_t)gridDim.x * blockDim.x) {
        const W *row = exps + i * n + 2;
        for (uint32_t j = 0; j < E; ++j) out[(uint64_t)j * s + i] = (OutT)row[j];
    }
}

static unsigned stream_grid(uint64_t s)
{
    return (unsigned)std::min<uint64_t>((s + 255) / 256, (uint64_t)num_sms() * 16);
}

cudaError_t launch_term_scan(const uint64_t *coeffs, const void *exps, uint32_t width, uint64_t s, uint32_t n,
                             uint64_t p, uint64_t *keys, CreateInfo *info, uint64_t *counts, uint64_t *base,
                             uint64_t *goff, uint32_t *gkeys, cudaStream_t st)
{
    const unsigned g = stream_grid(s);
    switch (width) {
    case 1: k_term_scan<uint8_t><<<g, 256, 0, st>>>(coeffs, (const uint8_t *)exps, s, n, p, keys, info); break;
    case 2: k_term_scan<uint16_t><<<g, 256, 0, st>>>(coeffs, (const uint16_t *)exps, s, n, p, keys, info); break;
    default: k_term_scan<uint32_t><<<g, 256, 0, st>>>(coeffs, (const uint32_t *)exps, s, n, p, keys, info); break;
    }
    const uint64_t nb = (s + kCreateBlock - 1) / kCreateBlock;
    k_group_count<<<(unsigned)nb, kCreateBlock, 0, st>>>(keys, s, counts);
    cudaError_t e = launch_scan_counts(counts, nb, base, st);   // base[nb] = number of groups
    if (e != cudaSuccess) return e;
    k_group_write<<<(unsigned)nb, kCreateBlock, 0, st>>>(keys, s, base, goff, gkeys);
    return cudaGetLastError();
}

cudaError_t launch_pack_exps(const void *exps, uint32_t width, uint64_t s, uint32_t n, uint32_t out_bytes,
                             void *out, cudaStream_t st)
{
    const unsigned g = stream_grid(s);
    const uint32_t E = n - 2;
    if (E == 0) return cudaSuccess;
#define PE_PACK(W, O) k_pack_exps<W, O><<<g, 256, 0, st>>>((const W *)exps, s, n, E, (O *)out)
    if (out_bytes == 1) {
        if (width == 1) PE_PACK(uint8_t, uint8_t);
        else if (width == 2) PE_PACK(uint16_t, uint8_t);
        else PE_PACK(uint32_t, uint8_t);
    } else {
        if (width == 1) PE_PACK(uint8_t, uint16_t);
        else if (width == 2) PE_PACK(uint16_t, uint16_t);
        else PE_PACK(uint32_t, uint16_t);
    }
#undef PE_PACK
    return cudaGetLastError();
}

}  // namespace pe
