// Step B without any allocation: for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory themselves: code running inside
// another framework's memory pool, an embedded runtime without allocator
// access, or a process that has promised never to grow its footprint after
// start-up.  This entry point serves them: the caller passes its inputs and
// its output, and every scratch byte the kernel needs (carry slots, chain
// buffers and arrival counters) comes from one file-scope device array of
// fixed size that the library reserves on each GPU where it is loaded.
//
// It runs the same arithmetic as the regular Step B (Barrett products with a
// per-term quotient, 96-bit lazy sums, group sums finished at the end) with a
// plan that needs no tables: each lane holds one term, a work unit is a run
// of whole 32-term slabs, and the groups come from the caller's offsets.
#include <algorithm>
#include <mutex>
#include "internal.h"
#include "modarith.cuh"
#include "stepb.cuh"

namespace pe {

constexpr size_t kNoAllocScratchBytes = 32u << 20;   // 32 MiB per device

// The scratch array.  In host code this name is only a host-side stand-in,
// never a device address: host code must use the address returned by
// cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocJob {
    const uint64_t *coeffs;   // s, sorted by group
    const uint64_t *m;        // s, monomial values in [0, p)
    const uint32_t *goff;     // G+1 term offsets of the groups
    uint64_t *out;            // T x G
    ulonglong2 *carry;        // 2U x T
    ulonglong2 *chain;        // U*Q x Tc
    uint32_t *counters;       // U*Q
    uint32_t s, G, U, Q, kslabs, Tc;
    uint64_t T, t0;
    ModCtx mc;
};

// Group of term i: the largest g with goff[g] <= i.
__device__ __forceinline__ uint32_t na_group_of(const uint32_t *goff, uint32_t G, uint32_t i)
{
    uint32_t lo = 0, hi = G;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(goff + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void na_close(const NoAllocJob &J, uint64_t row, uint32_t g, bool first_chain,
                                         bool at_end, int64_t lslot, int64_t rslot, uint64_t lo, uint32_t hi)
{
    if (first_chain && lslot >= 0)
        J.carry[(uint64_t)lslot * J.T + row] = make_ulonglong2(lo, hi);
    else if (at_end && rslot >= 0)
        J.carry[(uint64_t)rslot * J.T + row] = make_ulonglong2(lo, hi);
    else
        J.out[row * J.G + g] = reduce96(lo, hi, J.mc);
}

constexpr int kNaWarps = 2;   // 2 x 12.8 KB of static shared memory per block

__global__ void __launch_bounds__(kNaWarps * 32) k_stepB_noalloc(NoAllocJob J)
{
    __shared__ WarpSmem smem[kNaWarps];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t item = blockIdx.x * kNaWarps + (threadIdx.x >> 5);
    if (item >= J.U * J.Q) return;
    WarpSmem &sm = smem[threadIdx.x >> 5];
    const ModCtx &mc = J.mc;
    const uint32_t per_unit = 32u * J.kslabs;
    const uint32_t u = item % J.U, q = item / J.U;
    const uint32_t ca = u * per_unit, cb = min(J.s, ca + per_unit);
    const uint64_t r_begin = (uint64_t)q * J.Tc, r_end = min(J.T, r_begin + J.Tc);
    const uint32_t gL = na_group_of(J.goff, J.G, ca), gR = na_group_of(J.goff, J.G, cb - 1);
    const bool lopen = J.goff[gL] < ca;
    const bool ropen = J.goff[gR + 1] > cb;
    const int64_t lslot = lopen ? 2 * (int64_t)u : -1;
    const int64_t rslot = (ropen && !(lopen && gL == gR)) ? 2 * (int64_t)u + 1 : -1;
    ulonglong2 *chain = J.chain + (uint64_t)item * J.Tc;
    bool cur_first = true;
    uint32_t prev_last_gid = 0xffffffffu;

    for (uint32_t sb = ca; sb < cb; sb += 32) {
        const uint32_t i = sb + lane;
        const bool valid = i < cb;
        const uint32_t gid = valid ? na_group_of(J.goff, J.G, i) : 0xffffffffu;
        Lane<VAR_BARRETT> st[1];
        if (valid) {
            const uint64_t mR = canon(mont_mul(J.m[i], mc.r2, mc), mc.p);
            const uint64_t v0 = canon(mont_mul(J.coeffs[i], mont_pow(mR, J.t0 + r_begin, mc), mc), mc.p);
            st[0].init(v0, mR, mc);
        } else {
            st[0].zero();
        }
        const uint32_t nvalid = min(32u, cb - sb);
        const uint32_t prevg = __shfl_up_sync(FULL, gid, 1);
        const uint32_t bmask = __ballot_sync(FULL, valid && lane > 0 && gid != prevg);
        const uint32_t first_gid = __shfl_sync(FULL, gid, 0);
        const uint32_t last_gid = __shfl_sync(FULL, gid, nvalid - 1);
        sm.g[lane] = gid;
        const bool chain_in = sb > ca && first_gid == prev_last_gid;
        const bool last_slab = sb + 32 >= cb;
        const bool chain_out = !last_slab && J.goff[last_gid + 1] > sb + 32;
        if (!chain_in) cur_first = (sb == ca);
        const bool slab_first = cur_first;
        __syncwarp();
        for (uint64_t rs = r_begin; rs < r_end; rs += 32) {
            const uint32_t nt = (uint32_t)min((uint64_t)32, r_end - rs);
            ulonglong2 cin = make_ulonglong2(0, 0);
            if (chain_in && (uint32_t)lane < nt) cin = chain[(rs - r_begin) + lane];
            for (uint32_t tt = 0; tt < nt; ++tt) {
                uint64_t lo;
                uint32_t hi;
                lane_point<1, VAR_BARRETT>(st, mc, lo, hi);
                sm.lo[tt * kWalkStride + lane] = lo;
                sm.hi[tt * kWalkStride + lane] = (uint8_t)hi;
            }
            __syncwarp();
            if ((uint32_t)lane < nt) {
                const uint64_t row = rs + lane;
                uint64_t alo = cin.x;
                uint32_t ahi = (uint32_t)cin.y;
                bool first = slab_first;
                for (uint32_t l = 0; l < nvalid; ++l) {
                    if ((bmask >> l) & 1u) {
                        na_close(J, row, sm.g[l - 1], first, false, lslot, rslot, alo, ahi);
                        alo = 0;
                        ahi = 0;
                        first = false;
                    }
                    add96(alo, ahi, sm.lo[lane * kWalkStride + l], sm.hi[lane * kWalkStride + l]);
                }
                if (chain_out)
                    chain[row - r_begin] = make_ulonglong2(alo, ahi);
                else
                    na_close(J, row, sm.g[nvalid - 1], first, last_slab, lslot, rslot, alo, ahi);
            }
            __syncwarp();
        }
        cur_first = slab_first && bmask == 0;
        prev_last_gid = last_gid;
    }

    // Arrivals: the span of a group is named by its first unit ua; unit w
    // contributes slot 2w (its left partial) or 2ua+1 (the first unit's right one).
    __threadfence();
    __syncwarp();
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const bool has = side == 0 ? lslot >= 0 : rslot >= 0;
        if (!has) continue;
        const uint32_t g = side == 0 ? gL : gR;
        // Offsets that break the contract (decreasing, or past s) must not
        // send the span outside the carry slots and counters: clamp it to the
        // units that exist.  Such inputs give unspecified images, never a
        // stray access.
        const uint32_t ua = min(J.goff[g] / per_unit, J.U - 1);
        const uint32_t ub = max(ua, min((J.goff[g + 1] - 1) / per_unit, J.U - 1));
        uint32_t last = 0;
        if (lane == 0) last = atomicAdd(&J.counters[(uint64_t)ua * J.Q + q], 1u) + 1u == ub - ua + 1;
        last = __shfl_sync(FULL, last, 0);
        if (!last) continue;
        __threadfence();
        for (uint64_t row = r_begin + lane; row < r_end; row += 32) {
            ulonglong2 cv = __ldcg(&J.carry[(2 * (uint64_t)ua + 1) * J.T + row]);
            uint64_t alo = cv.x;
            uint32_t ahi = (uint32_t)cv.y;
            for (uint32_t w = ua + 1; w <= ub; ++w) {
                cv = __ldcg(&J.carry[(2 * (uint64_t)w) * J.T + row]);
                add96(alo, ahi, cv.x, (uint32_t)cv.y);
            }
            J.out[row * J.G + g] = reduce96(alo, ahi, mc);
        }
    }
}

// Work units of kslabs whole 32-term slabs and Q T-chunks of Tc points, with
// the byte offsets of the carry slots and chain buffers in the scratch array.
struct NoAllocShape {
    uint32_t U = 0, Q = 0, Tc = 0, kslabs = 0;
    size_t off_carry = 0, off_chain = 0, need = 0;
};

// Tile choice: whole slabs per unit, as few as fit the scratch, and enough
// T-chunks to give every SM work.  At least one unit per SM (or per slab when
// there are fewer slabs): a larger kslabs would leave most of the GPU idle, so
// such inputs are rejected (returns false).
static bool na_plan(uint64_t s, uint64_t T, NoAllocShape &out)
{
    const uint64_t items_target = (uint64_t)num_sms() * 16;
    const uint64_t slabs = (s + 31) / 32;
    const uint64_t min_units = std::min<uint64_t>(slabs, (uint64_t)num_sms());
    for (uint32_t k = 1; k <= (1u << 20); k *= 2) {
        const uint64_t U = (s + 32ull * k - 1) / (32ull * k);
        if (U < min_units) break;
        uint64_t Q = (items_target + U - 1) / U;
        Q = std::max<uint64_t>(1, std::min<uint64_t>(Q, std::max<uint64_t>(1, T / 32)));
        const uint64_t Tc = (T + Q - 1) / Q;
        Q = (T + Tc - 1) / Tc;
        const size_t off_carry = ((U * Q * 4 + 255) / 256) * 256;
        const size_t off_chain = off_carry + 2 * U * T * 16;
        const size_t need = off_chain + (k > 1 ? U * Q * Tc * 16 : 0);
        if (need <= kNoAllocScratchBytes) {
            out.U = (uint32_t)U;
            out.Q = (uint32_t)Q;
            out.Tc = (uint32_t)Tc;
            out.kslabs = k;
            out.off_carry = off_carry;
            out.off_chain = off_chain;
            out.need = need;
            return true;
        }
        if (U == 1) break;
    }
    return false;
}

// Scratch address for each device, looked up once with that device current.
static std::mutex g_na_mu;
static void *g_na_ptr[64] = {nullptr};

static pe_status na_scratch(void **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return PE_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_na_ptr[dev] = p;
    }
    *ptr = g_na_ptr[dev];
    return PE_OK;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace pe

using namespace pe;

extern "C" pe_status poly_eval_stepb_noalloc(uint64_t p, uint64_t s, uint64_t G, const uint64_t *coeffs,
                                             const uint64_t *m, const uint32_t *group_off, uint64_t T, uint64_t t0,
                                             uint64_t *out, void *stream)
{
    if (p < 3 || !(p & 1) || p >= (1ull << 62)) {
        set_error("p must be odd, at least 3 and below 2^62");
        return PE_ERR_PRIME;
    }
    if (!points_ok(T, t0) || !out_ok(T, G)) return PE_ERR_ARG;
    if (T == 0 || s == 0) return PE_OK;
    if (G == 0 || G > s || s >= 0xffffffffull) {
        set_error("sizes out of range (need 1 <= G <= s < 2^32 - 1, T <= 2^31)");
        return PE_ERR_ARG;
    }
    if (!coeffs || !m || !group_off || !out || !is_device_ptr(coeffs) || !is_device_ptr(m) ||
        !is_device_ptr(group_off) || !is_device_ptr(out)) {
        set_error("coeffs, m, group_off and out must be device pointers");
        return PE_ERR_ARG;
    }
    NoAllocShape sh;
    if (!na_plan(s, T, sh)) {
        set_error("input needs more scratch than the fixed %zu bytes (s*T too large for this entry point)",
                  kNoAllocScratchBytes);
        return PE_ERR_ARG;
    }
    NoAllocJob J{};
    J.U = sh.U;
    J.Q = sh.Q;
    J.Tc = sh.Tc;
    J.kslabs = sh.kslabs;
    const size_t off_carry = sh.off_carry, off_chain = sh.off_chain;
    void *base = nullptr;
    pe_status st = na_scratch(&base);
    if (st != PE_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    unsigned char *b = (unsigned char *)base;
    cudaError_t e = cudaMemsetAsync(b, 0, (size_t)J.U * J.Q * 4, cs);   // counters start at zero
    if (e != cudaSuccess) return cuda_fail(e, "clearing counters");
    J.coeffs = coeffs;
    J.m = m;
    J.goff = group_off;
    J.out = out;
    J.counters = (uint32_t *)b;
    J.carry = (ulonglong2 *)(b + off_carry);
    J.chain = (ulonglong2 *)(b + off_chain);
    J.s = (uint32_t)s;
    J.G = (uint32_t)G;
    J.T = T;
    J.t0 = t0;
    J.mc = make_modctx(p);
    const uint32_t nitems = J.U * J.Q;
    k_stepB_noalloc<<<(nitems + kNaWarps - 1) / kNaWarps, kNaWarps * 32, 0, cs>>>(J);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "Step B (no allocation)");
    return PE_OK;
}

extern "C" pe_status poly_eval_stepb_noalloc_shape(uint64_t s, uint64_t T, uint32_t shape[4])
{
    if (!shape) {
        set_error("shape must not be NULL");
        return PE_ERR_ARG;
    }
    shape[0] = shape[1] = shape[2] = shape[3] = 0;
    if (T == 0 || s == 0) return PE_OK;
    if (s >= 0xffffffffull || T > (1ull << 31)) {
        set_error("sizes out of range (need s < 2^32 - 1, T <= 2^31)");
        return PE_ERR_ARG;
    }
    NoAllocShape sh;
    if (!na_plan(s, T, sh)) {
        set_error("input needs more scratch than the fixed %zu bytes (s*T too large for this entry point)",
                  kNoAllocScratchBytes);
        return PE_ERR_ARG;
    }
    shape[0] = sh.U;
    shape[1] = sh.Q;
    shape[2] = sh.Tc;
    shape[3] = sh.kslabs;
    return PE_OK;
}
