// Step B of the matrix method (paper Sect. 2.3, Algorithm 1): T rounds of
// v_i <- v_i * m_i mod p, each followed by the coefficient reduction, the sum
// of v_i over every (x1, x2) group.
//
// Work decomposition (one warp per work item):
//  * The terms, sorted by group, are cut into lane chunks of at most K terms
//    of one group.  A lane keeps its chunk's v_i and multipliers in registers
//    across all the points of the item, so the terms are read once per item
//    (the paper's dependent evaluations T_d, Sect. 4.1, with the register file
//    as the cache).  The K chains of a lane are independent, which gives the
//    instruction-level parallelism that Sect. 4.2 obtains from T_i.
//  * 32 consecutive chunks form a slab; an item is `kslabs` consecutive slabs
//    (a "unit") over Tc consecutive points (a "T-chunk").  Items of later
//    T-chunks start from v_i = a_i * m_i^t by square-and-multiply (the
//    Gamma-jump of the Hu-Monagan parallelisation, Sect. 2.3.1, without the
//    extra vectors).
//  * Per point, each lane adds its K values lazily into 96 bits (the
//    reduction order does not matter: addition in F_p is associative) and
//    writes that partial to shared memory.  After 32 points the warp
//    transposes: lane t walks the 32 partials of point t in chunk order and
//    closes a group wherever the group id changes (a segmented sum whose
//    segment boundaries are warp-uniform, so the walk never diverges).
//  * A group cut by a slab boundary inside the item continues through a
//    per-item chain buffer; a group cut by an item boundary leaves a partial
//    in a carry slot, and the last item of that group and T-chunk to finish
//    (an arrival counter) adds the slots and writes the output.
// Results are reduced to [0, p) only when they are written out.
#pragma once
#include "common.h"
#include "modarith.cuh"

namespace pe {

enum : int { VAR_MONT = 1, VAR_FP64 = 2, VAR_BARRETT = 3, VAR_BARRETT32 = 4 };

constexpr int kWalkStride = 33;  // shared-memory row stride (conflict-free transpose)

// Per-warp transpose buffer.  The high word of a lane partial (K values below
// 2^64 each, K <= 16) is below 16, so it is kept in a byte.
struct WarpSmem {
    uint64_t lo[32 * kWalkStride];
    uint32_t g[32];
    uint8_t hi[32 * kWalkStride];
    uint8_t pad[(16 - (32 * kWalkStride) % 16) % 16];
};

template <int VAR>
struct Lane;

template <>
struct Lane<VAR_BARRETT> {
    uint64_t v, w, wq;
    __device__ __forceinline__ void init(uint64_t v0, uint64_t mR, const ModCtx &mc)
    {
        v = v0;
        w = canon(mont_redc(mR, 0, mc), mc.p);
        wq = barrett_quotient_from_mont(mR, mc);
    }
    __device__ __forceinline__ void zero() { v = 0; w = 0; wq = 0; }
};

// 32-bit lanes (p < 2^30): floor(m * 2^32 / p) is the top word of the 64-bit
// quotient floor(m * 2^64 / p).
template <>
struct Lane<VAR_BARRETT32> {
    uint32_t v, w, wq;
    __device__ __forceinline__ void init(uint64_t v0, uint64_t mR, const ModCtx &mc)
    {
        v = (uint32_t)v0;
        w = (uint32_t)canon(mont_redc(mR, 0, mc), mc.p);
        wq = (uint32_t)(barrett_quotient_from_mont(mR, mc) >> 32);
    }
    __device__ __forceinline__ void zero() { v = 0; w = 0; wq = 0; }
};

template <>
struct Lane<VAR_MONT> {
    uint64_t v, y;
    __device__ __forceinline__ void init(uint64_t v0, uint64_t mR, const ModCtx &) { v = v0; y = mR; }
    __device__ __forceinline__ void zero() { v = 0; y = 0; }
};

template <>
struct Lane<VAR_FP64> {
    double v, m;
    __device__ __forceinline__ void init(uint64_t v0, uint64_t mR, const ModCtx &mc)
    {
        v = (double)v0;
        m = (double)canon(mont_redc(mR, 0, mc), mc.p);
    }
    __device__ __forceinline__ void zero() { v = 0.0; m = 0.0; }
};

// One point for a lane's K terms: partial = sum of the current values, then
// every value advances by one power of m (the accumulate-then-multiply order
// of Algorithm 7 keeps the two operations independent).
template <int K, int VAR>
__device__ __forceinline__ void lane_point(Lane<VAR> (&st)[K], const ModCtx &mc, uint64_t &lo, uint32_t &hi)
{
    if constexpr (VAR == VAR_FP64) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            acc = fp64_addmod(acc, st[k].v, mc.pd);
            st[k].v = fp64_mulmod(st[k].v, st[k].m, mc.pd, mc.ud);
        }
        lo = (uint64_t)acc;
        hi = 0;
    } else if constexpr (VAR == VAR_BARRETT32) {
        // K values below 2^32 each: the sum fits in 64 bits.
        const uint32_t p = (uint32_t)mc.p;
        lo = 0;
        hi = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            lo += st[k].v;
            st[k].v = barrett_mul32(st[k].v, st[k].w, st[k].wq, p);
        }
    } else {
        lo = 0;
        hi = 0;
        const uint64_t np = 0ull - mc.p;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            add96(lo, hi, st[k].v);
            if constexpr (VAR == VAR_BARRETT)
                st[k].v = barrett_mul_lazy4_mad(st[k].v, st[k].w, st[k].wq, np);
            else
                st[k].v = mont_mul(st[k].v, st[k].y, mc);
        }
    }
}

// Monomial value of term i in Montgomery form (Step A, Sect. 2.3): the product
// of one power-table entry per evaluated variable, n-3 products.
template <typename ExpT>
__device__ __forceinline__ uint64_t monomial_mont(const ExpT *__restrict__ exps, uint64_t s, uint64_t i,
                                                  uint32_t E, const uint64_t *__restrict__ ptab, uint32_t dp1,
                                                  const ModCtx &mc)
{
    if (E == 0) return mc.r1;
    uint64_t x = ptab[exps[i]];
    for (uint32_t j = 1; j < E; ++j) x = mont_mul(x, ptab[(uint64_t)j * dp1 + exps[(uint64_t)j * s + i]], mc);
    return canon(x, mc.p);
}

__device__ __forceinline__ uint64_t fused_monomial(const StepBJob &J, uint64_t i)
{
    if (J.exp_bytes == 1)
        return monomial_mont((const uint8_t *)J.exps, J.s, i, J.E, J.ptab, J.dp1, J.mc);
    return monomial_mont((const uint16_t *)J.exps, J.s, i, J.E, J.ptab, J.dp1, J.mc);
}

// Where a finished group partial goes: a carry slot when the group crosses the
// item's left (first chain) or right (chain reaching the end) boundary,
// otherwise straight to the output.
__device__ __forceinline__ void close_group(const StepBJob &J, uint64_t row, uint32_t g, bool first_chain,
                                            bool at_end, int32_t lslot, int32_t rslot, uint64_t lo, uint32_t hi)
{
    if (first_chain && lslot >= 0)
        J.carry[(uint64_t)lslot * J.T + row] = make_ulonglong2(lo, hi);
    else if (at_end && rslot >= 0)
        J.carry[(uint64_t)rslot * J.T + row] = make_ulonglong2(lo, hi);
    else
        J.out[row * J.G + g] = reduce96(lo, hi, J.mc);
}

// Step A is fused (m_i computed from the exponents and power tables) when the
// job has no precomputed monomial array.
template <int K, int VAR>
__device__ __forceinline__ void stepb_item(const StepBJob &J, uint32_t item, WarpSmem &sm)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t u = item % J.U;
    const uint32_t q = item / J.U;
    const uint32_t c_begin = u * J.kslabs * 32u;
    const uint32_t c_end = min(J.NC, c_begin + J.kslabs * 32u);
    const uint64_t r_begin = (uint64_t)q * J.Tc;
    const uint64_t r_end = min(J.T, r_begin + J.Tc);
    const int32_t lslot = J.u_lslot[u], rslot = J.u_rslot[u];
    const ModCtx &mc = J.mc;
    ulonglong2 *chain = J.chain + (uint64_t)item * J.Tc;
    bool cur_first = true;

    for (uint32_t sb = c_begin; sb < c_end; sb += 32) {
        const uint32_t c = sb + lane;
        const bool valid = c < c_end;
        uint32_t start = 0, cnt = 0, gid = 0xffffffffu;
        if (valid) {
            start = J.cs[c];
            cnt = J.cs[c + 1] - start;
            gid = J.cg[c];
        }
        // Starting values a_i * m_i^(t0 + r_begin): precomputed by Step A for
        // plain runs, otherwise by square-and-multiply here (jump start).
        const uint64_t e = J.t0 + r_begin;
        Lane<VAR> st[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if ((uint32_t)k < cnt) {
                const uint64_t i = (uint64_t)start + k;
                const uint64_t mR = J.mR ? J.mR[i] : fused_monomial(J, i);
                const uint64_t v0 = J.vstart ? J.vstart[(uint64_t)(J.vs_base + q) * J.s + i]
                                             : canon(mont_mul(J.coeffs[i], mont_pow(mR, e, mc), mc), mc.p);
                st[k].init(v0, mR, mc);
            } else {
                st[k].zero();
            }
        }
        const uint32_t nvalid = min(32u, c_end - sb);
        const uint32_t prevg = __shfl_up_sync(FULL, gid, 1);
        const uint32_t bmask = __ballot_sync(FULL, valid && lane > 0 && gid != prevg);
        sm.g[lane] = gid;
        const bool chain_in = (sb > c_begin) && (J.cg[sb] == J.cg[sb - 1]);
        const bool last_slab = sb + 32 >= c_end;
        const bool chain_out = !last_slab && (J.cg[sb + 31] == J.cg[sb + 32]);
        if (!chain_in) cur_first = (sb == c_begin);
        const bool slab_first = cur_first;
        __syncwarp();

        for (uint64_t rs = r_begin; rs < r_end; rs += 32) {
            const uint32_t nt = (uint32_t)min((uint64_t)32, r_end - rs);
            ulonglong2 cin = make_ulonglong2(0, 0);
            if (chain_in && (uint32_t)lane < nt) cin = chain[(rs - r_begin) + lane];
            for (uint32_t tt = 0; tt < nt; ++tt) {
                uint64_t lo;
                uint32_t hi;
                lane_point<K, VAR>(st, mc, lo, hi);
                sm.lo[tt * kWalkStride + lane] = lo;
                // The 32-bit product's sums never reach 2^64 (values below
                // 2^31, fewer than 2^32 terms): its high word is always zero.
                if constexpr (VAR != VAR_BARRETT32) sm.hi[tt * kWalkStride + lane] = (uint8_t)hi;
            }
            __syncwarp();
            if ((uint32_t)lane < nt) {
                const uint64_t row = rs + lane;
                uint64_t alo = cin.x;
                uint32_t ahi = (uint32_t)cin.y;
                bool first = slab_first;
                const uint64_t *plo = sm.lo + lane * kWalkStride;
                const uint8_t *phi = sm.hi + lane * kWalkStride;
                for (uint32_t l = 0; l < nvalid; ++l) {
                    if ((bmask >> l) & 1u) {
                        close_group(J, row, sm.g[l - 1], first, false, lslot, rslot, alo, ahi);
                        alo = 0;
                        ahi = 0;
                        first = false;
                    }
                    if constexpr (VAR == VAR_BARRETT32)
                        alo += plo[l];
                    else
                        add96(alo, ahi, plo[l], phi[l]);
                }
                if (chain_out)
                    chain[row - r_begin] = make_ulonglong2(alo, ahi);
                else
                    close_group(J, row, sm.g[nvalid - 1], first, last_slab, lslot, rslot, alo, ahi);
            }
            __syncwarp();
        }
        cur_first = slab_first && (bmask == 0);
    }

    // Arrival at the item's boundary groups; the last item of a group and
    // T-chunk to arrive adds the carry slots and writes the output rows.
    __threadfence();
    __syncwarp();
    const int32_t spans[2] = {J.u_lspan[u], J.u_rspan[u]};
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const int32_t sp = spans[w];
        if (sp < 0) continue;
        const uint32_t ns = J.span_n[sp];
        uint32_t last = 0;
        if (lane == 0) last = (atomicAdd(&J.counters[(uint64_t)sp * J.Q + q], 1u) + 1u == ns);
        last = __shfl_sync(FULL, last, 0);
        if (!last) continue;
        __threadfence();
        const uint32_t g = J.span_g[sp], base = J.span_base[sp];
        for (uint64_t row = r_begin + lane; row < r_end; row += 32) {
            uint64_t alo = 0;
            uint32_t ahi = 0;
            for (uint32_t j = 0; j < ns; ++j) {
                const ulonglong2 cv = __ldcg(&J.carry[(uint64_t)(base + j) * J.T + row]);
                add96(alo, ahi, cv.x, (uint32_t)cv.y);
            }
            J.out[row * J.G + g] = reduce96(alo, ahi, mc);
        }
        __syncwarp();
        if (lane == 0) J.counters[(uint64_t)sp * J.Q + q] = 0u;  // ready for the next run
    }
}

}  // namespace pe
