// Internal definitions shared by the host library and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pe {

constexpr int kMaxEval = 64;  // evaluated variables x3..xn (n <= 66)

// Per-prime constants, computed once on the host (Sect. 3.1: p is a run-time value).
struct ModCtx {
    uint64_t p;         // the modulus, odd, p < 2^62
    uint64_t p2;        // 2p
    uint64_t pinv;      // p^-1 mod 2^64
    uint64_t pinv_neg;  // -p^-1 mod 2^64 (Montgomery reduction)
    uint64_t r1;        // 2^64 mod p  (Montgomery form of 1)
    uint64_t r2;        // 2^128 mod p (converts into Montgomery form)
    uint64_t w64q;      // floor(r1 * 2^64 / p), Barrett quotient for multiplier r1
    uint64_t one_q;     // floor(2^64 / p), Barrett quotient for multiplier 1
    double pd;          // (double)p   (Algorithm 2)
    double ud;          // 1/(double)p rounded to nearest (Algorithm 2)
};

ModCtx make_modctx(uint64_t p);  // host

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (thread-safe; the attribute is per device).
cudaError_t smem_limit_once(const void *func, int bytes);

struct BetaArg {
    uint64_t b[kMaxEval];
};

// Step B arguments for one polynomial (plain kernel) or one job (batched kernel).
struct StepBJob {
    const uint64_t *coeffs;   // s, sorted by group
    const uint64_t *mR;       // s, m_i * 2^64 mod p (Step A output), or nullptr when fused
    const void *exps;         // E x s exponents (fused Step A)
    const uint64_t *ptab;     // E x dp1 power tables in Montgomery form (fused Step A)
    const uint32_t *cs;       // NC+1 chunk starts (term index)
    const uint32_t *cg;       // NC chunk group ids
    const int32_t *u_lslot, *u_rslot, *u_lspan, *u_rspan;  // per unit
    const uint32_t *span_g, *span_base, *span_n;            // per span
    uint32_t *counters;       // spans x Q arrival counters (self-resetting)
    ulonglong2 *carry;        // slots x T partial sums (96-bit as lo, hi)
    ulonglong2 *chain;        // items x Tc chain partials between slabs
    uint64_t *out;            // T x G
    uint64_t s, T, t0, G;
    uint32_t NC, U, Q, kslabs, Tc;
    uint32_t E, dp1, exp_bytes;
    uint32_t K, var;          // lane chunk size and modular product (queue dispatch)
    const uint64_t *vstart;   // L x s starting values a_i m_i^t per item start row, or nullptr (jump start)
    uint32_t vs_base;         // row of vstart used by T-chunk 0 of this job
    uint32_t item0;           // first work item of this launch (plain kernel: one launch per T-chunk)
    ModCtx mc;
};

constexpr int kMaxStarts = 128;
constexpr int kMaxGaps = 4;

// Start rows (offsets from t0) of the work items of a plain run, strictly
// increasing, and the distinct gaps between consecutive rows: row k follows
// row k-1 by gap[gidx[k]]; entries of gap past ngap are 0; gap_hb is the
// highest bit set in any gap.
struct StartRows {
    uint32_t n;
    uint32_t row[kMaxStarts];
    uint32_t ngap, gap_hb;
    uint32_t gap[kMaxGaps];
    uint8_t gidx[kMaxStarts];
};

}  // namespace pe
