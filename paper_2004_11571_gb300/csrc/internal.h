// Host-side internals shared by the API, batch, tuner and server sources.
#pragma once
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/poly_eval.h"
#include "common.h"

namespace pe {

void set_error(const char *fmt, ...);
pe_status cuda_fail(cudaError_t e, const char *what);

// The library's allocation stream on the current device.  Buffers come from
// the device's stream-ordered memory pool (kept cached: release threshold at
// its maximum), so allocating and freeing never synchronizes the device.  A
// buffer is freed only once no queued work can still use it: callers of the
// public destroy functions are synchronized first, the server frees what its
// completed epochs released.
cudaStream_t alloc_stream();

// Testing aid (poly_eval_debug_fail_alloc): true when this device
// allocation is the one chosen to fail.
bool alloc_fault_now();

// Owned device allocation that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFreeAsync(p, alloc_stream());
        p = nullptr;
        bytes = 0;
    }
    // Allocates on `s` (the library stream by default) and waits for it, so the
    // buffer is usable from any stream on return.
    cudaError_t ensure(size_t n, cudaStream_t s = nullptr)
    {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) n = 16;
        if (alloc_fault_now()) return cudaErrorMemoryAllocation;
        if (!s) s = alloc_stream();
        cudaError_t e = cudaMallocAsync(&p, n, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    // The same without waiting: the buffer is usable by work queued on `s`
    // (and by other streams once they wait for that work).
    cudaError_t ensure_async(size_t n, cudaStream_t s)
    {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) n = 16;
        if (alloc_fault_now()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMallocAsync(&p, n, s);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// Runs fn(0) .. fn(n-1) on a persistent pool of host threads (the caller
// takes part); calls from several host threads take turns.
void host_parallel(unsigned n, const std::function<void(unsigned)> &fn);
unsigned host_pool_size();

// Host side of a Step B work decomposition: units of kslabs slabs, T-chunks
// of Tc points, and the groups that cross unit boundaries ("spans").
struct PlanHost {
    uint32_t K = 0, kslabs = 0, Tc = 0, wpb = 0;
    uint64_t T = 0;
    uint32_t NC = 0, U = 0, Q = 0, S = 0, nslots = 0;
    std::vector<int32_t> unit;    // 4U: lslot, rslot, lspan, rspan
    std::vector<uint32_t> span;   // 3*max(S,1): group, slot base, slot count
    size_t counter_bytes() const;
    size_t carry_bytes() const;
    size_t chain_bytes() const;
};

// Work decomposition of Step B for one (polynomial, tile shape, T).
struct Plan {
    PlanHost host;
    bool valid = false;
    uint32_t K = 0, kslabs = 0, Q = 0, Tc = 0, wpb = 0;
    uint64_t T = 0;
    uint32_t NC = 0, U = 0, S = 0, nslots = 0;
    DevBuf cs, cg, gfirst, unit, span, counters, carry, chain;
    uint64_t scratch_bytes() const { return counters.bytes + carry.bytes + chain.bytes; }
};

// Lane chunks of at most K terms of one group.  gfirst (the first chunk of
// each group, G+1 entries) is always on the host; the per-chunk arrays cs/cg
// are built on the host only where a batch copies them into its image (a
// plain run builds them on the device from gfirst and the group offsets).
struct HostChunks {
    uint32_t K = 0;
    uint32_t NC = 0;
    std::vector<uint32_t> gfirst;       // first chunk of each group, G+1
    std::vector<uint32_t> cs, cg;       // NC+1, NC (empty until build_chunks)
};

struct Tiles {
    uint32_t K = 0, kslabs = 0, Tc = 0, wpb = 0;
    uint32_t tailT = 0;   // points in the tail band of one-slab items (0: none)
};

struct PowJob;

// A planned batch laid out in a device arena (see batch.cu).
struct BatchImage {
    std::vector<unsigned char> host;          // bytes to upload at `base`
    std::vector<std::vector<uint64_t>> betas;
    std::vector<size_t> beta_off;
    // Jobs with the same prime, number of variables and point share one set of
    // power tables (the leader's); every job keeps a slot of its own so that
    // poly_eval_batch_set_beta can split a job off.
    std::vector<size_t> leader;               // per job: the job whose tables it reads
    std::vector<size_t> ptab_off;             // per job: its own table slot (offset from base)
    size_t off_jobs = 0, off_pow = 0;         // descriptor arrays (offsets from base)
    uint32_t tables = 0;                      // power-table sets computed per launch
    unsigned char *base = nullptr;
    size_t counters_off = 0, counters_bytes = 0;
    StepBJob *d_jobs = nullptr;
    PowJob *d_pow = nullptr;
    uint2 *d_items = nullptr;
    uint32_t *d_head = nullptr;
    uint32_t nitems = 0, njobs = 0, max_entries = 0;
    int grid = 0;
    double term_points = 0.0;
    // Jobs large enough to fill the GPU on their own take no part in the image:
    // they run as plain runs (precomputed starting values, their own tiles)
    // after the queue kernel, on the same stream.
    struct PlainRun {
        size_t j;
        pe_poly *poly;
        uint64_t T, t0;
        uint64_t *out;
    };
    std::vector<uint8_t> is_plain;            // per job
    std::vector<PlainRun> plain;
};

// Work (term-points) from which a batch job runs as a plain run.
constexpr double kPlainRunWork = 268435456.0;   // 2^28

// plain_runs = false keeps every job in the queue (server epochs, which overlap
// on several streams and mix large requests with small ones).
pe_status batch_build(const pe_job *jobs, size_t njobs, DevBuf &arena, BatchImage &img, bool plain_runs = true);
cudaError_t batch_enqueue(const BatchImage &img, cudaStream_t st);
// The plain runs of a batch (after batch_enqueue or the batch's graph).
pe_status batch_run_plain(const BatchImage &img, cudaStream_t st);

}  // namespace pe

struct FastPlan;
void fast_plan_delete(FastPlan *f);

struct pe_poly {
    uint64_t p = 0;
    uint32_t n = 0, E = 0;
    uint64_t s = 0, G = 0;
    int variant = 0;             // variant of the current plan
    int requested_variant = 0;   // as created (PE_MODMUL_AUTO: tuner's choice, else Barrett)
    pe::ModCtx mc{};
    uint32_t exp_bytes = 1;      // 1 or 2 on the device
    uint32_t dmax = 0;           // max exponent over x3..xn
    std::vector<uint64_t> group_off;   // G+1 (host)
    std::vector<uint32_t> keys;        // 2G (host)
    pe::DevBuf coeffs, mR, ptab, out_scratch, vstart;
    pe::DevBuf goff_dev;                // G+1 uint32 group offsets on the device (plain-run chunk tables)
    // Exponents of x3..xn (E rows of s), shared with the polynomials made by
    // poly_eval_create_like, and the permutation that put the input terms in
    // group order (empty when they already were).
    std::shared_ptr<pe::DevBuf> exps = std::make_shared<pe::DevBuf>();
    std::shared_ptr<const std::vector<uint32_t>> perm;
    std::unique_ptr<FastPlan, void (*)(FastPlan *)> fast{nullptr, fast_plan_delete};   // poly_eval_run_fast state
    pe::HostChunks chunks;
    pe::Plan plan;        // band of large items: rows [0, T - tail)
    pe::Plan tail_plan;   // band of small items: the last tail rows
    uint32_t tailT = 0;
    pe_tiles forced{};
    bool timing = false;
    std::vector<cudaEvent_t> events;   // 4 per timed run
    size_t events_used = 0;
    cudaEvent_t last_use = nullptr;    // end of the latest run; frees of this handle's buffers wait for it
    // A run into page-locked host memory: T-chunks rotate over the run's
    // stream and `aux[0..1]`; their downloads queue on `copy_st`, each after
    // its chunk's event; fork and join events tie them to the run's stream.
    cudaStream_t aux[2] = {nullptr, nullptr}, copy_st = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    std::vector<cudaEvent_t> chunk_ev;
    ~pe_poly()
    {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (cudaEvent_t e : chunk_ev) cudaEventDestroy(e);
        if (last_use) cudaEventDestroy(last_use);
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (join_ev) cudaEventDestroy(join_ev);
        for (cudaStream_t a : aux)
            if (a) cudaStreamDestroy(a);
        if (copy_st) cudaStreamDestroy(copy_st);
    }
    uint64_t device_bytes() const
    {
        return coeffs.bytes + (exps.use_count() == 1 ? exps->bytes : 0) + mR.bytes + ptab.bytes + out_scratch.bytes + vstart.bytes +
               goff_dev.bytes + plan.cs.bytes + plan.cg.bytes + plan.gfirst.bytes + plan.unit.bytes + plan.span.bytes +
               plan.scratch_bytes() + tail_plan.cs.bytes + tail_plan.cg.bytes + tail_plan.gfirst.bytes +
               tail_plan.unit.bytes + tail_plan.span.bytes + tail_plan.scratch_bytes();
    }
};

namespace pe {
int num_sms();

// The points t0 .. t0+T-1 must be representable: T <= 2^31 and t0 + T - 1 < 2^64.
// Sets the error message and returns false otherwise.
bool points_ok(uint64_t T, uint64_t t0);

// The T x G output must hold at most 2^60 values (its byte count fits in 64
// bits with room to spare).  Sets the error message and returns false otherwise.
bool out_ok(uint64_t T, uint64_t G);

// Fills the distinct-gap fields of the start rows (row[0..n) already set);
// false if the rows do not increase or have more than kMaxGaps distinct gaps.
bool plan_start_gaps(StartRows *sr);
// Chooses the tile shape for a run of T points (forced fields win).
Tiles choose_tiles(pe_poly *poly, uint64_t T, const pe_tiles *forced);
// Builds (or reuses) `pl` for the given tiles and T.
// With `queued`, allocations, uploads and the counter reset are queued on
// `st` (the plan is then valid for work queued after them on that stream);
// otherwise they complete before the call returns.
pe_status ensure_plan(pe_poly *poly, Plan &pl, const Tiles &t, uint64_t T, cudaStream_t st = nullptr,
                      bool queued = false);
void build_gfirst(pe_poly *P, uint32_t K);
void build_chunks(pe_poly *P, uint32_t K);
void build_plan_host(pe_poly *P, const Tiles &t, uint64_t T, PlanHost &ph);
void fill_job(StepBJob &J, pe_poly *P, const PlanHost &ph, const uint32_t *cs, const uint32_t *cg,
              const int32_t *unit, const uint32_t *span, uint32_t *counters, ulonglong2 *carry, ulonglong2 *chain,
              uint64_t t0, uint64_t *out_dev, const uint64_t *mR, const uint64_t *ptab, int variant);
// Fills a Step B job description from a poly and its current plan.
StepBJob make_job(pe_poly *poly, const Plan &pl, uint64_t t0, uint64_t *out_dev, bool fused);
pe_status check_beta(const pe_poly *poly, const uint64_t *beta, BetaArg *arg);
// Frees a polynomial whose device work is known to have completed (no device synchronization).
void destroy_idle(pe_poly *poly);
// poly_eval_create with control over host threads (the server parallelizes across uploads instead).
// host_threads: split host passes over the host pool.  allow_device: inputs of
// at least 2^14 terms may be checked, grouped and packed by kernels on the
// device (two synchronizations) instead of on the host; callers whose GPU is
// held by long kernels (the server) keep the host path, which needs only copies.
pe_status create_poly(const pe_poly_desc *desc, pe_poly **out, bool host_threads, bool allow_device = true);
}  // namespace pe
