// C ABI of the plain path: create / groups / run / destroy, tile planning.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <numeric>
#include <memory>
#include <thread>
#include "internal.h"
#include "kernels.h"
#include "tune.h"

namespace pe {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

// poly_eval_debug_fail_alloc: the countdown reaches 1 at the allocation that fails.
static std::atomic<long> g_alloc_countdown{0};

bool alloc_fault_now()
{
    long c = g_alloc_countdown.load(std::memory_order_relaxed);
    while (c > 0 && !g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
    }
    return c == 1;
}

pe_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PE_ERR_NOMEM : PE_ERR_CUDA;
}

ModCtx make_modctx(uint64_t p)
{
    ModCtx m{};
    m.p = p;
    m.p2 = 2 * p;
    uint64_t inv = p;                           // p*p = 1 mod 8: three correct bits
    for (int i = 0; i < 5; ++i) inv *= 2 - p * inv;  // Newton-Hensel, doubling the bits
    m.pinv = inv;
    m.pinv_neg = 0 - inv;
    const unsigned __int128 R = (unsigned __int128)1 << 64;
    m.r1 = (uint64_t)(R % p);
    m.r2 = (uint64_t)(((unsigned __int128)m.r1 * m.r1) % p);
    m.w64q = (uint64_t)(((unsigned __int128)m.r1 << 64) / p);
    m.one_q = (uint64_t)(R / p);
    m.pd = (double)p;
    m.ud = 1.0 / (double)p;
    return m;
}

cudaStream_t alloc_stream()
{
    static std::mutex mu;
    static cudaStream_t streams[64] = {nullptr};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev]) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    }
    return streams[dev];
}

void destroy_idle(pe_poly *P) { delete P; }

// Page-locked staging buffers for uploads, reused across calls and threads.
namespace {
struct Staging {
    void *p = nullptr;
    size_t bytes = 0;
};
std::mutex g_stage_mu;
std::vector<Staging> g_stage_free;

// Best fit: the smallest cached buffer that holds n bytes, so uploads of mixed
// sizes on several threads reuse buffers instead of pinning new ones
// (page-locking is slow, and freeing page-locked memory waits for the device).
Staging stage_acquire(size_t n)
{
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        size_t best = g_stage_free.size();
        for (size_t i = 0; i < g_stage_free.size(); ++i)
            if (g_stage_free[i].bytes >= n && (best == g_stage_free.size() || g_stage_free[i].bytes < g_stage_free[best].bytes))
                best = i;
        if (best < g_stage_free.size()) {
            Staging s = g_stage_free[best];
            g_stage_free.erase(g_stage_free.begin() + best);
            return s;
        }
    }
    Staging s;
    const size_t want = std::max<size_t>(n + n / 4, 1 << 20);
    if (cudaMallocHost(&s.p, want) == cudaSuccess) s.bytes = want;
    else {
        cudaGetLastError();
        s.p = nullptr;
    }
    return s;
}

std::vector<cudaStream_t> g_up_streams;   // idle upload streams (same mutex)

// A non-blocking stream for one upload, from a pool (uploads on several host
// threads then proceed in parallel instead of queueing on one stream).
cudaStream_t upload_stream_acquire()
{
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        if (!g_up_streams.empty()) {
            cudaStream_t s = g_up_streams.back();
            g_up_streams.pop_back();
            return s;
        }
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return s;
}

void upload_stream_release(cudaStream_t s)
{
    if (!s) return;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    g_up_streams.push_back(s);
}

// Cached page-locked bytes are kept up to a cap; above it the smallest
// buffers are released first.
constexpr size_t kStageCacheBytes = 4ull << 30;

void stage_release(Staging s)
{
    if (!s.p) return;
    std::vector<Staging> drop;
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        g_stage_free.push_back(s);
        size_t total = 0;
        for (const Staging &x : g_stage_free) total += x.bytes;
        while (total > kStageCacheBytes && g_stage_free.size() > 1) {
            size_t small = 0;
            for (size_t i = 1; i < g_stage_free.size(); ++i)
                if (g_stage_free[i].bytes < g_stage_free[small].bytes) small = i;
            total -= g_stage_free[small].bytes;
            drop.push_back(g_stage_free[small]);
            g_stage_free.erase(g_stage_free.begin() + small);
        }
    }
    for (const Staging &x : drop) cudaFreeHost(x.p);
}
}  // namespace

// ----------------------------------------------------------- host pool
namespace {
struct HostPool {
    // A job is published with a new generation; workers that pick it up are
    // counted in `active`, and run() returns only when every index is done and
    // no worker is still inside the job, so no worker ever holds a finished job.
    std::mutex run_mu;                 // one parallel call at a time
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::vector<std::thread> threads;
    const std::function<void(unsigned)> *job = nullptr;
    unsigned n = 0, finished = 0, active = 0;
    std::atomic<unsigned> next{0};
    uint64_t gen = 0;
    bool stop = false;
    HostPool()
    {
        const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        for (unsigned t = 1; t < hw; ++t) threads.emplace_back([this] { work(); });
    }
    void drain(const std::function<void(unsigned)> &fn, unsigned count)
    {
        unsigned done = 0;
        for (unsigned i; (i = next.fetch_add(1)) < count;) {
            fn(i);
            ++done;
        }
        std::lock_guard<std::mutex> lk(mu);
        finished += done;
    }
    void work()
    {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return stop || gen != seen; });
            if (stop) return;
            seen = gen;
            if (!job) continue;
            const std::function<void(unsigned)> *f = job;
            const unsigned count = n;
            ++active;
            lk.unlock();
            drain(*f, count);
            lk.lock();
            --active;
            done_cv.notify_all();
        }
    }
    void run(unsigned count, const std::function<void(unsigned)> &fn)
    {
        std::lock_guard<std::mutex> rl(run_mu);
        {
            std::unique_lock<std::mutex> lk(mu);
            done_cv.wait(lk, [&] { return active == 0; });
            job = &fn;
            n = count;
            finished = 0;
            next.store(0);
            ++gen;
        }
        cv.notify_all();
        drain(fn, count);
        std::unique_lock<std::mutex> lk(mu);
        done_cv.wait(lk, [&] { return finished == count && active == 0; });
        job = nullptr;
    }
};
HostPool &host_pool()
{
    static HostPool *pool = new HostPool();   // never destroyed: workers may outlive static destructors
    return *pool;
}
}  // namespace

void host_parallel(unsigned n, const std::function<void(unsigned)> &fn)
{
    if (n <= 1) {
        if (n) fn(0);
        return;
    }
    host_pool().run(n, fn);
}

unsigned host_pool_size() { return (unsigned)host_pool().threads.size() + 1; }

static constexpr int kMaxDevices = 64;

int num_sms()
{
    static std::atomic<int> cached[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

cudaError_t smem_limit_once(const void *func, int bytes)
{
    // (function, device) pairs already raised; a concurrent first call raises it twice, which is harmless
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> g(mu);
        for (const auto &d : done)
            if (d.first == func && d.second == dev) return cudaSuccess;
    }
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    done.emplace_back(func, dev);
    return cudaSuccess;
}

bool plan_start_gaps(StartRows *sr)
{
    sr->ngap = 0;
    sr->gap_hb = 0;
    for (int j = 0; j < kMaxGaps; ++j) sr->gap[j] = 0;   // unused entries have no bits
    uint32_t bits = 0;
    for (uint32_t k = 1; k < sr->n; ++k) {
        const uint32_t g = sr->row[k] - sr->row[k - 1];
        if (g == 0) return false;                   // rows must increase
        uint32_t j = 0;
        while (j < sr->ngap && sr->gap[j] != g) ++j;
        if (j == sr->ngap) {
            if (sr->ngap == (uint32_t)kMaxGaps) return false;
            sr->gap[sr->ngap++] = g;
        }
        sr->gidx[k] = (uint8_t)j;
        bits |= g;
    }
    while (bits >> (sr->gap_hb + 1)) ++sr->gap_hb;
    return true;
}

bool out_ok(uint64_t T, uint64_t G)
{
    if (G && T > (1ull << 60) / G) {
        set_error("the output of %llu x %llu values is above 2^60", (unsigned long long)T, (unsigned long long)G);
        return false;
    }
    return true;
}

bool points_ok(uint64_t T, uint64_t t0)
{
    if (T > (1ull << 31)) {
        set_error("T above 2^31");
        return false;
    }
    if (T && t0 > ~0ull - (T - 1)) {
        set_error("the last point t0 + T - 1 is above 2^64 - 1");
        return false;
    }
    return true;
}

pe_status check_beta(const pe_poly *poly, const uint64_t *beta, BetaArg *arg)
{
    memset(arg, 0, sizeof *arg);
    if (poly->E == 0) return PE_OK;
    if (!beta) {
        set_error("beta is NULL");
        return PE_ERR_ARG;
    }
    for (uint32_t j = 0; j < poly->E; ++j) {
        if (beta[j] == 0 || beta[j] >= poly->p) {
            set_error("beta[%u] = %llu is not in [1, p)", j, (unsigned long long)beta[j]);
            return PE_ERR_ARG;
        }
        arg->b[j] = beta[j];
    }
    return PE_OK;
}

static uint64_t count_chunks(const pe_poly *P, uint32_t K)
{
    uint64_t nc = 0;
    for (uint64_t g = 0; g < P->G; ++g) nc += (P->group_off[g + 1] - P->group_off[g] + K - 1) / K;
    return nc;
}

// Tail band shape for `tail` final points: one-slab items of at most 64 points.
static uint32_t tail_tc(uint64_t tail) { return (uint32_t)std::min<uint64_t>(tail, 64); }

// Tile shape.  Items are issued in order and each warp takes the next, so the
// run ends unevenly by about one item; measured on GB300, items of about 2% of
// a warp's share of the work (at least 128 slab-points, at most 512 points)
// balance that against the fixed cost of starting an item.  Small jobs use
// smaller items so that every warp gets one.
Tiles choose_tiles(pe_poly *P, uint64_t T, const pe_tiles *f)
{
    Tiles t;
    const TuneEntry *te = tune_lookup(P, T);
    t.wpb = (f && f->warps_per_block) ? f->warps_per_block : (te ? te->wpb : 4);
    t.wpb = std::min<uint32_t>(t.wpb, kMaxStepBWarps);
    if (f && f->K) {
        t.K = f->K;
    } else if (te) {
        t.K = te->K;
    } else {
        // Padded slots plus the per-chunk cost: a chunk costs K products+sums
        // and, per point, its partial's store and walk entry, about 1.2 of a
        // 64-bit product+sum and 2.4 of a 32-bit one (measured on GB300: K=16
        // with 168 registers and 12 warps per SM beats K=8 with 20 warps).
        const bool narrow = P->variant == PE_MODMUL_BARRETT32;
        const double walk = narrow ? 2.4 : 1.2;
        double best = 1e300;
        for (uint32_t K : {1u, 2u, 4u, 8u, 12u, 16u}) {
            const double nc = (double)count_chunks(P, K);
            const double c = nc * (K + walk);
            if (c < best * 0.98) {
                best = c;
                t.K = K;
            }
        }
    }
    if (f && f->slabs && f->tchunk) {
        t.kslabs = f->slabs;
        t.tailT = f->tail && f->tail < T ? f->tail : 0;
        t.Tc = (uint32_t)std::min<uint64_t>(f->tchunk, T - t.tailT);
        return t;
    }
    if (te && te->kslabs && te->Tc && !(f && (f->slabs || f->tchunk || f->K))) {   // measured shape
        t.kslabs = te->kslabs;
        t.tailT = te->tail && te->tail + 32 <= T ? te->tail : 0;
        t.Tc = (uint32_t)std::min<uint64_t>(te->Tc, T - t.tailT);
        const uint64_t q0 = (T - t.tailT + t.Tc - 1) / t.Tc, q1 = t.tailT ? (t.tailT + 63) / 64 : 0;
        if (q0 + q1 <= (uint64_t)kMaxStarts) return t;
        t.tailT = 0;   // too many start rows for this T: fall through to the rule
    }
    const uint64_t NC = count_chunks(P, t.K);
    int bps = 0;
    if (stepB_occupancy((int)t.K, P->variant, (int)t.wpb, &bps) != cudaSuccess || bps <= 0) bps = 1;
    const uint64_t R = (uint64_t)bps * t.wpb * num_sms();
    const uint64_t slabs = std::max<uint64_t>(1, (NC + 31) / 32);
    // Start rows are limited by kMaxStarts and by 1 GB of starting values.
    const uint64_t lmax = std::max<uint64_t>(
        1, std::min<uint64_t>(kMaxStarts, (1ull << 30) / (8 * std::max<uint64_t>(P->s, 1))));
    const double per_warp = (double)slabs * (double)T / (double)R;
    double target = std::max(128.0, 0.02 * per_warp);                 // slab-points per item
    if ((double)slabs * (double)T < target * (double)R)               // small job: one item per warp
        target = std::max(32.0, (double)slabs * (double)T / (double)R);
    uint64_t Tc = f && f->tchunk ? f->tchunk : (uint64_t)std::min<double>(512.0, target);
    Tc = std::max<uint64_t>(1, std::min<uint64_t>(Tc, T));
    Tc = std::max<uint64_t>(Tc, (T + lmax - 1) / lmax);               // start-row limit
    uint64_t k = f && f->slabs ? f->slabs : (uint64_t)std::max(1.0, std::floor(target / (double)Tc));
    k = std::max<uint64_t>(1, std::min<uint64_t>(k, slabs));
    t.kslabs = (uint32_t)k;
    t.Tc = (uint32_t)Tc;
    t.tailT = 0;
    // Few items per warp: the run would end unevenly by a sizeable fraction.
    // Reserve the last ~T/8 points for a band of one-slab, 64-point items that
    // run after the others (their starting values are precomputed, so they are
    // cheap), and make the other items twice as long.
    const double items = (double)((slabs + k - 1) / k) * (double)((T + Tc - 1) / Tc);
    if (!(f && (f->slabs || f->tchunk)) && T >= 512 && items / (double)R < 24.0) {
        const uint64_t tail = std::min<uint64_t>(256, std::max<uint64_t>(64, (T / 8 + 32) / 64 * 64));
        const uint64_t T0 = T - tail;
        uint64_t q0 = (T0 + std::min<uint64_t>(512, 2 * Tc) - 1) / std::min<uint64_t>(512, 2 * Tc);
        const uint64_t q1 = (tail + tail_tc(tail) - 1) / tail_tc(tail);
        q0 = std::max<uint64_t>(1, std::min<uint64_t>(q0, lmax > q1 ? lmax - q1 : 1));
        if (q0 + q1 <= lmax) {
            t.Tc = (uint32_t)((T0 + q0 - 1) / q0);
            t.tailT = (uint32_t)tail;
        }
    }
    return t;
}

void build_gfirst(pe_poly *P, uint32_t K)
{
    HostChunks &h = P->chunks;
    if (h.K == K && h.gfirst.size() == P->G + 1) return;
    h.K = K;
    h.cs.clear();
    h.cg.clear();
    h.gfirst.resize(P->G + 1);
    uint64_t nc = 0;
    for (uint64_t g = 0; g < P->G; ++g) {
        h.gfirst[g] = (uint32_t)nc;
        nc += (P->group_off[g + 1] - P->group_off[g] + K - 1) / K;
    }
    h.gfirst[P->G] = (uint32_t)nc;
    h.NC = (uint32_t)nc;
}

void build_chunks(pe_poly *P, uint32_t K)
{
    build_gfirst(P, K);
    HostChunks &h = P->chunks;
    if (h.cs.size() == (size_t)h.NC + 1) return;
    const uint64_t nc = h.NC;
    h.cs.resize(nc + 1);
    h.cg.resize(nc);
    uint32_t *cs = h.cs.data(), *cg = h.cg.data();
    const unsigned nth = nc >= (1u << 15) ? 2 * host_pool_size() : 1u;
    const std::function<void(unsigned)> fill = [&](unsigned t) {
        for (uint64_t g = P->G * t / nth; g < P->G * (t + 1) / nth; ++g) {
            uint64_t c = h.gfirst[g];
            for (uint64_t st = P->group_off[g]; st < P->group_off[g + 1]; st += K, ++c) {
                cs[c] = (uint32_t)st;
                cg[c] = (uint32_t)g;
            }
        }
    };
    host_parallel(nth, fill);
    cs[nc] = (uint32_t)P->s;
}

void build_plan_host(pe_poly *P, const Tiles &t, uint64_t T, PlanHost &ph)
{
    build_gfirst(P, t.K);
    const HostChunks &h = P->chunks;
    ph.K = t.K;
    ph.kslabs = t.kslabs;
    ph.Tc = t.Tc;
    ph.wpb = t.wpb;
    ph.T = T;
    ph.NC = h.NC;
    const uint32_t per_unit = 32u * t.kslabs;
    ph.U = (ph.NC + per_unit - 1) / per_unit;
    ph.Q = (uint32_t)((T + t.Tc - 1) / t.Tc);
    ph.unit.assign(4 * (size_t)ph.U, -1);   // lslot, rslot, lspan, rspan
    std::vector<uint32_t> sg, sbase, sn;
    uint32_t nslots = 0;
    for (uint64_t g = 0; g < P->G; ++g) {
        const uint32_t ua = h.gfirst[g] / per_unit, ub = (h.gfirst[g + 1] - 1) / per_unit;
        if (ub == ua) continue;
        const int32_t sp = (int32_t)sg.size();
        sg.push_back((uint32_t)g);
        sbase.push_back(nslots);
        sn.push_back(ub - ua + 1);
        ph.unit[1 * (size_t)ph.U + ua] = (int32_t)nslots;
        ph.unit[3 * (size_t)ph.U + ua] = sp;
        for (uint32_t u = ua + 1; u <= ub; ++u) {
            ph.unit[0 * (size_t)ph.U + u] = (int32_t)(nslots + (u - ua));
            ph.unit[2 * (size_t)ph.U + u] = sp;
        }
        nslots += ub - ua + 1;
    }
    ph.S = (uint32_t)sg.size();
    ph.nslots = nslots;
    ph.span.assign(3 * (size_t)std::max<uint32_t>(ph.S, 1), 0);
    for (uint32_t i = 0; i < ph.S; ++i) {
        ph.span[i] = sg[i];
        ph.span[ph.S + i] = sbase[i];
        ph.span[2 * (size_t)ph.S + i] = sn[i];
    }
}

size_t PlanHost::counter_bytes() const { return (size_t)std::max<uint32_t>(S, 1) * Q * 4; }
size_t PlanHost::carry_bytes() const { return nslots ? (size_t)nslots * T * 16 : 16; }
size_t PlanHost::chain_bytes() const { return kslabs > 1 ? (size_t)U * Q * Tc * 16 : 16; }

void fill_job(StepBJob &J, pe_poly *P, const PlanHost &ph, const uint32_t *cs, const uint32_t *cg,
              const int32_t *unit, const uint32_t *span, uint32_t *counters, ulonglong2 *carry, ulonglong2 *chain,
              uint64_t t0, uint64_t *out_dev, const uint64_t *mR, const uint64_t *ptab, int variant)
{
    J = StepBJob{};
    J.coeffs = P->coeffs.as<uint64_t>();
    J.mR = mR;
    J.exps = P->exps->p;
    J.ptab = ptab;
    J.cs = cs;
    J.cg = cg;
    J.u_lslot = unit;
    J.u_rslot = unit + ph.U;
    J.u_lspan = unit + 2 * (size_t)ph.U;
    J.u_rspan = unit + 3 * (size_t)ph.U;
    const uint32_t S = std::max<uint32_t>(ph.S, 1);
    J.span_g = span;
    J.span_base = span + S;
    J.span_n = span + 2 * (size_t)S;
    J.counters = counters;
    J.carry = carry;
    J.chain = chain;
    J.out = out_dev;
    J.s = P->s;
    J.T = ph.T;
    J.t0 = t0;
    J.G = P->G;
    J.NC = ph.NC;
    J.U = ph.U;
    J.Q = ph.Q;
    J.kslabs = ph.kslabs;
    J.Tc = ph.Tc;
    J.E = P->E;
    J.dp1 = P->dmax + 1;
    J.exp_bytes = P->exp_bytes;
    J.K = ph.K;
    J.var = (uint32_t)variant;
    J.mc = P->mc;
}

pe_status ensure_plan(pe_poly *P, Plan &pl, const Tiles &t, uint64_t T, cudaStream_t st, bool queued)
{
    if (pl.valid && pl.K == t.K && pl.kslabs == t.kslabs && pl.Tc == t.Tc && pl.T == T && pl.wpb == t.wpb)
        return PE_OK;
    pl.valid = false;
    PlanHost &ph = pl.host;
    build_plan_host(P, t, T, ph);
    const HostChunks &h = P->chunks;
    cudaError_t e;
    // Synchronous plans are built on the library stream and waited for.
    cudaStream_t ks = queued ? st : alloc_stream();
    auto alloc = [&](DevBuf &b, size_t n) { return b.ensure_async(n, ks); };
    if ((e = alloc(pl.cs, ((size_t)ph.NC + 1) * 4)) != cudaSuccess || (e = alloc(pl.cg, std::max<size_t>(ph.NC, 1) * 4)) != cudaSuccess ||
        (e = alloc(pl.gfirst, h.gfirst.size() * 4)) != cudaSuccess ||
        (e = alloc(pl.unit, ph.unit.size() * 4)) != cudaSuccess || (e = alloc(pl.span, ph.span.size() * 4)) != cudaSuccess ||
        (e = alloc(pl.counters, ph.counter_bytes())) != cudaSuccess)
        return cuda_fail(e, "plan alloc");
    if ((e = alloc(pl.carry, ph.carry_bytes())) != cudaSuccess) return cuda_fail(e, "carry alloc");
    if ((e = alloc(pl.chain, ph.chain_bytes())) != cudaSuccess) return cuda_fail(e, "chain alloc");
    if (!P->goff_dev.p) {   // the group offsets, once per handle
        std::vector<uint32_t> go(P->group_off.begin(), P->group_off.end());
        if ((e = P->goff_dev.ensure_async(go.size() * 4, ks)) != cudaSuccess ||
            (e = cudaMemcpyAsync(P->goff_dev.p, go.data(), go.size() * 4, cudaMemcpyHostToDevice, ks)) != cudaSuccess)
            return cuda_fail(e, "group offsets");
    }
    // Pageable sources are staged by the driver before these calls return.
    if ((e = cudaMemcpyAsync(pl.gfirst.p, h.gfirst.data(), h.gfirst.size() * 4, cudaMemcpyHostToDevice, ks)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pl.unit.p, ph.unit.data(), ph.unit.size() * 4, cudaMemcpyHostToDevice, ks)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pl.span.p, ph.span.data(), ph.span.size() * 4, cudaMemcpyHostToDevice, ks)) != cudaSuccess ||
        (e = cudaMemsetAsync(pl.counters.p, 0, pl.counters.bytes, ks)) != cudaSuccess ||
        (e = launch_chunk_tables(P->goff_dev.as<uint32_t>(), pl.gfirst.as<uint32_t>(), P->G, ph.K, P->s, ph.NC,
                                 pl.cs.as<uint32_t>(), pl.cg.as<uint32_t>(), ks)) != cudaSuccess)
        return cuda_fail(e, "plan upload");
    if (!queued && (e = cudaStreamSynchronize(ks)) != cudaSuccess) return cuda_fail(e, "plan upload");
    pl.K = t.K;
    pl.kslabs = t.kslabs;
    pl.Tc = t.Tc;
    pl.wpb = t.wpb;
    pl.T = T;
    pl.NC = ph.NC;
    pl.U = ph.U;
    pl.Q = ph.Q;
    pl.S = ph.S;
    pl.nslots = ph.nslots;
    pl.valid = true;
    return PE_OK;
}

StepBJob make_job(pe_poly *P, const Plan &pl, uint64_t t0, uint64_t *out_dev, bool fused)
{
    StepBJob J;
    fill_job(J, P, pl.host, pl.cs.as<uint32_t>(), pl.cg.as<uint32_t>(), pl.unit.as<int32_t>(),
             pl.span.as<uint32_t>(), pl.counters.as<uint32_t>(), pl.carry.as<ulonglong2>(),
             pl.chain.as<ulonglong2>(), t0, out_dev, fused ? nullptr : P->mR.as<uint64_t>(),
             P->ptab.as<uint64_t>(), P->variant);
    return J;
}

static inline uint32_t read_exp(const void *exps, uint32_t width, uint64_t idx)
{
    switch (width) {
    case 1: return ((const uint8_t *)exps)[idx];
    case 2: return ((const uint16_t *)exps)[idx];
    default: return ((const uint32_t *)exps)[idx];
    }
}

static pe_status check_prime(uint64_t p, int variant)
{
    if (p < 3 || (p & 1) == 0) {
        set_error("p = %llu must be odd and at least 3", (unsigned long long)p);
        return PE_ERR_PRIME;
    }
    if (p >= (1ull << 62)) {
        set_error("p must be below 2^62");
        return PE_ERR_PRIME;
    }
    if (variant == PE_MODMUL_FP64 && p >= (1ull << 50)) {
        set_error("the FP64 modular product (Algorithm 2) needs p < 2^50");
        return PE_ERR_PRIME;
    }
    if (variant == PE_MODMUL_BARRETT32 && p >= (1ull << 30)) {
        set_error("the 32-bit Barrett product needs p < 2^30");
        return PE_ERR_PRIME;
    }
    return PE_OK;
}

// Terms already in group order are checked, grouped and packed on the device
// (create.cu): the host only copies the raw arrays into page-locked staging
// (several threads) and reads back the flags and the group table.  Sets
// *fallback, and does nothing else, when the terms are not in group order or
// staging memory is unavailable; the host path then handles them.
static constexpr uint64_t kDeviceCreateMin = 1u << 14;
static constexpr uint64_t kEarlyGroups = 1u << 14;   // group-table entries fetched with the first wait

static pe_status create_poly_device(const pe_poly_desc *d, int variant, pe_poly **out, bool host_threads,
                                    bool *fallback)
{
    *fallback = false;
    const uint64_t s = d->s;
    const uint32_t n = d->n, w = d->exp_bytes, E = n - 2;
    const size_t cbytes = s * 8, ebytes = (size_t)s * n * w;
    const bool dev_in = (d->flags & PE_FLAG_DEVICE_PTRS) != 0;
    const uint64_t nb = (s + 1023) / 1024;
    std::unique_ptr<pe_poly> P(new pe_poly());
    DevBuf raw, keys, counts, base, goff, gkeys, info;
    Staging stg{};
    cudaStream_t us = upload_stream_acquire();
    auto finish = [&]() {   // waits for queued work before the scratch is freed
        cudaStreamSynchronize(us);
        upload_stream_release(us);
        stage_release(stg);
    };
    cudaError_t e;
    if ((e = P->coeffs.ensure_async(cbytes, us)) != cudaSuccess ||
        (!dev_in && (e = raw.ensure_async(ebytes, us)) != cudaSuccess) ||
        (e = keys.ensure_async(s * 8, us)) != cudaSuccess || (e = counts.ensure_async(nb * 8, us)) != cudaSuccess ||
        (e = base.ensure_async((nb + 1) * 8, us)) != cudaSuccess || (e = goff.ensure_async(s * 8, us)) != cudaSuccess ||
        (e = gkeys.ensure_async(s * 8, us)) != cudaSuccess ||
        (e = info.ensure_async(sizeof(CreateInfo), us)) != cudaSuccess ||
        (e = P->mR.ensure_async(s * 8, us)) != cudaSuccess) {
        finish();
        return cuda_fail(e, "device allocation");
    }
    const void *dexps = d->exps;
    auto page_locked = [](const void *p) {
        cudaPointerAttributes a{};
        const bool yes = cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost;
        cudaGetLastError();
        return yes;
    };
    if (!dev_in && page_locked(d->coeffs) && page_locked(d->exps)) {
        // Page-locked caller arrays are read by the copy engine directly (the
        // caller keeps them unchanged until create returns, which waits for it).
        if ((e = cudaMemcpyAsync(P->coeffs.p, d->coeffs, cbytes, cudaMemcpyHostToDevice, us)) != cudaSuccess ||
            (e = cudaMemcpyAsync(raw.p, d->exps, ebytes, cudaMemcpyHostToDevice, us)) != cudaSuccess) {
            finish();
            return cuda_fail(e, "uploading terms");
        }
        dexps = raw.p;
    } else if (!dev_in) {
        stg = stage_acquire(cbytes + ebytes);
        if (!stg.p) {
            finish();
            *fallback = true;
            return PE_OK;
        }
        unsigned char *dst = (unsigned char *)stg.p;
        const unsigned nth = host_threads ? 2 * host_pool_size() : 1u;
        const std::function<void(unsigned)> copy = [&](unsigned t) {
            const size_t c0 = cbytes * t / nth, c1 = cbytes * (t + 1) / nth;
            const size_t e0 = ebytes * t / nth, e1 = ebytes * (t + 1) / nth;
            memcpy(dst + c0, (const unsigned char *)d->coeffs + c0, c1 - c0);
            memcpy(dst + cbytes + e0, (const unsigned char *)d->exps + e0, e1 - e0);
        };
        host_parallel(nth, copy);
        if ((e = cudaMemcpyAsync(P->coeffs.p, dst, cbytes, cudaMemcpyHostToDevice, us)) != cudaSuccess ||
            (e = cudaMemcpyAsync(raw.p, dst + cbytes, ebytes, cudaMemcpyHostToDevice, us)) != cudaSuccess) {
            finish();
            return cuda_fail(e, "uploading terms");
        }
        dexps = raw.p;
    } else if ((e = cudaMemcpyAsync(P->coeffs.p, d->coeffs, cbytes, cudaMemcpyDeviceToDevice, us)) != cudaSuccess) {
        finish();
        return cuda_fail(e, "copying terms");
    }
    CreateInfo ci{};
    uint64_t G = 0;
    // With byte exponents the packed rows are bytes whatever the scan finds, so
    // the packing and a bounded copy of the group table are queued before the
    // first wait: a polynomial of at most kEarlyGroups groups needs one wait.
    const bool early = w == 1 && E > 0;
    const uint64_t early_groups = std::min<uint64_t>(s, kEarlyGroups);
    Staging gst{};
    if (early) {
        gst = stage_acquire(early_groups * 16);
        if ((e = P->exps->ensure_async((size_t)E * s, us)) != cudaSuccess) {
            finish();
            stage_release(gst);
            return cuda_fail(e, "device allocation");
        }
    }
    if ((e = cudaMemsetAsync(info.p, 0, sizeof(CreateInfo), us)) != cudaSuccess ||
        (e = cudaMemsetAsync(info.p, 0xff, sizeof(unsigned long long), us)) != cudaSuccess ||
        (e = launch_term_scan(P->coeffs.as<uint64_t>(), dexps, w, s, n, d->p, keys.as<uint64_t>(),
                              info.as<CreateInfo>(), counts.as<uint64_t>(), base.as<uint64_t>(), goff.as<uint64_t>(),
                              gkeys.as<uint32_t>(), us)) != cudaSuccess ||
        (early && (e = launch_pack_exps(dexps, 1, s, n, 1, P->exps->p, us)) != cudaSuccess) ||
        (early && gst.p &&
         ((e = cudaMemcpyAsync(gst.p, goff.p, early_groups * 8, cudaMemcpyDeviceToHost, us)) != cudaSuccess ||
          (e = cudaMemcpyAsync((unsigned char *)gst.p + early_groups * 8, gkeys.p, early_groups * 8,
                               cudaMemcpyDeviceToHost, us)) != cudaSuccess)) ||
        (e = cudaMemcpyAsync(&ci, info.p, sizeof ci, cudaMemcpyDeviceToHost, us)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&G, base.as<uint64_t>() + nb, 8, cudaMemcpyDeviceToHost, us)) != cudaSuccess ||
        (e = cudaStreamSynchronize(us)) != cudaSuccess) {
        finish();
        stage_release(gst);
        return cuda_fail(e, "scanning terms");
    }
    struct StageGuard {
        Staging &g;
        ~StageGuard() { stage_release(g); }
    } guard{gst};
    if (ci.bad != ~0ull) {
        uint64_t v = 0;
        if (dev_in)
            cudaMemcpy(&v, d->coeffs + ci.bad, 8, cudaMemcpyDeviceToHost);
        else
            v = d->coeffs[ci.bad];
        finish();
        set_error("coefficient %llu of term %llu is not reduced mod p", (unsigned long long)v, ci.bad);
        return PE_ERR_NOT_REDUCED;
    }
    if (ci.unsorted) {
        finish();
        *fallback = true;
        return PE_OK;
    }
    if (ci.dmax > 0xffff) {
        finish();
        set_error("exponent %u above 65535", ci.dmax);
        return PE_ERR_EXP_RANGE;
    }
    P->p = d->p;
    P->n = n;
    P->E = E;
    P->s = s;
    P->requested_variant = variant;
    P->variant = variant == PE_MODMUL_AUTO ? default_variant(d->p) : variant;
    P->mc = make_modctx(d->p);
    P->dmax = ci.dmax;
    P->exp_bytes = ci.dmax <= 0xff ? 1 : 2;
    P->G = G;
    P->group_off.resize(G + 1);
    P->keys.resize(2 * G);
    const size_t dp1 = ci.dmax + 1;
    if ((e = P->ptab.ensure_async((size_t)E * dp1 * 8, us)) != cudaSuccess) {
        finish();
        return cuda_fail(e, "device allocation");
    }
    if (early && gst.p && G <= early_groups) {   // everything arrived with the first wait
        memcpy(P->group_off.data(), gst.p, G * 8);
        memcpy(P->keys.data(), (const unsigned char *)gst.p + early_groups * 8, G * 8);
    } else if ((!early && (e = P->exps->ensure_async((size_t)E * s * P->exp_bytes, us)) != cudaSuccess) ||
               (e = cudaMemcpyAsync(P->group_off.data(), goff.p, G * 8, cudaMemcpyDeviceToHost, us)) != cudaSuccess ||
               (e = cudaMemcpyAsync(P->keys.data(), gkeys.p, 2 * G * 4, cudaMemcpyDeviceToHost, us)) != cudaSuccess ||
               (!early && (e = launch_pack_exps(dexps, w, s, n, P->exp_bytes, P->exps->p, us)) != cudaSuccess) ||
               (e = cudaStreamSynchronize(us)) != cudaSuccess) {
        finish();
        return cuda_fail(e, "packing terms");
    }
    P->group_off[G] = s;
    finish();
    *out = P.release();
    return PE_OK;
}

}  // namespace pe

using namespace pe;

extern "C" const char *poly_eval_last_error(void) { return g_err.c_str(); }

extern "C" pe_status poly_eval_debug_fail_alloc(uint32_t nth)
{
    g_alloc_countdown.store((long)nth);
    return PE_OK;
}

extern "C" pe_status poly_eval_create(const pe_poly_desc *d, pe_poly **out) { return create_poly(d, out, true); }

namespace {
// One host pass over terms i0..i1: the first coefficient not below p, the
// largest evaluated exponent, each term's (d, e) key, and whether the keys of
// the range are in descending order (the boundary with the previous range is
// checked by the caller).
struct ScanOut {
    uint32_t dmax = 0;
    uint64_t bad = ~0ull;
    char sorted = 1;
};

template <typename ExpT>
void scan_terms(const ExpT *exps, const uint64_t *coeffs, uint32_t n, uint64_t p, uint64_t i0, uint64_t i1,
                uint64_t *key, ScanOut &o)
{
    uint32_t dm = 0;
    uint64_t bad = ~0ull, prev = ~0ull;
    char srt = 1;
    for (uint64_t i = i0; i < i1; ++i) {
        const ExpT *e = exps + i * n;
        if (coeffs[i] >= p && bad == ~0ull) bad = i;
        const uint64_t k = ((uint64_t)e[0] << 32) | (uint64_t)e[1];
        key[i] = k;
        srt &= (char)(k <= prev);
        prev = k;
        for (uint32_t j = 2; j < n; ++j) dm = std::max<uint32_t>(dm, e[j]);
    }
    o.dmax = dm;
    o.bad = bad;
    o.sorted = srt;
}

// Structure-of-arrays packing of terms i0..i1 in group order (perm: the
// source term of each position, or NULL when the input is already in order).
template <typename ExpT, typename OutT>
void pack_terms(const ExpT *exps, const uint64_t *coeffs, const uint32_t *perm, uint32_t n, uint64_t s,
                uint64_t i0, uint64_t i1, uint64_t *sc, OutT *se)
{
    const uint32_t E = n - 2;
    for (uint64_t i = i0; i < i1; ++i) {
        const uint64_t o = perm ? perm[i] : i;
        sc[i] = coeffs[o];
        const ExpT *e = exps + o * n + 2;
        for (uint32_t j = 0; j < E; ++j) se[(size_t)j * s + i] = (OutT)e[j];
    }
}
}  // namespace

// Allocates a new handle's device arrays and uploads its packed terms
// (coefficients, then E rows of exponents) from `stage`: the allocations and
// both copies are queued on one upload stream and waited for once.  Releases
// the staging buffer; deletes P on failure.
static pe_status upload_packed(pe_poly *P, Staging stg, const unsigned char *stage, size_t se_bytes)
{
    const uint64_t s = P->s;
    const size_t dp1 = P->dmax + 1;
    cudaStream_t us = upload_stream_acquire();
    cudaError_t e;
    if ((e = P->coeffs.ensure_async(s * 8, us)) != cudaSuccess || (e = P->exps->ensure_async(se_bytes, us)) != cudaSuccess ||
        (e = P->mR.ensure_async(s * 8, us)) != cudaSuccess ||
        (e = P->ptab.ensure_async((size_t)P->E * dp1 * 8, us)) != cudaSuccess) {
        cudaStreamSynchronize(us);
        upload_stream_release(us);
        stage_release(stg);
        delete P;
        return cuda_fail(e, "device allocation");
    }
    if ((s && (e = cudaMemcpyAsync(P->coeffs.p, stage, s * 8, cudaMemcpyHostToDevice, us)) != cudaSuccess) ||
        (se_bytes && (e = cudaMemcpyAsync(P->exps->p, stage + s * 8, se_bytes, cudaMemcpyHostToDevice, us)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(us)) != cudaSuccess) {
        cudaStreamSynchronize(us);
        upload_stream_release(us);
        stage_release(stg);
        delete P;
        return cuda_fail(e, "uploading terms");
    }
    upload_stream_release(us);
    stage_release(stg);
    return PE_OK;
}

namespace {
// One pass over terms with byte exponents that are already in group order
// (descending (d, e)): checks the coefficients, records the groups and packs
// coefficients and exponent rows into staging.  Returns false as soon as a
// key rises (the input is not in group order; the caller sorts instead).
bool scan_pack_sorted_u8(const uint64_t *coeffs, const uint8_t *exps, uint32_t n, uint64_t s, uint64_t p,
                         uint64_t *sc, uint8_t *se, std::vector<uint64_t> &goff, std::vector<uint32_t> &keys,
                         uint32_t &dmax, uint64_t &bad)
{
    const uint32_t E = n - 2;
    uint64_t prev = ~0ull;
    uint32_t dm = 0;
    bad = ~0ull;
    goff.assign(1, 0);
    keys.clear();
    for (uint64_t i = 0; i < s; ++i) {
        const uint8_t *e = exps + i * n;
        const uint64_t c = coeffs[i];
        if (c >= p && bad == ~0ull) bad = i;
        sc[i] = c;
        const uint64_t k = ((uint64_t)e[0] << 32) | (uint64_t)e[1];
        if (k != prev) {
            if (i && k > prev) return false;
            if (i) goff.push_back(i);
            keys.push_back(e[0]);
            keys.push_back(e[1]);
            prev = k;
        }
        for (uint32_t j = 0; j < E; ++j) {
            const uint8_t x = e[2 + j];
            dm = std::max<uint32_t>(dm, x);
            se[(size_t)j * s + i] = x;
        }
    }
    goff.push_back(s);
    dmax = dm;
    return true;
}
}  // namespace

pe_status pe::create_poly(const pe_poly_desc *d, pe_poly **out, bool host_threads, bool allow_device)
{
    if (!out) {
        set_error("out is NULL");
        return PE_ERR_ARG;
    }
    *out = nullptr;
    if (!d) {
        set_error("desc is NULL");
        return PE_ERR_ARG;
    }
    if (d->n < 2 || d->n > PE_MAX_VARS) {
        set_error("n = %u is outside [2, %d]", d->n, PE_MAX_VARS);
        return PE_ERR_ARG;
    }
    if (d->exp_bytes != 1 && d->exp_bytes != 2 && d->exp_bytes != 4) {
        set_error("exp_bytes must be 1, 2 or 4");
        return PE_ERR_ARG;
    }
    if (d->s >= 0xffffffffull) {
        set_error("at most 2^32-2 terms");
        return PE_ERR_ARG;
    }
    if (d->s && (!d->coeffs || !d->exps)) {
        set_error("coeffs or exps is NULL");
        return PE_ERR_ARG;
    }
    int variant = d->variant;
    if (variant != PE_MODMUL_AUTO && variant != PE_MODMUL_MONT64 && variant != PE_MODMUL_FP64 &&
        variant != PE_MODMUL_BARRETT64 && variant != PE_MODMUL_BARRETT32) {
        set_error("unknown variant %d", (int)d->variant);
        return PE_ERR_ARG;
    }
    pe_status st = check_prime(d->p, variant);
    if (st != PE_OK) return st;
    if (allow_device && d->s >= kDeviceCreateMin) {
        bool fallback = false;
        st = create_poly_device(d, variant, out, host_threads, &fallback);
        if (!fallback) return st;
    }

    const uint64_t s = d->s;
    const uint32_t n = d->n, E = n - 2, w = d->exp_bytes;
    // Host views of the terms (device inputs are staged through the host).
    std::vector<uint64_t> hc;
    std::vector<uint8_t> he;
    const uint64_t *coeffs = d->coeffs;
    const void *exps = d->exps;
    if ((d->flags & PE_FLAG_DEVICE_PTRS) && s) {
        hc.resize(s);
        he.resize(s * n * w);
        cudaError_t e;
        if ((e = cudaMemcpy(hc.data(), d->coeffs, s * 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(he.data(), d->exps, s * n * w, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "reading device terms");
        coeffs = hc.data();
        exps = he.data();
    }
    // One pass (split over host threads for large inputs): reduced
    // coefficients, the largest evaluated exponent, (d, e) keys, sortedness.
    std::unique_ptr<uint64_t[]> key_buf(new uint64_t[std::max<uint64_t>(s, 1)]);   // not zero-filled
    uint64_t *key = key_buf.get();
    const unsigned nth = host_threads && s >= (1u << 18)
                             ? std::max(1u, std::min(8u, std::thread::hardware_concurrency())) : 1u;
    if (w == 1 && nth == 1 && s && n > 2) {
        // Byte exponents in group order (the usual input): one pass.
        Staging stg = stage_acquire(s * 8 + (size_t)(n - 2) * s);
        if (stg.p) {
            unsigned char *stage = (unsigned char *)stg.p;
            std::vector<uint64_t> goff;
            std::vector<uint32_t> gkeys;
            uint32_t dm = 0;
            uint64_t bad = ~0ull;
            if (scan_pack_sorted_u8(coeffs, (const uint8_t *)exps, n, s, d->p, (uint64_t *)stage, stage + s * 8, goff,
                                    gkeys, dm, bad)) {
                if (bad != ~0ull) {
                    stage_release(stg);
                    set_error("coefficient %llu of term %llu is not reduced mod p", (unsigned long long)coeffs[bad],
                              (unsigned long long)bad);
                    return PE_ERR_NOT_REDUCED;
                }
                pe_poly *P = new pe_poly();
                P->p = d->p;
                P->n = n;
                P->E = E;
                P->s = s;
                P->requested_variant = variant;
                P->variant = variant == PE_MODMUL_AUTO ? default_variant(d->p) : variant;
                P->mc = make_modctx(d->p);
                P->dmax = dm;
                P->exp_bytes = 1;
                P->group_off = std::move(goff);
                P->keys = std::move(gkeys);
                P->G = P->keys.size() / 2;
                const pe_status ust = upload_packed(P, stg, stage, (size_t)E * s);
                if (ust != PE_OK) return ust;
                *out = P;
                return PE_OK;
            }
            stage_release(stg);
        }
    }
    std::vector<uint32_t> t_dmax(nth, 0);
    std::vector<uint64_t> t_bad(nth, ~0ull);
    std::vector<char> t_sorted(nth, 1);
    auto scan = [&](unsigned t) {
        const uint64_t i0 = s * t / nth, i1 = s * (t + 1) / nth;
        ScanOut o;
        if (w == 1)
            scan_terms((const uint8_t *)exps, coeffs, n, d->p, i0, i1, key, o);
        else if (w == 2)
            scan_terms((const uint16_t *)exps, coeffs, n, d->p, i0, i1, key, o);
        else
            scan_terms((const uint32_t *)exps, coeffs, n, d->p, i0, i1, key, o);
        t_dmax[t] = o.dmax;
        t_bad[t] = o.bad;
        t_sorted[t] = o.sorted;
    };
    auto parallel = [&](auto fn) {
        const std::function<void(unsigned)> f = fn;
        if (nth == 1)
            f(0u);
        else
            host_parallel(nth, f);
    };
    parallel(scan);
    uint32_t dmax = 0;
    bool sorted = true;
    for (unsigned t = 0; t < nth; ++t) {
        if (t_bad[t] != ~0ull) {
            set_error("coefficient %llu of term %llu is not reduced mod p", (unsigned long long)coeffs[t_bad[t]],
                      (unsigned long long)t_bad[t]);
            return PE_ERR_NOT_REDUCED;
        }
        dmax = std::max(dmax, t_dmax[t]);
        sorted = sorted && t_sorted[t];
        const uint64_t b = s * t / nth;   // thread boundaries
        if (t && b && b < s && key[b] > key[b - 1]) sorted = false;
    }
    if (dmax > 0xffff) {
        set_error("exponent %u above 65535", dmax);
        return PE_ERR_EXP_RANGE;
    }
    // Group order: descending lex on (d, e); stable sort only when needed (Sect. 2.3).
    std::vector<uint32_t> perm;
    if (!sorted) {
        perm.resize(s);
        std::iota(perm.begin(), perm.end(), 0u);
        std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return key[a] > key[b]; });
    }
    auto src = [&](uint64_t i) -> uint64_t { return sorted ? i : perm[i]; };

    pe_poly *P = new pe_poly();
    P->p = d->p;
    P->n = n;
    P->E = E;
    P->s = s;
    P->requested_variant = variant;
    P->variant = variant == PE_MODMUL_AUTO ? default_variant(d->p) : variant;
    P->mc = make_modctx(d->p);
    P->dmax = dmax;
    P->exp_bytes = dmax <= 0xff ? 1 : 2;
    // Groups.
    P->group_off.push_back(0);
    for (uint64_t i = 0; i < s; ++i) {
        const uint64_t k = key[src(i)];
        if (i == 0 || k != key[src(i - 1)]) {
            if (i) P->group_off.push_back(i);
            P->keys.push_back((uint32_t)(k >> 32));
            P->keys.push_back((uint32_t)(k & 0xffffffffu));
        }
    }
    if (s) P->group_off.push_back(s);
    P->G = P->keys.size() / 2;
    // Structure-of-arrays packing, straight into page-locked staging:
    // coefficients, then E rows of exponents.
    const size_t se_bytes = (size_t)E * s * P->exp_bytes;
    Staging stg = stage_acquire(s * 8 + se_bytes);
    std::vector<uint8_t> fallback;
    if (!stg.p) fallback.resize(s * 8 + se_bytes);
    unsigned char *stage = stg.p ? (unsigned char *)stg.p : fallback.data();
    uint64_t *sc = (uint64_t *)stage;
    uint8_t *se = stage + s * 8;
    const uint32_t *pm = sorted ? nullptr : perm.data();
    auto pack = [&](unsigned t) {
        const uint64_t i0 = s * t / nth, i1 = s * (t + 1) / nth;
        const bool out8 = P->exp_bytes == 1;
        if (w == 1 && out8)
            pack_terms((const uint8_t *)exps, coeffs, pm, n, s, i0, i1, sc, se);
        else if (w == 1)
            pack_terms((const uint8_t *)exps, coeffs, pm, n, s, i0, i1, sc, (uint16_t *)se);
        else if (w == 2 && out8)
            pack_terms((const uint16_t *)exps, coeffs, pm, n, s, i0, i1, sc, se);
        else if (w == 2)
            pack_terms((const uint16_t *)exps, coeffs, pm, n, s, i0, i1, sc, (uint16_t *)se);
        else if (out8)
            pack_terms((const uint32_t *)exps, coeffs, pm, n, s, i0, i1, sc, se);
        else
            pack_terms((const uint32_t *)exps, coeffs, pm, n, s, i0, i1, sc, (uint16_t *)se);
    };
    parallel(pack);
    const pe_status ust = upload_packed(P, stg, stage, se_bytes);
    if (ust != PE_OK) return ust;
    if (!sorted) P->perm = std::make_shared<const std::vector<uint32_t>>(std::move(perm));
    *out = P;
    return PE_OK;
}

extern "C" pe_status poly_eval_create_like(const pe_poly *L, uint64_t p, const uint64_t *coeffs, uint32_t flags,
                                           pe_variant variant, pe_poly **out)
{
    if (!out) {
        set_error("out is NULL");
        return PE_ERR_ARG;
    }
    *out = nullptr;
    if (!L || (L->s && !coeffs)) {
        set_error("layout or coeffs is NULL");
        return PE_ERR_ARG;
    }
    if (variant != PE_MODMUL_AUTO && variant != PE_MODMUL_MONT64 && variant != PE_MODMUL_FP64 &&
        variant != PE_MODMUL_BARRETT64 && variant != PE_MODMUL_BARRETT32) {
        set_error("unknown variant %d", (int)variant);
        return PE_ERR_ARG;
    }
    pe_status st = check_prime(p, variant);
    if (st != PE_OK) return st;
    const uint64_t s = L->s;
    // Coefficients in the caller's order, on the host.
    std::vector<uint64_t> hc;
    const uint64_t *c = coeffs;
    cudaError_t e;
    if ((flags & PE_FLAG_DEVICE_PTRS) && s) {
        hc.resize(s);
        if ((e = cudaMemcpy(hc.data(), coeffs, s * 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "reading device coefficients");
        c = hc.data();
    }
    // Range check and copy into staging (in group order), split over the host pool.
    Staging stg = stage_acquire(std::max<uint64_t>(s, 1) * 8);
    std::vector<uint64_t> fallback;
    if (!stg.p) fallback.resize(std::max<uint64_t>(s, 1));
    uint64_t *sc = stg.p ? (uint64_t *)stg.p : fallback.data();
    const std::vector<uint32_t> *perm = L->perm.get();
    const unsigned nth = s >= (1u << 16) ? 2 * host_pool_size() : 1u;
    std::vector<uint64_t> t_bad(nth, ~0ull);
    const std::function<void(unsigned)> fill = [&](unsigned t) {
        const uint64_t i0 = s * t / nth, i1 = s * (t + 1) / nth;
        uint64_t bad = ~0ull;
        for (uint64_t i = i0; i < i1; ++i) {
            const uint64_t v = c[perm ? (*perm)[i] : i];
            if (v >= p && bad == ~0ull) bad = perm ? (*perm)[i] : i;
            sc[i] = v;
        }
        t_bad[t] = bad;
    };
    host_parallel(nth, fill);
    uint64_t bad = ~0ull;
    for (uint64_t b : t_bad) bad = std::min(bad, b);
    if (bad != ~0ull) {
        stage_release(stg);
        set_error("coefficient %llu of term %llu is not reduced mod p", (unsigned long long)c[bad],
                  (unsigned long long)bad);
        return PE_ERR_NOT_REDUCED;
    }
    std::unique_ptr<pe_poly> P(new pe_poly());
    P->p = p;
    P->n = L->n;
    P->E = L->E;
    P->s = s;
    P->G = L->G;
    P->requested_variant = variant;
    P->variant = variant == PE_MODMUL_AUTO ? default_variant(p) : variant;
    P->mc = make_modctx(p);
    P->exp_bytes = L->exp_bytes;
    P->dmax = L->dmax;
    P->group_off = L->group_off;
    P->keys = L->keys;
    P->exps = L->exps;
    P->perm = L->perm;
    cudaStream_t us = upload_stream_acquire();
    const size_t dp1 = P->dmax + 1;
    if ((e = P->coeffs.ensure_async(s * 8, us)) != cudaSuccess || (e = P->mR.ensure_async(s * 8, us)) != cudaSuccess ||
        (e = P->ptab.ensure_async((size_t)P->E * dp1 * 8, us)) != cudaSuccess ||
        (s && (e = cudaMemcpyAsync(P->coeffs.p, sc, s * 8, cudaMemcpyHostToDevice, us)) != cudaSuccess)) {
        cudaStreamSynchronize(us);
        upload_stream_release(us);
        stage_release(stg);
        return cuda_fail(e, "uploading coefficients");
    }
    e = cudaStreamSynchronize(us);
    upload_stream_release(us);
    stage_release(stg);
    if (e != cudaSuccess) return cuda_fail(e, "uploading coefficients");
    *out = P.release();
    return PE_OK;
}

// Waits for the device (as cudaFree would) so that no queued run can still
// read the polynomial's memory, then returns that memory to the pool.
extern "C" void poly_eval_destroy(pe_poly *P)
{
    if (!P) return;
    cudaDeviceSynchronize();
    delete P;
}

extern "C" pe_status poly_eval_groups(const pe_poly *P, uint64_t *G, uint32_t *keys)
{
    if (!P || !G) {
        set_error("NULL argument");
        return PE_ERR_ARG;
    }
    *G = P->G;
    if (keys && P->G) memcpy(keys, P->keys.data(), P->keys.size() * 4);
    return PE_OK;
}

extern "C" pe_status poly_eval_set_tiles(pe_poly *P, const pe_tiles *t)
{
    if (!P) {
        set_error("NULL poly");
        return PE_ERR_ARG;
    }
    pe_tiles z{};
    if (!t) t = &z;
    if (t->K && t->K != 1 && t->K != 2 && t->K != 4 && t->K != 8 && t->K != 12 && t->K != 16) {
        set_error("K must be 1, 2, 4, 8, 12 or 16");
        return PE_ERR_ARG;
    }
    if (t->warps_per_block > 8) {
        set_error("warps_per_block must be at most 8");
        return PE_ERR_ARG;
    }
    P->forced = *t;
    P->plan.valid = false;
    P->tail_plan.valid = false;
    return PE_OK;
}

// The product and tile shape of a run of T points (cheap: no plan tables).
static Tiles plan_tiles(pe_poly *P, uint64_t T)
{
    const int v = run_variant(P, T);
    if (v != P->variant) {
        P->variant = v;
        P->plan.valid = false;
        P->tail_plan.valid = false;
    }
    const Tiles tiles = choose_tiles(P, T, &P->forced);
    if (P->tailT != tiles.tailT) {
        P->plan.valid = false;
        P->tail_plan.valid = false;
        P->tailT = tiles.tailT;
    }
    return tiles;
}

// The plans (chunk, unit and span tables, scratch) of both bands for `tiles`.
static pe_status plan_build(pe_poly *P, uint64_t T, const Tiles &tiles, cudaStream_t st, bool queued)
{
    pe_status ps = ensure_plan(P, P->plan, tiles, T - tiles.tailT, st, queued);
    if (ps != PE_OK || !tiles.tailT) return ps;
    Tiles tt = tiles;
    tt.kslabs = 1;
    tt.Tc = tail_tc(tiles.tailT);
    return ensure_plan(P, P->tail_plan, tt, tiles.tailT, st, queued);
}

static pe_status plan_for(pe_poly *P, uint64_t T, Tiles *tiles, cudaStream_t st = nullptr, bool queued = false)
{
    *tiles = plan_tiles(P, T);
    return plan_build(P, T, *tiles, st, queued);
}

extern "C" pe_status poly_eval_plan_info(pe_poly *P, uint64_t T, pe_plan_info *info)
{
    if (!P || !info || T == 0) {
        set_error("bad argument");
        return PE_ERR_ARG;
    }
    Tiles t;
    pe_status st = plan_for(P, T, &t);
    if (st != PE_OK) return st;
    memset(info, 0, sizeof *info);
    info->tiles.K = t.K;
    info->tiles.slabs = t.kslabs;
    info->tiles.tchunk = t.Tc;
    info->tiles.warps_per_block = t.wpb;
    info->variant = (pe_variant)P->variant;
    info->chunks = P->plan.NC;
    info->items = (uint64_t)P->plan.U * P->plan.Q + (t.tailT ? (uint64_t)P->tail_plan.U * P->tail_plan.Q : 0);
    info->spans = P->plan.S;
    info->padded_terms = (uint64_t)P->plan.NC * t.K;
    {
        const TuneEntry *te = tune_lookup(P, T);
        info->method = P->requested_variant == PE_MODMUL_AUTO && !P->forced.K && !P->forced.slabs &&
                               !P->forced.tchunk && !P->forced.warps_per_block && !P->forced.tail && te &&
                               te->method == 1 && fast_applicable(P->p, T)
                           ? 1u
                           : 0u;
    }
    info->tail_points = t.tailT;
    return PE_OK;
}

extern "C" pe_status poly_eval_set_timing(pe_poly *P, int enable)
{
    if (!P) {
        set_error("NULL poly");
        return PE_ERR_ARG;
    }
    P->timing = enable != 0;
    return PE_OK;
}

extern "C" pe_status poly_eval_kernel_times(pe_poly *P, double ms[3], uint64_t *runs)
{
    if (!P || !ms) {
        set_error("NULL argument");
        return PE_ERR_ARG;
    }
    ms[0] = ms[1] = ms[2] = 0.0;
    const size_t nrun = P->events_used / 4;
    for (size_t r = 0; r < nrun; ++r) {
        cudaEvent_t *ev = &P->events[4 * r];
        cudaError_t e = cudaEventSynchronize(ev[3]);
        if (e != cudaSuccess) return cuda_fail(e, "timing");
        for (int k = 0; k < 3; ++k) {
            float x = 0.f;
            if ((e = cudaEventElapsedTime(&x, ev[k], ev[k + 1])) != cudaSuccess) return cuda_fail(e, "timing");
            ms[k] += x;
        }
    }
    if (runs) *runs = nrun;
    P->events_used = 0;
    return PE_OK;
}

extern "C" pe_status poly_eval_launches_per_run(pe_poly *P, uint64_t T, uint32_t *launches)
{
    if (!P || !launches) {
        set_error("NULL argument");
        return PE_ERR_ARG;
    }
    uint32_t n = 0;
    if (T && P->G) {
        if (P->E && P->dmax + 1) n++;   // power tables
        n++;                            // Step A
        n++;                            // Step B
    }
    *launches = n;
    return PE_OK;
}

extern "C" pe_status poly_eval_run(pe_poly *P, const uint64_t *beta, uint64_t T, uint64_t t0, uint64_t *out,
                                   void *stream)
{
    // The tuner's choice of method for this shape, unless a product or tiles were forced.
    if (P && P->requested_variant == PE_MODMUL_AUTO && !P->forced.K && !P->forced.slabs && !P->forced.tchunk &&
        !P->forced.warps_per_block && !P->forced.tail && fast_applicable(P->p, T)) {
        const TuneEntry *te = tune_lookup(P, T);
        if (te && te->method == 1) return poly_eval_run_fast(P, beta, T, t0, out, stream);
    }
    return run_matrix(P, beta, T, t0, out, stream);
}

constexpr uint64_t kPipelinedDownloadBytes = 16ull << 20;

// Step B into host memory: one launch per T-chunk (main band, then tail
// band), rotating over the run's stream and two more of the handle's streams;
// each chunk's rows are downloaded on a third stream as soon as that chunk's
// launch has finished.  Items of a later chunk fill the SMs as an earlier
// chunk's items finish (launches on two streams overlap), the copies never hold
// up a launch, and only the last chunks' copies remain after the compute.
// T-chunks share nothing but read-only plan tables: carries and arrival
// counters are per T-chunk, chain buffers per item.
static pe_status stepb_download_pipelined(pe_poly *P, const Tiles &t, StepBJob J0, StepBJob J1, uint64_t T0,
                                          uint64_t T, uint64_t *out, uint64_t *out_dev, cudaStream_t cs)
{
    cudaError_t e;
    for (cudaStream_t *a : {&P->aux[0], &P->aux[1], &P->copy_st})
        if (!*a && (e = cudaStreamCreateWithFlags(a, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "streams");
    const uint32_t nchunks = P->plan.Q + (T > T0 ? P->tail_plan.Q : 0);
    while (P->chunk_ev.size() < nchunks) {
        cudaEvent_t x;
        if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "events");
        P->chunk_ev.push_back(x);
    }
    if ((!P->fork_ev && (e = cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming)) != cudaSuccess) ||
        (!P->join_ev && (e = cudaEventCreateWithFlags(&P->join_ev, cudaEventDisableTiming)) != cudaSuccess))
        return cuda_fail(e, "events");
    if ((e = cudaEventRecord(P->fork_ev, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(P->aux[0], P->fork_ev, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(P->aux[1], P->fork_ev, 0)) != cudaSuccess)
        return cuda_fail(e, "fork");
    const cudaStream_t launch_st[3] = {cs, P->aux[0], P->aux[1]};
    const uint64_t G = P->G;
    const StepBJob none{};
    uint32_t k = 0;
    for (int band = 0; band < 2; ++band) {
        const Plan &pl = band == 0 ? P->plan : P->tail_plan;
        StepBJob J = band == 0 ? J0 : J1;
        const uint64_t rows = band == 0 ? T0 : T - T0, row0 = band == 0 ? 0 : T0;
        if (!rows) continue;
        for (uint32_t q = 0; q < pl.Q; ++q, ++k) {
            // Three launch streams: a chunk waits only for the chunk three
            // before it, so the tail band's chunks start as SMs free up.
            cudaStream_t st = launch_st[k % 3];
            J.item0 = q * pl.U;
            if ((e = launch_stepB((int)t.K, P->variant, J, pl.U, none, 0, (int)t.wpb, st)) != cudaSuccess)
                return cuda_fail(e, "Step B");
            const uint64_t r0 = row0 + (uint64_t)q * pl.Tc, r1 = std::min<uint64_t>(row0 + rows, r0 + pl.Tc);
            if ((e = cudaEventRecord(P->chunk_ev[k], st)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(P->copy_st, P->chunk_ev[k], 0)) != cudaSuccess ||
                (e = cudaMemcpyAsync(out + r0 * G, out_dev + r0 * G, (r1 - r0) * G * 8, cudaMemcpyDeviceToHost,
                                     P->copy_st)) != cudaSuccess)
                return cuda_fail(e, "copy back");
        }
    }
    // The copy stream waited for every chunk, so joining it covers every launch stream.
    if ((e = cudaEventRecord(P->join_ev, P->copy_st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cs, P->join_ev, 0)) != cudaSuccess)
        return cuda_fail(e, "join");
    return PE_OK;
}

pe_status pe::run_matrix(pe_poly *P, const uint64_t *beta, uint64_t T, uint64_t t0, uint64_t *out, void *stream)
{
    if (!P) {
        set_error("NULL poly");
        return PE_ERR_ARG;
    }
    if (!points_ok(T, t0) || !out_ok(T, P->G)) return PE_ERR_ARG;
    BetaArg barg;
    pe_status st = check_beta(P, beta, &barg);
    if (st != PE_OK) return st;
    if (T == 0 || P->G == 0) return PE_OK;
    if (!out) {
        set_error("out is NULL");
        return PE_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    // Runs of one handle share its scratch (power tables, monomials, starting
    // values, plans), so a run on any stream starts after the previous one has
    // finished; buffers replaced below are freed only after that run as well.
    if (P->last_use) {
        cudaStreamWaitEvent(cs, P->last_use, 0);
        cudaStreamWaitEvent(alloc_stream(), P->last_use, 0);
    }
    // Tiles first: the power tables and Step A need only the start rows, so
    // they are queued before the plan tables are built on the host.
    const Tiles t = plan_tiles(P, T);
    cudaPointerAttributes attr{};
    bool dev_out = false, pinned_out = false;
    if (cudaPointerGetAttributes(&attr, out) == cudaSuccess) {
        dev_out = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
        pinned_out = attr.type == cudaMemoryTypeHost;
    }
    cudaGetLastError();
    uint64_t *out_dev = out;
    cudaError_t e;
    if (!dev_out) {
        if ((e = P->out_scratch.ensure_async(T * P->G * 8, cs)) != cudaSuccess) return cuda_fail(e, "output scratch");
        out_dev = P->out_scratch.as<uint64_t>();
    }
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (P->timing) {
        while (P->events.size() < P->events_used + 4) {
            cudaEvent_t x;
            if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(e, "timing events");
            P->events.push_back(x);
        }
        for (int k = 0; k < 4; ++k) ev[k] = P->events[P->events_used + k];
        P->events_used += 4;
    }
    auto mark = [&](int k) {
        if (ev[k]) cudaEventRecord(ev[k], cs);
    };
    const uint32_t dp1 = P->dmax + 1;
    mark(0);
    if ((e = launch_powtab(barg, P->E, dp1, P->mc, P->ptab.as<uint64_t>(), cs)) != cudaSuccess)
        return cuda_fail(e, "power tables");
    mark(1);
    // Item start rows: band 0's T-chunks, then the tail band's (the plans'
    // T-chunks follow from the tiles alone).
    const uint64_t T0 = T - t.tailT;
    const uint32_t tc0 = t.Tc, tc1 = t.tailT ? tail_tc(t.tailT) : 1;
    const uint32_t q0 = (uint32_t)((T0 + tc0 - 1) / tc0), q1 = t.tailT ? (uint32_t)((t.tailT + tc1 - 1) / tc1) : 0;
    StartRows sr{};
    bool use_starts = q0 + q1 <= (uint32_t)kMaxStarts;
    if (use_starts) {
        for (uint32_t q = 0; q < q0; ++q) sr.row[sr.n++] = q * tc0;
        for (uint32_t q = 0; q < q1; ++q) sr.row[sr.n++] = (uint32_t)T0 + q * tc1;
        use_starts = plan_start_gaps(&sr);   // at most three distinct gaps (main band, band change, tail band)
    }
    if (use_starts) {
        if ((e = P->vstart.ensure_async((size_t)sr.n * P->s * 8, cs)) != cudaSuccess) return cuda_fail(e, "start values");
        e = launch_stepA_starts(P->exps->p, P->exp_bytes, P->coeffs.as<uint64_t>(), P->s, P->E,
                                P->ptab.as<uint64_t>(), dp1, P->mc, t0, sr, P->mR.as<uint64_t>(),
                                P->vstart.as<uint64_t>(), num_sms(), cs);
    } else {
        e = launch_stepA(P->exps->p, P->exp_bytes, P->s, P->E, P->ptab.as<uint64_t>(), dp1, P->mc,
                         P->mR.as<uint64_t>(), num_sms(), cs);
    }
    if (e != cudaSuccess) return cuda_fail(e, "Step A");
    if ((st = plan_build(P, T, t, cs, true)) != PE_OK) return st;
    if (P->plan.Q != q0 || (t.tailT && P->tail_plan.Q != q1)) {
        set_error("internal: plan and start rows disagree");
        return PE_ERR_ARG;
    }
    StepBJob J0 = make_job(P, P->plan, t0, out_dev, false);
    StepBJob J1{};
    uint32_t n1 = 0;
    if (t.tailT) {
        J1 = make_job(P, P->tail_plan, t0 + T0, out_dev + T0 * P->G, false);
        n1 = P->tail_plan.U * P->tail_plan.Q;
    }
    if (use_starts) {
        J0.vstart = J1.vstart = P->vstart.as<uint64_t>();
        J0.vs_base = 0;
        J1.vs_base = q0;
    }
    mark(2);
    // A large download into page-locked host memory overlaps the compute
    // chunk by chunk; small ones take one launch and one copy (extra launches
    // would cost more than the copy), and so do downloads into pageable memory
    // (a copy there returns only when it is done, which would stall the launches).
    const bool pipelined = pinned_out && T * P->G * 8 >= kPipelinedDownloadBytes && q0 + q1 >= 3;
    if (!pipelined) {
        if ((e = launch_stepB((int)t.K, P->variant, J0, P->plan.U * P->plan.Q, J1, n1, (int)t.wpb, cs)) != cudaSuccess)
            return cuda_fail(e, "Step B");
        if (!dev_out && (e = cudaMemcpyAsync(out, out_dev, T * P->G * 8, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
            return cuda_fail(e, "copy back");
    } else if ((st = stepb_download_pipelined(P, t, J0, J1, T0, T, out, out_dev, cs)) != PE_OK) {
        return st;
    }
    mark(3);
    if (!P->last_use && (e = cudaEventCreateWithFlags(&P->last_use, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "event");
    if ((e = cudaEventRecord(P->last_use, cs)) != cudaSuccess) return cuda_fail(e, "event");
    if (!dev_out && (e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "run");
    return PE_OK;
}
