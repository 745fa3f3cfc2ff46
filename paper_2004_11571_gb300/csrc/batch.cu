// Batched evaluation: many polynomials in one persistent kernel.
//
// Each job (polynomial, beta, T, t0) gets its own Step B plan; all plans,
// power tables and scratch live in one device arena.  Work items of every job
// are put in one queue ordered by decreasing estimated cost; a persistent
// kernel with a fixed number of warps per SM pops items with an atomic ticket
// (a warp that finishes early takes the next item, so the cheap items at the
// end of the queue fill the tail).  Step A runs fused into each item (the
// monomial values are formed from the exponents and the job's power tables),
// so a batch is three graph nodes: clear the counters, build every job's power
// tables, run the queue.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include "internal.h"
#include "modarith.cuh"
#include "stepb.cuh"
#include "tune.h"

namespace pe {

struct PowJob {
    const uint64_t *beta;
    uint64_t *ptab;
    uint32_t E, dp1;
    ModCtx mc;
};

// Power tables of every job: blockIdx.y selects the job (Sect. 2.3 tables).
__global__ void k_powtab_batch(const PowJob *__restrict__ jobs)
{
    const PowJob &J = jobs[blockIdx.y];
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= J.E * J.dp1) return;
    const uint32_t j = idx / J.dp1, e = idx - j * J.dp1;
    const uint64_t bR = canon(mont_mul(J.beta[j], J.mc.r2, J.mc), J.mc.p);
    J.ptab[idx] = mont_pow(bR, e, J.mc);
}

struct QueueSmem {
    WarpSmem w;
    StepBJob job;
};

template <int K, int VAR>
__device__ __forceinline__ void queue_item(const StepBJob &J, uint32_t item, WarpSmem &sm)
{
    stepb_item<K, VAR>(J, item, sm);
}

// The persistent Step B kernel: warps pop (job, item) pairs until the queue is empty.
__global__ void __launch_bounds__(128) k_stepB_queue(const StepBJob *__restrict__ jobs,
                                                     const uint2 *__restrict__ items, uint32_t nitems,
                                                     uint32_t *__restrict__ head)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    QueueSmem &qs = reinterpret_cast<QueueSmem *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    uint32_t cur_job = 0xffffffffu;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(head, 1u);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= nitems) break;
        const uint2 it = items[idx];
        if (it.x != cur_job) {   // stage the job description in shared memory
            const uint32_t *src = reinterpret_cast<const uint32_t *>(jobs + it.x);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&qs.job);
            for (uint32_t w = lane; w < sizeof(StepBJob) / 4; w += 32) dst[w] = src[w];
            cur_job = it.x;
            __syncwarp();
        }
        const StepBJob &J = qs.job;
        switch (J.K * 8 + J.var) {
        case 1 * 8 + VAR_BARRETT: queue_item<1, VAR_BARRETT>(J, it.y, qs.w); break;
        case 2 * 8 + VAR_BARRETT: queue_item<2, VAR_BARRETT>(J, it.y, qs.w); break;
        case 4 * 8 + VAR_BARRETT: queue_item<4, VAR_BARRETT>(J, it.y, qs.w); break;
        case 8 * 8 + VAR_BARRETT: queue_item<8, VAR_BARRETT>(J, it.y, qs.w); break;
        case 1 * 8 + VAR_MONT: queue_item<1, VAR_MONT>(J, it.y, qs.w); break;
        case 2 * 8 + VAR_MONT: queue_item<2, VAR_MONT>(J, it.y, qs.w); break;
        case 4 * 8 + VAR_MONT: queue_item<4, VAR_MONT>(J, it.y, qs.w); break;
        case 8 * 8 + VAR_MONT: queue_item<8, VAR_MONT>(J, it.y, qs.w); break;
        case 1 * 8 + VAR_FP64: queue_item<1, VAR_FP64>(J, it.y, qs.w); break;
        case 2 * 8 + VAR_FP64: queue_item<2, VAR_FP64>(J, it.y, qs.w); break;
        case 4 * 8 + VAR_FP64: queue_item<4, VAR_FP64>(J, it.y, qs.w); break;
        case 8 * 8 + VAR_FP64: queue_item<8, VAR_FP64>(J, it.y, qs.w); break;
        case 1 * 8 + VAR_BARRETT32: queue_item<1, VAR_BARRETT32>(J, it.y, qs.w); break;
        case 2 * 8 + VAR_BARRETT32: queue_item<2, VAR_BARRETT32>(J, it.y, qs.w); break;
        case 4 * 8 + VAR_BARRETT32: queue_item<4, VAR_BARRETT32>(J, it.y, qs.w); break;
        case 8 * 8 + VAR_BARRETT32: queue_item<8, VAR_BARRETT32>(J, it.y, qs.w); break;
        default: break;
        }
        __syncwarp();
    }
}

static constexpr int kQueueWarps = 4;

static size_t queue_smem() { return kQueueWarps * sizeof(QueueSmem); }

static cudaError_t queue_setup(int *blocks_per_sm)
{
    cudaError_t e = smem_limit_once((const void *)k_stepB_queue, (int)queue_smem());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_stepB_queue, kQueueWarps * 32,
                                                         queue_smem());
}

uint64_t queue_resident_warps()
{
    int bps = 0;
    if (queue_setup(&bps) != cudaSuccess || bps < 1) bps = 1;
    return (uint64_t)bps * kQueueWarps * num_sms();
}

// Chooses a job's tiles for a batch whose items should be about `w_target`
// slot-points each (slot-points = padded terms x points).
static Tiles batch_tiles(pe_poly *P, uint64_t T, double w_target)
{
    Tiles t;
    t.wpb = kQueueWarps;
    const TuneEntry *te = tune_lookup(P, T);
    if (te && te->K <= 8) {
        t.K = te->K;
    } else {
        double best = 1e300;
        for (uint32_t K : {1u, 2u, 4u, 8u}) {
            uint64_t nc = 0;
            for (uint64_t g = 0; g < P->G; ++g) nc += (P->group_off[g + 1] - P->group_off[g] + K - 1) / K;
            const double c = (double)nc * (K + 0.7);
            if (c < best * 0.98) {
                best = c;
                t.K = K;
            }
        }
    }
    uint64_t nc = 0;
    for (uint64_t g = 0; g < P->G; ++g) nc += (P->group_off[g + 1] - P->group_off[g] + t.K - 1) / t.K;
    const uint64_t slabs = std::max<uint64_t>(1, (nc + 31) / 32);
    const double one_slab = 32.0 * t.K * (double)T;
    if (one_slab <= w_target) {
        t.Tc = (uint32_t)T;
        t.kslabs = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(slabs, (uint64_t)(w_target / one_slab)));
    } else {
        t.kslabs = 1;
        uint64_t tc = (uint64_t)(w_target / (32.0 * t.K));
        tc = std::max<uint64_t>(64, (tc + 31) / 32 * 32);
        t.Tc = (uint32_t)std::min<uint64_t>(tc, T);
    }
    return t;
}

static int resolve_variant(pe_poly *P, uint64_t T) { return run_variant(P, T); }

namespace {

struct Layout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

}  // namespace

// Plans every job, lays the plans, power tables, scratch and the ordered work
// queue out in `arena` (grown only when too small) and fills `img.host` with
// the bytes to upload there.
pe_status batch_build(const pe_job *jobs, size_t njobs, DevBuf &arena, BatchImage &img, bool plain_runs)
{
    img = BatchImage{};
    if (njobs && !jobs) {
        set_error("jobs is NULL");
        return PE_ERR_ARG;
    }
    img.betas.resize(njobs);
    img.is_plain.assign(njobs, 0);
    double w_total = 0.0, w_queue = 0.0;
    for (size_t j = 0; j < njobs; ++j) {
        const pe_job &jb = jobs[j];
        if (!jb.poly || (jb.T && jb.poly->G && !jb.out)) {
            set_error("job %zu: NULL poly or out", j);
            return PE_ERR_ARG;
        }
        if (!points_ok(jb.T, jb.t0) || !out_ok(jb.T, jb.poly->G)) return PE_ERR_ARG;
        BetaArg ba;
        pe_status st = check_beta(jb.poly, jb.beta, &ba);
        if (st != PE_OK) return st;
        img.betas[j].assign(ba.b, ba.b + jb.poly->E);
        const double w = (double)jb.poly->s * (double)jb.T;
        w_total += w;
        if (plain_runs && w >= kPlainRunWork && jb.poly->G) {
            img.is_plain[j] = 1;
            img.plain.push_back({j, jb.poly, jb.T, jb.t0, jb.out});
        } else {
            w_queue += w;
        }
    }
    // a job in the queue: nonempty and not a plain run
    auto queued = [&](size_t j) { return jobs[j].T && jobs[j].poly->G && !img.is_plain[j]; };
    const uint64_t R = queue_resident_warps();
    const double w_target = std::max(w_queue / (8.0 * (double)R), 32.0 * 64.0);
    std::vector<PlanHost> ph(njobs);
    std::vector<std::vector<uint32_t>> cs(njobs), cg(njobs);
    std::vector<int> var(njobs);
    // Two regions: U (uploaded: descriptors, tables, betas, the queue) and S
    // (scratch, written by the kernels before it is read; counters cleared).
    Layout U, S;
    const size_t off_jobs = U.take(std::max<size_t>(njobs, 1) * sizeof(StepBJob));
    const size_t off_pow = U.take(std::max<size_t>(njobs, 1) * sizeof(PowJob));
    std::vector<size_t> o_cs(njobs), o_cg(njobs), o_unit(njobs), o_span(njobs), o_carry(njobs), o_chain(njobs),
        o_ptab(njobs), o_cnt(njobs);
    img.beta_off.assign(njobs, 0);
    // Power-table classes: (p, E, beta) -> leader; the class's table width is
    // its largest dmax + 1 (Sect. 2.3 tables, computed once per class).
    img.leader.resize(njobs);
    std::vector<uint32_t> dp1c(njobs, 1);
    {
        std::map<std::vector<uint64_t>, size_t> cls;
        for (size_t j = 0; j < njobs; ++j) {
            img.leader[j] = j;
            pe_poly *P = jobs[j].poly;
            if (!queued(j) || !P->E) continue;
            std::vector<uint64_t> key{P->p, P->E};
            key.insert(key.end(), img.betas[j].begin(), img.betas[j].end());
            auto it = cls.emplace(key, j).first;
            img.leader[j] = it->second;
            dp1c[it->second] = std::max(dp1c[it->second], P->dmax + 1);
        }
        for (size_t j = 0; j < njobs; ++j) dp1c[j] = dp1c[img.leader[j]];
    }
    for (size_t j = 0; j < njobs; ++j) {
        pe_poly *P = jobs[j].poly;
        if (!queued(j)) continue;
        const Tiles t = batch_tiles(P, jobs[j].T, w_target);
        build_plan_host(P, t, jobs[j].T, ph[j]);
        build_chunks(P, t.K);                  // the image holds the chunk tables
        cs[j] = P->chunks.cs;
        cg[j] = P->chunks.cg;
        var[j] = resolve_variant(P, jobs[j].T);
        o_cs[j] = U.take(cs[j].size() * 4);
        o_cg[j] = U.take(std::max<size_t>(cg[j].size(), 1) * 4);
        o_unit[j] = U.take(ph[j].unit.size() * 4);
        o_span[j] = U.take(ph[j].span.size() * 4);
        img.beta_off[j] = U.take((size_t)std::max<uint32_t>(P->E, 1) * 8);
        o_carry[j] = S.take(ph[j].carry_bytes());
        o_chain[j] = S.take(ph[j].chain_bytes());
        o_ptab[j] = S.take((size_t)std::max<uint32_t>(P->E, 1) * dp1c[j] * 8);
    }
    // Items, grouped by code path (K and product: the warps of an SM then run
    // the same instantiation of the item loop and share its instructions),
    // classes in decreasing order of their largest item, each by decreasing
    // cost (a slab-point of a K-term chunk costs K), so the queue ends on the
    // cheapest items.
    struct QItem {
        double cost;
        uint32_t cls;
        uint2 it;
    };
    std::vector<QItem> items;
    std::map<uint32_t, double> cls_max;
    for (size_t j = 0; j < njobs; ++j) {
        if (!queued(j)) continue;
        const PlanHost &p = ph[j];
        const uint32_t cls = p.K * 8 + (uint32_t)var[j];
        const double lg = std::log2((double)std::max<uint64_t>(2, jobs[j].t0 + jobs[j].T));
        for (uint32_t q = 0; q < p.Q; ++q) {
            const uint64_t tc = std::min<uint64_t>(p.Tc, p.T - (uint64_t)q * p.Tc);
            for (uint32_t u = 0; u < p.U; ++u) {
                const uint32_t chunks = std::min(p.NC - u * 32 * p.kslabs, 32 * p.kslabs);
                const double slabs = std::ceil(chunks / 32.0);
                const double cost = slabs * 32.0 * (p.K * (double)tc * 1.2 + (double)tc * 0.7 + p.K * lg * 3.0);
                items.push_back({cost, cls, make_uint2((uint32_t)j, q * p.U + u)});
                cls_max[cls] = std::max(cls_max[cls], cost);
            }
        }
    }
    {   // class order: decreasing largest item (ties by class code), looked up once per item
        std::vector<std::pair<double, uint32_t>> order;
        for (const auto &kv : cls_max) order.push_back({kv.second, kv.first});
        std::sort(order.begin(), order.end(), [](const auto &a, const auto &b) {
            return a.first != b.first ? a.first > b.first : a.second > b.second;
        });
        uint32_t rank_of[256] = {};
        for (size_t r = 0; r < order.size(); ++r) rank_of[order[r].second & 255] = (uint32_t)r;
        for (QItem &q : items) q.cls = rank_of[q.cls & 255] << 8 | (q.cls & 255);   // rank above the code
    }
    std::stable_sort(items.begin(), items.end(), [](const QItem &a, const QItem &b) {
        return a.cls != b.cls ? a.cls < b.cls : a.cost > b.cost;
    });
    for (QItem &q : items) q.cls &= 255;
    const size_t off_items = U.take(std::max<size_t>(items.size(), 1) * sizeof(uint2));
    // Counters (and the queue head) in one contiguous scratch block, cleared before each launch.
    const size_t cnt0 = S.off;
    const size_t off_head = S.take(256);
    for (size_t j = 0; j < njobs; ++j)
        if (queued(j)) o_cnt[j] = S.take(ph[j].counter_bytes());
    const size_t cnt1 = S.off;
    // Scratch offsets follow the uploaded region.
    const size_t up = U.off;
    for (size_t j = 0; j < njobs; ++j) {
        o_carry[j] += up;
        o_chain[j] += up;
        o_ptab[j] += up;
        o_cnt[j] += up;
    }
    img.counters_off = up + cnt0;
    img.counters_bytes = cnt1 - cnt0;
    cudaError_t e = arena.ensure(up + S.off);
    if (e != cudaSuccess) return cuda_fail(e, "batch arena");
    unsigned char *base = arena.as<unsigned char>();
    img.host.assign(up, 0);
    auto put = [&](size_t off, const void *src, size_t n) {
        if (n) memcpy(img.host.data() + off, src, n);
    };
    std::vector<StepBJob> hj(njobs);
    std::vector<PowJob> hp(njobs);
    for (size_t j = 0; j < njobs; ++j) {
        const pe_job &jb = jobs[j];
        pe_poly *P = jb.poly;
        if (!queued(j)) continue;
        put(o_cs[j], cs[j].data(), cs[j].size() * 4);
        put(o_cg[j], cg[j].data(), cg[j].size() * 4);
        put(o_unit[j], ph[j].unit.data(), ph[j].unit.size() * 4);
        put(o_span[j], ph[j].span.data(), ph[j].span.size() * 4);
        put(img.beta_off[j], img.betas[j].data(), img.betas[j].size() * 8);
        const size_t lead = img.leader[j];
        fill_job(hj[j], P, ph[j], (const uint32_t *)(base + o_cs[j]), (const uint32_t *)(base + o_cg[j]),
                 (const int32_t *)(base + o_unit[j]), (const uint32_t *)(base + o_span[j]),
                 (uint32_t *)(base + o_cnt[j]), (ulonglong2 *)(base + o_carry[j]), (ulonglong2 *)(base + o_chain[j]),
                 jb.t0, jb.out, nullptr, (const uint64_t *)(base + o_ptab[lead]), var[j]);
        hj[j].dp1 = dp1c[j];
        hp[j].beta = (const uint64_t *)(base + img.beta_off[j]);
        hp[j].ptab = (uint64_t *)(base + o_ptab[j]);
        hp[j].E = lead == j ? P->E : 0;   // followers read the leader's tables
        hp[j].dp1 = dp1c[j];
        hp[j].mc = P->mc;
        if (lead == j) ++img.tables;
        img.max_entries = std::max(img.max_entries, P->E * dp1c[j]);
    }
    put(off_jobs, hj.data(), njobs * sizeof(StepBJob));
    put(off_pow, hp.data(), njobs * sizeof(PowJob));
    img.off_jobs = off_jobs;
    img.off_pow = off_pow;
    img.ptab_off = o_ptab;
    std::vector<uint2> it(items.size());
    for (size_t i = 0; i < items.size(); ++i) it[i] = items[i].it;
    put(off_items, it.data(), it.size() * sizeof(uint2));
    img.base = base;
    img.d_jobs = (StepBJob *)(base + off_jobs);
    img.d_pow = (PowJob *)(base + off_pow);
    img.d_items = (uint2 *)(base + off_items);
    img.d_head = (uint32_t *)(base + up + off_head);
    img.nitems = (uint32_t)items.size();
    img.njobs = (uint32_t)njobs;
    int bps = 0;
    if ((e = queue_setup(&bps)) != cudaSuccess) return cuda_fail(e, "queue kernel setup");
    img.grid = std::max(1, bps) * num_sms();
    img.term_points = w_total;
    return PE_OK;
}

// Clears the counters, builds every job's power tables and runs the queue.
cudaError_t batch_kernels(const BatchImage &img, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(img.base + img.counters_off, 0, img.counters_bytes, st);
    if (e != cudaSuccess) return e;
    if (img.max_entries && img.njobs)
        k_powtab_batch<<<dim3((img.max_entries + 127) / 128, img.njobs), 128, 0, st>>>(img.d_pow);
    if (img.nitems)
        k_stepB_queue<<<img.grid, kQueueWarps * 32, queue_smem(), st>>>(img.d_jobs, img.d_items, img.nitems,
                                                                        img.d_head);
    return cudaGetLastError();
}

// Uploads the image (stream-ordered) and runs it.
cudaError_t batch_enqueue(const BatchImage &img, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(img.base, img.host.data(), img.host.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return batch_kernels(img, st);
}

pe_status batch_run_plain(const BatchImage &img, cudaStream_t st)
{
    for (const BatchImage::PlainRun &r : img.plain) {
        const pe_status s = run_matrix(r.poly, img.betas[r.j].data(), r.T, r.t0, r.out, st);
        if (s != PE_OK) return s;
    }
    return PE_OK;
}

}  // namespace pe

using namespace pe;

struct pe_batch {
    std::vector<pe_job> jobs;
    BatchImage img;
    DevBuf arena;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~pe_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
};

extern "C" pe_status poly_eval_batch_plan(const pe_job *jobs, size_t njobs, pe_batch **out)
{
    if (!out) {
        set_error("out is NULL");
        return PE_ERR_ARG;
    }
    *out = nullptr;
    pe_batch *B = new pe_batch();
    if (njobs && jobs) B->jobs.assign(jobs, jobs + njobs);
    pe_status st = batch_build(jobs, njobs, B->arena, B->img);
    if (st != PE_OK) {
        delete B;
        return st;
    }
    cudaError_t e = cudaMemcpy(B->img.base, B->img.host.data(), B->img.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete B;
        return cuda_fail(e, "batch upload");
    }
    // Capture the batch as a CUDA graph on a private stream.
    if ((e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        delete B;
        return cuda_fail(e, "graph capture");
    }
    cudaError_t le = batch_kernels(B->img, B->cap);
    e = cudaStreamEndCapture(B->cap, &B->graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
    if (e != cudaSuccess) {
        delete B;
        return cuda_fail(e, "graph build");
    }
    *out = B;
    return PE_OK;
}

extern "C" pe_status poly_eval_batch_launch(pe_batch *B, void *stream)
{
    if (!B) {
        set_error("NULL batch");
        return PE_ERR_ARG;
    }
    cudaError_t e = cudaGraphLaunch(B->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return batch_run_plain(B->img, (cudaStream_t)stream);
}

extern "C" pe_status poly_eval_batch_launches(const pe_batch *B, uint32_t *kernels, uint32_t *plain_jobs)
{
    if (!B) {
        set_error("NULL batch");
        return PE_ERR_ARG;
    }
    const BatchImage &I = B->img;
    uint32_t n = (I.max_entries && I.njobs ? 1u : 0u) + (I.nitems ? 1u : 0u);
    for (const BatchImage::PlainRun &r : I.plain) {
        uint32_t k = 0;
        if (poly_eval_launches_per_run(r.poly, r.T, &k) == PE_OK) n += k;
    }
    if (kernels) *kernels = n;
    if (plain_jobs) *plain_jobs = (uint32_t)I.plain.size();
    return PE_OK;
}

extern "C" pe_status poly_eval_batch_set_beta(pe_batch *B, size_t j, const uint64_t *beta)
{
    if (!B || j >= B->jobs.size()) {
        set_error("bad batch or job index");
        return PE_ERR_ARG;
    }
    BetaArg ba;
    pe_status st = check_beta(B->jobs[j].poly, beta, &ba);
    if (st != PE_OK) return st;
    const uint32_t E = B->jobs[j].poly->E;
    if (!E) return PE_OK;
    BatchImage &I = B->img;
    I.betas[j].assign(ba.b, ba.b + E);
    if (I.is_plain[j]) return PE_OK;   // a plain run reads its point from the host at launch
    cudaError_t e = cudaMemcpy(I.base + I.beta_off[j], I.betas[j].data(), E * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "beta upload");
    if (!B->jobs[j].T || !B->jobs[j].poly->G) return PE_OK;
    // A job that shared power tables leaves its class: it computes its own from
    // now on, and if it led the class the next member takes over the lead.
    const size_t lead = I.leader[j];
    std::vector<size_t> members;
    for (size_t k = 0; k < I.leader.size(); ++k)
        if (I.leader[k] == lead && k != j) members.push_back(k);
    if (members.empty()) return PE_OK;
    auto job_at = [&](size_t k) { return (StepBJob *)(I.host.data() + I.off_jobs) + k; };
    auto pow_at = [&](size_t k) { return (PowJob *)(I.host.data() + I.off_pow) + k; };
    std::vector<size_t> touched{j};
    I.leader[j] = j;
    job_at(j)->ptab = (const uint64_t *)(I.base + I.ptab_off[j]);
    pow_at(j)->E = E;
    if (lead == j) {
        const size_t nl = members[0];
        pow_at(nl)->E = B->jobs[nl].poly->E;
        for (size_t k : members) {
            I.leader[k] = nl;
            job_at(k)->ptab = (const uint64_t *)(I.base + I.ptab_off[nl]);
            touched.push_back(k);
        }
    } else {
        ++I.tables;
    }
    for (size_t k : touched) {
        if ((e = cudaMemcpy(I.base + I.off_jobs + k * sizeof(StepBJob), job_at(k), sizeof(StepBJob),
                            cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(I.base + I.off_pow + k * sizeof(PowJob), pow_at(k), sizeof(PowJob),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "batch descriptors");
    }
    if (lead == j) ++I.tables;
    return PE_OK;
}

extern "C" void poly_eval_batch_destroy(pe_batch *B)
{
    if (!B) return;
    cudaDeviceSynchronize();   // a launched graph may still be running
    delete B;
}

extern "C" pe_status poly_eval_batch(const pe_job *jobs, size_t njobs, void *stream)
{
    pe_batch *B = nullptr;
    pe_status st = poly_eval_batch_plan(jobs, njobs, &B);
    if (st != PE_OK) return st;
    st = poly_eval_batch_launch(B, stream);
    if (st == PE_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch");
    }
    poly_eval_batch_destroy(B);
    return st;
}
