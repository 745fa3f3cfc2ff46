// Server: continuous batching of evaluation requests.
//
// Clients submit requests (a polynomial to upload, or one already resident,
// with beta, T, t0 and a host output buffer).  Three stages run concurrently:
//  * upload threads take requests with a new polynomial from the backlog in
//    arrival order, admit them while their device memory fits under the cap
//    (evicting unreferenced uploads least recently used first), build the
//    polynomial on the device and move the request to the ready queue;
//    requests on a resident polynomial are ready at submit;
//  * the epoch thread, whenever one of its streams is free, packs ready
//    requests into one batch (persistent queue kernel, see batch.cu) in that
//    stream's reusable arena and launches it, so epochs on different streams
//    overlap on the GPU and requests that arrive meanwhile join the next one;
//  * completion: results go back by asynchronous copy into page-locked
//    buffers (others through a staging buffer) and tickets are marked done.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include "internal.h"

namespace pe {

using Clock = std::chrono::steady_clock;

struct SrvRequest {
    uint64_t ticket = 0;
    uint64_t resident_id = 0;         // 0: upload `desc`
    pe_poly_desc desc{};
    std::vector<uint64_t> coeffs;     // copies, unless the caller lends its arrays
    std::vector<uint8_t> exps;
    std::vector<uint64_t> beta;
    uint64_t T = 0, t0 = 0;
    uint64_t *out = nullptr;
    bool out_pinned = false;
    uint64_t reserved_id = 0;         // resident id of an upload, assigned at submit
    Clock::time_point submitted;
    pe_poly *poly = nullptr;          // once on the device
    uint64_t used_id = 0;             // store entry holding a reference for this request
    size_t out_off = 0, out_bytes = 0;
};

struct Resident {
    pe_poly *poly = nullptr;
    uint64_t bytes = 0;
    uint64_t last_use = 0;
    uint32_t refs = 0;                // queued or running requests using it
    bool pinned = false;              // registered by the client: never evicted
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf arena, outs;
    void *staging = nullptr;          // page-locked bounce buffer for pageable outputs
    size_t staging_bytes = 0;
    BatchImage img;
    std::vector<SrvRequest *> reqs;
    bool busy = false;
    double term_points = 0.0;
    uint64_t device_bytes = 0;        // arena + outs, published under the server mutex
};

static uint64_t poly_bytes_estimate(const pe_poly_desc &d)
{
    const uint64_t E = d.n >= 2 ? d.n - 2 : 0;
    return d.s * (8 + 8 + E * 2) + 4096;
}

// Epoch hold (see pe_server::launch).  Measured on the served mixture: paced
// streams ran with about half the p50 and a lower p99 at the same or higher
// rate, and bursts were no slower.
constexpr size_t kHoldJobs = 16;
constexpr double kHoldSeconds = 0.002;

static double since(Clock::time_point a) { return std::chrono::duration<double>(Clock::now() - a).count(); }

}  // namespace pe

using namespace pe;

struct pe_server {
    pe_server_cfg cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_upload;
    std::deque<SrvRequest *> backlog;   // new polynomials waiting for an upload thread
    std::deque<SrvRequest *> ready;     // on the device, waiting for an epoch
    std::unordered_map<uint64_t, int> status;   // ticket -> PE_PENDING / PE_OK / error
    std::unordered_map<uint64_t, Resident> store;
    uint64_t next_ticket = 1, next_id = 1, use_clock = 0;
    uint64_t resident_bytes = 0, reserved_bytes = 0;
    Slot slots[4];
    uint32_t nslots = 0;
    std::thread worker;
    std::vector<std::thread> uploaders;
    int uploading = 0;
    bool stop = false;
    bool paused = false;
    // statistics
    uint64_t submitted = 0, completed = 0, rejected = 0, epochs = 0, evictions = 0;
    std::vector<double> lat_ms;
    double term_points = 0.0, busy_s = 0.0;
    double t_upload = 0.0, t_plan = 0.0, t_launch = 0.0, t_finish = 0.0;
    Clock::time_point busy_since;
    int inflight = 0;
    bool shrink_wanted = false;        // set by an upload that cannot fit while nothing runs

    uint64_t slot_bytes() const
    {
        uint64_t b = 0;
        for (uint32_t i = 0; i < nslots; ++i) b += slots[i].device_bytes;
        return b;
    }

    uint64_t committed() const
    {
        uint64_t b = resident_bytes + reserved_bytes;
        for (uint32_t i = 0; i < nslots; ++i) b += slots[i].device_bytes;
        return b;
    }

    // Evicts unreferenced, unpinned residents (least recently used first) until
    // `need` more bytes fit under the cap.  Called with `mu` held.
    bool make_room(uint64_t need)
    {
        while (committed() + need > cfg.mem_cap_bytes) {
            uint64_t victim = 0, oldest = ~0ull;
            for (auto &kv : store)
                if (!kv.second.pinned && kv.second.refs == 0 && kv.second.last_use < oldest) {
                    oldest = kv.second.last_use;
                    victim = kv.first;
                }
            if (!victim) return false;
            Resident r = store[victim];
            store.erase(victim);
            resident_bytes -= r.bytes;
            destroy_idle(r.poly);          // refs == 0: the epochs that used it have completed
            ++evictions;
        }
        return true;
    }

    void release_ref(SrvRequest *r)    // with `mu` held
    {
        auto it = store.find(r->used_id);
        if (it != store.end() && it->second.refs) it->second.refs--;
    }

    void fail_locked(SrvRequest *r, int code)
    {
        release_ref(r);
        status[r->ticket] = code;
        delete r;
        cv_done.notify_all();
        cv_upload.notify_all();
    }

    // ---------------------------------------------------------------- uploads
    void upload_loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_upload.wait(lk, [&] { return stop || !backlog.empty(); });
            if (backlog.empty()) {
                if (stop) return;
                continue;
            }
            SrvRequest *r = backlog.front();
            const uint64_t need = poly_bytes_estimate(r->desc);
            if (!make_room(need)) {
                if (uploading == 0 && inflight == 0 && ready.empty() && slot_bytes() > 0) {
                    // Nothing runs: the epoch thread gives back the idle
                    // epochs' scratch (it grows again on demand), then retry.
                    shrink_wanted = true;
                    cv_work.notify_all();
                    cv_upload.wait_for(lk, std::chrono::milliseconds(1));
                    continue;
                }
                if (uploading == 0 && inflight == 0 && ready.empty()) {   // can never fit
                    backlog.pop_front();
                    ++rejected;
                    fail_locked(r, PE_ERR_ADMISSION);
                    continue;
                }
                cv_upload.wait_for(lk, std::chrono::milliseconds(1));     // wait for memory
                continue;
            }
            backlog.pop_front();
            reserved_bytes += need;
            ++uploading;
            lk.unlock();
            const Clock::time_point t0 = Clock::now();
            if (!(r->desc.flags & PE_FLAG_BORROW)) {
                r->desc.coeffs = r->coeffs.data();
                r->desc.exps = r->exps.data();
            }
            pe_poly *P = nullptr;
            // Host-side create: its only device work is the upload copies, which
            // do not wait for the epochs' kernels to leave the SMs.
            pe_status st = create_poly(&r->desc, &P, false, false);
            if (st == PE_OK && !out_ok(r->T, P->G)) {   // its output could not be addressed
                poly_eval_destroy(P);
                P = nullptr;
                st = PE_ERR_ARG;
            }
            std::vector<uint8_t>().swap(r->exps);
            std::vector<uint64_t>().swap(r->coeffs);
            const double dt = since(t0);
            lk.lock();
            --uploading;
            reserved_bytes -= need;
            t_upload += dt;
            if (st != PE_OK) {
                fail_locked(r, st);
                continue;
            }
            Resident res;
            res.poly = P;
            res.bytes = P->device_bytes();
            res.refs = 1;
            res.last_use = ++use_clock;
            store[r->reserved_id] = res;
            resident_bytes += res.bytes;
            r->poly = P;
            r->used_id = r->reserved_id;
            ready.push_back(r);
            cv_work.notify_one();
        }
    }

    // ------------------------------------------------------------- completion
    void finish(Slot &s)
    {
        const Clock::time_point now = Clock::now();
        for (SrvRequest *r : s.reqs)
            if (!r->out_pinned && r->out_bytes) memcpy(r->out, (unsigned char *)s.staging + r->out_off, r->out_bytes);
        std::lock_guard<std::mutex> lk(mu);
        for (SrvRequest *r : s.reqs) {
            release_ref(r);
            status[r->ticket] = PE_OK;
            lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->submitted).count());
            ++completed;
            delete r;
        }
        term_points += s.term_points;
        s.reqs.clear();
        s.busy = false;
        if (--inflight == 0) busy_s += std::chrono::duration<double>(now - busy_since).count();
        t_finish += since(now);
        cv_done.notify_all();
        cv_upload.notify_all();
    }

    void fail_all(std::vector<SrvRequest *> &reqs, int code)
    {
        std::lock_guard<std::mutex> lk(mu);
        for (SrvRequest *r : reqs) fail_locked(r, code);
        reqs.clear();
    }

    // ----------------------------------------------------------------- epochs
    // Packs ready requests into slot `s` and launches them as one epoch.
    bool launch(Slot &s)
    {
        std::vector<SrvRequest *> ok;
        {
            std::lock_guard<std::mutex> lk(mu);
            uint64_t need = 0;
            // While other epochs run, a small epoch waits briefly for more
            // requests: larger epochs use the GPU better, and the wait ends as
            // soon as kHoldJobs are ready or the oldest has waited kHoldSeconds.
            if (!stop && inflight > 0 && !ready.empty() && ready.size() < kHoldJobs &&
                std::chrono::duration<double>(Clock::now() - ready.front()->submitted).count() < kHoldSeconds)
                return false;
            while (!paused && !ready.empty() && ok.size() < cfg.max_epoch_jobs) {
                SrvRequest *r = ready.front();
                const uint64_t add = r->T * r->poly->G * 8 + r->poly->s * 24 + r->T * 1024;
                if (!make_room(need + add) && !ok.empty()) break;   // run what fits; a lone request always runs
                need += add;
                ready.pop_front();
                ok.push_back(r);
            }
        }
        if (ok.empty()) return false;
        const Clock::time_point t_pl0 = Clock::now();
        size_t total = 0;
        for (SrvRequest *r : ok) {
            r->out_bytes = r->T * r->poly->G * 8;
            r->out_off = total;
            total += (r->out_bytes + 255) / 256 * 256;
        }
        cudaError_t e = s.outs.ensure(std::max<size_t>(total, 256));
        bool need_staging = false;
        for (SrvRequest *r : ok) need_staging |= !r->out_pinned && r->out_bytes;
        if (e == cudaSuccess && need_staging && s.staging_bytes < total) {
            if (s.staging) cudaFreeHost(s.staging);
            s.staging = nullptr;
            s.staging_bytes = 0;
            e = cudaMallocHost(&s.staging, total);
            if (e == cudaSuccess) s.staging_bytes = total;
        }
        if (e != cudaSuccess) {
            cuda_fail(e, "server outputs");
            fail_all(ok, PE_ERR_NOMEM);
            return true;
        }
        std::vector<pe_job> jobs(ok.size());
        s.term_points = 0.0;
        for (size_t j = 0; j < ok.size(); ++j) {
            SrvRequest *r = ok[j];
            jobs[j].poly = r->poly;
            jobs[j].beta = r->beta.data();
            jobs[j].T = r->T;
            jobs[j].t0 = r->t0;
            jobs[j].out = (uint64_t *)(s.outs.as<unsigned char>() + r->out_off);
            s.term_points += (double)r->poly->s * (double)r->T;
        }
        // Every request runs in the epoch's queue kernel.  (Running requests of
        // at least 2^28 term-points as plain runs after it, as a batch does,
        // measured slower: 2,700-3,200 against 3,400-4,900 requests/s on bursts
        // of the served mixture; the large requests then stop sharing the SMs
        // with the small ones and each epoch ends on a lone plain run.)
        pe_status st = batch_build(jobs.data(), jobs.size(), s.arena, s.img, false);
        t_plan += since(t_pl0);
        const Clock::time_point t_la0 = Clock::now();
        if (st == PE_OK && (e = batch_enqueue(s.img, s.st)) != cudaSuccess) st = cuda_fail(e, "server epoch");
        for (size_t j = 0; st == PE_OK && j < ok.size(); ++j) {
            SrvRequest *r = ok[j];
            if (!r->out_bytes) continue;
            void *dst = r->out_pinned ? (void *)r->out : (void *)((unsigned char *)s.staging + r->out_off);
            if ((e = cudaMemcpyAsync(dst, jobs[j].out, r->out_bytes, cudaMemcpyDeviceToHost, s.st)) != cudaSuccess)
                st = cuda_fail(e, "server copy back");
        }
        if (st == PE_OK && (e = cudaEventRecord(s.done, s.st)) != cudaSuccess) st = cuda_fail(e, "server event");
        if (st != PE_OK) {
            cudaStreamSynchronize(s.st);
            fail_all(ok, st);
            return true;
        }
        s.reqs = ok;
        s.busy = true;
        t_launch += since(t_la0);
        std::lock_guard<std::mutex> lk(mu);
        s.device_bytes = s.arena.bytes + s.outs.bytes;   // the epoch thread alone resizes them
        if (inflight++ == 0) busy_since = Clock::now();
        ++epochs;
        return true;
    }

    void run()
    {
        cudaSetDevice(device);
        for (;;) {
            bool progressed = false;
            for (uint32_t i = 0; i < nslots; ++i) {
                Slot &s = slots[i];
                if (s.busy && cudaEventQuery(s.done) == cudaSuccess) {
                    finish(s);
                    progressed = true;
                } else if (s.busy) {
                    cudaGetLastError();   // clear cudaErrorNotReady
                }
            }
            for (uint32_t i = 0; i < nslots; ++i)
                if (!slots[i].busy && launch(slots[i])) progressed = true;
            std::unique_lock<std::mutex> lk(mu);
            if (shrink_wanted) {   // an upload cannot fit: release idle slots' device scratch
                shrink_wanted = false;
                for (uint32_t i = 0; i < nslots; ++i)
                    if (!slots[i].busy) {
                        slots[i].arena.release();
                        slots[i].outs.release();
                        slots[i].device_bytes = 0;
                    }
                cv_upload.notify_all();
            }
            bool any_busy = false;
            for (uint32_t i = 0; i < nslots; ++i) any_busy |= slots[i].busy;
            if (stop && backlog.empty() && ready.empty() && uploading == 0 && !any_busy) return;
            if (!progressed) {
                if (any_busy) {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                } else {
                    cv_work.wait_for(lk, std::chrono::milliseconds(2));
                }
            }
        }
    }
};

extern "C" pe_status poly_eval_server_create(const pe_server_cfg *cfg, pe_server **out)
{
    if (!out) {
        set_error("out is NULL");
        return PE_ERR_ARG;
    }
    *out = nullptr;
    pe_server *S = new pe_server();
    pe_server_cfg c{};
    if (cfg) c = *cfg;
    if (!c.mem_cap_bytes) c.mem_cap_bytes = 40ull << 30;
    if (!c.max_queue) c.max_queue = 4096;
    if (!c.max_epoch_jobs) c.max_epoch_jobs = 256;
    if (!c.streams) c.streams = 4;   // four epochs in flight: bursts ran 1.3x faster than with two
    c.streams = std::min<uint32_t>(c.streams, 4);
    S->cfg = c;
    cudaGetDevice(&S->device);
    S->nslots = c.streams;
    for (uint32_t i = 0; i < S->nslots; ++i) {
        Slot &s = S->slots[i];
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess) {
            delete S;
            return cuda_fail(e, "server streams");
        }
    }
    const unsigned nup = std::max(1u, std::min(8u, std::thread::hardware_concurrency() / 2));
    for (unsigned i = 0; i < nup; ++i) S->uploaders.emplace_back([S] { S->upload_loop(); });
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return PE_OK;
}

extern "C" pe_status poly_eval_server_register(pe_server *S, const pe_poly_desc *desc, uint64_t *resident_id)
{
    if (!S || !desc || !resident_id) {
        set_error("NULL argument");
        return PE_ERR_ARG;
    }
    pe_poly *P = nullptr;
    pe_status st = poly_eval_create(desc, &P);
    if (st != PE_OK) return st;
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->make_room(P->device_bytes())) {
        destroy_idle(P);
        set_error("resident store is full");
        return PE_ERR_ADMISSION;
    }
    Resident r;
    r.poly = P;
    r.bytes = P->device_bytes();
    r.pinned = true;
    r.last_use = ++S->use_clock;
    const uint64_t id = S->next_id++;
    S->store[id] = r;
    S->resident_bytes += r.bytes;
    *resident_id = id;
    return PE_OK;
}

extern "C" pe_status poly_eval_server_submit(pe_server *S, const pe_request *req, uint64_t *ticket)
{
    if (!S || !req || !ticket || !req->out || (!req->resident_id && !req->poly_desc)) {
        set_error("bad request");
        return PE_ERR_ARG;
    }
    if (!points_ok(req->T, req->t0)) return PE_ERR_ARG;
    SrvRequest *r = new SrvRequest();
    r->resident_id = req->resident_id;
    r->T = req->T;
    r->t0 = req->t0;
    r->out = req->out;
    cudaPointerAttributes a{};
    r->out_pinned = cudaPointerGetAttributes(&a, req->out) == cudaSuccess && a.type == cudaMemoryTypeHost;
    cudaGetLastError();
    uint32_t n = 0;
    if (!req->resident_id) {
        const pe_poly_desc &d = *req->poly_desc;
        if ((d.flags & PE_FLAG_DEVICE_PTRS) || (d.s && (!d.coeffs || !d.exps)) ||
            (d.exp_bytes != 1 && d.exp_bytes != 2 && d.exp_bytes != 4) || d.n < 2 || d.n > PE_MAX_VARS) {
            delete r;
            set_error("poly_desc must describe host arrays");
            return PE_ERR_ARG;
        }
        r->desc = d;
        const uint8_t *e = (const uint8_t *)d.exps;
        if (!(d.flags & PE_FLAG_BORROW)) {           // copy: the caller may reuse its arrays at once
            r->coeffs.assign(d.coeffs, d.coeffs + d.s);
            r->exps.assign(e, e + d.s * d.n * d.exp_bytes);
        }
        n = d.n;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (req->resident_id) {
        auto it = S->store.find(req->resident_id);
        if (it == S->store.end()) {
            delete r;
            set_error("unknown resident id");
            return PE_ERR_NOT_FOUND;
        }
        n = it->second.poly->n;
        if (!out_ok(req->T, it->second.poly->G)) {
            delete r;
            return PE_ERR_ARG;
        }
    }
    if (n > 2 && !req->beta) {
        delete r;
        set_error("beta is NULL");
        return PE_ERR_ARG;
    }
    if (S->backlog.size() + S->ready.size() >= S->cfg.max_queue) {
        ++S->rejected;
        delete r;
        set_error("queue full");
        return PE_ERR_ADMISSION;
    }
    if (n > 2) r->beta.assign(req->beta, req->beta + (n - 2));
    r->submitted = Clock::now();
    r->ticket = S->next_ticket++;
    S->status[r->ticket] = PE_PENDING;
    ++S->submitted;
    *ticket = r->ticket;
    if (req->resident_id) {
        Resident &res = S->store[req->resident_id];
        res.refs++;                         // keeps it resident until this request completes
        res.last_use = ++S->use_clock;
        r->poly = res.poly;
        r->used_id = req->resident_id;
        S->ready.push_back(r);
        S->cv_work.notify_one();
    } else {
        r->reserved_id = S->next_id++;
        if (req->new_resident_id) *req->new_resident_id = r->reserved_id;
        S->backlog.push_back(r);
        S->cv_upload.notify_one();
    }
    return PE_OK;
}

extern "C" pe_status poly_eval_server_poll(pe_server *S, uint64_t ticket, int64_t timeout_us)
{
    if (!S) {
        set_error("NULL server");
        return PE_ERR_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto done = [&] {
        auto it = S->status.find(ticket);
        return it == S->status.end() || it->second != PE_PENDING;
    };
    if (timeout_us < 0) S->cv_done.wait(lk, done);
    else if (timeout_us > 0) S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
    auto it = S->status.find(ticket);
    if (it == S->status.end()) {
        set_error("unknown ticket");
        return PE_ERR_NOT_FOUND;
    }
    const int st = it->second;
    if (st == PE_PENDING) return timeout_us == 0 ? PE_PENDING : PE_ERR_TIMEOUT;
    S->status.erase(it);
    return (pe_status)st;
}

extern "C" pe_status poly_eval_server_stats(pe_server *S, pe_server_stats *out)
{
    if (!S || !out) {
        set_error("NULL argument");
        return PE_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->epochs = S->epochs;
    out->term_points = S->term_points;
    out->busy_s = S->busy_s + (S->inflight ? since(S->busy_since) : 0);
    out->resident_bytes = S->resident_bytes;
    out->resident_polys = S->store.size();
    out->evictions = S->evictions;
    out->upload_s = S->t_upload;
    out->plan_s = S->t_plan;
    out->launch_s = S->t_launch;
    out->finish_s = S->t_finish;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
    }
    return PE_OK;
}

extern "C" pe_status poly_eval_server_pause(pe_server *S, int paused)
{
    if (!S) {
        set_error("NULL server");
        return PE_ERR_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->paused = paused != 0;
    }
    S->cv_work.notify_all();
    return PE_OK;
}

extern "C" void poly_eval_server_destroy(pe_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->paused = false;
    }
    S->cv_upload.notify_all();
    S->cv_work.notify_all();
    for (std::thread &t : S->uploaders)
        if (t.joinable()) t.join();
    if (S->worker.joinable()) S->worker.join();
    cudaDeviceSynchronize();
    for (uint32_t i = 0; i < S->nslots; ++i) {
        Slot &s = S->slots[i];
        if (s.staging) cudaFreeHost(s.staging);
        if (s.done) cudaEventDestroy(s.done);
        if (s.st) cudaStreamDestroy(s.st);
    }
    for (auto &kv : S->store) destroy_idle(kv.second.poly);
    for (SrvRequest *r : S->backlog) delete r;
    for (SrvRequest *r : S->ready) delete r;
    delete S;
}
