// Autotuner: times candidate tile shapes and modular products of the plain
// path on the current device and records the fastest for the polynomial's
// shape bucket (prime width, and log2 of s, T and the mean group size).  The
// paper tunes its (T_i, T_d, M) unrolling constants the same way, by
// measurement (Sect. 4.4); here the constants are the lane chunk size K, the
// warps per block and the modular product.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include "internal.h"
#include "tune.h"

namespace pe {

static std::mutex g_tune_mu;
static std::map<std::string, TuneEntry> g_tune;

static int lg(double x) { return (int)std::lround(std::log2(std::max(1.0, x))); }

std::string tune_key(const pe_poly *P, uint64_t T)
{
    char buf[96];
    snprintf(buf, sizeof buf, "p%d|s%d|T%d|gs%d", P->p < (1ull << 30) ? 30 : P->p < (1ull << 50) ? 50 : 62,
             lg((double)P->s), lg((double)T),
             lg((double)P->s / (double)std::max<uint64_t>(1, P->G)));
    return buf;
}

const TuneEntry *tune_lookup(const pe_poly *P, uint64_t T)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(P, T));
    return it == g_tune.end() ? nullptr : &it->second;
}

int default_variant(uint64_t p) { return p < (1ull << 30) ? PE_MODMUL_BARRETT32 : PE_MODMUL_BARRETT64; }

int run_variant(pe_poly *P, uint64_t T)
{
    if (P->requested_variant != PE_MODMUL_AUTO) return P->requested_variant;
    const TuneEntry *te = tune_lookup(P, T);
    return te ? te->variant : default_variant(P->p);
}

}  // namespace pe

using namespace pe;

extern "C" pe_status poly_eval_tune(pe_poly *P, uint64_t T, pe_tiles *best, double *best_ms)
{
    if (!P || T == 0) {
        set_error("bad argument");
        return PE_ERR_ARG;
    }
    if (P->G == 0) {
        set_error("empty polynomial");
        return PE_ERR_ARG;
    }
    if (!points_ok(T, 1) || !out_ok(T, P->G)) return PE_ERR_ARG;
    std::vector<uint64_t> beta(std::max<uint32_t>(P->E, 1));
    for (size_t j = 0; j < beta.size(); ++j) beta[j] = 2 + (j * 7919) % (P->p - 3);
    DevBuf out;
    cudaError_t e = out.ensure(T * P->G * 8);
    if (e != cudaSuccess) return cuda_fail(e, "tune output");
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const pe_tiles saved_tiles = P->forced;
    const int saved_req = P->requested_variant;
    std::vector<int> variants = {PE_MODMUL_BARRETT64, PE_MODMUL_MONT64};
    if (P->p < (1ull << 50)) variants.push_back(PE_MODMUL_FP64);
    if (P->p < (1ull << 30)) variants.push_back(PE_MODMUL_BARRETT32);
    if (saved_req != PE_MODMUL_AUTO) variants = {saved_req};
    TuneEntry bestE;
    bestE.ms = 1e300;
    pe_status result = PE_OK;
    for (int v : variants) {
        for (uint32_t K : {1u, 2u, 4u, 8u, 12u, 16u}) {
            for (uint32_t wpb : {2u, 4u}) {
                pe_tiles t{};
                t.K = K;
                t.warps_per_block = wpb;
                P->forced = t;
                P->requested_variant = v;
                P->plan.valid = false;
                P->tail_plan.valid = false;
                pe_status s = run_matrix(P, beta.data(), T, 1, out.as<uint64_t>(), st);  // warm-up + plan
                if (s != PE_OK) {
                    result = s;
                    break;
                }
                cudaEventRecord(a, st);
                for (int r = 0; r < 3; ++r) run_matrix(P, beta.data(), T, 1, out.as<uint64_t>(), st);
                cudaEventRecord(b, st);
                if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
                    result = cuda_fail(e, "tune");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (ms / 3.0 < bestE.ms) {
                    bestE.ms = ms / 3.0;
                    bestE.K = K;
                    bestE.wpb = wpb;
                    bestE.variant = v;
                }
            }
            if (result != PE_OK) break;
        }
        if (result != PE_OK) break;
    }
    // Item shape for the best product and chunk size: a few measured shapes
    // around the rule's (slabs per item, points per item, tail band).
    if (result == PE_OK) {
        const uint32_t cand[][3] = {{1, 128, 0}, {2, 128, 0}, {1, 224, 128}, {2, 224, 128}, {1, 256, 0},
                                    {2, 256, 0}, {1, 512, 0}, {2, 448, 128}};
        for (const auto &c : cand) {
            if (c[1] + c[2] > T) continue;
            pe_tiles ft{};
            ft.K = bestE.K;
            ft.warps_per_block = bestE.wpb;
            ft.slabs = c[0];
            ft.tchunk = c[1];
            ft.tail = c[2];
            P->forced = ft;
            P->requested_variant = bestE.variant;
            P->plan.valid = false;
            P->tail_plan.valid = false;
            pe_status s = run_matrix(P, beta.data(), T, 1, out.as<uint64_t>(), st);
            if (s != PE_OK) {
                result = s;
                break;
            }
            cudaEventRecord(a, st);
            for (int r = 0; r < 3; ++r) run_matrix(P, beta.data(), T, 1, out.as<uint64_t>(), st);
            cudaEventRecord(b, st);
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
                result = cuda_fail(e, "tune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms / 3.0 < bestE.ms * 0.995) {
                bestE.ms = ms / 3.0;
                bestE.kslabs = c[0];
                bestE.Tc = c[1];
                bestE.tail = c[2];
            }
        }
    }
    P->forced = saved_tiles;
    P->requested_variant = saved_req;
    P->plan.valid = false;
    P->tail_plan.valid = false;
    // The fast method (Sect. 2.3.1) where the prime allows it.
    if (result == PE_OK && saved_req == PE_MODMUL_AUTO && fast_applicable(P->p, T)) {
        pe_status s = poly_eval_run_fast(P, beta.data(), T, 1, out.as<uint64_t>(), st);
        if (s == PE_OK) {
            cudaEventRecord(a, st);
            for (int r = 0; r < 3; ++r) poly_eval_run_fast(P, beta.data(), T, 1, out.as<uint64_t>(), st);
            cudaEventRecord(b, st);
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
                result = cuda_fail(e, "tune");
            } else {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (ms / 3.0 < bestE.ms) {
                    bestE.ms = ms / 3.0;
                    bestE.method = 1;
                }
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    if (result != PE_OK) return result;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(P, T)] = bestE;
    }
    if (best) {
        pe_tiles f{};
        const Tiles t = choose_tiles(P, T, &f);
        best->K = t.K;
        best->slabs = t.kslabs;
        best->tchunk = t.Tc;
        best->warps_per_block = t.wpb;
    }
    if (best_ms) *best_ms = bestE.ms;
    return PE_OK;
}

extern "C" pe_status poly_eval_tune_save(const char *path)
{
    if (!path) {
        set_error("NULL path");
        return PE_ERR_ARG;
    }
    std::ofstream f(path);
    if (!f) {
        set_error("cannot write %s", path);
        return PE_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &kv : g_tune)
        f << "{\"key\": \"" << kv.first << "\", \"K\": " << kv.second.K << ", \"wpb\": " << kv.second.wpb
          << ", \"variant\": " << kv.second.variant << ", \"ms\": " << kv.second.ms << ", \"slabs\": "
          << kv.second.kslabs << ", \"tchunk\": " << kv.second.Tc << ", \"tail\": " << kv.second.tail
          << ", \"method\": " << kv.second.method << "}\n";
    return PE_OK;
}

extern "C" pe_status poly_eval_tune_load(const char *path)
{
    if (!path) {
        set_error("NULL path");
        return PE_ERR_ARG;
    }
    std::ifstream f(path);
    if (!f) {
        set_error("cannot read %s", path);
        return PE_ERR_ARG;
    }
    std::string line;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    while (std::getline(f, line)) {
        const size_t k0 = line.find("\"key\": \"");
        if (k0 == std::string::npos) continue;
        const size_t k1 = line.find('"', k0 + 8);
        TuneEntry t;
        unsigned K = 0, w = 0;
        int v = 0;
        double ms = 0;
        const size_t r = line.find("\"K\":");
        if (r == std::string::npos ||
            sscanf(line.c_str() + r, "\"K\": %u, \"wpb\": %u, \"variant\": %d, \"ms\": %lf", &K, &w, &v, &ms) != 4)
            continue;
        if ((K != 1 && K != 2 && K != 4 && K != 8 && K != 12 && K != 16) || w < 1 || w > 8 || v < 1 || v > 4) continue;
        t.K = K;
        t.wpb = w;
        t.variant = v;
        t.ms = ms;
        unsigned ks = 0, tc = 0, tl = 0;
        const size_t sp = line.find("\"slabs\":");
        if (sp != std::string::npos &&
            sscanf(line.c_str() + sp, "\"slabs\": %u, \"tchunk\": %u, \"tail\": %u", &ks, &tc, &tl) == 3) {
            t.kslabs = ks;
            t.Tc = tc;
            t.tail = tl;
        }
        unsigned meth = 0;
        const size_t mp = line.find("\"method\":");
        if (mp != std::string::npos && sscanf(line.c_str() + mp, "\"method\": %u", &meth) == 1 && meth <= 1)
            t.method = meth;
        g_tune[line.substr(k0 + 8, k1 - k0 - 8)] = t;
    }
    return PE_OK;
}
