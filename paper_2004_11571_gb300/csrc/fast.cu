// The asymptotically fast method (Sect. 2.3.1): the T images of a group from
// O(s log^2 T) products instead of the matrix method's s*T, for primes with
// p - 1 divisible by a power of two larger than 2T (so that NTTs of that
// order exist in F_p).
//
// For a group with terms y_i = a_i m_i^t0 (values at the first point) and
// monomial values m_i,
//     sum_{r>=0} b_(t0+r) z^r = sum_i y_i / (1 - m_i z) = N(z) / D(z),
// with D = prod_i (1 - m_i z) and deg N < deg D.  The group's terms are cut
// into blocks of B = Tp terms (Tp: T rounded up to a power of two, at least
// 64); every block's N/D comes from a product tree, its first T series
// coefficients from a Newton inversion of D, and the blocks of a group add up:
//   k_fast_leaf   : leaves 1 - m_i z and y_i, then the tree up to 32 terms per
//                   warp in shared memory (schoolbook, one output per lane)
//   k_fast_merge  : one tree level above 32 terms: N = Na Db + Nb Da and
//                   D = Da Db by NTTs of size 2L (cyclic; the one coefficient
//                   that wraps, the leading one of D, is computed directly)
//   k_fast_series : h = 1/D mod z^Tp by Newton (h <- h - z^k h (D h)_[k,2k)),
//                   then N h mod z^T
//   k_fast_sum    : the blocks of each group added, converted to [0, p)
// Values are in Montgomery form (x * 2^64 mod p), kept in [0, 2p); NTT
// twiddles are plain residues used by Shoup's fixed-multiplier product.
#include <algorithm>
#include <vector>
#include "internal.h"
#include "modarith.cuh"
#include "kernels.h"

namespace pe {

constexpr uint32_t kFastChunk = 32;
constexpr uint32_t kFastMaxT = 4096;
constexpr int kFastThreads = 512;

struct FastTab {
    const uint64_t *W, *Wq;     // w^j and Shoup quotients, j < Nmax/2 (w of order Nmax)
    const uint64_t *Wi, *Wiq;   // w^-j
    const uint64_t *ninv;       // [2 * log2 N]: N^-1 and its Shoup quotient
    uint32_t lognmax;
};

struct FastChunkT {
    uint32_t off, cnt;
};
struct FastPairT {
    uint32_t off, la, lb, pad;
};
struct FastBlockT {
    uint32_t off, d, parity, pad;
};

__device__ __forceinline__ uint64_t lazy2(uint64_t x, uint64_t p2) { return x >= p2 ? x - p2 : x; }

// Shoup's product x*w mod p for a twiddle w (wq = floor(w 2^64 / p)), in [0, 2p).
__device__ __forceinline__ uint64_t twmul(uint64_t x, uint64_t w, uint64_t wq, const ModCtx &mc)
{
    return lazy2(barrett_mul_lazy4_mad(x, w, wq, 0 - mc.p), mc.p2);
}

// Forward NTT (decimation in frequency, natural order in, bit-reversed out) of
// NA arrays of size N = 2^logN in shared memory, values in [0, 2p).  Two
// stages per pass (radix 4: the stage of half-size h, then h/2, on the four
// points s+j, s+j+h/2, s+j+h, s+j+3h/2), after one radix-2 stage if logN is odd.
template <int NA>
__device__ void ntt_fwd(uint64_t *const *arr, uint32_t logN, const FastTab &tb, const ModCtx &mc)
{
    const uint64_t p2 = mc.p2;
    const uint32_t N = 1u << logN;
    int logh = (int)logN - 1;
    if (logN & 1) {
        const uint32_t h = 1u << logh, sh = tb.lognmax - (uint32_t)(logh + 1);
        for (uint32_t j = threadIdx.x; j < h; j += blockDim.x) {
            const uint64_t w = tb.W[j << sh], wq = tb.Wq[j << sh];
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                uint64_t *a = arr[k];
                const uint64_t u = a[j], v = a[j + h];
                a[j] = lazy2(u + v, p2);
                a[j + h] = twmul(u - v + p2, w, wq, mc);
            }
        }
        __syncthreads();
        --logh;
    }
    for (; logh >= 1; logh -= 2) {
        const uint32_t h = 1u << logh, q = h >> 1;
        const uint32_t sh1 = tb.lognmax - (uint32_t)(logh + 1), sh2 = tb.lognmax - (uint32_t)logh;
        for (uint32_t b = threadIdx.x; b < N / 4; b += blockDim.x) {
            const uint32_t j = b & (q - 1), s = (b - j) << 2;
            const uint64_t w1 = tb.W[j << sh1], w1q = tb.Wq[j << sh1];
            const uint64_t w3 = tb.W[(j + q) << sh1], w3q = tb.Wq[(j + q) << sh1];
            const uint64_t w2 = tb.W[j << sh2], w2q = tb.Wq[j << sh2];
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                uint64_t *a = arr[k] + s + j;
                const uint64_t a0 = a[0], a1 = a[q], a2 = a[2 * q], a3 = a[3 * q];
                const uint64_t b0 = lazy2(a0 + a2, p2), b2 = twmul(a0 - a2 + p2, w1, w1q, mc);
                const uint64_t b1 = lazy2(a1 + a3, p2), b3 = twmul(a1 - a3 + p2, w3, w3q, mc);
                a[0] = lazy2(b0 + b1, p2);
                a[q] = twmul(b0 - b1 + p2, w2, w2q, mc);
                a[2 * q] = lazy2(b2 + b3, p2);
                a[3 * q] = twmul(b2 - b3 + p2, w2, w2q, mc);
            }
        }
        __syncthreads();
    }
}

// Inverse NTT (decimation in time, bit-reversed in, natural out), scaled by
// N^-1; radix 4 as above (stages of half-size q, then 2q), after one radix-2
// stage of half-size 1 (twiddle 1) if logN is odd.
template <int NA>
__device__ void ntt_inv(uint64_t *const *arr, uint32_t logN, const FastTab &tb, const ModCtx &mc)
{
    const uint64_t p2 = mc.p2;
    const uint32_t N = 1u << logN;
    uint32_t logh = 0;
    if (logN & 1) {
        for (uint32_t b = threadIdx.x; b < N / 2; b += blockDim.x) {
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                uint64_t *a = arr[k] + 2 * b;
                const uint64_t u = a[0], v = a[1];
                a[0] = lazy2(u + v, p2);
                a[1] = lazy2(u - v + p2, p2);
            }
        }
        __syncthreads();
        logh = 1;
    }
    for (; logh < logN; logh += 2) {
        const uint32_t q = 1u << logh;
        const uint32_t shq = tb.lognmax - (logh + 1), shh = tb.lognmax - (logh + 2);
        for (uint32_t b = threadIdx.x; b < N / 4; b += blockDim.x) {
            const uint32_t j = b & (q - 1), s = (b - j) << 2;
            const uint64_t wa = tb.Wi[j << shq], waq = tb.Wiq[j << shq];
            const uint64_t wb = tb.Wi[j << shh], wbq = tb.Wiq[j << shh];
            const uint64_t wc = tb.Wi[(j + q) << shh], wcq = tb.Wiq[(j + q) << shh];
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                uint64_t *a = arr[k] + s + j;
                const uint64_t a0 = a[0], a2 = a[2 * q];
                const uint64_t v1 = twmul(a[q], wa, waq, mc), v3 = twmul(a[3 * q], wa, waq, mc);
                const uint64_t b0 = lazy2(a0 + v1, p2), b1 = lazy2(a0 - v1 + p2, p2);
                const uint64_t b2 = lazy2(a2 + v3, p2), b3 = lazy2(a2 - v3 + p2, p2);
                const uint64_t v2 = twmul(b2, wb, wbq, mc), v4 = twmul(b3, wc, wcq, mc);
                a[0] = lazy2(b0 + v2, p2);
                a[2 * q] = lazy2(b0 - v2 + p2, p2);
                a[q] = lazy2(b1 + v4, p2);
                a[3 * q] = lazy2(b1 - v4 + p2, p2);
            }
        }
        __syncthreads();
    }
    const uint64_t ni = tb.ninv[2 * logN], niq = tb.ninv[2 * logN + 1];
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < NA; ++k) arr[k][i] = twmul(arr[k][i], ni, niq, mc);
    __syncthreads();
}

// Leaves and the first five tree levels, one warp per chunk of up to 32 terms
// of a block.  Node [a, a+d) keeps D_1..D_d at a..a+d-1 (D_0 = 1 implicit) and
// N_0..N_(d-1) at a..a+d-1.  At level L, lane k of a pair starting at q*2L
// computes D_(kk+1) and N_kk, kk = k - q*2L, from the two children.
__global__ void __launch_bounds__(128) k_fast_leaf(const FastChunkT *__restrict__ chunks, uint32_t nchunks,
                                                   const uint64_t *__restrict__ mR,
                                                   const uint64_t *__restrict__ coeffs, uint64_t t0, ModCtx mc,
                                                   uint64_t r2, uint64_t *__restrict__ Dout, uint64_t *__restrict__ Nout)
{
    __shared__ uint64_t sD[4][kFastChunk], sN[4][kFastChunk];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t c = blockIdx.x * 4 + w;
    if (c >= nchunks) return;   // whole warp
    const FastChunkT ch = chunks[c];
    const uint64_t p = mc.p;
    uint64_t *D = sD[w], *N = sN[w];
    if (lane < ch.cnt) {
        const uint64_t m = canon(mR[ch.off + lane], p);
        const uint64_t cR = canon(mont_mul(coeffs[ch.off + lane], r2, mc), p);
        D[lane] = m ? p - m : 0;                               // 1 - m z
        N[lane] = mont_mul(cR, mont_pow(m, t0, mc), mc);       // y = a m^t0
    } else {
        D[lane] = 0;
        N[lane] = 0;
    }
    __syncwarp();
    for (uint32_t L = 1; L < kFastChunk; L *= 2) {
        const uint32_t a0 = lane / (2 * L) * (2 * L), kk = lane - a0;
        const uint32_t la = ch.cnt > a0 ? min(L, ch.cnt - a0) : 0;
        const uint32_t lb = ch.cnt > a0 + la ? min(L, ch.cnt - a0 - la) : 0;
        uint64_t nd = D[lane], nn = N[lane];
        if (lb && kk < la + lb) {
            // D_(kk+1) = sum Da_i Db_(kk+1-i), Da_0 = Db_0 = 1 (r1 in Montgomery form)
            const uint32_t kd = kk + 1;
            uint64_t l = 0, m = 0;
            uint32_t h = 0;
            for (uint32_t i = kd > lb ? kd - lb : 0; i <= min(kd, la); ++i) {
                const uint64_t da = i ? D[a0 + i - 1] : mc.r1;
                const uint64_t db = kd - i ? D[a0 + L + kd - i - 1] : mc.r1;
                mac192(l, m, h, da, db);
            }
            nd = reduce192(l, m, h, r2, mc);
            l = m = 0;
            h = 0;
            // N_kk = sum Na_i Db_(kk-i) + sum Nb_i Da_(kk-i)
            for (uint32_t i = kk > lb ? kk - lb : 0; i <= min(kk, la - 1); ++i) {
                const uint64_t db = kk - i ? D[a0 + L + kk - i - 1] : mc.r1;
                mac192(l, m, h, N[a0 + i], db);
            }
            for (uint32_t i = kk > la ? kk - la : 0; i <= min(kk, lb - 1); ++i) {
                const uint64_t da = kk - i ? D[a0 + kk - i - 1] : mc.r1;
                mac192(l, m, h, N[a0 + L + i], da);
            }
            nn = reduce192(l, m, h, r2, mc);
        }
        __syncwarp();
        D[lane] = nd;
        N[lane] = nn;
        __syncwarp();
    }
    if (lane < ch.cnt) {
        Dout[ch.off + lane] = D[lane];
        Nout[ch.off + lane] = N[lane];
    }
}

// One tree level above 32 terms: the pair's children have degrees la, lb <= L.
__global__ void __launch_bounds__(kFastThreads) k_fast_merge(const FastPairT *__restrict__ pairs, uint32_t logL,
                                                             const uint64_t *__restrict__ Din,
                                                             const uint64_t *__restrict__ Nin,
                                                             uint64_t *__restrict__ Dout, uint64_t *__restrict__ Nout,
                                                             FastTab tb, ModCtx mc)
{
    extern __shared__ uint64_t sm[];
    const FastPairT pr = pairs[blockIdx.x];
    const uint32_t L = 1u << logL, N2 = 2 * L;
    const uint64_t p = mc.p, p2 = mc.p2;
    if (pr.lb == 0) {   // no partner: copied (uniform over the block)
        for (uint32_t i = threadIdx.x; i < pr.la; i += blockDim.x) {
            Dout[pr.off + i] = Din[pr.off + i];
            Nout[pr.off + i] = Nin[pr.off + i];
        }
        return;
    }
    uint64_t *X = sm, *Y = sm + N2, *C = sm + 2 * N2, *E = sm + 3 * N2;
    const uint64_t *Da = Din + pr.off, *Db = Din + pr.off + pr.la;
    const uint64_t *Na = Nin + pr.off, *Nb = Nin + pr.off + pr.la;
    for (uint32_t i = threadIdx.x; i < N2; i += blockDim.x) {
        X[i] = i == 0 ? mc.r1 : (i <= pr.la ? Da[i - 1] : 0);
        Y[i] = i == 0 ? mc.r1 : (i <= pr.lb ? Db[i - 1] : 0);
        C[i] = i < pr.la ? Na[i] : 0;
        E[i] = i < pr.lb ? Nb[i] : 0;
    }
    __syncthreads();
    {
        uint64_t *const arr[4] = {X, Y, C, E};
        ntt_fwd<4>(arr, logL + 1, tb, mc);
    }
    for (uint32_t i = threadIdx.x; i < N2; i += blockDim.x) {
        const uint64_t x = X[i], y = Y[i];
        C[i] = lazy2(mont_mul(C[i], y, mc) + mont_mul(E[i], x, mc), p2);
        X[i] = mont_mul(x, y, mc);
    }
    __syncthreads();
    {
        uint64_t *const arr[2] = {X, C};
        ntt_inv<2>(arr, logL + 1, tb, mc);
    }
    const uint32_t d = pr.la + pr.lb;
    for (uint32_t k = threadIdx.x; k < d; k += blockDim.x) {
        // D_(k+1): index 2L wraps onto 0 in the cyclic product, so the leading
        // coefficient of a full-size pair is the product of the children's.
        Dout[pr.off + k] = k + 1 < N2 ? X[k + 1] : mont_mul(Da[pr.la - 1], Db[pr.lb - 1], mc);
        Nout[pr.off + k] = C[k];
    }
}

// One block of a group: Newton inversion of D modulo z^Tp, then the first T
// coefficients of N/D, written to series[block][0..T).
__global__ void __launch_bounds__(kFastThreads) k_fast_series(const FastBlockT *__restrict__ blocks,
                                                              uint32_t logTp, uint32_t T,
                                                              const uint64_t *__restrict__ D0,
                                                              const uint64_t *__restrict__ N0,
                                                              const uint64_t *__restrict__ D1,
                                                              const uint64_t *__restrict__ N1,
                                                              uint64_t *__restrict__ series, FastTab tb, ModCtx mc)
{
    extern __shared__ uint64_t sm[];
    const FastBlockT bk = blocks[blockIdx.x];
    const uint32_t Tp = 1u << logTp;
    const uint64_t p = mc.p, p2 = mc.p2;
    const uint64_t *D = (bk.parity ? D1 : D0) + bk.off, *Nn = (bk.parity ? N1 : N0) + bk.off;
    uint64_t *h = sm, *X = sm + Tp, *Y = sm + 3 * Tp;
    if (threadIdx.x == 0) h[0] = mc.r1;
    __syncthreads();
    for (uint32_t logk = 0; logk < logTp; ++logk) {
        const uint32_t k = 1u << logk;
        // e = (D mod z^2k) * h with a cyclic product of size 2k: the product has
        // degree < 3k, so only its coefficients [0, k) wrap and e_[k,2k) is exact.
        for (uint32_t i = threadIdx.x; i < 2 * k; i += blockDim.x) {
            X[i] = i == 0 ? mc.r1 : (i <= bk.d ? D[i - 1] : 0);
            Y[i] = i < k ? h[i] : 0;
        }
        __syncthreads();
        {
            uint64_t *const arr[2] = {X, Y};
            ntt_fwd<2>(arr, logk + 1, tb, mc);
        }
        for (uint32_t i = threadIdx.x; i < 2 * k; i += blockDim.x) X[i] = mont_mul(X[i], Y[i], mc);
        __syncthreads();
        {
            uint64_t *const arr[1] = {X};
            ntt_inv<1>(arr, logk + 1, tb, mc);
        }
        // g = h * e_[k,2k) mod z^k, reusing the transform of h (still in Y).
        for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) X[i] = X[k + i];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) X[k + i] = 0;
        __syncthreads();
        {
            uint64_t *const arr[1] = {X};
            ntt_fwd<1>(arr, logk + 1, tb, mc);
        }
        for (uint32_t i = threadIdx.x; i < 2 * k; i += blockDim.x) X[i] = mont_mul(X[i], Y[i], mc);
        __syncthreads();
        {
            uint64_t *const arr[1] = {X};
            ntt_inv<1>(arr, logk + 1, tb, mc);
        }
        for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) h[k + i] = X[i] ? p2 - X[i] : 0;
        __syncthreads();
    }
    // N * h mod z^T, size 2Tp
    for (uint32_t i = threadIdx.x; i < 2 * Tp; i += blockDim.x) {
        X[i] = i < bk.d ? Nn[i] : 0;
        Y[i] = i < Tp ? h[i] : 0;
    }
    __syncthreads();
    {
        uint64_t *const arr[2] = {X, Y};
        ntt_fwd<2>(arr, logTp + 1, tb, mc);
    }
    for (uint32_t i = threadIdx.x; i < 2 * Tp; i += blockDim.x) X[i] = mont_mul(X[i], Y[i], mc);
    __syncthreads();
    {
        uint64_t *const arr[1] = {X};
        ntt_inv<1>(arr, logTp + 1, tb, mc);
    }
    for (uint32_t r = threadIdx.x; r < T; r += blockDim.x) series[(uint64_t)blockIdx.x * T + r] = X[r];
}

// out[r][g] = sum of the series of g's blocks, in [0, p).
__global__ void k_fast_sum(const uint32_t *__restrict__ gblk, uint64_t G, uint32_t T,
                           const uint64_t *__restrict__ series, uint64_t *__restrict__ out, ModCtx mc)
{
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G * T) return;
    const uint64_t g = idx / T, r = idx - g * T;
    uint64_t acc = 0;
    for (uint32_t b = gblk[g]; b < gblk[g + 1]; ++b) acc = lazy2(acc + series[(uint64_t)b * T + r], mc.p2);
    out[r * G + g] = canon(mont_redc(acc, 0, mc), mc.p);
}

// ------------------------------------------------------------------ host side

static uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((unsigned __int128)a * b % p); }
static uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t p)
{
    uint64_t r = 1 % p;
    for (b %= p; e; e >>= 1, b = mulmod_h(b, b, p))
        if (e & 1) r = mulmod_h(r, b, p);
    return r;
}
static uint64_t shoup_q(uint64_t w, uint64_t p) { return (uint64_t)(((unsigned __int128)w << 64) / p); }

}  // namespace pe

// Per-(polynomial, T) state of the fast method: the block structure, tile
// lists, twiddle tables and scratch.
struct FastPlan {
    uint64_t T = 0, p = 0;
    uint32_t logTp = 0, lognmax = 0;
    uint32_t nchunks = 0, nblocks = 0;
    size_t pairs_at = 0, blocks_at = 0;   // byte offsets in `tiles` (chunks first)
    std::vector<uint32_t> level_count;    // pairs per merge level (L = 32 * 2^level)
    std::vector<size_t> level_at;
    pe::DevBuf tiles, tables, gblk, D0, N0, D1, N1, series, out_scratch;
};

void fast_plan_delete(FastPlan *f) { delete f; }

using namespace pe;

static bool fast_applicable(uint64_t p, uint64_t T, uint32_t *logTp);

namespace pe {
bool fast_applicable(uint64_t p, uint64_t T)
{
    uint32_t l;
    return ::fast_applicable(p, T, &l);
}
}  // namespace pe

static bool fast_applicable(uint64_t p, uint64_t T, uint32_t *logTp)
{
    uint32_t lt = 6;
    while ((1ull << lt) < T) ++lt;
    *logTp = lt;
    const uint64_t nmax = 2ull << lt;
    return T >= 1 && T <= kFastMaxT && (p - 1) % nmax == 0;
}

static pe_status fast_prepare(pe_poly *P, uint64_t T, cudaStream_t st)
{
    FastPlan *F = P->fast.get();
    if (F && F->T == T && F->p == P->p) return PE_OK;
    if (!F) {
        P->fast.reset(new FastPlan());
        F = P->fast.get();
    }
    uint32_t logTp;
    fast_applicable(P->p, T, &logTp);
    const uint64_t p = P->p, Tp = 1ull << logTp, B = Tp;
    F->T = 0;   // set once everything below has succeeded
    F->p = 0;
    F->logTp = logTp;
    F->lognmax = logTp + 1;
    // Blocks of at most B terms per group; chunks of 32 within blocks; pairs per level.
    std::vector<FastBlockT> blocks;
    std::vector<uint32_t> gblk(P->G + 1);
    for (uint64_t g = 0; g < P->G; ++g) {
        gblk[g] = (uint32_t)blocks.size();
        for (uint64_t a = P->group_off[g]; a < P->group_off[g + 1]; a += B) {
            const uint32_t d = (uint32_t)std::min<uint64_t>(B, P->group_off[g + 1] - a);
            uint32_t levels = 0;
            for (uint64_t L = kFastChunk; L < d; L *= 2) ++levels;
            blocks.push_back({(uint32_t)a, d, levels & 1u, 0});
        }
    }
    gblk[P->G] = (uint32_t)blocks.size();
    std::vector<FastChunkT> chunks;
    for (const FastBlockT &b : blocks)
        for (uint32_t c = 0; c < b.d; c += kFastChunk) chunks.push_back({b.off + c, std::min(kFastChunk, b.d - c)});
    std::vector<FastPairT> pairs;
    F->level_count.clear();
    F->level_at.clear();
    for (uint64_t L = kFastChunk; L < B; L *= 2) {
        F->level_at.push_back(pairs.size());
        for (const FastBlockT &b : blocks)
            if (b.d > L)
                for (uint64_t ps = 0; ps < b.d; ps += 2 * L) {
                    const uint32_t la = (uint32_t)std::min<uint64_t>(L, b.d - ps);
                    const uint32_t lb = (uint32_t)std::min<uint64_t>(L, b.d - ps - la);
                    pairs.push_back({(uint32_t)(b.off + ps), la, lb, 0});
                }
        F->level_count.push_back((uint32_t)(pairs.size() - F->level_at.back()));
    }
    F->nchunks = (uint32_t)chunks.size();
    F->nblocks = (uint32_t)blocks.size();
    // Twiddles: w of order Nmax = 2Tp from an element whose power has order 2^e.
    const uint64_t nmax = 2 * Tp;
    uint64_t q = p - 1;
    uint32_t e2 = 0;
    while (!(q & 1)) {
        q >>= 1;
        ++e2;
    }
    uint64_t w = 0;
    for (uint64_t x = 2; x < 1000 && !w; ++x) {
        const uint64_t c = powmod_h(x, q, p);
        if (powmod_h(c, 1ull << (e2 - 1), p) == p - 1) w = powmod_h(c, 1ull << (e2 - F->lognmax), p);
    }
    if (!w) {
        set_error("no element of order 2^%u found: is p prime?", e2);
        return PE_ERR_PRIME;
    }
    const uint64_t half = nmax / 2, winv = powmod_h(w, p - 2, p);
    std::vector<uint64_t> tab(4 * half + 2 * (F->lognmax + 1), 0);
    uint64_t wj = 1, wij = 1;
    for (uint64_t j = 0; j < half; ++j) {
        tab[j] = wj;
        tab[half + j] = shoup_q(wj, p);
        tab[2 * half + j] = wij;
        tab[3 * half + j] = shoup_q(wij, p);
        wj = mulmod_h(wj, w, p);
        wij = mulmod_h(wij, winv, p);
    }
    for (uint32_t l = 1; l <= F->lognmax; ++l) {
        const uint64_t ni = powmod_h((1ull << l) % p, p - 2, p);
        tab[4 * half + 2 * l] = ni;
        tab[4 * half + 2 * l + 1] = shoup_q(ni, p);
    }
    auto al16 = [](size_t x) { return (x + 15) / 16 * 16; };
    F->pairs_at = al16(chunks.size() * sizeof(FastChunkT));
    F->blocks_at = al16(F->pairs_at + pairs.size() * sizeof(FastPairT));
    const size_t tile_bytes = F->blocks_at + blocks.size() * sizeof(FastBlockT);
    cudaError_t err;
    if ((err = F->tiles.ensure_async(std::max<size_t>(tile_bytes, 16), st)) != cudaSuccess ||
        (err = F->tables.ensure_async(tab.size() * 8, st)) != cudaSuccess ||
        (err = F->gblk.ensure_async(gblk.size() * 4, st)) != cudaSuccess ||
        (err = F->D0.ensure_async(P->s * 8, st)) != cudaSuccess || (err = F->N0.ensure_async(P->s * 8, st)) != cudaSuccess ||
        (err = F->D1.ensure_async(P->s * 8, st)) != cudaSuccess || (err = F->N1.ensure_async(P->s * 8, st)) != cudaSuccess ||
        (err = F->series.ensure_async((size_t)blocks.size() * T * 8, st)) != cudaSuccess)
        return cuda_fail(err, "fast method scratch");
    unsigned char *tp = (unsigned char *)F->tiles.p;
    if ((err = cudaMemcpyAsync(tp, chunks.data(), chunks.size() * sizeof(FastChunkT), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (err = cudaMemcpyAsync(tp + F->pairs_at, pairs.data(), pairs.size() * sizeof(FastPairT),
                               cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (err = cudaMemcpyAsync(tp + F->blocks_at, blocks.data(), blocks.size() * sizeof(FastBlockT),
                               cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (err = cudaMemcpyAsync(F->tables.p, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (err = cudaMemcpyAsync(F->gblk.p, gblk.data(), gblk.size() * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(err, "fast method upload");
    F->T = T;
    F->p = p;
    return PE_OK;
}

extern "C" pe_status poly_eval_run_fast(pe_poly *P, const uint64_t *beta, uint64_t T, uint64_t t0, uint64_t *out,
                                        void *stream)
{
    if (!P) {
        set_error("NULL poly");
        return PE_ERR_ARG;
    }
    BetaArg barg;
    pe_status st = check_beta(P, beta, &barg);
    if (st != PE_OK) return st;
    uint32_t logTp;
    if (T > kFastMaxT) {
        set_error("the fast method takes T <= %u", kFastMaxT);
        return PE_ERR_ARG;
    }
    if (!points_ok(T, t0)) return PE_ERR_ARG;
    if (T == 0 || P->G == 0) return PE_OK;
    if (!fast_applicable(P->p, T, &logTp)) {
        set_error("the fast method needs p - 1 divisible by %llu (NTTs of twice the padded T)",
                  (unsigned long long)(2ull << logTp));
        return PE_ERR_PRIME;
    }
    if (!out) {
        set_error("out is NULL");
        return PE_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    if (P->last_use) {
        cudaStreamWaitEvent(cs, P->last_use, 0);
        cudaStreamWaitEvent(alloc_stream(), P->last_use, 0);
    }
    if ((st = fast_prepare(P, T, cs)) != PE_OK) return st;
    FastPlan &F = *P->fast;
    cudaPointerAttributes attr{};
    bool dev_out = false;
    if (cudaPointerGetAttributes(&attr, out) == cudaSuccess)
        dev_out = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    cudaGetLastError();
    cudaError_t e;
    uint64_t *out_dev = out;
    if (!dev_out) {
        if ((e = F.out_scratch.ensure_async(T * P->G * 8, cs)) != cudaSuccess) return cuda_fail(e, "output scratch");
        out_dev = F.out_scratch.as<uint64_t>();
    }
    // Step A: monomial values.
    const uint32_t dp1 = P->dmax + 1;
    if ((e = launch_powtab(barg, P->E, dp1, P->mc, P->ptab.as<uint64_t>(), cs)) != cudaSuccess ||
        (e = launch_stepA(P->exps->p, P->exp_bytes, P->s, P->E, P->ptab.as<uint64_t>(), dp1, P->mc,
                          P->mR.as<uint64_t>(), num_sms(), cs)) != cudaSuccess)
        return cuda_fail(e, "Step A");
    const uint64_t p = P->p, Tp = 1ull << logTp, half = Tp;   // Nmax / 2 = Tp
    const uint64_t *tab = F.tables.as<uint64_t>();
    FastTab tb{tab, tab + half, tab + 2 * half, tab + 3 * half, tab + 4 * half, F.lognmax};
    const uint64_t r2 = P->mc.r2;
    const unsigned char *tp = (const unsigned char *)F.tiles.p;
    const FastChunkT *chunks = (const FastChunkT *)tp;
    const FastPairT *pairs = (const FastPairT *)(tp + F.pairs_at);
    const FastBlockT *blocks = (const FastBlockT *)(tp + F.blocks_at);
    uint64_t *Dbuf[2] = {F.D0.as<uint64_t>(), F.D1.as<uint64_t>()};
    uint64_t *Nbuf[2] = {F.N0.as<uint64_t>(), F.N1.as<uint64_t>()};
    k_fast_leaf<<<(F.nchunks + 3) / 4, 128, 0, cs>>>(chunks, F.nchunks, P->mR.as<uint64_t>(), P->coeffs.as<uint64_t>(),
                                                     t0, P->mc, r2, Dbuf[0], Nbuf[0]);
    if ((e = smem_limit_once((const void *)k_fast_merge, 4 * 2 * kFastMaxT / 2 * 8)) != cudaSuccess ||
        (e = smem_limit_once((const void *)k_fast_series, 5 * kFastMaxT * 8)) != cudaSuccess)
        return cuda_fail(e, "fast method shared memory");
    for (size_t lv = 0; lv < F.level_count.size(); ++lv) {
        if (!F.level_count[lv]) continue;   // no block reaches this level (the buffers' roles still alternate)
        const uint32_t logL = 5 + (uint32_t)lv, L = 1u << logL;
        const unsigned threads = std::min<unsigned>(kFastThreads, L);
        k_fast_merge<<<F.level_count[lv], threads, 4 * 2 * L * 8, cs>>>(pairs + F.level_at[lv], logL, Dbuf[lv & 1],
                                                                         Nbuf[lv & 1], Dbuf[(lv + 1) & 1],
                                                                         Nbuf[(lv + 1) & 1], tb, P->mc);
    }
    k_fast_series<<<F.nblocks, kFastThreads, 5 * Tp * 8, cs>>>(blocks, logTp, (uint32_t)T, Dbuf[0], Nbuf[0], Dbuf[1],
                                                              Nbuf[1], F.series.as<uint64_t>(), tb, P->mc);
    const uint64_t cells = P->G * T;
    k_fast_sum<<<(unsigned)((cells + 255) / 256), 256, 0, cs>>>(F.gblk.as<uint32_t>(), P->G, (uint32_t)T,
                                                             F.series.as<uint64_t>(), out_dev, P->mc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fast method");
    if (!P->last_use && (e = cudaEventCreateWithFlags(&P->last_use, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "event");
    if ((e = cudaEventRecord(P->last_use, cs)) != cudaSuccess) return cuda_fail(e, "event");
    if (!dev_out) {
        if ((e = cudaMemcpyAsync(out, out_dev, T * P->G * 8, cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
            (e = cudaStreamSynchronize(cs)) != cudaSuccess)
            return cuda_fail(e, "copy back");
    }
    (void)p;
    return PE_OK;
}
