// Interpolation from images at successive powers (Sect. 1).
//
// With evaluation points beta^t, t = t0, t0+1, ..., the images of one
// (x1, x2) coefficient with n terms are a_k = sum_i c_i z_i^(t0+k), where
// z_i = M_i(beta) is the value of the i-th monomial.  Recovering the c_i from
// a_0..a_{n-1} is a transposed Vandermonde system (Zippel's observation,
// Sect. 1), solved here in O(n^2) operations per coefficient:
//
//   P(z)  = prod_i (z - z_i) = sum_{j<=n} P_j z^j              (master polynomial)
//   R_l   = sum_{k=0}^{n-1-l} a_k P_{k+1+l},   l = 0..n-1      (correlation of a and P)
//   S_i   = R(z_i) = sum_l R_l z_i^l,   D_i = P'(z_i)
//   c_i   = S_i / D_i * z_i^(-t0).
//
// Why: the quotient Q_i(z) = P(z) / (z - z_i) vanishes at every z_j, j != i,
// and sum_k [z^k]Q_i * a_k = sum_j c_j z_j^t0 Q_i(z_j) = c_i z_i^t0 P'(z_i);
// expanding [z^k]Q_i = sum_{j>k} P_j z_i^(j-1-k) gives S_i = R(z_i).
//
// Kernels (all coefficients of a call in each launch, flat tile lists built
// on the host, 128 outputs per block):
//   k_vdm_init   : leaves z - z_i of the product tree, images gathered per coefficient
//   k_vdm_merge  : one level of the product tree: adjacent monic factors of
//                  degree L multiplied pairwise (schoolbook, exact 128-bit
//                  products summed in 192 bits, one reduction per output)
//   k_vdm_corr   : R_l and P'_l
//   k_vdm_horner : S_i and D_i by Horner with the fixed multiplier z_i
//                  (lazy Barrett product), then c_i
// The work is integer multiplies: about n^2/2 exact products for the tree,
// n^2/2 for the correlation and 2 n^2 fixed-multiplier products for Horner.
// Long sums are cut into chunks of at least 512 inputs so that a coefficient
// of thousands of terms still spreads over the whole GPU: each chunk's sum is
// a partial (k_vdm_sum adds the partials of the tree and the correlation);
// Horner over a chunk of 512 powers gives S_i = sum_k z_i^(512k) S_i^(k),
// which k_vdm_finish evaluates by Horner in z_i^512.
#include <algorithm>
#include <vector>
#include "internal.h"
#include "modarith.cuh"
#include "kernels.h"

namespace pe {

constexpr int kVdmTile = 128;        // outputs per block
constexpr uint32_t kVdmChunk = 512;  // shortest chunk of a long sum
constexpr uint32_t kVdmMaxChunks = 64;

struct VdmTile {
    uint32_t off;     // first term of the coefficient
    uint32_t n;       // its number of terms
    uint32_t j0;      // first output of the tile (index within the coefficient)
    uint32_t g;       // coefficient (column of the images)
    uint32_t kappa;   // input chunk of this tile
    uint32_t nchunk;  // chunks of this sum (1: no partials)
    uint32_t clen;    // chunk length of the coefficient
    uint32_t pad;
    uint64_t pbase;   // partial of chunk kappa, output j: part[pbase + kappa * n + j]
};

__device__ __forceinline__ uint64_t lazy2v(uint64_t x, uint64_t p2) { return x >= p2 ? x - p2 : x; }

// x in [0, 3p) to [0, p).
__device__ __forceinline__ uint64_t canon3(uint64_t x, const ModCtx &mc)
{
    x = x >= mc.p2 ? x - mc.p2 : x;
    return canon(x, mc.p);
}

// Number of tree levels a coefficient of n terms goes through: ceil(log2 n).
// Its master polynomial ends in buffer (levels mod 2).
__device__ __forceinline__ uint32_t tree_levels(uint32_t n) { return n <= 1 ? 0 : 32 - __clz(n - 1); }

// Leaves: factor z - z_i stored as its constant coefficient p - z_i; images
// of each coefficient gathered into consecutive words.  Flags nodes >= p.
__global__ void k_vdm_init(const VdmTile *__restrict__ tiles, const uint64_t *__restrict__ z,
                           const uint64_t *__restrict__ img, uint64_t lda, uint64_t p, uint64_t *__restrict__ leaf,
                           uint64_t *__restrict__ ag, uint32_t *__restrict__ flags)
{
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t j = t.j0 + threadIdx.x;
    if (j >= t.n) return;
    const uint64_t zi = z[t.off + j];
    if (zi >= p) atomicOr(flags, 1u);
    leaf[t.off + j] = zi == 0 || zi >= p ? 0 : p - zi;
    ag[t.off + j] = img[(uint64_t)j * lda + t.g];
}

// One level of the product tree: within a coefficient, the factors of terms
// [2qL, 2qL+L) and [2qL+L, 2qL+2L) (monic, degrees la and lb, non-leading
// coefficients stored in place of their terms) are multiplied; the product's
// la+lb non-leading coefficients replace them.  A factor without a partner is
// copied.  With several chunks, chunk kappa sums the products A_i B_(k-i)
// with i in [kappa*clen, (kappa+1)*clen) into a partial; chunk 0 also takes
// the terms of the two leading ones.
__global__ void __launch_bounds__(kVdmTile) k_vdm_merge(const VdmTile *__restrict__ tiles, uint32_t L,
                                                        const uint64_t *__restrict__ src, uint64_t *__restrict__ dst,
                                                        uint64_t *__restrict__ part, uint64_t r3, ModCtx mc)
{
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t j = t.j0 + threadIdx.x;
    if (j >= t.n) return;
    const uint32_t base = j / (2 * L) * (2 * L);
    const uint32_t la = min(L, t.n - base);
    const uint32_t lb = min(L, t.n - base - la);
    const uint32_t k = j - base;
    const uint64_t *A = src + t.off + base;
    const uint64_t *B = A + la;
    uint64_t *out = t.nchunk > 1 ? part + t.pbase + (uint64_t)t.kappa * t.n + j : dst + t.off + j;
    if (lb == 0) {
        *out = t.kappa == 0 ? A[k] : 0;
        return;
    }
    uint64_t l = 0, m = 0;
    uint32_t h = 0;
    const uint32_t c0 = t.kappa * t.clen, c1 = c0 + t.clen;
    const uint32_t i_lo = max(k + 1 > lb ? k + 1 - lb : 0, c0), i_hi = min(min(k, la - 1), c1 - 1);
    for (uint32_t i = i_lo; i <= i_hi; ++i) mac192(l, m, h, A[i], B[k - i]);
    if (t.kappa == 0) {
        if (k >= la) mac192(l, m, h, 1, B[k - la]);   // A's leading 1
        if (k >= lb) mac192(l, m, h, 1, A[k - lb]);   // B's leading 1
    }
    *out = reduce192(l, m, h, r3, mc);
}

// Sums the chunk partials of one output: mode 0 writes dst0 (a tree level),
// mode 1 writes R next to the coefficient's master polynomial (the buffer
// that does not hold it).
__global__ void __launch_bounds__(kVdmTile) k_vdm_sum(const VdmTile *__restrict__ tiles,
                                                      const uint64_t *__restrict__ part, uint64_t *dst0,
                                                      uint64_t *dst1, int mode, ModCtx mc)
{
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t j = t.j0 + threadIdx.x;
    if (j >= t.n) return;
    uint64_t acc = 0;
    for (uint32_t q = 0; q < t.nchunk; ++q) {
        acc += part[t.pbase + (uint64_t)q * t.n + j];
        acc = canon(acc, mc.p);
    }
    uint64_t *dst = mode == 0 ? dst0 : (tree_levels(t.n) & 1 ? dst0 : dst1);
    dst[t.off + j] = acc;
}

// R_l = sum_{k <= n-1-l} a_k P_{k+1+l} (P_n = 1) over chunk kappa of k, and
// (chunk 0) P'_l = (l+1) P_{l+1}.  buf0/Rout0 and buf1/Rout1 are the same two
// buffers: each column reads its P from one and writes its R to the other, so
// no element is both read and written.
__global__ void __launch_bounds__(kVdmTile) k_vdm_corr(const VdmTile *__restrict__ tiles, const uint64_t *buf0,
                                                       const uint64_t *buf1, const uint64_t *__restrict__ ag,
                                                       uint64_t *Rout0, uint64_t *Rout1, uint64_t *__restrict__ Dout,
                                                       uint64_t *__restrict__ part, uint64_t r3, ModCtx mc)
{
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t l = t.j0 + threadIdx.x;
    if (l >= t.n) return;
    const uint32_t levels = tree_levels(t.n);
    const uint64_t *P = (levels & 1 ? buf1 : buf0) + t.off;
    const uint64_t *a = ag + t.off;
    uint64_t lo = 0, mid = 0;
    uint32_t h = 0;
    const uint32_t kmax = t.n - 1 - l;                    // term k = kmax uses P_n = 1
    const uint32_t c0 = t.kappa * t.clen, c1 = min(c0 + t.clen, kmax);
    for (uint32_t k = c0; k < c1; ++k) mac192(lo, mid, h, a[k], P[k + 1 + l]);
    if (t.kappa == 0) {
        mac192(lo, mid, h, 1, a[kmax]);
        uint64_t dl = 0, dm = 0;
        uint32_t dh = 0;
        mac192(dl, dm, dh, (uint64_t)l + 1, l + 1 < t.n ? P[l + 1] : 1);
        Dout[t.off + l] = reduce192(dl, dm, dh, r3, mc);
    }
    const uint64_t r = reduce192(lo, mid, h, r3, mc);
    if (t.nchunk > 1)
        part[t.pbase + (uint64_t)t.kappa * t.n + l] = r;
    else
        ((levels & 1 ? Rout0 : Rout1) + t.off)[l] = r;
}

// c_i = S / D * z_i^(-t0), or a flag: D = 0 (repeated node) or a zero node
// with t0 > 0 sets bit 2 and the lowest such coefficient index.
__device__ __forceinline__ void vdm_finish(uint64_t S, uint64_t D, uint64_t zi, uint64_t zR, uint64_t t0_exp,
                                           bool t0_pos, uint32_t g, uint64_t *c, uint32_t *flags, const ModCtx &mc)
{
    const uint64_t p = mc.p;
    if (D == 0 || (zi == 0 && t0_pos)) {
        atomicOr(flags, 2u);
        atomicMin(flags + 1, g);
        *c = 0;
        return;
    }
    const uint64_t dinvR = mont_pow(canon(mont_mul(D, mc.r2, mc), p), p - 2, mc);   // D^-1 R (Fermat)
    const uint64_t ztR = mont_pow(zR, t0_exp, mc);                                 // z^-t0 R
    const uint64_t sR = canon(mont_mul(S, mc.r2, mc), p);
    const uint64_t cR = mont_mul(mont_mul(sR, dinvR, mc), ztR, mc);
    *c = canon(mont_redc(cR, 0, mc), p);
}

// Horner with the fixed multiplier z_i over chunk kappa of the powers:
// S^(kappa) = sum_{l in chunk} R_l z_i^(l - kappa*clen), and the same for P'.
// With one chunk the results are final and c_i is written.
__global__ void __launch_bounds__(kVdmTile) k_vdm_horner(const VdmTile *__restrict__ tiles,
                                                         const uint64_t *__restrict__ z,
                                                         const uint64_t *__restrict__ Rb0,
                                                         const uint64_t *__restrict__ Rb1,
                                                         const uint64_t *__restrict__ D, uint64_t *__restrict__ part_s,
                                                         uint64_t *__restrict__ part_d, uint64_t t0_exp, bool t0_pos,
                                                         uint64_t *__restrict__ c, uint32_t *__restrict__ flags,
                                                         ModCtx mc)
{
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t i = t.j0 + threadIdx.x;
    if (i >= t.n) return;
    const uint64_t *R = (tree_levels(t.n) & 1 ? Rb0 : Rb1) + t.off;
    const uint64_t *Dp = D + t.off;
    const uint64_t zi = z[t.off + i];
    const uint64_t np = 0 - mc.p;
    const uint64_t zR = canon(mont_mul(zi, mc.r2, mc), mc.p);
    const uint64_t wq = barrett_quotient_from_mont(zR, mc);
    const uint32_t c0 = t.kappa * t.clen, c1 = min(c0 + t.clen, t.n);
    uint64_t s = 0, d = 0;
    for (uint32_t l = c1; l-- > c0;) {
        s = barrett_mul_lazy4_mad(s, zi, wq, np);     // [0, 4p)
        d = barrett_mul_lazy4_mad(d, zi, wq, np);
        s = (s >= mc.p2 ? s - mc.p2 : s) + R[l];      // [0, 3p)
        d = (d >= mc.p2 ? d - mc.p2 : d) + Dp[l];
    }
    s = canon3(s, mc);
    d = canon3(d, mc);
    if (t.nchunk > 1) {
        const uint64_t at = t.pbase + (uint64_t)t.kappa * t.n + i;
        part_s[at] = s;
        part_d[at] = d;
        return;
    }
    vdm_finish(s, d, zi, zR, t0_exp, t0_pos, t.g, c + t.off + i, flags, mc);
}

// S = sum_k (z^clen)^k S^(k) by Horner in z^clen, the same for D, then c_i.
__global__ void __launch_bounds__(kVdmTile) k_vdm_finish(const VdmTile *__restrict__ tiles,
                                                         const uint64_t *__restrict__ z,
                                                         const uint64_t *__restrict__ part_s,
                                                         const uint64_t *__restrict__ part_d, uint64_t t0_exp,
                                                         bool t0_pos, uint64_t *__restrict__ c,
                                                         uint32_t *__restrict__ flags, ModCtx mc)
{
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t i = t.j0 + threadIdx.x;
    if (i >= t.n) return;
    const uint64_t zi = z[t.off + i];
    const uint64_t np = 0 - mc.p;
    const uint64_t zR = canon(mont_mul(zi, mc.r2, mc), mc.p);
    const uint64_t zLR = mont_pow(zR, t.clen, mc);                  // z^clen in Montgomery form
    const uint64_t zL = canon(mont_redc(zLR, 0, mc), mc.p);
    const uint64_t wq = barrett_quotient_from_mont(zLR, mc);
    uint64_t s = 0, d = 0;
    for (uint32_t q = t.nchunk; q-- > 0;) {
        const uint64_t at = t.pbase + (uint64_t)q * t.n + i;
        s = barrett_mul_lazy4_mad(s, zL, wq, np);
        d = barrett_mul_lazy4_mad(d, zL, wq, np);
        s = (s >= mc.p2 ? s - mc.p2 : s) + part_s[at];
        d = (d >= mc.p2 ? d - mc.p2 : d) + part_d[at];
    }
    vdm_finish(canon3(s, mc), canon3(d, mc), zi, zR, t0_exp, t0_pos, t.g, c + t.off + i, flags, mc);
}

// A whole column of at most 128 terms in one block (no partials, one launch
// for all such columns): P by multiplying in one factor z - z_k per step (one
// coefficient per thread, Montgomery form, Shoup product by the plain z_k),
// then R and P' (thread l), then Horner and c_i (thread i).
constexpr uint32_t kVdmSmall = 128;

__global__ void __launch_bounds__(kVdmSmall) k_vdm_small(const VdmTile *__restrict__ tiles,
                                                        const uint64_t *__restrict__ z,
                                                        const uint64_t *__restrict__ img, uint64_t lda,
                                                        uint64_t t0_exp, bool t0_pos, uint64_t *__restrict__ c,
                                                        uint32_t *__restrict__ flags, ModCtx mc)
{
    __shared__ uint64_t Zs[kVdmSmall], Pa[kVdmSmall + 1], A[kVdmSmall], R[kVdmSmall], Dd[kVdmSmall];
    const VdmTile t = tiles[blockIdx.x];
    const uint32_t n = t.n, i = threadIdx.x;
    const uint64_t p = mc.p, p2 = mc.p2, np = 0 - mc.p;
    uint64_t zi = 0;
    if (i < n) {
        zi = z[t.off + i];
        if (zi >= p) {
            atomicOr(flags, 1u);
            zi = 0;
        }
        Zs[i] = zi;
        A[i] = img[(uint64_t)i * lda + t.g];
    }
    if (i == 0) Pa[0] = mc.r1;   // P = 1
    __syncthreads();
    for (uint32_t k = 0; k < n; ++k) {   // P <- P (z - z_k): degree k -> k+1, leading coefficient stays 1
        const uint64_t zk = Zs[k];
        const uint64_t wq = barrett_quotient_from_mont(canon(mont_mul(zk, mc.r2, mc), p), mc);
        uint64_t nv = 0;
        if (i <= k) {
            const uint64_t below = i ? Pa[i - 1] : 0;
            const uint64_t prod = lazy2v(barrett_mul_lazy4_mad(Pa[i], zk, wq, np), p2);
            nv = lazy2v(below + p2 - prod, p2);
        }
        __syncthreads();
        if (i <= k) Pa[i] = nv;
        if (i == 0) Pa[k + 1] = mc.r1;
        __syncthreads();
    }
    if (i < n) {   // R_l = sum_{k <= n-1-l} a_k P_{k+1+l}, P'_l = (l+1) P_{l+1}, plain residues
        uint64_t lo = 0, mid = 0;
        uint32_t h = 0;
        for (uint32_t k = 0; k + i < n; ++k) mac192(lo, mid, h, A[k], Pa[k + 1 + i]);
        R[i] = reduce192(lo, mid, h, mc.r2, mc);
        lo = mid = 0;
        h = 0;
        mac192(lo, mid, h, (uint64_t)i + 1, Pa[i + 1]);
        Dd[i] = reduce192(lo, mid, h, mc.r2, mc);
    }
    __syncthreads();
    if (i < n) {
        const uint64_t zR = canon(mont_mul(zi, mc.r2, mc), p);
        const uint64_t wq = barrett_quotient_from_mont(zR, mc);
        uint64_t sv = 0, dv = 0;
        for (uint32_t l = n; l-- > 0;) {
            sv = barrett_mul_lazy4_mad(sv, zi, wq, np);
            dv = barrett_mul_lazy4_mad(dv, zi, wq, np);
            sv = lazy2v(sv, p2) + R[l];
            dv = lazy2v(dv, p2) + Dd[l];
        }
        vdm_finish(canon3(sv, mc), canon3(dv, mc), zi, zR, t0_exp, t0_pos, t.g, c + t.off + i, flags, mc);
    }
}

// Canonical values from Montgomery form.
__global__ void k_from_mont(const uint64_t *__restrict__ xR, uint64_t s, ModCtx mc, uint64_t *__restrict__ x)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (uint64_t)gridDim.x * blockDim.x)
        x[i] = canon(mont_redc(xR[i], 0, mc), mc.p);
}

// Appends the tiles of one column for one launch: every chunk kappa < nchunk
// (kappa fixed at 0 with nchunk kept, for the kernels that read all chunks).
static void add_tiles(std::vector<VdmTile> &v, uint32_t off, uint32_t n, uint32_t g, uint32_t nchunk,
                      uint32_t clen, uint64_t pbase, bool per_chunk)
{
    for (uint32_t q = 0; q < (per_chunk ? nchunk : 1u); ++q)
        for (uint32_t j0 = 0; j0 < n; j0 += kVdmTile) v.push_back({off, n, j0, g, q, nchunk, clen, 0, pbase});
}

// Optional kernel timing of the solver, per host thread: events around the
// leaves, the tree levels, the correlation and the Horner kernels.
struct VdmTiming {
    bool on = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double ms[4] = {0, 0, 0, 0};
    ~VdmTiming()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};
static thread_local VdmTiming g_vdm_timing;

// A launch over a range of the tile list.
struct VdmRange {
    size_t at = 0, count = 0;
};

}  // namespace pe

using namespace pe;

extern "C" pe_status poly_eval_vandermonde_solve(uint64_t p, uint64_t G, const uint64_t *off, const uint64_t *z,
                                                 const uint64_t *images, uint64_t rows, uint64_t lda, uint64_t t0,
                                                 uint64_t *c, void *stream)
{
    if (p < 3 || (p & 1) == 0 || p >= (1ull << 62)) {
        set_error("p = %llu must be odd, at least 3 and below 2^62", (unsigned long long)p);
        return PE_ERR_PRIME;
    }
    if (G && !off) {
        set_error("off is NULL");
        return PE_ERR_ARG;
    }
    if (G == 0) return PE_OK;
    if (off[0] != 0 || off[G] > 0xffffffffull || G > 0xffffffffull) {
        set_error("off[0] must be 0 and off[G] below 2^32");
        return PE_ERR_ARG;
    }
    uint64_t nmax = 0;
    for (uint64_t g = 0; g < G; ++g) {
        if (off[g + 1] < off[g]) {
            set_error("off must be nondecreasing (off[%llu] > off[%llu])", (unsigned long long)g,
                      (unsigned long long)(g + 1));
            return PE_ERR_ARG;
        }
        nmax = std::max(nmax, off[g + 1] - off[g]);
    }
    const uint64_t s = off[G];
    if (s == 0) return PE_OK;
    if (!z || !images || !c) {
        set_error("z, images and c must be device pointers");
        return PE_ERR_ARG;
    }
    if (nmax > (1ull << 24)) {
        set_error("a coefficient has %llu terms; at most 2^24 are supported", (unsigned long long)nmax);
        return PE_ERR_ARG;
    }
    if (nmax > rows || lda < G) {
        set_error("a coefficient has %llu terms but the images have %llu rows (lda %llu, G %llu)",
                  (unsigned long long)nmax, (unsigned long long)rows, (unsigned long long)lda,
                  (unsigned long long)G);
        return PE_ERR_ARG;
    }
    const ModCtx mc = make_modctx(p);
    const uint64_t r3 = (uint64_t)(((unsigned __int128)mc.r2 * mc.r1) % p);
    // Per column: chunk length (at least 512, at most 64 chunks) and the base
    // of its partials (chunks x terms words).  Larger columns first.
    // Columns of at most 128 terms go to the one-launch kernel; the rest
    // through the tree, correlation and Horner kernels.
    std::vector<uint64_t> order, small;
    uint64_t nlarge = 0;
    for (uint64_t g = 0; g < G; ++g) {
        const uint64_t n = off[g + 1] - off[g];
        if (n > kVdmSmall) {
            order.push_back(g);
            nlarge = std::max(nlarge, n);
        } else if (n) {
            small.push_back(g);
        }
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](uint64_t a, uint64_t b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    std::vector<uint32_t> clen(G, kVdmChunk);
    std::vector<uint64_t> pbase(G, 0);
    uint64_t part_words = 0;
    for (uint64_t g : order) {
        const uint64_t n = off[g + 1] - off[g];
        clen[g] = (uint32_t)std::max<uint64_t>(kVdmChunk, (n + kVdmMaxChunks - 1) / kVdmMaxChunks);
        pbase[g] = part_words;
        const uint64_t nch = (n + clen[g] - 1) / clen[g];
        if (nch > 1) part_words += nch * n;
    }
    auto chunks = [&](uint64_t g, uint64_t len) { return (uint32_t)std::max<uint64_t>(1, (len + clen[g] - 1) / clen[g]); };
    // Tile lists, one range per launch.
    std::vector<VdmTile> tiles;
    auto begin = [&]() { return VdmRange{tiles.size(), 0}; };
    auto end = [&](VdmRange &r) { r.count = tiles.size() - r.at; };
    auto column = [&](uint64_t g, uint32_t nch, bool per_chunk) {
        add_tiles(tiles, (uint32_t)off[g], (uint32_t)(off[g + 1] - off[g]), (uint32_t)g, nch, clen[g], pbase[g],
                  per_chunk);
    };
    VdmRange r_init = begin();
    for (uint64_t g : order) column(g, 1, false);
    end(r_init);
    std::vector<VdmRange> r_merge, r_msum;   // level L of the tree: coefficients with more than L terms
    std::vector<uint32_t> level_L;
    for (uint64_t L = 1; L < nlarge; L *= 2) {
        level_L.push_back((uint32_t)L);
        VdmRange m = begin();
        for (uint64_t g : order)
            if (off[g + 1] - off[g] > L) column(g, chunks(g, L), true);
        end(m);
        r_merge.push_back(m);
        VdmRange q = begin();
        for (uint64_t g : order)
            if (off[g + 1] - off[g] > L && chunks(g, L) > 1) column(g, chunks(g, L), false);
        end(q);
        r_msum.push_back(q);
    }
    VdmRange r_corr = begin();
    for (uint64_t g : order) column(g, chunks(g, off[g + 1] - off[g] - 1), true);
    end(r_corr);
    VdmRange r_csum = begin();
    for (uint64_t g : order)
        if (chunks(g, off[g + 1] - off[g] - 1) > 1) column(g, chunks(g, off[g + 1] - off[g] - 1), false);
    end(r_csum);
    VdmRange r_horner = begin();
    for (uint64_t g : order) column(g, chunks(g, off[g + 1] - off[g]), true);
    end(r_horner);
    VdmRange r_finish = begin();
    for (uint64_t g : order)
        if (chunks(g, off[g + 1] - off[g]) > 1) column(g, chunks(g, off[g + 1] - off[g]), false);
    end(r_finish);
    VdmRange r_small = begin();
    for (uint64_t g : small) tiles.push_back({(uint32_t)off[g], (uint32_t)(off[g + 1] - off[g]), 0, (uint32_t)g, 0, 1, 0, 0, 0});
    end(r_small);
    if (tiles.size() > 0x7fffffffull) {
        set_error("too many columns");
        return PE_ERR_ARG;
    }

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    DevBuf dtiles, b0, b1, ag, dD, part, flags;
    const uint64_t sl = order.empty() ? 1 : s;   // the general path's scratch
    if ((e = dtiles.ensure_async(tiles.size() * sizeof(VdmTile), st)) != cudaSuccess ||
        (e = b0.ensure_async(sl * 8, st)) != cudaSuccess || (e = b1.ensure_async(sl * 8, st)) != cudaSuccess ||
        (e = ag.ensure_async(sl * 8, st)) != cudaSuccess || (e = dD.ensure_async(sl * 8, st)) != cudaSuccess ||
        (e = part.ensure_async(std::max<uint64_t>(1, 2 * part_words) * 8, st)) != cudaSuccess ||
        (e = flags.ensure_async(8, st)) != cudaSuccess) {
        cudaStreamSynchronize(st);
        return cuda_fail(e, "interpolation scratch");
    }
    const uint32_t fl_init[2] = {0, 0xffffffffu};
    if ((e = cudaMemcpyAsync(dtiles.p, tiles.data(), tiles.size() * sizeof(VdmTile), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(flags.p, fl_init, 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        cudaStreamSynchronize(st);
        return cuda_fail(e, "interpolation upload");
    }
    const VdmTile *T = dtiles.as<VdmTile>();
    uint64_t *bufs[2] = {b0.as<uint64_t>(), b1.as<uint64_t>()};
    uint64_t *part_s = part.as<uint64_t>(), *part_d = part_s + part_words;
    VdmTiming &tm = g_vdm_timing;
    if (tm.on && !tm.ev[0])
        for (cudaEvent_t &x : tm.ev)
            if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(e, "timing events");
    auto mark = [&](int k) {
        if (tm.on) cudaEventRecord(tm.ev[k], st);
    };
    auto grid = [](const VdmRange &r) { return (unsigned)r.count; };
    const bool general = !order.empty();
    mark(0);
    if (general)
        k_vdm_init<<<grid(r_init), kVdmTile, 0, st>>>(T + r_init.at, z, images, lda, p, bufs[0], ag.as<uint64_t>(),
                                                  flags.as<uint32_t>());
    mark(1);
    for (size_t lv = 0; lv < r_merge.size(); ++lv) {
        uint64_t *dst = bufs[(lv + 1) & 1];
        k_vdm_merge<<<grid(r_merge[lv]), kVdmTile, 0, st>>>(T + r_merge[lv].at, level_L[lv], bufs[lv & 1], dst,
                                                            part_s, r3, mc);
        if (r_msum[lv].count)
            k_vdm_sum<<<grid(r_msum[lv]), kVdmTile, 0, st>>>(T + r_msum[lv].at, part_s, dst, dst, 0, mc);
    }
    mark(2);
    if (general)
        k_vdm_corr<<<grid(r_corr), kVdmTile, 0, st>>>(T + r_corr.at, bufs[0], bufs[1], ag.as<uint64_t>(), bufs[0],
                                                  bufs[1], dD.as<uint64_t>(), part_s, r3, mc);
    if (r_csum.count)
        k_vdm_sum<<<grid(r_csum), kVdmTile, 0, st>>>(T + r_csum.at, part_s, bufs[0], bufs[1], 1, mc);
    mark(3);
    const uint64_t t0_exp = (p - 1 - t0 % (p - 1)) % (p - 1);
    if (r_small.count)
        k_vdm_small<<<grid(r_small), kVdmSmall, 0, st>>>(T + r_small.at, z, images, lda, t0_exp, t0 > 0, c,
                                                        flags.as<uint32_t>(), mc);
    if (general)
        k_vdm_horner<<<grid(r_horner), kVdmTile, 0, st>>>(T + r_horner.at, z, bufs[0], bufs[1], dD.as<uint64_t>(),
                                                      part_s, part_d, t0_exp, t0 > 0, c, flags.as<uint32_t>(), mc);
    if (r_finish.count)
        k_vdm_finish<<<grid(r_finish), kVdmTile, 0, st>>>(T + r_finish.at, z, part_s, part_d, t0_exp, t0 > 0, c,
                                                          flags.as<uint32_t>(), mc);
    mark(4);
    uint32_t fl[2] = {0, 0};
    if ((e = cudaGetLastError()) != cudaSuccess) cudaStreamSynchronize(st);
    if (e != cudaSuccess ||
        (e = cudaMemcpyAsync(fl, flags.p, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "interpolation");
    if (tm.on)
        for (int k = 0; k < 4; ++k) {
            float ms = 0;
            cudaEventElapsedTime(&ms, tm.ev[k], tm.ev[k + 1]);
            tm.ms[k] = ms;
        }
    if (fl[0] & 1) {
        set_error("a node z_i is not below p");
        return PE_ERR_NOT_REDUCED;
    }
    if (fl[0] & 2) {
        set_error("singular system in coefficient %u: repeated node, or a zero node with t0 > 0", fl[1]);
        return PE_ERR_SINGULAR;
    }
    return PE_OK;
}

extern "C" pe_status poly_eval_monomials(pe_poly *P, const uint64_t *beta, uint64_t *z, uint64_t *off, void *stream)
{
    if (!P) {
        set_error("NULL poly");
        return PE_ERR_ARG;
    }
    BetaArg barg;
    pe_status st = check_beta(P, beta, &barg);
    if (st != PE_OK) return st;
    if (off) memcpy(off, P->group_off.data(), (P->G + 1) * sizeof(uint64_t));
    if (P->s == 0) return PE_OK;
    if (!z) {
        set_error("z is NULL");
        return PE_ERR_ARG;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    if (P->last_use) {
        cudaStreamWaitEvent(cs, P->last_use, 0);
        cudaStreamWaitEvent(alloc_stream(), P->last_use, 0);
    }
    cudaError_t e;
    const uint32_t dp1 = P->dmax + 1;
    if ((e = P->ptab.ensure((size_t)std::max(1u, P->E * dp1) * 8)) != cudaSuccess ||
        (e = P->mR.ensure(P->s * 8)) != cudaSuccess)
        return cuda_fail(e, "monomial scratch");
    if ((e = launch_powtab(barg, P->E, dp1, P->mc, P->ptab.as<uint64_t>(), cs)) != cudaSuccess ||
        (e = launch_stepA(P->exps->p, P->exp_bytes, P->s, P->E, P->ptab.as<uint64_t>(), dp1, P->mc,
                          P->mR.as<uint64_t>(), num_sms(), cs)) != cudaSuccess)
        return cuda_fail(e, "Step A");
    const unsigned grid = (unsigned)std::min<uint64_t>((P->s + 255) / 256, (uint64_t)num_sms() * 8);
    k_from_mont<<<grid, 256, 0, cs>>>(P->mR.as<uint64_t>(), P->s, P->mc, z);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "monomials");
    if (!P->last_use && (e = cudaEventCreateWithFlags(&P->last_use, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "event");
    if ((e = cudaEventRecord(P->last_use, cs)) != cudaSuccess) return cuda_fail(e, "event");
    return PE_OK;
}

extern "C" pe_status poly_eval_vandermonde_timing(int enable, double ms[4])
{
    if (ms)
        for (int k = 0; k < 4; ++k) ms[k] = g_vdm_timing.ms[k];
    if (enable >= 0) g_vdm_timing.on = enable != 0;
    return PE_OK;
}
