/*
 * CPU oracle for partial modular polynomial evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library and includes nothing of it.
 *
 * What it computes (paper Sect. 2.3, the definition of the bivariate images
 * below Eq. 1): for a prime p, terms (a_i, d_i, e_i, M_i) and a point beta in
 * F_p^{n-2},
 *
 *     out[t - t0][g] = sum_{i in group g} a_i * prod_{k=3..n} (beta_k^t)^{e_ik}  mod p
 *
 * for t = t0 .. t0+T-1, where group g collects the terms sharing (d_i, e_i)
 * and groups are numbered in descending lexicographic order of (d, e)
 * (Sect. 2.3: lex order with x1 > x2 > ... makes like monomials adjacent).
 *
 * Arithmetic: every product is (unsigned __int128)a*b % p, every sum is a
 * compare-and-subtract on values below p < 2^63, every power is binary
 * square-and-multiply.  Nothing is blocked, fused or reordered.
 *
 *   oracle_eval_direct : O1, the definition above.  A per-t table of
 *                        (beta_k^t)^e for e <= max degree is the only memo.
 *   oracle_eval_cells  : the same definition for a list of (t, g) cells.
 *   oracle_eval_matrix : O2, the matrix method's recurrence (Sect. 2.3):
 *                        m_i = M_i(beta) from power tables, then each term's
 *                        value at successive points by one product per
 *                        point, M_i(beta^t) = m_i^t.  It is the CPU baseline.
 *   oracle_power_sums  : the images of one (x1, x2) coefficient with known
 *                        monomial values z_i: a_k = sum_i c_i z_i^(t0+k).
 *   oracle_tvandermonde_solve : the inverse, interpolation from those images
 *                        (Sect. 1: with points at successive powers of beta the
 *                        linear systems of sparse interpolation are transposed
 *                        Vandermonde systems).  The oracle is the definition:
 *                        Gaussian elimination modulo p on the n x n system.
 *
 * Pins (tests under tests/): brute force with exact Python integers on tiny
 * inputs, Fermat's little theorem at Miller-Rabin-verified primes, the ring
 * homomorphisms eval(A+B) = eval(A)+eval(B) and eval(A*B) = eval(A)*eval(B),
 * the t0 = 0 and beta = 1 coefficient sums, the paper's gcd example
 * (Sect. 2.1) and small symmetric Toeplitz determinants (Sect. 2.2.1).
 * The interpolation functions are pinned by closed forms for n = 1 and 2
 * (Cramer's rule), exhaustive search over F_7^n, round trips through power
 * sums computed with exact Python integers, and recovery of a polynomial's
 * coefficients from images made by oracle_eval_direct.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- F_p ---- */

uint64_t oracle_mulmod(uint64_t a, uint64_t b, uint64_t p)
{
    return (uint64_t)(((u128)a * (u128)b) % (u128)p);
}

/* a, b < p < 2^63, so a + b does not wrap. */
uint64_t oracle_addmod(uint64_t a, uint64_t b, uint64_t p)
{
    uint64_t s = a + b;
    return s >= p ? s - p : s;
}

uint64_t oracle_powmod(uint64_t b, uint64_t e, uint64_t p)
{
    uint64_t r = 1 % p, x = b % p;
    while (e) {
        if (e & 1) r = oracle_mulmod(r, x, p);
        x = oracle_mulmod(x, x, p);
        e >>= 1;
    }
    return r;
}

/* -------------------------------------------------------------- groups ---- */

static int cmp_desc_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? 1 : (x > y ? -1 : 0);
}

static uint64_t term_key(const uint32_t *exps, uint32_t n, uint64_t i)
{
    return ((uint64_t)exps[i * n + 0] << 32) | (uint64_t)exps[i * n + 1];
}

/*
 * Distinct (d, e) keys in descending lexicographic order.
 *   keys_out  : capacity 2*s, receives (d, e) pairs of the G groups
 *   term_group: receives the group index of every term
 * Returns G.  Requires n >= 2.
 */
uint64_t oracle_group_keys(uint32_t n, uint64_t s, const uint32_t *exps,
                           uint32_t *keys_out, uint64_t *term_group)
{
    if (s == 0) return 0;
    uint64_t *k = (uint64_t *)malloc(s * sizeof(uint64_t));
    for (uint64_t i = 0; i < s; ++i) k[i] = term_key(exps, n, i);
    qsort(k, s, sizeof(uint64_t), cmp_desc_u64);
    uint64_t G = 0;
    for (uint64_t i = 0; i < s; ++i)
        if (i == 0 || k[i] != k[G - 1]) k[G++] = k[i];
    for (uint64_t g = 0; g < G; ++g) {
        keys_out[2 * g] = (uint32_t)(k[g] >> 32);
        keys_out[2 * g + 1] = (uint32_t)(k[g] & 0xffffffffu);
    }
    for (uint64_t i = 0; i < s; ++i) {           /* binary search, descending */
        uint64_t key = term_key(exps, n, i), lo = 0, hi = G;
        while (hi - lo > 1) {
            uint64_t mid = (lo + hi) / 2;
            if (k[mid] >= key) lo = mid; else hi = mid;
        }
        term_group[i] = lo;
    }
    free(k);
    return G;
}

static uint32_t max_exp(uint32_t n, uint64_t s, const uint32_t *exps, uint32_t j)
{
    uint32_t m = 0;
    for (uint64_t i = 0; i < s; ++i)
        if (exps[i * n + j] > m) m = exps[i * n + j];
    return m;
}

/* --------------------------------------------------------- O1: direct ---- */

int oracle_eval_direct(uint64_t p, uint32_t n, uint64_t s, const uint64_t *coeffs,
                       const uint32_t *exps, const uint64_t *beta, uint64_t T, uint64_t t0,
                       uint64_t G, const uint64_t *term_group, uint64_t *out)
{
    if (p < 2 || n < 2) return 1;
    uint32_t E = n - 2, dmax = 0;
    for (uint32_t j = 0; j < E; ++j) {
        uint32_t d = max_exp(n, s, exps, 2 + j);
        if (d > dmax) dmax = d;
    }
    uint64_t *pw = (uint64_t *)malloc((size_t)(E ? E : 1) * (dmax + 1) * sizeof(uint64_t));
    memset(out, 0, (size_t)T * G * sizeof(uint64_t));
    for (uint64_t r = 0; r < T; ++r) {
        uint64_t t = t0 + r;
        for (uint32_t j = 0; j < E; ++j) {            /* (beta_j^t)^e, e = 0..dmax */
            uint64_t gam = oracle_powmod(beta[j], t, p);
            pw[(size_t)j * (dmax + 1)] = 1 % p;
            for (uint32_t e = 1; e <= dmax; ++e)
                pw[(size_t)j * (dmax + 1) + e] = oracle_mulmod(pw[(size_t)j * (dmax + 1) + e - 1], gam, p);
        }
        uint64_t *row = out + r * G;
        for (uint64_t i = 0; i < s; ++i) {
            uint64_t v = coeffs[i] % p;
            for (uint32_t j = 0; j < E; ++j)
                v = oracle_mulmod(v, pw[(size_t)j * (dmax + 1) + exps[i * n + 2 + j]], p);
            row[term_group[i]] = oracle_addmod(row[term_group[i]], v, p);
        }
    }
    free(pw);
    return 0;
}

/* The same definition for individual cells (t, g); `t` is the absolute point index. */
int oracle_eval_cells(uint64_t p, uint32_t n, uint64_t s, const uint64_t *coeffs,
                      const uint32_t *exps, const uint64_t *beta, uint64_t G,
                      const uint64_t *term_group, uint64_t ncells, const uint64_t *cell_t,
                      const uint64_t *cell_g, uint64_t *vals)
{
    if (p < 2 || n < 2) return 1;
    uint32_t E = n - 2;
    /* CSR of terms by group */
    uint64_t *cnt = (uint64_t *)calloc(G + 1, sizeof(uint64_t));
    uint64_t *idx = (uint64_t *)malloc((s ? s : 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < s; ++i) cnt[term_group[i] + 1]++;
    for (uint64_t g = 0; g < G; ++g) cnt[g + 1] += cnt[g];
    uint64_t *fill = (uint64_t *)malloc((G + 1) * sizeof(uint64_t));
    memcpy(fill, cnt, (G + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < s; ++i) idx[fill[term_group[i]]++] = i;
    uint64_t *gam = (uint64_t *)malloc((E ? E : 1) * sizeof(uint64_t));
    for (uint64_t c = 0; c < ncells; ++c) {
        uint64_t t = cell_t[c], g = cell_g[c], acc = 0;
        if (g >= G) { vals[c] = ~(uint64_t)0; continue; }
        for (uint32_t j = 0; j < E; ++j) gam[j] = oracle_powmod(beta[j], t, p);
        for (uint64_t q = cnt[g]; q < cnt[g + 1]; ++q) {
            uint64_t i = idx[q], v = coeffs[i] % p;
            for (uint32_t j = 0; j < E; ++j)
                v = oracle_mulmod(v, oracle_powmod(gam[j], exps[i * n + 2 + j], p), p);
            acc = oracle_addmod(acc, v, p);
        }
        vals[c] = acc;
    }
    free(cnt); free(idx); free(fill); free(gam);
    return 0;
}

/* -------------------------------------------- O2: the matrix method ---- */

/*
 * The matrix method's recurrence (Sect. 2.3): since M_i(beta^t) = m_i^t with
 * m_i = M_i(beta), the term a_i M_i(beta^t) at point t is the one at point t-1
 * times m_i.  This evaluator takes the groups one at a time; for each term of
 * the group it computes m_i from power tables [beta_k^e, 0 <= e <= d_k]
 * (n-3 products), starts from a_i m_i^(t0-1), and walks the T points with one
 * product per point, adding each value into the group's row of T sums.  It
 * does the same sT products and sums as the paper's matrix method, in a
 * different order (the method itself advances every term by one point before
 * the next point; order does not matter in F_p).  Requires t0 >= 1.
 */
int oracle_eval_matrix(uint64_t p, uint32_t n, uint64_t s, const uint64_t *coeffs,
                       const uint32_t *exps, const uint64_t *beta, uint64_t T, uint64_t t0,
                       uint64_t G, const uint64_t *term_group, uint64_t *out)
{
    if (p < 2 || n < 2 || t0 < 1) return 1;
    uint32_t E = n - 2;
    /* terms of group g: members[first[g] .. first[g+1]) */
    uint64_t *first = (uint64_t *)calloc(G + 1, sizeof(uint64_t));
    uint64_t *members = (uint64_t *)malloc((s ? s : 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < s; ++i) first[term_group[i] + 1]++;
    for (uint64_t g = 0; g < G; ++g) first[g + 1] += first[g];
    uint64_t *next = (uint64_t *)malloc((G + 1) * sizeof(uint64_t));
    memcpy(next, first, (G + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < s; ++i) members[next[term_group[i]]++] = i;
    free(next);
    /* power tables: pw[j][e] = beta_j^e for e <= the largest exponent of x_{j+3} */
    uint32_t *deg = (uint32_t *)malloc((E ? E : 1) * sizeof(uint32_t));
    size_t cells = 0;
    for (uint32_t j = 0; j < E; ++j) { deg[j] = max_exp(n, s, exps, 2 + j); cells += deg[j] + 1; }
    uint64_t *pw = (uint64_t *)malloc((cells ? cells : 1) * sizeof(uint64_t));
    uint64_t **tab = (uint64_t **)malloc((E ? E : 1) * sizeof(uint64_t *));
    for (uint32_t j = 0, at = 0; j < E; at += deg[j] + 1, ++j) {
        tab[j] = pw + at;
        tab[j][0] = 1 % p;
        for (uint32_t e = 1; e <= deg[j]; ++e) tab[j][e] = oracle_mulmod(tab[j][e - 1], beta[j], p);
    }
    uint64_t *sums = (uint64_t *)malloc((T ? T : 1) * sizeof(uint64_t));
    for (uint64_t g = 0; g < G; ++g) {
        memset(sums, 0, (T ? T : 1) * sizeof(uint64_t));
        for (uint64_t q = first[g]; q < first[g + 1]; ++q) {
            const uint64_t i = members[q];
            uint64_t m = 1 % p;
            for (uint32_t j = 0; j < E; ++j) m = oracle_mulmod(m, tab[j][exps[i * n + 2 + j]], p);
            uint64_t v = oracle_mulmod(coeffs[i] % p, oracle_powmod(m, t0 - 1, p), p);
            for (uint64_t r = 0; r < T; ++r) {      /* v = a_i m_i^(t0+r) */
                v = oracle_mulmod(v, m, p);
                sums[r] = oracle_addmod(sums[r], v, p);
            }
        }
        for (uint64_t r = 0; r < T; ++r) out[r * G + g] = sums[r];
    }
    free(first); free(members); free(deg); free(pw); free(tab); free(sums);
    return 0;
}

/* ------------------------------------------ interpolation (Sect. 1) ---- */

/*
 * a_k = sum_{i<n} c_i * z_i^(t0+k) mod p for k = 0..K-1: the value at the
 * point beta^(t0+k) of one (x1, x2) coefficient whose terms have monomial
 * values z_i = M_i(beta) and coefficients c_i.
 */
int oracle_power_sums(uint64_t p, uint64_t n, const uint64_t *z, const uint64_t *c, uint64_t t0,
                      uint64_t K, uint64_t *a)
{
    if (p < 2) return 1;
    for (uint64_t k = 0; k < K; ++k) {
        uint64_t acc = 0;
        for (uint64_t i = 0; i < n; ++i)
            acc = oracle_addmod(acc, oracle_mulmod(c[i] % p, oracle_powmod(z[i], t0 + k, p), p), p);
        a[k] = acc;
    }
    return 0;
}

/*
 * Solves sum_{i<n} c_i * z_i^(t0+k) = a_k (k = 0..n-1) for c by Gaussian
 * elimination modulo the prime p: row k of the matrix holds z_i^(t0+k).  The
 * pivot of each column is the first nonzero entry at or below the diagonal;
 * inverses are a^(p-2) (Fermat).  Returns 0, or 1 if the matrix is singular
 * (two equal z_i, or a zero z_i with t0 > 0).
 */
int oracle_tvandermonde_solve(uint64_t p, uint64_t n, const uint64_t *z, const uint64_t *a,
                              uint64_t t0, uint64_t *c)
{
    if (p < 2) return 1;
    if (n == 0) return 0;
    uint64_t *A = (uint64_t *)malloc((size_t)n * (n + 1) * sizeof(uint64_t));  /* [A | a] */
    for (uint64_t k = 0; k < n; ++k) {
        for (uint64_t i = 0; i < n; ++i) A[k * (n + 1) + i] = oracle_powmod(z[i], t0 + k, p);
        A[k * (n + 1) + n] = a[k] % p;
    }
    int singular = 0;
    for (uint64_t col = 0; col < n && !singular; ++col) {
        uint64_t piv = col;
        while (piv < n && A[piv * (n + 1) + col] == 0) ++piv;
        if (piv == n) { singular = 1; break; }
        if (piv != col)
            for (uint64_t j = 0; j <= n; ++j) {
                uint64_t t = A[col * (n + 1) + j];
                A[col * (n + 1) + j] = A[piv * (n + 1) + j];
                A[piv * (n + 1) + j] = t;
            }
        uint64_t inv = oracle_powmod(A[col * (n + 1) + col], p - 2, p);
        for (uint64_t j = col; j <= n; ++j) A[col * (n + 1) + j] = oracle_mulmod(A[col * (n + 1) + j], inv, p);
        for (uint64_t r = 0; r < n; ++r) {                      /* eliminate the column elsewhere */
            if (r == col) continue;
            uint64_t f = A[r * (n + 1) + col];
            if (f == 0) continue;
            for (uint64_t j = col; j <= n; ++j) {
                uint64_t sub = oracle_mulmod(f, A[col * (n + 1) + j], p);
                A[r * (n + 1) + j] = oracle_addmod(A[r * (n + 1) + j], sub ? p - sub : 0, p);
            }
        }
    }
    if (!singular)
        for (uint64_t i = 0; i < n; ++i) c[i] = A[i * (n + 1) + n];
    free(A);
    return singular;
}
