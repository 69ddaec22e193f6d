/*
 * Plain CPU oracle for DKSS multiplication: C transcription of
 * oracle/dkss_oracle.py for sizes Python cannot finish (test infrastructure
 * only; the CUDA library never links or calls it and shares no code with it).
 *
 * It follows C. Lueders, "Fast Multiplication of Large Integers:
 * Implementation and Analysis of the DKSS Algorithm" (arXiv:1503.04955),
 * Section 3.2, in the same order and notation as the Python oracle:
 *   encode (Section 3.2.4, Fig. dkss:fig:encode), forward FFT by inner DFTs,
 *   bad multiplications and recursive outer DFTs (Section 3.2.5 i.-iii. and
 *   Section 4.2), componentwise products (Section 3.2.6), backwards transform
 *   as forward transform read at index -l and division by 2M (Sections 2.7,
 *   3.2.7, 3.2.8), decode by shifted additions (Section 3.2.8).
 *
 * Residues are unsigned __int128 values in [0, p^z) with p^z < 2^126.
 * Products are summed exactly in 256-bit accumulators and reduced once per
 * output coefficient by Horner's rule with the compiler's 128-bit remainder.
 * The root rho is an input (computed by the Python oracle, Section 3.2.3).
 *
 * Pins: tests/test_oracle_pins.py checks this file against the Python oracle
 * on small parameter sets, against brute-force DFTs and against exact integer
 * products (Python int and schoolbook) on every size it runs.
 *
 * Threads: when built with OpenMP, the loops whose iterations the thesis's
 * steps leave independent run on several host threads -- the inner DFTs of
 * the columns (step i.), the bad multiplications (step ii.), the outer DFTs of
 * the rows (step iii., top level only; deeper levels run inside one thread),
 * encoding, the componentwise products and the scaling.  Every iteration
 * writes its own outputs, so the result does not depend on the thread count;
 * oracle_set_threads() picks it (1 = the plain serial program).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

typedef struct {
    u128 q;          /* p^z */
    uint32_t m, h, u;
    uint64_t M, P2, mu;
    int red_shift;   /* bits fed per Horner step: 127 - bitlen(q) */
} par_t;

static int bitlen128(u128 x) {
    int n = 0;
    while (x) { n++; x >>= 1; }
    return n;
}

static u128 add_mod(u128 a, u128 b, u128 q) { u128 s = a + b; return s >= q ? s - q : s; }
static u128 sub_mod(u128 a, u128 b, u128 q) { return a >= b ? a - b : a + (q - b); }

/* acc (4 x 64-bit words, little-endian) += x * y, x and y < 2^127. */
static void mac256(uint64_t acc[4], u128 x, u128 y) {
    uint64_t x0 = (uint64_t)x, x1 = (uint64_t)(x >> 64);
    uint64_t y0 = (uint64_t)y, y1 = (uint64_t)(y >> 64);
    u128 p00 = (u128)x0 * y0, p01 = (u128)x0 * y1, p10 = (u128)x1 * y0, p11 = (u128)x1 * y1;
    uint64_t prod[4];
    u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
    prod[0] = (uint64_t)p00;
    prod[1] = (uint64_t)mid;
    u128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
    prod[2] = (uint64_t)hi;
    prod[3] = (uint64_t)(hi >> 64) + (uint64_t)(p11 >> 64);
    u128 carry = 0;
    for (int k = 0; k < 4; k++) {
        u128 s = (u128)acc[k] + prod[k] + carry;
        acc[k] = (uint64_t)s;
        carry = s >> 64;
    }
}

/* w (256 bits) mod q by Horner's rule over chunks of red_shift bits. */
static u128 reduce256(const uint64_t w[4], const par_t* par) {
    int top = 255;
    while (top >= 0 && !((w[top / 64] >> (top % 64)) & 1)) top--;
    u128 r = 0;
    int s = par->red_shift;
    for (int pos = top; pos >= 0; pos -= s) {
        int len = pos + 1 < s ? pos + 1 : s;
        u128 chunk = 0;
        for (int b = pos; b > pos - len; b--) chunk = (chunk << 1) | ((w[b / 64] >> (b % 64)) & 1);
        r = ((r << len) | chunk) % par->q;
    }
    return r;
}

/* ---- arithmetic in R = P[alpha]/(alpha^m+1) ---------------------------- */

/* out = x * alpha^k: cyclic shift, negated on wrap (alpha^m = -1). */
static void r_shift(u128* out, const u128* x, int64_t k, const par_t* par) {
    uint32_t m = par->m;
    k %= (int64_t)(2 * m);
    if (k < 0) k += 2 * m;
    for (uint32_t j = 0; j < m; j++) {
        uint64_t t = j + (uint64_t)k;
        int neg = 0;
        while (t >= m) { t -= m; neg = !neg; }
        out[t] = neg ? sub_mod(0, x[j], par->q) : x[j];
    }
}

/* out = x * y, the negacyclic convolution (Section 2.9.2, eq. ncycconv):
 * c_k = sum_{i+j=k} x_i y_j - sum_{i+j=m+k} x_i y_j, with -y_j taken as q - y_j. */
static void r_mul(u128* out, const u128* x, const u128* y, const par_t* par) {
    uint32_t m = par->m;
    uint64_t acc[64][4];
    memset(acc, 0, sizeof(uint64_t) * 4 * m);
    for (uint32_t i = 0; i < m; i++)
        for (uint32_t j = 0; j < m; j++) {
            if (i + j < m) mac256(acc[i + j], x[i], y[j]);
            else mac256(acc[i + j - m], x[i], sub_mod(0, y[j], par->q));
        }
    for (uint32_t k = 0; k < m; k++) out[k] = reduce256(acc[k], par);
}

/* ---- the FFT (Section 3.2.5, Section 4.2) ------------------------------- */

/* Length-n DFT of n elements of R with root alpha^step (n*step = 2m),
 * radix-2 decimation in time: X_k = E_k + w^k O_k, X_{k+n/2} = E_k - w^k O_k,
 * where E, O are the half-length DFTs of the even and odd elements
 * (Section 2.6; the thesis's inner FFT, Section 4.2). */
static void alpha_dft(u128* e, uint64_t n, uint32_t step, const par_t* par) {
    uint32_t m = par->m;
    if (n == 1) return;
    uint64_t half = n / 2;
    u128* ev = malloc(sizeof(u128) * m * half);
    u128* od = malloc(sizeof(u128) * m * half);
    for (uint64_t j = 0; j < half; j++) {
        memcpy(ev + j * m, e + (2 * j) * m, sizeof(u128) * m);
        memcpy(od + j * m, e + (2 * j + 1) * m, sizeof(u128) * m);
    }
    alpha_dft(ev, half, 2 * step, par);
    alpha_dft(od, half, 2 * step, par);
    u128 t[64];
    for (uint64_t k = 0; k < half; k++) {
        r_shift(t, od + k * m, (int64_t)(step * k), par);
        for (uint32_t c = 0; c < m; c++) {
            e[k * m + c] = add_mod(ev[k * m + c], t[c], par->q);
            e[(k + half) * m + c] = sub_mod(ev[k * m + c], t[c], par->q);
        }
    }
    free(ev);
    free(od);
}

/* rho^e = alpha^(e div mu) * rho^(e mod mu), table holds rho^s, s < mu. */
static void rho_power(u128* out, uint64_t e, const u128* table, const par_t* par) {
    e %= par->P2;
    r_shift(out, table + (e % par->mu) * par->m, (int64_t)(e / par->mu), par);
}

/* In place: a (n elements) <- its DFT with root rho^base_pow, natural order. */
static void dkss_fft(u128* a, uint64_t n, uint64_t base_pow, const u128* table, const par_t* par) {
    uint32_t m = par->m, two_m = 2 * m;
    if (n <= two_m) {
        alpha_dft(a, n, (uint32_t)(two_m / n), par);
        return;
    }
    uint64_t mu_n = n / two_m;
    u128* abar = malloc(sizeof(u128) * m * n);   /* row v, column l at (v*mu_n + l) */
    /* i. inner DFTs of the columns e_l(y) = sum_j a_{j mu + l} y^j */
#pragma omp parallel
    {
        u128* el = malloc(sizeof(u128) * m * two_m);
#pragma omp for schedule(static)
        for (int64_t li = 0; li < (int64_t)mu_n; li++) {
            uint64_t l = (uint64_t)li;
            for (uint32_t j = 0; j < two_m; j++)
                memcpy(el + j * m, a + (j * mu_n + l) * m, sizeof(u128) * m);
            alpha_dft(el, two_m, 1, par);
            for (uint32_t v = 0; v < two_m; v++)
                memcpy(abar + (v * mu_n + l) * m, el + v * m, sizeof(u128) * m);
        }
        free(el);
    }
    /* ii. bad multiplications abar_{v,l} *= rho^(v l base_pow) */
#pragma omp parallel for schedule(static)
    for (int64_t vl = 0; vl < (int64_t)(two_m * mu_n); vl++) {
        uint64_t v = (uint64_t)vl / mu_n, l = (uint64_t)vl % mu_n;
        if (l == 0) continue;
        u128 tw[64];
        u128* x = abar + (v * mu_n + l) * m;
        rho_power(tw, v * l * base_pow, table, par);
        r_mul(x, x, tw, par);
    }
    /* iii. outer DFTs of the rows, root rho^(2m base_pow); output f -> 2m f + v */
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t vi = 0; vi < (int32_t)two_m; vi++) {
        uint32_t v = (uint32_t)vi;
        u128* row = abar + v * mu_n * m;
        dkss_fft(row, mu_n, base_pow * two_m, table, par);
        for (uint64_t f = 0; f < mu_n; f++)
            memcpy(a + (two_m * f + v) * m, row + f * m, sizeof(u128) * m);
    }
    free(abar);
}

/* ---- encode / decode (Sections 3.2.4 and 3.2.8) ------------------------- */

static uint64_t get_bits(const uint64_t* a, uint64_t n_words, uint64_t pos, uint32_t len) {
    uint64_t v = 0;
    for (uint32_t b = 0; b < len; b++) {
        uint64_t bit = pos + b;
        if (bit / 64 < n_words && ((a[bit / 64] >> (bit % 64)) & 1)) v |= (uint64_t)1 << b;
    }
    return v;
}

static void encode(u128* out, const uint64_t* a, uint64_t n_words, const par_t* par) {
    memset(out, 0, sizeof(u128) * par->m * par->P2);
#pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < par->M; i++)
        for (uint32_t t = 0; t < par->h; t++)
            out[i * par->m + t] = get_bits(a, n_words, (uint64_t)par->u * (i * par->h + t), par->u);
}

/* c += v * 2^shift on a little-endian word array of length n. */
static void add_shifted(uint64_t* c, uint64_t n, u128 v, uint64_t shift) {
    uint64_t w = shift / 64, s = shift % 64;
    uint64_t parts[3];
    parts[0] = (uint64_t)(v << s);
    parts[1] = s ? (uint64_t)(v >> (64 - s)) : (uint64_t)(v >> 64);
    parts[2] = s ? (uint64_t)((v >> 64) >> (64 - s)) : 0;
    u128 carry = 0;
    for (uint64_t k = w; k < n; k++) {
        u128 add = (k - w < 3) ? parts[k - w] : 0;
        if (k - w >= 3 && carry == 0) break;
        u128 sum = (u128)c[k] + add + carry;
        c[k] = (uint64_t)sum;
        carry = sum >> 64;
    }
}

/* ---- entry points ------------------------------------------------------- */

static int make_par(par_t* par, uint64_t M, uint32_t m, uint32_t u, const uint64_t pz[2]) {
    par->q = ((u128)pz[1] << 64) | pz[0];
    par->m = m; par->h = m / 2; par->u = u;
    par->M = M; par->P2 = 2 * M; par->mu = M / m;
    int bl = bitlen128(par->q);
    if (bl > 126 || m > 64 || m < 2 || M < m || u > 64) return -1;
    par->red_shift = 127 - bl;
    return 0;
}

static void load_r(u128* dst, const uint64_t* src, uint64_t count) {
    for (uint64_t k = 0; k < count; k++) dst[k] = ((u128)src[2 * k + 1] << 64) | src[2 * k];
}

static void store_r(uint64_t* dst, const u128* src, uint64_t count) {
    for (uint64_t k = 0; k < count; k++) { dst[2 * k] = (uint64_t)src[k]; dst[2 * k + 1] = (uint64_t)(src[k] >> 64); }
}

static u128* build_table(const u128* rho, const par_t* par) {
    u128* table = malloc(sizeof(u128) * par->m * par->mu);
    memset(table, 0, sizeof(u128) * par->m);
    table[0] = 1;
    for (uint64_t s = 1; s < par->mu; s++) r_mul(table + s * par->m, table + (s - 1) * par->m, rho, par);
    return table;
}

/* Host threads for the loops above (OpenMP builds); returns the count in
 * effect, 1 when the library was built without OpenMP. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Negacyclic product of two elements of R (m residues of 2 words each). */
int oracle_r_mul(uint32_t m, const uint64_t pz[2], const uint64_t* x, const uint64_t* y, uint64_t* out) {
    par_t par;
    if (make_par(&par, m, m, 1, pz)) return -1;
    u128 X[64], Y[64], C[64];
    load_r(X, x, m); load_r(Y, y, m);
    r_mul(C, X, Y, &par);
    store_r(out, C, m);
    return 0;
}

/* Forward DFT with root rho of a length-2M vector over R (natural order). */
int oracle_fft(uint64_t M, uint32_t m, const uint64_t pz[2], const uint64_t* rho,
               const uint64_t* in, uint64_t* out) {
    par_t par;
    if (make_par(&par, M, m, 1, pz)) return -1;
    u128 R[64];
    load_r(R, rho, m);
    u128* table = build_table(R, &par);
    u128* a = malloc(sizeof(u128) * m * par.P2);
    load_r(a, in, (uint64_t)m * par.P2);
    dkss_fft(a, par.P2, 1, table, &par);
    store_r(out, a, (uint64_t)m * par.P2);
    free(a); free(table);
    return 0;
}

/* c = a * b (Section 3.2).  a, b: ceil(n_bits/64) words; c: 2*ceil(n_bits/64)
 * words.  Optional dumps (2M*m residues of 2 words, natural order, or NULL):
 * a_hat, b_hat, c_hat (componentwise products) and c_poly (after the
 * backwards transform and division by 2M). */
int oracle_dkss_mul(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, const uint64_t pz[2],
                    const uint64_t* rho, const uint64_t* a, const uint64_t* b, uint64_t* c,
                    uint64_t* a_hat, uint64_t* b_hat, uint64_t* c_hat, uint64_t* c_poly) {
    par_t par;
    if (make_par(&par, M, m, u, pz)) return -1;
    uint64_t nw = (n_bits + 63) / 64, len = (uint64_t)m * par.P2;
    u128 R[64];
    load_r(R, rho, m);
    u128* table = build_table(R, &par);
    u128* ea = malloc(sizeof(u128) * len);
    u128* eb = malloc(sizeof(u128) * len);
    encode(ea, a, nw, &par);
    encode(eb, b, nw, &par);
    dkss_fft(ea, par.P2, 1, table, &par);
    dkss_fft(eb, par.P2, 1, table, &par);
    if (a_hat) store_r(a_hat, ea, len);
    if (b_hat) store_r(b_hat, eb, len);
#pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < par.P2; i++) r_mul(ea + i * m, ea + i * m, eb + i * m, &par);
    if (c_hat) store_r(c_hat, ea, len);
    dkss_fft(ea, par.P2, 1, table, &par);
    /* backwards transform: element l is forward output (-l) mod 2M, divided by 2M */
    u128 inv = 1, two_m_p = par.P2 % par.q;
    {   /* inverse of 2M mod q by Fermat-free extended Euclid on u128 */
        __int128 t0 = 0, t1 = 1;
        u128 r0 = par.q, r1 = two_m_p;
        while (r1) {
            u128 qt = r0 / r1, tmp = r0 - qt * r1;
            __int128 tt = t0 - (__int128)qt * t1;
            r0 = r1; r1 = tmp; t0 = t1; t1 = tt;
        }
        inv = (u128)(t0 < 0 ? t0 + (__int128)par.q : t0);
    }
    memset(eb, 0, sizeof(u128) * len);
#pragma omp parallel for schedule(static)
    for (uint64_t l = 0; l < par.P2; l++) {
        uint64_t src = (par.P2 - l) % par.P2;
        for (uint32_t t = 0; t < m; t++) {
            uint64_t acc[4] = {0, 0, 0, 0};
            mac256(acc, ea[src * m + t], inv);
            eb[l * m + t] = reduce256(acc, &par);
        }
    }
    if (c_poly) store_r(c_poly, eb, len);
    memset(c, 0, sizeof(uint64_t) * 2 * nw);
    for (uint64_t i = 0; i < par.P2; i++)
        for (uint32_t t = 0; t < m; t++)
            if (eb[i * m + t]) add_shifted(c, 2 * nw, eb[i * m + t], (uint64_t)u * (i * par.h + t));
    free(ea); free(eb); free(table);
    return 0;
}

/* One output of the forward transform at frequency i = k*mu, where
 * rho^(k mu) = alpha^k (Section 3.2.3): a_hat_{k mu} = sum_j a_j alpha^(k j),
 * the plain definition with shifts and additions only.  Lets a test sample
 * the transform of operands too large for the full oracle.  out: m residues
 * of 2 words. */
int oracle_fft_alpha_point(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, const uint64_t pz[2],
                           const uint64_t* a, uint64_t k, uint64_t* out) {
    par_t par;
    if (make_par(&par, M, m, u, pz)) return -1;
    uint64_t nw = (n_bits + 63) / 64;
    u128 acc[64], el[64], t[64];
    memset(acc, 0, sizeof(acc));
    for (uint64_t j = 0; j < par.M; j++) {
        memset(el, 0, sizeof(el));
        for (uint32_t c = 0; c < par.h; c++) el[c] = get_bits(a, nw, (uint64_t)u * (j * par.h + c), u);
        r_shift(t, el, (int64_t)((k * j) % (2 * m)), &par);
        for (uint32_t c = 0; c < m; c++) acc[c] = add_mod(acc[c], t[c], par.q);
    }
    store_r(out, acc, m);
    return 0;
}
