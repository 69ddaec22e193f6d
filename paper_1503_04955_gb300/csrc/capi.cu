// C ABI of libdkss (declarations and contracts in include/dkss.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "plan.hpp"

using dkss_host::MontCtx;
using dkss_host::Relem;
using dkss_host::u128;

// test hook: DKSS_FAULT_* bits set by dkss_fault_inject (0 in normal use)
static std::atomic<uint32_t> g_fault{0};

namespace dkss_planning {

const uint64_t kCandidatePrimes[kNumCandidatePrimes] = {12289, 40961, 65537, 786433, 7340033, 23068673,
                                                        104857601, 167772161, 469762049, 998244353};

uint32_t fault_mask() { return g_fault.load(); }

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

uint32_t log2u(uint64_t x) {
    uint32_t r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

int bitlen(u128 x) {
    int n = 0;
    while (x) { ++n; x >>= 1; }
    return n;
}

// 2^bits mod q by doubling (bits may exceed 128)
u128 pow2_mod(int bits, u128 q) {
    u128 r = 1 % q;
    for (int i = 0; i < bits; ++i) {
        r <<= 1;            // r < q < 2^126: no overflow
        if (r >= q) r -= q;
    }
    return r;
}

// x < 2^bits for a 256-bit value held as 5 little-endian words
bool below_pow2(const uint64_t t[5], int bits) {
    for (int w = 4; w >= 0; --w) {
        int lo = 64 * w;
        if (t[w] == 0) continue;
        int top = lo + 63 - __builtin_clzll(t[w]);
        return top < bits;
    }
    return true;
}

}  // namespace dkss_planning

namespace {
using namespace dkss_planning;

typedef dkss_status (*run_mul_fn)(dkss_plan_s*, const uint64_t*, const uint64_t*, uint64_t*, cudaStream_t);
typedef dkss_status (*run_fwd_fn)(dkss_plan_s*, const uint64_t*, uint64_t*, cudaStream_t);
typedef dkss_status (*prep_fn)(dkss_plan_s*);

struct Kernels {
    run_mul_fn mul;
    run_fwd_fn fwd;
    prep_fn prep;
};

template <int m, int L, int LR>
Kernels kernels_for() {
    return Kernels{&dkss::run_mul<m, L, LR>, &dkss::run_forward<m, L, LR>, &dkss::prepare<m, L, LR>};
}

bool lookup(uint32_t m, uint32_t L, uint32_t LR, Kernels* k) {
#define DKSS_CASE(M_, L_, LR_) \
    if (m == M_ && L == L_ && LR == LR_) { *k = kernels_for<M_, L_, LR_>(); return true; }
#define DKSS_CASES(M_) \
    DKSS_CASE(M_, 2, 2) DKSS_CASE(M_, 2, 3) DKSS_CASE(M_, 3, 3) DKSS_CASE(M_, 3, 4) DKSS_CASE(M_, 4, 4) DKSS_CASE(M_, 4, 5)
    DKSS_CASES(16) DKSS_CASES(32) DKSS_CASES(64)
#undef DKSS_CASES
#undef DKSS_CASE
    return false;
}

}  // namespace

namespace dkss_planning {

// Everything of a plan that needs no device: parameter checks (Section 3.2
// steps 1-2), roots (Section 3.2.3) and the limb layout.
// Shape checks shared by every ring (Section 3.2 step 1).
static dkss_status check_shape(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u) {
    if (!is_pow2(M) || !is_pow2(m) || m < 2 || M < m || n_bits == 0 || u == 0 || u > 32) return DKSS_EPARAM;
    if (M >= ((uint64_t)1 << 40)) return DKSS_EPARAM;
    if ((u128)M * (m / 2) * u < n_bits) return DKSS_EPARAM;
    return DKSS_OK;
}

static dkss_status plan_ring(dkss_plan_s* pl, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, u128 p, uint32_t z,
                             u128 q, uint64_t zeta, u128 zeta_z);

dkss_status plan_host(dkss_plan_s* pl, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t p, uint32_t z) {
    if (check_shape(n_bits, M, m, u) != DKSS_OK || z == 0) return DKSS_EPARAM;
    const uint64_t P2 = 2 * M;
    if (p < 3 || !dkss_host::is_prime_u64(p) || (p - 1) % P2 != 0) return DKSS_EPARAM;
    u128 q = 1;
    for (uint32_t i = 0; i < z; ++i) {
        if (q > (((u128)1 << 126) / p)) return DKSS_EPARAM;
        q *= p;
    }
    const u128 umax = ((u128)1 << u) - 1;
    if (!(q > (u128)M * (m / 2) * umax * umax)) return DKSS_EPARAM;  // largest coefficient
    const uint64_t zeta = dkss_host::smallest_generator(p);
    return plan_ring(pl, n_bits, M, m, u, p, z, q, zeta, dkss_host::hensel_lift(zeta, p, z));
}

// z = 1 and the Proth prime p = h 2^n + 1 (Section 4.1: the thesis's primes).
dkss_status plan_host_proth(dkss_plan_s* pl, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t h,
                            uint32_t n) {
    if (check_shape(n_bits, M, m, u) != DKSS_OK) return DKSS_EPARAM;
    if (h == 0 || (h >> 32) != 0 || (h & 1) == 0 || n == 0 || n + (uint32_t)bitlen(h) > 126) return DKSS_EPARAM;
    if (((u128)1 << n) % (2 * M) != 0) return DKSS_EPARAM;          // 2M | p - 1
    if (!dkss_host::proth_is_prime(h, n)) return DKSS_EPARAM;
    const u128 p = ((u128)h << n) + 1;
    const u128 umax = ((u128)1 << u) - 1;
    if (!(p > (u128)M * (m / 2) * umax * umax)) return DKSS_EPARAM;
    const uint64_t zeta = dkss_host::proth_generator(h, n);
    if (zeta == 0) return DKSS_EPARAM;
    return plan_ring(pl, n_bits, M, m, u, p, 1, p, zeta, zeta);
}

// The Proth ring with the sparse reduction at a given LR: n = max(26 (LR-1),
// log2 2M) and the smallest odd h with p = h 2^n + 1 prime, above the
// coefficient bound, m p < 2^(26 LR - 2), and a plan with that LR.
bool proth_ring_lr(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint32_t LR, uint64_t* h_out,
                   uint32_t* n_out) {
    if (check_shape(n_bits, M, m, u) != DKSS_OK || LR < 3 || LR > 5) return false;
    const u128 umax = ((u128)1 << u) - 1;
    const u128 bound = (u128)M * (m / 2) * umax * umax;
    const uint32_t n = std::max<uint32_t>(26 * (LR - 1), log2u(2 * M));
    const int top = 26 * (int)LR - 2 - (int)log2u(m);       // m p < 2^(26 LR - 2)
    if (top <= (int)n || top > 126) return false;
    uint64_t h = (uint64_t)(bound >> n) + 1;
    h |= 1;
    for (int tries = 0; tries < 200000; ++tries, h += 2) {
        if ((h >> 32) != 0 || (int)(n + bitlen(h)) > top) break;
        if (!dkss_host::proth_is_prime(h, n)) continue;
        dkss_plan_s pl;
        if (plan_host_proth(&pl, n_bits, M, m, u, h, n) != DKSS_OK) continue;
        if (pl.LR != LR || !pl.q_sparse) continue;
        *h_out = h;
        *n_out = n;
        return true;
    }
    return false;
}

// Everything of a plan that needs no device, once the ring Z/qZ (q = p^z) and
// a (p-1)-th root of unity zeta_z mod q are fixed: limb layout, roots
// (Section 3.2.3) and the constants of the lazy arithmetic.
static dkss_status plan_ring(dkss_plan_s* pl, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, u128 p, uint32_t z,
                             u128 q, uint64_t zeta, u128 zeta_z) {
    const uint64_t P2 = 2 * M;
    if ((u128)m * q >= ((u128)1 << 127)) return DKSS_EUNSUPPORTED;  // host sums of m products; 4 m q < 2^130
    // limbs: one spare bit for sums, and m q^2 + R q < 2^(64L) for the REDC of m-term sums
    uint32_t L = (uint32_t)((bitlen(q) + 1 + 31) / 32);
    if (L < 2) L = 2;
    for (;; ++L) {
        if (L > 4) return DKSS_EUNSUPPORTED;
        // t = m q^2 + q 2^(32L) must stay below 2^(64L)
        uint64_t t[5] = {0, 0, 0, 0, 0};
        dkss_host::mac256(t, q, q * m);
        uint64_t add[6] = {0, 0, 0, 0, 0, 0};
        const int sh = 32 * (int)L;
        const uint64_t qw[2] = {(uint64_t)q, (uint64_t)(q >> 64)};
        for (int i = 0; i < 2; ++i) {
            const int bit = sh + 64 * i, w = bit / 64, s = bit % 64;
            add[w] |= qw[i] << s;
            if (s) add[w + 1] |= qw[i] >> (64 - s);
        }
        u128 carry = 0;
        for (int i = 0; i < 5; ++i) {
            u128 s2 = (u128)t[i] + add[i] + carry;
            t[i] = (uint64_t)s2;
            carry = s2 >> 64;
        }
        if (!carry && !add[5] && below_pow2(t, 64 * (int)L)) break;
    }
    if (m != 16 && m != 32 && m != 64) return DKSS_EUNSUPPORTED;
    if (P2 <= 2 * (uint64_t)m) return DKSS_EUNSUPPORTED;

    pl->n_bits = n_bits; pl->M = M; pl->P2 = P2; pl->mu_top = P2 / (2 * m); pl->p = p;
    pl->m = m; pl->u = u; pl->z = z; pl->L = L; pl->q = q;
    pl->log2_mu_top = log2u(pl->mu_top);
    // levels: ceil(log2 2M / log2 2m) - 1 radix-2m levels, then one of length <= 2m
    const uint32_t lg = log2u(P2), k = log2u(2 * m);
    pl->col_levels = (lg + k - 1) / k - 1;
    pl->r_last = P2 >> (k * pl->col_levels);
    for (uint32_t i = 0; i < 4; ++i) pl->q_limbs[i] = i < L ? (uint32_t)(q >> (32 * i)) : 0;
    {
        uint32_t q0 = (uint32_t)q, inv = q0;
        for (int i = 0; i < 5; ++i) inv *= 2 - q0 * inv;
        pl->nprime = 0u - inv;
    }
    const int RB = 32 * (int)L;
    pl->nsub = (uint32_t)(RB >= 128 ? 0 : (uint64_t)(((u128)m * q) >> RB)) + 1;
    // products in 26-bit limbs: 4 m q < R' = 2^(26 LR) keeps every REDC input of the
    // direct convolution and of the transform in R below q R'
    uint32_t LR = 2;
    while (LR <= 5 && (26 * LR < 127 && (((u128)m * q) >> (26 * LR - 2)) != 0)) ++LR;
    if (LR > 5 || LR < L || LR > L + 1) return DKSS_EUNSUPPORTED;
    pl->LR = LR;
    pl->i8_S = (uint32_t)((bitlen(q) + 7) / 8);   // bytes of a residue (INT8 form)
    for (uint32_t i = 0; i < 5; ++i) pl->q_rr[i] = i < LR ? (uint32_t)(q >> (26 * i)) & ((1u << 26) - 1) : 0;
    {
        uint32_t q0 = (uint32_t)q, inv = q0;
        for (int i = 0; i < 5; ++i) inv *= 2 - q0 * inv;
        pl->nprime26 = (0u - inv) & ((1u << 26) - 1);
    }
    pl->q_sparse = LR >= 3 && pl->q_rr[0] == 1;
    for (uint32_t i = 1; i + 1 < LR; ++i) pl->q_sparse = pl->q_sparse && pl->q_rr[i] == 0;

    // roots (Section 3.2.3)
    MontCtx c(q);
    u128 phi = q / p * (p - 1);
    dkss_host::Roots& r = pl->roots;
    r.zeta = zeta;
    r.zeta_z = zeta_z;
    u128 omega_m = c.pow(c.to(r.zeta_z), (p - 1) / P2);
    u128 gamma_m = c.pow(omega_m, pl->mu_top);
    r.omega = c.from(omega_m);
    r.gamma = c.from(gamma_m);
    Relem rho_m = dkss_host::rho_lagrange(c, omega_m, gamma_m, m, phi - 1);
    if (g_fault.load() & DKSS_FAULT_RHO) rho_m[1] = c.add(rho_m[1], c.r1);   // test hook: the checks must fail
    // checks the thesis fixes: rho^(2M/2m) = alpha, rho^M = -1
    Relem t1 = dkss_host::r_pow(c, rho_m, pl->mu_top);
    Relem t2 = dkss_host::r_pow(c, rho_m, M);
    for (uint32_t i = 0; i < m; ++i) {
        if (t1[i] != (i == 1 ? c.r1 : 0)) return DKSS_EPARAM;
        if (t2[i] != (i == 0 ? q - c.r1 : 0)) return DKSS_EPARAM;
    }
    r.rho.resize(m);
    for (uint32_t i = 0; i < m; ++i) r.rho[i] = c.from(rho_m[i]);
    // (2M)^-1 R'^2 mod q, the scaling factor applied through one Montgomery product
    const int RRB = 26 * (int)LR;
    u128 rdev = pow2_mod(RRB, q);
    u128 p2inv = c.pow(c.to(P2 % q), phi - 1);          // Montgomery form
    u128 rdev_m = c.to(rdev);
    u128 ks = c.from(c.mul(c.mul(p2inv, rdev_m), rdev_m));
    for (uint32_t i = 0; i < 5; ++i) pl->kscale[i] = i < LR ? (uint32_t)(ks >> (26 * i)) & ((1u << 26) - 1) : 0;
    // limits of the lazy transform in R (NTT form of the R-multiplications)
    pl->ntt_ok = ntt_lazy_bounds(m, LR, q, &pl->ntt_bias);
    pl->eval_levels = (pl->flags & DKSS_LEVELS_EVAL) && !(pl->flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC)) &&
                      m <= 32 && pl->ntt_ok && pl->ntt_bias.eval_ok;
    return DKSS_OK;
}

// rho^s R' mod q for s < mu_top (R' = 2^(26 LR)), m residues of LR 26-bit limbs each.
void build_table(const dkss_plan_s* pl, std::vector<uint32_t>& out) {
    const uint32_t m = pl->m, L = pl->LR;
    const uint64_t mu = pl->mu_top;
    out.assign(mu * m * L, 0);
    MontCtx c(pl->q);
    Relem rho_m(m);
    for (uint32_t i = 0; i < m; ++i) rho_m[i] = c.to(pl->roots.rho[i]);
    u128 rdev = pow2_mod(26 * (int)L, pl->q);
    unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    uint64_t chunks = std::min<uint64_t>(hw, mu);
    std::vector<std::thread> th;
    for (uint64_t ci = 0; ci < chunks; ++ci) {
        th.emplace_back([&, ci]() {
            uint64_t s0 = mu * ci / chunks, s1 = mu * (ci + 1) / chunks;
            Relem cur = dkss_host::r_pow(c, rho_m, s0);
            for (uint64_t s = s0; s < s1; ++s) {
                for (uint32_t t = 0; t < m; ++t) {
                    u128 v = c.mul(cur[t], rdev);   // rho^s_t * R' mod q
                    for (uint32_t w = 0; w < L; ++w)
                        out[(s * m + t) * L + w] = (uint32_t)(v >> (26 * w)) & ((1u << 26) - 1);
                }
                if (s + 1 < s1) cur = dkss_host::r_mul(c, cur, rho_m);
            }
        });
    }
    for (auto& t : th) t.join();
}

u128 to_dev(const MontCtx& c, u128 v_m, u128 rdev) { return c.mul(v_m, rdev); }

void put_rr(uint32_t* dst, u128 v, uint32_t LR) {
    for (uint32_t w = 0; w < LR; ++w) dst[w] = (uint32_t)(v >> (26 * w)) & ((1u << 26) - 1);
}

// the four base-p digits of a canonical residue (p-adic digit form, padic.cuh)
void put_pd(uint32_t* dst, u128 v, u128 p) {
    for (uint32_t k = 0; k < 4; ++k) {
        dst[k] = (uint32_t)(v % p);
        v /= p;
    }
}

// K (p, p-1, p-1, p-1): digits of K p^4, zero mod p^4
void put_pd_bias(uint32_t* dst, uint32_t K, u128 p) {
    for (uint32_t k = 0; k < 4; ++k) dst[k] = (uint32_t)(K * (k == 0 ? p : p - 1));
}

uint32_t brv(uint32_t x, uint32_t bits) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// Constants of the transform in R (ntt_rmul.cuh, NttLayout): psi = gamma.
// Constants of the transform in p-adic digits (padic.cuh, PdLayout): the
// entries of NttLayout as plain residues, biases K (p, p-1, p-1, p-1), then the
// digits of 2^(32j) mod p^4, j < 4.
// Residue index of the digits of 2^(32j) mod p^4 in that table (PdLayout<m>::POW32).
uint32_t pd_pow32_index(uint32_t m) {
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    const uint32_t Q = 2 * m + lg + 2, PSI = Q + 7 + lg + 1;
    return PSI + 2 * m;
}

void build_ntt_consts_pd(const dkss_plan_s* pl, std::vector<uint32_t>& out) {
    constexpr uint32_t Z = 4;
    const uint32_t m = pl->m;
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    const uint32_t Q = 2 * m + lg + 2, COUNT = pd_pow32_index(m);
    out.assign((size_t)(COUNT + 4) * Z, 0);
    MontCtx c(pl->q);
    const u128 phi = pl->q / pl->p * (pl->p - 1);
    const u128 psi = c.to(pl->roots.gamma);
    const u128 psi_inv = c.pow(psi, phi - 1);
    auto put = [&](uint32_t idx, u128 v_m) { put_pd(&out[(size_t)idx * Z], c.from(v_m), pl->p); };
    for (uint32_t k = 1; k < m; ++k) {
        put(k, c.pow(psi, brv(k, lg)));
        put(m + k, c.pow(psi_inv, brv(k, lg)));
    }
    for (uint32_t b = 0; b < lg; ++b) put_pd_bias(&out[(size_t)(2 * m + b) * Z], pl->pd_bias.kb[b], pl->p);
    put_pd_bias(&out[(size_t)(2 * m + lg) * Z], pl->pd_bias.kf, pl->p);
    put_pd_bias(&out[(size_t)(2 * m + lg + 1) * Z], pl->pd_bias.kf, pl->p);
    const u128 minv = c.pow(c.to(m), phi - 1);
    const u128 p2inv = c.pow(c.to(pl->P2 % pl->q), phi - 1);
    const u128 zlast = c.pow(psi_inv, brv(1, lg));
    put(Q + 1, minv);
    put(Q + 2, c.mul(zlast, minv));
    put(Q + 3, c.mul(minv, p2inv));
    put(Q + 4, c.mul(c.mul(zlast, minv), p2inv));
    put(Q + 5, c.to(1));
    put(Q + 6, zlast);
    u128 pw = 1;
    for (uint32_t j = 0; j < 4; ++j) {
        put_pd(&out[(size_t)(COUNT + j) * Z], pw, pl->p);
        pw = c.from(c.mul(c.to(pw), c.to(((u128)1 << 32) % pl->q)));
    }
}

void build_ntt_consts(const dkss_plan_s* pl, std::vector<uint32_t>& out) {
    if (pl->padic) {
        build_ntt_consts_pd(pl, out);
        return;
    }
    const uint32_t m = pl->m, LR = pl->LR;
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    // layout of NttLayout<m> (ntt_rmul.cuh)
    const uint32_t Q = 2 * m + lg + 2, PSI = Q + 7 + lg + 1, COUNT = PSI + 2 * m;
    out.assign((size_t)COUNT * LR, 0);
    MontCtx c(pl->q);
    const u128 rdev = pow2_mod(26 * (int)LR, pl->q);
    const u128 phi = pl->q / pl->p * (pl->p - 1);
    const u128 psi = c.to(pl->roots.gamma);
    const u128 psi_inv = c.pow(psi, phi - 1);
    for (uint32_t k = 1; k < m; ++k) {
        put_rr(&out[(size_t)k * LR], to_dev(c, c.pow(psi, brv(k, lg)), rdev), LR);
        put_rr(&out[(size_t)(m + k) * LR], to_dev(c, c.pow(psi_inv, brv(k, lg)), rdev), LR);
    }
    // lazy-arithmetic biases (ntt_bounds.cpp): backwards stages, forward, negation
    for (uint32_t b = 0; b < lg; ++b)
        for (uint32_t i = 0; i < LR; ++i) out[(size_t)(2 * m + b) * LR + i] = pl->ntt_bias.bwd[b][i];
    for (uint32_t i = 0; i < LR; ++i) {
        out[(size_t)(2 * m + lg) * LR + i] = pl->ntt_bias.fwd[i];
        out[(size_t)(2 * m + lg + 1) * LR + i] = pl->ntt_bias.neg[i];
    }
    put_rr(&out[(size_t)Q * LR], pl->q, LR);
    const u128 minv = c.pow(c.to(m), phi - 1);
    const u128 p2inv = c.pow(c.to(pl->P2 % pl->q), phi - 1);
    const u128 zlast = c.pow(psi_inv, brv(1, lg));
    put_rr(&out[(size_t)(Q + 1) * LR], to_dev(c, minv, rdev), LR);
    put_rr(&out[(size_t)(Q + 2) * LR], to_dev(c, c.mul(zlast, minv), rdev), LR);
    // componentwise products multiply two normal-form factors, so their scaling
    // constants carry one more R' to cancel the product's R'^-1
    const u128 rdev_m = c.to(rdev);
    put_rr(&out[(size_t)(Q + 3) * LR], to_dev(c, c.mul(c.mul(minv, p2inv), rdev_m), rdev), LR);
    put_rr(&out[(size_t)(Q + 4) * LR], to_dev(c, c.mul(c.mul(c.mul(zlast, minv), p2inv), rdev_m), rdev), LR);
    // last backwards stage after a prescaled componentwise product: 1 and psi^-1
    put_rr(&out[(size_t)(Q + 5) * LR], rdev, LR);
    put_rr(&out[(size_t)(Q + 6) * LR], to_dev(c, zlast, rdev), LR);
    // DFTs in evaluation coordinates: their stage biases and the powers psi^t, t < 2m
    for (uint32_t st = 0; st <= lg; ++st)
        for (uint32_t i = 0; i < LR; ++i) out[(size_t)(Q + 7 + st) * LR + i] = pl->ntt_bias.evl[st][i];
    u128 pt = c.to(1);
    for (uint32_t t = 0; t < 2 * m; ++t) {
        put_rr(&out[(size_t)(PSI + t) * LR], to_dev(c, pt, rdev), LR);
        pt = c.mul(pt, psi);
    }
}

// Bad twiddles of levels d >= 1 in evaluation coordinates (eval_levels.cuh):
// rho^e(gamma^(2j+1)) = omega^(e(2j+1)) for every e = e' b_d (b_d = (2m)^d),
// e' < 2M / b_d, at index i with j = brv(i), in device Montgomery form.  Level
// d's table starts at word offs[d].
void build_eval_level_tables(const dkss_plan_s* pl, std::vector<uint32_t>& out, std::vector<uint64_t>& offs) {
    const uint32_t m = pl->m, LR = pl->LR;
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    MontCtx c(pl->q);
    const u128 rdev = pow2_mod(26 * (int)LR, pl->q);
    const u128 om = c.to(pl->roots.omega);
    offs.assign(pl->col_levels + 1, 0);
    uint64_t total = 0, bp = 1;
    for (uint32_t d = 0; d < pl->col_levels; ++d) {
        offs[d] = total;
        if (d > 0) total += (pl->P2 / bp) * m * LR;
        bp *= 2 * m;
    }
    offs[pl->col_levels] = total;
    out.assign(total, 0);
    bp = 2 * m;
    for (uint32_t d = 1; d < pl->col_levels; ++d, bp *= 2 * m) {
        const uint64_t n = pl->P2 / bp;
        const u128 wb = c.pow(om, bp);   // omega^(b_d)
        unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        uint64_t chunks = std::min<uint64_t>(hw, n);
        std::vector<std::thread> th;
        for (uint64_t ci = 0; ci < chunks; ++ci) {
            th.emplace_back([&, ci]() {
                uint64_t e0 = n * ci / chunks, e1 = n * (ci + 1) / chunks;
                u128 w = c.pow(wb, e0);
                std::vector<u128> val(m);
                for (uint64_t e = e0; e < e1; ++e) {
                    u128 w2 = c.mul(w, w), cur = w;
                    for (uint32_t j = 0; j < m; ++j) {
                        val[j] = cur;
                        cur = c.mul(cur, w2);
                    }
                    for (uint32_t i = 0; i < m; ++i)
                        put_rr(&out[offs[d] + (e * m + i) * LR], to_dev(c, val[brv(i, lg)], rdev), LR);
                    w = c.mul(w, wb);
                }
            });
        }
        for (auto& t : th) t.join();
    }
}

// Evaluations of the bad twiddles: rho^s(gamma^(2j+1)) = omega^(s(2j+1)), stored
// for s < mu_top at index i with j = brv(i), in device Montgomery form; for the
// R-multiplications of the coefficient levels each entry also carries the
// backward transform's m^-1 (ntt_backward<RAW_LO>), for the levels in
// evaluation coordinates not.
void build_eval_table(const dkss_plan_s* pl, std::vector<uint32_t>& out, bool with_minv) {
    const uint32_t m = pl->m, LR = pl->padic ? 4u : pl->LR;
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    const uint64_t mu = pl->mu_top;
    out.assign(mu * m * LR, 0);
    MontCtx c(pl->q);
    const u128 rdev = pow2_mod(26 * (int)LR, pl->q);
    const u128 om = c.to(pl->roots.omega);
    const u128 phi = pl->q / pl->p * (pl->p - 1);
    const u128 scale = with_minv ? c.pow(c.to(m), phi - 1) : c.to(1);   // m^-1 or 1
    unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    uint64_t chunks = std::min<uint64_t>(hw, mu);
    std::vector<std::thread> th;
    for (uint64_t ci = 0; ci < chunks; ++ci) {
        th.emplace_back([&, ci]() {
            uint64_t s0 = mu * ci / chunks, s1 = mu * (ci + 1) / chunks;
            u128 ws = c.pow(om, s0);
            std::vector<u128> val(m);
            for (uint64_t s = s0; s < s1; ++s) {
                u128 w2 = c.mul(ws, ws), cur = ws;
                for (uint32_t j = 0; j < m; ++j) {
                    val[j] = cur;
                    cur = c.mul(cur, w2);
                }
                for (uint32_t i = 0; i < m; ++i) {
                    if (pl->padic) put_pd(&out[(s * m + i) * LR], c.from(c.mul(val[brv(i, lg)], scale)), pl->p);
                    else put_rr(&out[(s * m + i) * LR], to_dev(c, c.mul(val[brv(i, lg)], scale), rdev), LR);
                }
                ws = c.mul(ws, om);
            }
        });
    }
    for (auto& t : th) t.join();
}

}  // namespace dkss_planning

namespace {
using namespace dkss_planning;

void free_device(dkss_plan_s* pl) {
    cudaFree(pl->d_table);
    cudaFree(pl->d_work);
    cudaFree(pl->d_agg);
    cudaFree(pl->d_status);
    cudaFree(pl->d_stage);
    cudaFree(pl->d_ntt);
    cudaFree(pl->d_evtw);
    cudaFree(pl->d_table_minv);
    cudaFree(pl->d_half);
    pl->d_half = nullptr;
    pl->d_ntt = nullptr;
    pl->d_evtw = nullptr;
    pl->d_table_minv = nullptr;
    pl->d_table = nullptr; pl->d_work = nullptr; pl->d_agg = nullptr; pl->d_status = nullptr; pl->d_stage = nullptr;
}

bool overlap(const void* a, size_t an, const void* b, size_t bn) {
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bn && y < x + an;
}

void fill_consts(const dkss_plan_s* pl, uint64_t* consts, size_t n) {
    const uint64_t form = (pl->flags & DKSS_FORM_INT8TC)                          ? 2
                          : ((pl->flags & DKSS_RMUL_DIRECT) || !pl->ntt_ok)         ? 1
                          : pl->eval_levels                                          ? 3
                                                                                     : 0;
    uint64_t v[25] = {pl->P2, pl->mu_top, pl->L, (uint64_t)pl->col_levels + 1, (uint64_t)pl->q,
                      (uint64_t)(pl->q >> 64), pl->roots.zeta, (uint64_t)pl->roots.omega,
                      (uint64_t)(pl->roots.omega >> 64), (uint64_t)pl->roots.gamma,
                      (uint64_t)(pl->roots.gamma >> 64), pl->LR, form,
                      (uint64_t)(pl->ntt_ok && pl->ntt_bias.prescale),
                      (uint64_t)(pl->ntt_ok && pl->ntt_bias.eval_ok && pl->m <= 32), pl->ntt_bias.eval_skip,
                      pl->M, pl->m, pl->u, (uint64_t)pl->p, pl->z, (uint64_t)(pl->p >> 64), pl->q_sparse ? 1u : 0u,
                      pl->dev_bytes, pl->padic ? 1u : 0u};
    for (size_t i = 0; i < n && i < 25; ++i) consts[i] = v[i];
}

}  // namespace

namespace {
using namespace dkss_planning;

// One valid parameter set with its limb and level structure.
struct Cand {
    uint64_t M, p;
    uint32_t m, u, z, L, LR, levels;
    uint64_t r_last, P2;
    uint32_t S;   // bytes of p^z (INT8 form)
};

const uint64_t* kCandPrimes = dkss_planning::kCandidatePrimes;

// Every (M, m, u, p, z) for N-bit operands that dkss_plan accepts and this
// build has kernels for: m in {16, 32, 64}, u in {8, 16, 24, 32}, the smallest
// M with M (m/2) u >= N and 2M > 2m, each listed prime with 2M | p-1 and the
// smallest z above the coefficient bound (Section 3.2.2).
std::vector<Cand> enumerate_candidates(uint64_t n_bits) {
    static const uint32_t ms[] = {16, 32, 64};
    static const uint32_t us[] = {8, 16, 24, 32};
    std::vector<Cand> out;
    for (uint32_t m : ms)
        for (uint32_t u : us) {
            const uint64_t per = (uint64_t)(m / 2) * u;
            uint64_t M = 1;
            while (M * per < n_bits || M <= m) M <<= 1;
            for (size_t ip = 0; ip < kNumCandidatePrimes; ++ip) {
                const uint64_t p = kCandPrimes[ip];
                if ((p - 1) % (2 * M) != 0) continue;
                for (uint32_t z = 1; z <= 8; ++z) {
                    dkss_plan_s pl;
                    const dkss_status s = plan_host(&pl, n_bits, M, m, u, p, z);
                    if (s == DKSS_EPARAM) continue;     // p^z below the bound: try the next z
                    Kernels k;
                    if (s == DKSS_OK && lookup(pl.m, pl.L, pl.LR, &k))
                        out.push_back(Cand{M, p, m, u, z, pl.L, pl.LR, pl.col_levels + 1, pl.r_last, pl.P2, pl.i8_S});
                    break;   // the smallest z that passes the bound (or an unsupported one) ends the search
                }
            }
        }
    return out;
}

// The thesis's rule (Section 4.1): the largest u, then the smallest M m,
// then M/m closest to N / log2(N)^3; then the fewest limbs and p^z just
// above the coefficient bound (the smallest p^z of those left).
bool rule_less(const Cand& a, const Cand& b, uint64_t n_bits) {
    const double lg = std::log2((double)n_bits);
    const double target = std::log2((double)n_bits / (lg * lg * lg));
    auto key = [&](const Cand& c) {
        u128 q = 1;
        for (uint32_t i = 0; i < c.z; ++i) q *= c.p;
        return std::make_tuple(-(int)c.u, c.M * c.m, std::fabs(std::log2((double)c.M / c.m) - target), c.L, c.LR,
                               q);
    };
    return key(a) < key(b);
}

// Arithmetic work of a product with candidate c, for picking which
// candidates to time: R-multiplications ((3 levels' worth of twiddles + the
// componentwise products) of m log m Montgomery products of LR^2 limb
// products each) and the bytes of one pass per level over three polynomials.
double work_estimate(const Cand& c) {
    const double rmuls = (3.0 * (c.levels - 1) + 1.0) * (double)c.P2;
    const double lgm = std::log2((double)c.m);
    const double ops = rmuls * c.m * lgm * c.LR * c.LR;
    const double bytes = (double)c.P2 * c.m * c.L * 4.0 * (2.0 * c.levels + 1.0);
    return ops / 20.0 + bytes / 6.0;    // about 20 T multiply-adds/s against 6 TB/s
}

bool form_ok(const Cand& c, uint32_t flags) {
    if (flags & DKSS_FORM_INT8TC) return c.m >= 32 && c.S <= 16;   // a warp per element, at most 16 bytes
    return true;
}

// Measured operands are bounded so that timing a candidate stays cheap.
constexpr uint64_t kTuneMaxBits = (uint64_t)1 << 26;
constexpr int kTuneCandidates = 4;

std::mutex g_tune_mu;
std::map<std::tuple<int, uint64_t, uint32_t>, Cand> g_tune_cache;   // (device, N, flags) -> choice

// Median device time (ms) of one product with candidate c on the current
// device, operands of N bits with every limb 0x5a5a... (the top limb masked).
double time_candidate(uint64_t n_bits, const Cand& c, uint32_t flags, bool* ok) {
    *ok = false;
    dkss_plan_t pl = nullptr;
    if (dkss_plan(&pl, n_bits, c.M, c.m, c.u, c.p, c.z, flags & ~(uint32_t)DKSS_PROFILE) != DKSS_OK) return 0;
    const size_t nw = (n_bits + 63) / 64;
    uint64_t* buf = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> ts;
    if (cudaMalloc(&buf, 4 * nw * sizeof(uint64_t)) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMemsetAsync(buf, 0x5a, 2 * nw * sizeof(uint64_t), st) == cudaSuccess) {
        const int top = (int)(n_bits - 64 * (nw - 1));
        const uint64_t last = top < 64 ? (0x5a5a5a5a5a5a5a5aull & ((1ull << top) - 1)) : 0x5a5a5a5a5a5a5a5aull;
        bool good = cudaMemcpyAsync(buf + nw - 1, &last, 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                    cudaMemcpyAsync(buf + 2 * nw - 1, &last, 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;
        for (int rep = 0; good && rep < 4; ++rep) {
            good = cudaEventRecord(e0, st) == cudaSuccess &&
                   dkss_mul(pl, buf, buf + nw, buf + 2 * nw, (dkss_stream_t)st) == DKSS_OK &&
                   cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float t = 0;
            if (good && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0) ts.push_back(t);
        }
        *ok = good && dkss_sync_status(pl, (dkss_stream_t)st) == DKSS_OK && !ts.empty();
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    dkss_plan_destroy(pl);
    if (!*ok) return 0;
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

// Parameters for dkss_plan(..., 0, 0, 0, 0, 0, flags): the thesis's rule
// alone for large N or with DKSS_TUNE_RULE, else the fastest measured of the
// rule's choice and the candidates with the least estimated work; cached per
// (device, N, flags) for the life of the process.
dkss_status choose_params(uint64_t n_bits, uint32_t flags, Cand* out) {
    std::vector<Cand> all = enumerate_candidates(n_bits), cands;
    for (const Cand& c : all)
        if (form_ok(c, flags)) cands.push_back(c);
    if (cands.empty()) return DKSS_EUNSUPPORTED;
    const Cand rule = *std::min_element(cands.begin(), cands.end(),
                                        [&](const Cand& a, const Cand& b) { return rule_less(a, b, n_bits); });
    if ((flags & DKSS_TUNE_RULE) || n_bits > kTuneMaxBits) {
        *out = rule;
        return DKSS_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DKSS_ECUDA;
    const auto key = std::make_tuple(dev, n_bits, flags & ~(uint32_t)DKSS_PROFILE);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            return DKSS_OK;
        }
    }
    // candidates with the same kernels and shapes cost the same: keep one of each
    std::vector<Cand> uniq;
    for (const Cand& c : cands) {
        bool dup = false;
        for (const Cand& d : uniq)
            dup |= d.M == c.M && d.m == c.m && d.u == c.u && d.L == c.L && d.LR == c.LR && d.levels == c.levels &&
                   d.r_last == c.r_last;
        if (!dup) uniq.push_back(c);
    }
    std::sort(uniq.begin(), uniq.end(), [](const Cand& a, const Cand& b) { return work_estimate(a) < work_estimate(b); });
    std::vector<Cand> timed{rule};
    for (const Cand& c : uniq) {
        if ((int)timed.size() >= kTuneCandidates + 1) break;
        if (!(c.M == rule.M && c.m == rule.m && c.u == rule.u && c.L == rule.L && c.LR == rule.LR)) timed.push_back(c);
    }
    Cand best = rule;
    double best_ms = 0;
    bool any = false;
    for (const Cand& c : timed) {
        bool ok = false;
        const double ms = time_candidate(n_bits, c, flags, &ok);
        if (ok && (!any || ms < best_ms)) {
            best = c;
            best_ms = ms;
            any = true;
        }
    }
    *out = best;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = best;
    return DKSS_OK;
}

dkss_status finish_plan(dkss_plan_s* pl, dkss_status s, dkss_plan_t* plan);

}  // namespace

extern "C" {

uint32_t dkss_fault_inject(uint32_t mask) { return g_fault.exchange(mask); }

dkss_status dkss_plan(dkss_plan_t* plan, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t p, uint32_t z,
                      uint32_t flags) {
    if (!plan) return DKSS_EINVAL;
    *plan = nullptr;
    if (M == 0 && m == 0 && u == 0 && p == 0 && z == 0) {   // parameters chosen by the library
        if (n_bits == 0) return DKSS_EPARAM;
        Cand c{};
        const dkss_status cs = choose_params(n_bits, flags, &c);
        if (cs != DKSS_OK) return cs;
        M = c.M; m = c.m; u = c.u; p = c.p; z = c.z;
    }
    dkss_plan_s* pl = (g_fault.load() & DKSS_FAULT_HOST_ALLOC) ? nullptr : new (std::nothrow) dkss_plan_s;
    if (!pl) return DKSS_ENOMEM;
    pl->flags = flags;
    return finish_plan(pl, plan_host(pl, n_bits, M, m, u, p, z), plan);
}

dkss_status dkss_plan_proth(dkss_plan_t* plan, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t h,
                            uint32_t n, uint32_t flags) {
    if (!plan) return DKSS_EINVAL;
    *plan = nullptr;
    dkss_plan_s* pl = (g_fault.load() & DKSS_FAULT_HOST_ALLOC) ? nullptr : new (std::nothrow) dkss_plan_s;
    if (!pl) return DKSS_ENOMEM;
    pl->flags = flags;
    return finish_plan(pl, plan_host_proth(pl, n_bits, M, m, u, h, n), plan);
}

}  // extern "C"

namespace {
// Device half of a plan whose host half (pl, status s) is done: kernel
// lookup, tables, workspace.  Takes ownership of pl.
dkss_status finish_plan(dkss_plan_s* pl, dkss_status s, dkss_plan_t* plan) {
    const uint32_t flags = pl->flags;
    const uint64_t n_bits = pl->n_bits;
    Kernels k;
    if (s == DKSS_OK && !lookup(pl->m, pl->L, pl->LR, &k)) s = DKSS_EUNSUPPORTED;
    // the INT8 tensor-core form needs a warp per element and at most 16 bytes per residue
    if (s == DKSS_OK && (flags & DKSS_FORM_INT8TC) && (pl->m < 32 || pl->i8_S > 16)) s = DKSS_EUNSUPPORTED;
    if (s != DKSS_OK) {
        delete pl;
        return s;
    }
    // a ring outside the lazy transform's limits takes the direct convolution
    if (!pl->ntt_ok && !(flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC))) pl->flags |= DKSS_RMUL_DIRECT;
    // inner levels in evaluation coordinates: the NTT form, m <= 32, within their limits
    pl->eval_levels = pl->eval_levels && !(pl->flags & DKSS_RMUL_DIRECT);
    // m = 64 forward half-column DFTs: unreduced between stages where 2^7 p^z fits L words and the
    // top word of p^z is at least 2^8 (the final reduction's quotient estimate)
    {
        const uint32_t qtop = pl->q_limbs[pl->L - 1];
        pl->dft_lazy = pl->m == 64 && pl->L >= 3 && bitlen(pl->q) + 7 <= 32 * pl->L && qtop >= 256;
        pl->red_rcp = pl->dft_lazy ? (uint32_t)(((uint64_t)1 << 40) / ((uint64_t)qtop + 1)) : 0;
    }
    // m = 64 NTT kernels over p^4 with p < 2^30: p-adic digits (padic.cuh) within their limits,
    // where they take fewer multiply-adds than the Montgomery products: with fast carries
    // (floor(2^32/p) a power of two), or against five 26-bit limbs.  Four limbs with the
    // generic carries measured slower (p = 7340033: 12.3 against 11.3 ms at 2^28 bits).
    pl->padic = !(pl->flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC | DKSS_ARITH_MONT)) && pl->m == 64 &&
                pl->z == 4 && pl->p < ((u128)1 << 30) && !pl->q_sparse &&
                pd_lazy_bounds((uint64_t)pl->p, pl->m, pl->L, &pl->pd_bias) &&
                (pl->pd_bias.fast || pl->LR >= 5);
    if (pl->padic) {
        const uint64_t p = (uint64_t)pl->p;
        uint32_t s = 0;
        while ((p >> (s + 1)) != 0) ++s;
        pl->pd_s = s;
        pl->pd_nmu = (uint32_t)(((uint64_t)1 << 32) / p);
        pl->pd_mu = (uint64_t)((((u128)1) << (64 + s)) / p);
        pl->pd_fast = pl->pd_bias.fast;
        // residues of 4 words hold 4 digits as well: the forward levels keep them in HBM
        pl->pd_io = pl->L == 4 && pl->pd_bias.dft_ok;
        pl->pd_pw_off = (uint64_t)pd_pow32_index(pl->m) * 4;
        pl->pd_mu_lo = (uint32_t)((((u128)1) << 64) / p);
        while ((1u << (pl->pd_lg_nmu + 1)) <= pl->pd_nmu) ++pl->pd_lg_nmu;
    }
    if (cudaGetDevice(&pl->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess) {
        delete pl;
        return DKSS_ECUDA;
    }
    std::vector<uint32_t> table, ntt;
    if (pl->flags & (DKSS_RMUL_DIRECT | DKSS_FORM_INT8TC)) build_table(pl, table);
    else build_eval_table(pl, table, !pl->eval_levels);
    // levels in evaluation coordinates: dkss_forward still runs coefficient levels
    std::vector<uint32_t> table_minv;
    if (pl->eval_levels) build_eval_table(pl, table_minv, true);
    build_ntt_consts(pl, ntt);
    std::vector<uint32_t> evtw;
    if (pl->eval_levels) build_eval_level_tables(pl, evtw, pl->evtw_offs);
    pl->poly_words = pl->P2 * pl->m * pl->L;
    const uint64_t nw = (n_bits + 63) / 64;
    pl->n_tiles = (4 * nw + 2047) / 2048;
    bool ok = cudaMalloc(&pl->d_table, table.size() * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&pl->d_work, 2 * pl->poly_words * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&pl->d_agg, pl->n_tiles * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&pl->d_status, sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&pl->d_ntt, ntt.size() * sizeof(uint32_t)) == cudaSuccess &&
              (evtw.empty() || cudaMalloc(&pl->d_evtw, evtw.size() * sizeof(uint32_t)) == cudaSuccess) &&
              (table_minv.empty() || cudaMalloc(&pl->d_table_minv, table_minv.size() * sizeof(uint32_t)) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        free_device(pl);
        delete pl;
        return DKSS_ENOMEM;
    }
    pl->dev_bytes = 4 * (table.size() + 2 * pl->poly_words + pl->n_tiles + 1 + ntt.size() + evtw.size() +
                         table_minv.size());
    if (cudaMemcpy(pl->d_table, table.data(), table.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->d_ntt, ntt.data(), ntt.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!evtw.empty() &&
         cudaMemcpy(pl->d_evtw, evtw.data(), evtw.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!table_minv.empty() && cudaMemcpy(pl->d_table_minv, table_minv.data(), table_minv.size() * sizeof(uint32_t),
                                           cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(pl->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
        free_device(pl);
        delete pl;
        return DKSS_ECUDA;
    }
    dkss_status ps = k.prep(pl);
    if (ps != DKSS_OK) {
        free_device(pl);
        delete pl;
        return ps;
    }
    *plan = pl;
    return DKSS_OK;
}

}  // namespace

extern "C" {

dkss_status dkss_mul(dkss_plan_t pl, const uint64_t* a, const uint64_t* b, uint64_t* out, dkss_stream_t stream) {
    if (!pl || !a || !b || !out) return DKSS_EINVAL;
    const size_t nw = (pl->n_bits + 63) / 64;
    if (overlap(out, 16 * nw, a, 8 * nw) || overlap(out, 16 * nw, b, 8 * nw)) return DKSS_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pl->device) return DKSS_EINVAL;
    Kernels k;
    if (!lookup(pl->m, pl->L, pl->LR, &k)) return DKSS_EUNSUPPORTED;
    return k.mul(pl, a, b, out, (cudaStream_t)stream);
}

dkss_status dkss_sqr(dkss_plan_t pl, const uint64_t* a, uint64_t* out, dkss_stream_t stream) {
    return dkss_mul(pl, a, a, out, stream);
}

dkss_status dkss_mul_host(dkss_plan_t pl, const uint64_t* a_host, const uint64_t* b_host, uint64_t* out_host,
                          dkss_stream_t stream) {
    if (!pl || !a_host || !b_host || !out_host) return DKSS_EINVAL;
    const size_t nw = (pl->n_bits + 63) / 64;
    if (!pl->d_stage && cudaMalloc(&pl->d_stage, 4 * nw * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        pl->d_stage = nullptr;
        return DKSS_ENOMEM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* da = pl->d_stage;
    uint64_t* db = pl->d_stage + nw;
    uint64_t* dout = pl->d_stage + 2 * nw;
    if (cudaMemcpyAsync(da, a_host, nw * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(db, b_host, nw * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return DKSS_ECUDA;
    dkss_status s = dkss_mul(pl, da, db, dout, stream);
    if (s != DKSS_OK) return s;
    if (cudaMemcpyAsync(out_host, dout, 2 * nw * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DKSS_ECUDA;
    return DKSS_OK;
}

dkss_status dkss_forward(dkss_plan_t pl, const uint64_t* a, uint64_t* out, dkss_stream_t stream) {
    if (!pl || !a || !out) return DKSS_EINVAL;
    Kernels k;
    if (!lookup(pl->m, pl->L, pl->LR, &k)) return DKSS_EUNSUPPORTED;
    return k.fwd(pl, a, out, (cudaStream_t)stream);
}

dkss_status dkss_plan_info(dkss_plan_t pl, uint64_t* consts, size_t n_consts, uint64_t* rho_out) {
    if (!pl) return DKSS_EINVAL;
    if (consts) fill_consts(pl, consts, n_consts);
    if (rho_out)
        for (uint32_t i = 0; i < pl->m; ++i) {
            rho_out[2 * i] = (uint64_t)pl->roots.rho[i];
            rho_out[2 * i + 1] = (uint64_t)(pl->roots.rho[i] >> 64);
        }
    return DKSS_OK;
}

dkss_status dkss_plan_rho(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t p, uint32_t z,
                          uint64_t* rho_out, uint64_t* consts, size_t n_consts) {
    dkss_plan_s pl;
    dkss_status s = plan_host(&pl, n_bits, M, m, u, p, z);
    if (s != DKSS_OK) return s;
    return dkss_plan_info(&pl, consts, n_consts, rho_out);
}

dkss_status dkss_plan_proth_rho(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t h, uint32_t n,
                                uint64_t* rho_out, uint64_t* consts, size_t n_consts) {
    dkss_plan_s pl;
    dkss_status s = plan_host_proth(&pl, n_bits, M, m, u, h, n);
    if (s != DKSS_OK) return s;
    return dkss_plan_info(&pl, consts, n_consts, rho_out);
}

dkss_status dkss_proth_ring(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t* h_out, uint32_t* n_out) {
    if (!h_out || !n_out) return DKSS_EINVAL;
    if (check_shape(n_bits, M, m, u) != DKSS_OK) return DKSS_EPARAM;
    for (uint32_t LR = 3; LR <= 5; ++LR)
        if (proth_ring_lr(n_bits, M, m, u, LR, h_out, n_out)) return DKSS_OK;
    return DKSS_EUNSUPPORTED;
}

dkss_status dkss_plan_choose(uint64_t n_bits, uint32_t flags, uint64_t* params) {
    if (!params || n_bits == 0) return DKSS_EINVAL;
    Cand c{};
    const dkss_status s = choose_params(n_bits, flags, &c);
    if (s != DKSS_OK) return s;
    params[0] = c.M; params[1] = c.m; params[2] = c.u; params[3] = c.p; params[4] = c.z;
    return DKSS_OK;
}

dkss_status dkss_plan_candidates(uint64_t n_bits, uint64_t* rows, size_t max_rows, size_t* n_rows) {
    if (!n_rows || n_bits == 0) return DKSS_EINVAL;
    const std::vector<Cand> all = enumerate_candidates(n_bits);
    for (size_t i = 0; rows && i < all.size() && i < max_rows; ++i) {
        const Cand& c = all[i];
        const uint64_t v[10] = {c.M, c.m, c.u, c.p, c.z, c.L, c.LR, c.levels, c.r_last, c.P2};
        for (int k = 0; k < 10; ++k) rows[10 * i + k] = v[k];
    }
    *n_rows = all.size();
    return DKSS_OK;
}

uint32_t dkss_plan_launches(dkss_plan_t pl) { return pl ? pl->launches : 0; }

dkss_status dkss_sync_status(dkss_plan_t pl, dkss_stream_t stream) {
    if (!pl) return DKSS_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DKSS_ECUDA;
    uint32_t st = 0;
    if (cudaMemcpy(&st, pl->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return DKSS_ECUDA;
    if (cudaMemset(pl->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return DKSS_ECUDA;
    if (st & dkss::kStatusTimeout) return DKSS_ETIMEOUT;
    if (st) return DKSS_EDEVICE;
    return DKSS_OK;
}

dkss_status dkss_profile_read(dkss_plan_t pl, double* ms, uint64_t* counts, size_t n) {
    if (!pl) return DKSS_EINVAL;
    dkss_status status = DKSS_OK;
    for (auto& r : pl->prof) {
        float t = 0.f;
        if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess)
            status = DKSS_ECUDA;
        if (r.kind >= 0 && r.kind < 8) {
            pl->prof_ms[r.kind] += t;
            pl->prof_count[r.kind] += 1;
        }
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    pl->prof.clear();
    for (size_t i = 0; i < n && i < 8; ++i) {
        if (ms) ms[i] = pl->prof_ms[i];
        if (counts) counts[i] = pl->prof_count[i];
        pl->prof_ms[i] = 0;
        pl->prof_count[i] = 0;
    }
    return status;
}

dkss_status dkss_plan_destroy(dkss_plan_t pl) {
    if (!pl) return DKSS_OK;
    cudaDeviceSynchronize();
    dkss_profile_read(pl, nullptr, nullptr, 0);
    free_device(pl);
    delete pl;
    return DKSS_OK;
}

const char* dkss_status_str(dkss_status s) {
    switch (s) {
        case DKSS_OK: return "ok";
        case DKSS_EINVAL: return "invalid argument";
        case DKSS_EPARAM: return "parameters violate the DKSS conditions";
        case DKSS_ENOMEM: return "out of memory";
        case DKSS_EUNSUPPORTED: return "unsupported parameters or form";
        case DKSS_ECUDA: return "CUDA runtime error";
        case DKSS_ETIMEOUT: return "device-side wait timed out";
        case DKSS_EDEVICE: return "device-side inconsistency";
    }
    return "unknown status";
}

}  // extern "C"
