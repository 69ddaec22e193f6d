// Worst-case limb and value bounds of the lazy NTT-form R-multiplication
// (see ntt_bounds.hpp for what is checked and why).
#include "ntt_bounds.hpp"

#include <algorithm>
#include <vector>

namespace dkss_planning {
namespace {

using dkss_host::u128;
constexpr uint64_t kM26 = (1u << 26) - 1;

// Unsigned integer of any size, little-endian base 2^32 (bounds only).
struct Big {
    std::vector<uint32_t> w;
    static Big of(u128 x) {
        Big b;
        while (x) {
            b.w.push_back((uint32_t)x);
            x >>= 32;
        }
        return b;
    }
    void trim() {
        while (!w.empty() && w.back() == 0) w.pop_back();
    }
    Big operator+(const Big& o) const {
        Big r;
        uint64_t c = 0;
        for (size_t i = 0; i < std::max(w.size(), o.w.size()); ++i) {
            c += (i < w.size() ? w[i] : 0u) + (uint64_t)(i < o.w.size() ? o.w[i] : 0u);
            r.w.push_back((uint32_t)c);
            c >>= 32;
        }
        if (c) r.w.push_back((uint32_t)c);
        r.trim();
        return r;
    }
    Big operator*(const Big& o) const {
        Big r;
        r.w.assign(w.size() + o.w.size() + 1, 0);
        for (size_t i = 0; i < w.size(); ++i) {
            uint64_t c = 0;
            for (size_t j = 0; j < o.w.size(); ++j) {
                c += (uint64_t)w[i] * o.w[j] + r.w[i + j];
                r.w[i + j] = (uint32_t)c;
                c >>= 32;
            }
            for (size_t k = i + o.w.size(); c; ++k) {
                c += r.w[k];
                r.w[k] = (uint32_t)c;
                c >>= 32;
            }
        }
        r.trim();
        return r;
    }
    // floor(this / 2^bits)
    Big shr(unsigned bits) const {
        Big r;
        const size_t ws = bits / 32, bs = bits % 32;
        for (size_t i = ws; i < w.size(); ++i) {
            uint64_t v = w[i] >> bs;
            if (bs && i + 1 < w.size()) v |= (uint64_t)w[i + 1] << (32 - bs);
            r.w.push_back((uint32_t)v);
        }
        r.trim();
        return r;
    }
    int cmp(const Big& o) const {
        if (w.size() != o.w.size()) return w.size() < o.w.size() ? -1 : 1;
        for (size_t i = w.size(); i-- > 0;)
            if (w[i] != o.w[i]) return w[i] < o.w[i] ? -1 : 1;
        return 0;
    }
    // value if below 2^64, else UINT64_MAX
    uint64_t u64() const {
        if (w.size() > 2) return UINT64_MAX;
        return (w.size() > 0 ? w[0] : 0) | (w.size() > 1 ? (uint64_t)w[1] << 32 : 0);
    }
    static Big pow2(unsigned bits) {
        Big b;
        b.w.assign(bits / 32 + 1, 0);
        b.w[bits / 32] = 1u << (bits % 32);
        return b;
    }
    Big minus_one() const {   // this - 1 for this > 0
        Big r = *this;
        for (size_t i = 0; i < r.w.size(); ++i)
            if (r.w[i]-- != 0) break;
        r.trim();
        return r;
    }
};

// Worst case of a residue held as LR limbs: each limb's maximum and the value's.
struct Bnd {
    uint64_t l[5] = {0, 0, 0, 0, 0};
    Big v;
};

struct Ctx {
    uint32_t LR;
    u128 q;
    uint64_t qr[5];   // q in 26-bit limbs
    Big qb, rp;       // q, R' = 2^(26 LR)

    Bnd canonical() const {   // a residue below q, normalised limbs
        Bnd b;
        b.v = qb.minus_one();
        for (uint32_t i = 0; i + 1 < LR; ++i) b.l[i] = kM26;
        b.l[LR - 1] = b.v.shr(26 * (LR - 1)).u64();
        return b;
    }
    bool limbs_ok(const Bnd& b) const {
        for (uint32_t i = 0; i < LR; ++i)
            if (b.l[i] >= ((uint64_t)1 << 32)) return false;
        return true;
    }
    Bnd add(const Bnd& a, const Bnd& b) const {
        Bnd r;
        for (uint32_t i = 0; i < LR; ++i) r.l[i] = a.l[i] + b.l[i];
        r.v = a.v + b.v;
        return r;
    }
    Bnd max(const Bnd& a, const Bnd& b) const {
        Bnd r;
        for (uint32_t i = 0; i < LR; ++i) r.l[i] = std::max(a.l[i], b.l[i]);
        r.v = a.v.cmp(b.v) >= 0 ? a.v : b.v;
        return r;
    }
    // Montgomery product with 64-bit columns (rr_arith.cuh, lazy reduction);
    // false on any overflow.
    bool mmul(const Bnd& x, const Bnd& y, Bnd* out) const {
        if (!limbs_ok(x) || !limbs_ok(y)) return false;
        const u128 lim = (u128)1 << 64;
        u128 col[10] = {0};
        for (uint32_t a = 0; a < LR; ++a)
            for (uint32_t b = 0; b < LR; ++b) {
                col[a + b] += (u128)x.l[a] * y.l[b];
                if (col[a + b] >= lim) return false;
            }
        u128 carry = 0;
        for (uint32_t i = 0; i < LR; ++i) {
            const u128 acc = col[i] + carry + (u128)kM26 * qr[0];
            if (acc >= lim) return false;
            carry = acc >> 26;
            for (uint32_t k = 1; k < LR; ++k) {
                col[i + k] += (u128)kM26 * qr[k];
                if (col[i + k] >= lim) return false;
            }
        }
        for (uint32_t i = 0; i < LR; ++i) {
            const u128 v = col[LR + i] + carry;
            if (v >= lim) return false;
            carry = v >> 26;
        }
        // value: (T + Q q) / R' with T <= x.v y.v and Q < R'
        Bnd r;
        r.v = (x.v * y.v + rp.minus_one() * qb).shr(26 * LR);
        const Big top = r.v.shr(26 * (LR - 1));
        if (top.cmp(Big::pow2(32)) >= 0) return false;
        for (uint32_t i = 0; i + 1 < LR; ++i) r.l[i] = kM26;
        r.l[LR - 1] = top.u64();
        *out = r;
        return true;
    }
    // Smallest K with limbs of K q, after moving units down from higher limbs,
    // each at least need[i].
    bool bias(const Bnd& need, uint32_t* limbs, Bnd* as_bnd) const {
        for (uint64_t K = 1; K <= (1u << 16); ++K) {
            const Big v = qb * Big::of(K);
            int64_t n[5];
            for (uint32_t i = 0; i < LR; ++i) {
                const Big part = v.shr(26 * i);
                const uint64_t lo = part.w.empty() ? 0 : part.w[0];
                if (i + 1 < LR) {
                    n[i] = (int64_t)(lo & kM26);
                } else {
                    if (part.cmp(Big::pow2(40)) >= 0) return false;
                    n[i] = (int64_t)part.u64();
                }
            }
            for (uint32_t i = 0; i + 1 < LR; ++i) {
                if (n[i] < (int64_t)need.l[i]) {
                    const int64_t c = ((int64_t)need.l[i] - n[i] + (int64_t)kM26) >> 26;
                    n[i] += c << 26;
                    n[i + 1] -= c;
                }
            }
            bool ok = n[LR - 1] >= (int64_t)need.l[LR - 1];
            for (uint32_t i = 0; i < LR; ++i) ok = ok && n[i] >= 0 && n[i] < ((int64_t)1 << 32);
            if (!ok) continue;
            Bnd b;
            for (uint32_t i = 0; i < LR; ++i) {
                limbs[i] = (uint32_t)n[i];
                b.l[i] = (uint64_t)n[i];
            }
            b.v = v;
            *as_bnd = b;
            return true;
        }
        return false;
    }
    bool below_2q(const Bnd& b) const { return b.v.cmp((qb + qb).minus_one()) <= 0; }
};

}  // namespace

bool ntt_lazy_bounds(uint32_t m, uint32_t LR, u128 q, NttBiases* out) {
    if (LR < 2 || LR > 5 || m < 4 || m > 128 || (m & (m - 1)) != 0) return false;
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    if (lg > 7) return false;
    Ctx c;
    c.LR = LR;
    c.q = q;
    for (uint32_t i = 0; i < 5; ++i) c.qr[i] = i < LR ? (uint64_t)((q >> (26 * i)) & kM26) : 0;
    c.qr[LR - 1] = (uint64_t)(q >> (26 * (LR - 1)));
    c.qb = Big::of(q);
    c.rp = Big::pow2(26 * LR);
    *out = NttBiases{};
    const Bnd C = c.canonical();

    // input: canonical coefficients, or K q - y for the negated ones
    Bnd BN;
    if (!c.bias(C, out->neg, &BN)) return false;
    Bnd X = c.max(C, BN);
    // forward butterflies: t = hi z, lo + t, lo + BF - t.  BF must cover every
    // t; take it first for t < 2q, then again for the largest t that bias gives.
    auto forward = [&](const Bnd& BF, Bnd* Xout, Bnd* tmax) {
        Bnd x = X, tm;
        tm.v = Big();
        for (uint32_t s = 0; s < lg; ++s) {
            Bnd t;
            if (!c.mmul(x, C, &t) || !c.below_2q(t)) return false;
            for (uint32_t i = 0; i < LR; ++i)
                if (BF.l[i] < t.l[i]) return false;
            tm = s ? c.max(tm, t) : t;
            x = c.add(x, BF);
            if (!c.limbs_ok(x)) return false;
        }
        *Xout = x;
        *tmax = tm;
        return true;
    };
    Bnd t_need = C;
    t_need.v = (c.qb + c.qb).minus_one();
    t_need.l[LR - 1] = t_need.v.shr(26 * (LR - 1)).u64();
    Bnd BF, Xf, tmax;
    if (!c.bias(t_need, out->fwd, &BF) || !forward(BF, &Xf, &tmax)) return false;
    {
        uint32_t tight[5];
        Bnd BF2, Xf2, tmax2;
        if (c.bias(tmax, tight, &BF2) && forward(BF2, &Xf2, &tmax2)) {
            for (uint32_t i = 0; i < 5; ++i) out->fwd[i] = tight[i];
            Xf = Xf2;
        }
    }
    X = Xf;
    // DFTs of length <= 2m in evaluation coordinates (eval_levels.cuh): inputs below
    // 2q normalised, Cooley-Tukey butterflies t = b w (the first stage t = b), lo + t,
    // lo + BE - t for log2(2m) stages; then a product by a canonical constant, or a
    // by b after b is scaled (the last level's componentwise products)
    // Butterflies whose twiddle is 1 may take t = b unreduced (stage s with bit
    // s of eval_skip; always at stage 0, whose inputs are reduced), and then
    // stage s's bias covers the stage's inputs too.  Stages are admitted
    // greedily while the whole DFT stays within the limits.
    auto eval_dft = [&](uint32_t skip, NttBiases* o, Bnd* xout) {
        const Bnd E0 = t_need;   // below 2q, normalised
        Bnd x = E0;
        if (lg + 1 > 8) return false;
        o->eval_noscale = 0;
        for (uint32_t s = 0; s <= lg; ++s) {
            Bnd t;
            if (!c.mmul(x, C, &t) || !c.below_2q(t)) return false;
            const Bnd need = (skip >> s) & 1 ? c.max(t, x) : t;
            Bnd B;
            if (!c.bias(need, o->evl[s], &B)) return false;
            x = c.add(x, B);
            if (!c.limbs_ok(x)) return false;
            Bnd ab;   // after 2^(s+1)-point DFTs: a b without scaling b first
            if (c.mmul(x, x, &ab) && c.below_2q(ab)) o->eval_noscale |= 1u << (s + 1);
        }
        Bnd r1, r2, r3;
        if (!(c.mmul(x, C, &r1) && c.below_2q(r1) && c.mmul(x, r1, &r2) && c.below_2q(r2) && c.mmul(r2, C, &r3)))
            return false;
        *xout = x;
        return true;
    };
    {
        Bnd xe;
        uint32_t skip = 1;
        out->eval_ok = eval_dft(skip, out, &xe);
        for (uint32_t s = 1; s <= lg && out->eval_ok; ++s) {
            NttBiases trial = *out;
            if (eval_dft(skip | (1u << s), &trial, &xe)) skip |= 1u << s;
        }
        if (out->eval_ok) out->eval_ok = eval_dft(skip, out, &xe);
        out->eval_skip = skip;
    }
    // componentwise: by a canonical twiddle, or a by b (b scaled first when a b would not fit)
    Bnd P_tw, P_fin;
    if (!c.mmul(X, C, &P_tw)) return false;
    out->prescale = !(c.mmul(X, X, &P_fin) && c.below_2q(P_fin));
    if (out->prescale && !c.mmul(X, P_tw, &P_fin)) return false;
    Bnd U = c.max(P_tw, P_fin);
    // backwards butterflies: lo + hi, (lo + BB_b - hi) z; the last stage multiplies both
    for (uint32_t b = 0; b < lg; ++b) {
        if (b + 1 == lg) {   // the last stage first carry-propagates its inputs to 26-bit limbs
            if (!c.limbs_ok(U)) return false;
            const Big top = U.v.shr(26 * (LR - 1));
            if (top.cmp(Big::pow2(32)) >= 0) return false;
            for (uint32_t i = 0; i + 1 < LR; ++i) U.l[i] = kM26;
            U.l[LR - 1] = top.u64();
        }
        Bnd BB;
        if (!c.bias(U, out->bwd[b], &BB)) return false;
        const Bnd s = c.add(U, U), d = c.add(U, BB);
        if (!c.limbs_ok(s) || !c.limbs_ok(d)) return false;
        Bnd r1, r2;
        if (!c.mmul(d, C, &r2)) return false;
        if (b + 1 == lg) {
            if (!c.mmul(s, C, &r1) || !c.below_2q(r1) || !c.below_2q(r2)) return false;
            // with the twiddle table carrying m^-1, s itself is reduced (reduce_raw):
            // a quotient below 2^12, and q's top two limbs at least 2^18
            if (s.v.cmp(c.qb * Big::of((u128)1 << 12)) >= 0 || c.qb.shr(26 * (LR - 2)).cmp(Big::pow2(18)) < 0)
                return false;
        } else {
            U = c.max(s, r2);
        }
    }
    return true;
}

// Limits of the p-adic digit form (padic.cuh), z = 4 digits: the largest
// digit of every value and every product column, through ntt_forward_pd,
// the componentwise product, ntt_backward_pd and the conversions.
namespace {

struct PdCtx {
    uint64_t p, nmu;        // floor(2^32 / p)
    uint32_t nsh;           // ceil(log2 p)
    bool fast = false;      // fast carries (padic.cuh, ModPD<Z, true>)
    uint64_t mu_lo = 0;     // floor(2^64 / p) mod 2^32
    static constexpr uint64_t kW = (uint64_t)1 << 32;

    // a column below 2^64; with fast carries also c1 mu_lo + c0 nmu + 2^32 < 2^64
    bool col_ok(u128 col) const {
        if (col >> 64) return false;
        if (fast && (u128)(uint64_t)(col >> 32) * mu_lo + (u128)(kW - 1) * nmu + kW >= ((u128)1 << 64)) return false;
        return true;
    }
    // product of digits <= A and <= B: every column (with its carry) within col_ok
    bool mmul_ok(uint64_t A, uint64_t B) const {
        u128 carry = 0;
        for (int k = 0; k < 4; ++k) {
            const u128 col = (u128)(k + 1) * A * B + carry;
            if (!col_ok(col)) return false;
            carry = col / p + 1;
        }
        return true;
    }
    // pd_norm of digits <= V: every digit plus its carry (at most v >> nsh)
    // below 2^32; the result's digits are at most *out
    bool norm(uint64_t V, uint64_t* out) const {
        uint64_t C = 0;
        for (int it = 0; it < 8; ++it) C = (V + C) >> nsh;   // carry bound (fixed point)
        const uint64_t v = V + C;
        if (v >= kW) return false;
        // v - floor(v / 2^nsh) p is largest where floor(v / 2^nsh) is smallest:
        // below v (1 - p / 2^nsh) + p
        *out = ((v * (((uint64_t)1 << nsh) - p)) >> nsh) + p;
        return true;
    }
    // pd_canon of digits <= V: every digit plus its carry (at most v nmu / 2^32) below 2^32
    bool canon_ok(uint64_t V) const {
        uint64_t C = 0;
        for (int it = 0; it < 8; ++it) C = ((V + C) * nmu) >> 32;
        return V + C < kW;
    }
};

}  // namespace

namespace {

bool pd_schedule(const PdCtx& c, uint32_t m, uint32_t L, PdBiases* out);

}  // namespace

bool pd_lazy_bounds(uint64_t p, uint32_t m, uint32_t L, PdBiases* out) {
    *out = PdBiases{};
    if (p < 3 || p >= ((uint64_t)1 << 30) || L < 2 || L > 4) return false;
    PdCtx c;
    c.p = p;
    c.nmu = PdCtx::kW / p;
    c.nsh = 0;
    while (((uint64_t)1 << c.nsh) < p) ++c.nsh;
    if (!pd_schedule(c, m, L, out)) return false;
    // DFTs on digits (dft_dit_pd): canonical inputs; per stage a + y and a - y + 2 (p, p-1, ...),
    // both normalised; the bias covers a normalised digit; up to 7 stages, the last made canonical
    {
        uint64_t N = p - 1;
        out->dft_ok = true;
        for (int st = 0; st < 7 && out->dft_ok; ++st) {
            const uint64_t S = std::max(2 * N, N + 2 * p);
            uint64_t Nn;
            if (N > 2 * (p - 1) || !c.norm(S, &Nn) || !c.canon_ok(S)) out->dft_ok = false;
            else N = Nn;
        }
    }
    // fast carries when floor(2^32 / p) is a power of two and the columns allow them
    if ((c.nmu & (c.nmu - 1)) == 0) {
        PdCtx f = c;
        f.fast = true;
        f.mu_lo = (uint64_t)((((u128)1) << 64) / p) & (PdCtx::kW - 1);
        PdBiases tmp;
        out->fast = pd_schedule(f, m, L, &tmp);
    }
    out->ok = true;
    return true;
}

namespace {

bool pd_schedule(const PdCtx& c, uint32_t m, uint32_t L, PdBiases* out) {
    const uint64_t p = c.p;
    uint32_t lg = 0;
    while ((1u << lg) < m) ++lg;
    const uint64_t C = p - 1;   // a canonical digit
    // conversion from L words: sum_j w_j P_j with canonical P_j
    {
        u128 carry = 0;
        for (int k = 0; k < 4; ++k) {
            const u128 col = (k == 0 ? (u128)(PdCtx::kW - 1) : 0) + (u128)(L - 1) * (PdCtx::kW - 1) * C + carry;
            if (!c.col_ok(col)) return false;
            carry = col / p + 1;
        }
    }
    // forward: inputs canonical or negated (digits <= p), bias K = 1
    out->kf = 1;
    uint64_t V = p;
    for (uint32_t st = 0; st < lg; ++st) {
        if (!c.mmul_ok(V, C)) return false;
        V += p;   // lo + t, lo + D - t
        if (V >= PdCtx::kW) return false;
        if (st % 2 == 1 || st + 1 == lg) {
            if (!c.norm(V, &V)) return false;
        }
    }
    // componentwise: by a canonical twiddle, or a by b's evaluations made canonical
    if (!c.mmul_ok(V, C) || !c.canon_ok(V)) return false;
    // backwards: products canonical, sums normalised after every stage but the last
    uint64_t U = C;
    for (uint32_t b = 0; b < lg; ++b) {
        const uint64_t K = (U + C - 1) / C;   // bias digits K (p - 1) >= U
        if (K > 255) return false;
        out->kb[b] = (uint32_t)K;
        const uint64_t d = U + K * p, s = 2 * U;
        if (d >= PdCtx::kW || s >= PdCtx::kW || !c.mmul_ok(d, C)) return false;
        if (b + 1 == lg) {
            if (!c.mmul_ok(s, C) || !c.canon_ok(s)) return false;   // scaled, or made canonical
        } else {
            uint64_t sn;
            if (!c.norm(s, &sn)) return false;
            U = sn > C ? sn : C;
        }
    }
    return true;
}

}  // namespace

}  // namespace dkss_planning
