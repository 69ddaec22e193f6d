// Host-side number theory for a DKSS plan; see host_math.hpp.
#include "host_math.hpp"

namespace dkss_host {

void mac256(uint64_t acc[5], u128 x, u128 y) {
    uint64_t x0 = (uint64_t)x, x1 = (uint64_t)(x >> 64);
    uint64_t y0 = (uint64_t)y, y1 = (uint64_t)(y >> 64);
    u128 p00 = (u128)x0 * y0, p01 = (u128)x0 * y1, p10 = (u128)x1 * y0, p11 = (u128)x1 * y1;
    u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
    u128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
    uint64_t w[4] = {(uint64_t)p00, (uint64_t)mid, (uint64_t)hi, (uint64_t)(hi >> 64) + (uint64_t)(p11 >> 64)};
    u128 carry = 0;
    for (int k = 0; k < 4; ++k) {
        u128 s = (u128)acc[k] + w[k] + carry;
        acc[k] = (uint64_t)s;
        carry = s >> 64;
    }
    acc[4] += (uint64_t)carry;
}

MontCtx::MontCtx(u128 modulus) : q(modulus) {
    uint64_t q0 = (uint64_t)q;
    uint64_t inv = q0;                      // q0 odd: correct to 3 bits
    for (int i = 0; i < 6; ++i) inv *= 2 - q0 * inv;
    np = (uint64_t)0 - inv;
    r1 = ((u128)0 - q) % q;                 // 2^128 mod q
    r2 = r1;
    for (int i = 0; i < 128; ++i) r2 = add(r2, r2);
}

u128 MontCtx::redc256(const uint64_t tin[5]) const {
    uint64_t t[6] = {tin[0], tin[1], tin[2], tin[3], tin[4], 0};
    uint64_t qw[2] = {(uint64_t)q, (uint64_t)(q >> 64)};
    for (int i = 0; i < 2; ++i) {
        uint64_t qi = t[i] * np;
        u128 carry = 0;
        for (int k = 0; k < 2; ++k) {
            u128 s = (u128)qi * qw[k] + t[i + k] + carry;
            t[i + k] = (uint64_t)s;
            carry = s >> 64;
        }
        for (int k = i + 2; k < 6 && carry; ++k) {
            u128 s = (u128)t[k] + carry;
            t[k] = (uint64_t)s;
            carry = s >> 64;
        }
    }
    u128 r = ((u128)t[3] << 64) | t[2];
    // t[4], t[5] are zero under the caller's bound; r < 2q
    while (r >= q) r -= q;
    return r;
}

u128 MontCtx::mul(u128 a, u128 b) const {
    uint64_t t[5] = {0, 0, 0, 0, 0};
    mac256(t, a, b);
    return redc256(t);
}

u128 MontCtx::pow(u128 base_m, u128 e) const {
    u128 r = r1;
    while (e) {
        if (e & 1) r = mul(r, base_m);
        base_m = mul(base_m, base_m);
        e >>= 1;
    }
    return r;
}

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t n) { return (uint64_t)((u128)a * b % n); }

static uint64_t powmod64(uint64_t b, uint64_t e, uint64_t n) {
    uint64_t r = 1 % n;
    b %= n;
    while (e) {
        if (e & 1) r = mulmod64(r, b, n);
        b = mulmod64(b, b, n);
        e >>= 1;
    }
    return r;
}

bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t s : small) {
        if (n == s) return true;
        if (n % s == 0) return false;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; ++r; }
    for (uint64_t a : small) {
        uint64_t x = powmod64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r; ++i) {
            x = mulmod64(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

std::vector<uint64_t> prime_factors_u64(uint64_t n) {
    std::vector<uint64_t> f;
    if ((n & 1) == 0) {
        f.push_back(2);
        while ((n & 1) == 0) n >>= 1;
    }
    for (uint64_t d = 3; d <= n / d; d += 2) {
        if (n % d == 0) {
            f.push_back(d);
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) f.push_back(n);
    return f;
}

uint64_t smallest_generator(uint64_t p) {
    std::vector<uint64_t> f = prime_factors_u64(p - 1);
    for (uint64_t g = 2; g < p; ++g) {
        bool ok = true;
        for (uint64_t q : f)
            if (powmod64(g, (p - 1) / q, p) == 1) { ok = false; break; }
        if (ok) return g;
    }
    return 0;
}

int jacobi(u128 a, u128 n) {
    a %= n;
    int t = 1;
    while (a != 0) {
        while ((a & 1) == 0) {
            a >>= 1;
            const unsigned r = (unsigned)(n & 7);
            if (r == 3 || r == 5) t = -t;
        }
        u128 tmp = a;
        a = n;
        n = tmp;
        if ((a & 3) == 3 && (n & 3) == 3) t = -t;
        a %= n;
    }
    return n == 1 ? t : 0;
}

// Proth's theorem: p = h 2^n + 1 with h < 2^n is prime iff a^((p-1)/2) = -1
// (mod p) for some a.  With a quadratic non-residue a ((a/p) = -1, Jacobi
// symbol) the test is decisive: for prime p Euler's criterion gives -1.  A
// composite p with no such a below 2^16 (a perfect square, for example) is
// rejected as well.
bool proth_is_prime(uint64_t h, uint32_t n) {
    if (h == 0 || (h & 1) == 0 || n == 0 || n >= 126) return false;
    if (n < 64 && h >= ((uint64_t)1 << n)) return false;
    const u128 p = ((u128)h << n) + 1;
    if ((p >> 126) != 0) return false;
    if (p < 4) return p == 2 || p == 3;
    MontCtx c(p);
    for (uint64_t a = 3; a < 65536; ++a) {
        const int j = jacobi(a, p);
        if (j == 0) return (u128)a == p;     // a shares a factor with p
        if (j == 1) continue;
        return c.pow(c.to(a), (p - 1) / 2) == c.sub(0, c.r1);   // a^((p-1)/2) = -1
    }
    return false;
}

uint64_t proth_generator(uint64_t h, uint32_t n) {
    const u128 p = ((u128)h << n) + 1;
    std::vector<uint64_t> f = prime_factors_u64(h);   // odd prime factors of p - 1
    f.push_back(2);
    MontCtx c(p);
    for (uint64_t g = 2; g < 65536; ++g) {
        bool ok = true;
        for (uint64_t q : f)
            if (c.pow(c.to(g), (p - 1) / q) == c.r1) { ok = false; break; }
        if (ok) return g;
    }
    return 0;
}

u128 inverse_mod(u128 x, u128 q, u128 phi_minus_one) {
    MontCtx c(q);
    return c.from(c.pow(c.to(x), phi_minus_one));
}

// Newton/Hensel step for f(x) = x^(p-1) - 1: x <- x - f(x)/f'(x) mod p^(s+1).
u128 hensel_lift(uint64_t zeta, uint64_t p, uint32_t z) {
    u128 x = zeta % p;
    u128 ps = p;  // p^s
    for (uint32_t s = 1; s < z; ++s) {
        u128 mod = ps * p;
        MontCtx c(mod);
        u128 xm = c.to(x);
        u128 f = c.sub(c.pow(xm, p - 1), c.r1);                     // x^(p-1) - 1
        u128 fp = c.mul(c.to((u128)(p - 1)), c.pow(xm, p - 2));     // (p-1) x^(p-2)
        u128 phi = ps * (p - 1);                                    // phi(p^(s+1))
        u128 fp_inv = c.pow(fp, phi - 1);
        xm = c.sub(xm, c.mul(f, fp_inv));
        x = c.from(xm);
        ps = mod;
    }
    return x;
}

Relem r_mul(const MontCtx& c, const Relem& x, const Relem& y) {
    const size_t m = x.size();
    std::vector<uint64_t> acc(5 * m, 0);
    Relem ny(m);
    for (size_t j = 0; j < m; ++j) ny[j] = y[j] ? c.q - y[j] : 0;
    for (size_t i = 0; i < m; ++i) {
        if (!x[i]) continue;
        for (size_t j = 0; j < m; ++j) {
            size_t k = i + j;
            if (k < m) mac256(&acc[5 * k], x[i], y[j]);
            else mac256(&acc[5 * (k - m)], x[i], ny[j]);
        }
    }
    Relem out(m);
    for (size_t k = 0; k < m; ++k) out[k] = c.redc256(&acc[5 * k]);
    return out;
}

Relem r_pow(const MontCtx& c, const Relem& x, uint64_t e) {
    Relem r(x.size(), 0), b = x;
    r[0] = c.r1;
    while (e) {
        if (e & 1) r = r_mul(c, r, b);
        b = r_mul(c, b, b);
        e >>= 1;
    }
    return r;
}

Relem rho_lagrange(const MontCtx& c, u128 omega_m, u128 gamma_m, uint32_t m, u128 phi_minus_one) {
    std::vector<u128> gp(2 * m), op(2 * m);
    gp[0] = c.r1;
    op[0] = c.r1;
    for (uint32_t i = 1; i < 2 * m; ++i) {
        gp[i] = c.mul(gp[i - 1], gamma_m);
        op[i] = c.mul(op[i - 1], omega_m);
    }
    Relem rho(m, 0);
    for (uint32_t i = 1; i < 2 * m; i += 2) {
        std::vector<u128> li(1, c.r1);
        u128 denom = c.r1;
        for (uint32_t j = 1; j < 2 * m; j += 2) {
            if (j == i) continue;
            std::vector<u128> nl(li.size() + 1, 0);
            for (size_t k = 0; k < li.size(); ++k) {
                nl[k + 1] = c.add(nl[k + 1], li[k]);
                nl[k] = c.sub(nl[k], c.mul(li[k], gp[j]));
            }
            li.swap(nl);
            denom = c.mul(denom, c.sub(gp[i], gp[j]));
        }
        u128 scale = c.mul(op[i], c.pow(denom, phi_minus_one));
        for (uint32_t k = 0; k < m; ++k) rho[k] = c.add(rho[k], c.mul(scale, li[k]));
    }
    return rho;
}

}  // namespace dkss_host
