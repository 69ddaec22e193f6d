// Host-side number theory for a DKSS plan (thesis Section 3.2.2-3.2.3,
// Section 4.2): primality, generator, Hensel lifting, omega, gamma, rho by
// Lagrange interpolation and the table of rho^s.  Residues of Z/p^zZ with
// p^z < 2^126 are unsigned __int128; multiplication is Montgomery with
// R = 2^128 over two 64-bit words.
#pragma once
#include <cstdint>
#include <vector>

namespace dkss_host {

typedef unsigned __int128 u128;

// Arithmetic mod an odd q < 2^127 in Montgomery form (R = 2^128).
struct MontCtx {
    u128 q = 0;
    uint64_t np = 0;   // -q^-1 mod 2^64
    u128 r1 = 0;       // R mod q (Montgomery one)
    u128 r2 = 0;       // R^2 mod q
    explicit MontCtx(u128 modulus);
    u128 mul(u128 a, u128 b) const;            // a*b*R^-1 mod q
    u128 to(u128 x) const { return mul(x % q, r2); }
    u128 from(u128 x) const { return mul(x, 1); }
    u128 add(u128 a, u128 b) const { u128 s = a + b; return s >= q ? s - q : s; }
    u128 sub(u128 a, u128 b) const { return a >= b ? a - b : a + (q - b); }
    u128 pow(u128 base_m, u128 e) const;       // Montgomery in, Montgomery out
    // sum of n products (each operand < q) reduced once: needs n*q < 2^128
    u128 redc256(const uint64_t t[5]) const;
};

// 256-bit accumulator helpers
void mac256(uint64_t acc[5], u128 x, u128 y);

bool is_prime_u64(uint64_t n);                        // deterministic Miller-Rabin
std::vector<uint64_t> prime_factors_u64(uint64_t n);  // trial division
uint64_t smallest_generator(uint64_t p);
u128 hensel_lift(uint64_t zeta, uint64_t p, uint32_t z);  // (p-1)-th root of unity mod p^z
u128 inverse_mod(u128 x, u128 q, u128 phi_minus_one);     // x^(phi-1) mod q

// Proth numbers p = h 2^n + 1 (h odd, h < 2^n, p < 2^126): the thesis's
// primes (Section 4.1, its table of primes of that form).
int jacobi(u128 a, u128 n);                          // Jacobi symbol (a/n), n odd
bool proth_is_prime(uint64_t h, uint32_t n);         // Proth's theorem with a non-residue witness
uint64_t proth_generator(uint64_t h, uint32_t n);    // smallest generator of F_p^*, p - 1 = h 2^n

// Element of R: m residues in Montgomery form.
typedef std::vector<u128> Relem;
Relem r_mul(const MontCtx& c, const Relem& x, const Relem& y);     // negacyclic product
Relem r_pow(const MontCtx& c, const Relem& x, uint64_t e);

struct Roots {
    uint64_t zeta = 0;
    u128 zeta_z = 0, omega = 0, gamma = 0;   // normal form
    Relem rho;                               // normal form
};

// Lagrange interpolation of rho from (gamma^i, omega^i), i odd (eq. dkss:lagrange).
Relem rho_lagrange(const MontCtx& c, u128 omega_m, u128 gamma_m, uint32_t m, u128 phi_minus_one);

}  // namespace dkss_host
