"""Plain CPU oracle for DKSS multiplication (test infrastructure only).

This module is the correctness reference for the CUDA library.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product path never calls it and shares no code with it.

It follows C. Lueders, "Fast Multiplication of Large Integers: Implementation
and Analysis of the DKSS Algorithm" (arXiv:1503.04955), Chapter 3, step by
step and in the thesis's notation, using Python integers (exact, slow).  Every
function cites the passage it restates.  Heavy sizes use the C transcription in
``oracle/dkss_oracle.c`` (same steps, 128-bit residues); the root and parameter
math below feeds both.

Notation (Section 3.2): the ring P = Z/p^zZ, R = P[alpha]/(alpha^m + 1),
transform length 2M (called ``P2`` here), mu = 2M/2m, u input bits per inner
coefficient, h = m/2 inner coefficients filled per outer coefficient.

Pins: every function below is checked in ``tests/test_oracle_pins.py`` against
something other than itself (printed values of the thesis, closed forms,
invariants the thesis proves, brute force on tiny inputs, the exact integer
product).  None is parity-unpinned.
"""
from dataclasses import dataclass, field


# ---------------------------------------------------------------------------
# Integer helpers (Section 3.2.2: primality and roots)
# ---------------------------------------------------------------------------

def prime_factors(n):
    """Distinct prime factors of n > 0 by trial division."""
    out = []
    d = 2
    while d * d <= n:
        if n % d == 0:
            out.append(d)
            while n % d == 0:
                n //= d
        d += 1 if d == 2 else 2
    if n > 1:
        out.append(n)
    return out


def lucas_is_prime(n):
    """Lucas primality test (Section 3.2.2; Crandall-Pomerance Thm 4.1.1).

    n is prime iff some a has a^(n-1) = 1 (mod n) and a^((n-1)/q) != 1 (mod n)
    for every prime q dividing n-1.  The thesis uses it because p - 1 = h*2M
    is fully factored.  A composite n fails the Fermat condition for some
    a < n, so the scan terminates with False."""
    if n < 2:
        return False
    if n < 4:
        return True
    if n % 2 == 0:
        return False
    qs = prime_factors(n - 1)
    for a in range(2, n):
        if pow(a, n - 1, n) != 1:
            return False
        if all(pow(a, (n - 1) // q, n) != 1 for q in qs):
            return True
    return False


def smallest_generator(p):
    """Smallest generator zeta of F_p^* (Section 3.2.3 needs 'a generator';
    the smallest one is this project's reading of that choice)."""
    qs = prime_factors(p - 1)
    for g in range(2, p):
        if all(pow(g, (p - 1) // q, p) != 1 for q in qs):
            return g
    raise ValueError("no generator: p is not prime")


def hensel_lift(zeta, p, z):
    """Hensel lifting of f(x) = x^(p-1) - 1 from a root mod p to a root mod
    p^z (Section 3.2.3, Hensel's theorem): zeta_{s+1} = zeta_s - f(zeta_s)/f'(zeta_s)
    taken mod p^(s+1), repeated z-1 times."""
    x = zeta % p
    for s in range(1, z):
        mod = p ** (s + 1)
        f = (pow(x, p - 1, mod) - 1) % mod
        fprime = ((p - 1) * pow(x, p - 2, mod)) % mod
        x = (x - f * pow(fprime, -1, mod)) % mod
    return x


# ---------------------------------------------------------------------------
# Parameters (Section 3.2, steps 1-3)
# ---------------------------------------------------------------------------

@dataclass
class Params:
    n_bits: int      # N: operands are < 2^N
    M: int           # degree-bound of the encoded polynomials
    m: int           # degree-bound of elements of R
    u: int           # input bits per inner coefficient
    p: int
    z: int
    pz: int = field(init=False)
    P2: int = field(init=False)   # 2M, the transform length
    mu: int = field(init=False)   # 2M / 2m
    h: int = field(init=False)    # m / 2

    def __post_init__(self):
        self.pz = self.p ** self.z
        self.P2 = 2 * self.M
        self.mu = self.P2 // (2 * self.m)
        self.h = self.m // 2

    def check(self):
        """The conditions of Section 3.2 steps 1-2, with the exact coefficient
        bound of Section 3.2.2 (inner coefficients reach (1/2) M m (2^u - 1)^2)."""
        def pow2(x):
            return x >= 1 and x & (x - 1) == 0
        assert pow2(self.M) and pow2(self.m) and self.m >= 2 and self.M >= self.m
        assert self.M * self.h * self.u >= self.n_bits
        assert lucas_is_prime(self.p) and (self.p - 1) % self.P2 == 0
        assert self.pz > self.M * self.h * ((1 << self.u) - 1) ** 2
        return self


@dataclass
class Roots:
    zeta: int      # generator of F_p^*
    zeta_z: int    # its Hensel lift: a (p-1)-th root of unity mod p^z
    omega: int     # principal 2M-th root of unity in P
    gamma: int     # omega^mu, principal 2m-th root of unity in P
    rho: list      # principal 2M-th root of unity in R with rho^mu = alpha


def compute_roots(par):
    """zeta, zeta_z, omega = zeta_z^h with h = (p-1)/2M, gamma = omega^mu and rho
    by Lagrange interpolation (Section 3.2.3, eq. dkss:lagrange)."""
    zeta = smallest_generator(par.p)
    zeta_z = hensel_lift(zeta, par.p, par.z)
    omega = pow(zeta_z, (par.p - 1) // par.P2, par.pz)
    gamma = pow(omega, par.mu, par.pz)
    rho = rho_lagrange(omega, gamma, par.m, par.pz)
    return Roots(zeta, zeta_z, omega, gamma, rho)


def poly_mul_linear(poly, c, q):
    """(sum poly[k] x^k) * (x - c) mod q, full degree (no wrap)."""
    out = [0] * (len(poly) + 1)
    for k, a in enumerate(poly):
        out[k + 1] = (out[k + 1] + a) % q
        out[k] = (out[k] - a * c) % q
    return out


def rho_lagrange(omega, gamma, m, q):
    """rho(alpha) = sum over odd i in [1, 2m-1] of omega^i * l_i(alpha), with
    l_i(alpha) = prod over odd j != i of (alpha - gamma^j) / (gamma^i - gamma^j)
    (Section 3.2.3, eq. dkss:lagrange).  The result has degree < m."""
    odd = list(range(1, 2 * m, 2))
    rho = [0] * m
    for i in odd:
        li = [1]
        denom = 1
        gi = pow(gamma, i, q)
        for j in odd:
            if j == i:
                continue
            gj = pow(gamma, j, q)
            li = poly_mul_linear(li, gj, q)
            denom = denom * (gi - gj) % q
        scale = pow(omega, i, q) * pow(denom, -1, q) % q
        for k in range(m):
            rho[k] = (rho[k] + scale * li[k]) % q
    return rho


# ---------------------------------------------------------------------------
# Arithmetic in R = P[alpha]/(alpha^m + 1)
# ---------------------------------------------------------------------------

def r_zero(m):
    return [0] * m


def r_one(m):
    return [1] + [0] * (m - 1)


def r_add(x, y, q):
    return [(a + b) % q for a, b in zip(x, y)]


def r_sub(x, y, q):
    return [(a - b) % q for a, b in zip(x, y)]


def r_shift(x, k, q):
    """x * alpha^k: a cyclic shift where coefficients passing degree m wrap
    around with changed sign, because alpha^m = -1 (Section 3.2.5, i.)."""
    m = len(x)
    k %= 2 * m
    out = [0] * m
    for j, a in enumerate(x):
        t = j + k
        sign = 1
        while t >= m:
            t -= m
            sign = -sign
        out[t] = (out[t] + sign * a) % q
    return out


def r_mul(x, y, q):
    """Negacyclic convolution (Section 2.9.2, eq. ncycconv):
    c_k = sum_{i+j=k} x_i y_j - sum_{i+j=m+k} x_i y_j, taken mod q."""
    m = len(x)
    c = [0] * m
    for i in range(m):
        for j in range(m):
            if i + j < m:
                c[i + j] += x[i] * y[j]
            else:
                c[i + j - m] -= x[i] * y[j]
    return [v % q for v in c]


def r_pow(x, e, q):
    """x^e in R by binary exponentiation."""
    result = r_one(len(x))
    base = list(x)
    while e:
        if e & 1:
            result = r_mul(result, base, q)
        base = r_mul(base, base, q)
        e >>= 1
    return result


def r_alpha_pow(k, m, q):
    return r_shift(r_one(m), k, q)


# ---------------------------------------------------------------------------
# Encoding (Section 3.2.4 "Distribution of Input Bits", Fig. dkss:fig:encode)
# ---------------------------------------------------------------------------

def encode(a, par):
    """a < 2^N -> 2M outer coefficients in R.  Outer coefficient i < M takes the
    um/2-bit block i of a; inside it, inner coefficient t < m/2 takes u bits.
    Upper m/2 inner coefficients and upper M outer coefficients are zero."""
    mask = (1 << par.u) - 1
    out = []
    for i in range(par.P2):
        el = [0] * par.m
        if i < par.M:
            for t in range(par.h):
                el[t] = (a >> (par.u * (i * par.h + t))) & mask
        out.append(el)
    return out


def decode(c, par):
    """Evaluate inner polynomials at alpha = 2^u and outer ones at x = 2^(um/2)
    (Section 3.2.8); Python's integer addition performs the carries."""
    total = 0
    for i, el in enumerate(c):
        for t, v in enumerate(el):
            total += v << (par.u * (i * par.h + t))
    return total


# ---------------------------------------------------------------------------
# The FFT (Section 3.2.5 steps i-iii and Section 4.2)
# ---------------------------------------------------------------------------

def rho_table(rho, par):
    """rho^s for s in [0, mu), so that rho^i = alpha^r * rho^s with i = r*mu + s
    (Section 4.2, the precomputed powers)."""
    tab = [r_one(par.m)]
    for _ in range(1, par.mu):
        tab.append(r_mul(tab[-1], rho, par.pz))
    return tab


def rho_power(e, table, par):
    """rho^e = alpha^(e div mu) * rho^(e mod mu) (Section 4.2)."""
    e %= par.P2
    return r_shift(table[e % par.mu], e // par.mu, par.pz)


def alpha_dft(e, step, par):
    """Length-n DFT with root alpha^step (n * step = 2m): the plain definition
    E_v = sum_j e_j alpha^(step*j*v), using only shifts and additions
    (inner DFTs of Section 3.2.5 i.; the last level when the length is <= 2m)."""
    n = len(e)
    out = []
    for v in range(n):
        acc = r_zero(par.m)
        for j in range(n):
            acc = r_add(acc, r_shift(e[j], step * j * v, par.pz), par.pz)
        out.append(acc)
    return out


def dkss_fft(a, table, par, base_pow=1, dump=None):
    """DFT of the vector a (length n, a power of 2 dividing 2M) with root
    rho^base_pow, returned in natural order: out[k] = sum_j a_j rho^(base_pow*j*k).

    Section 3.2.5: write a as 2m rows of mu' = n/2m columns; i. inner DFTs of the
    columns e_l with root alpha give abar_{v,l} = e_l(alpha^v); ii. bad
    multiplications abar_{v,l} * rho^(v*l*base_pow); iii. outer DFTs of the rows
    with root rho^(2m*base_pow) by recursion, whose output f is element 2m*f + v.
    When n <= 2m the whole DFT is one alpha-power DFT (root alpha^(2m/n))."""
    n = len(a)
    two_m = 2 * par.m
    if n <= two_m:
        return alpha_dft(a, two_m // n, par)
    mu_n = n // two_m
    abar = [[None] * mu_n for _ in range(two_m)]
    for l in range(mu_n):
        e_l = [a[j * mu_n + l] for j in range(two_m)]
        E = alpha_dft(e_l, 1, par)
        for v in range(two_m):
            abar[v][l] = E[v]
    if dump is not None and base_pow == 1:
        dump["inner"] = [abar[v][l] for v in range(two_m) for l in range(mu_n)]
    for v in range(two_m):
        for l in range(1, mu_n):
            abar[v][l] = r_mul(abar[v][l], rho_power(v * l * base_pow, table, par), par.pz)
    out = [None] * n
    for v in range(two_m):
        sub = dkss_fft(abar[v], table, par, base_pow * two_m)
        for f in range(mu_n):
            out[two_m * f + v] = sub[f]
    return out


def dkss_inverse(c_hat, table, par):
    """Backwards transform (Sections 2.7 and 3.2.7): a forward transform again,
    read at index (-l) mod 2M, then division by 2M."""
    y = dkss_fft(c_hat, table, par)
    inv = pow(par.P2, -1, par.pz)
    return [[v * inv % par.pz for v in y[(-l) % par.P2]] for l in range(par.P2)]


# ---------------------------------------------------------------------------
# DKSS_MUL (Section 3.2 steps 1-8)
# ---------------------------------------------------------------------------

def dkss_mul(a, b, par, roots=None, stages=None):
    """c = a*b for 0 <= a, b < 2^N.  ``stages`` (a dict) receives natural-order
    dumps: 'a_inner' (abar after the level-1 inner DFTs, row-major v*mu + l),
    'a_hat', 'b_hat', 'c_hat' (pointwise products) and 'c' (after inverse and
    scaling)."""
    if roots is None:
        roots = compute_roots(par)
    table = rho_table(roots.rho, par)
    ea = encode(a, par)
    eb = encode(b, par)
    dump = {} if stages is not None else None
    a_hat = dkss_fft(ea, table, par, dump=dump)
    b_hat = dkss_fft(eb, table, par)
    c_hat = [r_mul(x, y, par.pz) for x, y in zip(a_hat, b_hat)]
    c_poly = dkss_inverse(c_hat, table, par)
    if stages is not None:
        stages.update(a_inner=dump.get("inner"), a_hat=a_hat, b_hat=b_hat,
                      c_hat=c_hat, c=c_poly)
    return decode(c_poly, par)


# ---------------------------------------------------------------------------
# Comparison multiplier (Section 2.3, OMUL): schoolbook on 64-bit words
# ---------------------------------------------------------------------------

def omul(a_words, b_words):
    """Ordinary schoolbook multiplication of little-endian 64-bit word lists."""
    base = 1 << 64
    c = [0] * (len(a_words) + len(b_words))
    for i, x in enumerate(a_words):
        carry = 0
        for j, y in enumerate(b_words):
            t = c[i + j] + x * y + carry
            c[i + j] = t % base
            carry = t // base
        c[i + len(b_words)] += carry
    return c


# ---------------------------------------------------------------------------
# System test of the implementation chapter: the Lucas-Lehmer test
# ---------------------------------------------------------------------------

def lucas_lehmer(p):
    """Last residue of the Lucas-Lehmer test of M_p = 2^p - 1, which the thesis
    runs with its DKSS square as a system test (implementation chapter, "system
    test"; the test as in Crandall-Pomerance Section 4.2.1): s_0 = 4,
    s_(k+1) = s_k^2 - 2 mod M_p for k < p - 2.  For an odd prime p, M_p is
    prime iff the result is 0.  Python integers throughout."""
    mp = (1 << p) - 1
    s = 4
    for _ in range(p - 2):
        s = (s * s - 2) % mp
    return s
