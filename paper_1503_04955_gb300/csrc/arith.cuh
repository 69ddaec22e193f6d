// Multi-limb modular arithmetic mod p^z on the integer pipe.
//
// A residue of P = Z/p^zZ (thesis Section 3.2, "inner coefficient") is L
// little-endian 32-bit limbs in [0, p^z).  Products are summed exactly in 2L
// limbs and reduced once with Montgomery's REDC (R = 2^(32L)).  The host plan
// guarantees m*(p^z)^2 + R*p^z < 2^(64L), so a sum of m products and its REDC
// never leave 2L limbs, and p^z < 2^(32L-1), so a sum of two residues fits.
#pragma once
#include <cstdint>

namespace dkss {

template <int L>
struct Mod {
    uint32_t q[L];     // p^z
    uint32_t nprime;   // -q^{-1} mod 2^32
    uint32_t nsub;     // conditional subtractions after REDC of an m-term sum
};

template <int L>
__device__ __forceinline__ bool geq(const uint32_t (&a)[L], const uint32_t (&b)[L]) {
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
        if (a[i] != b[i]) return a[i] > b[i];
    }
    return true;
}

// r = a - b, returns the borrow out.
template <int L>
__device__ __forceinline__ uint32_t sub_n(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L]) {
    uint32_t borrow = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        uint64_t d = (uint64_t)a[i] - b[i] - borrow;
        r[i] = (uint32_t)d;
        borrow = (uint32_t)(d >> 63);
    }
    return borrow;
}

template <int L>
__device__ __forceinline__ void add_n(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L]) {
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        uint64_t s = (uint64_t)a[i] + b[i] + carry;
        r[i] = (uint32_t)s;
        carry = (uint32_t)(s >> 32);
    }
}

// x <- x - q if x >= q
template <int L>
__device__ __forceinline__ void cond_sub(uint32_t (&x)[L], const Mod<L>& md) {
    uint32_t d[L];
    uint32_t borrow = sub_n<L>(d, x, md.q);
#pragma unroll
    for (int i = 0; i < L; ++i) x[i] = borrow ? x[i] : d[i];
}

// r = (a + b) mod q for a, b in [0, q)
template <int L>
__device__ __forceinline__ void add_mod(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                        const Mod<L>& md) {
    add_n<L>(r, a, b);
    cond_sub<L>(r, md);
}

// r = (a - b) mod q for a, b in [0, q)
template <int L>
__device__ __forceinline__ void sub_mod(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                        const Mod<L>& md) {
    uint32_t borrow = sub_n<L>(r, a, b);
    uint32_t t[L];
    add_n<L>(t, r, md.q);
#pragma unroll
    for (int i = 0; i < L; ++i) r[i] = borrow ? t[i] : r[i];
}

// r = (q - a) mod q
template <int L>
__device__ __forceinline__ void neg_mod(uint32_t (&r)[L], const uint32_t (&a)[L], const Mod<L>& md) {
    uint32_t nz = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) nz |= a[i];
    uint32_t t[L];
    sub_n<L>(t, md.q, a);
#pragma unroll
    for (int i = 0; i < L; ++i) r[i] = nz ? t[i] : 0u;
}

// acc (2L limbs) += x * y.  The caller guarantees no carry leaves acc.
template <int L>
__device__ __forceinline__ void mac(uint32_t (&acc)[2 * L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
    uint32_t prod[2 * L];
    {
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            uint64_t t = (uint64_t)x[0] * y[k] + carry;
            prod[k] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        prod[L] = carry;
    }
#pragma unroll
    for (int j = 1; j < L; ++j) {
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            uint64_t t = (uint64_t)x[j] * y[k] + prod[j + k] + carry;
            prod[j + k] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        prod[j + L] = carry;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < 2 * L; ++i) {
        uint64_t s = (uint64_t)acc[i] + prod[i] + carry;
        acc[i] = (uint32_t)s;
        carry = (uint32_t)(s >> 32);
    }
}

// Montgomery reduction: r = T * 2^(-32L) mod q, brought into [0, q) with
// nsub conditional subtractions (nsub from the host's bound on T).
template <int L>
__device__ __forceinline__ void redc(uint32_t (&r)[L], uint32_t (&T)[2 * L], const Mod<L>& md, uint32_t nsub) {
#pragma unroll
    for (int i = 0; i < L; ++i) {
        uint32_t qi = T[i] * md.nprime;
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            uint64_t t = (uint64_t)qi * md.q[k] + T[i + k] + carry;
            T[i + k] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
#pragma unroll
        for (int k = i + L; k < 2 * L; ++k) {
            uint64_t s = (uint64_t)T[k] + carry;
            T[k] = (uint32_t)s;
            carry = (uint32_t)(s >> 32);
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i) r[i] = T[L + i];
    for (uint32_t k = 0; k < nsub; ++k) cond_sub<L>(r, md);
}

// r = a * b * 2^(-32L) mod q for a, b in [0, q)
template <int L>
__device__ __forceinline__ void mont_mul(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                         const Mod<L>& md) {
    uint32_t T[2 * L];
#pragma unroll
    for (int i = 0; i < 2 * L; ++i) T[i] = 0;
    mac<L>(T, a, b);
    redc<L>(r, T, md, 1);
}

// ---- residue loads / stores (residue-major layout: L consecutive words) ----

template <int L>
__device__ __forceinline__ void ld_res(uint32_t (&x)[L], const uint32_t* p) {
    if constexpr (L == 4) {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else if constexpr (L == 2) {
        uint2 v = *reinterpret_cast<const uint2*>(p);
        x[0] = v.x; x[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < L; ++i) x[i] = p[i];
    }
}

template <int L>
__device__ __forceinline__ void st_res(uint32_t* p, const uint32_t (&x)[L]) {
    if constexpr (L == 4) {
        *reinterpret_cast<uint4*>(p) = make_uint4(x[0], x[1], x[2], x[3]);
    } else if constexpr (L == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(x[0], x[1]);
    } else {
#pragma unroll
        for (int i = 0; i < L; ++i) p[i] = x[i];
    }
}

}  // namespace dkss
