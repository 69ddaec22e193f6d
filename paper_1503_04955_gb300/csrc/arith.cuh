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

// Modular addition and subtraction with the limb carries in the condition-code
// chain (add.cc / addc / sub.cc / subc in one asm block, so nothing can come
// between the instructions of a chain): a + b, then a - q with its borrow
// choosing the result; a - b, then + (q & borrow mask).
template <int L>
__device__ __forceinline__ void add_mod_ptx(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                            const uint32_t (&q)[L]);
template <int L>
__device__ __forceinline__ void sub_mod_ptx(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                            const uint32_t (&q)[L]);

template <>
__device__ __forceinline__ void add_mod_ptx<2>(uint32_t (&r)[2], const uint32_t (&a)[2], const uint32_t (&b)[2],
                                          const uint32_t (&q)[2]) {
    asm("{\n\t.reg .u32 s0,s1,d0,d1,bw;\n\t.reg .pred p;\n\t"
        "add.cc.u32 s0, %2, %4;\n\t"
        "addc.u32 s1, %3, %5;\n\t"
        "sub.cc.u32 d0, s0, %6;\n\t"
        "subc.cc.u32 d1, s1, %7;\n\t"
        "subc.u32 bw, 0, 0;\n\t"
        "setp.ne.u32 p, bw, 0;\n\t"
        "selp.b32 %0, s0, d0, p;\n\t"
        "selp.b32 %1, s1, d1, p;\n\t"
        "}"
        : "=r"(r[0]), "=r"(r[1])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]), "r"(q[0]), "r"(q[1]));
}

template <>
__device__ __forceinline__ void add_mod_ptx<3>(uint32_t (&r)[3], const uint32_t (&a)[3], const uint32_t (&b)[3],
                                          const uint32_t (&q)[3]) {
    asm("{\n\t.reg .u32 s0,s1,s2,d0,d1,d2,bw;\n\t.reg .pred p;\n\t"
        "add.cc.u32 s0, %3, %6;\n\t"
        "addc.cc.u32 s1, %4, %7;\n\t"
        "addc.u32 s2, %5, %8;\n\t"
        "sub.cc.u32 d0, s0, %9;\n\t"
        "subc.cc.u32 d1, s1, %10;\n\t"
        "subc.cc.u32 d2, s2, %11;\n\t"
        "subc.u32 bw, 0, 0;\n\t"
        "setp.ne.u32 p, bw, 0;\n\t"
        "selp.b32 %0, s0, d0, p;\n\t"
        "selp.b32 %1, s1, d1, p;\n\t"
        "selp.b32 %2, s2, d2, p;\n\t"
        "}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(q[0]), "r"(q[1]), "r"(q[2]));
}

template <>
__device__ __forceinline__ void add_mod_ptx<4>(uint32_t (&r)[4], const uint32_t (&a)[4], const uint32_t (&b)[4],
                                          const uint32_t (&q)[4]) {
    asm("{\n\t.reg .u32 s0,s1,s2,s3,d0,d1,d2,d3,bw;\n\t.reg .pred p;\n\t"
        "add.cc.u32 s0, %4, %8;\n\t"
        "addc.cc.u32 s1, %5, %9;\n\t"
        "addc.cc.u32 s2, %6, %10;\n\t"
        "addc.u32 s3, %7, %11;\n\t"
        "sub.cc.u32 d0, s0, %12;\n\t"
        "subc.cc.u32 d1, s1, %13;\n\t"
        "subc.cc.u32 d2, s2, %14;\n\t"
        "subc.cc.u32 d3, s3, %15;\n\t"
        "subc.u32 bw, 0, 0;\n\t"
        "setp.ne.u32 p, bw, 0;\n\t"
        "selp.b32 %0, s0, d0, p;\n\t"
        "selp.b32 %1, s1, d1, p;\n\t"
        "selp.b32 %2, s2, d2, p;\n\t"
        "selp.b32 %3, s3, d3, p;\n\t"
        "}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(q[0]), "r"(q[1]), "r"(q[2]), "r"(q[3]));
}

template <>
__device__ __forceinline__ void sub_mod_ptx<2>(uint32_t (&r)[2], const uint32_t (&a)[2], const uint32_t (&b)[2],
                                          const uint32_t (&q)[2]) {
    asm("{\n\t.reg .u32 d0,d1,t0,t1,bw;\n\t.reg .pred p;\n\t"
        "sub.cc.u32 d0, %2, %4;\n\t"
        "subc.cc.u32 d1, %3, %5;\n\t"
        "subc.u32 bw, 0, 0;\n\t"
        "and.b32 t0, %6, bw;\n\t"
        "and.b32 t1, %7, bw;\n\t"
        "add.cc.u32 %0, d0, t0;\n\t"
        "addc.u32 %1, d1, t1;\n\t"
        "}"
        : "=r"(r[0]), "=r"(r[1])
        : "r"(a[0]), "r"(a[1]), "r"(b[0]), "r"(b[1]), "r"(q[0]), "r"(q[1]));
}

template <>
__device__ __forceinline__ void sub_mod_ptx<3>(uint32_t (&r)[3], const uint32_t (&a)[3], const uint32_t (&b)[3],
                                          const uint32_t (&q)[3]) {
    asm("{\n\t.reg .u32 d0,d1,d2,t0,t1,t2,bw;\n\t.reg .pred p;\n\t"
        "sub.cc.u32 d0, %3, %6;\n\t"
        "subc.cc.u32 d1, %4, %7;\n\t"
        "subc.cc.u32 d2, %5, %8;\n\t"
        "subc.u32 bw, 0, 0;\n\t"
        "and.b32 t0, %9, bw;\n\t"
        "and.b32 t1, %10, bw;\n\t"
        "and.b32 t2, %11, bw;\n\t"
        "add.cc.u32 %0, d0, t0;\n\t"
        "addc.cc.u32 %1, d1, t1;\n\t"
        "addc.u32 %2, d2, t2;\n\t"
        "}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(q[0]), "r"(q[1]), "r"(q[2]));
}

template <>
__device__ __forceinline__ void sub_mod_ptx<4>(uint32_t (&r)[4], const uint32_t (&a)[4], const uint32_t (&b)[4],
                                          const uint32_t (&q)[4]) {
    asm("{\n\t.reg .u32 d0,d1,d2,d3,t0,t1,t2,t3,bw;\n\t.reg .pred p;\n\t"
        "sub.cc.u32 d0, %4, %8;\n\t"
        "subc.cc.u32 d1, %5, %9;\n\t"
        "subc.cc.u32 d2, %6, %10;\n\t"
        "subc.cc.u32 d3, %7, %11;\n\t"
        "subc.u32 bw, 0, 0;\n\t"
        "and.b32 t0, %12, bw;\n\t"
        "and.b32 t1, %13, bw;\n\t"
        "and.b32 t2, %14, bw;\n\t"
        "and.b32 t3, %15, bw;\n\t"
        "add.cc.u32 %0, d0, t0;\n\t"
        "addc.cc.u32 %1, d1, t1;\n\t"
        "addc.cc.u32 %2, d2, t2;\n\t"
        "addc.u32 %3, d3, t3;\n\t"
        "}"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(q[0]), "r"(q[1]), "r"(q[2]), "r"(q[3]));
}

// r = (a + b) mod q for a, b in [0, q)  (q < 2^(32L-1), so a + b fits)
template <int L>
__device__ __forceinline__ void add_mod(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                        const Mod<L>& md) {
    add_mod_ptx<L>(r, a, b, md.q);
}

// r = (a - b) mod q for a, b in [0, q)
template <int L>
__device__ __forceinline__ void sub_mod(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                        const Mod<L>& md) {
    sub_mod_ptx<L>(r, a, b, md.q);
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
