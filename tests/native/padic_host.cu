// Host driver for the p-adic digit arithmetic (csrc/padic.cuh) and its limit
// check (csrc/ntt_bounds.cpp, pd_lazy_bounds), read by tests/test_padic_host.py.
// One request per input line, one answer line each:
//   mul p a0..a3 b0..b3          -> canonical digits of a b mod p^4
//   mulf p a0..a3 b0..b3         -> the same with fast carries (floor(2^32/p) = 2^e)
//   norm p x0..x3                -> pd_norm's digits
//   canon p x0..x3               -> pd_canon's digits
//   from p L w0..w(L-1) P0..P15  -> pd_from_words (P: digits of 2^(32j) mod p^4)
//   to p L d0..d3                -> pd_to_words's L words
//   from4 p w0..w3 P0..P15       -> pd_from_words4_large_p (p > 2^22)
//   bounds p m L                 -> ok kf kb0..kb6 fast dft_ok
#include <cstdio>
#include <cstring>
#include <iostream>
#include <sstream>
#include <string>

#include "../../paper_1503_04955_gb300/csrc/ntt_bounds.hpp"
#include "../../paper_1503_04955_gb300/csrc/padic.cuh"

using namespace dkss;

template <bool F = false>
static ModPD<4, F> make(uint64_t p) {
    ModPD<4, F> md;
    md.p = (uint32_t)p;
    md.nmu = (uint32_t)(((uint64_t)1 << 32) / p);
    uint32_t s = 0;
    while ((p >> (s + 1)) != 0) ++s;
    md.s = s;
    md.nsh = s + 1;   // p is odd: ceil(log2 p) = floor(log2 p) + 1
    md.mu = (uint64_t)((((unsigned __int128)1) << (64 + s)) / p);
    md.mu_lo = (uint32_t)((((unsigned __int128)1) << 64) / p);
    md.lg_nmu = 0;
    while ((1u << (md.lg_nmu + 1)) <= md.nmu) ++md.lg_nmu;
    return md;
}

template <int L>
static void from_words(std::istringstream& in, const ModPD<4>& md) {
    uint32_t w[L], pw[16], r[4];
    for (int j = 0; j < L; ++j) in >> w[j];
    for (int i = 0; i < 16; ++i) in >> pw[i];
    pd_from_words<L, 4>(r, w, pw, md);
    printf("%u %u %u %u\n", r[0], r[1], r[2], r[3]);
}

template <int L>
static void to_words(std::istringstream& in, const ModPD<4>& md) {
    uint32_t d[4], w[L];
    for (int k = 0; k < 4; ++k) in >> d[k];
    pd_to_words<L, 4>(w, d, md);
    for (int j = 0; j < L; ++j) printf(j ? " %u" : "%u", w[j]);
    printf("\n");
}

int main() {
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string op;
        uint64_t p;
        if (!(in >> op >> p)) continue;
        const ModPD<4> md = make(p);
        uint32_t a[4], b[4], r[4];
        if (op == "mul" || op == "mulf") {
            for (auto& v : a) in >> v;
            for (auto& v : b) in >> v;
            if (op == "mul") mmul<4>(r, a, b, md);
            else mmul<4>(r, a, b, make<true>(p));   // fast carries: floor(2^32/p) a power of two
            printf("%u %u %u %u\n", r[0], r[1], r[2], r[3]);
        } else if (op == "norm" || op == "canon") {
            for (auto& v : a) in >> v;
            if (op == "norm") {
                pd_norm<4>(a, md);
                printf("%u %u %u %u\n", a[0], a[1], a[2], a[3]);
            } else {
                pd_canon<4>(r, a, md);
                printf("%u %u %u %u\n", r[0], r[1], r[2], r[3]);
            }
        } else if (op == "from4") {   // the short conversion for p > 2^22
            uint32_t w[4], pw[16];
            for (auto& v : w) in >> v;
            for (auto& v : pw) in >> v;
            pd_from_words4_large_p(r, w, pw, md);
            printf("%u %u %u %u\n", r[0], r[1], r[2], r[3]);
        } else if (op == "from" || op == "to") {
            int L;
            in >> L;
            if (op == "from") {
                if (L == 2) from_words<2>(in, md);
                else if (L == 3) from_words<3>(in, md);
                else from_words<4>(in, md);
            } else {
                if (L == 2) to_words<2>(in, md);
                else if (L == 3) to_words<3>(in, md);
                else to_words<4>(in, md);
            }
        } else if (op == "bounds") {
            uint32_t m, L;
            in >> m >> L;
            dkss_planning::PdBiases bi;
            const bool ok = dkss_planning::pd_lazy_bounds(p, m, L, &bi);
            printf("%d %u", ok ? 1 : 0, bi.kf);
            for (int i = 0; i < 7; ++i) printf(" %u", bi.kb[i]);
            printf(" %d %d\n", bi.fast ? 1 : 0, bi.dft_ok ? 1 : 0);
        } else {
            printf("?\n");
        }
    }
    return 0;
}
