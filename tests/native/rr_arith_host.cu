// Host driver for the limb arithmetic of the R-multiplications
// (csrc/rr_arith.cuh, csrc/ntt_rmul.cuh): the same functions the kernels
// inline, called on the CPU so that tests/test_rr_arith_host.py can compare
// them with exact integer arithmetic without a GPU.
//
// One request per input line, decimal 32-bit words:
//   <op> <LR> <nprime> q[0..LR) x[0..LR) y[0..LR)
// op: mont (mont_mul_rr), mmul (lazy Montgomery product), rraw (reduce_raw
// of a lazy value), canon, norm
// (lz_norm of x), neg (neg_rr of x), rt<L> (to_rr then from_rr of the L
// words x[0..L), LR = limbs).  And the Lucas-Lehmer reduction of
// csrc/mersenne.cuh:
//   ll <p> c[0..2w)   (w = ceil(p/64), decimal 64-bit words)
// One output line per request: the result words.
#include <cinttypes>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_1503_04955_gb300/csrc/mersenne.cuh"
#include "../../paper_1503_04955_gb300/csrc/ntt_rmul.cuh"

namespace {

template <int LR>
void run(const char* op, uint32_t nprime, const uint32_t* q, const uint32_t* x, const uint32_t* y) {
    dkss::ModRR<LR> md;
    for (int i = 0; i < LR; ++i) md.q[i] = q[i];
    md.nprime = nprime;
    md.qtop_inv = dkss::qtop_reciprocal(q[LR - 1], q[LR - 2]);
    uint32_t a[LR], b[LR], r[LR];
    for (int i = 0; i < LR; ++i) {
        a[i] = x[i];
        b[i] = y[i];
        r[i] = 0;
    }
    if (!std::strcmp(op, "mont")) {
        dkss::mont_mul_rr<LR>(r, a, b, md);
    } else if (!std::strcmp(op, "mmul")) {
        dkss::mmul<LR>(r, a, b, md);
    } else if (!std::strcmp(op, "rraw")) {
        dkss::reduce_raw<LR>(r, a, md);
    } else if (!std::strcmp(op, "canon")) {
        dkss::canon<LR>(r, a, md);
    } else if (!std::strcmp(op, "norm")) {
        for (int i = 0; i < LR; ++i) r[i] = a[i];
        dkss::lz_norm<LR>(r);
    } else if (!std::strcmp(op, "neg")) {
        dkss::neg_rr<LR>(r, a, md);
    } else if (!std::strncmp(op, "rt", 2)) {
        const int L = op[2] - '0';
        uint32_t w[4] = {x[0], x[1], x[2], x[3]};
        uint32_t back[4] = {0, 0, 0, 0};
        if (L == 2) {
            uint32_t in[2] = {w[0], w[1]}, out[2];
            dkss::to_rr<2, LR>(r, in);
            dkss::from_rr<2, LR>(out, r);
            back[0] = out[0]; back[1] = out[1];
        } else if (L == 3) {
            uint32_t in[3] = {w[0], w[1], w[2]}, out[3];
            dkss::to_rr<3, LR>(r, in);
            dkss::from_rr<3, LR>(out, r);
            for (int i = 0; i < 3; ++i) back[i] = out[i];
        } else {
            uint32_t in[4] = {w[0], w[1], w[2], w[3]}, out[4];
            dkss::to_rr<4, LR>(r, in);
            dkss::from_rr<4, LR>(out, r);
            for (int i = 0; i < 4; ++i) back[i] = out[i];
        }
        for (int i = 0; i < LR; ++i) std::printf("%u ", r[i]);
        for (int i = 0; i < L; ++i) std::printf("%u%s", back[i], i + 1 < L ? " " : "");
        std::printf("\n");
        return;
    } else {
        std::printf("error\n");
        return;
    }
    for (int i = 0; i < LR; ++i) std::printf("%u%s", r[i], i + 1 < LR ? " " : "");
    std::printf("\n");
}

}  // namespace

int main() {
    char op[16];
    int LR;
    unsigned nprime;
    while (std::scanf("%15s", op) == 1) {
        if (!std::strcmp(op, "ll")) {
            unsigned p;
            if (std::scanf("%u", &p) != 1 || p < 3) return 4;
            const uint32_t w = (p + 63) / 64;
            std::vector<uint64_t> c(2 * w), s(w);
            for (uint32_t i = 0; i < 2 * w; ++i)
                if (std::scanf("%" SCNu64, &c[i]) != 1) return 4;
            dkss::ll_fold(c.data(), s.data(), p, w);
            for (uint32_t i = 0; i < w; ++i) std::printf("%" PRIu64 "%s", s[i], i + 1 < w ? " " : "\n");
            continue;
        }
        if (std::scanf("%d %u", &LR, &nprime) != 2) return 3;
        uint32_t q[5] = {0}, x[5] = {0}, y[5] = {0};
        if (LR < 2 || LR > 5) return 2;
        for (int i = 0; i < LR; ++i) if (std::scanf("%u", &q[i]) != 1) return 3;
        for (int i = 0; i < LR; ++i) if (std::scanf("%u", &x[i]) != 1) return 3;
        for (int i = 0; i < LR; ++i) if (std::scanf("%u", &y[i]) != 1) return 3;
        switch (LR) {
            case 2: run<2>(op, nprime, q, x, y); break;
            case 3: run<3>(op, nprime, q, x, y); break;
            case 4: run<4>(op, nprime, q, x, y); break;
            case 5: run<5>(op, nprime, q, x, y); break;
        }
    }
    return 0;
}
