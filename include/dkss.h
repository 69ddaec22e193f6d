/*
 * dkss.h -- C ABI of the GB300 DKSS multiplication library (libdkss.so).
 *
 * The library multiplies nonnegative integers a, b < 2^N exactly with the
 * De-Kurur-Saha-Saptharishi algorithm as implemented and analysed in
 * C. Lueders, "Fast Multiplication of Large Integers: Implementation and
 * Analysis of the DKSS Algorithm" (arXiv:1503.04955), Chapter 3:
 * encode into R[x] with R = (Z/p^zZ)[alpha]/(alpha^m+1), a 2M-point FFT whose
 * inner 2m-point butterflies use powers of alpha as negacyclic shifts and whose
 * outer "bad" twiddles rho^i are full R-multiplications, componentwise
 * products, the backwards FFT with scaling by (2M)^-1, and decoding with a
 * device-wide carry scan (Section 3.2, steps 4-8).
 *
 * Numbers are little-endian arrays of 64-bit words (Section 2.1): word k holds
 * bits [64k, 64k+64).  An N-bit operand has ceil(N/64) words and every bit at
 * or above N must be zero; a product has 2*ceil(N/64) words.
 *
 * All entry points return a dkss_status.  Argument and parameter errors are
 * reported synchronously and leave no work queued.  Work on the GPU is queued
 * on the caller's stream and returns at once; errors found by a kernel are
 * recorded in a per-plan device status word, read by dkss_sync_status().
 * A plan is not safe for concurrent calls from several host threads, and two
 * calls on one plan must not run concurrently on different streams (they
 * share the plan's workspace).
 */
#ifndef DKSS_H
#define DKSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dkss_plan_s* dkss_plan_t;
typedef struct CUstream_st* dkss_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    DKSS_OK = 0,
    DKSS_EINVAL = 1,       /* null pointer, aliasing output, size mismatch */
    DKSS_EPARAM = 2,       /* parameters violate Section 3.2 steps 1-2 (see dkss_plan) */
    DKSS_ENOMEM = 3,       /* device or host allocation failed */
    DKSS_EUNSUPPORTED = 4, /* valid parameters this build has no kernel for */
    DKSS_ECUDA = 5,        /* a CUDA runtime call failed */
    DKSS_ETIMEOUT = 6,     /* a bounded device-side wait gave up */
    DKSS_EDEVICE = 7       /* a kernel found an internal inconsistency */
} dkss_status;

enum {
    DKSS_FORM_IMAD = 1,    /* R-multiplications on the integer pipe (default) */
    DKSS_FORM_INT8TC = 2,  /* R-multiplications as exact INT8 tensor-core products
                              (mma.sync u8, byte slices of the residues); m >= 32 */
    DKSS_PROFILE = 4,      /* per-stage CUDA-event timing, read with dkss_profile_read */
    DKSS_DEBUG_CHECKS = 8, /* device-side range checks at the stage boundaries: every residue of
                              both transformed operands, of the componentwise products and of
                              the product polynomial must lie in [0, p^z) (Section 3.2); one
                              extra HBM pass per check; a failure makes dkss_sync_status return
                              DKSS_EDEVICE (the product itself is then not to be trusted) */
    DKSS_RMUL_DIRECT = 16, /* R-multiplications by the direct negacyclic convolution
                              (Section 2.9.2) instead of through the evaluation map of R */
    DKSS_ARITH_MONT = 512, /* NTT form with m = 64 over p^4, p < 2^30: keep the 26-bit-limb Montgomery
                              products instead of p-adic digits (each residue as four base-p
                              digits, a product as ten digit products and a carry chain;
                              Section 3.2.2's ring Z/p^zZ, no change of the transform).  Without
                              the flag the library takes the digits where they need fewer
                              multiply-adds: floor(2^32/p) a power of two, or five 26-bit limbs */
    DKSS_LEVELS_EVAL = 128 /* every radix-2m level but the first, and the last level, in the
                              evaluation coordinates of R (the CRT map of Section 3.2.3):
                              their inner DFTs become m independent DFTs over Z/p^zZ with
                              products instead of alpha-shifts, their bad twiddles pointwise
                              products.  The same transform with fewer Montgomery products;
                              NTT form and m <= 32 only, ignored otherwise.  By default every
                              inner DFT is the thesis's alpha-shift DFT */
};

/* dkss_plan with M = m = u = p = z = 0: parameters by the thesis's rule alone
   (Section 4.1), without timing candidates on the device */
#define DKSS_TUNE_RULE 32

/*
 * Build a plan for N-bit operands (thesis Section 3.2 steps 1-3, Section 4.1).
 *   n_bits  N, 64 <= N; operands are < 2^N.
 *   M = m = u = p = z = 0: the library chooses the parameters.  It lists the
 *           valid sets as dkss_plan_candidates does and ranks them by the
 *           thesis's rule (Section 4.1: p^z just above the coefficient bound,
 *           then the largest u, then the smallest M m, then M/m closest to
 *           N / log2(N)^3).  For N <= 2^26 (and without DKSS_TUNE_RULE) it
 *           then times one product with the rule's choice and with the four
 *           other sets of least estimated work on the current device and keeps
 *           the fastest; choices are cached per (device, N, flags) for the
 *           life of the process.  The thesis notes that its fixed rule leaves a
 *           staircase of run times that calibration should smooth out
 *           (Section 4.4).  dkss_plan_info reports the chosen set.
 *   M, m    powers of two, 16 <= m <= 64, M >= m, with 2M > 2m (at least one
 *           radix-2m level); the transform length is 2M.
 *   u       input bits per inner coefficient, 1 <= u <= 32, M*(m/2)*u >= N.
 *   p, z    p prime with 2M | p-1 (Section 3.2.2); the residue ring is
 *           Z/p^zZ; p^z must exceed the largest product coefficient
 *           M*(m/2)*(2^u-1)^2 (Section 3.2.2); m*p^z < 2^127 (so that
 *           products in 26-bit limbs stay within 5 limbs).
 *   flags   0 (inner DFTs by alpha-shifts, R-multiplications through the
 *           evaluation map of R on the integer pipe), DKSS_LEVELS_EVAL (inner
 *           levels in evaluation coordinates, m <= 32), DKSS_RMUL_DIRECT
 *           (direct convolution, integer pipe) or DKSS_FORM_INT8TC (INT8 tensor
 *           cores; DKSS_EUNSUPPORTED if m < 32), optionally | DKSS_PROFILE.
 * On the host it tests p (deterministic Miller-Rabin), finds the smallest
 * generator zeta of F_p^*, Hensel-lifts it to a (p-1)-th root of unity mod p^z,
 * forms omega = zeta_z^((p-1)/2M), gamma = omega^(2M/2m) and rho by Lagrange
 * interpolation (Section 3.2.3, eq. dkss:lagrange), checks rho^(2M/2m) = alpha
 * and rho^M = -1, and tabulates rho^s, s < 2M/2m (Section 4.2).  It then
 * allocates the device workspace (two transformed polynomials, the rho^s table,
 * carry-scan scratch) on the current device, which the plan owns.
 * Errors: DKSS_EINVAL (plan == NULL), DKSS_EPARAM, DKSS_EUNSUPPORTED,
 * DKSS_ENOMEM, DKSS_ECUDA.  On error *plan is set to NULL.
 */
dkss_status dkss_plan(dkss_plan_t* plan, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u,
                      uint64_t p, uint32_t z, uint32_t flags);

/*
 * A plan over Z/pZ (z = 1) with the Proth prime p = h 2^n + 1, the form of
 * the thesis's own primes (Section 4.1: z = 1 without Hensel lifting, and a
 * precomputed table of primes h 2^n + 1 with the smallest odd h for each bit
 * length).  Arguments as dkss_plan with p = h 2^n + 1 in place of (p, z):
 * h odd, 0 < h < 2^32, 2M | 2^n, p < 2^126, p prime (Proth's theorem with a
 * quadratic non-residue as witness) and above the coefficient bound
 * M (m/2) (2^u - 1)^2 (Section 3.2.2).
 * When n >= 26 (LR - 1) (LR: the 26-bit limbs of the plan's products) and p has
 * no other limbs, p = 1 mod 2^26: the Montgomery reductions of the default
 * form then need no digit product and one limb product per digit instead of
 * LR + 1 (the thesis's outlook proposes exploiting the Proth form in the
 * modular reductions, Section 5.1); dkss_plan_info reports whether it applies.
 * The products are the same as with any other valid ring.  Errors: as
 * dkss_plan.
 */
dkss_status dkss_plan_proth(dkss_plan_t* plan, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t h,
                            uint32_t n, uint32_t flags);

/* Host-only roots of a Proth plan: as dkss_plan_rho for dkss_plan_proth's ring. */
dkss_status dkss_plan_proth_rho(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t h, uint32_t n,
                                uint64_t* rho_out, uint64_t* consts, size_t n_consts);

/*
 * A Proth ring with the cheap reduction for the given N, M, m, u (host only):
 * the fewest product limbs LR in 3..5 and, for it, n = max(26 (LR - 1),
 * log2 2M) and the smallest odd h such that p = h 2^n + 1 is prime, above the
 * coefficient bound and m p < 2^(26 LR - 2) -- p just above the bound, as the
 * thesis's rule picks it (Section 4.1), within the limb layout.  *h, *n
 * receive the choice.  Errors: DKSS_EINVAL, DKSS_EPARAM (shape),
 * DKSS_EUNSUPPORTED (none found).
 */
dkss_status dkss_proth_ring(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t* h, uint32_t* n);

/*
 * out = a * b (thesis Section 3.2 steps 4-8).  a, b: device pointers to
 * ceil(N/64) words each; out: device pointer to 2*ceil(N/64) words, which must
 * not overlap a or b.  Queued on `stream`; the caller keeps a, b, out alive
 * until the stream reaches this work.  When a == b (the same pointer) the
 * product is a square and takes dkss_sqr's path.  Errors: DKSS_EINVAL,
 * DKSS_ECUDA.
 */
dkss_status dkss_mul(dkss_plan_t plan, const uint64_t* a, const uint64_t* b, uint64_t* out,
                     dkss_stream_t stream);

/*
 * out = a^2.  The forward transform (Section 3.2 step 5) runs once, on a
 * alone, and the componentwise products (step 6) square each element
 * (through the evaluation map of R, one forward transform per element instead
 * of two); the rest is the product's path.  This is the operation of the
 * thesis's system test, the Lucas-Lehmer test of Mersenne numbers
 * (implementation chapter, "system test"; see dkss_ll_step).  a: device
 * pointer to ceil(N/64) words; out: 2*ceil(N/64) words, not overlapping a.
 * Errors: as dkss_mul.
 */
dkss_status dkss_sqr(dkss_plan_t plan, const uint64_t* a, uint64_t* out, dkss_stream_t stream);

/*
 * One step of the Lucas-Lehmer test of M_p = 2^p - 1 after the square:
 * s = (c - 2) mod M_p for c = s_prev^2 < 2^(2p) (the thesis's system test, as
 * above; the test itself: s_0 = 4, s_(k+1) = s_k^2 - 2 mod M_p, and M_p is
 * prime iff s_(p-2) = 0 for odd prime p).  The thesis has no kernel for it;
 * the modular reduction folds c's high part onto its low part, since
 * 2^p = 1 mod M_p, and the result is the canonical residue in [0, M_p).
 *   c  device pointer, 2*w words (w = ceil(p/64)), little-endian, c < 2^(2p).
 *   s  device pointer, w words; receives the residue, bits >= p zero.  May
 *      not overlap c.
 *   p  2 < p < 2^26.
 * One thread of one CTA works through the words in order (a short serial
 * step beside the square; not part of the product's path).  Queued on
 * `stream`.  Errors: DKSS_EINVAL (null pointer, p out of range, overlap),
 * DKSS_ECUDA.
 */
dkss_status dkss_ll_step(const uint64_t* c, uint64_t* s, uint32_t p, dkss_stream_t stream);

/*
 * Same product from host memory: copies a and b (ceil(N/64) words each) to the
 * device, multiplies, copies the 2*ceil(N/64)-word product back to out_host
 * and waits for the stream.  Host buffers may be pageable or pinned.
 * Errors: as dkss_mul, plus DKSS_ENOMEM for the plan's staging buffers.
 */
dkss_status dkss_mul_host(dkss_plan_t plan, const uint64_t* a_host, const uint64_t* b_host,
                          uint64_t* out_host, dkss_stream_t stream);

/*
 * The forward transform alone (Section 3.2 step 5): writes
 * out[i] = a(rho^i), i < 2M, to out (device, 2M*m residues of 2 words each,
 * element-major, residue t of element i at words 2*(i*m+t), 2*(i*m+t)+1,
 * canonical in [0, p^z), natural order).  Used to compare stage results.
 * Errors: DKSS_EINVAL, DKSS_ECUDA.
 */
dkss_status dkss_forward(dkss_plan_t plan, const uint64_t* a, uint64_t* out, dkss_stream_t stream);

/* One job of a batch: operands of n_bits bits, device pointers as dkss_mul. */
typedef struct {
    const uint64_t* a;
    const uint64_t* b;
    uint64_t* out;
    uint64_t n_bits;
} dkss_job;

typedef struct dkss_batch_s* dkss_batch_t;

enum {
    DKSS_BATCH_RULE = 32,      /* size-class parameters by rule instead of measurement */
    DKSS_BATCH_NO_GRAPH = 64,  /* launch the persistent kernel directly, not from a graph */
    DKSS_BATCH_PROTH = 128,    /* every class over its own Proth prime (dkss_plan_proth) */
    DKSS_BATCH_NO_PROTH = 256  /* every class over the configured primes */
};

/*
 * Plan a batch of `count` independent products whose operands have the given
 * bit lengths (each job is Section 3.2 on its own).  Jobs are grouped into
 * size classes (operands up to the next power of two, at least 2^12 bits).
 * All classes share the limb layout of one kernel (m = 32, residues of three
 * 32-bit words, products in four 26-bit limbs); each class has its own M, u
 * and ring Z/p^zZ in that layout: either the smallest p^z above its
 * coefficient bound from the primes dkss_plan_candidates draws from, or its
 * own Proth prime p = h 2^n + 1 (z = 1, dkss_proth_ring), whose reductions
 * are cheaper (Section 4.1 and the outlook of Section 5.1).  Per class the
 * autotuner times one product with u = 32 and with u = 16 on the current
 * device (cached per device, class and ring family) and keeps the faster;
 * the ring family of the batch is the one with the smaller sum over classes
 * of jobs x time (DKSS_BATCH_PROTH, DKSS_BATCH_NO_PROTH force one;
 * DKSS_BATCH_RULE takes the configured primes and the largest valid u, the
 * thesis's own rule of Section 4.1, without timing).  The plan owns every
 * job's workspace and the class tables, and records one cooperative
 * persistent-kernel launch in a CUDA graph.  Operands up to 2^21 bits;
 * count <= 2^20.
 * Errors: DKSS_EINVAL, DKSS_EUNSUPPORTED (operand too long), DKSS_ENOMEM,
 * DKSS_ECUDA.  On error *batch is NULL.
 */
dkss_status dkss_batch_plan(dkss_batch_t* batch, const uint64_t* n_bits, size_t count, uint32_t flags);

/*
 * Run a planned batch: jobs is a host array of count entries whose n_bits
 * match the plan, in order; a, b, out are device pointers as for dkss_mul.
 * Copies the job pointers to the device (host-to-device copy on `stream`)
 * and launches the graph: one persistent kernel for all jobs.  Asynchronous;
 * calls on one batch plan must not overlap.  Errors: DKSS_EINVAL, DKSS_ECUDA.
 */
dkss_status dkss_batch_run(dkss_batch_t batch, const dkss_job* jobs, dkss_stream_t stream);

/*
 * Parameters chosen for job `job`: params[0..12] = M, m, u, p (low word), z,
 * the class's largest operand bits, transform levels, persistent grid size,
 * 1 if the launch is a graph, p's high word, 1 for a Proth ring, and its h
 * and n (p = h 2^n + 1; 0 otherwise).  n is the length of params.
 */
dkss_status dkss_batch_job_params(dkss_batch_t batch, size_t job, uint64_t* params, size_t n);

/* Free a batch plan (waits for the device).  NULL is a no-op. */
dkss_status dkss_batch_destroy(dkss_batch_t batch);

/*
 * Multiply `count` independent pairs of any sizes in one call: plans a batch
 * for these lengths (kept and reused while the lengths and flags stay the
 * same) and runs it.  jobs: host array.  Errors: as dkss_batch_plan and
 * dkss_batch_run.
 */
dkss_status dkss_mul_batch(const dkss_job* jobs, size_t count, uint32_t flags, dkss_stream_t stream);

/*
 * Host view of a plan's parameters (no device work).  rho_out (may be NULL)
 * receives rho's m coefficients as 2 words each; consts receives, in order:
 * 2M, 2M/2m, L (32-bit limbs per stored residue), transform levels, p^z low
 * word, p^z high word, generator zeta, omega low, omega high, gamma low,
 * gamma high, LR (26-bit limbs of the product arithmetic), the form of the
 * R-multiplications (0 through the evaluation map, 1 direct convolution,
 * 2 INT8 tensor cores, 3 inner levels in evaluation coordinates
 * (DKSS_LEVELS_EVAL);
 * a ring outside the evaluation-map form's limits on its unreduced sums gets
 * 1 unless the flags ask for 2), 1 when form 0 (every level on
 * coefficients) scales one factor of each componentwise product first (else
 * 0), 1 when the ring allows the inner levels in evaluation coordinates
 * (else 0), the mask of the stages of their DFTs whose butterflies with
 * twiddle 1 skip the product (bit s: stage s), then M, m, u, p (low word),
 * z (the parameters in effect, also when the library chose them), p's high
 * word (Proth primes above 2^64), 1 when the Montgomery reductions use the
 * sparse Proth modulus (dkss_plan_proth) else 0, and the bytes of device memory
 * the plan holds: its two transformed polynomials (the transform runs in
 * place, level by level, with no third polynomial for the thesis's
 * intermediate abar of Section 4.5), the twiddle tables and the carry-scan
 * scratch (0 for a host-only view), and 1 when the m = 64 transforms in R
 * compute in p-adic digits (see DKSS_ARITH_MONT) else 0.
 */
dkss_status dkss_plan_info(dkss_plan_t plan, uint64_t* consts, size_t n_consts, uint64_t* rho_out);

/*
 * Host-only computation of rho for the given parameters (same checks as
 * dkss_plan, no device allocation); rho_out receives m coefficients of 2 words.
 * Lets a CPU-only caller inspect the plan's root.  Errors: as dkss_plan.
 */
dkss_status dkss_plan_rho(uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint64_t p, uint32_t z,
                          uint64_t* rho_out, uint64_t* consts, size_t n_consts);

/*
 * Per-stage device times of the plan's calls since the last read (needs
 * DKSS_PROFILE at dkss_plan; CUDA events recorded on the caller's stream around
 * each kernel group).  Waits for those events.  Index k of ms (milliseconds
 * summed) and counts (groups timed): 0 forward inner DFTs (the first level
 * encodes), 1 forward bad multiplications, 2 last forward level +
 * componentwise products + first backwards level, 3 backwards bad
 * multiplications, 4 backwards inner DFTs, 5 decoding and carry scan.
 * Either array may be NULL; n is their length (at most 8 used).  Resets the
 * sums.  Errors: DKSS_EINVAL, DKSS_ECUDA.
 */
dkss_status dkss_profile_read(dkss_plan_t plan, double* ms, uint64_t* counts, size_t n);

/*
 * Largest product dkss_decode_static handles: its scratch holds one word per
 * tile of 2048 32-bit output windows, and a product has 4*ceil(N/64) windows,
 * so ceil(N/64) <= 2^27 (N <= 2^33).
 */
#define DKSS_DECODE_STATIC_MAX_TILES 262144

/*
 * Decoding and carry propagation (the last step of a product) that allocates
 * nothing.  The thesis has no counterpart.  It exists for callers that cannot
 * allocate device memory at the time of the call: a latency-bound loop whose
 * device memory is fixed before it starts (cudaMalloc and cudaFree may
 * synchronize the device and stall its other streams), or code running inside
 * a framework that owns the device's memory pool and gives its plugins no
 * allocator.  They still need the carry scan's scratch; here it is a
 * file-scope device array of DKSS_DECODE_STATIC_MAX_TILES + 1 words (1 MiB)
 * that every GPU which loads the library holds until the process exits.
 *
 *   c       device pointer: the product polynomial, 2M elements x m residues
 *           x L 32-bit limbs (word (e*m + t)*L + l), natural order, each
 *           residue the exact nonnegative coefficient (below 2^(32L)); the
 *           layout dkss_mul uses internally after the backwards transform.
 *   n_bits  N of the operands; out receives 2*ceil(N/64) words (device).
 *   M, m, u the encoding parameters (powers of two M, m with m <= 64,
 *           u <= 32, M*(m/2)*u >= N); L in [2, 4].
 * Result: out = sum over elements e and residues t of c[e][t] * 2^(u(e*m/2+t)),
 * the value decoded in Section 3.2.8 of a product of two N-bit operands.
 * Queued on `stream`.  Errors: DKSS_EINVAL (bad argument), DKSS_EUNSUPPORTED
 * (N beyond the static scratch, checked before any device work), DKSS_ECUDA.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * process, so make that first call before any stream capture; after
 * cudaDeviceReset the kept address is stale and later calls on that device
 * are not valid.  All calls share the scratch, which keeps the last call's
 * contents (only its status word is cleared by each call): calls whose work
 * overlaps on the GPU (different streams, or different host threads) race and
 * must be serialised by the caller.  A carry out of 2N bits (impossible for a
 * true product) is recorded in the scratch's status word and not reported.
 */
dkss_status dkss_decode_static(const uint32_t* c, uint64_t n_bits, uint64_t M, uint32_t m, uint32_t u, uint32_t L,
                               uint64_t* out, dkss_stream_t stream);

/*
 * Valid parameter sets for N-bit operands (host only, no device work): for
 * m in {16, 32, 64}, u in {8, 16, 24, 32}, the smallest M with M (m/2) u >= N
 * and 2M > 2m, each p of a fixed list of primes with 2M | p-1 (12289, 40961,
 * 65537, 786433, 7340033, 23068673, 104857601, 167772161, 469762049,
 * 998244353) and the smallest z with p^z above the coefficient bound
 * (Section 3.2.2), every set dkss_plan accepts and this build has kernels for.
 * rows receives up to max_rows rows of 10 words: M, m, u, p, z, L, LR,
 * transform levels, last-level length, 2M; *n_rows the number of valid sets
 * (may exceed max_rows; rows may be NULL to count).  The search space of the
 * autotuner.  Errors: DKSS_EINVAL.
 */
dkss_status dkss_plan_candidates(uint64_t n_bits, uint64_t* rows, size_t max_rows, size_t* n_rows);

/*
 * The parameters dkss_plan(plan, n_bits, 0, 0, 0, 0, 0, flags) uses:
 * params[0..4] = M, m, u, p, z.  With DKSS_TUNE_RULE, or for N > 2^26, this is
 * the thesis's rule alone and runs on the host only (no device needed);
 * otherwise candidates are timed on the current device as dkss_plan
 * describes (and the choice is cached).  flags: the form flags of the plan.
 * Errors: DKSS_EINVAL (params NULL, N = 0), DKSS_EUNSUPPORTED (no valid set
 * for this form), DKSS_ECUDA.
 */
dkss_status dkss_plan_choose(uint64_t n_bits, uint32_t flags, uint64_t* params);

/*
 * Cost model of the autotuner (the thesis has no counterpart; its Section 4.1
 * picks parameters by a fixed rule and notes that calibration should smooth
 * out the resulting staircase of run times).  A multilayer perceptron maps
 * DKSS_MLP_FEATURES features of a parameter set to a predicted log2 of the
 * product's device time: relu(W1 x + b1) -> relu(W2 h1 + b2) -> w3 . h2 + b3,
 * hidden width DKSS_MLP_HIDDEN.  params: DKSS_MLP_PARAMS floats, in order
 * W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.  All pointers are device
 * pointers; work is queued on `stream`.  This is the only floating point in
 * the library and it never enters a product.
 */
#define DKSS_MLP_FEATURES 12
#define DKSS_MLP_HIDDEN 32
#define DKSS_MLP_PARAMS 1505

/* y[n] = network(x[n]) for n < B; x is B rows of DKSS_MLP_FEATURES floats. */
dkss_status dkss_mlp_forward(const float* params, const float* x, size_t B, float* y, dkss_stream_t stream);

/*
 * grad (DKSS_MLP_PARAMS floats) = gradient of the mean squared error
 * mean_n (network(x[n]) - t[n])^2 with respect to params; *loss = that mean.
 * grad and loss are overwritten.  Summation order across samples is not fixed
 * (float atomics), so repeated calls agree to rounding only.
 */
dkss_status dkss_mlp_grad(const float* params, const float* x, const float* t, size_t B, float* grad, float* loss,
                          dkss_stream_t stream);

/*
 * One Adam step (beta1 = 0.9, beta2 = 0.999, eps = 1e-8; Kingma and Ba,
 * 2015) with learning rate lr; m1, m2 are the moment arrays (zero before step
 * 1) and step counts from 1.
 */
dkss_status dkss_mlp_adam(float* params, const float* grad, float* m1, float* m2, float lr, uint32_t step,
                          dkss_stream_t stream);

/*
 * Host-side fault injection for tests (the thesis has no counterpart).  mask
 * is process-wide and 0 by default; set it only while no other thread plans.
 *   DKSS_FAULT_RHO        plan math perturbs one coefficient of rho before it
 *                         checks rho^(2M/2m) = alpha and rho^M = -1 (Section
 *                         3.2.3), which must then reject it: dkss_plan and
 *                         dkss_plan_rho return DKSS_EPARAM.
 *   DKSS_FAULT_HOST_ALLOC dkss_plan's host allocation fails: it returns
 *                         DKSS_ENOMEM and sets *plan to NULL.
 *   DKSS_FAULT_RANGE      dkss_mul (product path, not the levels in evaluation
 *                         coordinates) overwrites residue 0 of the transformed
 *                         first operand with 2^(32L) - 1, which is not below
 *                         p^z, by a host-to-device copy queued after the
 *                         forward transform; with DKSS_DEBUG_CHECKS the range
 *                         check that follows must record it, and
 *                         dkss_sync_status returns DKSS_EDEVICE.
 * The injection is made on the host (plan math, host allocation, or a copy
 * of a host value into device memory); no kernel faults, traps or waits.
 * Returns the previous mask.
 */
enum { DKSS_FAULT_RHO = 1, DKSS_FAULT_HOST_ALLOC = 2, DKSS_FAULT_RANGE = 4 };
uint32_t dkss_fault_inject(uint32_t mask);

/* Kernel launches one dkss_mul call queues (for launch accounting). */
uint32_t dkss_plan_launches(dkss_plan_t plan);

/*
 * Wait for `stream`, then return and clear the plan's device status word:
 * DKSS_OK, or the first device-side error (DKSS_EDEVICE, DKSS_ETIMEOUT).
 */
dkss_status dkss_sync_status(dkss_plan_t plan, dkss_stream_t stream);

/* Free a plan and its device memory (waits for the device).  NULL is a no-op. */
dkss_status dkss_plan_destroy(dkss_plan_t plan);

/* Static text of a status code. */
const char* dkss_status_str(dkss_status s);

#ifdef __cplusplus
}
#endif

#endif /* DKSS_H */
