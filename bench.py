#!/usr/bin/env python3
"""Throughput of the DKSS_MUL hot path on GB300; prints one JSON line.

A step is one full product c = a*b of the 2^32-bit workload (M = 2^22,
m = 64, u = 32, p = 998244353, z = 4; the largest single-GPU workload):
encode, forward transforms of both operands, componentwise products,
backwards transform, decode and carry scan, all in libdkss's CUDA kernels.
Operands are seeded uniform random integers (--workload picks another size).

value      operand Gbit/s = 2N bits per product / device time per product
           (CUDA events on the launching stream; the transformed polynomials
           are 8 GiB each, far larger than L2, which is also flushed between
           steps by writing a 256 MiB buffer outside the timed events).
e2e        the same metric through dkss_mul_host (pinned host buffers,
           host->device copies of a and b and device->host copy of c inside
           the timed region).
roofline   the kernel group with the most device time, timed live with the
           library's per-stage CUDA events over the timed steps.
forms      the same product with every R-multiplication form (IMAD forms and
           the INT8 tensor-core form) and the TC-vs-IMAD ratios.
workloads  the other single-product workloads (65,536, 2^24 and 2^28 bits),
           each with its own form comparison.
batched    the 4096-product batch (one persistent kernel from a CUDA graph)
           against plain per-product launches.
thesis_points  the thesis's own operand lengths (its execution-time table)
           over z = 1 Proth rings, against its printed CPU times.
cpu_baseline  the CPU oracle (oracle/dkss_oracle.c) on all host cores and on
           one, on a bounded sample of the workload (oracle_sample).

--impl reference times that oracle alone on the host cores, same metric and
sample.  With torchrun (N > 1) every rank multiplies its own pair on its own
GPU (independent replicas; the product itself is not sharded).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
for _p in (ROOT, os.path.join(ROOT, "oracle")):
    if _p not in sys.path:
        sys.path.insert(0, _p)

import numpy as np  # noqa: E402

import dkss_synth as syn  # noqa: E402

METRIC = "DKSS_MUL operand Gbit/s and batched products/s on 1 GB300, bit-exact; TC vs IMAD"
WORKLOAD = "dkss_2p32b"
L2_FLUSH_BYTES = 256 << 20
SM_COUNT_GB300 = 152
IMAD_PER_SM_PER_CLK = 64          # 32-bit integer multiply-add lanes per SM per clock
SM_MAX_MHZ = 2070.0
HBM_GBS = 6782.1                  # STREAM-style copy bandwidth measured on a GB300 (HBM roofline denominator)
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture
# (profiles/stage_kernels_dkss_2p24b*.md); valid only for the kernel version captured.
FORM_FLAGS = {"ntt": 0, "mont": 512, "eval": 128, "direct": 16, "int8tc": 2}   # binding.ARITH_MONT, LEVELS_EVAL, ...
I8_TOPS = 150.0                   # mma.sync.m16n8k32 u8 throughput measured on a GB300 (2 ops per MAC)
NCU_TRAFFIC_BYTES = {("dkss_2p24b", "ntt", "fwd_twiddle"): 46.6e6,
                     ("dkss_2p24b", "eval", "fwd_twiddle"): 44.3e6}
# DRAM bytes (read + write) per element a bad-multiplication launch transforms,
# from one ncu capture of the same kernel on the 2^26-bit product with the same
# ring (profiles/stage_kernels_dkss_2p32b.md: 478 MB for 259,842 elements and
# 408 MB for 227,584); a full launch's traffic is this times its elements.
# The "mont" figures come from the 26-bit-limb Montgomery kernels, the "ntt"
# ones from the p-adic digit kernels with fast carries and digits in HBM
# (879.6 MB for 487,426 elements).
NCU_BYTES_PER_ELEMENT = {("dkss_2p32b", "mont", "config", "fwd_twiddle"): 1817.0,
                         ("dkss_2p26b_ring2p32", "mont", "config", "fwd_twiddle"): 1817.0,
                         ("dkss_2p32b", "ntt", "config", "fwd_twiddle"): 1805.0,
                         ("dkss_2p26b_ring2p32", "ntt", "config", "fwd_twiddle"): 1805.0}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(syn.WORKLOADS))
    ap.add_argument("--ring", default="config", choices=["config", "proth"],
                    help="the workload's ring p^z (config) or z = 1 with its Proth prime (dkss_proth_ring)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-batched", action="store_true", help="skip the 4096-product batched workload")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--no-forms", action="store_true", help="skip the R-multiplication form comparison")
    ap.add_argument("--form-budget-ms", type=float, default=4000.0,
                    help="device time per form and workload in the form comparison")
    ap.add_argument("--no-others", action="store_true", help="skip the other single-product workloads")
    ap.add_argument("--other-budget-ms", type=float, default=1000.0)
    ap.add_argument("--no-thesis-points", action="store_true",
                    help="skip the thesis's operand lengths over Proth rings")
    ap.add_argument("--thesis-budget-ms", type=float, default=600.0)
    ap.add_argument("--form", default="ntt", choices=["ntt", "mont", "eval", "direct", "int8tc"],
                    help="alpha-shift inner DFTs with R-multiplications through the evaluation map of R (ntt, the "
                         "default; p-adic digits for m = 64 over p^4), the same with 26-bit-limb Montgomery "
                         "products (mont), inner levels in evaluation coordinates (eval), the direct convolution, "
                         "or INT8 tensor-core byte-slice convolutions (int8tc)")
    return ap.parse_args()


def workload_config(name):
    w = syn.WORKLOADS[name]
    return {"workload": name, "n_bits": w["n_bits"], "M": w["M"], "m": w["m"], "u": w["u"], "p": w["p"],
            "z": w["z"], "products_per_step": 1}


def max_over_ranks(x, device, world):
    """Largest x over the ranks: a job's time is its slowest rank's (replicas
    only; no collective touches the data path)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbit_s(bits_per_rank_step, world, ms_per_step):
    """Whole-job operand Gbit/s: the operand bits all ranks multiplied in one
    step over the slowest rank's step time."""
    return bits_per_rank_step * world / (ms_per_step * 1e-3) / 1e9


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="dkss_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------ algorithmic counts ----

def modmul_imads(L):
    """32-bit multiply-adds of one Montgomery product of L-limb residues: L^2
    limb products (lo and hi halves) plus the reduction's L(L+1) products."""
    return 2 * L * L + L * (2 * L + 1)


def padic_mul_imads(z):
    """32-bit multiply-adds of one product mod p^z in p-adic digits: the
    z(z+1)/2 digit products of the truncated columns (lo and hi halves), and per
    column a Barrett carry: the high half of a 64 x 64-bit product by the
    reciprocal of p (seven multiply-adds) and one low product q p."""
    return z * (z + 1) + 8 * z


def rmul_imads(m, L, form, pointwise=False, padic_z=0):
    """Multiply-adds of one R-multiplication.
    direct: the negacyclic convolution (thesis eq. ncycconv), m^2 limb-level
      products and m reductions.
    ntt: through the evaluation map of R (forward transform of each variable
      factor, m/2 log2 m products; m pointwise products; backwards transform,
      m/2 (log2 m + 1) products including the final scaling)."""
    if form == "direct":
        return 2 * m * m * L * L + m * L * (2 * L + 1)
    lg = m.bit_length() - 1
    forwards = 2 if pointwise else 1
    per = padic_mul_imads(padic_z) if padic_z else modmul_imads(L)
    return (forwards * (m // 2) * lg + m + (m // 2) * (lg + 1)) * per


def nontrivial_dft_products(n):
    """Twiddle products of a radix-2 DIT of n points other than those by 1."""
    return sum(n // 2 - n // (2 << s) for s in range(1, n.bit_length() - 1))


def stage_work_eval(info, m, L):
    """Algorithmic multiply-adds of the levels-in-evaluation-coordinates form,
    by kernel group: level 0 maps every element to evaluation coordinates (m/2
    log m products) and multiplies its twiddle (m); levels d >= 1 run 2m-point
    DFTs over P per coordinate and pointwise twiddles; the last level r-point
    DFTs, the scaled componentwise products (2 per coordinate) and inverse DFTs;
    backwards, pointwise twiddles, DFTs, and level 0's return to coefficients
    (m/2 (log m + 1)).  Products by 1 are not counted."""
    P2, col_levels = info["P2"], info["levels"] - 1
    lg = m.bit_length() - 1
    r_last = P2 // (2 * m) ** col_levels
    nontrivial, length = [], P2
    for _ in range(col_levels):
        mu_d = length // (2 * m)
        nontrivial.append((P2 // length) * (mu_d - 1) * (2 * m - 1))
        length //= 2 * m
    cols = P2 // (2 * m)
    dft = cols * m * nontrivial_dft_products(2 * m)
    fwd = P2 * (m // 2) * lg + nontrivial[0] * m + sum(dft + nt * m for nt in nontrivial[1:])
    fin = 2 * (P2 // r_last) * m * nontrivial_dft_products(r_last) + 2 * P2 * m + (P2 // r_last) * m * nontrivial_dft_products(r_last)
    inv = P2 * (m // 2) * (lg + 1) + nontrivial[0] * m + sum(dft + nt * m for nt in nontrivial[1:])
    k = modmul_imads(L)
    return {"fwd_twiddle": (2 * fwd * k, col_levels), "final_pointwise": (fin * k, 1),
            "inv_twiddle": (inv * k, col_levels)}


def stage_work_i8(info, m):
    """Tensor-core operations of the INT8 form by kernel group (2 per u8
    multiply-accumulate): an R-multiplication of residues of S bytes is, for
    each of the S byte planes of one factor, an m x m Toeplitz matrix times
    the m x S matrix of the other factor's bytes, S^2 m^2 MACs.  Twiddles
    rho^0 = 1 are not work; every componentwise product is one
    R-multiplication.  The integer recombination and reduction are not
    counted (they run on the integer pipe)."""
    P2, col_levels = info["P2"], info["levels"] - 1
    S = (info["pz"].bit_length() + 7) // 8
    nontrivial, length = [], P2
    for _ in range(col_levels):
        mu_d = length // (2 * m)
        nontrivial.append((P2 // length) * (mu_d - 1) * (2 * m - 1))
        length //= 2 * m
    r = 2 * S * S * m * m
    return {"fwd_twiddle": (2 * sum(nontrivial) * r, col_levels), "final_pointwise": (P2 * r, 1),
            "inv_twiddle": (sum(nontrivial) * r, col_levels)}


def transformed_elements(info, m):
    """Elements each radix-2m level's bad multiplications transform (twiddle
    not 1), per operand."""
    out, length = [], info["P2"]
    for _ in range(info["levels"] - 1):
        mu_d = length // (2 * m)
        out.append((info["P2"] // length) * (mu_d - 1) * (2 * m - 1))
        length //= 2 * m
    return out


def stage_work(info, m, form):
    """Per kernel group: (algorithmic 32-bit multiply-adds per step, launches
    per step).  Twiddles rho^0 = 1 are not work; every other twiddle and every
    componentwise product is one R-multiplication (the direct form also scales
    each product coefficient by (2M)^-1 with one Montgomery product).  The
    inner DFTs have no products."""
    P2, L, col_levels = info["P2"], info["L"], info["levels"] - 1
    if form == "eval":
        return stage_work_eval(info, m, L)
    if form == "int8tc":
        return stage_work_i8(info, m)
    nontrivial = []
    length = P2
    for _ in range(col_levels):
        mu_d = length // (2 * m)
        nontrivial.append((P2 // length) * (mu_d - 1) * (2 * m - 1))
        length //= 2 * m
    # m = 64 over p^4: the NTT form's products are p-adic (plan info "padic")
    pz = info["z"] if info.get("padic") and form != "direct" else 0
    r = rmul_imads(m, L, form, padic_z=pz)
    rp = rmul_imads(m, L, form, pointwise=True, padic_z=pz)
    scale = P2 * m * modmul_imads(L) if form == "direct" else 0
    return {
        "fwd_twiddle": (2 * sum(nontrivial) * r, col_levels),
        "final_pointwise": (P2 * rp + scale, 1),
        "inv_twiddle": (sum(nontrivial) * r, col_levels),
    }


# ----------------------------------------------------------------- ours ----

CHECK_PRIMES = (2147483647, 2147483629, 2147483587)   # the three largest primes below 2^31


def limb_residues(limbs, primes=CHECK_PRIMES):
    """sum_k limbs[k] 2^(64k) mod q for each q < 2^31, vectorised: the powers
    2^(64k) mod q come from an outer product of block powers (every partial
    product stays below 2^62)."""
    x = np.asarray(limbs, dtype=np.uint64).reshape(-1)
    n = x.size
    out = []
    blk = 1 << 12
    nb = (n + blk - 1) // blk
    for q in primes:
        r = pow(2, 64, q)
        small = np.empty(blk, dtype=np.uint64)
        big = np.empty(nb, dtype=np.uint64)
        acc = 1
        for i in range(blk):
            small[i] = acc
            acc = acc * r % q
        rb, acc = acc, 1
        for j in range(nb):
            big[j] = acc
            acc = acc * rb % q
        total = 0
        for j0 in range(0, nb, 1 << 12):                       # slabs of 2^24 limbs
            j1 = min(nb, j0 + (1 << 12))
            pw = (big[j0:j1, None] * small[None, :]) % np.uint64(q)
            seg = x[j0 * blk:j1 * blk]
            pw = pw.reshape(-1)[:seg.size]
            total += int(np.sum(((seg % np.uint64(q)) * pw) % np.uint64(q), dtype=np.uint64))
        out.append(total % q)
    return out


def check_product(got, A, B, ra=None, rb=None):
    """Low word and residues mod three 31-bit primes against the operands'
    (a bounded check at any size; never the full product)."""
    if int(got[0]) != (int(A[0]) * int(B[0])) % (1 << 64):
        return False
    ra = ra or limb_residues(A)
    rb = rb or limb_residues(B)
    rc = limb_residues(got)
    return all(c == x * y % q for c, x, y, q in zip(rc, ra, rb, CHECK_PRIMES))


def time_steps(fn, steps, flush, stream):
    """Device ms per call of fn(): CUDA events on the launching stream around
    each call, L2 flushed (256 MiB write) outside the events."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.fill_(1)
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def steps_for(ms_estimate, budget_ms, lo=2, hi=200):
    return int(max(lo, min(hi, budget_ms // max(ms_estimate, 1e-3))))


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1503_04955_gb300 as dk
    from paper_1503_04955_gb300 import binding

    world, rank, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = syn.workload_params(args.workload)
    n_bits = cfg[0]
    A, B = syn.operand_pair(n_bits, syn.config_seed(syn.WORKLOADS[args.workload]["index"]), product=rank)
    flags = binding.FORM_PROFILE | FORM_FLAGS[args.form]
    if args.ring == "proth":      # the same N, M, m, u over the Proth ring of dkss_proth_ring
        h, n = dk.proth_ring(*cfg[:4])
        plan = dk.Plan.proth(*cfg[:4], h, n, flags=flags)
    else:
        plan = dk.Plan(*cfg, flags=flags)
    info = plan.info()
    plan_p = info["p"]
    a = torch.from_numpy(A.view(np.int64)).to(dev)
    b = torch.from_numpy(B.view(np.int64)).to(dev)
    out = torch.empty(2 * A.size, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(3, args.warmup)):
        plan.mul(a, b, out)
    torch.cuda.synchronize(dev)
    plan.profile_read()
    plan.sync_status()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    sampler = ClockSampler(gpu_index) if rank == 0 else None
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for e0, e1 in events:
        flush.fill_(1)                       # evict L2 (untimed: outside the events)
        e0.record(stream)
        plan.mul(a, b, out)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    step_ms = [e0.elapsed_time(e1) for e0, e1 in events]
    prof = plan.profile_read()
    plan.sync_status()
    total_ms = max_over_ranks(sum(step_ms), dev, world)
    ms_per_step = total_ms / args.steps
    value = job_gbit_s(2 * n_bits, world, ms_per_step)
    rab = (limb_residues(A), limb_residues(B))
    ok = check_product(out.cpu().numpy().view(np.uint64), A, B, *rab)

    # end to end through dkss_mul_host from pinned host memory
    a_h = torch.from_numpy(A.view(np.int64)).pin_memory()
    b_h = torch.from_numpy(B.view(np.int64)).pin_memory()
    c_h = torch.empty(2 * A.size, dtype=torch.int64).pin_memory()
    an, bn, cn = (x.numpy().view(np.uint64) for x in (a_h, b_h, c_h))
    plan.mul_host(an, bn, cn)
    e2e_steps = max(1, min(args.steps, args.e2e_steps, steps_for(ms_per_step, 8000)))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.mul_host(an, bn, cn)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dev, world)
    ok = ok and check_product(cn, A, B, *rab)
    e2e_value = job_gbit_s(2 * n_bits, world, e2e_s * 1e3)
    del a_h, b_h, c_h

    # squares of the same operand (dkss_mul with a == b: one forward transform)
    sq_steps = max(1, min(args.steps, 50, steps_for(ms_per_step, 4000)))
    sq_ms = sum(time_steps(lambda: plan.mul(a, a, out), sq_steps, flush, stream)) / sq_steps
    square = {"ms_per_step": round(sq_ms, 5), "speedup_vs_product": round(ms_per_step / sq_ms, 3),
              "bit_exact": bool(check_product(out.cpu().numpy().view(np.uint64), A, A, rab[0], rab[0]))}
    plan.profile_read()
    roofline = main_roofline(args, info, cfg, A, prof)
    launches = plan.launches * args.steps
    plan.close()

    forms = compare_forms(args.workload, args.form, dev, flush, a, b, out, ms_per_step, args.form_budget_ms, A, B,
                          rab) \
        if (rank == 0 and not args.no_forms) else None
    proth = proth_ring_time(args.workload, dev, flush, a, b, out, ms_per_step, args.form_budget_ms, A, B, rab) \
        if (rank == 0 and not args.no_forms) else None
    del a, b, out
    others = other_workloads(args, dev, flush) if (rank == 0 and not args.no_others) else None
    batched = run_batched(args, dev, flush) if (rank == 0 and not args.no_batched) else None
    thesis = thesis_points(args, dev, flush) if (rank == 0 and not args.no_thesis_points) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8" if args.form == "int8tc" else "u32",
            "data": "synthetic: SplitMix64 uniform operands in [0, 2^N)",
            "config": dict(workload_config(args.workload), form="int8tc" if args.form == "int8tc" else "imad",
                           ring="workload's p^z" if args.ring == "config" else "Proth prime %s (z = 1)" % plan_p,
                           rmul=args.form,
                           l2="inputs larger than L2 at 2^28 bits and up; also flushed between steps "
                              "(256 MiB write outside the timed events)",
                           parallelism="replicas" if world > 1 else "single GPU"),
            "products_per_s": round(world / (ms_per_step * 1e-3), 3),
            "bit_exact": bool(ok),
            "device_bytes": {"plan": info["dev_bytes"],
                             "bits_per_operand_bit": round(8 * info["dev_bytes"] / n_bits, 2)},
            "gpu_launches": launches,
            "e2e": {"value": round(e2e_value, 4), "unit": "Gbit/s", "h2d_bytes_per_step": 2 * A.nbytes,
                    "d2h_bytes_per_step": 2 * A.nbytes, "steps": e2e_steps},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "forms": forms,
            "proth_ring": proth,
            "square": square,
            "workloads": others,
            "batched": batched,
            "thesis_points": thesis,
            "clocks": clocks,
            "wall_s": round(wall, 3),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main_roofline(args, info, cfg, A, prof):
    """Roofline of the kernel group with the most device time (per-stage CUDA
    events of the library, on the launching stream, over the timed steps), and
    every group's own figure under 'stages'."""
    work = stage_work(info, cfg[2], args.form)
    dom = max((k for k in prof if k in work), key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    ops_per_step, launches_per_step = work[dom]
    ops_per_launch = ops_per_step / max(1, launches_per_step)
    avg_launch_ms = dom_ms / max(1, dom_n)
    achieved = ops_per_launch / (avg_launch_ms * 1e-3) / 1e12
    if args.form == "int8tc":
        bound, unit, peak = "tensor", "TOPS", I8_TOPS
        peak_basis = "mma.sync.m16n8k32 u8 throughput measured on a GB300 (2 ops per MAC)"
    else:
        bound, unit = "alu", "TIMAD/s"
        peak = SM_COUNT_GB300 * IMAD_PER_SM_PER_CLK * SM_MAX_MHZ * 1e6 / 1e12
        peak_basis = "152 SMs x 64 IMAD/clk x 2070 MHz (recipe unit counts and max clock)"
    # memory-bound groups: algorithmic bytes = one read and one write of the
    # polynomials they pass over (DFT levels), or of the product polynomial and
    # the product words (decode)
    poly_bytes = info["P2"] * cfg[2] * info["L"] * 4
    mem_bytes = {"fwd_dft": 2 * 2 * poly_bytes * (info["levels"] - 1),
                 "inv_dft": 2 * poly_bytes * (info["levels"] - 1),
                 "decode": poly_bytes + 4 * A.nbytes}
    stages = {}
    for k, (ms_tot, _) in prof.items():
        ms = ms_tot / args.steps
        if ms <= 0:
            continue
        if k in work:
            ach = work[k][0] / (ms * 1e-3) / 1e12
            stages[k] = {"bound": bound, "ms": round(ms, 4), "achieved": round(ach, 3), "unit": unit,
                         "frac": round(ach / peak, 4)}
        elif k in mem_bytes:
            ach = mem_bytes[k] / (ms * 1e-3) / 1e9
            stages[k] = {"bound": "hbm", "ms": round(ms, 4), "achieved": round(ach, 1), "unit": "GB/s",
                         "frac": round(ach / HBM_GBS, 4)}
    traffic = NCU_TRAFFIC_BYTES.get((args.workload, args.form, dom)) if args.ring == "config" else None
    per_elem = NCU_BYTES_PER_ELEMENT.get((args.workload, args.form, args.ring, dom))
    if per_elem is not None:
        elements = sum(transformed_elements(info, cfg[2])) * (2 if dom == "fwd_twiddle" else 1)
        traffic = round(per_elem * elements / max(1, launches_per_step))
    return {"bound": bound, "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": unit, "frac": round(achieved / peak, 4),
            "traffic": traffic,
            "stages": stages,
            "avg_launch_ms": round(avg_launch_ms, 4), "ops_per_launch": int(ops_per_launch),
            "peak_basis": peak_basis}


def other_workloads(args, dev, flush):
    """The other single-product workloads, default form, with the TC-vs-IMAD
    comparison of each: device ms per product, operand Gbit/s, products/s."""
    import torch

    import paper_1503_04955_gb300 as dk

    stream = torch.cuda.current_stream(dev)
    res = {}
    for name in ("dkss_65536b", "dkss_2p24b", "dkss_2p28b", "dkss_2p32b"):
        if name == args.workload:
            continue
        cfg = syn.workload_params(name)
        A, B = syn.operand_pair(cfg[0], syn.config_seed(syn.WORKLOADS[name]["index"]))
        a = torch.from_numpy(A.view(np.int64)).to(dev)
        b = torch.from_numpy(B.view(np.int64)).to(dev)
        out = torch.empty(2 * A.size, dtype=torch.int64, device=dev)
        with dk.Plan(*cfg) as plan:
            for _ in range(3):
                plan.mul(a, b, out)
            torch.cuda.synchronize(dev)
            t = time_steps(lambda: plan.mul(a, b, out), 2, flush, stream)
            steps = steps_for(min(t), args.other_budget_ms)
            ms = sum(time_steps(lambda: plan.mul(a, b, out), steps, flush, stream)) / steps
            rab = (limb_residues(A), limb_residues(B))
            ok = check_product(out.cpu().numpy().view(np.uint64), A, B, *rab)
        entry = {"ms_per_step": round(ms, 5), "latency_us": round(1e3 * ms, 2), "steps": steps,
                 "gbit_s": round(2 * cfg[0] / (ms * 1e-3) / 1e9, 4),
                 "products_per_s": round(1 / (ms * 1e-3), 2), "bit_exact": bool(ok)}
        if not args.no_forms:
            entry["forms"] = compare_forms(name, "ntt", dev, flush, a, b, out, ms, args.form_budget_ms, A, B, rab)
        if cfg[0] >= 1 << 24:
            entry["proth_ring"] = proth_ring_time(name, dev, flush, a, b, out, ms, args.form_budget_ms, A, B, rab)
        if not args.no_cpu_baseline:
            # the oracle (all host cores) on the whole workload: a few seconds up to 2^28 bits
            dt, c, cores = oracle_product_seconds(list(cfg), A, B, os.cpu_count() or 1)
            entry["cpu_oracle"] = {"seconds": round(dt, 3), "cores": cores,
                                   "gbit_s": round(2 * cfg[0] / dt / 1e9, 6),
                                   "bit_exact": bool(check_product(c, A, B, *rab)),
                                   "gpu_speedup": round(dt / (ms * 1e-3), 1)}
        res[name] = entry
        del a, b, out
    return res


def compare_forms(workload, main_form, dev, flush, a, b, out, ms_main, budget_ms, A, B, rab):
    """Device time per product of one workload with each R-multiplication
    form: through the evaluation map of R (alpha-shift inner DFTs, ntt; or
    inner levels in evaluation coordinates, eval) and the direct convolution
    on the integer pipe (IMAD), and INT8 tensor-core byte-slice products (TC).
    Each form's product is checked (low word and prime residues)."""
    import torch

    import paper_1503_04955_gb300 as dk
    from paper_1503_04955_gb300 import binding

    cfg = syn.workload_params(workload)
    res = {}
    stream = torch.cuda.current_stream(dev)
    for name, flags in (("ntt", 0), ("mont", binding.ARITH_MONT), ("eval", binding.LEVELS_EVAL),
                        ("direct", binding.RMUL_DIRECT), ("int8tc", binding.FORM_INT8TC)):
        if name == main_form:
            res[name] = {"ms_per_step": round(ms_main, 5)}
            continue
        try:
            plan = dk.Plan(*cfg, flags=flags)
        except dk.DkssError as e:
            res[name] = {"unsupported": str(e)}
            continue
        for _ in range(2):
            plan.mul(a, b, out)
        torch.cuda.synchronize(dev)
        t = time_steps(lambda: plan.mul(a, b, out), 1, flush, stream)
        steps = steps_for(t[0], budget_ms, lo=1, hi=50)
        ms = sum(time_steps(lambda: plan.mul(a, b, out), steps, flush, stream)) / steps
        ok = check_product(out.cpu().numpy().view(np.uint64), A, B, *rab)
        plan.close()
        res[name] = {"ms_per_step": round(ms, 5), "steps": steps, "bit_exact": bool(ok)}
    if all("ms_per_step" in res.get(k, {}) for k in ("int8tc", "direct", "ntt")):
        res["tc_vs_imad_direct"] = round(res["direct"]["ms_per_step"] / res["int8tc"]["ms_per_step"], 3)
        res["tc_vs_imad_ntt"] = round(res["ntt"]["ms_per_step"] / res["int8tc"]["ms_per_step"], 3)
    return res


def proth_ring_time(workload, dev, flush, a, b, out, ms_config, budget_ms, A, B, rab):
    """The same product (same N, M, m, u) over the Proth ring Z/pZ, p = h 2^n + 1
    of dkss_proth_ring (z = 1, the form of the thesis's primes), whose
    Montgomery reductions need no digit products: device ms per product in the
    default form, against the workload's own ring (p^z)."""
    import torch

    import paper_1503_04955_gb300 as dk

    n_bits, M, m, u = syn.workload_params(workload)[:4]
    try:
        h, n = dk.proth_ring(n_bits, M, m, u)
        plan = dk.Plan.proth(n_bits, M, m, u, h, n)
    except dk.DkssError as e:
        return {"unsupported": str(e)}
    info = plan.info()
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        plan.mul(a, b, out)
    torch.cuda.synchronize(dev)
    t = time_steps(lambda: plan.mul(a, b, out), 1, flush, stream)
    steps = steps_for(t[0], budget_ms, lo=1, hi=50)
    ms = sum(time_steps(lambda: plan.mul(a, b, out), steps, flush, stream)) / steps
    ok = check_product(out.cpu().numpy().view(np.uint64), A, B, *rab)
    plan.close()
    return {"h": h, "n": n, "p_bits": ((h << n) + 1).bit_length(), "L": info["L"], "LR": info["LR"],
            "sparse_reduction": bool(info["sparse"]), "ms_per_step": round(ms, 5), "steps": steps,
            "device_bytes": info["dev_bytes"], "bits_per_operand_bit": round(8 * info["dev_bytes"] / n_bits, 2),
            "gbit_s": round(2 * n_bits / (ms * 1e-3) / 1e9, 4),
            "speedup_vs_config_ring": round(ms_config / ms, 3), "bit_exact": bool(ok)}


# The thesis's execution times of DKSS_MUL at its most favourable lengths (its
# Section 4.4 table "Execution times of DKSS_MUL and SMUL"): operand length in
# 64-bit words and CPU cycles on one core of a 3.4 GHz Core i7-3770.
THESIS_TIMES = [(3648, 133948102), (7168, 288821718), (14336, 636214972), (28160, 1373645624),
                (56320, 2908271180), (110592, 6013189608), (221184, 13430829526), (434176, 29461464342),
                (868352, 62917787338), (1703936, 122680187946), (2752512, 199424397176),
                (5505024, 410390455672), (10878976, 892949727060), (21757952, 1917703330120),
                (42991616, 3965210546518), (85983232, 8145120758260)]
THESIS_HZ = 3.4e9


def thesis_points(args, dev, flush):
    """The thesis's operand lengths with its kind of ring: z = 1 and a Proth
    prime p = h 2^n + 1 (dkss_proth_ring) under the parameters its rule picks
    (largest u, smallest M m, M/m near N / log^3 N: dkss_plan_choose with the
    rule flag).  The thesis itself used u of 54 to 83 bits and 128- or 192-bit
    primes, which this build's limbs (u <= 32, p^z < 2^126) do not hold, so
    u is 32 here.  Device ms per product against the thesis's CPU time."""
    import torch

    import paper_1503_04955_gb300 as dk

    stream = torch.cuda.current_stream(dev)
    out_rows = []
    for words, cycles in THESIS_TIMES:
        n_bits = 64 * words
        M, m, u, _, _ = dk.plan_choose(n_bits, dk.TUNE_RULE)
        try:
            h, n = dk.proth_ring(n_bits, M, m, u)
            plan = dk.Plan.proth(n_bits, M, m, u, h, n)
        except dk.DkssError as e:
            out_rows.append({"words": words, "unsupported": str(e)})
            continue
        A, B = syn.operand_pair(n_bits, syn.config_seed(100), product=words)
        a = torch.from_numpy(A.view(np.int64)).to(dev)
        b = torch.from_numpy(B.view(np.int64)).to(dev)
        out = torch.empty(2 * A.size, dtype=torch.int64, device=dev)
        for _ in range(2):
            plan.mul(a, b, out)
        torch.cuda.synchronize(dev)
        t = time_steps(lambda: plan.mul(a, b, out), 1, flush, stream)
        steps = steps_for(t[0], args.thesis_budget_ms, lo=1, hi=20)
        ms = sum(time_steps(lambda: plan.mul(a, b, out), steps, flush, stream)) / steps
        ok = check_product(out.cpu().numpy().view(np.uint64), A, B)
        plan.close()
        thesis_s = cycles / THESIS_HZ
        out_rows.append({"words": words, "n_bits": n_bits, "M": M, "m": m, "u": u, "p": "%d*2^%d+1" % (h, n),
                         "ms_per_step": round(ms, 4), "gbit_s": round(2 * n_bits / (ms * 1e-3) / 1e9, 3),
                         "thesis_s": round(thesis_s, 4), "speedup_vs_thesis": round(thesis_s / (ms * 1e-3), 1),
                         "bit_exact": bool(ok)})
        del a, b, out
    return out_rows


def run_batched(args, dev, flush):
    """4096 products, operand lengths 2^x with x uniform in [14, 20] rounded to
    64-bit limbs: one persistent-kernel launch under a CUDA graph per step,
    against plain per-product dkss_mul launches with the same parameters."""
    import torch

    import paper_1503_04955_gb300 as dk

    w = syn.BATCH_WORKLOAD
    seed = syn.config_seed(w["index"])
    lengths = [int(n) for n in syn.log_uniform_lengths(w["count"], seed, w["lo_exp"], w["hi_exp"])]
    words = [syn.n_limbs(n) for n in lengths]
    total = sum(words)
    a_all = torch.empty(total, dtype=torch.int64, device=dev)
    b_all = torch.empty(total, dtype=torch.int64, device=dev)
    o_all = torch.zeros(2 * total, dtype=torch.int64, device=dev)
    a_l, b_l, o_l, ops = [], [], [], []
    off = 0
    for j, (n, wd) in enumerate(zip(lengths, words)):
        A, B = syn.operand_pair(n, seed, product=j)
        ops.append((A, B))
        a_all[off:off + wd] = torch.from_numpy(A.view(np.int64)).to(dev)
        b_all[off:off + wd] = torch.from_numpy(B.view(np.int64)).to(dev)
        a_l.append(a_all[off:off + wd])
        b_l.append(b_all[off:off + wd])
        o_l.append(o_all[2 * off:2 * off + 2 * wd])
        off += wd
    t0 = time.perf_counter()
    bt = dk.Batch(lengths)
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        bt.run(a_l, b_l, o_l)
    torch.cuda.synchronize(dev)
    steps = max(1, args.batched_steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.fill_(1)
        e0.record(stream)
        bt.run(a_l, b_l, o_l)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
    ok = all(check_product(o.cpu().numpy().view(np.uint64), A, B)
             for o, (A, B) in zip(o_l[::16], ops[::16]))
    classes = {}
    for j in range(len(lengths)):
        prm = bt.job_params(j)
        key = prm["class_bits"]
        if key not in classes:
            classes[key] = {"M": prm["M"], "u": prm["u"], "levels": prm["levels"], "jobs": 0,
                            "p_bits": prm["p"].bit_length(), "z": prm["z"], "proth": bool(prm["proth"])}
        classes[key]["jobs"] += 1
    graph = bool(bt.job_params(0)["graph"])
    grid = bt.job_params(0)["grid"]
    proth = bool(bt.job_params(0)["proth"])
    # plain per-product launches with each class's parameters (one plan per
    # distinct length: a plan is fixed to one N)
    plain_plans = {}
    for j, n in enumerate(lengths):
        if n not in plain_plans:
            plain_plans[n] = bt.class_plan(j)
    bt.close()
    for _ in range(2):
        for j, n in enumerate(lengths):
            plain_plans[n].mul(a_l[j], b_l[j], o_l[j])
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    e0.record(stream)
    for j, n in enumerate(lengths):
        plain_plans[n].mul(a_l[j], b_l[j], o_l[j])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1)
    for p in plain_plans.values():
        p.close()
    bits = 2 * sum(lengths)
    return {"workload": "dkss_batch_4096_log_uniform_2p14_2p20", "products": len(lengths),
            "operand_bits": bits, "ms_per_batch": round(ms, 4),
            "products_per_s": round(len(lengths) / (ms * 1e-3), 1),
            "operand_gbit_s": round(bits / (ms * 1e-3) / 1e9, 3),
            "plain_launches_ms": round(plain_ms, 4),
            "speedup_vs_plain_launches": round(plain_ms / ms, 3),
            "graph": graph, "persistent_grid": grid, "plan_s": round(plan_s, 3), "bit_exact_sampled": bool(ok),
            "rings": "Proth primes (z = 1, sparse reduction)" if proth else "configured primes (smallest p^z per class)",
            "classes": {str(k): v for k, v in sorted(classes.items())}}


# ------------------------------------------------------------- reference ----

# The oracle's full product at 2^32 bits takes about half an hour on 8 host
# threads; a bench step takes a bounded sample of the workload instead: one
# full product of operands 2^(32-SAMPLE_SHIFT) bits long with the same ring
# and encoding (m, u, p, z; M scaled with N), 2^23 bits for the 2^32-bit
# workload.  Smaller workloads are timed whole.
SAMPLE_MAX_BITS = 1 << 23


def oracle_sample(name):
    """(params, operands, description) of the oracle's timed sample of workload `name`."""
    cfg = list(syn.workload_params(name))
    n_bits = cfg[0]
    if n_bits <= SAMPLE_MAX_BITS:
        A, B = syn.operand_pair(n_bits, syn.config_seed(syn.WORKLOADS[name]["index"]))
        return cfg, A, B, "one full %s product" % name
    shift = (n_bits // SAMPLE_MAX_BITS).bit_length() - 1
    cfg[0] = n_bits >> shift
    cfg[1] = cfg[1] >> shift
    A, B = syn.operand_pair(cfg[0], syn.config_seed(syn.WORKLOADS[name]["index"]))
    desc = ("one full product of %d-bit operands with the %s ring and encoding (M=%d, m=%d, u=%d, p=%d, z=%d), "
            "the bounded sample of the %d-bit workload" % (cfg[0], name, cfg[1], cfg[2], cfg[3], cfg[4], cfg[5],
                                                            n_bits))
    return cfg, A, B, desc


def oracle_product_seconds(cfg, A, B, threads):
    import dkss_oracle
    import oracle_c
    par = dkss_oracle.Params(*cfg).check()
    rho = dkss_oracle.compute_roots(par).rho
    used = oracle_c.set_threads(threads)
    t0 = time.perf_counter()
    c, _ = oracle_c.dkss_mul(A, B, par, rho)
    dt = time.perf_counter() - t0
    return dt, c, used


def cpu_baseline(name):
    """The oracle (oracle/dkss_oracle.c as it stands) on the host cores: all of
    them (OpenMP over its independent loops) and one thread, on the workload's
    bounded sample; operand Gbit/s of the sample."""
    cfg, A, B, desc = oracle_sample(name)
    dt_all, c, cores = oracle_product_seconds(cfg, A, B, os.cpu_count() or 1)
    ok = check_product(c, A, B)
    dt_one, _, _ = oracle_product_seconds(cfg, A, B, 1)
    return {"value": round(2 * cfg[0] / dt_all / 1e9, 6), "unit": "Gbit/s", "cores": cores, "kind": "oracle",
            "sample": "%s: %.2f s on %d host threads" % (desc, dt_all, cores),
            "single_thread": {"value": round(2 * cfg[0] / dt_one / 1e9, 6), "cores": 1, "seconds": round(dt_one, 3)},
            "bit_exact_checked": bool(ok)}


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    name = args.workload
    cfg, A, B, desc = oracle_sample(name)
    small = syn.workload_params("dkss_65536b")
    Aw, Bw = syn.operand_pair(small[0], 7)
    cores = os.cpu_count() or 1
    for _ in range(max(3, args.warmup)):      # warm-up on the small workload (bounded)
        oracle_product_seconds(small, Aw, Bw, cores)
    budget_s = 150.0
    times = []
    while len(times) < args.steps:
        dt, c, used = oracle_product_seconds(cfg, A, B, cores)
        times.append(dt)
        if sum(times) + dt > budget_s:
            break
    mean = sum(times) / len(times)
    value = 2 * cfg[0] / mean / 1e9
    sample = "%s per step, %d host threads; %d of %d steps requested (capped at %.0f s)" % (
        desc, used, len(times), args.steps, budget_s)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gbit/s", "n_gpus": world,
        "steps": len(times), "warmup": max(3, args.warmup), "ms_per_step": round(mean * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128",
        "data": "synthetic: SplitMix64 uniform operands in [0, 2^N)",
        "config": dict(workload_config(name), form="cpu oracle"),
        "cpu_baseline": {"value": round(value, 6), "unit": "Gbit/s", "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "bit_exact": bool(check_product(c, A, B)),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
