#!/usr/bin/env python3
"""Write SHA-256 digests of the oracle's results for the large workloads.

The 2^32-bit product is too large for the oracle to run inside a GPU test
(about half an hour on 8 host threads and 32 GiB of host memory), so this
script runs it once and stores digests that the GPU tests compare against:

* the product c = a*b (2*ceil(N/64) little-endian 64-bit words), and
* the forward transform a_hat_i = a(rho^i), i < 2M (Section 3.2.5), in
  natural order, 2M*m canonical residues of two little-endian 64-bit words
  each (the layout dkss_forward writes),

each as the digest of the whole array and of CHUNKS equal consecutive slices
(so that a mismatch can be located).  Operands are the workload's seeded
operands from dkss_synth.  Only oracle/ and dkss_synth are used: no value
comes from the CUDA library.

Usage: python tests/golden/make_large_digests.py [workload ...] [--threads T]
Output: tests/golden/<workload>_digests.txt
"""
import argparse
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for _p in (ROOT, os.path.join(ROOT, "oracle")):
    if _p not in sys.path:
        sys.path.insert(0, _p)

import numpy as np  # noqa: E402

import dkss_oracle as o  # noqa: E402
import dkss_synth as syn  # noqa: E402
import oracle_c  # noqa: E402

CHUNKS = 16
RESIDUE_SEED = 0x5245534944       # seed of the random 61-bit primes below


def random_primes61(count, seed):
    """Random primes in [2^60, 2^61): candidates from a seeded generator,
    kept when they pass Miller-Rabin to the first twelve prime bases."""
    import random
    rng = random.Random(seed)
    out = []
    while len(out) < count:
        n = rng.randrange(1 << 60, 1 << 61) | 1
        d, s = n - 1, 0
        while d % 2 == 0:
            d //= 2
            s += 1
        ok = True
        for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            x = pow(a, d, n)
            if x in (1, n - 1):
                continue
            for _ in range(s - 1):
                x = x * x % n
                if x == n - 1:
                    break
            else:
                ok = False
                break
        if ok:
            out.append(n)
    return out


def digests(arr, chunks=CHUNKS):
    """(whole-array digest, [digest of each of `chunks` equal slices]) of a
    uint64 array, over its little-endian bytes."""
    flat = np.ascontiguousarray(arr, dtype="<u8").reshape(-1)
    assert flat.size % chunks == 0
    step = flat.size // chunks
    whole = hashlib.sha256()
    parts = []
    for k in range(chunks):
        b = memoryview(flat[k * step:(k + 1) * step]).cast("B")
        whole.update(b)
        parts.append(hashlib.sha256(b).hexdigest())
    return whole.hexdigest(), parts


def golden_path(name):
    return os.path.join(HERE, "%s_digests.txt" % name)


def read_golden(name):
    """Parse a digest file: {'product': (words, whole, [chunks]), 'a_hat': (...)}."""
    out = {}
    with open(golden_path(name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *rest = line.split()
            if key in ("product", "a_hat"):
                words, whole = int(rest[0]), rest[1]
                out[key] = (words, whole, [])
            elif key in ("product_chunk", "a_hat_chunk"):
                out[key[:-6]][2].append(rest[1])
            elif key == "residue":
                out.setdefault("residues", []).append((int(rest[0]), int(rest[1])))
            else:
                out[key] = rest
    return out


def write_one(name, threads):
    cfg = syn.workload_params(name)
    par = o.Params(*cfg).check()
    rho = o.compute_roots(par).rho
    A, B = syn.operand_pair(par.n_bits, syn.config_seed(syn.WORKLOADS[name]["index"]))
    used = oracle_c.set_threads(threads)
    t0 = time.time()
    c, d = oracle_c.dkss_mul(A, B, par, rho, dumps=("a_hat",))
    dt = time.time() - t0
    lines = [
        "# SHA-256 digests of the CPU oracle's results for workload %s" % name,
        "# (operands: dkss_synth.operand_pair(N, config_seed(%d)); natural order,"
        " little-endian 64-bit words)" % syn.WORKLOADS[name]["index"],
        "# written by tests/golden/make_large_digests.py (oracle/ only; %d host threads, %.0f s)" % (used, dt),
        "params %d %d %d %d %d %d" % cfg,
    ]
    # residues of the oracle's product mod random primes: a CPU test checks
    # them against (a mod q)(b mod q) mod q, which pins the stored product
    cint = syn.to_int(c)
    for q in random_primes61(4, RESIDUE_SEED):
        lines.append("residue %d %d" % (q, cint % q))
    del cint
    for key, arr in (("product", c), ("a_hat", d["a_hat"])):
        whole, parts = digests(arr)
        lines.append("%s %d %s" % (key, arr.size, whole))
        lines += ["%s_chunk %d %s" % (key, k, h) for k, h in enumerate(parts)]
    with open(golden_path(name), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("%s: oracle %.0f s on %d threads -> %s" % (name, dt, used, golden_path(name)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=["dkss_2p32b"])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for name in args.workloads:
        write_one(name, args.threads)


if __name__ == "__main__":
    main()
