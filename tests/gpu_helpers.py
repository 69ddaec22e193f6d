"""Shared helpers of the GPU parity tests (marshalling only)."""
import numpy as np

import dkss_synth as syn


def to_dev(limbs):
    import torch
    return torch.from_numpy(np.ascontiguousarray(limbs, dtype=np.uint64).view(np.int64)).cuda()


def to_host(t):
    return t.cpu().numpy().view(np.uint64)


def residues(flat_words2):
    """(…, 2) uint64 words -> flat list of Python ints."""
    arr = np.asarray(flat_words2).reshape(-1, 2).astype(np.uint64)
    return [int(lo) | (int(hi) << 64) for lo, hi in arr]


def random_primes61(count, seed):
    """Random primes in [2^60, 2^61) (Miller-Rabin with many bases; test-side helper)."""
    import random
    rng = random.Random(seed)
    out = []
    while len(out) < count:
        n = rng.randrange(1 << 60, 1 << 61) | 1
        if all(pow(b, n - 1, n) == 1 for b in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)):
            out.append(n)
    return out


def mod_int(limbs, q):
    return syn.to_int(limbs) % q
