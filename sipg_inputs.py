"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: only the counter-based random
generator, the named workload shapes and small helpers that turn them into
arguments.  Both sides of every parity check draw their inputs from here.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as in Vigna's public reference): the first
output of a SplitMix64 stream whose state is ``seed XOR i`` gives entry i, so
any entry can be produced independently.  u_i = 2 * ((z >> 11) * 2^-53) - 1 is
uniform in [-1, 1).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output for state(s) x (uint64 array): one step of the stream."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(n, seed, dtype=np.float64):
    """n values uniform in [-1, 1): u_i from splitmix64(seed XOR i)."""
    i = np.arange(n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed) ^ i)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (2.0 * u - 1.0).astype(dtype)


def uniform_ints(n, lo, hi, seed):
    """n integers uniform in [lo, hi] from the same stream (by modulo, tiny bias)."""
    i = np.arange(n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed) ^ i)
    return (lo + (z % np.uint64(hi - lo + 1)).astype(np.int64)).astype(np.int64)


# Seeds of the workloads
SEED_APPLY = 1910      # operator_apply input vector
SEED_RHS = 1911        # random right-hand side r uses SEED_RHS + r
SEED_EIG = 1910        # start vector of the eigenvalue estimate
SEED_BATCH = 2019      # draw of the batched problem set

# Named workloads: mesh cells per direction m, degree k, curved mapping flag.
WORKLOADS = {
    # 4^3 Cartesian unit cube, k=3, Dirichlet, manufactured sine RHS
    "cube4_k3": dict(m=4, k=3, deform=0),
    # 16^3 curved (x_i += 0.1 prod sin(pi x_j), degree-3 mapping), k=5
    "curved16_k5": dict(m=16, k=5, deform=1),
    # 32^3 Cartesian, k=4, mixed-precision V-cycle
    "cube32_k4": dict(m=32, k=4, deform=0),
    # 16^3 Cartesian, k=4, 32 right-hand sides
    "cube16_k4": dict(m=16, k=4, deform=0),
    # 32^3 curved, k=4, learned smoother
    "curved32_k4": dict(m=32, k=4, deform=1),
}

# Operator-apply sweep at about 16 MDoF for k = 1..8 (cells per direction)
SWEEP_M = {1: 126, 2: 84, 3: 63, 4: 50, 5: 42, 6: 36, 7: 32, 8: 28}


def batch_problems(count=16, seed=SEED_BATCH):
    """The batched set: m even in {8,...,24}, k in {2,...,6}, both drawn from seed."""
    ms = 8 + 2 * uniform_ints(count, 0, 8, seed)
    ks = uniform_ints(count, 2, 6, seed + 1)
    return [dict(m=int(m), k=int(k), deform=0) for m, k in zip(ms, ks)]
