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


# Proper rotations of the reference cube [0,1]^3: (axes, flips) with
# xi_old[a] = 1 - xi_new[axes[a]] if flips[a] else xi_new[axes[a]], determinant +1.
def cube_rotations():
    import itertools
    out = []
    for axes in itertools.permutations(range(3)):
        sign = 1
        for i in range(3):
            for j in range(i + 1, 3):
                if axes[i] > axes[j]:
                    sign = -sign
        for flips in itertools.product((0, 1), repeat=3):
            if sign * (-1) ** sum(flips) == 1:
                out.append((tuple(axes), tuple(flips)))
    return out


def scrambled_box(m, seed, distort=0.0, bc=(0, 0, 0, 0, 0, 0)):
    """An m0 x m1 x m2 hexahedral box on [0,1]^3 written as an unstructured mesh.

    Vertices are renumbered by a seeded permutation; cells are renumbered by
    another one, and every cell's local vertex order is turned by a seeded
    proper rotation of the reference cube; with distort > 0 every interior
    vertex moves by up to distort * h in each coordinate (seeded uniform), which
    makes the cells general trilinear hexahedra.  face_bc[e, f] is the code
    bc[side] of the box side a boundary face lies on (0 elsewhere).

    Returns vertices (nv, 3), cells (E, 8) (local vertex i + 2 j + 4 k at the
    reference corner (i, j, k)), face_bc (E, 6), and for the tests the cell map
    new -> old cell and every new cell's rotation (axes, flips) against the
    structured numbering of the box (cell i0 + m0 (i1 + m1 i2), local vertex of
    corner (i, j, k) at grid vertex (i0 + i, i1 + j, i2 + k)).
    """
    m = tuple(int(v) for v in (m if np.ndim(m) else (m, m, m)))
    g = (m[0] + 1, m[1] + 1, m[2] + 1)
    nv = g[0] * g[1] * g[2]
    vid = np.arange(nv)
    gx, gy, gz = vid % g[0], (vid // g[0]) % g[1], vid // (g[0] * g[1])
    X = np.stack([gx / m[0], gy / m[1], gz / m[2]], axis=1).astype(np.float64)
    if distort > 0:
        inner = (gx > 0) & (gx < m[0]) & (gy > 0) & (gy < m[1]) & (gz > 0) & (gz < m[2])
        for a in range(3):
            X[inner, a] += distort / m[a] * uniform(nv, seed + 10 + a)[inner]
    E = m[0] * m[1] * m[2]
    e = np.arange(E)
    i0, i1, i2 = e % m[0], (e // m[0]) % m[1], e // (m[0] * m[1])
    old_cells = np.zeros((E, 8), dtype=np.int64)
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, v >> 2
        old_cells[:, v] = (i0 + a) + g[0] * ((i1 + b) + g[1] * (i2 + c))
    # structured face codes: box side of each boundary face (old numbering)
    old_bc = np.zeros((E, 6), dtype=np.int64)
    ijk = (i0, i1, i2)
    for d in range(3):
        old_bc[ijk[d] == 0, 2 * d] = bc[2 * d]
        old_bc[ijk[d] == m[d] - 1, 2 * d + 1] = bc[2 * d + 1]
    vperm = np.argsort(splitmix64(np.uint64(seed) ^ np.arange(nv, dtype=np.uint64)))   # new -> old vertex
    vnew = np.empty(nv, dtype=np.int64)
    vnew[vperm] = np.arange(nv)                                                        # old -> new vertex
    cperm = np.argsort(splitmix64(np.uint64(seed + 1) ^ np.arange(E, dtype=np.uint64)))  # new -> old cell
    rots = cube_rotations()
    rsel = uniform_ints(E, 0, len(rots) - 1, seed + 2)
    cells = np.zeros((E, 8), dtype=np.int64)
    face_bc = np.zeros((E, 6), dtype=np.int64)
    rot = []
    for en in range(E):
        eo = cperm[en]
        axes, flips = rots[rsel[en]]
        rot.append((axes, flips))
        for v in range(8):
            xn = (v & 1, (v >> 1) & 1, v >> 2)
            xo = [(1 - xn[axes[a]]) if flips[a] else xn[axes[a]] for a in range(3)]
            cells[en, v] = vnew[old_cells[eo, xo[0] + 2 * xo[1] + 4 * xo[2]]]
        for f in range(6):
            d, s = divmod(f, 2)
            # new face xi_new[d] = s is the old face on axis a with axes[a] = d
            a = axes.index(d)
            so = (1 - s) if flips[a] else s
            face_bc[en, f] = old_bc[eo, 2 * a + so]
    return X[vperm], cells, face_bc, cperm, rot
