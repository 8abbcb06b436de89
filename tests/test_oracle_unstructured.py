"""Pins of the oracle's SIPG operator on unstructured hexahedral meshes.

The unstructured oracle finds which face points of two neighbours coincide from
their physical positions alone.  It is pinned by
  * the structured box: a box mesh written with shuffled vertex and cell numbers
    and every cell's local vertex order turned by a proper rotation of the cube
    gives the structured oracle's operator (Cartesian and curved, mixed
    boundary conditions), up to the matching renumbering of the degrees of
    freedom;
  * relabelling invariance on distorted (general trilinear) cells: shuffling
    and rotating the cells of such a mesh again permutes the operator;
  * symmetry, positive definiteness with Dirichlet faces, and the constant null
    space with Neumann faces only.
"""
import numpy as np
import pytest

import sipg_inputs
from oracle.dg import SIPG
from oracle.mesh import Mesh
from oracle.unstructured import HexMesh, USIPG


def dof_map(k, cperm, rot, n_cells):
    """new DoF index -> old (structured) DoF index for scrambled_box's renumbering."""
    n = k + 1
    n3 = n ** 3
    out = np.zeros(n_cells * n3, dtype=np.int64)
    for en in range(n_cells):
        axes, flips = rot[en]
        for p in range(n3):
            an = (p % n, (p // n) % n, p // (n * n))
            ao = [(n - 1 - an[axes[a]]) if flips[a] else an[axes[a]] for a in range(3)]
            out[en * n3 + p] = cperm[en] * n3 + ao[0] + n * ao[1] + n * n * ao[2]
    return out


def rescramble(V, C, F, seed):
    """The same mesh with cells shuffled and each cell's local order turned again."""
    E = len(C)
    cperm = np.argsort(sipg_inputs.splitmix64(np.uint64(seed) ^ np.arange(E, dtype=np.uint64)))
    rots = sipg_inputs.cube_rotations()
    rsel = sipg_inputs.uniform_ints(E, 0, len(rots) - 1, seed + 1)
    C2, F2, rot = np.zeros_like(C), np.zeros_like(F), []
    for en in range(E):
        eo = cperm[en]
        axes, flips = rots[rsel[en]]
        rot.append((axes, flips))
        for v in range(8):
            xn = (v & 1, (v >> 1) & 1, v >> 2)
            xo = [(1 - xn[axes[a]]) if flips[a] else xn[axes[a]] for a in range(3)]
            C2[en, v] = C[eo, xo[0] + 2 * xo[1] + 4 * xo[2]]
        for f in range(6):
            d, s = divmod(f, 2)
            a = axes.index(d)
            F2[en, f] = F[eo, 2 * a + ((1 - s) if flips[a] else s)]
    return V, C2, F2, cperm, rot


@pytest.mark.parametrize("k,deform", [(1, 0), (2, 1), (3, 0)])
def test_scrambled_box_reproduces_structured_operator(k, deform):
    m, bc = (3, 2, 2), (0, 1, 0, 0, 1, 0)
    V, C, F, cperm, rot = sipg_inputs.scrambled_box(m, 11, bc=bc)
    Au = USIPG(HexMesh(V, C, F, deform=deform), k).assemble().toarray()
    As = SIPG(Mesh(m, deform=deform, bc=bc), k).assemble().toarray()
    old = dof_map(k, cperm, rot, len(C))
    ref = As[np.ix_(old, old)]
    assert np.max(np.abs(Au - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_relabelling_a_distorted_mesh_permutes_the_operator():
    k = 2
    V, C, F, _, _ = sipg_inputs.scrambled_box((3, 3, 2), 21, distort=0.2, bc=(0, 0, 1, 0, 0, 1))
    A = USIPG(HexMesh(V, C, F), k).assemble().toarray()
    V2, C2, F2, cperm, rot = rescramble(V, C, F, 77)
    A2 = USIPG(HexMesh(V2, C2, F2), k).assemble().toarray()
    old = dof_map(k, cperm, rot, len(C))
    assert np.max(np.abs(A2 - A[np.ix_(old, old)])) <= 1e-12 * np.max(np.abs(A))
    # the distortion is real: the operator differs from the undistorted box's
    Vb, Cb, Fb, _, _ = sipg_inputs.scrambled_box((3, 3, 2), 21, bc=(0, 0, 1, 0, 0, 1))
    Ab = USIPG(HexMesh(Vb, Cb, Fb), k).assemble().toarray()
    assert np.max(np.abs(A - Ab)) > 1e-3 * np.max(np.abs(A))


def test_symmetric_spd_and_neumann_null_space_on_distorted_cells():
    k = 2
    V, C, F, _, _ = sipg_inputs.scrambled_box((2, 2, 2), 5, distort=0.2)
    A = USIPG(HexMesh(V, C, F, deform=1), k).assemble().toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-13 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A).min() > 0
    Vn, Cn, Fn, _, _ = sipg_inputs.scrambled_box((2, 2, 2), 5, distort=0.2, bc=(1,) * 6)
    An = USIPG(HexMesh(Vn, Cn, Fn), k).assemble()
    assert np.max(np.abs(An @ np.ones(An.shape[0]))) <= 1e-12 * abs(An).max()
