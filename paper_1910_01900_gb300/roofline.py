"""Algorithmic work of the operator apply, for roofline accounting.

flops_alg follows the count of the even-odd 1D kernels (Section 4 cites the
even-odd decomposition): one sweep over n^2 lines costs
n^2 (2 (ceil(n/2)^2 + floor(n/2)^2) + 2n) flops and a cell does 12 sweeps;
each interior face, per side and per direction (evaluation and integration)
costs one normal-derivative pass n^2 * 2n plus 4 face sweeps of
n (2 (ceil^2 + floor^2) + 2n) each, about 3 faces per cell with both sides
counted; pointwise 6 flops per cell point (Cartesian) or 18 (curved) and 12 per
face point per side; curved faces add 2 tangential-derivative sweeps per side
and direction.  The evaluation pass gets the forward half, the integration
pass the backward half plus the pointwise work.

bytes_alg: read u and write v (2 words per DoF); curved cells add the stored
geometry of the paper's scheme (J^-T and JxW per cell point, n^T J^-T and the
area element per face point and side).
"""


def flops_alg(k, curved):
    """(eval, integrate) algorithmic flops per DoF of one operator apply."""
    n = k + 1
    h, hc = n // 2, (n + 1) // 2
    line = 2 * (hc * hc + h * h) + 2 * n
    sweep = n * n * line
    face_sweep = n * line
    n3 = n ** 3
    per_side = n * n * 2 * n + 4 * face_sweep + (2 * face_sweep if curved else 0)
    cell_half = 6 * sweep
    face_half = 3 * 2 * per_side
    point = (18 if curved else 6) * n3 + 3 * 2 * 12 * n * n
    return (cell_half + face_half) / n3, (cell_half + face_half + point) / n3


def bytes_alg(k, curved, word):
    """Algorithmic bytes per DoF of one apply (word = 8 for FP64, 4 for FP32)."""
    n = k + 1
    b = 2 * word
    if curved:
        b += 10 * word                                   # J^-T (9) + JxW per cell point
        b += 3 * n * n * 2 * 4 * word / n ** 3           # per face point and side: n^T J^-T (3) + dA
    return b
