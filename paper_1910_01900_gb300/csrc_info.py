"""Facts about the compiled kernels that callers may want to check."""


def default_cells_per_block(n):
    """Cells per thread block of the DG passes for n points per direction (about 256 threads)."""
    return {2: 64, 3: 28, 4: 16, 5: 10, 6: 7, 7: 5, 8: 4, 9: 3}[n]


def tile_candidates(n):
    """The cells-per-block variants compiled for n (the autotuner picks among them)."""
    d = default_cells_per_block(n)
    return sorted({d, (d + 1) // 2, 2 * d, 1})
