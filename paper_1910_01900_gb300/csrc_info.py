"""Facts about the compiled kernels that callers may want to check."""


def default_cells_per_block(n):
    """Cells per thread block of the cell kernels for n points per direction (about 256 threads)."""
    return {2: 64, 3: 28, 4: 16, 5: 10, 6: 7, 7: 5, 8: 4, 9: 3}[n]


def max_cells_per_block(n, elem_bytes):
    """Widest block of a cell kernel: 768 threads (n^2 per cell) and 227 KB of shared
    memory (four tile arrays of n^2 * pitch values per cell, pitch n + 1 for even n)."""
    pitch = n + 1 if n % 2 == 0 else n
    return min(768 // (n * n), 232448 // (4 * pitch * n * n * elem_bytes))
