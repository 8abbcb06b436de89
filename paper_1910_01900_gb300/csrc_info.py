"""Facts about the compiled kernels that callers may want to check."""

# shared-memory values per cell of the cell kernels (four tile arrays with
# their bank-spreading pitches), per points per direction n = 2..9
CELL_VALUES = {2: 36, 3: 123, 4: 304, 5: 509, 6: 964, 7: 1457, 8: 2304, 9: 2929}


def default_cells_per_block(n):
    """Cells per thread block of the cell kernels for n points per direction (about 256 threads)."""
    return {2: 64, 3: 28, 4: 16, 5: 10, 6: 7, 7: 5, 8: 4, 9: 3}[n]


def max_cells_per_block(n, elem_bytes):
    """Widest block of a cell kernel: 768 threads (n^2 per cell) and 227 KB of shared
    memory (CELL_VALUES[n] values per cell)."""
    return min(768 // (n * n), 232448 // (CELL_VALUES[n] * elem_bytes))
