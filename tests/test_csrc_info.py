"""csrc_info's block-width tables agree with the constants the kernels are compiled with.

csrc_info.py restates two functions of csrc/sumfac.cuh for callers in Python
(default and largest cells per thread block); this reads the header as text and
checks that both give the same numbers for every tile size n = 2..9.
"""
import os
import re

from paper_1910_01900_gb300 import csrc_info

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1910_01900_gb300", "csrc",
                   "sumfac.cuh")


def _header():
    return open(HDR).read()


def test_default_cells_per_block_matches_header():
    src = _header()
    body = re.search(r"constexpr int default_cb\(int n\)\s*\{\s*return (.*?);\s*\}", src, re.S).group(1)
    pairs = dict((int(a), int(b)) for a, b in re.findall(r"n == (\d) \? (\d+)", body))
    last = int(re.search(r":\s*(\d+)\s*$", body.strip()).group(1))
    for n in range(2, 10):
        assert csrc_info.default_cells_per_block(n) == pairs.get(n, last), n


def test_max_cells_per_block_matches_header():
    src = _header()
    threads = int(re.search(r"constexpr int kCellThreads = (\d+);", src).group(1))
    smem = int(re.search(r"\((\d+) / \(cell_values\(n\) \* elem_bytes\)\)", src).group(1))
    body = re.search(r"constexpr int cell_values\(int n\)\s*\{\s*return (.*?);\s*\}", src, re.S).group(1)
    pairs = dict((int(a), int(b)) for a, b in re.findall(r"n == (\d) \? (\d+)", body))
    last = int(re.search(r":\s*(\d+)\s*$", body.strip()).group(1))
    for n in range(2, 10):
        cv = pairs.get(n, last)
        assert csrc_info.CELL_VALUES[n] == cv, n
        for eb in (4, 8):
            want = min(threads // (n * n), smem // (cv * eb))
            assert csrc_info.max_cells_per_block(n, eb) == want, (n, eb)
