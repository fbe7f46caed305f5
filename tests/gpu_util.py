"""Shared helpers of the GPU parity tests (no mining arithmetic here)."""
import numpy as np


def trace_tests(trace, m, n):
    tr = trace.astype(np.int64)
    return m * n + int((tr[:, 4] * (tr[:, 3] - tr[:, 2])).sum()) if len(tr) else m * n


def packbits_rows(row_ptr, items, n, m):
    """Bit rows with numpy's packbits (little bit order), independent of both
    the oracle's and the library's packers."""
    W = (m + 63) // 64
    dense = np.zeros((n, W * 64), dtype=np.uint8)
    lens = np.diff(row_ptr).astype(np.int64)
    dense[np.repeat(np.arange(n), lens), items.astype(np.int64)] = 1
    return np.packbits(dense, axis=1, bitorder="little").view("<u8").reshape(n, W)
