"""Seeded synthetic transaction databases, shared by the oracle side and the
CUDA side of the tests and the benchmark.

The paper evaluates on a synthetic IBM-Quest database (20M) and a real voltage
log (Tornado20M), Section 5.1 / Table 1; neither is available here, so these
planted-pattern recipes stand in for them. The module draws random rows only:
it returns CSR item lists (``row_ptr`` uint64[n+1], ``items`` uint32[nnz], rows
sorted and duplicate-free) and holds none of the mining arithmetic (no bit
packing, counting or lattice logic).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into _synth.so next to it (gcc, no FP contraction so
    the same seed gives the same rows on every host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, u32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        pu64 = ctypes.POINTER(u64)
        ppu32 = ctypes.POINTER(ctypes.POINTER(u32))
        lib.synth_planted.argtypes = [u64, u64, u32, u32, dbl, dbl, dbl, dbl, dbl, pu64, ppu32,
                                      pu64]
        lib.synth_planted.restype = ctypes.c_int
        lib.synth_dense.argtypes = [u64, u64, u32, dbl, dbl, dbl, u32, dbl, dbl, dbl, pu64, ppu32,
                                    pu64, ctypes.POINTER(dbl)]
        lib.synth_dense.restype = ctypes.c_int
        lib.synth_uniform.argtypes = [u64, u64, u64]
        lib.synth_uniform.restype = dbl
        lib.synth_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Database:
    """A transaction database as CSR item lists plus its mining parameters."""
    name: str
    n: int
    m: int
    row_ptr: np.ndarray          # uint64[n+1]
    items: np.ndarray            # uint32[nnz]
    minsup: int                  # integer support threshold (count)
    M: int                       # DIC block length
    params: dict = field(default_factory=dict)

    def rows(self):
        rp, it = self.row_ptr, self.items
        return [it[rp[t]:rp[t + 1]] for t in range(self.n)]

    def dense(self) -> np.ndarray:
        """0/1 uint8 matrix n x m (for small databases only)."""
        d = np.zeros((self.n, self.m), dtype=np.uint8)
        lens = np.diff(self.row_ptr).astype(np.int64)
        r = np.repeat(np.arange(self.n), lens)
        d[r, self.items.astype(np.int64)] = 1
        return d


def _take(ptr, nnz) -> np.ndarray:
    lib = _load()
    if nnz == 0:
        lib.synth_free(ctypes.cast(ptr, ctypes.c_void_p))
        return np.zeros(0, dtype=np.uint32)
    arr = np.ctypeslib.as_array(ptr, shape=(nnz,)).copy()
    lib.synth_free(ctypes.cast(ptr, ctypes.c_void_p))
    return arr


def planted(seed: int, n: int, m: int, n_patterns: int, pat_len_mean: float, tx_len_mean: float,
            carry: float = 0.5, keep_p: float = 0.5, noise_frac: float = 0.1):
    """Planted-pattern rows: a pool of n_patterns patterns (length
    Poisson(pat_len_mean) >= 1, floor(carry*len) items carried over from the
    previous pattern, weights Exp(1) normalised); each row has a
    Poisson(tx_len_mean) target length, Binomial(target, noise_frac) uniform
    noise items, and is then filled by weighted pattern draws keeping each
    item with probability keep_p. Returns (row_ptr, items)."""
    lib = _load()
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    out = ctypes.POINTER(ctypes.c_uint32)()
    nnz = ctypes.c_uint64(0)
    rc = lib.synth_planted(seed, n, m, n_patterns, pat_len_mean, carry, tx_len_mean, keep_p,
                           noise_frac, row_ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                           ctypes.byref(out), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"synth_planted failed ({rc})")
    return row_ptr, _take(out, nnz.value)


def dense(seed: int, n: int, m: int, zipf_s: float, noise_mean: float, cap: float,
          n_patterns: int, pat_len_mean: float, draws_mean: float, keep_p: float):
    """Dense rows: independent items with Zipf(zipf_s) popularity over a
    seeded random rank, each capped at `cap` and scaled to noise_mean items
    per row, plus Poisson(draws_mean) pattern draws (keep_p per item).
    Returns (row_ptr, items, q) with q the per-item noise probability."""
    lib = _load()
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    q = np.zeros(m, dtype=np.float64)
    out = ctypes.POINTER(ctypes.c_uint32)()
    nnz = ctypes.c_uint64(0)
    rc = lib.synth_dense(seed, n, m, zipf_s, noise_mean, cap, n_patterns, pat_len_mean,
                         draws_mean, keep_p,
                         row_ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                         ctypes.byref(out), ctypes.byref(nnz),
                         q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError(f"synth_dense failed ({rc})")
    return row_ptr, _take(out, nnz.value), q


def uniform(seed: int, stream: int, i: int) -> float:
    """The i-th value in [0,1) of a seeded stream (platform-independent)."""
    return _load().synth_uniform(seed, stream, i)


def minsup_count(n: int, frac: float) -> int:
    """Support fraction -> integer count ceil(frac*n), at least 1."""
    return max(1, int(math.ceil(frac * n - 1e-9)))


# ------------------------------------------------------------------ recipes
def planted_small(seed: int = 0) -> Database:
    """n=10,000, m=100, 200 patterns of Poisson(4) length, rows Poisson(10),
    minsup 2% (200), M=1,000."""
    n, m = 10_000, 100
    rp, it = planted(seed, n, m, 200, 4.0, 10.0)
    return Database("planted-small n=1e4 m=100", n, m, rp, it, 200, 1_000,
                    dict(seed=seed, n_patterns=200, pat_len=4, tx_len=10))


def planted_paper_scale(seed: int = 1, n: int = 1_000_000) -> Database:
    """n=1,000,000, m=1,000 (16 words per row), 2,000 patterns of mean
    length 6, rows of mean length 20, minsup 0.25% (2,500), M=10,000."""
    m = 1_000
    rp, it = planted(seed, n, m, 2_000, 6.0, 20.0)
    return Database(f"planted-paper-scale n={n} m=1000", n, m, rp, it, minsup_count(n, 0.0025),
                    min(10_000, max(1, n)), dict(seed=seed, n_patterns=2000, pat_len=6, tx_len=20))


def dense_zipf(seed: int = 2, n: int = 200_000) -> Database:
    """n=200,000, m=4,096 (64 words per row), Zipf(1.1) item popularity
    capped at 0.4 per item (360 noise items per row on average) plus 64
    planted patterns of mean length 10 (Poisson(4) draws per row, kept with
    p=0.9): about 400 items per row (~10% density); minsup 20%, M=20,000."""
    m = 4_096
    rp, it, q = dense(seed, n, m, 1.1, 360.0, 0.4, 64, 10.0, 4.0, 0.9)
    return Database(f"dense-zipf n={n} m=4096", n, m, rp, it, minsup_count(n, 0.20),
                    min(20_000, max(1, n)), dict(seed=seed, cap=0.4, zipf=1.1, q=q))


BATCH_M_CHOICES = (64, 128, 256, 512, 1024)


def batched_params(index: int, base_seed: int = 1000, n_lo: int = 1_000, n_hi: int = 200_000):
    """(seed, n, m, mean row length, mean pattern length, minsup fraction) of
    the index-th database of the batched recipe, without drawing its rows."""
    s = base_seed + index
    u = [uniform(s, 0, k) for k in range(5)]
    n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
    m = BATCH_M_CHOICES[min(4, int(u[1] * 5))]
    tx_len = min(5.0 + 35.0 * u[2], m / 16.0)
    pat_len = 2.0 + 6.0 * u[3]
    frac = 0.005 + 0.045 * u[4]
    return s, n, m, tx_len, pat_len, frac


def batched_db(index: int, base_seed: int = 1000, n_lo: int = 1_000, n_hi: int = 200_000) -> Database:
    """The index-th database of the batched recipe: n log-uniform in
    [n_lo, n_hi], m uniform from {64,...,1024}, mean row length U(5,40)
    capped at m/16 (rows at most 6.25% dense, so that two independent items
    are not frequent together even at 0.5% support; uncapped, a 64-item
    database with 40-item rows has ~10^11 frequent itemsets), mean pattern
    length U(2,8), pool of 2m patterns, minsup U(0.5%,5%) of n, M = n/10."""
    s, n, m, tx_len, pat_len, frac = batched_params(index, base_seed, n_lo, n_hi)
    rp, it = planted(s, n, m, 2 * m, pat_len, tx_len)
    return Database(f"batched#{index} n={n} m={m}", n, m, rp, it, minsup_count(n, frac),
                    max(1, n // 10), dict(seed=s, tx_len=tx_len, pat_len=pat_len, frac=frac))


def served_queries(n_queries: int, n_dbs: int, rate: float = 200.0, seed: int = 7000):
    """Poisson arrivals at `rate` req/s; each query: db id uniform in
    [0,n_dbs), minsup fraction log-uniform in [0.2%, 5%], block choice
    uniform from {n/20, n/10, n/4}. Returns a list of dicts."""
    t = 0.0
    out = []
    for i in range(n_queries):
        t += -math.log(1.0 - uniform(seed, 10, i)) / rate
        db = min(n_dbs - 1, int(uniform(seed, 11, i) * n_dbs))
        frac = math.exp(math.log(0.002) + uniform(seed, 12, i) * (math.log(0.05) - math.log(0.002)))
        mdiv = (20, 10, 4)[min(2, int(uniform(seed, 13, i) * 3))]
        out.append(dict(t=t, db=db, frac=frac, mdiv=mdiv))
    return out
