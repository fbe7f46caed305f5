"""CPU oracle for DIC frequent-itemset mining -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package. The product path (``paper_1812_10959_gb300``) never
imports, links or runs anything here, and shares no code with it.

Every function wraps a plain serial routine of ``dic_oracle.cpp``:
  * :func:`dic`          ParallelDIC, Algorithm 2 with Algorithms 3-5 (serial)
  * :func:`dic_classic`  serial DIC of Algorithm 1 (no first pass)
  * :func:`apriori`      level-wise Apriori, Section 3
  * :func:`bruteforce`   all subsets by sub-mask enumeration (m <= 24)
  * :func:`support`      support of given itemsets by tid-list intersection
  * :func:`pair_supports` co-occurrence counts of every item pair
  * :func:`pack`         BitMask of Section 4.1
  * :func:`rules`        association rules from frequent itemsets (Section 1's
                         second subtask), plain Python loops
  * :func:`paralleldic`  the paper's own parallel design on the host cores
                         (``paralleldic_omp.cpp``, OpenMP): the benchmark's
                         multi-core CPU baseline, pinned to :func:`dic`
Results are lists of ``(items_tuple, support)`` in canonical order (size, then
lexicographic), plus a per-stop trace for the DIC forms.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, textbook reductions, hand-worked example).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dic_oracle.cpp")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None
_PSRC = os.path.join(_HERE, "paralleldic_omp.cpp")
_PLIB = os.path.join(_HERE, "_paralleldic.so")
_plib = None

TRACE_COLUMNS = ("step", "stop", "first", "last", "dashed", "promoted", "pruned", "generated",
                 "solidified")


def build(force: bool = False) -> str:
    """Compile dic_oracle.cpp into _oracle.so (g++, plain -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def build_paralleldic(force: bool = False) -> str:
    """Compile paralleldic_omp.cpp into _paralleldic.so (g++ -O3 -fopenmp)."""
    if force or not os.path.exists(_PLIB) or os.path.getmtime(_PLIB) < os.path.getmtime(_PSRC):
        tmp = _PLIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _PSRC,
                               "-o", tmp])
        os.replace(tmp, _PLIB)
    return _PLIB


_REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                              ctypes.c_uint64)


def _pload():
    global _plib
    if _plib is None:
        lib = ctypes.CDLL(build_paralleldic())
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.pdic_mine.argtypes = [vp, vp, u64, u32, u32, u64, u64, ctypes.c_int,
                                  ctypes.POINTER(vp)]
        lib.pdic_mine.restype = ctypes.c_int
        lib.pdic_mine_sharded.argtypes = [vp, vp, u64, u32, u32, u64, u64, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, _REDUCE_FN, vp,
                                          ctypes.POINTER(vp)]
        lib.pdic_mine_sharded.restype = ctypes.c_int
        for name in ("pdic_result_count", "pdic_result_nitems", "pdic_result_trace_len",
                     "pdic_result_tests"):
            f = getattr(lib, name)
            f.argtypes = [vp]
            f.restype = u64
        lib.pdic_result_threads.argtypes = [vp]
        lib.pdic_result_threads.restype = ctypes.c_int
        lib.pdic_result_copy.argtypes = [vp, vp, vp, vp]
        lib.pdic_result_trace.argtypes = [vp, vp]
        lib.pdic_result_free.argtypes = [vp]
        _plib = lib
    return _plib


def paralleldic(row_ptr, items, n: int, m: int, minsup: int, M: int, max_stops: int = 0,
                threads: int = 0):
    """ParallelDIC with OpenMP on `threads` host threads (0 = all): Algorithm
    2 with the loop interchange and nested balancing of Algorithm 3 (Figures
    2-3), the same readings as :func:`dic`. Returns (OracleResult, threads)."""
    lib = _pload()
    rp, it = _csr(row_ptr, items)
    h = ctypes.c_void_p()
    if lib.pdic_mine(rp.ctypes.data, it.ctypes.data, n, m, minsup, M, max_stops, threads,
                     ctypes.byref(h)) != 0:
        raise ValueError("paralleldic: invalid arguments")
    return _presult(lib, h)


def paralleldic_sharded(row_ptr, items, n: int, m: int, minsup: int, M: int, rank: int,
                        world: int, reduce, max_stops: int = 0, threads: int = 0):
    """Transaction-sharded ParallelDIC (the data-distributed scheme of the
    paper's related work): this rank counts its share of every block and
    `reduce(counts)` must sum the uint64 numpy array `counts` across the
    ranks in place (called for the first pass and once per stop). Every rank
    returns the single-rank result and trace. Returns (OracleResult, threads)."""
    lib = _pload()
    rp, it = _csr(row_ptr, items)

    def cb(_ctx, ptr, length):
        try:
            reduce(np.ctypeslib.as_array(ptr, shape=(int(length),)))
            return 0
        except Exception:  # noqa: BLE001 (reported to the C side as a failure)
            return 1

    fn = _REDUCE_FN(cb)
    h = ctypes.c_void_p()
    rc = lib.pdic_mine_sharded(rp.ctypes.data, it.ctypes.data, n, m, minsup, M, max_stops,
                               threads, rank, world, fn, None, ctypes.byref(h))
    if rc == -2:
        raise RuntimeError("paralleldic_sharded: the counter reduction failed")
    if rc != 0:
        raise ValueError("paralleldic_sharded: invalid arguments")
    return _presult(lib, h)


def _presult(lib, h):
    cnt = lib.pdic_result_count(h)
    nit = lib.pdic_result_nitems(h)
    k = np.zeros(max(cnt, 1), dtype=np.uint32)
    items_out = np.zeros(max(nit, 1), dtype=np.uint32)
    sp = np.zeros(max(cnt, 1), dtype=np.uint64)
    lib.pdic_result_copy(h, k.ctypes.data, items_out.ctypes.data, sp.ctypes.data)
    out, p = [], 0
    for i in range(cnt):
        out.append((tuple(int(x) for x in items_out[p:p + k[i]]), int(sp[i])))
        p += int(k[i])
    tl = lib.pdic_result_trace_len(h)
    tr = np.zeros((max(tl, 1), len(TRACE_COLUMNS)), dtype=np.uint64)
    lib.pdic_result_trace(h, tr.ctypes.data)
    res = OracleResult(out, tr[:tl], int(lib.pdic_result_tests(h)), 0)
    used = int(lib.pdic_result_threads(h))
    lib.pdic_result_free(h)
    return res, used


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, u32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        pres = ctypes.POINTER(vp)
        for name in ("oracle_dic", "oracle_dic_classic"):
            f = getattr(lib, name)
            f.argtypes = [vp, vp, u64, u32, u32, u64, u64, ctypes.c_int, pres]
            f.restype = ctypes.c_int
        for name in ("oracle_apriori", "oracle_bruteforce"):
            f = getattr(lib, name)
            f.argtypes = [vp, vp, u64, u32, u32, pres]
            f.restype = ctypes.c_int
        lib.oracle_pack.argtypes = [vp, vp, u64, u32, vp]
        lib.oracle_support.argtypes = [vp, vp, u64, u32, vp, vp, u64, vp]
        lib.oracle_support.restype = ctypes.c_int
        lib.oracle_pair_supports.argtypes = [vp, vp, u64, u32, vp]
        for name in ("oracle_result_count", "oracle_result_nitems", "oracle_result_trace_len",
                     "oracle_result_tests", "oracle_result_violations"):
            f = getattr(lib, name)
            f.argtypes = [vp]
            f.restype = u64
        lib.oracle_trace_cols.restype = u32
        lib.oracle_result_copy.argtypes = [vp, vp, vp, vp]
        lib.oracle_result_trace.argtypes = [vp, vp]
        lib.oracle_result_free.argtypes = [vp]
        _lib = lib
    return _lib


@dataclass
class OracleResult:
    itemsets: list            # [(tuple(items), support)] canonical order
    trace: np.ndarray         # uint64 [stops, 9] (DIC forms); Apriori: per level
    tests: int                # candidate-transaction tests performed
    violations: int           # reading violations (must be 0)

    def as_dict(self):
        return {s: v for s, v in self.itemsets}


def _csr(row_ptr, items):
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    it = np.ascontiguousarray(items, dtype=np.uint32)
    if it.size == 0:
        it = np.zeros(1, dtype=np.uint32)
    return rp, it


def _result(handle) -> OracleResult:
    lib = _load()
    cnt = lib.oracle_result_count(handle)
    nit = lib.oracle_result_nitems(handle)
    k = np.zeros(max(cnt, 1), dtype=np.uint32)
    it = np.zeros(max(nit, 1), dtype=np.uint32)
    sp = np.zeros(max(cnt, 1), dtype=np.uint64)
    lib.oracle_result_copy(handle, k.ctypes.data, it.ctypes.data, sp.ctypes.data)
    out, p = [], 0
    for i in range(cnt):
        out.append((tuple(int(x) for x in it[p:p + k[i]]), int(sp[i])))
        p += int(k[i])
    tl = lib.oracle_result_trace_len(handle)
    tr = np.zeros((max(tl, 1), lib.oracle_trace_cols()), dtype=np.uint64)
    lib.oracle_result_trace(handle, tr.ctypes.data)
    res = OracleResult(out, tr[:tl], int(lib.oracle_result_tests(handle)),
                       int(lib.oracle_result_violations(handle)))
    lib.oracle_result_free(handle)
    return res


def _run(name, row_ptr, items, n, m, *args) -> OracleResult:
    lib = _load()
    rp, it = _csr(row_ptr, items)
    h = ctypes.c_void_p()
    rc = getattr(lib, name)(rp.ctypes.data, it.ctypes.data, n, m, *args, ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments (rc={rc})")
    return _result(h)


def dic(row_ptr, items, n: int, m: int, minsup: int, M: int, max_stops: int = 0,
        superset_loop: bool = True) -> OracleResult:
    """ParallelDIC (Algorithm 2): first pass, then COUNT / PRUNE /
    MAKECANDIDATES / CHECKFULLPASS per block of M rows with rewind.
    max_stops > 0 ends after that many stops (timing samples only);
    superset_loop=False skips Algorithm 4's superset loop (quadratic; the
    pinned runs show it never changes anything)."""
    return _run("oracle_dic", row_ptr, items, n, m, minsup, M, max_stops, int(superset_loop))


def dic_classic(row_ptr, items, n: int, m: int, minsup: int, M: int,
                max_stops: int = 0, superset_loop: bool = True) -> OracleResult:
    """Serial DIC of Algorithm 1 (every 1-itemset starts as a dashed circle)."""
    return _run("oracle_dic_classic", row_ptr, items, n, m, minsup, M, max_stops,
                int(superset_loop))


def apriori(row_ptr, items, n: int, m: int, minsup: int) -> OracleResult:
    """Level-wise Apriori (Section 3)."""
    return _run("oracle_apriori", row_ptr, items, n, m, minsup)


def bruteforce(row_ptr, items, n: int, m: int, minsup: int) -> OracleResult:
    """Every non-empty subset with support >= minsup (m <= 24)."""
    return _run("oracle_bruteforce", row_ptr, items, n, m, minsup)


def support(row_ptr, items, n: int, m: int, itemsets) -> np.ndarray:
    """Support count of each itemset (iterable of item sequences)."""
    lib = _load()
    rp, it = _csr(row_ptr, items)
    sets = [list(s) for s in itemsets]
    off = np.zeros(len(sets) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(s) for s in sets]) if sets else []
    flat = np.array([x for s in sets for x in s] or [0], dtype=np.uint32)
    out = np.zeros(max(len(sets), 1), dtype=np.uint64)
    rc = lib.oracle_support(rp.ctypes.data, it.ctypes.data, n, m, off.ctypes.data,
                            flat.ctypes.data, len(sets), out.ctypes.data)
    if rc != 0:
        raise ValueError("item id out of range")
    return out[:len(sets)]


def pair_supports(row_ptr, items, n: int, m: int) -> np.ndarray:
    """uint32 [m, m]: rows containing both a and b (diagonal: single items)."""
    lib = _load()
    rp, it = _csr(row_ptr, items)
    out = np.zeros((m, m), dtype=np.uint32)
    lib.oracle_pair_supports(rp.ctypes.data, it.ctypes.data, n, m, out.ctypes.data)
    return out


def pack(row_ptr, items, n: int, m: int) -> np.ndarray:
    """BitMask rows, uint64 [n, ceil(m/64)]."""
    lib = _load()
    rp, it = _csr(row_ptr, items)
    W = (m + 63) // 64
    out = np.zeros((max(n, 1), W), dtype=np.uint64)
    lib.oracle_pack(rp.ctypes.data, it.ctypes.data, n, m, out.ctypes.data)
    return out[:n]


def rules(itemsets, conf_num: int, conf_den: int) -> list:
    """Association rules from frequent itemsets, the second subtask of
    Section 1 (the paper leaves its definition to its reference [1]; the
    textbook one is taken): for every frequent Z with |Z| >= 2 and every
    non-empty proper subset X of Z, the rule X -> Z \\ X holds when its
    confidence supp(Z) / supp(X) is at least conf_num / conf_den, compared
    exactly as supp(Z) * conf_den >= conf_num * supp(X).

    `itemsets` is a list of (items_tuple, support), downward closed (every
    subset of a member is a member). Returns [(X, Z \\ X, supp(Z), supp(X))]
    sorted by X (size, then items) and then by Z \\ X (size, then items).
    Plain loops: small inputs only."""
    sup = {tuple(s): int(v) for s, v in itemsets}
    out = []
    for z, sz in sup.items():
        k = len(z)
        if k < 2:
            continue
        for code in range(1, (1 << k) - 1):
            x = tuple(z[b] for b in range(k) if code >> b & 1)
            y = tuple(z[b] for b in range(k) if not code >> b & 1)
            sx = sup[x]  # KeyError: not downward closed
            if sz * conf_den >= conf_num * sx:
                out.append((x, y, sz, sx))
    out.sort(key=lambda r: (len(r[0]), r[0], len(r[1]), r[1]))
    return out
