"""Python binding of the C ABI in include/dic.h (ctypes; argument marshalling
only). Every step of mining runs inside libdic.so on the GPU; there is no
Python or CPU fallback: importing this module fails if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdic.so")

DIC_OK, DIC_EINVAL, DIC_ENOMEM, DIC_ECUDA, DIC_ECAPACITY, DIC_ETIMEOUT, DIC_EBUSY = range(7)
PATHS = {"auto": 0, "rows": 1, "bitslice": 2, "tensor": 3}
TRACE_COLUMNS = ("step", "stop", "first", "last", "dashed", "promoted", "pruned", "generated",
                 "solidified")


class DicError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dic status {status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("count_path", ctypes.c_uint32),
                ("steps_per_sync", ctypes.c_uint32), ("use_graph", ctypes.c_uint32),
                ("profile", ctypes.c_uint32), ("max_candidates", ctypes.c_uint32),
                ("profile_every", ctypes.c_uint32), ("tile_words", ctypes.c_uint32),
                ("count_form", ctypes.c_uint32), ("algorithm", ctypes.c_uint32),
                ("prestage", ctypes.c_uint32), ("solo_rows", ctypes.c_uint32),
                ("stop_loop", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 3)]


class Stats(ctypes.Structure):
    _fields_ = [("tests", ctypes.c_uint64), ("stops", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("frequent", ctypes.c_uint64),
                ("l1", ctypes.c_uint32), ("words", ctypes.c_uint32),
                ("words_compact", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32),
                ("count_ms", ctypes.c_double), ("count_launches", ctypes.c_uint64),
                ("firstpass_ms", ctypes.c_double), ("mine_ms", ctypes.c_double),
                ("path_launches", ctypes.c_uint32 * 4), ("count_ops", ctypes.c_uint64),
                ("gram_ms", ctypes.c_double), ("gram_launches", ctypes.c_uint64),
                ("settle_ms", ctypes.c_double), ("gen_ms", ctypes.c_double),
                ("gen_launches", ctypes.c_uint64), ("gram_flops", ctypes.c_uint64),
                ("count_ops_timed", ctypes.c_uint64), ("setup_ms", ctypes.c_double),
                ("graph_ms", ctypes.c_double), ("collect_ms", ctypes.c_double),
                ("event_loop", ctypes.c_uint32), ("event_iters", ctypes.c_uint32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("reserved", "path_launches")}
        d["path_launches"] = list(self.path_launches)
        return d


class ServerMetrics(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("peak_slots", ctypes.c_uint32),
                ("reserved0", ctypes.c_uint32), ("peak_bytes", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("qps", ctypes.c_double),
                ("solo", ctypes.c_uint64), ("reserved", ctypes.c_uint32 * 6)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdic.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    pvp = ctypes.POINTER(vp)
    sig = {
        "dic_load_db": ([vp, u64, u32, pvp], i32),
        "dic_load_db_csr": ([vp, vp, u64, u32, pvp], i32),
        "dic_load_db_device": ([vp, u64, u32, vp, pvp], i32),
        "dic_db_free": ([vp], i32),
        "dic_db_rows": ([vp], u64),
        "dic_db_items": ([vp], u32),
        "dic_db_device_words": ([vp], vp),
        "dic_options_init": ([ctypes.POINTER(Options)], None),
        "dic_mine": ([vp, u32, u64, pvp], i32),
        "dic_mine_ex": ([vp, u32, u64, ctypes.POINTER(Options), vp, pvp], i32),
        "dic_mine_batch": ([vp, vp, vp, u32, ctypes.POINTER(Options), vp], i32),
        "dic_mine_async": ([vp, u32, u64, ctypes.POINTER(Options), vp, pvp], i32),
        "dic_mine_wait": ([vp, ctypes.c_int64, pvp], i32),
        "dic_result_count": ([vp], u64),
        "dic_result_words": ([vp], u32),
        "dic_result_copy": ([vp, vp, vp, vp], i32),
        "dic_result_trace_len": ([vp], u64),
        "dic_result_trace": ([vp, vp], i32),
        "dic_result_stats": ([vp, ctypes.POINTER(Stats)], i32),
        "dic_result_free": ([vp], None),
        "dic_minsup_count": ([u64, ctypes.c_double], u32),
        "dic_status_str": ([i32], ctypes.c_char_p),
        "dic_last_error": ([], ctypes.c_char_p),
        "dic_abi_version": ([], u32),
        "dic_server_create": ([u64, u32, ctypes.POINTER(Options), pvp], i32),
        "dic_server_submit": ([vp, vp, u32, u64, ctypes.POINTER(u64)], i32),
        "dic_server_wait": ([vp, u64, ctypes.c_int64, pvp], i32),
        "dic_server_stats": ([vp, ctypes.POINTER(ServerMetrics)], i32),
        "dic_server_destroy": ([vp], i32),
        "dic_rules_from_itemsets": ([vp, vp, vp, u64, u32, u32, u32, pvp], i32),
        "dic_rules_count": ([vp], u64),
        "dic_rules_copy": ([vp, vp, vp, vp, vp], i32),
        "dic_rules_free": ([vp], None),
        "dic_measure_alu_peak": ([ctypes.POINTER(ctypes.c_double)], i32),
        "dic_debug_fail_device_alloc": ([ctypes.c_int64], i32),
        "dic_debug_pool_used": ([ctypes.POINTER(u64)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc: int):
    if rc != DIC_OK:
        raise DicError(rc, (_lib.dic_last_error() or b"").decode())


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Database:
    """A device-resident transaction database (dic_db)."""

    def __init__(self, handle: int, n: int, m: int):
        self._h = ctypes.c_void_p(handle)
        self.n, self.m = n, m
        self.W = (m + 63) // 64

    @property
    def handle(self):
        return self._h

    def device_words_ptr(self) -> int:
        return _lib.dic_db_device_words(self._h) or 0

    def free(self):
        if self._h:
            _check(_lib.dic_db_free(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                _lib.dic_db_free(self._h)
        except Exception:
            pass


def load_db(words, n: int, m: int) -> Database:
    """Host bitmaps uint64 [n, ceil(m/64)] (numpy or pinned torch CPU tensor)."""
    if isinstance(words, np.ndarray):
        words = np.ascontiguousarray(words, dtype=np.uint64)
    h = ctypes.c_void_p()
    _check(_lib.dic_load_db(_ptr(words) if n else None, n, m, ctypes.byref(h)))
    return Database(h.value, n, m)


def load_db_csr(row_ptr, items, n: int, m: int) -> Database:
    """Host CSR item lists (row_ptr uint64[n+1], items uint32[nnz])."""
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    if isinstance(items, np.ndarray):
        items = np.ascontiguousarray(items, dtype=np.uint32)
        if items.size == 0:
            items = np.zeros(1, dtype=np.uint32)
    h = ctypes.c_void_p()
    _check(_lib.dic_load_db_csr(_ptr(row_ptr), _ptr(items), n, m, ctypes.byref(h)))
    return Database(h.value, n, m)


def load_db_device(words_tensor, n: int, m: int, stream=None) -> Database:
    """Device bitmaps (e.g. a CUDA torch int64 tensor [n, W]); copied."""
    h = ctypes.c_void_p()
    _check(_lib.dic_load_db_device(words_tensor.data_ptr() if n else None, n, m,
                                   _stream_handle(stream), ctypes.byref(h)))
    return Database(h.value, n, m)


@dataclass
class Result:
    W: int
    masks: np.ndarray     # uint64 [count, W]
    k: np.ndarray         # uint32 [count]
    support: np.ndarray   # uint32 [count]
    trace: np.ndarray     # uint64 [stops, 9]
    stats: dict

    def itemsets(self):
        """[(tuple(items), support)] in canonical order."""
        out = []
        for q in range(len(self.k)):
            its = []
            for w in range(self.W):
                x = int(self.masks[q, w])
                while x:
                    b = (x & -x).bit_length() - 1
                    its.append(w * 64 + b)
                    x &= x - 1
            out.append((tuple(its), int(self.support[q])))
        return out


def _result(h) -> Result:
    cnt = _lib.dic_result_count(h)
    W = _lib.dic_result_words(h)
    masks = np.zeros((max(cnt, 1), max(W, 1)), dtype=np.uint64)
    k = np.zeros(max(cnt, 1), dtype=np.uint32)
    sp = np.zeros(max(cnt, 1), dtype=np.uint32)
    _check(_lib.dic_result_copy(h, masks.ctypes.data, k.ctypes.data, sp.ctypes.data))
    tl = _lib.dic_result_trace_len(h)
    tr = np.zeros((max(tl, 1), len(TRACE_COLUMNS)), dtype=np.uint64)
    _check(_lib.dic_result_trace(h, tr.ctypes.data))
    st = Stats()
    _check(_lib.dic_result_stats(h, ctypes.byref(st)))
    _lib.dic_result_free(h)
    return Result(W, masks[:cnt], k[:cnt], sp[:cnt], tr[:tl], st.as_dict())


PROFILE_BITS = {"count": 1, "gram": 2, "settle": 4, "gen": 8}
PROFILE_ALL = 15


def profile_mask(profile) -> int:
    """True -> every kind; False/None -> none; an int is the DIC_PROFILE_*
    bitmask; a name or list of names from PROFILE_BITS selects kinds."""
    if profile is True:
        return PROFILE_ALL
    if not profile:
        return 0
    if isinstance(profile, int):
        return profile & PROFILE_ALL
    if isinstance(profile, str):
        profile = [profile]
    return sum(PROFILE_BITS[k] for k in set(profile))


COUNT_FORMS = {"auto": 0, "tiled": 1, "direct": 2}
ALGORITHMS = {"paralleldic": 0, "classic": 1}


PRESTAGE = {"auto": 0, "off": 1}
STOP_LOOPS = {"auto": 0, "events": 1, "per-stop": 2}


def options(path: str = "auto", steps_per_sync: int = 0, use_graph: bool = True,
            profile=False, max_candidates: int = 0, profile_every: int = 0,
            tile_words: int = 0, count_form: str = "auto",
            algorithm: str = "paralleldic", prestage: str = "auto",
            stop_loop: str = "auto") -> Options:
    o = Options()
    _lib.dic_options_init(ctypes.byref(o))
    o.count_path = PATHS[path]
    o.steps_per_sync = steps_per_sync
    o.use_graph = 1 if use_graph else 0
    o.profile = profile_mask(profile)
    o.profile_every = profile_every
    o.tile_words = tile_words
    o.count_form = COUNT_FORMS[count_form]
    o.algorithm = ALGORITHMS[algorithm]
    o.prestage = PRESTAGE[prestage]
    o.stop_loop = STOP_LOOPS[stop_loop]
    o.max_candidates = max_candidates
    return o


def mine(db: Database, minsup: int, M: int, path: str = "auto", stream=None,
         profile=False, steps_per_sync: int = 0, use_graph: bool = True,
         max_candidates: int = 0, profile_every: int = 0, tile_words: int = 0,
         count_form: str = "auto", algorithm: str = "paralleldic",
         prestage: str = "auto", stop_loop: str = "auto") -> Result:
    """All itemsets with support >= minsup (integer count), blocks of M rows.
    algorithm: "paralleldic" (Algorithm 2, first pass then pairs) or
    "classic" (Algorithm 1, every 1-itemset a dashed circle). prestage:
    "auto" (stage every block's columns, and count the pair cohort over the
    whole pass, before the loop when they fit) or "off" (per stop).
    stop_loop: "auto" (per stop, handing over to the event-driven form once
    promotions have stopped), "events" (event-driven where it applies: each
    cohort counted over its whole pass when born, only stops with promotions
    generate) or "per-stop" (every dashed itemset counted at every stop)."""
    o = options(path, steps_per_sync, use_graph, profile, max_candidates, profile_every,
                tile_words, count_form, algorithm, prestage, stop_loop)
    h = ctypes.c_void_p()
    _check(_lib.dic_mine_ex(db.handle, minsup, M, ctypes.byref(o), _stream_handle(stream),
                            ctypes.byref(h)))
    return _result(h)


class MineJob:
    """A mine running on the library's worker thread (dic_mine_async)."""

    def __init__(self, handle, db):
        self._h = handle
        self._db = db  # kept alive while the job runs

    def wait(self, timeout_ms: int = -1) -> Result:
        """The result; DicError(DIC_ETIMEOUT) if not finished in time (the
        job can be waited again)."""
        if not self._h:
            raise DicError(DIC_EINVAL, "job already waited")
        h = ctypes.c_void_p()
        rc = _lib.dic_mine_wait(self._h, timeout_ms, ctypes.byref(h))
        if rc == DIC_ETIMEOUT:
            _check(rc)
        self._h = None
        _check(rc)
        return _result(h)

    def __del__(self):
        try:
            if self._h:
                h = ctypes.c_void_p()
                if _lib.dic_mine_wait(self._h, -1, ctypes.byref(h)) == DIC_OK:
                    _lib.dic_result_free(h)
        except Exception:
            pass


def mine_async(db: Database, minsup: int, M: int, stream=None, **kw) -> MineJob:
    """Start a mine on the library's worker thread (dic_mine_async); the
    keyword arguments are those of mine()."""
    o = options(**kw)
    h = ctypes.c_void_p()
    _check(_lib.dic_mine_async(db.handle, minsup, M, ctypes.byref(o), _stream_handle(stream),
                               ctypes.byref(h)))
    return MineJob(h, db)


def mine_batch(dbs, minsups, Ms, path: str = "auto", profile=False, tile_words: int = 0,
               algorithm: str = "paralleldic"):
    """Mine several (db, minsup, M) queries together; returns a list of Result
    (ParallelDIC only: the library rejects algorithm="classic" here)."""
    cnt = len(dbs)
    handles = (ctypes.c_void_p * max(cnt, 1))(*[d.handle.value for d in dbs])
    ms = np.ascontiguousarray(minsups, dtype=np.uint32)
    Ms_ = np.ascontiguousarray(Ms, dtype=np.uint64)
    outs = (ctypes.c_void_p * max(cnt, 1))()
    o = options(path, profile=profile, tile_words=tile_words, algorithm=algorithm)
    _check(_lib.dic_mine_batch(ctypes.cast(handles, ctypes.c_void_p), ms.ctypes.data,
                               Ms_.ctypes.data, cnt, ctypes.byref(o),
                               ctypes.cast(outs, ctypes.c_void_p)))
    return [_result(ctypes.c_void_p(outs[i])) for i in range(cnt)]


def _items_of(mask_row) -> tuple:
    return tuple(int(w * 64 + b) for w, x in enumerate(mask_row) for b in range(64)
                 if (int(x) >> b) & 1)


def rules(res: Result, conf_num: int, conf_den: int, m: int | None = None) -> list:
    """Association rules X -> Z \\ X of the mined itemsets with confidence
    supp(Z) / supp(X) >= conf_num / conf_den (exact), evaluated on the GPU.
    Returns [(X, Z \\ X, supp(Z), supp(X))] in canonical order."""
    W = res.W
    masks = np.ascontiguousarray(res.masks, dtype=np.uint64).reshape(-1)
    k = np.ascontiguousarray(res.k, dtype=np.uint32)
    sp = np.ascontiguousarray(res.support, dtype=np.uint32)
    cnt = len(k)
    h = ctypes.c_void_p()
    _check(_lib.dic_rules_from_itemsets(masks.ctypes.data if cnt else None,
                                        k.ctypes.data if cnt else None,
                                        sp.ctypes.data if cnt else None, cnt,
                                        m if m is not None else W * 64, conf_num, conf_den,
                                        ctypes.byref(h)))
    try:
        nr = _lib.dic_rules_count(h)
        ante = np.zeros((max(nr, 1), W), dtype=np.uint64)
        cons = np.zeros((max(nr, 1), W), dtype=np.uint64)
        sz = np.zeros(max(nr, 1), dtype=np.uint32)
        sx = np.zeros(max(nr, 1), dtype=np.uint32)
        _check(_lib.dic_rules_copy(h, ante.ctypes.data, cons.ctypes.data, sz.ctypes.data,
                                   sx.ctypes.data))
    finally:
        _lib.dic_rules_free(h)
    return [(_items_of(ante[i]), _items_of(cons[i]), int(sz[i]), int(sx[i])) for i in range(nr)]


def measure_alu_peak() -> float:
    """Measured integer-ALU (lop3) issue rate of the current device, Top/s."""
    v = ctypes.c_double(0.0)
    _check(_lib.dic_measure_alu_peak(ctypes.byref(v)))
    return v.value


def debug_fail_device_alloc(after: int):
    """Test support: the calling thread's allocation number `after` (0-based)
    of the next mining calls fails as out of memory; -1 cancels."""
    _check(_lib.dic_debug_fail_device_alloc(after))


def debug_pool_used() -> int:
    """Test support: bytes in use in the device's stream-ordered pool."""
    v = ctypes.c_uint64(0)
    _check(_lib.dic_debug_pool_used(ctypes.byref(v)))
    return v.value


def minsup_count(n: int, frac: float) -> int:
    return _lib.dic_minsup_count(n, frac)


class Server:
    """Continuous-batching request server (dic_server_*): submit queries from
    any thread, wait for their results by ticket."""

    def __init__(self, hbm_budget_bytes: int = 120 << 30, max_slots: int = 64,
                 path: str = "auto", steps_per_sync: int = 0, solo_rows: int = 0):
        """solo_rows: queries on databases of at least this many rows are mined
        alone by the single-query path (0 = the library's default, 2^19)."""
        o = options(path, steps_per_sync)
        o.solo_rows = solo_rows
        h = ctypes.c_void_p()
        _check(_lib.dic_server_create(hbm_budget_bytes, max_slots, ctypes.byref(o),
                                      ctypes.byref(h)))
        self._h = h

    def submit(self, db: Database, minsup: int, M: int) -> int:
        t = ctypes.c_uint64()
        _check(_lib.dic_server_submit(self._h, db.handle, minsup, M, ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> Result:
        h = ctypes.c_void_p()
        _check(_lib.dic_server_wait(self._h, ticket, timeout_ms, ctypes.byref(h)))
        return _result(h)

    def stats(self) -> dict:
        m = ServerMetrics()
        _check(_lib.dic_server_stats(self._h, ctypes.byref(m)))
        return m.as_dict()

    def close(self):
        if self._h:
            _check(_lib.dic_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                _lib.dic_server_destroy(self._h)
        except Exception:
            pass
