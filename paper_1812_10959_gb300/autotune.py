"""Autotuner for the count configuration of a mining query.

The library's AUTO choice is a rule (TENSOR pairs when there are >= 256
frequent items and blocks of >= 2,048 rows, the widest BITSLICE tile that fits
shared memory, the direct count form for small windows). The tuner instead
times the candidate configurations on the query itself, through the C ABI,
checks that every one of them returns the same itemsets, supports and per-stop
trace (the configurations change the order in which bits are combined, never
a count), and keeps the fastest per query shape (the rule itself unless
another configuration beats it by more than the timing margin). Later
queries of the same shape reuse the choice without timing anything.

Shape key: device name, n, m, minsup, M (the lattice, and so the best
configuration, depends on the data as well; queries on one database with the
same parameters share it exactly). The cache is a dict, optionally persisted
as JSON.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time
from dataclasses import dataclass, field

# (path, tile_words, count_form): tile_words 0 = widest that fits
CANDIDATES = (
    ("auto", 0, "auto"),
    ("bitslice", 16, "auto"),
    ("bitslice", 8, "auto"),
    ("bitslice", 4, "auto"),
    ("bitslice", 16, "tiled"),
    ("tensor", 16, "auto"),
    ("tensor", 8, "auto"),
    ("tensor", 16, "tiled"),
)
BATCH_CANDIDATES = (0, 16, 8, 4)  # tile_words common to a batch round


@dataclass
class Choice:
    path: str
    tile_words: int
    count_form: str
    seconds: float
    timings: list = field(default_factory=list)  # [(path, tile_words, form, seconds)]

    def kwargs(self) -> dict:
        return dict(path=self.path, tile_words=self.tile_words, count_form=self.count_form)


def _signature(res) -> tuple:
    """What every configuration must reproduce exactly."""
    return (res.masks.tobytes(), res.k.tobytes(), res.support.tobytes(), res.trace.tobytes(),
            int(res.stats["tests"]))


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:  # noqa: BLE001 (no torch or no device: key on the library alone)
        return "cuda"


class Tuner:
    """Times CANDIDATES per query shape and remembers the fastest.

    `run(kwargs) -> (signature, seconds)` may be given to time something else
    than the library (tests); by default a configuration is timed as the wall
    time of `dic.mine`, which returns with the result on the host."""

    def __init__(self, cache_path: str | None = None, repeats: int = 2, run=None,
                 margin: float = 0.03):
        self.cache_path = cache_path
        self.repeats = max(1, repeats)
        self.margin = margin  # the first candidate (the rule) is kept unless beaten by this
        self.cache: dict = {}
        self._run = run
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    @staticmethod
    def key(n: int, m: int, minsup: int, M: int, device: str | None = None) -> str:
        return f"{device or _device_name()}|n={n}|m={m}|minsup={minsup}|M={M}"

    def _save(self):
        if self.cache_path:
            tmp = self.cache_path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def _time(self, db, minsup, M, kw):
        if self._run is not None:
            return self._run(kw)
        from . import dic
        dic.mine(db, minsup, M, **kw)  # warm-up: builds the stop graphs of this shape
        secs, sig = [], None
        for _ in range(self.repeats):
            t0 = time.perf_counter()
            res = dic.mine(db, minsup, M, **kw)
            secs.append(time.perf_counter() - t0)
            sig = _signature(res)
        return sig, statistics.median(secs)

    def tune(self, db, minsup: int, M: int, candidates=CANDIDATES) -> Choice:
        k = self.key(db.n, db.m, minsup, M)
        if k in self.cache:
            c = self.cache[k]
            return Choice(c["path"], c["tile_words"], c["count_form"], c["seconds"],
                          c.get("timings", []))
        ref, timings = None, []
        for path, tw, form in candidates:
            kw = dict(path=path, tile_words=tw, count_form=form)
            sig, sec = self._time(db, minsup, M, kw)
            if ref is None:
                ref = sig
            elif sig != ref:
                raise RuntimeError(f"configuration {kw} changed the mining result")
            timings.append((path, tw, form, sec))
        best = min(timings, key=lambda t: t[3])
        if timings[0][3] <= best[3] * (1.0 + self.margin):
            best = timings[0]  # within timing noise of the rule: keep the rule
        choice = Choice(best[0], best[1], best[2], best[3], timings)
        self.cache[k] = dict(path=choice.path, tile_words=choice.tile_words,
                             count_form=choice.count_form, seconds=choice.seconds,
                             timings=timings)
        self._save()
        return choice

    def mine(self, db, minsup: int, M: int, **kw):
        """dic.mine with the tuned configuration of this query shape."""
        from . import dic
        return dic.mine(db, minsup, M, **self.tune(db, minsup, M).kwargs(), **kw)

    def tune_batch(self, dbs, minsups, Ms, candidates=BATCH_CANDIDATES) -> Choice:
        """The tile width common to a batch round, timed on the batch itself."""
        from . import dic
        shape = ";".join(f"{d.n}x{d.m}:{s}:{M}" for d, s, M in zip(dbs, minsups, Ms))
        digest = hashlib.sha256(shape.encode()).hexdigest()[:16]
        k = f"{_device_name()}|batch|{digest}|{len(dbs)}"
        if k in self.cache:
            c = self.cache[k]
            return Choice("auto", c["tile_words"], "auto", c["seconds"], c.get("timings", []))
        ref, timings = None, []
        for tw in candidates:
            dic.mine_batch(dbs, minsups, Ms, tile_words=tw)
            t0 = time.perf_counter()
            out = dic.mine_batch(dbs, minsups, Ms, tile_words=tw)
            sec = time.perf_counter() - t0
            sig = [_signature(r) for r in out]
            if ref is None:
                ref = sig
            elif sig != ref:
                raise RuntimeError(f"tile_words={tw} changed a batched mining result")
            timings.append(("auto", tw, "auto", sec))
        best = min(timings, key=lambda t: t[3])
        self.cache[k] = dict(tile_words=best[1], seconds=best[3], timings=timings)
        self._save()
        return Choice("auto", best[1], "auto", best[3], timings)
