"""GB300-native (sm_103a) Dynamic Itemset Counting: the hot path of
ParallelDIC (Zymbler, Algorithms 2-5) as hand-written CUDA kernels behind the
C ABI of include/dic.h, with a thin ctypes binding (:mod:`.dic`)."""
from .dic import (Database, DicError, Result, load_db, load_db_csr, load_db_device, mine,
                  mine_batch, minsup_count)

__all__ = ["Database", "DicError", "Result", "load_db", "load_db_csr", "load_db_device", "mine",
           "mine_batch", "minsup_count"]
