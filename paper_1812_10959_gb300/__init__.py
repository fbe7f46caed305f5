"""GB300-native (sm_103a) Dynamic Itemset Counting: the hot path of
ParallelDIC (Zymbler, Algorithms 2-5) as hand-written CUDA kernels behind the
C ABI of include/dic.h, with a thin ctypes binding (:mod:`.dic`).

The binding is imported on first use of any exported name, so that the build
module (``paper_1812_10959_gb300.build``) can be imported before libdic.so
exists; using the binding without the library raises ImportError."""
import importlib

_EXPORTS = ("Database", "DicError", "MineJob", "Result", "Server", "load_db", "load_db_csr",
            "load_db_device", "mine", "mine_async", "mine_batch", "minsup_count", "rules")
__all__ = list(_EXPORTS) + ["dic"]


def __getattr__(name):
    if name in _EXPORTS or name == "dic":
        mod = importlib.import_module(__name__ + ".dic")
        return mod if name == "dic" else getattr(mod, name)
    raise AttributeError(name)
