"""GB300-native exact k-clique counting (arb-count) on a low out-degree orientation.

The public API lives in :mod:`paper_2002_10047_gb300.kclique` (imported lazily so
that the input generators in :mod:`paper_2002_10047_gb300.graphgen` can be used
without the CUDA library).
"""

__all__ = ["kclique", "graphgen"]


def __getattr__(name):
    if name in ("kclique", "graphgen"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
