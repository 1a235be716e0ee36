"""GB300-native Fast Folding Algorithm period search (Cameron et al. 2017).

The search (detrend, per-octave downsampling, FFA fold, Algorithm 1 boxcar
scoring, candidate reduction) runs in hand-written sm_103a CUDA kernels behind
a C ABI (``include/ffa.h``).  ``paper_1703_05581_gb300.ffa`` is the thin ctypes
binding; ``paper_1703_05581_gb300.synth`` draws seeded synthetic inputs.
Submodules are imported on first use so that the input generator works on a
machine without the CUDA library.
"""
import importlib

__all__ = ["ffa", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
