"""GB300 (sm_103a) spike delivery for time-driven simulation of balanced
random networks of LIF neurons with alpha-shaped currents (arXiv 2109.12855).

The compute path is the CUDA library ``libsnn.so`` behind the C ABI in
``include/snn.h``; ``paper_2109_12855_gb300.snn`` is its ctypes binding.
"""


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsnn.so for sm_103a (see ``paper_2109_12855_gb300.native``)."""
    from .native import build as _build
    return _build(force=force, verbose=verbose)
