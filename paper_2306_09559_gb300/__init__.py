"""GB300-native hot path of Multipolynomial Monte Carlo (arXiv:2306.09559).

The compute path is the C-ABI library ``libmpmc.so`` (hand-written CUDA for
sm_103a, declared in ``include/mpmc.h``); :mod:`.mpmc` is its thin ctypes
binding.  Importing this package is cheap: the library is only loaded when
:func:`paper_2306_09559_gb300.mpmc.lib` is first called, and that call
raises if the library has not been built.
"""

__all__ = ["synth", "configs"]
