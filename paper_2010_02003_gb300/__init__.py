"""GB300-native DG2 flood solver (slope-decoupled DG2 of Ayog et al., Sec. 2.1).

The compute path is the C-ABI library ``libdg2.so`` (hand-written CUDA for
sm_103a, declared in ``include/dg2.h``); :mod:`.binding` marshals arguments to
it.  Importing this package does not load the library; the first call into
:mod:`.binding` does, and raises if it has not been built.
"""

__all__ = ["binding", "inputs", "build"]
