"""GB300-native explicit time step of the sharp phase-field method (SPFM).

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``);
``spfm`` is its thin ctypes binding with the C names of ``include/spfm.h``.
"""
from . import spfm  # noqa: F401
from .spfm import Grid, SpfmError  # noqa: F401
