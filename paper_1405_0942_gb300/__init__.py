"""GB300-native (sm_103a) Lagrangian magneto-frictional relaxation with the
mimetic current (Candelaresi, Pontin & Hornig).

The compute path is the CUDA library ``libglemur.so`` behind the C ABI of
``include/glemur.h``; :mod:`.glemur` is its argument-marshalling binding.
"""
from .glemur import (DIRECT, FP64, MIMETIC, MIXED, GlemurError, Relaxation,  # noqa: F401
                     default_opts, lib, lib_path, workspace_bytes)
