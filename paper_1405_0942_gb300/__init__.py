"""GB300-native (sm_103a) Lagrangian magneto-frictional relaxation with the
mimetic current (Candelaresi, Pontin & Hornig).

The compute path is the CUDA library ``libglemur.so`` behind the C ABI of
``include/glemur.h``; :mod:`.glemur` is its argument-marshalling binding.
"""
from .glemur import (DIRECT, FP64, LOSS_ENERGY, LOSS_XI, MIMETIC, MIXED, NNN,  # noqa: F401
                     GlemurError, Relaxation, RelaxationFieldLoss, RelaxationLoss,
                     default_opts, forward_checkpoints, lib, lib_path, loss_and_field_gradient,
                     param_contract, relax_with_schedule, reverse_sweep, workspace_bytes)
