"""libqscatter: GB300 (sm_103a) beam phase-space integration of QScatter
(Amaro & Vranic, arXiv 2308.09348).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/qscatter.h``); :mod:`.binding` marshals arguments to it and
:mod:`.inputs` draws seeded synthetic beams.
"""
from . import inputs  # noqa: F401
from .binding import (MOMENT_FIELDS, Outputs, QsError, lib, qs_eval_samples,  # noqa: F401
                      qs_scatter, workspace_bytes)

__all__ = ["inputs", "MOMENT_FIELDS", "Outputs", "QsError", "lib", "qs_eval_samples",
           "qs_scatter", "workspace_bytes"]
