"""GB300-native penalised Cox / Fine-Gray cyclic coordinate descent.

The computation lives in ``libsurvgpu.so`` (CUDA, sm_103a; C ABI in
``include/survgpu.h``).  ``binding`` marshals arrays to it; ``synth`` builds
seeded synthetic cohorts.  Importing this package does not load the library;
the first call does, and raises if it is missing.
"""
from .binding import (SurvData, SurvError, Workspace, cox_fit, cox_nll, fg_fit, load,  # noqa: F401
                      loglik_grad_hess, surv_groups, surv_sort_desc)

__all__ = ["SurvData", "SurvError", "Workspace", "cox_fit", "cox_nll", "fg_fit", "load", "loglik_grad_hess",
           "surv_groups", "surv_sort_desc"]
