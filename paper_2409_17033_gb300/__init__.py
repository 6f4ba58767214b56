"""GB300 (sm_103a) implementation of the SP2 density-matrix, response and
dual-susceptibility path of arXiv 2409.17033, behind the C ABI of
include/sp2.h (libsp2.so, built from csrc/ by build.py).

The Python layer only marshals arguments; the library must be built, and
there is no CPU fallback.
"""
from .api import (Handle, SP2Error, make_opts, mlp_forward, mlp_loss_grad, mlp_train,
                  response_contract, sp2_adjoint, sp2_density, sp2_fermi,
                  sp2_nonorth_susceptibility, sp2_response, sp2_scf_response, sp2_susceptibility,
                  synchronize)
from .autograd import SP2Density, sp2_density_autograd

__all__ = ["Handle", "SP2Error", "make_opts", "sp2_density", "sp2_response",
           "sp2_susceptibility", "sp2_adjoint", "sp2_fermi", "sp2_nonorth_susceptibility",
           "sp2_scf_response", "mlp_forward",
           "mlp_loss_grad", "mlp_train", "response_contract", "SP2Density",
           "sp2_density_autograd", "synchronize"]
