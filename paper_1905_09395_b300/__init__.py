"""B300-native STEV: stabilized explicit, variable-load integration of stiff
chemical source terms (Buchheit et al., arXiv:1905.09395) behind a C ABI
(include/stev.h) with hand-written sm_103a CUDA kernels.

    from paper_1905_09395_b300 import Mechanism, synth
    mech_tables, T, P, Y, dt = synth.small_case()
    m = Mechanism(mech_tables)              # stev_mechanism_create
    T_out, Y_out, iters, status = m.solve(T_dev, P_dev, Y_dev, dt)   # stev_solve
"""
from .binding import (CELL_MAXITER, CELL_NONFINITE, CELL_OK, CELL_TRANGE, EXPORTS, FP64, MIXED,
                      THERMO_MLP, THERMO_MLP_CPH, THERMO_POLY, Mechanism, Options, Server, StevError,
                      default_options,
                      lib)

__all__ = ["Mechanism", "Server", "Options", "StevError", "default_options", "lib", "EXPORTS", "FP64",
           "MIXED", "THERMO_POLY", "THERMO_MLP", "THERMO_MLP_CPH", "CELL_OK", "CELL_MAXITER", "CELL_NONFINITE",
           "CELL_TRANGE"]
