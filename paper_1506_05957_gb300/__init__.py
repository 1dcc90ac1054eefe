"""GB300-native relaxed-p FMM-BEM (Wang, Layton & Barba, arXiv:1506.05957).

The compute path is libfmmbem.so (hand-written sm_103a CUDA behind the C ABI in
include/fmmbem.h); this package only builds and binds it.
"""
from .binding import (FmmBem, FmmBemError, FmmBemServer, fmmbem_default_opts, fmmbem_estimate_bytes,
                      fmmbem_expansion_eval, fmmbem_relaxed_p, lib, FMMBEM_LAPLACE, FMMBEM_STOKES, FMMBEM_FP64,
                      FMMBEM_MIXED, FMMBEM_MIXED_REFINED, FMMBEM_P_MAX, FMMBEM_LAYER_SINGLE, FMMBEM_LAYER_DOUBLE)

__all__ = ["FmmBem", "FmmBemError", "FmmBemServer", "fmmbem_default_opts", "fmmbem_estimate_bytes",
           "fmmbem_expansion_eval", "fmmbem_relaxed_p", "lib",
           "FMMBEM_LAPLACE", "FMMBEM_STOKES", "FMMBEM_FP64", "FMMBEM_MIXED", "FMMBEM_MIXED_REFINED", "FMMBEM_P_MAX",
           "FMMBEM_LAYER_SINGLE", "FMMBEM_LAYER_DOUBLE"]
