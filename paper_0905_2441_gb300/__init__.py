"""GB300 (sm_103a) library for the data-parallel hot path of population-based
MCMC and SMC samplers, after Lee, Yau, Giles, Doucet & Holmes (2009), "On the
utility of graphics cards to perform massively parallel simulation of
advanced Monte Carlo methods".

The compute lives in libsmc.so (hand-written CUDA, C ABI in include/smc.h);
this package binds it for torch CUDA tensors and drives the samplers.
Importing the package loads nothing; the first call loads libsmc.so and
fails loudly if it is missing -- there is no CPU path.
"""
from ._lib import (GMM_1D, GMM_DIAG, MOVE_MALA, MOVE_RW, OP_LOGLIK, OP_MOVE, OP_POPMCMC, PF_LG,
                   PF_FSV, PF_MSV, PREC_BF16SPLIT, PREC_FP32, RNG_ACCEPT, RNG_EXCHANGE, RNG_MOVE,
                   RNG_MULTINOMIAL, RNG_PFNOISE, RNG_PROPOSAL, RNG_RESAMPLE)

__all__ = ["GMM_1D", "GMM_DIAG", "MOVE_MALA", "MOVE_RW", "OP_LOGLIK", "OP_MOVE", "OP_POPMCMC",
           "PF_FSV", "PF_LG", "PF_MSV", "PREC_BF16SPLIT", "PREC_FP32", "RNG_ACCEPT", "RNG_EXCHANGE",
           "RNG_MOVE", "RNG_MULTINOMIAL", "RNG_PFNOISE", "RNG_PROPOSAL", "RNG_RESAMPLE"]


def __getattr__(name):
    # the torch-facing binding is imported on first use
    import importlib
    if name.startswith("__"):
        raise AttributeError(name)
    api = importlib.import_module(__name__ + ".api")
    if hasattr(api, name):
        return getattr(api, name)
    raise AttributeError(name)
