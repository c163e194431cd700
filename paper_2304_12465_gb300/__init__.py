"""GB300 (sm_103a) library for RPCholesky-preconditioned CG and KRILL in kernel
ridge regression ("Robust, randomized preconditioning for kernel ridge
regression", Diaz, Epperly, Frangella, Tropp, Webber).

The compute path is hand-written CUDA behind the C ABI of include/krr.h; this
package is a thin ctypes binding with the same call names.  There is no CPU
implementation: without the built library (and a GPU) every call fails.
"""
from .api import (  # noqa: F401
    Factor,
    KrillPreconditioner,
    KrrServer,
    krill_build,
    krill_solve,
    krr_kmatvec,
    krr_kmatvec_batched,
    krr_launch_count,
    krr_pcg_solve,
    krr_pcg_solve_batched,
    krr_predict,
    krr_pivoted_cholesky,
    krr_precond_apply,
    krr_rpc_sample,
    krr_rpcholesky,
    krr_server_footprint,
    krr_autotune_choice,
    krr_set_autotune,
    krr_set_pcg_graphs,
    krr_check_bounded_wait,
    krr_set_product_path,
    krr_set_product_variant,
    krr_autotune_variant,
    krr_set_profiling,
    krr_profile_collect,
    krr_sparse_sign,
    krr_version,
)
from ._native import KrrError, KrrInfo, SIGNATURES, load, library_path  # noqa: F401
