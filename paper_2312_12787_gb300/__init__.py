"""GB300-native Burton-Miller collocation BEM for 2D Helmholtz transmission problems.

The compute path is libbem.so (hand-written CUDA for sm_103a, C interface in include/bem.h); this
package holds its sources (csrc/), the in-tree build (build.py) and the ctypes binding (bem.py).
"""
from .bem import (  # noqa: F401
    Batch, BemError, Problem, bem_last_error, bem_test_set_fused_iteration, bem_test_set_wait_limit,
    bem_version, load, make_opts,
    BEM_OK, BEM_EINVAL, BEM_ENOMEM, BEM_ENOCONV, BEM_ETIMEOUT, BEM_ECUDA, BEM_ESTATE,
    BEM_FORM_MOD, BEM_FORM_ORIG, BEM_FORM_BETA1, BEM_FORM_CONV,
    BEM_PREC_FP64, BEM_PREC_MIXED, BEM_PREC_MIXED_TC, EXPORTS,
)
