"""FP64 CPU oracle for covariance-free EM (CoFEM) sparse Bayesian learning.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the paper's method, used to check the CUDA path.
Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
it; the library itself never does, and it shares no code with the CUDA path.

Modules and the passages they follow:
  philox     Philox4x64-10 (Salmon et al., SC'11) and the Rademacher probe rule
             (Alg. 1, "draw p_1..p_K").
  operators  Phi / Phi^T for dense and causal-convolution dictionaries
             (Sec. V-A "Dictionary", Sec. VI-A) and A V (Sec. III).
  em         classic EM with explicit covariance (Sec. II-B, Eqs. estep-params,
             mstep), the Woodbury/IRLS E-step (Sec. II-C, Eq. woodbury, beta
             restored), the log marginal likelihood (Eq. mle2), the rectified
             Gaussian prior's M-step and multi-task EM (Sec. III extensions).
  cofem      Alg. 1 (CovarianceFreeEM) with Alg. 2 (ParallelConjGradient) and
             the diagonal preconditioner (Sec. III-C); the diagonal estimation
             rule (Prop. 1, Eq. diag-estimate); multi-task CoFEM.

Every function is pinned by tests/test_oracle_*.py against something other
than itself (numpy's Philox, brute-force enumeration, closed forms, the two
independent EM routes, CG convergence theory).  No function here is marked
"parity unpinned".
"""
from .philox import philox4x64_10, probe_bits, rademacher_probes  # noqa: F401
from .operators import DenseOperator, ToeplitzOperator, DCTOperator, make_operator, apply_A  # noqa: F401
from .em import (estep_explicit, estep_woodbury, log_marginal_likelihood,  # noqa: F401
                 mstep, em, em_multitask, second_moment)
from .cofem import (cofem, cofem_multitask, pcg, diag_estimate, diag_estimate_general,  # noqa: F401
                    FLAG_CG_NOT_CONVERGED, FLAG_ALPHA_CLAMPED, FLAG_BREAKDOWN)
