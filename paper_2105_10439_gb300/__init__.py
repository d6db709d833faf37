"""GB300 (sm_103a) hot path of covariance-free EM (CoFEM) for sparse Bayesian
learning, behind the C ABI of include/cofem.h (libcofem.so).

Importing the package loads libcofem.so and raises ImportError if it has not
been built; there is no CPU fallback.
"""
from .binding import *  # noqa: F401,F403
from .binding import CoFEM, CofemError, LIB_PATH, lib  # noqa: F401
