"""FP64 CPU oracle for the NNEinFact multiplicative update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_2602_02759_gb300``), and
the product never imports it.

Contents:
  * ``oracle.core``  -- plain C loop nests (``nef_oracle.c``) behind ctypes:
    reconstruction (Eq. 2.1), einsum(einstr_l) numerator/denominator
    (Eq. 3.6-3.8), the update (Eq. 3.4), D_{alpha,beta} and g (App. B),
    Algorithm 1, and a sampled num/den for large-size parity checks; the same
    steps under the likelihood losses of App. B (negative binomial, binomial /
    Bernoulli on odds, Jensen-Shannon).
  * ``oracle.mlp``   -- FP64 forward/backward of the fold-in encoder MLP.

Parity pins (what checks this oracle against something other than itself)
live in ``tests/test_oracle_pins.py`` and ``tests/test_oracle_lik_pins.py``.
"""
from .core import (  # noqa: F401
    OracleModel,
    build,
    divergence,
    ginv,
    eta_of,
    lik_divergence,
    num_threads,
    set_num_threads,
)
