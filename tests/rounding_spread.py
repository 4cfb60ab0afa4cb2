"""The rounding floor of an oracle run, for the full-run parity bounds.

Two probes of how far a run amplifies rounding, both on the oracle alone:
the same run from the input times (1 +- 1e-16) (random signs), and the same
run in the oracle build whose final sums are added in the opposite order
(oracle.rounding_variant("reversed")).  The full-run bound of the GPU parity
tests is max(1e-10, 4 x the larger spread): where both roundings of the
oracle itself end more than 1e-10 apart, the 1e-10 bar is below what any FP64
implementation can meet (tests/test_oracle_rounding.py shows the cases).
"""
import numpy as np

import oracle


def spread(run, U0, rel):
    """run(U) -> final state of an oracle run from U; rel(a, b) -> error."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    base = run(U0)
    rng = np.random.default_rng(1)
    pert = run(U0 * (1 + 1e-16 * rng.choice([-1.0, 1.0], size=U0.shape)))
    with oracle.rounding_variant("reversed"):
        rev = run(U0)
    return max(rel(pert, base), rel(rev, base))


def run_bound(run, U0, rel, floor=1e-10):
    return max(floor, 4.0 * spread(run, U0, rel))
