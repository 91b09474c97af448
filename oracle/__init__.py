"""CPU oracle for the hard-to-round argument search of arXiv 1211.3056.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
baseline of bench.py may import this package; the CUDA library never calls
it and shares no code with it.

It is a plain, slow and exact restatement of what the hot path computes:

  fmath       exact-rational enclosures of exp, 2^x, log and their Taylor
              coefficients, correct rounding by Ziv's strategy;
  plan        output-binade segments, Taylor blocks, sub-intervals;
  poly        coefficients c_k, direct Horner for (b_i, alpha_i), search words;
  search      brute-force minimum (the definition of Eq. (1)), the
              three-distance geometry, the continued-fraction configurations,
              Algorithms 2 and 4 as lower bounds, difference tables;
  candidates  the full candidate list of a batch of jobs.

Parity pins (tests/test_oracle_*.py) tie each part to something outside
itself: the paper's printed examples (Figs. 3, 5, 6, 7 and Table 1), exact
points (2^1 = 2, exp(0) = 1, log(1) = 0), identities (exp(log x) = x,
log 2^k = k ln 2), the three-distance theorem, an independent libm
evaluation of every argument of the 24-bit toy format, and brute force.
"""
from . import fmath, plan, poly, search, candidates  # noqa: F401
