"""Tolerances of the GPU-vs-oracle parity tests, with their derivation.

Counts (joint, marginal, N) are compared bit-exactly.  MI: the epilogue sums
T(c) = c log2 c per shift in 64-bit fixed point (units of 2^-24), exactly and
in any order, with T(c) = c * L(c), L(c) = e 2^24 + round(log2(m) 2^24) for
c = m 2^e (m in [1, 2)) and log2(m) from the hardware lg2 approximation.  With
eps = max over every count c <= 2^22 of |L(c) 2^-24 - log2 c|, the MI of a shift
(Eq. finalentropy: joint, both marginal families and N each sum to N) is off by
at most 4 eps.  TERM_EPS is the bound asserted on eps by the exhaustive test
(test_gpu_entropy_term.py); MI_TOL = 4 TERM_EPS rounded up is the MI tolerance.
"""
TERM_EPS = 2.0 ** -22 + 2.0 ** -25   # documented lg2 error on [1, 2) plus the 2^-25 grid rounding
MI_TOL = 1.1e-6                      # >= 4 * TERM_EPS = 1.07e-6
