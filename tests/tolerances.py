"""Tolerances of the GPU-vs-oracle parity tests, with their derivation.

Counts (joint, marginal, N) are compared bit-exactly.  MI: the epilogue sums
T(c) = c log2 c per shift in 64-bit fixed point (units of 2^-23), exactly and
in any order, with T(c) = c * L(c), L(c) = e 2^23 + round(log2(m) 2^23) for
c = m 2^e (m in [1, 2)) and log2(m) from the hardware lg2 approximation.  With
eps = max over every count c <= 2^22 of |L(c) 2^-23 - log2 c|, the MI of a shift
(Eq. finalentropy: joint, both marginal families and N each sum to N) is off by
at most 4 eps.  The exhaustive test (test_gpu_entropy_term.py) measures eps over
every count a map can hold on GB300: 2.075e-7 (= 2^-22.20, at c = 2219005), and
asserts eps <= TERM_EPS; 4 TERM_EPS = 8.4e-7 is within MI_TOL = 1e-6, the
tolerance of an FP64 entropy reduction.
"""
TERM_EPS = 2.1e-7
MI_TOL = 1e-6
