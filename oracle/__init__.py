"""Oracle for truncated integer multiplication (Harvey, "Faster truncated integer
multiplication").

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or run anything in this
package. It shares no code, header, table or constant generator with the CUDA
library in ``paper_1703_00640_gb300/`` and never imports it.

Contents (each function cites the passage of the paper it follows):

- ``bigmul``   exact full product of uint64 limb arrays (C: schoolbook + Karatsuba)
               and the low / high products by their definitions (Section 1).
- ``trace``    exact integer trace of the method: digit splits (Algorithms 1-3,
               split step), the integer product coefficients w_i, the rounded
               coefficients 2^b L_i (Proposition 3.1) and 2^b H_i (Proposition 4.1),
               the overlap-add steps of Algorithms 2 and 3.
- ``series``   exact rational coefficients alpha_{k,r}, beta_{k,r} (Section 3.2),
               gamma_{k,r}, delta_{k,r} (Section 4.2), the auxiliary root rho
               (Lemma 4.2) and the maps alpha*, beta*, gamma-dagger, delta-dagger
               (Sections 3.3 and 4.3) in exact arithmetic for small N.
- ``fp64_ref`` Algorithms 1-3 step by step in numpy float64, with numpy's FFT as
               the Convolution black box (Section 2.1).
- ``plan``     the oracle's own choice of (b, N, lambda) from the FP64 error bound,
               with the convolution's error (eta_conv) derived for the arithmetic of
               the FFT kernels (Section 2.1's Convolution step).
- ``tft``      the truncated-FFT question at the end of Section 2.2 as an
               experiment: Algorithm 2 with a length-N cyclic product (any N) and
               with the product at the points of a truncated FFT, and the ring maps
               from R[X]/A(X) to both.
- ``division`` the reciprocal floor((2^(2k) - 1) / m) and floor division by
               definition, plus binary long division as a cross-check (Section 1
               names Barrett's reduction as an application of the high product).

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (the convolution bound also by
``tests/test_fft_error_bound.py``); none is "parity unpinned".
"""
