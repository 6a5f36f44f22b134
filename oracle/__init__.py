"""CPU FP64 oracle for the Kerdock fast sparsifying transform (arXiv 2105.05879).

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test
suite (``tests/``), ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or execute it.  The CUDA
library never calls it and shares no code, tables or constants with it: every
function here is written again, slowly and plainly, from the paper.

Modules
-------
field    GF(2^(k-1)) arithmetic, the field trace, the maps L_s and the Kerdock
         matrices M_s of Prop. 5, quadratic forms Q_M (Sec. 3).
kerdock  The real mutually unbiased bases u_{M,w} (Eq. "definition of
         vectors"), the sample vectors s_l = sqrt(d) Pi u_l of Algorithm 1, and
         the representation {A s_l} computed two ways: by its definition and by
         the sign-flip + fast Walsh-Hadamard route of Lemma 6.
query    The streaming step of Algorithm 1: sampling (SplitMix64 counter
         hash), coefficients s_l^T x, median of means (Theorem 3), top-S,
         exact refinement A_S x and the eps-hard threshold h_eps (Sec. 1.1),
         plus the dense truth h_eps(Ax).

Everything is float64 (numpy) or exact Python integers.  Parity pins: each
function is checked in ``tests/test_oracle_*.py`` against facts the paper and
mathematics fix (Prop. 1, 2, 4, 5, Lemma 2, Lemma 6, Theorem 3, closed forms
and brute force on tiny inputs).  No function here is "parity unpinned".
"""
