"""CPU oracle for the Lippmann-Schwinger HBS solver (Gopal & Martinsson, arXiv 2007.12718).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2007_12718_gb300/csrc``) and never consumes
a value produced there.

Everything is plain FP64 numpy / scipy, written to be checked against the
paper by eye:

* ``lattice``  -- lattice zeta constants and the corrected-quadrature weights
                  (Sec. 2.2, Eq. (8), Fig. 1).  The paper does not print the
                  weights; the reading used is stated in that module.
* ``kernel``   -- G(x,y) = (i/4) H0(kappa |x-y|)  (Eq. (2)).
* ``nystrom``  -- dense corrected Nystrom matrix (Eqs. (9)-(10)), dense LU
                  solve, FFT convolution matvec (Sec. 2.2 / Sec. 5),
                  fields at receivers (Eq. (1)).
* ``gmres``    -- right-preconditioned GMRES (Sec. 5).
* ``hbs``      -- HBS compression with proxy sources and CPQR row IDs
                  (Sec. 3.2, Eqs. (12)-(15)), Algorithm 1 (build) and
                  Algorithm 2 (apply) of Sec. 4.1.
* ``disk``     -- closed-form Bessel-series solution for a constant-b disk
                  (the Helmholtz form Eq. (4)), used only as a pin.

Parity status per function is stated in each module header.
"""
