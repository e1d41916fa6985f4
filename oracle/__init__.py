"""FP64 CPU oracle for the factorized stochastic three-point method (arXiv:1711.02384).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path (the seeded input generator is the one module
both sides use, and it holds none of the method's arithmetic).

Every function is the plain definition written out in complex128 numpy:

* ``gamma``       -- Euclidean Dirac matrices (chiral and Dirac-Pauli bases)
* ``momenta``     -- momentum sets p = 2*pi*k/L and the Fourier phases (Sec. 3, Eqs. 9-10)
* ``contractions``-- spectator part (Eq. 9), insertion part (Eq. 10), the baryon
                     spectator (our reading; the paper gives no formula) and the
                     noise-averaged combine (Eqs. 5 and 8)
* ``direct``      -- brute-force trace of Eq. 1 (and its baryon analogue) over all
                     sink/insertion site pairs, for tiny lattices
* ``freefield``   -- free (unit-link) Wilson propagator in closed form, the hopping
                     stencil, and random SU(3) gauge transformations

Pins (tests marked ``not gpu``) tie each function to something other than itself:
full spin-colour-site dilution equals the direct trace; k = 0 equals the site sum;
all L^3 momenta equal numpy's FFT; translation covariance; the free-field
propagator solves the Wilson equation and obeys gamma5-hermiticity; the free-field
correlator equals an independent momentum-space (convolution) evaluation; the
baryon colour factor and gauge invariance; the count of 93 momenta with k^2 <= 8.
"""
