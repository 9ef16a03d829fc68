"""FP64 CPU oracle for coil-sketched iterative MR reconstruction (Oscanoa et al.,
"Coil Sketching for computationally-efficient MR iterative reconstruction").

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of
what the method computes, written in NumPy/SciPy with complex128/float64 throughout.  It is
imported only by the test-suite, by the smoke check in ``__graft_entry__`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product library never
imports, links or calls it, and it shares no code with the CUDA sources.

Modules
-------
fourier   Cartesian SENSE operator (Sec. 2.1, Eq. 1-2, A = U F C) and a dense brute-force A.
nufft     Kaiser-Bessel gridding NUFFT with density compensation (Sec. 2.1, A = W^1/2 F C,
          Eq. 5), plus the exact non-uniform DFT it approximates.
binning   Grid coordinates, kernel boxes and the stable counting sort of samples to tiles.
coils     Coil PCA (SVD-based coil compression, Sec. 3.1 and Alg. 1), structured sketch
          (Sec. 2.3, S^t = S~^t (x) I_N with the virtual-coil block form) and sketched maps.
philox    Philox4x32-10 counter-based generator and the sketch entry distributions (Sec. 3.2).
wavelet   Periodised orthonormal Daubechies-4 (db4, 8 taps) multi-level DWT (Sec. 2.1, l1-wavelets).
tv        Periodic first-order differences and the dual projection of l1-TV (Sec. 2.1).
gfactor   Inverse g-factor by Monte Carlo pseudo-replicas and in closed form for SENSE (Sec. 3.2).
solvers   CG, FISTA, PDHG, power iteration, the sketched sub-problem (Eq. 9-10) and Algorithm 1.
fftlib    The DFT library calls (scipy.fft with a thread count, else numpy.fft).

Parity pins live in ``tests/test_oracle_*.py``: each function here is checked against
something other than itself (dense matrices built from Eq. 1, closed forms, invariants,
brute force on tiny inputs, published known-answer vectors).
"""
