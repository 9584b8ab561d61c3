"""FP64 CPU oracle for the Pulscan boxcar search (arXiv 2406.15186).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the accelerated path computes, written from the paper:

* ``fft``          -- own iterative radix-2 FFT and its adjoint (input to §2.2.2)
* ``normalise``    -- per-block median / MAD normalisation and power (§2.2.3, Eq. 8)
* ``boxcar``       -- recursive boxcar bank and per-segment maxima (§2.2.5, Algorithm 4)
* ``significance`` -- chi-square survival, Bonferroni, Gaussian sigma (§2.2.3, Eq. 9)
* ``pipeline``     -- the end-to-end search in the paper's order (width sampling, R-Block)
* ``harmonic``     -- harmonic summing by decimation and its search (§2.3)
* ``fidelity``     -- the paper's GPU approximations: median of medians (§2.5)
                      and the polynomial log p (§2.6)
* ``lse``          -- logsumexp relaxation of the segment maximum and its adjoint

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import it.  The CUDA library never does, and this package
imports nothing from the CUDA package: the two share no code.  Inputs (noise,
injected chirps) are passed in as arrays.

Every function is FP64.  Each one names the passage of the paper it follows.
"""
