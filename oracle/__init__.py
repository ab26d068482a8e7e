"""Plain, slow, single-threaded FP64 CPU oracle for the MujicΛ hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
C-ABI and the Python binding in ``paper_2604_26823_gb300``) imports, links or
calls anything here.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

What it computes (paper: "MujicΛ: Initial Condition Reconstruction on
Realistic Redshift Surveys with Augmented Optimization"):

* ``cosmology`` -- E(a), linear growth D1, second-order growth D2, the
  FastPM-style kick/drift factors, the Eisenstein-Hu no-wiggle P(k) table
  (Sec. 2.2.1 items 1-2; the P(k) table is input data for both sides).
* ``mesh`` -- DFT conventions, spectral derivative operators, CIC paint /
  readout and their derivatives (Sec. 2.2.1 item 2, Sec. 2.2.2 "CiC").
* ``model`` -- the forward model: white noise -> linear field -> 2LPT ->
  leapfrog PM steps -> RSD -> bias -> selection -> likelihood + prior
  (Sec. 2.2.1, Eq. galaxy_bias, Sec. 2.2.2), and its hand-derived adjoint
  (the gradient with respect to the white noise s).
* ``projection`` -- the projection operator P (z-score + reset, Sec. 2.3.1)
  and rank-order matching R (Sec. 2.3.2) in real and Fourier space.
* ``lbfgs`` -- the L-BFGS two-loop recursion and the projected
  backtracking line search (Sec. 2.3.1, Appendix B Table 1).
* ``anneal`` -- the resolution transfer of the white noise and the coarse
  data of the annealed reconstruction (Sec. 3, opening).
* ``analysis`` -- binned power / cross spectra and r_c (Sec. 3.2), Gaussian
  smoothing, the T-web classification, eigenvector cosines and the confusion
  matrix (Sec. 3.3).

Parity unpinned: the shape of the Eisenstein-Hu no-wiggle transfer function
between its k->0 limit and its normalisation is not pinned by any printed
value (the paper prints none); it is input data read identically by both
sides.  Reconstruction quality against the paper's figures is unpinned (the
paper's dataset is not available).
"""
