"""FP64 CPU oracle for the binned power-spectrum and bispectrum estimators of PolyBin3D (arXiv 2404.07249).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or execute anything in
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA path.

It is a plain, slow, obviously-correct restatement of the paper's definitions in float64, with numpy
FFTs, matrix products and LAPACK solves as the only library steps:

* ``binning``    -- k-grid, half-open shell bins, Legendre weights (Sec. 3.1, eq. xi-p-alpha-deriv;
                   Sec. 4.1, eq. Bk-Yam).
* ``ideal``      -- ideal (uniform-density, global line of sight) estimators: P_ell numerator and
                   Fisher (Sec. 3.4.1, eqs. pk-limit, fish-ideal-continuous), shell-filtered maps
                   g_b (Sec. 4.3.1, eq. g-ell-def), triplet sums and N_abc (eqs. beta-def, N-ell-def),
                   the ideal bispectrum (Sec. 4.4.1, eqs. bk-num-ideal, bk-fish-ideal2).
* ``philox``     -- Philox4x32-10 counter-based generator (Salmon et al., SC'11) + Box-Muller, used for
                   the Monte Carlo draws of the Fisher matrices (Sec. 3.3.2 and Sec. 4.3.4).
* ``unwindowed`` -- masked estimators with an FKP weighting (Sec. 2.4, eq. Sinv-fkp): P numerator and
                   Monte Carlo Fisher (Sec. 3.3, eqs. pk-num-fft, Q-alpha-global, fish-from-Q), the
                   bispectrum numerator with its linear term (Sec. 4.3.2, eq. b-numerator-practical),
                   the Q-derivatives and Monte Carlo Fisher (Sec. 4.3.4, eqs. bk-fish-def, Q-bis-global),
                   and the final F^-1 solves (eqs. pk-estimator-def, bk-estimator-def).
* ``brute``      -- brute-force closed-triangle counts and triple products in C (``brute.c``), the
                   independent pin for N_abc and S_abc.

Units.  Everything is computed in the discrete "pixel" convention (cell volume 1): integrals over
space become sums over cells, int_k becomes (1/N) sum_k, FT is numpy ``fftn`` and IFT is ``ifftn``
(with its 1/N).  Physical units follow by dV = V/N factors stated where they are applied.
"""
