"""Plain FP64 CPU oracle for the Basic Scheme on anisotropic patterns.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
link this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` use it.  It shares no code with the CUDA path.

Everything here follows Bergmann & Merkert, "FFT-based homogenization on
periodic anisotropic translation invariant spaces" (arXiv 1701.04685):

* ``lattice``    -- pattern P(M), generating set G(M^T), pattern DFT (Sec. 2.1,
                    Eqs. (Fouriermatrix), (FourierTransform)); an independent
                    Smith-normal-form index map used by the fast variant.
* ``material``   -- Mandel layout of Sym_d / SSym_d (Sec. 3.1) and isotropic
                    stiffness tensors.
* ``generators`` -- Fourier symbols of the Dirichlet kernel, the de la Vallee
                    Poussin means and the periodised box splines (Sec. 2.2,
                    Def. dlVP) and the orthonormalised alias weights
                    (Lemma FI:Props (iii)).
* ``green``      -- Green operator Gamma^0 (Def. projection, Eq. (gamma)) and the
                    periodised Green operator Gamma^p (Def.
                    gamma_tilde_fourier).
* ``scheme``     -- fixed-point iteration on Eq. (pde_coefficients), Cauchy
                    residual (Sec. 4) and the effective stiffness (Sec. 3.1).

* ``krylov``     -- conjugate gradients (Dirichlet, Galerkin form), GMRES and
                    BiCGStab on the same discrete equation as ``scheme`` (Krylov
                    solvers that the paper cites; not its iteration).
* ``fno``        -- forward pass and loss of the learned start (a Fourier
                    neural operator; not part of the paper's method); the GPU
                    gradients are checked against central finite differences
                    of this loss.

Parity status: every function is pinned by ``tests/test_oracle_*.py``.  The
reference-medium rule (``material.reference_medium_ms``) is a reading, since
the paper never states C0: it is pinned to its defining property (phase
spectra of C0^-1 C centred on 1) and the contraction bound that follows.
"""
