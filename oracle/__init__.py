"""CPU oracle for Galerkin FFT homogenization with stress and mixed control
(Lucarini & Segurado, arXiv:1901.06531).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the method, written to check the CUDA library against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library never calls it and has no CPU fallback through it.  It shares
no code with the CUDA path: its transform is the discrete Fourier transform
written out by its definition (one dense twiddle matrix per axis), its
projector, constitutive laws and Newton/CG loop are written here from the
paper's equations.

Modules
  dft        -- Eq. (eql_discrete2): the DFT pair F / F^-1 (forward 1/N)
  projector  -- Eq. (eq:G), (eq:Gnew), (eq:Gnewnew): the operator G-hat-star
  materials  -- P(F) and K = dP/dF (Eq. eq:lineariz) for the neo-Hookean and
                St Venant-Kirchhoff (cubic, rotated) laws
  solver     -- Eq. (linequil2ast) and (eq:mixedeqil): Newton + conjugate
                gradients under per-component stress/strain control
  dense      -- dense assembly of the linear operator for brute-force checks
  adjoint    -- adjoint sensitivity of the homogenized response (one CG solve
                with the projected tangent at a converged step)

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(naive DFT sums and library FFT, the projector's algebra and the reference
medium Green operator, energy finite differences, affine and laminate closed
forms, dense solves, central finite differences of full solves for the
adjoint).  None is "parity unpinned".
"""
from . import dft, projector, materials, solver, dense, adjoint  # noqa: F401
