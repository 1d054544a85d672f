"""FP64 CPU oracle of the cascaded central-moment lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow restatement of the method of
Premnath & Banerjee, "Inertial frame independent forcing for discrete velocity Boltzmann
equation" (arXiv:1202.6074), written in float64 with plain PyTorch CPU tensor operations.
Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The CUDA library never calls it and shares no code
with it; the product path fails loudly when the CUDA library is missing.

Modules
  lattice    velocity sets, rest weights, monomial orders, orthogonal basis K (Sec. 2)
  moments    raw and central moments, binomial frame shift, exact inverse (Secs. 7, 9)
  collision  hydrodynamics, source central moments, attractors, relaxation (Secs. 4-10)
  literal    the element-wise D2Q9 collision exactly as printed (Secs. 9-11)
  les        Smagorinsky eddy viscosity from the non-equilibrium stress (paper silent)
  stream     pull streaming, periodic and half-way bounce-back walls, initial state
  solver     the time loop, diagnostics and the configurations
  adjoint    gradient of a velocity loss w.r.t. the force field (torch.autograd)

Parity status: every function here is pinned by a ``-m "not gpu"`` test against values
or identities the paper prints, closed forms, or exact invariants, except where a
function's docstring says "parity unpinned".
"""
from . import lattice, moments, collision, literal, les, stream, solver  # noqa: F401
