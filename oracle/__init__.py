"""FP64 CPU oracle for the batched fiber-network RVE solve.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` (including ``bench.py --impl reference``) may import,
call or run it.  It shares no code, headers, constants or helpers with the
CUDA path; both consume the seeded inputs of ``rvegen``.

What it computes (Sec. 2 and Sec. 3.2 of the paper): for each RVE and
macroscale deformation gradient F, the static equilibrium of the truss
network with boundary nodes pinned to x = F X (affine BC, Eq. affine-bc),
i.e. the state the dynamic-relaxation loop of Algorithm 2 converges to
(residual -> 0), followed by the volume-averaged Cauchy stress of the fiber
virial (the identity after Eq. hill-mandel).  The route is the one the
paper calls the implicit method (Sec. 3.2): load-incremented Newton-Raphson
with a sparse direct solve, here in plain double precision with the steps
written out in the paper's order; see ``newton.py``.

Pins (tests/test_oracle_*.py): closed forms for a single fiber, the affine
regular lattice and rigid rotations; invariants (symmetry, objectivity,
Hill-Mandel boundary virial, translation, pruning); brute force with
scipy.optimize on 1-3 free nodes; finite-difference checks of force vs
energy and tangent vs force; the linear-elastic limit against an
independent linear solve.  The paper prints no numeric worked example, so
no value here is pinned to a printed number.
"""
from .fiber_law import axial_force, axial_stiffness, fiber_energy
from .network import convergence_threshold, prune, reference_force_scale
from .newton import Solution, solve
from .tangent import dsigma_dF
from .mandel import mandel_tangent
from .orientation import orientation_tensor, p2

__all__ = ["axial_force", "axial_stiffness", "fiber_energy", "prune",
           "reference_force_scale", "convergence_threshold", "Solution", "solve", "dsigma_dF", "mandel_tangent", "orientation_tensor", "p2"]
