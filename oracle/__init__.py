"""CPU FP64 oracle for the per-column Krylov (multiple-Arnoldi) Green's-function method.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import anything from this package. The CUDA library never calls it, and it
shares no code with the CUDA path: both consume the seeded inputs of ``workloads`` and nothing
else in common.

What it computes (Hoshi et al., arXiv 1210.1531):
  * the generalized shifted equation (zS - H) x = b with sparse real-symmetric H and positive
    definite S in an LCAO basis (Eq. 1), solved column by column, j being the parallel unit;
  * the one-body density matrix from the Fermi-Dirac energy integral of Im G (Eq. 2);
  * the chemical potential by bisection on the electron count (memory-saving workflow, Eq. 3);
  * the band energy Tr(rho H), equal to the sum of ICOHP (Eq. 6), and forces.

Modules
  slater_koster  two-centre s/p Hamiltonian and overlap blocks and their derivatives
  structure      neighbour lists, clusters and the block-sparse (BSR) pattern, brute force
  hamiltonian    dense and block-sparse H, S built from the Slater-Koster blocks
  exact          plain definitions: dense generalized diagonalisation, rho, mu, G(z) by solve
  krylov         the per-column Krylov build, projection and projected eigenproblem
  physics        Fermi function, bisection, density-matrix columns, energies, forces
  pipeline       the whole path over all (or sampled) columns of a workload
  cohp           COHP / ICOHP and their sigma / pi parts (Eqs. 4-8)

Every function names the passage of the paper (or the stated reading of it) that it follows.
"""
from . import slater_koster, structure, hamiltonian, exact, krylov, physics, pipeline, cohp  # noqa: F401
