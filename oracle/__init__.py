"""CPU complex128 oracle for the Hubbard-model VQE statevector path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (``paper_2408_00836_gb300``) and never imports it.

Everything here is the plain definition, written out slowly:

* fermionic operators from the Jordan-Wigner definition, applied to explicit
  basis-state lists of the fixed (N_up, N_dn) sector;
* the Hamiltonian of Eqs. 1, 2, 15 and 16 (hopping t_ij, on-site potential,
  on-site U_i, nearest-neighbour V_ij) as a sparse matrix;
* the Hamiltonian variational ansatz of Eq. 7 applied term by term, every
  term an exact exponential;
* the energy of Eq. 4 with an explicit H|psi>, its adjoint gradient (the
  recursion of Sec. 2.1) and central finite differences;
* a Lanczos ground-state solver with full re-orthogonalisation, standing in
  for the paper's DMRG reference energies.
"""

from .hubbard import *  # noqa: F401,F403
