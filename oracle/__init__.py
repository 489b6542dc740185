"""Plain FP64 CPU oracle for the Wilson-Dirac hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, the smoke check and the benchmark's CPU-baseline leg call it.  It
shares no code with the CUDA path: it works on canonical-layout numpy arrays
with whole-lattice shifts and einsum, in float64/complex128, with no blocking,
fusion or reordering beyond the definitions it cites.

The paper (Kamleh, "Evolving the COLA software library", Lattice 2022) names
the fermion-matrix inverter, the conjugate-gradient solver with 32-bit inner
and 64-bit outer precision (Fig. 2 discussion) and Hybrid Monte Carlo, but
writes no formula.  The operator, basis, boundary phases, even-odd split,
CG recurrence and force therefore follow the standard lattice-QCD
definitions, each stated where it is coded:

  wilson.py  gamma matrices, hopping term H, D = 1 - kappa H, H^dagger,
             even-odd blocks and the Schur operator Mhat, sampled-site H
  solve.py   Hestenes-Stiefel CG with true-residual confirmation, the
             even-odd normal-equation solve, shifted systems (A + sigma_i) x_i = b
             one CG per shift, dense matrices for brute force
  force.py   the fermion force dS/dU of S = phi^dag (D^dag D)^-1 phi
  clover.py  the clover (Sheikholeslami-Wohlert) term A(x), D_sw = A - kappa H,
             its even-odd Schur operator A_ee - kappa^2 H_eo A_oo^-1 H_oe and
             the clover term's parts of the fermion force and of the raw link gradient
  hmc.py     Wilson gauge action and force, momenta, leapfrog and Omelyan
             integrators, the Hamiltonian and the Metropolis step
  eig.py     the lowest eigenpairs of D^dag D and Mhat^dag Mhat (dense and
             Lanczos), and closed forms of both free-field spectra

Pins (tests/test_oracle_*.py, run without a GPU): gamma algebra; the free
field closed form (plane waves and the full D^dag D spectrum); gamma5
hermiticity and the adjoint identity; gauge covariance under random SU(3)
transformations; brute-force dense solves on 2^4; the Schur identity between
the even-odd and full solves; the force against central finite differences of
an exactly computed action and against the closed form S = |eta|^2 at
phi = D^dag eta; for the clover term the unit-gauge reduction, a constant
abelian field in closed form, the weak-field lattice curl, gauge covariance,
dense Schur identities and the tree-level cancellation of the Wilson lift of
Landau zero modes (which fixes its sign), and its force against finite
differences of the bilinear -2 Re Y^dag D_sw X and of the action, and its
raw link gradient against finite differences of link entries; for HMC the gauge force against
finite differences of the action, exact free motion, reversibility and the
second-order scaling of dH (with and without the clover term); for the eigenmodes the closed-form free-field
spectra of D^dag D and Mhat^dag Mhat (derived in eig.py).  Every function
here is pinned by at least one of them.
"""
from .wilson import (  # noqa: F401
    GAMMA, GAMMA5, IDENTITY4, parity_of_sites, even_mask, phased_links, hop,
    dirac, dirac_dag, hop_block, mhat, mhat_dag, mdagm_full, mdagm_eo,
    hop_sites, gamma5_apply,
)
from .solve import cg, solve_normal_full, solve_normal_eo, solve_dirac_eo, solve_shifted, dense_matrix  # noqa: F401
from .force import GELL_MANN, T_GEN, force_coeffs, dirac_link_grad, link_variation  # noqa: F401
