"""GB300-native Wilson-Dirac hot path of the COLA lattice-QCD library.

Kamleh, "Evolving the COLA software library" (Lattice 2022): a GPU
fermion-matrix inverter (CUDA, called through a C interface) with
mixed-precision conjugate gradient.  Here: libcola, a C-ABI shared library of
hand-written sm_103a kernels (include/cola.h), and this thin torch binding.

    import paper_2302_00850_gb300 as cola
    g = cola.Gauge(links, dims=(16, 16, 16, 32), kappa=0.125)
    x, info = cola.cg_solve(g, b, op="eo", inner="f16", delta=0.1)
    g.attach_clover(1.0)        # D = A - kappa H from here on
"""
from .api import (  # noqa: F401
    ColaError, EigInfo, Gauge, HmcInfo, SolveInfo, apply_clover, apply_dirac, cg_solve, cg_solve_batched, clover,
    debug_bounds, dirac, dirac_link_grad, dslash, eig_lowest, fermion_force, gauge_force, hmc_trajectory, link_update, mdagm, multishift_solve,
    pack, plaquette, unpack, F16, F32, F64, OP_EO, OP_FULL, SYS_DIRAC, SYS_NORMAL,
)
from .autograd import DiracOp, PseudofermionAction, SolveNormal  # noqa: F401
