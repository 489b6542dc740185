/*
 * cola.h -- C ABI of the GB300 Wilson-Dirac hot path.
 *
 * Kamleh, "Evolving the COLA software library" (Lattice 2022) describes a
 * GPU fermion-matrix inverter written in CUDA C/C++ and called through a
 * plain C interface (ISO C Binding) from Fortran; this header is that kind of
 * boundary.  The paper does not write the operator.  The library implements
 * the kappa-normalised Wilson matrix
 *
 *   (H psi)(x) = sum_mu (1 - gamma_mu) Ut_mu(x) psi(x+mu)
 *              + (1 + gamma_mu) Ut_mu(x-mu)^dag psi(x-mu),     D = 1 - kappa H,
 *
 * gamma matrices in the Hermitian chiral (DeGrand-Rossi) basis, Ut_mu(x) =
 * U_mu(x) * bc[mu] on links that cross the lattice boundary (x_mu = L_mu - 1).
 * Even-odd preconditioning uses the Schur operator on even sites,
 * Mhat = 1 - kappa^2 H_eo H_oe, whose determinant equals det D.  A handle may
 * carry a clover term A(x) (cola_clover_attach): then D = A - kappa H and
 * Mhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe.  Around the operator: CG solves
 * (plain FP64 or mixed precision, many right-hand sides, batches of
 * lattices), multi-shift CG, the fermion and gauge forces and an HMC
 * trajectory driver, and a Kalkreuter-Simma eigensolver.
 *
 * Conventions shared by every call:
 *  - Site index i = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2.
 *    All four extents must be even and >= 2.
 *  - Canonical spinor: complex128 [V][4 spin][3 colour], interleaved (re, im).
 *    Canonical gauge field: complex128 [4 mu][V][3][3], row-major 3x3.
 *    Multi-RHS canonical spinors: [nrhs][V][4][3].
 *  - Packed spinor (the layout the Dslash reads): both parities, even first,
 *    each parity a structure of arrays over its V/2 sites; per right-hand
 *    side cola_spinor_bytes(lat, prec, 1) bytes, right-hand side outermost.
 *  - Every pointer is a DEVICE pointer unless its comment says host.  The
 *    caller owns every buffer it passes; the library owns only what a handle
 *    holds (packed links, clover fields, solver workspace), released by
 *    cola_gauge_destroy.
 *  - All work is ordered on the given stream; calls return after enqueuing,
 *    except those that report results to the host (the solvers, the
 *    eigensolver, the HMC trajectory, cola_plaquette, cola_clover_attach,
 *    and cola_gauge_update / cola_link_update on a handle with a clover term,
 *    which rebuild it and read back its pivot flag), which synchronise the
 *    stream.  A call that first needs handle workspace allocates it then.
 *  - A handle is not thread-safe: its workspace is reused by every call, so
 *    calls on one handle must be ordered (one stream, or synchronised).
 *  - Errors are returned as cola_status codes; nothing aborts.  The message
 *    of the last failure on the calling thread is cola_last_error().
 */
#ifndef COLA_H
#define COLA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t; /* identical to CUDA's own typedef */

typedef enum {
    COLA_OK = 0,
    COLA_ERR_ARG = -1,           /* invalid argument: null pointer, odd extent, bad enum, size */
    COLA_ERR_CUDA = -2,          /* a CUDA runtime call failed (message has the CUDA error) */
    COLA_ERR_NOMEM = -3,         /* device allocation failed */
    COLA_ERR_NOT_CONVERGED = -4, /* max_iter reached; x holds the best iterate */
    COLA_ERR_BREAKDOWN = -5,     /* non-finite or non-positive CG scalar (e.g. NaN source) */
    COLA_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
    COLA_ERR_UNSUPPORTED = -7    /* precision not packed in this gauge handle */
} cola_status;

typedef enum { COLA_F64 = 0, COLA_F32 = 1, COLA_F16 = 2 } cola_prec;

enum { COLA_OP_FULL = 0, COLA_OP_EO = 1 };
enum { COLA_SYS_NORMAL = 0, COLA_SYS_DIRAC = 1 };
enum { COLA_PARITY_EVEN = 0, COLA_PARITY_ODD = 1, COLA_PARITY_BOTH = 2 };

/* Lattice and operator parameters.  bc[mu] = (re, im) of the phase on links
 * crossing the boundary in direction mu: (1,0) periodic, (-1,0) anti-periodic. */
typedef struct {
    int dims[4];     /* Lx, Ly, Lz, Lt */
    double kappa;    /* hopping parameter */
    double bc[4][2];
} cola_lattice;

/* Which packed copies of the links a handle holds.  prec_mask bit (1 << p)
 * requests precision p; recon[p] is 12 (rows 0-1 stored, row 2 rebuilt as
 * conj(row0 x row1)) or 18 (all rows stored).  FP16 links are SU(3) entries,
 * |u_ij| <= 1, so they are stored without a scale factor. */
typedef struct {
    unsigned prec_mask;
    int recon[3];
} cola_gauge_opts;

typedef struct cola_gauge_s *cola_gauge;

/* Pack the canonical FP64 links (device, [4][V][3][3] complex128, caller-owned,
 * read during the call's stream work only) into every requested precision.
 * The links must be SU(3) for recon 12.  On success *out owns device memory. */
cola_status cola_gauge_create(const cola_lattice *lat, const void *links_dev,
                              const cola_gauge_opts *opts, cudaStream_t stream,
                              cola_gauge *out);
cola_status cola_gauge_destroy(cola_gauge g);
/* Re-pack new links (same lattice, same layout as cola_gauge_create) into an
 * existing handle, keeping its precisions, reconstruction and workspace (an
 * HMC trajectory changes the links at every step). */
cola_status cola_gauge_update(cola_gauge g, const void *links_dev, cudaStream_t stream);

/* Bytes of one packed spinor field (both parities) times nrhs. */
size_t cola_spinor_bytes(const cola_lattice *lat, cola_prec prec, int nrhs);

/* canonical complex128 [nrhs][V][4][3] <-> packed.  FP16 stores each site as
 * half values scaled by that site's max |component| (an FP32 scale). */
cola_status cola_spinor_pack(cola_gauge g, void *packed_dev, const void *canon_dev,
                             cola_prec prec, int nrhs, cudaStream_t stream);
cola_status cola_spinor_unpack(cola_gauge g, void *canon_dev, const void *packed_dev,
                               cola_prec prec, int nrhs, cudaStream_t stream);

/* Hopping term on packed fields, for each of nrhs right-hand sides:
 *   out_p = a * in_self_p + b * H_{p,1-p} in_{1-p}
 * for p = parity (0 even, 1 odd) or both parities (2).  dagger != 0 applies
 * H^dag (projectors swapped).  in_self may be NULL when a == 0.  out must not
 * alias in.  FP64 accumulates in double, FP32/FP16 storage in float. */
cola_status cola_dslash_apply(cola_gauge g, void *out, const void *in, const void *in_self,
                              double a, double b, int parity, int dagger, cola_prec prec,
                              int nrhs, cudaStream_t stream);

/* out = D in (dagger: D^dag in) on packed fields, both parities, for each
 * of nrhs right-hand sides: D = 1 - kappa H, or A - kappa H when the handle
 * has a clover term.  out must not alias in. */
cola_status cola_dirac_apply(cola_gauge g, void *out, const void *in, int dagger, cola_prec prec,
                             int nrhs, cudaStream_t stream);

/* out = M^dag M in on packed fields.  op COLA_OP_FULL: M = D on the whole
 * lattice.  op COLA_OP_EO: M = Mhat on the even half (the odd half of out is
 * left as it was).  With a clover term D = A - kappa H and
 * Mhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe.  Uses workspace held by the
 * handle (allocated on first use). */
cola_status cola_mdagm_apply(cola_gauge g, void *out, const void *in, int op, cola_prec prec,
                             int nrhs, cudaStream_t stream);

/* The same operator as cola_mdagm_apply, for callers that cannot allocate
 * device memory when they call it (for example a service that reserves all
 * device memory up front).  The paper has no counterpart: it is an addition
 * of this library.  It calls no allocator; its temporaries live in one
 * static device array of 64 MiB that the library holds on each device until
 * the process exits.  A call needs cola_spinor_bytes(lat, prec, nrhs) bytes
 * of that array and returns COLA_ERR_ARG above 64 MiB.  Every call looks up
 * the array's device address in the current device's context
 * (cudaGetSymbolAddress), so a context that was reset and created again gets
 * the new address; the first call in a context may load the library's device
 * code there.  With
 * lazy module loading (the CUDA default) the array is reserved on a device
 * when this part of the library is first used there; with
 * CUDA_MODULE_LOADING=EAGER every process that loads the library reserves it
 * on each device it uses, even if it never calls this entry point.
 * All calls share the array: calls whose work overlaps on the GPU (other
 * streams, unordered threads) race, so order them. */
cola_status cola_mdagm_apply_noalloc(cola_gauge g, void *out, const void *in, int op, cola_prec prec,
                                     int nrhs, cudaStream_t stream);

/* Clover (Sheikholeslami-Wohlert) term.  The paper's list of COLA's physics
 * features cites clover-improved Wilson actions (FLIC fermions among them)
 * without writing them; this is the standard term in the kappa
 * normalisation above:
 *   A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_munu F_munu(x),
 *   sigma_munu = (i/2)[gamma_mu, gamma_nu],
 *   F_munu(x) = traceless part of (Q_munu(x) - Q_munu(x)^dag) / (8i),
 * Q_munu(x) the sum of the four plaquettes of the (mu, nu) plane touching x,
 * each oriented mu -> nu, from the links WITHOUT boundary phases.  Then
 * D = A - kappa H and the even-odd Schur operator is
 * Mhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe (det D = det A_oo det Mhat).
 *
 * cola_clover_attach builds A and A^-1 on every site from the handle's FP64
 * links (the handle must hold COLA_F64) and stores both in each precision
 * the handle holds (72 reals per site each; FP16 without a scale).  From then
 * on cola_dirac_apply, cola_mdagm_apply(_noalloc) and cola_cg_solve(_batched)
 * use the clover operator, cola_gauge_update rebuilds the term for the new
 * links, cola_fermion_force and cola_dirac_link_grad add the clover term's
 * parts, and cola_hmc_trajectory integrates the clover action.
 * cola_dslash_apply stays the bare hopping term.  csw = 0 removes the term.
 * The call waits for its stream (it reads back a pivot flag): it returns
 * COLA_ERR_BREAKDOWN, and leaves the handle without a clover term, if some
 * A(x) block has a zero or non-finite pivot in its LDL^dag factorisation. */
cola_status cola_clover_attach(cola_gauge g, double csw, cudaStream_t stream);
/* c_sw of the attached clover term, 0 if none (or g is NULL). */
double cola_clover_csw(cola_gauge g);
/* out_p = A_pp in_p (inverse != 0: A_pp^-1 in_p) on packed fields for
 * parity p (0, 1, or 2 = both) and nrhs right-hand sides; out may alias in.
 * COLA_ERR_UNSUPPORTED without a clover term. */
cola_status cola_clover_apply(cola_gauge g, void *out, const void *in, int parity, int inverse,
                              cola_prec prec, int nrhs, cudaStream_t stream);

typedef struct {
    double tol;      /* target true relative residual (e.g. 1e-10) */
    int max_iter;    /* iteration cap (CG steps) */
    int op;          /* COLA_OP_FULL or COLA_OP_EO */
    int system;      /* COLA_SYS_NORMAL: M^dag M x = b;  COLA_SYS_DIRAC: D x = b */
    int inner;       /* cola_prec of the inner iterations; COLA_F64 = plain FP64 CG */
    double delta;    /* reliable-update trigger: |r_inner| < delta * |r| at last update */
    int nrhs;        /* right-hand sides solved together (1..64) */
    int use_graph;   /* 1: run the iteration loop as one CUDA graph with device-side control */
} cola_solver_params;

typedef struct {
    int iters;             /* CG iterations */
    int reliable_updates;  /* FP64 residual recomputations, the initial one included */
    double true_rel_resid; /* |b - A x| / |b| (SYS_DIRAC: |b - D x| / |b|) recomputed in FP64 at the end */
    double seconds;        /* wall time of the call */
    int status;            /* cola_status of this right-hand side */
} cola_solve_info;

/* Solve for x in canonical FP64 layout ([nrhs][V][4][3] complex128, device).
 * On entry x holds the initial guess (zeros for a cold start); on return the
 * solution.  SYS_NORMAL + OP_FULL: D^dag D x = b.  SYS_NORMAL + OP_EO:
 * Mhat^dag Mhat x_e = b_e (odd sites of b ignored, of x set to zero).
 * SYS_DIRAC: D x = b (OP_EO through the Schur complement and its normal
 * equations, x_o = A_oo^-1 (b_o + kappa H_oe x_e), A = 1 without a clover
 * term).  Convergence is declared on the FP64 true residual of the system
 * solved: |b - A x| <= tol |b| for SYS_NORMAL; for SYS_DIRAC on the Dirac
 * residual |b - D x| <= tol |b| over the whole lattice (a right-hand side
 * whose normal equations met their target while its Dirac residual did not
 * is solved again from its x with a target scaled down by the ratio it
 * missed by; iters and reliable_updates then sum the passes, and after 6
 * passes it returns COLA_ERR_NOT_CONVERGED).  info has nrhs entries (host).
 * With clover terms, every handle of a batched solve must have one. */
cola_status cola_cg_solve(cola_gauge g, void *x_dev, const void *b_dev,
                          const cola_solver_params *params, cola_solve_info *info,
                          cudaStream_t stream);

/* Several lattices (up to 8, uneven volumes allowed) solved together: every
 * kernel of an iteration is one launch over all lattices and right-hand sides,
 * each (lattice, right-hand side) with its own CG scalars and convergence.
 * gauges[l], x_dev[l], b_dev[l] as in cola_cg_solve (distinct handles, the
 * same link reconstruction per precision); params (including nrhs) shared;
 * info has nlat * nrhs entries, lattice-major (host). */
cola_status cola_cg_solve_batched(int nlat, const cola_gauge *gauges, void *const *x_dev,
                                  const void *const *b_dev, const cola_solver_params *params,
                                  cola_solve_info *info, cudaStream_t stream);

/* Multi-shift CG: x_i = (A + shifts[i])^-1 b for nshift (1..64) shifts >= 0
 * at once, A = Mhat^dag Mhat (op COLA_OP_EO, even sites; odd sites of x set
 * to zero) or D^dag D (COLA_OP_FULL); the partial-fraction building block
 * of rational HMC.  x_dev: canonical FP64 [nshift][V][4][3] (device, output;
 * no initial guess); b_dev: canonical [V][4][3]; shifts: host array.
 * Phase 1 runs the shifted-CG recurrence (Jegerlehner 1996) on one Krylov
 * space down to tol_sloppy (0: tol for FP64, else max(tol, 1e-7)), in FP64
 * when params->inner is COLA_F64 and in FP32 storage otherwise (the handle
 * then needs FP32 links too); phase 2 refines all shifts together with the
 * mixed-precision CG of cola_cg_solve in params->inner (rows = shifts, FP64
 * reliable updates, FP64 true residual) down to params->tol.  params: system
 * must be NORMAL; nrhs ignored.  info: nshift entries (host); iters counts
 * both phases. */
cola_status cola_multishift_solve(cola_gauge g, void *x_dev, const void *b_dev, const double *shifts,
                                  int nshift, double tol_sloppy, const cola_solver_params *params,
                                  cola_solve_info *info, cudaStream_t stream);

/* Lowest eigenmodes of A = Mhat^dag Mhat (op COLA_OP_EO, even sites) or
 * D^dag D (COLA_OP_FULL) by the accelerated conjugate-gradient method of
 * Kalkreuter and Simma (1996), which the paper cites for COLA's eigensolver:
 * each vector minimises the Ritz functional <x, A x> / <x, x> by CG in the
 * complement of the ones before it, and every sweep ends with a
 * Rayleigh-Ritz diagonalisation of A on the span of all nev vectors.  FP64.
 * nextra guard vectors are iterated with the nev wanted ones but not tested
 * for convergence (they speed up levels close to the edge of the wanted set).
 * evecs_dev: canonical FP64 [nev + nextra][V][4][3] (device); on entry the
 * caller's starting vectors (e.g. Gaussian; they must be independent on the
 * operator's sites), on return orthonormal Ritz vectors, the first nev the
 * eigenvectors (odd sites zero for COLA_OP_EO).  evals: host [nev + nextra],
 * ascending.  Converged when every |A v_j - lambda_j v_j| <= tol lambda_j
 * for j < nev; COLA_ERR_NOT_CONVERGED after max_sweeps sweeps (the best
 * estimates are returned).  Uses the handle's workspace block that
 * cola_multishift_solve also uses. */
typedef struct {
    int nev;         /* eigenpairs wanted (>= 1) */
    int nextra;      /* guard vectors (>= 0); nev + nextra <= 64 */
    int op;          /* COLA_OP_EO or COLA_OP_FULL */
    double tol;      /* relative residual target */
    int max_sweeps;  /* sweeps (each: nev Ritz minimisations + one Rayleigh-Ritz step) */
    int max_cg;      /* CG steps per vector per sweep */
    double gamma;    /* a vector's minimisation stops once |gradient| fell by this factor */
} cola_eig_params;

typedef struct {
    int sweeps;
    int applications;     /* operator applications */
    double max_rel_resid; /* max_j |A v_j - lambda_j v_j| / lambda_j at return */
    double seconds;
    int status;
} cola_eig_info;

cola_status cola_eig_lowest(cola_gauge g, void *evecs_dev, double *evals, const cola_eig_params *params,
                            cola_eig_info *info, cudaStream_t stream);

/* Fermion force of S = phi^dag (D^dag D)^-1 phi given X = (D^dag D)^-1 phi and
 * Y = D X (canonical FP64, device).  Output force_dev: real FP64 [4][V][8],
 * F^a_mu(x) = dS/d eps^a for U_mu(x) -> (1 + i eps T^a) U_mu(x), T^a = lambda^a/2:
 * F^a = -2 kappa Im Tr[T^a Ut_mu(x) (P + Q^dag)], with
 * P_ba = sum_s [(1-gamma_mu) X(x+mu)]_sb conj(Y(x)_sa),
 * Q_ba = sum_s [(1+gamma_mu) X(x)]_sb conj(Y(x+mu)_sa).  Accumulated in FP64.
 * With a clover term (D = A - kappa H, Y = D X) the clover part is added:
 * dS = -2 Re Y^dag dA X = (kappa c_sw / 4) sum_x sum_{mu<nu} Im Tr[dQ_munu Gam_munu],
 * Gam_munu(x) = L + L^dag, L the traceless part of
 * Lam_ba = sum_st (sigma_munu)_st X(x)_tb conj(Y(x)_sa); each link collects the
 * two plaquettes of each of its three planes with Gam inserted at their four
 * corners (the links without boundary phases).  That part needs 384 bytes
 * of handle workspace per site. */
cola_status cola_fermion_force(cola_gauge g, double *force_dev, const void *X_dev,
                               const void *Y_dev, cudaStream_t stream);

/* Raw complex link gradient of a real loss through y = D psi, in the
 * convention grad = 2 dL/d conj(U) (PyTorch's), given g = that gradient on y:
 * grad_U_mu(x)_ab = -kappa conj(ph) [ sum_s g(x)_sa conj([(1-gamma_mu) psi(x+mu)]_sb)
 *                                    + sum_s [(1+gamma_mu) psi(x)]_sa conj(g(x+mu)_sb) ],
 * ph the link's boundary phase.  Canonical FP64 in and out ([4][V][3][3]).
 * With a clover term (D = A - kappa H) the clover part is added: with Gam
 * built from (X, Y) = (psi, g) as for cola_fermion_force, dL = Re g^dag dA psi
 * = -(kappa c_sw / 8) sum_x sum_{mu<nu} Im Tr[dQ_munu Gam_munu], and a factor
 * U (U^dag) of a leaf contributes -i (kappa c_sw / 8) M^dag (+i (kappa c_sw / 8) M),
 * M the rest of the leaf with Gam inserted; the links without boundary
 * phases; 384 bytes of handle workspace per site. */
cola_status cola_dirac_link_grad(cola_gauge g, void *grad_links_dev, const void *psi_dev,
                                 const void *gy_dev, cudaStream_t stream);

/* ---------------------------------------------------------------- HMC ----
 * Hybrid Monte Carlo around the fermion force (HMC is one of COLA's key
 * algorithms in the paper's overview; the formulas are the standard ones).
 * Links without fermion boundary phases enter the Wilson gauge action
 *   S_G = beta sum_x sum_{mu<nu} (1 - Re tr U_munu(x) / 3),
 *   U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.
 * Momenta and forces are real FP64 [4][V][8] coefficients of the generators
 * T^a = lambda^a / 2 (Gell-Mann); P_mu(x) = sum_a p^a T^a, kinetic energy
 * K = sum p^2 / 2; a force is dS/deps^a for U_mu(x) -> (1 + i eps T^a) U_mu(x),
 * as for cola_fermion_force.  Pseudofermions: phi = D^dag eta,
 * S_F = phi^dag (D^dag D)^-1 phi (whole-lattice D, FP64 Wilson).  H = K + S_G + S_F. */

/* Mean plaquette (1/6V) sum Re tr U_munu / 3 of the handle's FP64 links,
 * written to *plaq (host); waits for the stream. */
cola_status cola_plaquette(cola_gauge g, double *plaq, cudaStream_t stream);

/* force_dev = dS_G/deps^a (FP64 [4][V][8], device). */
cola_status cola_gauge_force(cola_gauge g, double beta, double *force_dev, cudaStream_t stream);

/* links_dev (canonical FP64 [4][V][3][3], device, the field the handle was
 * created or last updated from) <- exp(i eps P) U link by link, then the
 * handle is re-packed from it (and its clover term rebuilt) as by
 * cola_gauge_update.  The exponential is exact to FP64 rounding (power series
 * reduced by Cayley-Hamilton to three scalars, with scaling and squaring). */
cola_status cola_link_update(cola_gauge g, void *links_dev, const double *mom_dev, double eps,
                             cudaStream_t stream);

enum { COLA_INT_LEAPFROG = 0, COLA_INT_OMELYAN = 1 };

typedef struct {
    double beta;            /* gauge coupling */
    double tau;             /* trajectory length */
    int nsteps;             /* integration steps (step eps = tau / nsteps) */
    int integrator;         /* COLA_INT_LEAPFROG, or COLA_INT_OMELYAN (2MN, lambda = 0.1931833275037836) */
    double uniform;         /* Metropolis random number in [0, 1): accept if uniform <= exp(-dH) (0: always) */
    cola_solver_params md;  /* force solves X = (D^dag D)^-1 phi: op COLA_OP_FULL runs CG on D^dag D;
                               op COLA_OP_EO solves D W = gamma5 phi, then D X = gamma5 W, each
                               through the even-odd Schur complement (system is set per solve) */
    double action_tol;      /* tolerance of the final action solve */
} cola_hmc_params;

typedef struct {
    double dH, H0, H1;  /* H1 - H0, start and end Hamiltonians */
    int accepted;
    double plaquette;   /* mean plaquette of the links on return */
    int force_evals;    /* force evaluations of the trajectory */
    int cg_iters;       /* CG iterations summed over every solve */
    double seconds;
} cola_hmc_info;

/* One HMC update of the gauge field links_dev (canonical FP64, device, in
 * and out; the handle must be created from or last updated with it and hold
 * FP64 links; with a clover term D = A - kappa H throughout, the term rebuilt
 * after every link update) with momenta mom_dev (FP64 [4][V][8],
 * device, drawn by the caller from N(0, 1); on return the final momenta of
 * the trajectory) and pseudofermion source eta_dev (canonical spinor,
 * device, drawn by the caller; NULL for the pure gauge theory).
 * phi = D^dag eta; H0 = K + S_G + |eta|^2; the molecular-dynamics trajectory
 * (leapfrog: p -= eps/2 F; n x [U <- exp(i eps P) U; p -= eps F], the last
 * momentum step eps/2; Omelyan 2MN: p -= lam eps F; U <- exp(i eps/2 P) U;
 * p -= (1 - 2 lam) eps F; U <- exp(i eps/2 P) U; p -= lam eps F, the two
 * adjacent lam steps of consecutive steps merged), F = dS_G/deps +
 * dS_F/deps with X = (D^dag D)^-1 phi solved from a zero guess (see md); then H1 and
 * the Metropolis test.  On rejection links_dev and the handle are restored
 * bitwise.  Waits for the stream. */
cola_status cola_hmc_trajectory(cola_gauge g, void *links_dev, double *mom_dev, const void *eta_dev,
                                const cola_hmc_params *params, cola_hmc_info *info, cudaStream_t stream);

/* Thread-local message describing the last error returned on this thread. */
const char *cola_last_error(void);

/* Measurement aid with no counterpart in the paper: launches on `stream`
 * one kernel of `blocks` x `threads` threads, each running 8 independent
 * FP64 fused multiply-add chains for `steps` steps, and returns in *flop
 * (host) the floating-point operations that launch performs
 * (2 x 8 x steps x threads x blocks).  Timing the launch with events on the
 * same stream gives the FP64 arithmetic rate the FP64 hopping term is bound
 * by.  out (device) receives blocks x threads doubles (the chains' sums), so
 * that no work is optimised away.  Returns COLA_ERR_ARG unless threads is a
 * multiple of 32 in 32..256, blocks in 1..2^20 and steps a positive
 * multiple of 4.  Does not wait for the device. */
cola_status cola_probe_fp64_fma(double *out, int blocks, int threads, int steps, cudaStream_t stream,
                                double *flop);

/* Debug builds only (libcola compiled with -DCOLA_BOUNDS): every neighbour,
 * link and site index the kernels compute is checked against its extent; an
 * index out of range is counted, the kernel source line of the first one is
 * recorded, and the access is redirected to index 0 (no fault, wrong result).
 * Waits for the device, then returns in *count (host) the number of
 * violations since the last reset and in *first_line (host) that line, 0 if
 * none; reset != 0 zeroes the counters.  A default build returns
 * COLA_ERR_UNSUPPORTED. */
cola_status cola_debug_bounds(unsigned long long *count, int *first_line, int reset);

#ifdef __cplusplus
}
#endif
#endif /* COLA_H */
