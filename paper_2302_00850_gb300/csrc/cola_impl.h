// Internal host-side interfaces between the translation units of libcola.
#pragma once

#include <string>
#include <vector>

#include "cola_internal.cuh"

namespace cola {

// Lattices of one batched launch (a single lattice is a batch of one).
constexpr int kMaxBatch = 8;

// One lattice of a hopping-term launch.  Spinor pointers address whole packed
// fields (both parities, right-hand side 0); the kernel offsets them by
// parity and right-hand side.
struct DslashLat {
    Geom g;
    const void *links;            // packed links of this precision: [parity][mu][group][Vh]
    size_t link_parity_stride;    // bytes of one parity of links
    size_t link_dir_stride;       // bytes of one direction of one parity
    void *out;
    const void *in;
    const void *xin;              // xpay input, same layout as out (null if !xpay)
    const void *clv;              // clover field of the epilogue (A or A^-1, both parities), else null
    size_t clv_parity_stride;     // bytes of one parity of clv
    size_t parity_stride;         // bytes of one parity of one spinor field
    size_t rhs_stride;            // bytes of one right-hand side of a spinor field
    double a, b;                  // out = a xin + b H in
    int row0;                     // solver row (state, partials) of this lattice's rhs 0
    int block0;                   // first blockIdx.x of this lattice (set by launch_dslash)
    int nblocks;                  // site blocks of this lattice per parity (set by launch_dslash)
};

struct DslashArgs {
    int nlat;
    int nrhs;
    int rhs_per_block;            // threads per block along right-hand sides (blockDim.y)
    int rhs_per_thread;           // right-hand sides each thread carries (0 or 1: one)
    int parity0;                  // first output parity (blockIdx.z adds 0 or 1)
    DslashLat lat[kMaxBatch];
    CgState *state;               // solver mode: skip finished rows
    int filter_ru;                // with state: compute only rows with a pending reliable update
    int ngroups;                  // right-hand-side groups (set by launch_dslash)
    // With red != null (xpay epilogues only): each block also writes, per
    // solver row, the partial sum of |xin|^2 over its sites to
    // red[row * red_stride + parity block * nblocks + site block], for a
    // finishing kernel to sum in block order.
    double *red;
    int red_stride;
};

// Epilogue of a hopping-term launch, per output site x of parity p:
//   EPI_HOP         out = b H in
//   EPI_XPAY        out = a xin + b H in
//   EPI_CLOVER_X    out = a A(x) xin + b H in          (clv = A)
//   EPI_CLOVER_INV  out = A(x)^-1 (b H in)              (clv = A^-1)
enum DslashEpi : int { EPI_HOP = 0, EPI_XPAY = 1, EPI_CLOVER_X = 2, EPI_CLOVER_INV = 3 };

int default_dslash_block(int prec, int rhs_per_block);
// Within this scope (per thread), launch_dslash only autotunes configurations
// it has not seen and launches nothing else.
struct TuneOnlyScope {
    TuneOnlyScope();
    ~TuneOnlyScope();
};
// Fills block0/nblocks of every lattice and launches; block_x <= 0 picks the
// autotuned (or default) launch shape.
cudaError_t launch_dslash(int prec, int recon, DslashArgs &A, int nparity, bool dagger, int epi, int block_x,
                          cudaStream_t s);
// The clover epilogues (instantiated in their own translation unit); A's
// block0/nblocks/ngroups are already assigned, nb is the grid size.
cudaError_t launch_dslash_clover(int prec, int recon, const DslashArgs &A, int nparity, bool dagger, int epi, int bx,
                                 int nb, cudaStream_t s);

// ----------------------------------------------------------------- clover --
// sigma_munu restricted to the two chirality blocks, planes in the order
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): sig[plane][chi][2 s + t] = (re, im).
struct CloverSigma {
    double v[6][2][4][2];
};
// Builds A = 1 - coef sum sigma F and A^-1 (coef = kappa c_sw) on every site
// from the FP64 links and writes both into each non-null a[p] / ainv[p];
// *bad is set to 1 if a block of A has a zero or non-finite pivot.
cudaError_t launch_clover_build(const Geom &g, const void *links_f64, int recon, double coef, const CloverSigma &sig,
                                void *const a[3], void *const ainv[3], int *bad, cudaStream_t s);
// sigma_munu in the hopping kernel's basis, by plane and chirality block
const CloverSigma &clover_sigma();
// Bytes of scratch launch_clover_force needs (six Hermitian traceless 3x3
// matrices per site).
size_t clover_force_scratch_bytes(const Geom &g);
// force = coef F_clover (accumulate: force += ...), [4][V][8]: the clover
// term's part of dS/deps^a for S = phi^dag (D^dag D)^-1 phi from canonical
// FP64 X = (D^dag D)^-1 phi and Y = D X, with the FP64 links of the handle.
cudaError_t launch_clover_force(const Geom &g, const void *links_f64, int recon, double kappa, double csw,
                                const void *X, const void *Y, double *force, double coef, bool accumulate,
                                void *scratch, cudaStream_t s);
// grad += the clover term's part of the raw link gradient (PyTorch's
// convention, canonical [4][V][3][3] complex) of a real loss through
// y = D psi, given gy = dL/dy; same scratch as launch_clover_force.
cudaError_t launch_clover_link_grad(const Geom &g, const void *links_f64, int recon, double kappa, double csw,
                                    const void *psi, const void *gy, void *grad, void *scratch, cudaStream_t s);
// out_p = C_p in_p on the parities of parity_mask (1 even, 2 odd, 3 both).
cudaError_t launch_clover_apply(int prec, const Geom &g, const void *clv, void *out, const void *in, int nrhs,
                                int parity_mask, cudaStream_t s);

// ---------------------------------------------------------------- packing --
cudaError_t launch_pack_gauge(int prec, int recon, const Geom &g, void *packed, const void *canon,
                              cudaStream_t s);
cudaError_t launch_pack_spinor(int prec, const Geom &g, void *packed, const void *canon, int nrhs,
                               int parity_mask, cudaStream_t s);
cudaError_t launch_unpack_spinor(int prec, const Geom &g, void *canon, const void *packed, int nrhs,
                                 int parity_mask, cudaStream_t s);

// ------------------------------------------------------------ CG kernels --
// Batched vector kernels: per lattice up to kMaxVecs packed fields (slot
// meaning depends on the kernel), all of the precision prec[slot].  Each
// lattice covers nparity parity blocks (1: even half only; 2: whole lattice)
// of nrhs right-hand sides; rows are row0 + rhs.
constexpr int kMaxVecs = 6;

struct BlasLat {
    int vh;
    int row0;
    int block0;    // set by the launcher
    int nblocks;   // set by the launcher
    void *v[kMaxVecs];
};

struct BlasArgs {
    int nlat;
    int nparity;
    int nrhs;
    int prec[kMaxVecs];
    BlasLat lat[kMaxBatch];
    CgState *state;
    double *partials;     // [row][pstride] block partials of reductions
    int pstride;
    double *out;          // norm2 results per row
    double a, b;          // axpby coefficients
    int init;             // ru_residual: initial residual (every row, also writes p)
};

// Slots: update_xr (x, r, p, q); update_p (p, r); pq (mp, p); ru_accumulate (x_hi, x_lo);
// ru_residual (r_hi, b, ax, r_lo, p, x_hi); norm2 (v); convert (dst, src); axpby (dst, x, y).
// A row with CgState::shift = sigma != 0 solves (A + sigma) x = b: pq adds
// sigma |p|^2 (reading p), update_xr subtracts alpha (q + sigma p), and
// ru_residual subtracts sigma x_hi (reading x_hi); rows with sigma = 0 read
// and compute exactly what the unshifted solver does.
cudaError_t launch_cg_update_xr(BlasArgs &B, cudaStream_t s);
cudaError_t launch_cg_update_p(BlasArgs &B, cudaStream_t s);
cudaError_t launch_cg_pq(BlasArgs &B, cudaStream_t s);         // slot (mp): pq, rho, alpha
// pq, rho, alpha from block partials already in B.partials (B.lat[l].nblocks
// partials per row of lattice l, row stride B.pstride), e.g. left by a
// hopping launch with a fused reduction.
cudaError_t launch_finish_pq(const BlasArgs &B, cudaStream_t s);
// Row stride of the reduction scratch for lattices of vh sites per parity:
// enough for the vector kernels and for a hopping launch's block partials.
int reduce_stride(int vh);
cudaError_t launch_ru_accumulate(BlasArgs &B, bool force, cudaStream_t s);
cudaError_t launch_ru_residual(BlasArgs &B, cudaStream_t s);
cudaError_t launch_init_norms(BlasArgs &B, cudaStream_t s);   // st.b2 = |b|^2, st.tol2 *= |b|^2
cudaError_t launch_norm2(BlasArgs &B, cudaStream_t s);        // out[row] = |v|^2
cudaError_t launch_convert(BlasArgs &B, cudaStream_t s);
cudaError_t launch_any_nonzero(BlasArgs &B, unsigned *flags, cudaStream_t s);  // F64 slot (v); flags zeroed by caller
cudaError_t launch_axpby(BlasArgs &B, cudaStream_t s);
// Largest block count per row of the batched vector kernels (partials stride).
int blas_max_blocks(const BlasArgs &B);

// ----------------------------------------------------------------- force --
// force = coef F (accumulate: force += coef F), F the fermion force [4][V][8]
cudaError_t launch_force(const Geom &g, double kappa, const void *links_f64, int recon, double *force,
                         const void *X, const void *Y, cudaStream_t s, double coef = 1.0, bool accumulate = false);
cudaError_t launch_link_grad(const Geom &g, double kappa, void *grad, const void *psi, const void *gy,
                             cudaStream_t s);

// ----------------------------------------------------------------- gauge --
// out = coef * dS_G/deps (accumulate: out += ...), [4][V][8], from FP64 links
cudaError_t launch_gauge_force(const Geom &g, const void *links_f64, int recon, double beta, double coef, double *out,
                               bool accumulate, cudaStream_t s);
// doubles of reduction scratch the two reductions below need
size_t gauge_scratch_doubles(const Geom &g);
// *out = sum over sites and planes mu < nu of Re tr U_munu(x) / 3 (device)
cudaError_t launch_plaquette_sum(const Geom &g, const void *links_f64, int recon, double *scratch, double *out,
                                 cudaStream_t s);
// *out = scale * sum_k a[k] b[k] (device), deterministic
cudaError_t launch_dot(const double *a, const double *b, size_t n, double scale, double *scratch, double *out,
                       cudaStream_t s);
// out = gamma5 in on one canonical FP64 spinor field
cudaError_t launch_gamma5(const Geom &g, void *out, const void *in, cudaStream_t s);
// canonical links U_mu(x) <- exp(i eps P_mu(x)) U_mu(x)
cudaError_t launch_link_update(const Geom &g, void *links_canon, const double *mom, double eps, cudaStream_t s);

// ------------------------------------------------------------------ errors --
void set_error(const std::string &msg);

}  // namespace cola

// ------------------------------------------------------------ gauge handle --
// Owns the packed links of each requested precision and the solver
// workspace (device buffers grown on demand and kept until destroy).
struct cola_gauge_s {
    cola_lattice lat;
    cola::Geom geom;
    int device = 0;
    void *links[3] = {nullptr, nullptr, nullptr};  // [parity][mu][group][Vh] per precision
    // clover term (csw != 0): A and A^-1 in every precision of the links
    double csw = 0.0;
    void *clover[3] = {nullptr, nullptr, nullptr};
    void *clover_inv[3] = {nullptr, nullptr, nullptr};
    int recon[3] = {12, 12, 12};
    size_t link_parity_bytes[3] = {0, 0, 0};
    // workspace slots: each a device buffer reused across calls
    static constexpr int kSlots = 25;
    static constexpr int kSlotCloverFlag = kSlots - 1;  // the construction's pivot flag
    static constexpr int kSlotCloverForce = 23;         // the clover force's per-site matrices
    // HMC: saved links, phi, X, Y, two packed FP64 fields, reduction scratch
    static constexpr int kSlotHmc = 15;
    static constexpr int kSlotMultishift = 22;  // the multi-shift solver's workspace block
    void *slot[kSlots] = {};
    size_t slot_bytes[kSlots] = {};
    double *partials = nullptr;
    size_t partials_count = 0;
    cola::CgState *states = nullptr;   // device
    cola::CgState *h_states = nullptr; // pinned host mirror
    int states_count = 0;
    // the instantiated solve graph of the last graph-driven solve this handle
    // led, and the bytes of the configuration it was captured for
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<unsigned char> graph_key;
};

namespace cola {
// Device buffer of at least `bytes` in workspace slot `k` (grown if needed).
cola_status ws_slot(cola_gauge g, int k, size_t bytes, void **out);
// Reduction scratch: nrows rows of pstride block partials.
cola_status ws_reduce(cola_gauge g, size_t nrows, size_t pstride);
cola_status ws_states(cola_gauge g, int n);

// One lattice of an operator application: out = M^dag M in with temporaries
// t and mp (full packed fields of the same precision), solver rows from row0.
struct OpLat {
    cola_gauge g;
    void *out;
    const void *in;
    void *t;
    void *mp;
    int row0;
};

DslashLat make_dslash_lat(cola_gauge g, int prec, void *out, const void *in, const void *xin, double a, double b,
                          int row0);
DslashArgs make_dslash_args(cola_gauge g, int prec, void *out, const void *in, const void *xin, int nrhs,
                            int parity0, double a, double b);
// Sets L's epilogue clover field to g's A (inverse: A^-1) of precision prec.
void set_clover(DslashLat &L, cola_gauge g, int prec, bool inverse);
// Launch a (batched) hopping term with the links of `owner`'s reconstruction.
cola_status dslash_launch(cola_gauge owner, int prec, DslashArgs &A, int nparity, bool dagger, int epi,
                          cudaStream_t s);
// The CG solve of one lattice with per-right-hand-side shifts: row r solves
// (A + shifts[r]) x_r = b_r (shifts may be null); shared_b: b holds one field
// used by every row.  x holds the initial guesses on entry.
cola_status cg_solve_rows(cola_gauge g, void *x, const void *b, const cola_solver_params *prm, cola_solve_info *info,
                          cudaStream_t s, const double *shifts, bool shared_b);
// (Re)builds g's clover fields from its FP64 links (g->csw != 0); waits for
// the construction to read its pivot flag.
cola_status clover_rebuild(cola_gauge g, cudaStream_t s);
// Frees g's clover fields and sets g->csw = 0.
void clover_free(cola_gauge g);
// out = Mdag M in for every lattice of L (op EO: Mhat on even halves, with
// Mhat in left in mp; op FULL: D, with D in left in mp).  With st != nullptr
// rows are filtered by st (filter_ru: only rows with a pending reliable
// update).
// With red != null, the last launch of the composition (the one whose xpay
// input is M in) also leaves the block partials of |M in|^2 in red (row
// stride red_stride) and, in red_nb[l], the number of partials of each row of
// lattice l.
cola_status apply_mdagm_batch(int nlat, const OpLat *L, int prec, int op, int nrhs, CgState *st, bool filter_ru,
                              cudaStream_t s, double *red = nullptr, int red_stride = 0, int *red_nb = nullptr);
cola_status apply_mdagm(cola_gauge g, int prec, int op, void *out, const void *in, void *t, void *mp, int nrhs,
                        CgState *st, bool filter_ru, cudaStream_t s);
cola_status cuda_check(cudaError_t e, const char *what);

// COLA_LOG=1 in the environment: one line per solve / eigensolve / trajectory on stderr
bool log_enabled();
void log_line(const char *fmt, ...);

// Named range for profilers and tracers (NVTX; no cost without a tool attached).
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
};
}  // namespace cola
