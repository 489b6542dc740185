// Internal host-side interfaces between the translation units of libcola.
#pragma once

#include <string>

#include "cola_internal.cuh"

namespace cola {

// Arguments of one hopping-term launch.  Pointers address whole packed
// fields (both parities, right-hand side 0); the kernel offsets them by
// parity and right-hand side.
struct DslashArgs {
    Geom g;
    void *out;
    const void *in;
    const void *xin;              // xpay input, same layout as out (may be null if !xpay)
    const void *links;            // packed links of this precision: [parity][mu][group][Vh]
    size_t link_parity_stride;    // bytes of one parity of links
    size_t link_dir_stride;       // bytes of one direction of one parity
    size_t parity_stride;         // bytes of one parity of one spinor field
    size_t rhs_stride;            // bytes of one right-hand side of a spinor field
    int parity0;                  // first output parity (blockIdx.z adds 0 or 1)
    int nrhs;
    int rhs_per_block;
    double a, b;
    // fused |out|^2 reduction (when launched with red = true)
    double *partials;             // [nrhs][nblocks]
    unsigned *counters;           // one per right-hand-side group, zero between launches
    double *result;               // [nrhs] sums (when state == nullptr)
    CgState *state;               // solver mode: skips finished rows; with red, sets pq and alpha
    int filter_ru;                // with state: compute only rows with a pending reliable update
};

int default_dslash_block(int prec, int rhs_per_block);
cudaError_t launch_dslash(int prec, int recon, const DslashArgs &A, int nparity, bool dagger, bool xpay,
                          bool red, int block_x, cudaStream_t s);

// ---------------------------------------------------------------- packing --
cudaError_t launch_pack_gauge(int prec, int recon, const Geom &g, void *packed, const void *canon,
                              cudaStream_t s);
cudaError_t launch_pack_spinor(int prec, const Geom &g, void *packed, const void *canon, int nrhs,
                               int parity_mask, cudaStream_t s);
cudaError_t launch_unpack_spinor(int prec, const Geom &g, void *canon, const void *packed, int nrhs,
                                 int parity_mask, cudaStream_t s);

// ------------------------------------------------------------ CG kernels --
// Vector arguments address a field of `nparity` parity blocks starting at the
// given pointer (right-hand side 0); rhs_stride/parity_stride in bytes per
// precision of that vector.
struct VecRef {
    void *ptr;
    int prec;
    size_t parity_stride;
    size_t rhs_stride;
};

struct BlasDims {
    int vh;
    int nparity;   // 1 (even-odd) or 2 (whole lattice)
    int nrhs;
};

// x += alpha p; r -= alpha q; rho_new = |r|^2; decides reliable update / stop.
cudaError_t launch_cg_update_xr(const BlasDims &d, VecRef x, VecRef r, VecRef p, VecRef q, CgState *st,
                                double *partials, unsigned *counters, cudaStream_t s);
// p = r + (rho_new / rho) p for rows not done.
cudaError_t launch_cg_update_p(const BlasDims &d, VecRef p, VecRef r, CgState *st, bool only_ru_rows,
                               cudaStream_t s);
// x_hi += x_lo; x_lo = 0 (rows with a pending reliable update, or all rows if force).
cudaError_t launch_ru_accumulate(const BlasDims &d, VecRef xhi, VecRef xlo, CgState *st, bool force,
                                 cudaStream_t s);
// r_hi = b - Ax; r_lo = r_hi; (init: p = r_lo); rho_new = r2_last = |r_hi|^2; convergence.
cudaError_t launch_ru_residual(const BlasDims &d, VecRef rhi, VecRef b, VecRef ax, VecRef rlo, VecRef p,
                               CgState *st, bool force, bool init, double *partials, unsigned *counters,
                               cudaStream_t s);
// st.b2 = |b|^2 and st.tol2 = tol^2 |b|^2.
cudaError_t launch_init_norms(const BlasDims &d, VecRef b, CgState *st, double *partials, unsigned *counters,
                              cudaStream_t s);
// dst = src with precision conversion (both VecRefs of the same shape).
cudaError_t launch_convert(const BlasDims &d, VecRef dst, VecRef src, cudaStream_t s);
// ||v||^2 per right-hand side into out[rhs] (FP64 accumulation).
cudaError_t launch_norm2(const BlasDims &d, VecRef v, double *out, double *partials, unsigned *counters,
                         cudaStream_t s);
// dst = a*x + b*y per right-hand side, any precisions.
cudaError_t launch_axpby(const BlasDims &d, VecRef dst, double a, VecRef x, double b, VecRef y, cudaStream_t s);

// ----------------------------------------------------------------- force --
cudaError_t launch_force(const Geom &g, double kappa, const void *links_f64, int recon, double *force,
                         const void *X, const void *Y, cudaStream_t s);
cudaError_t launch_link_grad(const Geom &g, double kappa, void *grad, const void *psi, const void *gy,
                             cudaStream_t s);

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
    int recon[3] = {12, 12, 12};
    size_t link_parity_bytes[3] = {0, 0, 0};
    // workspace slots: each a device buffer reused across calls
    static constexpr int kSlots = 24;
    void *slot[kSlots] = {};
    size_t slot_bytes[kSlots] = {};
    double *partials = nullptr;
    size_t partials_count = 0;
    unsigned *counters = nullptr;
    size_t counters_count = 0;
    cola::CgState *states = nullptr;   // device
    cola::CgState *h_states = nullptr; // pinned host mirror
    int states_count = 0;
};

namespace cola {
// Device buffer of at least `bytes` in workspace slot `k` (grown if needed).
cola_status ws_slot(cola_gauge g, int k, size_t bytes, void **out);
// Reduction scratch for up to `nrows` rows of `nblocks` partials.
cola_status ws_reduce(cola_gauge g, size_t nrows, size_t nblocks);
cola_status ws_states(cola_gauge g, int n);

DslashArgs make_dslash_args(cola_gauge g, int prec, void *out, const void *in, const void *xin, int nrhs,
                            int parity0, double a, double b);
// out = Mdag M in (op EO: Mhat on even halves; op FULL: D).  t and mp are
// full-field temporaries of the same precision.  With st != nullptr the
// first xpay apply reduces |M in|^2 into st (pq, alpha), and rows are
// filtered by st (filter_ru: only rows with a pending reliable update).
cola_status apply_mdagm(cola_gauge g, int prec, int op, void *out, const void *in, void *t, void *mp, int nrhs,
                        CgState *st, bool filter_ru, bool reduce, cudaStream_t s);
cola_status cuda_check(cudaError_t e, const char *what);
}  // namespace cola
