// C ABI entry points: argument checks, gauge handles, workspace, and the
// operator compositions (D, Mhat, their normal operators) built from the
// hopping kernel.
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cola_impl.h"

namespace cola {

bool log_enabled() {
    static const bool on = [] {
        const char *e = getenv("COLA_LOG");
        return e && e[0] && e[0] != '0';
    }();
    return on;
}

void log_line(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    fprintf(stderr, "cola: %s\n", buf);
}

TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

#ifdef COLA_BOUNDS
// readers of the per-translation-unit bounds counters, registered at load time
static std::vector<BoundsReader> &bounds_readers() {
    static std::vector<BoundsReader> r;
    return r;
}
bool register_bounds_reader(BoundsReader r) {
    bounds_readers().push_back(r);
    return true;
}
#endif

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

cola_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return COLA_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? COLA_ERR_NOMEM : COLA_ERR_CUDA;
}

#define COLA_TRY(expr)                       \
    do {                                     \
        cola_status _st = (expr);            \
        if (_st != COLA_OK) return _st;      \
    } while (0)
#define COLA_CUDA(expr, what) COLA_TRY(cuda_check((expr), what))

static cola_status arg_error(const std::string &msg) {
    set_error(msg);
    return COLA_ERR_ARG;
}

static cola_status check_lattice(const cola_lattice *lat) {
    if (!lat) return arg_error("lattice is null");
    long long v = 1;
    for (int m = 0; m < 4; ++m) {
        if (lat->dims[m] < 2 || lat->dims[m] % 2)
            return arg_error("lattice extents must be even and >= 2 (dims[" + std::to_string(m) +
                             "] = " + std::to_string(lat->dims[m]) + ")");
        v *= lat->dims[m];
    }
    if (v > (1ll << 30)) return arg_error("lattice volume above 2^30 sites");
    if (!std::isfinite(lat->kappa)) return arg_error("kappa is not finite");
    for (int m = 0; m < 4; ++m)
        if (!std::isfinite(lat->bc[m][0]) || !std::isfinite(lat->bc[m][1]))
            return arg_error("boundary phase is not finite");
    return COLA_OK;
}

static Geom make_geom(const cola_lattice &lat) {
    Geom g;
    for (int m = 0; m < 4; ++m) g.L[m] = lat.dims[m];
    g.Lxh = g.L[0] / 2;
    g.V = g.L[0] * g.L[1] * g.L[2] * g.L[3];
    g.Vh = g.V / 2;
    g.stride[0] = 1;
    g.stride[1] = g.Lxh;
    g.stride[2] = g.Lxh * g.L[1];
    g.stride[3] = g.Lxh * g.L[1] * g.L[2];
    for (int m = 0; m < 4; ++m) {
        g.bc[m][0] = lat.bc[m][0];
        g.bc[m][1] = lat.bc[m][1];
        g.bc_trivial[m] = (lat.bc[m][0] == 1.0 && lat.bc[m][1] == 0.0);
    }
    g.div_xh = make_fastdiv(g.Lxh);
    g.div_y = make_fastdiv(g.L[1]);
    g.div_z = make_fastdiv(g.L[2]);
    return g;
}

static cola_status check_prec(cola_gauge g, int prec) {
    if (prec < 0 || prec > 2) return arg_error("precision must be COLA_F64, COLA_F32 or COLA_F16");
    if (!g->links[prec]) {
        set_error("gauge handle holds no links of precision " + std::to_string(prec));
        return COLA_ERR_UNSUPPORTED;
    }
    return COLA_OK;
}

cola_status ws_slot(cola_gauge g, int k, size_t bytes, void **out) {
    if (g->slot_bytes[k] < bytes) {
        if (g->slot[k]) cudaFree(g->slot[k]);
        g->slot[k] = nullptr;
        g->slot_bytes[k] = 0;
        COLA_CUDA(cudaMalloc(&g->slot[k], bytes), "workspace allocation");
        g->slot_bytes[k] = bytes;
    }
    *out = g->slot[k];
    return COLA_OK;
}

cola_status ws_reduce(cola_gauge g, size_t nrows, size_t pstride) {
    const size_t need = nrows * pstride;
    if (g->partials_count < need) {
        if (g->partials) cudaFree(g->partials);
        g->partials = nullptr;
        g->partials_count = 0;
        COLA_CUDA(cudaMalloc(&g->partials, need * sizeof(double)), "reduction scratch");
        g->partials_count = need;
    }
    return COLA_OK;
}

cola_status ws_states(cola_gauge g, int n) {
    if (g->states_count < n) {
        if (g->states) cudaFree(g->states);
        if (g->h_states) cudaFreeHost(g->h_states);
        g->states = nullptr;
        g->h_states = nullptr;
        g->states_count = 0;
        COLA_CUDA(cudaMalloc(&g->states, n * sizeof(CgState)), "solver state");
        COLA_CUDA(cudaMallocHost(&g->h_states, n * sizeof(CgState)), "solver state (host)");
        g->states_count = n;
    }
    return COLA_OK;
}

static int rhs_per_block_for(int nrhs) {
    if (nrhs <= 1) return 1;
    if (nrhs <= 4) return nrhs;
    return 4;
}

DslashLat make_dslash_lat(cola_gauge g, int prec, void *out, const void *in, const void *xin, double a, double b,
                          int row0) {
    DslashLat L;
    std::memset(&L, 0, sizeof(L));
    L.g = g->geom;
    L.links = g->links[prec];
    L.link_parity_stride = g->link_parity_bytes[prec];
    L.link_dir_stride = link_dir_bytes(prec, g->recon[prec], g->geom.Vh);
    L.out = out;
    L.in = in;
    L.xin = xin;
    L.parity_stride = spinor_parity_bytes(prec, g->geom.Vh);
    L.rhs_stride = 2 * L.parity_stride;
    L.a = a;
    L.b = b;
    L.row0 = row0;
    return L;
}

static DslashArgs empty_args(int nrhs, int parity0) {
    DslashArgs A;
    std::memset(&A, 0, sizeof(A));
    A.nrhs = nrhs;
    A.rhs_per_block = rhs_per_block_for(nrhs);
    A.parity0 = parity0;
    return A;
}

DslashArgs make_dslash_args(cola_gauge g, int prec, void *out, const void *in, const void *xin, int nrhs,
                            int parity0, double a, double b) {
    DslashArgs A = empty_args(nrhs, parity0);
    A.nlat = 1;
    A.lat[0] = make_dslash_lat(g, prec, out, in, xin, a, b, 0);
    return A;
}

cola_status dslash_launch(cola_gauge owner, int prec, DslashArgs &A, int nparity, bool dagger, int epi,
                          cudaStream_t s) {
    return cuda_check(launch_dslash(prec, owner->recon[prec], A, nparity, dagger, epi, 0, s), "dslash launch");
}

// With a clover term (every lattice of the batch has one, or none does):
//   Mhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe,  D = A - kappa H,
// the A_oo^-1 riding on the odd-parity hops (EPI_CLOVER_INV) and A on the
// xpay term (EPI_CLOVER_X); the sequence of launches is the same.
cola_status apply_mdagm_batch(int nlat, const OpLat *L, int prec, int op, int nrhs, CgState *st, bool filter_ru,
                              cudaStream_t s, double *red, int red_stride, int *red_nb) {
    cola_gauge owner = L[0].g;
    const bool clv = owner->csw != 0.0;
    const int epi_x = clv ? EPI_CLOVER_X : EPI_XPAY;
    const int epi_h = clv ? EPI_CLOVER_INV : EPI_HOP;
    auto batch = [&](int parity0, double a_coef, bool use_xin, int which) {
        // which: 0 in->t, 1 t->mp (xin = in), 2 mp->t, 3 t->out (xin = mp); full: 4 in->mp, 5 mp->out
        DslashArgs A = empty_args(nrhs, parity0);
        A.nlat = nlat;
        A.state = st;
        A.filter_ru = filter_ru;
        for (int l = 0; l < nlat; ++l) {
            const OpLat &o = L[l];
            const double k = o.g->lat.kappa;
            const double b = which >= 4 ? -k : (which == 1 || which == 3) ? -k * k : 1.0;
            void *out = which == 0 || which == 2 ? o.t : which == 1 || which == 4 ? o.mp : o.out;
            const void *in = which == 0 || which == 4 ? o.in : which == 1 || which == 3 ? o.t : o.mp;
            const void *xin = !use_xin ? nullptr : (which == 1 || which == 4) ? o.in : o.mp;
            A.lat[l] = make_dslash_lat(o.g, prec, out, in, xin, a_coef, b, o.row0);
            if (clv) set_clover(A.lat[l], o.g, prec, !use_xin);
        }
        return A;
    };
    if (op == COLA_OP_EO) {
        DslashArgs A = batch(1, 0.0, false, 0);
        COLA_TRY(dslash_launch(owner, prec, A, 1, false, epi_h, s));
        A = batch(0, 1.0, true, 1);
        COLA_TRY(dslash_launch(owner, prec, A, 1, false, epi_x, s));
        A = batch(1, 0.0, false, 2);
        COLA_TRY(dslash_launch(owner, prec, A, 1, true, epi_h, s));
        A = batch(0, 1.0, true, 3);  // xin = Mhat in: the fused reduction gives |Mhat in|^2
        A.red = red;
        A.red_stride = red_stride;
        COLA_TRY(dslash_launch(owner, prec, A, 1, true, epi_x, s));
        if (red_nb)
            for (int l = 0; l < nlat; ++l) red_nb[l] = A.lat[l].nblocks;
        return COLA_OK;
    }
    DslashArgs A = batch(0, 1.0, true, 4);
    COLA_TRY(dslash_launch(owner, prec, A, 2, false, epi_x, s));
    A = batch(0, 1.0, true, 5);  // xin = D in: the fused reduction gives |D in|^2
    A.red = red;
    A.red_stride = red_stride;
    COLA_TRY(dslash_launch(owner, prec, A, 2, true, epi_x, s));
    if (red_nb)
        for (int l = 0; l < nlat; ++l) red_nb[l] = 2 * A.lat[l].nblocks;
    return COLA_OK;
}

cola_status apply_mdagm(cola_gauge g, int prec, int op, void *out, const void *in, void *t, void *mp, int nrhs,
                        CgState *st, bool filter_ru, cudaStream_t s) {
    OpLat L = {g, out, in, t, mp, 0};
    return apply_mdagm_batch(1, &L, prec, op, nrhs, st, filter_ru, s);
}

}  // namespace cola

using namespace cola;

static cola_status check_rhs(int nrhs) {
    if (nrhs < 1 || nrhs > 65535) return arg_error("nrhs must be in 1..65535");
    return COLA_OK;
}

extern "C" {

const char *cola_last_error(void) { return g_last_error.c_str(); }

cola_status cola_debug_bounds(unsigned long long *count, int *first_line, int reset) {
    if (!count || !first_line) return arg_error("null argument to cola_debug_bounds");
    *count = 0;
    *first_line = 0;
#ifdef COLA_BOUNDS
    COLA_CUDA(cudaDeviceSynchronize(), "bounds counters");
    for (BoundsReader r : bounds_readers()) {
        unsigned long long c = 0;
        int line = 0;
        COLA_CUDA(r(&c, &line, reset != 0), "bounds counters");
        if (c && !*first_line) *first_line = line;
        *count += c;
    }
    return COLA_OK;
#else
    (void)reset;
    set_error("libcola was built without COLA_BOUNDS: no bounds checks to report");
    return COLA_ERR_UNSUPPORTED;
#endif
}

size_t cola_spinor_bytes(const cola_lattice *lat, cola_prec prec, int nrhs) {
    if (check_lattice(lat) != COLA_OK || prec < 0 || prec > 2 || nrhs < 1) return 0;
    const size_t vh = (size_t)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3] / 2;
    return 2 * spinor_parity_bytes(prec, (int)vh) * (size_t)nrhs;
}

cola_status cola_gauge_create(const cola_lattice *lat, const void *links_dev, const cola_gauge_opts *opts,
                              cudaStream_t stream, cola_gauge *out) {
    TraceRange trace_("cola_gauge_create");
    COLA_TRY(check_lattice(lat));
    if (!links_dev || !opts || !out) return arg_error("null argument to cola_gauge_create");
    if ((opts->prec_mask & 7u) == 0 || (opts->prec_mask & ~7u))
        return arg_error("prec_mask must request at least one of F64/F32/F16 and nothing else");
    for (int p = 0; p < 3; ++p)
        if ((opts->prec_mask >> p) & 1)
            if (opts->recon[p] != 12 && opts->recon[p] != 18) return arg_error("recon must be 12 or 18");
    *out = nullptr;
    cola_gauge g = new cola_gauge_s();
    g->lat = *lat;
    g->geom = make_geom(*lat);
    cudaGetDevice(&g->device);
    for (int p = 0; p < 3; ++p) {
        if (!((opts->prec_mask >> p) & 1)) continue;
        g->recon[p] = opts->recon[p];
        g->link_parity_bytes[p] = 4 * link_dir_bytes(p, g->recon[p], g->geom.Vh);
        cola_status st = cuda_check(cudaMalloc(&g->links[p], 2 * g->link_parity_bytes[p]), "link allocation");
        if (st == COLA_OK) st = cuda_check(launch_pack_gauge(p, g->recon[p], g->geom, g->links[p], links_dev, stream),
                                           "link packing");
        if (st != COLA_OK) {
            cola_gauge_destroy(g);
            return st;
        }
    }
    *out = g;
    return COLA_OK;
}

cola_status cola_gauge_update(cola_gauge g, const void *links_dev, cudaStream_t stream) {
    TraceRange trace_("cola_gauge_update");
    if (!g || !links_dev) return arg_error("null argument to cola_gauge_update");
    for (int p = 0; p < 3; ++p)
        if (g->links[p])
            COLA_TRY(cuda_check(launch_pack_gauge(p, g->recon[p], g->geom, g->links[p], links_dev, stream),
                                "link packing"));
    if (g->csw != 0.0) return clover_rebuild(g, stream);
    return COLA_OK;
}

cola_status cola_clover_attach(cola_gauge g, double csw, cudaStream_t stream) {
    TraceRange trace_("cola_clover_attach");
    if (!g) return arg_error("null gauge handle");
    if (!std::isfinite(csw)) return arg_error("c_sw is not finite");
    if (csw == 0.0) {
        cudaStreamSynchronize(stream);
        clover_free(g);
        return COLA_OK;
    }
    g->csw = csw;
    cola_status st = clover_rebuild(g, stream);
    if (st != COLA_OK) {
        const std::string msg = cola_last_error();
        cudaStreamSynchronize(stream);
        clover_free(g);
        set_error(msg);
    }
    return st;
}

double cola_clover_csw(cola_gauge g) { return g ? g->csw : 0.0; }

cola_status cola_clover_apply(cola_gauge g, void *out, const void *in, int parity, int inverse, cola_prec prec,
                              int nrhs, cudaStream_t stream) {
    TraceRange trace_("cola_clover_apply");
    if (!g || !out || !in) return arg_error("null argument to cola_clover_apply");
    if (parity < 0 || parity > 2) return arg_error("parity must be 0, 1 or 2");
    COLA_TRY(check_prec(g, prec));
    COLA_TRY(check_rhs(nrhs));
    if (g->csw == 0.0) {
        set_error("no clover term is attached to this gauge handle");
        return COLA_ERR_UNSUPPORTED;
    }
    const void *c = inverse ? g->clover_inv[prec] : g->clover[prec];
    return cuda_check(launch_clover_apply(prec, g->geom, c, out, in, nrhs, parity == 2 ? 3 : 1 << parity, stream),
                      "clover apply");
}

cola_status cola_gauge_destroy(cola_gauge g) {
    if (!g) return COLA_OK;
    cudaDeviceSynchronize();
    for (int p = 0; p < 3; ++p)
        if (g->links[p]) cudaFree(g->links[p]);
    clover_free(g);
    for (int k = 0; k < cola_gauge_s::kSlots; ++k)
        if (g->slot[k]) cudaFree(g->slot[k]);
    if (g->partials) cudaFree(g->partials);
    if (g->states) cudaFree(g->states);
    if (g->h_states) cudaFreeHost(g->h_states);
    if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
    delete g;
    return COLA_OK;
}


cola_status cola_spinor_pack(cola_gauge g, void *packed_dev, const void *canon_dev, cola_prec prec, int nrhs,
                             cudaStream_t stream) {
    TraceRange trace_("cola_spinor_pack");
    if (!g || !packed_dev || !canon_dev) return arg_error("null argument to cola_spinor_pack");
    if (prec < 0 || prec > 2) return arg_error("bad precision");
    COLA_TRY(check_rhs(nrhs));
    return cuda_check(launch_pack_spinor(prec, g->geom, packed_dev, canon_dev, nrhs, 3, stream), "spinor packing");
}

cola_status cola_spinor_unpack(cola_gauge g, void *canon_dev, const void *packed_dev, cola_prec prec, int nrhs,
                               cudaStream_t stream) {
    TraceRange trace_("cola_spinor_unpack");
    if (!g || !packed_dev || !canon_dev) return arg_error("null argument to cola_spinor_unpack");
    if (prec < 0 || prec > 2) return arg_error("bad precision");
    COLA_TRY(check_rhs(nrhs));
    return cuda_check(launch_unpack_spinor(prec, g->geom, canon_dev, packed_dev, nrhs, 3, stream),
                      "spinor unpacking");
}

cola_status cola_dslash_apply(cola_gauge g, void *out, const void *in, const void *in_self, double a, double b,
                              int parity, int dagger, cola_prec prec, int nrhs, cudaStream_t stream) {
    TraceRange trace_("cola_dslash_apply");
    if (!g || !out || !in) return arg_error("null argument to cola_dslash_apply");
    if (parity < 0 || parity > 2) return arg_error("parity must be 0, 1 or 2");
    if (a != 0.0 && !in_self) return arg_error("in_self is null but a != 0");
    if (out == in) return arg_error("out must not alias in");
    COLA_TRY(check_prec(g, prec));
    COLA_TRY(check_rhs(nrhs));
    const bool xpay = a != 0.0;
    DslashArgs A = make_dslash_args(g, prec, out, in, xpay ? in_self : nullptr, nrhs, parity == 2 ? 0 : parity, a, b);
    return dslash_launch(g, prec, A, parity == 2 ? 2 : 1, dagger != 0, xpay, stream);
}

cola_status cola_dirac_apply(cola_gauge g, void *out, const void *in, int dagger, cola_prec prec, int nrhs,
                             cudaStream_t stream) {
    TraceRange trace_("cola_dirac_apply");
    if (!g || !out || !in) return arg_error("null argument to cola_dirac_apply");
    if (out == in) return arg_error("out must not alias in");
    COLA_TRY(check_prec(g, prec));
    COLA_TRY(check_rhs(nrhs));
    DslashArgs A = make_dslash_args(g, prec, out, in, in, nrhs, 0, 1.0, -g->lat.kappa);
    if (g->csw != 0.0) set_clover(A.lat[0], g, prec, false);
    return dslash_launch(g, prec, A, 2, dagger != 0, g->csw != 0.0 ? EPI_CLOVER_X : EPI_XPAY, stream);
}

cola_status cola_mdagm_apply(cola_gauge g, void *out, const void *in, int op, cola_prec prec, int nrhs,
                             cudaStream_t stream) {
    TraceRange trace_("cola_mdagm_apply");
    if (!g || !out || !in) return arg_error("null argument to cola_mdagm_apply");
    if (op != COLA_OP_FULL && op != COLA_OP_EO) return arg_error("op must be COLA_OP_FULL or COLA_OP_EO");
    if (out == in) return arg_error("out must not alias in");
    COLA_TRY(check_prec(g, prec));
    COLA_TRY(check_rhs(nrhs));
    const size_t bytes = 2 * spinor_parity_bytes(prec, g->geom.Vh) * (size_t)nrhs;
    void *t, *mp;
    COLA_TRY(ws_slot(g, 0, bytes, &t));
    COLA_TRY(ws_slot(g, 1, bytes, &mp));
    return apply_mdagm(g, prec, op, out, in, t, mp, nrhs, nullptr, false, stream);
}

cola_status cola_fermion_force(cola_gauge g, double *force_dev, const void *X_dev, const void *Y_dev,
                               cudaStream_t stream) {
    TraceRange trace_("cola_fermion_force");
    if (!g || !force_dev || !X_dev || !Y_dev) return arg_error("null argument to cola_fermion_force");
    COLA_TRY(check_prec(g, COLA_F64));
    COLA_CUDA(launch_force(g->geom, g->lat.kappa, g->links[COLA_F64], g->recon[COLA_F64], force_dev, X_dev, Y_dev,
                           stream),
              "force launch");
    if (g->csw == 0.0) return COLA_OK;
    void *scratch;
    COLA_TRY(ws_slot(g, cola_gauge_s::kSlotCloverForce, clover_force_scratch_bytes(g->geom), &scratch));
    return cuda_check(launch_clover_force(g->geom, g->links[COLA_F64], g->recon[COLA_F64], g->lat.kappa, g->csw,
                                          X_dev, Y_dev, force_dev, 1.0, true, scratch, stream),
                      "clover force launch");
}

cola_status cola_dirac_link_grad(cola_gauge g, void *grad_links_dev, const void *psi_dev, const void *gy_dev,
                                 cudaStream_t stream) {
    TraceRange trace_("cola_dirac_link_grad");
    if (!g || !grad_links_dev || !psi_dev || !gy_dev) return arg_error("null argument to cola_dirac_link_grad");
    COLA_CUDA(launch_link_grad(g->geom, g->lat.kappa, grad_links_dev, psi_dev, gy_dev, stream),
              "link gradient launch");
    if (g->csw == 0.0) return COLA_OK;
    COLA_TRY(check_prec(g, COLA_F64));
    void *scratch;
    COLA_TRY(ws_slot(g, cola_gauge_s::kSlotCloverForce, clover_force_scratch_bytes(g->geom), &scratch));
    return cuda_check(launch_clover_link_grad(g->geom, g->links[COLA_F64], g->recon[COLA_F64], g->lat.kappa, g->csw,
                                              psi_dev, gy_dev, grad_links_dev, scratch, stream),
                      "clover link gradient launch");
}

}  // extern "C"
