// Conjugate-gradient solver with reliable updates (mixed precision) and
// multiple right-hand sides.
//
// The paper's GPU inverter is a conjugate-gradient solver run in mixed
// precision, 32-bit inner iterations inside a 64-bit outer solve (Fig. 2
// discussion, citing Clark et al.).  The inner iterations here keep p, q and
// r in the storage precision (FP32 or FP16 with a per-site scale, FP32
// arithmetic) and x_lo in FP32; b, x_hi and r_hi stay in FP64.  Whenever the
// inner residual falls below delta times the FP64 residual of the last
// update (or reaches the target), x_hi += x_lo and r_hi = b - A x_hi is
// recomputed in FP64 with the FP64 links (a reliable update); the search
// direction p is kept.  Convergence is declared only on that FP64 true
// residual.  With inner = FP64 the same loop is the plain FP64 CG, whose
// "reliable update" is the true-residual confirmation at convergence.
//
// Per iteration: four hopping-term launches for A = Mhat^dag Mhat, one
// reduction of <p, Ap> = |Mhat p|^2 that sets alpha, one fused x/r update
// that reduces |r|^2 and decides, optionally the FP64 update, and the p
// update.  All scalars stay on the device.  Two drivers run the
// loop: a host loop that reads the per-right-hand-side state after each
// update, or one CUDA graph whose while/if conditional nodes are set by a
// one-thread control kernel, so that a whole solve is a single launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <utility>
#include <vector>

#include "cola_impl.h"

namespace cola {

#define COLA_TRY(expr)                       \
    do {                                     \
        cola_status _st = (expr);            \
        if (_st != COLA_OK) return _st;      \
    } while (0)
#define COLA_CUDA(expr, what) COLA_TRY(cuda_check((expr), what))

// One-thread control: any row due for a reliable update -> the "if" node;
// any row still running -> the "while" node.
__global__ void control_ru_kernel(const CgState *st, int nrhs, cudaGraphConditionalHandle h_ru) {
    int any = 0;
    for (int r = 0; r < nrhs; ++r) any |= (st[r].ru && !st[r].done);
    cudaGraphSetConditional(h_ru, any ? 1u : 0u);
}
__global__ void control_loop_kernel(const CgState *st, int nrhs, cudaGraphConditionalHandle h_loop) {
    int running = 0;
    for (int r = 0; r < nrhs; ++r) running |= !st[r].done;
    cudaGraphSetConditional(h_loop, running ? 1u : 0u);
}

namespace {

enum Slot {
    S_T = 0, S_MP = 1,              // low-precision temporaries of the operator
    S_P = 2, S_Q = 3, S_RLO = 4, S_XLO = 5,
    S_B = 6, S_XHI = 7, S_RHI = 8, S_AX = 9, S_T64 = 10, S_MP64 = 11, S_BORIG = 12, S_NORMS = 13, S_FLAGS = 14,
};

// Vectors of one lattice of the batch (full packed fields x nrhs, held in
// that lattice's gauge-handle workspace).
struct LatCtx {
    cola_gauge g;
    int row0;
    void *t, *mp, *p, *q, *rlo, *xlo;
    void *b, *xhi, *rhi, *ax, *t64, *mp64, *borig;
};

struct SolveCtx {
    int nlat;
    LatCtx lat[kMaxBatch];
    cola_gauge owner;  // holds states and reduction scratch
    int prec, xprec, op, nrhs, nparity;
    int fuse_pq;       // <p, Ap> from the operator's last hopping launch (no shifted rows)
    int red_stride;    // row stride of the reduction scratch
};

enum VecId { V_T, V_MP, V_P, V_Q, V_RLO, V_XLO, V_B, V_XHI, V_RHI, V_AX, V_T64, V_MP64, V_BORIG };

void *vec(const LatCtx &L, VecId v) {
    switch (v) {
        case V_T: return L.t;
        case V_MP: return L.mp;
        case V_P: return L.p;
        case V_Q: return L.q;
        case V_RLO: return L.rlo;
        case V_XLO: return L.xlo;
        case V_B: return L.b;
        case V_XHI: return L.xhi;
        case V_RHI: return L.rhi;
        case V_AX: return L.ax;
        case V_T64: return L.t64;
        case V_MP64: return L.mp64;
        default: return L.borig;
    }
}

// Batched vector-kernel arguments over every lattice, slots from `ids`.
BlasArgs blas(const SolveCtx &c, std::initializer_list<std::pair<VecId, int>> ids, int nparity = -1) {
    BlasArgs B;
    std::memset(&B, 0, sizeof(B));
    B.nlat = c.nlat;
    B.nparity = nparity < 0 ? c.nparity : nparity;
    B.nrhs = c.nrhs;
    int k = 0;
    for (auto &id : ids) B.prec[k++] = id.second;
    for (int l = 0; l < c.nlat; ++l) {
        B.lat[l].vh = c.lat[l].g->geom.Vh;
        B.lat[l].row0 = c.lat[l].row0;
        k = 0;
        for (auto &id : ids) B.lat[l].v[k++] = vec(c.lat[l], id.first);
    }
    B.state = c.owner->states;
    B.partials = c.owner->partials;
    B.pstride = blas_max_blocks(B);
    return B;
}

cola_status mdagm(const SolveCtx &c, int prec, VecId out, VecId in, VecId t, VecId mp, CgState *st, bool filter_ru,
                  cudaStream_t s, double *red = nullptr, int *red_nb = nullptr) {
    OpLat L[kMaxBatch];
    for (int l = 0; l < c.nlat; ++l)
        L[l] = {c.lat[l].g, vec(c.lat[l], out), vec(c.lat[l], in), vec(c.lat[l], t), vec(c.lat[l], mp), c.lat[l].row0};
    return apply_mdagm_batch(c.nlat, L, prec, c.op, c.nrhs, st, filter_ru, s, red, c.red_stride, red_nb);
}

cola_status ru_block(const SolveCtx &c, cudaStream_t s) {
    BlasArgs B = blas(c, {{V_XHI, COLA_F64}, {V_XLO, c.xprec}});
    COLA_CUDA(launch_ru_accumulate(B, false, s), "reliable update (accumulate)");
    COLA_TRY(mdagm(c, COLA_F64, V_AX, V_XHI, V_T64, V_MP64, c.owner->states, true, s));
    B = blas(c, {{V_RHI, COLA_F64}, {V_B, COLA_F64}, {V_AX, COLA_F64}, {V_RLO, c.prec}, {V_P, c.prec},
                 {V_XHI, COLA_F64}});
    COLA_CUDA(launch_ru_residual(B, s), "reliable update (residual)");
    return COLA_OK;
}

cola_status iter_head(const SolveCtx &c, cudaStream_t s) {
    BlasArgs P = blas(c, {{V_MP, c.prec}, {V_P, c.prec}});  // <p, A p> = |M p|^2 (+ sigma |p|^2), alpha
    if (c.fuse_pq) {
        // the operator's last hopping launch reads M p as its xpay input and
        // leaves the block partials of |M p|^2; the finishing kernel sums them
        int nb[kMaxBatch];
        COLA_TRY(mdagm(c, c.prec, V_Q, V_P, V_T, V_MP, c.owner->states, false, s, c.owner->partials, nb));
        for (int l = 0; l < c.nlat; ++l) P.lat[l].nblocks = nb[l];
        P.pstride = c.red_stride;
        COLA_CUDA(launch_finish_pq(P, s), "cg <p, Ap>");
    } else {
        COLA_TRY(mdagm(c, c.prec, V_Q, V_P, V_T, V_MP, c.owner->states, false, s));
        COLA_CUDA(launch_cg_pq(P, s), "cg <p, Ap>");
    }
    BlasArgs B = blas(c, {{V_XLO, c.xprec}, {V_RLO, c.prec}, {V_P, c.prec}, {V_Q, c.prec}});
    COLA_CUDA(launch_cg_update_xr(B, s), "cg update x, r");
    return COLA_OK;
}

cola_status iter_tail(const SolveCtx &c, cudaStream_t s) {
    BlasArgs B = blas(c, {{V_P, c.prec}, {V_RLO, c.prec}});
    COLA_CUDA(launch_cg_update_p(B, s), "cg update p");
    return COLA_OK;
}

int total_rows(const SolveCtx &c) { return c.nlat * c.nrhs; }

cola_status read_states(const SolveCtx &c, cudaStream_t s) {
    COLA_CUDA(cudaMemcpyAsync(c.owner->h_states, c.owner->states, total_rows(c) * sizeof(CgState),
                              cudaMemcpyDeviceToHost, s),
              "state readback");
    COLA_CUDA(cudaStreamSynchronize(s), "solver synchronisation");
    return COLA_OK;
}

// Host-driven loop: one state readback per iteration.
cola_status run_host_loop(const SolveCtx &c, cudaStream_t s) {
    for (;;) {
        COLA_TRY(iter_head(c, s));
        COLA_TRY(read_states(c, s));
        bool any_ru = false, running = false;
        for (int r = 0; r < total_rows(c); ++r) {
            const CgState &st = c.owner->h_states[r];
            any_ru |= st.ru && !st.done;
        }
        if (any_ru) {
            COLA_TRY(ru_block(c, s));
            COLA_TRY(read_states(c, s));
        }
        for (int r = 0; r < total_rows(c); ++r) running |= !c.owner->h_states[r].done;
        if (!running) return COLA_OK;
        COLA_TRY(iter_tail(c, s));
    }
}

// Everything a captured solve graph depends on: the vectors and handles of
// every lattice, the solver's shape, and the state and reduction buffers.
std::vector<unsigned char> graph_key(const SolveCtx &c) {
    std::vector<unsigned char> k;
    auto put = [&k](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        k.insert(k.end(), b, b + n);
    };
    put(&c, sizeof(SolveCtx));  // zero-initialised, so padding compares equal
    void *extra[2] = {c.owner->states, c.owner->partials};
    put(extra, sizeof(extra));
    put(&c.owner->partials_count, sizeof(size_t));
    for (int l = 0; l < c.nlat; ++l) {  // the lattice data baked into every kernel argument
        const cola_gauge g = c.lat[l].g;
        put(&g->lat, sizeof(cola_lattice));
        put(g->links, sizeof(g->links));
        put(g->recon, sizeof(g->recon));
        put(&g->csw, sizeof(double));
        put(g->clover, sizeof(g->clover));
        put(g->clover_inv, sizeof(g->clover_inv));
    }
    return k;
}

// Whole loop as one graph: while (running) { head; if (ru) { ru_block } ; tail }.
// The instantiated graph is kept in the leading handle and launched again by
// later solves of the same configuration (HMC solves thousands of times).
cola_status run_graph_loop(const SolveCtx &c, cudaStream_t s) {
    std::vector<unsigned char> key = graph_key(c);
    if (c.owner->graph_exec && c.owner->graph_key == key) {
        COLA_CUDA(cudaGraphLaunch(c.owner->graph_exec, s), "graph launch");
        COLA_CUDA(cudaStreamSynchronize(s), "graph run");
        return read_states(c, s);
    }
    if (c.owner->graph_exec) {
        cudaGraphExecDestroy(c.owner->graph_exec);
        c.owner->graph_exec = nullptr;
        c.owner->graph_key.clear();
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    cola_status st = COLA_OK;
    const int nrows = total_rows(c);
    CgState *states = c.owner->states;
    auto fail = [&](cola_status e) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        return e;
    };
    if ((st = cuda_check(cudaGraphCreate(&graph, 0), "graph create")) != COLA_OK) return fail(st);
    cudaGraphConditionalHandle h_loop, h_ru;
    if ((st = cuda_check(cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault),
                         "graph conditional")) != COLA_OK)
        return fail(st);
    cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((st = cuda_check(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &wp), "graph while node")) != COLA_OK)
        return fail(st);
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if ((st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream")) != COLA_OK)
        return fail(st);
    if ((st = cuda_check(cudaGraphConditionalHandleCreate(&h_ru, body, 0, cudaGraphCondAssignDefault),
                         "graph conditional")) != COLA_OK)
        return fail(st);
    if ((st = cuda_check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                         "capture")) != COLA_OK)
        return fail(st);
    st = iter_head(c, cs);
    if (st == COLA_OK) {
        control_ru_kernel<<<1, 1, 0, cs>>>(states, nrows, h_ru);
        st = cuda_check(cudaGetLastError(), "control kernel");
    }
    cudaGraphNode_t ifnode = nullptr;
    cudaGraph_t ifbody = nullptr;
    if (st == COLA_OK) {
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edata = nullptr;
        size_t ndeps = 0;
        cudaGraph_t capg;
        st = cuda_check(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, &edata, &ndeps), "capture info");
        if (st == COLA_OK) {
            cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
            ip.conditional.handle = h_ru;
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            st = cuda_check(cudaGraphAddNode(&ifnode, capg, deps, edata, ndeps, &ip), "graph if node");
            if (st == COLA_OK) {
                ifbody = ip.conditional.phGraph_out[0];
                st = cuda_check(cudaStreamUpdateCaptureDependencies(cs, &ifnode, nullptr, 1,
                                                                    cudaStreamSetCaptureDependencies),
                                "capture dependencies");
            }
        }
    }
    if (st == COLA_OK) st = iter_tail(c, cs);
    if (st == COLA_OK) {
        control_loop_kernel<<<1, 1, 0, cs>>>(states, nrows, h_loop);
        st = cuda_check(cudaGetLastError(), "control kernel");
    }
    {
        cudaGraph_t out = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &out);
        if (st == COLA_OK) st = cuda_check(e, "end capture");
    }
    if (st != COLA_OK) return fail(st);
    if ((st = cuda_check(cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal),
                         "capture")) != COLA_OK)
        return fail(st);
    st = ru_block(c, cs);
    {
        cudaGraph_t out = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &out);
        if (st == COLA_OK) st = cuda_check(e, "end capture");
    }
    if (st != COLA_OK) return fail(st);
    if ((st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate")) != COLA_OK) return fail(st);
    if ((st = cuda_check(cudaGraphLaunch(exec, s), "graph launch")) != COLA_OK) return fail(st);
    if ((st = cuda_check(cudaStreamSynchronize(s), "graph run")) != COLA_OK) return fail(st);
    c.owner->graph_exec = exec;
    c.owner->graph_key = std::move(key);
    exec = nullptr;  // kept in the handle
    fail(COLA_OK);
    return read_states(c, s);
}

cola_status arg_error(const char *msg) {
    set_error(msg);
    return COLA_ERR_ARG;
}

cola_status check_params(const cola_solver_params *prm) {
    if (prm->op != COLA_OP_FULL && prm->op != COLA_OP_EO) return arg_error("op must be COLA_OP_FULL or COLA_OP_EO");
    if (prm->system != COLA_SYS_NORMAL && prm->system != COLA_SYS_DIRAC)
        return arg_error("system must be COLA_SYS_NORMAL or COLA_SYS_DIRAC");
    if (prm->inner < 0 || prm->inner > 2) return arg_error("inner precision must be F64, F32 or F16");
    if (prm->nrhs < 1 || prm->nrhs > 64) return arg_error("nrhs must be in 1..64");
    if (!(prm->tol > 0.0) || prm->max_iter < 0) return arg_error("tol must be > 0 and max_iter >= 0");
    if (prm->inner != COLA_F64 && !(prm->delta > 0.0 && prm->delta < 1.0))
        return arg_error("delta must be in (0, 1) for a mixed-precision solve");
    return COLA_OK;
}

// Solve every lattice of the batch together: one launch per kernel per
// iteration covers all lattices and right-hand sides.
// shifts (host, nrhs entries, may be null): right-hand side r solves
// (A + shifts[r]) x = b (normal system only).  shared_b: bs[l] holds one field
// that every right-hand side of lattice l solves with.
// row_tol / row_max_iter (host, one per row, may be null): per-row overrides
// of prm->tol and prm->max_iter for the CG's stopping test.
cola_status solve_batch_pass(int nlat, const cola_gauge *gs, void *const *xs, const void *const *bs,
                             const cola_solver_params *prm, cola_solve_info *info, cudaStream_t s,
                             const double *shifts, bool shared_b, const double *row_tol, const int *row_max_iter) {
    const auto t0 = std::chrono::steady_clock::now();
    COLA_TRY(check_params(prm));
    if (shifts && prm->system != COLA_SYS_NORMAL) return arg_error("shifted solves need the normal system");
    SolveCtx c;
    std::memset(&c, 0, sizeof(c));
    c.nlat = nlat;
    c.owner = gs[0];
    c.prec = prm->inner;
    c.xprec = prm->inner == COLA_F64 ? COLA_F64 : COLA_F32;
    c.op = prm->op;
    c.nrhs = prm->nrhs;
    c.nparity = prm->op == COLA_OP_EO ? 1 : 2;
    const bool dirac = prm->system == COLA_SYS_DIRAC;
    // D = A - kappa H with a clover term: every lattice of a batch has one, or none has
    const bool clv = gs[0]->csw != 0.0;
    const int epi_x = clv ? EPI_CLOVER_X : EPI_XPAY;
    const int epi_h = clv ? EPI_CLOVER_INV : EPI_HOP;
    int maxblocks = 0, nrows = nlat * c.nrhs;
    for (int l = 0; l < nlat; ++l) {
        cola_gauge g = gs[l];
        if (!g->links[COLA_F64]) {
            set_error("cola_cg_solve needs FP64 links in every gauge handle (reliable updates and residuals)");
            return COLA_ERR_UNSUPPORTED;
        }
        if (!g->links[c.prec]) {
            set_error("a gauge handle holds no links of the inner precision");
            return COLA_ERR_UNSUPPORTED;
        }
        if (g->recon[COLA_F64] != gs[0]->recon[COLA_F64] || g->recon[c.prec] != gs[0]->recon[c.prec])
            return arg_error("the gauge handles of a batch must use the same link reconstruction per precision");
        for (int m = 0; m < l; ++m)
            if (gs[m] == g) return arg_error("a gauge handle appears twice in the batch (use nrhs instead)");
        if ((g->csw != 0.0) != clv)
            return arg_error("either every gauge handle of a batch has a clover term or none has");
        const Geom &G = g->geom;
        LatCtx &L = c.lat[l];
        L.g = g;
        L.row0 = l * c.nrhs;
        const size_t lo = 2 * spinor_parity_bytes(c.prec, G.Vh) * c.nrhs;
        const size_t xb = 2 * spinor_parity_bytes(c.xprec, G.Vh) * c.nrhs;
        const size_t hi = 2 * spinor_parity_bytes(COLA_F64, G.Vh) * c.nrhs;
        COLA_TRY(ws_slot(g, S_T, lo, &L.t));
        COLA_TRY(ws_slot(g, S_MP, lo, &L.mp));
        COLA_TRY(ws_slot(g, S_P, lo, &L.p));
        COLA_TRY(ws_slot(g, S_Q, lo, &L.q));
        COLA_TRY(ws_slot(g, S_RLO, lo, &L.rlo));
        COLA_TRY(ws_slot(g, S_XLO, xb, &L.xlo));
        COLA_TRY(ws_slot(g, S_B, hi, &L.b));
        COLA_TRY(ws_slot(g, S_XHI, hi, &L.xhi));
        COLA_TRY(ws_slot(g, S_RHI, hi, &L.rhi));
        COLA_TRY(ws_slot(g, S_AX, hi, &L.ax));
        COLA_TRY(ws_slot(g, S_T64, hi, &L.t64));
        COLA_TRY(ws_slot(g, S_MP64, hi, &L.mp64));
        L.borig = nullptr;
        if (dirac) COLA_TRY(ws_slot(g, S_BORIG, hi, &L.borig));
        maxblocks = std::max(maxblocks, reduce_stride(G.Vh));
    }
    COLA_TRY(ws_reduce(c.owner, nrows, maxblocks));
    c.red_stride = maxblocks;
    c.fuse_pq = shifts == nullptr;
    COLA_TRY(ws_states(c.owner, nrows));
    CgState *hs = c.owner->h_states;

    // right-hand side of the CG system in b (packed FP64), initial guess in x_hi
    for (int l = 0; l < nlat; ++l) {
        LatCtx &L = c.lat[l];
        cola_gauge g = L.g;
        const Geom &G = g->geom;
        const double k = g->lat.kappa;
        if (!dirac) {
            const int pmask = prm->op == COLA_OP_EO ? 1 : 3;
            COLA_CUDA(launch_pack_spinor(COLA_F64, G, L.b, bs[l], shared_b ? 1 : c.nrhs, pmask, s), "pack b");
            const size_t hi1 = 2 * spinor_parity_bytes(COLA_F64, G.Vh);
            for (int r = 1; shared_b && r < c.nrhs; ++r)
                COLA_CUDA(cudaMemcpyAsync(static_cast<char *>(L.b) + r * hi1, L.b, hi1, cudaMemcpyDeviceToDevice, s),
                          "replicate b");
        } else {
            COLA_CUDA(launch_pack_spinor(COLA_F64, G, L.borig, bs[l], c.nrhs, 3, s), "pack b");
            if (prm->op == COLA_OP_EO) {
                // bhat_e = b_e + kappa H_eo A_oo^-1 b_o (into mp64);  b = Mhat^dag bhat
                // (without a clover term A = 1)
                const void *bo = L.borig;
                if (clv) {
                    COLA_CUDA(launch_clover_apply(COLA_F64, G, g->clover_inv[COLA_F64], L.t64, L.borig, c.nrhs, 2, s),
                              "A_oo^-1 b_o");
                    bo = L.t64;
                }
                DslashArgs A = make_dslash_args(g, COLA_F64, L.mp64, bo, L.borig, c.nrhs, 0, 1.0, k);
                COLA_TRY(dslash_launch(g, COLA_F64, A, 1, false, EPI_XPAY, s));
                A = make_dslash_args(g, COLA_F64, L.t64, L.mp64, nullptr, c.nrhs, 1, 0.0, 1.0);
                if (clv) set_clover(A.lat[0], g, COLA_F64, true);
                COLA_TRY(dslash_launch(g, COLA_F64, A, 1, true, epi_h, s));
                A = make_dslash_args(g, COLA_F64, L.b, L.t64, L.mp64, c.nrhs, 0, 1.0, -k * k);
                if (clv) set_clover(A.lat[0], g, COLA_F64, false);
                COLA_TRY(dslash_launch(g, COLA_F64, A, 1, true, epi_x, s));
            } else {
                DslashArgs A = make_dslash_args(g, COLA_F64, L.b, L.borig, L.borig, c.nrhs, 0, 1.0, -k);
                if (clv) set_clover(A.lat[0], g, COLA_F64, false);
                COLA_TRY(dslash_launch(g, COLA_F64, A, 2, true, epi_x, s));
            }
        }
        COLA_CUDA(launch_pack_spinor(COLA_F64, G, L.xhi, xs[l], c.nrhs, prm->op == COLA_OP_EO ? 1 : 3, s), "pack x0");
        COLA_CUDA(cudaMemsetAsync(L.xlo, 0, 2 * spinor_parity_bytes(c.xprec, G.Vh) * c.nrhs, s), "zero x_lo");
    }
    for (int r = 0; r < nrows; ++r) {
        CgState &st = hs[r];
        std::memset(&st, 0, sizeof(st));
        const double tol = row_tol ? row_tol[r] : prm->tol;
        st.tol2 = tol * tol;
        st.delta2 = prm->inner == COLA_F64 ? 0.0 : prm->delta * prm->delta;
        st.max_iter = row_max_iter ? row_max_iter[r] : prm->max_iter;
        st.shift = shifts ? shifts[r % c.nrhs] : 0.0;
        st.status = COLA_ERR_NOT_CONVERGED;
    }
    COLA_CUDA(cudaMemcpyAsync(c.owner->states, hs, nrows * sizeof(CgState), cudaMemcpyHostToDevice, s),
              "state upload");
    {
        BlasArgs B = blas(c, {{V_B, COLA_F64}});
        COLA_CUDA(launch_init_norms(B, s), "|b|^2");
    }
    // r = b - A x0 in FP64, r_lo = p = r.  A cold start (x0 all zero, the
    // usual case) skips the FP64 operator: A x0 = 0.
    {
        unsigned *d_flags;
        COLA_TRY(ws_slot(c.owner, S_FLAGS, nrows * sizeof(unsigned), reinterpret_cast<void **>(&d_flags)));
        COLA_CUDA(cudaMemsetAsync(d_flags, 0, nrows * sizeof(unsigned), s), "zero flags");
        BlasArgs B = blas(c, {{V_XHI, COLA_F64}});
        COLA_CUDA(launch_any_nonzero(B, d_flags, s), "x0 check");
        std::vector<unsigned> h(nrows);
        COLA_CUDA(cudaMemcpyAsync(h.data(), d_flags, nrows * sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                  "x0 check readback");
        COLA_CUDA(cudaStreamSynchronize(s), "x0 check");
        bool any = false;
        for (unsigned f : h) any |= f != 0;
        if (any) {
            COLA_TRY(mdagm(c, COLA_F64, V_AX, V_XHI, V_T64, V_MP64, nullptr, false, s));
        } else {
            for (int l = 0; l < nlat; ++l)
                COLA_CUDA(cudaMemsetAsync(c.lat[l].ax, 0, 2 * spinor_parity_bytes(COLA_F64, c.lat[l].g->geom.Vh) * c.nrhs,
                                          s),
                          "zero A x0");
        }
    }
    {
        BlasArgs B = blas(c, {{V_RHI, COLA_F64}, {V_B, COLA_F64}, {V_AX, COLA_F64}, {V_RLO, c.prec}, {V_P, c.prec},
                              {V_XHI, COLA_F64}});
        B.init = 1;
        COLA_CUDA(launch_ru_residual(B, s), "initial residual");
    }
    COLA_TRY(read_states(c, s));
    bool running = false;
    for (int l = 0; l < nlat; ++l) {
        const size_t hi1 = 2 * spinor_parity_bytes(COLA_F64, c.lat[l].g->geom.Vh);
        for (int r = 0; r < c.nrhs; ++r) {
            const CgState &st = hs[c.lat[l].row0 + r];
            running |= !st.done;
            if (st.b2 == 0.0)  // b = 0: the solution is x = 0 whatever the guess
                COLA_CUDA(cudaMemsetAsync(static_cast<char *>(c.lat[l].xhi) + r * hi1, 0, hi1, s), "zero x");
        }
    }
    if (running && prm->use_graph) {
        // Kernels launched while a stream is capturing are not autotuned, so
        // tune the inner and the FP64 operators here (only configurations not
        // seen before run, into buffers that are rewritten before use).
        TuneOnlyScope tune_only;
        COLA_TRY(mdagm(c, c.prec, V_Q, V_P, V_T, V_MP, nullptr, false, s));
        COLA_TRY(mdagm(c, COLA_F64, V_AX, V_XHI, V_T64, V_MP64, nullptr, false, s));
    }
    if (running) COLA_TRY(prm->use_graph ? run_graph_loop(c, s) : run_host_loop(c, s));
    {
        // a row stopped by breakdown may still hold work in x_lo
        BlasArgs B = blas(c, {{V_XHI, COLA_F64}, {V_XLO, c.xprec}});
        COLA_CUDA(launch_ru_accumulate(B, true, s), "final accumulate");
    }
    std::vector<double> dirac_res(nrows, -1.0);
    for (int l = 0; l < nlat; ++l) {
        LatCtx &L = c.lat[l];
        cola_gauge g = L.g;
        const Geom &G = g->geom;
        const double k = g->lat.kappa;
        if (dirac && prm->op == COLA_OP_EO) {
            // x_o = A_oo^-1 (b_o + kappa H_oe x_e)   (A = 1 without a clover term)
            DslashArgs A = make_dslash_args(g, COLA_F64, clv ? L.t64 : L.xhi, L.xhi, L.borig, c.nrhs, 1, 1.0, k);
            COLA_TRY(dslash_launch(g, COLA_F64, A, 1, false, EPI_XPAY, s));
            if (clv)
                COLA_CUDA(launch_clover_apply(COLA_F64, G, g->clover_inv[COLA_F64], L.xhi, L.t64, c.nrhs, 2, s),
                          "x_o = A_oo^-1 (...)");
        }
        if (prm->op == COLA_OP_EO && !dirac) {
            const size_t pb = spinor_parity_bytes(COLA_F64, G.Vh);
            for (int r = 0; r < c.nrhs; ++r)
                COLA_CUDA(cudaMemsetAsync(static_cast<char *>(L.xhi) + (2 * r + 1) * pb, 0, pb, s), "zero odd x");
        }
        COLA_CUDA(launch_unpack_spinor(COLA_F64, G, xs[l], L.xhi, c.nrhs, 3, s), "unpack x");
    }
    if (dirac) {
        // |b - D x| / |b| on the whole lattice, every lattice
        for (int l = 0; l < nlat; ++l) {
            LatCtx &L = c.lat[l];
            DslashArgs A = make_dslash_args(L.g, COLA_F64, L.ax, L.xhi, L.xhi, c.nrhs, 0, 1.0, -L.g->lat.kappa);
            if (clv) set_clover(A.lat[0], L.g, COLA_F64, false);
            COLA_TRY(dslash_launch(L.g, COLA_F64, A, 2, false, epi_x, s));
        }
        double *d_norms;
        COLA_TRY(ws_slot(c.owner, S_NORMS, 2 * nrows * sizeof(double), reinterpret_cast<void **>(&d_norms)));
        BlasArgs B = blas(c, {{V_RHI, COLA_F64}, {V_BORIG, COLA_F64}, {V_AX, COLA_F64}}, 2);
        B.a = 1.0;
        B.b = -1.0;
        COLA_CUDA(launch_axpby(B, s), "b - D x");
        B = blas(c, {{V_RHI, COLA_F64}}, 2);
        B.out = d_norms;
        COLA_CUDA(launch_norm2(B, s), "norm");
        B = blas(c, {{V_BORIG, COLA_F64}}, 2);
        B.out = d_norms + nrows;
        COLA_CUDA(launch_norm2(B, s), "norm");
        std::vector<double> h(2 * nrows);
        COLA_CUDA(cudaMemcpyAsync(h.data(), d_norms, 2 * nrows * sizeof(double), cudaMemcpyDeviceToHost, s),
                  "norm readback");
        COLA_CUDA(cudaStreamSynchronize(s), "sync");
        for (int r = 0; r < nrows; ++r) dirac_res[r] = h[nrows + r] > 0 ? std::sqrt(h[r] / h[nrows + r]) : 0.0;
    }
    COLA_TRY(read_states(c, s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    cola_status worst = COLA_OK;
    for (int r = 0; r < nrows; ++r) {
        const CgState &st = hs[r];
        info[r].iters = st.iter;
        info[r].reliable_updates = st.ru_count;
        info[r].true_rel_resid = dirac ? dirac_res[r] : st.b2 > 0 ? std::sqrt(st.r2_last / st.b2) : 0.0;
        info[r].seconds = secs;
        info[r].status = st.status;
        if (st.status != COLA_OK && worst == COLA_OK) worst = (cola_status)st.status;
    }
    bool stalled = false;
    for (int r = 0; r < nrows; ++r) stalled |= hs[r].status == COLA_ERR_NOT_CONVERGED && hs[r].iter < hs[r].max_iter;
    if (worst != COLA_OK)
        set_error(worst == COLA_ERR_BREAKDOWN ? "CG breakdown (non-finite or non-positive scalar)"
                  : stalled ? "CG stagnated: the FP64 true residual did not improve over 3 reliable updates "
                              "(is the tolerance below what FP64 reaches for this operator?)"
                            : "CG did not converge within max_iter");
    if (log_enabled())
        for (int r = 0; r < nrows; ++r)
            log_line("cg_solve row %d: status %d, %d iterations, %d reliable updates, true residual %.3e, %.3f s", r,
                     info[r].status, info[r].iters, info[r].reliable_updates, info[r].true_rel_resid, secs);
    return worst;
}

// Passes of the Dirac-system refinement before a row that still misses the
// tolerance is reported as not converged.
constexpr int kDiracPasses = 6;

// The Dirac system D x = b is solved through the normal equations (of Mhat on
// the even sites, or of D), whose CG stops on the normal-equation residual;
// the contract is the Dirac residual |b - D x| <= tol |b|.  So every row whose
// Dirac residual is still above tol is solved again from its current x with
// the normal-equation target scaled down by the ratio it missed by (halved
// again for margin), until every row meets tol.  Rows that already meet it
// start below their target and stop at once.  Iterations, reliable updates
// and seconds are summed over the passes.
cola_status solve_batch(int nlat, const cola_gauge *gs, void *const *xs, const void *const *bs,
                        const cola_solver_params *prm, cola_solve_info *info, cudaStream_t s,
                        const double *shifts = nullptr, bool shared_b = false) {
    if (prm->system != COLA_SYS_DIRAC)
        return solve_batch_pass(nlat, gs, xs, bs, prm, info, s, shifts, shared_b, nullptr, nullptr);
    COLA_TRY(check_params(prm));
    if (shifts) return arg_error("shifted solves need the normal system");
    const int nrows = nlat * prm->nrhs;
    std::vector<double> tol(nrows, prm->tol);
    std::vector<int> maxit(nrows, prm->max_iter);
    std::vector<cola_solve_info> cur(nrows);
    for (int r = 0; r < nrows; ++r) info[r] = {0, 0, -1.0, 0.0, COLA_ERR_NOT_CONVERGED};
    for (int pass = 0;; ++pass) {
        const cola_status st = solve_batch_pass(nlat, gs, xs, bs, prm, cur.data(), s, nullptr, false, tol.data(),
                                                maxit.data());
        if (st != COLA_OK && st != COLA_ERR_NOT_CONVERGED && st != COLA_ERR_BREAKDOWN) return st;
        bool again = false;
        for (int r = 0; r < nrows; ++r) {
            info[r].iters += cur[r].iters;
            info[r].reliable_updates += cur[r].reliable_updates;
            info[r].seconds += cur[r].seconds;
            info[r].true_rel_resid = cur[r].true_rel_resid;
            info[r].status = cur[r].status;
            maxit[r] = std::max(0, maxit[r] - cur[r].iters);
            if (cur[r].status == COLA_OK && !(cur[r].true_rel_resid <= prm->tol)) {
                again = true;
                tol[r] *= std::max(0.5 * prm->tol / cur[r].true_rel_resid, 1e-4);
            }
        }
        if (!again) return st;
        if (pass + 1 == kDiracPasses) {
            for (int r = 0; r < nrows; ++r)
                if (info[r].status == COLA_OK && !(info[r].true_rel_resid <= prm->tol))
                    info[r].status = COLA_ERR_NOT_CONVERGED;
            set_error("Dirac-system solve: the Dirac residual stayed above tol after refinement passes");
            return COLA_ERR_NOT_CONVERGED;
        }
    }
}

}  // namespace

cola_status cg_solve_rows(cola_gauge g, void *x, const void *b, const cola_solver_params *prm, cola_solve_info *info,
                          cudaStream_t s, const double *shifts, bool shared_b) {
    return solve_batch(1, &g, &x, &b, prm, info, s, shifts, shared_b);
}

}  // namespace cola

using namespace cola;

extern "C" cola_status cola_cg_solve(cola_gauge g, void *x_dev, const void *b_dev, const cola_solver_params *prm,
                                     cola_solve_info *info, cudaStream_t s) {
    TraceRange trace_("cola_cg_solve");
    if (!g || !x_dev || !b_dev || !prm || !info) return arg_error("null argument to cola_cg_solve");
    return solve_batch(1, &g, &x_dev, &b_dev, prm, info, s);
}

extern "C" cola_status cola_cg_solve_batched(int nlat, const cola_gauge *gauges, void *const *x_dev,
                                             const void *const *b_dev, const cola_solver_params *prm,
                                             cola_solve_info *info, cudaStream_t s) {
    TraceRange trace_("cola_cg_solve_batched");
    if (nlat < 1 || nlat > kMaxBatch) return arg_error("nlat must be in 1..8");
    if (!gauges || !x_dev || !b_dev || !prm || !info) return arg_error("null argument to cola_cg_solve_batched");
    for (int l = 0; l < nlat; ++l)
        if (!gauges[l] || !x_dev[l] || !b_dev[l]) return arg_error("null entry in a batch array");
    return solve_batch(nlat, gauges, x_dev, b_dev, prm, info, s);
}
