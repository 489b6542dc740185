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
// Per iteration: four hopping-term launches for A = Mhat^dag Mhat (the
// second also reduces <p, Ap> = |Mhat p|^2 and sets alpha), one fused
// x/r update that reduces |r|^2 and decides, optionally the FP64 update,
// and the p update.  All scalars stay on the device.  Two drivers run the
// loop: a host loop that reads the per-right-hand-side state after each
// update, or one CUDA graph whose while/if conditional nodes are set by a
// one-thread control kernel, so that a whole solve is a single launch.
#include <chrono>
#include <cstring>
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
    S_B = 6, S_XHI = 7, S_RHI = 8, S_AX = 9, S_T64 = 10, S_MP64 = 11, S_BORIG = 12,
};

struct SolveCtx {
    cola_gauge g;
    int prec, xprec, op, nrhs, nparity;
    void *t, *mp, *p, *q, *rlo, *xlo;
    void *b, *xhi, *rhi, *ax, *t64, *mp64, *borig;
    size_t lo_bytes, x_bytes, hi_bytes;
    BlasDims dims;
};

VecRef vref(void *p, int prec, const Geom &g) {
    VecRef v;
    v.ptr = p;
    v.prec = prec;
    v.parity_stride = spinor_parity_bytes(prec, g.Vh);
    v.rhs_stride = 2 * v.parity_stride;
    return v;
}

cola_status ru_block(SolveCtx &c, cudaStream_t s) {
    const Geom &G = c.g->geom;
    COLA_CUDA(launch_ru_accumulate(c.dims, vref(c.xhi, COLA_F64, G), vref(c.xlo, c.xprec, G), c.g->states, false, s),
              "reliable update (accumulate)");
    COLA_TRY(apply_mdagm(c.g, COLA_F64, c.op, c.ax, c.xhi, c.t64, c.mp64, c.nrhs, c.g->states, true, false, s));
    COLA_CUDA(launch_ru_residual(c.dims, vref(c.rhi, COLA_F64, G), vref(c.b, COLA_F64, G), vref(c.ax, COLA_F64, G),
                                 vref(c.rlo, c.prec, G), vref(c.p, c.prec, G), c.g->states, false, false,
                                 c.g->partials, c.g->counters, s),
              "reliable update (residual)");
    return COLA_OK;
}

cola_status iter_head(SolveCtx &c, cudaStream_t s) {
    const Geom &G = c.g->geom;
    COLA_TRY(apply_mdagm(c.g, c.prec, c.op, c.q, c.p, c.t, c.mp, c.nrhs, c.g->states, false, true, s));
    COLA_CUDA(launch_cg_update_xr(c.dims, vref(c.xlo, c.xprec, G), vref(c.rlo, c.prec, G), vref(c.p, c.prec, G),
                                  vref(c.q, c.prec, G), c.g->states, c.g->partials, c.g->counters, s),
              "cg update x, r");
    return COLA_OK;
}

cola_status iter_tail(SolveCtx &c, cudaStream_t s) {
    const Geom &G = c.g->geom;
    COLA_CUDA(launch_cg_update_p(c.dims, vref(c.p, c.prec, G), vref(c.rlo, c.prec, G), c.g->states, false, s),
              "cg update p");
    return COLA_OK;
}

cola_status read_states(SolveCtx &c, cudaStream_t s) {
    COLA_CUDA(cudaMemcpyAsync(c.g->h_states, c.g->states, c.nrhs * sizeof(CgState), cudaMemcpyDeviceToHost, s),
              "state readback");
    COLA_CUDA(cudaStreamSynchronize(s), "solver synchronisation");
    return COLA_OK;
}

// Host-driven loop: one state readback per iteration.
cola_status run_host_loop(SolveCtx &c, cudaStream_t s) {
    for (;;) {
        COLA_TRY(iter_head(c, s));
        COLA_TRY(read_states(c, s));
        bool any_ru = false, running = false;
        for (int r = 0; r < c.nrhs; ++r) {
            const CgState &st = c.g->h_states[r];
            any_ru |= st.ru && !st.done;
        }
        if (any_ru) {
            COLA_TRY(ru_block(c, s));
            COLA_TRY(read_states(c, s));
        }
        for (int r = 0; r < c.nrhs; ++r) running |= !c.g->h_states[r].done;
        if (!running) return COLA_OK;
        COLA_TRY(iter_tail(c, s));
    }
}

// Whole loop as one graph: while (running) { head; if (ru) { ru_block } ; tail }.
cola_status run_graph_loop(SolveCtx &c, cudaStream_t s) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    cola_status st = COLA_OK;
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
    // body part 1: iteration head, then the control kernel for the "if"
    if ((st = cuda_check(cudaGraphConditionalHandleCreate(&h_ru, body, 0, cudaGraphCondAssignDefault),
                         "graph conditional")) != COLA_OK)
        return fail(st);
    if ((st = cuda_check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                         "capture")) != COLA_OK)
        return fail(st);
    st = iter_head(c, cs);
    if (st == COLA_OK) {
        control_ru_kernel<<<1, 1, 0, cs>>>(c.g->states, c.nrhs, h_ru);
        st = cuda_check(cudaGetLastError(), "control kernel");
    }
    // if node appended to the capture
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
        control_loop_kernel<<<1, 1, 0, cs>>>(c.g->states, c.nrhs, h_loop);
        st = cuda_check(cudaGetLastError(), "control kernel");
    }
    {
        cudaGraph_t out = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &out);
        if (st == COLA_OK) st = cuda_check(e, "end capture");
    }
    if (st != COLA_OK) return fail(st);
    // the "if" body: the FP64 reliable update
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
    fail(COLA_OK);
    return read_states(c, s);
}

}  // namespace

static cola_status arg_error(const char *msg) {
    set_error(msg);
    return COLA_ERR_ARG;
}

}  // namespace cola

using namespace cola;

extern "C" cola_status cola_cg_solve(cola_gauge g, void *x_dev, const void *b_dev, const cola_solver_params *prm,
                                     cola_solve_info *info, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!g || !x_dev || !b_dev || !prm || !info) return arg_error("null argument to cola_cg_solve");
    if (prm->op != COLA_OP_FULL && prm->op != COLA_OP_EO) return arg_error("op must be COLA_OP_FULL or COLA_OP_EO");
    if (prm->system != COLA_SYS_NORMAL && prm->system != COLA_SYS_DIRAC)
        return arg_error("system must be COLA_SYS_NORMAL or COLA_SYS_DIRAC");
    if (prm->inner < 0 || prm->inner > 2) return arg_error("inner precision must be F64, F32 or F16");
    if (prm->nrhs < 1 || prm->nrhs > 64) return arg_error("nrhs must be in 1..64");
    if (!(prm->tol > 0.0) || prm->max_iter < 0) return arg_error("tol must be > 0 and max_iter >= 0");
    if (prm->inner != COLA_F64 && !(prm->delta > 0.0 && prm->delta < 1.0))
        return arg_error("delta must be in (0, 1) for a mixed-precision solve");
    if (!g->links[COLA_F64]) {
        set_error("cola_cg_solve needs FP64 links in the gauge handle (reliable updates and residuals)");
        return COLA_ERR_UNSUPPORTED;
    }
    if (!g->links[prm->inner]) {
        set_error("gauge handle holds no links of the inner precision");
        return COLA_ERR_UNSUPPORTED;
    }
    const Geom &G = g->geom;
    SolveCtx c;
    c.g = g;
    c.prec = prm->inner;
    c.xprec = prm->inner == COLA_F64 ? COLA_F64 : COLA_F32;
    c.op = prm->op;
    c.nrhs = prm->nrhs;
    c.nparity = prm->op == COLA_OP_EO ? 1 : 2;
    c.dims = {G.Vh, c.nparity, c.nrhs};
    c.lo_bytes = 2 * spinor_parity_bytes(c.prec, G.Vh) * c.nrhs;
    c.x_bytes = 2 * spinor_parity_bytes(c.xprec, G.Vh) * c.nrhs;
    c.hi_bytes = 2 * spinor_parity_bytes(COLA_F64, G.Vh) * c.nrhs;
    COLA_TRY(ws_slot(g, S_T, c.lo_bytes, &c.t));
    COLA_TRY(ws_slot(g, S_MP, c.lo_bytes, &c.mp));
    COLA_TRY(ws_slot(g, S_P, c.lo_bytes, &c.p));
    COLA_TRY(ws_slot(g, S_Q, c.lo_bytes, &c.q));
    COLA_TRY(ws_slot(g, S_RLO, c.lo_bytes, &c.rlo));
    COLA_TRY(ws_slot(g, S_XLO, c.x_bytes, &c.xlo));
    COLA_TRY(ws_slot(g, S_B, c.hi_bytes, &c.b));
    COLA_TRY(ws_slot(g, S_XHI, c.hi_bytes, &c.xhi));
    COLA_TRY(ws_slot(g, S_RHI, c.hi_bytes, &c.rhi));
    COLA_TRY(ws_slot(g, S_AX, c.hi_bytes, &c.ax));
    COLA_TRY(ws_slot(g, S_T64, c.hi_bytes, &c.t64));
    COLA_TRY(ws_slot(g, S_MP64, c.hi_bytes, &c.mp64));
    c.borig = nullptr;
    if (prm->system == COLA_SYS_DIRAC) COLA_TRY(ws_slot(g, S_BORIG, c.hi_bytes, &c.borig));
    // reduction scratch sized for the largest launch of this solve
    {
        const size_t blas_blocks = (size_t)(G.Vh * 2 + 255) / 256;
        const size_t ds_blocks = (size_t)((G.Vh + 31) / 32) * 2;
        COLA_TRY(ws_reduce(g, c.nrhs, blas_blocks > ds_blocks ? blas_blocks : ds_blocks));
    }
    COLA_TRY(ws_states(g, c.nrhs));

    const double k = g->lat.kappa;
    const int pmask_b = (prm->op == COLA_OP_EO && prm->system == COLA_SYS_NORMAL) ? 1 : 3;
    // right-hand side of the CG system in b (packed FP64)
    if (prm->system == COLA_SYS_NORMAL) {
        COLA_CUDA(launch_pack_spinor(COLA_F64, G, c.b, b_dev, c.nrhs, pmask_b, s), "pack b");
    } else {
        COLA_CUDA(launch_pack_spinor(COLA_F64, G, c.borig, b_dev, c.nrhs, 3, s), "pack b");
        if (prm->op == COLA_OP_EO) {
            // bhat_e = b_e + kappa H_eo b_o (into mp64);  b = Mhat^dag bhat
            DslashArgs A = make_dslash_args(g, COLA_F64, c.mp64, c.borig, c.borig, c.nrhs, 0, 1.0, k);
            COLA_CUDA(launch_dslash(COLA_F64, g->recon[COLA_F64], A, 1, false, true, false, 0, s), "source prep");
            A = make_dslash_args(g, COLA_F64, c.t64, c.mp64, nullptr, c.nrhs, 1, 0.0, 1.0);
            COLA_CUDA(launch_dslash(COLA_F64, g->recon[COLA_F64], A, 1, true, false, false, 0, s), "source prep");
            A = make_dslash_args(g, COLA_F64, c.b, c.t64, c.mp64, c.nrhs, 0, 1.0, -k * k);
            COLA_CUDA(launch_dslash(COLA_F64, g->recon[COLA_F64], A, 1, true, true, false, 0, s), "source prep");
        } else {
            // b = D^dag b
            DslashArgs A = make_dslash_args(g, COLA_F64, c.b, c.borig, c.borig, c.nrhs, 0, 1.0, -k);
            COLA_CUDA(launch_dslash(COLA_F64, g->recon[COLA_F64], A, 2, true, true, false, 0, s), "source prep");
        }
    }
    COLA_CUDA(launch_pack_spinor(COLA_F64, G, c.xhi, x_dev, c.nrhs, prm->op == COLA_OP_EO ? 1 : 3, s), "pack x0");
    COLA_CUDA(cudaMemsetAsync(c.xlo, 0, c.x_bytes, s), "zero x_lo");

    // per right-hand side state
    for (int r = 0; r < c.nrhs; ++r) {
        CgState &st = g->h_states[r];
        std::memset(&st, 0, sizeof(st));
        st.tol2 = prm->tol * prm->tol;
        st.delta2 = prm->inner == COLA_F64 ? 0.0 : prm->delta * prm->delta;
        st.max_iter = prm->max_iter;
        st.status = COLA_ERR_NOT_CONVERGED;
    }
    COLA_CUDA(cudaMemcpyAsync(g->states, g->h_states, c.nrhs * sizeof(CgState), cudaMemcpyHostToDevice, s),
              "state upload");
    COLA_CUDA(launch_init_norms(c.dims, vref(c.b, COLA_F64, G), g->states, g->partials, g->counters, s), "|b|^2");
    // r = b - A x0 in FP64, r_lo = p = r
    COLA_TRY(apply_mdagm(g, COLA_F64, c.op, c.ax, c.xhi, c.t64, c.mp64, c.nrhs, nullptr, false, false, s));
    COLA_CUDA(launch_ru_residual(c.dims, vref(c.rhi, COLA_F64, G), vref(c.b, COLA_F64, G), vref(c.ax, COLA_F64, G),
                                 vref(c.rlo, c.prec, G), vref(c.p, c.prec, G), g->states, true, true, g->partials,
                                 g->counters, s),
              "initial residual");
    COLA_TRY(read_states(c, s));
    bool running = false;
    for (int r = 0; r < c.nrhs; ++r) {
        running |= !g->h_states[r].done;
        if (g->h_states[r].b2 == 0.0)  // b = 0: the solution is x = 0 whatever the guess
            COLA_CUDA(cudaMemsetAsync(static_cast<char *>(c.xhi) + r * (c.hi_bytes / c.nrhs), 0, c.hi_bytes / c.nrhs, s),
                      "zero x");
    }
    if (running) COLA_TRY(prm->use_graph ? run_graph_loop(c, s) : run_host_loop(c, s));
    // a row stopped by breakdown may still hold work in x_lo
    COLA_CUDA(launch_ru_accumulate(c.dims, vref(c.xhi, COLA_F64, G), vref(c.xlo, c.xprec, G), g->states, true, s),
              "final accumulate");

    if (prm->system == COLA_SYS_DIRAC && prm->op == COLA_OP_EO) {
        // x_o = b_o + kappa H_oe x_e
        DslashArgs A = make_dslash_args(g, COLA_F64, c.xhi, c.xhi, c.borig, c.nrhs, 1, 1.0, k);
        COLA_CUDA(launch_dslash(COLA_F64, g->recon[COLA_F64], A, 1, false, true, false, 0, s), "odd reconstruction");
    }
    if (prm->op == COLA_OP_EO && prm->system == COLA_SYS_NORMAL) {
        const size_t pb = spinor_parity_bytes(COLA_F64, G.Vh);
        for (int r = 0; r < c.nrhs; ++r)
            COLA_CUDA(cudaMemsetAsync(static_cast<char *>(c.xhi) + (2 * r + 1) * pb, 0, pb, s), "zero odd x");
    }
    COLA_CUDA(launch_unpack_spinor(COLA_F64, G, x_dev, c.xhi, c.nrhs, 3, s), "unpack x");
    std::vector<double> dirac_res(c.nrhs, -1.0);
    if (prm->system == COLA_SYS_DIRAC) {
        // |b - D x| / |b| on the whole lattice
        const BlasDims full = {G.Vh, 2, c.nrhs};
        DslashArgs A = make_dslash_args(g, COLA_F64, c.ax, c.xhi, c.xhi, c.nrhs, 0, 1.0, -k);
        COLA_CUDA(launch_dslash(COLA_F64, g->recon[COLA_F64], A, 2, false, true, false, 0, s), "D x");
        COLA_CUDA(launch_axpby(full, vref(c.rhi, COLA_F64, G), 1.0, vref(c.borig, COLA_F64, G), -1.0,
                               vref(c.ax, COLA_F64, G), s),
                  "b - D x");
        double *d_norms;
        COLA_TRY(ws_slot(g, 13, 2 * c.nrhs * sizeof(double), reinterpret_cast<void **>(&d_norms)));
        COLA_CUDA(launch_norm2(full, vref(c.rhi, COLA_F64, G), d_norms, g->partials, g->counters, s), "norm");
        COLA_CUDA(launch_norm2(full, vref(c.borig, COLA_F64, G), d_norms + c.nrhs, g->partials, g->counters, s),
                  "norm");
        std::vector<double> h(2 * c.nrhs);
        COLA_CUDA(cudaMemcpyAsync(h.data(), d_norms, 2 * c.nrhs * sizeof(double), cudaMemcpyDeviceToHost, s),
                  "norm readback");
        COLA_CUDA(cudaStreamSynchronize(s), "sync");
        for (int r = 0; r < c.nrhs; ++r) dirac_res[r] = h[c.nrhs + r] > 0 ? std::sqrt(h[r] / h[c.nrhs + r]) : 0.0;
    }
    COLA_TRY(read_states(c, s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    cola_status worst = COLA_OK;
    for (int r = 0; r < c.nrhs; ++r) {
        const CgState &st = g->h_states[r];
        info[r].iters = st.iter;
        info[r].reliable_updates = st.ru_count;
        info[r].true_rel_resid = prm->system == COLA_SYS_DIRAC ? dirac_res[r]
                                 : st.b2 > 0                   ? std::sqrt(st.r2_last / st.b2)
                                                               : 0.0;
        info[r].seconds = secs;
        info[r].status = st.status;
        if (st.status != COLA_OK && worst == COLA_OK) worst = (cola_status)st.status;
    }
    if (worst != COLA_OK) set_error(worst == COLA_ERR_BREAKDOWN ? "CG breakdown (non-finite or non-positive scalar)"
                                                                : "CG did not converge within max_iter");
    return worst;
}
