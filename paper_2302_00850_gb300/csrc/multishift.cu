// Multi-shift conjugate gradient: x_i = (A + sigma_i)^-1 b for many shifts
// from one Krylov space (Jegerlehner, "Krylov space solvers for shifted
// linear systems", 1996), A = Mhat^dag Mhat (even-odd) or D^dag D.
//
// Rational HMC, one of COLA's HMC variants (the paper's overview of the
// library), applies rational functions of A through such partial-fraction
// sums.  CG on A + sigma_0 (sigma_0 the smallest shift) builds residuals
// r_k = R_k(A + sigma_0) b with R_k(0) = 1.  Those residuals are collinear
// with the CG residuals of every other shift: r^i_k = zeta^i_k r_k.  The
// polynomial recurrence
//   R_{k+1}(t) = (1 - a_k t + a_k b_{k-1} / a_{k-1}) R_k(t) - (a_k b_{k-1} / a_{k-1}) R_{k-1}(t)
// evaluated at t = -d_i (d_i = sigma_i - sigma_0), with zeta^i_k = 1 / R_k(-d_i),
// gives
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /
//                (a_k b_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} a_{k-1} (1 + d_i a_k)),
//   a^i_k = a_k zeta_{k+1} / zeta_k,   b^i_k = b_k (zeta_{k+1} / zeta_k)^2,
//   x^i += a^i_k p^i,   p^i = zeta_{k+1} r_{k+1} + b^i_k p^i,
// with zeta_0 = zeta_{-1} = 1, a_{-1} = 1, b_{-1} = 0.  Shift i has converged
// when |zeta^i| |r| <= tol |b|; the base shift converges last.
//
// Phase 1 runs this recurrence with r, every p^i and x^i in FP32 storage (FP64
// for a plain FP64 solve) down to tol_sloppy, with one operator application
// per iteration for all shifts; FP16 storage is not used there, since
// rounding every p^i to FP16 each iteration stalls the shifted solutions near
// 1e-3 (measured).  Phase 2 refines every shift at once from those x^i with
// the mixed-precision CG of solver.cu in the requested inner precision (one
// right-hand-side row per shift, row shifts sigma_i, FP64 reliable updates
// and an FP64 true residual) down to tol.  All scalars
// live on the device; the host reads the state every few iterations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cola_impl.h"

namespace cola {
namespace {

#define MS_TRY(expr)                    \
    do {                                \
        cola_status _st = (expr);       \
        if (_st != COLA_OK) return _st; \
    } while (0)
#define MS_CUDA(expr, what) MS_TRY(cuda_check((expr), what))

constexpr int kMaxShifts = 64;
constexpr int kBlk = 256;
constexpr int kCheckEvery = 4;  // iterations between host reads of the state

struct MsShift {
    double delta;              // sigma_i - sigma_0
    double z, z_prev, z_next;  // zeta_k, zeta_{k-1}, zeta_{k+1}
    double alpha, beta;        // a^i_k, b^i_k
    int done, done_next, iters, pad;
};

struct MsState {
    double rho, rho_new, pq, alpha, alpha_prev, beta_prev, b2, tol2, sigma0;
    int iter, max_iter, status, done, halted, nshift;
    MsShift sh[kMaxShifts];
};

struct MsArgs {
    int vh, nparity, nshift;
    char *b64;        // packed FP64 right-hand side
    char *r, *q, *mp, *p, *x;
    char *p0;         // p of the base shift (the smallest)
    size_t fb, fpb;   // bytes of one storage-precision field, of one of its parities
    size_t xb, xpb;   // the same for the x^i fields
    MsState *st;
    double *partials;
};

struct Site {
    int par, cb;
    bool ok;
};

__device__ __forceinline__ Site site_of(const MsArgs &A) {
    Site t;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    t.ok = s < A.vh * A.nparity;
    t.par = s >= A.vh;
    t.cb = s - t.par * A.vh;
    return t;
}

template <typename R>
__device__ __forceinline__ double nrm2(const Cx<R> (&v)[12]) {
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) a += (double)v[k].re * v[k].re + (double)v[k].im * v[k].im;
    return a;
}

__device__ __forceinline__ void partial(const MsArgs &A, double v) {
    __shared__ double sh[kBlk / 32];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) A.partials[blockIdx.x] = t;
}

// r = b; p^i = b; x^i = 0; partial |b|^2 (FP64)
template <int P, int PX>
__global__ void __launch_bounds__(kBlk) ms_init_kernel(const __grid_constant__ MsArgs A) {
    const Site t = site_of(A);
    double nb = 0.0;
    if (t.ok) {
        Cx<double> b[12];
        SpinorIO<COLA_F64>::load(A.b64 + t.par * spinor_parity_bytes(COLA_F64, A.vh), A.vh, t.cb, b);
        nb = nrm2(b);
        Cx<typename Prec<P>::real> v[12];
        Cx<typename Prec<PX>::real> z[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            v[k] = {(typename Prec<P>::real)b[k].re, (typename Prec<P>::real)b[k].im};
            z[k] = {0, 0};
        }
        SpinorIO<P>::store(A.r + t.par * A.fpb, A.vh, t.cb, v);
        for (int i = 0; i < A.nshift; ++i) {
            SpinorIO<P>::store(A.p + i * A.fb + t.par * A.fpb, A.vh, t.cb, v);
            SpinorIO<PX>::store(A.x + i * A.xb + t.par * A.xpb, A.vh, t.cb, z);
        }
    }
    partial(A, nb);
}

// partial <p_0, (A + sigma_0) p_0> = |M p_0|^2 + sigma_0 |p_0|^2
template <int P>
__global__ void __launch_bounds__(kBlk) ms_pq_kernel(const __grid_constant__ MsArgs A) {
    const Site t = site_of(A);
    double v = 0.0;
    if (!A.st->done && t.ok) {
        Cx<typename Prec<P>::real> m[12];
        SpinorIO<P>::load(A.mp + t.par * A.fpb, A.vh, t.cb, m);
        v = nrm2(m);
        if (A.st->sigma0 != 0.0) {
            SpinorIO<P>::load(A.p0 + t.par * A.fpb, A.vh, t.cb, m);
            v += A.st->sigma0 * nrm2(m);
        }
    }
    partial(A, v);
}

// r -= alpha (q + sigma_0 p_0); partial |r|^2
template <int P>
__global__ void __launch_bounds__(kBlk) ms_update_r_kernel(const __grid_constant__ MsArgs A) {
    using R = typename Prec<P>::real;
    const Site t = site_of(A);
    double v = 0.0;
    if (!A.st->done && t.ok) {
        Cx<R> r[12], q[12], p[12];
        SpinorIO<P>::load(A.r + t.par * A.fpb, A.vh, t.cb, r);
        SpinorIO<P>::load(A.q + t.par * A.fpb, A.vh, t.cb, q);
        const R a = (R)A.st->alpha;
        if (A.st->sigma0 != 0.0) {
            SpinorIO<P>::load(A.p0 + t.par * A.fpb, A.vh, t.cb, p);
            const R sg = (R)A.st->sigma0;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                q[k].re = fma(sg, p[k].re, q[k].re);
                q[k].im = fma(sg, p[k].im, q[k].im);
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            r[k].re -= a * q[k].re;
            r[k].im -= a * q[k].im;
        }
        SpinorIO<P>::store(A.r + t.par * A.fpb, A.vh, t.cb, r);
        v = nrm2(r);
    }
    partial(A, v);
}

// for every shift still running: x^i += a^i p^i;  p^i = zeta^i r + b^i p^i
template <int P, int PX>
__global__ void __launch_bounds__(kBlk) ms_update_xp_kernel(const __grid_constant__ MsArgs A) {
    using R = typename Prec<P>::real;
    using RX = typename Prec<PX>::real;
    const Site t = site_of(A);
    if (A.st->halted || !t.ok) return;
    Cx<R> r[12];
    SpinorIO<P>::load(A.r + t.par * A.fpb, A.vh, t.cb, r);
    for (int i = 0; i < A.nshift; ++i) {
        const MsShift &S = A.st->sh[i];
        if (S.done) continue;
        char *pi = A.p + i * A.fb + t.par * A.fpb;
        char *xi = A.x + i * A.xb + t.par * A.xpb;
        Cx<R> p[12];
        Cx<RX> x[12];
        SpinorIO<P>::load(pi, A.vh, t.cb, p);
        SpinorIO<PX>::load(xi, A.vh, t.cb, x);
        const RX ax = (RX)S.alpha;
        const R z = (R)S.z, b = (R)S.beta;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            x[k].re += ax * (RX)p[k].re;
            x[k].im += ax * (RX)p[k].im;
            p[k].re = fma(b, p[k].re, z * r[k].re);
            p[k].im = fma(b, p[k].im, z * r[k].im);
        }
        SpinorIO<PX>::store(xi, A.vh, t.cb, x);
        SpinorIO<P>::store(pi, A.vh, t.cb, p);
    }
}

enum MsFinish { MS_INIT, MS_PQ, MS_R };

// One block: sum the partials in block order, then the scalar recurrences.
template <int MODE>
__global__ void __launch_bounds__(kBlk) ms_finish_kernel(MsState *st, const double *partials, int nb, CgState *gate) {
    __shared__ double sh[kBlk / 32];
    double a = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) a += partials[k];
    const double tot = block_sum(a, sh);
    if (threadIdx.x != 0) return;
    MsState &S = *st;
    if constexpr (MODE == MS_INIT) {
        S.b2 = tot;
        S.rho = tot;
        S.tol2 *= tot;  // tol_sloppy^2 on entry
        if (tot == 0.0) {
            S.done = 1;
            S.status = COLA_OK;
            for (int i = 0; i < S.nshift; ++i) S.sh[i].done = S.sh[i].done_next = 1;
        }
        gate->done = S.done;
    } else if constexpr (MODE == MS_PQ) {
        if (S.done) {
            S.halted = 1;
            return;
        }
        for (int i = 0; i < S.nshift; ++i) S.sh[i].done = S.sh[i].done_next;
        S.pq = tot;
        S.alpha = S.rho / tot;
        if (!(tot > 0.0) || !isfinite(S.alpha)) {
            S.status = COLA_ERR_BREAKDOWN;
            S.done = S.halted = 1;
            gate->done = 1;
            return;
        }
        const double ak = S.alpha, ap = S.alpha_prev, bp = S.beta_prev;
        for (int i = 0; i < S.nshift; ++i) {
            MsShift &T = S.sh[i];
            if (T.done) continue;
            const double den = ak * bp * (T.z_prev - T.z) + T.z_prev * ap * (1.0 + T.delta * ak);
            T.z_next = T.z * T.z_prev * ap / den;
            T.alpha = ak * T.z_next / T.z;
            if (!isfinite(T.z_next) || !isfinite(T.alpha)) {
                S.status = COLA_ERR_BREAKDOWN;
                S.done = S.halted = 1;
                gate->done = 1;
                return;
            }
        }
    } else {  // MS_R
        if (S.done) return;
        S.rho_new = tot;
        S.iter += 1;
        if (!isfinite(tot)) {
            S.status = COLA_ERR_BREAKDOWN;
            S.done = 1;
            gate->done = 1;
            return;
        }
        const double beta = tot / S.rho;
        int all = 1;
        for (int i = 0; i < S.nshift; ++i) {
            MsShift &T = S.sh[i];
            if (T.done) continue;
            const double ratio = T.z_next / T.z;
            T.beta = beta * ratio * ratio;
            T.z_prev = T.z;
            T.z = T.z_next;
            T.iters = S.iter;
            T.done_next = (T.z * T.z * tot <= S.tol2) || (S.iter >= S.max_iter);
            all &= T.done_next;
        }
        S.alpha_prev = S.alpha;
        S.beta_prev = beta;
        S.rho = tot;
        if (all) {
            S.done = 1;
            S.status = S.iter >= S.max_iter ? COLA_ERR_NOT_CONVERGED : COLA_OK;
            gate->done = 1;
        }
    }
}

template <int P, int PX>
cudaError_t run_kernel(int which, const MsArgs &A, int nb, cudaStream_t s) {
    switch (which) {
        case 0: ms_init_kernel<P, PX><<<nb, kBlk, 0, s>>>(A); break;
        case 1: ms_pq_kernel<P><<<nb, kBlk, 0, s>>>(A); break;
        case 2: ms_update_r_kernel<P><<<nb, kBlk, 0, s>>>(A); break;
        default: ms_update_xp_kernel<P, PX><<<nb, kBlk, 0, s>>>(A); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_ms(int prec, int which, const MsArgs &A, int nb, cudaStream_t s) {
    switch (prec) {
        case COLA_F64: return run_kernel<COLA_F64, COLA_F64>(which, A, nb, s);
        case COLA_F32: return run_kernel<COLA_F32, COLA_F32>(which, A, nb, s);
        default: return run_kernel<COLA_F16, COLA_F32>(which, A, nb, s);
    }
}

cola_status arg_error(const std::string &m) {
    set_error(m);
    return COLA_ERR_ARG;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" cola_status cola_multishift_solve(cola_gauge g, void *x_dev, const void *b_dev, const double *shifts,
                                             int nshift, double tol_sloppy, const cola_solver_params *prm,
                                             cola_solve_info *info, cudaStream_t s) {
    TraceRange trace_("cola_multishift_solve");
    const auto t0 = std::chrono::steady_clock::now();
    if (!g || !x_dev || !b_dev || !shifts || !prm || !info) return arg_error("null argument to cola_multishift_solve");
    if (nshift < 1 || nshift > kMaxShifts) return arg_error("nshift must be in 1..64");
    if (prm->system != COLA_SYS_NORMAL) return arg_error("multi-shift solves need the normal system");
    if (prm->op != COLA_OP_FULL && prm->op != COLA_OP_EO) return arg_error("op must be COLA_OP_FULL or COLA_OP_EO");
    if (prm->inner < 0 || prm->inner > 2) return arg_error("inner precision must be F64, F32 or F16");
    if (!(prm->tol > 0.0 && prm->tol < 1.0) || prm->max_iter < 0) return arg_error("tol must be in (0, 1), max_iter >= 0");
    for (int i = 0; i < nshift; ++i)
        if (!std::isfinite(shifts[i]) || shifts[i] < 0.0) return arg_error("shifts must be finite and >= 0");
    const double tol1 = tol_sloppy > 0.0 ? std::max(tol_sloppy, prm->tol)
                                         : (prm->inner == COLA_F64 ? prm->tol : std::max(prm->tol, 1e-7));
    if (!(tol1 < 1.0)) return arg_error("tol_sloppy must be below 1");
    // phase 1 in FP64 for a plain FP64 solve, else in FP32 storage: rounding
    // every p^i to FP16 each iteration stalls the shifted solutions near 1e-3
    const int prec = prm->inner == COLA_F64 ? COLA_F64 : COLA_F32;
    if (!g->links[COLA_F64] || !g->links[prec] || !g->links[prm->inner]) {
        set_error("cola_multishift_solve needs FP64 links, and FP32 links plus links of the inner precision for a "
                  "mixed-precision solve");
        return COLA_ERR_UNSUPPORTED;
    }
    const Geom &G = g->geom;
    const int xprec = prec == COLA_F64 ? COLA_F64 : COLA_F32;
    const int nparity = prm->op == COLA_OP_EO ? 1 : 2;
    const size_t fb = 2 * spinor_parity_bytes(prec, G.Vh), xb = 2 * spinor_parity_bytes(xprec, G.Vh);
    const size_t b64b = 2 * spinor_parity_bytes(COLA_F64, G.Vh);
    const int nb = (G.Vh * nparity + kBlk - 1) / kBlk;
    // one workspace block: state, gate, partials, b64, r, q, t, mp, p^i, x^i
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t o_gate = al(sizeof(MsState)), o_part = o_gate + al(sizeof(CgState));
    const size_t o_b = o_part + al(nb * sizeof(double)), o_r = o_b + al(b64b), o_q = o_r + al(fb), o_t = o_q + al(fb);
    const size_t o_mp = o_t + al(fb), o_p = o_mp + al(fb), o_x = o_p + al(fb) * nshift;
    const size_t total = o_x + al(xb) * nshift;
    void *ws = nullptr;
    MS_TRY(ws_slot(g, cola_gauge_s::kSlotMultishift, total, &ws));
    char *w = static_cast<char *>(ws);
    MsArgs A;
    std::memset(&A, 0, sizeof(A));
    A.vh = G.Vh;
    A.nparity = nparity;
    A.nshift = nshift;
    A.b64 = w + o_b;
    A.r = w + o_r;
    A.q = w + o_q;
    A.mp = w + o_mp;
    A.p = w + o_p;
    A.x = w + o_x;
    A.fb = al(fb);
    A.fpb = spinor_parity_bytes(prec, G.Vh);
    A.xb = al(xb);
    A.xpb = spinor_parity_bytes(xprec, G.Vh);
    A.st = reinterpret_cast<MsState *>(w);
    A.partials = reinterpret_cast<double *>(w + o_part);
    CgState *gate = reinterpret_cast<CgState *>(w + o_gate);

    // base shift: the smallest (it converges last)
    int i0 = 0;
    for (int i = 1; i < nshift; ++i)
        if (shifts[i] < shifts[i0]) i0 = i;
    const double sigma0 = shifts[i0];
    A.p0 = A.p + i0 * A.fb;
    MsState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.alpha_prev = 1.0;
    hs.beta_prev = 0.0;
    hs.tol2 = tol1 * tol1;
    hs.sigma0 = sigma0;
    hs.max_iter = prm->max_iter;
    hs.nshift = nshift;
    hs.status = COLA_ERR_NOT_CONVERGED;
    for (int i = 0; i < nshift; ++i) {
        hs.sh[i].delta = shifts[i] - sigma0;
        hs.sh[i].z = hs.sh[i].z_prev = 1.0;
    }
    CgState hg;
    std::memset(&hg, 0, sizeof(hg));
    MS_CUDA(cudaMemcpyAsync(A.st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s), "state upload");
    MS_CUDA(cudaMemcpyAsync(gate, &hg, sizeof(hg), cudaMemcpyHostToDevice, s), "state upload");
    MS_CUDA(launch_pack_spinor(COLA_F64, G, A.b64, b_dev, 1, nparity == 1 ? 1 : 3, s), "pack b");
    MS_CUDA(launch_ms(prec, 0, A, nb, s), "multi-shift init");
    ms_finish_kernel<MS_INIT><<<1, kBlk, 0, s>>>(A.st, A.partials, nb, gate);
    MS_CUDA(cudaGetLastError(), "multi-shift init");

    // phase 1: shifted CG recurrence in the storage precision
    MsState cur;
    for (int it = 0;; ++it) {
        if (it % kCheckEvery == 0) {
            MS_CUDA(cudaMemcpyAsync(&cur, A.st, sizeof(MsState), cudaMemcpyDeviceToHost, s), "state readback");
            MS_CUDA(cudaStreamSynchronize(s), "multi-shift");
            if (cur.done) break;
        }
        MS_TRY(apply_mdagm(g, prec, prm->op, A.q, A.p0, w + o_t, A.mp, 1, gate, false, s));
        MS_CUDA(launch_ms(prec, 1, A, nb, s), "multi-shift <p, Ap>");
        ms_finish_kernel<MS_PQ><<<1, kBlk, 0, s>>>(A.st, A.partials, nb, gate);
        MS_CUDA(launch_ms(prec, 2, A, nb, s), "multi-shift r update");
        ms_finish_kernel<MS_R><<<1, kBlk, 0, s>>>(A.st, A.partials, nb, gate);
        MS_CUDA(launch_ms(prec, 3, A, nb, s), "multi-shift x, p update");
    }
    if (cur.status == COLA_ERR_BREAKDOWN) {
        set_error("multi-shift CG breakdown (non-finite or non-positive scalar)");
        for (int i = 0; i < nshift; ++i) info[i] = {cur.sh[i].iters, 0, -1.0, 0.0, COLA_ERR_BREAKDOWN};
        return COLA_ERR_BREAKDOWN;
    }
    // x^i -> x_dev[i] (canonical FP64; odd sites zero for the even-odd system)
    const size_t canon = (size_t)G.V * 12 * 16;
    for (int i = 0; i < nshift; ++i) {
        char *xi = static_cast<char *>(x_dev) + i * canon;
        if (nparity == 1) MS_CUDA(cudaMemsetAsync(xi, 0, canon, s), "zero x");
        MS_CUDA(launch_unpack_spinor(xprec, G, xi, A.x + i * A.xb, 1, nparity == 1 ? 1 : 3, s), "unpack x");
    }
    // phase 2: every shift refined at once (rows = shifts) from those guesses
    cola_solver_params p2 = *prm;
    p2.nrhs = nshift;
    p2.max_iter = std::max(0, prm->max_iter - cur.iter);
    std::vector<cola_solve_info> inf(nshift);
    cola_status st = cg_solve_rows(g, x_dev, b_dev, &p2, inf.data(), s, shifts, true);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < nshift; ++i) {
        info[i] = inf[i];
        info[i].iters += cur.sh[i].iters;
        info[i].seconds = secs;
        if (log_enabled())
            log_line("multishift shift %d (sigma %.4g): status %d, %d iterations (%d in the recurrence), true residual "
                     "%.3e, %.3f s", i, shifts[i], info[i].status, info[i].iters, cur.sh[i].iters,
                     info[i].true_rel_resid, secs);
    }
    return st;
}
