// Low-lying eigenmodes of A = Mhat^dag Mhat (even-odd) or D^dag D by the
// accelerated conjugate-gradient method of Kalkreuter and Simma (1996), the
// eigensolver the paper cites among COLA's key algorithms.
//
// Each vector v_j in turn minimises the Ritz functional mu(x) = <x, A x> / <x, x>
// over the complement of v_0 .. v_{j-1}, by conjugate gradients on the unit
// sphere: with the gradient g = (A - mu) x (projected), the search direction
// p (kept orthogonal to x), p^ = p / |p| and z = A p^, the minimum of mu over
// x cos t + p^ sin t is the lower eigenvalue of the 2x2 matrix
// [[a, b], [b, c]] (a = mu, b = Re <x, z>, c = <p^, z>):
//   mu' = (a + c) / 2 - R,  R = sqrt(((a - c) / 2)^2 + b^2),
//   cos 2t = -(a - c) / (2 R),  sin 2t = -b / R,
// and x, A x follow by the same rotation (no extra operator application).
// Then p = g' + beta (p - <x', p> x'), beta = |g'|^2 / |g|^2.  A vector's
// minimisation stops when |g| has fallen by gamma (or after max_cg steps).
// After every sweep over the vectors, the Rayleigh-Ritz step diagonalises A
// in span(v): H = V^dag A V (N x N, Hermitian), H = U diag(lambda) U^dag by
// cyclic complex Jacobi rotations in one thread block, V <- V U, A V <- (A V) U.
// Converged when every wanted |A v_j - lambda_j v_j| <= tol lambda_j (j < nev).
// nextra guard vectors above the wanted ones take part in every sweep and in
// the Rayleigh-Ritz step but not in the test: near-degenerate levels at the
// edge of the wanted set then converge at the rate of the gap to the guard
// levels rather than to the next wanted one (12 levels of an 8^3x16 field in
// 12 sweeps with 4 guards, none within 40 without).
//
// FP64 throughout: packed fields, the FP64 normal operator, reductions in
// fixed order (block partials, one finishing block per result).  The
// minimisation of each vector runs on the device: its scalars (the rotation
// of the line search, beta, the projection coefficients, the stopping test)
// are computed into device memory by one thread after the dot products they
// need are finished, the linear combinations read their coefficients from
// there, and the CG loop is a while node of a CUDA graph (one graph per
// vector index, built on first use in a call).  A CG step is 7 launches
// besides the operator: the rotation, the gradient and its dot products
// share one pass over the sites, as do the projection, the new direction and
// the dot products the next step starts from.  The host launches the graphs
// of a sweep back to back, runs the Rayleigh-Ritz step, and reads the
// residuals once per sweep.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cola_impl.h"

namespace cola {
namespace {

#define EIG_TRY(expr)                   \
    do {                                \
        cola_status _st = (expr);       \
        if (_st != COLA_OK) return _st; \
    } while (0)
#define EIG_CUDA(expr, what) EIG_TRY(cuda_check((expr), what))

constexpr int kMaxNev = 64;
constexpr int kMaxTerms = kMaxNev + 2;
constexpr int kBlk = 256;

struct Fields {
    int vh, nparity;
};

__device__ __forceinline__ bool site(const Fields &F, int &par, int &cb) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    par = s >= F.vh;
    cb = s - par * F.vh;
    return s < F.vh * F.nparity;
}

__device__ __forceinline__ const char *at(const char *f, int vh, int par) {
    return f + par * spinor_parity_bytes(COLA_F64, vh);
}

// out[k] partials: sum over sites of conj(a_k) b_k (re, im)
struct DotArgs {
    Fields F;
    int n;
    const char *a[kMaxTerms];
    const char *b[kMaxTerms];
    double *partials;  // [n][nb][2]
    int nb;
    unsigned re_only;  // bit k: pair k needs the real part only (its imaginary partial is 0)
};

// Pairs are taken four at a time with one block reduction per group, and a
// field shared by consecutive pairs (the basis dots <v_i, g> all read g) is
// loaded once.  The reduction order per pair is the same fixed order as
// block_sum: warp butterflies, then the warps in order.
constexpr int kDotGroup = 4;

// Block partials of one group of kDotGroup dots (re, im in v): warp
// butterflies, then the warps in order; results k0 .. min(k0 + kDotGroup, n)
// go to partials[k][blockIdx.x].  Every thread of the block calls it.
__device__ __forceinline__ void group_partials(double (&v)[2 * kDotGroup], int k0, int n, double *partials, int nb,
                                               double (*sh)[2 * kDotGroup]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 2 * kDotGroup; ++q) v[q] = warp_allsum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 2 * kDotGroup; ++q) sh[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 2 * kDotGroup) {
        const int k = k0 + (int)threadIdx.x / 2;
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sh[w][threadIdx.x];
        if (k < n) partials[((size_t)k * nb + blockIdx.x) * 2 + (threadIdx.x & 1)] = t;
    }
    __syncthreads();
}

// conj(a) b accumulated over the 12 components of one site, in the order
// every dot product of the eigensolver uses
__device__ __forceinline__ void site_dot(const Cx<double> (&a)[12], const Cx<double> (&b)[12], double &re,
                                         double &im) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        re = fma(a[c].re, b[c].re, fma(a[c].im, b[c].im, re));
        im = fma(a[c].re, b[c].im, fma(-a[c].im, b[c].re, im));
    }
}

// The real part alone (for |a|^2, and for dots whose imaginary part no
// step uses): the same multiply-adds as site_dot's real part.
__device__ __forceinline__ void site_dot_re(const Cx<double> (&a)[12], const Cx<double> (&b)[12], double &re) {
#pragma unroll
    for (int c = 0; c < 12; ++c) re = fma(a[c].re, b[c].re, fma(a[c].im, b[c].im, re));
}

// acc += w x over a site.  The vector work of the eigensolver runs on the
// FP64 pipe (one complex multiply-add is 4 FP64 operations per component, at
// 1/64 of the FP32 rate), so a real w takes the 2 multiply-adds that its
// non-zero part needs (the zero imaginary part only adds exact zeros), and
// w = 1 into an empty accumulator is a copy.
__device__ __forceinline__ void site_mac(Cx<double> (&acc)[12], double2 w, const Cx<double> (&x)[12], bool first) {
    if (w.y == 0.0) {
        if (first && w.x == 1.0) {
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = x[c];
            return;
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            acc[c].re = fma(w.x, x[c].re, first ? 0.0 : acc[c].re);
            acc[c].im = fma(w.x, x[c].im, first ? 0.0 : acc[c].im);
        }
        return;
    }
    const Cx<double> cw = {w.x, w.y};
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        if (first) acc[c] = {0.0, 0.0};
        cmac(acc[c], cw, x[c]);
    }
}

__global__ void __launch_bounds__(kBlk, 2) dots_kernel(const __grid_constant__ DotArgs A) {
    __shared__ double sh[kBlk / 32][2 * kDotGroup];
    int par, cb;
    const bool ok = site(A.F, par, cb);
    const char *pa = nullptr, *pb = nullptr;
    Cx<double> x[12], y[12];
    for (int k0 = 0; k0 < A.n; k0 += kDotGroup) {
        double v[2 * kDotGroup];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) {
            const int k = k0 + q;
            double re = 0.0, im = 0.0;
            if (ok && k < A.n) {
                if (A.a[k] != pa) {
                    pa = A.a[k];
                    SpinorIO<COLA_F64>::load(at(pa, A.F.vh, par), A.F.vh, cb, x);
                }
                if (A.b[k] != pb) {
                    pb = A.b[k];
                    SpinorIO<COLA_F64>::load(at(pb, A.F.vh, par), A.F.vh, cb, y);
                }
                if (k < 32 && ((A.re_only >> k) & 1u)) site_dot_re(x, y, re);
                else site_dot(x, y, re, im);
            }
            v[2 * q] = re;
            v[2 * q + 1] = im;
        }
        group_partials(v, k0, A.n, A.partials, A.nb, sh);
    }
}

// one block per result: out[k] = sum of its partials in block order
__global__ void __launch_bounds__(kBlk) dots_finish_kernel(const double *partials, int nb, double2 *out) {
    __shared__ double sh[kBlk / 32];
    const int k = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        re += partials[((size_t)k * nb + b) * 2];
        im += partials[((size_t)k * nb + b) * 2 + 1];
    }
    const double tr = block_sum(re, sh);
    __syncthreads();
    const double ti = block_sum(im, sh);
    if (threadIdx.x == 0) out[k] = make_double2(tr, ti);
}

// out = sum_k c_k in_k  (out may be one of the inputs: each site is read, then written)
struct CombArgs {
    Fields F;
    int n;
    char *out;
    const char *in[kMaxTerms];
    double2 c[kMaxTerms];
};

__global__ void __launch_bounds__(kBlk) lincomb_kernel(const __grid_constant__ CombArgs A) {
    int par, cb;
    if (!site(A.F, par, cb)) return;
    Cx<double> acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {0.0, 0.0};
    for (int k = 0; k < A.n; ++k) {
        Cx<double> x[12];
        SpinorIO<COLA_F64>::load(at(A.in[k], A.F.vh, par), A.F.vh, cb, x);
        site_mac(acc, A.c[k], x, k == 0);
    }
    SpinorIO<COLA_F64>::store(const_cast<char *>(at(A.out, A.F.vh, par)), A.F.vh, cb, acc);
}

// ------------------------------------------------------ device control --
// Coefficient sets of the linear combinations of one minimisation.
enum CoefSet { C_PROJ = 0, C_NORM, C_GRAD, C_PERP, C_ROT, C_DIR, kCoefSets };

// Scalars of the minimisation of one vector, on the device.
struct EigDev {
    double mu, gg, gg0, gg_new, pn, pn2, beta;
    double2 xpn;
    int k, stop, halt, cont, status, steps;
    double2 coef[kCoefSets][kMaxTerms];
};

// out = sum_k coef[k] in_k with coefficients read from device memory; skipped
// when the minimisation has halted (mask bit 0) or its loop has stopped
// (mask bit 1).
struct CombDevArgs {
    Fields F;
    int n;
    char *out;
    const char *in[kMaxTerms];
    const EigDev *e;
    int set;
    int mask;
};

__global__ void __launch_bounds__(kBlk) lincomb_dev_kernel(const __grid_constant__ CombDevArgs A) {
    if (((A.mask & 1) && A.e->halt) || ((A.mask & 2) && A.e->stop)) return;
    int par, cb;
    if (!site(A.F, par, cb)) return;
    Cx<double> acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {0.0, 0.0};
    for (int k = 0; k < A.n; ++k) {
        Cx<double> x[12];
        SpinorIO<COLA_F64>::load(at(A.in[k], A.F.vh, par), A.F.vh, cb, x);
        site_mac(acc, A.e->coef[A.set][k], x, k == 0);
    }
    SpinorIO<COLA_F64>::store(const_cast<char *>(at(A.out, A.F.vh, par)), A.F.vh, cb, acc);
}

enum CtlStep { CTL_PROJ, CTL_NORM, CTL_MU, CTL_GRAD0, CTL_LOOP0, CTL_PERP, CTL_ROT, CTL_GRAD, CTL_END };

struct CtlParams {
    int j;          // vector index: number of earlier vectors projected out
    int max_cg;
    double gamma, tol;
};

__device__ __forceinline__ bool keep_going(const EigDev &e, const CtlParams &p) {
    return !(e.gg <= p.gamma * p.gamma * e.gg0 || sqrt(e.gg) <= 0.1 * p.tol * fabs(e.mu) || e.gg == 0.0) &&
           e.k < p.max_cg;
}

// The gradient's norm after projecting out v_0 .. v_{j-1}: the dots are
// {<v_i, g>} (i < j), |g|^2, then optionally <x, p>.
__device__ __forceinline__ void gradient_norm(EigDev &e, const double2 *d, int j) {
    double n2 = d[j].x;
    e.coef[C_PROJ][0] = make_double2(1.0, 0.0);
    for (int i = 0; i < j; ++i) {
        e.coef[C_PROJ][1 + i] = make_double2(-d[i].x, -d[i].y);
        n2 -= d[i].x * d[i].x + d[i].y * d[i].y;
    }
    e.gg_new = fmax(n2, 0.0);
}

// The control steps (one thread); d holds the latest finished dot products.
template <int STEP>
__device__ __forceinline__ void ctl_step(EigDev &e, const double2 *d, const CtlParams &p,
                                         cudaGraphConditionalHandle h) {
    if constexpr (STEP == CTL_PROJ) {  // x -= sum_i <v_i, x> v_i
        e.coef[C_PROJ][0] = make_double2(1.0, 0.0);
        for (int i = 0; i < p.j; ++i) e.coef[C_PROJ][1 + i] = make_double2(-d[i].x, -d[i].y);
    } else if constexpr (STEP == CTL_NORM) {  // x /= |x|
        if (e.halt) return;
        if (!(d[0].x > 0.0) || !isfinite(d[0].x)) {
            e.halt = 1;
            e.status = COLA_ERR_BREAKDOWN;
            return;
        }
        e.coef[C_NORM][0] = make_double2(1.0 / sqrt(d[0].x), 0.0);
    } else if constexpr (STEP == CTL_MU) {  // mu = <x, A x>;  g = y - mu x
        e.mu = d[0].x;
        e.coef[C_GRAD][0] = make_double2(1.0, 0.0);
        e.coef[C_GRAD][1] = make_double2(-e.mu, 0.0);
    } else if constexpr (STEP == CTL_GRAD0) {
        gradient_norm(e, d, p.j);
        e.gg = e.gg0 = e.gg_new;
    } else if constexpr (STEP == CTL_LOOP0) {
        e.k = 0;
        e.stop = 0;
        e.cont = !e.halt && keep_going(e, p);
        cudaGraphSetConditional(h, e.cont ? 1u : 0u);
    } else if constexpr (STEP == CTL_PERP) {  // p -= <x, p> x; |p|
        const double2 xp = d[0];
        e.pn2 = d[1].x - (xp.x * xp.x + xp.y * xp.y);
        if (!(e.pn2 > 0.0)) {
            e.stop = 1;
            return;
        }
        e.pn = sqrt(e.pn2);
        e.coef[C_PERP][0] = make_double2(1.0, 0.0);
        e.coef[C_PERP][1] = make_double2(-xp.x, -xp.y);
    } else if constexpr (STEP == CTL_ROT) {  // exact line search on span(x, p^): d = {<x, z>, <p, z>}
        if (e.stop) return;
        const double a = e.mu, b = d[0].x / e.pn, cc = d[1].x / e.pn2;
        const double hh = 0.5 * (a - cc), R = sqrt(hh * hh + b * b);
        if (!(R > 0.0)) {
            e.stop = 1;
            return;
        }
        // cos 2t = -h / R, sin 2t = -b / R; half angle with cos t >= 0
        const double c2 = -hh / R, s2 = -b / R;
        const double ct = sqrt(fmax(0.0, 0.5 * (1.0 + c2)));
        const double st = ct > 1e-8 ? s2 / (2.0 * ct) : (s2 >= 0.0 ? 1.0 : -1.0) * sqrt(fmax(0.0, 0.5 * (1.0 - c2)));
        e.coef[C_ROT][0] = make_double2(ct, 0.0);
        e.coef[C_ROT][1] = make_double2(st / e.pn, 0.0);
        e.mu = 0.5 * (a + cc) - R;
        e.coef[C_GRAD][0] = make_double2(1.0, 0.0);
        e.coef[C_GRAD][1] = make_double2(-e.mu, 0.0);
    } else if constexpr (STEP == CTL_GRAD) {  // d = {<v_i, g'>}, |g'|^2, <x', p>;  p = g' + beta (p - <x', p> x')
        if (e.stop) return;
        gradient_norm(e, d, p.j);
        e.xpn = d[p.j + 1];
        e.beta = e.gg_new / e.gg;
        e.coef[C_DIR][0] = make_double2(1.0, 0.0);
        e.coef[C_DIR][1] = make_double2(e.beta, 0.0);
        e.coef[C_DIR][2] = make_double2(-e.beta * e.xpn.x, -e.beta * e.xpn.y);
    } else {  // CTL_END
        ++e.steps;  // operator applications of the loop (one per pass)
        if (!e.stop) e.gg = e.gg_new;
        e.k += 1;
        e.cont = !e.stop && !e.halt && keep_going(e, p);
        cudaGraphSetConditional(h, e.cont ? 1u : 0u);
    }
}

template <int STEP>
__global__ void eig_ctl_kernel(EigDev *ep, const double2 *d, const CtlParams p, cudaGraphConditionalHandle h) {
    ctl_step<STEP>(*ep, d, p, h);
}

// The CG loop's fused steps.  fin_ctl: one block sums the partials of n dot
// products in block order (as dots_finish_kernel does) and thread 0 runs a
// control step on them (CTL_GRAD is followed by CTL_END, which depends only
// on it).  rot_grad_dots: the rotation of the line search and the new
// gradient, x' = r0 x + r1 p^, y' = r0 y + r1 z, g = y' - mu x', with the
// partials of <v_i, g> (i < j), |g|^2 and <x', p^> in the same pass over the
// sites.  proj_dir_dots: the projection of g on the complement of
// v_0 .. v_{j-1} and the new direction p = g' + beta (p - <x', p> x'), with the
// partials of <x, p> and |p|^2 that the next step starts from.  Their linear
// combinations and dot products are those of lincomb_dev_kernel and
// dots_kernel in the same order (real coefficients and real dots skip only
// exact zeros), so the results are unchanged; the step runs 7 small
// launches instead of 16.
template <int STEP>
__global__ void __launch_bounds__(kBlk) fin_ctl_kernel(EigDev *ep, const double *partials, int nb, int n, double2 *d,
                                                       const CtlParams p, cudaGraphConditionalHandle h) {
    // warp w of block_sum holds threads 32 w + lane: one warp per result
    // replays them in turn, so each sum has block_sum's order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < n; k += nw) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < nw; ++w) {
            double re = 0.0, im = 0.0;
            for (int b = 32 * w + lane; b < nb; b += blockDim.x) {
                re += partials[((size_t)k * nb + b) * 2];
                im += partials[((size_t)k * nb + b) * 2 + 1];
            }
            tr += warp_allsum(re);
            ti += warp_allsum(im);
        }
        if (lane == 0) d[k] = make_double2(tr, ti);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl_step<STEP>(*ep, d, p, h);
        if constexpr (STEP == CTL_GRAD) ctl_step<CTL_END>(*ep, d, p, h);
    }
}

struct StepArgs {
    Fields F;
    int j;
    char *x, *y, *g, *p;
    const char *z;
    const char *v[kMaxTerms];
    const EigDev *e;
    double *partials;
    int nb;
};

__device__ __forceinline__ void load_site(const char *f, const Fields &F, int par, int cb, Cx<double> (&s)[12]) {
    SpinorIO<COLA_F64>::load(at(f, F.vh, par), F.vh, cb, s);
}
__device__ __forceinline__ void store_site(char *f, const Fields &F, int par, int cb, const Cx<double> (&s)[12]) {
    SpinorIO<COLA_F64>::store(const_cast<char *>(at(f, F.vh, par)), F.vh, cb, s);
}
// The basis dots <v_i, f> (i < j) of a register spinor f, then the two extra
// results (re, im pairs in extra), as partials j, j + 1.
__device__ __forceinline__ void basis_partials(const StepArgs &A, bool ok, int par, int cb, const Cx<double> (&f)[12],
                                               const double (&extra)[4], double (*sh)[2 * kDotGroup]) {
    const int n = A.j + 2;
    for (int k0 = 0; k0 < n; k0 += kDotGroup) {
        double v[2 * kDotGroup];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) {
            const int k = k0 + q;
            double re = 0.0, im = 0.0;
            if (k < A.j) {
                if (ok) {
                    Cx<double> a[12];
                    load_site(A.v[k], A.F, par, cb, a);
                    site_dot(a, f, re, im);
                }
            } else if (k < n) {
                re = extra[2 * (k - A.j)];
                im = extra[2 * (k - A.j) + 1];
            }
            v[2 * q] = re;
            v[2 * q + 1] = im;
        }
        group_partials(v, k0, n, A.partials, A.nb, sh);
    }
}

// Four spinors and the new gradient are live at once: one block per SM keeps
// them in registers.
__global__ void __launch_bounds__(kBlk, 1) rot_grad_dots_kernel(const __grid_constant__ StepArgs A) {
    __shared__ double sh[kBlk / 32][2 * kDotGroup];
    if (A.e->halt || A.e->stop) return;  // the same for every block
    int par, cb;
    const bool ok = site(A.F, par, cb);
    Cx<double> g[12];
    double extra[4] = {0.0, 0.0, 0.0, 0.0};  // |g|^2, <x', p^>
    if (ok) {
        const double2 *rc = A.e->coef[C_ROT], *gc = A.e->coef[C_GRAD];
        Cx<double> x[12], pp[12], t[12], xr[12];
        load_site(A.x, A.F, par, cb, x);
        load_site(A.p, A.F, par, cb, pp);
        site_mac(xr, rc[0], x, true);
        site_mac(xr, rc[1], pp, false);
        store_site(A.x, A.F, par, cb, xr);
        site_dot(xr, pp, extra[2], extra[3]);
        load_site(A.y, A.F, par, cb, x);  // y
        load_site(A.z, A.F, par, cb, t);  // z
        site_mac(pp, rc[0], x, true);      // y'
        site_mac(pp, rc[1], t, false);
        store_site(A.y, A.F, par, cb, pp);
        site_mac(g, gc[0], pp, true);
        site_mac(g, gc[1], xr, false);
        store_site(A.g, A.F, par, cb, g);
        site_dot_re(g, g, extra[0]);
    }
    basis_partials(A, ok, par, cb, g, extra, sh);
}

__global__ void __launch_bounds__(kBlk, 2) proj_dir_dots_kernel(const __grid_constant__ StepArgs A) {
    __shared__ double sh[kBlk / 32][2 * kDotGroup];
    if (A.e->halt || A.e->stop) return;  // the same for every block
    int par, cb;
    const bool ok = site(A.F, par, cb);
    double v[2 * kDotGroup] = {};
    if (ok) {
        const double2 *pc = A.e->coef[C_PROJ], *dc = A.e->coef[C_DIR];
        Cx<double> acc[12], t[12];
        // g' = sum_k C_PROJ[k] {g, v_0, .., v_{j-1}}_k (g itself when j = 0)
        load_site(A.g, A.F, par, cb, t);
        site_mac(acc, A.j > 0 ? pc[0] : make_double2(1.0, 0.0), t, true);
        for (int i = 0; i < A.j; ++i) {
            load_site(A.v[i], A.F, par, cb, t);
            site_mac(acc, pc[1 + i], t, false);
        }
        // p = sum_k C_DIR[k] {g', p, x}_k, the first term scaled in place
        if (!(dc[0].x == 1.0 && dc[0].y == 0.0)) {
            const Cx<double> w = {dc[0].x, dc[0].y};
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const Cx<double> g = acc[c];
                acc[c] = {0.0, 0.0};
                cmac(acc[c], w, g);
            }
        }
        load_site(A.p, A.F, par, cb, t);
        site_mac(acc, dc[1], t, false);
        load_site(A.x, A.F, par, cb, t);
        site_mac(acc, dc[2], t, false);
        store_site(A.p, A.F, par, cb, acc);
        site_dot(t, acc, v[0], v[1]);  // <x, p>
        site_dot_re(acc, acc, v[2]);   // |p|^2
    }
    group_partials(v, 0, 2, A.partials, A.nb, sh);
}

// Eigen-decomposition of the Hermitian n x n matrix H (row-major, destroyed)
// by cyclic Jacobi rotations; U receives the eigenvectors as columns and w
// the eigenvalues, ascending.  One block of blockDim.x >= n threads.
// A rotation of the pair (p, q), h = H_pq = r e^{i phi}, uses
//   G = [[c, -s e^{i phi}], [s e^{-i phi}, c]],  t = s / c = -sgn(tau) / (|tau| + sqrt(1 + tau^2)),
//   tau = (H_qq - H_pp) / (2 r),
// which makes (G^dag H G)_pq = e^{i phi} (r (c^2 - s^2) + (H_qq - H_pp) c s) vanish.
__global__ void herm_eig_kernel(int n, double2 *H, double2 *U, double *w, int *sweeps_out) {
    __shared__ double rot[4];  // c, s, cos phi, sin phi
    __shared__ int stop;
    const int k = threadIdx.x;
    for (int i = k; i < n * n; i += blockDim.x) U[i] = make_double2((i / n == i % n) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    int sweep = 0;
    for (; sweep < 100; ++sweep) {
        if (k == 0) {
            double off = 0.0, tot = 0.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    const double2 h = H[i * n + j];
                    const double m = h.x * h.x + h.y * h.y;
                    tot += m;
                    if (i != j) off += m;
                }
            stop = !(off > 1e-30 * tot);
        }
        __syncthreads();
        if (stop) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (k == 0) {
                    const double2 h = H[p * n + q];
                    const double r = sqrt(h.x * h.x + h.y * h.y);
                    if (r == 0.0) {
                        rot[0] = 1.0;
                        rot[1] = 0.0;
                        rot[2] = 1.0;
                        rot[3] = 0.0;
                    } else {
                        const double tau = (H[q * n + q].x - H[p * n + p].x) / (2.0 * r);
                        const double t = (tau >= 0.0 ? -1.0 : 1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        const double c = 1.0 / sqrt(1.0 + t * t);
                        rot[0] = c;
                        rot[1] = t * c;
                        rot[2] = h.x / r;
                        rot[3] = h.y / r;
                    }
                }
                __syncthreads();
                const double c = rot[0], s = rot[1], cp = rot[2], sp = rot[3];
                if (s != 0.0 && k < n) {
                    // columns: col_p' = c col_p + s e^{-i phi} col_q;  col_q' = -s e^{i phi} col_p + c col_q
                    const double2 a = H[k * n + p], b = H[k * n + q];
                    H[k * n + p] = make_double2(c * a.x + s * (cp * b.x + sp * b.y), c * a.y + s * (cp * b.y - sp * b.x));
                    H[k * n + q] = make_double2(c * b.x - s * (cp * a.x - sp * a.y), c * b.y - s * (cp * a.y + sp * a.x));
                    const double2 ua = U[k * n + p], ub = U[k * n + q];
                    U[k * n + p] = make_double2(c * ua.x + s * (cp * ub.x + sp * ub.y),
                                                c * ua.y + s * (cp * ub.y - sp * ub.x));
                    U[k * n + q] = make_double2(c * ub.x - s * (cp * ua.x - sp * ua.y),
                                                c * ub.y - s * (cp * ua.y + sp * ua.x));
                }
                __syncthreads();
                if (s != 0.0 && k < n) {
                    // rows: row_p' = c row_p + s e^{i phi} row_q;  row_q' = -s e^{-i phi} row_p + c row_q
                    const double2 a = H[p * n + k], b = H[q * n + k];
                    H[p * n + k] = make_double2(c * a.x + s * (cp * b.x - sp * b.y), c * a.y + s * (cp * b.y + sp * b.x));
                    H[q * n + k] = make_double2(c * b.x - s * (cp * a.x + sp * a.y), c * b.y - s * (cp * a.y - sp * a.x));
                }
                __syncthreads();
                if (s != 0.0 && k == 0) {
                    H[p * n + q] = make_double2(0.0, 0.0);
                    H[q * n + p] = make_double2(0.0, 0.0);
                    H[p * n + p].y = 0.0;
                    H[q * n + q].y = 0.0;
                }
                __syncthreads();
            }
    }
    if (k == 0) {
        // ascending eigenvalues; permute U's columns to match (selection sort)
        for (int i = 0; i < n; ++i) w[i] = H[i * n + i].x;
        for (int i = 0; i < n; ++i) {
            int m = i;
            for (int j = i + 1; j < n; ++j)
                if (w[j] < w[m]) m = j;
            if (m != i) {
                const double t = w[i];
                w[i] = w[m];
                w[m] = t;
                for (int r = 0; r < n; ++r) {
                    const double2 x = U[r * n + i];
                    U[r * n + i] = U[r * n + m];
                    U[r * n + m] = x;
                }
            }
        }
        *sweeps_out = sweep;
    }
}

struct Ctx {
    cola_gauge g;
    int op, nev;
    Fields F;
    size_t fb;
    int nb;
    std::vector<char *> V, W, T;
    char *x_y, *g_, *p, *z, *t, *mp;
    double *partials;
    double2 *dres;     // device results (dots)
    double2 *H, *Ud;   // N x N
    double *wd;
    int *sweeps;
    EigDev *e;         // scalars of the current minimisation
    cudaStream_t s;
    long applications = 0;
    std::vector<cudaGraphExec_t> ritz;  // one minimisation graph per vector index, built on first use
    ~Ctx() {
        for (cudaGraphExec_t x : ritz)
            if (x) cudaGraphExecDestroy(x);
    }
};

cola_status apply_a(Ctx &c, char *out, const char *in) {
    ++c.applications;
    return apply_mdagm(c.g, COLA_F64, c.op, out, in, c.t, c.mp, 1, nullptr, false, c.s);
}

// host copies of n complex dots conj(a_k) b_k
cola_status dots(Ctx &c, const std::vector<std::pair<const char *, const char *>> &ab, std::vector<double2> &out) {
    const int n = (int)ab.size();
    out.assign(n, make_double2(0.0, 0.0));
    if (n == 0) return COLA_OK;
    for (int k0 = 0; k0 < n; k0 += kMaxTerms) {
        const int m = std::min(kMaxTerms, n - k0);
        DotArgs A;
        std::memset(&A, 0, sizeof(A));
        A.F = c.F;
        A.n = m;
        for (int k = 0; k < m; ++k) {
            A.a[k] = ab[k0 + k].first;
            A.b[k] = ab[k0 + k].second;
        }
        A.partials = c.partials;
        A.nb = c.nb;
        dots_kernel<<<c.nb, kBlk, 0, c.s>>>(A);
        dots_finish_kernel<<<m, kBlk, 0, c.s>>>(c.partials, c.nb, c.dres);
        EIG_CUDA(cudaGetLastError(), "eigensolver reduction");
        EIG_CUDA(cudaMemcpyAsync(out.data() + k0, c.dres, m * sizeof(double2), cudaMemcpyDeviceToHost, c.s),
                 "reduction readback");
    }
    EIG_CUDA(cudaStreamSynchronize(c.s), "eigensolver reduction");
    return COLA_OK;
}

cola_status comb(Ctx &c, char *out, const std::vector<std::pair<const char *, double2>> &terms) {
    CombArgs A;
    std::memset(&A, 0, sizeof(A));
    A.F = c.F;
    A.n = (int)terms.size();
    A.out = out;
    for (int k = 0; k < A.n; ++k) {
        A.in[k] = terms[k].first;
        A.c[k] = terms[k].second;
    }
    lincomb_kernel<<<c.nb, kBlk, 0, c.s>>>(A);
    return cuda_check(cudaGetLastError(), "eigensolver linear combination");
}

double2 cplx(double re, double im = 0.0) { return make_double2(re, im); }

// x <- x - sum_{i<j} <v_i, x> v_i, twice (classical Gram-Schmidt, repeated)
cola_status project(Ctx &c, char *x, int j) {
    for (int rep = 0; rep < 2 && j > 0; ++rep) {
        std::vector<std::pair<const char *, const char *>> ab;
        for (int i = 0; i < j; ++i) ab.push_back({c.V[i], x});
        std::vector<double2> d;
        EIG_TRY(dots(c, ab, d));
        std::vector<std::pair<const char *, double2>> t = {{x, cplx(1.0)}};
        for (int i = 0; i < j; ++i) t.push_back({c.V[i], cplx(-d[i].x, -d[i].y)});
        EIG_TRY(comb(c, x, t));
    }
    return COLA_OK;
}

cola_status normalize(Ctx &c, char *x) {
    std::vector<double2> d;
    EIG_TRY(dots(c, {{x, x}}, d));
    if (!(d[0].x > 0.0) || !std::isfinite(d[0].x)) {
        set_error("eigensolver: a vector vanished after orthogonalisation (dependent initial vectors?)");
        return COLA_ERR_BREAKDOWN;
    }
    return comb(c, x, {{x, cplx(1.0 / std::sqrt(d[0].x))}});
}

// ------------------------------------------------ device-driven minimisation --
// Launches on stream st (capturing or not) with results left on the device.
void dots_dev(Ctx &c, cudaStream_t st, const std::vector<std::pair<const char *, const char *>> &ab,
              unsigned re_only = 0) {
    DotArgs A;
    std::memset(&A, 0, sizeof(A));
    A.re_only = re_only;
    A.F = c.F;
    A.n = (int)ab.size();
    for (int k = 0; k < A.n; ++k) {
        A.a[k] = ab[k].first;
        A.b[k] = ab[k].second;
    }
    A.partials = c.partials;
    A.nb = c.nb;
    dots_kernel<<<c.nb, kBlk, 0, st>>>(A);
    dots_finish_kernel<<<A.n, kBlk, 0, st>>>(c.partials, c.nb, c.dres);
}

void comb_dev(Ctx &c, cudaStream_t st, char *out, const std::vector<const char *> &in, int set, int mask) {
    CombDevArgs A;
    std::memset(&A, 0, sizeof(A));
    A.F = c.F;
    A.n = (int)in.size();
    A.out = out;
    for (int k = 0; k < A.n; ++k) A.in[k] = in[k];
    A.e = c.e;
    A.set = set;
    A.mask = mask;
    lincomb_dev_kernel<<<c.nb, kBlk, 0, st>>>(A);
}

template <int STEP>
void ctl(Ctx &c, cudaStream_t st, const CtlParams &p, cudaGraphConditionalHandle h = 0) {
    eig_ctl_kernel<STEP><<<1, 1, 0, st>>>(c.e, c.dres, p, h);
}

// The dots' block partials only (a fin_ctl launch finishes them).
void dots_part(Ctx &c, cudaStream_t st, const std::vector<std::pair<const char *, const char *>> &ab,
               unsigned re_only = 0) {
    DotArgs A;
    std::memset(&A, 0, sizeof(A));
    A.re_only = re_only;
    A.F = c.F;
    A.n = (int)ab.size();
    for (int k = 0; k < A.n; ++k) {
        A.a[k] = ab[k].first;
        A.b[k] = ab[k].second;
    }
    A.partials = c.partials;
    A.nb = c.nb;
    dots_kernel<<<c.nb, kBlk, 0, st>>>(A);
}

template <int STEP>
void fin_ctl(Ctx &c, cudaStream_t st, int n, const CtlParams &p, cudaGraphConditionalHandle h = 0) {
    fin_ctl_kernel<STEP><<<1, kBlk, 0, st>>>(c.e, c.partials, c.nb, n, c.dres, p, h);
}

StepArgs step_args(Ctx &c, int j, char *x) {
    StepArgs A;
    std::memset(&A, 0, sizeof(A));
    A.F = c.F;
    A.j = j;
    A.x = x;
    A.y = c.x_y;
    A.g = c.g_;
    A.p = c.p;
    A.z = c.z;
    for (int i = 0; i < j; ++i) A.v[i] = c.V[i];
    A.e = c.e;
    A.partials = c.partials;
    A.nb = c.nb;
    return A;
}

// {<v_i, f>} for i < j, then |f|^2, then the extra pairs
std::vector<std::pair<const char *, const char *>> against_basis(Ctx &c, int j, const char *f) {
    std::vector<std::pair<const char *, const char *>> ab;
    for (int i = 0; i < j; ++i) ab.push_back({c.V[i], f});
    ab.push_back({f, f});
    return ab;
}

std::vector<const char *> with_basis(Ctx &c, int j, const char *f) {
    std::vector<const char *> in = {f};
    for (int i = 0; i < j; ++i) in.push_back(c.V[i]);
    return in;
}

// The minimisation of v_j as one graph: project v_j on the complement of
// v_0 .. v_{j-1} (classical Gram-Schmidt, twice), normalise, y = A x, the
// projected gradient g = Q (y - mu x), p = g, then while the gradient has not
// fallen by gamma (and fewer than max_cg steps ran): p <- p - <x, p> x,
// z = A p, the exact line search on span(x, p^), x and y rotated, the new
// projected gradient, p = g' + beta (p - <x', p> x'); finally v_j is
// normalised again.  Every scalar stays on the device (EigDev).
cola_status build_ritz_graph(Ctx &c, int j, const CtlParams &p, cudaGraphExec_t *out) {
    char *x = c.V[j], *y = c.x_y, *g = c.g_, *pp = c.p, *z = c.z;
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphExec_t exec = nullptr;
    cola_status st = COLA_OK;
    auto fail = [&](cola_status e) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        return e;
    };
    if ((st = cuda_check(cudaGraphCreate(&graph, 0), "graph create")) != COLA_OK) return fail(st);
    cudaGraphConditionalHandle h;
    if ((st = cuda_check(cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault),
                         "graph conditional")) != COLA_OK)
        return fail(st);
    if ((st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream")) != COLA_OK)
        return fail(st);
    if ((st = cuda_check(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                         "capture")) != COLA_OK)
        return fail(st);
    // prologue
    for (int rep = 0; rep < 2 && j > 0; ++rep) {
        std::vector<std::pair<const char *, const char *>> ab;
        for (int i = 0; i < j; ++i) ab.push_back({c.V[i], x});
        dots_dev(c, cs, ab);
        ctl<CTL_PROJ>(c, cs, p);
        comb_dev(c, cs, x, with_basis(c, j, x), C_PROJ, 1);
    }
    dots_dev(c, cs, {{x, x}}, 1u);
    ctl<CTL_NORM>(c, cs, p);
    comb_dev(c, cs, x, {x}, C_NORM, 1);
    st = apply_mdagm(c.g, COLA_F64, c.op, y, x, c.t, c.mp, 1, nullptr, false, cs);
    if (st == COLA_OK) {
        dots_dev(c, cs, {{x, y}}, 1u);  // mu: the real part
        ctl<CTL_MU>(c, cs, p);
        comb_dev(c, cs, g, {y, x}, C_GRAD, 1);
        dots_dev(c, cs, against_basis(c, j, g), j < 32 ? 1u << j : 0u);  // |g|^2 real
        ctl<CTL_GRAD0>(c, cs, p);
        if (j > 0) comb_dev(c, cs, g, with_basis(c, j, g), C_PROJ, 1);
        st = cuda_check(cudaMemcpyAsync(pp, g, c.fb, cudaMemcpyDeviceToDevice, cs), "p = g");
        if (st == COLA_OK) dots_part(c, cs, {{x, pp}, {pp, pp}});  // the loop's first step starts from these
    }
    if (st == COLA_OK) {
        ctl<CTL_LOOP0>(c, cs, p, h);
        st = cuda_check(cudaGetLastError(), "eigensolver prologue");
    }
    // the loop as a while node after the prologue
    cudaGraph_t body = nullptr;
    if (st == COLA_OK) {
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edata = nullptr;
        size_t ndeps = 0;
        cudaGraph_t capg;
        st = cuda_check(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, &edata, &ndeps), "capture info");
        if (st == COLA_OK) {
            cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
            wp.conditional.handle = h;
            wp.conditional.type = cudaGraphCondTypeWhile;
            wp.conditional.size = 1;
            cudaGraphNode_t wnode;
            st = cuda_check(cudaGraphAddNode(&wnode, capg, deps, edata, ndeps, &wp), "graph while node");
            if (st == COLA_OK) {
                body = wp.conditional.phGraph_out[0];
                st = cuda_check(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1,
                                                                    cudaStreamSetCaptureDependencies),
                                "capture dependencies");
            }
        }
    }
    // epilogue: normalise v_j
    if (st == COLA_OK) {
        dots_dev(c, cs, {{x, x}}, 1u);
        ctl<CTL_NORM>(c, cs, p);
        comb_dev(c, cs, x, {x}, C_NORM, 1);
        st = cuda_check(cudaGetLastError(), "eigensolver epilogue");
    }
    {
        cudaGraph_t g_out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g_out);
        if (st == COLA_OK) st = cuda_check(e, "end capture");
    }
    if (st != COLA_OK) return fail(st);
    // the loop body
    if ((st = cuda_check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                         "capture")) != COLA_OK)
        return fail(st);
    fin_ctl<CTL_PERP>(c, cs, 2, p);  // <x, p>, |p|^2: partials of the prologue or of the previous step
    comb_dev(c, cs, pp, {pp, x}, C_PERP, 3);
    st = apply_mdagm(c.g, COLA_F64, c.op, z, pp, c.t, c.mp, 1, nullptr, false, cs);  // z = A p = pn A p^
    if (st == COLA_OK) {
        dots_part(c, cs, {{x, z}, {pp, z}}, 3u);  // the line search uses the real parts
        fin_ctl<CTL_ROT>(c, cs, 2, p);
        rot_grad_dots_kernel<<<c.nb, kBlk, 0, cs>>>(step_args(c, j, x));  // x, y, g; <v_i, g>, |g|^2, <x, p>
        fin_ctl<CTL_GRAD>(c, cs, j + 2, p, h);                            // and CTL_END: the loop condition
        proj_dir_dots_kernel<<<c.nb, kBlk, 0, cs>>>(step_args(c, j, x));  // p; <x, p>, |p|^2
        st = cuda_check(cudaGetLastError(), "eigensolver step");
    }
    {
        cudaGraph_t g_out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g_out);
        if (st == COLA_OK) st = cuda_check(e, "end capture");
    }
    if (st != COLA_OK) return fail(st);
    if ((st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate")) != COLA_OK) return fail(st);
    *out = exec;
    exec = nullptr;
    fail(COLA_OK);  // the graph and the capture stream are no longer needed
    return COLA_OK;
}

cola_status arg_error(const std::string &m) {
    set_error(m);
    return COLA_ERR_ARG;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" cola_status cola_eig_lowest(cola_gauge g, void *evecs_dev, double *evals, const cola_eig_params *prm,
                                       cola_eig_info *info, cudaStream_t s) {
    TraceRange trace_("cola_eig_lowest");
    const auto t0 = std::chrono::steady_clock::now();
    if (!g || !evecs_dev || !evals || !prm || !info) return arg_error("null argument to cola_eig_lowest");
    if (prm->nev < 1 || prm->nextra < 0 || prm->nev + prm->nextra > kMaxNev)
        return arg_error("nev must be >= 1, nextra >= 0 and nev + nextra <= 64");
    if (prm->op != COLA_OP_FULL && prm->op != COLA_OP_EO) return arg_error("op must be COLA_OP_FULL or COLA_OP_EO");
    if (!(prm->tol > 0.0 && prm->tol < 1.0)) return arg_error("tol must be in (0, 1)");
    if (prm->max_sweeps < 1 || prm->max_cg < 1) return arg_error("max_sweeps and max_cg must be >= 1");
    if (!(prm->gamma > 0.0 && prm->gamma < 1.0)) return arg_error("gamma must be in (0, 1)");
    if (!g->links[COLA_F64]) {
        set_error("cola_eig_lowest needs FP64 links in the gauge handle");
        return COLA_ERR_UNSUPPORTED;
    }
    const Geom &G = g->geom;
    const int N = prm->nev + prm->nextra;  // vectors iterated; the first nev are tested
    Ctx c;
    c.g = g;
    c.op = prm->op;
    c.nev = N;
    c.s = s;
    c.F = {G.Vh, prm->op == COLA_OP_EO ? 1 : 2};
    c.fb = 2 * spinor_parity_bytes(COLA_F64, G.Vh);
    c.nb = (G.Vh * c.F.nparity + kBlk - 1) / kBlk;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t nfield = 3 * (size_t)N + 6;
    const size_t o_part = al(c.fb) * nfield;
    const size_t o_res = o_part + al((size_t)kMaxTerms * c.nb * 2 * sizeof(double));
    const size_t o_h = o_res + al(kMaxTerms * sizeof(double2));
    const size_t o_u = o_h + al((size_t)N * N * sizeof(double2));
    const size_t o_w = o_u + al((size_t)N * N * sizeof(double2));
    const size_t o_sw = o_w + al(N * sizeof(double));
    const size_t o_e = o_sw + 256;
    const size_t total = o_e + al(sizeof(EigDev));
    void *ws = nullptr;
    EIG_TRY(ws_slot(g, cola_gauge_s::kSlotMultishift, total, &ws));  // shares the multi-shift block
    char *w = static_cast<char *>(ws);
    size_t o = 0;
    for (int i = 0; i < N; ++i, o += al(c.fb)) c.V.push_back(w + o);
    for (int i = 0; i < N; ++i, o += al(c.fb)) c.W.push_back(w + o);
    for (int i = 0; i < N; ++i, o += al(c.fb)) c.T.push_back(w + o);
    char *extra[6];
    for (int i = 0; i < 6; ++i, o += al(c.fb)) extra[i] = w + o;
    c.x_y = extra[0];
    c.g_ = extra[1];
    c.p = extra[2];
    c.z = extra[3];
    c.t = extra[4];
    c.mp = extra[5];
    c.partials = reinterpret_cast<double *>(w + o_part);
    c.dres = reinterpret_cast<double2 *>(w + o_res);
    c.H = reinterpret_cast<double2 *>(w + o_h);
    c.Ud = reinterpret_cast<double2 *>(w + o_u);
    c.wd = reinterpret_cast<double *>(w + o_w);
    c.sweeps = reinterpret_cast<int *>(w + o_sw);
    c.e = reinterpret_cast<EigDev *>(w + o_e);
    c.ritz.assign(N, nullptr);

    const size_t canon = (size_t)G.V * 12 * 16;
    const int pmask = c.F.nparity == 1 ? 1 : 3;
    for (int i = 0; i < N; ++i)
        EIG_CUDA(launch_pack_spinor(COLA_F64, G, c.V[i], static_cast<char *>(evecs_dev) + i * canon, 1, pmask, s),
                 "pack initial vectors");
    for (int i = 0; i < N; ++i) {
        // a starting vector (nearly) in the span of the earlier ones cannot be used
        std::vector<double2> n0, n1;
        EIG_TRY(dots(c, {{c.V[i], c.V[i]}}, n0));
        EIG_TRY(project(c, c.V[i], i));
        EIG_TRY(dots(c, {{c.V[i], c.V[i]}}, n1));
        if (!(n1[0].x > 1e-20 * n0[0].x)) {
            set_error("eigensolver: a starting vector vanished after orthogonalisation (dependent starting vectors)");
            return COLA_ERR_BREAKDOWN;
        }
        EIG_TRY(normalize(c, c.V[i]));
    }
    std::vector<double> lam(N, 0.0), res(N, 0.0);
    EIG_CUDA(cudaMemsetAsync(c.e, 0, sizeof(EigDev), s), "eigensolver state");
    {
        // the operator's launch shape is tuned outside the graph captures
        TuneOnlyScope tune_only;
        EIG_TRY(apply_mdagm(g, COLA_F64, c.op, c.z, c.V[0], c.t, c.mp, 1, nullptr, false, s));
    }
    int sweep = 0;
    bool converged = false;
    for (; sweep < prm->max_sweeps && !converged; ++sweep) {
        for (int j = 0; j < N; ++j) {
            if (!c.ritz[j]) {
                const CtlParams cp = {j, prm->max_cg, prm->gamma, prm->tol};
                EIG_TRY(build_ritz_graph(c, j, cp, &c.ritz[j]));
            }
            EIG_CUDA(cudaGraphLaunch(c.ritz[j], s), "eigensolver minimisation");
            ++c.applications;  // y = A x of the prologue; the loop's are counted on the device
        }
        // Rayleigh-Ritz on span(V)
        for (int i = 0; i < N; ++i) EIG_TRY(apply_a(c, c.W[i], c.V[i]));
        std::vector<std::pair<const char *, const char *>> ab;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) ab.push_back({c.V[i], c.W[j]});
        std::vector<double2> h;
        EIG_TRY(dots(c, ab, h));
        for (int i = 0; i < N; ++i)  // exactly Hermitian
            for (int j = i; j < N; ++j) {
                const double2 a = h[i * N + j], b = h[j * N + i];
                h[i * N + j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
                h[j * N + i] = make_double2(h[i * N + j].x, -h[i * N + j].y);
            }
        EIG_CUDA(cudaMemcpyAsync(c.H, h.data(), N * N * sizeof(double2), cudaMemcpyHostToDevice, s), "H upload");
        herm_eig_kernel<<<1, std::max(32, ((N + 31) / 32) * 32), 0, s>>>(N, c.H, c.Ud, c.wd, c.sweeps);
        EIG_CUDA(cudaGetLastError(), "Rayleigh-Ritz eigen-decomposition");
        std::vector<double2> U(N * N);
        EIG_CUDA(cudaMemcpyAsync(U.data(), c.Ud, N * N * sizeof(double2), cudaMemcpyDeviceToHost, s), "U readback");
        EIG_CUDA(cudaMemcpyAsync(lam.data(), c.wd, N * sizeof(double), cudaMemcpyDeviceToHost, s), "lambda readback");
        EIG_CUDA(cudaStreamSynchronize(s), "Rayleigh-Ritz");
        // V <- V U, W <- W U through T (V is copied back: the minimisation
        // graphs hold the addresses of the V buffers; W swaps)
        for (int j = 0; j < N; ++j) {
            std::vector<std::pair<const char *, double2>> t;
            for (int i = 0; i < N; ++i) t.push_back({c.V[i], U[i * N + j]});
            EIG_TRY(comb(c, c.T[j], t));
        }
        for (int j = 0; j < N; ++j)
            EIG_CUDA(cudaMemcpyAsync(c.V[j], c.T[j], c.fb, cudaMemcpyDeviceToDevice, s), "V = V U");
        for (int j = 0; j < N; ++j) {
            std::vector<std::pair<const char *, double2>> t;
            for (int i = 0; i < N; ++i) t.push_back({c.W[i], U[i * N + j]});
            EIG_TRY(comb(c, c.T[j], t));
        }
        std::swap(c.W, c.T);
        // residuals |W_j - lambda_j V_j| (V_j is unit)
        for (int j = 0; j < N; ++j) EIG_TRY(comb(c, c.T[j], {{c.W[j], cplx(1.0)}, {c.V[j], cplx(-lam[j])}}));
        ab.clear();
        for (int j = 0; j < N; ++j) ab.push_back({c.T[j], c.T[j]});
        EIG_TRY(dots(c, ab, h));
        EigDev he;
        EIG_CUDA(cudaMemcpyAsync(&he, c.e, sizeof(EigDev), cudaMemcpyDeviceToHost, s), "eigensolver state");
        EIG_CUDA(cudaStreamSynchronize(s), "eigensolver state");
        if (he.status != COLA_OK) {
            set_error("eigensolver: a vector vanished after orthogonalisation (dependent initial vectors?)");
            return (cola_status)he.status;
        }
        converged = true;
        for (int j = 0; j < N; ++j) {
            res[j] = std::sqrt(std::max(0.0, h[j].x));
            if (j < prm->nev) converged &= res[j] <= prm->tol * std::fabs(lam[j]);
        }
    }
    {
        EigDev he;
        EIG_CUDA(cudaMemcpyAsync(&he, c.e, sizeof(EigDev), cudaMemcpyDeviceToHost, s), "eigensolver state");
        EIG_CUDA(cudaStreamSynchronize(s), "eigensolver state");
        c.applications += he.steps;
    }
    for (int i = 0; i < N; ++i) {
        char *dst = static_cast<char *>(evecs_dev) + i * canon;
        if (c.F.nparity == 1) EIG_CUDA(cudaMemsetAsync(dst, 0, canon, s), "zero odd sites");
        EIG_CUDA(launch_unpack_spinor(COLA_F64, G, dst, c.V[i], 1, pmask, s), "unpack eigenvectors");
        evals[i] = lam[i];
    }
    EIG_CUDA(cudaStreamSynchronize(s), "eigensolver");
    double worst = 0.0;
    for (int j = 0; j < prm->nev; ++j) worst = std::max(worst, res[j] / std::max(std::fabs(lam[j]), 1e-300));
    info->sweeps = sweep;
    info->applications = (int)c.applications;
    info->max_rel_resid = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->status = converged ? COLA_OK : COLA_ERR_NOT_CONVERGED;
    if (log_enabled())
        log_line("eig_lowest: status %d, %d sweeps, %d operator applications, lambda_0 %.6e, max relative residual "
                 "%.3e, %.3f s", info->status, info->sweeps, info->applications, lam[0], worst, info->seconds);
    if (!converged) set_error("eigensolver did not converge within max_sweeps");
    return (cola_status)info->status;
}
