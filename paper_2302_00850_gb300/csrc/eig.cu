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
// fixed order (block partials, one finishing block per result).  The host
// drives the sweep and reads the few scalars of each step.
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
};

__global__ void __launch_bounds__(kBlk) dots_kernel(const __grid_constant__ DotArgs A) {
    __shared__ double sh[kBlk / 32];
    int par, cb;
    const bool ok = site(A.F, par, cb);
    for (int k = 0; k < A.n; ++k) {
        double re = 0.0, im = 0.0;
        if (ok) {
            Cx<double> x[12], y[12];
            SpinorIO<COLA_F64>::load(at(A.a[k], A.F.vh, par), A.F.vh, cb, x);
            SpinorIO<COLA_F64>::load(at(A.b[k], A.F.vh, par), A.F.vh, cb, y);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                re = fma(x[c].re, y[c].re, fma(x[c].im, y[c].im, re));
                im = fma(x[c].re, y[c].im, fma(-x[c].im, y[c].re, im));
            }
        }
        const double tr = block_sum(re, sh);
        __syncthreads();
        const double ti = block_sum(im, sh);
        __syncthreads();
        if (threadIdx.x == 0) {
            A.partials[((size_t)k * A.nb + blockIdx.x) * 2] = tr;
            A.partials[((size_t)k * A.nb + blockIdx.x) * 2 + 1] = ti;
        }
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
        const Cx<double> w = {A.c[k].x, A.c[k].y};
#pragma unroll
        for (int c = 0; c < 12; ++c) cmac(acc[c], w, x[c]);
    }
    SpinorIO<COLA_F64>::store(const_cast<char *>(at(A.out, A.F.vh, par)), A.F.vh, cb, acc);
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
    cudaStream_t s;
    long applications = 0;
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

// Ritz-functional CG for v_j over the complement of v_0 .. v_{j-1}.  Three
// host reads per step: {<x, p>, |p|^2}, {<x, A p>, <p, A p>} and
// {<v_i, g> (i < j), |g|^2, <x, p>}; the norms after a projection follow from
// those (|p - <x,p> x|^2 = |p|^2 - |<x,p>|^2 for unit x, and likewise for g).
cola_status ritz_cg(Ctx &c, int j, int max_cg, double gamma, double tol) {
    char *x = c.V[j], *y = c.x_y, *g = c.g_, *p = c.p, *z = c.z;
    EIG_TRY(project(c, x, j));
    EIG_TRY(normalize(c, x));
    EIG_TRY(apply_a(c, y, x));
    std::vector<double2> d;
    EIG_TRY(dots(c, {{x, y}}, d));
    double mu = d[0].x;
    // g = Q (y - mu x), one classical Gram-Schmidt pass
    auto gradient = [&](double &gg, double2 *xp) -> cola_status {
        EIG_TRY(comb(c, g, {{y, cplx(1.0)}, {x, cplx(-mu)}}));
        std::vector<std::pair<const char *, const char *>> ab;
        for (int i = 0; i < j; ++i) ab.push_back({c.V[i], g});
        ab.push_back({g, g});
        if (xp) ab.push_back({x, p});
        EIG_TRY(dots(c, ab, d));
        double n2 = d[j].x;
        if (j > 0) {
            std::vector<std::pair<const char *, double2>> t = {{g, cplx(1.0)}};
            for (int i = 0; i < j; ++i) {
                t.push_back({c.V[i], cplx(-d[i].x, -d[i].y)});
                n2 -= d[i].x * d[i].x + d[i].y * d[i].y;
            }
            EIG_TRY(comb(c, g, t));
        }
        gg = std::max(n2, 0.0);
        if (xp) *xp = d[j + 1];
        return COLA_OK;
    };
    double gg0 = 0.0;
    EIG_TRY(gradient(gg0, nullptr));
    double gg = gg0;
    EIG_CUDA(cudaMemcpyAsync(p, g, c.fb, cudaMemcpyDeviceToDevice, c.s), "p = g");
    for (int k = 0; k < max_cg; ++k) {
        if (gg <= gamma * gamma * gg0 || std::sqrt(gg) <= 0.1 * tol * std::fabs(mu) || gg == 0.0) break;
        // p <- p - <x, p> x (keep p orthogonal to x)
        EIG_TRY(dots(c, {{x, p}, {p, p}}, d));
        const double2 xp = d[0];
        const double pn2 = d[1].x - (xp.x * xp.x + xp.y * xp.y);
        if (!(pn2 > 0.0)) break;
        EIG_TRY(comb(c, p, {{p, cplx(1.0)}, {x, cplx(-xp.x, -xp.y)}}));
        const double pn = std::sqrt(pn2);
        EIG_TRY(apply_a(c, z, p));  // z = A p = pn A p^
        EIG_TRY(dots(c, {{x, z}, {p, z}}, d));
        const double a = mu, b = d[0].x / pn, cc = d[1].x / pn2;
        const double h = 0.5 * (a - cc), R = std::sqrt(h * h + b * b);
        if (!(R > 0.0)) break;
        // cos 2t = -h / R, sin 2t = -b / R; half angle with cos t >= 0
        const double c2 = -h / R, s2 = -b / R;
        const double ct = std::sqrt(std::max(0.0, 0.5 * (1.0 + c2)));
        const double st = ct > 1e-8 ? s2 / (2.0 * ct) : (s2 >= 0.0 ? 1.0 : -1.0) * std::sqrt(std::max(0.0, 0.5 * (1.0 - c2)));
        EIG_TRY(comb(c, x, {{x, cplx(ct)}, {p, cplx(st / pn)}}));
        EIG_TRY(comb(c, y, {{y, cplx(ct)}, {z, cplx(st / pn)}}));
        mu = 0.5 * (a + cc) - R;
        double gg_new = 0.0;
        double2 xpn;
        EIG_TRY(gradient(gg_new, &xpn));  // also <x', p>
        const double beta = gg_new / gg;
        // p = g' + beta (p - <x', p> x')
        EIG_TRY(comb(c, p, {{g, cplx(1.0)}, {p, cplx(beta)}, {x, cplx(-beta * xpn.x, -beta * xpn.y)}}));
        gg = gg_new;
    }
    return normalize(c, x);
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
    const size_t total = o_sw + 256;
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
    int sweep = 0;
    bool converged = false;
    for (; sweep < prm->max_sweeps && !converged; ++sweep) {
        for (int j = 0; j < N; ++j) EIG_TRY(ritz_cg(c, j, prm->max_cg, prm->gamma, prm->tol));
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
        // V <- V U, W <- W U (through T, then swap)
        for (int j = 0; j < N; ++j) {
            std::vector<std::pair<const char *, double2>> t;
            for (int i = 0; i < N; ++i) t.push_back({c.V[i], U[i * N + j]});
            EIG_TRY(comb(c, c.T[j], t));
        }
        std::swap(c.V, c.T);
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
        converged = true;
        for (int j = 0; j < N; ++j) {
            res[j] = std::sqrt(std::max(0.0, h[j].x));
            if (j < prm->nev) converged &= res[j] <= prm->tol * std::fabs(lam[j]);
        }
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
