// Gauge-field kernels of Hybrid Monte Carlo: the Wilson gauge action
// (plaquette sum) and its force, the link update U <- exp(i eps P) U, and
// deterministic FP64 dot products (kinetic energy, |eta|^2, phi^dag X).
//
// HMC is one of COLA's key algorithms (the paper's overview of the library);
// the paper writes no formula.  Definitions, with the links WITHOUT fermion
// boundary phases and the link-variation convention of the fermion force
// (U_mu(x) -> (1 + i eps T^a) U_mu(x), T^a = lambda^a / 2):
//   S_G = beta sum_x sum_{mu<nu} (1 - Re tr U_munu(x) / 3),
//   dS_G/deps^a = (beta / 3) Im Tr[T^a U_mu(x) V_mu(x)],
//   V_mu(x) = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//                          + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu).
// Momenta and forces are [4][V][8] real generator coefficients, links in the
// canonical [4][V][3][3] complex layout; all FP64, one thread per link.
#include "cola_impl.h"

namespace cola {

namespace {

constexpr int kThreads = 128;
constexpr int kRedThreads = 256;

__device__ __forceinline__ void lex_coords(const Geom &g, int i, int (&c)[4]) {
    c[0] = i % g.L[0];
    int r = i / g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
}

struct LinkField {
    Geom g;
    const char *links;  // packed FP64
    size_t dir_stride;
};

template <int RECON>
__device__ __forceinline__ void link_rel(const LinkField &F, const int (&c)[4], int mu, int d1, int s1, int d2,
                                         int s2, Cx<double> (&u)[9]) {
    int p[4] = {c[0], c[1], c[2], c[3]};
    p[d1] += s1;
    p[d2] += s2;
    link_at<RECON>(F.g, F.links, F.dir_stride, p, mu, u);
}

template <int RECON>
__global__ void __launch_bounds__(kThreads) gauge_force_kernel(const LinkField F, double coef, double *out,
                                                               int accumulate) {
    const Geom &g = F.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (i >= g.V) return;
    int c[4];
    lex_coords(g, i, c);
    Cx<double> v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = {0.0, 0.0};
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        Cx<double> w[9], u[9];
        // U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        link_rel<RECON>(F, c, nu, mu, 1, nu, 0, u);
        mat3_set(w, u, false);
        link_rel<RECON>(F, c, mu, nu, 1, mu, 0, u);
        mat3_rmul(w, u, true);
        link_rel<RECON>(F, c, nu, mu, 0, nu, 0, u);
        mat3_rmul(w, u, true);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            v[k].re += w[k].re;
            v[k].im += w[k].im;
        }
        // U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        link_rel<RECON>(F, c, nu, mu, 1, nu, -1, u);
        mat3_set(w, u, true);
        link_rel<RECON>(F, c, mu, nu, -1, mu, 0, u);
        mat3_rmul(w, u, true);
        link_rel<RECON>(F, c, nu, nu, -1, mu, 0, u);
        mat3_rmul(w, u, false);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            v[k].re += w[k].re;
            v[k].im += w[k].im;
        }
    }
    Cx<double> m[9], u[9];
    link_rel<RECON>(F, c, mu, 0, 0, 0, 0, u);
    mat3_set(m, u, false);
    mat3_rmul(m, v, false);
    double f[8];
    im_tr_lambda(m, f);  // Im Tr[lambda^a U V] = 2 Im Tr[T^a U V]
    store_force(out + ((size_t)mu * g.V + i) * 8, f, coef / 6.0, accumulate != 0);
}

// per site: sum over the six planes of Re tr U_munu(x) (block partial sums)
template <int RECON>
__global__ void __launch_bounds__(kRedThreads) plaquette_kernel(const LinkField F, double *partials) {
    __shared__ double sh[kRedThreads / 32];
    const Geom &g = F.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < g.V) {
        int c[4];
        lex_coords(g, i, c);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                Cx<double> w[9], u[9];
                link_rel<RECON>(F, c, mu, 0, 0, 0, 0, u);
                mat3_set(w, u, false);
                link_rel<RECON>(F, c, nu, mu, 1, mu, 0, u);
                mat3_rmul(w, u, false);
                link_rel<RECON>(F, c, mu, nu, 1, nu, 0, u);
                mat3_rmul(w, u, true);
                link_rel<RECON>(F, c, nu, 0, 0, 0, 0, u);
                mat3_rmul(w, u, true);
                s += w[0].re + w[4].re + w[8].re;
            }
    }
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// sum_k a[k] b[k] over n doubles (block partial sums)
__global__ void __launch_bounds__(kRedThreads) dot_kernel(const double *a, const double *b, size_t n,
                                                          double *partials) {
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) s = fma(a[k], b[k], s);
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// out[0] = scale * sum of n partials, in a fixed order
__global__ void __launch_bounds__(kRedThreads) finish_sum_kernel(const double *partials, int n, double scale,
                                                                 double *out) {
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += partials[k];
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) out[0] = scale * t;
}

// E = exp(A) for traceless 3x3 A (here anti-Hermitian).  By Cayley-Hamilton,
// A^3 = s A + d I with s = tr(A^2) / 2 and d = det A, so every power is
// A^k = al_k I + be_k A + ga_k A^2 with
//   (al, be, ga)_{k+1} = (ga_k d, al_k + ga_k s, be_k),
// and exp(A) = a I + b A + c A^2 with (a, b, c) = sum_k (al, be, ga)_k / k!:
// a scalar series (three complex numbers) and one 3x3 product.  A is first
// scaled by 2^-q to a Frobenius norm of at most 1 (at most 30 terms, fewer
// once a term falls below 1e-18; at the usual eps |P| ~ 0.1 about 10) and
// the result squared q times.
__device__ void exp_traceless(Cx<double> (&a)[9], Cx<double> (&e)[9]) {
    double n2 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) n2 += a[k].re * a[k].re + a[k].im * a[k].im;
    int q = 0;
    while (n2 > 1.0 && q < 60) {
        n2 *= 0.25;
        ++q;
    }
    const double sc = ldexp(1.0, -q);
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = {a[k].re * sc, a[k].im * sc};
    Cx<double> a2[9];
    mat3_set(a2, a, false);
    mat3_rmul(a2, a, false);
    const Cx<double> s = {0.5 * (a2[0].re + a2[4].re + a2[8].re), 0.5 * (a2[0].im + a2[4].im + a2[8].im)};
    // det A by cofactors of the first row
    Cx<double> d = cmul(a[0], Cx<double>{cmul(a[4], a[8]).re - cmul(a[5], a[7]).re,
                                         cmul(a[4], a[8]).im - cmul(a[5], a[7]).im});
    {
        const Cx<double> m1 = {cmul(a[3], a[8]).re - cmul(a[5], a[6]).re, cmul(a[3], a[8]).im - cmul(a[5], a[6]).im};
        const Cx<double> m2 = {cmul(a[3], a[7]).re - cmul(a[4], a[6]).re, cmul(a[3], a[7]).im - cmul(a[4], a[6]).im};
        const Cx<double> t1 = cmul(a[1], m1), t2 = cmul(a[2], m2);
        d = {d.re - t1.re + t2.re, d.im - t1.im + t2.im};
    }
    // k = 0: (1, 0, 0); the running term (al, be, ga) / k!
    Cx<double> al = {1.0, 0.0}, be = {0.0, 0.0}, ga = {0.0, 0.0};
    Cx<double> ca = al, cb = be, cc = ga;
    for (int k = 1; k <= 30; ++k) {
        const double r = 1.0 / k;
        const Cx<double> gd = cmul(ga, d), gs = cmul(ga, s);
        const Cx<double> nal = {gd.re * r, gd.im * r};
        const Cx<double> nbe = {(al.re + gs.re) * r, (al.im + gs.im) * r};
        const Cx<double> nga = {be.re * r, be.im * r};
        al = nal;
        be = nbe;
        ga = nga;
        ca = {ca.re + al.re, ca.im + al.im};
        cb = {cb.re + be.re, cb.im + be.im};
        cc = {cc.re + ga.re, cc.im + ga.im};
        // the sums are O(1): stop once a term no longer changes them in FP64
        // (each term is a function of the previous one alone, at most 2 / (k + 1) times
        // its size since |s|, |d| <= 1 after scaling, so the rest sums below 2e-18)
        if (fabs(al.re) + fabs(al.im) + fabs(be.re) + fabs(be.im) + fabs(ga.re) + fabs(ga.im) < 1e-18) break;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Cx<double> v = cmul(cb, a[k]);
        cmac(v, cc, a2[k]);
        if (k % 4 == 0) v = {v.re + ca.re, v.im + ca.im};
        e[k] = v;
    }
    for (int j = 0; j < q; ++j) {
        Cx<double> t[9];
        mat3_set(t, e, false);
        mat3_rmul(t, e, false);
#pragma unroll
        for (int k = 0; k < 9; ++k) e[k] = t[k];
    }
}

// U_mu(x) <- exp(i eps P_mu(x)) U_mu(x), P = sum_a p^a lambda^a / 2
__global__ void __launch_bounds__(kThreads) link_update_kernel(int V, double2 *links, const double *mom, double eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (i >= V) return;
    const size_t l = (size_t)mu * V + i;
    const double *p = mom + l * 8;
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    // P (Hermitian), then a = i eps P
    const Cx<double> P[9] = {
        {0.5 * (p[2] + r3 * p[7]), 0.0}, {0.5 * p[0], -0.5 * p[1]}, {0.5 * p[3], -0.5 * p[4]},
        {0.5 * p[0], 0.5 * p[1]}, {0.5 * (-p[2] + r3 * p[7]), 0.0}, {0.5 * p[5], -0.5 * p[6]},
        {0.5 * p[3], 0.5 * p[4]}, {0.5 * p[5], 0.5 * p[6]}, {-r3 * p[7], 0.0},
    };
    Cx<double> a[9], e[9], u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = {-eps * P[k].im, eps * P[k].re};
    exp_traceless(a, e);
    double2 *lu = links + l * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = {lu[k].x, lu[k].y};
    mat3_rmul(e, u, false);
#pragma unroll
    for (int k = 0; k < 9; ++k) lu[k] = make_double2(e[k].re, e[k].im);
}

// out = gamma5 in on canonical spinors (gamma5 = diag(1, 1, -1, -1) in the
// chiral basis): spins 2 and 3 change sign
__global__ void __launch_bounds__(kThreads) gamma5_kernel(int V, double2 *out, const double2 *in) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const double2 v = in[(size_t)i * 12 + c];
        out[(size_t)i * 12 + c] = c < 6 ? v : make_double2(-v.x, -v.y);
    }
}

int red_blocks(size_t n) {
    const size_t b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < 1184 ? b : 1184);  // 152 SMs x 8 resident blocks
}

}  // namespace

cudaError_t launch_gauge_force(const Geom &g, const void *links_f64, int recon, double beta, double coef, double *out,
                               bool accumulate, cudaStream_t s) {
    LinkField F{g, static_cast<const char *>(links_f64), link_dir_bytes(COLA_F64, recon, g.Vh)};
    dim3 grid((g.V + kThreads - 1) / kThreads, 4);
    if (recon == 12) gauge_force_kernel<12><<<grid, kThreads, 0, s>>>(F, coef * beta, out, accumulate);
    else gauge_force_kernel<18><<<grid, kThreads, 0, s>>>(F, coef * beta, out, accumulate);
    return cudaGetLastError();
}

size_t gauge_scratch_doubles(const Geom &g) {
    const size_t a = (g.V + kRedThreads - 1) / kRedThreads;
    return (a > 1184 ? a : 1184) + 8;
}

cudaError_t launch_plaquette_sum(const Geom &g, const void *links_f64, int recon, double *scratch, double *out,
                                 cudaStream_t s) {
    LinkField F{g, static_cast<const char *>(links_f64), link_dir_bytes(COLA_F64, recon, g.Vh)};
    const int nb = (g.V + kRedThreads - 1) / kRedThreads;
    if (recon == 12) plaquette_kernel<12><<<nb, kRedThreads, 0, s>>>(F, scratch);
    else plaquette_kernel<18><<<nb, kRedThreads, 0, s>>>(F, scratch);
    finish_sum_kernel<<<1, kRedThreads, 0, s>>>(scratch, nb, 1.0 / 3.0, out);
    return cudaGetLastError();
}

cudaError_t launch_dot(const double *a, const double *b, size_t n, double scale, double *scratch, double *out,
                       cudaStream_t s) {
    const int nb = red_blocks(n);
    dot_kernel<<<nb, kRedThreads, 0, s>>>(a, b, n, scratch);
    finish_sum_kernel<<<1, kRedThreads, 0, s>>>(scratch, nb, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_gamma5(const Geom &g, void *out, const void *in, cudaStream_t s) {
    gamma5_kernel<<<(g.V + kThreads - 1) / kThreads, kThreads, 0, s>>>(g.V, static_cast<double2 *>(out),
                                                                       static_cast<const double2 *>(in));
    return cudaGetLastError();
}

cudaError_t launch_link_update(const Geom &g, void *links_canon, const double *mom, double eps, cudaStream_t s) {
    dim3 grid((g.V + kThreads - 1) / kThreads, 4);
    link_update_kernel<<<grid, kThreads, 0, s>>>(g.V, static_cast<double2 *>(links_canon), mom, eps);
    return cudaGetLastError();
}

}  // namespace cola
