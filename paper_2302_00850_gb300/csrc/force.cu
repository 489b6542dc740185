// Link derivatives of the Wilson operator: the HMC fermion force and the raw
// complex link gradient used by the differentiable Dslash.
//
// Hybrid Monte Carlo is one of COLA's key algorithms (the paper's overview of
// the library).  For S = phi^dag (D^dag D)^-1 phi, X = (D^dag D)^-1 phi and
// Y = D X, a left variation U_mu(x) -> (1 + i eps T^a) U_mu(x) gives
//   dS/deps^a = -2 kappa Im Tr[T^a Ut_mu(x) (P + Q^dag)],
//   P = sum_s [(1 - gamma_mu) X(x+mu)]_s conj(Y(x)_s)^T,
//   Q = sum_s [(1 + gamma_mu) X(x)]_s conj(Y(x+mu)_s)^T.
// Each projector (1 +- gamma_mu) = R R^dag-like factorisation with R = [1; B^dag]
// in the chiral basis, so a spin sum of the projected outer product equals the
// sum over the two projected rows of both factors: the kernel projects X and
// Y to two-spinors and forms two 3x3 outer products instead of four.
// One thread per link, FP64 throughout.
#include "cola_impl.h"

namespace cola {

// rows 0, 1 of (1 + S gamma_mu) psi (the same projection the hopping kernel uses)
template <int MU, int S>
__device__ __forceinline__ void proj2(const Cx<double> (&p)[12], Cx<double> (&h)[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Cx<double> p0 = p[a], p1 = p[3 + a], p2 = p[6 + a], p3 = p[9 + a];
        if constexpr (MU == 0) {
            h[0][a] = {p0.re - S * p3.im, p0.im + S * p3.re};
            h[1][a] = {p1.re - S * p2.im, p1.im + S * p2.re};
        } else if constexpr (MU == 1) {
            h[0][a] = {p0.re - S * p3.re, p0.im - S * p3.im};
            h[1][a] = {p1.re + S * p2.re, p1.im + S * p2.im};
        } else if constexpr (MU == 2) {
            h[0][a] = {p0.re - S * p2.im, p0.im + S * p2.re};
            h[1][a] = {p1.re + S * p3.im, p1.im - S * p3.re};
        } else {
            h[0][a] = {p0.re + S * p2.re, p0.im + S * p2.im};
            h[1][a] = {p1.re + S * p3.re, p1.im + S * p3.im};
        }
    }
}

__device__ __forceinline__ void load_canon(const double2 *f, int site, Cx<double> (&s)[12]) {
    const double2 *p = f + (size_t)site * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 v = __ldg(p + c);
        s[c] = {v.x, v.y};
    }
}

// m += sum_k a_k b_k^dag  (3x3)
__device__ __forceinline__ void outer_acc(Cx<double> (&m)[9], const Cx<double> (&a)[2][3],
                                          const Cx<double> (&b)[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Cx<double> t = cmulc(a[k][i], b[k][j]);
                m[3 * i + j].re += t.re;
                m[3 * i + j].im += t.im;
            }
}

__device__ __forceinline__ void site_coords(const Geom &g, int i, int (&c)[4]) {
    c[0] = i % g.L[0];
    int r = i / g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
}

__device__ __forceinline__ int site_fwd(const Geom &g, int i, const int (&c)[4], int mu) {
    int step = 1;
    for (int k = 0; k < mu; ++k) step *= g.L[k];
    return COLA_BOUND(c[mu] == g.L[mu] - 1 ? i - (g.L[mu] - 1) * step : i + step, g.V);
}

template <int MU, int RECON>
__device__ void force_link(const Geom &g, double kappa, const void *links, int i, const int (&c)[4],
                           const double2 *X, const double2 *Y, double *out, double coef, bool accumulate) {
    const int j = site_fwd(g, i, c, MU);
    Cx<double> xs[12], ys[12];
    Cx<double> hx[2][3], hy[2][3];
    Cx<double> m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = {0.0, 0.0};
    // P = sum_k hx_k hy_k^dag with hx from X(x+mu), hy from Y(x), projector (1 - gamma)
    load_canon(X, j, xs);
    load_canon(Y, i, ys);
    proj2<MU, -1>(xs, hx);
    proj2<MU, -1>(ys, hy);
    outer_acc(m, hx, hy);
    // Q^dag = sum_k hy'_k hx'_k^dag with hx' from X(x), hy' from Y(x+mu), projector (1 + gamma)
    load_canon(X, i, xs);
    load_canon(Y, j, ys);
    proj2<MU, +1>(xs, hx);
    proj2<MU, +1>(ys, hy);
    outer_acc(m, hy, hx);
    // W = Ut m
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const size_t dir_bytes = link_dir_bytes(COLA_F64, RECON, g.Vh);
    const char *base = static_cast<const char *>(links) + (size_t)par * 4 * dir_bytes + (size_t)MU * dir_bytes;
    Cx<double> u[9];
    LinkIO<COLA_F64, RECON>::load(base, g.Vh, i >> 1, u);
    if (c[MU] == g.L[MU] - 1 && !g.bc_trivial[MU]) {
        const Cx<double> ph = {g.bc[MU][0], g.bc[MU][1]};
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = cmul(u[k], ph);
    }
    Cx<double> w[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Cx<double> s = cmul(u[3 * a], m[b]);
            cmac(s, u[3 * a + 1], m[3 + b]);
            cmac(s, u[3 * a + 2], m[6 + b]);
            w[3 * a + b] = s;
        }
    // F^a = -kappa Im Tr[lambda^a W], times coef, stored or added
    double fa[8];
    im_tr_lambda(w, fa);
    store_force(out + ((size_t)MU * g.V + i) * 8, fa, -kappa * coef, accumulate);
}

template <int RECON>
__global__ void __launch_bounds__(128) force_kernel(const Geom g, double kappa, const void *links, double *out,
                                                    const double2 *X, const double2 *Y, double coef, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    int c[4];
    site_coords(g, i, c);
    switch (blockIdx.y) {
        case 0: force_link<0, RECON>(g, kappa, links, i, c, X, Y, out, coef, accumulate); break;
        case 1: force_link<1, RECON>(g, kappa, links, i, c, X, Y, out, coef, accumulate); break;
        case 2: force_link<2, RECON>(g, kappa, links, i, c, X, Y, out, coef, accumulate); break;
        default: force_link<3, RECON>(g, kappa, links, i, c, X, Y, out, coef, accumulate); break;
    }
}

// grad_U_mu(x) = -kappa conj(ph) sum_k [hg_k hpsi_k^dag + hpsi'_k hg'_k^dag]
//   hg = (1-gamma) rows of g(x), hpsi = (1-gamma) rows of psi(x+mu),
//   hpsi' = (1+gamma) rows of psi(x), hg' = (1+gamma) rows of g(x+mu).
template <int MU>
__device__ void link_grad_one(const Geom &g, double kappa, int i, const int (&c)[4], const double2 *psi,
                              const double2 *gy, double2 *out) {
    const int j = site_fwd(g, i, c, MU);
    Cx<double> a[12], b[12];
    Cx<double> ha[2][3], hb[2][3];
    Cx<double> m[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = {0.0, 0.0};
    load_canon(gy, i, a);
    load_canon(psi, j, b);
    proj2<MU, -1>(a, ha);
    proj2<MU, -1>(b, hb);
    outer_acc(m, ha, hb);
    load_canon(psi, i, a);
    load_canon(gy, j, b);
    proj2<MU, +1>(a, ha);
    proj2<MU, +1>(b, hb);
    outer_acc(m, ha, hb);
    Cx<double> ph = {-kappa, 0.0};
    if (c[MU] == g.L[MU] - 1 && !g.bc_trivial[MU]) ph = {-kappa * g.bc[MU][0], kappa * g.bc[MU][1]};
    double2 *o = out + ((size_t)MU * g.V + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Cx<double> v = cmul(ph, m[k]);
        o[k] = make_double2(v.re, v.im);
    }
}

__global__ void __launch_bounds__(128) link_grad_kernel(const Geom g, double kappa, double2 *out,
                                                        const double2 *psi, const double2 *gy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    int c[4];
    site_coords(g, i, c);
    switch (blockIdx.y) {
        case 0: link_grad_one<0>(g, kappa, i, c, psi, gy, out); break;
        case 1: link_grad_one<1>(g, kappa, i, c, psi, gy, out); break;
        case 2: link_grad_one<2>(g, kappa, i, c, psi, gy, out); break;
        default: link_grad_one<3>(g, kappa, i, c, psi, gy, out); break;
    }
}

cudaError_t launch_force(const Geom &g, double kappa, const void *links_f64, int recon, double *force,
                         const void *X, const void *Y, cudaStream_t s, double coef, bool accumulate) {
    dim3 block(128), grid((g.V + 127) / 128, 4);
    const double2 *x = static_cast<const double2 *>(X);
    const double2 *y = static_cast<const double2 *>(Y);
    if (recon == 12) force_kernel<12><<<grid, block, 0, s>>>(g, kappa, links_f64, force, x, y, coef, accumulate);
    else force_kernel<18><<<grid, block, 0, s>>>(g, kappa, links_f64, force, x, y, coef, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_link_grad(const Geom &g, double kappa, void *grad, const void *psi, const void *gy,
                             cudaStream_t s) {
    dim3 block(128), grid((g.V + 127) / 128, 4);
    link_grad_kernel<<<grid, block, 0, s>>>(g, kappa, static_cast<double2 *>(grad),
                                            static_cast<const double2 *>(psi), static_cast<const double2 *>(gy));
    return cudaGetLastError();
}

}  // namespace cola
