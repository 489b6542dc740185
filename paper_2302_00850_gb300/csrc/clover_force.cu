// Clover part of the HMC fermion force.
//
// The paper's overview of COLA's physics features lists clover-improved
// fermions and HMC; it writes neither the action nor its force.  With the
// clover term A = 1 - kappa c_sw sum_{mu<nu} sigma_munu F_munu of clover.cu and
// S = phi^dag (D^dag D)^-1 phi, X = (D^dag D)^-1 phi, Y = D X, the variation
// dS = -2 Re Y^dag dA X of the clover term is
//   dS = (kappa c_sw / 4) sum_x sum_{mu<nu} Im Tr[dQ_munu(x) Gam_munu(x)],
//   Gam_munu = L + L^dag, L = Lam - tr Lam / 3,
//   Lam_munu(x)_ba = sum_st (sigma_munu)_st X(x)_tb conj(Y(x)_sa)
// (the traceless projection of F moves onto Lam, and the anti-Hermitian part
// of Q pairs with the Hermitian part of Lam).  Ordered pairs (mu, nu) and
// (nu, mu) give the same sum (Q_numu = Q_munu^dag, Gam_numu = -Gam_munu), so
// the link U_mu(y) collects, for each nu != mu, the two plaquettes of the
// (mu, nu) plane through it with Gam inserted at each of their four corners:
//   Z = U S+ - S- U^dag,
//   S+ = L2 L3 L4 G(y) + G(y+mu) L2 L3 L4 + L2 G(y+mu+nu) L3 L4 + L2 L3 G(y+nu) L4,
//        L2 = U_nu(y+mu), L3 = U_mu(y+nu)^dag, L4 = U_nu(y)^dag,
//   S- = G(y) M1 M2 M3 + M1 G(y-nu) M2 M3 + M1 M2 G(y-nu+mu) M3 + M1 M2 M3 G(y+mu),
//        M1 = U_nu(y-nu)^dag, M2 = U_mu(y-nu), M3 = U_nu(y-nu+mu),
// with G = Gam_munu (= -Gam_numu for mu > nu), and
//   dS/deps^a = (kappa c_sw / 4) Re Tr[T^a Z]   (U -> (1 + i eps T^a) U).
// Two kernels, FP64 throughout: Gam on every site (six planes, eight reals
// each: Gam is Hermitian and traceless), then one thread per link.
//
// The same sums give the clover part of the raw complex link gradient of a
// real loss through y = D psi (PyTorch's convention, grad = 2 dL/d conj(U)),
// with (X, Y) = (psi, dL/dy): dL = Re gy^dag dA psi is -1/2 of the form above,
// and a factor U (U^dag) of Im Tr[dU M] (Im Tr[dU^dag M]) has gradient -i M^dag
// (+i M), so per link grad = -i (kappa c_sw / 8) (S+^dag - S-).
#include "cola_impl.h"

namespace cola {
namespace {

using C64 = Cx<double>;

// Gam layout: [plane][8][V] doubles, plane = (0,1) (0,2) (0,3) (1,2) (1,3) (2,3),
// reals g00, g11 (g22 = -g00 - g11), then (0,1) (0,2) (1,2) as (re, im).
constexpr int kGamReals = 8;

__device__ __forceinline__ int plane_of(int mu, int nu) {  // mu < nu
    return mu == 0 ? nu - 1 : mu == 1 ? nu + 1 : 5;
}

// lam += s P for one entry s of sigma: an exact zero, a pure real or a pure
// imaginary s (all entries of sigma in the chirality blocks are one of
// these) takes 0 or 2 FP64 multiply-adds, a general one 4
__device__ __forceinline__ void sigma_mac(C64 &lam, double sr, double si, const C64 &P) {
    if (si == 0.0) {
        if (sr == 0.0) return;
        lam.re = fma(sr, P.re, lam.re);
        lam.im = fma(sr, P.im, lam.im);
    } else if (sr == 0.0) {
        lam.re = fma(-si, P.im, lam.re);
        lam.im = fma(si, P.re, lam.im);
    } else {
        lam.re = fma(sr, P.re, fma(-si, P.im, lam.re));
        lam.im = fma(sr, P.im, fma(si, P.re, lam.im));
    }
}

// The spin products of colour entry (b, a) of Lam: P[chi][s][t] = X_tb conj(Y_sa)
// within chirality block chi (spin index 2 chi + s, 2 chi + t).
__device__ __forceinline__ void spin_products(const C64 (&x)[12], const C64 (&y)[12], int b, int a,
                                              C64 (&P)[2][2][2]) {
#pragma unroll
    for (int chi = 0; chi < 2; ++chi)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const C64 xv = x[(2 * chi + t) * 3 + b], yv = y[(2 * chi + s) * 3 + a];
                P[chi][s][t] = {fma(xv.re, yv.re, xv.im * yv.im), fma(xv.im, yv.re, -xv.re * yv.im)};
            }
}

// Lam_p[b][a] = sum over chi, s, t of sigma_p[chi][s][t] P[chi][s][t]
__device__ __forceinline__ C64 plane_entry(const CloverSigma &sig, int p, const C64 (&P)[2][2][2]) {
    C64 lam = {0.0, 0.0};
#pragma unroll
    for (int chi = 0; chi < 2; ++chi)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int t = 0; t < 2; ++t)
                sigma_mac(lam, sig.v[p][chi][2 * s + t][0], sig.v[p][chi][2 * s + t][1], P[chi][s][t]);
    return lam;
}

// Gam_p = L + L^dag with L = Lam_p - tr Lam_p / 3 and
//   Lam_p[b][a] = sum over the chirality blocks of sigma_st X_tb conj(Y_sa).
// The 8 spin products of a colour entry serve all six planes, and of Lam
// only what Gam needs is formed: the real diagonal, and each off-diagonal
// pair (b, a), (a, b) together.
__global__ void __launch_bounds__(128) clover_gamma_kernel(const Geom g, const CloverSigma sig, const double2 *X,
                                                           const double2 *Y, double *gam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    C64 x[12], y[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const double2 a = __ldg(X + (size_t)i * 12 + c), b = __ldg(Y + (size_t)i * 12 + c);
        x[c] = {a.x, a.y};
        y[c] = {b.x, b.y};
    }
    double dg[6][3];
    C64 P[2][2][2];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        spin_products(x, y, b, b, P);
#pragma unroll
        for (int p = 0; p < 6; ++p) dg[p][b] = plane_entry(sig, p, P).re;
    }
    const size_t V = g.V;
    constexpr int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        C64 Q[2][2][2];
        spin_products(x, y, pairs[q][0], pairs[q][1], P);  // (b, a)
        spin_products(x, y, pairs[q][1], pairs[q][0], Q);  // (a, b)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const C64 ba = plane_entry(sig, p, P), ab = plane_entry(sig, p, Q);
            double *o = gam + (size_t)p * kGamReals * V + i;
            o[(2 + 2 * q) * V] = ba.re + ab.re;
            o[(3 + 2 * q) * V] = ba.im - ab.im;
        }
    }
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        const double tr = (dg[p][0] + dg[p][1] + dg[p][2]) / 3.0;
        double *o = gam + (size_t)p * kGamReals * V + i;
        o[0] = 2.0 * (dg[p][0] - tr);
        o[V] = 2.0 * (dg[p][1] - tr);
    }
}

__device__ __forceinline__ int lex_site(const Geom &g, const int (&p)[4]) {
    const int x = wrap_coord(p[0], g.L[0]), y = wrap_coord(p[1], g.L[1]);
    const int z = wrap_coord(p[2], g.L[2]), t = wrap_coord(p[3], g.L[3]);
    return COLA_BOUND(x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t)), g.V);
}

// G = sign Gam_plane at the site with coordinates p (wrapped)
__device__ __forceinline__ void gam_at(const Geom &g, const double *gam, int plane, double sign, const int (&p)[4],
                                       C64 (&m)[9]) {
    const double *q = gam + (size_t)plane * kGamReals * g.V + lex_site(g, p);
    const size_t V = g.V;
    const double d0 = sign * __ldg(q), d1 = sign * __ldg(q + V);
    const C64 e01 = {sign * __ldg(q + 2 * V), sign * __ldg(q + 3 * V)};
    const C64 e02 = {sign * __ldg(q + 4 * V), sign * __ldg(q + 5 * V)};
    const C64 e12 = {sign * __ldg(q + 6 * V), sign * __ldg(q + 7 * V)};
    m[0] = {d0, 0.0};
    m[4] = {d1, 0.0};
    m[8] = {-d0 - d1, 0.0};
    m[1] = e01;
    m[2] = e02;
    m[5] = e12;
    m[3] = {e01.re, -e01.im};
    m[6] = {e02.re, -e02.im};
    m[7] = {e12.re, -e12.im};
}

// c = a b
__device__ __forceinline__ void mul3(const C64 (&a)[9], const C64 (&b)[9], C64 (&c)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C64 s = cmul(a[3 * i], b[j]);
            cmac(s, a[3 * i + 1], b[3 + j]);
            cmac(s, a[3 * i + 2], b[6 + j]);
            c[3 * i + j] = s;
        }
}

// acc += a b
__device__ __forceinline__ void mac3(C64 (&acc)[9], const C64 (&a)[9], const C64 (&b)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cmac(acc[3 * i + j], a[3 * i], b[j]);
            cmac(acc[3 * i + j], a[3 * i + 1], b[3 + j]);
            cmac(acc[3 * i + j], a[3 * i + 2], b[6 + j]);
        }
}

// Products with the insertion matrix G (Hermitian, so its diagonal is real:
// only the real parts of g[0], g[4], g[8] are read), which saves the two
// multiply-adds by the zero imaginary parts of each diagonal entry.
// acc (+)= G b
template <bool ACC>
__device__ __forceinline__ void gmul_left(C64 (&acc)[9], const C64 (&gm)[9], const C64 (&b)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double d = gm[4 * i].re;
            C64 s = ACC ? acc[3 * i + j] : C64{0.0, 0.0};
            s.re = fma(d, b[3 * i + j].re, s.re);
            s.im = fma(d, b[3 * i + j].im, s.im);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k != i) cmac(s, gm[3 * i + k], b[3 * k + j]);
            acc[3 * i + j] = s;
        }
}
// acc (+)= a G
template <bool ACC>
__device__ __forceinline__ void gmul_right(C64 (&acc)[9], const C64 (&a)[9], const C64 (&gm)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double d = gm[4 * j].re;
            C64 s = ACC ? acc[3 * i + j] : C64{0.0, 0.0};
            s.re = fma(a[3 * i + j].re, d, s.re);
            s.im = fma(a[3 * i + j].im, d, s.im);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k != j) cmac(s, a[3 * i + k], gm[3 * k + j]);
            acc[3 * i + j] = s;
        }
}

// The specialised products where registers allow: with 12-real links the
// third-row reconstruction's temporaries leave no room for them without
// spilling, so those builds use the general products.
template <int RECON, bool ACC>
__device__ __forceinline__ void g_left(C64 (&acc)[9], const C64 (&gm)[9], const C64 (&b)[9]);
template <int RECON, bool ACC>
__device__ __forceinline__ void g_right(C64 (&acc)[9], const C64 (&a)[9], const C64 (&gm)[9]);

__device__ __forceinline__ void adj3(C64 (&m)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        m[4 * i].im = -m[4 * i].im;
#pragma unroll
        for (int j = i + 1; j < 3; ++j) {
            const C64 a = m[3 * i + j], b = m[3 * j + i];
            m[3 * i + j] = {b.re, -b.im};
            m[3 * j + i] = {a.re, -a.im};
        }
    }
}

template <int RECON, bool ACC>
__device__ __forceinline__ void g_left(C64 (&acc)[9], const C64 (&gm)[9], const C64 (&b)[9]) {
    if constexpr (RECON == 18) gmul_left<ACC>(acc, gm, b);
    else if constexpr (ACC) mac3(acc, gm, b);
    else mul3(gm, b, acc);
}
template <int RECON, bool ACC>
__device__ __forceinline__ void g_right(C64 (&acc)[9], const C64 (&a)[9], const C64 (&gm)[9]) {
    if constexpr (RECON == 18) gmul_right<ACC>(acc, a, gm);
    else if constexpr (ACC) mac3(acc, a, gm);
    else mul3(a, gm, acc);
}

// op(U_dir(y + dmu mu + dnu nu)), op = identity or adjoint
template <int RECON>
__device__ __forceinline__ void link_off(const Geom &g, const char *links, size_t dir_stride, const int (&c)[4],
                                         int dir, int mu, int dmu, int nu, int dnu, bool adj, C64 (&u)[9]) {
    int p[4] = {c[0], c[1], c[2], c[3]};
    p[mu] += dmu;
    p[nu] += dnu;
    link_at<RECON>(g, links, dir_stride, p, dir, u);
    if (adj) adj3(u);
}

// sign Gam_plane(y + dmu mu + dnu nu)
__device__ __forceinline__ void gam_off(const Geom &g, const double *gam, int plane, double sign, const int (&c)[4],
                                        int mu, int dmu, int nu, int dnu, C64 (&m)[9]) {
    int p[4] = {c[0], c[1], c[2], c[3]};
    p[mu] += dmu;
    p[nu] += dnu;
    gam_at(g, gam, plane, sign, p, m);
}

// GRAD = false: out is the force [4][V][8] (reals), coef multiplies Re Tr[lambda^a Z].
// GRAD = true: out is the raw link gradient [4][V][3][3] (double2), out += -i coef (S+^dag - S-).
template <int RECON, bool GRAD>
__global__ void __launch_bounds__(128) clover_force_kernel(const Geom g, const char *links, size_t dir_stride,
                                                           const double *gam, void *out, double coef,
                                                           int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (i >= g.V) return;
    int c[4];
    c[0] = i % g.L[0];
    int r = i / g.L[0];
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];

    C64 sp[9], sm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) sp[k] = sm[k] = {0.0, 0.0};
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const int plane = mu < nu ? plane_of(mu, nu) : plane_of(nu, mu);
        const double sign = mu < nu ? 1.0 : -1.0;
        // Each side's insertion sum in nested (Horner) form, 8 products of
        // 3x3 matrices instead of 9:
        //   S+ += L2 (L3 (L4 G(y) + G(y+nu) L4) + G(y+mu+nu) L3 L4) + G(y+mu) L2 L3 L4
        //   S- += M1 (M2 (G(y-nu+mu) M3 + M3 G(y+mu)) + G(y-nu) M2 M3) + G(y) M1 M2 M3
        C64 l2[9], l3[9], l4[9], gm[9], t[9], u[9];
        // ---- the plaquette on the +nu side: L2 = U_nu(y+mu), L3 = U_mu(y+nu)^dag, L4 = U_nu(y)^dag
        link_off<RECON>(g, links, dir_stride, c, nu, mu, 0, nu, 0, true, l4);   // L4
        gam_off(g, gam, plane, sign, c, mu, 0, nu, 0, gm);                      // G(y)
        g_right<RECON, false>(t, l4, gm);                                       // L4 G(y)
        gam_off(g, gam, plane, sign, c, mu, 0, nu, 1, gm);                      // G(y+nu)
        g_left<RECON, true>(t, gm, l4);                                          // + G(y+nu) L4
        link_off<RECON>(g, links, dir_stride, c, mu, mu, 0, nu, 1, true, l3);   // L3
        mul3(l3, t, u);                                                         // L3 (...)
        mul3(l3, l4, t);                                                        // L3 L4
        gam_off(g, gam, plane, sign, c, mu, 1, nu, 1, gm);                      // G(y+mu+nu)
        g_left<RECON, true>(u, gm, t);                                           // + G(y+mu+nu) L3 L4
        link_off<RECON>(g, links, dir_stride, c, nu, mu, 1, nu, 0, false, l2);  // L2
        mac3(sp, l2, u);                                                        // S+ += L2 (...)
        mul3(l2, t, u);                                                         // L2 L3 L4
        gam_off(g, gam, plane, sign, c, mu, 1, nu, 0, gm);                      // G(y+mu)
        g_left<RECON, true>(sp, gm, u);                                          // S+ += G(y+mu) L2 L3 L4
        // ---- the plaquette on the -nu side: M1 = U_nu(y-nu)^dag, M2 = U_mu(y-nu), M3 = U_nu(y-nu+mu)
        // (M1, M2, M3 reuse the registers of L2, L3, L4)
        link_off<RECON>(g, links, dir_stride, c, nu, mu, 1, nu, -1, false, l4); // M3
        gam_off(g, gam, plane, sign, c, mu, 1, nu, -1, gm);                     // G(y-nu+mu)
        g_left<RECON, false>(t, gm, l4);                                         // G(y-nu+mu) M3
        gam_off(g, gam, plane, sign, c, mu, 1, nu, 0, gm);                      // G(y+mu)
        g_right<RECON, true>(t, l4, gm);                                         // + M3 G(y+mu)
        link_off<RECON>(g, links, dir_stride, c, mu, mu, 0, nu, -1, false, l3); // M2
        mul3(l3, t, u);                                                         // M2 (...)
        mul3(l3, l4, t);                                                        // M2 M3
        gam_off(g, gam, plane, sign, c, mu, 0, nu, -1, gm);                     // G(y-nu)
        g_left<RECON, true>(u, gm, t);                                           // + G(y-nu) M2 M3
        link_off<RECON>(g, links, dir_stride, c, nu, mu, 0, nu, -1, true, l2);  // M1
        mac3(sm, l2, u);                                                        // S- += M1 (...)
        mul3(l2, t, u);                                                         // M1 M2 M3
        gam_off(g, gam, plane, sign, c, mu, 0, nu, 0, gm);                      // G(y)
        g_left<RECON, true>(sm, gm, u);                                          // S- += G(y) M1 M2 M3
    }
    if constexpr (GRAD) {
        double2 *o = static_cast<double2 *>(out) + ((size_t)mu * g.V + i) * 9;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const C64 v = {sp[3 * b + a].re - sm[3 * a + b].re, -sp[3 * b + a].im - sm[3 * a + b].im};
                double2 r = make_double2(coef * v.im, -coef * v.re);  // -i coef v
                if (accumulate) {
                    const double2 p = o[3 * a + b];
                    r.x += p.x;
                    r.y += p.y;
                }
                o[3 * a + b] = r;
            }
        return;
    }
    // Z = U S+ - S- U^dag; F^a = coef Re Tr[lambda^a Z] = coef Im Tr[lambda^a (i Z)]
    C64 u[9], z[9], w[9];
    link_at<RECON>(g, links, dir_stride, c, mu, u);
    mul3(u, sp, z);
    adj3(u);
    mul3(sm, u, w);
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = {-(z[k].im - w[k].im), z[k].re - w[k].re};  // i (z - w)
    double fa[8];
    im_tr_lambda(w, fa);
    store_force(static_cast<double *>(out) + ((size_t)mu * g.V + i) * 8, fa, coef, accumulate != 0);
}

}  // namespace

size_t clover_force_scratch_bytes(const Geom &g) { return (size_t)6 * kGamReals * g.V * sizeof(double); }

cudaError_t launch_clover_force(const Geom &g, const void *links_f64, int recon, double kappa, double csw,
                                const void *X, const void *Y, double *force, double coef, bool accumulate,
                                void *scratch, cudaStream_t s) {
    double *gam = static_cast<double *>(scratch);
    const dim3 block(128), grid1((g.V + 127) / 128), grid2((g.V + 127) / 128, 4);
    clover_gamma_kernel<<<grid1, block, 0, s>>>(g, clover_sigma(), static_cast<const double2 *>(X),
                                                static_cast<const double2 *>(Y), gam);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const char *l = static_cast<const char *>(links_f64);
    const size_t ds = link_dir_bytes(COLA_F64, recon, g.Vh);
    // dS/deps^a = (kappa c_sw / 4) Re Tr[T^a Z] = (kappa c_sw / 8) Re Tr[lambda^a Z]
    const double c = coef * kappa * csw / 8.0;
    if (recon == 12) clover_force_kernel<12, false><<<grid2, block, 0, s>>>(g, l, ds, gam, force, c, accumulate);
    else clover_force_kernel<18, false><<<grid2, block, 0, s>>>(g, l, ds, gam, force, c, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_clover_link_grad(const Geom &g, const void *links_f64, int recon, double kappa, double csw,
                                    const void *psi, const void *gy, void *grad, void *scratch, cudaStream_t s) {
    double *gam = static_cast<double *>(scratch);
    const dim3 block(128), grid1((g.V + 127) / 128), grid2((g.V + 127) / 128, 4);
    clover_gamma_kernel<<<grid1, block, 0, s>>>(g, clover_sigma(), static_cast<const double2 *>(psi),
                                                static_cast<const double2 *>(gy), gam);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const char *l = static_cast<const char *>(links_f64);
    const size_t ds = link_dir_bytes(COLA_F64, recon, g.Vh);
    // per link: grad += -i (kappa c_sw / 8) (S+^dag - S-)
    const double c = kappa * csw / 8.0;
    if (recon == 12) clover_force_kernel<12, true><<<grid2, block, 0, s>>>(g, l, ds, gam, grad, c, 1);
    else clover_force_kernel<18, true><<<grid2, block, 0, s>>>(g, l, ds, gam, grad, c, 1);
    return cudaGetLastError();
}

}  // namespace cola
