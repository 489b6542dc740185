// Clover (Sheikholeslami-Wohlert) term: construction of A(x) and A(x)^-1 from
// the FP64 links, and the stand-alone application C psi on one parity.
//
// The paper's overview of COLA's physics features cites clover-improved
// Wilson actions (FLIC fermions among them) without writing them out; the
// definitions used here are the standard ones in the kappa normalisation of
// the hopping kernel (Luscher, Sint, Sommer and Weisz 1996 for the sign):
//
//   Q_munu(x) = sum of the four plaquettes of the (mu, nu) plane at x, each
//               oriented mu -> nu (the clover leaves)
//   F_munu(x) = (Q - Q^dag) / (8i) minus its trace / 3   (Hermitian, traceless)
//   A(x)      = 1 - kappa c_sw sum_{mu<nu} sigma_munu F_munu(x),
//               sigma_munu = (i/2) [gamma_mu, gamma_nu]
//
// A is block diagonal in chirality (two Hermitian 6x6 blocks, layout in
// cola_internal.cuh).  Construction is setup work (once per gauge field): one
// thread per site in FP64, F from 24 plaquettes, the two blocks assembled
// and inverted by an LDL^dag factorisation without pivoting (A is Hermitian
// and, for the fields and c_sw of interest, close to 1; a zero or non-finite
// pivot is reported, not hidden).
#include <complex>

#include "cola_impl.h"

namespace cola {

namespace {

using C64 = Cx<double>;

struct BuildArgs {
    Geom g;
    const char *links;
    size_t link_parity_stride, link_dir_stride;
    double coef;  // kappa * c_sw
    CloverSigma sig;
    void *a[3];
    void *ainv[3];
    int *bad;
};

// One factor of a leaf: the link of direction `d` (0: mu, 1: nu) at offset
// (om, on) along (mu, nu) from the site, adjoint or not.
struct Factor {
    signed char om, on, d, adj;
};
// The four leaves, each a closed path starting and ending at the site:
//   U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//   U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
//   U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
//   U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
__constant__ Factor kLeaves[4][4] = {
    {{0, 0, 0, 0}, {1, 0, 1, 0}, {0, 1, 0, 1}, {0, 0, 1, 1}},
    {{0, 0, 1, 0}, {-1, 1, 0, 1}, {-1, 0, 1, 1}, {-1, 0, 0, 0}},
    {{-1, 0, 0, 1}, {-1, -1, 1, 1}, {-1, -1, 0, 0}, {0, -1, 1, 0}},
    {{0, -1, 1, 1}, {0, -1, 0, 0}, {1, -1, 1, 0}, {0, 0, 0, 1}},
};

__device__ __forceinline__ int lower(int i, int j) { return i * (i - 1) / 2 + j; }  // i > j

template <int RECON>
__global__ void __launch_bounds__(128) clover_build_kernel(const __grid_constant__ BuildArgs A) {
    const Geom &g = A.g;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y;
    if (cb >= g.Vh) return;
    const Coord c = cb_coord(g, cb, par);
    const int X[4] = {c.x, c.y, c.z, c.t};

    // F per plane: real diagonal (traceless) and the entries (0,1) (0,2) (1,2)
    double fd[6][3];
    C64 fo[6][3];
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            C64 q[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) q[k] = {0.0, 0.0};
            for (int leaf = 0; leaf < 4; ++leaf) {
                C64 w[9];
                for (int f = 0; f < 4; ++f) {
                    const Factor fa = kLeaves[leaf][f];
                    int p[4] = {X[0], X[1], X[2], X[3]};
                    p[mu] += fa.om;
                    p[nu] += fa.on;
                    C64 u[9];
                    link_at<RECON>(g, A.links, A.link_dir_stride, p, fa.d ? nu : mu, u);
                    if (f == 0) mat3_set(w, u, fa.adj != 0);
                    else mat3_rmul(w, u, fa.adj != 0);
                }
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    q[k].re += w[k].re;
                    q[k].im += w[k].im;
                }
            }
            // F = (Q - Q^dag) / (8i): diagonal Im Q_aa / 4; off-diagonal z / (8i) = (z.im, -z.re) / 8
            double d0 = q[0].im * 0.25, d1 = q[4].im * 0.25, d2 = q[8].im * 0.25;
            const double tr = (d0 + d1 + d2) / 3.0;
            fd[plane][0] = d0 - tr;
            fd[plane][1] = d1 - tr;
            fd[plane][2] = d2 - tr;
            const int ab[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const C64 qab = q[3 * ab[e][0] + ab[e][1]], qba = q[3 * ab[e][1] + ab[e][0]];
                const C64 z = {qab.re - qba.re, qab.im + qba.im};  // Q_ab - conj(Q_ba)
                fo[plane][e] = {z.im * 0.125, -z.re * 0.125};
            }
        }

    for (int chi = 0; chi < 2; ++chi) {
        // A block, packed: row i = 3 s + a (s the spin within the block)
        double m[kCloverReals];
        for (int i = 0; i < 6; ++i) {
            const int s = i / 3, a = i % 3;
            double v = 1.0;
            for (int p = 0; p < 6; ++p) v -= A.coef * A.sig.v[p][chi][3 * s][0] * fd[p][a];
            m[i] = v;
        }
        for (int i = 1; i < 6; ++i)
            for (int j = 0; j < i; ++j) {
                const int s = i / 3, a = i % 3, t = j / 3, b = j % 3;
                C64 v = {0.0, 0.0};
                for (int p = 0; p < 6; ++p) {
                    C64 f;
                    if (a == b) f = {fd[p][a], 0.0};
                    else if (a < b) f = fo[p][a + b - 1];
                    else {
                        const C64 o = fo[p][a + b - 1];  // F_ab = conj(F_ba)
                        f = {o.re, -o.im};
                    }
                    const C64 sg = {A.sig.v[p][chi][2 * s + t][0], A.sig.v[p][chi][2 * s + t][1]};
                    cmac(v, sg, f);
                }
                m[6 + 2 * lower(i, j)] = -A.coef * v.re;
                m[6 + 2 * lower(i, j) + 1] = -A.coef * v.im;
            }

        // A = L D L^dag, L unit lower triangular
        double d[6];
        C64 l[15];
        bool ok = true;
        for (int j = 0; j < 6; ++j) {
            double dj = m[j];
            for (int k = 0; k < j; ++k) {
                const C64 x = l[lower(j, k)];
                dj -= (x.re * x.re + x.im * x.im) * d[k];
            }
            ok = ok && isfinite(dj) && fabs(dj) > 1e-300;
            d[j] = dj;
            const double rdj = 1.0 / dj;
            for (int i = j + 1; i < 6; ++i) {
                C64 s = {m[6 + 2 * lower(i, j)], m[6 + 2 * lower(i, j) + 1]};
                for (int k = 0; k < j; ++k) {
                    const C64 lik = l[lower(i, k)], ljk = l[lower(j, k)];
                    const C64 t = cmulc(lik, ljk);  // l_ik conj(l_jk)
                    s.re -= t.re * d[k];
                    s.im -= t.im * d[k];
                }
                l[lower(i, j)] = {s.re * rdj, s.im * rdj};
            }
        }
        if (!ok) *A.bad = 1;
        // M = L^-1 (unit lower triangular)
        C64 mi[15];
        for (int i = 1; i < 6; ++i)
            for (int j = 0; j < i; ++j) {
                C64 s = {-l[lower(i, j)].re, -l[lower(i, j)].im};
                for (int k = j + 1; k < i; ++k) {
                    const C64 t = cmul(l[lower(i, k)], mi[lower(k, j)]);
                    s.re -= t.re;
                    s.im -= t.im;
                }
                mi[lower(i, j)] = s;
            }
        // A^-1 = M^dag D^-1 M: (i, j) = sum_{k >= i} conj(M_ki) M_kj / d_k, M_kk = 1
        double inv[kCloverReals];
        for (int i = 0; i < 6; ++i) {
            double v = 1.0 / d[i];
            for (int k = i + 1; k < 6; ++k) {
                const C64 x = mi[lower(k, i)];
                v += (x.re * x.re + x.im * x.im) / d[k];
            }
            inv[i] = v;
        }
        for (int i = 1; i < 6; ++i)
            for (int j = 0; j < i; ++j) {
                const C64 mij = mi[lower(i, j)];
                C64 v = {mij.re / d[i], mij.im / d[i]};
                for (int k = i + 1; k < 6; ++k) {
                    const C64 t = cmulc(mi[lower(k, j)], mi[lower(k, i)]);  // conj(M_ki) M_kj
                    v.re += t.re / d[k];
                    v.im += t.im / d[k];
                }
                inv[6 + 2 * lower(i, j)] = v.re;
                inv[6 + 2 * lower(i, j) + 1] = v.im;
            }

        const size_t po64 = par * clover_parity_bytes(COLA_F64, g.Vh) + chi * clover_block_bytes(COLA_F64, g.Vh);
        const size_t po32 = par * clover_parity_bytes(COLA_F32, g.Vh) + chi * clover_block_bytes(COLA_F32, g.Vh);
        const size_t po16 = par * clover_parity_bytes(COLA_F16, g.Vh) + chi * clover_block_bytes(COLA_F16, g.Vh);
        if (A.a[COLA_F64]) CloverIO<COLA_F64>::store(static_cast<char *>(A.a[COLA_F64]) + po64, g.Vh, cb, m);
        if (A.ainv[COLA_F64]) CloverIO<COLA_F64>::store(static_cast<char *>(A.ainv[COLA_F64]) + po64, g.Vh, cb, inv);
        if (A.a[COLA_F32]) CloverIO<COLA_F32>::store(static_cast<char *>(A.a[COLA_F32]) + po32, g.Vh, cb, m);
        if (A.ainv[COLA_F32]) CloverIO<COLA_F32>::store(static_cast<char *>(A.ainv[COLA_F32]) + po32, g.Vh, cb, inv);
        if (A.a[COLA_F16]) CloverIO<COLA_F16>::store(static_cast<char *>(A.a[COLA_F16]) + po16, g.Vh, cb, m);
        if (A.ainv[COLA_F16]) CloverIO<COLA_F16>::store(static_cast<char *>(A.ainv[COLA_F16]) + po16, g.Vh, cb, inv);
    }
}

template <int P>
__global__ void __launch_bounds__(128) clover_apply_kernel(Geom g, const char *clv, char *out, const char *in,
                                                           int par0) {
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.Vh) return;
    const int rhs = blockIdx.y;
    const int par = par0 + blockIdx.z;
    const size_t ps = spinor_parity_bytes(P, g.Vh);
    const size_t off = (size_t)rhs * 2 * ps + par * ps;
    Cx<typename Prec<P>::real> v[12];
    SpinorIO<P>::load(in + off, g.Vh, cb, v);
    clover_mul<P>(clv + par * clover_parity_bytes(P, g.Vh), g.Vh, cb, v);
    SpinorIO<P>::store(out + off, g.Vh, cb, v);
}

}  // namespace

cudaError_t launch_clover_build(const Geom &g, const void *links_f64, int recon, double coef, const CloverSigma &sig,
                                void *const a[3], void *const ainv[3], int *bad, cudaStream_t s) {
    BuildArgs A;
    A.g = g;
    A.links = static_cast<const char *>(links_f64);
    A.link_dir_stride = link_dir_bytes(COLA_F64, recon, g.Vh);
    A.link_parity_stride = 4 * A.link_dir_stride;
    A.coef = coef;
    A.sig = sig;
    for (int p = 0; p < 3; ++p) {
        A.a[p] = a[p];
        A.ainv[p] = ainv[p];
    }
    A.bad = bad;
    dim3 grid((g.Vh + 127) / 128, 2, 1);
    if (recon == 12) clover_build_kernel<12><<<grid, 128, 0, s>>>(A);
    else clover_build_kernel<18><<<grid, 128, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_clover_apply(int prec, const Geom &g, const void *clv, void *out, const void *in, int nrhs,
                                int parity_mask, cudaStream_t s) {
    if (parity_mask < 1 || parity_mask > 3 || nrhs < 1 || nrhs > 65535) return cudaErrorInvalidValue;
    dim3 grid((g.Vh + 127) / 128, nrhs, parity_mask == 3 ? 2 : 1);
    const int par0 = parity_mask == 2 ? 1 : 0;
    const char *c = static_cast<const char *>(clv);
    const char *i = static_cast<const char *>(in);
    char *o = static_cast<char *>(out);
    switch (prec) {
        case COLA_F64: clover_apply_kernel<COLA_F64><<<grid, 128, 0, s>>>(g, c, o, i, par0); break;
        case COLA_F32: clover_apply_kernel<COLA_F32><<<grid, 128, 0, s>>>(g, c, o, i, par0); break;
        default: clover_apply_kernel<COLA_F16><<<grid, 128, 0, s>>>(g, c, o, i, par0); break;
    }
    return cudaGetLastError();
}

// sigma_munu = (i/2)[gamma_mu, gamma_nu] in the DeGrand-Rossi basis of the
// hopping kernel, restricted to the chirality blocks (spins 0,1 and 2,3;
// the off-block entries vanish because sigma commutes with gamma5).
static CloverSigma make_sigma() {
    using Z = std::complex<double>;
    const Z i1(0.0, 1.0), o(0.0, 0.0), one(1.0, 0.0);
    const Z gam[4][4][4] = {
        {{o, o, o, i1}, {o, o, i1, o}, {o, -i1, o, o}, {-i1, o, o, o}},     // gamma_x
        {{o, o, o, -one}, {o, o, one, o}, {o, one, o, o}, {-one, o, o, o}}, // gamma_y
        {{o, o, i1, o}, {o, o, o, -i1}, {-i1, o, o, o}, {o, i1, o, o}},     // gamma_z
        {{o, o, one, o}, {o, o, o, one}, {one, o, o, o}, {o, one, o, o}},   // gamma_t
    };
    CloverSigma sg;
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            Z sm[4][4];
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    Z comm = 0.0;
                    for (int k = 0; k < 4; ++k) comm += gam[mu][r][k] * gam[nu][k][c] - gam[nu][r][k] * gam[mu][k][c];
                    sm[r][c] = 0.5 * i1 * comm;
                }
            for (int chi = 0; chi < 2; ++chi)
                for (int s = 0; s < 2; ++s)
                    for (int t = 0; t < 2; ++t) {
                        sg.v[plane][chi][2 * s + t][0] = sm[2 * chi + s][2 * chi + t].real();
                        sg.v[plane][chi][2 * s + t][1] = sm[2 * chi + s][2 * chi + t].imag();
                    }
        }
    return sg;
}

const CloverSigma &clover_sigma() {
    static const CloverSigma sig = make_sigma();
    return sig;
}

void set_clover(DslashLat &L, cola_gauge g, int prec, bool inverse) {
    L.clv = inverse ? g->clover_inv[prec] : g->clover[prec];
    L.clv_parity_stride = clover_parity_bytes(prec, g->geom.Vh);
}

cola_status clover_rebuild(cola_gauge g, cudaStream_t s) {
    if (!g->links[COLA_F64]) {
        set_error("the clover term is built from FP64 links: create the gauge handle with COLA_F64 in prec_mask");
        return COLA_ERR_UNSUPPORTED;
    }
    for (int p = 0; p < 3; ++p) {
        if (!g->links[p]) continue;
        const size_t bytes = 2 * clover_parity_bytes(p, g->geom.Vh);
        if (!g->clover[p]) {
            cola_status st = cuda_check(cudaMalloc(&g->clover[p], bytes), "clover allocation");
            if (st != COLA_OK) return st;
        }
        if (!g->clover_inv[p]) {
            cola_status st = cuda_check(cudaMalloc(&g->clover_inv[p], bytes), "clover allocation");
            if (st != COLA_OK) return st;
        }
    }
    int *bad = nullptr;
    cola_status st = ws_slot(g, cola_gauge_s::kSlotCloverFlag, sizeof(int), reinterpret_cast<void **>(&bad));
    if (st != COLA_OK) return st;
    st = cuda_check(cudaMemsetAsync(bad, 0, sizeof(int), s), "clover flag");
    if (st != COLA_OK) return st;
    const CloverSigma &sig = clover_sigma();
    st = cuda_check(launch_clover_build(g->geom, g->links[COLA_F64], g->recon[COLA_F64], g->lat.kappa * g->csw, sig,
                                        g->clover, g->clover_inv, bad, s),
                    "clover construction");
    if (st != COLA_OK) return st;
    int h_bad = 0;
    st = cuda_check(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s), "clover flag readback");
    if (st == COLA_OK) st = cuda_check(cudaStreamSynchronize(s), "clover construction");
    if (st != COLA_OK) return st;
    if (h_bad) {
        set_error("a clover block A(x) has a zero or non-finite pivot: A is singular for this field and c_sw");
        return COLA_ERR_BREAKDOWN;
    }
    return COLA_OK;
}

void clover_free(cola_gauge g) {
    for (int p = 0; p < 3; ++p) {
        if (g->clover[p]) cudaFree(g->clover[p]);
        if (g->clover_inv[p]) cudaFree(g->clover_inv[p]);
        g->clover[p] = g->clover_inv[p] = nullptr;
    }
    g->csw = 0.0;
}

}  // namespace cola
