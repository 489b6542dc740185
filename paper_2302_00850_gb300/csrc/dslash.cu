// Wilson hopping term on checkerboarded fields (the fermion-matrix kernel).
//
// The paper maps one lattice site to one GPU thread and notes that lattice
// codes are memory-bandwidth bound, so spending arithmetic to save traffic
// pays (its discussion of the GPU inverter).  This kernel follows that: one
// thread per output site and right-hand side; links stored as two rows and
// the third rebuilt in registers (recon 12); spinors in a structure-of-arrays
// checkerboard layout so that each 16-byte load of a warp is coalesced;
// FP16 storage with a per-site scale for the inner solver.
//
// For output parity p and each direction mu:
//   forward : (1 - s gamma_mu) Ut_mu(x) psi(x + mu)
//   backward: (1 + s gamma_mu) Ut_mu(x - mu)^dag psi(x - mu)
// with s = +1 for H and s = -1 for H^dag (projectors swapped).  Each
// projector has rank two, so the SU(3) multiply acts on a two-spinor and
// the other two spin rows are rebuilt from it (spin projection and
// reconstruction, gamma matrices in the DeGrand-Rossi basis).
#include "cola_impl.h"

namespace cola {

// a + s*i*b
template <typename R, int S>
__device__ __forceinline__ Cx<R> add_si(Cx<R> a, Cx<R> b) {
    if constexpr (S > 0) return {a.re - b.im, a.im + b.re};
    else return {a.re + b.im, a.im - b.re};
}
template <typename R, int S>
__device__ __forceinline__ Cx<R> add_s(Cx<R> a, Cx<R> b) {
    if constexpr (S > 0) return {a.re + b.re, a.im + b.im};
    else return {a.re - b.re, a.im - b.im};
}

// Two-spinor h = rows 0, 1 of (1 + S gamma_mu) psi.
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const Cx<R> (&psi)[12], Cx<R> (&h)[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Cx<R> p0 = psi[a], p1 = psi[3 + a], p2 = psi[6 + a], p3 = psi[9 + a];
        if constexpr (MU == 0) {         // gamma_x psi = (i p3, i p2, -i p1, -i p0)
            h[0][a] = add_si<R, S>(p0, p3);
            h[1][a] = add_si<R, S>(p1, p2);
        } else if constexpr (MU == 1) {  // gamma_y psi = (-p3, p2, p1, -p0)
            h[0][a] = add_s<R, -S>(p0, p3);
            h[1][a] = add_s<R, S>(p1, p2);
        } else if constexpr (MU == 2) {  // gamma_z psi = (i p2, -i p3, -i p0, i p1)
            h[0][a] = add_si<R, S>(p0, p2);
            h[1][a] = add_si<R, -S>(p1, p3);
        } else {                         // gamma_t psi = (p2, p3, p0, p1)
            h[0][a] = add_s<R, S>(p0, p2);
            h[1][a] = add_s<R, S>(p1, p3);
        }
    }
}

template <typename R>
__device__ __forceinline__ Cx<R> times_i(Cx<R> a, int s) {  // s*i*a
    return s > 0 ? Cx<R>{-a.im, a.re} : Cx<R>{a.im, -a.re};
}

// acc += full spinor rebuilt from w = U h (rows 2, 3 follow from rows 0, 1).
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate(Cx<R> (&acc)[12], const Cx<R> (&w)[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a].re += w[0][a].re;
        acc[a].im += w[0][a].im;
        acc[3 + a].re += w[1][a].re;
        acc[3 + a].im += w[1][a].im;
        Cx<R> r2, r3;
        if constexpr (MU == 0) {         // r2 = -S i w1, r3 = -S i w0
            r2 = times_i(w[1][a], -S);
            r3 = times_i(w[0][a], -S);
        } else if constexpr (MU == 1) {  // r2 = S w1, r3 = -S w0
            r2 = {S * w[1][a].re, S * w[1][a].im};
            r3 = {-S * w[0][a].re, -S * w[0][a].im};
        } else if constexpr (MU == 2) {  // r2 = -S i w0, r3 = S i w1
            r2 = times_i(w[0][a], -S);
            r3 = times_i(w[1][a], S);
        } else {                         // r2 = S w0, r3 = S w1
            r2 = {S * w[0][a].re, S * w[0][a].im};
            r3 = {S * w[1][a].re, S * w[1][a].im};
        }
        acc[6 + a].re += r2.re;
        acc[6 + a].im += r2.im;
        acc[9 + a].re += r3.re;
        acc[9 + a].im += r3.im;
    }
}

template <typename R>
__device__ __forceinline__ void su3_mul(const Cx<R> (&u)[9], const Cx<R> (&h)[2][3], Cx<R> (&w)[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Cx<R> s = cmul(u[3 * a], h[k][0]);
            cmac(s, u[3 * a + 1], h[k][1]);
            cmac(s, u[3 * a + 2], h[k][2]);
            w[k][a] = s;
        }
}

template <typename R>
__device__ __forceinline__ void su3_adj_mul(const Cx<R> (&u)[9], const Cx<R> (&h)[2][3], Cx<R> (&w)[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Cx<R> s = {R(0), R(0)};
            cmac_conj(s, u[a], h[k][0]);
            cmac_conj(s, u[3 + a], h[k][1]);
            cmac_conj(s, u[6 + a], h[k][2]);
            w[k][a] = s;
        }
}

template <typename R>
__device__ __forceinline__ void phase_mul(Cx<R> (&w)[2][3], R pr, R pi) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) w[k][a] = cmul(w[k][a], Cx<R>{pr, pi});
}

template <int P, int RECON, int MU, bool DAGGER>
__device__ __forceinline__ void hop_mu(const DslashArgs &A, const Coord &c, int cb, const char *in,
                                       const char *links_out, const char *links_in,
                                       Cx<typename Prec<P>::real> (&acc)[12]) {
    using R = typename Prec<P>::real;
    const Geom &g = A.g;
    constexpr int SF = DAGGER ? +1 : -1;  // forward projector 1 + SF gamma
    constexpr int SB = -SF;
    {
        const int nb = nbr_cb<MU, +1>(g, c, cb);
        Cx<R> psi[12];
        SpinorIO<P>::load(in, g.Vh, nb, psi);
        Cx<R> h[2][3];
        project<MU, SF>(psi, h);
        Cx<R> u[9];
        LinkIO<P, RECON>::load(links_out + MU * A.link_dir_stride, g.Vh, cb, u);
        Cx<R> w[2][3];
        su3_mul(u, h, w);
        if (!g.bc_trivial[MU] && coord_of<MU>(c) == g.L[MU] - 1)
            phase_mul(w, (R)g.bc[MU][0], (R)g.bc[MU][1]);
        accumulate<MU, SF>(acc, w);
    }
    {
        const int nb = nbr_cb<MU, -1>(g, c, cb);
        Cx<R> psi[12];
        SpinorIO<P>::load(in, g.Vh, nb, psi);
        Cx<R> h[2][3];
        project<MU, SB>(psi, h);
        Cx<R> u[9];
        LinkIO<P, RECON>::load(links_in + MU * A.link_dir_stride, g.Vh, nb, u);
        Cx<R> w[2][3];
        su3_adj_mul(u, h, w);
        if (!g.bc_trivial[MU] && coord_of<MU>(c) == 0)
            phase_mul(w, (R)g.bc[MU][0], -(R)g.bc[MU][1]);
        accumulate<MU, SB>(acc, w);
    }
}

// Grid: x over checkerboard sites, y over right-hand-side groups, z over the
// output parities (1 or 2).  Block: (sites, right-hand sides).
template <int P, int RECON, bool DAGGER, bool XPAY, bool RED>
__global__ void __launch_bounds__(256) dslash_kernel(const DslashArgs A) {
    using R = typename Prec<P>::real;
    __shared__ double sh[32];
    const Geom &g = A.g;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y * blockDim.y + threadIdx.y;
    const int par = A.parity0 + blockIdx.z;
    const bool row_ok = rhs < A.nrhs;
    bool live = row_ok;
    if (live && A.state) {
        const CgState &st = A.state[rhs];
        live = A.filter_ru ? (st.ru && !st.done) : !st.done;
    }
    double nrm = 0.0;
    if (cb < g.Vh && live) {
        const Coord c = cb_coord(g, cb, par);
        const char *in = static_cast<const char *>(A.in) + rhs * A.rhs_stride + (1 - par) * A.parity_stride;
        const char *lo = static_cast<const char *>(A.links) + par * A.link_parity_stride;
        const char *li = static_cast<const char *>(A.links) + (1 - par) * A.link_parity_stride;
        Cx<R> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
        hop_mu<P, RECON, 0, DAGGER>(A, c, cb, in, lo, li, acc);
        hop_mu<P, RECON, 1, DAGGER>(A, c, cb, in, lo, li, acc);
        hop_mu<P, RECON, 2, DAGGER>(A, c, cb, in, lo, li, acc);
        hop_mu<P, RECON, 3, DAGGER>(A, c, cb, in, lo, li, acc);
        const R b = (R)A.b;
        if constexpr (XPAY) {
            const R a = (R)A.a;
            Cx<R> xs[12];
            SpinorIO<P>::load(static_cast<const char *>(A.xin) + rhs * A.rhs_stride + par * A.parity_stride,
                              g.Vh, cb, xs);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[k].re = a * xs[k].re + b * acc[k].re;
                acc[k].im = a * xs[k].im + b * acc[k].im;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[k].re *= b;
                acc[k].im *= b;
            }
        }
        SpinorIO<P>::store(static_cast<char *>(A.out) + rhs * A.rhs_stride + par * A.parity_stride, g.Vh, cb,
                           acc);
        if constexpr (RED) {
            R s = R(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) s += acc[k].re * acc[k].re + acc[k].im * acc[k].im;
            nrm = (double)s;
        }
    }
    if constexpr (RED) {
        const int nblocks = gridDim.x * gridDim.z;
        const int bid = blockIdx.z * gridDim.x + blockIdx.x;
        double tot;
        if (reduce_rows_last_block(nrm, A.partials, A.counters + blockIdx.y, nblocks, bid, rhs, row_ok, sh,
                                   &tot)) {
            if (threadIdx.x == 0 && row_ok) {
                if (A.state) {
                    CgState &st = A.state[rhs];
                    if (!st.done) {
                        st.pq = tot;
                        st.rho = st.rho_new;
                        st.alpha = st.rho / tot;
                        if (!(tot > 0.0) || !isfinite(st.alpha)) {
                            st.status = COLA_ERR_BREAKDOWN;
                            st.done = 1;
                        }
                    }
                } else if (A.result) {
                    A.result[rhs] = tot;
                }
            }
        }
    }
}

template <int P, int RECON, bool DAGGER, bool XPAY, bool RED>
static cudaError_t launch_t(const DslashArgs &A, int nparity, int bx, cudaStream_t s) {
    const int by = A.rhs_per_block;
    dim3 block(bx, by, 1);
    dim3 grid((A.g.Vh + bx - 1) / bx, (A.nrhs + by - 1) / by, nparity);
    dslash_kernel<P, RECON, DAGGER, XPAY, RED><<<grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

template <int P, int RECON>
static cudaError_t launch_r(const DslashArgs &A, int nparity, bool dagger, bool xpay, bool red, int bx,
                            cudaStream_t s) {
    if (dagger) {
        if (xpay) return red ? launch_t<P, RECON, true, true, true>(A, nparity, bx, s)
                             : launch_t<P, RECON, true, true, false>(A, nparity, bx, s);
        return red ? launch_t<P, RECON, true, false, true>(A, nparity, bx, s)
                   : launch_t<P, RECON, true, false, false>(A, nparity, bx, s);
    }
    if (xpay) return red ? launch_t<P, RECON, false, true, true>(A, nparity, bx, s)
                         : launch_t<P, RECON, false, true, false>(A, nparity, bx, s);
    return red ? launch_t<P, RECON, false, false, true>(A, nparity, bx, s)
               : launch_t<P, RECON, false, false, false>(A, nparity, bx, s);
}

cudaError_t launch_dslash(int prec, int recon, const DslashArgs &A, int nparity, bool dagger, bool xpay,
                          bool red, int block_x, cudaStream_t s) {
    if (block_x <= 0) block_x = default_dslash_block(prec, A.rhs_per_block);
    switch (prec) {
        case COLA_F64:
            return recon == 12 ? launch_r<COLA_F64, 12>(A, nparity, dagger, xpay, red, block_x, s)
                               : launch_r<COLA_F64, 18>(A, nparity, dagger, xpay, red, block_x, s);
        case COLA_F32:
            return recon == 12 ? launch_r<COLA_F32, 12>(A, nparity, dagger, xpay, red, block_x, s)
                               : launch_r<COLA_F32, 18>(A, nparity, dagger, xpay, red, block_x, s);
        default:
            return recon == 12 ? launch_r<COLA_F16, 12>(A, nparity, dagger, xpay, red, block_x, s)
                               : launch_r<COLA_F16, 18>(A, nparity, dagger, xpay, red, block_x, s);
    }
}

int default_dslash_block(int prec, int rhs_per_block) {
    int bx = prec == COLA_F64 ? 128 : 128;
    while (bx * rhs_per_block > 256 && bx > 32) bx >>= 1;
    return bx;
}

}  // namespace cola
