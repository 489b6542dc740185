// Fused vector updates and FP64 reductions of the conjugate-gradient solver.
//
// The paper's benchmark solver uses 32-bit inner iterations and a 64-bit outer
// solver (its Fig. 2 discussion, after Clark et al.).  Here every CG scalar
// (alpha, beta, |r|^2, <p, Ap>) is reduced in FP64 on the device, and each
// update kernel also produces the next reduction so that one pass over the
// vectors does both.  Reductions are deterministic: each block writes one
// partial per row with a plain store, then a finishing kernel with one block
// per row sums the partials in block order and makes the solver's decisions
// (reliable update due, converged, iteration cap, breakdown) in CgState.  No
// floating-point atomics and no memory fences are involved, so repeated
// solves give identical results.  Every kernel walks one table of lattices
// (a batch of up to kMaxBatch lattices, each with nrhs right-hand sides), so
// a batch of uneven lattices is one launch per step.
#include <algorithm>

#include "cola_impl.h"

namespace cola {

static constexpr int kBlasBlock = 256;

// Site s of lattice l (s in [0, nparity * vh)) -> parity and checkerboard index.
struct SiteRef {
    int l, rhs, row, s, par, cb, bid;
    bool ok;
};

__device__ __forceinline__ SiteRef blas_site(const BlasArgs &B) {
    SiteRef r;
    int l = 0;
    while (l + 1 < B.nlat && (int)blockIdx.x >= B.lat[l + 1].block0) ++l;
    const BlasLat &L = B.lat[l];
    r.l = l;
    r.bid = (int)blockIdx.x - L.block0;
    r.s = r.bid * blockDim.x + threadIdx.x;
    r.rhs = blockIdx.y;
    r.row = L.row0 + r.rhs;
    r.ok = r.s < L.vh * B.nparity;
    r.par = r.s >= L.vh;
    r.cb = r.s - r.par * L.vh;
    return r;
}

__device__ __forceinline__ const char *vptr(const BlasArgs &B, const SiteRef &r, int k) {
    const size_t ps = spinor_parity_bytes(B.prec[k], B.lat[r.l].vh);
    return static_cast<const char *>(B.lat[r.l].v[k]) + (size_t)r.rhs * 2 * ps + r.par * ps;
}
__device__ __forceinline__ char *vptr_w(const BlasArgs &B, const SiteRef &r, int k) {
    return const_cast<char *>(vptr(B, r, k));
}

template <int PD, int PS>
__device__ __forceinline__ void cvt(const Cx<typename Prec<PS>::real> (&s)[12], Cx<typename Prec<PD>::real> (&d)[12]) {
    using RD = typename Prec<PD>::real;
#pragma unroll
    for (int k = 0; k < 12; ++k) d[k] = {(RD)s[k].re, (RD)s[k].im};
}

template <typename R>
__device__ __forceinline__ double site_norm2(const Cx<R> (&s)[12]) {
    R a = R(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) a += s[k].re * s[k].re + s[k].im * s[k].im;
    return (double)a;
}

// The block's partial of its row (every thread of the block takes part).
__device__ __forceinline__ void write_partial(const BlasArgs &B, const SiteRef &r, double v) {
    __shared__ double sh[kBlasBlock / 32];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) B.partials[(size_t)r.row * B.pstride + r.bid] = t;
}

// ---------------------------------------------------------------------------
// slots (x, r, p, q):  x += alpha p;  r -= alpha q;  partial |r|^2
template <int PX, int PV>
__global__ void __launch_bounds__(kBlasBlock) cg_update_xr_kernel(const __grid_constant__ BlasArgs B) {
    using RV = typename Prec<PV>::real;
    using RX = typename Prec<PX>::real;
    const SiteRef r = blas_site(B);
    const CgState &S = B.state[r.row];
    double nr = 0.0;
    if (!S.done && r.ok) {
        const double alpha = S.alpha;
        const int vh = B.lat[r.l].vh;
        Cx<RV> pv[12], qv[12], rv[12];
        Cx<RX> xv[12];
        SpinorIO<PV>::load(vptr(B, r, 2), vh, r.cb, pv);
        SpinorIO<PV>::load(vptr(B, r, 3), vh, r.cb, qv);
        SpinorIO<PV>::load(vptr(B, r, 1), vh, r.cb, rv);
        SpinorIO<PX>::load(vptr(B, r, 0), vh, r.cb, xv);
        const RV a = (RV)alpha;
        const RX ax = (RX)alpha;
        if (S.shift != 0.0) {  // q + sigma p is the shifted operator's A p
            const RV sg = (RV)S.shift;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                qv[k].re = fma(sg, pv[k].re, qv[k].re);
                qv[k].im = fma(sg, pv[k].im, qv[k].im);
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xv[k].re += ax * (RX)pv[k].re;
            xv[k].im += ax * (RX)pv[k].im;
            rv[k].re -= a * qv[k].re;
            rv[k].im -= a * qv[k].im;
        }
        SpinorIO<PX>::store(vptr_w(B, r, 0), vh, r.cb, xv);
        SpinorIO<PV>::store(vptr_w(B, r, 1), vh, r.cb, rv);
        nr = site_norm2(rv);
    }
    write_partial(B, r, nr);
}

// slots (p, r):  p = r + beta p,  beta = rho_new / rho
template <int PV>
__global__ void __launch_bounds__(kBlasBlock) cg_update_p_kernel(const __grid_constant__ BlasArgs B) {
    using RV = typename Prec<PV>::real;
    const SiteRef r = blas_site(B);
    const CgState &S = B.state[r.row];
    if (S.done || !r.ok) return;
    const int vh = B.lat[r.l].vh;
    const RV beta = (RV)(S.rho_new / S.rho);
    Cx<RV> pv[12], rv[12];
    SpinorIO<PV>::load(vptr(B, r, 0), vh, r.cb, pv);
    SpinorIO<PV>::load(vptr(B, r, 1), vh, r.cb, rv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        pv[k].re = rv[k].re + beta * pv[k].re;
        pv[k].im = rv[k].im + beta * pv[k].im;
    }
    SpinorIO<PV>::store(vptr_w(B, r, 0), vh, r.cb, pv);
}

// slots (mp, p):  partial |M p|^2 = <p, A p>  (+ sigma |p|^2 for a shifted row)
template <int PV>
__global__ void __launch_bounds__(kBlasBlock) cg_pq_kernel(const __grid_constant__ BlasArgs B) {
    const SiteRef r = blas_site(B);
    const CgState &S = B.state[r.row];
    double nr = 0.0;
    if (!S.done && r.ok) {
        Cx<typename Prec<PV>::real> m[12];
        SpinorIO<PV>::load(vptr(B, r, 0), B.lat[r.l].vh, r.cb, m);
        nr = site_norm2(m);
        if (S.shift != 0.0) {
            SpinorIO<PV>::load(vptr(B, r, 1), B.lat[r.l].vh, r.cb, m);
            nr += S.shift * site_norm2(m);
        }
    }
    write_partial(B, r, nr);
}

// slots (x_hi, x_lo):  x_hi += x_lo;  x_lo = 0
template <int PX>
__global__ void __launch_bounds__(kBlasBlock) ru_accumulate_kernel(const __grid_constant__ BlasArgs B, int force) {
    using RX = typename Prec<PX>::real;
    const SiteRef r = blas_site(B);
    const CgState &S = B.state[r.row];
    if (!(force || (S.ru && !S.done)) || !r.ok) return;
    const int vh = B.lat[r.l].vh;
    Cx<double> xh[12];
    Cx<RX> xl[12];
    SpinorIO<COLA_F64>::load(vptr(B, r, 0), vh, r.cb, xh);
    SpinorIO<PX>::load(vptr(B, r, 1), vh, r.cb, xl);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        xh[k].re += (double)xl[k].re;
        xh[k].im += (double)xl[k].im;
        xl[k] = {RX(0), RX(0)};
    }
    SpinorIO<COLA_F64>::store(vptr_w(B, r, 0), vh, r.cb, xh);
    SpinorIO<PX>::store(vptr_w(B, r, 1), vh, r.cb, xl);
}

__device__ __forceinline__ bool ru_live(const BlasArgs &B, const CgState &S) {
    return B.init ? true : (S.ru && !S.done);
}

// slots (r_hi, b, ax, r_lo, p, x_hi):  r_hi = b - ax (- sigma x_hi);  r_lo = r_hi;  (init: p = r_lo);
// partial |r_hi|^2
template <int PV>
__global__ void __launch_bounds__(kBlasBlock) ru_residual_kernel(const __grid_constant__ BlasArgs B) {
    const SiteRef r = blas_site(B);
    const CgState &S = B.state[r.row];
    double nr = 0.0;
    if (ru_live(B, S) && r.ok) {
        const int vh = B.lat[r.l].vh;
        Cx<double> bv[12], av[12];
        SpinorIO<COLA_F64>::load(vptr(B, r, 1), vh, r.cb, bv);
        SpinorIO<COLA_F64>::load(vptr(B, r, 2), vh, r.cb, av);
        if (S.shift != 0.0) {
            Cx<double> xv[12];
            SpinorIO<COLA_F64>::load(vptr(B, r, 5), vh, r.cb, xv);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                av[k].re = fma(S.shift, xv[k].re, av[k].re);
                av[k].im = fma(S.shift, xv[k].im, av[k].im);
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            bv[k].re -= av[k].re;
            bv[k].im -= av[k].im;
        }
        SpinorIO<COLA_F64>::store(vptr_w(B, r, 0), vh, r.cb, bv);
        Cx<typename Prec<PV>::real> lv[12];
        cvt<PV, COLA_F64>(bv, lv);
        SpinorIO<PV>::store(vptr_w(B, r, 3), vh, r.cb, lv);
        if (B.init) SpinorIO<PV>::store(vptr_w(B, r, 4), vh, r.cb, lv);
        nr = site_norm2(bv);
    }
    write_partial(B, r, nr);
}

// slot (v):  partial |v|^2
template <int P>
__global__ void __launch_bounds__(kBlasBlock) norm2_kernel(const __grid_constant__ BlasArgs B) {
    const SiteRef r = blas_site(B);
    double nr = 0.0;
    if (r.ok) {
        Cx<typename Prec<P>::real> a[12];
        SpinorIO<P>::load(vptr(B, r, 0), B.lat[r.l].vh, r.cb, a);
        nr = site_norm2(a);
    }
    write_partial(B, r, nr);
}

// ------------------------------------------------------------- finishing --
enum FinishMode { FIN_XR, FIN_PQ, FIN_RU, FIN_NORM, FIN_INIT };

// reliable updates without a new smallest true residual before a row stops
constexpr int kStallUpdates = 3;
// iterations without a 4x drop of the iterated |r|^2 before a true-residual check
constexpr int kPlateauIters = 500;
// (|r|/|b|)^2 below which FP64 CG checks its true residual every 100x drop of |r|
constexpr double kDeepRel2 = 1e-28;

// One block per row: sum the row's block partials in block order, then decide.
template <int MODE>
__global__ void __launch_bounds__(512) finish_kernel(const __grid_constant__ BlasArgs B) {
    __shared__ double sh[512 / 32];
    const int row = blockIdx.x;
    const int l = row / B.nrhs;  // rows are lattice-major
    const int nb = B.lat[l].nblocks;
    const double *part = B.partials + (size_t)row * B.pstride;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    int b = threadIdx.x;
    for (; b + 3 * (int)blockDim.x < nb; b += 4 * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] += part[b + k * blockDim.x];
    }
    for (; b < nb; b += blockDim.x) a[0] += part[b];
    const double tot = block_sum((a[0] + a[1]) + (a[2] + a[3]), sh);
    if (threadIdx.x != 0) return;
    if constexpr (MODE == FIN_NORM) {
        B.out[row] = tot;
    } else {
        CgState &S = B.state[row];
        if constexpr (MODE == FIN_INIT) {
            S.b2 = tot;
            S.tol2 = S.tol2 * tot;  // tol2 holds tol^2 on entry
            if (tot == 0.0) {
                S.done = 1;
                S.status = COLA_OK;
            }
        } else if constexpr (MODE == FIN_PQ) {
            if (S.done) return;
            S.pq = tot;
            S.rho = S.rho_new;
            S.alpha = S.rho / tot;
            if (!(tot > 0.0) || !isfinite(S.alpha)) {
                S.status = COLA_ERR_BREAKDOWN;
                S.done = 1;
            }
        } else if constexpr (MODE == FIN_XR) {
            if (S.done) return;
            S.rho_new = tot;
            S.iter += 1;
            if (!isfinite(tot)) {
                S.status = COLA_ERR_BREAKDOWN;
                S.done = 1;
            } else {
                // Two more triggers of an FP64 true residual, so that a solve whose
                // tolerance is out of reach is seen to stagnate even when delta never
                // fires (plain FP64 CG): a plateau of the iterated residual (no 4x drop
                // in kPlateauIters iterations), and, in FP64 CG below the level FP64
                // resolves (|r|/|b| < 1e-14), every further 100x drop of |r|.
                if (tot < 0.25 * S.rho_mark) {
                    S.rho_mark = tot;
                    S.it_mark = S.iter;
                }
                const bool deep = S.delta2 == 0.0 && tot < kDeepRel2 * S.b2 && tot < 1e-4 * S.r2_last;
                S.ru = (tot < S.delta2 * S.r2_last) || (tot <= S.tol2) || (S.iter >= S.max_iter) ||
                       (S.iter - S.it_mark >= kPlateauIters) || deep;
            }
        } else {  // FIN_RU
            if (!ru_live(B, S)) return;
            S.rho_new = tot;
            S.r2_last = tot;
            S.ru = 0;
            S.ru_count += 1;
            // stagnation: the FP64 true residual has not improved over kStallUpdates
            // reliable updates (a tolerance below what the precision reaches)
            if (S.r2_best == 0.0 || tot < S.r2_best) {
                S.r2_best = tot;
                S.stall = 0;
            } else {
                S.stall += 1;
            }
            S.rho_mark = tot;
            S.it_mark = S.iter;
            if (!isfinite(tot)) {
                S.status = COLA_ERR_BREAKDOWN;
                S.done = 1;
            } else if (tot <= S.tol2) {
                S.status = COLA_OK;
                S.done = 1;
            } else if (S.iter >= S.max_iter || S.stall >= kStallUpdates) {
                S.status = COLA_ERR_NOT_CONVERGED;
                S.done = 1;
            }
        }
    }
}

// slot (v):  flags[row] |= 1 if any stored bit of the row's field is nonzero
// (an initial guess of exactly zero lets the solver skip A x0).
__global__ void __launch_bounds__(kBlasBlock) any_nonzero_kernel(const __grid_constant__ BlasArgs B, unsigned *flags) {
    const SiteRef r = blas_site(B);
    bool nz = false;
    if (r.ok) {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(vptr(B, r, 0));
        const int vh = B.lat[r.l].vh;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const ulonglong2 v = __ldg(p + (size_t)c * vh + r.cb);
            nz |= ((v.x | v.y) << 1) != 0;  // -0.0 counts as zero
        }
    }
    if (__any_sync(0xffffffffu, nz) && (threadIdx.x & 31) == 0) atomicOr(flags + r.row, 1u);
}

// slots (dst, src)
template <int PD, int PS>
__global__ void __launch_bounds__(kBlasBlock) convert_kernel(const __grid_constant__ BlasArgs B) {
    const SiteRef r = blas_site(B);
    if (!r.ok) return;
    const int vh = B.lat[r.l].vh;
    Cx<typename Prec<PS>::real> a[12];
    Cx<typename Prec<PD>::real> b[12];
    SpinorIO<PS>::load(vptr(B, r, 1), vh, r.cb, a);
    cvt<PD, PS>(a, b);
    SpinorIO<PD>::store(vptr_w(B, r, 0), vh, r.cb, b);
}

// slots (dst, x, y):  dst = a x + b y (one precision)
template <int P>
__global__ void __launch_bounds__(kBlasBlock) axpby_kernel(const __grid_constant__ BlasArgs B) {
    using R = typename Prec<P>::real;
    const SiteRef r = blas_site(B);
    if (!r.ok) return;
    const int vh = B.lat[r.l].vh;
    Cx<R> xv[12], yv[12];
    SpinorIO<P>::load(vptr(B, r, 1), vh, r.cb, xv);
    SpinorIO<P>::load(vptr(B, r, 2), vh, r.cb, yv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        xv[k].re = (R)B.a * xv[k].re + (R)B.b * yv[k].re;
        xv[k].im = (R)B.a * xv[k].im + (R)B.b * yv[k].im;
    }
    SpinorIO<P>::store(vptr_w(B, r, 0), vh, r.cb, xv);
}

// ------------------------------------------------------------------ launch --
static dim3 blas_grid(BlasArgs &B) {
    int total = 0;
    for (int l = 0; l < B.nlat; ++l) {
        B.lat[l].block0 = total;
        B.lat[l].nblocks = (B.lat[l].vh * B.nparity + kBlasBlock - 1) / kBlasBlock;
        total += B.lat[l].nblocks;
    }
    return dim3(total, B.nrhs);
}

int blas_max_blocks(const BlasArgs &B) {
    int mx = 0;
    for (int l = 0; l < B.nlat; ++l) {
        const int nb = (B.lat[l].vh * B.nparity + kBlasBlock - 1) / kBlasBlock;
        if (nb > mx) mx = nb;
    }
    return mx;
}

template <int MODE>
static cudaError_t finish(const BlasArgs &B, cudaStream_t s) {
    finish_kernel<MODE><<<B.nlat * B.nrhs, 512, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_cg_update_xr(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[1] == COLA_F64) cg_update_xr_kernel<COLA_F64, COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[1] == COLA_F32) cg_update_xr_kernel<COLA_F32, COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else cg_update_xr_kernel<COLA_F32, COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : finish<FIN_XR>(B, s);
}

cudaError_t launch_cg_update_p(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[0] == COLA_F64) cg_update_p_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[0] == COLA_F32) cg_update_p_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else cg_update_p_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_cg_pq(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[0] == COLA_F64) cg_pq_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[0] == COLA_F32) cg_pq_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else cg_pq_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : finish<FIN_PQ>(B, s);
}

cudaError_t launch_finish_pq(const BlasArgs &B, cudaStream_t s) { return finish<FIN_PQ>(B, s); }

int reduce_stride(int vh) {
    // vector kernels: 256 sites per block over both parities; hopping
    // launches: at least 32 sites per block, both parities
    return std::max((2 * vh + kBlasBlock - 1) / kBlasBlock, 2 * ((vh + 31) / 32));
}

cudaError_t launch_ru_accumulate(BlasArgs &B, bool force, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[1] == COLA_F64) ru_accumulate_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B, force);
    else ru_accumulate_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(B, force);
    return cudaGetLastError();
}

cudaError_t launch_ru_residual(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[3] == COLA_F64) ru_residual_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[3] == COLA_F32) ru_residual_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else ru_residual_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : finish<FIN_RU>(B, s);
}

cudaError_t launch_init_norms(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    norm2_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : finish<FIN_INIT>(B, s);
}

cudaError_t launch_norm2(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[0] == COLA_F64) norm2_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[0] == COLA_F32) norm2_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else norm2_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : finish<FIN_NORM>(B, s);
}

cudaError_t launch_any_nonzero(BlasArgs &B, unsigned *flags, cudaStream_t s) {
    if (B.prec[0] != COLA_F64) return cudaErrorInvalidValue;
    any_nonzero_kernel<<<blas_grid(B), kBlasBlock, 0, s>>>(B, flags);
    return cudaGetLastError();
}

template <int PD>
static void convert_from(BlasArgs &B, dim3 g, cudaStream_t s) {
    if (B.prec[1] == COLA_F64) convert_kernel<PD, COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[1] == COLA_F32) convert_kernel<PD, COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else convert_kernel<PD, COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
}

cudaError_t launch_convert(BlasArgs &B, cudaStream_t s) {
    const dim3 g = blas_grid(B);
    if (B.prec[0] == COLA_F64) convert_from<COLA_F64>(B, g, s);
    else if (B.prec[0] == COLA_F32) convert_from<COLA_F32>(B, g, s);
    else convert_from<COLA_F16>(B, g, s);
    return cudaGetLastError();
}

cudaError_t launch_axpby(BlasArgs &B, cudaStream_t s) {
    if (B.prec[0] != B.prec[1] || B.prec[0] != B.prec[2]) return cudaErrorInvalidValue;
    const dim3 g = blas_grid(B);
    if (B.prec[0] == COLA_F64) axpby_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(B);
    else if (B.prec[0] == COLA_F32) axpby_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(B);
    else axpby_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(B);
    return cudaGetLastError();
}

}  // namespace cola
