// Fused vector updates and FP64 reductions of the conjugate-gradient solver.
//
// The paper's benchmark solver uses 32-bit inner iterations and a 64-bit outer
// solver (its Fig. 2 discussion, after Clark et al.).  Here every CG scalar
// (alpha, beta, |r|^2, <p, Ap>) is reduced in FP64 on the device, in a fixed
// block order so repeated solves give identical results, and each update
// kernel also produces the next reduction so that one pass over the vectors
// does both.  The last block of each reduction makes the solver's decisions
// (reliable update due, converged, iteration cap, breakdown) in CgState.
#include "cola_impl.h"

namespace cola {

template <int P>
__device__ __forceinline__ const char *vptr(const VecRef &v, int rhs, int par) {
    return static_cast<const char *>(v.ptr) + rhs * v.rhs_stride + par * v.parity_stride;
}
template <int P>
__device__ __forceinline__ char *vptr_w(const VecRef &v, int rhs, int par) {
    return static_cast<char *>(v.ptr) + rhs * v.rhs_stride + par * v.parity_stride;
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

// ---------------------------------------------------------------------------
// x += alpha p;  r -= alpha q;  rho_new = |r|^2
template <int PX, int PV>
__global__ void __launch_bounds__(256) cg_update_xr_kernel(const BlasDims d, const VecRef x, const VecRef r,
                                                           const VecRef p, const VecRef q, CgState *st,
                                                           double *partials, unsigned *counters) {
    using RV = typename Prec<PV>::real;
    using RX = typename Prec<PX>::real;
    __shared__ double sh[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    CgState &S = st[rhs];
    const bool live = !S.done;
    double nr = 0.0;
    if (live && s < d.vh * d.nparity) {
        const int par = s >= d.vh;
        const int cb = s - par * d.vh;
        const double alpha = S.alpha;
        Cx<RV> pv[12], qv[12], rv[12];
        Cx<RX> xv[12];
        SpinorIO<PV>::load(vptr<PV>(p, rhs, par), d.vh, cb, pv);
        SpinorIO<PV>::load(vptr<PV>(q, rhs, par), d.vh, cb, qv);
        SpinorIO<PV>::load(vptr<PV>(r, rhs, par), d.vh, cb, rv);
        SpinorIO<PX>::load(vptr<PX>(x, rhs, par), d.vh, cb, xv);
        const RV a = (RV)alpha;
        const RX ax = (RX)alpha;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            xv[k].re += ax * (RX)pv[k].re;
            xv[k].im += ax * (RX)pv[k].im;
            rv[k].re -= a * qv[k].re;
            rv[k].im -= a * qv[k].im;
        }
        SpinorIO<PX>::store(vptr_w<PX>(x, rhs, par), d.vh, cb, xv);
        SpinorIO<PV>::store(vptr_w<PV>(r, rhs, par), d.vh, cb, rv);
        nr = site_norm2(rv);
    }
    double tot;
    if (reduce_rows_last_block(nr, partials, counters + rhs, gridDim.x, blockIdx.x, rhs, true, sh, &tot)) {
        if (threadIdx.x == 0 && live) {
            S.rho_new = tot;
            S.iter += 1;
            if (!isfinite(tot)) {
                S.status = COLA_ERR_BREAKDOWN;
                S.done = 1;
            } else {
                S.ru = (tot < S.delta2 * S.r2_last) || (tot <= S.tol2) || (S.iter >= S.max_iter);
            }
        }
    }
}

// p = r + beta p, beta = rho_new / rho
template <int PV>
__global__ void __launch_bounds__(256) cg_update_p_kernel(const BlasDims d, const VecRef p, const VecRef r,
                                                          const CgState *st) {
    using RV = typename Prec<PV>::real;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    const CgState &S = st[rhs];
    if (S.done || s >= d.vh * d.nparity) return;
    const int par = s >= d.vh;
    const int cb = s - par * d.vh;
    const RV beta = (RV)(S.rho_new / S.rho);
    Cx<RV> pv[12], rv[12];
    SpinorIO<PV>::load(vptr<PV>(p, rhs, par), d.vh, cb, pv);
    SpinorIO<PV>::load(vptr<PV>(r, rhs, par), d.vh, cb, rv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        pv[k].re = rv[k].re + beta * pv[k].re;
        pv[k].im = rv[k].im + beta * pv[k].im;
    }
    SpinorIO<PV>::store(vptr_w<PV>(p, rhs, par), d.vh, cb, pv);
}

// x_hi += x_lo; x_lo = 0
template <int PX>
__global__ void __launch_bounds__(256) ru_accumulate_kernel(const BlasDims d, const VecRef xhi, const VecRef xlo,
                                                            const CgState *st, int force) {
    using RX = typename Prec<PX>::real;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    const CgState &S = st[rhs];
    if (!(force || (S.ru && !S.done)) || s >= d.vh * d.nparity) return;
    const int par = s >= d.vh;
    const int cb = s - par * d.vh;
    Cx<double> xh[12];
    Cx<RX> xl[12];
    SpinorIO<COLA_F64>::load(vptr<COLA_F64>(xhi, rhs, par), d.vh, cb, xh);
    SpinorIO<PX>::load(vptr<PX>(xlo, rhs, par), d.vh, cb, xl);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        xh[k].re += (double)xl[k].re;
        xh[k].im += (double)xl[k].im;
        xl[k] = {RX(0), RX(0)};
    }
    SpinorIO<COLA_F64>::store(vptr_w<COLA_F64>(xhi, rhs, par), d.vh, cb, xh);
    SpinorIO<PX>::store(vptr_w<PX>(xlo, rhs, par), d.vh, cb, xl);
}

// r_hi = b - Ax;  r_lo = r_hi;  (init: p = r_lo);  |r_hi|^2 -> decisions
template <int PV>
__global__ void __launch_bounds__(256) ru_residual_kernel(const BlasDims d, const VecRef rhi, const VecRef b,
                                                          const VecRef ax, const VecRef rlo, const VecRef p,
                                                          CgState *st, int force, int init, double *partials,
                                                          unsigned *counters) {
    __shared__ double sh[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    CgState &S = st[rhs];
    const bool live = force ? !S.done || init : (S.ru && !S.done);
    double nr = 0.0;
    if (live && s < d.vh * d.nparity) {
        const int par = s >= d.vh;
        const int cb = s - par * d.vh;
        Cx<double> bv[12], av[12];
        SpinorIO<COLA_F64>::load(vptr<COLA_F64>(b, rhs, par), d.vh, cb, bv);
        SpinorIO<COLA_F64>::load(vptr<COLA_F64>(ax, rhs, par), d.vh, cb, av);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            bv[k].re -= av[k].re;
            bv[k].im -= av[k].im;
        }
        SpinorIO<COLA_F64>::store(vptr_w<COLA_F64>(rhi, rhs, par), d.vh, cb, bv);
        Cx<typename Prec<PV>::real> lv[12];
        cvt<PV, COLA_F64>(bv, lv);
        SpinorIO<PV>::store(vptr_w<PV>(rlo, rhs, par), d.vh, cb, lv);
        if (init) SpinorIO<PV>::store(vptr_w<PV>(p, rhs, par), d.vh, cb, lv);
        nr = site_norm2(bv);
    }
    double tot;
    if (reduce_rows_last_block(nr, partials, counters + rhs, gridDim.x, blockIdx.x, rhs, true, sh, &tot)) {
        if (threadIdx.x == 0 && live) {
            S.rho_new = tot;
            S.r2_last = tot;
            S.ru = 0;
            S.ru_count += 1;
            if (!isfinite(tot)) {
                S.status = COLA_ERR_BREAKDOWN;
                S.done = 1;
            } else if (tot <= S.tol2) {
                S.status = COLA_OK;
                S.done = 1;
            } else if (S.iter >= S.max_iter) {
                S.status = COLA_ERR_NOT_CONVERGED;
                S.done = 1;
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(256) norm2_kernel(const BlasDims d, const VecRef v, double *out,
                                                    CgState *st, double *partials, unsigned *counters) {
    __shared__ double sh[32];
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    double nr = 0.0;
    if (s < d.vh * d.nparity) {
        const int par = s >= d.vh;
        const int cb = s - par * d.vh;
        Cx<typename Prec<P>::real> a[12];
        SpinorIO<P>::load(vptr<P>(v, rhs, par), d.vh, cb, a);
        nr = site_norm2(a);
    }
    double tot;
    if (reduce_rows_last_block(nr, partials, counters + rhs, gridDim.x, blockIdx.x, rhs, true, sh, &tot)) {
        if (threadIdx.x == 0) {
            if (out) out[rhs] = tot;
            if (st) {
                st[rhs].b2 = tot;
                st[rhs].tol2 = st[rhs].tol2 * tot;  // tol2 holds tol^2 on entry
                if (tot == 0.0) {
                    st[rhs].done = 1;
                    st[rhs].status = COLA_OK;
                }
            }
        }
    }
}

template <int PD, int PS>
__global__ void __launch_bounds__(256) convert_kernel(const BlasDims d, const VecRef dst, const VecRef src) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (s >= d.vh * d.nparity) return;
    const int par = s >= d.vh;
    const int cb = s - par * d.vh;
    Cx<typename Prec<PS>::real> a[12];
    Cx<typename Prec<PD>::real> b[12];
    SpinorIO<PS>::load(vptr<PS>(src, rhs, par), d.vh, cb, a);
    cvt<PD, PS>(a, b);
    SpinorIO<PD>::store(vptr_w<PD>(dst, rhs, par), d.vh, cb, b);
}

template <int P>
__global__ void __launch_bounds__(256) axpby_kernel(const BlasDims d, const VecRef dst, double a, const VecRef x,
                                                    double b, const VecRef y) {
    using R = typename Prec<P>::real;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (s >= d.vh * d.nparity) return;
    const int par = s >= d.vh;
    const int cb = s - par * d.vh;
    Cx<R> xv[12], yv[12];
    SpinorIO<P>::load(vptr<P>(x, rhs, par), d.vh, cb, xv);
    SpinorIO<P>::load(vptr<P>(y, rhs, par), d.vh, cb, yv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        xv[k].re = (R)a * xv[k].re + (R)b * yv[k].re;
        xv[k].im = (R)a * xv[k].im + (R)b * yv[k].im;
    }
    SpinorIO<P>::store(vptr_w<P>(dst, rhs, par), d.vh, cb, xv);
}

// ------------------------------------------------------------------ launch --
static constexpr int kBlasBlock = 256;
static dim3 blas_grid(const BlasDims &d) { return dim3((d.vh * d.nparity + kBlasBlock - 1) / kBlasBlock, d.nrhs); }

cudaError_t launch_cg_update_xr(const BlasDims &d, VecRef x, VecRef r, VecRef p, VecRef q, CgState *st,
                                double *partials, unsigned *counters, cudaStream_t s) {
    const dim3 g = blas_grid(d);
    if (r.prec == COLA_F64) cg_update_xr_kernel<COLA_F64, COLA_F64><<<g, kBlasBlock, 0, s>>>(d, x, r, p, q, st, partials, counters);
    else if (r.prec == COLA_F32) cg_update_xr_kernel<COLA_F32, COLA_F32><<<g, kBlasBlock, 0, s>>>(d, x, r, p, q, st, partials, counters);
    else cg_update_xr_kernel<COLA_F32, COLA_F16><<<g, kBlasBlock, 0, s>>>(d, x, r, p, q, st, partials, counters);
    return cudaGetLastError();
}

cudaError_t launch_cg_update_p(const BlasDims &d, VecRef p, VecRef r, CgState *st, bool, cudaStream_t s) {
    const dim3 g = blas_grid(d);
    if (p.prec == COLA_F64) cg_update_p_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(d, p, r, st);
    else if (p.prec == COLA_F32) cg_update_p_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(d, p, r, st);
    else cg_update_p_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(d, p, r, st);
    return cudaGetLastError();
}

cudaError_t launch_ru_accumulate(const BlasDims &d, VecRef xhi, VecRef xlo, CgState *st, bool force,
                                 cudaStream_t s) {
    const dim3 g = blas_grid(d);
    if (xlo.prec == COLA_F64) ru_accumulate_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(d, xhi, xlo, st, force);
    else ru_accumulate_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(d, xhi, xlo, st, force);
    return cudaGetLastError();
}

cudaError_t launch_ru_residual(const BlasDims &d, VecRef rhi, VecRef b, VecRef ax, VecRef rlo, VecRef p,
                               CgState *st, bool force, bool init, double *partials, unsigned *counters,
                               cudaStream_t s) {
    const dim3 g = blas_grid(d);
    if (rlo.prec == COLA_F64)
        ru_residual_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(d, rhi, b, ax, rlo, p, st, force, init, partials, counters);
    else if (rlo.prec == COLA_F32)
        ru_residual_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(d, rhi, b, ax, rlo, p, st, force, init, partials, counters);
    else
        ru_residual_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(d, rhi, b, ax, rlo, p, st, force, init, partials, counters);
    return cudaGetLastError();
}

cudaError_t launch_init_norms(const BlasDims &d, VecRef b, CgState *st, double *partials, unsigned *counters,
                              cudaStream_t s) {
    norm2_kernel<COLA_F64><<<blas_grid(d), kBlasBlock, 0, s>>>(d, b, nullptr, st, partials, counters);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const BlasDims &d, VecRef v, double *out, double *partials, unsigned *counters,
                         cudaStream_t s) {
    const dim3 g = blas_grid(d);
    if (v.prec == COLA_F64) norm2_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(d, v, out, nullptr, partials, counters);
    else if (v.prec == COLA_F32) norm2_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(d, v, out, nullptr, partials, counters);
    else norm2_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(d, v, out, nullptr, partials, counters);
    return cudaGetLastError();
}

template <int PD>
static void convert_from(const BlasDims &d, VecRef dst, VecRef src, cudaStream_t s) {
    const dim3 g = blas_grid(d);
    if (src.prec == COLA_F64) convert_kernel<PD, COLA_F64><<<g, kBlasBlock, 0, s>>>(d, dst, src);
    else if (src.prec == COLA_F32) convert_kernel<PD, COLA_F32><<<g, kBlasBlock, 0, s>>>(d, dst, src);
    else convert_kernel<PD, COLA_F16><<<g, kBlasBlock, 0, s>>>(d, dst, src);
}

cudaError_t launch_convert(const BlasDims &d, VecRef dst, VecRef src, cudaStream_t s) {
    if (dst.prec == COLA_F64) convert_from<COLA_F64>(d, dst, src, s);
    else if (dst.prec == COLA_F32) convert_from<COLA_F32>(d, dst, src, s);
    else convert_from<COLA_F16>(d, dst, src, s);
    return cudaGetLastError();
}

cudaError_t launch_axpby(const BlasDims &d, VecRef dst, double a, VecRef x, double b, VecRef y, cudaStream_t s) {
    if (dst.prec != x.prec || dst.prec != y.prec) return cudaErrorInvalidValue;
    const dim3 g = blas_grid(d);
    if (dst.prec == COLA_F64) axpby_kernel<COLA_F64><<<g, kBlasBlock, 0, s>>>(d, dst, a, x, b, y);
    else if (dst.prec == COLA_F32) axpby_kernel<COLA_F32><<<g, kBlasBlock, 0, s>>>(d, dst, a, x, b, y);
    else axpby_kernel<COLA_F16><<<g, kBlasBlock, 0, s>>>(d, dst, a, x, b, y);
    return cudaGetLastError();
}

}  // namespace cola
