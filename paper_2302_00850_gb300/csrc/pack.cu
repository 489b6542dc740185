// Canonical <-> checkerboard structure-of-arrays packing of spinors and links.
//
// Canonical fields are complex128 with site index i = x + Lx(y + Ly(z + Lz t));
// the packed fields split sites by parity (x+y+z+t) mod 2 and store, for each
// parity, one array per storage group over the Vh = V/2 sites of that parity
// (checkerboard index cb = i / 2), so that a warp reading one group for 32
// consecutive sites issues one coalesced transaction.
//
// Packed spinors hold psi' = S psi, S = (gamma_t + gamma5) / sqrt(2), a
// unitary and Hermitian spin rotation (S S = 1): with u = spins 0, 1 and
// d = spins 2, 3 of the canonical chiral basis, u' = (u + d) / sqrt(2) and
// d' = (u - d) / sqrt(2).  In that basis gamma_t is diag(1, 1, -1, -1), so
// the time hops of the hopping term project by selecting two spins, and
// gamma_x, gamma_y, gamma_z are minus their canonical forms.
#include "cola_impl.h"

namespace cola {

// s <- S s on one site (canonical <-> packed spin basis; S is its own inverse)
__device__ __forceinline__ void spin_rotate(Cx<double> (&s)[12]) {
    constexpr double r = 0.70710678118654752440;  // 1 / sqrt(2)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const Cx<double> u = s[k], d = s[6 + k];
        s[k] = {(u.re + d.re) * r, (u.im + d.im) * r};
        s[6 + k] = {(u.re - d.re) * r, (u.im - d.im) * r};
    }
}

__device__ __forceinline__ void site_parity_cb(const Geom &g, int i, int &par, int &cb) {
    int x = i % g.L[0];
    int r = i / g.L[0];
    int y = r % g.L[1];
    r /= g.L[1];
    int z = r % g.L[2];
    int t = r / g.L[2];
    par = (x + y + z + t) & 1;
    cb = COLA_BOUND(i >> 1, g.Vh);
}

template <int P>
__global__ void pack_spinor_kernel(const Geom g, void *packed, const double2 *canon, int nrhs, int pmask) {
    using R = typename Prec<P>::real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.V || rhs >= nrhs) return;
    int par, cb;
    site_parity_cb(g, i, par, cb);
    if (!((pmask >> par) & 1)) return;
    const double2 *src = canon + ((size_t)rhs * g.V + i) * 12;
    Cx<double> sd[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) sd[c] = {src[c].x, src[c].y};
    spin_rotate(sd);
    Cx<R> s[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) s[c] = {(R)sd[c].re, (R)sd[c].im};
    const size_t pbytes = spinor_parity_bytes(P, g.Vh);
    char *dst = static_cast<char *>(packed) + (size_t)rhs * 2 * pbytes + par * pbytes;
    SpinorIO<P>::store(dst, g.Vh, cb, s);
}

// The F16 loader returns float; the F64 path needs double output.  A plain
// loader per precision is kept here so that unpacking reads exactly what a
// kernel would read.
template <int P>
__global__ void unpack_spinor_kernel(const Geom g, double2 *canon, const void *packed, int nrhs, int pmask) {
    using R = typename Prec<P>::real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.V || rhs >= nrhs) return;
    int par, cb;
    site_parity_cb(g, i, par, cb);
    if (!((pmask >> par) & 1)) return;
    const size_t pbytes = spinor_parity_bytes(P, g.Vh);
    const char *src = static_cast<const char *>(packed) + (size_t)rhs * 2 * pbytes + par * pbytes;
    Cx<R> s[12];
    SpinorIO<P>::load(src, g.Vh, cb, s);
    Cx<double> sd[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) sd[c] = {(double)s[c].re, (double)s[c].im};
    spin_rotate(sd);
    double2 *dst = canon + ((size_t)rhs * g.V + i) * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) dst[c] = make_double2(sd[c].re, sd[c].im);
}

template <int P, int RECON>
__global__ void pack_gauge_kernel(const Geom g, void *packed, const double2 *canon) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int mu = blockIdx.y;
    if (i >= g.V) return;
    int par, cb;
    site_parity_cb(g, i, par, cb);
    const double2 *u = canon + ((size_t)mu * g.V + i) * 9;
    const size_t dir_bytes = link_dir_bytes(P, RECON, g.Vh);
    char *base = static_cast<char *>(packed) + (size_t)par * 4 * dir_bytes + (size_t)mu * dir_bytes;
    constexpr int ncplx = RECON == 12 ? 6 : 9;
    if constexpr (P == COLA_F64) {
        double2 *d = reinterpret_cast<double2 *>(base);
        for (int k = 0; k < ncplx; ++k) d[(size_t)k * g.Vh + cb] = u[k];
    } else if constexpr (P == COLA_F32) {
        float4 *d = reinterpret_cast<float4 *>(base);
        constexpr int ng = RECON == 12 ? 3 : 5;
        for (int k = 0; k < ng; ++k) {
            double2 a = u[2 * k];
            double2 b = (2 * k + 1 < ncplx) ? u[2 * k + 1] : make_double2(0.0, 0.0);
            d[(size_t)k * g.Vh + cb] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        }
    } else {  // 16-byte groups of four complexes, then the last two complexes (8 bytes)
        constexpr int n16 = link16_groups_f16(RECON);
        uint32_t w[4 * n16 + 2];
        for (int k = 0; k < 4 * n16 + 2; ++k) {
            const double2 a = k < ncplx ? u[k] : make_double2(0.0, 0.0);
            w[k] = f2h((float)a.x, (float)a.y);
        }
        uint4 *d = reinterpret_cast<uint4 *>(base);
        for (int k = 0; k < n16; ++k) d[(size_t)k * g.Vh + cb] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        reinterpret_cast<uint2 *>(d + (size_t)n16 * g.Vh)[cb] = make_uint2(w[4 * n16], w[4 * n16 + 1]);
    }
}

cudaError_t launch_pack_gauge(int prec, int recon, const Geom &g, void *packed, const void *canon,
                              cudaStream_t s) {
    dim3 block(128), grid((g.V + 127) / 128, 4);
    const double2 *c = static_cast<const double2 *>(canon);
    if (prec == COLA_F64) {
        if (recon == 12) pack_gauge_kernel<COLA_F64, 12><<<grid, block, 0, s>>>(g, packed, c);
        else pack_gauge_kernel<COLA_F64, 18><<<grid, block, 0, s>>>(g, packed, c);
    } else if (prec == COLA_F32) {
        if (recon == 12) pack_gauge_kernel<COLA_F32, 12><<<grid, block, 0, s>>>(g, packed, c);
        else pack_gauge_kernel<COLA_F32, 18><<<grid, block, 0, s>>>(g, packed, c);
    } else {
        if (recon == 12) pack_gauge_kernel<COLA_F16, 12><<<grid, block, 0, s>>>(g, packed, c);
        else pack_gauge_kernel<COLA_F16, 18><<<grid, block, 0, s>>>(g, packed, c);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_spinor(int prec, const Geom &g, void *packed, const void *canon, int nrhs,
                               int parity_mask, cudaStream_t s) {
    dim3 block(128), grid((g.V + 127) / 128, nrhs);
    const double2 *c = static_cast<const double2 *>(canon);
    if (prec == COLA_F64) pack_spinor_kernel<COLA_F64><<<grid, block, 0, s>>>(g, packed, c, nrhs, parity_mask);
    else if (prec == COLA_F32) pack_spinor_kernel<COLA_F32><<<grid, block, 0, s>>>(g, packed, c, nrhs, parity_mask);
    else pack_spinor_kernel<COLA_F16><<<grid, block, 0, s>>>(g, packed, c, nrhs, parity_mask);
    return cudaGetLastError();
}

cudaError_t launch_unpack_spinor(int prec, const Geom &g, void *canon, const void *packed, int nrhs,
                                 int parity_mask, cudaStream_t s) {
    dim3 block(128), grid((g.V + 127) / 128, nrhs);
    double2 *c = static_cast<double2 *>(canon);
    if (prec == COLA_F64) unpack_spinor_kernel<COLA_F64><<<grid, block, 0, s>>>(g, c, packed, nrhs, parity_mask);
    else if (prec == COLA_F32) unpack_spinor_kernel<COLA_F32><<<grid, block, 0, s>>>(g, c, packed, nrhs, parity_mask);
    else unpack_spinor_kernel<COLA_F16><<<grid, block, 0, s>>>(g, c, packed, nrhs, parity_mask);
    return cudaGetLastError();
}

}  // namespace cola
