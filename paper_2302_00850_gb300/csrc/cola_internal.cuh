// Internal device-side building blocks: lattice geometry, packed field
// accessors, complex arithmetic, SU(3) link reconstruction and block
// reductions.  Shared by every kernel translation unit of libcola.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/cola.h"

namespace cola {

// ----------------------------------------------------------- bounds checks --
// A debug build (-DCOLA_BOUNDS) checks every computed neighbour, link and site
// index against its extent before it is used.  An index out of range is
// counted, the source line of the first one is recorded, and the access is
// redirected to index 0 so that nothing faults; cola_debug_bounds() reports
// the count.  Each translation unit keeps its own counter (device variables
// have internal linkage without relocatable device code) and registers a
// reader with the library at load time.  Default builds compile the checks
// away: COLA_BOUND(i, n) is then the bare index.
#ifdef COLA_BOUNDS
static __device__ unsigned long long g_bounds_count;
static __device__ int g_bounds_line;

__device__ __forceinline__ int bound_check(long long i, long long n, int line) {
    if (i < 0 || i >= n) {
        if (atomicAdd(&g_bounds_count, 1ull) == 0ull) g_bounds_line = line;
        return 0;
    }
    return (int)i;
}
#define COLA_BOUND(i, n) ::cola::bound_check((long long)(i), (long long)(n), __LINE__)

using BoundsReader = cudaError_t (*)(unsigned long long *count, int *line, bool reset);
bool register_bounds_reader(BoundsReader r);

// this translation unit's counter and first line (reset: zero them after reading)
static cudaError_t bounds_read_local(unsigned long long *count, int *line, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(count, g_bounds_count, sizeof(*count));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(line, g_bounds_line, sizeof(*line));
    if (e == cudaSuccess && reset) {
        const unsigned long long zc = 0;
        const int zl = 0;
        e = cudaMemcpyToSymbol(g_bounds_count, &zc, sizeof(zc));
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds_line, &zl, sizeof(zl));
    }
    return e;
}
[[maybe_unused]] static const bool g_bounds_registered = register_bounds_reader(&bounds_read_local);
#else
#define COLA_BOUND(i, n) (i)
#endif

// ---------------------------------------------------------------- geometry --
// Division by a fixed divisor d through a multiply-high (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> l for 0 <= n < 2^31.
struct FastDiv {
    unsigned m, l;
    __host__ __device__ __forceinline__ int div(int n) const {
        return (int)((__umulhi_host_dev((unsigned)n, m) + (unsigned)n) >> l);
    }
    static __host__ __device__ __forceinline__ unsigned __umulhi_host_dev(unsigned a, unsigned b) {
#ifdef __CUDA_ARCH__
        return __umulhi(a, b);
#else
        return (unsigned)(((unsigned long long)a * b) >> 32);
#endif
    }
};

inline FastDiv make_fastdiv(int d) {
    FastDiv f{0u, 0u};
    if (d > 1) {
        unsigned l = 0;
        while ((1ull << l) < (unsigned long long)d) ++l;
        f.l = l;
        f.m = (unsigned)((((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d) + 1ull);
    }
    return f;
}

// Per-lattice constants passed by value to every kernel.
struct Geom {
    int L[4];        // Lx, Ly, Lz, Lt
    int Lxh;         // Lx / 2
    int Vh;          // sites of one parity
    int V;
    int stride[4];   // checkerboard-index offset of a +1 step in y, z, t (x unused)
    double bc[4][2]; // boundary phase per direction
    int bc_trivial[4];
    FastDiv div_xh, div_y, div_z;  // by Lxh, Ly, Lz
};

// Site coordinates of checkerboard index cb on parity `par`.
struct Coord {
    int x, y, z, t;
};

__device__ __forceinline__ Coord cb_coord(const Geom &g, int cb, int par) {
    Coord c;
    const int r1 = g.div_xh.div(cb);
    const int xh = cb - r1 * g.Lxh;
    const int r2 = g.div_y.div(r1);
    c.y = r1 - r2 * g.L[1];
    c.t = g.div_z.div(r2);
    c.z = r2 - c.t * g.L[2];
    c.x = 2 * xh + ((par + c.y + c.z + c.t) & 1);
    return c;
}

// Checkerboard index of the neighbour of site (c, cb) one step in direction mu
// (dir = +1 forward, -1 backward).  The neighbour has the opposite parity.
template <int MU, int DIR>
__device__ __forceinline__ int nbr_cb(const Geom &g, const Coord &c, int cb) {
    if constexpr (MU == 0) {
        int xn = c.x + DIR;
        if (DIR > 0 && xn == g.L[0]) xn = 0;
        if (DIR < 0 && xn < 0) xn = g.L[0] - 1;
        return COLA_BOUND(cb - (c.x >> 1) + (xn >> 1), g.Vh);
    } else {
        const int coord = (MU == 1) ? c.y : (MU == 2) ? c.z : c.t;
        const int L = g.L[MU];
        const int s = g.stride[MU];
        if (DIR > 0) return COLA_BOUND((coord == L - 1) ? cb - (L - 1) * s : cb + s, g.Vh);
        return COLA_BOUND((coord == 0) ? cb + (L - 1) * s : cb - s, g.Vh);
    }
}

template <int MU>
__device__ __forceinline__ int coord_of(const Coord &c) {
    return MU == 0 ? c.x : MU == 1 ? c.y : MU == 2 ? c.z : c.t;
}

// ----------------------------------------------------------------- complex --
template <typename R>
struct Cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ Cx<R> cmulc(Cx<R> a, Cx<R> b) {
    return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// acc += a * b
template <typename R>
__device__ __forceinline__ void cmac(Cx<R> &acc, Cx<R> a, Cx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc -= a * b
template <typename R>
__device__ __forceinline__ void cmsub(Cx<R> &acc, Cx<R> a, Cx<R> b) {
    acc.re = fma(-a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(-a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cmac_conj(Cx<R> &acc, Cx<R> a, Cx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------- precision traits --
template <int P>
struct Prec;
template <>
struct Prec<COLA_F64> {
    using real = double;
    static constexpr size_t site_bytes = 192;  // 24 doubles
    static constexpr int link_cplx_per_group = 1;
};
template <>
struct Prec<COLA_F32> {
    using real = float;
    static constexpr size_t site_bytes = 96;  // 24 floats
    static constexpr int link_cplx_per_group = 2;
};
template <>
struct Prec<COLA_F16> {
    using real = float;
    static constexpr size_t site_bytes = 52;  // 24 halves + FP32 scale
    static constexpr int link_cplx_per_group = 2;
};

__host__ __device__ constexpr size_t spinor_parity_bytes(int prec, int vh) {
    return (size_t)vh * (prec == COLA_F64 ? 192 : prec == COLA_F32 ? 96 : 52);
}

// Number of storage groups of one link (3x3 or its first two rows).
// FP16 links: 16-byte groups of four complexes, then one 8-byte group.
__host__ __device__ constexpr int link16_groups_f16(int recon) { return recon == 12 ? 1 : 2; }
// Bytes per site of one direction of the packed links (the layout is below).
__host__ __device__ constexpr size_t link_site_bytes(int prec, int recon) {
    return prec == COLA_F64 ? (recon == 12 ? 6 : 9) * 16
         : prec == COLA_F32 ? (recon == 12 ? 3 : 5) * 16
                            : link16_groups_f16(recon) * 16 + 8;
}
// Bytes of one direction of one parity of the packed links.
__host__ __device__ constexpr size_t link_dir_bytes(int prec, int recon, int vh) {
    return link_site_bytes(prec, recon) * vh;
}

// --------------------------------------------------------- spinor access --
// A parity field: pointer to the first byte of one parity of one RHS.
// Layout per precision (Vh sites, cb fastest):
//   F64: 12 arrays of double2 (complex c = 3*spin + colour)
//   F32:  6 arrays of float4  (complexes 2k, 2k+1)
//   F16:  3 arrays of uint4   (8 halves = complexes 4k..4k+3, scaled),
//         then Vh floats (per-site scale)
template <int P>
struct SpinorIO;

template <>
struct SpinorIO<COLA_F64> {
    // values without any site scale, and the scale (1 unless FP16)
    __device__ static __forceinline__ double load_raw(const void *base, int vh, int cb, Cx<double> (&s)[12]) {
        load(base, vh, cb, s);
        return 1.0;
    }
    __device__ static __forceinline__ void load(const void *base, int vh, int cb, Cx<double> (&s)[12]) {
        const double2 *p = reinterpret_cast<const double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 v = __ldg(p + (size_t)c * vh + cb);
            s[c] = {v.x, v.y};
        }
    }
    __device__ static __forceinline__ void store(void *base, int vh, int cb, const Cx<double> (&s)[12]) {
        double2 *p = reinterpret_cast<double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; ++c) p[(size_t)c * vh + cb] = make_double2(s[c].re, s[c].im);
    }
};

template <>
struct SpinorIO<COLA_F32> {
    __device__ static __forceinline__ float load_raw(const void *base, int vh, int cb, Cx<float> (&s)[12]) {
        load(base, vh, cb, s);
        return 1.0f;
    }
    __device__ static __forceinline__ void load(const void *base, int vh, int cb, Cx<float> (&s)[12]) {
        const float4 *p = reinterpret_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = __ldg(p + (size_t)k * vh + cb);
            s[2 * k] = {v.x, v.y};
            s[2 * k + 1] = {v.z, v.w};
        }
    }
    __device__ static __forceinline__ void store(void *base, int vh, int cb, const Cx<float> (&s)[12]) {
        float4 *p = reinterpret_cast<float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[(size_t)k * vh + cb] = make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
    }
};

__device__ __forceinline__ float2 h2f(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <>
struct SpinorIO<COLA_F16> {
    __device__ static __forceinline__ float load_raw(const void *base, int vh, int cb, Cx<float> (&s)[12]) {
        const uint4 *p = reinterpret_cast<const uint4 *>(base);
        const float sc = __ldg(reinterpret_cast<const float *>(p + (size_t)3 * vh) + cb);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(p + (size_t)k * vh + cb);
            float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            s[4 * k + 0] = {a.x, a.y};
            s[4 * k + 1] = {b.x, b.y};
            s[4 * k + 2] = {c.x, c.y};
            s[4 * k + 3] = {d.x, d.y};
        }
        return sc;
    }
    __device__ static __forceinline__ void load(const void *base, int vh, int cb, Cx<float> (&s)[12]) {
        const uint4 *p = reinterpret_cast<const uint4 *>(base);
        const float sc = __ldg(reinterpret_cast<const float *>(p + (size_t)3 * vh) + cb);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(p + (size_t)k * vh + cb);
            float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            s[4 * k + 0] = {a.x * sc, a.y * sc};
            s[4 * k + 1] = {b.x * sc, b.y * sc};
            s[4 * k + 2] = {c.x * sc, c.y * sc};
            s[4 * k + 3] = {d.x * sc, d.y * sc};
        }
    }
    __device__ static __forceinline__ void store(void *base, int vh, int cb, const Cx<float> (&s)[12]) {
        uint4 *p = reinterpret_cast<uint4 *>(base);
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(s[c].re), fabsf(s[c].im)));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v;
            v.x = f2h(s[4 * k + 0].re * inv, s[4 * k + 0].im * inv);
            v.y = f2h(s[4 * k + 1].re * inv, s[4 * k + 1].im * inv);
            v.z = f2h(s[4 * k + 2].re * inv, s[4 * k + 2].im * inv);
            v.w = f2h(s[4 * k + 3].re * inv, s[4 * k + 3].im * inv);
            p[(size_t)k * vh + cb] = v;
        }
        reinterpret_cast<float *>(p + (size_t)3 * vh)[cb] = m;
    }
};

// ----------------------------------------------------------- link access --
// One direction of one parity of the packed links: arrays of groups over Vh
// sites.  F64 groups are one complex (double2); F32 groups two complexes
// (float4).  F16 groups are four complexes (16 bytes: 8 halves), then one
// group of the last two complexes (8 bytes), so that a link is two 16-byte
// and 8-byte loads (recon 12: 16 + 8 bytes; recon 18: 16 + 16 + 8).
// Entries are row-major u00 u01 u02 u10 ...; with recon 18 the last group of
// F32/F16 is half padding.
template <int P, int RECON>
struct LinkIO;

template <typename R>
__device__ __forceinline__ void reconstruct_row2(Cx<R> (&u)[9]) {
    // row2 = conj(row0 x row1), exact for SU(3).  Each component is one
    // multiply-add chain: t = a b, then t -= c d continuing it (8 operations
    // instead of two products and a subtraction).
    Cx<R> t = cmul(u[1], u[5]);
    cmsub(t, u[2], u[4]);
    Cx<R> r6 = {t.re, -t.im};
    t = cmul(u[2], u[3]);
    cmsub(t, u[0], u[5]);
    Cx<R> r7 = {t.re, -t.im};
    t = cmul(u[0], u[4]);
    cmsub(t, u[1], u[3]);
    u[6] = r6;
    u[7] = r7;
    u[8] = {t.re, -t.im};
}

template <int RECON>
struct LinkIO<COLA_F64, RECON> {
    __device__ static __forceinline__ void load(const void *dir_base, int vh, int cb, Cx<double> (&u)[9]) {
        const double2 *p = reinterpret_cast<const double2 *>(dir_base);
        constexpr int n = RECON == 12 ? 6 : 9;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            double2 v = __ldg(p + (size_t)k * vh + cb);
            u[k] = {v.x, v.y};
        }
        if constexpr (RECON == 12) reconstruct_row2(u);
    }
};

template <int RECON>
struct LinkIO<COLA_F32, RECON> {
    __device__ static __forceinline__ void load(const void *dir_base, int vh, int cb, Cx<float> (&u)[9]) {
        const float4 *p = reinterpret_cast<const float4 *>(dir_base);
        if constexpr (RECON == 12) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float4 v = __ldg(p + (size_t)k * vh + cb);
                u[2 * k] = {v.x, v.y};
                u[2 * k + 1] = {v.z, v.w};
            }
            reconstruct_row2(u);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 v = __ldg(p + (size_t)k * vh + cb);
                u[2 * k] = {v.x, v.y};
                u[2 * k + 1] = {v.z, v.w};
            }
            float4 v = __ldg(p + (size_t)4 * vh + cb);
            u[8] = {v.x, v.y};
        }
    }
};

template <int RECON>
struct LinkIO<COLA_F16, RECON> {
    __device__ static __forceinline__ void load(const void *dir_base, int vh, int cb, Cx<float> (&u)[9]) {
        constexpr int n16 = link16_groups_f16(RECON);
        const uint4 *p = reinterpret_cast<const uint4 *>(dir_base);
        uint32_t w[4 * n16 + 2];
#pragma unroll
        for (int k = 0; k < n16; ++k) {
            const uint4 v = __ldg(p + (size_t)k * vh + cb);
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p + (size_t)n16 * vh) + cb);
        w[4 * n16] = v.x;
        w[4 * n16 + 1] = v.y;
        constexpr int ncplx = RECON == 12 ? 6 : 9;
#pragma unroll
        for (int k = 0; k < ncplx; ++k) {
            const float2 a = h2f(w[k]);
            u[k] = {a.x, a.y};
        }
        if constexpr (RECON == 12) reconstruct_row2(u);
    }
};

// ------------------------------------------- links by lattice coordinates --
// Gauge-field kernels (plaquettes, staples, clover leaves) visit links at
// arbitrary offsets from a site: these read one FP64 link of the packed
// field at coordinates p (each within one step of the lattice, wrapped
// periodically), and multiply 3x3 matrices in registers.
__device__ __forceinline__ int wrap_coord(int x, int l) { return x < 0 ? x + l : x >= l ? x - l : x; }

template <int RECON>
__device__ __forceinline__ void link_at(const Geom &g, const char *links, size_t link_dir_stride, const int (&p)[4],
                                        int mu, Cx<double> (&u)[9]) {
    const int x = wrap_coord(p[0], g.L[0]), y = wrap_coord(p[1], g.L[1]);
    const int z = wrap_coord(p[2], g.L[2]), t = wrap_coord(p[3], g.L[3]);
    const int par = (x + y + z + t) & 1;
    const int cb = COLA_BOUND((x >> 1) + g.Lxh * (y + g.L[1] * (z + g.L[2] * t)), g.Vh);
    LinkIO<COLA_F64, RECON>::load(links + (size_t)(4 * par + mu) * link_dir_stride, g.Vh, cb, u);
}

// w = op(u), op = identity or adjoint
__device__ __forceinline__ void mat3_set(Cx<double> (&w)[9], const Cx<double> (&u)[9], bool adj) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) w[3 * i + j] = adj ? Cx<double>{u[3 * j + i].re, -u[3 * j + i].im} : u[3 * i + j];
}

// w <- w op(u)
__device__ __forceinline__ void mat3_rmul(Cx<double> (&w)[9], const Cx<double> (&u)[9], bool adj) {
    Cx<double> r[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Cx<double> s = {0.0, 0.0};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (adj) cmac(s, w[3 * i + k], Cx<double>{u[3 * j + k].re, -u[3 * j + k].im});
                else cmac(s, w[3 * i + k], u[3 * k + j]);
            }
            r[3 * i + j] = s;
        }
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = r[k];
}

// f_a = Im Tr[lambda^a w] for the Gell-Mann matrices lambda^1..8
__device__ __forceinline__ void im_tr_lambda(const Cx<double> (&w)[9], double (&f)[8]) {
    f[0] = w[3].im + w[1].im;
    f[1] = w[1].re - w[3].re;
    f[2] = w[0].im - w[4].im;
    f[3] = w[6].im + w[2].im;
    f[4] = w[2].re - w[6].re;
    f[5] = w[7].im + w[5].im;
    f[6] = w[5].re - w[7].re;
    f[7] = (w[0].im + w[4].im - 2.0 * w[8].im) * 0.57735026918962576451;  // 1/sqrt(3)
}

// out[0..7] = coef f (accumulate: out += coef f); one link's eight
// generator coefficients of a force or momentum field [4][V][8]
__device__ __forceinline__ void store_force(double *out, const double (&f)[8], double coef, bool accumulate) {
#pragma unroll
    for (int a = 0; a < 8; ++a) out[a] = accumulate ? fma(coef, f[a], out[a]) : coef * f[a];
}

// ---------------------------------------------------------- clover access --
// The clover matrix A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_munu F_munu(x)
// (or its inverse) commutes with gamma5 = diag(1, 1, -1, -1), so it is two
// Hermitian 6x6 blocks per site: chirality 0 acts on spins 0, 1 and
// chirality 1 on spins 2, 3, with block row 3 (spin mod 2) + colour, i.e.
// components 6 chi .. 6 chi + 5 of a spinor.  A block is stored as 36 reals:
// the 6 (real) diagonal entries, then the 15 entries below the diagonal row
// by row, (1,0) (2,0) (2,1) (3,0) ... (5,4), each as (re, im).
// Layout: [parity][chirality][group][Vh]; a group holds 2 reals (F64,
// double2), 4 reals (F32, float4) or 4 halves (F16, uint2: no scale, the
// entries of A and of a well-conditioned A^-1 are O(1)).
constexpr int kCloverReals = 36;

__host__ __device__ constexpr size_t clover_block_bytes(int prec, int vh) {
    return (size_t)kCloverReals * (prec == COLA_F64 ? 8 : prec == COLA_F32 ? 4 : 2) * vh;
}
__host__ __device__ constexpr size_t clover_parity_bytes(int prec, int vh) { return 2 * clover_block_bytes(prec, vh); }

template <int P>
struct CloverIO;

template <>
struct CloverIO<COLA_F64> {
    __device__ static __forceinline__ void load(const void *blk, int vh, int cb, double (&m)[kCloverReals]) {
        const double2 *p = reinterpret_cast<const double2 *>(blk);
#pragma unroll
        for (int k = 0; k < kCloverReals / 2; ++k) {
            const double2 v = __ldg(p + (size_t)k * vh + cb);
            m[2 * k] = v.x;
            m[2 * k + 1] = v.y;
        }
    }
    __device__ static __forceinline__ void store(void *blk, int vh, int cb, const double (&m)[kCloverReals]) {
        double2 *p = reinterpret_cast<double2 *>(blk);
#pragma unroll
        for (int k = 0; k < kCloverReals / 2; ++k) p[(size_t)k * vh + cb] = make_double2(m[2 * k], m[2 * k + 1]);
    }
};

template <>
struct CloverIO<COLA_F32> {
    __device__ static __forceinline__ void load(const void *blk, int vh, int cb, float (&m)[kCloverReals]) {
        const float4 *p = reinterpret_cast<const float4 *>(blk);
#pragma unroll
        for (int k = 0; k < kCloverReals / 4; ++k) {
            const float4 v = __ldg(p + (size_t)k * vh + cb);
            m[4 * k] = v.x;
            m[4 * k + 1] = v.y;
            m[4 * k + 2] = v.z;
            m[4 * k + 3] = v.w;
        }
    }
    __device__ static __forceinline__ void store(void *blk, int vh, int cb, const double (&m)[kCloverReals]) {
        float4 *p = reinterpret_cast<float4 *>(blk);
#pragma unroll
        for (int k = 0; k < kCloverReals / 4; ++k)
            p[(size_t)k * vh + cb] = make_float4((float)m[4 * k], (float)m[4 * k + 1], (float)m[4 * k + 2],
                                                 (float)m[4 * k + 3]);
    }
};

template <>
struct CloverIO<COLA_F16> {
    __device__ static __forceinline__ void load(const void *blk, int vh, int cb, float (&m)[kCloverReals]) {
        const uint2 *p = reinterpret_cast<const uint2 *>(blk);
#pragma unroll
        for (int k = 0; k < kCloverReals / 4; ++k) {
            const uint2 v = __ldg(p + (size_t)k * vh + cb);
            const float2 a = h2f(v.x), b = h2f(v.y);
            m[4 * k] = a.x;
            m[4 * k + 1] = a.y;
            m[4 * k + 2] = b.x;
            m[4 * k + 3] = b.y;
        }
    }
    __device__ static __forceinline__ void store(void *blk, int vh, int cb, const double (&m)[kCloverReals]) {
        uint2 *p = reinterpret_cast<uint2 *>(blk);
#pragma unroll
        for (int k = 0; k < kCloverReals / 4; ++k) {
            uint2 v;
            v.x = f2h((float)m[4 * k], (float)m[4 * k + 1]);
            v.y = f2h((float)m[4 * k + 2], (float)m[4 * k + 3]);
            p[(size_t)k * vh + cb] = v;
        }
    }
};

// o = M v for one Hermitian block in the packed form above.
template <typename R>
__device__ __forceinline__ void herm6_mul(const R (&m)[kCloverReals], const Cx<R> *v, Cx<R> (&o)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) o[i] = {m[i] * v[i].re, m[i] * v[i].im};
    int k = 6;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            const Cx<R> l = {m[k], m[k + 1]};
            k += 2;
            cmac(o[i], l, v[j]);       // below the diagonal: M_ij = l
            cmac_conj(o[j], l, v[i]);  // above it: M_ji = conj(l)
        }
}

// v <- C v for the clover field C (A or A^-1) of one parity at site cb, v in
// the packed spin basis (v' = S v, S = (gamma_t + gamma5) / sqrt(2)).  The
// chirality blocks act on the canonical spins 0, 1 and 2, 3, i.e. on
// (v'_u + v'_d) / sqrt(2) and (v'_u - v'_d) / sqrt(2); the two factors
// 1 / sqrt(2) of the rotations in and out combine to one 1 / 2.
template <int P>
__device__ __forceinline__ void clover_mul(const char *parity_base, int vh, int cb,
                                           Cx<typename Prec<P>::real> (&v)[12]) {
    using R = typename Prec<P>::real;
    Cx<R> w[12];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        w[k] = {v[k].re + v[6 + k].re, v[k].im + v[6 + k].im};
        w[6 + k] = {v[k].re - v[6 + k].re, v[k].im - v[6 + k].im};
    }
    Cx<R> o[2][6];
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        R m[kCloverReals];
        CloverIO<P>::load(parity_base + chi * clover_block_bytes(P, vh), vh, cb, m);
        herm6_mul(m, w + 6 * chi, o[chi]);
    }
    const R h = R(0.5);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        v[k] = {h * (o[0][k].re + o[1][k].re), h * (o[0][k].im + o[1][k].im)};
        v[6 + k] = {h * (o[0][k].re - o[1][k].re), h * (o[0][k].im - o[1][k].im)};
    }
}

}  // namespace cola

namespace cola {

// ------------------------------------------------------ solver state (device) --
// One per right-hand side; all CG scalars live on the device so that the
// iteration needs no host round trip.
struct CgState {
    double rho;      // <r, r> of the residual the current alpha uses
    double rho_new;  // <r, r> after the latest update
    double pq;       // <p, A p> = |M p|^2
    double alpha;
    double r2_last;  // |r_hi|^2 at the last reliable update (FP64 true residual)
    double b2;       // |b|^2
    double tol2;     // tol^2 |b|^2
    double delta2;   // delta^2
    double shift;    // sigma: this row solves (A + sigma) x = b
    double r2_best;  // smallest FP64 true |r|^2 so far (0: none yet)
    double rho_mark; // iterated |r|^2 at the last 4x drop (or the last reliable update)
    int it_mark;     // iteration of rho_mark
    int stall;       // reliable updates since r2_best last improved
    int iter;
    int max_iter;
    int ru;          // a reliable update is due
    int ru_count;
    int done;
    int status;
};

// Deterministic grid reductions (no floating-point atomics, no fences):
// every block of a reducing vector kernel writes one partial per row with a
// plain store, and a one-block-per-row finishing kernel sums those partials
// in block order and applies the solver's decision.  The kernel boundary
// orders the partial stores before the finisher reads them.

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a one-dimensional block in a fixed order; valid in thread 0.
// `sh` holds at least blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_allsum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) t += sh[w];
    return t;
}

}  // namespace cola
