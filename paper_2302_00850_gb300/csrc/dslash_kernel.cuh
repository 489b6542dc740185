// Hopping-term kernel templates (the fermion-matrix kernel), included by the
// translation units that instantiate them: dslash.cu (plain and xpay
// epilogues, launch shapes, autotuning) and dslash_clover.cu (clover
// epilogues).
//
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
// reconstruction).  Packed spinors are in the rotated spin basis of the
// packing (psi' = S psi, S = (gamma_t + gamma5) / sqrt(2)), where
// gamma_x, gamma_y, gamma_z are minus their DeGrand-Rossi forms and
// gamma_t = diag(1, 1, -1, -1): a time hop's projector 1 +- gamma_t is twice
// the projection on spins 0, 1 or on spins 2, 3, with nothing to add and
// half the rows to accumulate.
#pragma once

#include <type_traits>

#include "cola_impl.h"

#ifndef COLA_DSLASH_MINB
#define COLA_DSLASH_MINB 2
#endif

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

// Two-spinor h = rows 0, 1 of (1 + S gamma_mu) psi, gamma_mu in the
// DeGrand-Rossi (canonical) basis.
template <int MU, int S, typename R>
__device__ __forceinline__ void project_chiral(const Cx<R> (&psi)[12], Cx<R> (&h)[2][3]) {
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

// Two-spinor h of (1 + S gamma_mu) psi in the packed basis: for the space
// directions the canonical projection with -S; for time the spins the
// projector keeps (0, 1 for S = +1, 2, 3 for S = -1), the factor 2 being
// applied at accumulation.
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const Cx<R> (&psi)[12], Cx<R> (&h)[2][3]) {
    if constexpr (MU < 3) {
        project_chiral<MU, -S>(psi, h);
    } else {
        constexpr int off = S > 0 ? 0 : 6;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h[0][a] = psi[off + a];
            h[1][a] = psi[off + 3 + a];
        }
    }
}

template <typename R>
__device__ __forceinline__ Cx<R> times_i(Cx<R> a, int s) {  // s*i*a
    return s > 0 ? Cx<R>{-a.im, a.re} : Cx<R>{a.im, -a.re};
}

// acc += sc * (full spinor rebuilt from w = U h); rows 2, 3 follow from rows 0, 1
// (canonical basis).  sc carries the neighbour's FP16 site scale and a real
// boundary phase, so both cost nothing beyond the fused multiply-adds of
// the accumulation.
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate_chiral(Cx<R> (&acc)[12], const Cx<R> (&w)[2][3], R sc) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a].re = fma(sc, w[0][a].re, acc[a].re);
        acc[a].im = fma(sc, w[0][a].im, acc[a].im);
        acc[3 + a].re = fma(sc, w[1][a].re, acc[3 + a].re);
        acc[3 + a].im = fma(sc, w[1][a].im, acc[3 + a].im);
        if constexpr (MU == 0) {         // r2 = -S i w1, r3 = -S i w0;  i(x + iy) = -y + ix
            acc[6 + a].re = fma(S * sc, w[1][a].im, acc[6 + a].re);
            acc[6 + a].im = fma(-S * sc, w[1][a].re, acc[6 + a].im);
            acc[9 + a].re = fma(S * sc, w[0][a].im, acc[9 + a].re);
            acc[9 + a].im = fma(-S * sc, w[0][a].re, acc[9 + a].im);
        } else if constexpr (MU == 1) {  // r2 = S w1, r3 = -S w0
            acc[6 + a].re = fma(S * sc, w[1][a].re, acc[6 + a].re);
            acc[6 + a].im = fma(S * sc, w[1][a].im, acc[6 + a].im);
            acc[9 + a].re = fma(-S * sc, w[0][a].re, acc[9 + a].re);
            acc[9 + a].im = fma(-S * sc, w[0][a].im, acc[9 + a].im);
        } else if constexpr (MU == 2) {  // r2 = -S i w0, r3 = S i w1
            acc[6 + a].re = fma(S * sc, w[0][a].im, acc[6 + a].re);
            acc[6 + a].im = fma(-S * sc, w[0][a].re, acc[6 + a].im);
            acc[9 + a].re = fma(-S * sc, w[1][a].im, acc[9 + a].re);
            acc[9 + a].im = fma(S * sc, w[1][a].re, acc[9 + a].im);
        } else {                         // r2 = S w0, r3 = S w1
            acc[6 + a].re = fma(S * sc, w[0][a].re, acc[6 + a].re);
            acc[6 + a].im = fma(S * sc, w[0][a].im, acc[6 + a].im);
            acc[9 + a].re = fma(S * sc, w[1][a].re, acc[9 + a].re);
            acc[9 + a].im = fma(S * sc, w[1][a].im, acc[9 + a].im);
        }
    }
}

// The same in the packed basis: for time, 2 sc w goes to the two spins the
// projector keeps and nothing to the others.
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate(Cx<R> (&acc)[12], const Cx<R> (&w)[2][3], R sc) {
    if constexpr (MU < 3) {
        accumulate_chiral<MU, -S>(acc, w, sc);
    } else {
        constexpr int off = S > 0 ? 0 : 6;
        const R s2 = R(2) * sc;
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[off + 3 * k + a].re = fma(s2, w[k][a].re, acc[off + 3 * k + a].re);
                acc[off + 3 * k + a].im = fma(s2, w[k][a].im, acc[off + 3 * k + a].im);
            }
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

// Scale of a hop crossing the boundary: a real phase folds into sc, a
// complex one multiplies w.
template <typename R>
__device__ __forceinline__ void boundary_phase(const Geom &g, int mu, bool conj_phase, Cx<R> (&w)[2][3], R &sc) {
    const R pr = (R)g.bc[mu][0];
    const R pi = conj_phase ? -(R)g.bc[mu][1] : (R)g.bc[mu][1];
    if (pi == R(0)) sc *= pr;
    else phase_mul(w, pr, pi);
}

// Rows 0 and 1 of acc += sc * c (no reconstruction: c is a sum of hops).
template <typename R>
__device__ __forceinline__ void accumulate01(Cx<R> (&acc)[12], const Cx<R> (&c)[2][3], R sc) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a].re = fma(sc, c[0][a].re, acc[a].re);
        acc[a].im = fma(sc, c[0][a].im, acc[a].im);
        acc[3 + a].re = fma(sc, c[1][a].re, acc[3 + a].re);
        acc[3 + a].im = fma(sc, c[1][a].im, acc[3 + a].im);
    }
}

// Rows 2 and 3 of the reconstruction of d with projector sign S, times sc
// (canonical basis; the space directions of the packed basis use -S).
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate23(Cx<R> (&acc)[12], const Cx<R> (&d)[2][3], R sc) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if constexpr (MU == 0) {
            acc[6 + a].re = fma(S * sc, d[1][a].im, acc[6 + a].re);
            acc[6 + a].im = fma(-S * sc, d[1][a].re, acc[6 + a].im);
            acc[9 + a].re = fma(S * sc, d[0][a].im, acc[9 + a].re);
            acc[9 + a].im = fma(-S * sc, d[0][a].re, acc[9 + a].im);
        } else if constexpr (MU == 1) {
            acc[6 + a].re = fma(S * sc, d[1][a].re, acc[6 + a].re);
            acc[6 + a].im = fma(S * sc, d[1][a].im, acc[6 + a].im);
            acc[9 + a].re = fma(-S * sc, d[0][a].re, acc[9 + a].re);
            acc[9 + a].im = fma(-S * sc, d[0][a].im, acc[9 + a].im);
        } else if constexpr (MU == 2) {
            acc[6 + a].re = fma(S * sc, d[0][a].im, acc[6 + a].re);
            acc[6 + a].im = fma(-S * sc, d[0][a].re, acc[6 + a].im);
            acc[9 + a].re = fma(-S * sc, d[1][a].im, acc[9 + a].re);
            acc[9 + a].im = fma(S * sc, d[1][a].re, acc[9 + a].im);
        } else {
            acc[6 + a].re = fma(S * sc, d[0][a].re, acc[6 + a].re);
            acc[6 + a].im = fma(S * sc, d[0][a].im, acc[6 + a].im);
            acc[9 + a].re = fma(S * sc, d[1][a].re, acc[9 + a].re);
            acc[9 + a].im = fma(S * sc, d[1][a].im, acc[9 + a].im);
        }
    }
}

// c += U^dag h (continues the multiply-add chains that produced c).
template <typename R>
__device__ __forceinline__ void su3_adj_mul_add(const Cx<R> (&u)[9], const Cx<R> (&h)[2][3], Cx<R> (&c)[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cmac_conj(c[k][a], u[a], h[k][0]);
            cmac_conj(c[k][a], u[3 + a], h[k][1]);
            cmac_conj(c[k][a], u[6 + a], h[k][2]);
        }
}

// Both hops of direction mu, results scaled by bs (the output factor b).
// The forward and backward reconstructions differ only in the sign of their
// lower two rows, so away from the boundary both hops enter as
//   rows 0,1 += bs (w_f + w_b),   rows 2,3 += bs C_f (w_f - w_b),
// with c = w_f + w_b built by continuing w_f's multiply-add chains and
// w_f - w_b = 2 w_f - c: twelve multiply-adds fewer than two full
// reconstructions.  Hops that cross the boundary (phase) or carry an FP16
// site scale take the general form.
template <int P, int MU, bool DAGGER>
__device__ __forceinline__ void hop_pair_apply(const Geom &g, const Cx<typename Prec<P>::real> (&uf)[9],
                                               const Cx<typename Prec<P>::real> (&ub)[9],
                                               const Cx<typename Prec<P>::real> (&hf)[2][3],
                                               const Cx<typename Prec<P>::real> (&hb)[2][3],
                                               typename Prec<P>::real scf, typename Prec<P>::real scb, bool edge_f,
                                               bool edge_b, Cx<typename Prec<P>::real> (&acc)[12],
                                               typename Prec<P>::real bs);

template <int P, int RECON, int MU, bool DAGGER>
__device__ __forceinline__ void hop_mu(const DslashLat &A, const Coord &c, int cb, const char *in,
                                       const char *links_out, const char *links_in,
                                       Cx<typename Prec<P>::real> (&acc)[12], typename Prec<P>::real bs) {
    using R = typename Prec<P>::real;
    const Geom &g = A.g;
    constexpr int SF = DAGGER ? +1 : -1;  // forward projector 1 + SF gamma
    constexpr int SB = -SF;
    const int nbf = nbr_cb<MU, +1>(g, c, cb);
    const int nbb = nbr_cb<MU, -1>(g, c, cb);
    Cx<R> hf[2][3], hb[2][3], uf[9], ub[9];
    R scf, scb;
    {
        Cx<R> psi[12];
        scf = SpinorIO<P>::load_raw(in, g.Vh, nbf, psi);
        project<MU, SF>(psi, hf);
    }
    LinkIO<P, RECON>::load(links_out + MU * A.link_dir_stride, g.Vh, cb, uf);
    {
        Cx<R> psi[12];
        scb = SpinorIO<P>::load_raw(in, g.Vh, nbb, psi);
        project<MU, SB>(psi, hb);
    }
    LinkIO<P, RECON>::load(links_in + MU * A.link_dir_stride, g.Vh, nbb, ub);
    const bool edge_f = !g.bc_trivial[MU] && coord_of<MU>(c) == g.L[MU] - 1;
    const bool edge_b = !g.bc_trivial[MU] && coord_of<MU>(c) == 0;
    hop_pair_apply<P, MU, DAGGER>(g, uf, ub, hf, hb, scf, scb, edge_f, edge_b, acc, bs);
}

// Both hops of direction mu for NR right-hand sides of one site: each link is
// loaded (and its third row rebuilt) once and applied to every right-hand
// side, so link traffic and link arithmetic are shared by NR outputs.
// in0 addresses right-hand side 0 of this thread; live[k] masks finished or
// absent right-hand sides.
template <int P, int RECON, int MU, bool DAGGER, int NR>
__device__ __forceinline__ void hop_mu_mrhs(const DslashLat &A, const Coord &c, int cb, const char *in0,
                                            const char *links_out, const char *links_in,
                                            Cx<typename Prec<P>::real> (&acc)[NR][12], typename Prec<P>::real bs,
                                            const bool (&live)[NR]) {
    using R = typename Prec<P>::real;
    const Geom &g = A.g;
    constexpr int SF = DAGGER ? +1 : -1;
    constexpr int SB = -SF;
    const int nbf = nbr_cb<MU, +1>(g, c, cb);
    const int nbb = nbr_cb<MU, -1>(g, c, cb);
    Cx<R> uf[9], ub[9];
    LinkIO<P, RECON>::load(links_out + MU * A.link_dir_stride, g.Vh, cb, uf);
    LinkIO<P, RECON>::load(links_in + MU * A.link_dir_stride, g.Vh, nbb, ub);
    const bool edge_f = !g.bc_trivial[MU] && coord_of<MU>(c) == g.L[MU] - 1;
    const bool edge_b = !g.bc_trivial[MU] && coord_of<MU>(c) == 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (!live[k]) continue;
        const char *in = in0 + (size_t)k * A.rhs_stride;
        Cx<R> hf[2][3], hb[2][3];
        R scf, scb;
        {
            Cx<R> psi[12];
            scf = SpinorIO<P>::load_raw(in, g.Vh, nbf, psi);
            project<MU, SF>(psi, hf);
        }
        {
            Cx<R> psi[12];
            scb = SpinorIO<P>::load_raw(in, g.Vh, nbb, psi);
            project<MU, SB>(psi, hb);
        }
        hop_pair_apply<P, MU, DAGGER>(g, uf, ub, hf, hb, scf, scb, edge_f, edge_b, acc[k], bs);
    }
}

// The forward hop (link uf, projected neighbour hf with site scale scf) and
// the backward hop (ub, hb, scb) of direction mu, accumulated into acc with
// the output factor bs.
template <int P, int MU, bool DAGGER>
__device__ __forceinline__ void hop_pair_apply(const Geom &g, const Cx<typename Prec<P>::real> (&uf)[9],
                                               const Cx<typename Prec<P>::real> (&ub)[9],
                                               const Cx<typename Prec<P>::real> (&hf)[2][3],
                                               const Cx<typename Prec<P>::real> (&hb)[2][3],
                                               typename Prec<P>::real scf, typename Prec<P>::real scb, bool edge_f,
                                               bool edge_b, Cx<typename Prec<P>::real> (&acc)[12],
                                               typename Prec<P>::real bs) {
    using R = typename Prec<P>::real;
    constexpr int SF = DAGGER ? +1 : -1;
    constexpr int SB = -SF;
    Cx<R> wf[2][3];
    su3_mul(uf, hf, wf);
    // time hops each fill half the rows, so the pairing below only pays for space
    if (MU < 3 && P != COLA_F16 && !edge_f && !edge_b) {
        Cx<R> cs[2][3];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) cs[k][a] = wf[k][a];
        su3_adj_mul_add(ub, hb, cs);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                wf[k][a].re = fma(R(2), wf[k][a].re, -cs[k][a].re);
                wf[k][a].im = fma(R(2), wf[k][a].im, -cs[k][a].im);
            }
        accumulate01(acc, cs, bs);
        accumulate23<MU, -SF>(acc, wf, bs);  // packed basis: gamma_mu' = -gamma_mu for space
    } else {
        R sf = scf * bs, sb = scb * bs;
        if (edge_f) boundary_phase(g, MU, false, wf, sf);
        accumulate<MU, SF>(acc, wf, sf);
        Cx<R> wb[2][3];
        su3_adj_mul(ub, hb, wb);
        if (edge_b) boundary_phase(g, MU, true, wb, sb);
        accumulate<MU, SB>(acc, wb, sb);
    }
}

// ------------------------------------------------------------------ staged --
// The FP16/FP32 kernels are limited by how many bytes each SM keeps in
// flight, not by arithmetic: a thread that loads one hop at a time leaves
// HBM idle.  The staged variant has each thread copy the raw bytes of its
// next NSTAGE-1 hops (neighbour spinor, its FP16 scale, the link) into its
// own shared-memory slots with asynchronous copies (cp.async), then computes
// hop j from shared memory while hops j+1.. are in flight.  Copies do not
// occupy registers, so the pipeline depth is not bounded by the register
// file.  Each thread reads only what it copied itself, so completion needs
// cp.async.wait_group only, no block barrier.  Shared layout per stage:
// [chunk][thread] so that a warp's 16-byte reads are conflict-free.

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// The same without allocating in L1 (.cg), for the neighbour spinors: L2
// serves their reuse, and the copies ran faster at 32^3x64 than through L1
__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Raw bytes of one hop: spinor chunks of 16 B (+ one 4-byte FP16 scale) and
// link chunks of 16 B (FP32: two complexes each; FP16: four) plus, for
// FP16, one 8-byte chunk of the last two complexes.
template <int P, int RECON>
struct HopLayout {
    static constexpr int spin16 = P == COLA_F32 ? 6 : 3;
    static constexpr int scale4 = P == COLA_F16 ? 1 : 0;
    static constexpr int link16 = P == COLA_F32 ? (RECON == 12 ? 3 : 5) : link16_groups_f16(RECON);
    static constexpr int link8 = P == COLA_F16 ? 1 : 0;
    static constexpr int bytes = spin16 * 16 + scale4 * 4 + link16 * 16 + link8 * 8;
};

// The staged kernel always runs kStagedThreads threads per block (sites x
// right-hand sides), so every shared-memory offset is a compile-time constant
// plus one per-thread term.
constexpr int kStagedThreads = 128;

template <int P, int RECON>
struct Stage {
    using L = HopLayout<P, RECON>;
    static constexpr int T = kStagedThreads;
    char *base;  // this stage's area
    __device__ uint4 *spin(int k, int tid) const { return reinterpret_cast<uint4 *>(base) + k * T + tid; }
    __device__ float *scale(int tid) const {
        return reinterpret_cast<float *>(base + L::spin16 * 16 * T) + tid;
    }
    __device__ uint4 *link16(int k, int tid) const {
        return reinterpret_cast<uint4 *>(base + (L::spin16 * 16 + L::scale4 * 4) * T) + k * T + tid;
    }
    __device__ uint2 *link8(int tid) const {
        return reinterpret_cast<uint2 *>(base + (L::spin16 * 16 + L::scale4 * 4 + L::link16 * 16) * T) + tid;
    }
};

// hop j = 2*mu + (0 forward, 1 backward)
template <int J>
struct Hop {
    static constexpr int MU = J / 2;
    static constexpr int DIR = (J % 2 == 0) ? +1 : -1;
};

template <int P, int RECON, int J>
__device__ __forceinline__ void stage_issue(const DslashLat &A, const Coord &c, int cb, const char *in,
                                            const char *links_out, const char *links_in, const Stage<P, RECON> &st,
                                            int tid) {
    using L = HopLayout<P, RECON>;
    constexpr int MU = Hop<J>::MU, DIR = Hop<J>::DIR;
    const Geom &g = A.g;
    const int nb = nbr_cb<MU, DIR>(g, c, cb);
#pragma unroll
    for (int k = 0; k < L::spin16; ++k) cp_async16_cg(st.spin(k, tid), in + ((size_t)k * g.Vh + nb) * 16);
    if constexpr (L::scale4) cp_async4(st.scale(tid), in + (size_t)L::spin16 * 16 * g.Vh + (size_t)nb * 4);
    const char *lb = (DIR > 0 ? links_out : links_in) + MU * A.link_dir_stride;
    const int lcb = DIR > 0 ? cb : nb;
#pragma unroll
    for (int k = 0; k < L::link16; ++k) cp_async16(st.link16(k, tid), lb + ((size_t)k * g.Vh + lcb) * 16);
    if constexpr (L::link8) cp_async8(st.link8(tid), lb + (size_t)L::link16 * 16 * g.Vh + (size_t)lcb * 8);
}

// FP16 spin projection straight from storage.  PTX for sm_100 and later
// adds one FP16 operand to one FP32 operand with an FP32 result
// (add/sub.rn.f32.f16); the FP16 value enters exactly, so a + b is rounded
// once, exactly as converting a first and adding in FP32 would do, and one
// conversion per component is saved.  A stored complex is a half2 word
// (real part in the low half).
__device__ __forceinline__ float hadd_lo(uint32_t a, float b) {
    float r;
    asm("{.reg .b16 l, h;\n mov.b32 {l, h}, %1;\n add.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float hadd_hi(uint32_t a, float b) {
    float r;
    asm("{.reg .b16 l, h;\n mov.b32 {l, h}, %1;\n add.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float hsub_lo(uint32_t a, float b) {
    float r;
    asm("{.reg .b16 l, h;\n mov.b32 {l, h}, %1;\n sub.rn.f32.f16 %0, l, %2;}" : "=f"(r) : "r"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float hsub_hi(uint32_t a, float b) {
    float r;
    asm("{.reg .b16 l, h;\n mov.b32 {l, h}, %1;\n sub.rn.f32.f16 %0, h, %2;}" : "=f"(r) : "r"(a), "f"(b));
    return r;
}
// a + s b and a + s i b for a stored half2 complex a and an FP32 complex b
template <int S>
__device__ __forceinline__ Cx<float> hadd_s(uint32_t a, Cx<float> b) {
    if constexpr (S > 0) return {hadd_lo(a, b.re), hadd_hi(a, b.im)};
    else return {hsub_lo(a, b.re), hsub_hi(a, b.im)};
}
template <int S>
__device__ __forceinline__ Cx<float> hadd_si(uint32_t a, Cx<float> b) {
    if constexpr (S > 0) return {hsub_lo(a, b.im), hadd_hi(a, b.re)};
    else return {hadd_lo(a, b.im), hsub_hi(a, b.re)};
}
__device__ __forceinline__ Cx<float> h2cx(uint32_t w) {
    const float2 f = h2f(w);
    return {f.x, f.y};
}

// Two-spinor h of (1 + S gamma_mu) psi from a stored FP16 spinor in the
// packed basis (unscaled; the site scale is applied with the hop's scale).
// The same combinations as project<MU, S>.
template <int MU, int SP>
__device__ __forceinline__ void project_h16(const uint32_t (&p)[12], Cx<float> (&h)[2][3]) {
    if constexpr (MU == 3) {  // packed basis: the kept spins, converted
        constexpr int off = SP > 0 ? 0 : 6;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h[0][a] = h2cx(p[off + a]);
            h[1][a] = h2cx(p[off + 3 + a]);
        }
        return;
    }
    constexpr int S = -SP;  // packed basis: gamma_mu' = -gamma_mu for space
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if constexpr (MU == 0) {
            h[0][a] = hadd_si<S>(p[a], h2cx(p[9 + a]));
            h[1][a] = hadd_si<S>(p[3 + a], h2cx(p[6 + a]));
        } else if constexpr (MU == 1) {
            h[0][a] = hadd_s<-S>(p[a], h2cx(p[9 + a]));
            h[1][a] = hadd_s<S>(p[3 + a], h2cx(p[6 + a]));
        } else if constexpr (MU == 2) {
            h[0][a] = hadd_si<S>(p[a], h2cx(p[6 + a]));
            h[1][a] = hadd_si<-S>(p[3 + a], h2cx(p[9 + a]));
        } else {
            h[0][a] = hadd_s<S>(p[a], h2cx(p[6 + a]));
            h[1][a] = hadd_s<S>(p[3 + a], h2cx(p[9 + a]));
        }
    }
}

// Raw bytes of one hop (neighbour spinor, its FP16 scale, the link) as
// loaded from memory, before any conversion.
template <int P, int RECON>
struct HopRaw {
    using L = HopLayout<P, RECON>;
    uint4 spin[L::spin16];
    float scale;
    uint4 link16[L::link16];
    uint2 link8;
};

template <int P, int RECON>
__device__ __forceinline__ HopRaw<P, RECON> stage_load_raw(const Stage<P, RECON> &st, int tid) {
    using H = HopRaw<P, RECON>;
    H r;
#pragma unroll
    for (int k = 0; k < H::L::spin16; ++k) r.spin[k] = *st.spin(k, tid);
    r.scale = H::L::scale4 ? *st.scale(tid) : 1.0f;
#pragma unroll
    for (int k = 0; k < H::L::link16; ++k) r.link16[k] = *st.link16(k, tid);
    r.link8 = H::L::link8 ? *st.link8(tid) : make_uint2(0u, 0u);
    return r;
}

// Hop J of output site c from its raw bytes: projection, link (third row
// rebuilt for recon 12), SU(3) product, boundary phase, accumulation.
template <int P, int RECON, int J, bool DAGGER>
__device__ __forceinline__ void hop_compute(const Geom &g, const Coord &c, const HopRaw<P, RECON> &r,
                                            Cx<float> (&acc)[12], float bs) {
    using L = HopLayout<P, RECON>;
    constexpr int MU = Hop<J>::MU, DIR = Hop<J>::DIR;
    constexpr int SF = DAGGER ? +1 : -1;
    constexpr int S = DIR > 0 ? SF : -SF;
    float sc = bs;
    Cx<float> h[2][3];
    if constexpr (P == COLA_F16) {
        uint32_t raw[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            raw[4 * k + 0] = r.spin[k].x;
            raw[4 * k + 1] = r.spin[k].y;
            raw[4 * k + 2] = r.spin[k].z;
            raw[4 * k + 3] = r.spin[k].w;
        }
        sc *= r.scale;
        project_h16<MU, S>(raw, h);
    } else {
        Cx<float> psi[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = *reinterpret_cast<const float4 *>(&r.spin[k]);
            psi[2 * k] = {v.x, v.y};
            psi[2 * k + 1] = {v.z, v.w};
        }
        project<MU, S>(psi, h);
    }
    Cx<float> u[9];
    if constexpr (P == COLA_F16) {
        uint32_t w[4 * L::link16 + 2];
#pragma unroll
        for (int k = 0; k < L::link16; ++k) {
            w[4 * k] = r.link16[k].x;
            w[4 * k + 1] = r.link16[k].y;
            w[4 * k + 2] = r.link16[k].z;
            w[4 * k + 3] = r.link16[k].w;
        }
        w[4 * L::link16] = r.link8.x;
        w[4 * L::link16 + 1] = r.link8.y;
#pragma unroll
        for (int k = 0; k < (RECON == 12 ? 6 : 9); ++k) u[k] = h2cx(w[k]);
    } else {
#pragma unroll
        for (int k = 0; k < L::link16; ++k) {
            const float4 v = *reinterpret_cast<const float4 *>(&r.link16[k]);
            if (2 * k < 9) u[2 * k] = {v.x, v.y};
            if (2 * k + 1 < 9) u[2 * k + 1] = {v.z, v.w};
        }
    }
    if constexpr (RECON == 12) reconstruct_row2(u);
    Cx<float> w[2][3];
    if constexpr (DIR > 0) su3_mul(u, h, w);
    else su3_adj_mul(u, h, w);
    if (!g.bc_trivial[MU] && coord_of<MU>(c) == (DIR > 0 ? g.L[MU] - 1 : 0)) boundary_phase(g, MU, DIR < 0, w, sc);
    accumulate<MU, S>(acc, w, sc);
}

template <int P, int RECON, int J, bool DAGGER>
__device__ __forceinline__ void stage_compute(const DslashLat &A, const Coord &c, const Stage<P, RECON> &st,
                                              int tid, Cx<float> (&acc)[12], float bs) {
    hop_compute<P, RECON, J, DAGGER>(A.g, c, stage_load_raw(st, tid), acc, bs);
}

template <int P, int RECON, bool DAGGER, int NS, int J>
__device__ __forceinline__ void staged_step(const DslashLat &A, const Coord &c, int cb, const char *in,
                                            const char *lo, const char *li, char *smem, int T, int tid,
                                            Cx<float> (&acc)[12], float bs) {
    using L = HopLayout<P, RECON>;
    if constexpr (J + NS - 1 < 8) {
        Stage<P, RECON> nx{smem + ((J + NS - 1) % NS) * L::bytes * kStagedThreads};
        stage_issue<P, RECON, J + NS - 1>(A, c, cb, in, lo, li, nx, tid);
    }
    cp_async_commit();
    cp_async_wait<NS - 1>();
    Stage<P, RECON> cur{smem + (J % NS) * L::bytes * kStagedThreads};
    stage_compute<P, RECON, J, DAGGER>(A, c, cur, tid, acc, bs);
    if constexpr (J < 7) staged_step<P, RECON, DAGGER, NS, J + 1>(A, c, cb, in, lo, li, smem, T, tid, acc, bs);
}

template <int P, int RECON, bool DAGGER, int NS, int J>
__device__ __forceinline__ void staged_prologue(const DslashLat &A, const Coord &c, int cb, const char *in,
                                                const char *lo, const char *li, char *smem, int T, int tid) {
    using L = HopLayout<P, RECON>;
    if constexpr (J < NS - 1) {
        Stage<P, RECON> st{smem + J * L::bytes * kStagedThreads};
        stage_issue<P, RECON, J>(A, c, cb, in, lo, li, st, tid);
        cp_async_commit();
        staged_prologue<P, RECON, DAGGER, NS, J + 1>(A, c, cb, in, lo, li, smem, T, tid);
    }
}

template <int P, int RECON, bool DAGGER, int NS>
__device__ __forceinline__ void hops_staged(const DslashLat &A, const Coord &c, int cb, const char *in,
                                            const char *lo, const char *li, Cx<float> (&acc)[12], float bs) {
    extern __shared__ __align__(16) char smem_dyn[];
    constexpr int T = kStagedThreads;  // blockDim.x * blockDim.y, enforced by launch_dslash
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    staged_prologue<P, RECON, DAGGER, NS, 0>(A, c, cb, in, lo, li, smem_dyn, T, tid);
    staged_step<P, RECON, DAGGER, NS, 0>(A, c, cb, in, lo, li, smem_dyn, T, tid, acc, bs);
}

// |s|^2 of one site, accumulated in the storage real type like the vector
// kernels' reductions.
template <typename R>
__device__ __forceinline__ double site_norm2_d(const Cx<R> (&s)[12]) {
    R a = R(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) a += s[k].re * s[k].re + s[k].im * s[k].im;
    return (double)a;
}

// Fused reduction of a hopping launch: the sum of v over the threads of each
// block row (one right-hand side), in a fixed order, written by the row's
// first thread to dst_row(threadIdx.y) if write.  Every thread of the block
// must call it.  Warps that lie within one row (blockDim.x a multiple of 32)
// reduce by shuffles; other shapes sum the row serially.
__device__ __forceinline__ void block_row_sum(double v, bool write, double *dst) {
    __shared__ double sh[256];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((blockDim.x & 31) == 0) {
        v = warp_allsum(v);
        if ((tid & 31) == 0) sh[tid >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0 && write) {
            const int wpr = blockDim.x >> 5;
            double t = 0.0;
            for (int w = 0; w < wpr; ++w) t += sh[threadIdx.y * wpr + w];
            *dst = t;
        }
    } else {
        sh[tid] = v;
        __syncthreads();
        if (threadIdx.x == 0 && write) {
            double t = 0.0;
            for (int i = 0; i < (int)blockDim.x; ++i) t += sh[threadIdx.y * blockDim.x + i];
            *dst = t;
        }
    }
}

// Grid: x over (site block, right-hand-side group) pairs of every lattice of
// the batch, group fastest (lattice l owns [block0, block0 + nblocks *
// ngroups)), so that the blocks reading the same links run back to back and
// find them in L1/L2; z over the output parities (1 or 2).
// Block: (sites, right-hand sides).
// Register budget: FP16/FP32 at two 256-thread blocks per SM (128 registers,
// no spills); FP64 is bound by the FP64 pipe and keeps its full register set.
// The staged kernels always run 128-thread blocks.
#ifndef COLA_STAGED_MINB
#define COLA_STAGED_MINB 5
#endif
// depth of the staged pipeline: while a thread computes one hop, the next
// stages - 1 are in flight.  With the 16 + 8 byte FP16 links, 4 stages ran
// the plain 32^3x64 parity apply in 67.0 us against 69.6 us for 3 (5 blocks
// of 39 KB per SM), while the even-odd operator (two of its four launches
// with the xpay epilogue) and the clover operator were no faster or slower
// with 4: the plain hop takes 4 stages, the other epilogues COLA_STAGES.
#ifndef COLA_STAGES
#define COLA_STAGES 3
#endif
#ifndef COLA_STAGES_HOP
#define COLA_STAGES_HOP 4
#endif
template <int P, int NS>
struct LaunchShape {
    static constexpr int threads = NS > 0 ? 128 : 256;
    static constexpr int min_blocks = P == COLA_F64 ? 1 : NS > 0 ? COLA_STAGED_MINB : COLA_DSLASH_MINB;
};

template <int P, int RECON, bool DAGGER, int EPI, int NS>
__global__ void __launch_bounds__(LaunchShape<P, NS>::threads, LaunchShape<P, NS>::min_blocks)
    dslash_kernel(const __grid_constant__ DslashArgs A) {
    using R = typename Prec<P>::real;
    int l = 0;
    while (l + 1 < A.nlat && (int)blockIdx.x >= A.lat[l + 1].block0) ++l;
    const DslashLat &L = A.lat[l];
    const Geom &g = L.g;
    const int rel = (int)blockIdx.x - L.block0;
    const int grp = A.ngroups == 1 ? 0 : rel % A.ngroups;
    const int sblk = A.ngroups == 1 ? rel : rel / A.ngroups;
    const int cb = sblk * blockDim.x + threadIdx.x;
    const int rhs = grp * blockDim.y + threadIdx.y;
    const int row = L.row0 + rhs;
    const int par = A.parity0 + blockIdx.z;
    const bool row_ok = rhs < A.nrhs;
    bool live = row_ok;
    if (live && A.state) {
        const CgState &st = A.state[row];
        live = A.filter_ru ? (st.ru && !st.done) : !st.done;
    }
    const bool have = cb < g.Vh && live;
    Cx<R> acc[12];
    double red_v = 0.0;  // |xin|^2 at this site (fused reduction)
    if (have) {
        const Coord c = cb_coord(g, cb, par);
        const char *in = static_cast<const char *>(L.in) + rhs * L.rhs_stride + (1 - par) * L.parity_stride;
        const char *lo = static_cast<const char *>(L.links) + par * L.link_parity_stride;
        const char *li = static_cast<const char *>(L.links) + (1 - par) * L.link_parity_stride;
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
        if constexpr (NS > 0 && P != COLA_F64) {
            hops_staged<P, RECON, DAGGER, NS>(L, c, cb, in, lo, li, acc, (float)L.b);
        } else {
            hop_mu<P, RECON, 0, DAGGER>(L, c, cb, in, lo, li, acc, (R)L.b);
            hop_mu<P, RECON, 1, DAGGER>(L, c, cb, in, lo, li, acc, (R)L.b);
            hop_mu<P, RECON, 2, DAGGER>(L, c, cb, in, lo, li, acc, (R)L.b);
            hop_mu<P, RECON, 3, DAGGER>(L, c, cb, in, lo, li, acc, (R)L.b);
        }
        // the factor b is already in every hop's scale
        if constexpr (EPI == EPI_XPAY || EPI == EPI_CLOVER_X) {
            const R a = (R)L.a;
            Cx<R> xs[12];
            SpinorIO<P>::load(static_cast<const char *>(L.xin) + rhs * L.rhs_stride + par * L.parity_stride,
                              g.Vh, cb, xs);
            if (A.red) red_v = site_norm2_d(xs);
            if constexpr (EPI == EPI_CLOVER_X)
                clover_mul<P>(static_cast<const char *>(L.clv) + par * L.clv_parity_stride, g.Vh, cb, xs);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                acc[k].re = fma(a, xs[k].re, acc[k].re);
                acc[k].im = fma(a, xs[k].im, acc[k].im);
            }
        }
        if constexpr (EPI == EPI_CLOVER_INV)
            clover_mul<P>(static_cast<const char *>(L.clv) + par * L.clv_parity_stride, g.Vh, cb, acc);
    }
    if (have)
        SpinorIO<P>::store(static_cast<char *>(L.out) + rhs * L.rhs_stride + par * L.parity_stride, g.Vh, cb, acc);
    if constexpr (EPI == EPI_XPAY || EPI == EPI_CLOVER_X) {
        if (A.red)
            block_row_sum(red_v, row_ok,
                          A.red + (size_t)row * A.red_stride + blockIdx.z * L.nblocks + sblk);
    }
}

// Multi-right-hand-side variant (direct loads): each thread carries NR
// right-hand sides of one site, so every link is loaded and reconstructed
// once per NR outputs.  Grid x runs over (site block, right-hand-side group)
// pairs as in dslash_kernel; a group is blockDim.y x NR right-hand sides.
template <int P, int RECON, bool DAGGER, int EPI, int NR>
__device__ __forceinline__ void dslash_mrhs_body(const DslashArgs &A, const DslashLat &L, int cb, int rhs0, int par,
                                                 const bool (&live)[NR], double (&red_v)[NR]);

template <int P, int RECON, bool DAGGER, int EPI, int NR>
__global__ void __launch_bounds__(256, 1) dslash_mrhs_kernel(const __grid_constant__ DslashArgs A) {
    int l = 0;
    while (l + 1 < A.nlat && (int)blockIdx.x >= A.lat[l + 1].block0) ++l;
    const DslashLat &L = A.lat[l];
    const Geom &g = L.g;
    const int rel = (int)blockIdx.x - L.block0;
    const int grp = A.ngroups == 1 ? 0 : rel % A.ngroups;
    const int sblk = A.ngroups == 1 ? rel : rel / A.ngroups;
    const int cb = sblk * blockDim.x + threadIdx.x;
    const int rhs0 = (grp * blockDim.y + threadIdx.y) * NR;
    const int par = A.parity0 + blockIdx.z;
    bool live[NR];
    bool any = false;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int rhs = rhs0 + k;
        bool ok = rhs < A.nrhs && cb < g.Vh;
        if (ok && A.state) {
            const CgState &st = A.state[L.row0 + rhs];
            ok = A.filter_ru ? (st.ru && !st.done) : !st.done;
        }
        live[k] = ok;
        any |= ok;
    }
    double red_v[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) red_v[k] = 0.0;
    if (any) dslash_mrhs_body<P, RECON, DAGGER, EPI, NR>(A, L, cb, rhs0, par, live, red_v);
    if constexpr (EPI == EPI_XPAY || EPI == EPI_CLOVER_X) {
        if (A.red)
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                block_row_sum(red_v[k], rhs0 + k < A.nrhs,
                              A.red + (size_t)(L.row0 + rhs0 + k) * A.red_stride + blockIdx.z * L.nblocks + sblk);
                __syncthreads();  // the shared sums are reused for the next right-hand side
            }
    }
}

template <int P, int RECON, bool DAGGER, int EPI, int NR>
__device__ __forceinline__ void dslash_mrhs_body(const DslashArgs &A, const DslashLat &L, int cb, int rhs0, int par,
                                                 const bool (&live)[NR], double (&red_v)[NR]) {
    using R = typename Prec<P>::real;
    const Geom &g = L.g;
    const Coord c = cb_coord(g, cb, par);
    const char *in0 = static_cast<const char *>(L.in) + (size_t)rhs0 * L.rhs_stride + (1 - par) * L.parity_stride;
    const char *lo = static_cast<const char *>(L.links) + par * L.link_parity_stride;
    const char *li = static_cast<const char *>(L.links) + (1 - par) * L.link_parity_stride;
    Cx<R> acc[NR][12];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
        for (int j = 0; j < 12; ++j) acc[k][j] = {R(0), R(0)};
    hop_mu_mrhs<P, RECON, 0, DAGGER, NR>(L, c, cb, in0, lo, li, acc, (R)L.b, live);
    hop_mu_mrhs<P, RECON, 1, DAGGER, NR>(L, c, cb, in0, lo, li, acc, (R)L.b, live);
    hop_mu_mrhs<P, RECON, 2, DAGGER, NR>(L, c, cb, in0, lo, li, acc, (R)L.b, live);
    hop_mu_mrhs<P, RECON, 3, DAGGER, NR>(L, c, cb, in0, lo, li, acc, (R)L.b, live);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (!live[k]) continue;
        const size_t roff = (size_t)(rhs0 + k) * L.rhs_stride + par * L.parity_stride;
        if constexpr (EPI == EPI_XPAY || EPI == EPI_CLOVER_X) {
            const R a = (R)L.a;
            Cx<R> xs[12];
            SpinorIO<P>::load(static_cast<const char *>(L.xin) + roff, g.Vh, cb, xs);
            if (A.red) red_v[k] = site_norm2_d(xs);
            if constexpr (EPI == EPI_CLOVER_X)
                clover_mul<P>(static_cast<const char *>(L.clv) + par * L.clv_parity_stride, g.Vh, cb, xs);
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                acc[k][j].re = fma(a, xs[j].re, acc[k][j].re);
                acc[k][j].im = fma(a, xs[j].im, acc[k][j].im);
            }
        }
        if constexpr (EPI == EPI_CLOVER_INV)
            clover_mul<P>(static_cast<const char *>(L.clv) + par * L.clv_parity_stride, g.Vh, cb, acc[k]);
        SpinorIO<P>::store(static_cast<char *>(L.out) + roff, g.Vh, cb, acc[k]);
    }
}

// Right-hand sides per thread the multi-right-hand-side kernel is built for
// (FP32 storage, direct loads); other precisions and the staged kernels carry
// one right-hand side per thread.
__host__ __device__ constexpr bool mrhs_supported(int prec, int nr) {
    return nr == 1 || (prec == COLA_F32 && (nr == 2 || nr == 4));
}

// Pipeline depth of the staged kernels: FP16 storage moves half the bytes
// per load of FP32, so it needs the deeper pipeline; FP32 keeps direct loads
// (measured on GB300 at 32^3x64).  COLA_DSLASH_STAGES=0 or 3 overrides.
static inline int staged_depth(int prec) {
    static const int env_ns = [] {
        const char *e = getenv("COLA_DSLASH_STAGES");
        return e ? atoi(e) : -1;
    }();
    if (prec == COLA_F64) return 0;
    if (env_ns >= 0) return env_ns == 0 ? 0 : COLA_STAGES;
    return prec == COLA_F16 ? COLA_STAGES : 0;
}

template <int P, int RECON, bool DAGGER, int EPI, int NS>
static cudaError_t launch_ns(const DslashArgs &A, int nparity, int bx, int total_blocks, cudaStream_t s) {
    const int by = A.rhs_per_block;
    dim3 block(bx, by, 1);
    dim3 grid(total_blocks, 1, nparity);
    size_t smem = 0;
    if constexpr (NS > 0 && P != COLA_F64) {
        smem = (size_t)NS * HopLayout<P, RECON>::bytes * bx * by;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(dslash_kernel<P, RECON, DAGGER, EPI, NS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
            attr_set = true;
        }
    }
    dslash_kernel<P, RECON, DAGGER, EPI, NS><<<grid, block, smem, s>>>(A);
    return cudaGetLastError();
}

template <int P, int RECON, bool DAGGER, int EPI, int NR>
static cudaError_t launch_mrhs(const DslashArgs &A, int nparity, int bx, int total_blocks, cudaStream_t s) {
    dim3 block(bx, A.rhs_per_block, 1);
    dim3 grid(total_blocks, 1, nparity);
    dslash_mrhs_kernel<P, RECON, DAGGER, EPI, NR><<<grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

template <int P, int RECON, bool DAGGER, int EPI>
static cudaError_t launch_t(const DslashArgs &A, int nparity, int bx, int nb, cudaStream_t s) {
    if constexpr (P == COLA_F32) {
        if (A.rhs_per_thread == 2) return launch_mrhs<P, RECON, DAGGER, EPI, 2>(A, nparity, bx, nb, s);
        if (A.rhs_per_thread == 4) return launch_mrhs<P, RECON, DAGGER, EPI, 4>(A, nparity, bx, nb, s);
    }
    if (A.rhs_per_thread > 1) return cudaErrorInvalidValue;
    if constexpr (P == COLA_F64) {
        return launch_ns<P, RECON, DAGGER, EPI, 0>(A, nparity, bx, nb, s);
    } else {
        if (staged_depth(P) == 0) return launch_ns<P, RECON, DAGGER, EPI, 0>(A, nparity, bx, nb, s);
        return launch_ns<P, RECON, DAGGER, EPI, EPI == EPI_HOP ? COLA_STAGES_HOP : COLA_STAGES>(A, nparity, bx, nb, s);
    }
}

// Launch with epilogue E0 or E1 (epi selects), both daggers.
template <int P, int RECON, int E0, int E1>
static cudaError_t launch_r(const DslashArgs &A, int nparity, bool dagger, int epi, int bx, int nb, cudaStream_t s) {
    if (dagger) return epi == E1 ? launch_t<P, RECON, true, E1>(A, nparity, bx, nb, s)
                                 : launch_t<P, RECON, true, E0>(A, nparity, bx, nb, s);
    return epi == E1 ? launch_t<P, RECON, false, E1>(A, nparity, bx, nb, s)
                     : launch_t<P, RECON, false, E0>(A, nparity, bx, nb, s);
}

template <int E0, int E1>
static cudaError_t launch_pr(int prec, int recon, const DslashArgs &A, int nparity, bool dagger, int epi, int bx,
                             int nb, cudaStream_t s) {
    switch (prec) {
        case COLA_F64:
            return recon == 12 ? launch_r<COLA_F64, 12, E0, E1>(A, nparity, dagger, epi, bx, nb, s)
                               : launch_r<COLA_F64, 18, E0, E1>(A, nparity, dagger, epi, bx, nb, s);
        case COLA_F32:
            return recon == 12 ? launch_r<COLA_F32, 12, E0, E1>(A, nparity, dagger, epi, bx, nb, s)
                               : launch_r<COLA_F32, 18, E0, E1>(A, nparity, dagger, epi, bx, nb, s);
        default:
            return recon == 12 ? launch_r<COLA_F16, 12, E0, E1>(A, nparity, dagger, epi, bx, nb, s)
                               : launch_r<COLA_F16, 18, E0, E1>(A, nparity, dagger, epi, bx, nb, s);
    }
}

}  // namespace cola
