// Hybrid Monte Carlo driver and the gauge-field entry points of the C ABI
// (plaquette, gauge force, link update, one HMC trajectory).
//
// HMC (Duane, Kennedy, Pendleton and Roweth 1987) is one of COLA's key
// algorithms (the paper's overview of the library).  The trajectory runs on
// the device throughout: forces accumulate straight into the momenta
// (p += coef F), links are exponentiated in place and re-packed into the
// handle, and the Hamiltonian's terms are deterministic FP64 reductions read
// back at the start and the end.  Each fermion force is a CG solve of
// D^dag D X = phi from a zero guess (so that the trajectory is reversible up
// to the solver tolerance), Y = D X, and the fermion-force kernel (plus the
// clover force when the handle has a clover term: D = A - kappa H throughout,
// in phi = D^dag eta, the solves, Y and the force).
#include <chrono>
#include <cmath>
#include <string>

#include "cola_impl.h"

namespace cola {
namespace {

#define HMC_TRY(expr)                   \
    do {                                \
        cola_status _st = (expr);       \
        if (_st != COLA_OK) return _st; \
    } while (0)
#define HMC_CUDA(expr, what) HMC_TRY(cuda_check((expr), what))

cola_status arg_error(const std::string &msg) {
    set_error(msg);
    return COLA_ERR_ARG;
}

cola_status need_f64(cola_gauge g) {
    if (!g->links[COLA_F64]) {
        set_error("this call needs FP64 links in the gauge handle");
        return COLA_ERR_UNSUPPORTED;
    }
    return COLA_OK;
}

size_t link_canon_bytes(const Geom &G) { return (size_t)4 * G.V * 9 * 16; }
size_t mom_doubles(const Geom &G) { return (size_t)4 * G.V * 8; }
size_t spinor_canon_bytes(const Geom &G) { return (size_t)G.V * 12 * 16; }

// reduction scratch and a few device result doubles
cola_status red_scratch(cola_gauge g, double **scratch, double **res) {
    const size_t n = gauge_scratch_doubles(g->geom);
    void *p = nullptr;
    HMC_TRY(ws_slot(g, cola_gauge_s::kSlotHmc + 6, (n + 8) * sizeof(double), &p));
    *scratch = static_cast<double *>(p);
    *res = *scratch + n;
    return COLA_OK;
}

cola_status read_doubles(const double *dev, double *host, int n, cudaStream_t s) {
    HMC_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, s), "result readback");
    HMC_CUDA(cudaStreamSynchronize(s), "reduction");
    return COLA_OK;
}

cola_status repack(cola_gauge g, const void *links, cudaStream_t s) {
    for (int p = 0; p < 3; ++p)
        if (g->links[p])
            HMC_CUDA(launch_pack_gauge(p, g->recon[p], g->geom, g->links[p], links, s), "link packing");
    if (g->csw != 0.0) return clover_rebuild(g, s);
    return COLA_OK;
}

// out = D in (dagger: D^dag in) on canonical FP64 fields, through packed buffers
cola_status dirac_canon(cola_gauge g, void *out, const void *in, bool dagger, void *pa, void *pb, cudaStream_t s) {
    HMC_CUDA(launch_pack_spinor(COLA_F64, g->geom, pa, in, 1, 3, s), "pack");
    HMC_TRY(cola_dirac_apply(g, pb, pa, dagger ? 1 : 0, COLA_F64, 1, s));
    HMC_CUDA(launch_unpack_spinor(COLA_F64, g->geom, out, pb, 1, 3, s), "unpack");
    return COLA_OK;
}

struct Traj {
    cola_gauge g;
    void *links;
    double *mom;
    const void *eta;
    const cola_hmc_params *prm;
    cudaStream_t s;
    void *saved, *phi, *X, *Y, *pa, *pb;
    void *clv_scratch = nullptr;
    double *scratch, *res;
    int force_evals = 0;
    int cg_iters = 0;
};

// X = (D^dag D)^-1 phi from a zero guess, to tolerance tol.  md.op FULL: CG
// on D^dag D.  md.op EO: X = D^-1 gamma5 D^-1 gamma5 phi (D^-dag =
// gamma5 D^-1 gamma5), two Dirac-system solves through the even-odd Schur
// complement, each on half the lattice with a better conditioned operator;
// Y is scratch until the caller sets Y = D X.
cola_status solve_x(Traj &T, double tol) {
    const Geom &G = T.g->geom;
    cola_solver_params md = T.prm->md;
    md.nrhs = 1;
    md.tol = tol;
    cola_solve_info info;
    if (md.op != COLA_OP_EO) {
        md.op = COLA_OP_FULL;
        md.system = COLA_SYS_NORMAL;
        HMC_CUDA(cudaMemsetAsync(T.X, 0, spinor_canon_bytes(G), T.s), "zero guess");
        cola_status st = cola_cg_solve(T.g, T.X, T.phi, &md, &info, T.s);
        T.cg_iters += info.iters;
        return st;
    }
    md.system = COLA_SYS_DIRAC;
    HMC_CUDA(launch_gamma5(G, T.Y, T.phi, T.s), "gamma5");
    HMC_CUDA(cudaMemsetAsync(T.X, 0, spinor_canon_bytes(G), T.s), "zero guess");
    cola_status st = cola_cg_solve(T.g, T.X, T.Y, &md, &info, T.s);
    T.cg_iters += info.iters;
    if (st != COLA_OK) return st;
    HMC_CUDA(launch_gamma5(G, T.Y, T.X, T.s), "gamma5");
    HMC_CUDA(cudaMemsetAsync(T.X, 0, spinor_canon_bytes(G), T.s), "zero guess");
    st = cola_cg_solve(T.g, T.X, T.Y, &md, &info, T.s);
    T.cg_iters += info.iters;
    return st;
}

// p += coef F(U)
cola_status force(Traj &T, double coef) {
    cola_gauge g = T.g;
    const Geom &G = g->geom;
    ++T.force_evals;
    HMC_CUDA(launch_gauge_force(G, g->links[COLA_F64], g->recon[COLA_F64], T.prm->beta, coef, T.mom, true, T.s),
             "gauge force");
    if (!T.eta) return COLA_OK;
    HMC_TRY(solve_x(T, T.prm->md.tol));
    HMC_TRY(dirac_canon(g, T.Y, T.X, false, T.pa, T.pb, T.s));
    HMC_CUDA(launch_force(G, g->lat.kappa, g->links[COLA_F64], g->recon[COLA_F64], T.mom, T.X, T.Y, T.s, coef, true),
             "fermion force");
    if (g->csw != 0.0)
        HMC_CUDA(launch_clover_force(G, g->links[COLA_F64], g->recon[COLA_F64], g->lat.kappa, g->csw, T.X, T.Y, T.mom,
                                     coef, true, T.clv_scratch, T.s),
                 "clover force");
    return COLA_OK;
}

// U <- exp(i eps P) U and re-pack
cola_status update(Traj &T, double eps) {
    HMC_CUDA(launch_link_update(T.g->geom, T.links, T.mom, eps, T.s), "link update");
    return repack(T.g, T.links, T.s);
}

// K + S_G (+ S_F with a solve when with_fermions), reduced on the device
cola_status hamiltonian(Traj &T, bool fermion_solve, double *h, double *plaq_mean) {
    cola_gauge g = T.g;
    const Geom &G = g->geom;
    HMC_CUDA(launch_dot(T.mom, T.mom, mom_doubles(G), 0.5, T.scratch, T.res + 0, T.s), "kinetic energy");
    HMC_CUDA(launch_plaquette_sum(G, g->links[COLA_F64], g->recon[COLA_F64], T.scratch, T.res + 1, T.s), "plaquette");
    int n = 2;
    if (T.eta) {
        if (fermion_solve) {
            HMC_TRY(solve_x(T, T.prm->action_tol));
            HMC_CUDA(launch_dot(static_cast<const double *>(T.phi), static_cast<const double *>(T.X),
                                spinor_canon_bytes(G) / 8, 1.0, T.scratch, T.res + 2, T.s),
                     "phi^dag X");
        } else {
            HMC_CUDA(launch_dot(static_cast<const double *>(T.eta), static_cast<const double *>(T.eta),
                                spinor_canon_bytes(G) / 8, 1.0, T.scratch, T.res + 2, T.s),
                     "|eta|^2");
        }
        n = 3;
    }
    double r[3] = {0.0, 0.0, 0.0};
    HMC_TRY(read_doubles(T.res, r, n, T.s));
    const double nplaq = 6.0 * G.V;
    *h = r[0] + T.prm->beta * (nplaq - r[1]) + r[2];
    if (plaq_mean) *plaq_mean = r[1] / nplaq;
    return COLA_OK;
}

cola_status integrate(Traj &T) {
    const int n = T.prm->nsteps;
    const double eps = T.prm->tau / n;
    if (T.prm->integrator == COLA_INT_LEAPFROG) {
        HMC_TRY(force(T, -0.5 * eps));
        for (int k = 0; k < n; ++k) {
            HMC_TRY(update(T, eps));
            HMC_TRY(force(T, k + 1 < n ? -eps : -0.5 * eps));
        }
        return COLA_OK;
    }
    const double lam = 0.1931833275037836;
    HMC_TRY(force(T, -lam * eps));
    for (int k = 0; k < n; ++k) {
        HMC_TRY(update(T, 0.5 * eps));
        HMC_TRY(force(T, -(1.0 - 2.0 * lam) * eps));
        HMC_TRY(update(T, 0.5 * eps));
        HMC_TRY(force(T, k + 1 < n ? -2.0 * lam * eps : -lam * eps));
    }
    return COLA_OK;
}

cola_status check_hmc_params(const cola_hmc_params *p) {
    if (!std::isfinite(p->beta) || p->beta < 0.0) return arg_error("beta must be finite and >= 0");
    if (!std::isfinite(p->tau) || p->tau <= 0.0) return arg_error("tau must be finite and > 0");
    if (p->nsteps < 1 || p->nsteps > 100000) return arg_error("nsteps must be in 1..100000");
    if (p->integrator != COLA_INT_LEAPFROG && p->integrator != COLA_INT_OMELYAN)
        return arg_error("integrator must be COLA_INT_LEAPFROG or COLA_INT_OMELYAN");
    if (!(p->uniform >= 0.0 && p->uniform < 1.0)) return arg_error("uniform must be in [0, 1)");
    if (!(p->action_tol > 0.0 && p->action_tol < 1.0)) return arg_error("action_tol must be in (0, 1)");
    if (!(p->md.tol > 0.0 && p->md.tol < 1.0)) return arg_error("md.tol must be in (0, 1)");
    return COLA_OK;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" {

cola_status cola_plaquette(cola_gauge g, double *plaq, cudaStream_t stream) {
    TraceRange trace_("cola_plaquette");
    if (!g || !plaq) return arg_error("null argument to cola_plaquette");
    HMC_TRY(need_f64(g));
    double *scratch, *res;
    HMC_TRY(red_scratch(g, &scratch, &res));
    HMC_CUDA(launch_plaquette_sum(g->geom, g->links[COLA_F64], g->recon[COLA_F64], scratch, res, stream), "plaquette");
    double sum = 0.0;
    HMC_TRY(read_doubles(res, &sum, 1, stream));
    *plaq = sum / (6.0 * g->geom.V);
    return COLA_OK;
}

cola_status cola_gauge_force(cola_gauge g, double beta, double *force_dev, cudaStream_t stream) {
    TraceRange trace_("cola_gauge_force");
    if (!g || !force_dev) return arg_error("null argument to cola_gauge_force");
    if (!std::isfinite(beta)) return arg_error("beta is not finite");
    HMC_TRY(need_f64(g));
    return cuda_check(launch_gauge_force(g->geom, g->links[COLA_F64], g->recon[COLA_F64], beta, 1.0, force_dev, false,
                                         stream),
                      "gauge force");
}

cola_status cola_link_update(cola_gauge g, void *links_dev, const double *mom_dev, double eps, cudaStream_t stream) {
    TraceRange trace_("cola_link_update");
    if (!g || !links_dev || !mom_dev) return arg_error("null argument to cola_link_update");
    if (!std::isfinite(eps)) return arg_error("eps is not finite");
    HMC_CUDA(launch_link_update(g->geom, links_dev, mom_dev, eps, stream), "link update");
    return repack(g, links_dev, stream);
}

cola_status cola_hmc_trajectory(cola_gauge g, void *links_dev, double *mom_dev, const void *eta_dev,
                                const cola_hmc_params *params, cola_hmc_info *info, cudaStream_t stream) {
    TraceRange trace_("cola_hmc_trajectory");
    if (!g || !links_dev || !mom_dev || !params || !info) return arg_error("null argument to cola_hmc_trajectory");
    HMC_TRY(check_hmc_params(params));
    HMC_TRY(need_f64(g));
    const auto t0 = std::chrono::steady_clock::now();
    const Geom &G = g->geom;
    Traj T;
    T.g = g;
    T.links = links_dev;
    T.mom = mom_dev;
    T.eta = eta_dev;
    T.prm = params;
    T.s = stream;
    const int k = cola_gauge_s::kSlotHmc;
    const size_t sp = spinor_canon_bytes(G), pk = 2 * spinor_parity_bytes(COLA_F64, G.Vh);
    HMC_TRY(ws_slot(g, k + 0, link_canon_bytes(G), &T.saved));
    HMC_TRY(red_scratch(g, &T.scratch, &T.res));
    if (eta_dev) {
        if (params->md.op != COLA_OP_FULL && params->md.op != COLA_OP_EO)
            return arg_error("md.op must be COLA_OP_FULL or COLA_OP_EO");
        HMC_TRY(ws_slot(g, k + 1, sp, &T.phi));
        HMC_TRY(ws_slot(g, k + 2, sp, &T.X));
        HMC_TRY(ws_slot(g, k + 3, sp, &T.Y));
        HMC_TRY(ws_slot(g, k + 4, pk, &T.pa));
        HMC_TRY(ws_slot(g, k + 5, pk, &T.pb));
        if (g->csw != 0.0)
            HMC_TRY(ws_slot(g, cola_gauge_s::kSlotCloverForce, clover_force_scratch_bytes(G), &T.clv_scratch));
    }
    HMC_CUDA(cudaMemcpyAsync(T.saved, links_dev, link_canon_bytes(G), cudaMemcpyDeviceToDevice, stream), "save links");
    if (eta_dev) HMC_TRY(dirac_canon(g, T.phi, eta_dev, true, T.pa, T.pb, stream));
    double h0 = 0.0, h1 = 0.0, plaq = 0.0;
    HMC_TRY(hamiltonian(T, false, &h0, nullptr));
    HMC_TRY(integrate(T));
    HMC_TRY(hamiltonian(T, true, &h1, &plaq));
    const double dh = h1 - h0;
    const bool accept = params->uniform <= std::exp(-dh);  // NaN rejects
    if (!accept) {
        HMC_CUDA(cudaMemcpyAsync(links_dev, T.saved, link_canon_bytes(G), cudaMemcpyDeviceToDevice, stream),
                 "restore links");
        HMC_TRY(repack(g, links_dev, stream));
        double sum = 0.0;
        HMC_CUDA(launch_plaquette_sum(G, g->links[COLA_F64], g->recon[COLA_F64], T.scratch, T.res, stream),
                 "plaquette");
        HMC_TRY(read_doubles(T.res, &sum, 1, stream));
        plaq = sum / (6.0 * G.V);
    }
    info->dH = dh;
    info->H0 = h0;
    info->H1 = h1;
    info->accepted = accept ? 1 : 0;
    info->plaquette = plaq;
    info->force_evals = T.force_evals;
    info->cg_iters = T.cg_iters;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (log_enabled())
        log_line("hmc_trajectory: dH %.6e (%s), plaquette %.6f, %d force evaluations, %d CG iterations, %.3f s", dh,
                 accept ? "accepted" : "rejected", plaq, T.force_evals, T.cg_iters, info->seconds);
    return COLA_OK;
}

}  // extern "C"
