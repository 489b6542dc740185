"""Python API over the C ABI (include/cola.h), on torch CUDA tensors.

torch supplies device memory, the current stream and autograd plumbing; every
step of the Wilson-Dirac path (packing, hopping term, solver, force) runs in
libcola's CUDA kernels.  There is no CPU implementation here and no fallback:
calls on tensors that are not CUDA tensors raise.

Canonical layouts (complex128, x fastest):
  spinor  [Lt, Lz, Ly, Lx, 4, 3], or [nrhs, Lt, Lz, Ly, Lx, 4, 3]
  links   [4, Lt, Lz, Ly, Lx, 3, 3]
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import F16, F32, F64, OP_EO, OP_FULL, SYS_DIRAC, SYS_NORMAL, ColaError, check  # noqa: F401

PREC = {"f64": F64, "f32": F32, "f16": F16, F64: F64, F32: F32, F16: F16}
OPS = {"full": OP_FULL, "eo": OP_EO, OP_FULL: OP_FULL, OP_EO: OP_EO}
SYSTEMS = {"normal": SYS_NORMAL, "dirac": SYS_DIRAC, SYS_NORMAL: SYS_NORMAL, SYS_DIRAC: SYS_DIRAC}


def _stream(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _ptr(t: torch.Tensor) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("libcola takes CUDA tensors (no CPU path)")
    if not t.is_contiguous():
        raise ValueError("libcola takes contiguous tensors")
    return t.data_ptr()


def _complex_field(t: torch.Tensor, numel: int, what: str):
    if t.dtype != torch.complex128:
        raise TypeError(f"{what} must be complex128")
    if t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, expected {numel}")
    return _ptr(t)


class Gauge:
    """Packed links of one lattice (a cola_gauge handle).

    links: complex128 CUDA tensor [4, Lt, Lz, Ly, Lx, 3, 3] (SU(3) for recon 12)
    dims: (Lx, Ly, Lz, Lt); bc: per-direction boundary phase (complex)
    precisions: any of "f64", "f32", "f16"; recon: dict precision -> 12 or 18
    """

    def __init__(self, links, dims, kappa, bc=(1, 1, 1, -1), precisions=("f64", "f32", "f16"), recon=None):
        self.lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        self.bc = tuple(complex(b) for b in bc)
        lx, ly, lz, lt = self.dims
        self.volume = lx * ly * lz * lt
        self.lat = _lib.Lattice()
        for m in range(4):
            self.lat.dims[m] = self.dims[m]
            self.lat.bc[m][0] = self.bc[m].real
            self.lat.bc[m][1] = self.bc[m].imag
        self.lat.kappa = self.kappa
        recon = dict(recon or {})
        self.recon = {}
        opts = _lib.GaugeOpts()
        opts.prec_mask = 0
        for p in precisions:
            pi = PREC[p]
            opts.prec_mask |= 1 << pi
            r = int(recon.get(p, recon.get(pi, 18 if pi == F64 else 12)))
            opts.recon[pi] = r
            self.recon[pi] = r
        self.precisions = {PREC[p] for p in precisions}
        self.device = links.device
        self.handle = ctypes.c_void_p()
        check(self.lib.cola_gauge_create(ctypes.byref(self.lat), _complex_field(links, 4 * self.volume * 9, "links"),
                                         ctypes.byref(opts), _stream(self.device), ctypes.byref(self.handle)))

    def attach_clover(self, csw):
        """Attach the clover term A = 1 - kappa c_sw sum sigma F (csw = 0 removes it).

        Builds A and A^-1 from the FP64 links (the handle must hold "f64");
        afterwards the Dirac operator, the normal operators and the solves use
        D = A - kappa H.  Waits for the construction.
        """
        check(self.lib.cola_clover_attach(self.handle, float(csw), _stream(self.device)))

    @property
    def csw(self) -> float:
        return float(self.lib.cola_clover_csw(self.handle))

    def update(self, links):
        """Re-pack new links (same lattice) into this handle, keeping its workspace."""
        check(self.lib.cola_gauge_update(self.handle, _complex_field(links, 4 * self.volume * 9, "links"),
                                         _stream(self.device)))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.cola_gauge_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spinor_shape(self, nrhs=None):
        lx, ly, lz, lt = self.dims
        base = (lt, lz, ly, lx, 4, 3)
        return base if nrhs is None else (nrhs,) + base

    def spinor_bytes(self, prec, nrhs=1) -> int:
        return int(self.lib.cola_spinor_bytes(ctypes.byref(self.lat), PREC[prec], int(nrhs)))

    def empty_packed(self, prec, nrhs=1) -> torch.Tensor:
        return torch.empty(self.spinor_bytes(prec, nrhs), dtype=torch.uint8, device=self.device)


def _nrhs_of(g: Gauge, psi: torch.Tensor):
    n = psi.numel() // (g.volume * 12)
    if n * g.volume * 12 != psi.numel():
        raise ValueError("spinor size is not a multiple of V * 12")
    return n


def pack(g: Gauge, psi: torch.Tensor, prec="f64") -> torch.Tensor:
    """Canonical complex128 spinor(s) -> packed field in precision `prec`."""
    nrhs = _nrhs_of(g, psi)
    out = g.empty_packed(prec, nrhs)
    check(g.lib.cola_spinor_pack(g.handle, _ptr(out), _ptr(psi), PREC[prec], nrhs, _stream(g.device)))
    return out


def unpack(g: Gauge, packed: torch.Tensor, prec="f64", nrhs=None) -> torch.Tensor:
    n = 1 if nrhs is None else nrhs
    out = torch.empty(g.spinor_shape(nrhs), dtype=torch.complex128, device=g.device)
    check(g.lib.cola_spinor_unpack(g.handle, _ptr(out), _ptr(packed), PREC[prec], n, _stream(g.device)))
    return out


def dslash(g: Gauge, out, inp, in_self=None, a=0.0, b=1.0, parity=2, dagger=False, prec="f64", nrhs=1):
    """out_p = a in_self_p + b H_{p,1-p} in_{1-p} on packed fields (parity 0, 1 or 2 = both)."""
    check(g.lib.cola_dslash_apply(g.handle, _ptr(out), _ptr(inp), _ptr(in_self) if in_self is not None else None,
                                  float(a), float(b), int(parity), int(bool(dagger)), PREC[prec], int(nrhs),
                                  _stream(g.device)))
    return out


def mdagm(g: Gauge, out, inp, op="eo", prec="f64", nrhs=1):
    """out = M^dag M in on packed fields (op "eo": Mhat on the even half; "full": D)."""
    check(g.lib.cola_mdagm_apply(g.handle, _ptr(out), _ptr(inp), OPS[op], PREC[prec], int(nrhs), _stream(g.device)))
    return out


def dirac(g: Gauge, out, inp, dagger=False, prec="f64", nrhs=1):
    """out = D in (or D^dag in) on packed fields; D = A - kappa H with a clover term."""
    check(g.lib.cola_dirac_apply(g.handle, _ptr(out), _ptr(inp), int(bool(dagger)), PREC[prec], int(nrhs),
                                 _stream(g.device)))
    return out


def clover(g: Gauge, out, inp, parity=2, inverse=False, prec="f64", nrhs=1):
    """out_p = A_pp in_p (inverse: A_pp^-1 in_p) on packed fields, parity 0, 1 or 2 = both."""
    check(g.lib.cola_clover_apply(g.handle, _ptr(out), _ptr(inp), int(parity), int(bool(inverse)), PREC[prec],
                                  int(nrhs), _stream(g.device)))
    return out


def apply_dirac(g: Gauge, psi: torch.Tensor, dagger=False, prec="f64") -> torch.Tensor:
    """D psi (or D^dag psi) on canonical complex128 fields, through the packed kernels."""
    nrhs = _nrhs_of(g, psi)
    pin = pack(g, psi, prec)
    pout = g.empty_packed(prec, nrhs)
    dirac(g, pout, pin, dagger=dagger, prec=prec, nrhs=nrhs)
    return unpack(g, pout, prec, None if psi.dim() == 6 else nrhs).reshape(psi.shape)


def apply_clover(g: Gauge, psi: torch.Tensor, inverse=False, prec="f64") -> torch.Tensor:
    """A psi (or A^-1 psi) on canonical complex128 fields, through the packed kernels."""
    nrhs = _nrhs_of(g, psi)
    pin = pack(g, psi, prec)
    pout = g.empty_packed(prec, nrhs)
    clover(g, pout, pin, parity=2, inverse=inverse, prec=prec, nrhs=nrhs)
    return unpack(g, pout, prec, None if psi.dim() == 6 else nrhs).reshape(psi.shape)


@dataclass
class SolveInfo:
    iters: int
    reliable_updates: int
    true_rel_resid: float
    seconds: float
    status: int


def cg_solve(g: Gauge, b: torch.Tensor, x0: torch.Tensor | None = None, tol=1e-10, max_iter=100000, op="eo",
             system="normal", inner="f64", delta=0.1, use_graph=False, raise_on_error=True):
    """Solve with CG (see cola_cg_solve).  Returns (x, [SolveInfo per right-hand side])."""
    nrhs = _nrhs_of(g, b)
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    prm = _lib.SolverParams(float(tol), int(max_iter), OPS[op], SYSTEMS[system], PREC[inner], float(delta), nrhs,
                            int(bool(use_graph)))
    infos = (_lib.SolveInfo * nrhs)()
    st = g.lib.cola_cg_solve(g.handle, _ptr(x), _complex_field(b, nrhs * g.volume * 12, "b"), ctypes.byref(prm),
                             infos, _stream(g.device))
    res = [SolveInfo(i.iters, i.reliable_updates, i.true_rel_resid, i.seconds, i.status) for i in infos]
    if st != 0 and (raise_on_error or st not in (-4, -5)):
        check(st)
    return x, res


def cg_solve_batched(gauges, bs, x0s=None, tol=1e-10, max_iter=100000, op="eo", system="normal", inner="f64",
                     delta=0.1, use_graph=False, raise_on_error=True):
    """Solve several lattices together (cola_cg_solve_batched).

    gauges: list of Gauge (distinct, same device); bs: matching list of sources,
    each with the same number of right-hand sides.  Returns (xs, infos) with
    infos[l][r] the SolveInfo of lattice l, right-hand side r.
    """
    nlat = len(gauges)
    if nlat != len(bs) or nlat < 1:
        raise ValueError("gauges and bs must be non-empty lists of the same length")
    nrhs = _nrhs_of(gauges[0], bs[0])
    xs = []
    for l, (g, b) in enumerate(zip(gauges, bs)):
        if _nrhs_of(g, b) != nrhs:
            raise ValueError("every lattice of a batch must have the same number of right-hand sides")
        _complex_field(b, nrhs * g.volume * 12, "b")
        xs.append(torch.zeros_like(b) if x0s is None else x0s[l].clone())
    lib = gauges[0].lib
    hs = (ctypes.c_void_p * nlat)(*[g.handle.value for g in gauges])
    xp = (ctypes.c_void_p * nlat)(*[_ptr(x) for x in xs])
    bp = (ctypes.c_void_p * nlat)(*[_ptr(b) for b in bs])
    prm = _lib.SolverParams(float(tol), int(max_iter), OPS[op], SYSTEMS[system], PREC[inner], float(delta), nrhs,
                            int(bool(use_graph)))
    infos = (_lib.SolveInfo * (nlat * nrhs))()
    st = lib.cola_cg_solve_batched(nlat, hs, xp, bp, ctypes.byref(prm), infos, _stream(gauges[0].device))
    res = [[SolveInfo(i.iters, i.reliable_updates, i.true_rel_resid, i.seconds, i.status)
            for i in infos[l * nrhs:(l + 1) * nrhs]] for l in range(nlat)]
    if st != 0 and (raise_on_error or st not in (-4, -5)):
        check(st)
    return xs, res


def multishift_solve(g: Gauge, b: torch.Tensor, shifts, tol=1e-10, max_iter=100000, op="eo", inner="f64",
                     delta=0.1, tol_sloppy=0.0, use_graph=False, raise_on_error=True):
    """x_i = (A + shifts[i])^-1 b for all shifts at once (see cola_multishift_solve).

    Returns (x [nshift, Lt, Lz, Ly, Lx, 4, 3] complex128, [SolveInfo per shift]).
    """
    shifts = [float(v) for v in shifts]
    n = len(shifts)
    x = torch.empty((n,) + g.spinor_shape(), dtype=torch.complex128, device=g.device)
    prm = _lib.SolverParams(float(tol), int(max_iter), OPS[op], SYSTEMS["normal"], PREC[inner], float(delta), 1,
                            int(bool(use_graph)))
    infos = (_lib.SolveInfo * n)()
    sh = (ctypes.c_double * n)(*shifts)
    st = g.lib.cola_multishift_solve(g.handle, _ptr(x), _complex_field(b, g.volume * 12, "b"), sh, n,
                                     float(tol_sloppy), ctypes.byref(prm), infos, _stream(g.device))
    res = [SolveInfo(i.iters, i.reliable_updates, i.true_rel_resid, i.seconds, i.status) for i in infos]
    if st != 0 and (raise_on_error or st not in (-4, -5)):
        check(st)
    return x, res


@dataclass
class EigInfo:
    sweeps: int
    applications: int
    max_rel_resid: float
    seconds: float
    status: int


def eig_lowest(g: Gauge, v0: torch.Tensor, nev: int | None = None, op="eo", tol=1e-8, max_sweeps=50, max_cg=40,
               gamma=0.1, raise_on_error=True):
    """Lowest eigenpairs of Mhat^dag Mhat ("eo") or D^dag D ("full") (see cola_eig_lowest).

    v0: starting vectors, complex128 [nev + nextra, Lt, Lz, Ly, Lx, 4, 3] (e.g.
    Gaussian); rows beyond nev (default: all rows) are guard vectors.
    Returns (eigenvalues float64 [nev], eigenvectors [nev, ...], EigInfo).
    """
    nvec = v0.shape[0]
    nev = nvec if nev is None else int(nev)
    vecs = v0.detach().clone().contiguous()
    _complex_field(vecs, nvec * g.volume * 12, "v0")
    vals = (ctypes.c_double * nvec)()
    prm = _lib.EigParams(nev, nvec - nev, OPS[op], float(tol), int(max_sweeps), int(max_cg), float(gamma))
    info = _lib.EigInfo()
    st = g.lib.cola_eig_lowest(g.handle, _ptr(vecs), vals, ctypes.byref(prm), ctypes.byref(info), _stream(g.device))
    if st != 0 and (raise_on_error or st != -4):
        check(st)
    return (torch.tensor(list(vals)[:nev], dtype=torch.float64), vecs[:nev],
            EigInfo(info.sweeps, info.applications, info.max_rel_resid, info.seconds, info.status))


def fermion_force(g: Gauge, X: torch.Tensor, Y: torch.Tensor) -> torch.Tensor:
    """F^a_mu(x) = dS/deps^a for S = phi^dag (D^dag D)^-1 phi, X = (D^dag D)^-1 phi, Y = D X.

    With a clover term attached, D = A - kappa H and the clover term's force is included."""
    lx, ly, lz, lt = g.dims
    out = torch.empty((4, lt, lz, ly, lx, 8), dtype=torch.float64, device=g.device)
    check(g.lib.cola_fermion_force(g.handle, _ptr(out), _complex_field(X, g.volume * 12, "X"),
                                   _complex_field(Y, g.volume * 12, "Y"), _stream(g.device)))
    return out


def dirac_link_grad(g: Gauge, psi: torch.Tensor, gy: torch.Tensor) -> torch.Tensor:
    """Raw complex link gradient (torch convention) of a real loss through y = D psi, given dL/dy
    (with a clover term attached, D = A - kappa H and the clover part is included)."""
    lx, ly, lz, lt = g.dims
    out = torch.empty((4, lt, lz, ly, lx, 3, 3), dtype=torch.complex128, device=g.device)
    check(g.lib.cola_dirac_link_grad(g.handle, _ptr(out), _complex_field(psi, g.volume * 12, "psi"),
                                     _complex_field(gy, g.volume * 12, "gy"), _stream(g.device)))
    return out


# ------------------------------------------------------------------- HMC --
INTEGRATORS = {"leapfrog": 0, "omelyan": 1}


@dataclass
class HmcInfo:
    dH: float
    H0: float
    H1: float
    accepted: bool
    plaquette: float
    force_evals: int
    cg_iters: int
    seconds: float


def plaquette(g: Gauge) -> float:
    """Mean plaquette of the handle's links."""
    out = ctypes.c_double()
    check(g.lib.cola_plaquette(g.handle, ctypes.byref(out), _stream(g.device)))
    return out.value


def _mom_field(t: torch.Tensor, g: Gauge) -> int:
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != 4 * g.volume * 8:
        raise ValueError("momenta/forces must be contiguous float64 CUDA tensors of 4*V*8 elements")
    return t.data_ptr()


def gauge_force(g: Gauge, beta: float) -> torch.Tensor:
    """dS_G/deps^a of the Wilson gauge action, float64 [4, Lt, Lz, Ly, Lx, 8]."""
    lx, ly, lz, lt = g.dims
    out = torch.empty((4, lt, lz, ly, lx, 8), dtype=torch.float64, device=g.device)
    check(g.lib.cola_gauge_force(g.handle, float(beta), _mom_field(out, g), _stream(g.device)))
    return out


def link_update(g: Gauge, links: torch.Tensor, mom: torch.Tensor, eps: float) -> torch.Tensor:
    """links <- exp(i eps P) links in place (and the handle re-packed); returns links."""
    check(g.lib.cola_link_update(g.handle, _complex_field(links, 4 * g.volume * 9, "links"), _mom_field(mom, g),
                                 float(eps), _stream(g.device)))
    return links


def hmc_trajectory(g: Gauge, links: torch.Tensor, mom: torch.Tensor, eta: torch.Tensor | None, beta: float,
                   tau: float, nsteps: int, integrator="leapfrog", uniform=0.5, md_tol=1e-10, md_inner="f64",
                   delta=0.1, action_tol=1e-12, use_graph=True, md_op="full") -> HmcInfo:
    """One HMC update (see cola_hmc_trajectory); links and mom are updated in place.

    md_op "full": force solves by CG on D^dag D; "eo": two even-odd Dirac-system solves.
    """
    md = _lib.SolverParams(float(md_tol), 100000, OPS[md_op], SYSTEMS["normal"], PREC[md_inner], float(delta), 1,
                           int(bool(use_graph)))
    prm = _lib.HmcParams(float(beta), float(tau), int(nsteps), INTEGRATORS[integrator], float(uniform), md,
                         float(action_tol))
    info = _lib.HmcInfo()
    eta_p = None if eta is None else _complex_field(eta, g.volume * 12, "eta")
    check(g.lib.cola_hmc_trajectory(g.handle, _complex_field(links, 4 * g.volume * 9, "links"), _mom_field(mom, g),
                                    eta_p, ctypes.byref(prm), ctypes.byref(info), _stream(g.device)))
    return HmcInfo(info.dH, info.H0, info.H1, bool(info.accepted), info.plaquette, info.force_evals, info.cg_iters,
                   info.seconds)


def debug_bounds(reset: bool = False) -> tuple[int, int]:
    """(violations, kernel source line of the first) of the bounds-checking debug build
    (COLA_LIB=.../_build_bounds/libcola.so); waits for the device; reset zeroes the counters.
    A default build raises ColaError (COLA_ERR_UNSUPPORTED)."""
    lib = _lib.load()
    count, line = ctypes.c_ulonglong(0), ctypes.c_int(0)
    check(lib.cola_debug_bounds(ctypes.byref(count), ctypes.byref(line), int(bool(reset))))
    return int(count.value), int(line.value)


def probe_fp64_fma(out: torch.Tensor, blocks: int, threads: int = 256, steps: int = 4096) -> float:
    """Launch the FP64 fused-multiply-add probe on the current stream (no wait);
    returns the flop count of the launch.  out: float64 on the device with at
    least blocks * threads elements."""
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < blocks * threads:
        raise ValueError("out must be a CUDA float64 tensor of at least blocks * threads elements")
    flop = ctypes.c_double(0.0)
    check(_lib.load().cola_probe_fp64_fma(_ptr(out), int(blocks), int(threads), int(steps), _stream(out.device),
                                          ctypes.byref(flop)))
    return float(flop.value)
