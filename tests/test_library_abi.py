"""The C-ABI library builds, loads and exports what include/cola.h declares (CPU only).

Also checks host-side argument validation, which runs before any CUDA call,
and that the ctypes structures match the C layout (compiled with gcc).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cola.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cola_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_00850_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["cola_dslash_apply", "cola_mdagm_apply", "cola_cg_solve", "cola_fermion_force"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2302_00850_gb300 import _lib

    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_struct_layout_matches_c(tmp_path):
    from paper_2302_00850_gb300 import _lib

    prog = tmp_path / "sz.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "cola.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(cola_lattice), sizeof(cola_gauge_opts),"
        " sizeof(cola_solver_params), sizeof(cola_solve_info), offsetof(cola_solver_params, delta),"
        " offsetof(cola_solve_info, true_rel_resid), offsetof(cola_lattice, bc));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(_lib.Lattice), ctypes.sizeof(_lib.GaugeOpts), ctypes.sizeof(_lib.SolverParams),
            ctypes.sizeof(_lib.SolveInfo), _lib.SolverParams.delta.offset, _lib.SolveInfo.true_rel_resid.offset,
            _lib.Lattice.bc.offset]
    assert got == want


def _lattice(dims, kappa=0.12):
    from paper_2302_00850_gb300 import _lib

    lat = _lib.Lattice()
    for m in range(4):
        lat.dims[m] = dims[m]
        lat.bc[m][0] = 1.0
    lat.bc[3][0] = -1.0
    lat.kappa = kappa
    return lat


def test_spinor_bytes(lib):
    lat = _lattice((4, 4, 4, 8))
    v = 4 * 4 * 4 * 8
    assert lib.cola_spinor_bytes(ctypes.byref(lat), 0, 1) == v * 192
    assert lib.cola_spinor_bytes(ctypes.byref(lat), 1, 3) == 3 * v * 96
    assert lib.cola_spinor_bytes(ctypes.byref(lat), 2, 2) == 2 * v * 52
    assert lib.cola_spinor_bytes(ctypes.byref(_lattice((4, 5, 4, 8))), 0, 1) == 0


def test_argument_errors_before_any_cuda_call(lib):
    from paper_2302_00850_gb300 import _lib

    h = ctypes.c_void_p()
    opts = _lib.GaugeOpts()
    opts.prec_mask = 1
    opts.recon[0] = 18
    dummy = ctypes.c_void_p(1)
    assert lib.cola_gauge_create(ctypes.byref(_lattice((4, 3, 4, 4))), dummy, ctypes.byref(opts), None,
                                 ctypes.byref(h)) == -1
    assert b"even" in lib.cola_last_error()
    opts.recon[0] = 14
    assert lib.cola_gauge_create(ctypes.byref(_lattice((4, 4, 4, 4))), dummy, ctypes.byref(opts), None,
                                 ctypes.byref(h)) == -1
    assert b"recon" in lib.cola_last_error()
    opts.prec_mask = 0
    assert lib.cola_gauge_create(ctypes.byref(_lattice((4, 4, 4, 4))), dummy, ctypes.byref(opts), None,
                                 ctypes.byref(h)) == -1
    assert lib.cola_cg_solve(None, None, None, None, None, None) == -1
    assert lib.cola_dslash_apply(None, None, None, None, 0.0, 1.0, 0, 0, 0, 1, None) == -1
    assert lib.cola_dirac_apply(None, None, None, 0, 0, 1, None) == -1
    assert lib.cola_clover_attach(None, 1.0, None) == -1
    assert lib.cola_clover_apply(None, None, None, 2, 0, 0, 1, None) == -1
    assert lib.cola_clover_csw(None) == 0.0
    assert lib.cola_plaquette(None, None, None) == -1
    assert lib.cola_gauge_force(None, 5.6, None, None) == -1
    assert lib.cola_link_update(None, None, None, 0.1, None) == -1
    assert lib.cola_gauge_destroy(None) == 0


def test_hmc_parameter_errors_before_any_cuda_call(lib):
    from paper_2302_00850_gb300 import _lib

    fake = ctypes.c_void_p(1)  # never dereferenced: parameters are checked first
    info = _lib.HmcInfo()
    md = _lib.SolverParams(1e-10, 100, 0, 0, 0, 0.1, 1, 0)
    for kw in [dict(beta=-1.0), dict(tau=0.0), dict(nsteps=0), dict(integrator=2), dict(uniform=1.0),
               dict(uniform=-0.1), dict(action_tol=0.0)]:
        p = dict(beta=5.6, tau=1.0, nsteps=4, integrator=0, uniform=0.5, action_tol=1e-12)
        p.update(kw)
        prm = _lib.HmcParams(p["beta"], p["tau"], p["nsteps"], p["integrator"], p["uniform"], md, p["action_tol"])
        assert lib.cola_hmc_trajectory(fake, fake, fake, None, ctypes.byref(prm), ctypes.byref(info), None) == -1, kw
    assert lib.cola_hmc_trajectory(None, fake, fake, None, None, ctypes.byref(info), None) == -1


def test_multishift_parameter_errors_before_any_cuda_call(lib):
    from paper_2302_00850_gb300 import _lib

    fake = ctypes.c_void_p(1)
    info = (_lib.SolveInfo * 2)()
    good = (ctypes.c_double * 2)(0.0, 0.5)
    bad = (ctypes.c_double * 2)(0.0, -0.5)
    prm = _lib.SolverParams(1e-10, 100, 1, 0, 0, 0.1, 1, 0)
    assert lib.cola_multishift_solve(None, fake, fake, good, 2, 0.0, ctypes.byref(prm), info, None) == -1
    assert lib.cola_multishift_solve(fake, fake, fake, good, 0, 0.0, ctypes.byref(prm), info, None) == -1
    assert lib.cola_multishift_solve(fake, fake, fake, good, 65, 0.0, ctypes.byref(prm), info, None) == -1
    assert lib.cola_multishift_solve(fake, fake, fake, bad, 2, 0.0, ctypes.byref(prm), info, None) == -1
    dirac = _lib.SolverParams(1e-10, 100, 1, 1, 0, 0.1, 1, 0)
    assert lib.cola_multishift_solve(fake, fake, fake, good, 2, 0.0, ctypes.byref(dirac), info, None) == -1


def test_eig_parameter_errors_before_any_cuda_call(lib):
    from paper_2302_00850_gb300 import _lib

    fake = ctypes.c_void_p(1)
    vals = (ctypes.c_double * 4)()
    info = _lib.EigInfo()
    for kw in [dict(nev=0), dict(nev=65), dict(nev=60, nextra=5), dict(nextra=-1), dict(op=3), dict(tol=0.0),
               dict(max_sweeps=0), dict(max_cg=0), dict(gamma=1.0)]:
        p = dict(nev=4, nextra=0, op=1, tol=1e-8, max_sweeps=5, max_cg=10, gamma=0.1)
        p.update(kw)
        prm = _lib.EigParams(p["nev"], p["nextra"], p["op"], p["tol"], p["max_sweeps"], p["max_cg"], p["gamma"])
        assert lib.cola_eig_lowest(fake, fake, vals, ctypes.byref(prm), ctypes.byref(info), None) == -1, kw
    assert lib.cola_eig_lowest(None, fake, vals, None, ctypes.byref(info), None) == -1


def test_solver_parameter_errors_before_any_cuda_call(lib):
    from paper_2302_00850_gb300 import _lib

    fake = ctypes.c_void_p(1)  # never dereferenced: parameters are checked first
    info = (_lib.SolveInfo * 1)()
    for kw in [dict(nrhs=0), dict(nrhs=65), dict(tol=0.0), dict(max_iter=-1), dict(op=7), dict(system=3),
               dict(inner=5), dict(inner=2, delta=1.5)]:
        p = dict(tol=1e-10, max_iter=10, op=1, system=0, inner=0, delta=0.1, nrhs=1, use_graph=0)
        p.update(kw)
        prm = _lib.SolverParams(p["tol"], p["max_iter"], p["op"], p["system"], p["inner"], p["delta"], p["nrhs"],
                                p["use_graph"])
        assert lib.cola_cg_solve(fake, fake, fake, ctypes.byref(prm), info, None) == -1, kw
    hs = (ctypes.c_void_p * 1)(1)
    prm = _lib.SolverParams(1e-10, 10, 1, 0, 0, 0.1, 1, 0)
    assert lib.cola_cg_solve_batched(0, hs, hs, hs, ctypes.byref(prm), info, None) == -1
    assert lib.cola_cg_solve_batched(9, hs, hs, hs, ctypes.byref(prm), info, None) == -1


def test_fp64_probe_parameter_errors_before_any_cuda_call(lib):
    fake = ctypes.c_void_p(1)  # never dereferenced: parameters are checked first
    flop = ctypes.c_double(0.0)
    for blocks, threads, steps in [(0, 256, 4096), (1216, 33, 4096), (1216, 512, 4096), (1216, 256, 4098),
                                   (1216, 256, 0)]:
        assert lib.cola_probe_fp64_fma(fake, blocks, threads, steps, None, ctypes.byref(flop)) == -1
    assert lib.cola_probe_fp64_fma(None, 1216, 256, 4096, None, ctypes.byref(flop)) == -1
    assert lib.cola_probe_fp64_fma(fake, 1216, 256, 4096, None, None) == -1
