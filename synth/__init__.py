"""Seeded synthetic inputs for the Wilson-Dirac hot path.

This module is the one piece shared by the oracle, the tests, the smoke check
and the benchmark.  It holds input construction only (random numbers, gauge
links drawn near the identity, Gaussian and point sources); it holds none of
the operator, solver or force arithmetic.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw i of stream (seed) is mix(seed + (i + 1) * 0x9E3779B97F4A7C15).
Uniforms take the top 53 bits; normals use the Box-Muller transform on
consecutive uniform pairs (u1, u2) -> sqrt(-2 ln(1 - u1)) * (cos, sin)(2 pi u2).

Layouts (canonical, x fastest; site i = x + Lx*(y + Ly*(z + Lz*t))):
  spinor  complex128 [Lt, Lz, Ly, Lx, 4 spin, 3 colour]
  gauge   complex128 [4 mu, Lt, Lz, Ly, Lx, 3, 3]   (mu = x, y, z, t)

Seeds: 230200850 + 16 * config + stream, stream 0 = gauge field,
1 = sources, 2 = finite-difference direction, 3 = gauge transformation.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 230200850


def seed_for(config: int, stream: int) -> int:
    """Seed of stream `stream` for workload number `config`."""
    return BASE_SEED + 16 * config + stream


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 sequence for `seed`."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + idx * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, count: int, chunk: int = 1 << 24) -> np.ndarray:
    """`count` standard normals (Box-Muller on consecutive uniform pairs)."""
    out = np.empty(count, dtype=np.float64)
    npairs = (count + 1) // 2
    done = 0
    while done < npairs:
        n = min(chunk, npairs - done)
        u = uniforms(seed, 2 * done, 2 * n).reshape(n, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
        th = 2.0 * np.pi * u[:, 1]
        pair = np.stack([r * np.cos(th), r * np.sin(th)], axis=1).reshape(-1)
        lo = 2 * done
        hi = min(count, lo + 2 * n)
        out[lo:hi] = pair[: hi - lo]
        done += n
    return out


def complex_normals(seed: int, shape) -> np.ndarray:
    """Standard complex Gaussians (E|z|^2 = 1), drawn re then im in C order."""
    n = int(np.prod(shape))
    g = normals(seed, 2 * n) * np.sqrt(0.5)
    return (g[0::2] + 1j * g[1::2]).reshape(shape)


def lattice_volume(dims) -> int:
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def _check_dims(dims):
    if len(dims) != 4 or any(int(d) < 2 or int(d) % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even numbers >= 2, got {dims}")


def _reunitarise(m):
    """Gram-Schmidt on rows 0 and 1; row 2 = conj(row0 x row1) (an SU(3) matrix)."""
    import torch

    r0 = m[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = m[..., 1, :]
    r1 = r1 - (torch.sum(r0.conj() * r1, dim=-1, keepdim=True)) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    c0 = r0[..., 1] * r1[..., 2] - r0[..., 2] * r1[..., 1]
    c1 = r0[..., 2] * r1[..., 0] - r0[..., 0] * r1[..., 2]
    c2 = r0[..., 0] * r1[..., 1] - r0[..., 1] * r1[..., 0]
    r2 = torch.stack([c0, c1, c2], dim=-1).conj()
    return torch.stack([r0, r1, r2], dim=-2)


def su3_near_identity(seed: int, n: int, eps: float, device="cpu"):
    """n matrices exp(i*eps*H), H = (A + A^dag)/2 - tr/3, A standard complex Gaussian.

    Returns a torch complex128 tensor [n, 3, 3] on `device`, re-unitarised so
    that each matrix is SU(3) to rounding and its third row is exactly the
    conjugate cross product of the first two.
    """
    import torch

    a = torch.from_numpy(complex_normals(seed, (n, 3, 3))).to(device)
    h = 0.5 * (a + a.conj().transpose(-1, -2))
    tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1) / 3.0
    h = h - tr[:, None, None] * torch.eye(3, dtype=h.dtype, device=device)
    u = torch.linalg.matrix_exp(1j * eps * h)
    return _reunitarise(u)


def gauge_field(dims, eps: float, seed: int, device="cpu", as_numpy: bool = True):
    """Links U_mu(x) = exp(i*eps*H) per site and direction.

    Draw order: canonical site order, then mu, then the 9 entries of A
    row-major (re then im).  Returned as [4, Lt, Lz, Ly, Lx, 3, 3].
    """
    _check_dims(dims)
    lx, ly, lz, lt = dims
    v = lattice_volume(dims)
    u = su3_near_identity(seed, v * 4, eps, device=device)
    u = u.reshape(lt, lz, ly, lx, 4, 3, 3).permute(4, 0, 1, 2, 3, 5, 6).contiguous()
    return u.cpu().numpy() if as_numpy else u


def unit_gauge(dims) -> np.ndarray:
    _check_dims(dims)
    lx, ly, lz, lt = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gaussian_spinor(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Standard complex Gaussian source, draw order site, spin, colour (re, im).

    With nrhs given, returns [nrhs, Lt, Lz, Ly, Lx, 4, 3], right-hand side outermost.
    """
    _check_dims(dims)
    lx, ly, lz, lt = dims
    shape = (lt, lz, ly, lx, 4, 3)
    if nrhs is None:
        return complex_normals(seed, shape)
    return complex_normals(seed, (nrhs,) + shape)


def point_sources(dims) -> np.ndarray:
    """The 12 spin-colour unit sources at the origin: [12, Lt, Lz, Ly, Lx, 4, 3]."""
    _check_dims(dims)
    lx, ly, lz, lt = dims
    s = np.zeros((12, lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    for k in range(12):
        s[k, 0, 0, 0, 0, k // 3, k % 3] = 1.0
    return s


def random_su3_field(dims, seed: int, eps: float = 1.0) -> np.ndarray:
    """One SU(3) matrix per site (for gauge transformations): [Lt, Lz, Ly, Lx, 3, 3]."""
    _check_dims(dims)
    lx, ly, lz, lt = dims
    u = su3_near_identity(seed, lattice_volume(dims), eps)
    return u.reshape(lt, lz, ly, lx, 3, 3).numpy()


def su3_direction(dims, seed: int) -> np.ndarray:
    """Real coefficients c_a ~ N(0, 1), a = 0..7, per link: [4, Lt, Lz, Ly, Lx, 8]."""
    _check_dims(dims)
    lx, ly, lz, lt = dims
    return normals(seed, 4 * lattice_volume(dims) * 8).reshape(4, lt, lz, ly, lx, 8)


# ------------------------------------------------------------------ device --
# The same SplitMix64 / Box-Muller recipe evaluated with torch on a device,
# in chunks, for lattices whose inputs would take minutes on the host.  The
# integer stream is bit-identical to the host one (64-bit wrap-around
# multiplication; logical shifts emulated by masking the arithmetic ones); the
# normals agree with the host ones to rounding (a different log / cos / sin).

def _device_uniforms(seed: int, start: int, count: int, device):
    import torch

    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)

    def as_i64(v):
        v &= (1 << 64) - 1
        return v - (1 << 64) if v >= (1 << 63) else v

    def lshr(z, k):  # logical right shift of the 64-bit pattern
        return (z >> k) & ((1 << (64 - k)) - 1)

    z = as_i64(seed) + idx * as_i64(int(GOLDEN))
    z = (z ^ lshr(z, 30)) * as_i64(int(_M1))
    z = (z ^ lshr(z, 27)) * as_i64(int(_M2))
    z = z ^ lshr(z, 31)
    return lshr(z, 11).to(torch.float64) * (2.0 ** -53)


def _device_normals(seed: int, start_pair: int, npairs: int, device):
    import torch

    u = _device_uniforms(seed, 2 * start_pair, 2 * npairs, device).reshape(npairs, 2)
    r = torch.sqrt(-2.0 * torch.log1p(-u[:, 0]))
    th = 2.0 * np.pi * u[:, 1]
    return torch.stack([r * torch.cos(th), r * torch.sin(th)], dim=1).reshape(-1)


def gauge_field_device(dims, eps: float, seed: int, device="cuda", chunk: int = 1 << 22):
    """gauge_field computed on `device` in chunks of `chunk` links: a torch
    complex128 tensor [4, Lt, Lz, Ly, Lx, 3, 3] (same draw order and recipe)."""
    import torch

    _check_dims(dims)
    lx, ly, lz, lt = dims
    n = lattice_volume(dims) * 4
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        g = _device_normals(seed, s * 9, m * 9, device) * np.sqrt(0.5)  # 18 normals (9 pairs) per matrix
        a = torch.complex(g[0::2], g[1::2]).reshape(m, 3, 3)
        h = 0.5 * (a + a.conj().transpose(-1, -2))
        h = h - (torch.diagonal(h, dim1=-2, dim2=-1).sum(-1) / 3.0)[:, None, None] * eye
        out[s:s + m] = _reunitarise(torch.linalg.matrix_exp(1j * eps * h))
    return out.reshape(lt, lz, ly, lx, 4, 3, 3).permute(4, 0, 1, 2, 3, 5, 6).contiguous()


def gaussian_spinor_device(dims, seed: int, device="cuda", chunk: int = 1 << 24):
    """gaussian_spinor computed on `device` (same draw order and recipe)."""
    import torch

    _check_dims(dims)
    lx, ly, lz, lt = dims
    n = lattice_volume(dims) * 12  # complex numbers = normal pairs
    out = torch.empty(n, dtype=torch.complex128, device=device)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        g = _device_normals(seed, s, m, device) * np.sqrt(0.5)
        out[s:s + m] = torch.complex(g[0::2], g[1::2])
    return out.reshape(lt, lz, ly, lx, 4, 3)
