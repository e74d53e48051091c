"""Seeded synthetic workloads for the variable-coefficient staggered Stokes solver.

This module is the one place that draws random numbers.  It builds the
coefficient fields (cell-centred density rho and shear viscosity mu), the
right-hand side (face forcing f, cell divergence data g) and the problem
description (grid, boundary conditions, theta = 1/dt) for each benchmark
configuration.  It holds none of the solver's arithmetic: both the CPU oracle
and the CUDA path receive the arrays it returns.

Storage layout (shared with the C ABI):
  * cell arrays have numpy shape (nz, ny, nx) (nz = 1 in 2D), x fastest;
  * the a-component face array has the same shape except that the a-axis
    extent is n_a + 1 when axis a has walls (faces 0 and n_a lie on the walls
    and are stored as zeros) and n_a when axis a is periodic.

The fields stand in for the paper's bubble tests (Sec. 4, Eq. varcoeff_def):
smooth log-normal fields scaled to a stated max/min contrast, or sharp
circular inclusions, at h = 1 so that the viscous CFL number is 1 when
theta = 1 (Sec. 4.3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, NOSLIP, FREESLIP = 0, 1, 2


@dataclass
class Problem:
    dim: int
    n: tuple            # (nx, ny, nz), nz = 1 in 2D
    bc: tuple           # 6 codes: x_lo, x_hi, y_lo, y_hi, z_lo, z_hi
    h: float
    theta: float        # 1/dt; 0 for steady flow
    rho: np.ndarray     # cell array
    mu: np.ndarray      # cell array
    b_u: list           # face arrays, one per velocity component
    b_p: np.ndarray     # cell array
    precond: int = 1    # 1..5: P1..P5
    name: str = ""
    meta: dict = field(default_factory=dict)


def face_shape(n, bc, a):
    """numpy shape of the a-component face array."""
    ext = list(n)
    if bc[2 * a] != PERIODIC:
        ext[a] += 1
    return (ext[2], ext[1], ext[0])


def cell_shape(n):
    return (n[2], n[1], n[0])


def _pad_n(n):
    n = list(n) + [1] * (3 - len(n))
    return tuple(int(v) for v in n)


def _cell_centres(n, h):
    nx, ny, nz = n
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h,
                          (np.arange(nx) + 0.5) * h, indexing="ij")
    return x, y, z


def smooth_field_2d(n, h, seed, modes=8, kmax=4):
    """Sum of `modes` random cosines a cos(2 pi k.x/L + phi); k integer with
    components in [-kmax, kmax], k != 0; a ~ N(0,1), phi ~ U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    x, y, _ = _cell_centres(n, h)
    Lx, Ly = n[0] * h, n[1] * h
    s = np.zeros(cell_shape(n))
    m = 0
    while m < modes:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if not k.any():
            continue
        a = rng.standard_normal()
        phi = rng.uniform(0.0, 2.0 * math.pi)
        s += a * np.cos(2 * math.pi * (k[0] * x / Lx + k[1] * y / Ly) + phi)
        m += 1
    return s


def smooth_field_3d(n, h, seed, kmax=8):
    """All integer wavevectors with |k_a| <= kmax, k != 0, amplitude
    N(0,1)/(1+|k|^2) and a uniform random phase, evaluated at cell centres by
    separable synthesis (independent of resolution)."""
    rng = np.random.default_rng(seed)
    ks = np.arange(-kmax, kmax + 1)
    K = len(ks)
    amp = rng.standard_normal((K, K, K))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=(K, K, K))
    kz, ky, kx = np.meshgrid(ks, ks, ks, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    c = amp / (1.0 + k2) * np.exp(1j * phase)
    c[k2 == 0] = 0.0
    nx, ny, nz = n
    ex = np.exp(2j * math.pi * np.outer(ks, (np.arange(nx) + 0.5) / nx))  # (K, nx)
    ey = np.exp(2j * math.pi * np.outer(ks, (np.arange(ny) + 0.5) / ny))
    ez = np.exp(2j * math.pi * np.outer(ks, (np.arange(nz) + 0.5) / nz))
    t = np.einsum("abc,cx->abx", c, ex)      # (kz, ky, x)
    t = np.einsum("abx,by->ayx", t, ey)      # (kz, y, x)
    t = np.einsum("ayx,az->zyx", t, ez)      # (z, y, x)
    return np.real(t)


def contrast_scale(s, contrast):
    """exp(c (s - midrange)) with max/min equal to `contrast` on the grid and
    geometric midrange 1."""
    lo, hi = float(s.min()), float(s.max())
    if contrast == 1.0 or hi == lo:
        return np.ones_like(s)
    c = math.log(contrast) / (hi - lo)
    return np.exp(c * (s - 0.5 * (hi + lo)))


def inclusions_2d(n, h, seed, count=20, rmin=0.02, rmax=0.06, mu_in=1e4, mu_out=1.0):
    """`count` non-overlapping disks (radius U(rmin, rmax) L, centre U[r, L-r]^2,
    rejection sampled); mu = mu_in at cells whose centre is inside a disk."""
    rng = np.random.default_rng(seed)
    L = n[0] * h
    disks = []
    tries = 0
    while len(disks) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place inclusions")
        r = rng.uniform(rmin, rmax) * L
        cx, cy = rng.uniform(r, L - r, size=2)
        if all((cx - dx) ** 2 + (cy - dy) ** 2 > (r + dr) ** 2 for dx, dy, dr in disks):
            disks.append((cx, cy, r))
    x, y, _ = _cell_centres(n, h)
    mu = np.full(cell_shape(n), mu_out)
    for cx, cy, r in disks:
        mu[(x - cx) ** 2 + (y - cy) ** 2 < r * r] = mu_in
    return mu, disks


def random_rhs(n, bc, dim, seed_f, seed_g, g_zero=False):
    """f ~ N(0,1) on every face that carries an unknown (wall faces 0) and
    g ~ N(0,1) with its mean removed; b_u = f, b_p = -g."""
    rng = np.random.default_rng(seed_f)
    b_u = []
    for a in range(dim):
        f = rng.standard_normal(face_shape(n, bc, a))
        if bc[2 * a] != PERIODIC:
            sl = [slice(None)] * 3
            sl[2 - a] = 0
            f[tuple(sl)] = 0.0
            sl[2 - a] = -1
            f[tuple(sl)] = 0.0
        b_u.append(f)
    if g_zero:
        g = np.zeros(cell_shape(n))
    else:
        g = np.random.default_rng(seed_g).standard_normal(cell_shape(n))
        g -= g.mean()
    return b_u, -g


def config_c1(n=32):
    """2D unsteady, n x n periodic; rho, mu contrast 10 smooth fields; theta=1; P1."""
    N = _pad_n((n, n))
    bc = (PERIODIC,) * 6
    rho = contrast_scale(smooth_field_2d(N, 1.0, 1), 10.0)
    mu = contrast_scale(smooth_field_2d(N, 1.0, 2), 10.0)
    b_u, b_p = random_rhs(N, bc, 2, 3, 4)
    return Problem(2, N, bc, 1.0, 1.0, rho, mu, b_u, b_p, precond=1,
                   name=f"2d_unsteady_periodic_{n}x{n}")


def config_c2(n=512, smooth=False):
    """2D steady, n x n no-slip walls, 20 disks of mu=1e4 in mu=1, rho=1; P2."""
    N = _pad_n((n, n))
    bc = (NOSLIP,) * 4 + (PERIODIC, PERIODIC)
    mu, disks = inclusions_2d(N, 1.0, 5)
    if smooth:
        x, y, _ = _cell_centres(N, 1.0)
        dist = np.full(cell_shape(N), np.inf)
        for cx, cy, r in disks:
            dist = np.minimum(dist, np.sqrt((x - cx) ** 2 + (y - cy) ** 2) - r)
        mu = 0.5 * (1e4 + 1) - 0.5 * (1e4 - 1) * np.tanh(dist / 1.0)
    rho = np.ones(cell_shape(N))
    b_u, b_p = random_rhs(N, bc, 2, 3, 4)
    return Problem(2, N, bc, 1.0, 0.0, rho, mu, b_u, b_p, precond=2,
                   name=f"2d_steady_noslip_inclusions_{n}x{n}", meta={"disks": disks})


def config_c3(n=128):
    """3D unsteady, n^3 periodic; rho contrast 1e2, mu contrast 1e3; theta=1; P1."""
    N = _pad_n((n, n, n))
    bc = (PERIODIC,) * 6
    rho = contrast_scale(smooth_field_3d(N, 1.0, 6), 1e2)
    mu = contrast_scale(smooth_field_3d(N, 1.0, 7), 1e3)
    b_u, b_p = random_rhs(N, bc, 3, 3, 4)
    return Problem(3, N, bc, 1.0, 1.0, rho, mu, b_u, b_p, precond=1,
                   name=f"3d_unsteady_periodic_{n}^3")


def config_c4_sizes(count=64, seed=8):
    idx = np.random.default_rng(seed).integers(0, 4, size=count)
    return [int((64, 128, 256, 512)[i]) for i in idx]


def config_c4_instance(i, n):
    """Instance i of the batched workload: 2D periodic n x n, rho = 1,
    mu contrast 1e3 (seed 100+i), theta = 1, random forcing; P1."""
    N = _pad_n((n, n))
    bc = (PERIODIC,) * 6
    mu = contrast_scale(smooth_field_2d(N, 1.0, 100 + i), 1e3)
    rho = np.ones(cell_shape(N))
    b_u, b_p = random_rhs(N, bc, 2, 1000 + i, 2000 + i)
    return Problem(2, N, bc, 1.0, 1.0, rho, mu, b_u, b_p, precond=1,
                   name=f"batched_instance_{i}_{n}x{n}")


def config_c5(n=64, target=False):
    """3D steady, n^3 no-slip walls; mu contrast 1e2 (seed 9; seed 10 for the
    target field), rho = 1; f ~ N(0,1) (seed 11), g = 0; P2."""
    N = _pad_n((n, n, n))
    bc = (NOSLIP,) * 6
    mu = contrast_scale(smooth_field_3d(N, 1.0, 10 if target else 9), 1e2)
    rho = np.ones(cell_shape(N))
    b_u, b_p = random_rhs(N, bc, 3, 11, 0, g_zero=True)
    return Problem(3, N, bc, 1.0, 0.0, rho, mu, b_u, b_p, precond=2,
                   name=f"3d_steady_noslip_{n}^3")


def generic(dim, n, bc, theta=1.0, rho_contrast=10.0, mu_contrast=10.0, seed=0, precond=1,
            h=1.0):
    """A small seeded problem of any shape, for parity tests."""
    N = _pad_n(n)
    if dim == 2:
        rho = contrast_scale(smooth_field_2d(N, h, seed + 1), rho_contrast)
        mu = contrast_scale(smooth_field_2d(N, h, seed + 2), mu_contrast)
    else:
        rho = contrast_scale(smooth_field_3d(N, h, seed + 1, kmax=3), rho_contrast)
        mu = contrast_scale(smooth_field_3d(N, h, seed + 2, kmax=3), mu_contrast)
    b_u, b_p = random_rhs(N, bc, dim, seed + 3, seed + 4)
    return Problem(dim, N, tuple(bc), h, theta, rho, mu, b_u, b_p, precond=precond,
                   name=f"generic_{dim}d_{'x'.join(map(str, N[:dim]))}")


def random_face_vector(n, bc, dim, seed):
    """Random velocity (wall faces 0) and pressure, e.g. for b = M x tests."""
    rng = np.random.default_rng(seed)
    u = []
    for a in range(dim):
        f = rng.standard_normal(face_shape(n, bc, a))
        if bc[2 * a] != PERIODIC:
            sl = [slice(None)] * 3
            sl[2 - a] = 0
            f[tuple(sl)] = 0.0
            sl[2 - a] = -1
            f[tuple(sl)] = 0.0
        u.append(f)
    p = rng.standard_normal(cell_shape(n))
    return u, p


def bubble(dim, n, r_mu=100.0, r_rho=100.0, theta=0.0, seed=12, bc_kind=NOSLIP, precond=1):
    """The bubble test of Sec. 4 (Eq. varcoeff_def): a sphere (disk in 2D) of
    radius L/4 at the centre of a box of side L = n h with no-slip walls;
    mu = f(x; r_mu), rho = f(x; r_rho) with
    f(x; r) = (r+1)/2 + (r-1)/2 tanh(d(x, Gamma)/eps) + 0.1 R,
    d the signed distance to the sphere (positive outside), eps = h and
    R ~ U(0, 1) per cell.  The forcing is f ~ N(0,1), g ~ N(0,1) mean-free."""
    N = _pad_n((n,) * dim)
    bc = (bc_kind,) * (2 * dim) + (PERIODIC,) * (6 - 2 * dim)
    h = 1.0
    L = n * h
    x, y, z = _cell_centres(N, h)
    rr = (x - L / 2) ** 2 + (y - L / 2) ** 2
    if dim == 3:
        rr = rr + (z - L / 2) ** 2
    dist = np.sqrt(rr) - L / 4
    rng = np.random.default_rng(seed)

    def f(r):
        return 0.5 * (r + 1) + 0.5 * (r - 1) * np.tanh(dist / h) + 0.1 * rng.uniform(size=dist.shape)

    mu = f(r_mu)
    rho = f(r_rho)
    b_u, b_p = random_rhs(N, bc, dim, seed + 1, seed + 2)
    return Problem(dim, N, bc, h, theta, rho, mu, b_u, b_p, precond=precond,
                   name=f"bubble_{dim}d_{n}_r{r_mu:g}")
