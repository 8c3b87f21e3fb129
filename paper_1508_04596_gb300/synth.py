"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This module holds workload descriptions and random-input generators only; none
of the method's arithmetic (no residual, interpolation or stabilisation) lives
here.  Both the oracle and the CUDA path consume what it produces.

The paper (Sec. 6.1) optimises a heat sink in a cavity; its designs are not
available, so design fields are generated:
  * ``smoothed_random``: gamma ~ U[0,1] per element (NumPy PCG64, seeded), a
    3x3x3 box filter (mean over the in-domain neighbours), then gamma = 1
    (fluid) outside the design column;
  * ``fins``: a 4x4 array of square vertical pins (pitch 0.125 L, half-width
    0.03125 L) in the design column with a linear solid-to-fluid ramp over two
    elements, seeded noise of amplitude 0.05, clamped to [0,1];
    the solid density rho is converted to the paper's gamma = 1 - rho.
The design column is the set of elements whose centroid has x, y in
[0.25, 0.75] L and z in [0, 0.75 Lz].
"""
import numpy as np

# name: (nx, ny, nz, h, Gr, Pr, patch mode, design generator, seed)
WORKLOADS = {
    "cavity12_gr1e3": dict(nx=12, ny=12, nz=12, h=1 / 12, Gr=1e3, Pr=0.71,
                           patch="dirichlet", design="smoothed_random", seed=0),
    "fins64_gr1e4": dict(nx=64, ny=64, nz=64, h=1 / 64, Gr=1e4, Pr=0.71,
                         patch="dirichlet", design="fins", seed=1),
    "cavity128_gr1e5": dict(nx=128, ny=128, nz=128, h=1 / 128, Gr=1e5, Pr=0.71,
                            patch="dirichlet", design="smoothed_random", seed=2),
    "cavity96_gr1e5_flux": dict(nx=96, ny=96, nz=96, h=1 / 96, Gr=1e5, Pr=0.71,
                                patch="flux", design="smoothed_random", seed=3),
    "tall192x192x384_gr1e6": dict(nx=192, ny=192, nz=384, h=1 / 192, Gr=1e6, Pr=0.71,
                                  patch="flux", design="smoothed_random", seed=5),
}
# material parameters common to all workloads: RAMP q = 1, alpha_max = 1e4,
# solid-to-fluid conductivity ratio 10 (Ck = k_f / k_s = 0.1)
MATERIAL = dict(alpha_max=1e4, q_alpha=1.0, q_f=1.0, Ck=0.1)


def elem_centroids(nx, ny, nz, h):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([(i.ravel() + 0.5) * h, (j.ravel() + 0.5) * h, (k.ravel() + 0.5) * h], 1)


def design_column(nx, ny, nz, h):
    c = elem_centroids(nx, ny, nz, h)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    return ((c[:, 0] >= 0.25 * Lx) & (c[:, 0] <= 0.75 * Lx)
            & (c[:, 1] >= 0.25 * Ly) & (c[:, 1] <= 0.75 * Ly)
            & (c[:, 2] <= 0.75 * Lz))


def box_filter3(a):
    """Mean over the in-domain 3x3x3 neighbourhood of a [nz, ny, nx] array."""
    s = np.zeros_like(a)
    c = np.zeros_like(a)
    nz, ny, nx = a.shape
    one = np.ones_like(a)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                dst = (slice(max(0, -dz), nz - max(0, dz)), slice(max(0, -dy), ny - max(0, dy)),
                       slice(max(0, -dx), nx - max(0, dx)))
                src = (slice(max(0, dz), nz - max(0, -dz)), slice(max(0, dy), ny - max(0, -dy)),
                       slice(max(0, dx), nx - max(0, -dx)))
                s[dst] += a[src]
                c[dst] += one[src]
    return s / c


def smoothed_random(nx, ny, nz, h, seed):
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    g = box_filter3(g).ravel()
    g[~design_column(nx, ny, nz, h)] = 1.0
    return g


def fins(nx, ny, nz, h, seed):
    rng = np.random.default_rng(seed)
    Lx, Ly = nx * h, ny * h
    c = elem_centroids(nx, ny, nz, h)
    centres = 0.25 + 0.0625 + 0.125 * np.arange(4)
    dx = np.min(np.abs(c[:, 0:1] / Lx - centres[None, :]), axis=1) * Lx
    dy = np.min(np.abs(c[:, 1:2] / Ly - centres[None, :]), axis=1) * Ly
    dinf = np.maximum(dx, dy)
    hw = 0.03125 * Lx
    rho = np.clip(1.0 - (dinf - hw) / (2.0 * h), 0.0, 1.0)
    rho = np.clip(rho + 0.05 * rng.uniform(-1.0, 1.0, size=rho.shape), 0.0, 1.0)
    gam = 1.0 - rho
    gam[~design_column(nx, ny, nz, h)] = 1.0
    return gam


def design(name_or_cfg, seed=None):
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    s = cfg["seed"] if seed is None else seed
    gen = {"smoothed_random": smoothed_random, "fins": fins}[cfg["design"]]
    return gen(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"], s)


def design_step(name_or_cfg, gam, seed, amp=0.02):
    """A synthetic optimiser step: gamma + amp * (box-filtered U[-1,1] noise) inside
    the design column, clipped to [0, 1] (the next design of an optimisation run,
    whose state solve is warm-started from the current one)."""
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    nx, ny, nz, h = cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"]
    rng = np.random.default_rng(seed)
    d = box_filter3(rng.uniform(-1.0, 1.0, size=(nz, ny, nx))).ravel()
    col = design_column(nx, ny, nz, h)
    out = np.array(gam, dtype=float, copy=True)
    out[col] = np.clip(out[col] + amp * d[col], 0.0, 1.0)
    return out


def random_state(nx, ny, nz, seed, scale=(1.0, 1.0, 1.0, 1.0, 1.0)):
    """Random nodal state, [5, Nn], N(0, scale_f^2) per field (Dirichlet values
    are imposed by whoever consumes it)."""
    rng = np.random.default_rng(seed)
    Nn = (nx + 1) * (ny + 1) * (nz + 1)
    return rng.standard_normal((5, Nn)) * np.asarray(scale)[:, None]


def random_design(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=nx * ny * nz)
