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
  * ``quarter``: the paper's quarter cavity (solid source block, design domain
    at 1 - v_f with small seeded noise, fluid elsewhere).
The regions (design column, quarter-cavity blocks) are defined in
``cavity``, the package's statement of the problem set-up; this module only
draws random fields on them.
"""
import numpy as np

from . import cavity as _cavity
# the cavity regions, re-exported for the input generators' users
from .cavity import QUARTER, design_column, elem_centroids, quarter_regions  # noqa: F401

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
    # The paper's own set-up (Sec. 6.1-6.2): the quarter of a closed unit cavity
    # (x, y in [0, 1/2], z in [0, 1] vertical; symmetry planes at x = y = 1/2),
    # mesh 80 x 80 x 160 (the paper's 80 x 160 x 80 with its middle index
    # vertical), Pr = 1, Ck = 1e-2, first continuation step q_f = 0.881,
    # q_alpha = 8, alpha_max = 1e5, heat source block s0 = 1e4.
    "quarter80x80x160_gr1e3": dict(nx=80, ny=80, nz=160, h=1 / 160, Gr=1e3, Pr=1.0,
                                   patch="none", bcs="quarter", design="quarter", seed=7,
                                   material=dict(alpha_max=1e5, q_alpha=8.0, q_f=0.881, Ck=1e-2)),
    "quarter80x80x160_gr1e6": dict(nx=80, ny=80, nz=160, h=1 / 160, Gr=1e6, Pr=1.0,
                                   patch="none", bcs="quarter", design="quarter", seed=7,
                                   material=dict(alpha_max=1e5, q_alpha=8.0, q_f=0.881, Ck=1e-2)),
    # the paper's larger meshes of the same quarter cavity (Sec. 6.4): 160 x 320 x 160
    # elements, 41,603,205 unknowns, and 320 x 640 x 320 elements, 330,246,405
    # unknowns (middle index vertical there, z here)
    "quarter160x160x320_gr1e3": dict(nx=160, ny=160, nz=320, h=1 / 320, Gr=1e3, Pr=1.0,
                                     patch="none", bcs="quarter", design="quarter", seed=7,
                                     material=dict(alpha_max=1e5, q_alpha=8.0, q_f=0.881, Ck=1e-2)),
    "quarter320x320x640_gr1e3": dict(nx=320, ny=320, nz=640, h=1 / 640, Gr=1e3, Pr=1.0,
                                     patch="none", bcs="quarter", design="quarter", seed=7,
                                     material=dict(alpha_max=1e5, q_alpha=8.0, q_f=0.881, Ck=1e-2)),
}
# material parameters common to all workloads: RAMP q = 1, alpha_max = 1e4,
# solid-to-fluid conductivity ratio 10 (Ck = k_f / k_s = 0.1)
MATERIAL = dict(alpha_max=1e4, q_alpha=1.0, q_f=1.0, Ck=0.1)


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


def quarter_design(nx, ny, nz, h, seed):
    """Solid source block (gamma = 0), the design domain at the volume fraction
    of the paper (gamma = 1 - v_f, the uniform start of an optimisation) with
    seeded smoothed noise of amplitude 0.02, fluid elsewhere."""
    src, des = quarter_regions(nx, ny, nz, h)
    rng = np.random.default_rng(seed)
    noise = box_filter3(rng.uniform(-1.0, 1.0, size=(nz, ny, nx))).ravel()
    g = np.ones(nx * ny * nz)
    g[des] = np.clip(1.0 - QUARTER["vf"] + 0.02 * noise[des], 0.0, 1.0)
    g[src] = 0.0
    return g


def source(name_or_cfg):
    """Element heat source s_e of a workload (cavity.source)."""
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    return _cavity.source(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"], cfg.get("bcs") == "quarter")


def material(name_or_cfg):
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    return dict(cfg.get("material", MATERIAL))


def design(name_or_cfg, seed=None):
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    s = cfg["seed"] if seed is None else seed
    gen = {"smoothed_random": smoothed_random, "fins": fins, "quarter": quarter_design}[cfg["design"]]
    return gen(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"], s)


def design_step(name_or_cfg, gam, seed, amp=0.02):
    """A synthetic optimiser step: gamma + amp * (box-filtered U[-1,1] noise) inside
    the design column, clipped to [0, 1] (the next design of an optimisation run,
    whose state solve is warm-started from the current one)."""
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    nx, ny, nz, h = cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"]
    rng = np.random.default_rng(seed)
    d = box_filter3(rng.uniform(-1.0, 1.0, size=(nz, ny, nx))).ravel()
    col = (quarter_regions(nx, ny, nz, h)[1] if cfg.get("bcs") == "quarter"
           else design_column(nx, ny, nz, h))
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
