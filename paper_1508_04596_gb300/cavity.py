"""Regions of the cavity problems: where the design variables, the heat source
and the passive solid sit.

* The paper's set-up (Sec. 6.1): a closed unit cavity with a heat-source block
  of solid material (0.1 wide, 0.05 high, s0 = 1e4) at the middle of the bottom
  and a 0.75 x 0.75 x 0.75 design domain on top of it, volume fraction 5 %;
  by symmetry only a quarter is computed.  Here the vertical is z and the
  quarter's symmetry planes are the faces x = nx h and y = ny h, so both blocks
  sit against those faces.
* The benchmark cavities (a heated patch of the bottom, no source block): the
  design column is the set of elements whose centroid has x, y in
  [0.25, 0.75] L and z in [0, 0.75 Lz].

Element masks are boolean arrays over the elements in the library's order
e = i + nx (j + ny k).
"""
import numpy as np

# Quarter-cavity geometry (fractions of the full unit cavity): heat-source block
# 0.1 x 0.1 wide (half-width 0.05 in the quarter), 0.05 high; design domain 0.75 x
# 0.75 wide (half-width 0.375) and 0.75 high, sitting on top of the source block.
QUARTER = dict(source_half=0.05, source_height=0.05, design_half=0.375, design_height=0.75,
               s0=1e4, vf=0.05)


def elem_centroids(nx, ny, nz, h):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([(i.ravel() + 0.5) * h, (j.ravel() + 0.5) * h, (k.ravel() + 0.5) * h], 1)


def design_column(nx, ny, nz, h):
    """Design elements of the benchmark cavities: the central half-width column
    above the heated base, three quarters of the height."""
    c = elem_centroids(nx, ny, nz, h)
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    return ((c[:, 0] >= 0.25 * Lx) & (c[:, 0] <= 0.75 * Lx)
            & (c[:, 1] >= 0.25 * Ly) & (c[:, 1] <= 0.75 * Ly)
            & (c[:, 2] <= 0.75 * Lz))


def quarter_regions(nx, ny, nz, h):
    """Source-block and design-domain element masks of the quarter cavity
    (Sec. 6.1), whose symmetry planes are the faces x = nx h and y = ny h."""
    c = elem_centroids(nx, ny, nz, h)
    Lx, Ly = nx * h, ny * h
    q = QUARTER
    near = lambda half: (c[:, 0] >= Lx - half) & (c[:, 1] >= Ly - half)
    src = near(q["source_half"]) & (c[:, 2] <= q["source_height"])
    des = (near(q["design_half"]) & (c[:, 2] > q["source_height"])
           & (c[:, 2] <= q["source_height"] + q["design_height"]))
    return src, des


def source(nx, ny, nz, h, quarter):
    """Element heat source s_e (Sec. 2): s0 in the source block of the quarter
    cavity, zero elsewhere (and everywhere for the benchmark cavities)."""
    s = np.zeros(nx * ny * nz)
    if quarter:
        src, _ = quarter_regions(nx, ny, nz, h)
        s[src] = QUARTER["s0"]
    return s


def design_regions(nx, ny, nz, h, quarter):
    """(active design elements, values of the passive elements): the source block
    is solid (gamma = 0), every other passive element fluid (gamma = 1)."""
    if quarter:
        src, des = quarter_regions(nx, ny, nz, h)
    else:
        src, des = np.zeros(nx * ny * nz, bool), design_column(nx, ny, nz, h)
    fixed = np.ones(nx * ny * nz)
    fixed[src] = 0.0
    return des, fixed
