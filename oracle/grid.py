"""Structured hexahedral grid and boundary conditions (oracle; test infrastructure only).

Grid (Sec. 4, Sec. 6.1): ``nx x ny x nz`` cubic trilinear elements of edge ``h``
on the box ``[0, nx h] x [0, ny h] x [0, nz h]``; z is vertical.  Five unknowns
per node, (u, v, w, p, T), on every node including Dirichlet ones (the DOF counts
of Sec. 6.3/6.4, 41,603,205 = 5*161*321*161, are reproduced that way).

Numbering (row-major, x fastest):
  node    n = i + (nx+1) * (j + (ny+1) * k)
  element e = i + nx * (j + ny * k)
  local node a = ia + 2 ja + 4 ka  of element (i,j,k) is node (i+ia, j+ja, k+ka)
  global unknown of field f at node n: f * Nn + n   (structure of arrays)

Boundary conditions (readings of Sec. 6.1 and of the benchmark set-up):
  velocity per face: NOSLIP (all 3 components 0), FREE (traction-free, natural),
                     SYMMETRY (normal component 0)
  temperature per face: ADIABATIC (natural) or DIRICHLET(value)
  a rectangular patch on the bottom face (z = 0), closed interval in x and y
  with tolerance 1e-12 * L, either DIRICHLET(value) or FLUX(q into the domain)
  on the bottom faces whose four nodes all lie in the patch.
  Precedence of Dirichlet temperature values on shared nodes:
  -x, +x, -y, +y faces first (in that order), then the patch, then -z, then +z.
  Dirichlet always wins over natural conditions.
  Optionally one pressure node is pinned (closed cavities).
"""
import numpy as np

NOSLIP, FREE, SYMMETRY = 0, 1, 2
ADIABATIC, DIRICHLET = 0, 1
PATCH_NONE, PATCH_DIRICHLET, PATCH_FLUX = 0, 1, 2
NF = 5  # u, v, w, p, T


class Grid:
    def __init__(self, nx, ny, nz, h):
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.Nn = (nx + 1) * (ny + 1) * (nz + 1)
        self.E = nx * ny * nz
        self.ndof = NF * self.Nn
        self.L = np.array([nx * h, ny * h, nz * h])

    def node(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def node_ijk(self):
        """Integer (i, j, k) of every node, shape [Nn, 3]."""
        k, j, i = np.meshgrid(np.arange(self.nz + 1), np.arange(self.ny + 1),
                              np.arange(self.nx + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def node_xyz(self):
        return self.node_ijk() * self.h

    def elem_ijk(self):
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny),
                              np.arange(self.nx), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def connectivity(self):
        """Global node of local node a of every element, shape [E, 8]."""
        eijk = self.elem_ijk()
        conn = np.empty((self.E, 8), dtype=np.int64)
        for a in range(8):
            ia, ja, ka = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn[:, a] = self.node(eijk[:, 0] + ia, eijk[:, 1] + ja, eijk[:, 2] + ka)
        return conn

    def elem_centroids(self):
        return (self.elem_ijk() + 0.5) * self.h


class BCs:
    """Face boundary conditions of the cavity set-up (reading of Sec. 6.1)."""

    def __init__(self, vel_bc=(NOSLIP, NOSLIP, NOSLIP, NOSLIP, NOSLIP, FREE),
                 T_bc=(DIRICHLET, DIRICHLET, DIRICHLET, DIRICHLET, ADIABATIC, DIRICHLET),
                 T_val=(0.0, 0.0, 0.0, 0.0, 0.0, 0.0),
                 patch=(1.0 / 3, 2.0 / 3, 1.0 / 3, 2.0 / 3),
                 patch_mode=PATCH_DIRICHLET, patch_val=1.0, p_pin=-1):
        self.vel_bc = tuple(vel_bc)
        self.T_bc = tuple(T_bc)
        self.T_val = tuple(float(t) for t in T_val)
        self.patch = tuple(float(p) for p in patch)  # fractions of Lx, Ly
        self.patch_mode = int(patch_mode)
        self.patch_val = float(patch_val)
        self.p_pin = int(p_pin)


def _on_faces(g):
    ijk = g.node_ijk()
    n = [g.nx, g.ny, g.nz]
    faces = []
    for d in range(3):
        faces.append(ijk[:, d] == 0)
        faces.append(ijk[:, d] == n[d])
    return faces  # -x, +x, -y, +y, -z, +z


def patch_nodes(g, bc):
    """Bottom-face nodes inside the closed patch rectangle (tolerance 1e-12 L)."""
    xyz = g.node_xyz()
    tol = 1e-12 * max(g.L)
    x0, x1 = bc.patch[0] * g.L[0], bc.patch[1] * g.L[0]
    y0, y1 = bc.patch[2] * g.L[1], bc.patch[3] * g.L[1]
    return ((g.node_ijk()[:, 2] == 0)
            & (xyz[:, 0] >= x0 - tol) & (xyz[:, 0] <= x1 + tol)
            & (xyz[:, 1] >= y0 - tol) & (xyz[:, 1] <= y1 + tol))


def dirichlet(g, bc):
    """Dirichlet mask [5, Nn] (bool) and prescribed values [5, Nn]."""
    faces = _on_faces(g)
    mask = np.zeros((NF, g.Nn), dtype=bool)
    val = np.zeros((NF, g.Nn))
    for f, on in enumerate(faces):
        d = f // 2
        if bc.vel_bc[f] == NOSLIP:
            mask[0:3, on] = True
        elif bc.vel_bc[f] == SYMMETRY:
            mask[d, on] = True
    # temperature, in precedence order: the first Dirichlet source to claim a node wins
    claimed = np.zeros(g.Nn, dtype=bool)

    def claim(sel, value):
        new = sel & ~claimed
        mask[4, new] = True
        val[4, new] = value
        claimed[new] = True

    for f in range(4):
        if bc.T_bc[f] == DIRICHLET:
            claim(faces[f], bc.T_val[f])
    if bc.patch_mode == PATCH_DIRICHLET:
        claim(patch_nodes(g, bc), bc.patch_val)
    for f in (4, 5):
        if bc.T_bc[f] == DIRICHLET:
            claim(faces[f], bc.T_val[f])
    if bc.p_pin >= 0:
        mask[3, bc.p_pin] = True
    return mask, val


def patch_faces(g, bc):
    """Element ids whose bottom face (local nodes 0..3) lies entirely in the patch."""
    inpatch = patch_nodes(g, bc)
    conn = g.connectivity()
    bottom = g.elem_ijk()[:, 2] == 0
    allin = inpatch[conn[:, 0]] & inpatch[conn[:, 1]] & inpatch[conn[:, 2]] & inpatch[conn[:, 3]]
    return np.nonzero(bottom & allin)[0]


def neumann_rhs(g, bc):
    """The flux term  -int_{Gamma_q} N_a q dA  of the energy rows, as a [5, Nn] array.

    Each patch face is a square of side h; 2x2 Gauss integrates the bilinear
    N_a exactly, giving h^2/4 at each of its four nodes."""
    out = np.zeros((NF, g.Nn))
    if bc.patch_mode != PATCH_FLUX:
        return out
    conn = g.connectivity()
    for e in patch_faces(g, bc):
        for a in range(4):
            out[4, conn[e, a]] -= bc.patch_val * g.h * g.h / 4.0
    return out
