"""Plain FP64 CPU oracle of the SIMP state solve, compliance and sensitivities.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
(and its `--impl reference` arm) use it.  It shares no code with the CUDA
library; the only common module is the seeded input generator.

What it computes, step by step, in the paper's notation (arXiv 2605.04735):

  * E_e = Emin + rho_e^p (E0 - Emin)                       Sec. 2.1, Eq. (1)
  * k_e = E_e k0_e, K(rho) = sum_e k_e (assembled), K U = F Sec. 2.1.1, Eq. (2)
  * J = U^T K U = sum_e u_e^T k_e u_e  (compliance)        Sec. 2.1.1, Eq. (2)
  * dJ/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e    Sec. 2.1.2, Eq. (3)

The paper names k0 (the element matrix for unit Young's modulus) but not the
element formulation; the reading used here is the standard trilinear 8-node
brick with full 2x2x2 Gauss-Legendre integration of B^T D B, isotropic D with
(E = 1, nu), Voigt order (xx, yy, zz, yz, xz, xy) and engineering shear
strains.  The paper's setup (Sec. 4.1) uses a structured hexahedral mesh,
E0 = 1, nu = 0.3, p = 3.  It does not say how K U = F is solved; the oracle
solves it directly (Cholesky of the assembled free-free block), which is the
definition of the exact discrete solution every iterative solver approaches.

Mesh conventions: nodes (i, j, k), 0 <= i <= nx etc., at (i, j, k) * h;
node n = i + (nx+1) (j + (ny+1) k); DOF = 3 n + c (c = x, y, z);
element e = i + nx (j + ny k) with local node order
(0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

LOCAL_NODES = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                        [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)

BC_CANTILEVER, BC_MBB, BC_ROLLER_BOX, BC_CORNERS, BC_MBB_STRIP = 0, 1, 2, 3, 4
LOAD_EDGE_XL_BOTTOM, LOAD_EDGE_X0_TOP, LOAD_FACE_XL_TRACTION = 0, 1, 2
LOAD_DISC_XL, LOAD_HALFDISC_X0_TOP = 3, 4

# The paper's test problems (Sec. 4.2, 4.3) on a 2 x 1 x 1 domain: supports and
# load regions in units of the unit cross-section edge (ny elements).
CORNER_FRACTION = 0.3   # corner support squares, 0.3 x 0.3 (Sec. 4.2)
DISC_FRACTION = 0.1     # load disc / half-disc radius 0.1 (Sec. 4.2, 4.3)


# --------------------------------------------------------------------------
# Element matrix k0 (Sec. 2.1.2: "element stiffness matrix for unit Young's
# modulus"); trilinear brick, Gauss-Legendre quadrature.
# --------------------------------------------------------------------------
def lame(E: float, nu: float):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def constitutive_matrix(E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """Isotropic 6x6 D in Voigt order (xx, yy, zz, yz, xz, xy), engineering shear."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_gradients(xi: float, eta: float, zeta: float) -> np.ndarray:
    """dN_a/d(xi, eta, zeta) for the 8 trilinear shape functions, shape (8, 3)."""
    s = 2.0 * LOCAL_NODES - 1.0            # node coordinates in [-1, 1]^3
    g = np.empty((8, 3))
    for a in range(8):
        sa, ta, ua = s[a]
        g[a, 0] = sa * (1 + eta * ta) * (1 + zeta * ua) / 8.0
        g[a, 1] = ta * (1 + xi * sa) * (1 + zeta * ua) / 8.0
        g[a, 2] = ua * (1 + xi * sa) * (1 + eta * ta) / 8.0
    return g


def strain_displacement(dNdx: np.ndarray) -> np.ndarray:
    """B (6 x 24) mapping u_e = [u_x, u_y, u_z per local node] to Voigt strain."""
    B = np.zeros((6, 24))
    for a in range(8):
        nx_, ny_, nz_ = dNdx[a]
        c = 3 * a
        B[0, c + 0] = nx_
        B[1, c + 1] = ny_
        B[2, c + 2] = nz_
        B[3, c + 1] = nz_
        B[3, c + 2] = ny_
        B[4, c + 0] = nz_
        B[4, c + 2] = nx_
        B[5, c + 0] = ny_
        B[5, c + 1] = nx_
    return B


def element_stiffness(h: float = 1.0, nu: float = 0.3, E: float = 1.0, ngauss: int = 2) -> np.ndarray:
    """k0 = integral over the cube [0, h]^3 of B^T D B, by ngauss^3 Gauss points."""
    pts, wts = np.polynomial.legendre.leggauss(ngauss)
    D = constitutive_matrix(E, nu)
    jac = h / 2.0                      # x = (xi + 1) h / 2 in each direction
    detJ = jac ** 3
    K = np.zeros((24, 24))
    for a, wa in zip(pts, wts):
        for b, wb in zip(pts, wts):
            for c, wc in zip(pts, wts):
                dN = shape_gradients(a, b, c) / jac
                B = strain_displacement(dN)
                K += wa * wb * wc * detJ * (B.T @ D @ B)
    return K


def rigid_body_modes(h: float = 1.0) -> np.ndarray:
    """The 6 rigid motions (3 translations, 3 infinitesimal rotations) of one element, (24, 6)."""
    X = LOCAL_NODES * h
    R = np.zeros((24, 6))
    for a in range(8):
        x, y, z = X[a]
        R[3 * a:3 * a + 3, 0] = [1, 0, 0]
        R[3 * a:3 * a + 3, 1] = [0, 1, 0]
        R[3 * a:3 * a + 3, 2] = [0, 0, 1]
        R[3 * a:3 * a + 3, 3] = [0, -z, y]    # rotation about x
        R[3 * a:3 * a + 3, 4] = [z, 0, -x]    # rotation about y
        R[3 * a:3 * a + 3, 5] = [-y, x, 0]    # rotation about z
    return R


# --------------------------------------------------------------------------
# Structured mesh, boundary conditions and loads
# --------------------------------------------------------------------------
class Grid:
    def __init__(self, nx: int, ny: int, nz: int, h: float = 1.0):
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    def node(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def node_ijk(self):
        """(n_nodes, 3) integer coordinates of every node, in node order."""
        k, j, i = np.meshgrid(np.arange(self.nz + 1), np.arange(self.ny + 1),
                              np.arange(self.nx + 1), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def element_ijk(self):
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                              indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def element_nodes(self) -> np.ndarray:
        """(n_elem, 8) global node numbers in the local order."""
        e = self.element_ijk()
        cols = []
        for a in range(8):
            d = LOCAL_NODES[a]
            cols.append(self.node(e[:, 0] + d[0], e[:, 1] + d[1], e[:, 2] + d[2]))
        return np.stack(cols, axis=1)

    def element_dofs(self) -> np.ndarray:
        """(n_elem, 24) global DOF numbers: [3 n_a + c] for a = 0..7, c = 0..2."""
        en = self.element_nodes()
        return (3 * en[:, :, None] + np.arange(3)[None, None, :]).reshape(self.n_elem, 24)


def fixed_dofs(grid: Grid, bc: int) -> np.ndarray:
    """Boolean mask over DOFs that the boundary condition holds at zero.

    Cantilever: every component on the face x = 0.
    MBB half-beam: u_x on x = 0 (symmetry), u_z on the line x = L, z = 0
    (roller), plus u_y at the single node (L, ny/2, 0): the roller and the
    symmetry plane leave the y translation free, which makes K singular, and
    pinning one node removes only that rigid motion (no strain, no load work).
    Roller box (test problem): u_x on x = 0, u_y on y = 0, u_z on z = 0.
    """
    ijk = grid.node_ijk()
    i, j, k = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    m = np.zeros((grid.n_nodes, 3), dtype=bool)
    if bc == BC_CANTILEVER:
        m[i == 0, :] = True
    elif bc == BC_MBB:
        if grid.ny % 2:
            raise ValueError("MBB needs an even ny for the y pin")
        m[i == 0, 0] = True
        m[(i == grid.nx) & (k == 0), 2] = True
        m[(i == grid.nx) & (k == 0) & (j == grid.ny // 2), 1] = True
    elif bc == BC_ROLLER_BOX:
        m[i == 0, 0] = True
        m[j == 0, 1] = True
        m[k == 0, 2] = True
    elif bc == BC_CORNERS:
        # Sec. 4.2: x = 0 face fixed on four 0.3 x 0.3 corner squares (in units of
        # the cross-section edge: ny and nz elements span 1.0)
        cj = int(np.floor(CORNER_FRACTION * grid.ny + 1e-9))
        ck = int(np.floor(CORNER_FRACTION * grid.nz + 1e-9))
        in_j = (j <= cj) | (j >= grid.ny - cj)
        in_k = (k <= ck) | (k >= grid.nz - ck)
        m[(i == 0) & in_j & in_k, :] = True
    elif bc == BC_MBB_STRIP:
        # Sec. 4.3: u_x = 0 on x = 0; u_z = 0 on the bottom strip of one element at
        # x = L; plus the same single u_y pin as BC_MBB (rigid y translation)
        if grid.ny % 2:
            raise ValueError("MBB needs an even ny for the y pin")
        m[i == 0, 0] = True
        m[(i >= grid.nx - 1) & (k == 0), 2] = True
        m[(i == grid.nx) & (k == 0) & (j == grid.ny // 2), 1] = True
    else:
        raise ValueError(bc)
    return m.reshape(-1)


def load_vector(grid: Grid, load: int, magnitude: float = 1.0) -> np.ndarray:
    """Consistent nodal forces.

    Edge loads: a total force `magnitude` in -z spread uniformly along a line
    of ny segments of length h; each segment sends half of its share to each
    end node (interior nodes magnitude/ny, the two ends magnitude/(2 ny)).
    Face traction: uniform traction `magnitude` in +x on x = L; each face quad
    (area h^2) sends a quarter of its force to each of its four nodes.
    """
    f = np.zeros((grid.n_nodes, 3))
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    if load in (LOAD_EDGE_XL_BOTTOM, LOAD_EDGE_X0_TOP):
        i, k = (nx, 0) if load == LOAD_EDGE_XL_BOTTOM else (0, nz)
        for s in range(ny):                       # segment between j = s and s + 1
            share = magnitude / ny
            f[grid.node(i, s, k), 2] -= share / 2.0
            f[grid.node(i, s + 1, k), 2] -= share / 2.0
    elif load == LOAD_FACE_XL_TRACTION:
        for k in range(nz):
            for j in range(ny):
                fq = magnitude * h * h / 4.0
                for dj, dk in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    f[grid.node(nx, j + dj, k + dk), 0] += fq
    elif load in (LOAD_DISC_XL, LOAD_HALFDISC_X0_TOP):
        # total `magnitude` in -z as a uniform traction on the face quads whose
        # centroids lie in the disc (Sec. 4.2: radius 0.1 about the centre of
        # x = L) or half-disc (Sec. 4.3: radius 0.1 about (0, 0.5, 1) on the top
        # face); each quad sends a quarter of its share to each corner
        rad = DISC_FRACTION * ny
        quads = []
        if load == LOAD_DISC_XL:
            for k in range(nz):
                for j in range(ny):
                    if (j + 0.5 - ny / 2.0) ** 2 + (k + 0.5 - nz / 2.0) ** 2 <= rad * rad:
                        quads.append([grid.node(nx, j + a, k + b) for a, b in
                                      ((0, 0), (1, 0), (1, 1), (0, 1))])
        else:
            for j in range(ny):
                for i in range(nx):
                    if (i + 0.5) ** 2 + (j + 0.5 - ny / 2.0) ** 2 <= rad * rad:
                        quads.append([grid.node(i + a, j + b, nz) for a, b in
                                      ((0, 0), (1, 0), (1, 1), (0, 1))])
        if not quads:
            raise ValueError("load region holds no face quad")
        share = magnitude / len(quads) / 4.0
        for q in quads:
            for nd in q:
                f[nd, 2] -= share
    else:
        raise ValueError(load)
    return f.reshape(-1)


# --------------------------------------------------------------------------
# SIMP interpolation, assembly, solve (Sec. 2.1, Eqs. (1)-(2))
# --------------------------------------------------------------------------
def simp_modulus(rho: np.ndarray, E0: float = 1.0, Emin: float = 1e-9, p: float = 3.0) -> np.ndarray:
    """Eq. (1): E_e = Emin + rho_e^p (E0 - Emin), in FP64."""
    r = np.asarray(rho, dtype=np.float64)
    return Emin + r ** p * (E0 - Emin)


def assemble(grid: Grid, E: np.ndarray, k0: np.ndarray) -> sp.csr_matrix:
    """K = sum_e E_e k0 scattered by element DOFs (all DOFs, no BC applied)."""
    ed = grid.element_dofs()
    rows = np.repeat(ed, 24, axis=1).ravel()
    cols = np.tile(ed, (1, 24)).ravel()
    vals = (E[:, None] * k0.ravel()[None, :]).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(grid.n_dof, grid.n_dof)).tocsr()
    K.sum_duplicates()
    return K


def x_outer_permutation(grid: Grid) -> np.ndarray:
    """DOF permutation with the x index slowest: keeps the band of K narrow
    (about 3 (ny+1)(nz+1)) for beams that are long in x."""
    ijk = grid.node_ijk()
    key = ijk[:, 2] + (grid.nz + 1) * (ijk[:, 1] + (grid.ny + 1) * ijk[:, 0])
    node_order = np.argsort(key, kind="stable")
    return (3 * node_order[:, None] + np.arange(3)[None, :]).reshape(-1)


def solve_direct(K: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray, grid: Grid | None = None,
                 dense_limit: int = 3000) -> np.ndarray:
    """u with u = 0 on fixed DOFs and K_ff u_f = f_f solved by Cholesky.

    Small systems: dense Cholesky (LAPACK potrf).  Larger ones: banded
    Cholesky (LAPACK pbtrf) of K_ff in the x-outermost DOF order.
    """
    free = np.flatnonzero(~fixed)
    if grid is not None and free.size > dense_limit:
        perm = x_outer_permutation(grid)
        perm = perm[~fixed[perm]]
        A = K[perm][:, perm].tocoo()
        lower = A.row >= A.col
        r, c, v = A.row[lower], A.col[lower], A.data[lower]
        bw = int((r - c).max())
        ab = np.zeros((bw + 1, perm.size))
        ab[r - c, c] = v
        cb = sla.cholesky_banded(ab, lower=True, overwrite_ab=True, check_finite=False)
        x = sla.cho_solve_banded((cb, True), f[perm], check_finite=False)
        u = np.zeros_like(f)
        u[perm] = x
        return u
    A = K[free][:, free].toarray()
    c = sla.cho_factor(A, lower=True, check_finite=False)
    u = np.zeros_like(f)
    u[free] = sla.cho_solve(c, f[free], check_finite=False)
    return u


def solve_cg(K: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray, rtol: float = 1e-12,
             maxiter: int = 200000) -> np.ndarray:
    """Independent check: Jacobi-preconditioned CG (scipy) on K_ff."""
    free = np.flatnonzero(~fixed)
    A = K[free][:, free].tocsr()
    d = A.diagonal()
    M = sp.diags(1.0 / d)
    x, info = spla.cg(A, f[free], rtol=rtol, atol=0.0, maxiter=maxiter, M=M)
    if info != 0:
        raise RuntimeError(f"CG did not converge (info={info})")
    u = np.zeros_like(f)
    u[free] = x
    return u


def residual(K: sp.csr_matrix, f: np.ndarray, u: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """r = f - K u restricted to free DOFs (fixed entries set to 0)."""
    r = f - K @ u
    r[fixed] = 0.0
    return r


# --------------------------------------------------------------------------
# Compliance and sensitivities (Sec. 2.1.1 Eq. (2), Sec. 2.1.2 Eq. (3))
# --------------------------------------------------------------------------
def element_energies(grid: Grid, u: np.ndarray, k0: np.ndarray) -> np.ndarray:
    """u_e^T k0 u_e for every element."""
    ue = u[grid.element_dofs()]
    return np.einsum("ei,ij,ej->e", ue, k0, ue)


def compliance(f: np.ndarray, u: np.ndarray) -> float:
    """J = F^T U (equal to U^T K U at equilibrium)."""
    return float(f @ u)


def compliance_energy(grid: Grid, u: np.ndarray, E: np.ndarray, k0: np.ndarray) -> float:
    """J = sum_e u_e^T k_e u_e with k_e = E_e k0 (Eq. (2), right-hand form)."""
    return float(E @ element_energies(grid, u, k0))


def sensitivity(grid: Grid, u: np.ndarray, rho: np.ndarray, k0: np.ndarray, E0: float = 1.0,
                Emin: float = 1e-9, p: float = 3.0) -> np.ndarray:
    """Eq. (3): dJ/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T k0 u_e."""
    r = np.asarray(rho, dtype=np.float64)
    return -p * r ** (p - 1.0) * (E0 - Emin) * element_energies(grid, u, k0)


# --------------------------------------------------------------------------
# Matrix-free checks for grids too large to assemble: (K u) at chosen nodes,
# computed one node at a time from the elements around it.
# --------------------------------------------------------------------------
def apply_at_nodes(grid: Grid, E: np.ndarray, k0: np.ndarray, u: np.ndarray,
                   nodes: np.ndarray) -> np.ndarray:
    """(K u) restricted to the listed nodes, shape (len(nodes), 3); no BC applied."""
    out = np.zeros((len(nodes), 3))
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    for t, n in enumerate(nodes):
        i = n % (nx + 1)
        j = (n // (nx + 1)) % (ny + 1)
        k = n // ((nx + 1) * (ny + 1))
        for a in range(8):                         # element whose local node a is n
            ei, ej, ek = i - LOCAL_NODES[a, 0], j - LOCAL_NODES[a, 1], k - LOCAL_NODES[a, 2]
            if not (0 <= ei < nx and 0 <= ej < ny and 0 <= ek < nz):
                continue
            e = ei + nx * (ej + ny * ek)
            nodes_e = [grid.node(ei + d[0], ej + d[1], ek + d[2]) for d in LOCAL_NODES]
            ue = np.concatenate([u[3 * m:3 * m + 3] for m in nodes_e])
            out[t] += E[e] * (k0[3 * a:3 * a + 3] @ ue)
    return out


def element_energies_at(grid: Grid, u: np.ndarray, k0: np.ndarray, elems: np.ndarray) -> np.ndarray:
    """u_e^T k0 u_e for the listed elements only."""
    nx, ny = grid.nx, grid.ny
    out = np.zeros(len(elems))
    for t, e in enumerate(elems):
        i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
        nodes_e = [grid.node(i + d[0], j + d[1], k + d[2]) for d in LOCAL_NODES]
        ue = np.concatenate([u[3 * m:3 * m + 3] for m in nodes_e])
        out[t] = ue @ k0 @ ue
    return out


# --------------------------------------------------------------------------
# One full oracle solve of a problem
# --------------------------------------------------------------------------
class Problem:
    """An assembled FP64 problem: grid, BC, load, densities -> K, f, fixed mask."""

    def __init__(self, nx, ny, nz, bc, load, rho, E0=1.0, Emin=1e-9, nu=0.3, p=3.0, h=1.0,
                 load_magnitude=1.0):
        self.grid = Grid(nx, ny, nz, h)
        self.E0, self.Emin, self.nu, self.p = E0, Emin, nu, p
        self.rho = np.asarray(rho, dtype=np.float64)
        self.k0 = element_stiffness(h, nu)
        self.E = simp_modulus(self.rho, E0, Emin, p)
        self.K = assemble(self.grid, self.E, self.k0)
        self.f = load_vector(self.grid, load, load_magnitude)
        self.fixed = fixed_dofs(self.grid, bc)
        self.f[self.fixed] = 0.0

    def solve(self) -> np.ndarray:
        return solve_direct(self.K, self.f, self.fixed, self.grid)

    def compliance(self, u):
        return compliance(self.f, u)

    def sensitivity(self, u):
        return sensitivity(self.grid, u, self.rho, self.k0, self.E0, self.Emin, self.p)

    def rel_residual(self, u) -> float:
        r = residual(self.K, self.f, u, self.fixed)
        return float(np.linalg.norm(r) / np.linalg.norm(self.f))
