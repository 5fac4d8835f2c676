"""Plain FP64 CPU oracle for the guarded floor-selection state solve.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It shares no code with
the CUDA library (it imports nothing from the package, and the package imports
nothing from here); it is slow on purpose and written to be checked against the
paper by eye.

Every function is in FP64 and names the passage it follows (paper arXiv
2607.26382, sections / equations / algorithm by their labels):

* mesh, DOF numbering, clamped face, tip load ........ Sec. 3.1 "Discretization",
  Table "geometries" (cantilever: x=0 face fixed, unit point load at the tip centre)
* hex8 element stiffness K0 (E0=1, nu=0.3, 2x2x2 Gauss)  Sec. 3.1 "Discretization"
* floor scaling E_e = rho_min + (1-rho_min) rho^p ....... Eq. (floor_scaling)
* frozen operator K = sum_e E_e K_e on free DOFs ........ Eq. (frozen_operator)
* relative residual eta = ||f - K u|| / ||f|| ........... Eq. (relative_residual)
* GMG V-cycle, 2:1 trilinear transfer ................... Table "solver-config"
* line-searched, rejectable coarse correction ......... Table "solver-config" (coarse correction)
* Chebyshev smoother (alternative to node-block Jacobi) . Table "solver-config" (names a
  Chebyshev smoother; degree and interval are readings, see below)
* right-preconditioned FGMRES, residual history ......... Sec. 3.2 "Which residual
  counts", Table "residual-semantics", Sec. 3.5 "Why a flexible Krylov method"
* probe features r50/r100 and trigger rule .............. Sec. 3.4, Eq. (trigger)
* guarded policy ........................................ Algorithm 1 (floor_policy)
* conditioning diagnostic kappa, direct residual, screen  Sec. 4.1.3 (Figure conditioning)
* true-residual checks during the probe, their detector . Sec. 4.1.1 (the checkpointed
  variant the paper leaves untested; the detector is a reading, see below)
* compliance and sensitivity ............................ Sec. 3.1 (after Eq. projection)

Readings where the paper is silent (the CUDA side takes the same ones):
coarse levels are rediscretised with the mean of the 8 child moduli (the paper's
Galerkin operators P^T K P are available as coarse="galerkin", to compare the two);
restriction is the transpose of trilinear prolongation, both masked;
damped 3x3 node-block Jacobi (the node-block operator of Table solver-config) with
omega=0.6, 2 pre + 2 post sweeps from x=0 (point Jacobi at omega=0.6 is unstable on
high-contrast fields: omega*lambda_max(D^-1 K) exceeds 2); coarsest level is a
dense Cholesky solve on free DOFs; FGMRES uses classical Gram-Schmidt with one
re-orthogonalisation; a cycle-start true residual overwrites the history entry
at that iteration count; happy breakdown when h_{j+1,j} <= 1e-14 * ||K z_j||.
Chebyshev smoothing (optional): Chebyshev semi-iteration of degree nu1 / nu2 on
D_b^{-1} K over [lambda_max / 30, 1.1 lambda_max], D_b the same 3x3 node blocks;
lambda_max of each level from 15 power iterations started from the all-ones vector
on free DOFs.
Line-searched coarse correction (optional, ls_ratio = theta > 0; the first adaptive
component of Table solver-config, step and acceptance test readings): the prolongated
correction c is scaled by the energy-optimal alpha = (c.r)/(c.K c), computed from the
residual, and dropped unless alpha >= theta. (Minimising ||r - alpha K c|| instead, or
rejecting on the residual norm before post-smoothing, cripples this V-cycle: measured.)
Fine-level adaptive correction (optional, fine_steps > 0; Table solver-config): after
the V-cycle, fine_steps steps of an inner FGMRES(fine_steps) on the fine-level residual
equation, preconditioned by the node-block Jacobi operator, applied only if it lowers
the recomputed residual norm.
Coarse-level inner Krylov solve (optional, coarse_steps > 0; Table solver-config's "10
inner Krylov steps with restart 10 on the coarse level"): the coarsest level of a
hierarchy with two or more levels is solved by coarse_steps steps of an inner
FGMRES(coarse_steps) from 0, preconditioned by its node-block Jacobi operator, instead
of exactly (reading: the coarse level is the coarsest one, the inner preconditioner the
one the fine-level correction uses).
True-residual checks (optional): every c steps of the probe the current iterate is
formed as at a cycle end and its guard residual recomputed; the detector fires when
one exceeds ratio (default 10) times the projected estimate of the same step, and a
firing detector escalates like Eq. (trigger).

Bridge geometry (Table geometries; oracle only, the CUDA path keeps the clamped face):
BridgeMesh fixes every DOF of the nodes (0, 0, z) and y, z of the nodes (x_max, 0, z) for
z in {0, Lz/2, Lz}; bridge_load is a unit pressure on the top face as consistent nodal
forces. Coarse meshes inherit their fixed sets by injection (Mesh.coarsen).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force on tiny grids, paper values). None is
"parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# Local node order of a hex8 element (offsets in x, y, z): bottom face
# counter-clockwise, then top face counter-clockwise.
LOCAL_NODES = ((0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
               (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1))

# FGMRES stop flags
CONVERGED = 0      # projected (or cycle-start true) residual <= tol
MAX_ITERS = 1      # budget k_max reached
BREAKDOWN = 2      # h_{j+1,j} ~ 0 without convergence

# Policy outcomes (Algorithm 1)
ACCEPTED = 0
NO_ADMISSIBLE_FLOOR = 1


# ----------------------------------------------------------------------------
# a1: mesh, DOFs, mask, load (Sec. 3.1, Table geometries)
# ----------------------------------------------------------------------------
class Mesh:
    """Structured nx*ny*nz grid of cubic hex8 elements with edge h.

    node n(i,j,k) = i + (nx+1)*(j + (ny+1)*k); DOF 3n+c, c in {x,y,z};
    element e = ex + nx*(ey + ny*ez). Cantilever support: every DOF of the
    nodes on the x=0 face is fixed.
    """

    def __init__(self, nx: int, ny: int, nz: int, h: float = 1.0):
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
        self.n_dof = 3 * self.n_nodes
        self.n_elem = nx * ny * nz
        ex, ey, ez = self._element_coords()
        conn = np.empty((self.n_elem, 8), dtype=np.int64)
        for a, (ox, oy, oz) in enumerate(LOCAL_NODES):
            conn[:, a] = self.node(ex + ox, ey + oy, ez + oz)
        self.conn = conn
        edof = np.empty((self.n_elem, 24), dtype=np.int64)
        for a in range(8):
            for c in range(3):
                edof[:, 3 * a + c] = 3 * conn[:, a] + c
        self.edof = edof
        i = np.arange(self.n_nodes) % (nx + 1)
        fixed_node = i == 0
        self.fixed = np.repeat(fixed_node, 3)
        self.free = ~self.fixed

    def node(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def coarsen(self) -> "Mesh":
        """The 2:1 coarser mesh (edge 2h). Its fixed set is the fine one injected: coarse
        node (I, J, K) fixes component c iff fine node (2I, 2J, 2K) does (for the clamped
        face this is again every DOF of the x = 0 nodes)."""
        mc = Mesh(self.nx // 2, self.ny // 2, self.nz // 2, self.h * 2.0)
        n = np.arange(mc.n_nodes)
        I, J, K = n % (mc.nx + 1), (n // (mc.nx + 1)) % (mc.ny + 1), n // ((mc.nx + 1) * (mc.ny + 1))
        fine = self.node(2 * I, 2 * J, 2 * K)
        mc.fixed = self.fixed.reshape(-1, 3)[fine].ravel().copy()
        mc.free = ~mc.fixed
        return mc

    def _element_coords(self):
        e = np.arange(self.n_elem)
        ex = e % self.nx
        ey = (e // self.nx) % self.ny
        ez = e // (self.nx * self.ny)
        return ex, ey, ez

    def node_coords(self):
        n = np.arange(self.n_nodes)
        i = n % (self.nx + 1)
        j = (n // (self.nx + 1)) % (self.ny + 1)
        k = n // ((self.nx + 1) * (self.ny + 1))
        return i * self.h, j * self.h, k * self.h


class BridgeMesh(Mesh):
    """The paper's bridge geometry (Table geometries: a 3.0 x 1.0 x 0.5 box, y up): every
    DOF fixed at the nodes (0, 0, z) and rollers free in x at (x_max, 0, z), for z at the
    two faces and the mid-plane of the depth. Reading: the supports sit on nodes
    k in {0, nz/2, nz}, so nz is even (the paper's 90x30x15 and 210x70x35 meshes put
    z = 0.25 between nodes). The x-extent carries no constraint (any nx)."""

    def __init__(self, nx: int, ny: int, nz: int, h: float = 1.0):
        if nz % 2:
            raise ValueError("bridge supports need even nz")
        super().__init__(nx, ny, nz, h)
        fixed = np.zeros(self.n_dof, dtype=bool)
        for k in (0, nz // 2, nz):
            n0, n1 = self.node(0, 0, k), self.node(nx, 0, k)
            fixed[3 * n0:3 * n0 + 3] = True        # fully fixed
            fixed[3 * n1 + 1:3 * n1 + 3] = True    # roller: y and z fixed, free in x
        self.fixed = fixed
        self.free = ~fixed


def bridge_load(mesh: Mesh, p: float = 1.0) -> np.ndarray:
    """Unit pressure on the top face y = ny h, pointing down (-y), as consistent nodal
    forces by tributary area (Sec. 3.1): each top face of area h^2 gives -p h^2 / 4 to
    each of its four corner nodes (bilinear face, uniform pressure)."""
    f = np.zeros(mesh.n_dof)
    ex, ez = np.meshgrid(np.arange(mesh.nx), np.arange(mesh.nz), indexing="ij")
    share = -p * mesh.h * mesh.h / 4.0
    for dx in (0, 1):
        for dz in (0, 1):
            nodes = mesh.node(ex + dx, mesh.ny, ez + dz).ravel()
            np.add.at(f, 3 * nodes + 1, share)
    f[mesh.fixed] = 0.0
    return f


def cantilever_load(mesh: Mesh) -> np.ndarray:
    """Unit point load in -z at the centre node of the free end x = nx*h.

    The paper's cantilever carries a unit point load at the centre of the free
    end with ||f|| = 1 (Sec. 3.1, Table geometries); the workloads here load in -z.
    """
    if mesh.ny % 2 or mesh.nz % 2:
        raise ValueError("cantilever load needs even ny and nz")
    f = np.zeros(mesh.n_dof)
    n = mesh.node(mesh.nx, mesh.ny // 2, mesh.nz // 2)
    f[3 * n + 2] = -1.0
    return f


# ----------------------------------------------------------------------------
# a2: hex8 element stiffness (Sec. 3.1 "Discretization")
# ----------------------------------------------------------------------------
def isotropic_D(E: float, nu: float) -> np.ndarray:
    """6x6 isotropic elasticity matrix, strain order (xx,yy,zz,xy,yz,zx), engineering shear."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] += 2.0 * mu
        D[3 + i, 3 + i] = mu
    return D


def strain_displacement(grad: np.ndarray) -> np.ndarray:
    """B (6x24) from the 8 shape-function gradients grad[a] = (dN/dx, dN/dy, dN/dz)."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = grad[a]
        B[0, 3 * a + 0] = gx
        B[1, 3 * a + 1] = gy
        B[2, 3 * a + 2] = gz
        B[3, 3 * a + 0] = gy
        B[3, 3 * a + 1] = gx
        B[4, 3 * a + 1] = gz
        B[4, 3 * a + 2] = gy
        B[5, 3 * a + 0] = gz
        B[5, 3 * a + 2] = gx
    return B


def element_stiffness(h: float = 1.0, E: float = 1.0, nu: float = 0.3, gauss: int = 2) -> np.ndarray:
    """K_e = integral over the cube [0,h]^3 of B^T D B, by gauss^3-point Gauss quadrature.

    Trilinear shape functions N_a = prod_d (1 + s_ad xi_d)/8 on the reference
    cube [-1,1]^3 with s_ad = +-1 from LOCAL_NODES; the map x = h(xi+1)/2 has
    Jacobian (h/2) I.
    """
    D = isotropic_D(E, nu)
    pts, wts = np.polynomial.legendre.leggauss(gauss)
    s = 2.0 * np.array(LOCAL_NODES, dtype=np.float64) - 1.0  # (8,3) signs
    K = np.zeros((24, 24))
    detJ = (h / 2.0) ** 3
    for a_, wa in zip(pts, wts):
        for b_, wb in zip(pts, wts):
            for c_, wc in zip(pts, wts):
                xi = np.array([a_, b_, c_])
                fac = 1.0 + s * xi[None, :]          # (8,3)
                dN = np.empty((8, 3))
                dN[:, 0] = s[:, 0] * fac[:, 1] * fac[:, 2] / 8.0
                dN[:, 1] = fac[:, 0] * s[:, 1] * fac[:, 2] / 8.0
                dN[:, 2] = fac[:, 0] * fac[:, 1] * s[:, 2] / 8.0
                grad = dN * (2.0 / h)
                B = strain_displacement(grad)
                K += wa * wb * wc * detJ * (B.T @ D @ B)
    return K


# ----------------------------------------------------------------------------
# a3: floor scaling (Eq. floor_scaling) and the level hierarchy
# ----------------------------------------------------------------------------
def young_modulus(rho_hat: np.ndarray, rho_min: float, p: float) -> np.ndarray:
    """E_e = rho_min + (1 - rho_min) * rho_hat_e^p  (E0 = 1).

    Integer p is evaluated by repeated multiplication, otherwise with pow.
    """
    rho_hat = np.asarray(rho_hat, dtype=np.float64)
    if float(p) == int(p) and p >= 1:
        rp = rho_hat.copy()
        for _ in range(int(p) - 1):
            rp = rp * rho_hat
    else:
        rp = np.power(rho_hat, p)
    return rho_min + (1.0 - rho_min) * rp


def coarsen_modulus(mesh: Mesh, E: np.ndarray) -> np.ndarray:
    """Coarse element modulus = arithmetic mean of its 8 children (rediscretisation)."""
    E3 = np.asarray(E).reshape(mesh.nz, mesh.ny, mesh.nx)
    s = np.zeros((mesh.nz // 2, mesh.ny // 2, mesh.nx // 2))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                s = s + E3[dz::2, dy::2, dx::2]
    return (s / 8.0).ravel()


# ----------------------------------------------------------------------------
# a4: matrix-free frozen operator (Eq. frozen_operator)
# ----------------------------------------------------------------------------
def apply_K(mesh: Mesh, E: np.ndarray, K0: np.ndarray, u: np.ndarray) -> np.ndarray:
    """y = M sum_e E_e P_e^T K0 P_e (M u); M zeroes the fixed DOFs.

    Element contributions are summed in element order (np.bincount accumulates
    in order of appearance).
    """
    um = np.where(mesh.fixed, 0.0, u)
    ue = um[mesh.edof]                              # (n_e, 24)
    ye = (ue @ K0.T) * np.asarray(E)[:, None]
    y = np.bincount(mesh.edof.ravel(), weights=ye.ravel(), minlength=mesh.n_dof)
    y[mesh.fixed] = 0.0
    return y


def apply_K_at_nodes(mesh: Mesh, E: np.ndarray, K0: np.ndarray, u: np.ndarray,
                     nodes) -> np.ndarray:
    """(K u) at the 3 DOFs of each listed node, one node at a time (for sampled checks)."""
    out = np.zeros((len(nodes), 3))
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    for t, n in enumerate(nodes):
        n = int(n)
        i = n % (nx + 1)
        j = (n // (nx + 1)) % (ny + 1)
        k = n // ((nx + 1) * (ny + 1))
        if mesh.fixed[3 * n:3 * n + 3].all():
            continue
        acc = np.zeros(3)
        for a, (ox, oy, oz) in enumerate(LOCAL_NODES):
            ex, ey, ez = i - ox, j - oy, k - oz
            if not (0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz):
                continue
            e = ex + nx * (ey + ny * ez)
            dofs = mesh.edof[e]
            ue = np.where(mesh.fixed[dofs], 0.0, u[dofs])
            acc += E[e] * (K0[3 * a:3 * a + 3, :] @ ue)
        out[t] = np.where(mesh.fixed[3 * n:3 * n + 3], 0.0, acc)
    return out


def assemble_sparse(mesh: Mesh, E: np.ndarray, K0: np.ndarray, constrained: bool = True):
    """Assembled sum_e E_e K_e (CSR); if constrained, fixed rows/cols are zeroed."""
    rows = np.repeat(mesh.edof, 24, axis=1).ravel()
    cols = np.tile(mesh.edof, (1, 24)).ravel()
    vals = (np.asarray(E)[:, None, None] * K0[None, :, :]).reshape(mesh.n_elem, -1).ravel()
    K = sp.coo_matrix((vals, (rows, cols)), shape=(mesh.n_dof, mesh.n_dof)).tocsr()
    if constrained:
        m = sp.diags(mesh.free.astype(np.float64))
        K = (m @ K @ m).tocsr()
    return K


def assemble_dense_free(mesh: Mesh, E: np.ndarray, K0: np.ndarray) -> np.ndarray:
    """Dense free-DOF operator, element by element."""
    K = np.zeros((mesh.n_dof, mesh.n_dof))
    for e in range(mesh.n_elem):
        d = mesh.edof[e]
        K[np.ix_(d, d)] += E[e] * K0
    f = mesh.free
    return K[np.ix_(f, f)]


def operator_diagonal(mesh: Mesh, E: np.ndarray, K0: np.ndarray) -> np.ndarray:
    """diag(K) scattered element by element; fixed DOFs get 1."""
    d = np.bincount(mesh.edof.ravel(),
                    weights=(np.asarray(E)[:, None] * np.diag(K0)[None, :]).ravel(),
                    minlength=mesh.n_dof)
    d[mesh.fixed] = 1.0
    return d


def node_block_diagonal(mesh: Mesh, E: np.ndarray, K0: np.ndarray) -> np.ndarray:
    """The 3x3 diagonal block of K at every node, (n_nodes, 3, 3), scattered element by
    element (the "3x3 node-block Jacobi operator" of Table solver-config). Fixed nodes
    get the identity."""
    Db = np.zeros((mesh.n_nodes, 3, 3))
    for a in range(8):
        blk = K0[3 * a:3 * a + 3, 3 * a:3 * a + 3]
        contrib = np.asarray(E)[:, None, None] * blk[None, :, :]
        for r in range(3):
            for c in range(3):
                Db[:, r, c] += np.bincount(mesh.conn[:, a], weights=contrib[:, r, c],
                                           minlength=mesh.n_nodes)
    return _mask_blocks(Db, mesh)


def _mask_blocks(Db: np.ndarray, mesh: Mesh) -> np.ndarray:
    """Node blocks of the constrained operator: fixed rows and columns become those of
    the identity (a fully fixed node gets I; a roller keeps only its free entries)."""
    m = (~mesh.fixed).reshape(-1, 3).astype(np.float64)
    Db = Db * m[:, :, None] * m[:, None, :]
    Db[:, np.arange(3), np.arange(3)] += 1.0 - m
    return Db


# ----------------------------------------------------------------------------
# a5: transfers, smoother, coarsest solve, V-cycle (Table solver-config)
# ----------------------------------------------------------------------------
def _linear_interp_1d(n_fine_el: int) -> sp.csr_matrix:
    """1D nodal linear interpolation from n_fine_el/2 coarse elements to n_fine_el."""
    nf, nc = n_fine_el + 1, n_fine_el // 2 + 1
    rows, cols, vals = [], [], []
    for i in range(nf):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation(fine: Mesh) -> sp.csr_matrix:
    """Trilinear 2:1 prolongation over DOFs (unmasked): (P_z (x) P_y (x) P_x) (x) I_3."""
    Px = _linear_interp_1d(fine.nx)
    Py = _linear_interp_1d(fine.ny)
    Pz = _linear_interp_1d(fine.nz)
    Pn = sp.kron(Pz, sp.kron(Py, Px)).tocsr()
    return sp.kron(Pn, sp.identity(3)).tocsr()


@dataclass
class Level:
    mesh: Mesh
    E: np.ndarray
    K0: np.ndarray
    blockdiag: np.ndarray               # (n_nodes, 3, 3) node blocks of K
    P: sp.csr_matrix | None = None      # prolongation from the next coarser level
    chol: tuple | None = None           # coarsest only: Cholesky factor of free block
    lam: float = 0.0                    # Chebyshev smoothing: lambda_max(D_b^{-1} K) estimate
    K: sp.csr_matrix | None = None      # Galerkin coarse levels: the assembled P^T K P (else matrix-free)


@dataclass
class Hierarchy:
    levels: list = field(default_factory=list)
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.6
    smoother: str = "jacobi"            # or "chebyshev"
    coarse: str = "rediscretised"       # or "galerkin"
    ls_ratio: float = 0.0               # > 0: line-searched, rejectable coarse correction (theta)
    fine_steps: int = 0                 # > 0: fine-level adaptive correction, inner FGMRES(fine_steps)
    coarse_steps: int = 0               # > 0: coarsest level by inner FGMRES(coarse_steps), not exactly


def level_apply(level: Level, x: np.ndarray) -> np.ndarray:
    """K_l x on a level: matrix-free sum_e E_e K0 (rediscretised), or the assembled
    Galerkin operator; fixed entries of the result are 0 either way."""
    if level.K is not None:
        return level.K @ np.where(level.mesh.fixed, 0.0, x)
    return apply_K(level.mesh, level.E, level.K0, x)


def _blocks_of(K: sp.csr_matrix, mesh: Mesh) -> np.ndarray:
    """The 3x3 diagonal blocks of an assembled operator (fixed nodes: identity)."""
    n = mesh.n_nodes
    D = np.zeros((n, 3, 3))
    for a in range(3):
        for b in range(3):
            D[:, a, b] = np.asarray(K[np.arange(n) * 3 + a, np.arange(n) * 3 + b]).ravel()
    return _mask_blocks(D, mesh)


def build_hierarchy(mesh: Mesh, E_fine: np.ndarray, n_levels: int, nu: float = 0.3,
                    nu1: int = 2, nu2: int = 2, omega: float = 0.6, smoother: str = "jacobi",
                    coarse: str = "rediscretised", ls_ratio: float = 0.0, fine_steps: int = 0,
                    coarse_steps: int = 0) -> Hierarchy:
    """Level l has (nx, ny, nz)/2^l elements of edge h*2^l. coarse="rediscretised":
    modulus = child mean and K0(h_l), applied matrix-free (this build's reading);
    coarse="galerkin": K_{l+1} = P^T K_l P with P the masked trilinear prolongation, the
    coarse operator of Table solver-config, assembled (used to compare the two).
    With smoother="chebyshev" every smoothing level also gets lam (its lambda_max)."""
    if coarse not in ("rediscretised", "galerkin"):
        raise ValueError(coarse)
    H = Hierarchy(nu1=nu1, nu2=nu2, omega=omega, smoother=smoother, coarse=coarse, ls_ratio=ls_ratio,
                  fine_steps=fine_steps, coarse_steps=coarse_steps)
    m, E = mesh, np.asarray(E_fine, dtype=np.float64)
    Kg = None
    for l in range(n_levels):
        K0 = element_stiffness(m.h, 1.0, nu)
        if Kg is None:
            H.levels.append(Level(m, E, K0, node_block_diagonal(m, E, K0)))
        else:
            H.levels.append(Level(m, E, K0, _blocks_of(Kg, m), K=Kg))
        if l == n_levels - 1:
            break
        if m.nx % 2 or m.ny % 2 or m.nz % 2:
            raise ValueError("grid not divisible for the requested level count")
        P = prolongation(m)
        H.levels[-1].P = P
        mc = m.coarsen()
        if coarse == "galerkin":
            Kf = H.levels[-1].K if H.levels[-1].K is not None else assemble_sparse(m, E, K0)
            Pm = sp.diags(m.free.astype(np.float64)) @ P @ sp.diags(mc.free.astype(np.float64))
            Kg = (Pm.T @ Kf @ Pm).tocsr()
        E = coarsen_modulus(m, E)
        m = mc
    last = H.levels[-1]
    if last.K is not None:
        f = last.mesh.free
        Kc = last.K.toarray()[np.ix_(f, f)]
    else:
        Kc = assemble_dense_free(last.mesh, last.E, last.K0)
    last.chol = sla.cho_factor(Kc, lower=True)
    if smoother == "chebyshev":
        for lev in H.levels[:-1]:
            lev.lam = level_lambda_max(lev)
    return H


def coarse_solve(level: Level, b: np.ndarray) -> np.ndarray:
    x = np.zeros_like(b)
    x[level.mesh.free] = sla.cho_solve(level.chol, b[level.mesh.free])
    return x


def coarse_krylov(level: Level, b: np.ndarray, steps: int) -> np.ndarray:
    """The coarse-level solve of Table solver-config: `steps` steps of an inner
    FGMRES(steps) from x = 0 on the level's operator, preconditioned by its 3x3 node-block
    Jacobi operator (b = 0 gives x = 0)."""
    if not np.any(b):
        return np.zeros_like(b)
    return fgmres(lambda w: level_apply(level, w), lambda w: block_jacobi_apply(level, w), b,
                  restart=steps, kmax=steps, tol=0.0).x


def jacobi_sweep(level: Level, x: np.ndarray, b: np.ndarray, omega: float) -> np.ndarray:
    """Damped node-block Jacobi: x <- x + omega D_b^{-1} (b - K x), D_b the 3x3 node blocks."""
    r = b - level_apply(level, x)
    dx = np.linalg.solve(level.blockdiag, r.reshape(-1, 3, 1)).reshape(-1)
    return x + omega * dx


def block_jacobi_apply(level: Level, r: np.ndarray) -> np.ndarray:
    """D_b^{-1} r with the 3x3 node blocks."""
    return np.linalg.solve(level.blockdiag, r.reshape(-1, 3, 1)).reshape(-1)


def power_lambda_max(apply_M, v0: np.ndarray, iters: int = 15) -> float:
    """Power method for the largest eigenvalue of M: v_0 = v0/||v0||, then at each step
    w = M v, estimate ||w|| (with ||v|| = 1), v = w/||w||; the last estimate is returned."""
    v = v0 / np.linalg.norm(v0)
    lam = 0.0
    for _ in range(iters):
        w = apply_M(v)
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


def level_lambda_max(level: Level, iters: int = 15) -> float:
    """lambda_max(D_b^{-1} K) of a level by 15 power iterations from ones on free DOFs."""
    v0 = np.where(level.mesh.fixed, 0.0, 1.0)
    return power_lambda_max(lambda v: block_jacobi_apply(level, level_apply(level, v)),
                            v0, iters)


def chebyshev_coefficients(lam: float, degree: int):
    """Chebyshev semi-iteration on [lam/30, 1.1 lam] (theta = centre, delta = half
    width, sigma = theta/delta): step 0 d = (1/theta) D^{-1} r; step k >= 1
    rho_k = 1/(2 sigma - rho_{k-1}), d = rho_k rho_{k-1} d + (2 rho_k/delta) D^{-1} r,
    rho_0 = 1/sigma. Returns [(c1, c2)] with d <- c1 d + c2 D^{-1} r."""
    a, b = lam / 30.0, 1.1 * lam
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    coefs = [(0.0, 1.0 / theta)]
    rho = 1.0 / sigma
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        coefs.append((rho_new * rho, 2.0 * rho_new / delta))
        rho = rho_new
    return coefs


def chebyshev_smooth(level: Level, x: np.ndarray, b: np.ndarray, lam: float, degree: int) -> np.ndarray:
    """degree steps of Chebyshev semi-iteration for K x = b preconditioned by D_b: the
    error is multiplied by T_m((theta - M)/delta) / T_m(theta/delta), M = D_b^{-1} K."""
    d = np.zeros_like(b)
    for c1, c2 in chebyshev_coefficients(lam, degree):
        r = b - level_apply(level, x)
        d = c1 * d + c2 * block_jacobi_apply(level, r)
        x = x + d
    return x


def _smooth(H: Hierarchy, lev: Level, x: np.ndarray, b: np.ndarray, nu: int) -> np.ndarray:
    if H.smoother == "chebyshev":
        return chebyshev_smooth(lev, x, b, lev.lam, nu)
    for _ in range(nu):
        x = jacobi_sweep(lev, x, b, H.omega)
    return x


def line_search(r: np.ndarray, c: np.ndarray, q: np.ndarray, theta: float):
    """The line search on a coarse correction c with q = K c (Table solver-config, "coarse
    correction"; both the step and the acceptance test are readings): the step minimising
    the energy error along c, alpha = (c.r)/(c.q) -- computed from the residual r, and 1
    for an exact Galerkin coarse correction -- and the correction is kept only when that
    ratio passes the acceptance test alpha >= theta. Returns (alpha, kept), alpha = 0
    when rejected.""" 
    cr, cq = float(c @ r), float(c @ q)
    if not cq > 0.0:
        return 0.0, False
    alpha = cr / cq
    kept = alpha >= theta
    return (alpha if kept else 0.0), kept


def vcycle(H: Hierarchy, b: np.ndarray, l: int = 0) -> np.ndarray:
    """One V-cycle on level l for right-hand side b (fixed entries of b are zero)."""
    lev = H.levels[l]
    if l == len(H.levels) - 1:
        if H.coarse_steps > 0 and l > 0:
            return coarse_krylov(lev, b, H.coarse_steps)
        return coarse_solve(lev, b)
    x = _smooth(H, lev, np.zeros_like(b), b, H.nu1)
    r = b - level_apply(lev, x)
    coarse = H.levels[l + 1]
    bc = lev.P.T @ r
    bc[coarse.mesh.fixed] = 0.0
    xc = vcycle(H, bc, l + 1)
    corr = lev.P @ xc
    corr[lev.mesh.fixed] = 0.0
    if H.ls_ratio > 0.0:   # the correction scaled by the residual line search, or rejected
        alpha, _ = line_search(r, corr, level_apply(lev, corr), H.ls_ratio)
        x = x + alpha * corr
    else:
        x = x + corr
    return _smooth(H, lev, x, b, H.nu2)


# ----------------------------------------------------------------------------
# a6: right-preconditioned FGMRES(m) with CGS2 and Givens rotations
# ----------------------------------------------------------------------------
def precondition(H: Hierarchy, v: np.ndarray) -> np.ndarray:
    """The preconditioner the outer FGMRES applies: one V-cycle, then (fine_steps > 0) the
    fine-level adaptive correction of Table solver-config: fine_steps steps of an inner
    FGMRES(fine_steps) from d = 0 on K d = r, r = v - K z, preconditioned by the 3x3
    node-block Jacobi operator, applied only if it reduces the recomputed residual norm
    (||v - K (z + d)|| < ||r||)."""
    z = vcycle(H, v)
    if H.fine_steps <= 0:
        return z
    lev = H.levels[0]
    r = v - level_apply(lev, z)
    d = fgmres(lambda w: level_apply(lev, w), lambda w: block_jacobi_apply(lev, w), r,
               restart=H.fine_steps, kmax=H.fine_steps, tol=0.0).x
    if np.linalg.norm(v - level_apply(lev, z + d)) < np.linalg.norm(r):
        z = z + d
    return z


@dataclass
class SolveResult:
    x: np.ndarray
    history: np.ndarray      # history[k], k = 0..iters
    iters: int
    flag: int
    stop_estimate: float
    checks: list = field(default_factory=list)   # (k, history[k], recomputed eta_k) per true-residual check


def fgmres(apply_A, precond, f: np.ndarray, restart: int = 30, kmax: int = 200,
           tol: float = 1e-6, x0: np.ndarray | None = None,
           breakdown_rtol: float = 1e-14, check_every: int = 0, check_upto: int = 0,
           true_res=None) -> SolveResult:
    """Flexible GMRES (Saad 1993) preconditioned on the right, restarted every `restart` steps.

    History semantics (Table residual-semantics): at the start of every cycle the
    entry at the current iteration count is the true residual ||f - A x|| / ||f||;
    within the cycle each Arnoldi step k records the Givens-projected estimate
    |g_{j+1}| / ||f||. The solver stops when the recorded value is <= tol
    (converged), at k = kmax, or on breakdown.

    True-residual checks (the periodic checkpoints Sec. 4.1.1 names as untested): with
    check_every = c > 0, after every step k with k % c == 0 and k <= check_upto that
    does not end the solve, the iterate x_k = x + Z_J y_J (y_J from the current
    triangular system, as at a cycle end) is formed and eta_k = true_res(x_k) (default
    ||f - A x_k|| / ||f||) recorded beside history[k]. The solve itself is unchanged.
    """
    fnorm = float(np.linalg.norm(f))
    x = np.zeros_like(f) if x0 is None else x0.astype(np.float64).copy()
    hist = {}
    checks = []
    k = 0
    flag = MAX_ITERS
    while True:
        r = f - apply_A(x)
        beta = float(np.linalg.norm(r))
        hist[k] = beta / fnorm
        if hist[k] <= tol:
            flag = CONVERGED
            break
        if k >= kmax:
            flag = MAX_ITERS
            break
        m = restart
        V = [r / beta]
        Z = []
        Hm = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        J = 0
        stop = None
        for j in range(m):
            z = precond(V[j])
            Z.append(z)
            w = apply_A(z)
            w_norm0 = float(np.linalg.norm(w))
            h = np.array([V[i] @ w for i in range(j + 1)])
            for i in range(j + 1):
                w = w - h[i] * V[i]
            h2 = np.array([V[i] @ w for i in range(j + 1)])
            for i in range(j + 1):
                w = w - h2[i] * V[i]
            h = h + h2
            hnext = float(np.linalg.norm(w))
            Hm[:j + 1, j] = h
            Hm[j + 1, j] = hnext
            for i in range(j):
                a, b = Hm[i, j], Hm[i + 1, j]
                Hm[i, j] = cs[i] * a + sn[i] * b
                Hm[i + 1, j] = -sn[i] * a + cs[i] * b
            a, b = Hm[j, j], Hm[j + 1, j]
            rho = math.hypot(a, b)
            if rho == 0.0:
                # The new column adds nothing (K z_j lies in the span already and
                # is orthogonal to the rotated residual): breakdown, drop the step.
                stop = BREAKDOWN
                break
            cs[j], sn[j] = a / rho, b / rho
            Hm[j, j] = rho
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k += 1
            J = j + 1
            hist[k] = abs(g[j + 1]) / fnorm
            if hist[k] <= tol:
                stop = CONVERGED
                break
            if k >= kmax:
                stop = MAX_ITERS
                break
            if hnext <= breakdown_rtol * w_norm0:
                stop = BREAKDOWN
                break
            if check_every > 0 and k % check_every == 0 and k <= check_upto:
                yk = sla.solve_triangular(Hm[:J, :J], g[:J], lower=False)
                xk = x.copy()
                for i in range(J):
                    xk = xk + yk[i] * Z[i]
                eta = true_res(xk) if true_res is not None else float(np.linalg.norm(f - apply_A(xk))) / fnorm
                checks.append((k, hist[k], eta))
            V.append(w / hnext)
        if J > 0:
            y = sla.solve_triangular(Hm[:J, :J], g[:J], lower=False)
            for i in range(J):
                x = x + y[i] * Z[i]
        if stop is not None:
            flag = stop
            break
    history = np.array([hist[i] for i in range(k + 1)])
    return SolveResult(x=x, history=history, iters=k, flag=flag, stop_estimate=float(history[k]), checks=checks)


# ----------------------------------------------------------------------------
# a7: acceptance guard (Eq. relative_residual, Table residual-semantics)
# ----------------------------------------------------------------------------
def true_residual(mesh: Mesh, E: np.ndarray, K0: np.ndarray, f: np.ndarray, u: np.ndarray) -> float:
    """eta = ||M (f - K u)||_2 / ||M f||_2, recomputed in FP64 on free DOFs."""
    fm = np.where(mesh.fixed, 0.0, f)
    r = fm - apply_K(mesh, E, K0, u)
    return float(np.linalg.norm(r) / np.linalg.norm(fm))


# ----------------------------------------------------------------------------
# floor-conditioning diagnostic (Sec. 4.1.3)
# ----------------------------------------------------------------------------
def conditioning(mesh: Mesh, E: np.ndarray, K0: np.ndarray, f: np.ndarray):
    """Extreme eigenvalues of the free-DOF operator (dense symmetric eigensolver) and the
    guard residual of the direct solution (Cholesky of the free block): the reduced
    diagnostic that relates kappa = lambda_max / lambda_min to the attained residual."""
    Kf = assemble_dense_free(mesh, E, K0)
    ev = sla.eigvalsh(Kf)
    u = np.zeros(mesh.n_dof)
    u[mesh.free] = sla.cho_solve(sla.cho_factor(Kf, lower=True), np.asarray(f)[mesh.free])
    return float(ev[0]), float(ev[-1]), true_residual(mesh, E, K0, f, u)


def conditioning_screen(lambda_min: float, lambda_max: float, rho_min: float, tau: float) -> float:
    """The floor screen: kappa ~ c / rho_min with c = kappa rho_min measured at rho_min, so
    kappa eps <= tau needs rho_min >= c eps / tau (eps = 2^-52, our reading of the paper's eps)."""
    c = lambda_max / lambda_min * rho_min
    return c * 2.0 ** -52 / tau


# ----------------------------------------------------------------------------
# a8: probe features, trigger rule, guarded policy (Sec. 3.4, Eq. trigger, Algorithm 1)
# ----------------------------------------------------------------------------
@dataclass
class Thresholds:
    r50_escalate: float = 1e-2     # r50 >= this -> escalate
    r100_stall: float = 1e-4       # r100 >= this ...
    plateau_ratio: float = 0.6     # ... and r100/r50 >= this -> escalate
    checkpoint_a: int = 50
    checkpoint_b: int = 100


def probe_features(history: np.ndarray, k_stop: int, th: Thresholds = Thresholds()):
    """r50 = eta_{min(50,k_stop)}, r100 = eta_{min(100,k_stop)} from the recorded history."""
    r50 = float(history[min(th.checkpoint_a, k_stop)])
    r100 = float(history[min(th.checkpoint_b, k_stop)])
    return r50, r100


def trigger_rule(r50: float, r100: float, th: Thresholds = Thresholds()) -> bool:
    """Eq. (trigger): escalate iff r50 >= 1e-2 or (r100 >= 1e-4 and r100/r50 >= 0.6)."""
    return (r50 >= th.r50_escalate) or (r100 >= th.r100_stall and r100 / r50 >= th.plateau_ratio)


def true_check_detector(checks, ratio: float) -> bool:
    """The checkpointed detector (our reading of the variant Sec. 4.1.1 leaves untested):
    it fires when a recomputed true residual exceeds ratio times the projected estimate
    recorded at the same step, i.e. the estimate the probe features are read from no
    longer tracks the residual the guard will measure."""
    return any(eta > ratio * est for (_, est, eta) in checks)


def candidate_floors(escalate: bool, rho0: float, ladder):
    """Algorithm 1: C = ladder if the rule fires, else (rho0, ladder) in order."""
    return list(ladder) if escalate else [rho0] + list(ladder)


@dataclass
class Attempt:
    rho_min: float
    iters: int
    flag: int
    stop_estimate: float
    eta: float
    accepted: bool


@dataclass
class SelectResult:
    status: int
    floor_index: int          # index into (rho0, ladder...) of the accepted floor, -1 if none
    rho_min: float
    u: np.ndarray | None
    eta: float
    r50: float
    r100: float
    escalated: bool
    attempts: list
    probe_iters_run: int = 0
    checks: list = field(default_factory=list)   # the probe's true-residual checks
    detector: bool = False                       # true_check_detector fired


@dataclass
class SolverSetup:
    """Everything fixed for a frozen state: mesh, stored density, exponent, solver settings."""
    mesh: Mesh
    rho_hat: np.ndarray
    p: float = 3.0
    nu: float = 0.3
    n_levels: int = 3
    restart: int = 30
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.6
    smoother: str = "jacobi"
    coarse: str = "rediscretised"
    ls_ratio: float = 0.0
    fine_steps: int = 0
    coarse_steps: int = 0


def solve_at_floor(setup: SolverSetup, f: np.ndarray, rho_min: float, kmax: int, tol: float,
                   check_every: int = 0, check_upto: int = 0):
    """Frozen-state solve K(rho_min) u = f with GMG-preconditioned FGMRES from u0 = 0
    (with check_every > 0: true-residual checks, the guard's eta, up to step check_upto)."""
    mesh = setup.mesh
    E = young_modulus(setup.rho_hat, rho_min, setup.p)
    H = build_hierarchy(mesh, E, setup.n_levels, setup.nu, setup.nu1, setup.nu2, setup.omega, setup.smoother,
                        setup.coarse, setup.ls_ratio, setup.fine_steps, setup.coarse_steps)
    K0 = H.levels[0].K0
    fm = np.where(mesh.fixed, 0.0, f)
    res = fgmres(lambda v: apply_K(mesh, E, K0, v), lambda v: precondition(H, v), fm,
                 restart=setup.restart, kmax=kmax, tol=tol, check_every=check_every, check_upto=check_upto,
                 true_res=lambda x: true_residual(mesh, E, K0, f, x))
    return res, E, K0


def guarded_policy(probe_fn, attempt_fn, rho0: float, ladder, tau: float = 1e-6,
                   kmax: int = 200, probe_iters: int = 100, th: Thresholds = Thresholds(),
                   selector: str = "rule", first_index: int | None = None,
                   true_check_ratio: float | None = None) -> SelectResult:
    """Algorithm 1 as pure control logic.

    probe_fn(rho0, iters) -> SolveResult of the probe solve (history used for r50/r100);
    attempt_fn(rho_min, kmax) -> (SolveResult, eta) for an independent solve from u0 = 0
    followed by the recomputed FP64 true residual (the acceptance guard).

    selector: "rule" (Eq. trigger on the probe), "full" (no probe, C = (rho0, ladder)),
    "given" (no probe; start at ``first_index`` of (rho0, ladder) -- e.g. chosen by a
    learned selector -- and continue up the ladder), or "reuse" (the cost reduction the
    paper names for the optimisation loop and leaves untested: attempt the previous
    decision, ``first_index``, with no probe; if the guard rejects it, run "rule" from
    scratch, the rejected attempt recorded first). Floor indices refer to (rho0, ladder...).

    true_check_ratio (rule selector): when given, the probe's true-residual checks
    (probe.checks) also escalate if true_check_detector fires (our reading of the
    checkpointed detector variant of Sec. 4.1.1).
    """
    floors = [rho0] + list(ladder)
    if selector == "reuse":
        res, eta = attempt_fn(floors[int(first_index)], kmax)
        first = Attempt(floors[int(first_index)], res.iters, res.flag, res.stop_estimate, eta, eta <= tau)
        if eta <= tau:
            return SelectResult(ACCEPTED, int(first_index), floors[int(first_index)], res.x, eta,
                                float("nan"), float("nan"), int(first_index) > 0, [first], 0)
        out = guarded_policy(probe_fn, attempt_fn, rho0, ladder, tau, kmax, probe_iters, th, "rule",
                             true_check_ratio=true_check_ratio)
        out.attempts = [first] + out.attempts
        return out
    r50 = r100 = float("nan")
    escalated = False
    probe_k = 0
    checks, detector = [], False
    if selector == "rule":
        probe = probe_fn(rho0, probe_iters)
        probe_k = probe.iters
        r50, r100 = probe_features(probe.history, probe.iters, th)
        checks = list(probe.checks)
        detector = true_check_ratio is not None and true_check_detector(checks, true_check_ratio)
        escalated = trigger_rule(r50, r100, th) or detector
        cand = candidate_floors(escalated, rho0, ladder)
        start = 1 if escalated else 0
    elif selector == "full":
        cand, start = floors, 0
    elif selector == "given":
        start = int(first_index)
        cand = floors[start:]
        escalated = start > 0
    else:
        raise ValueError(selector)
    attempts = []
    for idx, rm in enumerate(cand):
        res, eta = attempt_fn(rm, kmax)
        ok = eta <= tau
        attempts.append(Attempt(rm, res.iters, res.flag, res.stop_estimate, eta, ok))
        if ok:
            return SelectResult(ACCEPTED, start + idx, rm, res.x, eta, r50, r100, escalated, attempts,
                                probe_k, checks, detector)
    return SelectResult(NO_ADMISSIBLE_FLOOR, -1, float("nan"), None, float("nan"), r50, r100,
                        escalated, attempts, probe_k, checks, detector)


def select_floor(setup: SolverSetup, f: np.ndarray, rho0: float, ladder, tau: float = 1e-6,
                 kmax: int = 200, probe_iters: int = 100, th: Thresholds = Thresholds(),
                 selector: str = "rule", first_index: int | None = None,
                 true_check_every: int = 0, true_check_ratio: float = 10.0) -> SelectResult:
    """Algorithm 1 on a frozen state: GMG-FGMRES solves plus the FP64 acceptance guard
    (with true_check_every > 0: the probe's true-residual checks and their detector)."""

    def probe_fn(rm, iters):
        return solve_at_floor(setup, f, rm, iters, tau, true_check_every, iters)[0]

    def attempt_fn(rm, km):
        res, E, K0 = solve_at_floor(setup, f, rm, km, tau)
        return res, true_residual(setup.mesh, E, K0, f, res.x)

    return guarded_policy(probe_fn, attempt_fn, rho0, ladder, tau, kmax, probe_iters, th,
                          selector, first_index, true_check_ratio if true_check_every > 0 else None)


# ----------------------------------------------------------------------------
# a12: compliance, sensitivity, density filter, OC update (Sec. 3.1)
# ----------------------------------------------------------------------------
def compliance(f: np.ndarray, u: np.ndarray) -> float:
    """C = f^T u."""
    return float(f @ u)


def sensitivity(mesh: Mesh, rho_hat: np.ndarray, rho_min: float, p: float, K0: np.ndarray,
                u: np.ndarray) -> np.ndarray:
    """dC/drho_e = -p (1 - rho_min) rho_e^{p-1} u_e^T K0 u_e (self-adjoint compliance)."""
    um = np.where(mesh.fixed, 0.0, u)
    ue = um[mesh.edof]
    energy = np.einsum("ei,ij,ej->e", ue, K0, ue)
    return -p * (1.0 - rho_min) * np.power(rho_hat, p - 1.0) * energy


def filter_weights(mesh: Mesh, r_min: float) -> sp.csr_matrix:
    """Linear-hat filter H_ee' = max(0, r_min - dist(e,e')) between element centres (in cells)."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    R = int(math.ceil(r_min)) - 1      # integer offsets with |d| < r_min
    ex, ey, ez = mesh._element_coords()
    rows, cols, vals = [], [], []
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                w = r_min - math.sqrt(dx * dx + dy * dy + dz * dz)
                if w <= 0:
                    continue
                jx, jy, jz = ex + dx, ey + dy, ez + dz
                ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
                e = np.nonzero(ok)[0]
                rows.append(e)
                cols.append(jx[ok] + nx * (jy[ok] + ny * jz[ok]))
                vals.append(np.full(e.size, w))
    Hf = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(mesh.n_elem, mesh.n_elem)).tocsr()
    return Hf


def density_filter(Hf: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    """rho_tilde_e = sum_e' H_ee' x_e' / sum_e' H_ee'."""
    return (Hf @ x) / np.asarray(Hf.sum(axis=1)).ravel()


def density_filter_adjoint(Hf: sp.csr_matrix, g: np.ndarray) -> np.ndarray:
    """Chain rule through the filter: dC/dx_e' = sum_e H_ee' g_e / sum_e'' H_ee''."""
    return Hf.T @ (g / np.asarray(Hf.sum(axis=1)).ravel())


def oc_update(x: np.ndarray, dc: np.ndarray, dv: np.ndarray, volfrac: float,
              move: float = 0.2, tol: float = 1e-3, max_bisect: int = 200) -> np.ndarray:
    """Optimality-criteria update with move limit; bisection on the volume multiplier.

    x_new = clip(x * sqrt(-dc / (lam dv)), max(0, x-move), min(1, x+move)), with lam
    bisected until mean(x_new) matches volfrac (relative bracket width < tol).
    """
    l1, l2 = 0.0, 1e9
    xnew = x
    for _ in range(max_bisect):
        if (l2 - l1) / (l1 + l2) <= tol:
            break
        lmid = 0.5 * (l1 + l2)
        be = np.sqrt(np.maximum(-dc, 0.0) / (lmid * dv))
        xnew = np.clip(x * be, np.maximum(0.0, x - move), np.minimum(1.0, x + move))
        if xnew.mean() > volfrac:
            l1 = lmid
        else:
            l2 = lmid
    return xnew


def oc_iteration(mesh: Mesh, x: np.ndarray, f: np.ndarray, p: float, volfrac: float, r_min: float,
                 move: float, policy_kw: dict, n_levels: int):
    """One guarded SIMP-OC iteration (Sec. 3.1 with Algorithm 1 as the state solve).

    rho_hat = filter(x); select_floor on rho_hat; if accepted: C = f^T u,
    dc = sensitivity at the accepted floor, chained through the filter adjoint
    together with the unit volume sensitivity; x <- OC update. Returns
    (x_new, SelectResult, C)."""
    Hf = filter_weights(mesh, r_min)
    rho = density_filter(Hf, x)
    setup = SolverSetup(mesh, rho, p=p, n_levels=n_levels)
    res = select_floor(setup, f, **policy_kw)
    if res.status != ACCEPTED:
        return x.copy(), res, float("nan")
    C = compliance(f, res.u)
    dc = sensitivity(mesh, rho, res.rho_min, p, element_stiffness(mesh.h), res.u)
    dcx = density_filter_adjoint(Hf, dc)
    dvx = density_filter_adjoint(Hf, np.ones(mesh.n_elem))
    return oc_update(x, dcx, dvx, volfrac, move), res, C


# ----------------------------------------------------------------------------
# a11: learned first-floor selector (not in the paper; its analogue is Eq. trigger)
# MLP 6 -> 32 -> 32 -> 4, tanh hidden layers, softmax + cross-entropy, Adam.
# Parameters are one flat vector: W1 (32x6, [out][in]), b1 (32), W2 (32x32), b2,
# W3 (4x32), b3 (4): 1412 numbers.
# ----------------------------------------------------------------------------
MLP_SIZES = (6, 32, 32, 4)


def mlp_unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for a, b in zip(MLP_SIZES[:-1], MLP_SIZES[1:]):
        W = theta[o:o + a * b].reshape(b, a)
        o += a * b
        c = theta[o:o + b]
        o += b
        out.append((W, c))
    assert o == theta.size
    return out


def mlp_n_params():
    return sum(a * b + b for a, b in zip(MLP_SIZES[:-1], MLP_SIZES[1:]))


def selector_features(r50, r100, rho_hat):
    """x = [log10 r50, log10 r100, r100/r50, fraction of voxels at floor (rho_hat == 0),
    mean rho_hat, std rho_hat] (population std)."""
    rho_hat = np.asarray(rho_hat, dtype=np.float64)
    return np.array([math.log10(max(r50, 1e-30)), math.log10(max(r100, 1e-30)), r100 / r50,
                     float(np.mean(rho_hat == 0.0)), float(np.mean(rho_hat)), float(np.std(rho_hat))])


def mlp_forward(theta, X, mu, sd):
    """Logits for rows of X, after standardising with (mu, sd)."""
    (W1, b1), (W2, b2), (W3, b3) = mlp_unpack(theta)
    Z = (np.asarray(X, dtype=np.float64) - mu) / sd
    H1 = np.tanh(Z @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    return H2 @ W3.T + b3


def mlp_loss_grad(theta, X, y, mu, sd):
    """Mean cross-entropy over the rows and its gradient (same flat layout as theta)."""
    (W1, b1), (W2, b2), (W3, b3) = mlp_unpack(theta)
    Z = (np.asarray(X, dtype=np.float64) - mu) / sd
    n = Z.shape[0]
    H1 = np.tanh(Z @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    L = H2 @ W3.T + b3
    L = L - L.max(axis=1, keepdims=True)
    P = np.exp(L)
    P /= P.sum(axis=1, keepdims=True)
    y = np.asarray(y, dtype=np.int64)
    loss = float(-np.mean(np.log(P[np.arange(n), y])))
    D3 = P.copy()
    D3[np.arange(n), y] -= 1.0
    D3 /= n
    gW3, gb3 = D3.T @ H2, D3.sum(0)
    D2 = (D3 @ W3) * (1.0 - H2 * H2)
    gW2, gb2 = D2.T @ H1, D2.sum(0)
    D1 = (D2 @ W2) * (1.0 - H1 * H1)
    gW1, gb1 = D1.T @ Z, D1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
