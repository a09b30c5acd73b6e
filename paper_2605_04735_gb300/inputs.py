"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds only input recipes: density fields, problem sizes and the
serving request stream.  It contains none of the method's arithmetic (no
element matrix, no interpolation E(rho), no solve), so both the CUDA path and
the CPU oracle may read what it produces without sharing computation.

Conventions (the same on both sides, stated here once):
  * element e = i + nx*(j + ny*k) for i < nx, j < ny, k < nz (x fastest);
  * densities are float32 in [0, 1], one per element, in that order;
  * every generator takes an explicit integer seed and uses
    numpy.random.Generator(PCG64(seed)).

The workloads stand in for the paper's 40x20x20 cantilever / MBB problems of
Sec. 4.1 (same E0 = 1, nu = 0.3, p = 3), at the grid sizes named below.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 2605_04735

# boundary-condition and load codes, mirrored by include/topo.h
BC_CANTILEVER = 0          # x = 0 face clamped (all three components)
BC_MBB = 1                 # u_x = 0 on x = 0, u_z = 0 on line (x = L, z = 0), u_y pin
BC_ROLLER_BOX = 2          # normal rollers on the x = 0, y = 0, z = 0 planes
LOAD_EDGE_XL_BOTTOM = 0    # unit -z load along the edge x = L, z = 0
LOAD_EDGE_X0_TOP = 1       # unit -z load along the edge x = 0, z = H
LOAD_FACE_XL_TRACTION = 2  # uniform unit +x traction on the face x = L
BC_CORNERS = 3             # paper Sec. 4.2: four 0.3 x 0.3 corner supports on x = 0
BC_MBB_STRIP = 4           # paper Sec. 4.3: symmetry x = 0, one-element strip support at x = L
LOAD_DISC_XL = 3           # paper Sec. 4.2: -z on a disc of radius 0.1 at the centre of x = L
LOAD_HALFDISC_X0_TOP = 4   # paper Sec. 4.3: -z on a half-disc of radius 0.1 at (0, 0.5, 1)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def density_uniform(nx: int, ny: int, nz: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """i.i.d. U[lo, hi] element densities (float32, element order)."""
    r = rng(seed).uniform(lo, hi, size=nx * ny * nz)
    return r.astype(np.float32)


def density_cone_smoothed(nx: int, ny: int, nz: int, seed: int, radius: float = 1.5,
                          lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    """U[0,1] field smoothed by a cone (linear hat) weight of the given radius.

    w(d) = max(0, radius - d) over element centroids d apart (in element
    units), normalised by the in-domain sum of weights, then clipped to
    [lo, hi].  With radius 1.5 the stencil is self (1.5), six face neighbours
    (0.5) and twelve edge neighbours (1.5 - sqrt 2); corners get 0.
    """
    raw = rng(seed).uniform(0.0, 1.0, size=(nz, ny, nx))
    num = np.zeros_like(raw)
    den = np.zeros_like(raw)
    reach = int(np.floor(radius))
    for dk in range(-reach, reach + 1):
        for dj in range(-reach, reach + 1):
            for di in range(-reach, reach + 1):
                w = radius - np.sqrt(di * di + dj * dj + dk * dk)
                if w <= 0.0:
                    continue
                # target slice t receives source slice s = t + d
                tk = slice(max(0, -dk), nz - max(0, dk))
                tj = slice(max(0, -dj), ny - max(0, dj))
                ti = slice(max(0, -di), nx - max(0, di))
                sk = slice(max(0, dk), nz - max(0, -dk))
                sj = slice(max(0, dj), ny - max(0, -dj))
                si = slice(max(0, di), nx - max(0, -di))
                num[tk, tj, ti] += w * raw[sk, sj, si]
                den[tk, tj, ti] += w
    rho = np.clip(num / den, lo, hi)
    return rho.reshape(-1).astype(np.float32)


def void_spheres(nx: int, ny: int, nz: int, n_voids: int, seed: int,
                 rmin: float = 4.0, rmax: float = 16.0):
    """Seeded sphere centres (uniform in the box) and radii (uniform [rmin, rmax])."""
    g = rng(seed)
    centres = g.uniform(0.0, 1.0, size=(n_voids, 3)) * np.array([nx, ny, nz], dtype=np.float64)
    radii = g.uniform(rmin, rmax, size=n_voids)
    return centres, radii


def density_voids(nx: int, ny: int, nz: int, n_voids: int, seed: int, slope: float = 8.0,
                  floor: float = 1e-3, rmin: float = 4.0, rmax: float = 16.0) -> np.ndarray:
    """Near-binary field: logistic step of slope 8 of the distance to spherical voids.

    d_e = min_k (|x_e - c_k| - r_k) in element units (x_e = element centroid),
    rho_e = max(floor, 1 / (1 + exp(-slope * d_e))), rounded to float32.
    Elements farther than 5 element lengths from every sphere surface get
    rho = 1 exactly: there 1/(1 + exp(-40)) already rounds to 1.0f, so the
    bounding-box shortcut below does not change a single float32 value.
    """
    centres, radii = void_spheres(nx, ny, nz, n_voids, seed, rmin, rmax)
    margin = 5.0
    d = np.full((nz, ny, nx), np.inf)
    for (cx, cy, cz), r in zip(centres, radii):
        lo = np.floor(np.array([cx, cy, cz]) - r - margin - 0.5).astype(int)
        hi = np.ceil(np.array([cx, cy, cz]) + r + margin + 0.5).astype(int)
        i0, j0, k0 = np.maximum(lo, 0)
        i1, j1, k1 = np.minimum(hi, [nx, ny, nz])
        if i0 >= i1 or j0 >= j1 or k0 >= k1:
            continue
        zc = (np.arange(k0, k1) + 0.5 - cz)[:, None, None]
        yc = (np.arange(j0, j1) + 0.5 - cy)[None, :, None]
        xc = (np.arange(i0, i1) + 0.5 - cx)[None, None, :]
        dist = np.sqrt(xc * xc + yc * yc + zc * zc) - r
        sub = d[k0:k1, j0:j1, i0:i1]
        np.minimum(sub, dist, out=sub)
    with np.errstate(over="ignore"):
        rho = 1.0 / (1.0 + np.exp(-slope * np.minimum(d, 1e3)))
    rho = np.maximum(floor, rho)
    return rho.reshape(-1).astype(np.float32)


def levelset_voids(nx: int, ny: int, nz: int, n_voids: int, seed: int, rmin: float = 2.0,
                   rmax: float = 6.0) -> np.ndarray:
    """Nodal level set of a block with spherical voids (phi < 0 is material):
    phi_n = max_k (r_k - |x_n - c_k|) at the nodes x_n = (i, j, k), i.e. the
    signed distance to the union of the void balls outside overlaps, with the
    seeded centres and radii of `void_spheres`.  Node order i + (nx+1)(j + (ny+1)k),
    float64."""
    centres, radii = void_spheres(nx, ny, nz, n_voids, seed, rmin, rmax)
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    phi = np.full(X.shape[0], -np.inf)
    for c, r in zip(centres, radii):
        np.maximum(phi, r - np.linalg.norm(X - np.asarray(c), axis=1), out=phi)
    return phi


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    bc: int
    load: int
    recipe: str          # "uniform", "cone", "voids"
    seed: int
    n_voids: int = 0

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    def density(self) -> np.ndarray:
        if self.recipe == "uniform":
            return density_uniform(self.nx, self.ny, self.nz, 0.01, 1.0, self.seed)
        if self.recipe == "cone":
            return density_cone_smoothed(self.nx, self.ny, self.nz, self.seed)
        if self.recipe == "voids":
            return density_voids(self.nx, self.ny, self.nz, self.n_voids, self.seed)
        raise ValueError(self.recipe)


# The paper's own test problems (Sec. 4.1: 40 x 20 x 20 on 2 x 1 x 1, SIMP from a
# uniform 0.4, V_f = 0.4), run by the SIMP loop rather than the solve benchmark.
PAPER_PROBLEMS = {
    "paper_cantilever_40x20x20": (40, 20, 20, BC_CORNERS, LOAD_DISC_XL),
    "paper_mbb_40x20x20": (40, 20, 20, BC_MBB_STRIP, LOAD_HALFDISC_X0_TOP),
}

# The five workloads (sizes, BCs, loads and density recipes).
WORKLOADS = {
    "cantilever_24x12x12": Workload("cantilever_24x12x12", 24, 12, 12, BC_CANTILEVER,
                                    LOAD_EDGE_XL_BOTTOM, "uniform", SEED_BASE + 0),
    "mbb_96x32x32": Workload("mbb_96x32x32", 96, 32, 32, BC_MBB, LOAD_EDGE_X0_TOP,
                             "cone", SEED_BASE + 1),
    "cantilever_voids_192x96x96": Workload("cantilever_voids_192x96x96", 192, 96, 96,
                                           BC_CANTILEVER, LOAD_EDGE_XL_BOTTOM, "voids",
                                           SEED_BASE + 2, n_voids=40),
    "cantilever_voids_320x160x160": Workload("cantilever_voids_320x160x160", 320, 160, 160,
                                             BC_CANTILEVER, LOAD_EDGE_XL_BOTTOM, "voids",
                                             SEED_BASE + 4, n_voids=120),
}


def fd_elements(rho: np.ndarray, count: int, seed: int) -> np.ndarray:
    """Seeded element sample for finite-difference checks: half drawn from
    elements with 0.05 < rho < 0.95 (where the gradient is informative), half
    uniformly from all elements."""
    g = rng(seed)
    mid = np.flatnonzero((rho > 0.05) & (rho < 0.95))
    half = count // 2
    a = g.choice(mid, size=min(half, mid.size), replace=False) if mid.size else np.array([], int)
    b = g.choice(rho.size, size=count - a.size, replace=False)
    return np.unique(np.concatenate([a, b]))


@dataclasses.dataclass
class Request:
    """One serving request: a design that is re-solved `n_steps` times."""
    rid: int
    arrival: float       # seconds after the stream starts
    nx: int
    ny: int
    nz: int
    bc: int
    load: int
    rho0: np.ndarray     # initial density (float32)
    n_steps: int
    factor_seed: int

    def factor(self, step: int) -> np.ndarray:
        """Multiplicative perturbation in [0.95, 1.05] applied before solve `step` (>= 1)."""
        n = self.nx * self.ny * self.nz
        return rng(self.factor_seed + step).uniform(0.95, 1.05, size=n)


def perturb(rho: np.ndarray, factor: np.ndarray) -> np.ndarray:
    """SIMP-style density step of the serving stream: clip(rho * factor, 1e-3, 1)."""
    return np.clip(rho.astype(np.float64) * factor, 1e-3, 1.0).astype(np.float32)


def serving_stream(n_requests: int = 64, n_steps: int = 30, rate: float = 1.0,
                   ny_choices=tuple(range(12, 65, 4)), seed: int = SEED_BASE + 3,
                   max_ny: int | None = None) -> list[Request]:
    """Seeded request stream: half cantilever, half MBB, aspect 2:1:1 grids with
    ny drawn uniformly from ny_choices, cone-smoothed densities, Poisson
    arrivals at `rate` requests per second, and the per-step density factors."""
    g = rng(seed)
    choices = [c for c in ny_choices if max_ny is None or c <= max_ny]
    t = 0.0
    out = []
    kinds = np.array([0, 1] * ((n_requests + 1) // 2))[:n_requests]
    g.shuffle(kinds)
    for rid in range(n_requests):
        t += g.exponential(1.0 / rate) if rate > 0 else 0.0
        ny = int(g.choice(choices))
        nx, nz = 2 * ny, ny
        seed_r = int(g.integers(0, 2**31 - 1))
        rho0 = density_cone_smoothed(nx, ny, nz, seed_r)
        if kinds[rid] == 0:
            bc, load = BC_CANTILEVER, LOAD_EDGE_XL_BOTTOM
        else:
            bc, load = BC_MBB, LOAD_EDGE_X0_TOP
        out.append(Request(rid, t, nx, ny, nz, bc, load, rho0, n_steps, seed_r + 1))
    return out
