"""Problem descriptions (no solver arithmetic) -- see the package docstring."""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class ProblemSpec:
    """One eigenproblem, described by its mesh and decomposition parameters.

    kind    : "p1_2d" | "p1_3d" | "q1_3d" | "morley_2d" | "bfs_2d" | "p1_lshape" | "q1_lshape"
    n       : elements per direction, (nx, ny) or (nx, ny, nz)
    length  : domain edge lengths; the domain is the box [0, Lx] x [0, Ly] (x [0, Lz])
    kappa   : per-element coefficient (layout in the package docstring), None = 1
    nsub    : subdomains per direction; n[d] must be a multiple of nsub[d]
    delta   : overlap width delta in fine element layers
    k       : number of wanted eigenpairs (the paper's s)
    tol     : relative residual tolerance of the stop test
    tau     : the initial eigenproblem of Algorithm 3.1 Step 1 is solved on the
              coarse grid refined tau times (H~ = H / 2^tau); tau = 0 uses J_H
    partition : "boxes" (nsub boxes per axis grown by delta element layers) or
              "triangles" (p1_2d on a square grid: the partition of Example 6.1, every
              coarse square cut along its SW->NE diagonal into two coarse triangles,
              each grown by delta rings of fine triangles; 2 delta < n / nsub)
    """

    kind: str
    n: Tuple[int, ...]
    length: Tuple[float, ...]
    nsub: Tuple[int, ...]
    delta: int
    k: int
    kappa: Optional[np.ndarray] = None
    tol: float = 1e-8
    tau: int = 0
    name: str = ""
    extra: dict = field(default_factory=dict)
    partition: str = "boxes"

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def h(self) -> Tuple[float, ...]:
        return tuple(L / m for L, m in zip(self.length, self.n))

    @property
    def n_dofs(self) -> int:
        """Interior grid nodes (Dirichlet data removed); for morley_2d the interior
        points of the half-grid (2 nx - 1)(2 ny - 1), for bfs_2d four dofs per interior
        node (clamped data removed)."""
        if self.kind == "p1_lshape":
            n = self.n[0]
            return (n - 1) ** 2 - (n // 2) ** 2
        if self.kind == "q1_lshape":
            nx, ny, nz = self.n
            return (nx - 1) * (ny - 1) * (nz - 1) - (nx // 2) * (ny // 2) * (nz - 1)
        out = 4 if self.kind == "bfs_2d" else 1
        for m in self.n:
            out *= (2 * m - 1) if self.kind == "morley_2d" else (m - 1)
        return out

    @property
    def n_coarse(self) -> int:
        """Coarse dimension: interior subdomain-grid nodes, four dofs each for the plate
        elements (their coarse space is BFS on the subdomain grid)."""
        if self.kind == "p1_lshape":
            S = self.nsub[0]
            return (S - 1) ** 2 - (S // 2) ** 2
        if self.kind == "q1_lshape":
            sx, sy, sz = self.nsub
            return (sx - 1) * (sy - 1) * (sz - 1) - (sx // 2) * (sy // 2) * (sz - 1)
        out = 4 if self.kind in ("bfs_2d", "morley_2d") else 1
        for m in self.nsub:
            out *= m - 1
        return out

    def kappa_array(self) -> np.ndarray:
        """The coefficient array with its documented shape (ones when kappa is None)."""
        if self.kappa is not None:
            return np.ascontiguousarray(self.kappa, dtype=np.float64)
        if self.kind == "p1_2d":
            nx, ny = self.n
            return np.ones((ny, nx, 2), dtype=np.float64)
        nx, ny, nz = self.n
        return np.ones((nz, ny, nx), dtype=np.float64)

    def validate(self) -> None:
        if self.kind not in ("p1_2d", "p1_3d", "q1_3d", "morley_2d", "bfs_2d", "p1_lshape", "q1_lshape"):
            raise ValueError(f"unknown kind {self.kind}")
        want_dim = 2 if self.kind in ("p1_2d", "morley_2d", "bfs_2d", "p1_lshape") else 3
        if self.dim != want_dim or len(self.length) != want_dim or len(self.nsub) != want_dim:
            raise ValueError("dimension mismatch")
        for m, s in zip(self.n, self.nsub):
            if m % s != 0:
                raise ValueError("element count must be a multiple of the subdomain count")
        if self.kind in ("morley_2d", "bfs_2d", "p1_lshape") and (
                self.kappa is not None or self.n[0] != self.n[1] or self.length[0] != self.length[1]):
            raise ValueError(f"{self.kind}: square domain and square cells, no coefficient")
        if self.kind == "p1_lshape" and (self.n[0] % 2 or self.nsub[0] % 2):
            raise ValueError("p1_lshape: even cell and subdomain counts (the removed quadrant is a union of both)")
        if self.kind == "q1_lshape" and (self.n[0] % 2 or self.n[1] % 2 or self.nsub[0] % 2 or self.nsub[1] % 2
                                         or self.kappa is not None):
            raise ValueError("q1_lshape: even x / y cell and subdomain counts, no coefficient")
        if self.partition not in ("boxes", "triangles"):
            raise ValueError(f"unknown partition {self.partition}")
        if self.partition == "triangles" and (self.kind != "p1_2d" or self.n[0] != self.n[1]
                                              or self.nsub[0] != self.nsub[1]
                                              or not 2 * self.delta < self.n[0] // self.nsub[0]):
            raise ValueError("triangles: p1_2d on a square grid with 2 delta < n / nsub")
        if self.k >= self.n_coarse:
            raise ValueError("k must be smaller than the coarse space dimension")
        ms = {m // s for m, s in zip(self.n, self.nsub)}
        if len(ms) != 1:
            raise ValueError("subdomains must span the same number of elements on every axis")
        if (ms.pop() % (1 << self.tau)) != 0:
            raise ValueError("the initial grid H/2^tau must be a union of fine cells")

    def initial_grid(self) -> "ProblemSpec":
        """The same problem with the subdomain grid refined tau times (the grid H~ of
        Algorithm 3.1 Step 1); only its coarse interpolation is used."""
        from dataclasses import replace
        return replace(self, nsub=tuple(s << self.tau for s in self.nsub), tau=0)


def _centroids_2d(nx: int, ny: int, Lx: float, Ly: float):
    """Centroids of the two triangles of every square of the uniform grid.

    Returns (cx, cy) with shape (ny, nx, 2), triangle 0 = below the SW->NE
    diagonal, triangle 1 = above it.
    """
    hx, hy = Lx / nx, Ly / ny
    i = np.arange(nx, dtype=np.float64)[None, :]
    j = np.arange(ny, dtype=np.float64)[:, None]
    cx = np.empty((ny, nx, 2))
    cy = np.empty((ny, nx, 2))
    # triangle 0: (0,0),(1,0),(1,1) in square-local units -> centroid (2/3, 1/3)
    cx[:, :, 0] = (i + 2.0 / 3.0) * hx + 0 * j
    cy[:, :, 0] = (j + 1.0 / 3.0) * hy + 0 * i
    # triangle 1: (0,0),(1,1),(0,1) -> centroid (1/3, 2/3)
    cx[:, :, 1] = (i + 1.0 / 3.0) * hx + 0 * j
    cy[:, :, 1] = (j + 2.0 / 3.0) * hy + 0 * i
    return cx, cy


def kappa_field_2d(nx: int, ny: int, Lx: float, Ly: float, kind: str, rng=None) -> np.ndarray:
    """Per-triangle coefficient samples.

    kind "sin"    : kappa = 1 + 0.5 sin(2 pi x) sin(2 pi y)      (smooth, in [0.5, 1.5])
    kind "random" : kappa = 2**zeta, zeta = sum_{p,q=1..3} c_pq cos(p pi x) cos(q pi y),
                    c_pq ~ U(-1, 1) from ``rng``, rescaled so max |zeta| = 1
                    (kappa in [0.5, 2]).
    """
    cx, cy = _centroids_2d(nx, ny, Lx, Ly)
    if kind == "sin":
        return 1.0 + 0.5 * np.sin(2 * np.pi * cx) * np.sin(2 * np.pi * cy)
    if kind == "random":
        if rng is None:
            raise ValueError("random kappa needs an rng")
        c = rng.uniform(-1.0, 1.0, size=(3, 3))
        zeta = np.zeros_like(cx)
        for p in range(3):
            for q in range(3):
                zeta += c[p, q] * np.cos((p + 1) * np.pi * cx) * np.cos((q + 1) * np.pi * cy)
        zeta /= max(np.abs(zeta).max(), 1e-300)
        return np.power(2.0, zeta)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def config_c1() -> ProblemSpec:
    """-Laplace u = lambda u on the unit square, P1, h = 1/32 (961 dofs), k = 6,
    4 x 4 subdomains (H = 8h), overlap 2 layers.  The initial eigenproblem uses
    H~ = H/2 (tau = 1): on J_H itself (9 coarse functions) the sixth coarse
    eigenvalue exceeds the smallest local Dirichlet eigenvalue, and the shifted
    local matrices of the first iteration would be indefinite."""
    return ProblemSpec("p1_2d", (32, 32), (1.0, 1.0), (4, 4), 2, 6, tau=1, name="c1_unit_square_p1_h32")


def config_c2() -> ProblemSpec:
    """-div(kappa grad u) = lambda u on [0,1] x [0,1.001], kappa = 1 + 0.5 sin sin,
    P1, 512 x 512 elements (261121 dofs), k = 12, 16 x 16 subdomains, overlap 2 layers."""
    nx = ny = 512
    kap = kappa_field_2d(nx, ny, 1.0, 1.001, "sin")
    return ProblemSpec("p1_2d", (nx, ny), (1.0, 1.001), (16, 16), 2, 12, kappa=kap,
                       name="c2_kappa_rect_p1_h512")


def config_c2_scaled(n: int) -> ProblemSpec:
    """C2's operator and coefficient on n x n elements with C2's subdomain shape (32
    elements per side, overlap 2 layers), k = 12: the same local band windows as C2
    at 1-17M dofs, for bandwidth measurements beyond the L2 cache."""
    kap = kappa_field_2d(n, n, 1.0, 1.001, "sin")
    return ProblemSpec("p1_2d", (n, n), (1.0, 1.001), (n // 32, n // 32), 2, 12, kappa=kap,
                       name=f"c2_scaled_p1_h{n}")


def config_c3() -> ProblemSpec:
    """-Laplace u = lambda u on the unit cube, P1 Kuhn tetrahedra, 64^3 cubes
    (250047 dofs), k = 10, 8 x 8 x 8 subdomains, overlap 1 layer."""
    return ProblemSpec("p1_3d", (64, 64, 64), (1.0, 1.0, 1.0), (8, 8, 8), 1, 10,
                       name="c3_unit_cube_p1tet_h64")


def config_c4() -> ProblemSpec:
    """Clamped plate Delta^2 u = lambda u on the unit square, Morley elements on
    256 x 256 squares (261121 dofs), k = 8 (including near-multiple pairs),
    8 x 8 subdomains, overlap 2 layers."""
    return ProblemSpec("morley_2d", (256, 256), (1.0, 1.0), (8, 8), 2, 8, name="c4_clamped_plate_morley_h256")


def config_small_morley(n: int = 32, ns: int = 4, delta: int = 2, k: int = 6, tau: int = 0) -> ProblemSpec:
    """A small clamped-plate case (Morley), for parity with the oracle."""
    return ProblemSpec("morley_2d", (n, n), (1.0, 1.0), (ns, ns), delta, k, tau=tau,
                       name=f"small_morley_{n}_{ns}_d{delta}_k{k}")


def config_c4_bfs() -> ProblemSpec:
    """The clamped plate of C4 with the paper's conforming element (BFS) instead of Morley:
    256 x 256 squares (260100 dofs), k = 8, 8 x 8 subdomains, overlap 2 layers."""
    return ProblemSpec("bfs_2d", (256, 256), (1.0, 1.0), (8, 8), 2, 8, name="c4_clamped_plate_bfs_h256")


def config_small_bfs(n: int = 32, ns: int = 4, delta: int = 2, k: int = 4, tau: int = 0) -> ProblemSpec:
    """A small clamped-plate case with BFS elements, for parity with the oracle."""
    return ProblemSpec("bfs_2d", (n, n), (1.0, 1.0), (ns, ns), delta, k, tau=tau,
                       name=f"small_bfs_{n}_{ns}_d{delta}_k{k}")


def config_small_2d(nx: int = 48, ny: int = 36, nsx: int = 4, nsy: int = 3, delta: int = 2,
                    k: int = 5, kappa: str = "sin", Lx: float = 1.0, Ly: float = 0.751, tau: int = 1) -> ProblemSpec:
    """A small variable-coefficient 2-D case with unequal sides (ragged subdomain sizes)."""
    kap = kappa_field_2d(nx, ny, Lx, Ly, kappa, rng=np.random.default_rng(0)) if kappa else None
    return ProblemSpec("p1_2d", (nx, ny), (Lx, Ly), (nsx, nsy), delta, k, kappa=kap, tau=tau,
                       name=f"small2d_{nx}x{ny}_{nsx}x{nsy}_d{delta}_k{k}")


def config_small_3d(n: int = 12, ns: int = 3, delta: int = 1, k: int = 4, kind: str = "p1_3d") -> ProblemSpec:
    return ProblemSpec(kind, (n, n, n), (1.0, 1.0, 1.0), (ns, ns, ns), delta, k,
                       name=f"small3d_{kind}_{n}_{ns}_d{delta}_k{k}")


def config_table1_col1() -> ProblemSpec:
    """Section 6, Example 6.1 / Table 1 first column: (0, pi)^2, P1, 128 x 128 squares
    (16129 dofs), s = 19.  The subdomain grid here is a box grid (8 x 8, overlap 4
    layers = H/4); the printed eigenvalues do not depend on the decomposition."""
    return ProblemSpec("p1_2d", (128, 128), (np.pi, np.pi), (8, 8), 4, 19, name="table1_col1")


def config_table5(n: int) -> ProblemSpec:
    """Section 6, Example 6.3 / Table 5: (0, pi)^3, trilinear elements, n^3 cubes,
    s = 20, 8 x 8 x 8 subdomains (H = pi/8), overlap H/2."""
    return ProblemSpec("q1_3d", (n, n, n), (np.pi, np.pi, np.pi), (8, 8, 8), max(1, n // 16), 20,
                       name=f"table5_n{n}")


def config_table3_col1() -> ProblemSpec:
    """Section 6, Example 6.2 / Table 3 first column: -Laplace u = lambda u on the L-shaped
    domain (-pi, pi)^2 minus [0, pi) x (-pi, 0], P1 on the 128 x 128 grid of the square
    (squares split SW->NE) restricted to the domain (12033 dofs), s = 20.  The subdomain
    grid is the paper's H = pi/8 (16 x 16 boxes over the square, those in the removed
    quadrant dropped) with delta / H = 1/4 (2 layers); the printed eigenvalues do not
    depend on the decomposition."""
    return ProblemSpec("p1_lshape", (128, 128), (2 * np.pi, 2 * np.pi), (16, 16), 2, 20, name="table3_col1")


def config_table7_col1() -> ProblemSpec:
    """Section 6, Example 6.4 / Table 7 first column: -Laplace u = lambda u on the prism
    (0, 2 pi) x (0, 2 pi) x (0, pi) minus [pi, 2 pi) x [pi, 2 pi) x (0, pi), trilinear
    elements on 32 x 32 x 16 cubes of side pi/16 (10575 dofs), s = 20; subdomains are the
    paper's N = 1536 cubes of side H = pi/8 with delta / H = 1/2 (one layer)."""
    return ProblemSpec("q1_lshape", (32, 32, 16), (2 * np.pi, 2 * np.pi, np.pi), (16, 16, 8), 1, 20,
                       name="table7_col1")


def config_small_lshape(n: int = 32, ns: int = 8, delta: int = 1, k: int = 4) -> ProblemSpec:
    """A small L-shaped case (P1), for parity with the oracle."""
    return ProblemSpec("p1_lshape", (n, n), (2 * np.pi, 2 * np.pi), (ns, ns), delta, k,
                       name=f"small_lshape_{n}_{ns}_d{delta}_k{k}")


@dataclass
class ServingRequest:
    rid: int
    arrival: float          # in units of the mean inter-arrival time
    spec: ProblemSpec


def serving_stream(n_requests: int = 64, seed: int = 0) -> List[ServingRequest]:
    """Poisson stream of mixed 2-D P1 eigenproblems (seeded, PCG64).

    Per request: elements per side in {64, 128, 256, 512}; kappa = 2**zeta with a
    random smooth zeta (kappa in [0.5, 2]); k ~ U{4..16}; subdomains per side
    drawn from {4, 8, 16}, then raised (doubling) until the subdomain is at most
    64 elements wide and the coarse space has more than k + 2 functions;
    overlap 2 layers; initial grid H/2 (tau = 1).  Arrival gaps are exponential with unit mean; the caller
    scales them to seconds.
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for rid in range(n_requests):
        t += float(rng.exponential(1.0))
        n = int(rng.choice([64, 128, 256, 512]))
        k = int(rng.integers(4, 17))
        ns = int(rng.choice([4, 8, 16]))
        while n // ns > 64 or (ns - 1) ** 2 <= k + 2:
            ns *= 2
        kap = kappa_field_2d(n, n, 1.0, 1.0, "random", rng=rng)
        # tau = 1: the Step 1 eigenproblem on the grid H/2 (Section 3), whose
        # initial Ritz values stay below the local Dirichlet spectra for every k drawn
        spec = ProblemSpec("p1_2d", (n, n), (1.0, 1.0), (ns, ns), 2, k, kappa=kap, tau=1,
                           name=f"req{rid}_n{n}_k{k}_ns{ns}")
        out.append(ServingRequest(rid, t, spec))
    return out
