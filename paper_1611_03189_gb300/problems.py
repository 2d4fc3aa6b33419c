"""Seeded synthetic inputs for the hierarchical solver.

This module builds the *inputs* of the method only: finite-difference matrices in
CSR form, the leaf clustering and right-hand sides.  It holds none of the
solver's arithmetic, so both the CUDA path and the FP64 oracle may use it.

Workloads (Sec. 7 of the paper, "Numerical tests"): the d-dimensional Poisson
problem -div(alpha grad u) = f on [0,1]^d with u = 0 on the boundary, discretised
by the second-order five-point (2D) or seven-point (3D) stencil on an interior
grid.  The matrix is not scaled by 1/h^2: the truncation rule is relative, so the
scaling does not change any decision.

Coefficient models:
  * constant (alpha = 1), Tables 1-3;
  * piecewise constant, 1e-5 on [1/4,3/4]^2 and 1 elsewhere, Table 4;
  * uniform random in [0,1] per grid point, Table 5;
  * log-normal random field exp(s*g), g a Gaussian-smoothed white noise field
    (length scale 8 cells) normalised to mean 0 and variance 1.

Face coefficient between grid points i and j is (a_i + a_j)/2; a face on the
Dirichlet boundary uses a_i.  Row i of A has A_ii = sum of its face
coefficients and A_ij = -(face coefficient) for each interior neighbour j.

Leaf clustering (Sec. 3, "the block partitioning ... forms N = 2^L red nodes",
satisfied "by recursively bisecting"): coordinate bisection of the grid box,
splitting the longest axis (ties: lowest axis) at floor(len/2), to depth L.
Leaves come out in sibling order (children of one parent are consecutive).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    """A sparse SPD system with its clustering.

    rowptr/col/val: CSR of A (int32, int32, float64), original grid ordering.
    perm: perm[p] = original index of the p-th unknown in cluster order (int32).
    leaf_ptr: leaf_ptr[i]..leaf_ptr[i+1] is leaf i in cluster order (int32),
        len = 2^L + 1.
    shape: grid shape (nx, ny) or (nx, ny, nz); index = x + nx*(y + ny*z).
    """

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    perm: np.ndarray
    leaf_ptr: np.ndarray
    shape: tuple
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def nleaf(self) -> int:
        return len(self.leaf_ptr) - 1

    @property
    def levels(self) -> int:
        return int(round(math.log2(self.nleaf)))

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


# ---------------------------------------------------------------------------
# coefficient fields
# ---------------------------------------------------------------------------

def coef_constant(shape) -> np.ndarray:
    return np.ones(int(np.prod(shape)))


def coef_piecewise(shape, low: float = 1e-5) -> np.ndarray:
    """alpha = low inside [1/4,3/4]^d, 1 elsewhere (grid point x_i = (i+1)h)."""
    axes = [(np.arange(s) + 1.0) / (s + 1.0) for s in shape]
    grids = np.meshgrid(*axes, indexing="ij")  # grids[d][i0, i1, ...]
    inside = np.ones(grids[0].shape, dtype=bool)
    for g in grids:
        inside &= (g >= 0.25) & (g <= 0.75)
    a = np.where(inside, low, 1.0)
    # flatten with x fastest: index = x + nx*(y + ny*z)
    return a.transpose(*reversed(range(len(shape)))).reshape(-1)


def coef_uniform(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=int(np.prod(shape)))


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(4 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def coef_lognormal(shape, s: float, seed: int, sigma: float = 8.0) -> np.ndarray:
    """a = exp(s*g): g = N(0,1) white noise convolved with a Gaussian of
    standard deviation `sigma` cells (truncated at 4 sigma, zero padded),
    renormalised to mean 0 and variance 1."""
    rng = np.random.default_rng(seed)
    # array axes ordered (z, y, x) so that C order flattening has x fastest
    g = rng.standard_normal(tuple(reversed(shape)))
    k = _gauss_kernel(sigma)
    r = len(k) // 2
    for ax in range(g.ndim):
        # zero-padded convolution, centred (valid for fields shorter than the kernel)
        g = np.apply_along_axis(lambda v: np.convolve(v, k, mode="full")[r:r + len(v)], ax, g)
    g = (g - g.mean()) / g.std()
    return np.exp(s * g).reshape(-1)


# ---------------------------------------------------------------------------
# stencil assembly
# ---------------------------------------------------------------------------

def stencil_matrix(shape, coef: np.ndarray):
    """CSR (rowptr, col, val) of the 5-/7-point operator with face coefficients
    (a_i + a_j)/2 and boundary faces a_i.  Columns sorted within a row."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    n = int(np.prod(shape))
    a = np.asarray(coef, dtype=np.float64)
    assert a.shape == (n,)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for s in shape:
        coords.append(rem % s)
        rem //= s
    strides = [int(np.prod(shape[:k])) for k in range(d)]
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for ax in range(d):
        for step in (-1, 1):
            c = coords[ax] + step
            inside = (c >= 0) & (c < shape[ax])
            j = idx + step * strides[ax]
            face = np.where(inside, 0.5 * (a + a[np.clip(j, 0, n - 1)]), a)
            diag += face
            rows.append(idx[inside])
            cols.append(j[inside])
            vals.append(-face[inside])
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), c.astype(np.int32), v


# ---------------------------------------------------------------------------
# clustering: coordinate bisection in sibling order
# ---------------------------------------------------------------------------

def bisect_clusters(shape, levels: int):
    """Recursive coordinate bisection of the grid box to depth `levels`.

    Returns (perm, leaf_ptr).  Each box splits its longest axis (ties: the
    lowest axis index) at floor(len/2); the low half is the first child.
    Within a leaf, unknowns keep ascending original index."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    strides = [int(np.prod(shape[:k])) for k in range(d)]
    boxes = [tuple((0, s) for s in shape)]
    for _ in range(levels):
        nxt = []
        for box in boxes:
            lens = [hi - lo for lo, hi in box]
            ax = int(np.argmax(lens))
            if lens[ax] < 2:
                raise ValueError("clustering too deep: a box cannot be split")
            lo, hi = box[ax]
            mid = lo + lens[ax] // 2
            b0 = list(box)
            b1 = list(box)
            b0[ax] = (lo, mid)
            b1[ax] = (mid, hi)
            nxt.append(tuple(b0))
            nxt.append(tuple(b1))
        boxes = nxt
    perm_parts = []
    leaf_ptr = [0]
    for box in boxes:
        rng = [np.arange(lo, hi) for lo, hi in box]
        mesh = np.meshgrid(*rng, indexing="ij")
        ids = sum(m.astype(np.int64) * st for m, st in zip(mesh, strides))
        ids = np.sort(ids.reshape(-1))
        perm_parts.append(ids)
        leaf_ptr.append(leaf_ptr[-1] + len(ids))
    perm = np.concatenate(perm_parts).astype(np.int32)
    return perm, np.asarray(leaf_ptr, dtype=np.int32)


def levels_for(n: int, leaf_size: int) -> int:
    return max(0, int(round(math.log2(n / leaf_size))))


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def make_problem(shape, coef: np.ndarray, leaf_size: int = 16, levels: int | None = None,
                 name: str = "") -> Problem:
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    rowptr, col, val = stencil_matrix(shape, coef)
    L = levels_for(n, leaf_size) if levels is None else levels
    perm, leaf_ptr = bisect_clusters(shape, L)
    return Problem(n, rowptr, col, val, perm, leaf_ptr, shape, name)


def convdiff2d(nx: int, beta: float, theta: float = 0.6, leaf_size: int = 16, levels=None) -> Problem:
    """Nonsymmetric input (an M-matrix with the five-point pattern): the 2D
    Poisson stencil plus first-order upwind convection -div grad u + w . grad u,
    w = (cos theta, sin theta) with cell strength beta (the convection term of
    a row is beta times the upwind difference).  The pattern is structurally
    symmetric; the values are not."""
    ny = nx
    shape = (nx, ny)
    n = nx * ny
    rowptr, col, val = stencil_matrix(shape, coef_constant(shape))
    val = val.copy()
    wx, wy = beta * math.cos(theta), beta * math.sin(theta)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    for ax, w, stride, size in ((0, wx, 1, nx), (1, wy, nx, ny)):
        coord = (rows // stride) % size
        # upwind: w > 0 differences with the lower neighbour, w < 0 with the upper
        up = -stride if w > 0 else stride
        aw = abs(w)
        is_diag = col == rows
        val[is_diag] += aw
        is_up = (col == rows + up) & (((coord > 0) if w > 0 else (coord < size - 1)))
        val[is_up] -= aw
    L = levels_for(n, leaf_size) if levels is None else levels
    perm, leaf_ptr = bisect_clusters(shape, L)
    return Problem(n, rowptr, col, val, perm, leaf_ptr, shape, f"convdiff2d_{nx}_b{beta}")


def poisson2d(nx: int, ny: int | None = None, leaf_size: int = 16, levels=None) -> Problem:
    ny = nx if ny is None else ny
    return make_problem((nx, ny), coef_constant((nx, ny)), leaf_size, levels,
                        f"poisson2d_{nx}x{ny}")


def poisson3d(nx: int, ny: int | None = None, nz: int | None = None, leaf_size: int = 64,
              levels=None) -> Problem:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return make_problem((nx, ny, nz), coef_constant((nx, ny, nz)), leaf_size, levels,
                        f"poisson3d_{nx}x{ny}x{nz}")


def diffusion2d(nx: int, s: float, seed: int, leaf_size: int = 16, levels=None,
                ny: int | None = None) -> Problem:
    ny = nx if ny is None else ny
    return make_problem((nx, ny), coef_lognormal((nx, ny), s, seed), leaf_size, levels,
                        f"diffusion2d_{nx}x{ny}_s{s}_seed{seed}")


def diffusion3d(nx: int, s: float, seed: int, leaf_size: int = 64, levels=None) -> Problem:
    shape = (nx, nx, nx)
    return make_problem(shape, coef_lognormal(shape, s, seed), leaf_size, levels,
                        f"diffusion3d_{nx}_s{s}_seed{seed}")


def piecewise2d(nx: int, leaf_size: int = 8, levels=None) -> Problem:
    return make_problem((nx, nx), coef_piecewise((nx, nx)), leaf_size, levels,
                        f"piecewise2d_{nx}")


def random2d(nx: int, seed: int, leaf_size: int = 8, levels=None) -> Problem:
    return make_problem((nx, nx), coef_uniform((nx, nx), seed), leaf_size, levels,
                        f"random2d_{nx}_seed{seed}")


def rhs(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """b ~ N(0,1) from numpy.random.default_rng(seed); shape (n,) or (n, nrhs)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.standard_normal(n)
    return rng.standard_normal((nrhs, n)).T.copy()


def batched_sides(count: int, seed: int, lo: int = 32, hi: int = 256) -> list[int]:
    """Grid sides round(exp(U(ln lo, ln hi))) for the batched workload."""
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(u))) for u in rng.uniform(math.log(lo), math.log(hi), count)]


def laplacian_eigvec_2d(nx: int, ny: int, j: int = 1, k: int = 1) -> np.ndarray:
    """sin(j pi x h) sin(k pi y h) on the interior grid, index x + nx*y
    (the (j,k) eigenvector of the constant-coefficient 5-point operator)."""
    x = (np.arange(nx) + 1.0) / (nx + 1.0)
    y = (np.arange(ny) + 1.0) / (ny + 1.0)
    return (np.sin(k * math.pi * y)[:, None] * np.sin(j * math.pi * x)[None, :]).reshape(-1)


def laplacian_eigval_2d(nx: int, ny: int, j: int = 1, k: int = 1) -> float:
    """4 - 2cos(j pi hx) - 2cos(k pi hy), hx = 1/(nx+1), hy = 1/(ny+1)."""
    return 4.0 - 2.0 * math.cos(j * math.pi / (nx + 1)) - 2.0 * math.cos(k * math.pi / (ny + 1))
