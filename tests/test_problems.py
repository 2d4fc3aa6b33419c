"""Checks of the synthetic input generators against closed forms."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1611_03189_gb300 import problems as P


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 7), (64, 64)])
@pytest.mark.parametrize("jk", [(1, 1), (2, 3)])
def test_poisson2d_eigenpairs_closed_form(nx, ny, jk):
    """The 5-point operator has eigenvectors sin(j pi x h) sin(k pi y h) with
    eigenvalues 4 - 2cos(j pi hx) - 2cos(k pi hy)."""
    pb = P.make_problem((nx, ny), P.coef_constant((nx, ny)), leaf_size=max(1, nx * ny // 4))
    A = pb.to_scipy()
    v = P.laplacian_eigvec_2d(nx, ny, *jk)
    lam = P.laplacian_eigval_2d(nx, ny, *jk)
    assert np.linalg.norm(A @ v - lam * v) <= 1e-12 * np.linalg.norm(v)


def test_poisson2d_extreme_eigenvalues_and_condition():
    nx = 16
    pb = P.poisson2d(nx, leaf_size=16)
    w = np.linalg.eigvalsh(pb.to_scipy().toarray())
    lo = P.laplacian_eigval_2d(nx, nx, 1, 1)
    hi = P.laplacian_eigval_2d(nx, nx, nx, nx)
    assert abs(w[0] - lo) < 1e-12 and abs(w[-1] - hi) < 1e-12


def test_poisson3d_stencil_row_structure():
    pb = P.poisson3d(6, leaf_size=27)
    A = pb.to_scipy().toarray()
    assert np.allclose(A, A.T)
    assert np.all(np.diag(A) == 6.0)
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off)) <= {-1.0, 0.0}
    # interior point has 6 neighbours
    i = 2 + 6 * (2 + 6 * 2)
    assert np.count_nonzero(off[i]) == 6


@pytest.mark.parametrize("maker", [
    lambda: P.diffusion2d(20, 2.0, 3, leaf_size=8),
    lambda: P.piecewise2d(16),
    lambda: P.random2d(16, 5),
])
def test_variable_coefficient_matrices_are_spd_m_matrices(maker):
    pb = maker()
    A = pb.to_scipy().toarray()
    assert np.allclose(A, A.T, rtol=0, atol=0)
    assert np.all(A - np.diag(np.diag(A)) <= 0)
    # diagonally dominant with strict dominance on boundary rows -> SPD
    assert np.linalg.eigvalsh(A)[0] > 0


def test_face_coefficients_average_rule():
    shape = (5, 4)
    a = np.arange(1, 21, dtype=float)
    rp, c, v = P.stencil_matrix(shape, a)
    A = np.zeros((20, 20))
    for i in range(20):
        A[i, c[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    # interior neighbour (x=1,y=1) -> (x=2,y=1)
    i, j = 1 + 5 * 1, 2 + 5 * 1
    assert A[i, j] == -(a[i] + a[j]) / 2
    # corner point (0,0): two boundary faces use a_i, two interior faces average
    d = 2 * a[0] + (a[0] + a[1]) / 2 + (a[0] + a[5]) / 2
    assert A[0, 0] == pytest.approx(d)


def test_lognormal_field_is_normalised():
    a = P.coef_lognormal((64, 48), 2.0, seed=7)
    g = np.log(a) / 2.0
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12


@pytest.mark.parametrize("shape,levels", [((64, 64), 8), ((13, 9), 3), ((8, 8, 8), 3)])
def test_bisection_clusters_are_sibling_ordered_boxes(shape, levels):
    perm, leaf_ptr = P.bisect_clusters(shape, levels)
    n = int(np.prod(shape))
    assert sorted(perm.tolist()) == list(range(n))
    assert len(leaf_ptr) == 2 ** levels + 1 and np.all(np.diff(leaf_ptr) > 0)
    strides = [int(np.prod(shape[:k])) for k in range(len(shape))]

    def coords(ids):
        return np.stack([(ids // st) % s for st, s in zip(strides, shape)], axis=1)

    # every subtree (range of leaves at any depth) is a full axis-aligned box
    for depth in range(levels + 1):
        width = 2 ** (levels - depth)
        for t in range(2 ** depth):
            ids = perm[leaf_ptr[t * width]:leaf_ptr[(t + 1) * width]]
            c = coords(ids.astype(np.int64))
            ext = c.max(0) - c.min(0) + 1
            assert int(np.prod(ext)) == len(ids)


def test_bisection_64x64_gives_4x4_leaves():
    perm, leaf_ptr = P.bisect_clusters((64, 64), 8)
    assert np.all(np.diff(leaf_ptr) == 16)


def test_rhs_is_seeded_standard_normal():
    b1 = P.rhs(1000, 3)
    b2 = P.rhs(1000, 3)
    assert np.array_equal(b1, b2)
    assert np.array_equal(b1, np.random.default_rng(3).standard_normal(1000))
    B = P.rhs(50, 1, nrhs=4)
    assert B.shape == (50, 4)


def test_batched_sides_are_log_uniform_in_range():
    s = P.batched_sides(256, 0)
    assert len(s) == 256 and min(s) >= 32 and max(s) <= 256
    # log-uniform: median near sqrt(32*256) = 90.5
    assert 60 < float(np.median(s)) < 130


def test_levels_for():
    assert P.levels_for(4096, 16) == 8
    assert P.levels_for(262144, 16) == 14
    assert P.levels_for(64 ** 3, 64) == 12
    assert math.isclose(2 ** P.levels_for(128 ** 3, 64), 128 ** 3 / 64)


@pytest.mark.parametrize("beta,theta", [(0.5, 0.6), (4.0, 0.6), (2.0, 2.5)])
def test_upwind_convection_diffusion_is_a_nonsymmetric_m_matrix(beta, theta):
    """convdiff2d: the five-point pattern (structurally symmetric), values of
    -Laplace + first-order upwind w . grad with w = beta (cos t, sin t):
    diagonal 4 + |w_x| + |w_y|, the upwind neighbour of each axis -1 - |w_a|,
    the downwind one -1; rows weakly diagonally dominant, so an M-matrix."""
    nx = 7
    pb = P.convdiff2d(nx, beta, theta=theta, leaf_size=4)
    A = sp.csr_matrix((pb.val, pb.col, pb.rowptr), shape=(pb.n, pb.n)).toarray()
    pat = A != 0
    assert (pat == pat.T).all() and np.abs(A - A.T).max() > 0.5 * beta * min(abs(math.cos(theta)), 1)
    wx, wy = beta * math.cos(theta), beta * math.sin(theta)
    i = 3 + nx * 3                                   # an interior point
    assert A[i, i] == pytest.approx(4 + abs(wx) + abs(wy))
    for w, stride in ((wx, 1), (wy, nx)):
        up, down = (i - stride, i + stride) if w > 0 else (i + stride, i - stride)
        assert A[i, up] == pytest.approx(-1 - abs(w))
        assert A[i, down] == pytest.approx(-1.0)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert (np.diag(A) >= off - 1e-12).all() and (A - np.diag(np.diag(A)) <= 0).all()
