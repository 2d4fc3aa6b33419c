"""Pins of the nonsymmetric (LU) variant of the oracle (reading R16), none of
which re-types its formulas:

* the literal dense extended system (oracle/dense_emulator.py with lu=True:
  the well-separated blocks moved onto a black/red pair, the pivot
  eliminated by an explicit dense Schur complement, no M_ss, P_ss or Q_ss
  formed) gives the same A_H^-1 at eps > 0, to rounding;
* eps = 0 keeps complete bases, so the factorization is exact: the apply
  equals a dense solve of the nonsymmetric A (Sec. 3.2: the extension is an
  equivalent system) -- this fixes the elimination algebra (M_ss, P_ss, Q_ss,
  the ordered-pair Schur update, A_nr, A_rn, A_rr);
* on a symmetric A the variant must reproduce the symmetric oracle (ranks and
  apply), which the dense emulator and the closed forms pin independently;
* GC keeps the constant exact on the RIGHT for any eps (Sec. 6 argument:
  phi_s and A_sW phi_W lie in span U), A_H^-1 (A 1) = 1, and LoRaSp does not
  (negative control) -- this fixes the nonsymmetric red-node blocks at eps > 0;
* the joint compression bounds both sides: ||A_sW - U U^T A_sW||_2 and
  ||A_Ws - A_Ws U U^T||_2 are at most eps ||[A_sW, A_Ws^T]||_2 (LoRaSp), with
  U orthonormal;
* as a preconditioner of GMRES (Sec. 7's outer solver) it converges on a
  convection-dominated problem in a handful of steps, more with a larger eps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hsolver as H
from oracle import hsolver_lu as HL
from oracle.dense_emulator import DenseEmulator
from paper_1611_03189_gb300 import problems as P


def _dense(pb):
    return sp.csr_matrix((pb.val, pb.col, pb.rowptr), shape=(pb.n, pb.n)).toarray()


def _factor(pb, eps, variant, **kw):
    return HL.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, eps, variant, **kw)


@pytest.mark.parametrize("nbr_dist", [1, 2])
@pytest.mark.parametrize("beta", [0.5, 4.0])
@pytest.mark.parametrize("variant", [HL.LORASP, HL.GC_CONSTANT])
def test_eps0_equals_a_dense_solve_of_the_nonsymmetric_matrix(beta, variant, nbr_dist):
    pb = P.convdiff2d(16, beta, leaf_size=4)
    A = _dense(pb)
    assert np.abs(A - A.T).max() > 0.1 * beta      # the input is nonsymmetric
    F = _factor(pb, 0.0, variant, nbr_dist=nbr_dist)
    if nbr_dist == 2:
        # red nodes made next to live neighbours (A_nr, A_rn exercised)
        assert any(r.wsep and r.nbrs for lv in F.levels for r in lv.supers)
    B = P.rhs(pb.n, 3, nrhs=2)
    X = np.linalg.solve(A, B)
    Z = HL.apply(F, B)
    assert np.max(np.abs(Z - X)) <= 1e-12 * np.max(np.abs(X))


@pytest.mark.parametrize("nbr_dist", [1, 2])
@pytest.mark.parametrize("variant", [HL.LORASP, HL.GC_CONSTANT])
@pytest.mark.parametrize("eps", [0.1, 0.3])
def test_symmetric_input_reproduces_the_symmetric_oracle(variant, eps, nbr_dist):
    pb = P.diffusion2d(16, 1.0, 3, leaf_size=4)
    F = _factor(pb, eps, variant, nbr_dist=nbr_dist)
    G = H.factor(pb.n, pb.rowptr, pb.col, pb.val, pb.perm, pb.leaf_ptr, eps, variant, nbr_dist=nbr_dist)
    assert [r.k for lv in F.levels for r in lv.supers] == [r.k for lv in G.levels for r in lv.supers]
    B = P.rhs(pb.n, 5, nrhs=2)
    Za, Zb = HL.apply(F, B), H.apply(G, B)
    assert np.max(np.abs(Za - Zb)) <= 1e-12 * np.max(np.abs(Zb))


@pytest.mark.parametrize("nbr_dist", [1, 2])
@pytest.mark.parametrize("eps", [0.1, 0.3])
def test_gc_keeps_the_constant_on_the_right_and_lorasp_does_not(eps, nbr_dist):
    pb = P.convdiff2d(16, 2.0, leaf_size=4)
    A = _dense(pb)
    one = np.ones(pb.n)
    F = _factor(pb, eps, HL.GC_CONSTANT, nbr_dist=nbr_dist)
    assert any(r.k < r.m for lv in F.levels for r in lv.supers if r.wsep)   # it truncated
    # the records are nonsymmetric: prolongation and restriction differ
    recs = [r for lv in F.levels for r in lv.supers if r.wsep and 0 < r.k < r.m]
    assert max(np.abs(r.Q - r.P.T).max() for r in recs) > 1e-3
    assert np.max(np.abs(HL.apply(F, A @ one) - one)) <= 1e-12
    Fl = _factor(pb, eps, HL.LORASP, nbr_dist=nbr_dist)
    assert np.max(np.abs(HL.apply(Fl, A @ one) - one)) > 1e-4


@pytest.mark.parametrize("nbr_dist", [1, 2])
def test_joint_compression_bounds_both_sides(nbr_dist):
    pb = P.convdiff2d(16, 2.0, leaf_size=4)
    eps = 0.2
    F = _factor(pb, eps, HL.LORASP, keep_U=True, nbr_dist=nbr_dist)
    checked = 0
    for lv in F.levels:
        for r in lv.supers:
            if not r.wsep or r.m == 0:
                continue
            U, AsW, AWs = r.U, r.AsW, r.AWs
            assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
            nb = np.linalg.norm(np.hstack([AsW, AWs.T]), 2)
            assert np.linalg.norm(AsW - U @ (U.T @ AsW), 2) <= eps * nb * (1 + 1e-12)
            assert np.linalg.norm(AWs - (AWs @ U) @ U.T, 2) <= eps * nb * (1 + 1e-12)
            checked += 1
    assert checked > 10


def test_gmres_with_the_lu_preconditioner_converges():
    pb = P.convdiff2d(32, 4.0, leaf_size=8)
    b = P.rhs(pb.n, 1)
    steps = {}
    for eps in (0.05, 0.3):
        F = _factor(pb, eps, HL.GC_CONSTANT)
        x, it, rel = HL.gmres_solve(F, pb.rowptr, pb.col, pb.val, b, rtol=1e-10)
        assert rel <= 1e-10
        steps[eps] = it
    assert steps[0.05] <= steps[0.3] <= 40
    assert steps[0.05] <= 12


def test_singular_pivot_is_reported():
    # a zero row block: A_ss is singular at the first elimination
    pb = P.convdiff2d(8, 1.0, leaf_size=4)
    val = pb.val.copy()
    rows = np.repeat(np.arange(pb.n), np.diff(pb.rowptr))
    val[rows == int(pb.perm[0])] = 0.0
    with pytest.raises(HL.Singular):
        HL.factor(pb.n, pb.rowptr, pb.col, val, pb.perm, pb.leaf_ptr, 0.1, HL.LORASP)


@pytest.mark.parametrize("nbr_dist", [1, 2])
@pytest.mark.parametrize("eps", [0.1, 0.3])
@pytest.mark.parametrize("variant", [HL.LORASP, HL.GC_CONSTANT])
@pytest.mark.parametrize("nx", [8, 12])
def test_matches_the_literal_extended_system(nx, variant, eps, nbr_dist):
    pb = P.convdiff2d(nx, 2.0, leaf_size=4)
    F = _factor(pb, eps, variant, nbr_dist=nbr_dist)
    E = DenseEmulator(_dense(pb), pb.perm, pb.leaf_ptr, eps, variant, nbr_dist=nbr_dist, lu=True)
    B = P.rhs(pb.n, 8, nrhs=2)
    Z = HL.apply(F, B)
    Ze = np.column_stack([E.solve(B[:, j]) for j in range(2)])
    assert np.max(np.abs(Z - Ze)) <= 1e-12 * np.max(np.abs(Ze))


@pytest.mark.parametrize("nbr_dist", [1, 2])
@pytest.mark.parametrize("eps", [0.1, 0.3])
def test_gc_user_keeps_the_callers_vectors_on_the_right(eps, nbr_dist):
    """Sec. 6 with caller-supplied vectors (one, then two): A_H^-1 (A phi) =
    phi on the nonsymmetric input; the literal extended system agrees."""
    pb = P.convdiff2d(16, 2.0, leaf_size=4)
    A = _dense(pb)
    p1 = P.laplacian_eigvec_2d(16, 16, 1, 2)
    Phi = np.column_stack([p1, P.laplacian_eigvec_2d(16, 16, 2, 1)])
    for phi in (p1, Phi):
        F = _factor(pb, eps, HL.GC_USER, nbr_dist=nbr_dist, phi=phi)
        assert np.max(np.abs(HL.apply(F, A @ phi) - phi)) <= 1e-12 * np.max(np.abs(phi))
    E = DenseEmulator(A, pb.perm, pb.leaf_ptr, eps, HL.GC_USER, phi=p1, nbr_dist=nbr_dist, lu=True)
    F = _factor(pb, eps, HL.GC_USER, nbr_dist=nbr_dist, phi=p1)
    b = P.rhs(pb.n, 4)
    zb = E.solve(b)
    assert np.max(np.abs(HL.apply(F, b) - zb)) <= 1e-12 * np.max(np.abs(zb))
