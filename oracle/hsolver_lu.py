"""FP64 CPU oracle of the nonsymmetric (LU) variant of the hierarchical
solver -- TEST INFRASTRUCTURE.

Like oracle/hsolver.py, this is a plain, slow statement of what the method
computes; only the test suite may import it.  The CUDA library has no LU
variant: this module defines and pins it.

The paper treats SPD matrices only (Sec. 2) and writes its elimination as a
Cholesky factorization (Sec. 3.2); it names GMRES as the outer solver of its
experiments (Sec. 7).  For a nonsymmetric A with a structurally symmetric
pattern this module takes the following reading (R16):

  * Blocks A_xy and A_yx are independent (no transpose relation).
  * Compression (Sec. 3.2 eq. local_compression, generalised): one
    orthonormal basis U (m x k) serves both sides of super node s.  U spans
    the leading left singular vectors of B = [A_sW, A_Ws^T] with
    sigma_i > eps ||B||_2, so that A_sW ~ U U^T A_sW and A_Ws ~ A_Ws U U^T.
    GC (Sec. 6): U = [U_1, U_2], U_1 = orth[phi_s, A_sW phi_W], U_2 from the
    truncated SVD of (I - U_1 U_1^T) B at the same threshold.  Then A_H phi =
    A phi (the right-hand preservation of Sec. 6: A_sW phi_W and phi_s lie in
    span U).
  * Extension and elimination (the nonsymmetric counterpart of eqs.
    extended_rearranged and eliminated), with Y = A_ss^-1 U,
    Z^T = U^T A_ss^-1 and S = U^T A_ss^-1 U (k x k):
      M_ss = A_ss^-1 - Y S^-1 Z^T
      P_ss = S^-1 Z^T                 (restriction; P_ss of Appendix A)
      Q_ss = Y S^-1                   (prolongation; P_ss^T when A = A^T)
      Schur update on the neighbours, every ordered pair (n, n'):
        A_nn' <- A_nn' - A_ns M_ss A_sn'
      red node r: A_rr = S^-1, A_nr = A_ns Q_ss, A_rn = P_ss A_sn,
        A_wr = A_Ws U (per w), A_rw = U^T A_sW, phi_r = U^T phi_s.
    For A = A^T every quantity reduces to the symmetric one (Q_ss = P_ss^T,
    A_rn = A_nr^T), which the tests use as a pin against oracle/hsolver.py.
  * Apply (Algorithm 2, generalised): forward in elimination order,
    phi_n -= A_ns M_ss phi_s and phi_r += P_ss phi_s; the parent solve; backward
    in reverse order, x_s = M_ss (phi_s - sum_n A_sn x_n) + Q_ss x_r.
  * Pivots: A_ss^-1 by LU with partial pivoting; a singular A_ss or S raises
    Singular (the counterpart of NOT_SPD).  The root: dense LU.

Everything else (leaves, merge, adjacency R1, canonical waves R4, R5, R6,
tolerance R2, GC basis R3) is as in oracle/hsolver.py, whose helpers this
module calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from oracle import hsolver as H

LORASP = H.LORASP
GC_CONSTANT = H.GC_CONSTANT
GC_USER = H.GC_USER


class Singular(RuntimeError):
    """A pivot block (A_ss, S or the root) is singular."""


@dataclass
class LuRecord:
    key: int
    wave: int
    m: int
    k: int
    nbrs: list
    A_sn: list          # A_{s n}, m x |n|
    A_ns: list          # A_{n s}, |n| x m
    M: np.ndarray       # M_ss, m x m
    P: np.ndarray       # P_ss, k x m (restriction)
    Q: np.ndarray       # Q_ss, m x k (prolongation)
    wsep: list
    margin: float = math.inf
    U: object = None        # the basis (keep_U)
    AsW: object = None      # A_sW at elimination time (keep_U)
    AWs: object = None      # A_Ws at elimination time (keep_U)


@dataclass
class LuLevel:
    level: int
    nsup: int
    sup_size: dict
    red_size: dict
    supers: list = field(default_factory=list)


@dataclass
class LuFactor:
    n: int
    perm: np.ndarray
    leaf_ptr: np.ndarray
    L: int
    levels: list
    root_size: int
    root_lu: object
    eps: float
    variant: int


def _leaf_blocks_full(n, rowptr, col, val, perm, leaf_ptr):
    """Every block A[I_i, I_j] of the leaf partition with a structural
    nonzero, each orientation from its own entries, and the leaf adjacency."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    nleaf = len(leaf_ptr) - 1
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    leaf_of = np.repeat(np.arange(nleaf), np.diff(leaf_ptr))
    sizes = np.diff(leaf_ptr)
    blocks, adj = {}, set()
    for i in range(n):
        pi = inv[i]
        a = leaf_of[pi]
        for e in range(rowptr[i], rowptr[i + 1]):
            pj = inv[col[e]]
            b = leaf_of[pj]
            blk = blocks.get((a, b))
            if blk is None:
                blk = blocks[(a, b)] = np.zeros((sizes[a], sizes[b]))
            blk[pi - leaf_ptr[a], pj - leaf_ptr[b]] += val[e]
            if a != b:
                adj.add((a, b))
                adj.add((b, a))
    for (a, b) in list(blocks):
        if (b, a) not in blocks:
            raise ValueError("the pattern must be structurally symmetric")
    return blocks, adj


def factor(n, rowptr, col, val, perm, leaf_ptr, eps, variant=LORASP, keep_U=False, nbr_dist=1,
           phi=None) -> LuFactor:
    """Hierarchical LU factorization (Algorithm 1 with the R16 elimination).
    variant: LORASP, GC_CONSTANT (right-hand preservation of the constant) or
    GC_USER (of the caller's vectors phi: an n-vector, or n x p for several,
    original ordering).
    keep_U: keep each compressed node's basis U and blocks A_sW, A_Ws in its
    record.  nbr_dist: the neighbour rule, 1 (R1) or 2 (R14, as in
    oracle/hsolver.py); only with 2 do compressed super nodes of the
    five-point problems still have neighbours when they are eliminated."""
    perm = np.asarray(perm, dtype=np.int64)
    leaf_ptr = np.asarray(leaf_ptr, dtype=np.int64)
    nleaf = len(leaf_ptr) - 1
    L = int(round(math.log2(nleaf)))
    if 2 ** L != nleaf:
        raise ValueError("number of leaves must be a power of two")
    if variant not in (LORASP, GC_CONSTANT, GC_USER):
        raise ValueError("variant must be LORASP, GC_CONSTANT or GC_USER")
    blocks, leaf_adj = _leaf_blocks_full(n, rowptr, col, val, perm, leaf_ptr)
    use_phi = variant in (GC_CONSTANT, GC_USER)
    phi_perm = np.asarray(phi, dtype=np.float64)[perm] if variant == GC_USER else np.ones(n)
    red_size = {i: int(leaf_ptr[i + 1] - leaf_ptr[i]) for i in range(nleaf)}
    red_leaves = {i: (i,) for i in range(nleaf)}
    red_phi = {i: phi_perm[leaf_ptr[i]:leaf_ptr[i + 1]].copy() for i in range(nleaf)}
    levels = []
    for lev in range(L, 1, -1):
        nsup = 2 ** (lev - 1)
        owner = {}
        for i in range(nsup):
            for c in (2 * i, 2 * i + 1):
                for a in red_leaves.get(c, ()):
                    owner[a] = i
        coarse_adj = {(owner[a], owner[b]) for a, b in leaf_adj
                      if a in owner and b in owner and owner[a] != owner[b]}
        if nbr_dist == 2:
            direct = {}
            for x, y in coarse_adj:
                direct.setdefault(x, set()).add(y)
            coarse_adj = coarse_adj | {(x, y) for x in direct for z in direct[x] for y in direct.get(z, ())
                                       if y != x}

        def adjacent(x, y):
            return ((x - nsup if x >= nsup else x), (y - nsup if y >= nsup else y)) in coarse_adj

        # merge (Sec. 3): super node i = red 2i u red 2i+1, blocks 2 x 2
        sup_size, sup_phi, sup_parts, sup_leaves = {}, {}, {}, {}
        for i in range(nsup):
            parts = [c for c in (2 * i, 2 * i + 1) if c in red_size]
            if not parts:
                continue
            sup_parts[i] = parts
            sup_leaves[i] = sum((red_leaves[c] for c in parts), ())
            sup_size[i] = sum(red_size[c] for c in parts)
            if use_phi:
                sup_phi[i] = np.concatenate([red_phi[c] for c in parts])
        cur = {}
        for (i, j) in {(a // 2, b // 2) for (a, b) in blocks}:
            blk = np.zeros((sup_size[i], sup_size[j]))
            ro = 0
            for a in sup_parts[i]:
                co = 0
                for b in sup_parts[j]:
                    if (a, b) in blocks:
                        blk[ro:ro + red_size[a], co:co + red_size[b]] = blocks[(a, b)]
                    co += red_size[b]
                ro += red_size[a]
            cur[(i, j)] = blk
        blocks = cur
        size = dict(sup_size)
        vphi = dict(sup_phi)
        nbr_of = {}
        for (i, j) in blocks:
            if i != j:
                nbr_of.setdefault(i, set()).add(j)

        def has_block(x, y):
            return y in nbr_of.get(x, ())

        lv = LuLevel(lev, nsup, sup_size, {})
        for widx, wave in enumerate(H.canonical_waves(list(sup_size), has_block)):
            for s in wave:
                rec = _eliminate(s, nsup, blocks, nbr_of, size, vphi, adjacent, eps, variant, use_phi, widx,
                                 keep_U)
                lv.supers.append(rec)
                if rec.wsep:
                    lv.red_size[s] = rec.k
        nxt = {}
        for (x, y), blk in blocks.items():
            assert x >= nsup and y >= nsup, "super node left uneliminated"
            nxt[(x - nsup, y - nsup)] = blk
        blocks = nxt
        levels.append(lv)
        red_size = dict(lv.red_size)
        red_phi = {i: vphi[nsup + i] for i in red_size} if use_phi else {}
        red_leaves = {i: sup_leaves[i] for i in red_size}
    # root (R6): dense LU of the last super node
    if L == 0:
        root_size = red_size.get(0, 0)
        A_root = blocks.get((0, 0), np.zeros((root_size, root_size)))
    else:
        parts = [c for c in (0, 1) if c in red_size]
        root_size = sum(red_size[c] for c in parts)
        A_root = np.zeros((root_size, root_size))
        ro = 0
        for a in parts:
            co = 0
            for b in parts:
                if (a, b) in blocks:
                    A_root[ro:ro + red_size[a], co:co + red_size[b]] = blocks[(a, b)]
                co += red_size[b]
            ro += red_size[a]
    root_lu = None
    if root_size:
        root_lu = sla.lu_factor(A_root, check_finite=True)
        if np.min(np.abs(np.diag(root_lu[0]))) == 0.0:
            raise Singular("the root block is singular")
    return LuFactor(n, perm, leaf_ptr, L, levels, root_size, root_lu, eps, variant)


def _set(blocks, nbr_of, x, y, blk):
    blocks[(x, y)] = blk
    if x != y:
        nbr_of.setdefault(x, set()).add(y)
        nbr_of.setdefault(y, set()).add(x)


def _eliminate(s, nsup, blocks, nbr_of, size, vphi, adjacent, eps, variant, use_phi, widx, keep_U=False):
    """Compress, extend and eliminate super node s (R16)."""
    m = size[s]
    others = sorted(nbr_of.get(s, ()))
    N = [x for x in others if adjacent(s, x)]
    W = [x for x in others if not adjacent(s, x)]
    A_ss = blocks[(s, s)]
    if W:
        wtot = sum(size[w] for w in W)
        B = np.hstack([blocks[(s, w)] for w in W] + [blocks[(w, s)].T for w in W]) if m else np.zeros((0, 2 * wtot))
        if use_phi:
            # B @ [phi_W; 0] = A_sW phi_W: the GC candidates of Sec. 6
            pw = np.concatenate([vphi[w] for w in W])
            phi_w = np.concatenate([pw, np.zeros((wtot,) + pw.shape[1:])])
            U, margin = H._compress(B, eps, variant, vphi[s], phi_w)
        else:
            U, margin = H._compress(B, eps, variant)
    else:
        U, margin = np.zeros((m, 0)), math.inf
    AsW = np.hstack([blocks[(s, w)] for w in W]) if (keep_U and W) else None
    AWs = np.vstack([blocks[(w, s)] for w in W]) if (keep_U and W) else None
    k = U.shape[1]
    if m:
        lu = sla.lu_factor(A_ss)
        if np.min(np.abs(np.diag(lu[0]))) <= 1e-14 * max(1.0, np.max(np.abs(np.diag(lu[0])))):
            raise Singular(f"super node {s}: A_ss is singular")
        Ainv = sla.lu_solve(lu, np.eye(m))
    else:
        Ainv = np.zeros((0, 0))
    Y = Ainv @ U                      # A_ss^-1 U
    Zt = U.T @ Ainv                   # U^T A_ss^-1
    S = U.T @ Y                       # U^T A_ss^-1 U
    if k:
        Slu = sla.lu_factor(S)
        if np.min(np.abs(np.diag(Slu[0]))) <= 1e-14 * max(1.0, np.max(np.abs(np.diag(Slu[0])))):
            raise Singular(f"super node {s}: S = U^T A_ss^-1 U is singular")
        Sinv = sla.lu_solve(Slu, np.eye(k))
    else:
        Sinv = np.zeros((0, 0))
    M = Ainv - Y @ Sinv @ Zt
    P = Sinv @ Zt
    Q = Y @ Sinv
    A_sn = [blocks[(s, x)].copy() for x in N]
    A_ns = [blocks[(x, s)].copy() for x in N]
    # Schur complement on the neighbours, every ordered pair
    for n1, a_n1s in zip(N, A_ns):
        t = a_n1s @ M
        for n2, a_sn2 in zip(N, A_sn):
            upd = t @ a_sn2
            old = blocks.get((n1, n2))
            _set(blocks, nbr_of, n1, n2, (old - upd) if old is not None else -upd)
    if W:
        r = nsup + s
        size[r] = k
        _set(blocks, nbr_of, r, r, Sinv)
        for x, a_sx, a_xs in zip(N, A_sn, A_ns):
            _set(blocks, nbr_of, x, r, a_xs @ Q)           # A_nr = A_ns Q_ss
            _set(blocks, nbr_of, r, x, P @ a_sx)           # A_rn = P_ss A_sn
        for w in W:
            _set(blocks, nbr_of, w, r, blocks[(w, s)] @ U)     # A_wr = A_ws U
            _set(blocks, nbr_of, r, w, U.T @ blocks[(s, w)])   # A_rw = U^T A_sw
        if use_phi:
            vphi[r] = U.T @ vphi[s]
    for x in others:
        del blocks[(s, x)]
        del blocks[(x, s)]
        nbr_of[x].discard(s)
    del blocks[(s, s)]
    nbr_of.pop(s, None)
    return LuRecord(s, widx, m, k, N, A_sn, A_ns, M, P, Q, W, margin, U if keep_U else None, AsW, AWs)


def apply(F: LuFactor, r: np.ndarray) -> np.ndarray:
    """z = A_H^-1 r (original ordering; 1-D, or 2-D with one column per rhs)."""
    r = np.asarray(r, dtype=np.float64)
    vec = r.ndim == 1
    R = r[:, None] if vec else r
    rp = R[F.perm]
    nleaf = len(F.leaf_ptr) - 1
    red = {i: rp[F.leaf_ptr[i]:F.leaf_ptr[i + 1]] for i in range(nleaf)}
    x_red = _solve_level(F, 0, red, R.shape[1])
    xp = np.vstack([x_red[i] for i in range(nleaf)])
    out = np.empty_like(R)
    out[F.perm] = xp
    return out[:, 0] if vec else out


def _solve_level(F: LuFactor, li: int, red: dict, nrhs: int) -> dict:
    if li == len(F.levels):
        parts = sorted(red)
        if not parts:
            return {}
        b = np.vstack([red[i] for i in parts])
        x = sla.lu_solve(F.root_lu, b) if F.root_size else b
        out, o = {}, 0
        for i in parts:
            ni = red[i].shape[0]
            out[i] = x[o:o + ni]
            o += ni
        return out
    lv = F.levels[li]
    nsup = lv.nsup
    phi = {i: np.vstack([red[c] for c in (2 * i, 2 * i + 1) if c in red]) for i in lv.sup_size}
    for i, k in lv.red_size.items():
        phi[nsup + i] = np.zeros((k, nrhs))
    for rec in lv.supers:                        # forward substitution, restriction
        t = rec.M @ phi[rec.key]
        for x, a_xs in zip(rec.nbrs, rec.A_ns):
            phi[x] = phi[x] - a_xs @ t
        if rec.wsep:
            phi[nsup + rec.key] = phi[nsup + rec.key] + rec.P @ phi[rec.key]
    psi = _solve_level(F, li + 1, {i: phi[nsup + i] for i in lv.red_size}, nrhs)
    x = {nsup + i: psi[i] for i in lv.red_size}
    for rec in reversed(lv.supers):              # prolongation, backward substitution
        v = phi[rec.key].copy()
        for y, a_sy in zip(rec.nbrs, rec.A_sn):
            v = v - a_sy @ x[y]
        xs = rec.M @ v
        if rec.wsep:
            xs = xs + rec.Q @ x[nsup + rec.key]
        x[rec.key] = xs
    out = {}
    for i in lv.sup_size:
        o = 0
        for c in (2 * i, 2 * i + 1):
            if c in red:
                nc = red[c].shape[0]
                out[c] = x[i][o:o + nc]
                o += nc
    return out


def gmres_solve(F: LuFactor, rowptr, col, val, b, rtol=1e-10, maxit=300, restart=0):
    """Right-preconditioned GMRES with this factorization (Sec. 7's outer
    solver; the same iteration as oracle.hsolver.gmres_solve)."""
    return H.gmres_solve(None, rowptr, col, val, b, rtol, maxit, restart, precond=lambda v: apply(F, v))
