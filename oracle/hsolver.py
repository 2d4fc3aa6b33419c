"""FP64 CPU oracle of the hierarchical solver (LoRaSp and GC) -- TEST INFRASTRUCTURE.

This is a plain, slow statement of what the method computes, used only to check
the CUDA library.  Only the test suite, the package's smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.

What it follows (arXiv 1611.03189, Yang, Pouransari, Darve):
  * Sec. 2.1 and Sec. 3: 2^L leaf clusters ("red nodes"), merged pairwise into
    super nodes, level by level (Algorithm 1).
  * Sec. 3.1: adjacency is taken in the original graph and never changes;
    two clusters are well separated when they are not neighbours.
  * Sec. 3.2, eqs. (local_compression)-(eliminated): compression of the
    well-separated block A_sw by truncated SVD, extension with a black node
    y_b and a red node y_r, block elimination of [x_s; y_b].
  * Sec. 6: the GC compression, U = [U_1, U_2] with U_1 an orthonormal basis
    of [phi_s, A_sw phi_w] and U_2 the truncated SVD of (I - U_1 U_1^T) A_sw;
    the parent red node preserves U^T phi_s.
  * Appendix A, Algorithm 2 with P_ss = S^-1 U^T A_ss^-1 and
    M_ss = A_ss^-1 - P_ss^T S P_ss: the solve (forward substitution,
    restriction, parent solve, prolongation, backward substitution).
  * Sec. 7: preconditioned Krylov iteration stopped at relative residual
    1e-10; the stationary iteration x_{k+1} = x_k + A_H^-1 (b - A x_k).

Readings where the paper is silent or ambiguous:
  R1 well separated = no edge of the ORIGINAL graph between the two leaf sets.
  R2 truncation: keep sigma_i > eps * ||A_sw||_2 (strict); GC applies the same
     threshold to the singular values of (I - U_1 U_1^T) A_sw.  eps = 0 means no
     truncation: the red node keeps a complete orthonormal basis (k = m).
  R3 GC basis: modified Gram-Schmidt with one re-orthogonalisation;
     u_1 = phi_s/||phi_s||, u_2 added only when the remainder of A_sw phi_w
     exceeds 1e-12 ||A_sw phi_w||.  With several preserved vectors (phi an
     m x p matrix) the candidates are the columns of phi_s, then those of
     A_sw phi_w, each kept under the same rule.
  R4 elimination order ("a given ordering", Sec. 3.2): canonical waves.  Within
     a level, repeatedly take, in ascending super-node index, a maximal set of
     super nodes no two of which share a block; eliminate that set, repeat.
  R5 a super node with no well-separated block is eliminated exactly: no
     compression and no red node (Sec. 3.2: the first super node has A_sw = 0).
     A red node exists iff its super node had a well-separated block.
  R6 the top of the tree: the last super node (level 1) is factored densely.
  R7 Algorithm 1 writes "compress A_sn, A_ns"; the compressed block is A_sw.
  R11 adaptive tolerance (Sec. 7): the paper's level l runs from the root to
     l_max at the leaves; here the super nodes of level l (l = L for the pairs of
     leaves, down to 2) play level l with l_max = L, and the tolerance list is
     indexed by j = L - l (levels above the leaves), so one list serves problems
     of different depth.
  R12 Appendix B, first-order one-sided projection (variant GC_PROJ): U_1 are
     the left singular vectors of C = [X_s, A_sw X_w] with
     sigma_i > max(eps1, 1e-12) sigma_1(C) (the 1e-12 floor drops the
     rounding-level directions of dependent columns, as R3 does); U_2 and the
     threshold eps ||A_sw||_2 are those of GC.  The appendix does not say what
     the parent red node keeps of X: as in Sec. 6, X_r = U^T X_s.  The caller
     passes the columns of X already scaled (e_i / lambda_i in the appendix).
  R15 symmetric diagonal scaling (an option the paper does not mention): the
     factorization of D^-1/2 A D^-1/2 (D = diag A).  With a 1e-5 coefficient
     jump, GC-constant on A itself loses definiteness (R9): the constant
     vector in U_1 mixes the O(1) rows of A_sw into the 1e-5 rows.  Scaled,
     the rows have one scale and the GMRES counts come close to Table 4.
  R14 neighbour rule of the experiments (Sec. 7 uses a geometric rule: well
     separated when the distance exceeds the cluster size; the C ABI carries
     no coordinates): with nbr_dist = 2, two super nodes of a level are also
     neighbours when they share a neighbour at that level (distance 2 in the
     level's cluster graph).  nbr_dist = 1 is R1.

Node keys inside a level: super node i -> i, red node made from super node i ->
nsup + i.  Blocks are stored in both orientations, kept consistent.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

LORASP = 0
GC_CONSTANT = 1
GC_USER = 2
GC_PROJ = 3  # Appendix B, first-order one-sided projection (R12)

MGS_DROP = 1e-12  # R3


class NotSPD(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# compression (Sec. 3.2 eq. local_compression; Sec. 6 eq. preserve)
# ---------------------------------------------------------------------------

def _columns(x) -> np.ndarray:
    """A vector or an m x p matrix as an m x p matrix."""
    x = np.asarray(x, dtype=np.float64)
    return x.reshape(x.shape[0], -1)


def gc_basis(phi_s: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Orthonormal U_1 spanning [phi_s, a] by MGS with one re-orthogonalisation (R3).

    phi_s and a = A_sw phi_w are vectors, or m x p matrices when p vectors are
    preserved; the candidates are phi_s's columns, then a's, and one is kept
    when its remainder exceeds MGS_DROP times its norm."""
    P = _columns(phi_s)
    m = P.shape[0]
    cols = []
    for c in np.hstack([P, _columns(a)]).T:
        nc = float(np.linalg.norm(c))
        if nc == 0.0:
            continue
        v = c.copy()
        for _ in range(2 if cols else 0):
            for u in cols:
                v = v - u * float(u @ v)
        nv = float(np.linalg.norm(v))
        if nv > MGS_DROP * nc:
            cols.append(v / nv)
    if not cols:
        return np.zeros((m, 0))
    return np.column_stack(cols)


def proj_basis(C: np.ndarray, eps1: float) -> np.ndarray:
    """Appendix B (first-order one-sided projection), first truncated SVD: the
    left singular vectors of C = [X_s, A_sw X_w] with
    sigma_i > max(eps1, MGS_DROP) sigma_1(C) (R12)."""
    C = _columns(C)
    m = C.shape[0]
    if C.size == 0:
        return np.zeros((m, 0))
    Uc, sc, _ = np.linalg.svd(C, full_matrices=False)
    if sc[0] == 0.0:
        return np.zeros((m, 0))
    k = int(np.count_nonzero(sc > max(eps1, MGS_DROP) * sc[0]))
    return Uc[:, :k].copy()


def complete_basis(U1: np.ndarray, m: int) -> np.ndarray:
    """Orthonormal basis of the complement of span(U1): eigenvectors of
    I - U1 U1^T with eigenvalue 1."""
    P = np.eye(m) - U1 @ U1.T
    w, V = np.linalg.eigh(P)
    return V[:, w > 0.5]


def _margin(sv: np.ndarray, thr: float) -> float:
    """min_i |sv_i - thr| / thr (inf for thr = 0 or no values)."""
    if thr <= 0.0 or sv.size == 0:
        return math.inf
    return float(np.min(np.abs(sv - thr)) / thr)


def compress(B: np.ndarray, eps: float, variant: int, phi_s=None, phi_w=None, eps1: float = 0.0):
    """Return U (m x k, orthonormal columns) for the well-separated block B = A_sw.

    LoRaSp: leading left singular vectors of B with sigma_i > eps ||B||_2.
    GC: U = [U_1, U_2], U_1 = orth[phi_s, B phi_w], U_2 = leading left singular
    vectors of (I - U_1 U_1^T) B with sigma_i > eps ||B||_2.
    GC_PROJ (Appendix B): as GC, with U_1 the left singular vectors of
    [phi_s, B phi_w] above eps1 times its norm (R12).
    """
    return _compress(B, eps, variant, phi_s, phi_w, eps1)[0]


def _gap_margin(sv: np.ndarray, j: int) -> float:
    """Relative gap (sv[j-1] - sv[j]) / sv[j-1] where a rank cap of j cuts the
    descending list sv (inf when nothing is cut)."""
    if j <= 0 or j >= sv.size or sv[j - 1] <= 0.0:
        return math.inf
    return float((sv[j - 1] - sv[j]) / sv[j - 1])


def _compress(B: np.ndarray, eps: float, variant: int, phi_s=None, phi_w=None, eps1: float = 0.0, cap=None):
    """compress(), and the margin of its rank decisions (SuperRecord.margin).
    cap: the largest rank kept (max_rank_ratio; None: no cap): the leading
    singular vectors, the GC basis U_1 always whole; a cap that binds adds the
    relative gap at the cut to the margin."""
    m = B.shape[0]
    if m == 0:
        return np.zeros((0, 0)), math.inf
    if variant == LORASP:
        if eps == 0.0:
            return np.eye(m), math.inf
        Ub, sb, _ = np.linalg.svd(B, full_matrices=False)
        normB = sb[0] if sb.size else 0.0
        k = int(np.count_nonzero(sb > eps * normB))
        margin = _margin(sb, eps * normB)
        if cap is not None and k > cap:
            k = cap
            margin = min(margin, _gap_margin(sb, cap))
        return Ub[:, :k].copy(), margin
    margin = math.inf
    if variant == GC_PROJ:
        C1 = np.hstack([_columns(phi_s), _columns(B @ phi_w)])
        U1 = proj_basis(C1, eps1)
        s1 = np.linalg.svd(C1, compute_uv=False)
        if s1.size and s1[0] > 0.0:
            margin = _margin(s1, max(eps1, MGS_DROP) * s1[0])
    else:
        U1 = gc_basis(phi_s, B @ phi_w)
    if eps == 0.0:
        return np.hstack([U1, complete_basis(U1, m)]), margin
    normB = float(np.linalg.svd(B, compute_uv=False)[0]) if B.size else 0.0
    C = B - U1 @ (U1.T @ B)
    Uc, sc, _ = np.linalg.svd(C, full_matrices=False)
    k2 = int(np.count_nonzero(sc > eps * normB))
    margin = min(margin, _margin(sc, eps * normB))
    if cap is not None:
        lim = max(cap - U1.shape[1], 0)
        if k2 > lim:
            k2 = lim
            margin = min(margin, _gap_margin(sc, lim))
    return np.hstack([U1, Uc[:, :k2]]), margin


# ---------------------------------------------------------------------------
# factorization records
# ---------------------------------------------------------------------------

@dataclass
class SuperRecord:
    """What the solve needs from the elimination of one super node."""

    key: int
    wave: int
    m: int
    k: int
    nbrs: list            # keys of N(s), ascending
    A_sn: list            # A_{s n} blocks, m x |n|
    M: np.ndarray         # M_ss = A_ss^-1 - P_ss^T S P_ss   (m x m)
    P: np.ndarray         # P_ss = S^-1 U^T A_ss^-1          (k x m)
    wsep: list = field(default_factory=list)   # keys of W(s), for inspection
    U: np.ndarray | None = None
    # smallest relative distance |sigma_i - threshold| / threshold among the
    # singular values behind this node's rank decisions (inf when none): ranks
    # from another implementation may differ only where this is tiny
    margin: float = math.inf


@dataclass
class LevelRecord:
    level: int
    nsup: int
    sup_size: dict        # super index -> size
    red_size: dict        # red index (next level) -> size
    supers: list          # SuperRecord in elimination order
    waves: list           # list of lists of super indices


@dataclass
class Factor:
    n: int
    perm: np.ndarray
    leaf_ptr: np.ndarray
    L: int
    levels: list          # LevelRecord, leaf level first
    root_size: int
    root_chol: np.ndarray | None
    eps: float
    variant: int
    partial: bool = False  # only the first levels were factored (no solve)
    dscale: np.ndarray | None = None  # R15: D^-1/2 (original order) when scaled

    def ranks(self):
        """{level: {super index: k}} for every super node with a red node."""
        out = {}
        for lv in self.levels:
            out[lv.level] = {r.key: r.k for r in lv.supers if r.wsep}
        return out


# ---------------------------------------------------------------------------
# symbolic helpers
# ---------------------------------------------------------------------------

def _leaf_blocks(n, rowptr, col, val, perm, leaf_ptr):
    """Dense leaf blocks A[I_a, I_b] of the permuted matrix, and the leaf adjacency."""
    nleaf = len(leaf_ptr) - 1
    iperm = np.empty(n, dtype=np.int64)
    iperm[np.asarray(perm, dtype=np.int64)] = np.arange(n)
    leaf_of = np.repeat(np.arange(nleaf), np.diff(leaf_ptr))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    pr = iperm[rows]
    pc = iperm[np.asarray(col, dtype=np.int64)]
    la, lb = leaf_of[pr], leaf_of[pc]
    ra = pr - leaf_ptr[la]
    cb = pc - leaf_ptr[lb]
    blocks = {}
    order = np.lexsort((lb, la))
    la, lb, ra, cb, v = la[order], lb[order], ra[order], cb[order], np.asarray(val)[order]
    bounds = np.flatnonzero(np.diff(la * nleaf + lb)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [len(la)]])
    adj = set()
    for s0, e0 in zip(starts, ends):
        a, b = int(la[s0]), int(lb[s0])
        blk = np.zeros((leaf_ptr[a + 1] - leaf_ptr[a], leaf_ptr[b + 1] - leaf_ptr[b]))
        np.add.at(blk, (ra[s0:e0], cb[s0:e0]), v[s0:e0])
        blocks[(a, b)] = blk
        if a != b:
            adj.add((a, b))
    return blocks, adj


def canonical_waves(supers, has_block):
    """R4: greedy maximal sets in ascending index with no block between members."""
    remaining = sorted(supers)
    while remaining:
        wave = []
        for s in remaining:
            if all(not has_block(s, t) for t in wave):
                wave.append(s)
        taken = set(wave)
        remaining = [s for s in remaining if s not in taken]
        yield wave          # the caller eliminates the wave before the next one is formed


# ---------------------------------------------------------------------------
# factorization (Algorithm 1)
# ---------------------------------------------------------------------------

def eps_schedule_gc(eps: float, L: int) -> list:
    """Adaptive tolerance of the GC variant (Sec. 7, Table 3): eps_l =
    eps 2^((l - l_max)/3), constant eps at the leaf level and smaller towards
    the root.  Entry j is the tolerance of the super nodes j levels above the
    leaves (level L - j, R11); L - 1 entries cover levels L..2."""
    return [eps * 2.0 ** (-j / 3.0) for j in range(L - 1)]


def eps_schedule_lorasp(eps: float, L: int, h: float) -> list:
    """Adaptive tolerance of LoRaSp in Sec. 7 (the HChols-like choice with one
    factor h dropped): eps_l = eps h 2^((l_max - l)/3), small at the leaves and
    growing towards the root; h is the grid spacing.  Indexed like
    eps_schedule_gc."""
    return [eps * h * 2.0 ** (j / 3.0) for j in range(L - 1)]


def factor(n, rowptr, col, val, perm, leaf_ptr, eps, variant=GC_CONSTANT, phi=None,
           order="waves", keep_U=False, eps_level=None, eps1=0.0, nbr_dist=1, levels=None,
           scale=False, max_rank_ratio=0.0) -> Factor:
    """Hierarchical factorization.

    n, rowptr, col, val: CSR of the SPD matrix A in original ordering.
    perm, leaf_ptr: clustering; perm[p] = original index of unknown p.
    eps: truncation tolerance (R2).  variant: LORASP, GC_CONSTANT, GC_USER or
        GC_PROJ (Appendix B; eps1 is its first tolerance, R12).
    eps_level: optional per-level tolerances (Sec. 7 adaptive choice): entry j
        is used instead of eps for the super nodes j levels above the leaves
        (level L - j); it needs L - 1 entries.
    phi: for GC_USER and GC_PROJ, the vector to preserve (original ordering),
        or an n x p array of p vectors.
    nbr_dist: 1, neighbours are joined by an edge of the original graph (R1);
        2, also the nodes of a level that share a neighbour (R14).
    levels: factor only that many levels above the leaves and return a
        partial record (ranks and margins to compare; it cannot be applied).
    scale: factor D^-1/2 A D^-1/2 (D = diag A) instead of A (R15); apply()
        then returns D^-1/2 A_H'^-1 D^-1/2 r.  GC-constant preserves the
        constant vector of the scaled system; GC_USER / GC_PROJ vectors are
        mapped to it (D^1/2 phi), so that they stay preserved for A.
    order: "waves" (R4), "waves-reversed" (same waves, each eliminated in
        descending order) or "sequential" (ascending super index, one at a time).
    max_rank_ratio: 0, or a cap on the rank of every truncation (eps > 0):
        k <= max(floor(ratio m), 1), keeping the leading singular vectors (GC:
        U_1 whole, then the leading ones of the projected block).  Not in the
        paper: a bound on the size of the red nodes a caller may impose.
    """
    rowptr = np.asarray(rowptr, dtype=np.int64)
    perm = np.asarray(perm, dtype=np.int64)
    leaf_ptr = np.asarray(leaf_ptr, dtype=np.int64)
    nleaf = len(leaf_ptr) - 1
    L = int(round(math.log2(nleaf)))
    if 2 ** L != nleaf:
        raise ValueError("number of leaves must be a power of two")
    dscale = None
    if scale:
        # R15: symmetric diagonal scaling, D^-1/2 A D^-1/2
        rows = np.repeat(np.arange(n), np.diff(rowptr))
        col_a = np.asarray(col, dtype=np.int64)
        diag = np.zeros(n)
        np.add.at(diag, rows[rows == col_a], np.asarray(val, dtype=np.float64)[rows == col_a])
        if np.any(diag <= 0.0):
            raise NotSPD("a diagonal entry is not positive")
        dscale = 1.0 / np.sqrt(diag)
        val = np.asarray(val, dtype=np.float64) * dscale[rows] * dscale[col_a]
    blocks, leaf_adj = _leaf_blocks(n, rowptr, col, val, perm, leaf_ptr)
    use_phi = variant in (GC_CONSTANT, GC_USER, GC_PROJ)
    if variant in (GC_USER, GC_PROJ):
        ph = np.asarray(phi, dtype=np.float64)
        if dscale is not None:
            ph = ph / (dscale if ph.ndim == 1 else dscale[:, None])
        phi_perm = ph[perm]
    else:
        phi_perm = np.ones(n)

    # level-L red nodes = leaves
    red_size = {i: int(leaf_ptr[i + 1] - leaf_ptr[i]) for i in range(nleaf)}
    red_leaves = {i: (i,) for i in range(nleaf)}
    red_phi = {i: phi_perm[leaf_ptr[i]:leaf_ptr[i + 1]].copy() for i in range(nleaf)}
    all_levels = []

    if eps_level is not None and len(eps_level) < L - 1:
        raise ValueError("eps_level needs L - 1 entries (levels L..2)")
    for lev in range(L, 1, -1):
        if levels is not None and L - lev >= levels:
            return Factor(n, perm, leaf_ptr, L, all_levels, -1, None, eps, variant, partial=True, dscale=dscale)
        nsup = 2 ** (lev - 1)
        eps_l = float(eps_level[L - lev]) if eps_level is not None else eps
        # leaf sets of the super nodes: union of the leaf sets of the red nodes that
        # exist (a red node inherits the leaf set of its super node, Sec. 3.2)
        owner = {}
        for i in range(nsup):
            for c in (2 * i, 2 * i + 1):
                for a in red_leaves.get(c, ()):
                    owner[a] = i
        coarse_adj = set()
        for a, b in leaf_adj:
            if a in owner and b in owner and owner[a] != owner[b]:
                coarse_adj.add((owner[a], owner[b]))
        if nbr_dist == 2:
            # R14: also the super nodes of this level that share a neighbour
            direct = {}
            for x, y in coarse_adj:
                direct.setdefault(x, set()).add(y)
            coarse_adj = coarse_adj | {(x, y) for x in direct for z in direct[x] for y in direct.get(z, ())
                                       if y != x}

        def adjacent(x, y):
            return ((x - nsup if x >= nsup else x), (y - nsup if y >= nsup else y)) in coarse_adj

        # --- merge (Sec. 3: I^s_i = I^r_{2i-1} u I^r_{2i}) ---
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
        pairs = {}
        for (a, b) in blocks:
            pairs.setdefault((a // 2, b // 2), None)
        for (i, j) in pairs:
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

        records = []
        waves = []
        new_red_size = {}
        new_red_phi = {}
        if order in ("waves", "waves-reversed"):
            wave_iter = canonical_waves(list(sup_size), has_block)
        elif order == "sequential":
            wave_iter = ([s] for s in sorted(sup_size))
        else:
            raise ValueError(order)
        for widx, wave in enumerate(wave_iter):
            waves.append(list(wave))
            # within a wave the eliminations are independent (R4); "waves-reversed"
            # eliminates each wave in descending order to test exactly that
            for s in (reversed(wave) if order == "waves-reversed" else wave):
                rec = _eliminate(s, nsup, blocks, nbr_of, size, vphi, adjacent, eps_l,
                                 variant, use_phi, widx, keep_U, eps1, max_rank_ratio)
                records.append(rec)
                if rec.wsep:
                    new_red_size[s] = rec.k
                    if use_phi:
                        new_red_phi[s] = vphi[nsup + s]
        # --- parent level: red node nsup+i becomes red i ---
        nxt = {}
        for (x, y), blk in blocks.items():
            assert x >= nsup and y >= nsup, "super node left uneliminated"
            nxt[(x - nsup, y - nsup)] = blk
        blocks = nxt
        all_levels.append(LevelRecord(lev, nsup, sup_size, dict(new_red_size), records, waves))
        red_size = new_red_size
        red_phi = new_red_phi
        red_leaves = {i: sup_leaves[i] for i in new_red_size}

    # --- root (R6) ---
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
    root_chol = None
    if root_size:
        try:
            root_chol = np.linalg.cholesky(A_root)
        except np.linalg.LinAlgError as e:
            raise NotSPD("root block is not positive definite") from e
    return Factor(n, perm, leaf_ptr, L, all_levels, root_size, root_chol, eps, variant, dscale=dscale)


def _set_block(blocks, nbr_of, x, y, blk):
    blocks[(x, y)] = blk
    blocks[(y, x)] = blk.T.copy() if x != y else blk
    if x != y:
        nbr_of.setdefault(x, set()).add(y)
        nbr_of.setdefault(y, set()).add(x)


def rank_cap(m: int, max_rank_ratio: float):
    """Largest rank a super node of size m keeps under max_rank_ratio (None:
    no cap): floor(ratio m), at least 1."""
    if not max_rank_ratio or max_rank_ratio <= 0.0:
        return None
    return max(1, int(math.floor(max_rank_ratio * m)))


def _eliminate(s, nsup, blocks, nbr_of, size, vphi, adjacent, eps, variant, use_phi, widx,
               keep_U, eps1=0.0, max_rank_ratio=0.0):
    """Compress, extend and eliminate super node s (Sec. 3.2)."""
    m = size[s]
    cap = rank_cap(m, max_rank_ratio) if eps > 0.0 else None
    others = sorted(nbr_of.get(s, ()))
    N = [x for x in others if adjacent(s, x)]
    W = [x for x in others if not adjacent(s, x)]
    A_ss = blocks[(s, s)]

    # compression of the well-separated block (eq. local_compression / Sec. 6)
    if W:
        B = np.hstack([blocks[(s, w)] for w in W]) if m else np.zeros((0, sum(size[w] for w in W)))
        if use_phi:
            phi_w = np.concatenate([vphi[w] for w in W])
            U, margin = _compress(B, eps, variant, vphi[s], phi_w, eps1, cap)
        else:
            U, margin = _compress(B, eps, variant, cap=cap)
    else:
        U, margin = np.zeros((m, 0)), math.inf
    k = U.shape[1]

    # elimination of [x_s; y_b] (eq. extended_rearranged, K = L K_2 L^T).
    # The quantities of Sec. 3.2 and Appendix A are formed through the Cholesky
    # factor A_ss = L L^T and a Householder QR of L^-1 U = Q R (Q_perp completes
    # Q to an orthogonal matrix), never through an explicit S^-1:
    #   S        = U^T A_ss^-1 U            = R^T R
    #   P_ss     = S^-1 U^T A_ss^-1         = R^-1 Q^T L^-1
    #   M_ss     = A_ss^-1 - P_ss^T S P_ss  = L^-T (I - Q Q^T) L^-1 = (L^-T Q_perp)(L^-T Q_perp)^T
    #   A_rr     = S^-1                     = R^-1 R^-T
    #   A_nr     = A_ns A_ss^-1 U S^-1      = (L^-1 A_sn)^T Q R^-T
    #   A_ns M_ss A_sn' (the Schur term of ~~A_nn')  = (Q_perp^T L^-1 A_sn)^T (Q_perp^T L^-1 A_sn')
    try:
        Lc = np.linalg.cholesky(A_ss) if m else np.zeros((0, 0))
    except np.linalg.LinAlgError as e:
        raise NotSPD(f"super node {s}: A_ss is not positive definite") from e

    def linv(X):                      # L^-1 X
        return sla.solve_triangular(Lc, X, lower=True) if m else X

    def ltinv(X):                     # L^-T X
        return sla.solve_triangular(Lc, X, lower=True, trans="T") if m else X

    Ut = linv(U)
    Qfull, Rfull = np.linalg.qr(Ut, mode="complete") if m else (np.zeros((0, 0)), np.zeros((0, k)))
    Q, Qp, R = Qfull[:, :k], Qfull[:, k:], Rfull[:k, :]
    if k and np.min(np.abs(np.diag(R))) <= 1e-14 * max(1.0, np.max(np.abs(np.diag(R)))):
        raise NotSPD(f"super node {s}: S = U^T A_ss^-1 U is singular")
    Rinv = sla.solve_triangular(R, np.eye(k), lower=False) if k else np.zeros((0, 0))

    Gt = {n_: linv(blocks[(s, n_)]) for n_ in N}           # L^-1 A_sn
    Gp = {n_: Qp.T @ Gt[n_] for n_ in N}                    # Q_perp^T L^-1 A_sn

    # Schur complement on the neighbours: ~~A_nn' = A_nn' - A_ns M_ss A_sn'
    for i1, n1 in enumerate(N):
        for n2 in N[i1:]:
            upd = Gp[n1].T @ Gp[n2]
            if (n1, n2) in blocks:
                new = blocks[(n1, n2)] - upd
            else:
                new = -upd
            _set_block(blocks, nbr_of, n1, n2, new)

    # factor records of Appendix A
    P = Rinv @ ltinv(Q).T                                                 # R^-1 Q^T L^-1
    Wp = ltinv(Qp)
    M = Wp @ Wp.T                                                         # L^-T Q_perp Q_perp^T L^-1
    A_sn = [blocks[(s, n_)].copy() for n_ in N]
    if W:
        r = nsup + s
        size[r] = k
        _set_block(blocks, nbr_of, r, r, Rinv @ Rinv.T)              # A_rr = S^-1
        for n_ in N:                                                  # A_nr = A_ns A_ss^-1 U S^-1
            _set_block(blocks, nbr_of, n_, r, Gt[n_].T @ Q @ Rinv.T)
        for w in W:                                                   # A_wr = R, R^T = U^T A_sw
            _set_block(blocks, nbr_of, w, r, (U.T @ blocks[(s, w)]).T)
        if use_phi:
            vphi[r] = U.T @ vphi[s]                                   # Sec. 6: preserve U^T phi_s
    # remove s
    for x in others:
        del blocks[(s, x)]
        del blocks[(x, s)]
        nbr_of[x].discard(s)
    del blocks[(s, s)]
    nbr_of.pop(s, None)
    return SuperRecord(s, widx, m, k, N, A_sn, M, P, W, U if keep_U else None, margin)


# ---------------------------------------------------------------------------
# solve (Algorithm 2)
# ---------------------------------------------------------------------------

def apply(F: Factor, r: np.ndarray) -> np.ndarray:
    """z = A_H^-1 r (r in original ordering; 1-D or 2-D with columns as RHS)."""
    if F.partial:
        raise ValueError("a partial factorization (levels=...) cannot be applied")
    r = np.asarray(r, dtype=np.float64)
    if F.dscale is not None:
        # R15: A_H^-1 = D^-1/2 A_H'^-1 D^-1/2
        ds = F.dscale if r.ndim == 1 else F.dscale[:, None]
        return ds * apply(Factor(F.n, F.perm, F.leaf_ptr, F.L, F.levels, F.root_size, F.root_chol, F.eps,
                                 F.variant), ds * r)
    vec = r.ndim == 1
    R = r[:, None] if vec else r
    rp = R[F.perm]
    red = {i: rp[F.leaf_ptr[i]:F.leaf_ptr[i + 1]] for i in range(len(F.leaf_ptr) - 1)}
    x_red = _solve_level(F, 0, red, R.shape[1])
    xp = np.vstack([x_red[i] for i in range(len(F.leaf_ptr) - 1)]) if x_red else np.zeros_like(rp)
    out = np.empty_like(R)
    out[F.perm] = xp
    return out[:, 0] if vec else out


def _solve_level(F: Factor, li: int, red: dict, nrhs: int) -> dict:
    """Solve on the system whose red nodes are `red` (dict index -> rhs)."""
    if li == len(F.levels):
        # root: dense solve of the one remaining super node (or leaf if L == 0)
        parts = sorted(red)
        if not parts:
            return {}
        b = np.vstack([red[i] for i in parts])
        x = sla.cho_solve((F.root_chol, True), b) if F.root_size else b
        out, o = {}, 0
        for i in parts:
            ni = red[i].shape[0]
            out[i] = x[o:o + ni]
            o += ni
        return out
    lv = F.levels[li]
    nsup = lv.nsup
    phi = {}
    for i, sz in lv.sup_size.items():
        phi[i] = np.vstack([red[c] for c in (2 * i, 2 * i + 1) if c in red])
    for i, k in lv.red_size.items():
        phi[nsup + i] = np.zeros((k, nrhs))          # parent right-hand sides start at 0
    # forward substitution and restriction, in elimination order
    for rec in lv.supers:
        t = rec.M @ phi[rec.key]
        for n_, A_sn in zip(rec.nbrs, rec.A_sn):
            phi[n_] = phi[n_] - A_sn.T @ t              # phi_n = r_n - A_ns M_ss r_s
        if rec.wsep:
            phi[nsup + rec.key] = phi[nsup + rec.key] + rec.P @ phi[rec.key]   # restriction
    # parent level solve
    parent = {i: phi[nsup + i] for i in lv.red_size}
    psi = _solve_level(F, li + 1, parent, nrhs)
    x = {}
    for i in lv.red_size:
        x[nsup + i] = psi[i]
    # prolongation and backward substitution, in reverse elimination order
    for rec in reversed(lv.supers):
        v = phi[rec.key].copy()
        for n_, A_sn in zip(rec.nbrs, rec.A_sn):
            v = v - A_sn @ x[n_]
        xs = rec.M @ v
        if rec.wsep:
            xs = xs + rec.P.T @ x[nsup + rec.key]
        x[rec.key] = xs
    # split super solutions back into the red nodes of this level
    out = {}
    for i in lv.sup_size:
        o = 0
        for c in (2 * i, 2 * i + 1):
            if c in red:
                nc = red[c].shape[0]
                out[c] = x[i][o:o + nc]
                o += nc
    return out


# ---------------------------------------------------------------------------
# outer iterations (Sec. 7)
# ---------------------------------------------------------------------------

def csr_matvec(rowptr, col, val, x):
    import scipy.sparse as sp

    n = len(rowptr) - 1
    return sp.csr_matrix((val, col, rowptr), shape=(n, n)) @ x


def pcg(F: Factor, rowptr, col, val, b, rtol=1e-10, maxit=500):
    """Preconditioned CG, x_0 = 0, stop when ||r_k|| <= rtol ||b|| on the
    recursive residual.  Returns (x, iterations, true relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0, 0.0
    z = apply(F, r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = csr_matvec(rowptr, col, val, p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if float(np.linalg.norm(r)) <= rtol * nb:
            break
        z = apply(F, r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    true_res = float(np.linalg.norm(b - csr_matvec(rowptr, col, val, x))) / nb
    return x, it, true_res


def stationary(F: Factor, rowptr, col, val, x_star, tol=1e-6, maxit=2000):
    """x_{k+1} = x_k + A_H^-1 (b - A x_k), b = A x*, x_0 = 0; iterations until
    ||x_k - x*|| / ||x_0 - x*|| < tol (Sec. 7.1)."""
    b = csr_matvec(rowptr, col, val, x_star)
    x = np.zeros_like(x_star)
    e0 = float(np.linalg.norm(x_star))
    for it in range(1, maxit + 1):
        x = x + apply(F, b - csr_matvec(rowptr, col, val, x))
        if float(np.linalg.norm(x - x_star)) < tol * e0:
            return it
    return maxit


def gmres_solve(F: Factor, rowptr, col, val, b, rtol=1e-10, maxit=300, restart=0, precond=None):
    """Right-preconditioned GMRES (Sec. 7, Tables 2-5), x_0 = 0: Arnoldi on
    A A_H^-1 with modified Gram-Schmidt, the Hessenberg least-squares problem
    solved directly at every step, stop when its residual is below rtol ||b||;
    restart every `restart` steps (0: never), x += A_H^-1 V y at the end of a
    cycle.  Returns (x, Arnoldi steps, true relative residual).  precond:
    the map v -> A_H^-1 v (default: apply(F, v))."""
    if precond is None:
        precond = lambda v: apply(F, v)  # noqa: E731
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    m = restart if 0 < restart < maxit else maxit
    total = 0
    done = False
    while not done and total < maxit:
        r = b - csr_matvec(rowptr, col, val, x)
        beta = float(np.linalg.norm(r))
        if beta < rtol * nb:
            break
        V = [r / beta]
        Hm = np.zeros((m + 1, m))
        y = np.zeros(0)
        for j in range(m):
            if total >= maxit:
                break
            w = csr_matvec(rowptr, col, val, precond(V[j]))
            for i in range(j + 1):
                Hm[i, j] = float(V[i] @ w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = float(np.linalg.norm(w))
            total += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hm[:j + 2, :j + 1], e1, rcond=None)
            res = float(np.linalg.norm(Hm[:j + 2, :j + 1] @ y - e1))
            if res < rtol * nb or Hm[j + 1, j] == 0.0:
                done = True
                break
            V.append(w / Hm[j + 1, j])
        if y.size:
            x = x + precond(np.column_stack(V[:y.size]) @ y)
    rel = float(np.linalg.norm(b - csr_matvec(rowptr, col, val, x))) / nb
    return x, total, rel


def gmres(F: Factor, rowptr, col, val, b, rtol=1e-10, maxit=300):
    """Right-preconditioned unrestarted GMRES; iterations to ||b - A x|| < rtol ||b||."""
    return gmres_solve(F, rowptr, col, val, b, rtol, maxit)[1]
