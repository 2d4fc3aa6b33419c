"""Brute-force dense emulator of the extended system -- TEST INFRASTRUCTURE.

An independent check of the block-sparse oracle on tiny grids.  It keeps one
dense matrix over all current unknowns and, for every super node, literally
builds the extended matrix of Sec. 3.2 (eq. extended_rearranged): unknowns
[x_s, y_b, rest, y_r] with the well-separated block replaced by U R^T and moved
onto the black/red pair, then eliminates the pivot [x_s, y_b] by an explicit
dense Schur complement K_rest - C P^-1 C^T (eq. eliminated).  The solve replays
the eliminations as plain block forward/backward substitution with P^-1.

It shares no arithmetic with oracle/hsolver.py: blocks are found from the
nonzero pattern of the dense matrix, adjacency from the original matrix,
compression is recomputed from the dense well-separated block, and no M_ss or
P_ss is ever formed.  Only the truncation rule (Sec. 3.2 / Sec. 6, readings
R2-R5 of the oracle) is the same by definition.

With lu=True the matrix may be nonsymmetric (reading R16 of the LU variant,
oracle/hsolver_lu.py): the basis U compresses [A_sw, A_ws^T] jointly, the
extended matrix keeps A_ws U in the rest rows of the red column and U^T A_sw
in the red row's rest columns, and the pivot's lower and upper couplings are
kept apart (no transposes), so the same literal construction checks the LU
variant.
"""
from __future__ import annotations

import math

import numpy as np

LORASP, GC_CONSTANT, GC_USER, GC_PROJ = 0, 1, 2, 3


def _orth_phi(phi_s, a):
    # candidates: every column of phi_s, then every column of a (Sec. 6, one or
    # several preserved vectors)
    m = len(phi_s)
    cand = list(np.reshape(phi_s, (m, -1)).T) + list(np.reshape(a, (m, -1)).T)
    cols = []
    for c in cand:
        nc = np.linalg.norm(c)
        if nc == 0:
            continue
        v = np.array(c, dtype=float)
        if cols:
            for _ in range(2):
                for u in cols:
                    v -= u * (u @ v)
        if np.linalg.norm(v) > 1e-12 * nc:
            cols.append(v / np.linalg.norm(v))
    return np.array(cols).T.reshape(m, len(cols))


def _proj_phi(phi_s, a, eps1):
    # Appendix B, one-sided projection: dominant left singular subspace of [X_s, A_sw X_w]
    m = len(phi_s)
    C = np.hstack([np.reshape(phi_s, (m, -1)), np.reshape(a, (m, -1))])
    u, sv, _ = np.linalg.svd(C, full_matrices=False)
    if sv[0] == 0:
        return np.zeros((m, 0))
    return u[:, : int(np.sum(sv > max(eps1, 1e-12) * sv[0]))]


def _truncate(B, eps, variant, phi_s, phi_w, eps1=0.0):
    m = B.shape[0]
    if variant == LORASP:
        if eps == 0:
            return np.eye(m)
        u, sv, _ = np.linalg.svd(B)
        return u[:, : int(np.sum(sv > eps * sv[0]))]
    U1 = _proj_phi(phi_s, B @ phi_w, eps1) if variant == GC_PROJ else _orth_phi(phi_s, B @ phi_w)
    if eps == 0:
        q, _ = np.linalg.qr(np.hstack([U1, np.eye(m)]))
        return np.hstack([U1, q[:, U1.shape[1]:m]])
    C = (np.eye(m) - U1 @ U1.T) @ B
    u, sv, _ = np.linalg.svd(C)
    nb = np.linalg.svd(B, compute_uv=False)[0]
    return np.hstack([U1, u[:, : int(np.sum(sv > eps * nb))]])


class DenseEmulator:
    """Dense extended-system factorization; `solve(b)` returns A_H^-1 b."""

    def __init__(self, A_dense, perm, leaf_ptr, eps, variant=GC_CONSTANT, phi=None, eps1=0.0, nbr_dist=1,
                 lu=False):
        n = A_dense.shape[0]
        self.lu = lu
        perm = np.asarray(perm)
        self.perm = perm
        Ap = A_dense[np.ix_(perm, perm)]
        nleaf = len(leaf_ptr) - 1
        L = int(round(math.log2(nleaf)))
        cells = [np.arange(leaf_ptr[i], leaf_ptr[i + 1]) for i in range(nleaf)]
        # leaf adjacency from the original pattern
        pattern = Ap != 0

        def touching(la, lb):
            return bool(pattern[np.ix_(np.concatenate([cells[a] for a in la]),
                                       np.concatenate([cells[b] for b in lb]))].any())

        self.level_sets = []     # leaf sets of the current level's super nodes

        def adjacent(la, lb):
            if touching(la, lb):
                return True
            # distance 2: a super node of this level touches both
            return nbr_dist == 2 and any(touching(la, lz) and touching(lz, lb) and set(lz) != set(la)
                                         and set(lz) != set(lb) for lz in self.level_sets)

        self.eps1 = eps1
        phi0 = np.asarray(phi, dtype=float)[perm] if variant in (GC_USER, GC_PROJ) else np.ones(n)
        # current system: matrix K over unknowns; groups: key -> (index list, leaf set)
        K = Ap.copy()
        vphi = phi0.copy()
        groups = {("leaf", i): (list(range(leaf_ptr[i], leaf_ptr[i + 1])), (i,)) for i in range(nleaf)}
        self.steps = []       # (pivot idx, rest idx, P, C, n_new) per elimination
        red_of_level = [("leaf", i) for i in range(nleaf)]
        for lev in range(L, 1, -1):
            nsup = 2 ** (lev - 1)
            supers = []
            for i in range(nsup):
                parts = [red_of_level[c] for c in (2 * i, 2 * i + 1) if red_of_level[c] is not None]
                if not parts:
                    continue
                idx = sum((groups[p][0] for p in parts), [])
                leaves = sum((groups[p][1] for p in parts), ())
                for p in parts:
                    del groups[p]
                groups[("s", lev, i)] = (idx, leaves)
                supers.append(("s", lev, i))
            self.level_sets = [groups[s][1] for s in supers]
            new_red = [None] * nsup

            def coupled(g, h):
                return bool(np.any(K[np.ix_(groups[g][0], groups[h][0])] != 0))

            remaining = list(supers)
            while remaining:
                wave = []
                for s in remaining:
                    if all(not coupled(s, t) for t in wave):
                        wave.append(s)
                remaining = [s for s in remaining if s not in wave]
                for s in wave:
                    K, vphi = self._eliminate(K, vphi, groups, s, adjacent, eps, variant, new_red, lev)
            red_of_level = new_red
        # root
        self.K_root = K
        self.root_groups = list(groups)

    def _eliminate(self, K, vphi, groups, s, adjacent, eps, variant, new_red, lev):
        Is, ls = groups[s]
        others = [g for g in sorted(groups, key=str) if g != s and np.any(K[np.ix_(Is, groups[g][0])] != 0)]
        N = [g for g in others if adjacent(ls, groups[g][1])]
        W = [g for g in others if not adjacent(ls, groups[g][1])]
        Iw = sum((groups[g][0] for g in W), [])
        m = len(Is)
        total = K.shape[0]
        rest = [i for i in range(total) if i not in set(Is)]
        if W and self.lu:
            # one basis for both sides: [A_sw, A_ws^T]; GC candidates A_sw phi_w
            B = np.hstack([K[np.ix_(Is, Iw)], K[np.ix_(Iw, Is)].T])
            U = _truncate(B, eps, variant, vphi[Is], np.concatenate([vphi[Iw], np.zeros(len(Iw))]), self.eps1)
        elif W:
            B = K[np.ix_(Is, Iw)]
            U = _truncate(B, eps, variant, vphi[Is], vphi[Iw], self.eps1)
        else:
            U = np.zeros((m, 0))
        k = U.shape[1]
        # extended matrix over [x_s, y_b, rest, y_r]
        nr = len(rest)
        E = np.zeros((m + k + nr + k, m + k + nr + k))
        sl_s = slice(0, m)
        sl_b = slice(m, m + k)
        sl_o = slice(m + k, m + k + nr)
        sl_r = slice(m + k + nr, m + 2 * k + nr)
        E[sl_s, sl_s] = K[np.ix_(Is, Is)]
        E[sl_o, sl_o] = K[np.ix_(rest, rest)]
        Ksr = K[np.ix_(Is, rest)].copy()
        wpos = [rest.index(i) for i in Iw]
        Ksr[:, wpos] = 0.0                     # A_sw moved onto the black/red nodes
        E[sl_s, sl_o] = Ksr
        if self.lu:
            Krs = K[np.ix_(rest, Is)].copy()
            Krs[wpos, :] = 0.0                 # A_ws moved onto the red node
            E[sl_o, sl_s] = Krs
        else:
            E[sl_o, sl_s] = Ksr.T
        E[sl_s, sl_b] = U
        E[sl_b, sl_s] = U.T
        E[sl_b, sl_r] = -np.eye(k)
        E[sl_r, sl_b] = -np.eye(k)
        R = (U.T @ K[np.ix_(Is, Iw)]).T         # (U^T A_sw)^T
        Rfull = np.zeros((nr, k))
        Rfull[wpos, :] = R
        if self.lu:
            Rcol = np.zeros((nr, k))
            Rcol[wpos, :] = K[np.ix_(Iw, Is)] @ U   # A_ws U
            E[sl_o, sl_r] = Rcol
        else:
            E[sl_o, sl_r] = Rfull
        E[sl_r, sl_o] = Rfull.T
        piv = list(range(0, m + k))
        keep = list(range(m + k, m + 2 * k + nr))
        P = E[np.ix_(piv, piv)]
        C = E[np.ix_(keep, piv)]
        Cu = E[np.ix_(piv, keep)]
        Knew = E[np.ix_(keep, keep)] - C @ np.linalg.solve(P, Cu)
        # bookkeeping: map old rest indices -> new positions 0..nr-1, red at the end
        self.steps.append((Is, rest, P, C, Cu, m, k))
        pos = {old: i for i, old in enumerate(rest)}
        del groups[s]
        for g in list(groups):
            idx, lv = groups[g]
            groups[g] = ([pos[i] for i in idx], lv)
        newphi = vphi[rest]
        if W:
            key = ("r", lev, s[2])
            groups[key] = (list(range(nr, nr + k)), ls)
            new_red[s[2]] = key
            newphi = np.concatenate([newphi, U.T @ vphi[Is]])
        else:
            Knew = Knew[:nr, :nr]
        return Knew, newphi

    def solve(self, b):
        b = np.asarray(b, dtype=np.float64)
        cur = b[self.perm]
        saved = []
        for (Is, rest, P, C, Cu, m, k) in self.steps:
            top = np.concatenate([cur[Is], np.zeros(k)])
            lower = np.concatenate([cur[rest], np.zeros(k)])
            lower = lower - C @ np.linalg.solve(P, top)
            saved.append(top)
            cur = lower if k else lower[: len(rest)]
        x = np.linalg.solve(self.K_root, cur) if cur.size else cur
        for (Is, rest, P, C, Cu, m, k), top in zip(reversed(self.steps), reversed(saved)):
            psi = x
            xtop = np.linalg.solve(P, top - Cu @ psi)
            full = np.empty(len(rest) + m)
            full[rest] = psi[: len(rest)]
            full[Is] = xtop[:m]
            x = full
        out = np.empty_like(x)
        out[self.perm] = x
        return out

