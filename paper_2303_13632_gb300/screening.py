"""Schwarz screening and 8-fold unique quartet enumeration (input preparation of the
batched workload; not part of the timed path).

Pairs (i, j) are unordered with the larger angular momentum first.  A quartet of pairs
(P, Q) is kept when Q_P Q_Q >= tau, where Q_P = sqrt(max |(ab|ab)|) over the pair's
components (Cauchy-Schwarz: |(ab|cd)| <= sqrt((ab|ab)(cd|cd)), and the largest entry of
the positive semidefinite matrix (ab|a'b') lies on its diagonal).  Of the eight equivalent
orderings (Sec. II-B) one is kept: the pair whose class has more components is the bra
(canonical classes, Eq. 3); for pairs of the same class the bra has the lower rank in the
list sorted by decreasing Q.  Every unique screened quartet is thus a quartet of one of the
55 canonical classes.
"""
from __future__ import annotations

import numpy as np

from .workloads import ShellSet, shell_size


def unique_pairs(shells: ShellSet) -> np.ndarray:
    """[n_pairs, 2] shell ids (i, j), i != j or i == j, each unordered pair once, the shell
    with the larger L (then the larger id) first."""
    n = len(shells.L)
    i, j = np.triu_indices(n)
    L = np.asarray(shells.L)
    swap = (L[i] < L[j]) | ((L[i] == L[j]) & (i < j))
    a = np.where(swap, j, i)
    b = np.where(swap, i, j)
    return np.stack([a, b], axis=1).astype(np.int32)


def pair_class(shells: ShellSet, pairs: np.ndarray) -> np.ndarray:
    L = np.asarray(shells.L)
    return (L[pairs[:, 0]] * 4 + L[pairs[:, 1]]).astype(np.int32)


def pair_size(pc) -> np.ndarray:
    pc = np.asarray(pc)
    return np.array([shell_size(p // 4) * shell_size(p % 4) for p in np.ravel(pc)]).reshape(pc.shape)


class ScreenedQuartets:
    """Pairs grouped by pair class and sorted by decreasing Schwarz factor, with the counts
    of unique screened quartets per (bra pair class, ket pair class)."""

    def __init__(self, shells: ShellSet, pairs: np.ndarray, qfac: np.ndarray, tau: float):
        self.shells = shells
        self.tau = tau
        pc = pair_class(shells, pairs)
        self.groups = {}
        for c in np.unique(pc):
            sel = np.nonzero(pc == c)[0]
            order = sel[np.argsort(-qfac[sel], kind="stable")]
            self.groups[int(c)] = (pairs[order], qfac[order])
        self.combos = []  # (bra class, ket class) with bra as canonical
        for cb in self.groups:
            for ck in self.groups:
                nb, nk = pair_size(cb), pair_size(ck)
                if nb > nk or cb == ck:
                    self.combos.append((cb, ck))

    def ket_counts(self, cb: int, ck: int) -> np.ndarray:
        """Kets kept for each bra pair of class cb (in the group's order)."""
        pb, qb = self.groups[cb]
        pk, qk = self.groups[ck]
        with np.errstate(divide="ignore"):
            need = np.where(qb > 0, self.tau / qb, np.inf)
        # qk is decreasing: number of kets with qk >= need
        n = np.searchsorted(-qk, -need, side="right")
        if cb == ck:
            n = np.minimum(n, np.arange(len(pb)) + 1)
        return n.astype(np.int64)

    def class_counts(self):
        """{canonical class id: number of unique screened quartets}."""
        out = {}
        for cb, ck in self.combos:
            cls = cb * 16 + ck
            out[cls] = out.get(cls, 0) + int(self.ket_counts(cb, ck).sum())
        return out

    def sample(self, rng: np.random.Generator, eri_budget: int) -> np.ndarray:
        """A seeded sample of whole bra rows (a bra pair with all its kept kets) drawn over
        all class combinations until about eri_budget ERIs are collected; returns [n, 4]."""
        rows = []
        for cb, ck in self.combos:
            cnt = self.ket_counts(cb, ck)
            for r in np.nonzero(cnt > 0)[0]:
                rows.append((cb, ck, int(r), int(cnt[r])))
        order = rng.permutation(len(rows))
        quartets, eris = [], 0
        for k in order:
            cb, ck, r, n = rows[k]
            pb, _ = self.groups[cb]
            pk, _ = self.groups[ck]
            q = np.empty((n, 4), dtype=np.int32)
            q[:, 0:2] = pb[r]
            q[:, 2:4] = pk[:n]
            quartets.append(q)
            eris += n * pair_size(cb) * pair_size(ck)
            if eris >= eri_budget:
                break
        return np.concatenate(quartets) if quartets else np.zeros((0, 4), dtype=np.int32)
