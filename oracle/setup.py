"""AMG setup phase (Sec. 2.2): Ruge-Stueben coarsening, direct interpolation,
Galerkin coarse operators.  Plain FP64, Python loops; test infrastructure only.

Readings where the paper is silent (it names only "classical Ruge-Stueben,
theta = 0.25", Sec. 4, and "at most 10 levels", Table train_hyper):

* strength: j is a strong dependency of i iff j != i and
  -a_ij >= theta * max_{k != i} (-a_ik), with that maximum > 0;
* C/F splitting: the classical first pass only.  Points with no strong
  connection in either direction become F.  Then repeatedly the undecided
  point with the largest measure lambda becomes C (ties: lowest index) and
  its undecided strong dependents become F.  lambda_k starts at |S_k^T|;
  each time an undecided point that strongly depends on k becomes C,
  lambda_k drops by 1, and each time one becomes F it rises by 1
  (lambda = |S^T cap U| + 2 |S^T cap F|).  No second pass;
* direct interpolation (C rows identity): for an F point i with strong
  C-neighbours C_i, w_ij = -alpha_i a_ij / d_i with
  alpha_i = sum_{k != i, a_ik < 0} a_ik / sum_{k in C_i} a_ik and
  d_i = a_ii + sum_{k != i, a_ik > 0} a_ik (positive couplings lumped onto
  the diagonal; strong couplings are always negative).  An F point with no
  strong C-neighbour gets an empty row;
* Galerkin product keeps the structural pattern of P^T A P (entries that
  cancel to 0.0 stay in the pattern);
* stop coarsening when n <= max_coarse, when the hierarchy has max_levels
  levels, or when a coarse level would keep more than 90% of the points (or
  none).

Parallel split (device setup; not the paper's coarsening, which is RS): PMIS
of De Sterck, Yang and Heys (2006), on the same strength graph.  Measure
lambda_i = |S_i^T| + r_i with r_i in [0, 1) the level's random numbers
(an input: splitmix64 doubles, workloads.uniform01(seed + level, n_l)), summed
in FP64.  Points that strongly influence no point (|S_i^T| = 0) start as F.
Each round, over the undecided points U and using the states at the start of
the round: i joins C when it beats every undecided j in S_i u S_i^T
(lambda_i > lambda_j, ties to the lower index); then every undecided point
with a strong dependency among the new C points becomes F.  Rounds repeat
until no point is undecided.  Interpolation and Galerkin product as for RS.

Block-local Ruge-Stueben split (device setup, coarsening "rs-blocks"; the
domain-decomposed form of the paper's RS): the rows are cut into
consecutive blocks of B rows and the classical first pass above runs on
each block's induced strength subgraph independently (S and S^T restricted
to pairs inside the block; its isolation rule applies to the restricted
lists).  With one block (B >= n) this is the RS split itself.  B is the
largest of 4096, 2048, ..., 128 for which no block holds more than 32768
strong pairs (128 always fits: 128 * 127 < 32768), so each block's graph
fits one CTA's shared memory.  Strong connections between blocks are
ignored by the blocks' passes, so a point can end F with strong
dependencies but none on a C point (all its couplings leave its block; its
interpolation row would be empty).  Repair (reading): every such point
becomes C, all decided from the split the blocks produced.  "rs-blocks-h1"
then adds the second pass below (random numbers as for PMIS).

Optional second pass after PMIS (coarsening "pmis-h1"), a round-parallel form
of the RS second pass: a pair (i, j) of F points with j in S_i violates when
no C point is a strong dependency of both (S_i n S_j n C empty).  Each
round counts v_j, the violating pairs whose second point is j, and every j
with v_j > 0 that beats each such candidate in S_j u S_j^T (measure v + r
with the level's random numbers, ties to the lower index) becomes C; rounds
repeat until no pair violates.  Afterwards every strong F-F connection has a
common strong C point, the property classical interpolation formulas rely
on (denser coarse levels, faster convergence with direct interpolation).
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass
from itertools import chain

import numpy as np
import scipy.sparse as sp

from workloads import CSR, uniform01

F_PT, C_PT, U_PT = 0, 1, -1


def _rows(A: CSR) -> np.ndarray:
    return np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))


def strength(A: CSR, theta: float):
    """S[i] = sorted strong dependencies of i; ST[i] = points strongly depending on i."""
    n = A.n_rows
    S = []
    for i in range(n):
        lo, hi = A.row_ptr[i], A.row_ptr[i + 1]
        cols = A.col[lo:hi]
        neg = -A.val[lo:hi]
        off = cols != i
        if not off.any():
            S.append(np.zeros(0, dtype=np.int64))
            continue
        m = neg[off].max()
        if m <= 0.0:
            S.append(np.zeros(0, dtype=np.int64))
            continue
        S.append(cols[off & (neg >= theta * m)].astype(np.int64))
    ST = [[] for _ in range(n)]
    for i in range(n):
        for j in S[i]:
            ST[j].append(i)
    ST = [np.array(t, dtype=np.int64) for t in ST]
    return S, ST


def rs_split(n: int, S, ST) -> np.ndarray:
    """Classical Ruge-Stueben first pass; returns 1 for C points, 0 for F."""
    state = np.full(n, U_PT, dtype=np.int64)
    lam = np.array([len(t) for t in ST], dtype=np.int64)
    for i in range(n):
        if len(S[i]) == 0 and len(ST[i]) == 0:
            state[i] = F_PT
    heap = [(-int(lam[i]), i) for i in range(n) if state[i] == U_PT]
    heapq.heapify(heap)
    while heap:
        neg_l, i = heapq.heappop(heap)
        if state[i] != U_PT or -neg_l != lam[i]:
            continue  # stale entry
        state[i] = C_PT
        for j in ST[i]:
            if state[j] == U_PT:
                state[j] = F_PT
                for k in S[j]:
                    if state[k] == U_PT:
                        lam[k] += 1
                        heapq.heappush(heap, (-int(lam[k]), int(k)))
        for k in S[i]:
            if state[k] == U_PT:
                lam[k] -= 1
                heapq.heappush(heap, (-int(lam[k]), int(k)))
    return (state == C_PT).astype(np.int64)


RS_BLOCK_SIZES = (4096, 2048, 1024, 512, 256, 128)
RS_BLOCK_MAX_PAIRS = 32768


def rs_block_pairs(n: int, S, B: int) -> int:
    """Largest number of strong pairs (i, j), j in S_i, inside one block of B rows."""
    counts = np.zeros((n + B - 1) // B, dtype=np.int64)
    for i in range(n):
        counts[i // B] += sum(1 for j in S[i] if int(j) // B == i // B)
    return int(counts.max()) if len(counts) else 0


def rs_block_size(n: int, S) -> int:
    """Block size of the block-local RS split (see the module notes)."""
    for B in RS_BLOCK_SIZES:
        if rs_block_pairs(n, S, B) <= RS_BLOCK_MAX_PAIRS:
            return B
    return RS_BLOCK_SIZES[-1]


def block_rs_split(n: int, S, ST, B: int) -> np.ndarray:
    """The RS first pass on each block's induced strength subgraph; 1 for C, 0 for F."""
    split = np.zeros(n, dtype=np.int64)
    for b0 in range(0, n, B):
        b1 = min(n, b0 + B)
        Sl = [np.array([int(j) - b0 for j in S[i] if b0 <= int(j) < b1], dtype=np.int64) for i in range(b0, b1)]
        STl = [np.array([int(j) - b0 for j in ST[i] if b0 <= int(j) < b1], dtype=np.int64) for i in range(b0, b1)]
        split[b0:b1] = rs_split(b1 - b0, Sl, STl)
    return split


def rs_repair(n: int, S, split) -> np.ndarray:
    """F points with strong dependencies but no strong C point become C (all
    decided from the given split)."""
    split = np.array(split, dtype=np.int64, copy=True)
    orphan = [i for i in range(n) if split[i] == 0 and len(S[i]) > 0 and not any(split[int(j)] for j in S[i])]
    split[orphan] = C_PT
    return split


def pmis_split(n: int, S, ST, r) -> np.ndarray:
    """PMIS C/F split with random numbers r (n doubles in [0, 1)); 1 for C, 0 for F."""
    state = np.full(n, U_PT, dtype=np.int64)
    lam = [float(len(ST[i])) + float(r[i]) for i in range(n)]
    for i in range(n):
        if len(ST[i]) == 0:
            state[i] = F_PT

    def beats(i, j):
        return lam[i] > lam[j] or (lam[i] == lam[j] and i < j)

    while (state == U_PT).any():
        new_c = {i for i in range(n) if state[i] == U_PT and
                 all(beats(i, int(j)) for j in chain(S[i], ST[i]) if state[j] == U_PT)}
        for j in range(n):
            if state[j] == U_PT and j not in new_c and any(int(k) in new_c for k in S[j]):
                state[j] = F_PT
        for i in new_c:
            state[i] = C_PT
    return (state == C_PT).astype(np.int64)


def second_pass(n: int, S, ST, split, r) -> np.ndarray:
    """Round-parallel second pass (see the module notes); returns the new split."""
    split = np.array(split, dtype=np.int64, copy=True)
    while True:
        C = split == C_PT
        cs = [set(int(k) for k in S[i] if C[k]) for i in range(n)]
        v = np.zeros(n, dtype=np.int64)
        for i in range(n):
            if C[i]:
                continue
            for j in S[i]:
                j = int(j)
                if not C[j] and not (cs[i] & cs[j]):
                    v[j] += 1
        if not v.any():
            return split
        w = [float(v[j]) + float(r[j]) for j in range(n)]
        promote = [j for j in range(n) if v[j] > 0 and
                   all(v[k] == 0 or w[j] > w[k] or (w[j] == w[k] and j < k) for k in chain(S[j], ST[j]))]
        split[promote] = C_PT


def direct_interpolation(A: CSR, S, split: np.ndarray) -> CSR:
    """Direct interpolation P (n x n_c); C points map to themselves."""
    n = A.n_rows
    cidx = np.cumsum(split) - 1
    nc = int(split.sum())
    rp, cols, vals = [0], [], []
    for i in range(n):
        if split[i] == C_PT:
            cols.append(int(cidx[i]))
            vals.append(1.0)
            rp.append(len(cols))
            continue
        lo, hi = A.row_ptr[i], A.row_ptr[i + 1]
        strong_c = set(int(j) for j in S[i] if split[j] == C_PT)
        if not strong_c:
            rp.append(len(cols))
            continue
        a_ii = 0.0
        neg_all = 0.0
        pos_all = 0.0
        neg_c = 0.0
        for p in range(lo, hi):
            j, a = int(A.col[p]), float(A.val[p])
            if j == i:
                a_ii += a
            elif a < 0.0:
                neg_all += a
                if j in strong_c:
                    neg_c += a
            elif a > 0.0:
                pos_all += a
        d = a_ii + pos_all
        alpha = neg_all / neg_c
        for p in range(lo, hi):
            j = int(A.col[p])
            if j in strong_c:
                cols.append(int(cidx[j]))
                vals.append(-alpha * float(A.val[p]) / d)
        rp.append(len(cols))
    return CSR(n, nc, np.array(rp, dtype=np.int32), np.array(cols, dtype=np.int32),
               np.array(vals, dtype=np.float64))


def _to_scipy(M: CSR):
    return sp.csr_matrix((M.val, M.col, M.row_ptr), shape=(M.n_rows, M.n_cols))


def _from_scipy(M) -> CSR:
    M = M.tocsr()
    M.sort_indices()
    return CSR(M.shape[0], M.shape[1], M.indptr.astype(np.int32), M.indices.astype(np.int32),
               M.data.astype(np.float64))


def transpose(M: CSR) -> CSR:
    return _from_scipy(_to_scipy(M).T)


def galerkin(A: CSR, P: CSR) -> CSR:
    """A_c = P^T A P on the structural pattern of the product."""
    As, Ps = _to_scipy(A), _to_scipy(P)
    ones = lambda M: sp.csr_matrix((np.ones_like(M.data), M.indices, M.indptr), shape=M.shape)
    pattern = (ones(Ps).T @ ones(As) @ ones(Ps)).tocsr()
    pattern.sort_indices()
    numeric = (Ps.T @ As @ Ps).tocoo()
    prow = np.repeat(np.arange(pattern.shape[0], dtype=np.int64), np.diff(pattern.indptr))
    pkey = prow * pattern.shape[1] + pattern.indices
    nkey = numeric.row.astype(np.int64) * pattern.shape[1] + numeric.col
    vals = np.zeros(pattern.nnz)
    np.add.at(vals, np.searchsorted(pkey, nkey), numeric.data)
    return CSR(pattern.shape[0], pattern.shape[1], pattern.indptr.astype(np.int32),
               pattern.indices.astype(np.int32), vals)


@dataclass
class Level:
    A: CSR
    P: CSR | None = None   # n_l x n_{l+1}
    R: CSR | None = None   # n_{l+1} x n_l, R = P^T
    split: np.ndarray | None = None


def build_hierarchy(A: CSR, theta: float = 0.25, max_levels: int = 10, max_coarse: int = 64,
                    coarsening: str = "rs", seed: int = 0):
    """Setup-AMG-Hierarchy of Algorithm 1: list of Level, finest first.
    coarsening "rs" (the paper's), "pmis" or "pmis-h1" (PMIS then the
    second pass), "rs-blocks" or "rs-blocks-h1" (the block-local RS split,
    then the second pass); level l draws its random numbers from
    uniform01(seed + l, n_l)."""
    if coarsening not in ("rs", "pmis", "pmis-h1", "rs-blocks", "rs-blocks-h1"):
        raise ValueError(f"unknown coarsening {coarsening!r}")
    levels = [Level(A)]
    while len(levels) < max_levels and levels[-1].A.n_rows > max_coarse:
        Al = levels[-1].A
        S, ST = strength(Al, theta)
        if coarsening == "rs":
            split = rs_split(Al.n_rows, S, ST)
        else:
            r = uniform01(seed + len(levels) - 1, Al.n_rows)
            if coarsening.startswith("pmis"):
                split = pmis_split(Al.n_rows, S, ST, r)
            else:
                split = rs_repair(Al.n_rows, S, block_rs_split(Al.n_rows, S, ST, rs_block_size(Al.n_rows, S)))
            if coarsening.endswith("-h1"):
                split = second_pass(Al.n_rows, S, ST, split, r)
        nc = int(split.sum())
        if nc == 0 or nc > 0.9 * Al.n_rows:
            break
        P = direct_interpolation(Al, S, split)
        levels[-1].P = P
        levels[-1].R = transpose(P)
        levels[-1].split = split
        levels.append(Level(galerkin(Al, P)))
    return levels
