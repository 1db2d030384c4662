"""Generic tensor operation, equivalent sparsity patterns and strength reduction
(oracle; test infrastructure).

* ``einsum_bruteforce``  Eq. gentensorop: U_i = sum_{j in R_U(i)} prod_k T^k[pi_k(j)], a
  plain loop over the global index space G (indices ordered lexically, Sec. 4.2.1).
* ``result_pattern``     the same sum over G with + read as OR and * as AND (boolean
  tensors, no cancellation assumed, Sec. 4.2.2).
* ``eqspp``              Eq. compeqspp: Theta^k_q = OR_{l in R_{T^k}(q)} AND_m Theta^m[pi_m(l)].
* ``strength_reduce``    exhaustive search over all binary Product / IndexSum trees with
  the sparse cost of Sec. 4.3 (a product V = X x Y costs nnz(V) multiplications, a
  summation W = sum_i Z costs nnz(Z) - nnz(W) additions); intermediates are formed
  explicitly.  Every index is summed as soon as it occurs in a single remaining term and
  not in the result (summing earlier never increases a later product's non-zeros).
Index strings follow the DSL: letters only, one letter per dimension, no repeated letter
inside one tensor (the trace T_ii is excluded, Sec. 4.2.1 footnote).
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np


def _check(out_idx, operands):
    sizes = {}
    for idx, arr in operands:
        if not idx.isalpha() or len(set(idx)) != len(idx):
            raise ValueError(f"invalid index string {idx!r}")
        if len(idx) != np.ndim(arr):
            raise ValueError("index string length must equal the tensor dimension")
        for c, n in zip(idx, np.shape(arr)):
            if sizes.setdefault(c, n) != n:
                raise ValueError(f"inconsistent size for index {c}")
    if len(set(out_idx)) != len(out_idx) or not set(out_idx) <= set(sizes):
        raise ValueError("invalid result index string")
    return sizes


def einsum_bruteforce(out_idx: str, operands):
    """Eq. gentensorop by a loop over every point of the global index space."""
    sizes = _check(out_idx, operands)
    glob = sorted(sizes)
    U = np.zeros([sizes[c] for c in out_idx])
    for j in itertools.product(*[range(sizes[c]) for c in glob]):
        point = dict(zip(glob, j))
        prod = 1.0
        for idx, arr in operands:
            prod *= arr[tuple(point[c] for c in idx)]
        U[tuple(point[c] for c in out_idx)] += prod
    return U


def result_pattern(out_idx: str, patterns):
    """Boolean sparsity pattern of U (OR over R_U(i) of AND of the operand patterns)."""
    sizes = _check(out_idx, patterns)
    glob = sorted(sizes)
    U = np.zeros([sizes[c] for c in out_idx], dtype=bool)
    for j in itertools.product(*[range(sizes[c]) for c in glob]):
        point = dict(zip(glob, j))
        if all(p[tuple(point[c] for c in idx)] for idx, p in patterns):
            U[tuple(point[c] for c in out_idx)] = True
    return U


def eqspp(out_idx: str, patterns):
    """Equivalent sparsity patterns of every operand, Eq. compeqspp."""
    sizes = _check(out_idx, patterns)
    glob = sorted(sizes)
    hats = [np.zeros(np.shape(p), dtype=bool) for _, p in patterns]
    for j in itertools.product(*[range(sizes[c]) for c in glob]):
        point = dict(zip(glob, j))
        keys = [tuple(point[c] for c in idx) for idx, _ in patterns]
        if all(p[k] for (_, p), k in zip(patterns, keys)):
            for h, k in zip(hats, keys):
                h[k] = True
    return hats


# ------------------------------------------------------------------ strength reduction
def _product_pattern(ia, pa, ib, pb):
    idx = ia + ''.join(c for c in ib if c not in ia)
    shape = [0] * len(idx)
    for n, c in enumerate(idx):
        if c in ia:
            shape[n] = pa.shape[ia.index(c)]
        else:
            shape[n] = pb.shape[ib.index(c)]
    a = np.transpose(pa, [ia.index(c) for c in idx if c in ia]).reshape(
        [shape[n] if c in ia else 1 for n, c in enumerate(idx)])
    b = np.transpose(pb, [ib.index(c) for c in idx if c in ib]).reshape(
        [shape[n] if c in ib else 1 for n, c in enumerate(idx)])
    return idx, np.logical_and(a, b)


def _sum_out(idx, pat, keep):
    axes = tuple(n for n, c in enumerate(idx) if c not in keep)
    if not axes:
        return idx, pat, 0
    w = np.any(pat, axis=axes)
    cost = int(pat.sum()) - int(w.sum())
    return ''.join(c for c in idx if c in keep), w, cost


def strength_reduce(out_idx: str, patterns, names=None):
    """Minimal-cost binary tree over all ways of pairing the operands.  Returns
    (cost, tree): a tree is a leaf name, ('*', left, right) or ('sum', indices, child).

    The search enumerates every unordered split of every subset of operands into two
    parts; since the term built from a subset (its indices after early summation and its
    pattern) depends only on the subset, the minimum over splits of
    cost(left) + cost(right) + nnz(product) + summation cost is the minimum over all
    trees (memoised by subset)."""
    _check(out_idx, patterns)
    n = len(patterns)
    names = names or [f"T{i}" for i in range(n)]
    leaf_idx = [idx for idx, _ in patterns]

    def reduce_term(idx, pat, group, tree):
        keep = set(out_idx)
        for i in range(n):
            if i not in group:
                keep |= set(leaf_idx[i])
        nidx, npat, cost = _sum_out(idx, pat, keep)
        if nidx != idx:
            tree = ('sum', ''.join(c for c in idx if c not in nidx), tree)
        return nidx, npat, cost, tree

    @lru_cache(maxsize=None)
    def build(group):
        if len(group) == 1:
            (i,) = group
            idx, pat = patterns[i]
            return reduce_term(idx, np.asarray(pat, dtype=bool), group, names[i])
        items = sorted(group)
        first, rest = items[0], items[1:]
        best = None
        for r in range(len(rest)):
            for combo in itertools.combinations(rest, r):
                left = frozenset((first,) + combo)
                right = group - left
                li, lp, lc, lt = build(left)
                ri, rp, rc, rt = build(right)
                pidx, ppat = _product_pattern(li, lp, ri, rp)
                sidx, spat, scost, tree = reduce_term(pidx, ppat, group, ('*', lt, rt))
                total = lc + rc + int(ppat.sum()) + scost
                if best is None or total < best[2]:
                    best = (sidx, spat, total, tree)
        return best

    idx, _, cost, tree = build(frozenset(range(n)))
    if set(idx) != set(out_idx):
        raise ValueError("result indices do not match the expression")
    return cost, tree


def naive_cost(out_idx: str, patterns):
    """Cost of the unreduced evaluation: one n-ary product over G ((n-1) multiplications
    per non-zero point) followed by one summation."""
    sizes = _check(out_idx, patterns)
    glob = ''.join(sorted(sizes))
    idx, pat = patterns[0][0], np.asarray(patterns[0][1], dtype=bool)
    for i2, p2 in patterns[1:]:
        idx, pat = _product_pattern(idx, pat, i2, np.asarray(p2, dtype=bool))
    nz = int(pat.sum())
    _, w, scost = _sum_out(idx, pat, set(out_idx))
    return (len(patterns) - 1) * nz + scost


def tree_cost(out_idx: str, patterns, tree, names=None):
    """Sparse cost of a given binary tree (leaves by name), with early summation."""
    names = names or [f"T{i}" for i in range(len(patterns))]
    lookup = {nm: (idx, np.asarray(p, dtype=bool)) for nm, (idx, p) in zip(names, patterns)}

    def leaves(t):
        if isinstance(t, str):
            return [t]
        return leaves(t[1]) + leaves(t[2])

    def ev(t):
        if isinstance(t, str):
            idx, pat = lookup[t]
            used = leaves(t)
            cost = 0
        else:
            li, lp, lc = ev(t[1])
            ri, rp, rc = ev(t[2])
            idx, pat = _product_pattern(li, lp, ri, rp)
            cost = lc + rc + int(pat.sum())
            used = leaves(t)
        keep = set(out_idx)
        for nm in names:
            if nm not in used:
                keep |= set(lookup[nm][0])
        idx2, pat2, sc = _sum_out(idx, pat, keep)
        return idx2, pat2, cost + sc

    return ev(tree)[2]
