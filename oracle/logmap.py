"""Loop-over-GEMM cost and brute-force search over temporaries' index orders
(oracle; test infrastructure).

Sec. 4.5: every binary contraction C = sum A * B is implemented as a loop over GEMMs;
its cost is the tuple (s, l + r, -f) compared lexicographically, ties broken by l, where
s counts operands whose GEMM slice has a non-unit leading stride, l (r) is 1 if the left
(right) GEMM operand is read transposed (column-major storage), and f counts the indices
fused into the GEMM.  Reading of the paper used here: a GEMM takes one block of
consecutive free indices of the left operand (M, also consecutive in C), one of the right
operand (N, consecutive in C, after M), and one of contracted indices (K, consecutive and
in the same order in both operands); a block is empty only when its index class is empty;
indices of C that occur in both operands are always loops; both operand roles are tried.
The tree cost is the sum over binary nodes; the optimum over all index orders of the
temporaries is found here by enumeration (the library uses dynamic programming,
Eqs. permopt, permcost, subproblem).
"""
from __future__ import annotations

import itertools


def _runs(src, allowed, other):
    out = [] if allowed else [""]
    for p in range(len(src)):
        for ln in range(1, len(src) - p + 1):
            g = src[p:p + ln]
            if g[-1] not in allowed:
                break
            if g in other:
                out.append(g)
    return out


def _pos(s, g):
    return -1 if not g else s.index(g[0])


def min_log(c: str, a: str, b: str):
    best = None
    for L, R in ((a, b), (b, a)):
        mset = [x for x in L if x in c and x not in R]
        kset = [x for x in L if x in R and x not in c]
        nset = [x for x in R if x in c and x not in L]
        for M in _runs(L, mset, c):
            for N in _runs(R, nset, c):
                for K in _runs(L, kset, R):
                    if M and N and _pos(c, M) > _pos(c, N):
                        continue
                    s = 0
                    first = M or N
                    if first and _pos(c, first) != 0:
                        s += 1
                    starts = [x for x in (_pos(L, M), _pos(L, K)) if x >= 0]
                    if starts and min(starts) > 0:
                        s += 1
                    starts = [x for x in (_pos(R, K), _pos(R, N)) if x >= 0]
                    if starts and min(starts) > 0:
                        s += 1
                    lt = 1 if (M and K and _pos(L, K) < _pos(L, M)) else 0
                    rt = 1 if (K and N and _pos(R, N) < _pos(R, K)) else 0
                    cost = (s, lt + rt, -(len(M) + len(N) + len(K)), lt)
                    if best is None or cost < best:
                        best = cost
    return best


def tree_cost(tree, orders):
    """tree: ('leaf', idx) | ('node', name, left, right); orders: name -> index order."""
    total = (0, 0, 0, 0)

    def order_of(t):
        return t[1] if t[0] == 'leaf' else orders[t[1]]

    def walk(t):
        nonlocal total
        if t[0] == 'leaf':
            return
        walk(t[2])
        walk(t[3])
        c = min_log(order_of(t), order_of(t[2]), order_of(t[3]))
        total = tuple(x + y for x, y in zip(total, c))

    walk(tree)
    return total


def best_orders(tree, root_order):
    """Minimum tree cost over all index orders of the non-root internal nodes."""
    internal = []

    def collect(t):
        if t[0] == 'node':
            collect(t[2])
            collect(t[3])
            internal.append(t)

    collect(tree)
    root_name = tree[1]
    free = [t for t in internal if t[1] != root_name]
    choices = [list(itertools.permutations(t[4])) for t in free]
    best = None
    for combo in itertools.product(*choices):
        orders = {t[1]: ''.join(o) for t, o in zip(free, combo)}
        orders[root_name] = root_order
        c = tree_cost(tree, orders)
        if best is None or c < best:
            best = c
    return best
