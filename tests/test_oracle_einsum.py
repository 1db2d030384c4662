"""Pins of the generic einsum, EQSPP and strength-reduction oracles (Sec. 4.1-4.3)."""
import itertools

import numpy as np
import pytest

from oracle import basis
from oracle import einsum as es


def test_einsum_matrix_product_and_mode2():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 4))
    B = rng.standard_normal((4, 2))
    assert np.allclose(es.einsum_bruteforce('ij', [('ik', A), ('kj', B)]), A @ B)
    # the paper's mode-2 product example C_ijk = A_ilk B_jl
    A3 = rng.standard_normal((2, 2, 2))
    B2 = rng.standard_normal((2, 2))
    ref = np.tensordot(A3, B2, axes=([1], [1])).transpose(0, 2, 1)
    assert np.allclose(es.einsum_bruteforce('ijk', [('ilk', A3), ('jl', B2)]), ref)


def test_einsum_rejects_trace_and_bad_lengths():
    with pytest.raises(ValueError):
        es.einsum_bruteforce('', [('ii', np.eye(2))])
    with pytest.raises(ValueError):
        es.einsum_bruteforce('i', [('ij', np.ones(3))])


def test_eqspp_block_example():
    """(K1 0) (Q11 Q12; Q21 Q22) (A1; 0) = K1 Q11 A1: only the Q11 block survives."""
    K = np.array([[1, 1, 0, 0]], dtype=bool)            # 1 x 4, blocks of 2
    Q = np.ones((4, 4), dtype=bool)
    A = np.array([[1], [1], [0], [0]], dtype=bool)      # 4 x 1
    hats = es.eqspp('ij', [('ik', K), ('kl', Q), ('lj', A)])
    expect = np.zeros((4, 4), dtype=bool)
    expect[:2, :2] = True
    assert np.array_equal(hats[1], expect)
    assert np.array_equal(hats[0], K) and np.array_equal(hats[2], A)


def _random_case(rng):
    sizes = {'i': 3, 'j': 2, 'k': 3, 'l': 2}
    specs = [('ik', 0.6), ('kjl', 0.5), ('l', 0.8)]
    pats = [(idx, rng.random([sizes[c] for c in idx]) < d) for idx, d in specs]
    return 'ij', pats


@pytest.mark.parametrize("seed", range(8))
def test_eqspp_definition(seed):
    """Condition 1: masking with the EQSPPs leaves U unchanged; condition 2: clearing any
    remaining non-zero changes U (generic values, no cancellation)."""
    rng = np.random.default_rng(seed)
    out, pats = _random_case(rng)
    hats = es.eqspp(out, pats)
    vals = [rng.uniform(1, 2, p.shape) * p for _, p in pats]
    U = es.einsum_bruteforce(out, [(idx, v) for (idx, _), v in zip(pats, vals)])
    masked = [v * h for v, h in zip(vals, hats)]
    Uh = es.einsum_bruteforce(out, [(idx, v) for (idx, _), v in zip(pats, masked)])
    assert np.allclose(U, Uh)
    for t, h in enumerate(hats):
        for pos in zip(*np.nonzero(h)):
            trial = [m.copy() for m in masked]
            trial[t][pos] = 0.0
            Ut = es.einsum_bruteforce(out, [(idx, v) for (idx, _), v in zip(pats, trial)])
            assert not np.allclose(Ut, U)
    assert all((h <= p).all() for h, (_, p) in zip(hats, pats))


@pytest.mark.parametrize("N", [2, 3])
def test_tce_example(N):
    """S_abij = A_acik B_befl C_dfjk D_cdel: 4N^10 naive vs 6N^6 reduced (Sec. 2.2); with the
    sparse cost the counts are exactly 4N^10 - N^4 and 6N^6 - 3N^4."""
    d = lambda s: (s, np.ones((N,) * len(s), bool))
    pats = [d('acik'), d('befl'), d('dfjk'), d('cdel')]
    cost, tree = es.strength_reduce('abij', pats, ['A', 'B', 'C', 'D'])
    assert cost == 6 * N ** 6 - 3 * N ** 4
    assert es.naive_cost('abij', pats) == 4 * N ** 10 - N ** 4
    assert tree == ('sum', 'ck', ('*', 'A', ('sum', 'fd', ('*', ('sum', 'el', ('*', 'B', 'D')), 'C'))))


def test_paper_kernel_example_tree():
    """C_ij = A_lj B_ikl w_k reduces to sum_l A_lj (sum_k B_ikl w_k) (Fig. strengthred_ast)."""
    N = 4
    pats = [('lj', np.ones((N, N), bool)), ('ikl', np.ones((N, N, N), bool)), ('k', np.ones(N, bool))]
    cost, tree = es.strength_reduce('ij', pats, ['A', 'B', 'w'])
    assert tree == ('sum', 'l', ('*', 'A', ('sum', 'k', ('*', 'B', 'w'))))
    assert cost == 4 * N ** 3 - 2 * N ** 2


def _all_trees(names):
    if len(names) == 1:
        yield names[0]
        return
    first, rest = names[0], names[1:]
    for r in range(len(rest)):
        for combo in itertools.combinations(rest, r):
            left = [first, *combo]
            right = [x for x in rest if x not in combo]
            for lt in _all_trees(left):
                for rt in _all_trees(right):
                    yield ('*', lt, rt)


@pytest.mark.parametrize("seed", range(4))
def test_strength_reduction_is_exhaustive(seed):
    """The subset DP equals the minimum over an explicit enumeration of all trees."""
    rng = np.random.default_rng(seed)
    sizes = {'a': 3, 'b': 2, 'c': 3, 'd': 2, 'e': 2}
    specs = ['ab', 'bc', 'cd', 'de', 'ea']
    pats = [(s, rng.random([sizes[c] for c in s]) < 0.7) for s in specs]
    names = [f'T{i}' for i in range(5)]
    cost, _ = es.strength_reduce('ac', pats, names)
    brute = min(es.tree_cost('ac', pats, t, names) for t in _all_trees(names))
    assert cost == brute


def test_madness_order():
    """R_ijk = S_xyz XL_xl XR_li YL_ym YR_mj ZL_zn ZR_nk (Sec. 7): for rank q < p the
    optimum first contracts S with the three low-rank L factors (down to q^3 entries) and
    then expands with the R factors; for q = p each L-R pair is multiplied first."""
    specs = ['xyz', 'xl', 'li', 'ym', 'mj', 'zn', 'nk']
    names = ['S', 'XL', 'XR', 'YL', 'YR', 'ZL', 'ZR']
    l_first = ('*', ('*', ('*', ('*', ('*', ('*', 'S', 'XL'), 'YL'), 'ZL'), 'XR'), 'YR'), 'ZR')
    pairs = ('*', ('*', ('*', 'S', ('*', 'XL', 'XR')), ('*', 'YL', 'YR')), ('*', 'ZL', 'ZR'))
    for p, q, order in ((3, 2, l_first), (4, 2, l_first), (4, 4, pairs)):
        shp = {'x': p, 'y': p, 'z': p, 'i': p, 'j': p, 'k': p, 'l': q, 'm': q, 'n': q}
        pats = [(s, np.ones([shp[c] for c in s], bool)) for s in specs]
        cost, _ = es.strength_reduce('ijk', pats, names)
        assert cost == es.tree_cost('ijk', pats, order, names)
        assert cost < es.naive_cost('ijk', pats) / 50


def _chain(N, s, j, h):
    m = basis.float_matrices(N)
    Rh, f, R = (m['Rhat'][s] != 0), (m['f'][h] != 0), (m['R'][j] != 0)
    B = R.shape[0]
    return [('km', Rh), ('mn', f), ('ln', R), ('lq', np.ones((B, 9), bool)),
            ('pq', np.ones((9, 9), bool))]


def test_seissol_neighbour_chain_orders():
    """Single simulation: Rhat((f(R^T I))A) attains the minimum at order 6; 8-32 fused
    simulations: (Rhat f)((R I) A) is the optimum (Sec. 5.1.3)."""
    names = ['Rh', 'f', 'R', 'I', 'A']
    single = ('*', 'Rh', ('*', ('*', 'f', ('*', 'R', 'I')), 'A'))
    fused = ('*', ('*', 'Rh', 'f'), ('*', ('*', 'R', 'I'), 'A'))
    for s, j, h in ((0, 3, 0), (3, 2, 1), (2, 1, 2)):
        pats = _chain(5, s, j, h)
        cost, _ = es.strength_reduce('kp', pats, names)
        assert es.tree_cost('kp', pats, single, names) == cost
    pats = _chain(3, 0, 3, 0)
    B = pats[3][1].shape[0]
    for S in (8, 32):
        pats3 = pats[:3] + [('slq', np.ones((S, B, 9), bool)), pats[4]]
        cost3, _ = es.strength_reduce('skp', pats3, names)
        assert es.tree_cost('skp', pats3, fused, names) == cost3


@pytest.mark.parametrize("seed", range(6))
def test_result_pattern_is_support_of_positive_einsum(seed):
    """With positive values on the non-zeros (no cancellation possible), the boolean
    result pattern is exactly the support of Eq. gentensorop's result; masking the
    operands with their EQSPPs leaves the result pattern unchanged."""
    rng = np.random.default_rng(100 + seed)
    out, pats = _random_case(rng)
    vals = [rng.uniform(0.5, 2.0, p.shape) * p for _, p in pats]
    U = es.einsum_bruteforce(out, [(idx, v) for (idx, _), v in zip(pats, vals)])
    P = es.result_pattern(out, pats)
    assert P.dtype == bool and P.shape == U.shape
    assert np.array_equal(P, U != 0)
    hats = es.eqspp(out, pats)
    assert np.array_equal(es.result_pattern(out, [(idx, h) for (idx, _), h in zip(pats, hats)]), P)


def test_result_pattern_block_product():
    """Block-diagonal times block-diagonal with matching blocks stays block-diagonal; with
    the second operand's blocks swapped the product has the off-diagonal blocks."""
    D = np.zeros((4, 4), dtype=bool)
    D[:2, :2] = D[2:, 2:] = True
    X = np.zeros((4, 4), dtype=bool)
    X[:2, 2:] = X[2:, :2] = True
    assert np.array_equal(es.result_pattern('ij', [('ik', D), ('kj', D)]), D)
    assert np.array_equal(es.result_pattern('ij', [('ik', D), ('kj', X)]), X)
    # an all-false operand gives an all-false result
    assert not es.result_pattern('ij', [('ik', D), ('kj', np.zeros((4, 4), dtype=bool))]).any()


def _tree_leaves(t):
    if isinstance(t, str):
        return [t]
    if t[0] == 'sum':
        return _tree_leaves(t[2])
    return _tree_leaves(t[1]) + _tree_leaves(t[2])


def _evaluate_tree(out_idx, operands, tree, names, early=True):
    """Values of a binary tree: each '*' node is the pairwise product over the union of
    its children's indices (numpy.einsum), each 'sum' node sums exactly the indices it
    names.  With early=True a '*'-only tree also sums, after each product, every index
    that neither the result nor an operand outside the subtree carries."""
    lookup = dict(zip(names, operands))

    def ev(t):
        if isinstance(t, str):
            idx, arr = lookup[t]
        elif t[0] == 'sum':
            cidx, carr = ev(t[2])
            assert set(t[1]) <= set(cidx)
            idx = ''.join(c for c in cidx if c not in t[1])
            return idx, np.einsum(f'{cidx}->{idx}', carr)
        else:
            li, la = ev(t[1])
            ri, ra = ev(t[2])
            idx = li + ''.join(c for c in ri if c not in li)
            arr = np.einsum(f'{li},{ri}->{idx}', la, ra)
        if early:
            used = _tree_leaves(t)
            keep = set(out_idx).union(*(set(lookup[n][0]) for n in names if n not in used))
            nidx = ''.join(c for c in idx if c in keep)
            if nidx != idx:
                arr = np.einsum(f'{idx}->{nidx}', arr)
                idx = nidx
        return idx, arr

    idx, arr = ev(tree)
    assert set(idx) == set(out_idx)
    return np.einsum(f'{idx}->{out_idx}', arr)


@pytest.mark.parametrize("seed", range(3))
def test_every_contraction_order_gives_the_same_values(seed):
    """Sec. 4.3: strength reduction only reorders an exact sum of products, so every
    binary tree (with early summation) evaluates Eq. gentensorop to rounding, and so does
    the tree the subset search returns, evaluated by its own 'sum' nodes alone (a sum
    placed before an operand that still carries the index would change the values)."""
    rng = np.random.default_rng(200 + seed)
    sizes = {'a': 3, 'b': 2, 'c': 3, 'd': 2, 'e': 2}
    specs = ['ab', 'bc', 'cd', 'de', 'ea']
    vals = [rng.standard_normal([sizes[c] for c in s]) * (rng.random([sizes[c] for c in s]) < 0.7)
            for s in specs]
    ops = list(zip(specs, vals))
    names = [f'T{i}' for i in range(5)]
    ref = es.einsum_bruteforce('ac', ops)
    scale = es.einsum_bruteforce('ac', [(s, np.abs(v)) for s, v in ops]).max()
    trees = list(_all_trees(names))
    assert len(trees) == 105                                  # (2n - 3)!! for n = 5
    for t in trees:
        got = _evaluate_tree('ac', ops, t, names)
        assert np.abs(got - ref).max() <= 1e-14 * scale
    _, best = es.strength_reduce('ac', [(s, v != 0) for s, v in ops], names)
    got = _evaluate_tree('ac', ops, best, names, early=False)
    assert np.abs(got - ref).max() <= 1e-14 * scale


def test_madness_tree_values():
    """The tree the search returns for the low-rank separated operator of Sec. 7 (rank 2,
    p = 3) evaluates, by its own 'sum' nodes, to Eq. gentensorop."""
    rng = np.random.default_rng(7)
    specs = ['xyz', 'xl', 'li', 'ym', 'mj', 'zn', 'nk']
    names = ['S', 'XL', 'XR', 'YL', 'YR', 'ZL', 'ZR']
    shp = {'x': 3, 'y': 3, 'z': 3, 'i': 3, 'j': 3, 'k': 3, 'l': 2, 'm': 2, 'n': 2}
    ops = [(s, rng.standard_normal([shp[c] for c in s])) for s in specs]
    _, tree = es.strength_reduce('ijk', [(s, np.ones(v.shape, bool)) for s, v in ops], names)
    ref = es.einsum_bruteforce('ijk', ops)
    scale = es.einsum_bruteforce('ijk', [(s, np.abs(v)) for s, v in ops]).max()
    got = _evaluate_tree('ijk', ops, tree, names, early=False)
    assert np.abs(got - ref).max() <= 1e-14 * scale
