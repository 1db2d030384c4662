"""Host-side pins of the library's planner (no device work): EQSPP, strength-reduced
non-zero flops and trees, and the index-permutation dynamic program, each against the
oracle's brute force or the paper's worked examples (Sec. 4.2-4.5, 5.1.3-5.1.4)."""
import re

import numpy as np
import pytest

from oracle import basis, logmap
from oracle import einsum as es
from paper_1903_11521_gb300 import Plan, YtError


def dense(name, shape):
    return (name, shape, None, None)


def parse_order(text):
    """Parses the planner's tree string into (tree, orders) for oracle.logmap."""
    text = re.sub(r"^[-0-9.e+]+\*", "", text)
    pos = 0
    counter = [0]
    orders = {}

    def expr():
        nonlocal pos
        summed = ''
        if text.startswith('sum_', pos):
            m = re.compile(r'sum_([A-Za-z]+)').match(text, pos)
            summed = m.group(1)
            pos = m.end()
        if text[pos] == '(':
            pos += 1
            left = expr()
            assert text[pos] == '*'
            pos += 1
            right = expr()
            assert text[pos] == ')'
            pos += 1
            m = re.compile(r'\[([A-Za-z]+)\]').match(text, pos)
            pos = m.end()
            counter[0] += 1
            name = f"t{counter[0]}"
            orders[name] = m.group(1)
            return ('node', name, left, right, m.group(1))
        m = re.compile(r'([A-Za-z_][A-Za-z0-9_]*)\[([A-Za-z]+)\]').match(text, pos)
        pos = m.end()
        idx = m.group(2)
        if summed:
            assert text[pos] == ')'
            pos += 1
            idx = ''.join(c for c in idx if c not in summed)
        return ('leaf', idx)

    tree = expr()
    return tree, orders


def test_tce_counts_and_order():
    N = 2
    plan = Plan('S[abij] = A[acik] * B[befl] * C[dfjk] * D[cdel]',
                [dense(n, (N,) * 4) for n in 'SABCD'])
    st = plan.stats()
    assert st['nz_flops'] == 6 * N ** 6 - 3 * N ** 4
    assert st['naive_flops'] == 4 * N ** 10 - N ** 4
    assert st['order'].startswith('sum_ck(A[acik]*sum_fd(sum_el(B[befl]*D[cdel])')


def test_paper_kernel_example():
    N = 5
    plan = Plan('C[ij] = 2.0 * A[lj] * B[ikl] * w[k]',
                [dense('C', (N, N)), dense('A', (N, N)), dense('B', (N, N, N)), dense('w', (N,))])
    st = plan.stats()
    assert 'sum_l(A[lj]*sum_k(B[ikl]*w[k])' in st['order']
    assert st['nz_flops'] == 4 * N ** 3 - 2 * N ** 2 + N * N      # + the scalar's multiplications


def _random_case(rng):
    sizes = {c: int(rng.integers(2, 4)) for c in 'ijklmn'}
    specs = [('ik', 0.6), ('kjl', 0.5), ('lm', 0.7), ('mn', 0.8)]
    out = 'ijn'
    pats = [(idx, rng.random([sizes[c] for c in idx]) < d) for idx, d in specs]
    for _, p in pats:
        p.flat[0] = True
    return out, pats, sizes


@pytest.mark.parametrize("seed", range(6))
def test_eqspp_and_strength_reduction_match_oracle(seed):
    rng = np.random.default_rng(seed)
    out, pats, sizes = _random_case(rng)
    names = ['A', 'B', 'C', 'D']
    tensors = [dense('U', tuple(sizes[c] for c in out))]
    tensors += [(n, p.shape, p, None) for n, (_, p) in zip(names, pats)]
    expr = f"U[{out}] = " + ' * '.join(f"{n}[{idx}]" for n, (idx, _) in zip(names, pats))
    plan = Plan(expr, tensors)
    hats = es.eqspp(out, pats)
    for n, h in zip(names, hats):
        assert np.array_equal(plan.eqspp(0, n), h)
    masked = [(idx, h) for (idx, _), h in zip(pats, hats)]
    cost, _ = es.strength_reduce(out, masked, names)
    assert plan.stats()['nz_flops'] == cost


@pytest.mark.parametrize("seed", range(5))
def test_permutation_dp_equals_brute_force(seed):
    """The planner's index orders of the temporaries (dynamic program) attain the minimum
    of the LoG cost over all orders (enumeration)."""
    rng = np.random.default_rng(100 + seed)
    sizes = {c: 2 for c in 'abcdefg'}
    choices = [('abc', 'cd', 'de', 'abe'), ('ab', 'bcd', 'de', 'ace'), ('abd', 'bc', 'cde', 'ae')]
    specs = choices[seed % 3]
    out = specs[-1]
    factors = specs[:-1]
    names = ['A', 'B', 'C']
    tensors = [dense('U', tuple(sizes[c] for c in out))]
    tensors += [dense(n, tuple(sizes[c] for c in f)) for n, f in zip(names, factors)]
    perm = list(factors)
    rng.shuffle(perm)
    expr = f"U[{out}] = " + ' * '.join(f"{names[factors.index(f)]}[{f}]" for f in perm)
    st = Plan(expr, tensors).stats()
    tree, orders = parse_order(st['order'])
    chosen = logmap.tree_cost(tree, orders)
    assert chosen == tuple(st['log_cost'])
    assert logmap.best_orders(tree, out) == tuple(st['log_cost'])


def test_seissol_neighbour_chain_single_simulation():
    """Sec. 5.1.3 / 5.1.4: order Rhat((f(R^T I))A) with temporaries alpha_nq, beta_mq,
    gamma_mp (one transposed left operand R^T, one transposed right operand A^T)."""
    m = basis.float_matrices(5)
    B, Bt = 56, 21
    plan = Plan('Q[kp] += Rh[km] * f[mn] * R[ln] * I[lq] * A[pq]',
                [dense('Q', (B, 9)), ('Rh', (B, Bt), None, m['Rhat'][0]),
                 ('f', (Bt, Bt), None, m['f'][0]), ('R', (B, Bt), None, m['R'][3]),
                 dense('I', (B, 9)), dense('A', (9, 9))])
    st = plan.stats()
    assert st['order'] == 'sum_m(Rh[km]*sum_q(sum_n(f[mn]*sum_l(R[ln]*I[lq])[nq])[mq]*A[pq])[mp])[kp]'
    assert tuple(st['log_cost']) == (0, 2, -12, 1)
    tree, orders = parse_order(st['order'])
    assert logmap.best_orders(tree, 'kp') == (0, 2, -12, 1)


def test_seissol_neighbour_chain_fused_simulations():
    """8 fused simulations: (Rhat f)((R I) A) with alpha_snq, beta_snp, gamma_kn."""
    m = basis.float_matrices(3)
    B, Bt, S = 20, 10, 8
    plan = Plan('Q[skp] += Rh[km] * f[mn] * R[ln] * I[slq] * A[pq]',
                [dense('Q', (S, B, 9)), ('Rh', (B, Bt), None, m['Rhat'][0]),
                 ('f', (Bt, Bt), None, m['f'][0]), ('R', (B, Bt), None, m['R'][3]),
                 dense('I', (S, B, 9)), dense('A', (9, 9))])
    st = plan.stats()
    assert st['order'] == 'sum_n(sum_m(Rh[km]*f[mn])[kn]*sum_q(sum_l(R[ln]*I[slq])[snq]*A[pq])[snp])[skp]'


def test_volume_eqspp_zero_block():
    """EQSPP of I in Q += Khat I A*: only the first C(N+2,3) rows (Sec. 5.1.2, reading of
    the zero block)."""
    N = 3
    m = basis.float_matrices(N)
    B = basis.n_basis(N)
    plan = Plan('Q[kp] += Kh[kl] * I[lq] * A[pq]',
                [dense('Q', (B, 9)), ('Kh', (B, B), None, m['Khat'][0]), dense('I', (B, 9)),
                 ('A', (9, 9), None, np.ones((9, 9)))])
    eq = plan.eqspp(0, 'I')
    rows = np.nonzero(eq.any(axis=1))[0]
    assert rows.max() + 1 <= (N + 2) * (N + 1) * N // 6


@pytest.mark.parametrize("expr,status", [
    ("Q[kp] += K[kl] * I[lq", 2),           # missing bracket
    ("Q[kp] = K[kk] * I[kp]", 2),           # trace
    ("Q[kp] = X[kl] * I[lp]", 2),           # unknown tensor
    ("Q[kp] = K[kl] * J[lp]", 3),           # inconsistent size of l
    ("Q[kp] = K[k] * I[kp]", 3),            # wrong number of indices
    ("K[kl] = Q[kp] * I[lp]", 1),           # constant on the left
])
def test_parse_errors(expr, status):
    tensors = [dense('Q', (4, 3)), ('K', (4, 4), None, np.eye(4)), dense('I', (4, 3)),
               dense('J', (5, 3))]
    with pytest.raises(YtError) as info:
        Plan(expr, tensors)
    assert info.value.status == status
