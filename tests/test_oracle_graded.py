"""Pins of the oracle's pairwise operations against what the paper fixes.

Each test checks the oracle against something other than itself: the
paper's printed sign formulas (Eqs. transposition, standardcontract,
swapdefn, the parity identity of Sec. II.B), a textbook reduction (bosonic
legs -> numpy.einsum), the literal outer-product definition, and the fusion
identity of Sec. IV.A.
"""
import itertools

import numpy as np
import pytest

import oracle as O
import workloads as W


def rand_t(legs, parity, seed):
    return O.embed_blocks(legs, parity, W.random_blocks(legs, parity, seed))


def pv(leg):
    return O.index_parity(leg[0], leg[1])


LEGSETS = [
    [(2, 1, 0), (1, 2, 1), (2, 2, 0), (1, 1, 1)],
    [(1, 1, 1), (3, 1, 0), (2, 3, 1), (1, 2, 0), (2, 1, 1)],
]


@pytest.mark.parametrize("legs", LEGSETS)
@pytest.mark.parametrize("parity", [0, 1])
def test_transpose_equals_adjacent_swaps(legs, parity):
    """A general permutation as a product of adjacent swaps, each carrying the
    sign (-1)^{p_i p_j} of Eq. (transposition)."""
    t = rand_t(legs, parity, 3)
    r = len(legs)
    for seed in range(6):
        perm = W.random_perm(r, seed)
        cur = list(range(r))
        data = t.data.copy()
        lg = list(legs)
        # bubble sort cur towards perm, one adjacent swap at a time
        target = {v: i for i, v in enumerate(perm)}
        changed = True
        while changed:
            changed = False
            for u in range(r - 1):
                if target[cur[u]] > target[cur[u + 1]]:
                    pu = pv(lg[u]).reshape([-1 if k == u else 1 for k in range(r)])
                    pw = pv(lg[u + 1]).reshape([-1 if k == u + 1 else 1 for k in range(r)])
                    data = data * (1.0 - 2.0 * ((pu * pw) & 1))
                    data = np.swapaxes(data, u, u + 1)
                    lg[u], lg[u + 1] = lg[u + 1], lg[u]
                    cur[u], cur[u + 1] = cur[u + 1], cur[u]
                    changed = True
        got = O.transpose(t, perm)
        assert np.array_equal(got.data, data)
        assert got.legs == lg


def test_transpose_bosonic_and_involution():
    legs = [(3, 0, 0), (2, 0, 1), (4, 0, 0)]
    t = rand_t(legs, 0, 1)
    assert np.array_equal(O.transpose(t, [2, 0, 1]).data, np.transpose(t.data, [2, 0, 1]))
    f = rand_t(LEGSETS[1], 1, 2)
    for seed in range(5):
        perm = W.random_perm(5, seed)
        inv = list(np.argsort(perm))
        back = O.transpose(O.transpose(f, perm), inv)
        assert np.array_equal(back.data, f.data)


def test_contract_bosonic_reduces_to_einsum():
    """Bosonic legs are entirely even (Sec. II.D remark): no sign survives."""
    a = rand_t([(3, 0, 0), (4, 0, 1), (2, 0, 0), (5, 0, 1)], 0, 5)
    b = rand_t([(2, 0, 1), (5, 0, 0), (3, 0, 0)], 0, 6)
    got = O.contract(a, b, [3, 2], [1, 0])
    want = np.einsum("ijkl,kls->ijs", a.data, b.data)
    assert np.allclose(got.data, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("pa,pb", [(0, 0), (1, 0), (1, 1)])
def test_contract_worked_example(pa, pb):
    """Eq. (standardcontract): C_ijlmnr = sum_k (-1)^{p_k(p_l+p_m+p_n)} A_ijkl B_mnkr
    for the ordered contraction F(AB) (A earlier: A's k incoming)."""
    la = [(1, 2, 0), (2, 1, 1), (2, 2, 1), (1, 1, 0)]  # i j k l
    lb = [(2, 1, 0), (1, 2, 1), (2, 2, 0), (1, 1, 1)]  # m n k r
    a, b = rand_t(la, pa, 7), rand_t(lb, pb, 8)
    p = [pv(x) for x in la] + [pv(x) for x in lb]
    pk, pl, pm, pn = p[2], p[3], p[4], p[5]
    # sign(k, l, m, n)
    expo = pk[:, None, None, None] * (pl[None, :, None, None] + pm[None, None, :, None] + pn[None, None, None, :])
    sgn = 1.0 - 2.0 * (expo & 1)
    want = np.einsum("ijkl,mnkr,klmn->ijlmnr", a.data, b.data, sgn)
    got = O.contract(a, b, [2], [2])
    assert np.allclose(got.data, want, rtol=1e-13, atol=1e-13)
    got2 = O.contract(a, b, [2], [2], arrows=False)
    assert np.allclose(got2.data, want, rtol=1e-13, atol=1e-13)


def test_parity_identity_exhaustive():
    """Sec. II.B: (p_m+p_r)(p_k+p_s) + (p_r+p_k)p_n + (p_s+p_m)p_n = p_A p_B + p_n
    (mod 2), with p_A = p_m+p_n+p_r and p_B = p_k+p_n+p_s."""
    for pm, pr, pk, ps, pn in itertools.product((0, 1), repeat=5):
        pa, pb = (pm + pn + pr) % 2, (pk + pn + ps) % 2
        lhs = ((pm + pr) * (pk + ps) + (pr + pk) * pn + (ps + pm) * pn) % 2
        assert lhs == (pa * pb + pn) % 2


@pytest.mark.parametrize("pa,pb", [(0, 0), (0, 1), (1, 1)])
def test_swap_rule(pa, pb):
    """Eq. (swapdefn)/(swapeq): with T_mrks = F(A_mnr B_kns) and
    B~ = (-1)^{p_n}(-1)^{p_A p_B} B, F(B~ A) = (-1)^{(p_m+p_r)(p_k+p_s)} T_mrks."""
    la = [(2, 1, 0), (2, 2, 1), (1, 2, 0)]  # m n r
    lb = [(1, 1, 1), (2, 2, 0), (2, 1, 1)]  # k n s
    a, b = rand_t(la, pa, 11), rand_t(lb, pb, 12)
    t = O.contract(a, b, [1], [1], arrows=False)  # legs m r k s
    bt = O.flip_legs(b, [1])
    if pa & pb:
        bt = O.GTensor(-bt.data, bt.legs, bt.parity)
    tt = O.contract(bt, a, [1], [1], arrows=False)  # legs k s m r
    pm, pr, pk, ps = pv(la[0]), pv(la[2]), pv(lb[0]), pv(lb[2])
    expo = (pm[:, None, None, None] + pr[None, :, None, None]) * (pk[None, None, :, None] + ps[None, None, None, :])
    want = np.transpose(t.data * (1.0 - 2.0 * (expo & 1)), [2, 3, 0, 1])
    assert np.allclose(tt.data, want, rtol=1e-13, atol=1e-13)


def test_contract_matches_literal_outer_product():
    la = [(1, 2, 0), (2, 1, 1), (1, 1, 0), (2, 1, 1)]
    lb = [(2, 1, 0), (1, 1, 1), (1, 2, 1), (2, 2, 0)]
    for pa, pb in [(0, 0), (1, 0), (1, 1)]:
        a, b = rand_t(la, pa, 21), rand_t(lb, pb, 22)
        for ax, ay in [([1], [0]), ([0, 3], [2, 0]), ([3, 0, 2], [0, 2, 1])]:
            got = O.contract(a, b, ax, ay)
            lit = O.contract_outer_literal(a, b, ax, ay)
            assert np.allclose(got.data, lit.data, rtol=1e-12, atol=1e-12)
            assert got.check_symmetry()


def test_contract_operand_order_local_formalism():
    """Locally ordered formalism: op(X,Y) and op(Y,X) agree up to the leg
    reordering of the result (the arrow decides the bond parity) and, for two
    odd tensors, the phase (-1)^{p_A p_B} of Eq. (swapeq)."""
    la = [(1, 2, 0), (2, 1, 1), (1, 1, 0), (2, 1, 1)]
    lb = [(2, 1, 0), (1, 1, 1), (1, 2, 1), (2, 2, 0)]
    for pa, pb in [(0, 0), (1, 1)]:
        a, b = rand_t(la, pa, 31), rand_t(lb, pb, 32)
        ax, ay = [3, 0, 2], [0, 2, 1]
        xy = O.contract(a, b, ax, ay)
        yx = O.contract(b, a, ay, ax)
        # yx legs: [free_b, free_a]; bring to [free_a, free_b]
        nb = b.rank - len(ay)
        na = a.rank - len(ax)
        back = O.transpose(yx, list(range(nb, nb + na)) + list(range(nb)))
        phase = -1.0 if (pa & pb) else 1.0
        assert np.allclose(phase * back.data, xy.data, rtol=1e-12, atol=1e-12)


def test_fusion_identity_one_by_one():
    """Sec. IV.A: contracting a group of legs at once gives the same parity
    contributions as contracting the modes one by one."""
    la = [(1, 2, 1), (2, 1, 1), (1, 1, 0), (2, 2, 1)]
    lb = [(2, 2, 0), (1, 1, 1), (1, 2, 0), (2, 1, 0)]
    for pa, pb in [(0, 0), (1, 0), (1, 1)]:
        a, b = rand_t(la, pa, 41), rand_t(lb, pb, 42)
        ax, ay = [0, 1, 3], [2, 3, 0]
        once = O.contract(a, b, ax, ay)
        t = O.contract(a, b, [ax[0]], [ay[0]])
        fa = [k for k in range(a.rank) if k != ax[0]]
        fb = [k for k in range(b.rank) if k != ay[0]]
        ids = [("a", k) for k in fa] + [("b", k) for k in fb]
        for x, y in zip(ax[1:], ay[1:]):
            i, j = ids.index(("a", x)), ids.index(("b", y))
            t = O.trace_pair(t, i, j)
            ids = [v for v in ids if v not in (("a", x), ("b", y))]
        assert np.allclose(t.data, once.data, rtol=1e-12, atol=1e-12)


def test_embed_extract_roundtrip():
    legs = LEGSETS[1]
    blocks = W.random_blocks(legs, 1, 9)
    t = O.embed_blocks(legs, 1, blocks)
    assert t.check_symmetry()
    back = O.extract_blocks(t)
    for bits, arr in blocks:
        assert np.array_equal(back[bits], arr)
