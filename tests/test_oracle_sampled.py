"""Pins of the oracle's entry-by-entry checker (``transpose_sign_at``,
``contract_sampled``) against the dense oracle operations it shortcuts.

``transpose_sign_at`` restates the sign of Eq. (transposition) for a single
index tuple; ``contract_sampled`` computes single entries of a permuted
contraction as one row of [free | bond] X times one column of [bond | free] Y
(the matricisation of Eq. standardcontract) times that sign.  Both are checked
here against ``transpose`` and ``contract`` (themselves pinned by brute force,
the bosonic einsum reduction and the paper's worked signs in
``test_oracle_graded.py``) on every parity-allowed entry of small tensors and
on sampled entries of the reduced microbenchmark shapes, with odd tensors,
both arrow conventions and odd-sector legs; a planted inversion-test mistake
must fail.
"""
import importlib
import itertools

import numpy as np
import pytest

import oracle as O
import workloads as W

OC = importlib.import_module("oracle.compress")  # the submodule (the package re-exports a function of that name)


def _random_legs(g, r):
    return [(int(g.integers(0, 4)), int(g.integers(1, 4)), int(g.integers(0, 2))) for _ in range(r)]


def test_transpose_sign_at_every_entry():
    """Every allowed entry of a transposed tensor equals the sign times the
    input entry, for random legs, parities and permutations (ranks 1-5)."""
    for seed in range(30):
        g = W.rng(seed)
        r = int(g.integers(1, 6))
        legs = _random_legs(g, r)
        p = int(g.integers(0, 2))
        t = O.embed_blocks(legs, p, W.random_blocks(legs, p, seed))
        perm = W.random_perm(r, seed + 100)
        out = O.transpose(t, perm)
        dims = [a + b for a, b, _ in legs]
        for idx in itertools.product(*[range(d) for d in dims]):
            if sum(int(i >= l[0]) for i, l in zip(idx, legs)) % 2 != p:
                continue
            s = OC.transpose_sign_at(legs, perm, idx)
            assert out.data[tuple(idx[q] for q in perm)] == s * t.data[idx]


def _check_sampled(x, y, ax, ay, perm, n, seed, arrows=True):
    full = O.contract(x, y, ax, ay, arrows=arrows)
    if perm is not None:
        full = O.transpose(full, perm)
    idx, vals = O.contract_sampled(x, y, ax, ay, perm, n, seed, arrows=arrows)
    ref = np.array([full.data[i] for i in idx])
    scale = max(float(np.max(np.abs(full.data), initial=0.0)), 1e-300)
    # only parity-allowed entries are sampled
    for i in idx:
        assert sum(int(v >= l[0]) for v, l in zip(i, full.legs)) % 2 == full.parity
    return float(np.max(np.abs(vals - ref), initial=0.0)) / scale


@pytest.mark.parametrize("name", ["T1", "T2", "T3", "T4"])
def test_contract_sampled_reduced_cases(name):
    """Sampled entries of the four microbenchmark contractions (every sector
    dimension divided by 4, T4 by 8) equal the dense permuted contraction."""
    case = W.tensordot_case(name, seed=0, shrink=8 if name == "T4" else 4)
    x = O.embed_blocks(case["legs_a"], 0, W.random_blocks(case["legs_a"], 0, case["seed_a"]))
    y = O.embed_blocks(case["legs_b"], 0, W.random_blocks(case["legs_b"], 0, case["seed_b"]))
    err = _check_sampled(x, y, case["axes_a"], case["axes_b"], case["out_perm"], 300, 9)
    assert err <= 1e-13


def test_contract_sampled_random_odd_cases():
    """Random ranks, odd and even tensors, mixed arrows, both arrow
    conventions, with and without an output permutation."""
    worst = 0.0
    for seed in range(40):
        g = W.rng(1000 + seed)
        n = int(g.integers(1, 4))
        ra, rb = n + int(g.integers(0, 3)), n + int(g.integers(0, 3))
        la, lb = _random_legs(g, ra), _random_legs(g, rb)
        ax = [int(v) for v in g.permutation(ra)[:n]]
        ay = [int(v) for v in g.permutation(rb)[:n]]
        for a, b in zip(ax, ay):
            lb[b] = (la[a][0], la[a][1], 1 - la[a][2])
        pa, pb = int(g.integers(0, 2)), int(g.integers(0, 2))
        rc = ra + rb - 2 * n
        if rc == 0:
            continue
        perm = [int(v) for v in g.permutation(rc)] if seed % 3 else None
        free = [l for k, l in enumerate(la) if k not in ax] + [l for k, l in enumerate(lb) if k not in ay]
        allowed = sum(int(np.prod(W.block_shape(free, bits))) for bits in W.block_bits(free, pa ^ pb))
        if allowed == 0:
            continue  # a result with no parity-allowed entry has nothing to sample
        x = O.embed_blocks(la, pa, W.random_blocks(la, pa, 2 * seed))
        y = O.embed_blocks(lb, pb, W.random_blocks(lb, pb, 2 * seed + 1))
        worst = max(worst, _check_sampled(x, y, ax, ay, perm, 60, seed, arrows=bool(seed % 2)))
    assert worst <= 1e-13


def test_planted_inversion_mistake_fails(monkeypatch):
    """A sign that counts the non-inverted pairs instead of the inverted ones
    (a flipped comparison) must break the pin above."""

    def wrong(legs, perm, index):
        par = [int(index[k] >= legs[k][0]) for k in range(len(legs))]
        s = 0
        for u in range(len(perm)):
            for v in range(u + 1, len(perm)):
                if perm[u] < perm[v]:
                    s ^= par[perm[u]] & par[perm[v]]
        return -1.0 if s else 1.0

    monkeypatch.setattr(OC, "transpose_sign_at", wrong)
    case = W.tensordot_case("T2", seed=0, shrink=4)
    x = O.embed_blocks(case["legs_a"], 0, W.random_blocks(case["legs_a"], 0, case["seed_a"]))
    y = O.embed_blocks(case["legs_b"], 0, W.random_blocks(case["legs_b"], 0, case["seed_b"]))
    assert _check_sampled(x, y, case["axes_a"], case["axes_b"], case["out_perm"], 200, 3) > 0.1
