"""Seeded random inputs: graded block data, leg permutations, tensordot cases.

Nothing here computes a fermionic sign, a contraction or a decomposition.  A
"block" is identified by its tuple of per-leg parity bits (0 = even sector,
1 = odd sector); a graded leg is ``(d_even, d_odd, dual)`` with ``dual = 1``
for an incoming ('-') leg and ``0`` for an outgoing ('+') leg, the labelling
of the paper's symmetry rule (Sec. II.A).
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = [
    "rng",
    "block_bits",
    "block_shape",
    "random_blocks",
    "random_perm",
    "tensordot_case",
    "TENSORDOT_CASES",
    "flip_duals",
]


def rng(seed: int) -> np.random.Generator:
    """Counter-free PCG64 stream for one seed (used for every draw here)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def block_bits(legs, parity):
    """All parity-bit tuples of a tensor with total parity ``parity``.

    Ordered by the integer whose bit k is the bit of leg k (leg 0 least
    significant).  Blocks of zero size are included.
    """
    r = len(legs)
    out = []
    for m in range(1 << r):
        bits = tuple((m >> k) & 1 for k in range(r))
        if sum(bits) % 2 == (parity & 1):
            out.append(bits)
    return out


def block_shape(legs, bits):
    return tuple(leg[1] if b else leg[0] for leg, b in zip(legs, bits))


def random_blocks(legs, parity, seed, scale=1.0):
    """i.i.d. N(0, scale^2) entries for every allowed block, drawn in block order."""
    g = rng(seed)
    out = []
    for bits in block_bits(legs, parity):
        shp = block_shape(legs, bits)
        out.append((bits, scale * g.standard_normal(shp)))
    return out


def random_perm(r, seed):
    return [int(v) for v in rng(seed).permutation(r)]


def flip_duals(legs):
    return [(d0, d1, 1 - du) for (d0, d1, du) in legs]


# Shapes of the single-tensordot microbenchmark: site tensors of rank 5 (four
# virtual legs D = 8 split 4+4, physical leg 4 split 2+2) and boundary
# environments of rank 6 (chi = 64 split 32+32 on the two outer legs, four
# D legs).  Canonical leg orders:
#   A  = [D, D, D, D, phys]      duals + + + + +
#   B  = [D, D, D, D, phys]      duals - - - - -
#   E  = [chi, D, D, D, D, chi]  duals + - - - - -
#   E' = E with every dual flipped
_D = (4, 4)
_P = (2, 2)
_CHI = (32, 32)


def _site(dual):
    return [(_D[0], _D[1], dual)] * 4 + [(_P[0], _P[1], dual)]


def _env():
    return [(_CHI[0], _CHI[1], 0)] + [(_D[0], _D[1], 1)] * 4 + [(_CHI[0], _CHI[1], 1)]


# name -> (legs_a, legs_b, canonical axes_a, canonical axes_b)
TENSORDOT_CASES = {
    # E . A over two D legs: dense (M, K, N) = (262144, 64, 256)
    "T1": (_env, lambda: _site(0), (1, 2), (0, 1)),
    # E . A over three D legs: (32768, 512, 32)
    "T2": (_env, lambda: _site(0), (1, 2, 3), (0, 1, 2)),
    # A . B over two D legs: (256, 64, 256)
    "T3": (lambda: _site(0), lambda: _site(1), (0, 1), (0, 1)),
    # E . E' over (chi, D, D): (4096, 4096, 4096)
    "T4": (_env, lambda: flip_duals(_env()), (3, 4, 5), (3, 4, 5)),
}


def _scale_legs(legs, shrink):
    """Divide every sector dimension by ``shrink`` (rounded up, floor 1)."""
    if shrink == 1:
        return legs
    return [(max(1, -(-d0 // shrink)), max(1, -(-d1 // shrink)), du) for (d0, d1, du) in legs]


def tensordot_case(name, seed=0, permute=True, shrink=1):
    """One tensordot instance of the microbenchmark family.

    Returns a dict with the stored leg lists (after a seeded random leg
    permutation of each input), the contracted axes in stored numbering, a
    seeded random output permutation, the parity of each input (both even)
    and the seeds of the block data.  ``shrink`` divides every sector
    dimension, for small parity cases of the same structure.
    """
    la_f, lb_f, ca, cb = TENSORDOT_CASES[name]
    legs_a = _scale_legs(la_f(), shrink)
    legs_b = _scale_legs(lb_f(), shrink)
    ra, rb = len(legs_a), len(legs_b)
    if permute:
        pa = random_perm(ra, 1000 * seed + 11)
        pb = random_perm(rb, 1000 * seed + 13)
    else:
        pa, pb = list(range(ra)), list(range(rb))
    # stored leg s holds canonical leg p[s]
    sa = [legs_a[p] for p in pa]
    sb = [legs_b[p] for p in pb]
    axes_a = [pa.index(c) for c in ca]
    axes_b = [pb.index(c) for c in cb]
    rc = ra + rb - 2 * len(ca)
    out_perm = random_perm(rc, 1000 * seed + 17) if permute else list(range(rc))
    return {
        "name": name,
        "legs_a": sa,
        "legs_b": sb,
        "parity_a": 0,
        "parity_b": 0,
        "axes_a": axes_a,
        "axes_b": axes_b,
        "out_perm": out_perm,
        "seed_a": 1000 * seed + 1,
        "seed_b": 1000 * seed + 2,
    }


def all_bit_tuples(r):
    return list(itertools.product((0, 1), repeat=r))
