"""The boundary-MPS row sweep (the tree of the 6 x 6 gradient): a valid SSA tree
for open lattices up to 6 x 6 -- every input and every intermediate consumed
exactly once, one tensor left -- whose column structure is the one its
docstring states; and, on a 2 x 3 lattice, the exact network value along it
equals the value along a site sweep (the value does not depend on the order of
contraction, Sec. II)."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def check_ssa(tree, n):
    alive = set(range(n))
    for s, (a, b) in enumerate(tree):
        assert a in alive and b in alive and a != b, (s, a, b)
        alive -= {a, b}
        alive.add(n + s)
    assert alive == {n + len(tree) - 1} and len(tree) == n - 1


@pytest.mark.parametrize("lx,ly", [(2, 2), (2, 3), (3, 3), (4, 5), (6, 6)])
def test_boundary_mps_tree_is_a_valid_ssa_tree(lx, ly):
    n = lx * ly
    site_tree = W.boundary_mps_tree(lx, ly)
    check_ssa(site_tree, n)
    check_ssa(W.double_layer_tree(n, site_tree), 2 * n)
    # row x > 0 joins the column tensors one site at a time: site (x, y) is
    # absorbed by column y's tensor before any site of row x + 1
    absorbed = [b for a, b in site_tree if b < n]
    assert absorbed == [x * ly + y for x in range(1, lx) for y in range(ly)]


def test_boundary_tree_value_equals_site_sweep():
    n, edges = W.square_lattice(2, 3)
    lay = W.peps_layout(n, edges, (1, 1), (2, 2))
    net = O.norm_network(lay, O.ket_tensors(lay, W.random_peps(lay, 7)))
    values = []
    for site_tree in (W.boundary_mps_tree(2, 3), W.site_sweep_tree(list(range(n)))):
        r, lg, _ = O.contract_tree(net, W.double_layer_tree(n, site_tree), normalize=True)
        values.append(float(r.data) * np.exp(lg))
    assert abs(values[0] - values[1]) <= 1e-12 * abs(values[1])
