"""The ctypes binding's packing of network descriptions (no GPU): every
field of every ftn_network / ftn_tree struct reads back what the network
dicts hold, for networks with and without bonds, trees and positions."""
import ctypes as C


class _Handle:
    def __init__(self, v):
        self.handle = C.c_void_p(v)


def test_network_arrays_round_trip():
    from paper_2410_02215_gb300 import ftn as F

    nets = []
    for i in range(7):
        if i % 3 == 0:
            nets.append({"tensors": [_Handle(100 + i)], "bonds": [], "tree": [], "positions": None})
        else:
            nets.append({"tensors": [_Handle(200 + i), _Handle(300 + i), _Handle(400 + i)],
                         "bonds": [(0, 1, 1, 0), (1, 2, 2, 0), (0, 0, 2, 1)], "tree": [(0, 1), (3, 2)],
                         "positions": [2, 0, 1] if i % 2 else None, "policy": ["exact", "early", "late"][i % 3],
                         "chi": 4 * i})
    n, na, ta, keep = F._network_arrays(nets)
    assert n == len(nets) and len(keep) == 6
    for i, job in enumerate(nets):
        N, T = na[i], ta[i]
        assert [N.tensors[k] for k in range(N.n_tensors)] == [t.handle.value for t in job["tensors"]]
        assert [N.bonds[k] for k in range(4 * N.n_bonds)] == [v for b in job["bonds"] for v in b]
        assert [T.pairs[k] for k in range(2 * T.n_steps)] == [v for p in job["tree"] for v in p]
        pos = [N.positions[k] for k in range(N.n_tensors)] if N.positions else None
        assert pos == job["positions"]
        assert T.policy == F.POLICY_NAMES[job.get("policy", "exact")] and T.chi == job.get("chi", 0)
    assert F._network_arrays([])[0] == 0


def test_cluster_structure_matches_network_assembly():
    """The structure kept per cluster function (bonds, positions, tree as
    int32 arrays) is what cluster_network assembles for the same term, with
    and without the operator, on a random 3-regular graph."""
    import numpy as np

    import workloads as W
    from paper_2410_02215_gb300 import peps

    class _T:
        def __init__(self, rank):
            self.rank = rank

    n, edges = W.random_regular_graph(12, 3, 5)
    lay = W.peps_layout(n, edges, (2, 1), (2, 2))
    kets = [_T(len(lay["legs"][s])) for s in range(n)]

    def cfn(targets):
        sites = W.cluster_sites(lay, targets, 1)
        return (sites, W.dangling_bonds(lay, sites), W.cluster_tree(lay, sites, targets, True),
                W.cluster_tree(lay, sites, targets, False))

    for targets in [tuple(lay["edges"][0]), tuple(lay["edges"][5]), (3,)]:
        st = peps._cluster_structure(lay, kets, cfn, targets)
        sites, dang, tr_op, tr_norm = cfn(list(targets))
        assert st["sites"] == list(sites) and st["dang"] == list(dang)
        for with_op, tree in ((True, tr_op), (False, tr_norm)):
            _t, bonds, pos = peps.cluster_network(lay, kets, kets, sites, dang, lambda s, a: None,
                                                  object() if with_op else None, targets)
            b, p, t = st[with_op]
            assert b.tolist() == [list(x) for x in bonds]
            assert p.tolist() == list(pos)
            assert t.tolist() == [list(x) for x in tree]
