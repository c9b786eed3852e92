"""Host checks of the seeded input generators (no GED-Walk arithmetic lives there)."""
import numpy as np

import graphgen as gg


def _rows(g):
    return [g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist() for v in range(g.n)]


def test_from_edges_is_symmetric_sorted_without_loops_or_repeats():
    g = gg.from_edges(5, [(0, 1), (1, 0), (2, 2), (3, 1), (0, 1), (4, 3)])
    rows = _rows(g)
    assert rows == [[1], [0, 3], [], [1, 4], [3]]


def test_from_arcs_keeps_direction_and_drops_loops_and_repeats():
    g = gg.from_arcs(4, [(0, 1), (0, 1), (1, 1), (2, 0), (0, 3), (3, 2)])
    assert _rows(g) == [[1, 3], [], [0], [2]]


def test_generators_are_seeded_and_well_formed():
    for make in (lambda s: gg.rmat(10, 8, seed=s), lambda s: gg.rmat(10, 8, seed=s, directed=True),
                 lambda s: gg.erdos_renyi(500, 6, s), lambda s: gg.barabasi_albert(500, 3, s),
                 lambda s: gg.random_digraph(60, 0.1, s)):
        a, b, c = make(1), make(1), make(2)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
        assert not (np.array_equal(a.row_ptr, c.row_ptr) and np.array_equal(a.col_idx, c.col_idx))
        for v, row in enumerate(_rows(a)):
            assert row == sorted(set(row)) and v not in row


def test_rmat_directed_symmetrises_to_the_undirected_graph():
    # the same tuples: symmetrising the arcs gives the undirected generator's graph
    d = gg.rmat(9, 8, seed=4, directed=True)
    u = gg.rmat(9, 8, seed=4)
    src = np.repeat(np.arange(d.n), np.diff(d.row_ptr))
    s = gg.from_edges(d.n, np.stack([src, d.col_idx], axis=1))
    assert np.array_equal(s.row_ptr, u.row_ptr) and np.array_equal(s.col_idx, u.col_idx)


def test_random_groups_sizes_and_members():
    off, mem = gg.random_groups(1000, 50, 3, 9, 5)
    sizes = np.diff(off)
    assert len(sizes) == 50 and sizes.min() >= 3 and sizes.max() <= 9
    for j in range(50):
        grp = mem[off[j]:off[j + 1]]
        assert len(set(grp.tolist())) == len(grp) and grp.min() >= 0 and grp.max() < 1000
