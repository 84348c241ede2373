"""Sorts within rows (option row_sorts): the setup's products whose entries
come row by row (vertex renumbering, Schur complement, W = L P) sort each
row's entries on its own instead of radix sorting all of them by (row,
column). Both orders are the same stable order, so the hierarchy must be the
same bit for bit: every level's CSR, map and the solves (which also read W).
The graphs reach every path of the within-row sort: rows of one entry, lane
groups, bitonic block sorts of 64..512 entries, radix block sorts of
1024..16384 entries in shared memory, one block per row of up to 65536
entries with global scratch, and the hubs' rows beyond, radix sorted by the
whole GPU (the star's centre when renumbered; the two hubs of K_2,m, whose
Schur rows hold m fill entries of one key each, summed in a fixed order)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def k2m(inputs, m):
    leaves = np.arange(2, m + 2, dtype=np.int64)
    u = np.concatenate([np.zeros(m, np.int64), np.ones(m, np.int64)])
    v = np.concatenate([leaves, leaves])
    return inputs.from_edges(m + 2, u, v, weights="uniform", seed=4)


GRAPHS = {
    "grid2d_40": (lambda I: I.grid2d(40, 40, weights="uniform", seed=1), {}),
    "chunglu_20k": (lambda I: I.chung_lu(20000, m_target=100000, seed=3), {}),
    "chunglu_20k_elim3": (lambda I: I.chung_lu(20000, m_target=100000, seed=3), {"elim_rounds": 3}),
    "rmat_13": (lambda I: I.rmat(13, seed=2), {}),
    "rmat_13_random_order": (lambda I: I.rmat(13, seed=2), {"reorder": 2}),
    "grid3d_12_kept_order": (lambda I: I.grid3d(12, 12, 12), {"reorder": 0}),
    "star_70000": (lambda I: I.star(70000, weights="uniform", seed=3), {}),
    "star_20000": (lambda I: I.star(20000, weights="uniform", seed=3), {}),
    "star_12000": (lambda I: I.star(12000, weights="uniform", seed=3), {}),
    "k2_70000": (lambda I: k2m(I, 70000), {}),
    "k2_20000": (lambda I: k2m(I, 20000), {}),
    "k2_12000": (lambda I: k2m(I, 12000), {}),
    "k2_6000": (lambda I: k2m(I, 6000), {}),
    "star_1500": (lambda I: I.star(1500, weights="uniform", seed=3), {}),
    "complete_3000w": (lambda I: I.complete(3000, weights="uniform", seed=5), {}),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_row_sorts_same_hierarchy(lgmod, inputs, name):
    make, kw = GRAPHS[name]
    g = make(inputs)
    A = lgmod.Hierarchy(g, row_sorts=1, **kw)
    B = lgmod.Hierarchy(g, row_sorts=0, **kw)
    assert A.nlevels == B.nlevels
    for l in range(A.nlevels):
        assert A.level_info(l) == B.level_info(l)
        for a, b in zip(A.level(l), B.level(l)):
            if a is None or b is None:
                assert a is None and b is None
            else:
                np.testing.assert_array_equal(a, b)
    assert lgmod.lg_hier_bytes(A.h) == lgmod.lg_hier_bytes(B.h)
    b = inputs.rhs(g.n, seed=9)
    for prec in (lgmod.FP64, lgmod.FP32_HIER):
        x1, i1 = A.solve(b, precision=prec)
        x2, i2 = B.solve(b, precision=prec)
        assert i1.status == lgmod.OK and i1.iterations == i2.iterations
        np.testing.assert_array_equal(x1, x2)
    A.close()
    B.close()
