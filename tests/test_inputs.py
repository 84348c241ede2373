"""The seeded synthetic input generators give valid inputs for the solver
(symmetric positive weights, sorted columns, no self-loops, one connected
component: the oracle's graph check) with the shapes they state. CPU only."""

import numpy as np
import pytest

GENERATORS = {
    "grid2d": lambda I: I.grid2d(17, 11),
    "grid3d": lambda I: I.grid3d(6, 5, 4, weights="uniform"),
    "road_like": lambda I: I.road_like(40, 30, seed=2),
    "chung_lu": lambda I: I.chung_lu(5000, m_target=25000, seed=3),
    "rmat": lambda I: I.rmat(11, seed=4),
    "random": lambda I: I.random_graph(700, 5, seed=5),
    "star": lambda I: I.star(50),
    "path": lambda I: I.path(90, weights="uniform"),
    "cycle": lambda I: I.cycle(90),
    "complete": lambda I: I.complete(25),
}


@pytest.mark.parametrize("name", list(GENERATORS))
def test_generator_output_is_a_valid_connected_graph(oracle, inputs, name):
    g = GENERATORS[name](inputs)
    assert oracle.check_graph(g) == oracle.OK
    assert np.all(g.w > 0.0)


def test_grid_edge_counts(inputs):
    g = inputs.grid2d(7, 5)
    assert g.n == 35 and g.rowptr[-1] == 2 * (6 * 5 + 7 * 4)
    g = inputs.grid3d(3, 4, 5)
    assert g.n == 60 and g.rowptr[-1] == 2 * (2 * 4 * 5 + 3 * 3 * 5 + 3 * 4 * 4)


def test_chung_lu_degrees_are_heavy_tailed(inputs):
    g = inputs.chung_lu(20000, m_target=100000, seed=3)
    deg = np.diff(g.rowptr)
    assert deg.max() > 20 * deg.mean()


def test_rmat_on_the_device_generator_runs_on_cpu(oracle, inputs):
    torch = pytest.importorskip("torch")
    n, rp, cl, w = inputs.rmat_device(12, seed=6, device="cpu")
    g = inputs.Graph(int(n), rp.numpy(), cl.numpy(), w.numpy())
    assert oracle.check_graph(g) == oracle.OK  # the largest component, symmetric, sorted
    assert 2000 < g.n < 4096
    assert torch.is_tensor(rp)


def test_rhs_columns_are_mean_zero(inputs):
    B = inputs.rhs(500, 3, seed=7)
    assert B.shape == (500, 3)
    np.testing.assert_allclose(B.mean(axis=0), 0.0, atol=1e-14)
    assert np.array_equal(inputs.rhs(500, seed=7), inputs.rhs(500, seed=7))


def test_serving_mix(oracle, inputs):
    gs = inputs.serving_mix(8, 500, 5000, seed=9)
    assert len(gs) == 8
    for g in gs:
        assert oracle.check_graph(g) == oracle.OK
        assert 30 <= g.n <= 5200


def test_chung_lu_on_the_device_generator_runs_on_cpu(oracle, inputs):
    pytest.importorskip("torch")
    n, rp, cl, w = inputs.chung_lu_device(6000, m_target=30000, seed=4, device="cpu")
    g = inputs.Graph(int(n), rp.numpy(), cl.numpy(), w.numpy())
    assert oracle.check_graph(g) == oracle.OK  # the largest component, symmetric, sorted
    assert 3000 < g.n <= 6000
    assert g.w.min() >= 0.5 and g.w.max() < 1.5
    deg = np.diff(g.rowptr)
    assert deg.max() > 10 * deg.mean()  # heavy-tailed, as the host recipe


def test_serving_mix_on_the_device_matches_the_host_recipe(oracle, inputs):
    pytest.importorskip("torch")
    host = inputs.serving_mix(8, 500, 5000, seed=9)
    dev = inputs.serving_mix_device(8, 500, 5000, seed=9, device="cpu")
    assert len(dev) == 8
    for g, (name, n, rp, cl, w) in zip(host, dev):
        gd = inputs.Graph(int(n), rp.numpy(), cl.numpy(), w.numpy())
        assert oracle.check_graph(gd) == oracle.OK
        kind = g.name.split("_")[0]
        assert name.split("_")[0] == kind  # same type per slot
        if kind == "grid2d" or kind == "grid3d":
            assert np.array_equal(gd.rowptr, g.rowptr) and np.array_equal(gd.col, g.col)
