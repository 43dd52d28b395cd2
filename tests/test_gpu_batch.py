"""Batched execution: uneven boxes in one launch per kernel class (CUDA graph) evolve bit for bit
like the same boxes stepped alone, before and after autotuning the launch shapes."""
import numpy as np
import pytest

from paper_1608_08748_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_08748_gb300 import build as B
    B.build()
    import paper_1608_08748_gb300 as M
    return M


SHAPES = [(16, 24, 40), (5, 6, 7), (32, 16, 8), (9, 33, 17), (24, 24, 24)]


def make(M, precision, k):
    ic = I.turbulence(8, mach=1.0 + 2.0 * k, beta=0.3 + 0.5 * k, seed=40 + k, shape=SHAPES[k])
    if k == 2:
        ic["options"] = dict(ic["options"], bc_x=1)  # an outflow box in the mix
    return M.from_ic(ic, precision=precision)


def assert_same(a, b):
    for k in ["rho", "E", "mom", "B", "rho_h2"]:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_solo_bitwise(M, precision):
    solo = [make(M, precision, k) for k in range(len(SHAPES))]
    mixed = [make(M, precision, k) for k in range(len(SHAPES))]
    batch = M.Batch(mixed)
    for _ in range(6):
        for s in solo:
            s.step(0.4, sync=False)
        batch.step(0.4)
    batch.sync()
    for s, m in zip(solo, mixed):
        s.sync()
        assert_same(s.get_state(), m.get_state())
        assert s.diagnostics()["t"] == m.diagnostics()["t"]


def test_tuning_keeps_results_and_shapes_are_valid(M):
    solo = [make(M, 1, k) for k in range(len(SHAPES))]
    mixed = [make(M, 1, k) for k in range(len(SHAPES))]
    batch = M.Batch(mixed)
    ms = batch.tune(0.4, reps=1)
    assert ms > 0
    for cls in ["prim", "euler_face", "lag_face", "post"]:
        block, mult = batch.shape(cls)
        assert block in (64, 128, 256, 512) and mult in (0, 4, 16)
    for _ in range(3):
        for s in solo:
            s.step(0.4, sync=False)
        batch.step(0.4)
    batch.sync()
    for s, m in zip(solo, mixed):
        s.sync()
        assert_same(s.get_state(), m.get_state())


def test_batch_of_one_matches_the_oracle(M, oracle_mod):
    from test_gpu_parity import compare
    ic = I.turbulence(8, mach=4.0, seed=5, shape=(12, 14, 10))
    g = M.from_ic(ic)
    b = M.Batch([g])
    b.set_shape("euler_face", 64, 4)  # a persistent grid, another tile size
    for _ in range(5):
        b.step(0.4)
    b.sync()
    o = oracle_mod.run(ic, steps=5)
    compare(g.get_state(), o.get_state())


def make_chem(M, precision, k):
    """Boxes with H/H2 chemistry: with the H+ network (k = 0), with heating/cooling (k = 1), plain (k = 2)."""
    ic = dict(I.turbulence(8, mach=2.0 + k, beta=0.5, seed=50 + k, shape=SHAPES[k], T_K=3000.0))
    ic["rho_h2"] = 0.05 * ic["rho"]
    opts = dict(ic["options"])
    if k == 0:
        ic["rho_hp"] = 0.01 * ic["rho"]
        opts.update(ions=1, heatcool=1)
    elif k == 1:
        opts.update(heatcool=1)
    ic["options"] = opts
    return M.from_ic(ic, precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_with_ions_equals_solo_bitwise(M, precision):
    # a batch with one H+ box runs the kernels with the ion code for every box; the other boxes must
    # still evolve exactly as alone (where the kernels without the ion code run)
    solo = [make_chem(M, precision, k) for k in range(3)]
    mixed = [make_chem(M, precision, k) for k in range(3)]
    batch = M.Batch(mixed)
    for _ in range(6):
        for s in solo:
            s.step(0.4, sync=False)
        batch.step(0.4)
    batch.sync()
    for s, m in zip(solo, mixed):
        s.sync()
        assert_same(s.get_state(), m.get_state())
        assert np.array_equal(s.get_ions(), m.get_ions())
