"""The multi-process oracle march (oracle/parallel.py) is the serial oracle's march, face for
face and bit for bit, whole and truncated.  CPU only (2 spawn workers)."""
import numpy as np
import pytest

from synth import sphere_net, tiny_net

RAY = np.array([[1.0, 0.37, 0.21]]) / np.linalg.norm([1.0, 0.37, 0.21])


def _same(a, b):
    assert [f.key for f in a.faces] == [f.key for f in b.faces]
    for fa, fb in zip(a.faces, b.faces):
        assert fa.edges == fb.edges and fa.ndeg == fb.ndeg
        assert np.array_equal(fa.verts, fb.verts) and np.array_equal(fa.aF, fb.aF)
    assert a.failed == b.failed and a.empty == b.empty and a.degenerate == b.degenerate


@pytest.mark.parametrize("make,dirs,max_cells", [
    (lambda: sphere_net(seed=21, width=32, depth=4, sigma=0.05), RAY, 1500),
    (lambda: tiny_net((6, 5, 4), 12), np.random.default_rng(5).normal(size=(16, 3)), None),
])
def test_level_march_is_the_serial_march(oracle_mod, make, dirs, max_cells):
    from oracle.parallel import LevelMarcher
    mlp = make()
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    net = oracle_mod.OracleNet(mlp)
    seeds = oracle_mod.seed_cells(net, np.zeros((len(dirs), 3)), dirs)
    ref = oracle_mod.march(net, seeds, max_cells=max_cells)
    with LevelMarcher(mlp, workers=2) as lm:
        got = lm.march(seeds, max_cells=max_cells)
        _same(ref, got)
        if max_cells is not None:
            _same(oracle_mod.march(net, seeds, max_cells=max_cells // 3), lm.march(seeds, max_cells=max_cells // 3))
