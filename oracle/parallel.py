"""Algorithm 1 on all host cores: the oracle's march, level by level.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by the benchmark's CPU-baseline
leg and the test suite, never by the library.

Breadth-first order makes the FIFO queue of Alg. 1 a sequence of levels: the cells of level
t+1 are the unseen neighbours of the faces of level t, in the order the serial loop would
enqueue them.  Here every cell of a level is solved (``oracle.solve_cell``, the same Alg. 2
per cell) by a pool of worker processes, and the level's faces are then expanded in queue
order on the parent.  The discovery order, hence each cell's entry plane and entry point,
is the serial loop's, so the mesh is the serial oracle's mesh, face for face and bit for bit.
Nothing of the per-cell arithmetic changes: this only runs it on more cores.

Workers are started with the ``spawn`` method: a forked copy of a process that has touched
a GPU is not safe to use.
"""
from __future__ import annotations

import multiprocessing as mp

import numpy as np

from . import oracle as O

_net = None
_box = O.DEFAULT_BOX
_delta = O.DEFAULT_DELTA


def _init(mlp, box, delta):
    global _net, _box, _delta
    _net = O.OracleNet(mlp)
    _box, _delta = box, delta


def _solve(batch):
    """Alg. 2 on a batch of (key, entry plane, entry point): [(face or None, rc, face area)]."""
    out = []
    for key, start, x in batch:
        f, rc = O.solve_cell(_net, key, start, x, _box, _delta)
        out.append((f, rc, f.area() if f is not None else 0.0))
    return out


def _ping(_):
    return _net is not None


class LevelMarcher:
    """A pool of `workers` processes, each holding the oracle's copy of one MLP.

    Every wait on the pool is bounded by `timeout` seconds (a worker that dies while starting
    would otherwise leave the pool's map waiting forever): TimeoutError, and the pool is
    terminated."""

    def __init__(self, mlp, workers: int, box=O.DEFAULT_BOX, delta=O.DEFAULT_DELTA, timeout: float = 120.0):
        O.build()
        self.mlp, self.box, self.delta, self.workers = mlp, box, delta, int(workers)
        self.N = mlp.N
        self.timeout = float(timeout)
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_init, initargs=(mlp, box, delta))
        if not all(self._map(_ping, range(self.workers))):
            self.terminate()
            raise RuntimeError("oracle workers did not start")

    def _map(self, fn, items):
        try:
            return self.pool.map_async(fn, items).get(self.timeout)
        except mp.TimeoutError:
            self.terminate()
            raise TimeoutError(f"oracle pool gave no answer within {self.timeout:.0f} s") from None

    def terminate(self):
        if self.pool is not None:
            self.pool.terminate()
            self.pool.join()
            self.pool = None

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def march(self, seeds, max_cells=None) -> O.Mesh:
        """Alg. 1 from `seeds` = [(key, point on its face)], breadth first; the first
        `max_cells` cells of the serial FIFO order when given."""
        mesh = O.Mesh(self.N, self.box, seeds=list(seeds))
        seen, level = set(), []
        for key, x in seeds:
            if key not in seen:
                seen.add(key)
                level.append((key, None, np.asarray(x, dtype=np.float64)))
        area_min = 1e-24 * self.box * self.box
        done = 0
        while level:
            if max_cells is not None:
                level = level[:max(0, max_cells - done)]
                if not level:
                    break
            chunk = -(-len(level) // self.workers)          # one batch per worker and level
            batches = [level[i:i + chunk] for i in range(0, len(level), chunk)]
            solved = [r for part in self._map(_solve, batches) for r in part]
            done += len(level)
            nxt = []
            for (key, _, _), (f, rc, area) in zip(level, solved):
                if f is None:
                    mesh.failed.append((key, rc))
                    continue
                if area <= area_min:
                    mesh.empty += 1
                    mesh.empty_cells.append((key, f))
                    continue
                mesh.faces.append(f)
                mesh.degenerate += f.ndeg
                m = len(f.edges)
                for j, e in enumerate(f.edges):
                    if e < self.N:
                        nk = key ^ (1 << e)
                        if nk not in seen:
                            seen.add(nk)
                            nxt.append((nk, e, 0.5 * (f.verts[j] + f.verts[(j + 1) % m])))
            level = nxt
        return mesh
