"""Writes the oracle-derived fixtures in this folder.  Calls only oracle/ and synth/ (and the
hashing helpers of tests/meshcheck.py, which name keys and cycles and compute nothing of the
method).

Run from the repository root:  python tests/golden/make_golden.py [--whole]
--whole also writes whole_mesh_oracle.json: order-independent digests of the oracle's whole
meshes of the large workloads (Alg. 1 run to completion on every host core; about an hour of
CPU time).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from synth import polytope_max_of_planes, proposal_target_net  # noqa: E402


def polytope12():
    mlp = polytope_max_of_planes()
    net, mesh = O.mesh_from_rays(mlp, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
    faces = sorted(mesh.faces, key=lambda f: f.key)
    return {
        "what": "analytic faces of the 12-plane max-of-planes net (3-12-6-3-2-1, seed 1), one +x ray, box 1.5",
        "written_by": "tests/golden/make_golden.py (oracle only)",
        "N": mlp.N,
        "faces": [{"key": f.key, "edges": f.edges, "area": round(f.area(), 12)} for f in faces],
    }


# the large workloads whose whole oracle mesh is digested: (name, generator, generator call, box)
WHOLE = [("learned_target_256x8", proposal_target_net, "synth.proposal_target_net()", 1.5)]


def whole_mesh(name, gen, call, box, workers):
    """The oracle's whole mesh of one workload (one +x seed ray), digested order-independently:
    face count, corners, vertices (assembled by combinatorial key), open faces, Euler
    characteristic, two 64-bit sums over the face keys and one over the keys with their edge
    cycles (tests/meshcheck.digest)."""
    import time

    from oracle.parallel import LevelMarcher
    from tests import meshcheck
    mlp = gen()
    net = O.OracleNet(mlp)
    seeds = O.seed_cells(net, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
    t0 = time.perf_counter()
    with LevelMarcher(mlp, workers=workers, box=box, timeout=3600.0) as lm:
        mesh = lm.march(seeds)
    dt = time.perf_counter() - t0
    d = meshcheck.digest(meshcheck.ArrayMesh(mesh, mlp.N), mlp.N)
    empty = [{"key": f"{k:x}", "edges": f.edges, "verts": f.verts.tolist(), "area": f.area()}
             for k, f in mesh.empty_cells]
    return {"name": name, "net": call, "N": mlp.N, "box": box, "seed_ray": "origin, +x, R = 2",
            "oracle": {"empty": mesh.empty, "degenerate": mesh.degenerate, "failed": len(mesh.failed),
                       "cells": len(mesh.faces) + mesh.empty + len(mesh.failed), "empty_cells": empty},
            "digest": d, "oracle_seconds": round(dt, 1), "workers": workers}


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "polytope12_oracle.json"), "w") as fh:
        json.dump(polytope12(), fh, separators=(",", ":"))
        fh.write("\n")
    if "--whole" in sys.argv:
        workers = os.cpu_count() or 1
        out = {"what": "digests of the oracle's whole meshes (Alg. 1 to completion, Alg. 2 per cell, FP64)",
               "written_by": "tests/golden/make_golden.py --whole (oracle only)",
               "meshes": [whole_mesh(*w, workers) for w in WHOLE]}
        with open(os.path.join(here, "whole_mesh_oracle.json"), "w") as fh:
            json.dump(out, fh, indent=1)
            fh.write("\n")
