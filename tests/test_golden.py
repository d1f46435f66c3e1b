"""The oracle still reproduces its committed fixture (drift check)."""
import json
import os

import numpy as np

from synth import polytope_max_of_planes

HERE = os.path.dirname(os.path.abspath(__file__))


def test_polytope12_fixture(oracle_mod):
    ref = json.load(open(os.path.join(HERE, "golden", "polytope12_oracle.json")))
    net, mesh = oracle_mod.mesh_from_rays(polytope_max_of_planes(), np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
    got = {f.key: f for f in mesh.faces}
    assert set(got) == {f["key"] for f in ref["faces"]}
    for f in ref["faces"]:
        g = got[f["key"]]
        assert g.edges == f["edges"]
        assert abs(g.area() - f["area"]) < 1e-11
