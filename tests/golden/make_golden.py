"""Writes the oracle-derived fixtures in this folder.  Calls only oracle/ and synth/.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from synth import polytope_max_of_planes  # noqa: E402


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


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "polytope12_oracle.json"), "w") as fh:
        json.dump(polytope12(), fh, separators=(",", ":"))
        fh.write("\n")
