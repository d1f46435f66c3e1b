"""am_assign_vertices_noalloc: the vertex assignment for callers that cannot allocate device
memory (inside a CUDA graph capture, or under a framework that owns every device byte).
It must group corners into vertices exactly as am_march's own assembly does, call after
call, although every call reuses the same static scratch table.  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from synth import polytope_max_of_planes, sphere_net

pytestmark = pytest.mark.gpu


def _march(mlp):
    import paper_2106_10031_gb300 as am
    with am.Mesher(max_cells=1 << 17, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
        m.march()
        return m.get_mesh(nid)


def _device_inputs(mesh):
    import torch
    dev = torch.device("cuda:0")
    return {"keys": torch.from_numpy(mesh.face_keys.view(np.int64).copy()).to(dev),
            "off": torch.from_numpy(mesh.face_offsets.astype(np.int64)).to(dev),
            "planes": torch.from_numpy(mesh.edge_planes.astype(np.int32)).to(dev),
            "out": torch.full((len(mesh.edge_planes),), -7, dtype=torch.int32, device=dev),
            "nv": torch.zeros(1, dtype=torch.int64, device=dev)}


def _call(lib, mesh, N, b, stream=None):
    return lib.am_assign_vertices_noalloc(C.c_void_p(b["keys"].data_ptr()), mesh.face_keys.shape[1],
                                          C.c_void_p(b["off"].data_ptr()), C.c_void_p(b["planes"].data_ptr()),
                                          mesh.n_faces, len(mesh.edge_planes), N, C.c_void_p(b["out"].data_ptr()),
                                          C.c_void_p(b["nv"].data_ptr()), stream)


def _noalloc(lib, mesh, N, b):
    import torch
    torch.cuda.synchronize()
    st = _call(lib, mesh, N, b)
    torch.cuda.synchronize()
    return st


def _same_grouping(a, b):
    # a and b assign the same vertex to the same corners (up to renumbering)
    fwd, bwd = {}, {}
    for x, y in zip(a.tolist(), b.tolist()):
        if fwd.setdefault(x, y) != y or bwd.setdefault(y, x) != x:
            return False
    return True


def test_noalloc_matches_march_assembly_on_consecutive_calls():
    import torch

    from paper_2106_10031_gb300 import native
    lib = native.load()
    sphere, poly = sphere_net(), polytope_max_of_planes()
    ms, mp = _march(sphere), _march(poly)
    calls = [(ms, sphere.N), (ms, sphere.N), (mp, poly.N), (ms, sphere.N)]
    bufs = [_device_inputs(mesh) for mesh, _ in calls]      # caller-owned inputs and outputs
    torch.cuda.synchronize()
    free, raw = [], []
    for (mesh, N), b in zip(calls, bufs):
        raw.append(_noalloc(lib, mesh, N, b))
        free.append(torch.cuda.mem_get_info(0)[0])
    results = []
    for (mesh, N), b, st in zip(calls, bufs, raw):
        out, nv = b["out"].cpu().numpy(), int(b["nv"].item())
        assert st == 0
        assert nv == len(mesh.xyz)
        assert out.min() >= 0 and out.max() == nv - 1
        assert _same_grouping(out, mesh.face_vertices)
        results.append(out)
    # repeated calls give the same grouping; after the first call nothing more is allocated
    assert _same_grouping(results[0], results[1]) and _same_grouping(results[0], results[3])
    assert min(free[1:]) >= free[1]


def test_noalloc_rejects_oversize_input():
    from paper_2106_10031_gb300 import native
    lib = native.load()
    one = C.c_void_p(8)   # never dereferenced: the size check comes first
    st = lib.am_assign_vertices_noalloc(one, 1, one, one, 10, (1 << 21) + 1, 16, one, one, None)
    assert st == 3        # AM_ERR_CAPACITY


def test_noalloc_large_then_small_on_one_stream_without_sync():
    # the second call clears only the part of the shared table it uses; queued behind the
    # first on one stream with no synchronisation between them, both must still group right
    import torch

    from paper_2106_10031_gb300 import native
    lib = native.load()
    big, small = sphere_net(), polytope_max_of_planes()
    mb, msm = _march(big), _march(small)
    bb, bs = _device_inputs(mb), _device_inputs(msm)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    s1 = _call(lib, mb, big.N, bb, C.c_void_p(stream.cuda_stream))
    s2 = _call(lib, msm, small.N, bs, C.c_void_p(stream.cuda_stream))
    stream.synchronize()
    assert s1 == 0 and s2 == 0
    for mesh, b in ((mb, bb), (msm, bs)):
        out, nv = b["out"].cpu().numpy(), int(b["nv"].item())
        assert nv == len(mesh.xyz)
        assert out.min() >= 0 and _same_grouping(out, mesh.face_vertices)


def test_noalloc_reports_a_face_over_the_corner_limit():
    # a face of 63 corners (one more than the 6-bit corner field keys) next to a valid mesh:
    # the count comes back negative (-1) and the long face's corners are -1
    import torch

    from paper_2106_10031_gb300 import native
    lib = native.load()
    poly = polytope_max_of_planes()
    mesh = _march(poly)
    nf = mesh.n_faces
    long_planes = np.arange(63, dtype=np.int32) % poly.N
    keys = np.vstack([mesh.face_keys, mesh.face_keys[:1]])
    off = np.concatenate([mesh.face_offsets, [mesh.face_offsets[-1] + 63]]).astype(np.int64)
    planes = np.concatenate([mesh.edge_planes, long_planes]).astype(np.int32)
    dev = torch.device("cuda:0")
    b = {"keys": torch.from_numpy(keys.view(np.int64).copy()).to(dev), "off": torch.from_numpy(off).to(dev),
         "planes": torch.from_numpy(planes).to(dev),
         "out": torch.full((len(planes),), -7, dtype=torch.int32, device=dev),
         "nv": torch.zeros(1, dtype=torch.int64, device=dev)}
    torch.cuda.synchronize()
    st = lib.am_assign_vertices_noalloc(C.c_void_p(b["keys"].data_ptr()), keys.shape[1], C.c_void_p(b["off"].data_ptr()),
                                        C.c_void_p(b["planes"].data_ptr()), nf + 1, len(planes), poly.N,
                                        C.c_void_p(b["out"].data_ptr()), C.c_void_p(b["nv"].data_ptr()), None)
    torch.cuda.synchronize()
    assert st == 0                                   # asynchronous: the error comes back in the count
    assert int(b["nv"].item()) == -1
    out = b["out"].cpu().numpy()
    assert np.all(out[off[nf]:] == -1)
    # the next call on a valid mesh starts from a clean table and error word
    bb = _device_inputs(mesh)
    assert _noalloc(lib, mesh, poly.N, bb) == 0
    assert int(bb["nv"].item()) == len(mesh.xyz)
    assert _same_grouping(bb["out"].cpu().numpy(), mesh.face_vertices)
