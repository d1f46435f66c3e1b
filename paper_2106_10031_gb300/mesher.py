"""Python face of the C ABI: a context that loads nets, seeds, marches and returns meshes.

Thin marshalling over ``native`` (numpy in, numpy out).  The network format is any object
with the attributes of ``synth.MLP`` (weights, biases, w_out, b_out, latent, skip_layer).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import native as nt


class AMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{nt.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


PRECISIONS = {"fp64": nt.AM_PREC_FP64, "mixed": nt.AM_PREC_MIXED, "tensor": nt.AM_PREC_TENSOR,
              "sliced": nt.AM_PREC_SLICED}


def _points(a, what: str) -> np.ndarray:
    """A C-contiguous (n, 3) FP64 copy of `a` (one point per row), n >= 1; ValueError otherwise,
    before any array reaches the C side."""
    x = np.ascontiguousarray(np.atleast_2d(np.asarray(a, dtype=np.float64)))
    if x.ndim != 2 or x.shape[1] != 3 or x.shape[0] < 1:
        raise ValueError(f"{what}: expected an (n, 3) array of points, got shape {np.shape(a)}")
    return x


def _key_array(keys, N: int) -> np.ndarray:
    """Activation patterns as a C-contiguous (n, ceil(N/64)) uint64 array (n >= 0): the device
    reads exactly that many words per pattern, so any other width is refused here."""
    kw = (int(N) + 63) // 64
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    if k.ndim != 2 or k.shape[1] != kw:
        raise ValueError(f"keys: expected an (n, {kw}) uint64 array for a net of {N} units, got shape {k.shape}")
    return k


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def device_N(mlp) -> int:
    """Plane ids (and key bits) of a net on the device: its units, plus one pooling row per head
    of a max-pooled net (Sec. 5.2)."""
    heads = getattr(mlp, "heads", None) or []
    return int(mlp.N) + (len(heads) if len(heads) >= 2 else 0)


@dataclass
class Mesh:
    """Assembled mesh of one net (all arrays host numpy)."""
    xyz: np.ndarray            # (V, 3) float64
    face_offsets: np.ndarray   # (F + 1,) int64
    face_vertices: np.ndarray  # (corners,) int32
    edge_planes: np.ndarray    # (corners,) int32
    face_keys: np.ndarray      # (F, key_words) uint64
    n_open_faces: int

    @property
    def n_faces(self) -> int:
        return len(self.face_offsets) - 1

    def faces(self):
        o = self.face_offsets
        return [self.face_vertices[o[i]:o[i + 1]] for i in range(self.n_faces)]

    def face_edges(self, i):
        o = self.face_offsets
        return self.edge_planes[o[i]:o[i + 1]]


def _host_view(mesh: Mesh) -> nt.am_mesh:
    """am_mesh over the arrays of `mesh` (already C-contiguous, of the binding's dtypes); the
    C side checks offsets and indices, the array lengths are checked here."""
    F, K = len(mesh.face_offsets) - 1, len(mesh.face_vertices)
    if (F < 0 or mesh.xyz.ndim != 2 or mesh.xyz.shape[1] != 3 or mesh.edge_planes.shape != (K,)
            or mesh.face_keys.ndim != 2 or mesh.face_keys.shape[0] != F):
        raise ValueError("mesh arrays of inconsistent lengths")
    m = nt.am_mesh()
    m.n_vertices, m.n_faces, m.n_corners = len(mesh.xyz), mesh.n_faces, len(mesh.face_vertices)
    m.key_words = mesh.face_keys.shape[1] if mesh.face_keys.ndim == 2 and mesh.face_keys.shape[1] else 1
    m.n_open_faces = mesh.n_open_faces
    m.xyz = mesh.xyz.ctypes.data_as(C.POINTER(C.c_double))
    m.face_offsets = mesh.face_offsets.ctypes.data_as(C.POINTER(C.c_int64))
    m.face_vertices = mesh.face_vertices.ctypes.data_as(C.POINTER(C.c_int32))
    m.edge_planes = mesh.edge_planes.ctypes.data_as(C.POINTER(C.c_int32))
    m.face_keys = mesh.face_keys.ctypes.data_as(C.POINTER(C.c_uint64))
    return m


def _host_arrays(mesh: Mesh) -> Mesh:
    return Mesh(np.ascontiguousarray(mesh.xyz, dtype=np.float64).copy(),
                np.ascontiguousarray(mesh.face_offsets, dtype=np.int64).copy(),
                np.ascontiguousarray(mesh.face_vertices, dtype=np.int32).copy(),
                np.ascontiguousarray(mesh.edge_planes, dtype=np.int32).copy(),
                np.ascontiguousarray(mesh.face_keys, dtype=np.uint64).copy(), int(mesh.n_open_faces))


def canonicalize(mesh: Mesh, lib_path=None) -> Mesh:
    """am_mesh_canonicalize on a copy: faces by key, rings from their canonical corner,
    vertices by first appearance (host only; no GPU needed)."""
    out = _host_arrays(mesh)
    st = nt.load(lib_path).am_mesh_canonicalize(C.byref(_host_view(out)))
    if st != nt.AM_OK:
        raise AMError(st, "inconsistent mesh arrays")
    return out


def triangulate(mesh: Mesh, lib_path=None) -> np.ndarray:
    """am_mesh_triangulate: (T, 3) int32 vertex indices, fans from each face's first corner."""
    lib = nt.load(lib_path)
    src = _host_arrays(mesh)
    view = _host_view(src)
    n = C.c_int64(0)
    st = lib.am_mesh_triangulate(C.byref(view), None, C.byref(n))
    if st != nt.AM_OK:
        raise AMError(st, "inconsistent mesh arrays")
    tri = np.zeros((n.value, 3), dtype=np.int32)
    st = lib.am_mesh_triangulate(C.byref(view), tri.ctypes.data, C.byref(n))
    if st != nt.AM_OK:
        raise AMError(st, "triangulation failed")
    return tri


class Mesher:
    def __init__(self, device: int = 0, max_cells: int = 1 << 20, max_neurons: int = 4096, max_width: int = 512,
                 max_face_verts: int = 32, hash_slots: int = 0, stream: int | None = None, lib_path=None):
        self.lib = nt.load(lib_path)
        self._keep = []
        opts = nt.am_ctx_opts(device=device, stream=stream, max_cells=max_cells, hash_slots=hash_slots,
                              max_face_verts=max_face_verts, max_neurons=max_neurons, max_width=max_width)
        self.ctx = C.c_void_p()
        st = self.lib.am_create(C.byref(self.ctx), C.byref(opts))
        if st != nt.AM_OK:
            msg = self.lib.am_last_error(self.ctx).decode() if self.ctx else ""
            self.lib.am_destroy(self.ctx)
            self.ctx = None
            raise AMError(st, msg)
        self.device = device
        self.nets = []

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.am_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int, ok=(nt.AM_OK,)):
        if st not in ok:
            raise AMError(st, self.lib.am_last_error(self.ctx).decode())
        return st

    # ---- am_load_mlp
    def load_mlp(self, mlp) -> int:
        L = len(mlp.weights)
        Ws = [np.ascontiguousarray(w, dtype=np.float64) for w in mlp.weights]
        bs = [np.ascontiguousarray(b, dtype=np.float64) for b in mlp.biases]
        w_out = np.ascontiguousarray(mlp.w_out, dtype=np.float64)
        width = (C.c_int * L)(*[int(w.shape[0]) for w in Ws])
        Wp = (C.POINTER(C.c_double) * L)(*[_dp(w) for w in Ws])
        bp = (C.POINTER(C.c_double) * L)(*[_dp(b) for b in bs])
        z = None if mlp.latent is None else np.ascontiguousarray(mlp.latent, dtype=np.float64).ravel()
        # the C side reads W_l as n_l x fan_l: every shape is checked here first
        in_dim = 3 + (0 if z is None else len(z))
        skip = int(mlp.skip_layer)
        if L < 1 or len(bs) != L or not (skip == 0 or 2 <= skip <= L):
            raise ValueError(f"{L} weight matrices, {len(bs)} bias vectors, skip layer {skip}")
        for l, (w, b) in enumerate(zip(Ws, bs), start=1):
            fan = in_dim if l == 1 else Ws[l - 2].shape[0] + (in_dim if l == skip else 0)
            if w.ndim != 2 or w.shape[1] != fan or b.shape != (w.shape[0],):
                raise ValueError(f"layer {l}: W {w.shape}, b {b.shape}; expected ({w.shape[0]}, {fan}) and "
                                 f"({w.shape[0]},)")
        if w_out.shape != (Ws[-1].shape[0],):
            raise ValueError(f"w_out {w_out.shape}; expected ({Ws[-1].shape[0]},)")
        # residual shortcuts {l: (src, S or None)}: S is n_l x n_src (n_src = 3 for x)
        sc = dict(getattr(mlp, "shortcuts", None) or {})
        src_arr, S_ptrs, S_keep = None, None, []
        if sc:
            src = [-1] * L
            S_ptrs = (C.POINTER(C.c_double) * L)()
            for l, (s0, S) in sc.items():
                l, s0 = int(l), int(s0)
                if not (1 <= l <= L and 0 <= s0 < l):
                    raise ValueError(f"shortcut into layer {l} from {s0}: the source must be an earlier layer")
                n_l, n_s = Ws[l - 1].shape[0], 3 if s0 == 0 else Ws[s0 - 1].shape[0]
                src[l - 1] = s0
                if S is None:
                    if n_s != n_l:
                        raise ValueError(f"identity shortcut into layer {l}: {n_s} source units, {n_l} units")
                else:
                    S = np.ascontiguousarray(S, dtype=np.float64)
                    if S.shape != (n_l, n_s):
                        raise ValueError(f"shortcut into layer {l}: S {S.shape}; expected ({n_l}, {n_s})")
                    S_keep.append(S)
                    S_ptrs[l - 1] = _dp(S)
            src_arr = (C.c_int * L)(*src)
        # final max pooling over heads [(w_i, b_i)] (Sec. 5.2)
        heads = list(getattr(mlp, "heads", None) or [])
        wh = bh = None
        if len(heads) == 1 or len(heads) > 64:
            raise ValueError(f"{len(heads)} pooling heads: none, or 2..64")
        if heads:
            wh = np.ascontiguousarray(np.stack([np.asarray(w, dtype=np.float64) for w, _ in heads]))
            bh = np.ascontiguousarray([float(b) for _, b in heads], dtype=np.float64)
            if wh.shape != (len(heads), Ws[-1].shape[0]):
                raise ValueError(f"pooling heads {wh.shape}; expected ({len(heads)}, {Ws[-1].shape[0]})")
        d = nt.am_mlp_desc(latent_dim=0 if z is None else len(z), latent=None if z is None else _dp(z),
                           n_hidden=L, width=width, W=Wp, b=bp, skip_layer=int(mlp.skip_layer),
                           w_out=_dp(w_out), b_out=float(mlp.b_out), slope=float(getattr(mlp, "slope", 0.0)),
                           shortcut_src=src_arr, shortcut_S=S_ptrs, n_heads=len(heads),
                           w_heads=None if wh is None else _dp(wh), b_heads=None if bh is None else _dp(bh))
        nid = C.c_int(-1)
        self._check(self.lib.am_load_mlp(self.ctx, C.byref(d), C.byref(nid)))
        self.nets.append(mlp)
        return nid.value

    def reset(self):
        self._check(self.lib.am_reset(self.ctx))

    def release_nets(self):
        self._check(self.lib.am_release_nets(self.ctx))
        self.nets = []

    # ---- am_seed
    def seed(self, net_id: int, origins, dirs, R: float = 2.0) -> int:
        o, d = _points(origins, "origins"), _points(dirs, "dirs")
        if o.shape != d.shape:
            raise ValueError(f"origins {o.shape} and dirs {d.shape} differ in shape")
        n = C.c_int(0)
        self._check(self.lib.am_seed(self.ctx, int(net_id), _dp(o), _dp(d), int(o.shape[0]), float(R), C.byref(n)))
        return n.value

    # ---- customised triggers (Sec. 4.3)
    def seed_sphere_trace(self, net_id: int, starts, eta: float = 1.0, max_steps: int = 64,
                          eps: float = 1e-12) -> tuple:
        """am_seed_sphere_trace: (new seed cells, (n, 3) seed point per start, NaN where none)."""
        x = _points(starts, "starts")
        pts = np.zeros_like(x)
        n = C.c_int(0)
        self._check(self.lib.am_seed_sphere_trace(self.ctx, int(net_id), x.ctypes.data, int(x.shape[0]), float(eta),
                                                  int(max_steps), float(eps), C.byref(n), pts.ctypes.data))
        return n.value, pts

    def seed_pairs(self, net_id: int, points, max_pairs: int) -> tuple:
        """am_seed_pairs: (pairs formed, new seed cells, (n_pairs, 3) seed point per pair)."""
        x = _points(points, "points")
        if int(max_pairs) < 1:
            raise ValueError("max_pairs must be at least 1")
        pts = np.zeros((int(max_pairs), 3))
        npair, n = C.c_int(0), C.c_int(0)
        self._check(self.lib.am_seed_pairs(self.ctx, int(net_id), x.ctypes.data, int(x.shape[0]), int(max_pairs),
                                           C.byref(npair), C.byref(n), pts.ctypes.data))
        return npair.value, n.value, pts[:npair.value]

    # ---- am_march
    def march(self, box: float = 1.5, delta: float = 1e-10, precision: int = nt.AM_PREC_FP64,
              max_cells: int = 0, candidates: int = nt.AM_CAND_NEAREST, schedule: int = nt.AM_SCHED_PERSISTENT,
              grid_blocks: int = 0) -> int:
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        if isinstance(schedule, str):
            schedule = {"persistent": nt.AM_SCHED_PERSISTENT, "levels": nt.AM_SCHED_LEVELS}[schedule]
        if isinstance(candidates, str):
            candidates = {"nearest": nt.AM_CAND_NEAREST, "learned": nt.AM_CAND_LEARNED,
                          "none": nt.AM_CAND_NONE}[candidates]
        op = nt.am_march_opts(box=box, delta=delta, precision=precision, max_cells=max_cells,
                              candidates=candidates, schedule=schedule, grid_blocks=grid_blocks)
        return self._check(self.lib.am_march(self.ctx, C.byref(op)), ok=(nt.AM_OK, nt.AM_INCOMPLETE))

    def stats(self) -> dict:
        s = nt.am_stats_t()
        self._check(self.lib.am_get_stats(self.ctx, C.byref(s)))
        out = {k: getattr(s, k) for k, _ in nt.am_stats_t._fields_}
        out["phase_cycles"] = list(out["phase_cycles"])
        return out

    # ---- launch shapes
    def set_tuning(self, compose_tile_cells: int | None = None, rank1_period: int | None = None,
                   clip_kernel: int | None = None, check_kernel: int | None = None):
        """Launch shapes of the sliced path; None keeps the current value."""
        cur = self.get_tuning()
        pick = lambda v, k: cur[k] if v is None else v  # noqa: E731
        t = nt.am_tuning(compose_tile_cells=pick(compose_tile_cells, "compose_tile_cells"),
                         rank1_period=pick(rank1_period, "rank1_period"), clip_kernel=pick(clip_kernel, "clip_kernel"),
                         check_kernel=pick(check_kernel, "check_kernel"))
        self._check(self.lib.am_set_tuning(self.ctx, C.byref(t)))

    def get_tuning(self) -> dict:
        t = nt.am_tuning()
        self._check(self.lib.am_get_tuning(self.ctx, C.byref(t)))
        return {k: getattr(t, k) for k, _ in nt.am_tuning._fields_}

    def autotune_compose(self, net_id: int, keys=None, n: int = 4096, reps: int = 5, cache: str | None = None,
                         seed: int = 0) -> dict:
        """Pick the sliced compose's tile shape for net_id by timing every candidate
        (am_autotune_compose) on `keys` ((n, ceil(N/64)) uint64 activation patterns; random
        patterns when None: the tensor work does not depend on them).  With `cache` (a JSON
        file path) a result stored for the same device, layer widths and precision is reused
        without timing, and a new one is stored."""
        import json
        import os

        import torch
        net = self.nets[net_id]
        dev = torch.device("cuda", self.device)
        cache_key = f"{torch.cuda.get_device_name(dev)}|sm_{''.join(map(str, torch.cuda.get_device_capability(dev)))}" \
                    f"|{'x'.join(map(str, net.widths))}|sliced"
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if cache_key in table:
                self.set_tuning(compose_tile_cells=int(table[cache_key]["compose_tile_cells"]))
                return dict(table[cache_key], cached=True)
        kw = (device_N(net) + 63) // 64
        if keys is None:
            g = torch.Generator(device="cpu").manual_seed(seed)
            k = torch.randint(-2**62, 2**62, (n, kw), generator=g, dtype=torch.int64).to(dev)
        else:
            k = torch.as_tensor(_key_array(keys, device_N(net)).view(np.int64), device=dev)
        n = k.shape[0]
        rows = torch.empty((n, device_N(net) + 1, 4), dtype=torch.float64, device=dev)
        pts = (nt.am_tune_point * 8)()
        cnt = C.c_int(0)
        self._check(self.lib.am_autotune_compose(self.ctx, net_id, C.c_void_p(k.data_ptr()), n,
                                                 C.c_void_p(rows.data_ptr()), reps, pts, 8, C.byref(cnt)))
        res = {"compose_tile_cells": self.get_tuning()["compose_tile_cells"], "cells": int(n),
               "candidates": [{"compose_tile_cells": pts[i].compose_tile_cells, "ms": pts[i].ms}
                              for i in range(cnt.value)]}
        if cache:
            table[cache_key] = res
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return dict(res, cached=False)

    def autotune_march(self, net_id: int, origins, dirs, R: float = 2.0, max_cells: int = 0, reps: int = 2,
                       box: float = 1.5, delta: float = 1e-10, candidates: str = "nearest") -> dict:
        """Time every precision x schedule of the march on net_id from the given rays
        (am_autotune_march) and return the fastest ({'precision', 'schedule'} as names, and every
        candidate's median ms).  The context holds no cells afterwards."""
        o, d = _points(origins, "origins"), _points(dirs, "dirs")
        if o.shape != d.shape:
            raise ValueError(f"origins {o.shape} and dirs {d.shape} differ in shape")
        cand = {"nearest": nt.AM_CAND_NEAREST, "learned": nt.AM_CAND_LEARNED, "none": nt.AM_CAND_NONE}[candidates]
        best = nt.am_march_opts(box=box, delta=delta, candidates=cand)
        pts = (nt.am_march_point * 8)()
        cnt = C.c_int(0)
        self._check(self.lib.am_autotune_march(self.ctx, net_id, _dp(o), _dp(d), int(o.shape[0]), float(R),
                                               int(max_cells), int(reps), C.byref(best), pts, 8, C.byref(cnt)))
        pname = {v: k for k, v in PRECISIONS.items()}
        sname = {nt.AM_SCHED_PERSISTENT: "persistent", nt.AM_SCHED_LEVELS: "levels"}
        return {"precision": pname[best.precision], "schedule": sname[best.schedule],
                "candidates": [{"precision": pname[pts[i].precision], "schedule": sname[pts[i].schedule],
                                "ms": pts[i].ms} for i in range(cnt.value)]}

    # ---- compose only
    def compose(self, net_id: int, keys, precision="fp64"):
        """Rows of the cells with activation patterns `keys` ((n, ceil(N/64)) uint64): returns
        (rows (n, N + 1, 4) float64, sign-adjusted neuron rows then a_F; err (n, N + 1))."""
        import torch
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        N = device_N(self.nets[net_id])
        dev = torch.device("cuda", self.device)
        k = torch.as_tensor(_key_array(keys, N).view(np.int64), device=dev)
        n = k.shape[0]
        rows = torch.empty((n, N + 1, 4), dtype=torch.float64, device=dev)
        err = torch.empty((n, N + 1), dtype=torch.float32, device=dev)
        self._check(self.lib.am_compose(self.ctx, net_id, C.c_void_p(k.data_ptr()), n, precision,
                                        C.c_void_p(rows.data_ptr()), C.c_void_p(err.data_ptr())))
        return rows.cpu().numpy(), err.cpu().numpy()

    def compose_neighbors(self, net_id: int, parent_keys, parent_rows, flips):
        """am_compose_neighbors: rows (n, N + 1, 4) float64 of the cells parent_keys[i] ^ e_flips[i]
        from the parents' rows ((n, N + 1, 4) float64, as compose() returns them) by the rank-1
        update on the tensor cores."""
        import torch
        N = device_N(self.nets[net_id])
        dev = torch.device("cuda", self.device)
        k = torch.as_tensor(_key_array(parent_keys, N).view(np.int64), device=dev)
        n = k.shape[0]
        pr = np.ascontiguousarray(parent_rows, dtype=np.float64)
        fl = np.ascontiguousarray(flips, dtype=np.int32)
        if pr.shape != (n, N + 1, 4) or fl.shape != (n,):
            raise ValueError(f"parent_rows {pr.shape}, flips {fl.shape}; expected ({n}, {N + 1}, 4) and ({n},)")
        rows_in = torch.as_tensor(pr, device=dev)
        f = torch.as_tensor(fl, device=dev)
        out = torch.empty((n, N + 1, 4), dtype=torch.float64, device=dev)
        self._check(self.lib.am_compose_neighbors(self.ctx, net_id, C.c_void_p(k.data_ptr()),
                                                  C.c_void_p(rows_in.data_ptr()), C.c_void_p(f.data_ptr()), n,
                                                  C.c_void_p(out.data_ptr())))
        return out.cpu().numpy()

    # ---- learned proposal (device arrays are torch CUDA tensors)
    def proposal_init(self, n_in: int, hidden: int, n_out: int, max_batch: int = 4096, seed: int = 0):
        self._check(self.lib.am_proposal_init(self.ctx, n_in, hidden, n_out, max_batch, seed))
        self.prop_shape = (n_in, hidden, n_out)

    def proposal_samples(self, net_id: int = 0, max_samples: int = 1 << 40):
        """(X, Y) training samples (torch CUDA tensors) from the last march's mesh of net_id."""
        import torch
        n = C.c_int64()
        self._check(self.lib.am_proposal_samples(self.ctx, net_id, None, None, max_samples, C.byref(n)))
        L, N = self.nets[net_id].L, self.nets[net_id].N
        dev = torch.device("cuda", self.device)
        X = torch.empty((max(n.value, 1), 7 + L), dtype=torch.float32, device=dev)
        Y = torch.empty((max(n.value, 1), N), dtype=torch.float32, device=dev)
        self._check(self.lib.am_proposal_samples(self.ctx, net_id, C.c_void_p(X.data_ptr()),
                                                 C.c_void_p(Y.data_ptr()), max_samples, C.byref(n)))
        return X[:n.value], Y[:n.value]

    def proposal_n_params(self) -> int:
        I, H, O = self.prop_shape
        return H * I + H + H * H + H + O * H + O

    def proposal_params(self) -> np.ndarray:
        n = self.proposal_n_params()
        p = np.zeros(n, dtype=np.float32)
        self._check(self.lib.am_proposal_get_params(self.ctx, p.ctypes.data_as(C.c_void_p), n))
        return p

    def proposal_set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.am_proposal_set_params(self.ctx, p.ctypes.data_as(C.c_void_p), len(p)))

    def _prop_rows(self, T, cols: int, what: str):
        """A float32 CUDA tensor on this context's device with `cols` columns, contiguous: the
        kernels read rows x cols floats from its data pointer, so nothing else gets through."""
        import torch
        if not isinstance(T, torch.Tensor) or not T.is_cuda or T.device.index != self.device:
            raise ValueError(f"{what}: expected a CUDA tensor on device {self.device}")
        if T.dtype != torch.float32 or T.dim() != 2 or T.shape[1] != cols:
            raise ValueError(f"{what}: expected (n, {cols}) float32, got {tuple(T.shape)} {T.dtype}")
        return T.contiguous()

    def _prop_xy(self, X, Y=None):
        shape = getattr(self, "prop_shape", None)
        if shape is None:
            raise ValueError("no proposal: call proposal_init first")
        X = self._prop_rows(X, shape[0], "X")
        if Y is None:
            return X, None
        Y = self._prop_rows(Y, shape[2], "Y")
        if Y.shape[0] != X.shape[0]:
            raise ValueError(f"X has {X.shape[0]} rows, Y {Y.shape[0]}")
        return X, Y

    def proposal_forward(self, X):
        import torch
        X, _ = self._prop_xy(X)
        Z = torch.empty((X.shape[0], self.prop_shape[2]), dtype=torch.float32, device=X.device)
        self._check(self.lib.am_proposal_forward(self.ctx, C.c_void_p(X.data_ptr()), X.shape[0],
                                                 C.c_void_p(Z.data_ptr())))
        return Z

    def proposal_grad(self, X, Y):
        X, Y = self._prop_xy(X, Y)
        n = self.proposal_n_params()
        g = np.zeros(n, dtype=np.float32)
        loss = C.c_float()
        self._check(self.lib.am_proposal_grad(self.ctx, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                              X.shape[0], g.ctypes.data_as(C.c_void_p), n, C.byref(loss)))
        return float(loss.value), g

    def proposal_train(self, X, Y, batch: int, steps: int, lr: float) -> np.ndarray:
        X, Y = self._prop_xy(X, Y)
        losses = np.zeros(max(int(steps), 0), dtype=np.float32)
        self._check(self.lib.am_proposal_train(self.ctx, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                               X.shape[0], batch, steps, float(lr),
                                               losses.ctypes.data_as(C.c_void_p)))
        return losses

    # ---- am_get_mesh
    def get_mesh(self, net_id: int) -> Mesh:
        m = nt.am_mesh()
        self._check(self.lib.am_get_mesh(self.ctx, int(net_id), C.byref(m)))
        xyz = np.zeros((m.n_vertices, 3))
        off = np.zeros(m.n_faces + 1, dtype=np.int64)
        fv = np.zeros(m.n_corners, dtype=np.int32)
        fe = np.zeros(m.n_corners, dtype=np.int32)
        keys = np.zeros((m.n_faces, m.key_words), dtype=np.uint64)
        m.xyz = xyz.ctypes.data_as(C.POINTER(C.c_double))
        m.face_offsets = off.ctypes.data_as(C.POINTER(C.c_int64))
        m.face_vertices = fv.ctypes.data_as(C.POINTER(C.c_int32))
        m.edge_planes = fe.ctypes.data_as(C.POINTER(C.c_int32))
        m.face_keys = keys.ctypes.data_as(C.POINTER(C.c_uint64))
        if m.n_faces == 0:
            return Mesh(xyz, off, fv, fe, keys, 0)
        self._check(self.lib.am_get_mesh(self.ctx, int(net_id), C.byref(m)))
        return Mesh(xyz, off, fv, fe, keys, int(m.n_open_faces))

    def get_mesh_device(self, net_id: int) -> dict:
        """Zero-copy device view of one net's mesh (am_get_mesh_device): a dict of CUDA torch
        tensors aliasing the context's own assembly buffers -- xyz (V, 3) float64, face_offsets
        (F + 1,) int64 starting at 0, face_vertices and edge_planes (corners,) int32, face_keys
        (F, key_words) int64 holding the uint64 key bits.  Valid until the next march, reset,
        release of the nets or close; each tensor keeps this Mesher object alive.  The tensors
        are not marked read-only (torch has no such flag) but must not be written."""
        import torch
        m = nt.am_mesh()
        self._check(self.lib.am_get_mesh_device(self.ctx, int(net_id), C.byref(m)))
        dev = torch.device("cuda", self.device)

        def view(ptr, shape, typestr):
            n = int(np.prod(shape))
            if n == 0:
                return torch.empty(shape, dtype={"<f8": torch.float64, "<i8": torch.int64,
                                                 "<i4": torch.int32}[typestr], device=dev)
            holder = _DeviceArray(C.cast(ptr, C.c_void_p).value, shape, typestr, self)
            return torch.as_tensor(holder, device=dev)

        V, F, K, kw = int(m.n_vertices), int(m.n_faces), int(m.n_corners), int(m.key_words)
        return {"xyz": view(m.xyz, (V, 3), "<f8"),
                "face_offsets": view(m.face_offsets, (F + 1,), "<i8"),
                "face_vertices": view(m.face_vertices, (K,), "<i4"),
                "edge_planes": view(m.edge_planes, (K,), "<i4"),
                "face_keys": view(m.face_keys, (F, kw), "<i8")}


class _DeviceArray:
    """__cuda_array_interface__ holder for a context-owned device array."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}


def mesh_net(mlp, origins, dirs, R=2.0, box=1.5, delta=1e-10, **ctx_kw):
    """Convenience: one net, one march; returns (Mesh, stats)."""
    with Mesher(**ctx_kw) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, origins, dirs, R)
        m.march(box=box, delta=delta)
        return m.get_mesh(nid), m.stats()
