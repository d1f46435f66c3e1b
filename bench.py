"""Benchmark: analytic faces per second of analytic marching on one GB300.

One step = the whole hot path on one mesh: forget the previous cells, trigger the seed cells
on the device (the random-pair trigger of Sec. 4.3.2: F at 16384 fixed uniform samples of
[-1.4, 1.4]^3, up to 1024 pairs of opposite sign, each bisected to its cell; --seeding ray: one
ray along +x instead), march every analytic cell to completion (compose, clip, emit, hash
march) and assemble the mesh.  The workload is the learned-proposal target net, 3-[256]x8-1
(N = 2048 ReLUs; geometric init, seed 5, every parameter perturbed by N(0, 0.05^2), output bias
recentred), clipped to the box [-1.5, 1.5]^3: 1.81e6 faces, the same mesh from either seeding.  The
headline is the mixed-precision path -- the compose of each breadth-first level's cells on the
tcgen05 tensor cores (error-free BF16 digit planes) and the certified clip -- with the learned
constraint proposal (trained before timing on the plain method's meshes of 32 other nets of the
same shape, seeds 100-131).  The comparison legs time the plain FP64 method on the same net
(every cutting row clipped), the nearest-row candidates, the decoder-shaped net and the
3-[64]x4-1 sphere net.  Inputs (the net, the proposal) are resident in HBM when the timed
region starts; the e2e leg repeats the step through the C ABI from pinned host buffers (net
upload, seed samples, mesh download) inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision sliced|fp64|mixed]
                  [--candidates learned|nearest|none] [--seeding pairs|ray] [--impl reference]

Multi-GPU: each rank meshes its own copy of the workload (replicas, no collective on the
data path); the job's value is the faces of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "analytic faces/sec on 1 GB300 (oracle-exact mesh); mixed+learned vs plain FP64"
UNIT = "faces/s"
WORKLOAD_NET = "3-[256]x8-1 geometric-init SDF MLP (seed 5, sigma 0.05, recentred; N = 2048)"
SEEDINGS = {
    "pairs": "seeded by the random-pair trigger (Sec. 4.3.2: 16384 uniform samples in [-1.4, 1.4]^3, up to 1024 "
             "sign-change pairs bisected to their cells)",
    "ray": "1 seed ray +x",
}
PAIR_SAMPLES, PAIR_MAX = 16384, 1024
SEEDING = "pairs"                                  # the step's seeding; --seeding sets it


def workload_name(seeding=None) -> str:
    return f"{WORKLOAD_NET}, {SEEDINGS[seeding or SEEDING]}, box 1.5, whole mesh"


def pair_samples():
    from synth import trigger_points
    return trigger_points(PAIR_SAMPLES, seed=5, box=1.4)


def oracle_seeds(O, net, o, d):
    """The oracle's seed cells for the step's seeding (the same samples or ray as the GPU's)."""
    if SEEDING == "pairs":
        return [x for x in O.seed_pairs(net, pair_samples(), PAIR_MAX) if x is not None]
    return O.seed_cells(net, o, d)


def seed_step(m, nid, o, d, seeding=None):
    """The step's seed cells: the random-pair trigger on the fixed samples, or the one ray."""
    if (seeding or SEEDING) == "pairs":
        m.seed_pairs(nid, pair_samples(), PAIR_MAX)
    else:
        m.seed(nid, o, d)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12     # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (derived)
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12   # 128 FFMA/clk/SM x 152 SMs x 2.07 GHz (derived)


def _measured_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0                              # fallback figure for a GB300


BF16_PEAK_TFLOPS = _measured_bf16_peak()


def _measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0                              # fallback figure for a GB300


HBM_PEAK_GBS = _measured_hbm_peak()


# DRAM bytes per cell of clip_warp_kernel (sliced, learned candidates, the step's net) from the
# committed ncu capture (every clip launch of the first 399,997 cells of the step's march: 15
# levels), valid while the kernel source is the one captured; the bench scales it to the cells
# of an average launch
TRAFFIC_CAPTURE = {"sha256_prefix": "e0e3939a8554252b", "source": "am_clip_warp.cu", "precision": "sliced",
                   "candidates": "learned", "cells": 399997, "bytes": 27015762432 + 1479644928}


def captured_traffic(precision, candidates, cells_per_launch):
    import hashlib
    c = TRAFFIC_CAPTURE
    if not c["sha256_prefix"]:
        return None
    src = os.path.join(ROOT, "paper_2106_10031_gb300", "csrc", c["source"])
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if h == c["sha256_prefix"] and (precision, candidates) == (c["precision"], c["candidates"]):
        return c["bytes"] / c["cells"] * cells_per_launch
    return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="sliced", choices=["sliced", "fp64", "mixed"])
    p.add_argument("--schedule", default="auto", choices=["auto", "persistent", "levels"],
                   help="auto: the level schedule for sliced, the persistent one otherwise")
    p.add_argument("--candidates", default="learned", choices=["nearest", "learned", "none"])
    p.add_argument("--no-compare", action="store_true", help="skip the comparison legs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--decoder-only", action="store_true",
                   help="run only the decoder leg, both paths on the whole mesh, and print its JSON")
    p.add_argument("--batch-only", action="store_true",
                   help="run only the 64-net batch leg (nets sharded over the ranks) and print its JSON")
    p.add_argument("--triggers-only", action="store_true",
                   help="run only the customised-trigger leg (sphere tracing, random pairs) and print its JSON")
    p.add_argument("--compose-only", action="store_true",
                   help="run only the compose benchmark (am_compose on the decoder) and print its JSON")
    p.add_argument("--seeding", default="pairs", choices=["pairs", "ray"],
                   help="the step's seed cells: the random-pair trigger (Sec. 4.3.2) on 16384 fixed samples, or one "
                        "ray along +x")
    p.add_argument("--seeds-only", action="store_true",
                   help="run only the many-seeds leg (1024 sphere-traced seeds vs one ray) and print its JSON")
    p.add_argument("--march-once", action="store_true",
                   help="march the workload once (after --warmup marches) with --precision and --candidates, "
                        "nothing else timed: the program a profiler captures")
    p.add_argument("--max-cells", type=int, default=0, help="with --march-once: stop after this many cells")
    p.add_argument("--net", default="target", choices=["target", "decoder"],
                   help="with --march-once: the 3-[256]x8-1 workload net or the (3+256)-[512]x8-1 decoder")
    p.add_argument("--rank1-period", type=int, default=0,
                   help="with --march-once: a full compose every this many generations (1 = every cell in "
                        "full; 0 = the library default)")
    p.add_argument("--clip-kernel", default="warp", choices=["warp", "block"],
                   help="with --march-once: the sliced level's clip, one warp or one block per cell")
    p.add_argument("--check-kernel", default="warp", choices=["warp", "tensor"],
                   help="with --march-once: the dense check of every row at every vertex in the warp clip "
                        "(CUDA cores) or on the tcgen05 tensor cores")
    return p.parse_args()


def workload():
    from synth import proposal_target_net
    return proposal_target_net(), np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])


class Dist:
    def __init__(self, n_gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def allreduce(self, x: float, op: str) -> float:
        if not self.pg:
            return x
        import torch
        dev = f"cuda:{self.local}" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# algorithmic work of the cell kernel


def algorithmic_work(mlp, mesh) -> dict:
    """Work the cell kernels must do per mesh, from the mesh's cell keys (the method's own work,
    not what a dense or exhaustive evaluation would do).

    row_col_products: masked multiply-adds of the compose (Cor. 1), per cell the sum over l >= 2
    of n_l x |active(l-1)| row-column products, plus a_F over |active(L)|; each covers the 4
    columns of an affine row, so 8 flops (compose_flops = 8 x row_col_products).
    checks: (row, vertex) sign tests of the all-row check, (N + 6) x |face| per cell, 8 flops each
    (a 4-term dot product).
    Learned candidates add the proposal's forward pass, 2 (I H + H H + H N) flops per cell."""
    widths = mlp.widths
    N = mlp.N
    keys = np.ascontiguousarray(mesh.face_keys)
    rc = np.zeros(len(keys), dtype=np.int64)
    r = np.cumsum([0] + widths)
    for c0 in range(0, len(keys), 65536):
        bits = np.unpackbits(keys[c0:c0 + 65536].view(np.uint8), axis=1, bitorder="little")[:, :N]
        for l in range(1, len(widths)):
            rc[c0:c0 + 65536] += widths[l] * bits[:, r[l - 1]:r[l]].sum(1, dtype=np.int64)
        rc[c0:c0 + 65536] += bits[:, r[-2]:r[-1]].sum(1, dtype=np.int64)
    checks = (N + 6) * np.diff(mesh.face_offsets)
    I, H = 7 + len(widths), 256
    prop = 2 * (I * H + H * H + H * N) * len(keys)
    return {"row_col_products": int(rc.sum()), "checks": int(checks.sum()), "compose_flops": int(8 * rc.sum()),
            "check_flops": int(8 * checks.sum()), "proposal_flops": int(prop),
            "fp64_flops": int(8 * rc.sum() + 8 * checks.sum())}


def cpu_baseline(mlp, o, d, budget_s=10.0):
    """The oracle as it stands on this host, on a bounded prefix of the same march (breadth-first
    order): the first n cells, n sized to about budget_s of single-thread time, timed single-
    threaded; then the first 4 n cells on every host core (oracle/parallel.py: the same per-cell
    arithmetic, each breadth-first level solved by a pool of spawned processes; the mesh is the
    serial one).  `value` is the all-core figure; if the pool cannot run, the single-thread one."""
    from oracle import oracle as O
    O.build()
    net = O.OracleNet(mlp)
    seeds = oracle_seeds(O, net, o, d)
    probe = 200
    t0 = time.perf_counter()
    O.march(net, seeds, max_cells=probe)
    per = (time.perf_counter() - t0) / probe
    n = max(probe, min(60000, int(budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    mesh = O.march(net, seeds, max_cells=n)
    dt = time.perf_counter() - t0
    faces = len(mesh.faces)
    model = cpu_model()
    single = {"value": faces / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": model,
              "sample": f"first {n} cells of the breadth-first march of the bench workload ({faces} faces) in "
                        f"{dt:.1f} s, single thread (plain C per cell + Python loop)"}
    try:
        from oracle.parallel import LevelMarcher
        cores = host_cores()
        with LevelMarcher(mlp, workers=cores, timeout=600.0) as lm:
            t0 = time.perf_counter()
            pm = lm.march(seeds, max_cells=4 * n)
            dtp = time.perf_counter() - t0
        fp = len(pm.faces)
        return {"value": fp / dtp, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": model,
                "sample": f"first {4 * n} cells of the breadth-first march of the bench workload ({fp} faces) in "
                          f"{dtp:.1f} s on {cores} processes, one breadth-first level at a time (per cell: plain C + "
                          f"Python)",
                "single_thread": single}
    except Exception as e:                          # noqa: BLE001 -- the single-thread figure stands
        single["all_cores_unavailable"] = f"{type(e).__name__}: {e}"
        return single


def oracle_agreement(mlp, mesh, box=1.5, sample=200, golden=None):
    """The headline mesh against the oracle.  Whole mesh: the face-key set and every edge cycle
    through the digests of the oracle's whole mesh (`golden`, from load_golden), and closure
    (every neuron edge shared by exactly two faces).  Coordinates: `sample` faces, uniform over
    the mesh, re-solved one by one by the oracle (edge cycles exact; vertex error relative to
    max(1, |v|))."""
    from oracle import oracle as O
    from tests import meshcheck, parity
    d = meshcheck.digest(mesh, mlp.N)
    out = {"faces": d["faces"], "vertices": d["vertices"], "euler": d["euler"], "open_faces": d["open_faces"]}
    try:
        meshcheck.closure(mesh, mlp.N)
        out["closed"] = True
    except AssertionError as e:
        out["closed"] = f"no: {e}"
    if golden is not None:
        keys = ("faces", "corners", "vertices", "open_faces", "euler", "keys0", "keys1", "cycles")
        out["oracle_faces"] = golden["digest"]["faces"]
        out["whole_mesh_identical"] = all(d[k] == golden["digest"][k] for k in keys)
    O.build()
    net = O.OracleNet(mlp)
    rng = np.random.default_rng(0)
    errs, cycles = [], 0
    for i in rng.choice(mesh.n_faces, min(sample, mesh.n_faces), replace=False):
        k, e_g, v_g = parity.face_at(mesh, int(i))
        try:
            f, rc = O.solve_cell(net, k, None, v_g.mean(0), box)
        except (ValueError, OverflowError):          # not a key of this net
            f, rc = None, -1
        if rc != 0 or f is None or f.edges != e_g:
            cycles += 1
            continue
        errs.append(np.linalg.norm(f.verts - v_g, axis=1) / np.maximum(1.0, np.linalg.norm(f.verts, axis=1)))
    e = np.concatenate(errs) if errs else np.zeros(1)
    out.update({"sampled_faces": int(min(sample, mesh.n_faces)), "sampled_edge_cycles_differing": cycles,
                "max_rel_vertex_err": float(e.max()), "p99_rel_vertex_err": float(np.quantile(e, 0.99))})
    return out


def run_reference(args, dist):
    """The oracle as it stands, as the reference arm, on every host core: each step is a bounded
    sample of the bench workload, the first `cells` cells of its breadth-first march, one level
    at a time in a pool of spawned processes (oracle/parallel.py; the mesh is the serial
    march's).  If the pool cannot run, each step is the first 1000 cells, single-threaded."""
    if dist.rank != 0:
        return 0
    mlp, o, d = workload()
    from oracle import oracle as O
    O.build()
    net = O.OracleNet(mlp)
    seeds = oracle_seeds(O, net, o, d)
    cells = 12000
    lm, cores = None, 1
    try:
        from oracle.parallel import LevelMarcher
        cores = host_cores()
        lm = LevelMarcher(mlp, workers=cores, timeout=600.0)
    except Exception:                               # noqa: BLE001 -- single-thread fallback below
        lm, cores = None, 1
    try:
        if lm is not None:
            def step():
                return lm.march(seeds, max_cells=cells)
            sample = (f"each step: the first {cells} cells of the breadth-first march on {cores} processes, one "
                      f"level at a time")
        else:
            def step():
                return O.march(net, seeds, max_cells=1000)
            sample = "each step: the first 1000 cells of the breadth-first march, single thread"
        for _ in range(max(0, args.warmup)):
            step()
        t0 = time.perf_counter()
        faces = 0
        for _ in range(args.steps):
            faces += len(step().faces)
        dt = time.perf_counter() - t0
    finally:
        if lm is not None:
            lm.close()
    v = faces / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(), "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def e2e_leg(mlp, o, d, steps, device, stream_ptr, precision, schedule, candidates, prop=None):
    """Same step through the C ABI with host buffers: upload the net from pinned memory, seed
    from pinned host sample points (or a pinned host ray), march, copy the mesh back into pinned
    host buffers.  A learned
    proposal (prop = (params, (n_in, hidden, n_out))) is loaded once, untimed."""
    import torch

    from paper_2106_10031_gb300 import native as nt
    lib = nt.load()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()  # noqa: E731
    Wp = [pin(w) for w in mlp.weights]
    bp = [pin(b) for b in mlp.biases]
    wo = pin(mlp.w_out)
    ray_o, ray_d = pin(o), pin(d)
    pts = pin(pair_samples()) if SEEDING == "pairs" else None
    L = mlp.L
    dp = lambda t: C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double))  # noqa: E731
    desc = nt.am_mlp_desc(latent_dim=0, latent=None, n_hidden=L, width=(C.c_int * L)(*mlp.widths),
                          W=(C.POINTER(C.c_double) * L)(*[dp(w) for w in Wp]),
                          b=(C.POINTER(C.c_double) * L)(*[dp(b) for b in bp]), skip_layer=0,
                          w_out=dp(wo), b_out=float(mlp.b_out))
    ctx = C.c_void_p()
    shp = ctx_shape(mlp)
    opts = nt.am_ctx_opts(device=device, stream=stream_ptr, max_cells=shp["max_cells"], hash_slots=0, max_face_verts=32,
                          max_neurons=shp["max_neurons"], max_width=shp["max_width"])
    assert lib.am_create(C.byref(ctx), C.byref(opts)) == 0, lib.am_last_error(ctx)
    cand = {"nearest": nt.AM_CAND_NEAREST, "learned": nt.AM_CAND_LEARNED, "none": nt.AM_CAND_NONE}[candidates]
    if cand == nt.AM_CAND_LEARNED:
        params, (n_in, hidden, n_out) = prop
        assert lib.am_proposal_init(ctx, n_in, hidden, n_out, 1024, 0) == 0
        assert lib.am_proposal_set_params(ctx, params.ctypes.data_as(C.c_void_p), len(params)) == 0
    mo = nt.am_march_opts(box=1.5, delta=1e-10, precision=precision, max_cells=0, candidates=cand, schedule=schedule)
    bufs = None
    h2d = sum(w.numel() * 8 for w in Wp + bp) + wo.numel() * 8 + (pts.numel() * 8 if pts is not None else 48)
    d2h = 0

    def step():
        nonlocal bufs, d2h
        assert lib.am_release_nets(ctx) == 0
        nid = C.c_int()
        assert lib.am_load_mlp(ctx, C.byref(desc), C.byref(nid)) == 0
        ns = C.c_int()
        if pts is not None:
            npair = C.c_int()
            assert lib.am_seed_pairs(ctx, nid, dp(pts), int(pts.shape[0]), PAIR_MAX, C.byref(npair), C.byref(ns),
                                     None) == 0, lib.am_last_error(ctx)
        else:
            assert lib.am_seed(ctx, nid, dp(ray_o), dp(ray_d), 1, 2.0, C.byref(ns)) == 0
        assert lib.am_march(ctx, C.byref(mo)) == 0, lib.am_last_error(ctx)
        m = nt.am_mesh()
        assert lib.am_get_mesh(ctx, nid, C.byref(m)) == 0
        if bufs is None:
            bufs = {"xyz": torch.empty(3 * m.n_vertices + 3, dtype=torch.float64).pin_memory(),
                    "off": torch.empty(m.n_faces + 1, dtype=torch.int64).pin_memory(),
                    "fv": torch.empty(m.n_corners + 1, dtype=torch.int32).pin_memory(),
                    "fe": torch.empty(m.n_corners + 1, dtype=torch.int32).pin_memory(),
                    "keys": torch.empty(m.n_faces * m.key_words + 1, dtype=torch.int64).pin_memory()}
            d2h = (3 * m.n_vertices * 8 + (m.n_faces + 1) * 8 + 2 * m.n_corners * 4 + m.n_faces * m.key_words * 8)
        m.xyz = C.cast(C.c_void_p(bufs["xyz"].data_ptr()), C.POINTER(C.c_double))
        m.face_offsets = C.cast(C.c_void_p(bufs["off"].data_ptr()), C.POINTER(C.c_int64))
        m.face_vertices = C.cast(C.c_void_p(bufs["fv"].data_ptr()), C.POINTER(C.c_int32))
        m.edge_planes = C.cast(C.c_void_p(bufs["fe"].data_ptr()), C.POINTER(C.c_int32))
        m.face_keys = C.cast(C.c_void_p(bufs["keys"].data_ptr()), C.POINTER(C.c_uint64))
        assert lib.am_get_mesh(ctx, nid, C.byref(m)) == 0
        return m.n_faces

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    faces = 0
    for _ in range(steps):
        faces += step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    lib.am_destroy(ctx)
    return {"value": faces / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": dt / steps * 1e3}


def measure(m, nid, o, d, steps, precision, schedule, flush, stream, candidates="nearest", max_cells=0):
    """K timed steps; L2 flushed before each (outside the events).  Returns totals."""
    import torch

    samples = pair_samples() if SEEDING == "pairs" else None

    def step():
        m.reset()
        if samples is not None:
            m.seed_pairs(nid, samples, PAIR_MAX)
        else:
            m.seed(nid, o, d)
        m.march(precision=precision, schedule=schedule, candidates=candidates, max_cells=max_cells)

    total_ms, cell_ms, compose_ms, clip_ms, launches, cell_launches = 0.0, 0.0, 0.0, 0.0, 0, 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        st = m.stats()
        cell_ms += st["ms_cell_kernels"]
        compose_ms += st["ms_compose"]
        clip_ms += st["ms_clip"]
        cell_launches += st["cell_launches"]
        launches += st["kernel_launches"]
    return {"total_ms": total_ms, "cell_ms": cell_ms, "compose_ms": compose_ms, "clip_ms": clip_ms,
            "launches": launches, "cell_launches": cell_launches, "stats": m.stats()}


def compose_leg(dev, n_cells=4000, reps=5):
    """The compose step alone (am_compose) on the decoder-shaped net, (3 + 256) -> [512] x 8 -> 1
    with skip-concat at layer 4, for the patterns of the first n_cells cells of its march, in the
    four precisions.  Dense work per cell: 8 n_l n_{l-1} flops over the hidden layers (4 columns
    of the cell's affine maps, Cor. 1); the split-BF16 path issues 4 m16n8k16 MMAs per 16 x 16
    weight tile, the sliced path 36 digit-plane products per layer (the tile shape picked by the
    autotuner on these patterns)."""
    import ctypes as C

    import torch

    import paper_2106_10031_gb300 as am
    from synth import decoder_net
    mlp = decoder_net()
    out = {"workload": f"decoder (3+256)-[512]x8-1, skip at 4; patterns of the first {n_cells} cells"}
    with am.Mesher(device=dev, max_cells=1 << 16, max_neurons=4096, max_width=512) as m:
        nid = m.load_mlp(mlp)
        m.seed(nid, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))
        m.march(max_cells=n_cells)
        keys = m.get_mesh(nid).face_keys
        N, n = mlp.N, keys.shape[0]
        k = torch.as_tensor(np.ascontiguousarray(keys).view(np.int64), device=f"cuda:{dev}")
        rows = torch.empty((n, N + 1, 4), dtype=torch.float64, device=f"cuda:{dev}")
        err = torch.empty((n, N + 1), dtype=torch.float32, device=f"cuda:{dev}")
        w = mlp.widths
        dense = n * sum(8 * w[l] * w[l - 1] for l in range(1, mlp.L))
        issued = n * sum(4 * 2 * 16 * 16 * 8 * ((w[l] + 15) // 16) * ((w[l - 1] + 15) // 16) for l in range(1, mlp.L))
        out["autotune"] = m.autotune_compose(nid, keys=keys, reps=3)      # picks the sliced tile shape
        for name, code in (("fp64", 0), ("mixed", 1), ("tensor", 2), ("sliced", 3)):
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc = m.lib.am_compose(m.ctx, nid, C.c_void_p(k.data_ptr()), n, code, C.c_void_p(rows.data_ptr()),
                                      C.c_void_p(err.data_ptr()))
                ts.append(time.perf_counter() - t0)
                assert rc == 0, m.lib.am_last_error(m.ctx)
            dt = statistics.median(ts)
            out[name] = {"cells_per_s": n / dt, "ms": dt * 1e3, "dense_tflops": dense / dt / 1e12}
        t = out["tensor"]
        t["issued_tflops"] = issued / (t["ms"] / 1e3) / 1e12
        t["roofline"] = {"bound": "tensor", "achieved": t["issued_tflops"], "peak": BF16_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": t["issued_tflops"] / BF16_PEAK_TFLOPS,
                         "peak_source": "measured cuBLAS bf16 burst"}
        out["tensor_speedup_vs_fp64"] = out["fp64"]["ms"] / t["ms"]
        sl = out["sliced"]
        # 36 plane products per layer for each real cell's 4 columns (rows padded to the 128-row
        # tile and K to 64; the tile's padding columns are not counted)
        sl["issued_tflops"] = 36 * 2 * 4 * n * sum(-(-w[l] // 128) * 128 * (-(-w[l - 1] // 64) * 64)
                                                   for l in range(1, mlp.L)) / (sl["ms"] / 1e3) / 1e12
        sl["roofline"] = {"bound": "tensor", "achieved": sl["issued_tflops"], "peak": BF16_PEAK_TFLOPS,
                          "unit": "TFLOP/s", "frac": sl["issued_tflops"] / BF16_PEAK_TFLOPS,
                          "peak_source": "measured cuBLAS bf16 burst", "scope": "whole am_compose call"}
        out["sliced_speedup_vs_fp64"] = out["fp64"]["ms"] / sl["ms"]
    return out


def decoder_leg(dev, fp64_cells=2_000_000, reps=1):
    """The decoder-shaped workload, (3 + 256) -> [512] x 8 -> 1 with skip-concat of [x; z] at
    hidden layer 4 (N = 4096), one seed ray along +x, box 1.5: its whole mesh (1.4e7 faces) with
    the sliced path, timed by am_march's CUDA events (seeding outside), against the plain FP64
    path (compose and clip in one persistent kernel) on the first fp64_cells cells of the same
    march (0 = the whole mesh; the FP64 march of all 1.4e7 cells takes about 100 s).  Rooflines
    of the two sliced kernels over their own device time: the compose's useful flops (8 per
    masked multiply-add of Cor. 1, four columns) and issued tensor flops, and the clip's
    algorithmic bytes (the FP32 rows its check reads, (N + 1) x 16 B per cell, the key and the face record)."""
    import paper_2106_10031_gb300 as am
    from synth import decoder_net
    mlp = decoder_net()
    o, d = np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])
    out = {"workload": "decoder (3+256)-[512]x8-1, skip at 4, seed 3, one +x ray, box 1.5"}
    with am.Mesher(device=dev, max_cells=16_000_000, max_neurons=4096, max_width=512) as m:
        nid = m.load_mlp(mlp)
        for prec, cells in (("sliced", 0), ("fp64", fp64_cells)):
            m.reset()
            m.seed(nid, o, d)
            m.march(precision=prec, max_cells=20000)            # warm-up
            runs = []
            for _ in range(reps):
                m.reset()
                m.seed(nid, o, d)
                m.march(precision=prec, max_cells=cells)
                runs.append(m.stats())
            st = min(runs, key=lambda x: x["ms_march"])
            out[prec] = {"faces": st["faces"], "cells": st["cells"], "whole_mesh": cells == 0, "ms": st["ms_march"],
                         "faces_per_s": st["faces"] / (st["ms_march"] / 1e3), "levels": st["levels"],
                         "launches": st["kernel_launches"], "degenerate": st["degenerate"],
                         "empty_faces": st["empty_faces"]}
            if prec == "sliced":
                mesh = m.get_mesh(nid)
                work = algorithmic_work(mlp, mesh)
                cells_n = st["cells"]
                issued = 2 * st["tensor_macs"]                  # BF16 digit-plane products issued
                useful = work["compose_flops"]
                del mesh
                out[prec]["ms_compose"], out[prec]["ms_clip"] = st["ms_compose"], st["ms_clip"]
                out[prec]["compose_roofline"] = {
                    "kernel": "oz_gemm_kernel + oz_prep_kernel", "bound": "tensor",
                    "achieved": useful / (st["ms_compose"] / 1e3) / 1e12, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": useful / (st["ms_compose"] / 1e3) / 1e12 / BF16_PEAK_TFLOPS,
                    "issued_tflops": issued / (st["ms_compose"] / 1e3) / 1e12,
                    "counts": "achieved: useful flops of Cor. 1 (8 per masked multiply-add, 4 columns); issued: "
                              "the BF16 digit-plane products the compose launched (36 per layer on the padded "
                              "tiles; one column per rank-1 cell, four per full compose)"}
                kw = (mlp.N + 63) // 64
                clip_bytes = cells_n * ((mlp.N + 1) * 16 + 8 * kw + 64) + st["corners"] * 28
                gbs = clip_bytes / (st["ms_clip"] / 1e3) / 1e9
                out[prec]["clip_roofline"] = {"kernel": "clip_warp_kernel (+ the block kernel on its fallback list)",
                                              "bound": "hbm",
                                              "achieved": gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                              "frac": gbs / HBM_PEAK_GBS, "bytes_per_cell": clip_bytes / cells_n}
        out["sliced_speedup_vs_fp64"] = out["sliced"]["faces_per_s"] / out["fp64"]["faces_per_s"]
    return out


def trigger_leg(dev, n_starts=1024, n_samples=4096, reps=5):
    """The customised triggers (Sec. 4.3) on the 3-[64]x4-1 sphere net, with the paper's 1024
    initial points: sphere tracing from n_starts points uniform in [-1.4, 1.4]^3 (eta 1, at most
    64 steps, eps 1e-12) and the random-pair dichotomy on n_samples points uniform in
    [-1.5, 1.5]^3 (up to 1024 pairs).  Each call is timed whole on the host clock (copy of the
    points in, the trigger kernels, the dichotomy, the push of the seed cells, the copy of the
    seed points out), best of `reps` after one warm-up; the oracle's time for the same call on a
    64-point sample is reported beside it.  Afterwards the march from all traced seeds against
    the march from one seed: the same mesh, and the breadth-first depth (levels) of each."""
    import paper_2106_10031_gb300 as am
    from synth import sphere_net, trigger_points
    mlp = sphere_net(seed=2, width=64, depth=4, sigma=0.05)
    starts = trigger_points(n_starts, seed=4, box=1.4)
    samples = trigger_points(n_samples, seed=7, box=1.5)
    out = {"workload": f"{mlp.name}: {n_starts} sphere-tracing starts, {n_samples} samples for up to 1024 pairs"}
    with am.Mesher(device=dev, max_cells=1 << 18, max_neurons=max(64, mlp.N), max_width=max(mlp.widths)) as m:
        nid = m.load_mlp(mlp)
        for name, call in (("sphere_trace", lambda: m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12)),
                           ("pairs", lambda: m.seed_pairs(nid, samples, 1024))):
            times, res = [], None
            for _ in range(reps + 1):                   # the first call warms up
                m.reset()
                t0 = time.perf_counter()
                res = call()
                times.append(time.perf_counter() - t0)
            best = min(times[1:])
            pts = res[-1]
            n_in = n_starts if name == "sphere_trace" else n_samples
            out[name] = {"ms": best * 1e3, "points_per_s": n_in / best, "seeds": int(np.sum(~np.isnan(pts[:, 0]))),
                         "new_cells": int(res[-2] if name == "pairs" else res[0])}
        # parallel marching from many seeds (Sec. 4.2): the same mesh, a shallower breadth-first
        # walk; the depth is counted by the level schedule, the persistent one gives the time
        seedings = {"traced_seeds": lambda: m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12),
                    "one_seed": lambda: m.seed(nid, np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]))}
        out["march_by_seeding"] = {"precision": "fp64", "candidates": "nearest"}
        for sched in ("persistent", "levels"):         # warm-up: first launches of both schedules
            m.reset()
            seedings["one_seed"]()
            m.march(schedule=sched)
        for name, seed in seedings.items():
            row = {}
            for sched in ("persistent", "levels"):
                m.reset()
                seed()
                m.march(schedule=sched)
                st = m.stats()
                row[sched] = {"faces": st["faces"], "ms_march": st["ms_march"], "levels": st["levels"]}
            out["march_by_seeding"][name] = row
    out["cpu_baseline"] = trigger_cpu_baseline(mlp, starts[:64], samples[:256])
    return out


def shard_nets(n_nets: int, rank: int, world: int) -> list:
    """Indices of the nets a rank meshes: round robin over the net index.  The nets are
    independent problems, so the ranks exchange nothing on the data path; the round robin
    spreads the batch's mix of small and large nets."""
    return list(range(rank, n_nets, world))


def batch_leg(dist, max_cells=0, precision="mixed", reps=1, box=2.0, capacity=60_000_000):
    """The 64-net batch: batch_nets(master_seed=4) (widths 32-256, depths 4-8, sigma in
    [0.02, 0.1]), one seed ray along +x per net, box [-2, 2]^3 (some of the deeper nets reach
    past 1.5), all of a rank's nets in one persistent launch, marched to completion (3.05e7
    faces in all), or the first max_cells cells of the job (split evenly over the ranks).
    Sharded by net (shard_nets); value = all ranks' faces / the slowest rank's march time, by
    am_march's CUDA events; strong scaling (the total work is fixed)."""
    import paper_2106_10031_gb300 as am
    from synth import batch_nets
    nets = batch_nets()
    mine = [nets[i] for i in shard_nets(len(nets), dist.rank, dist.world)]
    cells = max_cells // dist.world
    o, d = np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])
    with am.Mesher(device=dist.local, max_cells=(cells + 4096) if cells else capacity // dist.world,
                   max_neurons=max(n.N for n in mine), max_width=max(max(n.widths) for n in mine)) as m:
        ids = [m.load_mlp(n) for n in mine]
        runs, unseeded = [], 0
        for _ in range(reps + 1):                   # the first run warms up
            m.reset()
            unseeded = 0
            for i in ids:
                try:
                    m.seed(i, o, d)
                except am.AMError:
                    unseeded += 1
            dist.barrier()
            m.march(box=box, precision=precision, max_cells=cells)
            runs.append(m.stats())
        st = min(runs[1:], key=lambda x: x["ms_march"])
    faces = dist.allreduce(float(st["faces"]), "sum")
    ms = dist.allreduce(float(st["ms_march"]), "max")
    return {"workload": f"64 nets of batch_nets(master_seed=4), box {box}, "
                        f"{'the whole batch' if not max_cells else f'first {max_cells} cells of the job'}, {precision}",
            "n_gpus": dist.world, "scaling": "strong", "sharding": "nets round robin over the ranks, no exchange",
            "faces": int(faces), "ms": ms, "faces_per_s": faces / (ms / 1e3),
            "rank0": {"nets": len(mine), "unseeded_nets": unseeded, "cells": int(st["cells"]),
                      "faces": int(st["faces"]), "ms": float(st["ms_march"])}}


def trigger_cpu_baseline(mlp, starts, samples):
    """The oracle's triggers as they stand, single-threaded, on a sample of the trigger leg's
    points: sphere tracing from `starts`, random pairs (up to 64) from `samples`."""
    from oracle import oracle as orc
    net = orc.OracleNet(mlp)
    t0 = time.perf_counter()
    orc.seed_sphere_trace(net, starts, eta=1.0, max_steps=64, eps=1e-12)
    t_tr = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.seed_pairs(net, samples, 64)
    t_pr = time.perf_counter() - t0
    return {"kind": "oracle", "cores": 1, "sample": f"{len(starts)} starts / {len(samples)} samples",
            "sphere_trace_points_per_s": len(starts) / t_tr, "pairs_points_per_s": len(samples) / t_pr}


def train_proposal(m, mlp, o, d, cells=40000, per_net=12000, steps=3000):
    """The learned proposal, trained outside every timed region on the plain method's faces of
    the 32 training nets (synth.proposal_train_nets: the target's shape and recipe, seeds
    100-131; the target net, seed 5, is not among them): the first `cells` cells of each net's
    march, at most `per_net` samples each, shuffled.  Then its held-out recall@32 on the target
    net's own faces (its first `cells` cells).  Leaves the context holding the target net only."""
    import torch

    from synth import proposal_train_nets
    Xs, Ys = [], []
    t0 = time.perf_counter()
    for net in proposal_train_nets():
        m.reset()
        m.release_nets()
        nid = m.load_mlp(net)
        m.seed(nid, o, d)
        m.march(precision="sliced", candidates="nearest", max_cells=cells)
        X, Y = m.proposal_samples(nid, max_samples=per_net)
        Xs.append(X.clone())
        Ys.append(Y.to(torch.bfloat16))
    label_s = time.perf_counter() - t0
    X = torch.cat(Xs)
    Y = torch.cat(Ys).float()
    del Xs, Ys
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(0)).to(X.device)
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    m.proposal_init(7 + mlp.L, 256, mlp.N, max_batch=1024, seed=0)
    t0 = time.perf_counter()
    losses = m.proposal_train(X, Y, batch=1024, steps=steps, lr=2e-3)
    train_s = time.perf_counter() - t0
    n_samples = int(X.shape[0])
    del X, Y, perm
    m.reset()
    m.release_nets()
    nid = m.load_mlp(mlp)
    m.seed(nid, o, d)
    m.march(precision="sliced", candidates="nearest", max_cells=cells)
    Xt, Yt = m.proposal_samples(nid, max_samples=20000)
    recall = proposal_recall(m, Xt, Yt, 32)
    del Xt, Yt
    m.reset()
    return nid, {"train_nets": "synth.proposal_train_nets(): seeds 100-131", "samples": n_samples,
                 "label_march_s": label_s, "steps": steps, "batch": 1024, "train_s": train_s,
                 "loss_first": float(losses[:5].mean()), "loss_last": float(losses[-50:].mean()),
                 "heldout_recall_at_32": recall, "heldout": "the target net (seed 5), its first 40000 cells"}


def leg(m, nid, o, d, steps, precision, schedule, flush, stream, candidates, dist, max_cells=0):
    measure(m, nid, o, d, 1, precision, schedule, flush, stream, candidates, max_cells=min(20000, max_cells or 20000))
    p = measure(m, nid, o, d, steps, precision, schedule, flush, stream, candidates, max_cells)
    p_ms = dist.allreduce(p["total_ms"], "max")
    st = p["stats"]
    faces = dist.allreduce(float(st["faces"] * steps), "sum")
    return {"value": faces / (p_ms / 1e3), "unit": UNIT, "ms_per_step": p_ms / steps, "steps": steps,
            "faces": st["faces"], "whole_mesh": max_cells == 0, "precision": precision, "schedule": schedule,
            "candidates": candidates, "cuts_per_cell": st["cuts"] / max(1, st["cells"]),
            "corrected_frac": st["fixups"] / max(1, st["cells"]), "refined_cells": st["refined_cells"],
            "ms_compose": p["compose_ms"] / steps, "ms_clip": p["clip_ms"] / steps}


def run_ours(args, dist):
    import torch

    import paper_2106_10031_gb300 as am
    from paper_2106_10031_gb300 import native as nt
    mlp, o, d = workload()
    base = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(mlp, o, d)                   # before any GPU work
    dev = dist.local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    prec = args.precision
    sched = schedule_for(prec, args.schedule)
    m = am.Mesher(device=dev, stream=stream.cuda_stream, **ctx_shape(mlp))
    nid = m.load_mlp(mlp)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")   # > 129 MB L2
    warm = max(args.warmup, 3)
    train = None
    if args.candidates == "learned" or not args.no_compare:
        nid, train = train_proposal(m, mlp, o, d)
    if prec == "sliced":
        train_tune = m.autotune_compose(nid, n=512, reps=3)       # batches of a breadth-first level
    else:
        train_tune = None
    measure(m, nid, o, d, 1, prec, sched, flush, stream, args.candidates, max_cells=20000)
    measure(m, nid, o, d, warm, prec, sched, flush, stream, args.candidates)
    mesh = m.get_mesh(nid)
    faces_per_step = mesh.n_faces
    work = algorithmic_work(mlp, mesh)
    torch.cuda.synchronize()
    dist.barrier()
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed steps
        r = measure(m, nid, o, d, args.steps, prec, sched, flush, stream, args.candidates)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    dist.barrier()
    mesh = m.get_mesh(nid)
    agreement = oracle_agreement(mlp, mesh, golden=load_golden()) if dist.rank == 0 else None
    del mesh
    max_ms = dist.allreduce(r["total_ms"], "max")
    all_faces = dist.allreduce(float(faces_per_step * args.steps), "sum")
    value = all_faces / (max_ms / 1e3)
    legs = None
    if not args.no_compare:
        legs = {}
        for name, p2, c2, k, cells in (("plain_fp64", "fp64", "none", 1, 0), ("fp64_nearest", "fp64", "nearest", 2, 0),
                                       ("sliced_nearest", "sliced", "nearest", 3, 0),
                                       ("fp64_learned", "fp64", "learned", 2, 0),
                                       ("sliced_learned", "sliced", "learned", 3, 0)):
            if (p2, c2) == (prec, args.candidates):
                continue
            g = leg(m, nid, o, d, k, p2, schedule_for(p2, "auto"), flush, stream, c2, dist, cells)
            g["headline_speedup"] = value / g["value"]
            legs[name] = g
        legs["proposal_training"] = train
        legs["compose_autotune"] = train_tune
    e2e = None
    if not args.no_e2e:
        prop = (m.proposal_params(), m.prop_shape) if args.candidates == "learned" else None
        from paper_2106_10031_gb300.mesher import PRECISIONS
        pcode = PRECISIONS[prec]
        scode = nt.AM_SCHED_LEVELS if sched == "levels" else nt.AM_SCHED_PERSISTENT
        e2e = e2e_leg(mlp, o, d, max(2, min(args.steps, 5)), dev, stream.cuda_stream, pcode, scode, args.candidates,
                      prop)
        e2e_ms = dist.allreduce(e2e.pop("ms_per_step") * max(2, min(args.steps, 5)), "max")
        e2e["value"] = dist.allreduce(float(faces_per_step * max(2, min(args.steps, 5))), "sum") / (e2e_ms / 1e3)
    m.close()
    if not args.no_compare:
        legs["many_seeds"] = seeds_leg(dev)
        legs["decoder"] = decoder_leg(dev)
        legs["sphere64x4"] = sphere_leg(dev)
        legs["compose"] = compose_leg(dev)
    if dist.rank != 0:
        return 0
    st = r["stats"]
    # the dominant kernel of the step by device time (the committed launch list): on the sliced
    # path the warp clip (one launch per level, with the block kernel on its fallback list in the
    # same event range), an HBM-bound pass over the rows the compose wrote; otherwise the march
    # kernel.  The compose on the tensor cores (product + prep kernels) is reported beside it.
    cell_ms, comp_ms = r["cell_ms"] if prec != "sliced" else r["clip_ms"], r["compose_ms"]
    kw = (mlp.N + 63) // 64
    per_cell = (mlp.N + 1) * 16 + 8 * kw + 64 if prec == "sliced" else 8 * kw + 64
    byts = (st["cells"] * per_cell + st["corners"] * 28) * args.steps
    ach = byts / (cell_ms / 1e3) / 1e9
    if prec == "sliced":
        kname = "clip_warp_kernel (+ march_range_kernel<double-float> on its fallback list)" \
            if args.candidates != "none" else "march_range_kernel<double-float>"
    else:
        kname = "march_persistent_kernel" if sched == "persistent" else "march_range_kernel"
    launches_per_step = max(1, st["levels"]) if sched == "levels" else 1
    roof = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": HBM_PEAK_GBS, "unit": "GB/s",
            "frac": ach / HBM_PEAK_GBS, "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
            "counts": "algorithmic bytes: the FP32 rows the all-row check reads ((N + 1) x 16 B per cell on the "
                      "sliced path: the hi words of the pairs), the key and the face record (28 B per corner)",
            "units": f"{st['cells']} cells per step in {launches_per_step} launches"}
    roof["traffic"] = captured_traffic(prec, args.candidates, st["cells"] / launches_per_step)
    roof["launch_ms"] = cell_ms / max(1, args.steps) / launches_per_step
    if prec == "sliced":
        cach = work["compose_flops"] * args.steps / (comp_ms / 1e3) / 1e12
        roof["compose"] = {"kernel": "oz_gemm_kernel + oz_prep_kernel + rank-1 kernels (tcgen05)", "bound": "tensor",
                           "achieved": cach, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": cach / BF16_PEAK_TFLOPS,
                           "peak_source": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)",
                           "counts": "useful flops of Cor. 1: 8 per masked multiply-add (4 columns)",
                           "issued_tflops": 2 * st["tensor_macs"] / (comp_ms / args.steps / 1e3) / 1e12,
                           "ms_per_step": comp_ms / args.steps}
    roof["share_of_step"] = {"compose": r["compose_ms"] / max(r["total_ms"], 1e-9),
                             "clip": r["clip_ms"] / max(r["total_ms"], 1e-9),
                             "cell_kernels": r["cell_ms"] / max(r["total_ms"], 1e-9)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": warm, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"sliced": "bf16-digits+f64", "mixed": "f32x2+f64",
                                                          "fp64": "f64"}[prec],
        "data": "synthetic",
        "config": {"workload": workload_name(), "faces_per_step": faces_per_step, "precision": prec,
                   "candidates": args.candidates, "schedule": sched, "parallelism": f"replicas x{dist.world}",
                   "l2": "flushed before every step (256 MiB write); the step's inputs exceed L2"},
        "roofline": roof,
        "algorithmic_work": work,
        "legs": legs,
        "exactness": {"refined_cells": st["refined_cells"], "close_calls": st["close_calls"],
                      "fixups": st["fixups"], "cuts_per_cell": st["cuts"] / max(1, st["cells"]),
                      "degenerate": st["degenerate"], "empty_faces": st["empty_faces"], "vs_oracle": agreement},
        "cpu_baseline": base,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": int(r["launches"]),
    }
    print(json.dumps(line))
    return 0


def ctx_shape(mlp) -> dict:
    """Context capacities for one net of this shape marched to completion (3-[256]x8-1: 1.81e6
    cells)."""
    return {"max_cells": 1 << 22, "max_neurons": max(64, mlp.N), "max_width": max(mlp.widths)}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def schedule_for(precision: str, schedule: str) -> str:
    if schedule != "auto":
        return schedule
    return "levels" if precision == "sliced" else "persistent"


def sphere_leg(dev, steps=3):
    """The 3-[64]x4-1 sphere net (seed 2, sigma 0.05; 43,780 faces, one +x ray, box 1.5) in one
    persistent launch per step: mixed precision and FP64 with nearest-row candidates, and the
    plain FP64 method (every cutting row clipped)."""
    import paper_2106_10031_gb300 as am
    from synth import sphere_net
    mlp = sphere_net(seed=2, width=64, depth=4, sigma=0.05)
    o, d = np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]])
    out = {"workload": "3-[64]x4-1 geometric-init SDF MLP (seed 2, sigma 0.05), one +x ray, box 1.5"}
    with am.Mesher(device=dev, max_cells=1 << 17, max_neurons=256, max_width=64) as m:
        nid = m.load_mlp(mlp)
        for name, prec, cand in (("mixed_nearest", "mixed", "nearest"), ("fp64_nearest", "fp64", "nearest"),
                                 ("plain_fp64", "fp64", "none")):
            runs = []
            for _ in range(steps + 1):
                m.reset()
                m.seed(nid, o, d)
                m.march(precision=prec, candidates=cand)
                runs.append(m.stats())
            st = min(runs[1:], key=lambda x: x["ms_march"])
            out[name] = {"faces": st["faces"], "ms": st["ms_march"], "faces_per_s": st["faces"] / (st["ms_march"] / 1e3),
                         "levels": st["levels"]}
    return out


def proposal_recall(m, X, Y, k=32) -> float:
    """Share of a sample's edge neurons (labels 1) among its k best-scored rows, averaged over
    the samples (the proposal's forward pass on the device)."""
    import torch
    Z = m.proposal_forward(X)
    top = torch.topk(Z, k, dim=1).indices
    hit = torch.gather(Y, 1, top).sum(1)
    return float((hit / Y.sum(1).clamp(min=1)).mean().item())


def load_golden(name="learned_target_256x8"):
    """The oracle's whole-mesh digest of a workload from tests/golden/whole_mesh_oracle.json
    (written by the oracle alone), or None."""
    gpath = os.path.join(ROOT, "tests", "golden", "whole_mesh_oracle.json")
    if not os.path.exists(gpath):
        return None
    with open(gpath) as f:
        g = [x for x in json.load(f)["meshes"] if x["name"] == name]
    return g[0] if g else None


def seeds_leg(dev, n_starts=1024, reps=2):
    """Parallel marching from many trigger points (Sec. 4.2, Sec. 4.3.1): the bench workload
    seeded by sphere tracing from the paper's 1024 initial points (uniform in [-1.4, 1.4]^3; eta 1,
    at most 64 steps), marched with the sliced path: the same mesh as from the one +x ray (face
    keys and edge cycles compared through the whole-mesh digest), a much shallower breadth-first
    walk, hence fewer and fuller levels.  Seeding is timed apart from the march."""
    import paper_2106_10031_gb300 as am
    from synth import trigger_points
    from tests import meshcheck
    mlp, o, d = workload()
    starts = trigger_points(n_starts, seed=4, box=1.4)
    out = {"workload": f"{workload_name('ray')}; seedings compared: one ray, {n_starts} sphere-traced starts, "
                       f"random pairs", "precision": "sliced",
           "candidates": "nearest"}
    digests = {}
    with am.Mesher(device=dev, **ctx_shape(mlp)) as m:
        nid = m.load_mlp(mlp)
        samples = trigger_points(16 * n_starts, seed=5, box=1.4)
        for name, seed in (("one_ray", lambda: m.seed(nid, o, d)),
                           ("traced_seeds", lambda: m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=64, eps=1e-12)),
                           ("traced_seeds_8_steps", lambda: m.seed_sphere_trace(nid, starts, eta=1.0, max_steps=8,
                                                                                 eps=1e-12)),
                           ("pair_seeds", lambda: m.seed_pairs(nid, samples, n_starts))):
            runs = []
            for _ in range(reps + 1):                   # the first run warms up
                m.reset()
                t0 = time.perf_counter()
                seed()
                t_seed = time.perf_counter() - t0
                m.march(precision="sliced", candidates="nearest")
                runs.append((m.stats(), t_seed))
            st, t_seed = min(runs[1:], key=lambda x: x[0]["ms_march"])
            digests[name] = meshcheck.digest(m.get_mesh(nid), mlp.N)
            out[name] = {"faces": st["faces"], "ms_march": st["ms_march"],
                         "faces_per_s": st["faces"] / (st["ms_march"] / 1e3), "levels": st["levels"],
                         "cells_per_level": st["cells"] / max(1, st["levels"]), "seed_ms": t_seed * 1e3,
                         "ms_compose": st["ms_compose"], "ms_clip": st["ms_clip"]}
    out["same_mesh"] = all(digests[k] == digests["one_ray"] for k in digests)
    out["speedup_vs_one_ray"] = out["traced_seeds"]["faces_per_s"] / out["one_ray"]["faces_per_s"]
    for k in ("traced_seeds", "traced_seeds_8_steps", "pair_seeds"):
        out[k]["same_mesh"] = digests[k] == digests["one_ray"]
        out[k]["seeded_march_ms"] = out[k]["ms_march"] + out[k]["seed_ms"]
    return out



def march_once(dev, args):
    """The step's march alone, for a profiler and for the launch-shape comparisons: the workload
    net seeded as the step is (--seeding; the decoder from one +x ray), the chosen precision and
    candidates, args.warmup untimed
    marches first, then one march (args.max_cells cells, 0 = all; the context is sized to it)
    whose am_march CUDA-event times are printed.  Learned candidates come from an untrained
    proposal of the step's shape: the same forward-pass work per level without the training's
    launches in front of a capture (which candidates it picks does not change the launches)."""
    import paper_2106_10031_gb300 as am
    mlp, o, d = workload()
    shape = ctx_shape(mlp)
    if args.net == "decoder":
        from synth import decoder_net
        mlp = decoder_net()
        shape = {"max_cells": 16_000_000, "max_neurons": 4096, "max_width": 512}
    if args.max_cells:
        shape["max_cells"] = min(shape["max_cells"], max(1 << 16, 2 * args.max_cells))
    prec = args.precision
    with am.Mesher(device=dev, **shape) as m:
        nid = m.load_mlp(mlp)
        m.set_tuning(rank1_period=args.rank1_period or None, clip_kernel=0 if args.clip_kernel == "warp" else 1,
                     check_kernel=0 if args.check_kernel == "warp" else 1)
        if args.candidates == "learned":
            m.proposal_init(7 + mlp.L, 256, mlp.N, max_batch=1024, seed=0)
        for _ in range(max(0, args.warmup) + 1):
            m.reset()
            if args.net == "decoder":
                m.seed(nid, o, d)
            else:
                seed_step(m, nid, o, d)
            m.march(precision=prec, schedule=schedule_for(prec, args.schedule), candidates=args.candidates,
                    max_cells=args.max_cells)
        st = m.stats()
        m_tuning = m.get_tuning()
    return {"net": mlp.name, "precision": prec, "candidates": args.candidates, "tuning": m_tuning,
            "max_cells": args.max_cells,
            "faces": st["faces"], "ms_march": st["ms_march"], "levels": st["levels"],
            "kernel_launches": st["kernel_launches"], "ms_compose": st["ms_compose"], "ms_clip": st["ms_clip"],
            "clip_fallbacks": st["clip_fallbacks"], "tensor_macs": st["tensor_macs"]}

def main():
    global SEEDING
    args = parse()
    SEEDING = args.seeding
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, dist)
        if args.compose_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "compose", **compose_leg(dist.local)}))
            return 0
        if args.decoder_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "decoder", **decoder_leg(dist.local, fp64_cells=0)}))
            return 0
        if args.batch_only:
            out = batch_leg(dist, precision=args.precision if args.precision != "sliced" else "mixed")
            if dist.rank == 0:
                print(json.dumps({"leg": "batch64", **out}))
            return 0
        if args.march_once:
            if dist.rank == 0:
                print(json.dumps({"leg": "march_once", **march_once(dist.local, args)}))
            return 0
        if args.seeds_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "many_seeds", **seeds_leg(dist.local)}))
            return 0
        if args.triggers_only:
            if dist.rank == 0:
                print(json.dumps({"leg": "triggers", **trigger_leg(dist.local)}))
            return 0
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
