#!/usr/bin/env python
"""Throughput benchmark of the narrow-band SDF path on one GB300 (one JSON line on stdout).

Default workload (--workload c2): a 50,000-triangle displaced, jittered torus soup
(R=0.3, r=0.1), grid 512^3 on [0,1]^3, band half-width 4h.  One step is the whole
path: sdf_build_features (weld, pair, records) + sdf_narrow_band_list (bin, scan
conversion + merge + dense write of the field and the compact band list, FP64
re-decision) + sdf_band_list_l2 (L = sum_band (d - 0.01)^2 and its vertex adjoint,
fused in one pass over the band list).  With --schedule cell or --shard slabs the
adjoint takes the dense path instead (dense winners, sdf_narrow_band_backward with the
upstream gradient formed once from the first forward).  --workload c4 times the
2,097,152-triangle knot tube on 1024^3, band 3h (forward only).

value = band points produced per second (all ranks), device-timed with CUDA events;
e2e = the same metric through the public API with host buffers (pinned H2D of the
soup, D2H of the SDF and the vertex gradient inside the timed region).
--impl reference times the FP64 CPU oracle on a bounded slab of the same workload.
Multi-GPU (torchrun): by default each rank evaluates one z-slab of the grid (the whole mesh's
features, the slab's layers) with the vertex gradient summed over the ranks by one all-reduce
(strong scaling); --shard replicas runs an independent copy of the workload per rank instead (weak
scaling, no data-path collective).
Timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "narrow-band grid points/s and fwd+adjoint ms at 1 GB300 vs plain fwd; fraction of HBM roofline"
UNIT = "band points/s"

WORKLOADS = {
    "c1": dict(index=1, adjoint=False, winner=False,
               desc="icosphere nu=4 r=0.3 (320 triangles), grid 64^3 on [0,1]^3, band 3h, forward"),
    "c2": dict(index=2, adjoint=True, winner=True,
               desc="displaced jittered torus R=0.3 r=0.1 (50,000 triangles), grid 512^3 on [0,1]^3, band 4h, "
                    "forward + loss and vertex adjoint of sum_band (d - 0.01)^2"),
    "c3": dict(index=3, adjoint=False, winner=False, batch=True,
               desc="batch of 64 seeded uneven meshes (log-uniform 1e3..2e5 triangles; displaced icospheres, "
                    "displaced tori, unions of 2-4 overlapping rotated boxes), per-mesh grids N in {64, 96, ..., 384} "
                    "on [0,1]^3, band 3h; forward of all 64 problems as one launch sequence replayed from a "
                    "CUDA graph, autotuned tile shape"),
    "c4": dict(index=4, adjoint=False, winner=False,
               desc="(3,7) torus-knot tube r=0.04 + 0.005 noise (2,097,152 triangles), grid 1024^3 on [0,1]^3, "
                    "band 3h, forward"),
    "c5": dict(index=5, adjoint=True, winner=True,
               desc="displaced icosphere nu=100 (200,000 triangles), grid 512^3 on [0,1]^3, band 4h, "
                    "forward + vertex adjoint"),
    "c5fit": dict(index=5, adjoint=True, winner=True, fit=True,
                  desc="shape fitting: displaced icosphere nu=100 (200,000 triangles), grid 512^3, band 4h; "
                       "one plain gradient-descent step on the welded vertices of "
                       "sum_band (d - d_ellipsoid(0.35, 0.25, 0.2))^2 (position update, forward with the "
                       "compact band list, loss and vertex gradient fused in one pass over the list)"),
}
WORKLOADS["cluster"] = dict(
    index=None, adjoint=False, winner=False, cluster=True,
    desc="very uneven triangle sizes: a coarse icosphere (320 triangles, r=0.3) and a separate dense "
         "cluster (icosphere nu=60, 72,000 triangles of radius 2e-4); build time against a uniform "
         "icosphere of 72,000 triangles, and the forward on 256^3, band 3h")
FIT_LR = 1e-4  # fixed learning rate of the shape-fitting workload

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_tile launch on a workload at
# its default grid, from the ncu capture summarised in the named profile.  A figure is reported only
# while the tile kernel's code still hashes to the captured one: first 16 hex digits of the sha256
# of band.cu with // comments and blank lines removed (code_hash below).
TILE_TRAFFIC = {
    "c2": {"bytes": 17_360_896 + 500_167_168, "band_cu_code_hash": "939fae67774dff57",
           "profile": "profiles/k_tile_torus_50k_512.md", "warp_instructions": 172_031_890},
}
# Instruction issue is the other roof of the tile kernel (its band work): 152 SMs x 4 schedulers x
# 1 warp instruction per clock at the 2070 MHz maximum SM clock.
ISSUE_PEAK = 152 * 4 * 2070e6  # warp instructions per second


def code_hash(path: str) -> str:
    import hashlib
    import re
    lines = []
    with open(path) as f:
        for line in f.read().splitlines():
            line = re.sub(r"//.*$", "", line).rstrip()
            if line.strip():
                lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def tile_traffic(name: str, default_grid: bool, key: str = "bytes"):
    rec = TILE_TRAFFIC.get(name)
    if rec is None or not default_grid:
        return None
    if code_hash(os.path.join(ROOT, "paper_1903_00353_gb300", "csrc", "band.cu")) != rec["band_cu_code_hash"]:
        return None
    return rec.get(key)


def step_stats(step_ms) -> dict:
    """Median and minimum of this rank's per-step times (the paper quotes the minimum of several
    runs); the line's ms_per_step stays the mean of the timed region."""
    a = np.asarray(step_ms, dtype=np.float64)
    return {"ms_per_step_median": float(np.median(a)), "ms_per_step_min": float(a.min())}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


_RATES = None


def measured_rates(sdf, dev) -> dict:
    """Rates of the merge's 64-bit atomicMin (shared memory: the tile kernel; global memory within L2
    and beyond it: the paper's schedule) and of FP64 FMAs, measured once per process with the
    library's rate probes (each launch sized to about 2 ms, CUDA events on the launching stream,
    best of 3 after a warm-up)."""
    global _RATES
    if _RATES is not None:
        return _RATES
    import torch
    buf = torch.full((1 << 28,), -1, dtype=torch.int64, device=dev)  # 2 GiB: beyond L2
    cases = {"smem_atomic_min_per_s": (sdf.PROBE_SMEM_ATOMIC_MIN, buf[: 1 << 12], 4096),
             "l2_atomic_min_per_s": (sdf.PROBE_GLOBAL_ATOMIC_MIN, buf[: 1 << 21], 256),  # 16 MiB footprint
             "hbm_atomic_min_per_s": (sdf.PROBE_GLOBAL_ATOMIC_MIN, buf, 256),  # 2 GiB footprint
             "fp64_flops_per_s": (sdf.PROBE_FP64_FMA, buf[:1], 256)}
    out = {}
    for key, (kind, b, iters) in cases.items():
        def timed(it):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ops = sdf.probe_rate(kind, b, it)
            e1.record()
            e1.synchronize()
            return ops, e0.elapsed_time(e1)
        _, ms = timed(iters)
        iters = int(min(1 << 22, max(1, iters * 2.0 / max(ms, 1e-3))))
        best = 0.0
        for _ in range(3):
            ops, ms = timed(iters)
            best = max(best, ops / (ms / 1e3))
        out[key] = best
    del buf
    torch.cuda.empty_cache()
    out["how"] = ("sdf_probe_rate: atomicMin(u64) on 32 KB of shared memory per CTA (lane l on word l + 32m); "
                  "on pseudo-random words of a 16 MiB (L2) and a 2 GiB (HBM) footprint; FP64 FMA chains")
    _RATES = out
    return out


def atomic_roof(ops: int, rates: dict, space: str, hbm_bytes: int, hbm_gbs: float, measured_ms: float) -> dict:
    """The atomic side of the roofline max(bytes / HBM bandwidth, atomics / atomic rate): the merge's
    (point, region) atomicMin count over the measured rate of the space it runs in."""
    key = {"shared": "smem_atomic_min_per_s", "global": "hbm_atomic_min_per_s"}[space]
    t_atomic = ops / rates[key] * 1e3
    t_hbm = hbm_bytes / (hbm_gbs * 1e9) * 1e3
    t_roof = max(t_atomic, t_hbm)
    return {"ops": int(ops), "space": space, "rate": rates[key], "rate_unit": "atomicMin(u64)/s",
            "rate_source": "measured in this run (sdf_probe_rate)", "atomic_ms": t_atomic, "hbm_ms": t_hbm,
            "roof_ms": t_roof, "bound": "atomic" if t_atomic > t_hbm else "hbm",
            "frac_of_max_roof": t_roof / measured_ms}


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background (200 ms period)."""
    Q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid and ("GPU-" + self.uuid) != parts[0]:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


class StepClocks:
    """Per-step SM clock and clock-event reasons, read through NVML (read-only queries) right after
    each timed step; empty when NVML is not available."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid: str | None):
        import ctypes
        self.mhz, self.reasons, self.h = [], set(), None
        try:
            self.L = ctypes.CDLL("libnvidia-ml.so.1")
            if self.L.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            u = uuid if uuid is None or uuid.startswith("GPU-") else "GPU-" + uuid
            if u is None or self.L.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) != 0:
                return
            self.h = h
        except Exception:
            self.h = None

    def read(self):
        if self.h is None:
            return
        import ctypes
        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        if self.L.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz)) == 0:  # NVML_CLOCK_SM
            self.mhz.append(int(mhz.value))
        fn = getattr(self.L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(self.L, "nvmlDeviceGetCurrentClocksThrottleReasons")
        if fn(self.h, ctypes.byref(rs)) == 0:
            for bit, name in self.REASONS.items():
                if rs.value & bit:
                    self.reasons.add(name)

    def summary(self):
        if not self.mhz:
            return None
        a = np.asarray(self.mhz, dtype=np.float64)
        return {"per_step_sm_mhz_median": float(np.median(a)), "per_step_sm_mhz_min": float(a.min()),
                "steps_read": int(a.size), "reasons": sorted(self.reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def record_bytes(feats) -> int:
    """Feature-record bytes the tile kernel reads once (face 4+2 float4, edge 5 float4 + class,
    vertex 2 float4 + class + one float4 plane per corner)."""
    T, E, V = feats.n_tri, feats.n_edge, feats.n_vert
    return T * 96 + E * 81 + V * 33 + 3 * T * 16


def cpu_baseline(soup, N, w, target_s: float = 12.0):
    """The oracle as it stands on a z-slab of the workload grid: rate of band points produced."""
    import oracle
    t0 = time.perf_counter()
    om = oracle.OracleMesh.from_soup(soup)
    t_build = time.perf_counter() - t0
    z = soup[..., 2].ravel()
    kmid = int(np.clip(np.median(z) * N, 0, N - 1))
    layers, band, spent = 1, 0, 0.0
    while True:
        k0 = max(0, kmid - layers // 2)
        t1 = time.perf_counter()
        d = om.narrow_band((N, N, layers), (0.0, 0.0, k0 / N), 1.0 / N, w)
        dt = time.perf_counter() - t1
        band, spent = int(np.isfinite(d).sum()), dt
        if dt > target_s / 4 or layers * 2 > N:
            break
        layers *= 2
    frac = layers / N
    rate = band / (spent + t_build * frac)
    one, brute = _oracle_extras(om, near_surface_points(soup, 20_000, 353_402, w))
    return {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{layers} of {N} z-layers through the mesh middle ({band} band points, {spent:.1f} s) "
                      f"plus the oracle's mesh build ({t_build:.2f} s) prorated by {frac:.4f}",
            "one_core": one, "brute_force": brute}


def _oracle_extras(om, pts, n_one: int = 20_000, n_brute: int = 4):
    """The oracle on one core (the first n_one points) and the literal brute-force loop (every
    point against every triangle, the plain definition of Eq. 1) on n_brute points."""
    import oracle
    cores = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        om.sdf_points(pts[:n_one], pruned=True)
        t1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    t0 = time.perf_counter()
    om.sdf_points(pts[:n_brute], pruned=False)
    tb = time.perf_counter() - t0
    return ({"points_per_s": n_one / t1, "cores": 1, "sample": f"{n_one} points near the surface, pruned search"},
            {"pairs_per_s": n_brute * om.T / tb, "sample": f"{n_brute} points x {om.T} triangles, literal loop"})


def near_surface_points(soup, n, seed, spread):
    """Seeded points near the surface: random points of random triangles moved along the normal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = soup.astype(np.float64)
    t = rng.integers(0, s.shape[0], size=n)
    bc = rng.dirichlet([1, 1, 1], size=n)
    base = np.einsum("ij,ijk->ik", bc, s[t])
    nrm = np.cross(s[t, 1] - s[t, 0], s[t, 2] - s[t, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return base + nrm * rng.uniform(-spread, spread, size=(n, 1))


def cpu_baseline_sampled(soup, N, w, band_total, n_points: int = 1_000_000):
    """The oracle as it stands on 10^6 grid points sampled near the surface of a large workload:
    band points produced per second on all cores, the time per point, the full band's time
    extrapolated from it (labelled), a one-core figure and the literal brute-force rate."""
    import oracle
    t0 = time.perf_counter()
    om = oracle.OracleMesh.from_soup(soup)
    t_build = time.perf_counter() - t0
    pts = near_surface_points(soup, n_points, 353_404, w)
    ijk = np.clip(np.rint(pts * N - 0.5).astype(np.int64), 0, N - 1)
    idx = np.unique(ijk[:, 0] + N * (ijk[:, 1] + N * ijk[:, 2]))
    t0 = time.perf_counter()
    d, _, _ = om.band_points((N, N, N), (0.0, 0.0, 0.0), 1.0 / N, w, idx)
    dt = time.perf_counter() - t0
    band = int(np.isfinite(d).sum())
    per_point = dt / idx.size
    one, brute = _oracle_extras(om, oracle.grid_points((N, N, N), (0, 0, 0), 1.0 / N, idx[:20_000]))
    return {"value": band / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{idx.size} grid points near the surface ({band} in the band), {dt:.1f} s; mesh build "
                      f"{t_build:.1f} s not included",
            "seconds_per_point": per_point,
            "full_band_seconds_extrapolated": per_point * band_total,
            "extrapolation": "time per sampled point x the band points of the full grid (a labelled estimate, "
                             "not a measurement)",
            "one_core": one, "brute_force": brute}


def batch_problems():
    """The 64 (soup, N, w) problems of the batch workload (band 3h)."""
    import meshgen
    return [(m.soup(seed=353_300 + i), N, 3.0 / N) for i, (m, N) in enumerate(meshgen.batch_meshes())]


def median_problem(problems):
    """The batch problem whose grid size times triangle count is the median (a sample for the oracle)."""
    order = sorted(range(len(problems)), key=lambda i: problems[i][0].shape[0] * problems[i][1] ** 3)
    return problems[order[len(order) // 2]]


def run_reference(args, wl):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import meshgen
    import oracle
    if wl.get("batch"):
        soup, N, w = median_problem(batch_problems())
    else:
        soup = meshgen.config_soup(wl["index"])
        N, cells = meshgen.CONFIG_GRID[wl["index"]]
        w = cells / N
    om = oracle.OracleMesh.from_soup(soup)
    z = soup[..., 2].ravel()
    kmid = int(np.clip(np.median(z) * N, 0, N - 1))
    layers = 2
    # each step evaluates a bounded slab of the workload (the oracle as it stands)
    def step(i):
        k0 = (kmid - layers * 4 + layers * (i % 8)) % max(1, N - layers)
        d = om.narrow_band((N, N, layers), (0.0, 0.0, k0 / N), 1.0 / N, w)
        return int(np.isfinite(d).sum())
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    band = sum(step(i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    value = band / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "sample": f"{layers} z-layers per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{layers} of {N} z-layers per step near the mesh middle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ellipsoid_target(N, dev):
    """Exact SDF of the ellipsoid (0.35, 0.25, 0.2) at the cell centres (float32), in z slabs."""
    import torch
    import meshgen
    c = (torch.arange(N, device=dev, dtype=torch.float64) + 0.5) / N
    out = torch.empty((N, N, N), dtype=torch.float32, device=dev)
    Y, X = torch.meshgrid(c, c, indexing="ij")
    for k0 in range(0, N, 32):
        k1 = min(N, k0 + 32)
        Z = c[k0:k1].view(-1, 1, 1).expand(k1 - k0, N, N)
        P = torch.stack([X.expand(k1 - k0, N, N), Y.expand(k1 - k0, N, N), Z], dim=-1)
        out[k0:k1] = meshgen.ellipsoid_sdf_torch(P).to(torch.float32)
    return out


def run_fit(args, wl, sdf, soup_np, soup, grid, w, N, dev, world, rank):
    """Shape-fitting workload: every step is one plain gradient-descent step on the welded vertices."""
    import torch
    import torch.distributed as tdist
    target = ellipsoid_target(N, dev)
    feats = sdf.sdf_build_features(soup)
    X = feats.vertices().clone()
    dist = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    gv = torch.zeros_like(X)
    # one synchronous forward sizes the band list (a quarter of spare room: the band changes little
    # over the steps, and an overflow would be reported by the status check after the loop)
    _, bl = sdf.sdf_narrow_band_list(feats, grid, w, out=dist)
    bl = sdf.BandList(len(bl) + len(bl) // 4 + 4096, device=dev)

    def fit_step(ev=None):
        """Positions in, forward with the compact band list, loss and vertex gradient fused over
        the list, update: all in the library's kernels except the update (a 1 MB axpy)."""
        if ev:
            ev[0].record()
        feats.update_positions(X)
        sdf.sdf_narrow_band_list(feats, grid, w, out=dist, band_list=bl, flags=sdf.FLAG_NO_SYNC)
        if ev:
            ev[1].record()
        gv.zero_()
        loss, _, band = sdf.band_list_l2(feats, grid, bl, dist, target, grad_vertices=gv)
        X.sub_(FIT_LR * gv)
        if ev:
            ev[2].record()
        return loss, band

    losses = []
    for _ in range(args.warmup):
        losses.append(fit_step()[0])
    torch.cuda.synchronize()
    launches0 = sdf.kernel_launches()
    per, bands = [], []
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    with ClockSampler(uuid) as clk:
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            l, b = fit_step(evs)
            losses.append(l)
            bands.append(b)
            per.append(evs)
        torch.cuda.synchronize()
    launches = sdf.kernel_launches() - launches0
    feats.status()  # raises if a forward without synchronisation outgrew its scratch
    times = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])] for e in per])
    total_ms = float(times.sum())
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    band_total = int(sum(int(b) for b in bands))
    value = band_total * world / (total_ms / 1e3)
    loss_curve = [float(x) for x in losses]
    # end to end: vertex positions from pinned host memory each step, loss read back each step
    Xh = X.cpu().pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, min(args.steps, 10))
    e2e_band = 0
    for _ in range(e2e_steps):
        X.copy_(Xh, non_blocking=True)
        l, b = fit_step()
        e2e_band += int(b)
        float(l)
    e2e_s = time.perf_counter() - t0
    if rank != 0:
        return
    fwd_ms, rest_ms = (float(x) for x in times.mean(axis=0))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, **step_stats(times.sum(axis=1)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "triangles": int(soup_np.shape[0]), "grid": [N, N, N], "band_w": w,
                   "lr": FIT_LR, "l2": "inputs of the dense loss (> L2) streamed every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "fwd_ms": fwd_ms, "loss_and_adjoint_ms": rest_ms, "loss_curve": loss_curve,
        "e2e": {"value": e2e_band * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(Xh.numel() * 4),
                "d2h_bytes_per_step": 4},
        "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
        "cpu_baseline": None, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_cluster(args, wl, sdf, local, world, rank):
    """Build time of a mesh with a dense cluster of tiny triangles (many distinct vertices under one
    spatial weld key) against a uniform mesh of about the same size, and its forward."""
    import torch
    import meshgen
    dev = torch.device("cuda", local)
    soups = {"cluster": meshgen.dense_cluster().soup(seed=353_901),
             "uniform": meshgen.icosphere(60, radius=0.3).soup(seed=353_902)}
    res = {}
    for name, s_np in soups.items():
        soup = torch.from_numpy(s_np).to(dev)
        for _ in range(args.warmup):
            sdf.sdf_build_features(soup).destroy()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f = sdf.sdf_build_features(soup)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            f.destroy()
        res[name] = {"triangles": int(s_np.shape[0]), "build_ms_median": float(np.median(ms)),
                     "build_ms_min": float(min(ms))}
    # the cluster mesh's forward on 256^3, band 3h
    N = 256
    grid, w = sdf.Grid.cube(N), 3.0 / N
    f = sdf.sdf_build_features(torch.from_numpy(soups["cluster"]).to(dev))
    out = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        sdf.sdf_narrow_band(f, grid, w, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sdf.sdf_narrow_band(f, grid, w, out=out)
    e1.record()
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / args.steps
    band = int(torch.isfinite(out).sum())
    if rank != 0:
        return
    line = {"metric": METRIC, "value": band / (fwd_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fwd_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "grid": [N, N, N], "band_w": w, "band_points": band},
            "build": res, "build_cluster_over_uniform": res["cluster"]["build_ms_median"] / res["uniform"]["build_ms_median"],
            "gpu_launches": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def run_batch(args, wl, sdf, local, world, rank):
    """Batch workload: all 64 problems in one launch sequence (one persistent tile kernel) captured
    in a CUDA graph; one step = one replay.  Also times the plain path (64 single-problem calls)."""
    import torch
    import torch.distributed as tdist
    dev = torch.device("cuda", local)
    problems = batch_problems()
    soups = [torch.from_numpy(s).to(dev) for s, _, _ in problems]
    grids = [sdf.Grid.cube(N) for _, N, _ in problems]
    ws = [w for _, _, w in problems]
    t0 = time.perf_counter()
    feats = [sdf.sdf_build_features(s) for s in soups]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    outs = [torch.empty(g.shape, dtype=torch.float32, device=dev) for g in grids]
    t0 = time.perf_counter()
    batch = sdf.sdf_batch_create(feats, grids, ws, out=outs, autotune=True, timing=True)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    band_points = sum(int(torch.isfinite(o).sum()) for o in outs)
    stats = batch.status()
    info = batch.info()
    rec_bytes = sum(record_bytes(f) for f in feats)
    grid_points = sum(g.nx * g.ny * g.nz for g in grids)

    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    launches0 = sdf.kernel_launches()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            batch.run()
    torch.cuda.synchronize()
    per_replay = sdf.kernel_launches() - launches0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    per, tile_ms = [], []
    with ClockSampler(uuid) as clk:
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1))
            tile_ms.append(batch.timing()["tile"])
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
    launches = per_replay * args.steps
    total_ms = float(sum(per))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = band_points * args.steps * world / (total_ms / 1e3)

    # the plain path on the same problems: 64 single-problem calls (each synchronises once)
    for f, g, w, o in zip(feats, grids, ws, outs):
        sdf.sdf_narrow_band(f, g, w, out=o)
    torch.cuda.synchronize()
    plain = []
    for _ in range(max(3, min(args.steps, 5))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for f, g, w, o in zip(feats, grids, ws, outs):
            sdf.sdf_narrow_band(f, g, w, out=o)
        e1.record(stream)
        e1.synchronize()
        plain.append(e0.elapsed_time(e1))
    plain_ms = float(np.mean(plain))

    # end to end: soups from pinned host memory, 64 builds, one batched list call, all fields read back;
    # two output sets and two streams let the copy-out of step i overlap the work of step i + 1
    soups_host = [torch.from_numpy(s).pin_memory() for s, _, _ in problems]
    outs_host = [torch.empty(g.shape, dtype=torch.float32).pin_memory() for g in grids]
    outs2 = [outs, [torch.empty_like(o) for o in outs]]
    sc, sx = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    computed = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    handles = []

    def e2e_step(i):
        b = i & 1
        with torch.cuda.stream(sc):
            if i >= 2:
                sc.wait_event(copied[b])
            fl = [sdf.sdf_build_features(sh.to(dev, non_blocking=True), stream=sc) for sh in soups_host]
            sdf.sdf_narrow_band(fl, grids, ws, out=outs2[b], stream=sc)
            computed[b].record(sc)
        with torch.cuda.stream(sx):
            sx.wait_event(computed[b])
            for oh, o in zip(outs_host, outs2[b]):
                oh.copy_(o, non_blocking=True)
            copied[b].record(sx)
        handles.extend(fl)

    for i in range(2):  # fill the two-stage pipeline
        e2e_step(i)
    e2e_steps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(2, 2 + e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    for f in handles:
        f.destroy()
    e2e = {"value": band_points * e2e_steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(sum(s.nbytes for s, _, _ in problems)),
           "d2h_bytes_per_step": int(4 * grid_points)}

    hbm, peak_kind = peaks()
    tile_avg_ms = float(np.mean(tile_ms))
    alg_bytes = 4 * grid_points + rec_bytes
    achieved = alg_bytes / (tile_avg_ms / 1e3) / 1e9
    roofline = {"kernel": "k_tile (all 64 problems in one persistent launch)", "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_kind,
                "traffic": None, "algorithmic_bytes": int(alg_bytes), "avg_ms": tile_avg_ms}
    roofline["atomic"] = atomic_roof(stats["candidates"], measured_rates(sdf, dev), "shared", alg_bytes, hbm,
                                     tile_avg_ms)
    del graph
    batch.destroy()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        s_np, N, w = median_problem(problems)
        cpu = cpu_baseline(s_np, N, w)
        cpu["sample"] = f"median problem of the batch ({s_np.shape[0]} triangles, {N}^3): " + cpu["sample"]
    tris = [s.shape[0] for s, _, _ in problems]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, **step_stats(per), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "meshes": len(problems), "triangles_total": int(sum(tris)),
                   "triangles_min_max": [int(min(tris)), int(max(tris))], "grid_points_total": int(grid_points),
                   "band_points": band_points, "tile_shape": list(info["tile"]),
                   "l2": "outputs (%.1f GB) larger than L2" % (4 * grid_points / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "batch_ms": total_ms / args.steps, "plain_ms": plain_ms, "plain_over_batch": plain_ms / (total_ms / args.steps),
        "autotune_ms_per_run": info["tuned_ms"], "build_all_s": build_s, "batch_create_s": create_s,
        "candidates_per_band_point": stats["candidates"] / max(1, stats["band_points"]),
        "fp64_points": stats["fp64_points"], "tile_region_pairs": stats["pairs"],
        "roofline": roofline, "rates": measured_rates(sdf, dev), "cpu_baseline": cpu, "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": int(launches), "gpu_launches_per_step": per_replay,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c4", action="store_true", help="leave the knot-tube record out of the default line")
    ap.add_argument("--grid", type=int, default=None, help="override the grid size N (same mesh, same band in cells)")
    ap.add_argument("--schedule", default="tile", choices=["tile", "cell"],
                    help="forward schedule: the binned tile kernel, or the paper's thread-per-region cell loop "
                         "(schedule comparison)")
    ap.add_argument("--shard", default="slabs", choices=["replicas", "slabs"],
                    help="N > 1: one z-slab of the grid per rank with the vertex gradient summed over the ranks "
                         "(slabs, strong scaling: the partitioning of the method, the default) or every rank "
                         "running the whole workload (replicas, weak scaling)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    import torch.distributed as tdist

    import meshgen
    import paper_1903_00353_gb300 as sdf

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        tdist.barrier()
    sdf.load_library()
    if wl.get("batch"):
        run_batch(args, wl, sdf, local, world, rank)
        if world > 1:
            tdist.destroy_process_group()
        return
    if wl.get("cluster"):
        run_cluster(args, wl, sdf, local, world, rank)
        if world > 1:
            tdist.destroy_process_group()
        return
    line = run_single(args, args.workload, wl, sdf, world, rank, local)
    # the default workload's line also carries the 2.1M-triangle knot tube at 1024^3 (forward only),
    # the workload the roofline target is stated for
    if line is not None and args.workload == "c2" and not args.grid and args.schedule == "tile" and world == 1 \
            and not args.no_c4:
        sub = run_single(args, "c4", WORKLOADS["c4"], sdf, world, rank, local)
        keep = ("value", "unit", "ms_per_step", "ms_per_step_median", "ms_per_step_min", "config", "build_ms",
                "fwd_ms", "candidates_per_band_point", "fp64_points", "tile_region_pairs", "rows", "rows_hit",
                "roofline", "sparse", "cpu_baseline", "clocks", "e2e", "gpu_launches")
        line["c4"] = {k: sub[k] for k in keep if k in sub}
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def run_single(args, name, wl, sdf, world, rank, local):
    """One single-mesh workload: the timed steps, the end-to-end loop, the roofline records and
    (rank 0) the CPU baseline.  Returns the JSON line's dict on rank 0, else None."""
    import torch
    import torch.distributed as tdist

    import meshgen
    soup_np = meshgen.config_soup(wl["index"])
    N, cells = meshgen.CONFIG_GRID[wl["index"]]
    if args.grid:
        N = args.grid
        wl = dict(wl, desc=wl["desc"].replace(f"{meshgen.CONFIG_GRID[wl['index']][0]}^3", f"{N}^3"))
    w = cells / N
    from paper_1903_00353_gb300 import slabs
    shard = args.shard == "slabs" and world > 1
    grid = slabs.slab_grid(sdf.Grid.cube(N), world, rank) if shard else sdf.Grid.cube(N)
    dev = torch.device("cuda", local)
    soup = torch.from_numpy(soup_np).to(dev)
    dist = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    win = torch.empty(grid.shape, dtype=torch.int32, device=dev) if wl["winner"] else None
    gv = None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    if wl.get("fit"):
        run_fit(args, wl, sdf, soup_np, soup, grid, w, N, dev, world, rank)
        return None

    # upstream gradient of L = sum_band (d - 0.01)^2 from one forward (same mesh every step)
    sched_flag = sdf.FLAG_CELL_LOOP if args.schedule == "cell" else 0
    feats = sdf.sdf_build_features(soup)
    sdf.sdf_narrow_band(feats, grid, w, out=dist, winner=win if win is not None else False, flags=sched_flag)
    band_points = int(torch.isfinite(dist).sum())
    band_total = band_points * world  # replicas: every rank produces the same band
    if shard:  # slabs: the ranks' bands partition the whole grid's band
        t = torch.tensor([band_points], dtype=torch.int64, device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.SUM)
        band_total = int(t.item())
    stats = feats.status()
    rec_bytes = record_bytes(feats)
    g = None
    # the adjoint runs over the compact band list (loss and gradient fused) on the tile schedule;
    # the paper's schedule and z-slabs keep the dense winners and the dense upstream gradient
    use_list = bool(wl["adjoint"]) and args.schedule == "tile" and not shard
    target = torch.full(grid.shape, 0.01, dtype=torch.float32, device=dev) if wl["adjoint"] else None
    bls = [None, None]
    if wl["adjoint"]:
        g = torch.where(torch.isfinite(dist), 2.0 * (dist - 0.01), torch.zeros_like(dist))
        gv = torch.zeros(feats.n_vert, 3, dtype=torch.float32, device=dev)
    if use_list:
        bls = [sdf.BandList(band_points + band_points // 4 + 4096, device=dev) for _ in range(2)]
        win = None
    feats.destroy()

    def step(timed_events=None):
        ev = timed_events
        if ev:
            ev[0].record()
        f = sdf.sdf_build_features(soup)
        if ev:
            ev[1].record()
        # no status read inside the step: the caller checks each step's status after its events
        if use_list:
            sdf.sdf_narrow_band_list(f, grid, w, out=dist, band_list=bls[0], flags=sdf.FLAG_TIMING | sdf.FLAG_NO_SYNC)
        else:
            sdf.sdf_narrow_band(f, grid, w, out=dist, winner=win if win is not None else False,
                                flags=sdf.FLAG_TIMING | sdf.FLAG_NO_SYNC | sched_flag)
        if ev:
            ev[2].record()
        if use_list:  # L = sum_band (d - 0.01)^2 and dL/dV in one pass over the band list
            gv.zero_()
            sdf.band_list_l2(f, grid, bls[0], dist, target, grad_vertices=gv, flags=sdf.FLAG_TIMING)
        elif wl["adjoint"]:
            gv.zero_()
            sdf.sdf_narrow_band_backward(f, grid, w, g, winner=win, grad_vertices=gv, flags=sdf.FLAG_TIMING)
            if shard:
                slabs.all_reduce_sum(gv)  # the one exchange: dL/dV summed over the slabs
        if ev:
            ev[3].record()
        return f

    for _ in range(args.warmup):
        f = step()
        f.status()  # raises if the step's forward outgrew its scratch or its band list
        f.destroy()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    per = []
    tile_ms, tile_calls = 0.0, 0
    launches0 = sdf.kernel_launches()
    step_clk = StepClocks(uuid)
    with ClockSampler(uuid) as clk:
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 between timed steps
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            f = step(evs)
            torch.cuda.synchronize()
            step_clk.read()  # the SM clock right after the step, while it is still at its loaded value
            f.status()
            t = f.timing()
            tile_ms += t["tile"][0]
            tile_calls += t["tile"][1]
            f.destroy()
            per.append([evs[0].elapsed_time(evs[1]), evs[1].elapsed_time(evs[2]), evs[2].elapsed_time(evs[3])])
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()
    launches = sdf.kernel_launches() - launches0
    per = np.array(per)
    total_ms = float(per.sum())
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = band_total * args.steps / (total_ms / 1e3)
    build_ms, fwd_ms, adj_ms = (float(x) for x in per.mean(axis=0))

    # end to end through the public API with host buffers: every step copies the soup in from
    # pinned host memory and the field (and the vertex gradient) out to pinned host memory.  Two
    # buffer sets and two streams let the copy-out of step i overlap the work of step i + 1.
    soup_host = torch.from_numpy(soup_np).pin_memory()
    sc, sx = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    dists = [dist, torch.empty_like(dist)]
    wins = [win, torch.empty_like(win)] if win is not None else [None, None]
    gvs = [gv, torch.empty_like(gv)] if gv is not None else [None, None]
    dist_hosts = [torch.empty(grid.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    gv_hosts = [torch.empty(gv.shape, dtype=torch.float32).pin_memory() for _ in range(2)] if gv is not None else None
    computed = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    handles = []
    if wl["adjoint"]:  # the dense path's gradient buffer
        ge = torch.empty_like(dist)

    def e2e_step(i):
        b = i & 1
        with torch.cuda.stream(sc):
            if i >= 2:
                sc.wait_event(copied[b])  # the copy-out of step i - 2 has left these buffers
            s_dev = soup_host.to(dev, non_blocking=True)
            f = sdf.sdf_build_features(s_dev, stream=sc)
            if use_list:
                sdf.sdf_narrow_band_list(f, grid, w, out=dists[b], band_list=bls[b], flags=sdf.FLAG_NO_SYNC,
                                         stream=sc)
                gvs[b].zero_()
                sdf.band_list_l2(f, grid, bls[b], dists[b], target, grad_vertices=gvs[b], stream=sc)
            else:
                sdf.sdf_narrow_band(f, grid, w, out=dists[b], winner=wins[b] if wins[b] is not None else False,
                                    flags=sched_flag | sdf.FLAG_NO_SYNC, stream=sc)
            if wl["adjoint"] and not use_list:
                sdf.band_l2_loss(dists[b], target, grad=ge, stream=sc)  # dL/dd of sum_band (d - 0.01)^2
                gvs[b].zero_()
                sdf.sdf_narrow_band_backward(f, grid, w, ge, winner=wins[b], grad_vertices=gvs[b], stream=sc)
                if shard:
                    slabs.all_reduce_sum(gvs[b])
            computed[b].record(sc)
        with torch.cuda.stream(sx):
            sx.wait_event(computed[b])
            dist_hosts[b].copy_(dists[b], non_blocking=True)
            if gv is not None:
                gv_hosts[b].copy_(gvs[b], non_blocking=True)
            copied[b].record(sx)
        handles.append(f)  # released after the timed loop (releasing synchronises the device)

    for i in range(2):  # fill the two-stage pipeline
        e2e_step(i)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(2, 2 + e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    for f in handles:
        f.status()  # every step's forward completed within its scratch and band list
        f.destroy()
    e2e = {"value": band_total * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(soup_np.nbytes),
           "d2h_bytes_per_step": int(dist.numel() * 4 + (gv.numel() * 4 if gv is not None else 0))}

    hbm, peak_kind = peaks()
    tile_avg_ms = tile_ms / max(1, tile_calls)
    npts = grid.nx * grid.ny * grid.nz
    # output bytes of the tile kernel: the field, and the band list (8 B per band point) or the
    # dense winners
    alg_bytes = 4 * npts + (8 * band_points if use_list else (4 * npts if win is not None else 0)) + rec_bytes
    achieved = alg_bytes / (tile_avg_ms / 1e3) / 1e9
    kname = ("k_cell_loop + k_decode_keys (the paper's schedule: region walk, global atomicMin, decode)"
             if args.schedule == "cell" else "k_tile (scan conversion + merge + dense write)")
    roofline = {"kernel": kname, "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": peak_kind,
                "traffic": tile_traffic(name, not args.grid and not shard and args.schedule == "tile" and use_list),
                "algorithmic_bytes": int(alg_bytes),
                "avg_ms": tile_avg_ms}
    rates = measured_rates(sdf, dev)
    # every (point, region) candidate is one 64-bit atomicMin: in shared memory in the tile kernel, in
    # global memory (8 B keys per grid point) in the paper's schedule
    roofline["atomic"] = atomic_roof(stats["candidates"], rates, "global" if args.schedule == "cell" else "shared",
                                     alg_bytes, hbm, tile_avg_ms)
    # the issue roof: warp instructions of the same ncu capture / the live duration
    instr = tile_traffic(name, not args.grid and not shard and args.schedule == "tile" and use_list,
                         "warp_instructions")
    if instr:
        roofline["issue"] = {"bound": "alu", "achieved": instr / (tile_avg_ms / 1e3), "peak": ISSUE_PEAK,
                             "unit": "warp instructions/s", "frac": instr / (tile_avg_ms / 1e3) / ISSUE_PEAK,
                             "warp_instructions": instr}

    # The sparse forward (a project addition, labelled as such): the same tile kernel writing only the
    # band list with distances (12 B per band point) and no dense field, so no +inf fill.  Its tile
    # kernel time and the roofline of its own bytes (list + feature records), and the issue roof.
    sparse = None
    if args.schedule == "tile" and not shard:
        sbl = sdf.BandList(band_points + band_points // 4 + 4096, device=dev)
        fs = sdf.sdf_build_features(soup)
        for _ in range(3):
            sdf.sdf_narrow_band_sparse(fs, grid, w, band_list=sbl)
        fs.timing(reset=True)
        s_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        for _ in range(s_steps):
            flush.fill_(1.0)
            sdf.sdf_narrow_band_sparse(fs, grid, w, band_list=sbl, flags=sdf.FLAG_TIMING | sdf.FLAG_NO_SYNC)
        torch.cuda.synchronize()
        fs.status()
        ts = fs.timing()
        s_tile = ts["tile"][0] / max(1, ts["tile"][1])
        s_fwd = (ts["bin"][0] + ts["tile"][0] + ts["fp64"][0]) / max(1, ts["tile"][1])
        s_bytes = 12 * band_points + rec_bytes
        sparse = {"what": "sdf_narrow_band_sparse: band list (index, winner) + distances, no dense field "
                          "(a project addition; the paper writes the dense array)",
                  "band_points_per_s": band_total / (s_fwd / 1e3), "fwd_device_ms": s_fwd, "tile_ms": s_tile,
                  "roofline": {"kernel": "k_tile (sparse)", "bound": "hbm", "algorithmic_bytes": int(s_bytes),
                               "achieved": s_bytes / (s_tile / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                               "frac": s_bytes / (s_tile / 1e3) / 1e9 / hbm, "peak_source": peak_kind}}
        fs.destroy()
        del sbl
    if rank != 0:
        return None
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(soup_np, N, w) if name != "c4" else cpu_baseline_sampled(soup_np, N, w, band_total)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, **step_stats(per.sum(axis=1)), "higher_is_better": True,
        "scaling": "strong" if shard else "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "triangles": int(soup_np.shape[0]), "grid": [N, N, N], "band_w": w,
                   "band_points": band_points, "l2": "flushed between timed steps (256 MiB write)",
                   "schedule": args.schedule,
                   "adjoint": ("loss and vertex gradient fused over the compact band list" if use_list else
                               "dense upstream gradient and winners") if wl["adjoint"] else None,
                   "parallelism": (f"z-slabs x{world}" if shard else "replicas") if world > 1 else "single GPU"},
        "build_ms": build_ms, "fwd_ms": fwd_ms, "adjoint_ms": adj_ms if wl["adjoint"] else None,
        "fwd_adjoint_ms": fwd_ms + adj_ms if wl["adjoint"] else None,
        "fwd_adjoint_over_fwd": (fwd_ms + adj_ms) / fwd_ms if wl["adjoint"] else None,
        "candidates_per_band_point": stats["candidates"] / max(1, stats["band_points"]),
        "fp64_points": stats["fp64_points"], "tile_region_pairs": stats["pairs"], "rows": stats["rows"],
        "rows_hit": stats["rows_hit"],
        "roofline": roofline, "rates": measured_rates(sdf, dev), "sparse": sparse, "cpu_baseline": cpu,
        "clocks": dict(clk.summary(), per_step=step_clk.summary()), "e2e": e2e,
        "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
    }
    return line


if __name__ == "__main__":
    main()
