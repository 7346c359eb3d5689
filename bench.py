#!/usr/bin/env python
"""Throughput of the whole Lagrangian step of the IP + MLS-IBM method on GB300.

One step = internal forces of the four potentials, MLS interpolation at every
face centroid with the direct-forcing marker force, probe gradient and
traction, node update, and spreading onto the staggered grid (with the
previous step's footprint cleared), as three kernel launches of ibm_step.

Metric: Lagrangian node-steps/s (vertices x steps / device time).  Default
workload: 1000 icosphere level-3 drops (642 nodes, 1280 faces each), radii
U[0.015, 0.03], Poisson-disk placed in the unit periodic box, 512^3 MAC grid,
frozen velocity = 32 random divergence-free Fourier modes (amplitude 1,
wavenumbers 1-8), k_s ~ U[0.5, 2], k_b ~ U[0.005, 0.02] per body.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun every rank runs its own independent replica (bodies do not
interact), so the job scales weakly with no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1612_03399_gb300 import workloads as W  # noqa: E402

METRIC = "Lagrangian node-steps/s (force+MLS interp+advance+spread), % HBM roofline"
UNIT = "node-steps/s"

WORKLOADS = {
    "drops1000": (lambda seed: W.batched_drops(1000, 3, 512, seed=seed),
                  "1000 icosphere-L3 drops (642 nodes, 1280 faces each), radii U[0.015,0.03], "
                  "Poisson-disk placed, 512^3 MAC grid, 32-mode divergence-free Fourier velocity "
                  "(amplitude 1, |k| 1-8), k_s~U[0.5,2], k_b~U[0.005,0.02]"),
    "uneven4096": (lambda seed: W.uneven_bodies(4096, 768, seed=seed),
                   "4096 closed bodies, icosphere levels 2/3/4/5 w.p. 0.4/0.3/0.2/0.1, radius "
                   "0.005*2^(L-2), ellipsoid stretch U[1,1.5], 768^3 MAC grid, Fourier velocity"),
    "drop64": (lambda seed: W.single_drop(3, 64),
               "one icosphere-L3 drop r=0.25 in frozen shear u=y-0.5, 64^3 grid"),
    "membranes": (lambda seed: W.membranes(8, 512, seed=seed),
                  "closed ellipsoidal membrane (655362 nodes) + two clamped leaflet sheets "
                  "(~100k faces each), 512^3 grid, Fourier velocity amplitude 2"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="drops1000", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--patch", type=int, default=0)
    ap.add_argument("--marker-patch", type=int, default=0, choices=[0, 128, 256],
                    help="faces per marker-kernel block; 0: picked by measurement")
    ap.add_argument("--spread-variant", type=int, default=0, choices=[0, 1, 2],
                    help="1: spread inside the marker kernel (atomic flush); 2: tile-owned "
                         "spread kernels; 0: the library's default")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the other spread variant on the headline workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the uneven-bodies and membrane workloads")
    ap.add_argument("--integrator", default="symplectic", choices=["symplectic", "hamming"],
                    help="hamming: the strong-coupling predictor-corrector step (ibm_step_pc), "
                         "steps launched one by one")
    ap.add_argument("--bodies", type=int, default=0,
                    help="profiling only: fewer drops on the same grid (drops1000 workload)")
    ap.add_argument("--coupled", action="store_true",
                    help="the coupled step (ibm_flow_step: RK3 Navier-Stokes with the IBM "
                         "forcing per substep, then the body update) on the workload's bodies "
                         "and grid, dt at CFL 0.5 of the initial field, nu = mu = 0.01")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (independent replicas; barrier + max over ranks)
# ---------------------------------------------------------------------------

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(ws, val, device):
    if ws == 1:
        return val
    import torch.distributed as dist
    t = torch.tensor([val], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(ws, val, device):
    if ws == 1:
        return val
    import torch.distributed as dist
    t = torch.tensor([val], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(ws, units_local, steps, ms_local, device):
    """Whole-job throughput of independent replicas: the units every rank
    processed (summed over ranks) times steps, over the slowest rank's time.
    Returns (units per second, max ms)."""
    t_max = reduce_max(ws, ms_local, device)
    units = reduce_sum(ws, float(units_local), device)
    return units * steps / (t_max * 1e-3), t_max


# ---------------------------------------------------------------------------
# algorithmic byte model of the two main kernels
# ---------------------------------------------------------------------------

def touched_nodes(wl, x, ctx, device):
    """Unique grid nodes per velocity component touched by the centroid
    stencils and by the centroid-or-probe stencils (3x3x3 nearest-node
    supports on the MAC lattices)."""
    n = wl.grid.n
    h = torch.tensor(wl.grid.h, dtype=torch.float64, device=device)
    origins = torch.tensor(np.concatenate([np.repeat(b.origin[None], len(b.tri), 0)
                                           for b in wl.bodies]), device=device)
    tri = torch.tensor(np.concatenate([b.tri + int(ctx.v_off[i]) for i, b in enumerate(wl.bodies)]),
                       dtype=torch.long, device=device)
    closed = torch.tensor(np.concatenate([np.full(len(b.tri), b.closed) for b in wl.bodies]),
                          device=device)
    X = x.double().T
    xa, xb, xc = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    c = (xa + xb + xc) / 3 + origins
    N = torch.cross(xb - xa, xc - xa, dim=1)
    nrm = N / N.norm(dim=1, keepdim=True)
    ph = float(h.mean())
    s = torch.tensor([-1, 0, 1], device=device)
    offs = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))
    res_c, res_all = [], []
    for comp in range(3):
        mark_c = torch.zeros(n[0] * n[1] * n[2], dtype=torch.bool, device=device)
        mark_a = torch.zeros_like(mark_c)
        for which, P in enumerate([c, c + ph * nrm, (c - ph * nrm)[~closed]]):
            for chunk in torch.split(P, 1 << 18):
                t = chunk / h - torch.tensor(offs[comp], dtype=torch.float64, device=device)
                ic = torch.floor(t + 0.5).long()
                ix = torch.remainder(ic[:, 0:1] + s, n[0])
                iy = torch.remainder(ic[:, 1:2] + s, n[1])
                iz = torch.remainder(ic[:, 2:3] + s, n[2])
                flat = ((iz[:, :, None, None] * n[1] + iy[:, None, :, None]) * n[0]
                        + ix[:, None, None, :]).reshape(-1)
                mark_a[flat] = True
                if which == 0:
                    mark_c[flat] = True
        res_c.append(int(mark_c.sum()))
        res_all.append(int(mark_a.sum()))
    return res_c, res_all


def byte_model(wl, ctx, x, device):
    """Algorithmic bytes per launch of the step's kernels, counted as the
    byte model of the hot path states: state x, v read and written (48 B per
    vertex), rest data (l0, theta0 per edge, A0 per face), and on the grid
    4 B per component and unique node read by the centroid and probe
    stencils plus 4 B per component and unique node written by the spread.
    `marker_fused` is the marker kernel of spread variant 1 (interpolation,
    traction and spread), `marker` that of variant 2 (interpolation and
    traction; its per-marker outputs, about 28 B, count as written), `spread`
    the tile-owned spread (those outputs read, the nodes written).  The
    `_rmw` figures count the spread's nodes as read and written (8 B), what
    float atomics into the fields move."""
    nv = sum(len(b.rest) for b in wl.bodies)
    nf = sum(len(b.tri) for b in wl.bodies)
    ne = ctx.E
    centre_nodes, all_nodes = touched_nodes(wl, x, ctx, device)
    grid_in = 4 * sum(all_nodes)
    grid_out = 4 * sum(centre_nodes)
    state_in = nv * 24                      # x, v gathered (each vertex once)
    out = {
        "marker_fused": state_in + nf * 12 + grid_in + grid_out,
        "marker_fused_rmw": state_in + nf * 12 + grid_in + 2 * grid_out,
        "marker": state_in + nf * 28 + grid_in,
        "spread": nf * 28 + grid_out,
        "force": (nv * (12 + 12 + 24 + 1)   # x, v read; x', v' written; clamp flag
                  + ne * 12                 # l0, (cos, sin) theta0
                  + nf * (4 + 12)),         # A0_f, F_ext read
        # the coupled step's forcing launch (interpolate and spread at the
        # centroids, no probe): x, v gathered, centroid velocity nodes read,
        # force nodes read-modify-written
        "forcing": state_in + 4 * sum(centre_nodes) + 8 * sum(centre_nodes),
        "step": nv * 48 + ne * 12 + nf * 4 + grid_in + grid_out,
        "nodes_centre": centre_nodes, "nodes_all": all_nodes,
    }
    return out


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def ncu_traffic(kernel_key):
    """DRAM bytes per launch of `kernel_key` from the committed ncu summary,
    or None when the kernel's sources changed since those counters were
    taken (each kernel carries the digest of the files it is built from)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        from paper_1612_03399_gb300 import build as B
        d = json.load(open(p))
        if d.get("digests", {}).get(kernel_key) != B.kernel_digest(kernel_key):
            return None
        return d.get("kernels", {}).get(kernel_key)
    except Exception:
        return None


def ncu_instructions(kernel_key):
    """Warp instructions per unit (marker, or own vertex for the force
    kernel) of `kernel_key` from the committed ncu summary (the drop
    workload's count), or None when the kernel's sources changed since it
    was taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        from paper_1612_03399_gb300 import build as B
        d = json.load(open(p))
        if d.get("digests", {}).get(kernel_key) != B.kernel_digest(kernel_key):
            return None
        return d.get("instructions", {}).get(kernel_key)
    except Exception:
        return None


def issue_roofline(kernel_key, units, ms, clk, device_index):
    """The kernel against its compute-side bound, instruction issue: warp
    instructions per launch (ncu's count per unit -- marker, or own vertex
    for the force kernel -- x the units of a launch) / its mean duration,
    against 4 schedulers per SM issuing one warp instruction per clock each,
    at the SM clock sampled during the timed region."""
    ipf = ncu_instructions(kernel_key)
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
    if not ipf or not mhz:
        return None
    n_sm = torch.cuda.get_device_properties(device_index).multi_processor_count
    peak = n_sm * 4 * mhz * 1e6
    achieved = ipf * units / (ms * 1e-3)
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp-instr/s",
            "frac": achieved / peak, "inst_per_unit": ipf, "sm_mhz": mhz, "sms": n_sm}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class _NvmlSampler:
    """SM clock and throttle reasons read through NVML (libnvidia-ml, read-only
    queries) every millisecond from a background thread, so that even a
    timed region of a few milliseconds gets several samples."""
    # clocks event reason bits (nvml.h)
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, index):
        import ctypes
        import threading
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(self.lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        self.ctypes, self.threading = ctypes, threading
        mx = ctypes.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx))
        self.max_mhz = float(mx.value)
        self.samples = []
        self.stop_flag = False
        self.thread = None

    def read(self):
        c = self.ctypes
        mhz, rs = c.c_uint(), c.c_ulonglong()
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, c.byref(mhz))
        self.reasons_fn(self.h, c.byref(rs))
        return float(mhz.value), int(rs.value)

    def start(self):
        import time as _t
        self.read()

        def loop():
            while not self.stop_flag:
                self.samples.append(self.read())
                _t.sleep(0.001)
        self.thread = self.threading.Thread(target=loop, daemon=True)
        self.thread.start()
        while not self.samples:
            _t.sleep(0.0005)

    def stop(self):
        self.stop_flag = True
        self.thread.join(1.0)
        sm = [m for m, _ in self.samples]
        reasons = sorted(n for n, b in self.BITS.items() if any(r & b for _, r in self.samples))
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "source": "nvml"}


class Clocks:
    """Clocks and throttle reasons during a timed region: NVML when the
    driver's library is there, else nvidia-smi sampling every 10 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.skip = 0
        self.nvml = None

    def start(self):
        try:
            self.nvml = _NvmlSampler(self.index)
            self.nvml.start()
            return
        except Exception:
            self.nvml = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "10"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler delivers readings
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
            self.skip = sum(1 for line in open(self.path) if line.strip())
        except Exception:
            self.proc = None

    def stop(self):
        if self.nvml is not None:
            try:
                return self.nvml.stop()
            except Exception:
                return None
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        # readings taken before the timed region started are dropped, but one
        # is kept when the region was shorter than the sampling interval
        rows = rows[self.skip:] or rows[-1:]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_rate(wl, n_bodies, steps, fields_cpu=None):
    """Time the FP64 oracle, as it stands, on the first n_bodies bodies of the
    workload (same grid and field) for `steps` steps; node-steps/s."""
    from oracle import ibm_oracle as O
    sub = wl.bodies[:n_bodies]
    ob = [O.Body(b.rest, b.tri, b.origin, closed=b.closed, clamped=b.clamped, ks=b.ks, kb=b.kb,
                 ka=b.ka, kA=b.kA, kv=b.kv, mass=b.mass) for b in sub]
    prm = O.Params(wl.grid.n, wl.grid.L, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    if fields_cpu is None:
        fields_cpu = W.sample_field(wl.field, wl.grid, device="cpu", dtype=torch.float64)
    xs = [torch.tensor(b.rest) for b in sub]
    vs = [torch.zeros_like(x) for x in xs]
    nodes = sum(len(b.rest) for b in sub)
    t0 = time.perf_counter()
    for _ in range(steps):
        out = O.step(ob, xs, vs, fields_cpu, prm)
        xs = [t.detach() for t in out["x_next"]]
        vs = [t.detach() for t in out["v_next"]]
    dt = time.perf_counter() - t0
    return nodes * steps / dt, dt, nodes


def run_reference(args, ws, rank):
    if rank != 0:
        return
    make, descr = WORKLOADS[args.workload]
    wl = make(1)
    fields = W.sample_field(wl.field, wl.grid, device="cpu", dtype=torch.float64)
    # warm-up (allocator, threads), which also sizes the sample: up to 8
    # bodies per step, about a minute of oracle work over all the steps
    _, t1, _ = oracle_sample_rate(wl, 1, 1, fields)
    steps = max(1, args.steps)
    nb = max(1, min(len(wl.bodies), 8, int(60.0 / (t1 * steps))))
    rate, secs, nodes = oracle_sample_rate(wl, nb, steps, fields)
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": descr, "sample_bodies": nb},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{nb} bodies ({nodes} nodes) of the workload, {args.steps} steps"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GB300 arm
# ---------------------------------------------------------------------------

PHASES = ["pre", "marker", "spread", "force"]


def time_steps(ctx, wl, fields, f, state, n_steps, flush, stream, clocks=None):
    """Time n_steps (rounded up to even) of the whole step as replays of a
    2-step CUDA graph, L2 flushed before every replay; CUDA events on the
    library's stream.  Returns (total ms, steps, clock record)."""
    xa, va, xb, vb = state
    graph = ctx.graph(xa, va, xb, vb, fields, f, n_steps=2)
    graph.launch()
    torch.cuda.synchronize()
    n_rep = (n_steps + 1) // 2
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks is not None:
        clocks.start()
    total = 0.0
    for _ in range(n_rep):
        flush.zero_()
        ev0.record(stream)
        graph.launch()
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    ctx.check_device_error()
    graph.close()
    return total, 2 * n_rep, clk


def phase_steps(ctx, wl, fields, f, state, n_steps, flush):
    """The same steps launched one by one with CUDA events between the
    kernels: mean (set-up or clear, marker, spread, force) ms and the mean
    step ms."""
    xa, va, xb, vb = state
    stream = torch.cuda.current_stream(xa.device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.set_phase_timing(True)
    phases, step_ms = [], 0.0
    for _ in range(n_steps):
        flush.zero_()
        ev0.record(stream)
        ctx.step(xa, va, fields, xb, vb, f)
        ev1.record(stream)
        ev1.synchronize()
        step_ms += ev0.elapsed_time(ev1)
        phases.append(ctx.phase_times())
        xa, va, xb, vb = xb, vb, xa, va
    ctx.set_phase_timing(False)
    return np.array(phases).mean(0), step_ms / n_steps, (xa, va, xb, vb)


def kernel_roofline(variant, mean_ph, bm, peak, peak_kind):
    """Per-kernel achieved GB/s (algorithmic bytes / mean event time) and the
    dominant kernel's roofline record."""
    keys = ({"marker": "marker_fused", "force": "force"} if variant == 1 else
            {"marker": "marker", "spread": "spread", "force": "force"})
    per = {}
    for k, n in enumerate(PHASES):
        if n not in keys or mean_ph[k] <= 0:
            continue
        b = bm[keys[n]]
        per[n] = {"algorithmic_bytes": b, "ms": float(mean_ph[k]),
                  "achieved_gbs": b / (mean_ph[k] * 1e-3) / 1e9,
                  "frac": b / (mean_ph[k] * 1e-3) / 1e9 / peak}
    dom = max(per, key=lambda n: per[n]["ms"])
    rec = {"bound": "hbm", "kernel": dom, "achieved": per[dom]["achieved_gbs"], "peak": peak,
           "peak_kind": peak_kind, "unit": "GB/s", "frac": per[dom]["frac"],
           "algorithmic_bytes": per[dom]["algorithmic_bytes"]}
    if variant == 1 and dom == "marker":
        rmw = bm["marker_fused_rmw"] / (per[dom]["ms"] * 1e-3) / 1e9
        rec["frac_rmw"] = rmw / peak
    return rec, per


def extra_workload(args, name, variant, device, flush, peak, peak_kind, patch):
    """One of the larger configurations: whole-step throughput (graph
    replays, L2 flushed), phases one by one, dominant kernel's roofline."""
    from paper_1612_03399_gb300 import _lib
    make, descr = WORKLOADS[name]
    wl = make(1)
    fields = W.sample_field(wl.field, wl.grid, device=device, dtype=torch.float32)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha, patch_size=patch,
                       device=device.index, spread_variant=variant,
                       marker_patch=getattr(args, "marker_patch_used", 0))
    stream = torch.cuda.current_stream(device)
    nx, ny, nz = wl.grid.n
    f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=device) for _ in range(3))
    xa, va = ctx.init_state()
    xb, vb = torch.empty_like(xa), torch.empty_like(va)
    bm = byte_model(wl, ctx, xa, device)
    for _ in range(3):
        ctx.step(xa, va, fields, xb, vb, f)
        xa, va, xb, vb = xb, vb, xa, va
    mean_ph, _, st = phase_steps(ctx, wl, fields, f, (xa, va, xb, vb), 6, flush)
    n = max(6, min(args.steps, 20))
    total, steps, clk = time_steps(ctx, wl, fields, f, st, n, flush, stream, Clocks(device.index))
    roof, per = kernel_roofline(ctx.spread_variant, mean_ph, bm, peak, peak_kind)
    out = {"workload": descr, "bodies": ctx.B, "vertices": ctx.V, "faces": ctx.F,
           "grid": list(wl.grid.n), "spread_variant": ctx.spread_variant,
           "ms_per_step": total / steps, "value": ctx.V * steps / (total * 1e-3), "unit": UNIT,
           "steps": steps, "phases_ms": dict(zip(PHASES, map(float, mean_ph))),
           "roofline": roof, "kernels": per,
           "step_algorithmic_gbs": bm["step"] / (total / steps * 1e-3) / 1e9, "clocks": clk}
    ctx.close()
    del fields, f, xa, va, xb, vb
    torch.cuda.empty_cache()
    return out


def differentiation_workload(device):
    """The differentiation configuration: 256 icosphere-L4 drops in linear
    shear on 256^3, 50 steps with a checkpoint every 10, loss sum over drops
    of (D - D*)^2; one calibration iteration = 50 forward, 50 recomputed and
    50 adjoint steps and the Taylor-deformation adjoint (torch.autograd over
    ibm_step / ibm_backward / ibm_taylor_backward).  Wall time per iteration
    after a first one."""
    from paper_1612_03399_gb300.autograd import Simulation
    from paper_1612_03399_gb300.calibrate import calibrate
    wl = W.shear_drops(256, 4, 256)
    sim = Simulation(wl.bodies, wl.grid, wl.field, dt=1e-3, mu=1.0, device=device.index)
    x0, v0 = sim.ctx.init_state()
    n_steps = 50
    _, hist = calibrate(sim, x0, v0, wl.notes["D_target"], n_steps, 10, iters=4, lr=0.1)
    secs = [h["seconds"] for h in hist[1:]]
    per = statistics.median(secs)
    out = {"workload": "256 icosphere-L4 drops (2562 nodes each), r = 0.04, linear shear, 256^3 "
                       "grid; 50 steps, checkpoint every 10; loss sum (D - D*)^2, D* ~ U[0.05, 0.3]",
           "bodies": sim.ctx.B, "vertices": sim.ctx.V, "seconds_per_iteration": per,
           "forward_node_steps_per_s_through_fwd_bwd": sim.ctx.V * n_steps / per,
           "losses": [h["loss"] for h in hist]}
    sim.ctx.close()
    return out


def run_gb300(args, ws, rank, local):
    from paper_1612_03399_gb300 import _lib
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    make, descr = WORKLOADS[args.workload]
    if args.bodies and args.workload == "drops1000":
        make = lambda seed: W.batched_drops(args.bodies, 3, 512, seed=seed)  # noqa: E731
        descr = descr.replace("1000 icosphere", f"{args.bodies} icosphere")
    wl = make(1 + rank)
    fields = W.sample_field(wl.field, wl.grid, device=device, dtype=torch.float32)
    tuned = None
    patch = args.patch
    if patch == 0:
        # force-kernel patch size picked by measurement on this workload
        from paper_1612_03399_gb300.autotune import autotune_patch_size
        patch, tuned = autotune_patch_size(wl.bodies, wl.grid, fields, dt=wl.dt, mu=wl.mu,
                                           alpha=wl.alpha, device=local)
    mtuned = None
    mpatch = args.marker_patch
    if mpatch == 0:
        # marker-kernel patch size (faces per block) picked by measurement too
        from paper_1612_03399_gb300.autotune import autotune_marker_patch
        mpatch, mtuned = autotune_marker_patch(wl.bodies, wl.grid, fields, dt=wl.dt, mu=wl.mu,
                                               alpha=wl.alpha, device=local, patch_size=patch)
    args.marker_patch_used = mpatch
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                       patch_size=patch, device=local, spread_variant=args.spread_variant,
                       marker_patch=mpatch)
    variant = ctx.spread_variant
    stream = torch.cuda.current_stream(device)
    nx, ny, nz = wl.grid.n
    f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=device) for _ in range(3))
    xa, va = ctx.init_state()
    xb, vb = torch.empty_like(xa), torch.empty_like(va)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)   # > L2 (129 MB)
    if args.integrator == "hamming":
        return run_hamming(args, ws, rank, ctx, wl, descr, fields, f, xa, va, xb, vb, flush,
                           device, patch)
    bytes_model = byte_model(wl, ctx, xa, device) if rank == 0 else None
    for _ in range(max(args.warmup, 3)):
        ctx.step(xa, va, fields, xb, vb, f)
        xa, va, xb, vb = xb, vb, xa, va
    ctx.check_device_error()
    torch.cuda.synchronize()
    # per-kernel phase times (CUDA events between the step's launches) for the
    # roofline: the same steps launched one by one
    mean_ph, step_ms, (xa, va, xb, vb) = phase_steps(ctx, wl, fields, f, (xa, va, xb, vb),
                                                     args.steps, flush)
    # the timed steps: the whole step captured in a CUDA graph, two steps per
    # replay (ping-pong state), L2 flushed before every replay
    barrier(ws)
    torch.cuda.synchronize()
    total_ms, n_steps, clk = time_steps(ctx, wl, fields, f, (xa, va, xb, vb), args.steps, flush,
                                        stream, Clocks(local))
    barrier(ws)
    value, t_max = job_rate(ws, ctx.V, n_steps, total_ms, device)
    value_steps, _ = job_rate(ws, ctx.V, 1, step_ms, device)

    # end to end through the public API with host buffers (pinned): one
    # ibm_step_host per step, which copies x, v in (beside the footprint
    # clear) and has the force kernel write x', v' into host memory
    e2e = None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if not args.no_e2e:
        xh = xa.cpu().pin_memory()
        vh = va.cpu().pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        vo = torch.empty_like(vh).pin_memory()
        ctx.step_host(xh, vh, fields, xo, vo, f)   # first call: the context's copies
        xh, xo = xo, xh
        vh, vo = vo, vh
        barrier(ws)
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            ctx.step_host(xh, vh, fields, xo, vo, f)
            ev1.record(stream)
            ev1.synchronize()
            e2e_ms += ev0.elapsed_time(ev1)
            xh, xo = xo, xh
            vh, vo = vo, vh
        e2e_value, _ = job_rate(ws, ctx.V, args.steps, e2e_ms, device)
        nbytes = 2 * 3 * ctx.V * 4
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    counters = ctx.counters()
    ctx.close()
    if rank != 0:
        return
    peak, peak_kind = hbm_peak()
    roof, per = kernel_roofline(variant, mean_ph, bytes_model, peak, peak_kind)
    # counters are recorded per marker patch size (256: "marker", 128: "marker_p128")
    rkey = roof["kernel"] if roof["kernel"] != "marker" or mpatch == 256 else f"marker_p{mpatch}"
    roof["traffic"] = ncu_traffic(rkey)
    if variant == 1 and args.workload == "drops1000" and roof["kernel"] == "marker":
        # per-marker instruction count measured on this workload's drops
        roof["issue"] = issue_roofline(rkey, int(sum(len(b.tri) for b in wl.bodies)),
                                       per["marker"]["ms"], clk, local)
        # the force kernel against the same bound (instructions per own vertex)
        if "force" in per:
            per["force"]["issue"] = issue_roofline("force", int(ctx.V), per["force"]["ms"], clk,
                                                   local)
    launches = 3 if variant == 1 else 6
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": n_steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_max / n_steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": descr, "bodies": int(sum(1 for _ in wl.bodies)),
                   "vertices": int(sum(len(b.rest) for b in wl.bodies)),
                   "faces": int(sum(len(b.tri) for b in wl.bodies)),
                   "grid": list(wl.grid.n), "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"{ws} independent replica(s)", "patch_size": patch,
                   "marker_patch": mpatch, "autotune_marker_ms": mtuned,
                   "spread_variant": variant, "autotune_force_ms": tuned},
        "roofline": roof,
        "phases_ms": dict(zip(PHASES, map(float, mean_ph))),
        "kernels": per,
        "step_algorithmic_gbs": bytes_model["step"] / (t_max / n_steps * 1e-3) / 1e9,
        "gpu_launches": launches * n_steps,
        "timing": "CUDA graph of 2 captured steps per replay; value_no_graph times the same "
                  "steps launched one by one (with phase events)",
        "value_no_graph": value_steps,
        "counters": counters,
        "e2e": e2e,
        "clocks": clk,
    }
    if not args.no_variants and ws == 1 and args.workload == "drops1000" and not args.bodies:
        # the other spread variant on the same workload, for the choice of default
        other = 1 if variant == 2 else 2
        ctx2 = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                            patch_size=patch, device=local, spread_variant=other,
                            marker_patch=mpatch)
        xa, va = ctx2.init_state()
        xb, vb = torch.empty_like(xa), torch.empty_like(va)
        for t in f:
            t.zero_()
        for _ in range(3):
            ctx2.step(xa, va, fields, xb, vb, f)
            xa, va, xb, vb = xb, vb, xa, va
        ph2, _, st = phase_steps(ctx2, wl, fields, f, (xa, va, xb, vb), 10, flush)
        tot2, n2, _ = time_steps(ctx2, wl, fields, f, st, max(10, args.steps), flush, stream)
        roof2, per2 = kernel_roofline(other, ph2, bytes_model, peak, peak_kind)
        line["other_variant"] = {"spread_variant": other, "ms_per_step": tot2 / n2,
                                 "value": ctx2.V * n2 / (tot2 * 1e-3),
                                 "phases_ms": dict(zip(PHASES, map(float, ph2))),
                                 "roofline": roof2}
        ctx2.close()
    if not args.no_variants and ws == 1 and args.workload == "drops1000" and not args.bodies:
        # what the float32 closed form of the MLS moment solve saves: the
        # interpolation and probe traction of every marker, closed form in
        # float32 against the general 4x4 solve and geometry in float64
        ctx3 = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                            patch_size=patch, device=local, marker_patch=mpatch)
        xa, va = ctx3.init_state()
        va.uniform_(-0.1, 0.1)
        times = {}
        for name, fn in (("fp32_closed_form", ctx3.interpolate), ("fp64_general", ctx3.interpolate_fp64)):
            fn(xa, va, fields)
            torch.cuda.synchronize()
            tot = 0.0
            for _ in range(3):
                flush.zero_()
                ev0.record(stream)
                fn(xa, va, fields)
                ev1.record(stream)
                ev1.synchronize()
                tot += ev0.elapsed_time(ev1)
            times[name] = tot / 3
        ctx3.check_device_error()
        ctx3.close()
        line["mls_precision"] = {"interpolate_ms": times,
                                 "fp64_over_fp32": times["fp64_general"] / times["fp32_closed_form"],
                                 "what": "U, F_marker and the probe traction of every marker "
                                         "(ibm_interpolate vs ibm_interpolate_fp64)"}
    if not args.no_extra and ws == 1 and args.workload == "drops1000" and not args.bodies:
        del fields, f
        torch.cuda.empty_cache()
        line["extra_workloads"] = {
            name: extra_workload(args, name, variant, device, flush, peak, peak_kind, patch)
            for name in ("uneven4096", "membranes")}
        line["extra_workloads"]["differentiation"] = differentiation_workload(device)
        fields = None
    if not args.no_cpu_baseline and ws == 1:
        if fields is None:
            fields = W.sample_field(wl.field, wl.grid, device=device, dtype=torch.float32)
        fields_cpu = tuple(t.double().cpu() for t in fields)
        oracle_sample_rate(wl, 1, 1, fields_cpu)
        nb = 16
        rate, secs, nodes = oracle_sample_rate(wl, nb, 2, fields_cpu)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": torch.get_num_threads(),
                                "kind": "oracle",
                                "sample": f"{nb} of the {len(wl.bodies)} bodies ({nodes} nodes) on "
                                          f"the full grid and field, 2 steps, {secs:.1f} s"}
    print(json.dumps(line), flush=True)


def run_hamming(args, ws, rank, ctx, wl, descr, fields, f, xa, va, xb, vb, flush, device,
                patch):
    """Throughput of the strong-coupling step (ibm_step_pc): Hamming's
    predictor-corrector, two acceleration evaluations per step, after the
    three Runge-Kutta start-up steps; steps launched one by one."""
    stream = torch.cuda.current_stream(device)
    ctx.pc_reset()
    for _ in range(3 + max(args.warmup, 3)):
        ctx.step_pc(xa, va, fields, xb, vb, f)
        xa, va, xb, vb = xb, vb, xa, va
    ctx.check_device_error()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(device.index)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        ctx.step_pc(xa, va, fields, xb, vb, f)
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
        xa, va, xb, vb = xb, vb, xa, va
    clk = clocks.stop()
    ctx.check_device_error()
    barrier(ws)
    value, t_max = job_rate(ws, ctx.V, args.steps, total, device)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": descr, "integrator": "Hamming predictor-corrector (ibm_step_pc)",
                   "bodies": ctx.B, "vertices": ctx.V, "grid": list(wl.grid.n),
                   "l2": "flushed between timed steps (256 MiB write)", "patch_size": patch},
        # per step: clear, marker, force (acceleration), predictor, marker, force, corrector
        "gpu_launches": 7 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the coupled step (flow solved)
# ---------------------------------------------------------------------------

COUPLED_NU, COUPLED_CFL = 1e-2, 0.5


def cfl_dt(fields, h, cfl):
    """Time step with sum_d max|u_d| dt / h_d = cfl: the explicit RK3
    advection is stable for centred differences up to sqrt(3)."""
    rate = sum(float(f.abs().max()) / hd for f, hd in zip(fields, h))
    return cfl / rate


def flow_bytes(n, widths):
    """Algorithmic bytes per time step of the flow solver's own kernels
    (float32 fields of N cells, spectra of NC = nz ny (nx/2+1) complex
    values), summed over the three substeps: what each kernel must read and
    write once.  `widths` are the substeps' viscous-solve widths (-1: Fourier
    path); the u* update moves the same bytes on both paths (R or du read,
    u read and written) and is named for the kernel that ran it."""
    N = n[0] * n[1] * n[2]
    NC = n[2] * n[1] * (n[0] // 2 + 1)
    n_fourier = sum(1 for w in widths if w < 0)
    upd = {0: "cn_solve", 3: "add"}.get(n_fourier, "update")
    out = {
        # u, v, w, p read; H and R (3 each) written; H_prev (3) read in substeps 1, 2
        "rhs": 4 * N * (3 * (4 + 6) + 2 * 3),
        upd: 3 * 4 * N * 9,                   # R or du, u read, u written (3 components)
        "div": 3 * 4 * N * 7,                 # u*, f read (3 + 3), divergence written
        "poisson_scale": 3 * NC * 8 * 2,
        "project": 3 * 4 * N * 12,            # u*, f, phi, p read; u, p written
    }
    if n_fourier:
        out["cn_scale"] = n_fourier * 3 * NC * 8 * 2   # three spectra read and written
    return out


def run_coupled(args, ws, rank, local):
    from paper_1612_03399_gb300 import _lib
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    make, descr = WORKLOADS[args.workload]
    if args.workload == "drops1000":
        # the direct forcing needs faces no larger than about two grid cells
        # (its per-marker gain is about A_l/h^2 with the narrow MLS kernel);
        # the level-3 drops have faces up to 2.2 h^2 on 512^3, 0.6 h^2 on 256^3
        make = lambda seed: W.batched_drops(1000, 3, 256, seed=seed)  # noqa: E731
        descr = descr.replace("512^3", "256^3")
    wl = make(1 + rank)
    fields = W.sample_field(wl.field, wl.grid, device=device, dtype=torch.float32)
    dt = cfl_dt(fields, wl.grid.h, COUPLED_CFL)
    hm = sum(wl.grid.h) / 3
    max_face_h2 = max(float(np.linalg.norm(np.cross(b.rest[b.tri[:, 1]] - b.rest[b.tri[:, 0]],
                                                     b.rest[b.tri[:, 2]] - b.rest[b.tri[:, 0]]),
                                            axis=1).max()) / 2 for b in wl.bodies) / hm ** 2
    ctx = _lib.Context(wl.bodies, wl.grid, dt=dt, mu=COUPLED_NU, alpha=wl.alpha,
                       patch_size=args.patch if args.patch else 256, device=local,
                       marker_patch=args.marker_patch)
    flow = _lib.Flow(wl.grid, nu=COUPLED_NU, dt=dt, device=local)
    stream = torch.cuda.current_stream(device)
    u = tuple(t.clone() for t in fields)
    p = torch.zeros_like(u[0])
    f = tuple(torch.zeros_like(u[0]) for _ in range(3))
    xa, va = ctx.init_state()
    xb, vb = torch.empty_like(xa), torch.empty_like(va)
    bytes_model = byte_model(wl, ctx, xa, device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def step():
        nonlocal xa, va, xb, vb
        flow.step(u, p, ctx=ctx, x=xa, v=va, x_out=xb, v_out=vb, f=f)
        xa, va, xb, vb = xb, vb, xa, va

    for _ in range(max(args.warmup, 3)):
        step()
    ctx.check_device_error()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ctx.check_device_error()
    barrier(ws)
    value, t_max = job_rate(ws, ctx.V, args.steps, total, device)
    ncell = wl.grid.n[0] * wl.grid.n[1] * wl.grid.n[2]
    cells, _ = job_rate(ws, ncell, args.steps, total, device)
    # phases: the same steps with CUDA events between the kernels
    flow.set_phase_timing(True)
    phases = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        step()
        phases.append(flow.phase_times())
    flow.set_phase_timing(False)
    ph = {k: float(np.mean([q[k] for q in phases])) for k in phases[0]}
    e2e = None
    if not args.no_e2e:
        xh, vh = xa.cpu().pin_memory(), va.cpu().pin_memory()
        xo, vo = torch.empty_like(xh).pin_memory(), torch.empty_like(vh).pin_memory()
        barrier(ws)
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            xa.copy_(xh, non_blocking=True)
            va.copy_(vh, non_blocking=True)
            flow.step(u, p, ctx=ctx, x=xa, v=va, x_out=xb, v_out=vb, f=f)
            xo.copy_(xb, non_blocking=True)
            vo.copy_(vb, non_blocking=True)
            ev1.record(stream)
            ev1.synchronize()
            e2e_ms += ev0.elapsed_time(ev1)
            xh, xo = xo, xh
            vh, vo = vo, vh
        e2e_value, _ = job_rate(ws, ctx.V, args.steps, e2e_ms, device)
        nbytes = 2 * 3 * ctx.V * 4
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes,
               "note": "body state (x, v) copied in and out every step; the flow fields are "
                       "the device-resident Eulerian state"}
    ctx.check_device_error()
    if rank != 0:
        return
    widths = flow.solve_widths()
    fb = flow_bytes(wl.grid.n, widths)
    # the forcing launches (marker kernel, interpolate and spread), three per
    # step; their phase also holds the zeroing of the three force fields, so
    # the rate derived from it is a lower bound
    fb["forcing"] = 3 * bytes_model["forcing"]
    ph_k = dict(ph, forcing=ph["ibm_forcing"], cn_solve=ph["update"], add=ph["update"])
    own = {k: ph_k[k] for k in fb}
    dom = max(own, key=own.get)
    peak, peak_kind = hbm_peak()
    achieved = fb[dom] / (ph_k[dom] * 1e-3) / 1e9
    fft_ms = sum(ph[k] for k in ("fft_fwd3", "fft_inv3", "fft_fwd1", "fft_inv1"))
    step_ms = sum(ph.values())
    line = {
        "metric": "Lagrangian node-steps/s, coupled step (RK3 flow + IBM forcing per substep + "
                  "body update)",
        "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "cell_steps_per_s": cells,
        "config": {"workload": descr + f"; flow solved: dt {dt:.3g} (CFL {COUPLED_CFL} of the "
                   "initial field), nu = mu = 0.01, p0 = 0",
                   "viscous_solve_widths": list(widths), "marker_patch": ctx.marker_patch,
                   "bodies": ctx.B, "vertices": ctx.V, "faces": ctx.F, "grid": list(wl.grid.n),
                   "max_face_area_h2": max_face_h2,
                   "l2": "flushed between timed steps (256 MiB write); fields of 64 MiB each",
                   "parallelism": f"{ws} independent replica(s)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(dom), "algorithmic_bytes": fb[dom] / 3},
        "phases_ms": ph,
        "fft_share": fft_ms / step_ms,
        "other_kernel": {k: {"algorithmic_bytes_per_step": fb[k],
                             "achieved_gbs": fb[k] / (ph_k[k] * 1e-3) / 1e9} for k in fb},
        # per step: 3 x (rhs, [cn_scale,] add or cn_solve, marker, div, poisson_scale,
        # project) + marker + force; cuFFT's own kernels and the memsets not counted
        "gpu_launches": (20 + sum(1 for w in widths if w < 0)) * args.steps,
        "timing": "coupled steps launched one by one; phases from CUDA events between the "
                  "kernels of separately timed steps",
        "e2e": e2e,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = coupled_oracle_rate(wl)
    print(json.dumps(line), flush=True)


def coupled_oracle_rate(wl):
    """The flow oracle's coupled step, as it stands, on the host cores: one
    step of 4 of the bodies on a 128^3 grid (the full 512^3 FFTs in float64
    take minutes); rates per node-step and per cell-step."""
    from oracle import ibm_oracle as O
    from oracle import ns_oracle as N
    sub = wl.bodies[:4]
    n = (128, 128, 128)
    grid = W.Grid(n, wl.grid.L)
    ob = [O.Body(b.rest, b.tri, b.origin, closed=b.closed, clamped=b.clamped, ks=b.ks, kb=b.kb,
                 ka=b.ka, kA=b.kA, kv=b.kv, mass=b.mass) for b in sub]
    u = W.sample_field(wl.field, grid, device="cpu", dtype=torch.float64)
    dt = cfl_dt(u, grid.h, COUPLED_CFL)
    u = torch.stack(list(u))
    prm = O.Params(n, wl.grid.L, dt=dt, mu=COUPLED_NU, alpha=wl.alpha)
    flow = N.Flow(n, wl.grid.L, nu=COUPLED_NU, dt=dt)
    p = torch.zeros(u.shape[1:], dtype=torch.float64)
    xs = [torch.tensor(b.rest) for b in sub]
    vs = [torch.zeros_like(x) for x in xs]
    t0 = time.perf_counter()
    N.coupled_step(ob, xs, vs, u, p, flow, prm)
    secs = time.perf_counter() - t0
    nodes = sum(len(b.rest) for b in sub)
    return {"value": nodes / secs, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "cell_steps_per_s": n[0] * n[1] * n[2] / secs,
            "sample": f"1 coupled step of {len(sub)} bodies ({nodes} nodes) on a 128^3 grid, "
                      f"{secs:.1f} s"}


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.coupled:
        run_coupled(args, ws, rank, local)
    else:
        run_gb300(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
