#!/usr/bin/env python
"""Benchmark of the per-step cloth solve.

Workload: the 512x512 hanging cloth (262,144 vertices, 522,242 triangles),
1 m wide in the x-z plane, top row pinned and swept 0.2 m at 1 Hz, dt 1/200 s,
self-collision on; every step iterates until the PD residual falls to 1e-3
of its value at z.  Forms: mixed16 (the headline: FP16 basis of 256 modes
scaled by a power of two, tcgen05 projections, FP64 reduced solves), mixed
(the same with a BF16 basis) and fp32 (all FP32).  Metric: ms per time step
(lower is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  With N > 1 (torchrun) every rank runs its own
replica (the cloth does not shard; "replicas only"), timing is max over
ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/step at 262K-vertex cloth (plain FP32 vs mixed) at 1e-3 residual; % HBM peak"
SIDE = 512
WORKLOAD = ("hanging swept cloth 512x512 (262,144 vertices, 522,242 triangles, 1 m, top row pinned and "
            "swept 0.2 m at 1 Hz), dt 1/200 s, self-collision on, iterate to 1e-3 relative PD residual")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=SIDE)
    ap.add_argument("--forms", default="mixed16,mixed,fp32",
                    help="comma list of mixed16 (FP16 basis), mixed (BF16 basis), fp32; the first is the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-side", type=int, default=32,
                    help="grid side of the oracle's sample (CPU baseline, reference arm, error report)")
    ap.add_argument("--error-steps", type=int, default=2,
                    help="steps of the per-form error report against the oracle (0: skip)")
    ap.add_argument("--error-side", type=int, default=64,
                    help="grid side of the per-form error report against the oracle")
    ap.add_argument("--sweeps", type=int, default=28, help="Chebyshev steps per LG iteration")
    ap.add_argument("--cheb-ratio", type=float, default=300.0, help="Chebyshev interval ratio b/a")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form comparison")
    ap.add_argument("--launch-overlap", type=int, default=1, choices=[0, 1],
                    help="1: Chebyshev steps launched as programmatic dependents (default)")
    ap.add_argument("--loop-control", type=int, default=1, choices=[0, 1, 2, 3],
                    help="stopping tests of the LG loops: 1 on the device in a CUDA graph while loop (default); "
                         "3 on the device, the host enqueueing each iteration ahead as one graph launch; 2 the "
                         "same with kernel launches; 0 on the host")
    ap.add_argument("--graph-unroll", type=int, default=1, help="LG iterations per pass of a graph loop (1..8)")
    ap.add_argument("--cheb-source", type=int, default=-1, choices=[-1, 0, 1, 2, 3],
                    help="matrix of the Chebyshev steps: -1 automatic, 0 ELL arrays, 1 row tiles, 2 patch tiles, 3 two steps a launch")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="1: launch shapes and the broad-phase grid timed on the handle's data in the warm-up")
    ap.add_argument("--loop-ahead", type=int, default=1, choices=[0, 1, 2],
                    help="LG iterations enqueued beyond the last decision read (loop control 2, 3)")
    ap.add_argument("--no-launch-count", action="store_true",
                    help="skip the CUDA activity trace (e.g. when running under ncu)")
    return ap.parse_args()


# form name -> pdc_params.precision, and the arithmetic types each form computes in
FORMS = {"mixed16": 2, "mixed": 1, "fp32": 0}
DTYPES = {"mixed16": "f16+f32+f64", "mixed": "bf16+f32+f64", "fp32": "f32"}


def solver_params(pc, precision, sweeps=28, cheb_ratio=300.0, overlap=1, loop_control=1, graph_unroll=1,
                  loop_ahead=1, autotune=1, cheb_source=-1):
    p = pc.pdc_default_params()
    p.loop_control = loop_control  # stopping tests of the LG loops on the device
    p.graph_unroll = graph_unroll
    p.loop_ahead = loop_ahead
    p.launch_overlap = overlap  # Chebyshev steps as programmatic dependent launches
    p.tol_rel_residual = 1e-3
    p.max_outer = 2
    p.max_inner = 400
    p.warm_iters = 5
    p.r_warm = 256
    p.r_reuse = 32
    p.precision = precision
    p.sweep_kind = 1        # Jacobi-preconditioned Chebyshev iteration for the sweeps
    p.jacobi_sweeps = sweeps
    p.cheb_ratio = cheb_ratio
    p.accel = 2             # Anderson mixing of the LG iterates
    p.aa_depth = 6
    p.solve_cycles = 1
    p.autotune = autotune   # launch shapes (first step) and broad-phase grid (8th pass) timed in the warm-up
    p.cheb_source = cheb_source
    p.eig_iters = 12
    return p


def max_over_ranks(value, device=None):
    """Largest value over the ranks of the default process group (the value
    itself on one rank); the timing of a multi-rank run is the slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_form(pc, torch, scene, precision, steps, warmup, dev_index, launch_count=True, sweeps=28, cheb_ratio=300.0,
             overlap=1, loop_control=1, graph_unroll=1, loop_ahead=1, autotune=1, cheb_source=-1):
    """Warm-up, timed region (device), profiled replay, e2e through host buffers."""
    import numpy as np
    stream = torch.cuda.Stream()
    p = solver_params(pc, precision, sweeps, cheb_ratio, overlap, loop_control, graph_unroll, loop_ahead, autotune,
                      cheb_source)
    t_setup = time.time()
    h = pc.pdc_create(scene.verts, scene.tris, scene.pins, scene.density, scene.k_stretch, scene.k_bend, p,
                      stream.cuda_stream)
    setup_s = time.time() - t_setup
    dt = p.dt
    total = warmup + steps
    # scripted pin targets for every step, resident on the device
    pins = np.stack([scene.pins_at((k + 1) * dt) for k in range(total)]).astype(np.float32)
    pins_d = torch.from_numpy(pins).to(f"cuda:{dev_index}")
    k = 0

    def one_step():
        nonlocal k
        pc.pdc_set_pin_targets_device(h, pins_d[k].data_ptr())
        pc.pdc_step(h, dt)
        k += 1

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    # checkpoint: the profiled replay, the launch count and the end-to-end
    # run repeat the timed steps from the same positions and velocities
    x_ck, v_ck = pc.pdc_get_state(h, scene.n)
    k_ck = k

    def restore():
        nonlocal k
        pc.pdc_set_state(h, x_ck, v_ck)
        k = k_ck
        torch.cuda.synchronize()

    # ---- timed region: device events on the library's stream
    clocks = ClockSampler(dev_index)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    # ---- profiled replay of the same steps (per-kernel event timing; the
    # profiler drives the LG loops from the host, same kernels)
    restore()
    pc.pdc_set_profiling(h, True)
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    kt = pc.pdc_get_kernel_times(h)
    pc.pdc_set_profiling(h, False)
    # ---- kernel launches of the library per step, counted by the CUDA
    # activity profiler over a replay of the same number of steps
    restore()
    launches, busy, gaps, kern_ms = count_launches(torch, one_step, steps) if launch_count else (None,) * 4
    restore()
    # ---- e2e through the public API with host buffers: pin targets h2d, positions d2h
    pin_host = torch.empty(pins.shape[1:], dtype=torch.float32).pin_memory()
    pos_host = torch.empty((scene.n, 3), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    st_list = []
    t0 = time.perf_counter()
    for j in range(steps):
        pin_host.numpy()[:] = scene.pins_at((k + 1) * dt)
        lib = pc.lib()
        pc._check(h, lib.pdc_set_pin_targets(h, pin_host.data_ptr(), 0))
        pc.pdc_step(h, dt)
        k += 1
        pc._check(h, lib.pdc_get_positions(h, pos_host.data_ptr(), 0))
        st_list.append(pc.pdc_get_stats(h))  # a host-side struct copy
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
    x = pos_host.numpy().copy()
    tuning = pc.pdc_get_tuning(h)
    pc.pdc_destroy(h)
    iters = [s["warm_iters"] + s["inner_iters"] for s in st_list]
    return dict(ms=ms / steps, setup_s=setup_s, clocks=clk, kernels=kt, e2e_ms=e2e_ms,
                h2d=int(pins.shape[1] * 12), d2h=int(scene.n * 12), iters=statistics.mean(iters),
                rel_res=statistics.mean(s["rel_residual"] for s in st_list),
                cand=statistics.mean(s["n_candidates"] for s in st_list),
                toi=min(s["t_toi"] for s in st_list), finite=bool(np.isfinite(x).all()),
                device_loops=statistics.mean(s["device_loops"] for s in st_list), device_busy=busy, idle_gaps=gaps,
                kernel_ms=kern_ms, launches=launches, tuning=tuning)


def solver_like(pc, p):
    """A copy of a pdc_params structure."""
    q = pc.pdc_default_params()
    for name, _ in p._fields_:
        v = getattr(p, name)
        if name == "gravity":
            for i in range(3):
                q.gravity[i] = v[i]
        else:
            setattr(q, name, v)
    return q


def run_batched(pc, torch, steps=5, warmup=5, dev_index=0):
    """Batched form (64 drapes of sides 16..192 over their own spheres, about
    0.9 M vertices, FP32, 32 LG iterations per step): one batched handle
    against the same 64 cloths stepped one after another on 64 handles.
    Instances are placed 2 m apart so that none touches another; each takes
    its own line-search fraction on the batched handle."""
    import numpy as np
    import workloads as wl
    scenes = wl.batched_drape()
    p = pc.pdc_default_params()
    for k, v in dict(fixed_iters=1, warm_iters=5, max_outer=1, max_inner=27, sweep_kind=1, jacobi_sweeps=16,
                     cheb_ratio=300.0, r_warm=32, r_reuse=32, eig_iters=4, precision=0).items():
        setattr(p, k, v)
    shifted = []
    for k, sc in enumerate(scenes):
        d = np.array([2.0 * (k % 8), 2.0 * (k // 8), 0.0], np.float32)
        obs = [(o.verts + d).astype(np.float32) for o in sc.obstacles]
        shifted.append(((sc.verts + d).astype(np.float32), sc.tris, sc.pins, sc.density, sc.k_stretch, sc.k_bend,
                        obs, [o.tris for o in sc.obstacles]))
    stream = torch.cuda.Stream()
    # one batched handle, every instance with its own line-search fraction
    # (its sphere attached to it)
    t0 = time.time()
    pb = solver_like(pc, p)
    pb.instance_line_search = 1
    pb.autotune = 1  # launch shapes timed on the batch's own data at the first step
    h, off = pc.pdc_create_batch([s[:6] for s in shifted], pb, stream.cuda_stream)
    for k, s in enumerate(shifted):
        for ov, ot in zip(s[6], s[7]):
            pc.pdc_set_obstacle_instance(h, pc.pdc_add_obstacle(h, ov, ot), k)
    setup_b = time.time() - t0
    for _ in range(warmup):
        pc.pdc_step(h, p.dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pc.pdc_step(h, p.dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / steps
    tuning = pc.pdc_get_tuning(h)
    gl = pc.pdc_get_stats(h)["device_loops"]
    pc.pdc_destroy(h)
    # the same cloths on separate handles, stepped in turn on one stream
    t0 = time.time()
    hs = []
    for s in shifted:
        hh = pc.pdc_create(s[0], s[1], s[2], s[3], s[4], s[5], p, stream.cuda_stream)
        for ov, ot in zip(s[6], s[7]):
            pc.pdc_add_obstacle(hh, ov, ot)
        hs.append(hh)
    setup_s = time.time() - t0
    for _ in range(warmup):
        for hh in hs:
            pc.pdc_step(hh, p.dt)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for hh in hs:
            pc.pdc_step(hh, p.dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1) / steps
    for hh in hs:
        pc.pdc_destroy(hh)
    return {"workload": "64 drapes over their own spheres, sides 16..192 (%d vertices), FP32, 32 LG iterations "
                        "per step, Chebyshev 16 steps per iteration, basis r=32" % int(off[-1]),
            "instances": len(shifted), "vertices": int(off[-1]), "steps": steps,
            "ms_per_step_batched": round(ms_b, 3), "ms_per_step_separate_handles": round(ms_s, 3),
            "speedup": round(ms_s / ms_b, 2), "setup_s_batched": round(setup_b, 1),
            "setup_s_separate": round(setup_s, 1), "device_loops_per_step": gl,
            "line_search": "per instance", "tuning": tuning}


def init_trace(torch):
    """Starts and stops one CUDA activity trace session, so that the tracer
    is set up before any CUDA graph is instantiated (kernels of graphs
    instantiated earlier would not be recorded)."""
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]):
            torch.cuda.synchronize()
    except Exception:
        pass


def count_launches(torch, one_step, steps):
    """Kernels launched by the library (names beginning with k_) during
    `steps` steps, from torch.profiler's CUDA activity trace; the share of
    the traced interval (first kernel start to last kernel end) in which some
    kernel ran; the largest idle gaps between consecutive kernels, summed by
    the pair of kernels around them; and the time per step in which some
    kernel ran (ms).  The trace lengthens the relaunch of a CUDA-graph while
    node's body (the gaps before each LG iteration's first kernel), so the
    busy share of the traced interval understates the untraced one; the
    kernel time per step against the untraced ms/step does not.  (None,) * 4
    if the trace is unavailable."""
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            for _ in range(steps):
                one_step()
            torch.cuda.synchronize()
        import re
        pat = re.compile(r"(?:^|[\s:])k_\w+")
        short = re.compile(r"(k_\w+)")
        n = 0
        spans = []
        for ev in prof.events():
            if str(getattr(ev, "device_type", "")).endswith("CUDA"):
                nm = ev.name or ""
                if pat.search(nm):
                    n += 1
                tr = getattr(ev, "time_range", None)
                if tr is not None and tr.end > tr.start:
                    m = short.search(nm)
                    spans.append((tr.start, tr.end, m.group(1) if m else nm[:24]))
        busy, gaps = None, None
        if spans:
            spans.sort()
            tot, cs, ce, last = 0.0, spans[0][0], spans[0][1], spans[0][2]
            acc = {}
            for a, b, nm in spans[1:]:
                if a > ce:
                    tot += ce - cs
                    key = last + " -> " + nm
                    g = acc.setdefault(key, [0, 0.0])
                    g[0] += 1
                    g[1] += a - ce
                    cs, ce = a, b
                else:
                    ce = max(ce, b)
                if b >= ce:
                    last = nm
            tot += ce - cs
            span = max(spans[-1][1] - spans[0][0], 1e-9)
            busy = round(tot / span, 4)
            top = sorted(acc.items(), key=lambda kv: -kv[1][1])[:10]
            gaps = {k: {"count": v[0], "us_per_step": round(v[1] / steps, 1)} for k, v in top}
        kern_ms = round(tot / 1e3 / steps, 3) if spans else None
        return n, busy, gaps, kern_ms
    except Exception:
        return None, None, None, None


# profiled regions that enclose other profiled regions (not kernels themselves)
PARENTS = {"broad_phase", "partial_ccd"}
# DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, one
# capture at 512x512) of the kernels that can be the dominant one; the file
# under profiles/ gives the command
TRAFFIC = {"cheb_sweep": 35386880.0}


def l2_copy_peak(pc, stream, mbytes=40):
    """Copy bandwidth of a working set that stays in L2 (mbytes of read plus
    written bytes per pass, 129 MB of L2): the library's persistent copy
    kernel, 400 passes per launch, best of 5, CUDA events; counted like the
    HBM copy peak (read + written bytes)."""
    return max(pc.pdc_measure_copy_bandwidth(mbytes << 20, 400, stream) for _ in range(5))


# working set of the dominant kernel per launch at the benchmark size (bytes):
# the patch tiles of H (1,024 x 21.5 KB) and the residual, three Chebyshev
# iterates, diagonal and iterate streams (float4, 4.2 MB each)
WORKING_SET = {"cheb_sweep": 22.0e6 + 6 * 4.19e6}
L2_BYTES = 129e6


def roofline(kernels, pk, ms_step, l2_gbs=None):
    """Dominant kernel (largest total time among the profiled leaf regions),
    achieved algorithmic bytes per launch / event time against the measured
    copy peak of the memory level its working set lives in: the L2 copy peak
    measured in this run when the working set fits in L2, else the HBM copy
    peak of MEASURED_PEAKS.json (both given)."""
    leaves = {k: v for k, v in kernels.items() if k not in PARENTS}
    best = max(leaves.items(), key=lambda kv: kv[1]["total_ms"])
    name, d = best
    per_launch_ms = d["total_ms"] / max(d["launches"], 1)
    bytes_per_launch = d["algo_bytes"] / max(d["launches"], 1)
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
    hbm = float(pk.get("hbm_gbs", 6800.0))
    ws = WORKING_SET.get(name)
    in_l2 = ws is not None and ws < 0.5 * L2_BYTES and l2_gbs
    peak = l2_gbs if in_l2 else hbm
    return {"kernel": name, "bound": "l2" if in_l2 else "hbm", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": TRAFFIC.get(name), "launches": d["launches"],
            "ms_per_launch": round(per_launch_ms, 5), "bytes_per_launch": bytes_per_launch,
            "working_set_bytes": ws, "hbm_peak": hbm, "hbm_frac": round(achieved / hbm, 4),
            "peak_source": ("L2 copy measured in this run (persistent copy kernel, 40 MB working set), of measured"
                            if in_l2 else
                            ("HBM copy of MEASURED_PEAKS.json, of measured" if not pk.get("_fallback") else "fallback"))}


ORACLE_PARAMS = "pd.Params(tol_rel_residual=1e-3, max_outer=2, max_inner=400, warm_iters=5)"


def oracle_from_states(side, states_path, out_path):
    """Runs, in a separate one-thread process, one FP64 oracle step of the
    swept cloth at side x side from each stored state (x*, v*, t) with the
    benchmark's stopping rule; stores the results and per-step times."""
    code = r'''
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
import workloads as wl
from oracle import pd, build
build.build()
sc = wl.hanging_swept(side=%d)
d = np.load(%r)
o = pd.Oracle(sc, %s)
xs, ts, its, res = [], [], [], []
m = o.model
for k in range(len(d["t"])):
    o.x, o.v, o.t = d["x"][k].astype(np.float64), d["v"][k].astype(np.float64), float(d["t"][k])
    z = o.x + o.p.dt * o.v + o.p.dt ** 2 * np.asarray(o.p.gravity)[None, :]
    z[~m.free] = sc.pins_at(o.t + o.p.dt)
    t0 = time.time()
    x, v, st = o.step()
    ts.append(time.time() - t0)
    xs.append(x)
    its.append(st.warm_iters + st.inner_iters)
    res.append(float(st.rel_residual))
np.savez(%r, x=np.array(xs), s=np.array(ts), iters=np.array(its), res=np.array(res))
''' % (ROOT, side, states_path, ORACLE_PARAMS, out_path)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)


def error_vs_oracle(pc, torch, forms, side, warm, steps, dev_index):
    """Per-step error of each form against the FP64 oracle, on the same swept
    cloth at side x side (the oracle's brute-force broad phase and exact
    sparse solves make the full 512 x 512 size impractical).  Start states:
    the first form's trajectory after `warm` steps.  From each state every
    form takes one production step (x* + u exactly, from the step's
    displacement), the oracle one step with the same stopping rule; reported
    per step: max and RMS vertex distance / bounding-box diagonal, the
    residual the form reports, the oracle's residual (R11, FP64) at the
    form's x* + u (only for steps without active collision springs and
    without an impact), and the residual at which the oracle's own stopping
    test ended (before its exit positions are rounded to float32)."""
    import numpy as np
    import workloads as wl
    from oracle import pd
    scene = wl.hanging_swept(side=side)
    dt = 1.0 / 200
    first = list(forms)[0]
    h = pc.pdc_create(scene.verts, scene.tris, scene.pins, scene.density, scene.k_stretch, scene.k_bend,
                      solver_params(pc, FORMS[first]))
    states = []
    for k in range(warm + steps):
        if k >= warm:
            x, v = pc.pdc_get_state(h, scene.n)
            states.append((x, v, k * dt))
        pc.pdc_set_pin_targets(h, scene.pins_at((k + 1) * dt))
        pc.pdc_step(h, dt)
    pc.pdc_destroy(h)
    fd, spath = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    opath = spath.replace(".npz", "_out.npz")
    np.savez(spath, x=np.array([s[0] for s in states]), v=np.array([s[1] for s in states]),
             t=np.array([s[2] for s in states]))
    r = oracle_from_states(side, spath, opath)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    od = np.load(opath)
    os.unlink(spath)
    os.unlink(opath)
    m = pd.Model(scene.verts, scene.tris, scene.pins, scene.density, scene.k_stretch, scene.k_bend, dt)
    g = np.array([0.0, 0.0, -9.8])
    out = {"grid": "%dx%d (%d vertices), the benchmark's scene and settings" % (side, side, scene.n),
           "start_states": "%s trajectory after %d steps" % (first, warm), "steps": steps,
           "oracle": {"rel_residual": [round(float(v), 6) for v in od["res"]],
                      "lg_iters": [int(v) for v in od["iters"]], "s_per_step": [round(float(v), 2) for v in od["s"]]},
           "forms": {}}
    for f in forms:
        h = pc.pdc_create(scene.verts, scene.tris, scene.pins, scene.density, scene.k_stretch, scene.k_bend,
                          solver_params(pc, FORMS[f]))
        rec = {"err_max": [], "err_rms": [], "rel_residual_reported": [], "rel_residual_oracle_at_form": [],
               "n_active": []}
        for k, (x, v, t) in enumerate(states):
            pc.pdc_set_state(h, x, v)
            pc.pdc_set_pin_targets(h, scene.pins_at(t + dt))
            pc.pdc_step(h, dt)
            st = pc.pdc_get_stats(h)
            xg = x.astype(np.float64) + pc.pdc_get_displacement(h, scene.n).astype(np.float64)
            d = np.linalg.norm(xg - od["x"][k], axis=1)
            rec["err_max"].append(float(d.max() / m.L))
            rec["err_rms"].append(float(np.sqrt(np.mean(d * d)) / m.L))
            rec["rel_residual_reported"].append(st["rel_residual"])
            rec["n_active"].append(st["n_active"])
            z = x.astype(np.float64) + dt * v.astype(np.float64) + dt * dt * g[None, :]
            z[scene.pins] = scene.pins_at(t + dt)
            ok = st["n_active"] == 0 and st["t_toi"] >= 2.0
            rec["rel_residual_oracle_at_form"].append(
                float(np.linalg.norm(m.residual(xg, z)) / np.linalg.norm(m.residual(z, z))) if ok else None)
        pc.pdc_destroy(h)
        out["forms"][f] = rec
    out["_oracle_ms"] = [float(v) * 1e3 for v in od["s"]]
    out["_oracle_side"] = side
    return out


def cpu_baseline(side, steps, warmup, budget_s=150.0):
    """The FP64 oracle as it stands on a bounded sample: its own trajectory
    of the same scene at side x side, `warmup` untimed then up to `steps`
    timed steps, in a separate one-thread process, stopping once budget_s
    of timed work is spent.  ms/step is scaled linearly by vertex count to
    512 x 512: a lower bound of the oracle at full size, whose brute-force
    broad phase and sparse factorisations grow faster than linearly."""
    code = r'''
import os, sys, time, json
sys.path.insert(0, %r)
import workloads as wl
from oracle import pd, build
build.build()
sc = wl.hanging_swept(side=%d)
o = pd.Oracle(sc, %s)
for k in range(%d):
    o.step()
ts = []
for k in range(%d):
    t0 = time.time()
    o.step()
    ts.append(time.time() - t0)
    if sum(ts) > %r:
        break
print(json.dumps({"s": ts, "n": sc.n, "cores": os.cpu_count()}))
''' % (ROOT, side, ORACLE_PARAMS, warmup, max(steps, 1), budget_s)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        return {"value": None, "error": out.stderr[-300:]}
    d = json.loads(out.stdout.strip().splitlines()[-1])
    scale = (SIDE * SIDE) / d["n"]
    per = [t * 1e3 * scale for t in d["s"]]
    return {"value": round(statistics.mean(per), 1), "unit": "ms/step", "cores": 1, "kind": "oracle",
            "per_step": per,
            "sample": "%d oracle steps (after %d untimed, of %d asked) of the same swept-cloth scene at %dx%d "
                      "(%d vertices), one thread on a %d-core host, ms/step scaled linearly by vertex count to "
                      "512x512 (a lower bound at full size)" % (len(d["s"]), warmup, max(steps, 1), side, side,
                                                               d["n"], d["cores"])}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        if rank != 0:
            return
        r = cpu_baseline(a.cpu_sample_side, steps=max(a.steps, 1), warmup=a.warmup)
        if r["value"] is None:
            print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + r.get("error", "")}))
            return
        base = r
        vals = r["per_step"]
        v = statistics.mean(vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/step", "n_gpus": a.gpus,
                          "steps": a.steps, "warmup": a.warmup, "ms_per_step": v, "higher_is_better": False,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": WORKLOAD},
                          "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": base["sample"], "value": v,
                                           "unit": "ms/step"},
                          "e2e": {"value": v, "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2403_19272_gb300 import build as libbuild
    libbuild.build()
    from paper_2403_19272_gb300 import pdcloth as pc
    import workloads as wl
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    scene = wl.hanging_swept(side=a.side)
    if not a.no_launch_count:
        init_trace(torch)
    forms = {}
    for f in a.forms.split(","):
        forms[f] = run_form(pc, torch, scene, FORMS[f], a.steps, a.warmup, local,
                            not a.no_launch_count, a.sweeps, a.cheb_ratio, a.launch_overlap, a.loop_control,
                            a.graph_unroll, a.loop_ahead, a.autotune, a.cheb_source)
    head = list(forms)[0]
    ms = forms[head]["ms"]
    ms = max_over_ranks(ms, f"cuda:{local}")
    if rank != 0:
        return
    pk = peaks()
    l2 = l2_copy_peak(pc, torch.cuda.current_stream().cuda_stream)
    rl = roofline(forms[head]["kernels"], pk, ms, l2)
    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": "ms/step", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": head, "basis": "r=256 (r_reuse=32 with collision springs)",
                   "l2": "inputs larger than L2 (basis 134 MB in 16 bits / 268 MB FP32 plus matrices and state)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "loop_control": a.loop_control, "loop_ahead": a.loop_ahead, "autotune": a.autotune},
        "forms": {f: {"ms_per_step": round(d["ms"], 3), "lg_iters_per_step": d["iters"],
                      "vertex_iters_per_s": round(scene.n * d["iters"] / (d["ms"] * 1e-3), 1),
                      "gpu_launches": d["launches"],
                      "rel_residual": d["rel_res"], "candidates": d["cand"], "min_toi": d["toi"],
                      "device_loops_per_step": d["device_loops"], "device_busy": d["device_busy"],
                      "kernel_ms_per_step": d["kernel_ms"],
                      "setup_s": round(d["setup_s"], 2), "e2e_ms_per_step": round(d["e2e_ms"], 3),
                      "tuning": d["tuning"]}
                  for f, d in forms.items()},
        "roofline": rl,
        "clocks": forms[head]["clocks"],
        "e2e": {"value": round(forms[head]["e2e_ms"], 3), "unit": "ms/step",
                "h2d_bytes_per_step": forms[head]["h2d"], "d2h_bytes_per_step": forms[head]["d2h"]},
        "gpu_launches": forms[head]["launches"],
        "idle_gaps": forms[head]["idle_gaps"],
        "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3),
                        "GBps": round(v["algo_bytes"] / max(v["total_ms"], 1e-9) / 1e6, 1)}
                    for k, v in forms[head]["kernels"].items()},
    }
    if not a.no_batched and world == 1:
        try:
            line["batched"] = run_batched(pc, torch, dev_index=local)
        except Exception as e:  # reported, not fatal for the headline
            line["batched"] = {"error": str(e)[:200]}
    if a.error_steps > 0 and world == 1:
        try:
            ev = error_vs_oracle(pc, torch, list(forms), a.error_side, 5, a.error_steps, local)
        except Exception as e:  # reported, not fatal for the headline
            ev = {"error": str(e)[:300]}
        oms = ev.pop("_oracle_ms", None)
        oside = ev.pop("_oracle_side", None)
        line["error_vs_oracle"] = ev
        if oms and not a.no_cpu_baseline:
            # the oracle steps of the error report are the CPU baseline's sample
            scale = (SIDE * SIDE) / float(oside * oside)
            per = [t * scale for t in oms]
            line["cpu_baseline"] = {
                "value": round(statistics.mean(per), 1), "unit": "ms/step", "cores": 1, "kind": "oracle",
                "per_step": [round(v, 1) for v in per],
                "sample": "%d oracle steps of the same swept-cloth scene at %dx%d (%d vertices) from the states of the "
                          "error report, one thread on a %d-core host, ms/step scaled linearly by vertex count to "
                          "512x512 (a lower bound at full size)" % (len(oms), oside, oside, oside * oside,
                                                                    os.cpu_count())}
    if "cpu_baseline" not in line and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a.cpu_sample_side, 2, 3, budget_s=30.0)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
