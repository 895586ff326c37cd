"""Benchmark of the GB300 Fast Haar transform.

Headline workload: one 4096 x 4096 fp32 piecewise-smooth image, 5-level 2D
Fast Haar analysis followed by the full synthesis (DWT + IDWT round trip).
One step = one round trip of one image.  The metric is input samples
(pixels) per second through the round trip, in Gsamples/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  For N > 1 it is launched with
torch.distributed.run, one process per GPU; the transform has no exchange
step, so every rank runs an independent replica and the value is the sum of
all ranks' samples over the slowest rank's time ("weak" scaling).

``--impl reference`` times the FP64 CPU oracle (the plain definition of the
filter bank) on the host instead, one full round trip of the same image per
step; it runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Haar DWT+IDWT Gsamples/s & %HBM roofline; bf16/ragged/bwd vs plain fp32"
UNIT = "Gsamples/s"
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth (context beside the measured peak)
N_SETS = 4  # rotating input/coefficient/output sets: 4 x 192 MB > L2


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--soak-s", type=float, default=1.5,
                    help="seconds of untimed steps before the timed region (clocks settle)")
    ap.add_argument("--no-forms", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows-once", action="store_true",
                    help="run the main operation of every row once on a case larger than L2 "
                         "(for a profiler capture) and exit; prints no JSON line")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (measurement only: no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(elapsed_ms: float, units: float, world: int, device=None):
    """(max elapsed over ranks, sum of units over ranks)."""
    if world == 1:
        return elapsed_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks sampled during the measurement
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
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
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


# translation units each timed kernel is built from
KERNEL_UNITS = {"k_dwt2d_fast": ("haar_tin_f32.cu", "haar_api.cu"),
                "k_idwt2d_fast": ("haar_tin_f32.cu", "haar_api.cu")}


def kernel_source_hash(units=("haar_tin_f32.cu", "haar_api.cu")):
    """Hash of the code (comments and layout stripped) of the given
    translation units and every file they include (quoted includes, followed
    recursively): a change anywhere else in the library, or in comments, does
    not touch the recorded counters of these kernels."""
    import hashlib
    import re
    dirs = [os.path.join(ROOT, "paper_1002_2184_gb300", "csrc"), os.path.join(ROOT, "include")]
    seen, todo = set(), list(units)
    while todo:
        name = todo.pop()
        if name in seen:
            continue
        for d in dirs:
            path = os.path.join(d, name)
            if os.path.exists(path):
                seen.add(name)
                with open(path) as f:
                    todo += re.findall(r'^\s*#\s*include\s+"([^"]+)"', f.read(), re.M)
                break
    h = hashlib.sha256()
    for name in sorted(seen):
        for d in dirs:
            path = os.path.join(d, name)
            if os.path.exists(path):
                with open(path) as f:
                    h.update(name.encode())
                    h.update(code_only(f.read()).encode())
                break
    return h.hexdigest()[:16]


def code_only(text: str) -> str:
    """C/C++/CUDA source with comments removed and whitespace collapsed, so
    that an edit of comments or layout alone keeps the hash (string literals
    are kept as they are)."""
    import re
    tok = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"', re.S)
    text = tok.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
    return " ".join(text.split())


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    src = kernel_source_hash(KERNEL_UNITS.get(kernel, ("haar_tin_f32.cu", "haar_api.cu")))
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        kv = dict(p.split("=", 1) for p in ln.split() if "=" in p)
        if kv.get("kernel") == kernel and kv.get("source_sha") == src:
            return float(kv["dram_bytes_per_launch"])
    return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1002_2184_gb300 import api, build, synth
    build.build()

    cfg = synth.Image2D()
    H, W, L = cfg.h, cfg.w, cfg.levels
    px = H * W
    xs = [torch.from_numpy(synth.piecewise_smooth_image(H, W, cfg.seed, i).astype(np.float32))
          .to(dev) for i in range(N_SETS)]
    cs = [torch.empty_like(x) for x in xs]
    ys = [torch.empty_like(x) for x in xs]
    stream = torch.cuda.current_stream(dev)
    plans = [api.Plan(xs[s], cs[s], L, ys[s]) for s in range(N_SETS)]
    # each input set has its own stream: a step's IDWT follows its DWT, and
    # steps on different sets (independent data) may overlap, so the drain of
    # one launch overlaps the ramp-up of the next step's first one
    streams = [torch.cuda.Stream(dev) for _ in range(N_SETS)]

    def step(k):
        s = k % N_SETS
        plans[s].dwt(streams[s])
        plans[s].idwt(streams[s])

    # Every timed run is one CUDA graph replay: the launches are recorded once
    # (programmatic dependent launch edges included), so host launch cost is
    # not what is measured.  The step graph forks the four set streams from
    # the capture stream and joins them at the end.
    def capture(body):
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(stream)
        with torch.cuda.graph(g, stream=cap):
            body(cap)
        torch.cuda.synchronize(dev)
        return g

    def steps_body(n):
        def body(cap):
            for st in streams:
                st.wait_stream(cap)
            for k in range(n):
                step(k)
            for st in streams:
                cap.wait_stream(st)
        return body

    def serial_body(n):
        def body(cap):
            for k in range(n):
                s_ = k % N_SETS
                plans[s_].dwt(cap)
                plans[s_].idwt(cap)
        return body

    def single_body(n, which):
        def body(cap):
            for k in range(n):
                getattr(plans[k % N_SETS], which)(cap)
        return body

    for k in range(N_SETS):  # eager warm-up (and a correctness reference)
        step(k)
    torch.cuda.synchronize(dev)
    g_steps = capture(steps_body(args.steps))
    g_warm = capture(steps_body(max(3, args.warmup)))
    g_serial = capture(serial_body(args.steps))
    g_dwt = capture(single_body(args.steps, "dwt"))
    g_idwt = capture(single_body(args.steps, "idwt"))

    def replay_ms(g):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.replay()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    g_warm.replay()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(dev.index if world == 1 else local)
    sampler.start()
    t_end = time.time() + args.soak_s
    while time.time() < t_end:
        g_warm.replay()
        torch.cuda.synchronize(dev)

    # timed region: exactly K steps (one graph replay), events at its ends
    barrier(world)
    torch.cuda.synchronize(dev)
    elapsed_ms = replay_ms(g_steps)
    barrier(world)

    # the same K steps strictly one after the other on one stream (reported
    # beside the value: the per-step time of a single image in isolation)
    serial_ms = replay_ms(g_serial) / args.steps

    # per-kernel launch duration: K back-to-back launches of each kernel
    # alone, same rotating buffers
    dwt_ms = replay_ms(g_dwt) / args.steps
    idwt_ms = replay_ms(g_idwt) / args.steps
    clocks = sampler.stop()

    max_ms, units = aggregate(elapsed_ms, float(px) * args.steps, world, dev)
    value = units / (max_ms * 1e-3) / 1e9

    # correctness guard on the timed data: the round trip reproduces the input
    err = float(torch.linalg.vector_norm((ys[0] - xs[0]).double()) /
                torch.linalg.vector_norm(xs[0].double()))
    head = (host64(xs[0]), host64(cs[0]), host64(ys[0]))  # checked against the oracle

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    alg_bytes = 8.0 * px  # read 4 B + write 4 B per pixel, per kernel
    dom = "k_dwt2d_fast" if dwt_ms >= idwt_ms else "k_idwt2d_fast"
    dom_ms = max(dwt_ms, idwt_ms)
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {
        "bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
        "unit": "GB/s", "frac": round(achieved / hbm, 4), "peak_source": peak_src,
        "traffic": recorded_traffic(dom),
        "algorithmic_bytes_per_launch": alg_bytes,
        "duration_source": "CUDA events around one graph replay of K back-to-back launches "
                           "of the kernel alone (rotating buffer sets), right after the timed "
                           "region",
        "kernels": {
            "k_dwt2d_fast": {"avg_us": round(dwt_ms * 1e3, 2),
                             "gbs": round(alg_bytes / (dwt_ms * 1e-3) / 1e9, 1),
                             "frac": round(alg_bytes / (dwt_ms * 1e-3) / 1e9 / hbm, 4)},
            "k_idwt2d_fast": {"avg_us": round(idwt_ms * 1e3, 2),
                              "gbs": round(alg_bytes / (idwt_ms * 1e-3) / 1e9, 1),
                              "frac": round(alg_bytes / (idwt_ms * 1e-3) / 1e9 / hbm, 4)},
        },
        "step_roofline": {"ideal_us": round(2 * alg_bytes / (hbm * 1e9) * 1e6, 2),
                          "measured_us": round(max_ms / args.steps * 1e3, 2),
                          "frac": round(2 * alg_bytes / (hbm * 1e9) / (max_ms / args.steps * 1e-3), 4)},
        "nominal_gbs": NOMINAL_HBM_GBS,
        "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
    }

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"2D fp32 image {H}x{W}, {L}-level DWT then full IDWT",
                   "h": H, "w": W, "levels": L, "batch_per_gpu": 1,
                   "l2": f"rotating {N_SETS} input/coef/output sets "
                         f"({N_SETS * 3 * px * 4 / 2**20:.0f} MiB) > L2; the IDWT reads the "
                         "coefficients its DWT just wrote",
                   "streams": f"one per input set ({N_SETS}): steps on different sets may "
                              "overlap, a step's IDWT always follows its DWT",
                   "launch": "the K timed steps are one CUDA graph replay (captured once, "
                             "programmatic dependent launch edges kept)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "gpu_launches": 2 * args.steps,
        "serial_ms_per_step": round(serial_ms, 5),
        "serial_frac_of_ideal": round(2 * alg_bytes / (hbm * 1e9) / (serial_ms * 1e-3), 4),
        "round_trip_rel_l2": err,
    }
    if clocks:
        out["clocks"] = clocks

    if not args.no_e2e:
        out["e2e"] = e2e_ours(api, synth, dev, cfg, max(10, min(args.steps, 50)), world)
    if not args.no_forms:
        out["forms"] = forms(api, synth, dev, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["accuracy"] = cpu_leg(synth, cfg, head, out.get("forms"))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def e2e_ours(api, synth, dev, cfg, steps, world):
    """Same metric through the public API with host buffers: every step
    copies one image from pinned host memory, runs DWT + IDWT and copies the
    reconstruction back to pinned host memory.  Two device buffer sets and
    three streams overlap the upload of step k+1, the transforms of step k
    and the download of step k-1."""
    import torch
    H, W, L = cfg.h, cfg.w, cfg.levels
    host_in = torch.from_numpy(
        synth.piecewise_smooth_image(H, W, cfg.seed, 0).astype(np.float32)).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    x = [torch.empty(host_in.shape, dtype=torch.float32, device=dev) for _ in range(2)]
    c = [torch.empty_like(x[0]) for _ in range(2)]
    y = [torch.empty_like(x[0]) for _ in range(2)]
    plans = [api.Plan(x[i], c[i], L, y[i]) for i in range(2)]
    s_up, s_cmp, s_dn = (torch.cuda.Stream(dev) for _ in range(3))
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_x_free = [torch.cuda.Event() for _ in range(2)]
    ev_y_ready = [torch.cuda.Event() for _ in range(2)]
    ev_y_free = [torch.cuda.Event() for _ in range(2)]

    def run(n):
        for k in range(n):
            i = k % 2
            with torch.cuda.stream(s_up):
                if k >= 2:
                    s_up.wait_event(ev_x_free[i])
                x[i].copy_(host_in, non_blocking=True)
                ev_in[i].record(s_up)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[i])
                if k >= 2:
                    s_cmp.wait_event(ev_y_free[i])
                plans[i].dwt(s_cmp)
                ev_x_free[i].record(s_cmp)
                plans[i].idwt(s_cmp)
                ev_y_ready[i].record(s_cmp)
            with torch.cuda.stream(s_dn):
                s_dn.wait_event(ev_y_ready[i])
                host_out[i].copy_(y[i], non_blocking=True)
                ev_y_free[i].record(s_dn)

    run(4)
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize(dev)
    el_ms = (time.perf_counter() - t0) * 1e3
    ms, units = aggregate(el_ms, float(H * W) * steps, world, dev)
    ok = all(bool(torch.allclose(h, host_in, atol=1e-5)) for h in host_out)

    # the host link alone: the same uploads and downloads, overlapped the
    # same way, with no transform in between (the ceiling for this metric)
    def link(n):
        for k in range(n):
            i = k % 2
            with torch.cuda.stream(s_up):
                x[i].copy_(host_in, non_blocking=True)
            with torch.cuda.stream(s_dn):
                host_out[i].copy_(y[i], non_blocking=True)

    link(4)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    link(steps)
    torch.cuda.synchronize(dev)
    link_ms = (time.perf_counter() - t0) * 1e3 / steps
    step_ms = el_ms / steps
    return {"value": round(units / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": H * W * 4, "d2h_bytes_per_step": H * W * 4,
            "steps": steps, "round_trip_ok": ok,
            "ms_per_step": round(step_ms, 4),
            "link_only_ms_per_step": round(link_ms, 4),
            "frac_of_link": round(link_ms / step_ms, 4),
            "timing": "host wall clock from the first upload to the last download, "
                      "device synchronised at both ends; link_only = the same copies "
                      "without the transforms"}


def cpu_leg(synth, cfg, head, forms_out, min_seconds=6.0):
    """The host-side leg of the benchmark (rank 0, one GPU only): the FP64
    oracle as it stands timed on this host's cores, the FP32 CPU baseline
    (the same method as a plain loop, one core), and the accuracy of every
    sampled GPU result against the oracle.

    head: host copies (x, coef, recon) of the headline image as the GPU
    produced them.  forms_out: the forms dict, whose entries get their
    "accuracy" here.  Returns (cpu_baseline dict, headline accuracy dict)."""
    import concurrent.futures as cf
    import oracle
    from oracle import cpu_baseline as fp32cpu
    H, W, L = cfg.h, cfg.w, cfg.levels
    x = synth.piecewise_smooth_image(H, W, cfg.seed, 0).astype(np.float32).astype(np.float64)
    oracle.lib()

    # (a) the oracle, one thread, the full headline image
    reps, t0 = 0, time.perf_counter()
    while True:
        c_ref = oracle.dwt2d(x, L)
        oracle.idwt2d(c_ref, L)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    out = {"value": round(H * W * reps / el / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{reps} round trips of the full {H}x{W} image, {L} levels, FP64 C oracle, "
                     f"one thread ({el:.1f} s)"}
    head_acc = {"vs": "FP64 oracle", "sample": f"the {H}x{W} image of input set 0",
                "coef": err_stats([(head[1], c_ref)]),
                "recon": err_stats([(head[2], oracle.idwt2d(c_ref, L))])}

    # (b) the same method as a plain FP32 loop, one core, -O3
    xf = x.astype(np.float32)
    fp32cpu.dwt2d_f32(xf, L)
    reps, t0 = 0, time.perf_counter()
    while True:
        fp32cpu.idwt2d_f32(fp32cpu.dwt2d_f32(xf, L), L)
        reps += 1
        el = time.perf_counter() - t0
        if el >= 2.0:
            break
    out["fp32_fast_haar_one_core"] = {
        "value": round(H * W * reps / el / 1e9, 4), "unit": UNIT, "cores": 1,
        "kind": "the Fast Haar butterfly as a plain FP32 loop (gcc -O3, no SIMD intrinsics)",
        "sample": f"{reps} round trips of the {H}x{W} image ({el:.1f} s)"}

    # (c) the oracle on every host core, one image per thread, on the
    # precision, ragged and differentiation workloads (bounded samples)
    cores = os.cpu_count() or 1
    multi = {"cores": cores, "kind": "oracle, one image per thread"}
    with cf.ThreadPoolExecutor(max_workers=cores) as pool:
        def timed(jobs, px, seconds=2.0):
            # whole rounds of the job list until `seconds` have passed
            rounds, t = 0, time.perf_counter()
            while True:
                list(pool.map(lambda f: f(), jobs))
                rounds += 1
                el = time.perf_counter() - t
                if el >= seconds:
                    return round(rounds * px / el / 1e9, 5), round(el, 2)

        pcfg = synth.PrecisionBatch()
        imgs = [synth.piecewise_smooth_image(pcfg.h, pcfg.w, pcfg.seed, i) for i in range(cores)]
        v, el = timed([lambda a=a: oracle.idwt2d(oracle.dwt2d(a, pcfg.levels), pcfg.levels)
                       for a in imgs], cores * pcfg.h * pcfg.w)
        multi["precision"] = {"value": v, "unit": UNIT, "seconds": el,
                              "sample": f"rounds of {cores} images of {pcfg.h}x{pcfg.w}, "
                                        f"{pcfg.levels} levels, DWT + IDWT"}
        rcfg = synth.RaggedBatch()
        items = synth.ragged_shapes(rcfg)[:2 * cores]
        rim = [synth.piecewise_smooth_image(h, w, rcfg.seed, i) for i, (h, w, _) in
               enumerate(items)]
        v, el = timed([lambda a=a, lv=lv: oracle.idwt2d(oracle.dwt2d(a, lv), lv)
                       for a, (_, _, lv) in zip(rim, items)], sum(h * w for h, w, _ in items))
        multi["ragged"] = {"value": v, "unit": UNIT, "seconds": el,
                           "sample": f"rounds of the first {len(items)} images of the ragged "
                                     "batch, DWT + IDWT"}
        gcfg = synth.GradBatch()
        _, C, gh, gw = gcfg.shape
        gim = [synth.piecewise_smooth_image(gh, gw, gcfg.seed, i)[None, None] for i in
               range(cores)]
        v, el = timed([lambda a=a: (oracle.denoise_loss(a, gcfg.levels, gcfg.threshold,
                                                        gcfg.l1_weight),
                                    oracle.denoise_loss_grad(a, gcfg.levels, gcfg.threshold,
                                                             gcfg.l1_weight))
                       for a in gim], cores * gh * gw)
        multi["backward"] = {"value": v, "unit": UNIT, "seconds": el,
                             "sample": f"rounds of {cores} channels of {gh}x{gw}, loss and "
                                       "gradient"}
    out["multi_core"] = multi

    # (d) accuracy of every sampled result
    for form, entry, check in ACCURACY:
        res = check(oracle)
        tgt = forms_out.get(form) if forms_out else None
        if tgt is None:
            continue
        (tgt[entry] if entry else tgt)["accuracy"] = res
    return out, head_acc


# ---------------------------------------------------------------------------
# secondary forms, each next to the plain fp32 path on the same GPU
# ---------------------------------------------------------------------------
# Accuracy of each result against the FP64 oracle.  The GPU side only copies
# its outputs for a few sampled items to host memory here; the oracle runs in
# the CPU-baseline leg (cpu_leg), which fills in each form's "accuracy".
ACCURACY = []  # (form name, entry name or None, function(oracle) -> dict)


def err_stats(pairs):
    """max-abs and relative L2 over (result, reference) pairs of float64
    arrays; rel-L2 is over all pairs together."""
    num = den = mx = scale = 0.0
    for got, ref in pairs:
        d = got - ref
        num += float(np.sum(d * d))
        den += float(np.sum(ref * ref))
        mx = max(mx, float(np.max(np.abs(d))) if d.size else 0.0)
        scale = max(scale, float(np.max(np.abs(ref))) if ref.size else 0.0)
    return {"max_abs": mx, "rel_l2": (num / den) ** 0.5 if den > 0 else num ** 0.5,
            "max_abs_over_max_ref": mx / scale if scale > 0 else mx}


def host64(t):
    return t.detach().double().cpu().numpy()


def time_med(fn, reps=50, warmup=3, min_group_ms=0.25):
    """Per-call device time: the median over ``reps`` groups of back-to-back
    calls, CUDA events on the current stream between the groups (no gap and
    no synchronisation between them).  A group holds enough calls to last
    about ``min_group_ms``, so short calls are not dominated by the event."""
    import math
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(3):
        fn()
    b.record()
    torch.cuda.synchronize()
    one = max(a.elapsed_time(b) / 3, 1e-4)
    g = max(1, int(math.ceil(min_group_ms / one)))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record()
    for r in range(reps):
        for _ in range(g):
            fn()
        ev[r + 1].record()
    torch.cuda.synchronize()
    return statistics.median(ev[r].elapsed_time(ev[r + 1]) / g for r in range(reps))


def forms(api, synth, dev, world):
    import torch
    res = {}

    # 1D signal, 2^16 samples, one level: launch-bound, reported as latency
    sc = synth.Signal1D()
    x1 = torch.from_numpy(synth.signal_1d(sc.n, sc.seed).astype(np.float32)).to(dev)
    c1 = torch.empty_like(x1)
    y1 = torch.empty_like(x1)
    p1 = api.Plan(x1, c1, sc.levels, y1, one_d=True)
    p1.dwt()
    p1.idwt()
    torch.cuda.synchronize()
    g1 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g1):
        p1.dwt()
        p1.idwt()

    ms_eager = time_med(lambda: (p1.dwt(), p1.idwt()))
    ms = time_med(g1.replay)
    s1 = (host64(x1), host64(c1), host64(y1))

    def check_signal(orc, s1=s1, L=sc.levels):
        ref = orc.dwt1d(s1[0], L)
        return {"vs": "FP64 oracle", "sample": "the whole signal",
                "coef": err_stats([(s1[1], ref)]),
                "recon": err_stats([(s1[2], orc.idwt1d(ref, L))])}
    ACCURACY.append(("signal_1d", None, check_signal))
    res["signal_1d"] = {"workload": f"1D fp32 signal n={sc.n}, {sc.levels} level, DWT+IDWT",
                        "us_per_round_trip": round(ms * 1e3, 2),
                        "us_per_round_trip_eager": round(ms_eager * 1e3, 2),
                        "gsamples_s": round(sc.n / (ms * 1e-3) / 1e9, 3),
                        "note": "launch-latency bound (two launches of 1 MiB traffic "
                                "in total); graph replay; data resident in L2"}
    res["signal_1d_batch"] = signal_batch_form(api, synth, dev)
    res["volume_3d"] = volume_form(api, synth, dev)
    res["filter_bank_1d"] = filter_form(api, synth, dev)
    res["denoise_2d"] = denoise2d_form(api, synth, dev)

    # precision form: 64 x 2048^2, 4 levels; bf16 / fp16 / u8-in vs fp32
    pc = synth.PrecisionBatch()
    distinct = 8
    base = np.stack([synth.piecewise_smooth_image(pc.h, pc.w, pc.seed, i)
                     for i in range(distinct)])
    x64 = torch.from_numpy(base).to(dev)
    rep = pc.batch // distinct
    xf = x64.float().repeat(rep, 1, 1)
    px = pc.batch * pc.h * pc.w
    entry = {"workload": f"{pc.batch} x {pc.h}x{pc.w} images ({distinct} distinct, repeated), "
                         f"{pc.levels}-level 2D DWT+IDWT, FP32 arithmetic"}
    for name, xdt, cdt, ydt in [("fp32", torch.float32, torch.float32, torch.float32),
                                ("bf16", torch.bfloat16, torch.bfloat16, torch.bfloat16),
                                ("fp16", torch.float16, torch.float16, torch.float16),
                                ("u8_in_bf16_coef_fp32_out", torch.uint8, torch.bfloat16,
                                 torch.float32)]:
        if xdt == torch.uint8:
            x = (xf.clamp(0, 1) * 255).round().to(torch.uint8)
        else:
            x = xf.to(xdt)
        c = torch.empty(x.shape, dtype=cdt, device=dev)
        y = torch.empty(x.shape, dtype=ydt, device=dev)
        plan = api.Plan(x, c, pc.levels, y)

        def rt():
            plan.dwt()
            plan.idwt()

        ms = time_med(rt)
        nbytes = px * (x.element_size() + 2 * c.element_size() + y.element_size())
        dwt_ms = time_med(plan.dwt)
        idwt_ms = time_med(plan.idwt)
        entry[name] = {"ms": round(ms, 4), "gsamples_s": round(px / (ms * 1e-3) / 1e9, 2),
                       "hbm_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                       "dwt_gbs": round(px * (x.element_size() + c.element_size())
                                        / (dwt_ms * 1e-3) / 1e9, 1),
                       "idwt_gbs": round(px * (c.element_size() + y.element_size())
                                         / (idwt_ms * 1e-3) / 1e9, 1)}
        # three images spread over the batch: the stored input (exactly what
        # the GPU read), its stored coefficients and reconstruction
        picks = (0, pc.batch * 37 // 64, pc.batch - 1)
        smp = [(host64(x[i]), host64(c[i]), host64(y[i])) for i in picks]

        def check(orc, smp=smp, L=pc.levels, picks=picks):
            refs = [orc.dwt2d(xi, L) for xi, _, _ in smp]
            rec = [orc.idwt2d(r, L) for r in refs]
            return {"vs": "FP64 oracle on the stored input values",
                    "sample": f"images {list(picks)} of the batch",
                    "coef": err_stats([(ci, r) for (_, ci, _), r in zip(smp, refs)]),
                    "recon": err_stats([(yi, r) for (_, _, yi), r in zip(smp, rec)])}
        ACCURACY.append(("precision", name, check))
        del x, c, y, plan
    for name in ("bf16", "fp16", "u8_in_bf16_coef_fp32_out"):
        entry[name]["speedup_vs_fp32"] = round(entry["fp32"]["ms"] / entry[name]["ms"], 3)
    res["precision"] = entry
    del xf, x64
    torch.cuda.empty_cache()

    res["ragged"] = ragged_form(api, synth, dev, entry["fp32"]["gsamples_s"])
    torch.cuda.empty_cache()
    res["backward"] = grad_form(api, synth, dev)
    torch.cuda.empty_cache()
    return res


def grad_form(api, synth, dev):
    """32 x 3 x 512 x 512 fp32, 3 levels: forward + backward of the wavelet
    denoising loss, fused (graph replay and eager autograd) and composed from
    separate differentiable ops, next to the plain fp32 DWT + IDWT round trip
    of the same batch."""
    import torch
    from paper_1002_2184_gb300 import autograd as ad
    gc_ = synth.GradBatch()
    B, C, H, W = gc_.shape
    imgs = [torch.from_numpy(synth.piecewise_smooth_image(H, W, gc_.seed, i).astype(np.float32))
            for i in range(8)]
    x = torch.stack([imgs[i % 8] for i in range(B * C)]).reshape(gc_.shape).to(dev)
    px = x.numel()
    L, t, lam = gc_.levels, gc_.threshold, gc_.l1_weight
    # four input sets (4 x (x + grad) = 800 MB > L2) rotate inside the graph,
    # so each step's forward reads its batch from DRAM; the backward re-reads
    # the same batch right after, as a training step would
    sets = 4
    xs = [x] + [x.roll(k, dims=0).contiguous() for k in range(1, sets)]
    plans = [ad.DenoisePlan(xk, L, t, lam) for xk in xs]
    for pl in plans:
        pl.forward()
        pl.backward()
    torch.cuda.synchronize()
    # one stream per set inside the graph (forked from and joined back to the
    # capture stream): sets are independent batches, so one set's read-only
    # forward can overlap another set's backward
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    side = [torch.cuda.Stream(dev) for _ in range(sets)]
    with torch.cuda.graph(g, stream=cap):
        for st in side:
            st.wait_stream(cap)
        for pl, st in zip(plans, side):
            pl.forward(st)
            pl.backward(stream=st)
        for st in side:
            cap.wait_stream(st)
    ms_graph = time_med(g.replay) / sets
    # each direction alone, 16 calls back to back on one stream over the
    # rotating sets, replayed as one graph: the forward (loss kernel + the
    # one-thread finalize) reads x, 4 B per pixel; the backward reads x and
    # writes the gradient, 8 B per pixel
    calls = 16

    def graphed(call):
        gg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gg):
            for k in range(calls):
                call(k % sets)
        return gg

    g_fwd = graphed(lambda k: plans[k].forward())
    g_bwd = graphed(lambda k: plans[k].backward())
    ms_fwd = time_med(g_fwd.replay) / calls
    ms_bwd = time_med(g_bwd.replay) / calls

    xr = x.clone().requires_grad_(True)

    def fused_eager():
        xr.grad = None
        ad.denoise_loss(xr, L, t, lam).backward()

    def unfused_eager():
        xr.grad = None
        ad.denoise_loss_unfused(xr, L, t, lam).backward()

    ms_fused = time_med(fused_eager)
    ms_unfused = time_med(unfused_eager)
    # loss and gradient of the whole batch from the fused kernels
    pl0 = plans[0]
    loss_gpu = float(pl0.forward().item())
    grad_gpu = host64(pl0.backward())
    x_host = host64(x)

    def check_grad(orc, x_host=x_host, loss_gpu=loss_gpu, grad_gpu=grad_gpu):
        loss_ref = orc.denoise_loss(x_host, L, t, lam)[0]
        g_ref = orc.denoise_loss_grad(x_host, L, t, lam)
        return {"vs": "FP64 oracle (closed-form gradient)", "sample": "the whole batch",
                "loss_gpu": loss_gpu, "loss_oracle": loss_ref,
                "loss_rel_err": abs(loss_gpu - loss_ref) / abs(loss_ref),
                "grad": err_stats([(grad_gpu, g_ref)])}
    ACCURACY.append(("backward", None, check_grad))
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    rt = api.Plan(x, c, L, y)
    ms_rt = time_med(lambda: (rt.dwt(), rt.idwt()))
    peaks = measured_peaks()
    hbm = (peaks or {}).get("hbm_gbs") or 6800.0
    gbs = 12.0 * px / (ms_graph * 1e-3) / 1e9
    return {"workload": f"{B}x{C}x{H}x{W} fp32, {L} levels, soft threshold {t}, L1 weight {lam}",
            "l2": f"{sets} rotating input sets in one graph, one stream each "
                  f"(per-step time = replay / {sets})",
            "fused_graph_ms": round(ms_graph, 4),
            "fused_graph_gsamples_s": round(px / (ms_graph * 1e-3) / 1e9, 2),
            "fused_hbm_gbs": round(gbs, 1), "fused_frac_of_hbm": round(gbs / hbm, 4),
            "fused_algorithmic_bytes_per_px": 12,
            "alone": f"{calls} calls on one stream over the {sets} sets, one graph replay",
            "forward_alone_ms": round(ms_fwd, 4),
            "forward_alone_frac_of_hbm": round(4.0 * px / (ms_fwd * 1e-3) / 1e9 / hbm, 4),
            "backward_alone_ms": round(ms_bwd, 4),
            "backward_alone_frac_of_hbm": round(8.0 * px / (ms_bwd * 1e-3) / 1e9 / hbm, 4),
            "fused_autograd_ms": round(ms_fused, 4),
            "unfused_autograd_ms": round(ms_unfused, 4),
            "plain_fp32_dwt_idwt_ms": round(ms_rt, 4),
            "fwd_bwd_over_plain_round_trip": round(ms_graph / ms_rt, 3)}


def _hbm():
    peaks = measured_peaks()
    return (peaks or {}).get("hbm_gbs") or 6800.0


def signal_batch_form(api, synth, dev):
    """64 signals of 2^20 fp32 samples (the signal generator), 8 levels:
    DWT + IDWT round trip and the one-pass shrinkage (soft threshold 1.0)."""
    import torch
    rows, n, L = 64, 1 << 20, 8
    base = [torch.from_numpy(synth.signal_1d(n, synth.Signal1D.seed, i).astype(np.float32))
            for i in range(4)]
    x = torch.stack([base[i % 4] for i in range(rows)]).to(dev)
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    plan = api.Plan(x, c, L, y, one_d=True)
    ms_rt = time_med(lambda: (plan.dwt(), plan.idwt()))
    ms_dn = time_med(lambda: api.denoise1d(x, L, 1.0, out=y))
    # the paper's comparison, existing vs fast, at scale: one level of the
    # undecimated direct form (every convolution output computed, 12 B per
    # sample) against the Fast Haar analysis (the decimated outputs only)
    u = torch.empty((rows, 2, n), dtype=x.dtype, device=dev)
    p1 = api.Plan(x, c, 1, y, one_d=True)
    ms_direct = time_med(lambda: api.swt1d(x, 1, out=u))
    ms_fast = time_med(p1.dwt)
    same = bool(torch.equal(u[:, 1, ::2], c[:, n // 2:]))
    px = rows * n
    hbm = _hbm()
    return {"workload": f"{rows} x 2^20 fp32 signals, {L} levels",
            "existing_vs_fast_1_level": {"undecimated_ms": round(ms_direct, 4),
                                         "fast_haar_ms": round(ms_fast, 4),
                                         "ratio": round(ms_direct / ms_fast, 3),
                                         "decimated_direct_equals_fast": same},
            "round_trip_ms": round(ms_rt, 4),
            "round_trip_gsamples_s": round(px / (ms_rt * 1e-3) / 1e9, 2),
            "round_trip_frac_of_hbm": round(16.0 * px / (ms_rt * 1e-3) / 1e9 / hbm, 4),
            "denoise_ms": round(ms_dn, 4),
            "denoise_gsamples_s": round(px / (ms_dn * 1e-3) / 1e9, 2),
            "denoise_frac_of_hbm": round(8.0 * px / (ms_dn * 1e-3) / 1e9 / hbm, 4),
            "denoise_bytes_per_sample": 8}


def lattice_taps(angles):
    """An orthonormal low-pass of length 2 * len(angles) from a paraunitary
    lattice of plane rotations and two-sample delays (each stage keeps the
    double-shift orthogonality the bank's perfect reconstruction needs)."""
    c, s = np.cos(angles[0]), np.sin(angles[0])
    h0, h1 = np.array([c, s]), np.array([-s, c])
    for th in angles[1:]:
        c, s = np.cos(th), np.sin(th)
        a, b = np.concatenate([h0, [0.0, 0.0]]), np.concatenate([[0.0, 0.0], h1])
        h0, h1 = c * a + s * b, -s * a + c * b
    return tuple(float(v) for v in h0)


def filter_form(api, synth, dev):
    """The same polyphase bank with longer orthonormal low-pass filters:
    64 x 2^20 fp32 signals, 8 levels, DWT + IDWT, K = 2 (Haar), 4
    (Daubechies-4) and 8 (a lattice filter) through the general K-tap
    kernels; the round trip and each direction alone (back-to-back
    launches)."""
    import torch
    rows, n, L = 64, 1 << 20, 8
    base = [torch.from_numpy(synth.signal_1d(n, synth.Signal1D.seed, i).astype(np.float32))
            for i in range(4)]
    x = torch.stack([base[i % 4] for i in range(rows)]).to(dev)
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    px = rows * n
    out = {"workload": f"{rows} x 2^20 fp32 signals, {L} levels, DWT + IDWT, periodic"}
    for name, taps in (("haar_k2", api.HAAR2), ("daubechies4_k4", api.DAUBECHIES4),
                       ("lattice_k8", lattice_taps([0.2, 0.5, -0.4, 0.9]))):
        ms = time_med(lambda: (api.filter_dwt1d(x, L, taps, out=c),
                               api.filter_idwt1d(c, L, taps, out=y)))
        ok = float(torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)) <= 1e-6
        dwt_ms = time_med(lambda: api.filter_dwt1d(x, L, taps, out=c))
        idwt_ms = time_med(lambda: api.filter_idwt1d(c, L, taps, out=y))
        out[name] = {"ms": round(ms, 4), "gsamples_s": round(px / (ms * 1e-3) / 1e9, 2),
                     "frac_of_hbm": round(16.0 * px / (ms * 1e-3) / 1e9 / _hbm(), 4),
                     "dwt_frac_of_hbm": round(8.0 * px / (dwt_ms * 1e-3) / 1e9 / _hbm(), 4),
                     "idwt_frac_of_hbm": round(8.0 * px / (idwt_ms * 1e-3) / 1e9 / _hbm(), 4),
                     "round_trip_ok": ok}
    # short rows: 16384 signals of 4096 samples, one chunk each, so every
    # staged window wraps around its row
    xs = x.reshape(-1, 4096)
    cs, ys = c.reshape(-1, 4096), y.reshape(-1, 4096)
    taps = api.DAUBECHIES4
    dwt_ms = time_med(lambda: api.filter_dwt1d(xs, L, taps, out=cs))
    idwt_ms = time_med(lambda: api.filter_idwt1d(cs, L, taps, out=ys))
    ok = float(torch.linalg.vector_norm(ys - xs) / torch.linalg.vector_norm(xs)) <= 1e-6
    out["daubechies4_k4_16384x4096"] = {
        "dwt_frac_of_hbm": round(8.0 * px / (dwt_ms * 1e-3) / 1e9 / _hbm(), 4),
        "idwt_frac_of_hbm": round(8.0 * px / (idwt_ms * 1e-3) / 1e9 / _hbm(), 4),
        "round_trip_ok": ok}
    return out


def volume_form(api, synth, dev):
    """3D: a 512^3 fp32 volume (slices of the image generator; 512 MiB, larger
    than L2), 3 levels, DWT + IDWT round trip."""
    import torch
    side, L = 512, 3
    sl = [torch.from_numpy(synth.piecewise_smooth_image(side, side, 77, i).astype(np.float32))
          for i in range(8)]
    x = torch.stack([sl[i % 8] for i in range(side)]).to(dev)
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    ms = time_med(lambda: (api.dwt3d(x, L, out=c), api.idwt3d(c, L, out=y)))
    ok = float(torch.linalg.vector_norm(y - x) / torch.linalg.vector_norm(x)) <= 1e-6
    px = x.numel()
    return {"workload": f"{side}^3 fp32 volume, {L} levels, DWT + IDWT",
            "ms": round(ms, 4), "gsamples_s": round(px / (ms * 1e-3) / 1e9, 2),
            "frac_of_hbm": round(16.0 * px / (ms * 1e-3) / 1e9 / _hbm(), 4), "round_trip_ok": ok}


def denoise2d_form(api, synth, dev):
    """One-pass soft shrinkage (t = 0.05, 5 levels) of 4 x 4096 x 4096 fp32
    images next to the DWT + IDWT round trip of the same batch."""
    import torch
    cfg = synth.Image2D()
    im = torch.from_numpy(synth.piecewise_smooth_image(cfg.h, cfg.w, cfg.seed, 0)
                          .astype(np.float32)).to(dev)
    x = im.expand(4, cfg.h, cfg.w).contiguous()
    y = torch.empty_like(x)
    c = torch.empty_like(x)
    plan = api.Plan(x, c, cfg.levels, y)
    ms_rt = time_med(lambda: (plan.dwt(), plan.idwt()))
    ms_dn = time_med(lambda: api.denoise2d(x, cfg.levels, 0.05, out=y))
    px = x.numel()
    hbm = _hbm()
    return {"workload": f"4 x {cfg.h}x{cfg.w} fp32 images, {cfg.levels} levels, soft t=0.05",
            "denoise_ms": round(ms_dn, 4),
            "denoise_gsamples_s": round(px / (ms_dn * 1e-3) / 1e9, 2),
            "denoise_frac_of_hbm": round(8.0 * px / (ms_dn * 1e-3) / 1e9 / hbm, 4),
            "round_trip_ms": round(ms_rt, 4),
            "speedup_vs_round_trip": round(ms_rt / ms_dn, 3)}


def ragged_form(api, synth, dev, dense_fp32_gsamples):
    """512 images, sides uniform on {64, ..., 2048}, levels 3..6: one
    persistent launch per direction (autotuned unit shape and grid, replayed
    from a CUDA graph) against a per-image loop of the plain path."""
    import torch
    from paper_1002_2184_gb300 import autotune
    rc = synth.RaggedBatch()
    items = synth.ragged_shapes(rc)
    px = sum(h * w for h, w, _ in items)
    # inputs: crops of 8 distinct 2048 x 2048 piecewise-smooth images
    base = [torch.from_numpy(synth.piecewise_smooth_image(2048, 2048, rc.seed, i)
                             .astype(np.float32)).to(dev) for i in range(8)]
    probe = api.RaggedPlan(items, dev)
    x = probe.empty()
    for i, v in enumerate(probe.views(x)):
        h, w, _ = items[i]
        v.copy_(base[i % 8][:h, :w])
    del base
    unit, bps, rep = autotune.tune_ragged(items, dev, x, reps=3, use_cache=False)
    plan = api.RaggedPlan(items, dev, unit, bps)
    c = plan.empty()
    y = plan.empty()
    plan.dwt(x, c)
    plan.idwt(c, y)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.dwt(x, c)
        plan.idwt(c, y)
    ms = time_med(g.replay)
    ok = plan.status() == 0
    err = float(torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double()))
    picks = sorted(np.random.default_rng(2184).choice(len(items), size=6, replace=False).tolist())
    xv_, cv_, yv_ = plan.views(x), plan.views(c), plan.views(y)
    smp = [(host64(xv_[i]), host64(cv_[i]), host64(yv_[i]), items[i][2]) for i in picks]

    def check_ragged(orc, smp=smp, picks=picks):
        refs = [orc.dwt2d(xi, L) for xi, _, _, L in smp]
        rec = [orc.idwt2d(r, L) for r, (_, _, _, L) in zip(refs, smp)]
        return {"vs": "FP64 oracle", "sample": f"images {picks} "
                f"({', '.join(f'{a.shape[0]}x{a.shape[1]} L{L}' for a, _, _, L in smp)})",
                "coef": err_stats([(ci, r) for (_, ci, _, _), r in zip(smp, refs)]),
                "recon": err_stats([(yi, r) for (_, _, yi, _), r in zip(smp, rec)])}
    ACCURACY.append(("ragged", None, check_ragged))
    # the plain path: one strided-batch plan per image, launched one by one
    per = [api.Plan(xv, cv, items[i][2], yv) for i, (xv, cv, yv) in
           enumerate(zip(plan.views(x), plan.views(c), plan.views(y)))]

    def loop():
        for p_ in per:
            p_.dwt()
            p_.idwt()

    ms_loop = time_med(loop, warmup=1)
    peaks = measured_peaks()
    hbm = (peaks or {}).get("hbm_gbs") or 6800.0
    gbs = 16.0 * px / (ms * 1e-3) / 1e9
    return {"workload": f"{len(items)} fp32 images, sides uniform on {{64..2048}} step 64, "
                        f"levels 3..6, {px} px",
            "ms": round(ms, 4), "gsamples_s": round(px / (ms * 1e-3) / 1e9, 2),
            "hbm_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 4),
            "unit": rep["unit_name"], "blocks_per_sm": bps,
            "autotune_ms": rep["timings"], "graph_replay": True, "queue_ok": ok,
            "round_trip_rel_l2": err,
            "per_image_loop_ms": round(ms_loop, 3),
            "speedup_vs_per_image_loop": round(ms_loop / ms, 2),
            "vs_dense_fp32_gsamples": round(px / (ms * 1e-3) / 1e9 / dense_fp32_gsamples, 3)}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def rows_once():
    """Each row's main operation once, on cases larger than L2, for an ncu
    capture of the kernels behind every row: the headline image (4096^2
    fp32, 5-level DWT + IDWT), the ragged batch (first 64 images of the
    ragged shape list), the fused loss (32 x 3 x 512^2), 1D signals
    (64 x 2^20: 8-level DWT + IDWT, shrinkage, one undecimated level,
    Daubechies-4 bank, 8-tap lattice bank), 2D shrinkage (4 x 4096^2), bf16
    2D (64 x 2048^2, 4 levels), uint8 -> bf16 analysis of the same batch and
    a 512^3 volume (3 levels)."""
    import torch
    from paper_1002_2184_gb300 import api, build, synth
    from paper_1002_2184_gb300 import autograd as ad
    build.build()
    dev = torch.device("cuda", 0)
    torch.manual_seed(0)
    x = torch.rand(4096, 4096, device=dev)
    c, y = torch.empty_like(x), torch.empty_like(x)
    ph = api.Plan(x, c, 5, y)
    ph.dwt()
    ph.idwt()
    del x, c, y, ph
    rp = api.RaggedPlan(synth.ragged_shapes()[:64], dev, 0, 6)
    xr = rp.empty()
    xr.normal_()
    cr, yr = rp.empty(), rp.empty()
    rp.dwt(xr, cr)
    rp.idwt(cr, yr)
    del xr, cr, yr
    gb = synth.GradBatch()
    x = torch.randn(gb.shape, device=dev) * 0.3 + 0.5
    pl = ad.DenoisePlan(x, gb.levels, gb.threshold, gb.l1_weight)
    pl.forward()
    pl.backward()
    del x, pl
    x = torch.randn(64, 1 << 20, device=dev)
    c, y = torch.empty_like(x), torch.empty_like(x)
    p1 = api.Plan(x, c, 8, y, one_d=True)
    p1.dwt()
    p1.idwt()
    api.denoise1d(x, 8, 1.0, out=y)
    api.swt1d(x, 1, out=torch.empty(64, 2, 1 << 20, device=dev))
    api.filter_dwt1d(x, 8, api.DAUBECHIES4, out=c)
    api.filter_idwt1d(c, 8, api.DAUBECHIES4, out=y)
    k8 = lattice_taps([0.2, 0.5, -0.4, 0.9])
    api.filter_dwt1d(x, 8, k8, out=c)
    api.filter_idwt1d(c, 8, k8, out=y)
    del x, c, y
    x = torch.randn(4, 4096, 4096, device=dev)
    api.denoise2d(x, 5, 0.05, out=torch.empty_like(x))
    del x
    x = torch.randn(64, 2048, 2048, device=dev, dtype=torch.bfloat16)
    c, y = torch.empty_like(x), torch.empty_like(x)
    pb = api.Plan(x, c, 4, y)
    pb.dwt()
    pb.idwt()
    u = (torch.rand(64, 2048, 2048, device=dev) * 255).to(torch.uint8)
    pu = api.Plan(u, c, 4)
    pu.dwt()
    del x, c, y, u
    x = torch.randn(512, 512, 512, device=dev)
    c, y = torch.empty_like(x), torch.empty_like(x)
    api.dwt3d(x, 3, out=c)
    api.idwt3d(c, 3, out=y)
    torch.cuda.synchronize()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1002_2184_gb300 import synth
    import oracle
    cfg = synth.Image2D()
    H, W, L = cfg.h, cfg.w, cfg.levels
    img = synth.piecewise_smooth_image(H, W, cfg.seed, 0).astype(np.float32).astype(np.float64)
    # each step: DWT + IDWT of the full image, as the GPU arm's step
    oracle.lib()
    for k in range(args.warmup):
        oracle.idwt2d(oracle.dwt2d(img, L), L)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.idwt2d(oracle.dwt2d(img, L), L)
    el = time.perf_counter() - t0
    value = H * W * args.steps / el / 1e9
    sample = (f"each step: DWT+IDWT of the full {H}x{W} image, {L} levels, FP64 C oracle, "
              "one thread")
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"2D fp32 image {H}x{W}, {L}-level DWT then full IDWT",
                   "h": H, "w": W, "levels": L, "batch_per_gpu": 1,
                   "parallelism": "host CPU, one thread"},
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.rows_once:
        rows_once()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
