"""Benchmark of the P-SPIR hot path on the 3D ring workload.

Workload (RING3D): 24 blocks x 13 x 13 crystals x 4 block rings (312 crystals
per ring, 52 rings), 1.9 mm crystals on a 2.2 mm pitch, radius 130 mm; 8 x 8
entry sub-positions, 32 x 8 angle nodes; 44,732,688 LORs (ring difference
<= 15, fan +-104); spread +-3 x +-3 crystals; 160 x 160 x 104 voxels of
0.8 mm; seeded uniform-cylinder phantom.

One step = one pass of the whole hot path: response table, class spreads,
geometric rows G (count, scan, fill), sensitivity A^T 1 and one MLEM iteration
(forward y = S G x, ratio, back-projection G^T S^T r, update).  The matrix
(~32 GB) is regenerated every step, so inputs are far larger than L2.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "RING3D"
METRIC = "PSF matrix nonzeros/s (psf_sysmat_rows, whole step) and PSF fwd+back LOR*voxel/s"
UNIT = "nnz/s"


def _env_int(k, d):
    return int(os.environ.get(k, d))


def dist_info():
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    return rank, world, local


def job_rate(total_ms: float, units_per_rank: float, device) -> tuple:
    """Whole-job throughput of replicas: the slowest rank's time (max over
    ranks) and the units all ranks processed divided by it.  Single process:
    the local time."""
    import torch

    world = 1
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        world = torch.distributed.get_world_size()
        tt = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = tt.item()
    return total_ms, world * units_per_rank / (total_ms * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU leg
def cpu_sample(n_tclass: int = 2, batch: int = 48):
    """Time the FP64 oracle on a bounded sample of the workload.

    The sample is n_tclass transaxial spread classes with all their members:
    every rotation of each class's crystal pair by whole blocks (24) times all
    1,372 ring pairs, and the spreads of those classes for all 31 ring
    differences.  The oracle builds the table once, then, `batch` classes at a
    time (bounded host memory), the spreads (one per class, the same
    amortisation as the full job), the chord rows, and projects forward and
    back with them.  Returns (nnz/s, seconds, threads, description)."""
    import numpy as np

    import oracle
    from paper_1607_06170_gb300 import inputs as I

    oracle.build()
    w = I.workload(WORKLOAD)
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    nt, nb, R = I.n_transaxial(s), s["nt_block"], s["n_blocks"]
    tp = I.transaxial_pairs(s, w["lors"]["fan_half"])
    cls = tp[tp[:, 0] < nb]
    # classes at evenly spaced quantiles of the list (central to oblique chords)
    pick = cls[((np.arange(n_tclass) + 0.5) / n_tclass * len(cls)).astype(int)]
    rp = I.ring_pairs(s, w["lors"]["max_ring_diff"]).astype(np.int64)
    Dm = w["lors"]["max_ring_diff"]
    x = I.phantom_cylinder(im, 1).reshape(-1).astype(np.float64)
    nv = x.size
    n_lors = nnz = n_reps = 0
    dt = 0.0
    t0 = time.perf_counter()
    T, _ = oracle.table_build(s, t)
    dt += time.perf_counter() - t0
    for c0 in range(0, len(pick), batch):
        lors, reps = [], []
        for a, b in pick[c0:c0 + batch]:
            for k in range(R):
                ta, tb_ = (a + k * nb) % nt, (b + k * nb) % nt
                lo, hi = min(ta, tb_), max(ta, tb_)
                ra_, rb_ = (rp[:, 0], rp[:, 1]) if ta < tb_ else (rp[:, 1], rp[:, 0])
                lors.append(np.stack([ra_ * nt + lo, rb_ * nt + hi], 1))
            for d in range(-Dm, Dm + 1):
                ra = max(0, -d)
                reps.append((ra * nt + a, (ra + d) * nt + b))
        lors = np.concatenate(lors).astype(np.int32)
        reps = np.array(reps, dtype=np.int32)
        t0 = time.perf_counter()
        oracle.spread(s, t, T, reps, Wt, Wa)
        G = oracle.rows_geom(s, im, lors)
        y = oracle.csr_fwd(G, x)
        oracle.csr_back(G, y, nv)
        dt += time.perf_counter() - t0
        n_lors += len(lors)
        nnz += int(G[0][-1])
        n_reps += len(reps)
        del G, y
    desc = (f"{n_lors} LORs ({n_tclass} transaxial classes x {R} rotations x {len(rp)} ring "
            f"pairs, {nnz} nnz) + {n_reps} class spreads + table; rows, forward, back")
    return nnz / dt, dt, oracle.threads(), desc


def run_reference(args):
    rank, world, _ = dist_info()
    if world > 1 and rank != 0:
        return
    # each step: the oracle on one bounded sample (one transaxial class)
    for _ in range(args.warmup):
        cpu_sample(16)
    rates, times = [], []
    desc, cores = "", 1
    for _ in range(args.steps):
        r, dt, cores, desc = cpu_sample(16)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
def stencil_pairs(s, ls, Wt, Wa):
    """Exact number of (output LOR, source LOR) products in one application of
    the spread S over a structured LOR set: transaxial (pair, partner) pairs
    in the set times axial (ring pair, ring pair) pairs in the set."""
    import numpy as np

    from paper_1607_06170_gb300 import inputs as I

    nt, F, Dm = I.n_transaxial(s), ls["fan_half"], ls["max_ring_diff"]
    tp = I.transaxial_pairs(s, F)
    a, b = tp[:, 0].astype(np.int64), tp[:, 1].astype(np.int64)
    n_t = 0
    for d1 in range(-Wt, Wt + 1):
        for d2 in range(-Wt, Wt + 1):
            pa, pb = (a - d1) % nt, (b - d2) % nt
            d = np.abs(pa - pb)
            n_t += int(((pa != pb) & (d >= nt // 2 - F) & (d <= nt // 2 + F)).sum())
    nr = I.n_rings(s)
    ra, rb = np.meshgrid(np.arange(nr), np.arange(nr), indexing="ij")
    n_a = 0
    for o1 in range(-Wa, Wa + 1):
        for o2 in range(-Wa, Wa + 1):
            sa, sb = ra - o1, rb - o2
            ok = (np.abs(ra - rb) <= Dm) & (sa >= 0) & (sa < nr) & (sb >= 0) & (sb < nr)
            n_a += int((ok & (np.abs(sa - sb) <= Dm)).sum())
    return n_t * n_a


# kernel -> (bound, algorithmic work per launch, unit): bytes a launch must move
# through HBM, or FP32 FLOPs it must execute
def n_comp_classes(s, ls):
    """Classes that are the smallest index of their orbit under the axial and
    transaxial reflections (the ones psf_bin_spread_classes computes)."""
    Nb = s["nt_block"]
    Nt = s["n_blocks"] * Nb
    F, Dm = ls["fan_half"], ls["max_ring_diff"]
    D = 2 * Dm + 1
    lo = [max(a + Nt // 2 - F, a + 1) for a in range(Nb)]
    start = [0]
    for a in range(Nb):
        start.append(start[-1] + max(min(a + Nt // 2 + F, Nt - 1) - lo[a] + 1, 0))

    def t_image(tp):
        a0 = max(a for a in range(Nb) if start[a] <= tp)
        b0 = lo[a0] + tp - start[a0]
        ma, mb = (Nb - 1 - a0) % Nt, (Nb - 1 - b0) % Nt
        sw = ma > mb
        a1, b1 = (mb, ma) if sw else (ma, mb)
        a10 = a1 % Nb
        return start[a10] + (b1 - (a1 - a10)) - lo[a10], sw

    n = 0
    for tp in range(start[Nb]):
        tpt, sw = t_image(tp)
        for d in range(-Dm, Dm + 1):
            dt = -d if sw else d
            c = tp * D + d + Dm
            n += c == min(c, tp * D - d + Dm, tpt * D + dt + Dm, tpt * D - dt + Dm)
    return n


def kernel_model(name, s, t, ls, Wt, Wa, n_lors, n_cls, nnz, nv, vb=4):
    # vb: bytes of a stored value (4 FP32; 2 for BF16/FP16 rows, which add a
    # 4-byte FP32 scale per row)
    ent = (4.0 + vb) * nnz + (4.0 * n_lors if vb < 4 else 0.0)
    if name == "set_fill_kernel":  # writes column + chord, reads row_ptr
        return "hbm", ent + 8.0 * n_lors, "GB/s"
    if name.startswith("csr_fwd"):  # column + value, row_ptr, LOR value, image
        return "hbm", ent + 12.0 * n_lors + 4.0 * nv, "GB/s"
    if name.startswith(("csr_back_pair", "csr_back_patch")):
        # column + value, row_ptr, two LOR values, image pair
        return "hbm", ent + 16.0 * n_lors + 8.0 * nv, "GB/s"
    if name == "spread_q_kernel":  # one FMA per sub-LOR and quadrant entry pair
        # of the classes the kernel computes (one per orbit of the two reflections)
        nsub = (t["n_sub_t"] * t["n_sub_a"]) ** 2
        return "alu", 2.0 * n_comp_classes(s, ls) * nsub * ((Wt + 1) * (Wa + 1)) ** 2, "TFLOP/s"
    if name.startswith("stencil"):  # one FMA per (output LOR, source LOR) pair
        return "alu", 2.0 * stencil_pairs(s, ls, Wt, Wa), "TFLOP/s"
    return None, None, None


def kernel_traffic(name):
    """DRAM bytes per launch from the committed ncu capture of this kernel,
    or None when one of the kernel's source files (the record's "source", a
    path or a list of paths; sha1 of their concatenated bytes) has changed
    since the capture."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))[name]
        srcs = rec["source"] if isinstance(rec["source"], list) else [rec["source"]]
        src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in srcs)
    except (OSError, ValueError, KeyError):
        return None
    if hashlib.sha1(src).hexdigest() != rec["sha1"]:
        return None
    return rec["bytes_per_launch"]


def kern_hbm_first(name, kern):
    """Sort key of the mixed step's roofline kernel: the HBM-bound kernel with
    the most device time (the 16-bit rows change only the HBM-bound kernels)."""
    hbm = name == "set_fill_kernel" or name.startswith(("csr_fwd", "csr_back_pair",
                                                          "csr_back_patch"))
    return (hbm, kern[name]["ms_per_step"])


def roofline(name, ms_per_launch, peaks, clocks, s, t, ls, Wt, Wa, n_lors, n_cls, nnz, nv,
             vb=4):
    bound, work, unit = kernel_model(name, s, t, ls, Wt, Wa, n_lors, n_cls, nnz, nv, vb)
    out = {"kernel": name, "ms_per_launch": ms_per_launch, "bound": bound}
    if bound is None:
        return out
    sm_mhz = float(clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0))
    if bound == "hbm":
        peak, src = float(peaks.get("hbm_gbs", 6800.0)), "measured" if peaks else "fallback"
        achieved = work / 1e9 / (ms_per_launch * 1e-3)
    else:  # FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x sampled SM clock
        peak, src = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12, "derived"
        achieved = work / 1e12 / (ms_per_launch * 1e-3)
    tr = kernel_traffic(name) if vb == 4 else None
    out.update({"achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": tr / 1e9 if tr is not None else None, "traffic_unit": "GB",
                "work_per_launch": work, "peak_source": src})
    return out


def run_gpu(args):
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    w = I.workload(WORKLOAD)
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    n_lors, n_cls = P.lor_set_size(s, ls)
    # replicas: every rank runs the whole workload on its own GPU
    x_host = torch.from_numpy(I.phantom_cylinder(im, 1).reshape(-1)).pin_memory()
    x = x_host.to(dev)
    L = P.lor_set_list(s, ls, device=dev)
    row_ptr = torch.empty(n_lors + 1, dtype=torch.int64, device=dev)
    # size query once, then buffers of that capacity are reused by every step
    _, col, val = P.sysmat_rows_set(s, im, ls, device=dev)
    nnz = col.numel()
    st = torch.cuda.current_stream()
    stages = ["table", "classes", "spread", "rows", "forward", "ratio", "back_sens", "update"]
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for k in stages}
    y_meas = None

    def step(x_in, y_in, record=None, inputs_ready=None):
        def mark(k, i):
            if record is not None:
                ev[k][i].record(st)

        mark("table", 0)
        T, eta = P.response_build(s, t, device=dev)
        mark("table", 1)
        mark("classes", 0)
        C = P.lor_set_classes(s, ls, device=dev)
        mark("classes", 1)
        mark("spread", 0)
        WC = P.bin_spread_classes(s, t, T, eta, ls, C, Wt, Wa)
        mark("spread", 1)
        mark("rows", 0)
        P.sysmat_rows_set(s, im, ls, buffers=(row_ptr, col, val))
        mark("rows", 1)
        M.set_spread(s, ls, Wt, Wa, WC)
        if inputs_ready is not None:  # image and data copied on a side stream
            st.wait_event(inputs_ready)
        # one MLEM iteration from the current image, with the sensitivity image
        # A^T 1 formed in the same pass over the rows as the back-projection
        mark("forward", 0)
        yh = M.forward(x_in)
        mark("forward", 1)
        mark("ratio", 0)
        r = P.em_ratio(y_in, yh)
        mark("ratio", 1)
        mark("back_sens", 0)
        bp, sens = M.back_sens(r)
        mark("back_sens", 1)
        mark("update", 0)
        x_out = x_in.clone()
        P.em_update(x_out, bp, sens, 1e-12)
        mark("update", 1)
        return x_out

    # one projector plan over the reused CSR buffers; measured data = noiseless
    # projection of the phantom (computed once)
    M = P.Matrix(row_ptr, col, val, nv).set_image(im)
    T0, e0 = P.response_build(s, t, device=dev)
    WC0 = P.bin_spread_classes(s, t, T0, e0, ls, P.lor_set_classes(s, ls, device=dev), Wt, Wa)
    P.sysmat_rows_set(s, im, ls, buffers=(row_ptr, col, val))
    M.set_spread(s, ls, Wt, Wa, WC0)
    M.autotune()  # launch choices of the projector kernels (CUDA-event timed, once)
    if args.stencil_form is not None:  # pinned (profiling runs: ncu's per-launch gaps
        M.set_stencil_form(args.stencil_form)  # skew the timing of the 3-launch form 5)
    y_meas = M.forward(x).clone()
    y_host = y_meas.cpu().pin_memory()
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(x, y_meas)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    P.timing_enable(True)  # CUDA events around every library kernel launch
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    stage_ms = {k: [] for k in stages}
    torch.cuda.synchronize()
    t0.record(st)
    xi = x
    for _ in range(args.steps):
        xi = step(x, y_meas, record=True)
        torch.cuda.synchronize()  # rows stage synchronises anyway; read stage events
        for k in stages:
            stage_ms[k].append(ev[k][0].elapsed_time(ev[k][1]))
    t1.record(st)
    torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    clocks = clk.stop()
    ktimes = P.timing_read()
    P.timing_enable(False)
    total_ms, value = job_rate(total_ms, nnz * args.steps, dev)
    ms_step = total_ms / args.steps
    med = {k: statistics.median(v) for k, v in stage_ms.items()}
    rows_rate = nnz / (med["rows"] * 1e-3)
    # LOR x voxel products of the projections: forward (nnz), back and
    # sensitivity (nnz each, one pass) over their stage times
    fb = 3 * nnz / ((med["forward"] + med["back_sens"]) * 1e-3)

    # end to end through the public API with host buffers: the pinned output
    # buffer and the copy stream are made once, one untimed step warms the
    # device allocator's cache for the per-step input copies, then each timed
    # step copies its inputs up, runs, and copies the image back
    e2e_steps = max(1, min(args.steps, 3))
    out_host = torch.empty(x_host.shape, dtype=x_host.dtype, pin_memory=True)
    copy_st = torch.cuda.Stream(device=dev)

    def e2e_step():
        # the step's inputs go up on a side stream while the table, spreads and
        # rows are computed; the projections wait for them
        copy_st.wait_stream(st)
        with torch.cuda.stream(copy_st):
            xd = x_host.to(dev, non_blocking=True)
            yd = y_host.to(dev, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(copy_st)
        xd.record_stream(st)
        yd.record_stream(st)
        xo = step(xd, yd, inputs_ready=ready)
        out_host.copy_(xo, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    # the slowest rank's wall time, the units of all ranks
    _, e2e_rate = job_rate((time.perf_counter() - te) * 1e3, nnz * e2e_steps, dev)
    e2e = {"value": e2e_rate, "unit": UNIT,
           "h2d_bytes_per_step": int(x_host.numel() * 4 + y_host.numel() * 4),
           "d2h_bytes_per_step": int(out_host.numel() * 4)}

    # the plain FP32 GPU form of the same step (outside the timed region): the
    # per-LOR tracer instead of the structured-set generator, grid-stride CSR
    # projectors, the plain one-output-per-thread stencil, and the sensitivity
    # as a separate back-projection of ones; same spread kernel
    Mp = P.Matrix(row_ptr, col, val, nv)
    plain_stages = ["table", "classes", "spread", "rows", "forward", "ratio", "back", "sens",
                    "update"]
    pev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for k in plain_stages}

    def plain_step(x_in, y_in):
        def mark(k, i):
            pev[k][i].record(st)

        mark("table", 0)
        T, eta = P.response_build(s, t, device=dev)
        mark("table", 1)
        mark("classes", 0)
        C = P.lor_set_classes(s, ls, device=dev)
        mark("classes", 1)
        mark("spread", 0)
        WC = P.bin_spread(s, t, T, eta, C, Wt, Wa)
        mark("spread", 1)
        mark("rows", 0)
        P.sysmat_rows(s, im, L, buffers=(row_ptr, col, val, None))
        mark("rows", 1)
        Mp.set_spread(s, ls, Wt, Wa, WC).set_launch(0).set_stencil_form(1)
        mark("forward", 0)
        yh = Mp.forward(x_in)
        mark("forward", 1)
        mark("ratio", 0)
        r = P.em_ratio(y_in, yh)
        mark("ratio", 1)
        mark("back", 0)
        bp = Mp.back(r)
        mark("back", 1)
        mark("sens", 0)
        sens = Mp.back(torch.ones_like(r))
        mark("sens", 1)
        mark("update", 0)
        x_out = x_in.clone()
        P.em_update(x_out, bp, sens, 1e-12)
        mark("update", 1)
        return x_out

    plain_step(x, y_meas)  # warm-up
    torch.cuda.synchronize()
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(st)
    plain_step(x, y_meas)
    pb.record(st)
    torch.cuda.synchronize()
    plain_ms = pa.elapsed_time(pb)
    plain = {"ms_per_step": plain_ms, "value": nnz / (plain_ms * 1e-3), "unit": UNIT,
             "speedup": plain_ms / ms_step,
             "stage_ms": {k: pev[k][0].elapsed_time(pev[k][1]) for k in plain_stages},
             "form": "per-LOR tracer rows, grid-stride CSR projectors, plain stencil, "
                     "sensitivity as a back-projection of ones; same spread kernel"}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass

    # the same step with mixed-precision G rows (outside the timed region):
    # BF16 values with a per-row FP32 scale, FP32 accumulation; columns and row
    # pointers are those of the FP32 rows (the same buffers are rewritten)
    mixed = None
    if not args.no_mixed:
        del Mp
        Mp = None
        val16 = torch.empty(nnz, dtype=torch.bfloat16, device=dev)
        scale16 = torch.empty(n_lors, dtype=torch.float32, device=dev)
        Mm = P.Matrix(row_ptr, col, val16, nv, row_scale=scale16).set_image(im)

        def mixed_step(x_in, y_in):
            T, eta = P.response_build(s, t, device=dev)
            C = P.lor_set_classes(s, ls, device=dev)
            WC = P.bin_spread_classes(s, t, T, eta, ls, C, Wt, Wa)
            P.sysmat_rows_set_typed(s, im, ls, "bf16", buffers=(row_ptr, col, val16, scale16))
            Mm.set_spread(s, ls, Wt, Wa, WC)
            yh = Mm.forward(x_in)
            r = P.em_ratio(y_in, yh)
            bp, sens = Mm.back_sens(r)
            x_out = x_in.clone()
            P.em_update(x_out, bp, sens, 1e-12)
            return x_out

        P.sysmat_rows_set_typed(s, im, ls, "bf16", buffers=(row_ptr, col, val16, scale16))
        Mm.set_spread(s, ls, Wt, Wa, WC0)
        Mm.autotune()
        if args.stencil_form is not None:
            Mm.set_stencil_form(args.stencil_form)
        for _ in range(max(1, args.warmup)):
            mixed_step(x, y_meas)
        torch.cuda.synchronize()
        P.timing_enable(True)
        ma, mb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ma.record(st)
        for _ in range(args.steps):
            xm = mixed_step(x, y_meas)
        mb.record(st)
        torch.cuda.synchronize()
        mixed_ms = ma.elapsed_time(mb) / args.steps
        mk = P.timing_read()
        P.timing_enable(False)
        mkern = {k: {"launches_per_step": n / args.steps, "ms_per_step": ms / args.steps,
                     "ms_per_launch": ms / n} for k, (n, ms) in mk.items()}
        mtop = max(mkern, key=lambda k: kern_hbm_first(k, mkern))
        # the updated image against the FP32 step's from the same input
        rel = float((xm - xi).norm() / xi.norm())
        mixed = {"dtype": "bf16", "row_scale": "f32", "accumulate": "f32",
                 "ms_per_step": mixed_ms, "value": nnz / (mixed_ms * 1e-3), "unit": UNIT,
                 "speedup_vs_f32_step": ms_step / mixed_ms,
                 "image_rel_l2_vs_f32_step": rel,
                 "kernels": {k: v["ms_per_step"] for k, v in mkern.items()},
                 "roofline": roofline(mtop, mkern[mtop]["ms_per_launch"], peaks, clocks, s, t,
                                      ls, Wt, Wa, n_lors, n_cls, nnz, nv, vb=2)}
        del Mm, val16, scale16

    # roofline of the dominant kernel: the library kernel with the most device
    # time per step (CUDA events around each launch, timed region only)
    kern = {k: {"launches_per_step": n / args.steps, "ms_per_step": ms / args.steps,
                "ms_per_launch": ms / n} for k, (n, ms) in ktimes.items()}
    top = max(kern, key=lambda k: kern[k]["ms_per_step"])
    roof = roofline(top, kern[top]["ms_per_launch"], peaks, clocks, s, t, ls, Wt, Wa,
                    n_lors, n_cls, nnz, nv)
    launches = sum(n for n, _ in ktimes.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_lors": n_lors, "nnz": nnz, "n_classes": n_cls,
                   "image": [im["nx"], im["ny"], im["nz"]], "voxel_mm": im["dx"],
                   "l2": "inputs larger than L2 (%.0f GB matrix regenerated per step)"
                         % ((8.0 * nnz + 8.0 * n_lors) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "sysmat_nnz_per_s": rows_rate,
        "fwdback_lor_voxel_per_s": fb,
        "stage_ms": med,
        "kernels": kern,
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "plain_fp32": plain,
        "mixed": mixed,
        "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        r, dt, cores, desc = cpu_sample(480)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc, "seconds": dt}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile_case(args):
    """One stage of the step on a configuration small enough for a kernel
    capture (a few GB on the device): 'spread' = all class spreads; 'stencil' =
    S and S^T over the full LOR space with an empty G; 'rows' = chord rows of
    the first 2M LORs; 'csr' = forward/back with those rows; 'back_patch' =
    the pair back-projection with per-pair shared-memory accumulation over the
    rows of the fan narrowed to +-10."""
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P

    B.build()
    dev = torch.device("cuda", 0)
    w = I.workload(WORKLOAD)
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    case = args.profile_case
    for _ in range(2):
        if case in ("spread", "stencil"):
            T, eta = P.response_build(s, t, device=dev)
            WC = P.bin_spread_classes(s, t, T, eta, ls, P.lor_set_classes(s, ls, device=dev),
                                      Wt, Wa)
        if case == "stencil":
            n, _ = P.lor_set_size(s, ls)
            rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
            M = P.Matrix(rp, torch.zeros(1, dtype=torch.int32, device=dev),
                         torch.zeros(1, device=dev), nv).set_spread(s, ls, Wt, Wa, WC)
            M.autotune()  # 8 stencil launches (2 forms x 2 directions x 2), then the tuned ones
            if args.stencil_form is not None:
                M.set_stencil_form(args.stencil_form)
            x = torch.rand(nv, device=dev)
            y = M.forward(x)
            M.back(y)
        if case == "back_patch":
            # the bench step's pair back-projection over the rows of the fan
            # narrowed to +-10 (~7 GB on the device), pair form -3
            l10 = dict(ls, fan_half=10)
            T, eta = P.response_build(s, t, device=dev)
            WC = P.bin_spread_classes(s, t, T, eta, l10, P.lor_set_classes(s, l10, device=dev),
                                      Wt, Wa)
            rp, col, val = P.sysmat_rows_set(s, im, l10, device=dev)
            M = P.Matrix(rp, col, val, nv).set_spread(s, l10, Wt, Wa, WC).set_image(im)
            r = torch.rand(rp.numel() - 1, device=dev)
            M.back_sens(r)
            info = {"rows": rp.numel() - 1, "nnz": col.numel()}
        if case == "rows_set":
            # same scanner and image, fan narrowed to +-10 so the capture holds ~3 GB
            rows_set = P.sysmat_rows_set(s, im, dict(ls, fan_half=10), device=dev)
            info = {"rows": rows_set[0].numel() - 1, "nnz": rows_set[1].numel()}
        if case in ("rows", "csr"):
            L = P.lor_set_list(s, ls, device=dev)[: 2_000_000].contiguous()
            rp, col, val, _ = P.sysmat_rows(s, im, L)
            info = {"rows": rp.numel() - 1, "nnz": col.numel()}
            if case == "csr":
                M = P.Matrix(rp, col, val, nv)
                M.set_launch(64, 512)  # the work-queue launch the bench step's autotuner picks
                y = M.forward(torch.rand(nv, device=dev))
                M.back(y)
                M.back_sens(y)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "ok": True,
                      **(info if case in ("rows_set", "rows", "csr", "back_patch") else {})}))


VH_K = (60, 240, 960, 3840, 15360)


def run_voxel_homog(args):
    """The paper's voxel-driven generator (Sec. 2.3, Eq. 11-12) on the planar
    ring: the dense matrix from k lines per pixel for growing k (the
    k-convergence the paper describes), its generation time, the relative
    change of the disc phantom's projection against the largest k, and the
    projection's correlation with the LOR-driven A = S G of the library.
    Prints one JSON object."""
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P

    B.build()
    dev = torch.device("cuda", 0)
    w = I.workload("RING2D")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"]
    x = torch.from_numpy(I.phantom_discs(im, 0).reshape(-1)).to(dev)
    T, eta = P.response_build(s, t, device=dev)
    L = P.lor_set_list(s, ls, device=dev)
    WL = P.bin_spread(s, t, T, eta, L, Wt, Wa)
    ptr, col2, val2, _ = P.sysmat_rows(s, im, L, WL, Wt, Wa)
    y_lor = P.Matrix(ptr, col2, val2, nv).forward(x).double()
    st = torch.cuda.current_stream()
    rows, proj = [], {}
    for k in VH_K:
        P.voxel_homog(s, t, T, eta, im, ls, k, Wt)  # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        A = P.voxel_homog(s, t, T, eta, im, ls, k, Wt)
        b.record(st)
        torch.cuda.synchronize()
        y = (A.double() @ x.double())
        proj[k] = y
        c = float(torch.corrcoef(torch.stack([y, y_lor]))[0, 1])
        rows.append({"k": k, "ms": a.elapsed_time(b), "lines_per_s": nv * k / (a.elapsed_time(b) * 1e-3),
                     "corr_with_lor_driven": c})
        del A
    ref = proj[VH_K[-1]]
    for r in rows:
        r["proj_rel_change_vs_kmax"] = float(torch.linalg.norm(proj[r["k"]] - ref) / torch.linalg.norm(ref))
    print(json.dumps({"voxel_homog": "RING2D", "n_lors": int(L.shape[0]), "pixels": nv,
                      "window_t": Wt, "rows": rows}))


def run_ring2d(args):
    """The planar-ring workloads, small enough to stay in L2 and bound by
    launches: RING2D with the disc phantom (FP32 rows) and RING2D_ELLIPSES
    with the 8-ellipse phantom and the merged PSF rows A = S G stored as FP32,
    BF16 and FP16 (16-bit values with a per-row FP32 scale, FP32 accumulation).
    Each time is the median of 20 CUDA-event-timed runs after 3 warm-ups: the
    response table, the LOR spreads, the rows through psf_sysmat_rows
    (allocation of the outputs and the size query included), and one MLEM
    iteration (forward, ratio, back-projection, update) launched one kernel at
    a time and replayed from a CUDA graph that holds 10 iterations.  The image
    after 10 iterations of each 16-bit form is compared with the FP32 one
    (their errors against the FP64 oracle are the test suite's).  Prints one
    JSON object."""
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P
    from paper_1607_06170_gb300.torch_api import mlem

    B.build()
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()

    def timed(fn, reps=20, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {"ring2d": True}
    for name, phantom, dtypes in (("RING2D", I.phantom_discs, ("f32",)),
                                  ("RING2D_ELLIPSES", I.phantom_ellipses, ("f32", "bf16", "f16"))):
        w = I.workload(name)
        s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
        Wt, Wa = w["window"]
        nv = im["nx"] * im["ny"] * im["nz"]
        L = P.lor_set_list(s, ls, device=dev)
        T, eta = P.response_build(s, t, device=dev)
        Wl = P.bin_spread(s, t, T, eta, L, Wt, Wa)
        res = {"n_lors": int(L.shape[0]), "pixels": nv,
               "table_ms": timed(lambda: P.response_build(s, t, device=dev)),
               "spread_ms": timed(lambda: P.bin_spread(s, t, T, eta, L, Wt, Wa))}
        xt = torch.from_numpy(phantom(im, w["index"]).reshape(-1).astype("float32")).to(dev)
        ptr, col, val, _ = P.sysmat_rows(s, im, L, Wl, Wt, Wa)
        y = P.Matrix(ptr, col, val, nv).forward(xt).clone()  # noiseless data (FP32 rows)
        images = {}
        for dt in dtypes:
            ptr, col, val, scale = P.sysmat_rows(s, im, L, Wl, Wt, Wa, dtype=dt)
            nnz = int(col.numel())
            rows_ms = timed(lambda: P.sysmat_rows(s, im, L, Wl, Wt, Wa, dtype=dt))
            M = P.Matrix(ptr, col, val, nv, row_scale=scale)
            sens = M.sensitivity(device=dev)
            floor = 1e-12 * float(sens.max())
            yhat, ratio, bp = torch.empty_like(y), torch.empty_like(y), torch.empty_like(sens)
            x = torch.ones_like(sens)
            P.em_update(x, sens, sens, floor)

            def iteration():
                M.forward(x, out=yhat)
                P.em_ratio(y, yhat, out=ratio)
                M.back(ratio, out=bp)
                P.em_update(x, bp, sens, floor)

            eager_ms = timed(iteration)
            g = torch.cuda.CUDAGraph()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                for _ in range(10):
                    iteration()
            graph_ms = timed(g.replay) / 10
            images[dt] = mlem(M, y, iters=10, graph=True)
            res[dt] = {"nnz": nnz, "rows_ms": rows_ms, "rows_nnz_per_s": nnz / (rows_ms * 1e-3),
                       "mlem_iteration_us_eager": eager_ms * 1e3,
                       "mlem_iteration_us_graph": graph_ms * 1e3}
        for dt in dtypes[1:]:
            res[dt]["image_rel_l2_vs_f32_after_10"] = float(
                torch.linalg.norm(images[dt] - images["f32"]) / torch.linalg.norm(images["f32"]))
        out[name] = res
    print(json.dumps(out))


PAPER_ITERATION_S = 43.0  # Table 2: one PSF reconstruction iteration on the paper's GPU


def run_eplus(args):
    """The paper's own workload (Sec. 4, Tables 1-3): the Eplus-260-like
    scanner (2 x 24 modules of 16 x 16 crystals), histogram organisation of
    192 angles x 199 bins per ring pair (ring difference <= 1), 380 x 380 x 63
    image.  Times the system-matrix generation (response table, class spreads,
    G rows) and one MLEM iteration (forward, ratio, back-projection with the
    sensitivity, update) with the full window and with top-5 spreads (the
    paper's N), and sets them beside the paper's one-iteration GPU time (43 s,
    other hardware and code: context only).  Prints one JSON object."""
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P

    B.build()
    dev = torch.device("cuda", 0)
    w = I.workload("EPLUS260")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    st = torch.cuda.current_stream()
    x = torch.from_numpy(I.phantom_cylinder(im, w["index"]).reshape(-1)).to(dev)
    view, bins = P.sino_bins(s, ls, device=dev)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        out = fn()
        b.record(st)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    def generate():
        T, eta = P.response_build(s, t, device=dev)
        WC = P.bin_spread_classes(s, t, T, eta, ls, P.lor_set_classes(s, ls, device=dev), Wt, Wa)
        return WC, P.sysmat_rows_set(s, im, ls, device=dev)

    generate()  # warm-up (allocations, first launches)
    (WC, (rp, col, val)), gen_ms = timed(generate)
    nnz = int(col.numel())
    res = {}
    for name in ("full window", "top-5"):
        M = P.Matrix(rp, col, val, nv)
        if name == "full window":
            M.set_spread(s, ls, Wt, Wa, WC)
        else:
            idx, wk = P.spread_topn(WC, Wt, Wa, 5)
            M.set_spread_topn(s, ls, Wt, Wa, idx, wk)
        M.autotune()
        y = M.forward(x).clone()

        def iteration():
            xi = torch.ones(nv, device=dev)
            r = P.em_ratio(y, M.forward(xi))
            bp, sens = M.back_sens(r)
            P.em_update(xi, bp, sens, 1e-12)
            return xi

        iteration()
        ms = min(timed(iteration)[1] for _ in range(3))
        res[name] = {"iteration_ms": ms, "vs_paper_iteration": PAPER_ITERATION_S * 1e3 / ms}
        del M
    print(json.dumps({
        "eplus260": True, "n_lors": int(rp.numel() - 1), "nnz": nnz,
        "sinogram": {"views": int(view.max()) + 1, "bins": int(bins.max()) + 1,
                     "ring_pairs": P.len_ring_pairs(s, ls)},
        "image": [im["nx"], im["ny"], im["nz"]], "voxel_mm": [im["dx"], im["dy"], im["dz"]],
        "matrix_generation_ms": gen_ms, "rows_nnz_per_s_incl_table_spreads": nnz / (gen_ms * 1e-3),
        "iteration": res, "paper_iteration_s": PAPER_ITERATION_S,
        "note": "paper's time: one PSF OSEM iteration on its GPU (Table 2), other hardware; "
                "context, not a target"}))


def run_listmode(args):
    """List-mode OSEM (the next step named in Sec. 5) on the 104-ring
    workload: 10M seeded three-sphere events mapped to set rows, the
    factored projector with top-N (N = 5, the paper's choice) class spreads
    (G stored: it fits in HBM), one OSEM iteration over 10 subsets of 1M
    events, timed with CUDA events after a one-subset warm-up.  Reports
    events/s, the projections' LOR x voxel/s (forward and back over nnz(G)
    per sub-iteration) and the row generation rate.  Prints one JSON object."""
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P
    from paper_1607_06170_gb300.torch_api import listmode_osem

    B.build()
    dev = torch.device("cuda", 0)
    w = I.workload("RING3D_LM")
    s, t, im, ls, lm = w["scanner"], w["table"], w["image"], w["lors"], w["listmode"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    events = I.listmode_events(w, lm["events"], w["index"], device=dev)
    rows = P.event_rows(s, ls, events)
    del events
    T, eta = P.response_build(s, t, device=dev)
    WCf = P.bin_spread_classes(s, t, T, eta, ls, P.lor_set_classes(s, ls, device=dev), Wt, Wa)
    idx, wk = P.spread_topn(WCf, Wt, Wa, lm["n_keep"])
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    rp, col, val = P.sysmat_rows_set(s, im, ls, device=dev)
    b.record(st)
    torch.cuda.synchronize()
    rows_ms = a.elapsed_time(b)
    nnz = int(col.numel())
    M = P.Matrix(rp, col, val, nv).set_spread_topn(s, ls, Wt, Wa, idx, wk)
    M.autotune()
    sens = M.sensitivity()
    torch.cuda.synchronize()
    a.record(st)
    M.build_sparse_adjoint()  # once per plan: the transpose of the top-N S
    b.record(st)
    torch.cuda.synchronize()
    transpose_ms = a.elapsed_time(b)
    n_sub = lm["events"] // lm["subset_events"]
    listmode_osem(M, rows[: lm["subset_events"]].contiguous(), 1, 1, sens=sens)  # warm-up
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    P.timing_enable(True)
    a.record(st)
    x = listmode_osem(M, rows, n_sub, 1, sens=sens)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    kt = P.timing_read()
    P.timing_enable(False)
    clocks = clk.stop()
    # the same iteration with the full 49 x 49 window (the dense stencil)
    Mf = P.Matrix(rp, col, val, nv).set_spread(s, ls, Wt, Wa, WCf)
    Mf.autotune()
    sens_f = Mf.sensitivity()
    listmode_osem(Mf, rows[: lm["subset_events"]].contiguous(), 1, 1, sens=sens_f)
    torch.cuda.synchronize()
    a.record(st)
    listmode_osem(Mf, rows, n_sub, 1, sens=sens_f)
    b.record(st)
    torch.cuda.synchronize()
    ms_full = a.elapsed_time(b)
    del Mf

    def timed_osem(Mx, sens_x):
        """One OSEM iteration over the 10 subsets after a one-subset warm-up
        (CUDA events), with the library's per-kernel times."""
        listmode_osem(Mx, rows[: lm["subset_events"]].contiguous(), 1, 1, sens=sens_x)
        torch.cuda.synchronize()
        P.timing_enable(True)
        a.record(st)
        xx = listmode_osem(Mx, rows, n_sub, 1, sens=sens_x)
        b.record(st)
        torch.cuda.synchronize()
        kx = P.timing_read()
        P.timing_enable(False)
        return a.elapsed_time(b), xx, {k: round(v[1], 3) for k, v in kx.items() if v[1] > 0.05}

    # BF16 weights: the stored rows in BF16 with a per-row FP32 scale (FP32
    # accumulation), same columns and row pointers, the same top-N spreads
    val16 = torch.empty(nnz, dtype=torch.bfloat16, device=dev)
    sc16 = torch.empty(rp.numel() - 1, dtype=torch.float32, device=dev)
    P.sysmat_rows_set_typed(s, im, ls, "bf16", buffers=(rp, col, val16, sc16))
    Mb = P.Matrix(rp, col, val16, nv, row_scale=sc16).set_spread_topn(s, ls, Wt, Wa, idx, wk)
    Mb.autotune()
    Mb.build_sparse_adjoint()
    ms_b, xb, kb = timed_osem(Mb, sens)
    # and with the top-N weights in BF16 too (one FP32 scale per class)
    w16, wsc = P.spread_topn_bf16(wk)
    Mb.set_spread_topn(s, ls, Wt, Wa, idx, w16, scale=wsc)
    Mb.build_sparse_adjoint()
    ms_bw, xbw, kbw = timed_osem(Mb, sens)
    del Mb, val16, sc16
    # rows generated on the fly per subset (no stored matrix): the subset's
    # source rows traced for the masked forward, the rows with S^T r != 0
    # traced for the back-projection; same top-N spreads, same sensitivity
    Mo = P.Matrix.traced(s, im, ls).set_spread_topn(s, ls, Wt, Wa, idx, wk)
    Mo.build_sparse_adjoint()
    ms_o, xo_img, ko = timed_osem(Mo, sens)
    Mo.check()
    del Mo
    rel = lambda u, v: float((u - v).norm() / v.norm())
    print(json.dumps({
        "bf16_rows": {"iteration_ms": ms_b, "events_per_s": lm["events"] / (ms_b * 1e-3),
                      "stored_bytes": int(nnz * 6 + 4 * (rp.numel() - 1)),
                      "image_rel_l2_vs_f32_rows": rel(xb, x), "kernels_ms": kb},
        "bf16_rows_bf16_weights": {"iteration_ms": ms_bw,
                                   "events_per_s": lm["events"] / (ms_bw * 1e-3),
                                   "weight_bytes": int(idx.numel() * 6 + 4 * idx.shape[0]),
                                   "image_rel_l2_vs_f32_rows": rel(xbw, x), "kernels_ms": kbw},
        "traced_rows": {"iteration_ms": ms_o, "events_per_s": lm["events"] / (ms_o * 1e-3),
                        "stored_bytes": 0, "image_rel_l2_vs_f32_rows": rel(xo_img, x),
                        "kernels_ms": ko},
        "full_window": {"iteration_ms": ms_full, "events_per_s": lm["events"] / (ms_full * 1e-3)},
        "listmode": "RING3D_LM", "events": lm["events"], "subsets": n_sub,
        "n_keep": lm["n_keep"], "n_lors": int(rp.numel() - 1), "nnz": nnz,
        "image": [im["nx"], im["ny"], im["nz"]], "iteration_ms": ms,
        "events_per_s": lm["events"] / (ms * 1e-3),
        "lor_voxel_per_s": 2 * n_sub * nnz / (ms * 1e-3),
        "rows_ms": rows_ms, "rows_nnz_per_s": nnz / (rows_ms * 1e-3),
        "transpose_ms": transpose_ms,
        "kernels_ms": {k: round(v[1], 3) for k, v in kt.items() if v[1] > 0.05},
        "image_sum": float(x.double().sum()), "clocks": clocks,
        "data": "synthetic (seeded three-sphere events)"}))


TOPN_KEEP = (3, 5, 7, 16, 32, 64)


def run_topn_table(args):
    """Table 3 counterpart: one MLEM iteration of the RING3D workload with the
    full 49 x 49 window and with the class spreads truncated to their top N
    entries (psf_spread_topn), per N: the selection time, the S and S^T kernel
    times, the iteration time (forward, ratio, back-projection with
    sensitivity, update; G rows generated once) and the relative L2 change of
    the projection of the phantom and of the image after three iterations
    against the full window.  Prints one JSON object."""
    import torch

    from paper_1607_06170_gb300 import build as B
    from paper_1607_06170_gb300 import inputs as I
    from paper_1607_06170_gb300 import psf as P

    B.build()
    dev = torch.device("cuda", 0)
    w = I.workload(WORKLOAD)
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    x = torch.from_numpy(I.phantom_cylinder(im, 1).reshape(-1)).to(dev)
    T, eta = P.response_build(s, t, device=dev)
    WC = P.bin_spread_classes(s, t, T, eta, ls, P.lor_set_classes(s, ls, device=dev), Wt, Wa)
    rp, col, val = P.sysmat_rows_set(s, im, ls, device=dev)
    M = P.Matrix(rp, col, val, nv).set_spread(s, ls, Wt, Wa, WC)
    _, (bc, bt) = M.autotune()
    y = M.forward(x).clone()
    st = torch.cuda.current_stream()

    def iterate(Mx, x0, n_iter):
        xi = x0.clone()
        ms = []
        for _ in range(n_iter):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            r = P.em_ratio(y, Mx.forward(xi))
            bp, sens = Mx.back_sens(r)
            P.em_update(xi, bp, sens, 1e-12)
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return xi, ms

    def kernels_of(Mx):
        P.timing_enable(True)
        Mx.forward(x)
        Mx.back_sens(y)
        torch.cuda.synchronize()
        kt = P.timing_read()
        P.timing_enable(False)
        return {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in kt.items()
                if k.startswith(("stencil", "topn_s", "sens_"))}

    ones = torch.ones(nv, device=dev)
    iterate(M, ones, 1)
    x_full, ms_full = iterate(M, ones, 3)
    y_full = M.forward(x)
    rows = [{"n_keep": "full (2401)", "iteration_ms": round(min(ms_full), 2),
             "spread_kernels_ms": kernels_of(M), "proj_rel_l2": 0.0, "image_rel_l2": 0.0}]
    for n in TOPN_KEEP:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        idx, wk = P.spread_topn(WC, Wt, Wa, n)
        b.record(st)
        torch.cuda.synchronize()
        Mn = P.Matrix(rp, col, val, nv).set_spread_topn(s, ls, Wt, Wa, idx, wk)
        Mn.set_launch(bc, bt if bc > 0 else 256)  # the full-window plan's tuned back launch
        iterate(Mn, ones, 1)
        xn, ms = iterate(Mn, ones, 3)
        yn = Mn.forward(x)
        rel = lambda u, v: float(torch.linalg.norm((u - v).double()) / torch.linalg.norm(v.double()))
        rows.append({"n_keep": n, "select_ms": round(a.elapsed_time(b), 3),
                     "iteration_ms": round(min(ms), 2), "spread_kernels_ms": kernels_of(Mn),
                     "proj_rel_l2": rel(yn, y_full), "image_rel_l2": rel(xn, x_full)})
        del Mn
    print(json.dumps({"topn_table": WORKLOAD, "n_lors": int(rp.numel() - 1), "nnz": int(col.numel()),
                      "note": "iteration = forward + ratio + back-projection with sensitivity + "
                              "update, G stored once; rel_l2 against the full window",
                      "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision (BF16 G rows) step")
    ap.add_argument("--stencil-form", type=int, default=None,
                    help="pin the LOR-space stencil form after autotuning (0-5)")
    ap.add_argument("--profile-case",
                    choices=["spread", "stencil", "rows", "rows_set", "csr", "back_patch"],
                    help="run one stage on a small-memory setup (for kernel captures)")
    ap.add_argument("--topn-table", action="store_true",
                    help="time the MLEM iteration with top-N truncated spreads (Table 3)")
    ap.add_argument("--listmode", action="store_true",
                    help="time one list-mode OSEM iteration on the 104-ring workload")
    ap.add_argument("--eplus", action="store_true",
                    help="matrix generation and one MLEM iteration on the paper's scanner")
    ap.add_argument("--voxel-homog", action="store_true",
                    help="the voxel-driven generator's k-convergence on the planar ring")
    ap.add_argument("--ring2d", action="store_true",
                    help="planar-ring timings: rows and MLEM iterations, eager and graphed")
    args = ap.parse_args()
    if args.topn_table:
        run_topn_table(args)
        return
    if args.listmode:
        run_listmode(args)
        return
    if args.eplus:
        run_eplus(args)
        return
    if args.voxel_homog:
        run_voxel_homog(args)
        return
    if args.ring2d:
        run_ring2d(args)
        return
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
