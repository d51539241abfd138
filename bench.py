"""Benchmark of the Tucker-compressed FFT-VIE solve on GB300.

Headline workload (the memory headline): 256^3 voxels (512^3 padded), 5 mm
voxels at 298 MHz, seeded ellipsoidal tissue contrast, 8 z-directed dipoles on
a 0.15 m ring as right-hand sides in one batch, HOSVD at 1e-6, mixed-precision
GMRES(50) with FP64 iterative refinement to a relative residual of 1e-5.
One step = one GMRES(50) restart cycle of the 8-RHS system (50 Arnoldi steps:
pad/FFT, Tucker rebuild + product, inverse FFT/crop, contrast, Gram-Schmidt,
Givens; the cycle-end true residual) followed by its FP64 refinement residual.
`value` = operator applications (right-hand-side matvecs, FP32 and FP64) per
second over the timed steps.  The same steps on the uncompressed-spectra path,
complete solves of both paths to 1e-5, the device memory of each path, the
64^3 plane-wave solve and the FP64 CPU oracle are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--mode headline|solve64|...]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Tucker-VIE matvecs/s & GMRES solve time vs uncompressed FFT path, same GB300"
UNIT = "matvecs/s"
L2_BYTES = 129 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--n", type=int, default=64, help="grid edge (default: the 64^3 solve)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-n64", action="store_true", help="headline: skip the 64^3 solve summary")
    p.add_argument("--only-steps", action="store_true",
                   help="headline: warm-up and timed steps only (a short command for profilers; "
                        "the timed steps run inside the NVTX range timed_steps)")
    p.add_argument("--no-batched", action="store_true", help="skip the 96^3 16-RHS solve")
    p.add_argument("--no-cp", action="store_true", help="skip the Tucker+CP (rank 32) measurement")
    p.add_argument("--mode", default="headline",
                   choices=["headline", "solve64", "matvec", "solve1", "ranks", "tolerance",
                            "refinement", "mixed"],
                   help="headline: the 256^3 8-dipole workload (default); solve64: the 64^3 "
                        "plane-wave solve with its extras; matvec: only K timed batched matvecs; "
                        "solve1: K solves only "
                        "(small commands for profilers); ranks: the multilinear rank of "
                        "the Green's tensors against frequency (Sec. VI.A, Fig. 4); tolerance: "
                        "operator error against the HOSVD tolerance (Sec. VI.C, Fig. 7); "
                        "refinement: solve time and memory of the three paths as a sphere's "
                        "grid is refined (Sec. VI.D, Fig. 9)")
    p.add_argument("--max-n", type=int, default=300, help="ranks: largest grid edge built")
    p.add_argument("--no-graph", action="store_true", help="solve1: direct launches")
    p.add_argument("--orth", type=int, default=1, choices=[1, 2],
                   help="Gram-Schmidt passes (2 = DGKS-conditional second pass)")
    p.add_argument("--batch", type=int, default=1, help="right-hand sides per matvec (matvec mode)")
    p.add_argument("--path", default="tucker", choices=["tucker", "uncompressed"])
    p.add_argument("--rebuild", default="tensor_cores", choices=["tensor_cores", "mma_sync", "tcgen05", "simt"],
                   help="matvec / solve1: how the Tucker path rebuilds the Green's fibres")
    p.add_argument("--record-traffic", metavar="NCU_CSV",
                   help="turn an ncu CSV of dram__bytes_read.sum / dram__bytes_write.sum per launch "
                        "into the row of --family in profiles/roofline_traffic.md, then exit")
    p.add_argument("--family", help="kernel family of --record-traffic (e.g. fused_tucker)")
    p.add_argument("--kernel", default="", help="--record-traffic: regex on the kernel name")
    p.add_argument("--capture", default="", help="--record-traffic: the ncu command, for the record")
    p.add_argument("--workload", default="", help="--record-traffic: the captured launches, for the record")
    return p.parse_args()


# ---------------------------------------------------------------------------
# DRAM traffic of the roofline kernel, from ncu captures (profiles/roofline_traffic.md).
# A row is used only while the library sources are unchanged since its capture.
# ---------------------------------------------------------------------------
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.md")
TRAFFIC_HEADER = ("| family | kernel | sources | launches | dram bytes per launch | workload | capture |\n"
                  "|---|---|---|---|---|---|---|\n")


def sources_digest():
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1811_00484_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                    [os.path.join(ROOT, "include", "vie.h")]):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_rows():
    rows = {}
    if os.path.exists(TRAFFIC_FILE):
        for line in open(TRAFFIC_FILE):
            cells = [c.strip() for c in line.strip().strip("|").split("|")]
            if len(cells) == 7 and cells[0] not in ("family", "---"):
                rows[cells[0]] = cells
    return rows


def recorded_traffic(family):
    r = traffic_rows().get(family)
    if r is None or r[2] != sources_digest():
        return None
    return float(r[4])


def record_traffic(args):
    import csv
    rows = list(csv.reader(open(args.record_traffic)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[hi]
    ki, mi, vi, ui = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    idx = hdr.index("ID")
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    names = set()
    import re
    pat = re.compile(args.kernel) if args.kernel else None
    for r in rows[hi + 1:]:
        if len(r) <= vi or r[mi] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        if pat is not None and not pat.search(r[ki]):
            continue
        per[r[idx]] = per.get(r[idx], 0.0) + float(r[vi].replace(",", "")) * scale[r[ui]]
        names.add(r[ki].split("(")[0].replace("void ", "").strip())
    if not per:
        raise SystemExit("no dram__bytes rows in " + args.record_traffic)
    table = traffic_rows()
    table[args.family] = [args.family, " ".join(sorted(names)), sources_digest(), str(len(per)),
                          f"{sum(per.values()) / len(per):.0f}", args.workload.replace("|", "/"),
                          args.capture.replace("|", "/")]
    with open(TRAFFIC_FILE, "w") as fh:
        fh.write("# DRAM traffic of the roofline kernel families\n\n"
                 "Written by `bench.py --record-traffic` from ncu captures of `dram__bytes_read.sum` + "
                 "`dram__bytes_write.sum` (one pass per launch) of a few launches of each family in the "
                 "bench's own launch shape. `sources` is a digest of the library sources at capture time: "
                 "`bench.py` reports a row's traffic only while the sources still match it, and null "
                 "otherwise.\n\n")
        fh.write(TRAFFIC_HEADER)
        for k in sorted(table):
            fh.write("| " + " | ".join(table[k]) + " |\n")
    print(json.dumps({"family": args.family, "launches": len(per),
                      "dram_bytes_per_launch": sum(per.values()) / len(per)}))


def reduce_ranks(t_local, count_local, world):
    """Whole-job figures from the per-rank ones: the slowest rank's time (max) and the
    operator applications of all ranks (sum).  One rank: unchanged."""
    if world == 1:
        return t_local, count_local
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=dev)
    c = torch.tensor([float(count_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_matvec_rate(wl, seconds=15.0, max_matvecs=None):
    """Oracle Tucker matvecs (FP64 numpy: FFT, rebuilt spectra, product) per second."""
    import numpy as np
    from oracle import embed, hosvd, kernel, matvec

    k0 = kernel.wavenumber(wl.freq_hz)
    Ghat = embed.green_spectra(kernel.toeplitz_tensor(*wl.n, wl.h, k0), *wl.n)
    rebuilt = hosvd.rebuild_components(hosvd.compress_components(Ghat, wl.tol_svd))
    w = wl.einc * wl.chi
    count, t0 = 0, time.perf_counter()
    while True:
        w = matvec.apply_system(rebuilt, wl.chi, w / np.linalg.norm(w))
        count += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_matvecs and count >= max_matvecs):
            break
    return count / el, count, el


def bench_config(n, world):
    """The workload both arms report (the native arm times it on the GPU, the
    reference arm samples the oracle's operator applications of it)."""
    return {"workload": f"solve {n[0]}^3 voxels ({2*n[0]}^3 padded), plane wave, HOSVD 1e-6, "
                        "GMRES(50) to 1e-6 + FP64 refinement",
            "global_batch": world, "parallelism": f"replicas x{world}",
            "l2": "solve working set (Krylov basis 51 x 6.3 MB) > L2; isolated matvecs flush L2"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads
    wl = workloads.solve_n64() if args.n == 64 else workloads.make("custom", args.n, 1, incident="plane")
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_matvec_rate(wl, seconds=0.0, max_matvecs=1)
    rates, t_total, n_total = [], 0.0, 0
    for _ in range(args.steps):
        r, c, el = oracle_matvec_rate(wl, seconds=5.0)
        rates.append(r)
        t_total += el
        n_total += c
    value = n_total / t_total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": bench_config(wl.n, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_total} FP64 oracle system matvecs (the operator "
                                       f"applications the solve counts; Tucker-rebuilt spectra) of "
                                       f"this workload in {t_total:.1f} s, one step a ~5 s sample"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


HEADLINE_WORKLOAD = ("memory headline: 256^3 voxels (512^3 padded, 5 mm, 298 MHz), 8 z-dipoles on a "
                     "0.15 m ring in one batch, HOSVD 1e-6, GMRES(50) + FP64 refinement to 1e-5; one "
                     "step = one restart cycle of the 8-RHS system and its FP64 refinement residual")


def headline_config(world):
    return {"workload": HEADLINE_WORKLOAD, "global_batch": 8 * world,
            "parallelism": f"replicas x{world}",
            "l2": "inputs > L2 (an 8-RHS vector is 3.2 GB, the Krylov basis 164 GB): no flush needed"}


def oracle_sample_rate(wl, J, seconds, max_voxels=None, seed=0):
    """The oracle's plain BTTB product (oracle.matvec.matvec_at) at successive
    uniformly drawn output voxels, for every right-hand side of J, until `seconds`
    have passed.  Returns (right-hand-side matvecs per second, voxels, seconds,
    threads used = process CPU time / wall time)."""
    import numpy as np
    from oracle import kernel, matvec

    k0 = kernel.wavenumber(wl.freq_hz)
    rng = np.random.default_rng(seed)
    t0, c0 = time.perf_counter(), time.process_time()
    nvox = 0
    while True:
        m = tuple(int(rng.integers(0, v)) for v in wl.n)
        matvec.matvec_at(J, wl.h, k0, [m])
        nvox += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_voxels and nvox >= max_voxels):
            break
    used = (time.process_time() - c0) / el
    rate = nvox * J.shape[0] / float(np.prod(wl.n)) / el
    return rate, nvox, el, used


def run_reference_headline(args):
    """Reference arm on the headline workload: the FP64 oracle's plain BTTB definition
    at sampled output voxels (each step one voxel, all three components, the seeded
    current J of the workload), as right-hand-side matvecs per second."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads

    wl = workloads.memory_n256()
    J = wl.J
    for w in range(args.warmup):
        oracle_sample_rate(wl, J, 0.0, max_voxels=1, seed=1000 + w)
    t_total, v_total, used = 0.0, 0, []
    for k in range(args.steps):
        _, nv, el, u = oracle_sample_rate(wl, J, 0.0, max_voxels=1, seed=k)
        t_total += el
        v_total += nv
        used.append(u)
    value = v_total * J.shape[0] / float(wl.n[0] * wl.n[1] * wl.n[2]) / t_total
    cores = max(1, round(statistics.median(used)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": headline_config(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the oracle's BTTB definition (kernel formed per output voxel) "
                                       f"at {v_total} sampled output voxels of the 256^3 workload's "
                                       f"current (3 components, 1 right-hand side) in {t_total:.1f} s; "
                                       "one step one voxel; value = fraction of a matvec per second"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_headline(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1811_00484_gb300 as vie
    import workloads

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def used_bytes():
        free, total = torch.cuda.mem_get_info()
        return total - free

    wl = workloads.memory_n256()
    n = wl.n
    mem0 = used_bytes()
    barrier()
    t0 = time.perf_counter()
    op = vie.Operator(n, wl.h, wl.freq_hz, wl.tol_svd, store_uncompressed=True)
    barrier()
    setup_s = time.perf_counter() - t0
    chi = torch.from_numpy(wl.chi.astype(np.complex64)).cuda()
    einc = op.incident_dipole(wl.dipoles)                    # c64 [8, 3, n, n, n]
    B = einc.shape[0]
    w = torch.empty_like(einc)
    step_kw = dict(tol=1e-5, restart=50, max_outer=1, max_refine=1, refine=False,
                   raise_on_failure=False)

    def timed_steps(path, k, chi_, einc_):
        mv = 0
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        start.record()
        for _ in range(k):
            _, inf = op.solve(chi_, einc_, path=path, out=w, **step_kw)
            mv += inf["matvecs"]
        stop.record()
        barrier()
        return start.elapsed_time(stop) / 1e3, mv

    for _ in range(args.warmup):
        op.solve(chi, einc, out=w, **step_kw)
    op.solve(chi, einc, path="uncompressed", out=w, **step_kw)
    # one step with every kernel family instrumented: the breakdown
    kern, dom = {}, None
    if not args.only_steps:
        vie.profile_start()
        timed_steps("tucker", 1, chi, einc)
        kern = vie.profile_stop()
        dom = max((k for k in kern if kern[k]["bytes"] > 0), key=lambda k: kern[k]["ms"])
    # timed region (the headline): no instrumentation inside the library
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        t_tucker, mv_tucker = timed_steps("tucker", args.steps, chi, einc)
        torch.cuda.nvtx.range_pop()
    clocks = clk.summary()
    if args.only_steps:
        if rank == 0:
            print(json.dumps({"mode": "only-steps", "metric": METRIC, "steps": args.steps,
                              "ms_per_step": 1e3 * t_tucker / args.steps,
                              "value": mv_tucker / t_tucker, "unit": UNIT, "clocks": clocks}))
        op.close()
        return
    k_unc = min(args.steps, 5)
    t_unc, mv_unc = timed_steps("uncompressed", k_unc, chi, einc)
    # the roofline kernel's launches timed with CUDA events on their stream
    k_roof = min(args.steps, 3)
    vie.profile_start([dom])
    t_roof, _ = timed_steps("tucker", k_roof, chi, einc)
    kern_live = vie.profile_stop()

    # end to end: contrast and incident fields from pinned host memory, solution back
    chi_h = torch.from_numpy(wl.chi.astype(np.complex64)).pin_memory()
    einc_h = einc.cpu().pin_memory()
    w_h = torch.empty_like(einc_h).pin_memory()
    k_e2e = min(args.steps, 3)
    # Two sets of device buffers (allocated once, outside the timed region) and a
    # copy stream: step k+1's inputs go in, and step k's solution comes out, while
    # the next solve runs, as a serving loop would overlap them.  Every step still
    # copies its own inputs from pinned host memory and reads its solution back.
    c_d = [torch.empty_like(chi_h, device="cuda") for _ in range(2)]
    e_d = [torch.empty_like(einc_h, device="cuda") for _ in range(2)]
    w_d = [w, torch.empty_like(w)]
    w_hs = [w_h, torch.empty_like(w_h).pin_memory()]
    comp, copy = torch.cuda.current_stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]      # a slot's inputs are on the device
    ev_done = [torch.cuda.Event() for _ in range(2)]    # a slot's solve has finished

    def copy_in(slot):
        with torch.cuda.stream(copy):
            c_d[slot].copy_(chi_h, non_blocking=True)
            e_d[slot].copy_(einc_h, non_blocking=True)
            ev_in[slot].record(copy)

    barrier()
    e2e_start = time.perf_counter()
    mv_e2e = 0
    copy_in(0)
    for k in range(k_e2e):
        slot = k % 2
        if k + 1 < k_e2e:
            # the other slot was last read by step k-1's solve and copy-out, both
            # ordered before this point on the copy stream
            copy_in(1 - slot)
        comp.wait_event(ev_in[slot])
        _, inf = op.solve(c_d[slot], e_d[slot], out=w_d[slot], **step_kw)
        mv_e2e += inf["matvecs"]
        ev_done[slot].record(comp)
        with torch.cuda.stream(copy):
            copy.wait_event(ev_done[slot])
            w_hs[slot].copy_(w_d[slot], non_blocking=True)
    copy.synchronize()
    barrier()
    t_e2e = time.perf_counter() - e2e_start
    del c_d, e_d, w_d, w_hs

    # complete refined solves of both paths to 1e-5
    solves = {}
    for path in ("tucker", "uncompressed"):
        barrier()
        ts = time.perf_counter()
        _, inf = op.solve(chi, einc, tol=1e-5, restart=50, max_outer=200, max_refine=20, path=path,
                          out=w)
        barrier()
        solves[path] = {"s": time.perf_counter() - ts, "iterations": inf["iterations"],
                        "matvecs": inf["matvecs"], "refine_steps": inf["refine_steps"],
                        "relres": inf["relres"], "converged": inf["converged"]}
    peak_used = used_bytes() - mem0
    info = op.info()

    # Section V.A's factor-wise setup at the same grid (no stored spectra): time and scratch
    barrier()
    t0 = time.perf_counter()
    op_fw = vie.Operator(n, wl.h, wl.freq_hz, wl.tol_svd, setup="factorwise")
    barrier()
    setup_fw_s = time.perf_counter() - t0
    info_fw = op_fw.info()
    op_fw.close()

    # isolated batched matvecs (the 8 incident fields), both paths
    def matvec_ms(path, reps=3):
        op.matvec(einc, path=path, out=w)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            op.matvec(einc, path=path, out=w)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    mv_ms = {p: matvec_ms(p) for p in ("tucker", "uncompressed")}
    vie.profile_start()
    op.matvec(einc, out=w)
    kern_mv = vie.profile_stop()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, nv, el, used = oracle_sample_rate(wl, wl.J, 15.0)
        cpu = {"value": rate, "unit": UNIT, "cores": max(1, round(used)), "kind": "oracle",
               "sample": f"the oracle's BTTB definition at {nv} sampled output voxels of the 256^3 "
                         f"workload's current (3 components, 1 right-hand side) in {el:.1f} s "
                         f"(fraction of a matvec per second)"}

    t_tucker, mv_all = reduce_ranks(t_tucker, mv_tucker, world)
    t_unc, mv_unc_all = reduce_ranks(t_unc, mv_unc, world)
    t_e2e, mv_e2e_all = reduce_ranks(t_e2e, mv_e2e, world)
    value = mv_all / t_tucker
    peak, peak_kind = measured_peaks()

    def gbs(e):
        return e["bytes"] / (e["ms"] * 1e-3) / 1e9 if e["ms"] > 0 else 0.0

    tot = max(1e-9, sum(x["ms"] for x in kern.values()))
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3), "share": round(v["ms"] / tot, 4),
                   "GBps": round(gbs(v), 1)} for k, v in kern.items()}
    d = kern_live[dom]
    traffic = recorded_traffic(dom)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(gbs(d), 1), "peak": peak,
                "unit": "GB/s", "frac": round(gbs(d) / peak, 4),
                "traffic": round(traffic) if traffic is not None else None,
                "bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
                "timing": f"CUDA events around every launch of the family on its stream, over {k_roof} "
                          "further steps",
                "instrumented_ms_per_step": 1e3 * t_roof / k_roof,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    mb = lambda v: round(v / 1e6, 1)
    dev_t, dev_s = info["device_bytes_tucker"], info["device_bytes_spectra"]
    ws, sws = info["matvec_workspace_bytes"], info["solver_workspace_bytes"]
    memory = {"unit": "MB", "ranks": info["ranks"],
              "tucker_cores_factors_c64": mb(info["tucker_bytes"]),
              "slab_cores_c64": mb(info["slab_bytes"]),
              "rebuild_scratch": mb(info["rebuild_scratch_bytes"]),
              "operator_tucker_all": mb(dev_t),
              "operator_spectra_c64_c128": mb(dev_s),
              "uncompressed_spectra_c64": mb(info["uncompressed_bytes"]),
              "matvec_workspace": mb(ws), "solver_workspace": mb(sws),
              "path_total_tucker": mb(dev_t + ws + sws),
              "path_total_uncompressed": mb(dev_s + ws + sws),
              "process_peak_used": mb(peak_used),
              "setup_s": round(setup_s, 2),
              "setup_scratch": mb(info["setup_scratch_bytes"]),
              "setup_factorwise_s": round(setup_fw_s, 2),
              "setup_factorwise_scratch": mb(info_fw["setup_scratch_bytes"]),
              "setup_factorwise_same_ranks": info_fw["ranks"] == info["ranks"]}
    f = kern_mv.get("fused_tucker")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_tucker / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": headline_config(world),
        "step": {"tucker_ms": 1e3 * t_tucker / args.steps, "uncompressed_ms": 1e3 * t_unc / k_unc,
                 "uncompressed_matvecs_per_s": mv_unc_all / t_unc, "uncompressed_steps": k_unc,
                 "matvecs_per_step": mv_tucker / args.steps},
        "solve": solves,
        "matvec": {"tucker_ms": mv_ms["tucker"], "uncompressed_ms": mv_ms["uncompressed"],
                   "batch": B, "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                                               "GBps": round(gbs(v), 1)} for k, v in kern_mv.items()}},
        "memory": memory,
        "clocks": clocks,
        "e2e": {"value": mv_e2e_all / t_e2e, "unit": UNIT, "steps": k_e2e,
                "h2d_bytes_per_step": chi_h.numel() * 8 + einc_h.numel() * 8,
                "d2h_bytes_per_step": w_h.numel() * 8,
                "copies": "pinned host buffers; each step's copy-in and copy-out run on a copy "
                          "stream beside the neighbouring steps' solves (two device buffer sets)"},
        "cpu_baseline": cpu,
        "roofline": roofline,
        "roofline_fused_matvec": None if not f else {
            "kernel": "fused_tucker (one batched matvec, B=8)", "bound": "hbm",
            "achieved": round(gbs(f), 1), "peak": peak, "unit": "GB/s", "frac": round(gbs(f) / peak, 4),
            "avg_launch_us": 1e3 * f["ms"] / f["launches"]},
        "kernels": kernels,
        "kernels_note": "per-family breakdown from one separately profiled step (all families "
                        "instrumented); the timed steps run without instrumentation",
        "gpu_launches": int(sum(v["launches"] for v in kern.values())) * args.steps,
    }
    # the 64^3 solve after the headline operator and its buffers are released
    op.close()
    del w, einc, chi, chi_h, einc_h, w_h
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_n64:
        line["n64"] = solve64_summary(args)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def solve64_summary(args):
    """The 64^3 plane-wave solve (GMRES(50) to 1e-6 + FP64 refinement) on both paths,
    three solves each, and one matvec's error against the oracle."""
    import numpy as np
    import torch

    import paper_1811_00484_gb300 as vie
    import workloads
    from oracle import embed, kernel, matvec

    wl = workloads.solve_n64()
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd, store_uncompressed=True)
    chi = torch.from_numpy(wl.chi.astype(np.complex64)).cuda()
    einc = torch.from_numpy(wl.einc.astype(np.complex64)).cuda()
    out = {"workload": "solve 64^3 voxels (128^3 padded), plane wave, HOSVD 1e-6, GMRES(50) to 1e-6 "
                       "+ FP64 refinement"}
    for path in ("tucker", "uncompressed"):
        op.solve(chi, einc, tol=1e-6, path=path)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mv = 0
        for _ in range(3):
            _, inf = op.solve(chi, einc, tol=1e-6, path=path)
            mv += inf["matvecs"]
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 3
        out[path] = {"ms_per_solve": ms, "matvecs_per_s": mv / (3 * ms * 1e-3),
                     "iterations": inf["iterations"], "relres": inf["relres"]}
    k0 = kernel.wavenumber(wl.freq_hz)
    Ghat = embed.green_spectra(kernel.toeplitz_tensor(*wl.n, wl.h, k0), *wl.n)
    ref = matvec.matvec_fft(Ghat, wl.J)
    y = op.matvec(torch.from_numpy(wl.J.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    out["matvec_rel_err_vs_oracle"] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    inf = op.info()
    out["memory_MB"] = {"operator_tucker_all": round(inf["device_bytes_tucker"] / 1e6, 2),
                        "uncompressed_spectra_c64": round(inf["uncompressed_bytes"] / 1e6, 2)}
    op.close()
    return out


def run_solve1_mode(args):
    """K solves of the bench workload and nothing else (for ncu captures)."""
    import numpy as np
    import torch

    import paper_1811_00484_gb300 as vie
    import workloads

    wl = workloads.solve_n64() if args.n == 64 else workloads.make("custom", args.n, 1, incident="plane")
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd, store_uncompressed=args.path == "uncompressed",
                      rebuild=args.rebuild)
    chi = torch.from_numpy(wl.chi.astype(np.complex64)).cuda()
    einc = torch.from_numpy(wl.einc.astype(np.complex64)).cuda()
    kw = dict(tol=1e-6, restart=50, path=args.path, use_graph=not args.no_graph, orth=args.orth)
    for _ in range(args.warmup):
        op.solve(chi, einc, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_solve")
    infos = [op.solve(chi, einc, **kw)[1] for _ in range(args.steps)]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    print(json.dumps({"mode": "solve1", "n": args.n, "path": args.path, "rebuild": op.info()["rebuild_kernel"],
                      "graph": not args.no_graph,
                      "orth": args.orth, "ms_per_solve": 1e3 * el / args.steps,
                      "iterations": infos[-1]["iterations"], "refine_steps": infos[-1]["refine_steps"],
                      "relres": infos[-1]["relres"],
                      "matvecs_per_s": sum(i["matvecs"] for i in infos) / el}))


def run_matvec_mode(args):
    """K batched matvecs of the bench workload, nothing else (for ncu captures)."""
    import numpy as np
    import torch

    import paper_1811_00484_gb300 as vie
    import workloads

    wl = workloads.make("matvec", args.n, seed=1, B=args.batch, tol_svd=1e-6)
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd, store_uncompressed=args.path == "uncompressed",
                      rebuild=args.rebuild)
    J = torch.from_numpy(wl.J.astype(np.complex64)).cuda()
    Y = torch.empty_like(J)
    for _ in range(args.warmup):
        op.matvec(J, path=args.path, out=Y)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_matvec")
    a.record()
    for _ in range(args.steps):
        op.matvec(J, path=args.path, out=Y)
    b.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"mode": "matvec", "n": args.n, "batch": args.batch, "path": args.path,
                      "rebuild": op.info()["rebuild_kernel"],
                      "ms_per_matvec_batch": ms, "matvecs_per_s": args.batch / (ms * 1e-3)}))


def run_mixed_mode(args):
    """The mixed-size batch (48^3, 64^3, 80^3 grids, four ring dipoles each, beside the
    96^3 sixteen-dipole batch): one multi-grid matvec as one persistent cooperative
    launch, as one launch per stage, and as separate per-operator matvecs; then the
    three solves to 1e-6 run concurrently (vie_solve_multi) and one after another."""
    import numpy as np
    import torch

    import paper_1811_00484_gb300 as vie
    import workloads

    wls = workloads.mixed_grids()
    ops = [vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd) for wl in wls]
    chis = [torch.from_numpy(wl.chi.astype(np.complex64)).cuda() for wl in wls]
    eincs = [op.incident_dipole(wl.dipoles) for op, wl in zip(ops, wls)]
    Js = [(c[None, None] * e).contiguous() for c, e in zip(chis, eincs)]
    outs = [torch.empty_like(J) for J in Js]

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = max(args.steps, 10)
    line = {"mode": "mixed", "grids": [list(wl.n) for wl in wls], "rhs_per_grid": 4,
            "matvec_ms": {
                "persistent_one_launch": timed(lambda: vie.matvec_multi(ops, Js, outs, mode="persistent"), reps),
                "one_launch_per_stage": timed(lambda: vie.matvec_multi(ops, Js, outs, mode="staged"), reps),
                "separate_operators": timed(lambda: [op.matvec(J, out=o) for op, J, o in zip(ops, Js, outs)],
                                            reps)}}
    kw = dict(tol=1e-6, restart=50)
    vie.solve_multi(ops, chis, eincs, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = [r[1] for r in vie.solve_multi(ops, chis, eincs, **kw)]
    torch.cuda.synchronize()
    line["solve_concurrent_ms"] = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    for op, c, e in zip(ops, chis, eincs):
        op.solve(c, e, **kw)
    torch.cuda.synchronize()
    line["solve_sequential_ms"] = 1e3 * (time.perf_counter() - t0)
    line["iterations"] = [i["iterations"] for i in infos]
    print(json.dumps(line))
    for op in ops:
        op.close()


def smooth7(n):
    """The 7-smooth integer nearest to n (the padded edge 2 n must factor into 2, 3, 5, 7)."""
    def ok(v):
        for p in (2, 3, 5, 7):
            while v % p == 0:
                v //= p
        return v == 1
    for d in range(0, n):
        for v in (n - d, n + d):
            if v >= 1 and ok(v):
                return v
    return 1


def run_ranks_mode(args):
    """Maximum Tucker rank over the six components against frequency, for a cube
    of unit edge at resolutions lambda/10, lambda/20, lambda/30 and HOSVD tolerance
    1e-8, f = 0.3 i GHz, i = 1..10: the sweep of Sec. VI.A (Fig. 4), with the
    point-collocated dyadic kernel in place of the paper's PWL components.  The
    edge n is the 7-smooth integer nearest to (cube edge) / (lambda / m); h = 1/n,
    so the cube stays exactly 1 m and the resolution is reported as lambda / h."""
    import torch

    import paper_1811_00484_gb300 as vie

    c0 = 299792458.0
    for per in (10, 20, 30):
        for i in range(1, 11):
            f = 0.3e9 * i
            lam = c0 / f
            n = smooth7(max(2, round(per / lam)))
            if n > args.max_n:
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op = vie.Operator((n, n, n), 1.0 / n, f, 1e-8)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            ranks = op.info()["ranks"]
            op.close()
            print(json.dumps({"mode": "ranks", "f_ghz": round(f / 1e9, 3), "per_lambda": per,
                              "n": n, "lambda_over_h": round(lam * n, 2), "tol": 1e-8,
                              "max_rank": max(max(r) for r in ranks), "ranks": ranks,
                              "setup_s": round(dt, 3)}), flush=True)


def run_tolerance_mode(args):
    """Operator error against the HOSVD tolerance on the bench workload (Sec. VI.C,
    Fig. 7): for each tol, the FP64 Tucker matvec and the FP32 Tucker+CP matvec
    (32 terms, 300 ALS sweeps) against the FP64 matvec with the stored
    uncompressed spectra, relative L2 over one random field."""
    import numpy as np
    import torch

    import paper_1811_00484_gb300 as vie
    import workloads

    wl = workloads.make("tolerance", args.n, seed=1, tol_svd=1e-6)
    J64 = torch.from_numpy(wl.J).to(torch.complex128).cuda()
    ref = None
    for e in range(2, 10):
        tol = 10.0 ** (-e)
        op = vie.Operator(wl.n, wl.h, wl.freq_hz, tol, store_uncompressed=ref is None)
        if ref is None:
            ref = op.matvec(J64, path="uncompressed")
        nref = torch.linalg.vector_norm(ref).item()
        err_t = torch.linalg.vector_norm(op.matvec(J64) - ref).item() / nref
        cp_err = op.tucker_cp(32, tol=1e-10, max_iter=300, seed=0)
        y_cp = op.matvec(J64.to(torch.complex64), path="tucker_cp").to(torch.complex128)
        err_cp = torch.linalg.vector_norm(y_cp - ref).item() / nref
        inf = op.info()
        print(json.dumps({"mode": "tolerance", "n": args.n, "tol": tol,
                          "max_rank": max(max(r) for r in inf["ranks"]),
                          "tucker_bytes": inf["tucker_bytes"], "tucker_matvec_rel_err": err_t,
                          "cp_rank": 32, "cp_core_rel_err_max": max(cp_err),
                          "cp_matvec_rel_err": err_cp}), flush=True)
        op.close()


def run_refinement_mode(args):
    """Scaling of the three paths as the grid of the refinement study's sphere is
    refined (Sec. VI.D, Fig. 9): a homogeneous sphere of radius 0.15 m in a 0.3 m
    cube, HOSVD tol 1e-8, plane wave, GMRES(50) to 1e-5 with FP64 refinement, on
    the uncompressed, HOSVD and Tucker+CP (32 terms, 1000 ALS sweeps) paths.
    Grid edges n = 32 .. 160 (9.4 to 1.9 mm voxels; the paper's 10 .. 2 mm with
    the padded edge a multiple of 32).  Each path is solved twice, the second
    solve is timed.  Memory: the six components as each path holds them (c64)."""
    import numpy as np
    import torch

    import paper_1811_00484_gb300 as vie
    import workloads

    for n in (32, 64, 96, 128, 160):
        if n > args.max_n:
            continue
        wl = workloads.sphere(n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd, store_uncompressed=True)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        chi = torch.from_numpy(wl.chi.astype(np.complex64)).cuda()
        einc = torch.from_numpy(wl.einc.astype(np.complex64)).cuda()
        line = {"mode": "refinement", "n": n, "h_mm": round(1e3 * wl.h, 3),
                "unknowns": 3 * n ** 3, "setup_s": round(setup, 3)}
        for path in ("uncompressed", "tucker", "tucker_cp"):
            if path == "tucker_cp":
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                errs = op.tucker_cp(32, tol=1e-12, max_iter=1000, seed=0)
                torch.cuda.synchronize()
                line["cp_als_s"] = round(time.perf_counter() - t0, 3)
                line["cp_core_rel_err_max"] = max(errs)
            try:
                op.solve(chi, einc, tol=1e-5, path=path)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, inf = op.solve(chi, einc, tol=1e-5, path=path)
                torch.cuda.synchronize()
                line[path] = {"solve_ms": round(1e3 * (time.perf_counter() - t0), 2),
                              "iterations": inf["iterations"], "refine_steps": inf["refine_steps"],
                              "relres": inf["relres"]}
            except vie.VieError as e:
                line[path] = {"error": str(e)}
        info = op.info()
        line["max_rank"] = max(max(r) for r in info["ranks"])
        line["bytes"] = {"uncompressed": info["uncompressed_bytes"], "tucker": info["tucker_bytes"],
                         "tucker_cp": info["cp_bytes"]}
        print(json.dumps(line), flush=True)
        op.close()


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.record_traffic:
        return record_traffic(args)
    if args.impl == "reference":
        return run_reference(args) if args.mode == "solve64" else run_reference_headline(args)
    if args.mode == "matvec":
        return run_matvec_mode(args)
    if args.mode == "solve1":
        return run_solve1_mode(args)
    if args.mode == "ranks":
        return run_ranks_mode(args)
    if args.mode == "tolerance":
        return run_tolerance_mode(args)
    if args.mode == "refinement":
        return run_refinement_mode(args)
    if args.mode == "solve64":
        return run_solve64(args)
    if args.mode == "mixed":
        return run_mixed_mode(args)
    return run_headline(args)


def run_solve64(args):
    """The 64^3 plane-wave solve (GMRES(50) to 1e-6, FP64 refinement): one step is one
    complete solve; with isolated matvecs, cuFFT, Tucker+CP and the 96^3 batch."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1811_00484_gb300 as vie
    import workloads

    wl = workloads.solve_n64() if args.n == 64 else workloads.make("custom", args.n, 1, incident="plane")
    n = wl.n
    op = vie.Operator(n, wl.h, wl.freq_hz, wl.tol_svd, store_uncompressed=True)
    info = op.info()
    chi = torch.from_numpy(wl.chi.astype(np.complex64)).cuda()
    einc = torch.from_numpy(wl.einc.astype(np.complex64)).cuda()
    chi_h = torch.from_numpy(wl.chi.astype(np.complex64)).pin_memory()
    einc_h = torch.from_numpy(wl.einc.astype(np.complex64)).pin_memory()
    w_h = torch.empty_like(einc_h).pin_memory()
    solve_kw = dict(tol=1e-6, restart=50, max_outer=200, max_refine=20, orth=args.orth)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed_solves(path, steps):
        mv = 0
        its = []
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.nvtx.range_push(f"{path}_solve")
        start.record()
        for _ in range(steps):
            w, inf = op.solve(chi, einc, path=path, **solve_kw)
            mv += inf["matvecs"]
            its.append(inf)
        stop.record()
        torch.cuda.nvtx.range_pop()
        barrier()
        return start.elapsed_time(stop) / 1e3, mv, its

    for _ in range(args.warmup):
        op.solve(chi, einc, **solve_kw)
        op.solve(chi, einc, path="uncompressed", **solve_kw)

    # one profiled solve with every kernel family instrumented: the breakdown
    vie.profile_start()
    timed_solves("tucker", 1)
    kern = vie.profile_stop()
    # the roofline kernel: the family with the most time among those that move
    # algorithmic bytes (the small latency-bound kernels have none to count)
    dom = max((k for k in kern if kern[k]["bytes"] > 0), key=lambda k: kern[k]["ms"])
    # timed region (the headline): the library runs without events
    with ClockSampler(local) as clk:
        t_tucker, mv_tucker, it_tucker = timed_solves("tucker", args.steps)
    clocks = clk.summary()
    t_unc, mv_unc, it_unc = timed_solves("uncompressed", args.steps)
    # the roofline kernel's launch durations: the same K solves again, with CUDA
    # events on the launching stream around every launch of the dominant family
    # (event nodes between kernels cost time of their own, so they stay out of
    # the headline solves)
    vie.profile_start([dom])
    t_tucker_ev, _, _ = timed_solves("tucker", args.steps)
    kern_live = vie.profile_stop()

    # end to end: host buffers in, host solution out, through the same C-ABI solve
    c_d = torch.empty_like(chi_h, device="cuda")
    e_d = torch.empty_like(einc_h, device="cuda")
    w_d = torch.empty_like(einc_h, device="cuda")
    barrier()
    e2e_start = time.perf_counter()
    mv_e2e = 0
    for _ in range(args.steps):
        c_d.copy_(chi_h, non_blocking=True)
        e_d.copy_(einc_h, non_blocking=True)
        w, inf = op.solve(c_d, e_d, out=w_d, **solve_kw)
        mv_e2e += inf["matvecs"]
        w_h.copy_(w, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    barrier()
    t_e2e = time.perf_counter() - e2e_start

    # isolated matvec rates (B = 1), L2 flushed between timed launches
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    J = torch.from_numpy(wl.J.astype(np.complex64)).cuda()

    def matvec_rate(path, reps=20):
        for _ in range(3):
            op.matvec(J, path=path)
        torch.cuda.nvtx.range_push(f"{path}_matvec")
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            op.matvec(J, path=path)
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        torch.cuda.nvtx.range_pop()
        return reps / (tot / 1e3), tot / reps

    mv_rate_t, mv_ms_t = matvec_rate("tucker")
    mv_rate_u, mv_ms_u = matvec_rate("uncompressed")

    # cuFFT beside it: zero-pad, 3-D FFT of the three components, inverse 3-D FFT and
    # crop (the FFT work of one traditional matvec, no product), same L2 flush
    P = tuple(2 * v for v in n)
    padded = torch.zeros((1, 3) + P, dtype=torch.complex64, device="cuda")

    def cufft_once():
        padded[..., :n[0], :n[1], :n[2]] = J
        X = torch.fft.fftn(padded, dim=(-3, -2, -1))
        return torch.fft.ifftn(X, dim=(-3, -2, -1))[..., :n[0], :n[1], :n[2]]

    for _ in range(3):
        cufft_once()
    cufft_tot = 0.0
    for _ in range(20):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        cufft_once()
        b.record()
        torch.cuda.synchronize()
        cufft_tot += a.elapsed_time(b)
    cufft_ms = cufft_tot / 20
    # fused kernel alone at B = 1 (isolated matvecs, L2 flushed), for its HBM fraction
    vie.profile_start()
    matvec_rate("tucker", reps=10)
    kern_mv = vie.profile_stop()

    # Tucker+CP (Algorithm 2) on the same operator, after the headline runs: CP-ALS
    # with 32 terms on each core, then isolated matvecs and one solve on that path
    # (its inner FP32 GMRES applies eq. (17); FP64 refinement residuals the Tucker model)
    tucker_cp = None
    if not args.no_cp:
        barrier()
        t0 = time.perf_counter()
        cp_err = op.tucker_cp(32, tol=1e-10, max_iter=300, seed=0)
        barrier()
        t_als = time.perf_counter() - t0
        mv_rate_cp, mv_ms_cp = matvec_rate("tucker_cp")
        op.solve(chi, einc, path="tucker_cp", **solve_kw)
        t_cp, mv_cp, it_cp = timed_solves("tucker_cp", 1)
        icp = op.info()
        tucker_cp = {"rank": 32, "als_ms": 1e3 * t_als, "als_sweeps": list(icp["cp_sweeps"]),
                     "core_rel_err_max": max(cp_err), "cp_bytes": icp["cp_bytes"],
                     "matvec_ms": mv_ms_cp, "matvecs_per_s": mv_rate_cp,
                     "solve_ms": 1e3 * t_cp, "solve_matvecs": mv_cp,
                     "iterations": it_cp[-1]["iterations"], "refine_steps": it_cp[-1]["refine_steps"],
                     "relres": it_cp[-1]["relres"]}

    # the batched workload: 96^3 (192^3 padded), 16 ring-dipole right-hand sides in one
    # solve, HOSVD 1e-6; one warm-up and one timed solve, no instrumentation
    batched = None
    if not args.no_batched:
        wb = workloads.dipoles_n96()
        opb = vie.Operator(wb.n, wb.h, wb.freq_hz, wb.tol_svd)
        chib = torch.from_numpy(wb.chi.astype(np.complex64)).cuda()
        eb = opb.incident_dipole(wb.dipoles, dtype=torch.complex64)
        opb.solve(chib, eb, **solve_kw)
        barrier()
        tb0 = time.perf_counter()
        _, infb = opb.solve(chib, eb, **solve_kw)
        barrier()
        tb = time.perf_counter() - tb0
        ib = opb.info()
        batched = {"workload": f"solve {wb.n[0]}^3 voxels ({2 * wb.n[0]}^3 padded), "
                               f"{wb.dipoles.shape[0]} ring-dipole right-hand sides, HOSVD 1e-6, "
                               "GMRES(50) to 1e-6 + FP64 refinement",
                   "ms_per_solve": 1e3 * tb, "matvecs": infb["matvecs"],
                   "matvecs_per_s": infb["matvecs"] / tb, "relres": infb["relres"],
                   "tucker_bytes": ib["tucker_bytes"], "uncompressed_bytes": ib["uncompressed_bytes"]}
        opb.close()

    # accuracy of one matvec against the oracle (FP64 numpy), rank 0 only
    acc = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import embed, kernel, matvec
        k0 = kernel.wavenumber(wl.freq_hz)
        Ghat = embed.green_spectra(kernel.toeplitz_tensor(*n, wl.h, k0), *n)
        ref = matvec.matvec_fft(Ghat, wl.J)
        y = op.matvec(J).cpu().numpy().astype(np.complex128)
        acc = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
        rate, count, el = oracle_matvec_rate(wl, seconds=15.0)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{count} FP64 oracle system matvecs ({n[0]}^3, Tucker-rebuilt spectra) "
                         f"in {el:.1f} s"}

    # whole job: matvecs of every rank over the slowest rank's time
    t_tucker, mv_all = reduce_ranks(t_tucker, mv_tucker, world)
    t_unc, mv_unc_all = reduce_ranks(t_unc, mv_unc, world)
    t_e2e, mv_e2e_all = reduce_ranks(t_e2e, mv_e2e, world)
    value = mv_all / t_tucker
    peak, peak_kind = measured_peaks()

    def gbs(e):
        return e["bytes"] / (e["ms"] * 1e-3) / 1e9 if e["ms"] > 0 else 0.0

    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "share": round(v["ms"] / max(1e-9, sum(x["ms"] for x in kern.values())), 4),
                   "GBps": round(gbs(v), 1)} for k, v in kern.items()}
    d = kern_live[dom]
    traffic = recorded_traffic(dom)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(gbs(d), 1), "peak": peak,
                "unit": "GB/s", "frac": round(gbs(d) / peak, 4),
                "traffic": round(traffic) if traffic is not None else None,
                "bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
                "timing": "CUDA events around every launch of the family on its stream, over a second "
                          "run of the K timed solves",
                "instrumented_ms_per_step": 1e3 * t_tucker_ev / args.steps,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    f = kern_mv.get("fused_tucker")
    roofline_fused = None
    if f:
        roofline_fused = {"kernel": "fused_tucker (isolated matvec, B=1, L2 flushed)", "bound": "hbm",
                          "achieved": round(gbs(f), 1), "peak": peak, "unit": "GB/s",
                          "frac": round(gbs(f) / peak, 4), "avg_launch_us": 1e3 * f["ms"] / f["launches"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_tucker / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": bench_config(n, world),
        "solve": {"tucker_ms": 1e3 * t_tucker / args.steps,
                  "uncompressed_ms": 1e3 * t_unc / args.steps,
                  "iterations": it_tucker[-1]["iterations"], "refine_steps": it_tucker[-1]["refine_steps"],
                  "relres": it_tucker[-1]["relres"],
                  "uncompressed_matvecs_per_s": mv_unc_all / t_unc},
        "matvec": {"tucker_per_s": mv_rate_t, "tucker_ms": mv_ms_t,
                   "uncompressed_per_s": mv_rate_u, "uncompressed_ms": mv_ms_u,
                   "rel_err_vs_oracle": acc,
                   "cufft_pad_fft_ifft_crop_ms": cufft_ms},
        "memory": {"tucker_bytes": info["tucker_bytes"], "uncompressed_bytes": info["uncompressed_bytes"],
                   "slab_bytes": info["slab_bytes"],
                   "rebuild_scratch_bytes": info["rebuild_scratch_bytes"], "ranks": info["ranks"]},
        "batched": batched,
        "tucker_cp": tucker_cp,
        "clocks": clocks,
        "e2e": {"value": mv_e2e_all / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": chi_h.numel() * 8 + einc_h.numel() * 8,
                "d2h_bytes_per_step": w_h.numel() * 8},
        "cpu_baseline": cpu,
        "roofline": roofline,
        "roofline_fused": roofline_fused,
        "kernels": kernels,
        "kernels_note": "per-family breakdown from one separately profiled solve (all families "
                        "instrumented); the timed solves instrument only the roofline kernel",
        "gpu_launches": int(sum(v["launches"] for v in kern.values())) * args.steps,
    }
    if rank == 0:
        print(json.dumps(line))
    op.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
