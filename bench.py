#!/usr/bin/env python
"""Throughput of the even-odd Wilson matrix on GB300.

One step = M_eo^dag (M_eo psi): both a1-a7 rows of the hot path (neighbour
indexing, projection, link multiply, reconstruction, the two hops of Eq. 4 with
the diagonal term, and the adjoint), i.e. the normal-operator application a
CG iteration on M_eo^dag M_eo performs. Workload: 32^3 x 64 periodic lattice,
kappa = 0.13, links exp(i 0.4 H) with H random traceless Hermitian (seed 0),
Gaussian even source (seed 0), FP32 storage and arithmetic, 18-real links.
GFlop/s counts 1344 flop per site per M_eo (1320 per hopping site plus the
kappa^2 scale and the subtraction).

``python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]``
prints one JSON line on rank 0. Under torchrun each rank runs an independent
replica (the operator has no data-path exchange on one lattice per GPU).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "M_eo GFlop/s & HBM-roofline %, FP32 vs 16-bit; solve time to 1e-10 vs FP64"
DIMS = (32, 32, 32, 64)
KAPPA = 0.13
EPS = 0.4
FLOP_PER_SITE = 1344  # per M_eo per lattice site


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--linkfmt", type=int, default=18)
    ap.add_argument("--algo", type=int, default=0,
                    help="0: two hop launches, 1: fused, 2: fused through the TMA-staged pipeline")
    ap.add_argument("--lookahead", type=int, default=4,
                    help="t-slices the fused kernel's first hop runs ahead of the second")
    ap.add_argument("--staged", action=argparse.BooleanOptionalAction, default=True,
                    help="FP32 18-real single-RHS hops fed by TMA through a shared-memory ring "
                         "(measured faster than the one-site-per-thread kernel at 32^3 x 64)")
    ap.add_argument("--staged-rows", type=int, default=0, help="lattice rows per staged tile (0: auto)")
    ap.add_argument("--staged-depth", type=int, default=0, help="stages of the staged ring (0: auto)")
    ap.add_argument("--threads", type=int, default=128, help="threads per CTA of the hop kernels")
    ap.add_argument("--order", type=int, default=1,
                    help="1: second hop walks the sites downward (reads the freshest part first)")
    ap.add_argument("--ff", action="store_true",
                    help="main step in float-float arithmetic (wilson_eo_apply_ff64, complex128 spinors)")
    ap.add_argument("--no-variants", action="store_true", help="skip the other precisions")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip multi-RHS, batch and force measurements")
    ap.add_argument("--no-solve", action="store_true", help="skip the 48^3x96 solve comparison")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end measurement (for profiling runs)")
    ap.add_argument("--only-solve", action="store_true", help="run only the solve comparison")
    ap.add_argument("--solve-dims", type=int, nargs=4, default=[48, 48, 48, 96])
    ap.add_argument("--solve-variants", nargs="*", default=None,
                    help="only these entries of the solve comparison (e.g. mixed_f16_two_pass)")
    ap.add_argument("--only-multi-rhs", type=int, default=0, metavar="N",
                    help="run only M_eo then M_eo^dag on N Gaussian right-hand sides (launch "
                         "configuration autotuned for N) and print its timing; for profiling")
    ap.add_argument("--tile-links", type=int, default=-1, metavar="N",
                    help="with --only-multi-rhs: hops over tiles with links in shared memory, N "
                         "right-hand sides per pass (0: off); default: autotuned")
    ap.add_argument("--tile-rpt", type=int, default=1, metavar="R",
                    help="with --tile-links: right-hand sides per thread sharing each link read (1, 2)")
    ap.add_argument("--dims", type=int, nargs=4, default=None,
                    help="lattice extents (default 32 32 32 64, the benchmark workload)")
    args = ap.parse_args()
    if args.dims:
        global DIMS
        DIMS = tuple(args.dims)
    return args


def staged_main(args):
    """The main line's hops run staged (FP32 18-real, two-launch algorithm)."""
    return args.staged and args.prec == "f32" and args.linkfmt == 18 and not args.ff and not args.algo


def workload_config(args, world):
    """The workload both arms measure (the same dict in both JSON lines)."""
    link_bytes = 144 if args.ff else {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}[args.prec]
    if args.linkfmt == 12 and not args.ff:
        link_bytes = link_bytes * 2 // 3
    links_mb = 4 * int(np.prod(DIMS)) * link_bytes / 1e6
    return {"workload": workload_name(args), "lattice": list(DIMS), "kappa": KAPPA,
            "links": f"exp(i*{EPS}*H), {18 if args.ff else args.linkfmt}-real", "prec": args.prec,
            "flop_per_site_per_meo": FLOP_PER_SITE,
            "l2": f"inputs larger than L2 ({links_mb:.0f} MB of links per hop pass)"
                  if links_mb > 129 else f"links {links_mb:.0f} MB per hop pass (L2 129 MB)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def workload_name(args):
    prec = "float-float (FP64-class)" if args.ff else {"f64": "FP64", "f32": "FP32", "f16": "FP16 storage",
                                                        "bf16": "BF16 storage"}[args.prec]
    links = 18 if args.ff else args.linkfmt
    return (f"M_eo^dag M_eo, {'x'.join(map(str, DIMS))}, {prec}, {links}-real links, "
            f"kappa={KAPPA}, exp(i*{EPS}*H) links")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def fields(seed=0):
    import gen

    U = gen.gauge_field(DIMS, "smooth", seed=seed, eps=EPS)
    psi = gen.gaussian_spinor(DIMS, seed=seed)[0]
    return U, psi


# sources that define the FP32 hopping kernels whose DRAM traffic ncu measured
HOP_SOURCES = ("weo_fields.cuh", "weo_dslash.cuh", "weo_launch.cuh", "dslash_f32.cu")


def sources_for(label):
    """Source files a kernel label's code comes from."""
    if label.startswith("fused_staged"):
        return HOP_SOURCES + ("fused_staged.cu", "weo_tma.cuh")
    if label.startswith("fused_"):
        return HOP_SOURCES + ("fused.cu",)
    if label.startswith("hop_staged"):
        return HOP_SOURCES + ("hop_staged.cu",)
    return HOP_SOURCES


def kernel_source_hash(files=HOP_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2303_08609_gb300", "csrc")
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stored_traffic(label):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel source
    it was taken from is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(label)
    if not e or e.get("source_hash") != kernel_source_hash(sources_for(label)):
        return None
    return e.get("bytes_per_launch")


# algorithmic bytes per launch of each hopping-kernel kind, per lattice site V
# (V/2 output sites): input spinors once + all 4V links once + output once,
# + the axpy addend for the second hop.
def algo_bytes_per_site(label):
    if label.startswith("fused_staged_"):
        # one M_eo: even input once, every link once (the pair blocks are read
        # by both hops, the second time from L2), even output once
        return 96 / 2 + 4 * 72 + 96 / 2
    if label.startswith("fused_"):
        # one M_eo: even input once, all 4V links once, even output once (FP32 spinors)
        lk = {"f32": 72, "f16": 36, "bf16": 36}[label.split("_")[1]]
        if "_l12" in label:
            lk = lk * 2 // 3
        return 96 / 2 + 4 * lk + 96 / 2
    if label.startswith("hop_f32") or label.startswith("hop_staged_f32"):
        sp, lk = 96, (48 if "_l12" in label else 72)
    elif label.startswith("hop_f64") or label.startswith("hop_ff"):
        sp, lk = 192, (96 if "_l12" in label else 144)
    elif label.startswith("hop_to16"):
        lk = 24 if "_l12" in label else 36
        return (96 + 52) / 2 + 4 * lk
    elif label.startswith("hop_from16"):
        lk = 24 if "_l12" in label else 36
        return (52 + 96 + 96) / 2 + 4 * lk
    else:
        return None
    n_sp = 3 if "_axpy" in label else 2
    return n_sp * sp / 2 + 4 * lk


# minimal traffic of one M_eo per lattice site V: the even input once, every
# link once and the even output once (the odd intermediate never leaves the
# chip). Against it, the "useful-work" fraction credits fusion and compression.
def useful_bytes_per_site(prec, fmt):
    sp = {"f64": 192, "f32": 96, "f16": 52, "bf16": 52}[prec]
    lk = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}[prec]
    if fmt == 12:
        lk = lk * 2 // 3
    if prec in ("f16", "bf16"):
        sp = 96  # the API's spinors are FP32 for 16-bit handles
    return sp / 2 + 4 * lk + sp / 2


def run_ours(args, rank, world, local):
    import torch

    import paper_2303_08609_gb300 as weo

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    U, psi = fields()
    V = int(np.prod(DIMS))
    vh = V // 2
    # the handle's spinor dtype: complex128 for FP64 handles, complex64 otherwise
    x_host = np.ascontiguousarray(np.moveaxis(psi, 0, -1)).astype(
        np.complex128 if args.prec == "f64" or args.ff else np.complex64)
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    op = weo.WilsonEO(DIMS, KAPPA, torch.from_numpy(U).to(dev), prec=args.prec,
                      linkfmt=args.linkfmt)

    def configure(o):
        if args.algo:
            weo.wilson_eo_set_algorithm(o.handle, {1: "fused", 2: "fused_staged"}[args.algo],
                                        args.lookahead, 128)
        weo.wilson_eo_set_launch(o.handle, args.threads, 1, args.order)
        if staged_main(args):
            weo.wilson_eo_set_staging(o.handle, True, args.staged_rows, args.staged_depth)

    configure(op)
    stream = torch.cuda.current_stream(dev)
    staged_mb = None

    def step():
        if args.ff:
            weo.wilson_eo_apply_ff64(op.handle, y, x, 1, False, stream)
            weo.wilson_eo_apply_ff64(op.handle, z, y, 1, True, stream)
        else:
            weo.wilson_eo_apply(op.handle, y, x, 1, stream)
            weo.wilson_eo_apply_dag(op.handle, z, y, 1, stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if staged_main(args):
        # the staged hop's per-tile link blocks: 576 B per site of each output
        # parity, beside the packed links (counted in device_mb too)
        staged_mb = round(576 * V / 1e6, 1)
    device_mb = round(weo.wilson_eo_info(op.handle).get("device_bytes", 0) / 1e6, 1)

    # ---- timed region: device events on the launching stream
    weo.wilson_eo_profile(op.handle, True)
    weo.wilson_eo_profile_read(op.handle, reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_total = e0.elapsed_time(e1)
    weo.wilson_eo_check(op.handle, stream)
    prof = weo.wilson_eo_profile_read(op.handle, reset=True)
    weo.wilson_eo_profile(op.handle, False)
    flops_step = 2 * FLOP_PER_SITE * V
    ms_step, value = replica_summary(ms_total / args.steps, flops_step, world, dev)
    launches = int(sum(c for _, c in prof.values()))

    # ---- roofline of the dominant kernel
    label, (kms, kcnt) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_ms = kms / kcnt
    per_site = algo_bytes_per_site(label)
    algo = per_site * V
    peak, peak_kind = measured_peaks()
    achieved = algo / (avg_ms * 1e-3) / 1e9
    traffic = stored_traffic(label)
    # the single hops (D_oe-type, no axpy): 1320 flop per output site, V/2 sites;
    # the second hops add kappa^2 scale and the subtraction: 1368 per output site
    hops = {k: round((1368 if "_axpy" in k else 1320) * (V // 2) / (ms / cnt * 1e-3) / 1e9, 1)
            for k, (ms, cnt) in prof.items()}
    useful = useful_bytes_per_site(args.prec, args.linkfmt)
    link_bytes = 144 if args.ff else {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}[args.prec]
    links_mb = 4 * V * (link_bytes * 2 // 3 if args.linkfmt == 12 and not args.ff else link_bytes) / 1e6
    roofline = {"bound": "hbm", "kernel": label, "achieved": round(achieved, 1),
                "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": int(algo), "avg_launch_ms": round(avg_ms, 5),
                "kernel_share": {k: round(v[0] / sum(w[0] for w in prof.values()), 4)
                                 for k, v in sorted(prof.items())},
                "useful_work": {"model": f"minimal traffic of M_eo (input, links, output once): "
                                         f"{useful:g} B per site",
                                "bytes_per_step": int(2 * useful * V),
                                "frac": round(2 * useful * V / (ms_step * 1e-3) / 1e9 / peak, 4)}}

    # ---- sampled parity of this run's output (M_eo^dag M_eo at 64 sites)
    check = None
    if rank == 0:
        try:
            import oracle

            sites = np.sort(np.random.default_rng(7).choice(vh, 64, replace=False))
            got_y = np.moveaxis(y[:, :, torch.from_numpy(sites).to(dev)].cpu().numpy(), -1, 0)
            want_y = oracle.meo_sites(U, KAPPA, psi, DIMS, sites)
            check = {"meo_rel_l2_64_sites": float(np.linalg.norm(got_y - want_y)
                                                  / np.linalg.norm(want_y))}
        except Exception as exc:  # pragma: no cover
            check = {"error": repr(exc)}

    # ---- end to end through the public API: every step copies its input from
    # pinned host memory, applies M_eo then M_eo^dag, and copies its result back
    # to pinned host memory. Two to four handles on as many streams take the
    # steps in turn, so one step's copies overlap the others' kernels (pinned
    # host arrays make the calls asynchronous); the best of them is reported,
    # with the one-stream figure beside it.
    nb = x_host.nbytes
    NS_E2E = 1 if args.no_e2e else 4  # handles / streams taking the steps in turn
    ops2 = [op]
    for _ in range(NS_E2E - 1):
        o_ = weo.WilsonEO(DIMS, KAPPA, torch.from_numpy(U).to(dev), prec=args.prec,
                          linkfmt=args.linkfmt)
        configure(o_)
        ops2.append(o_)
    streams = [stream] + [torch.cuda.Stream(dev) for _ in range(NS_E2E - 1)]
    xh = [torch.from_numpy(x_host).pin_memory() for _ in range(NS_E2E)]
    zh = [torch.empty_like(xh[0]).pin_memory() for _ in range(NS_E2E)]
    ys = [y] + [torch.empty_like(y) for _ in range(NS_E2E - 1)]

    def e2e_steps(count, nstreams):
        for k in range(count):
            j = k % nstreams
            if args.ff:
                weo.wilson_eo_apply_ff64(ops2[j].handle, ys[j], xh[j], 1, False, streams[j])
                weo.wilson_eo_apply_ff64(ops2[j].handle, zh[j], ys[j], 1, True, streams[j])
            else:
                weo.wilson_eo_apply(ops2[j].handle, ys[j], xh[j], 1, streams[j])
                weo.wilson_eo_apply_dag(ops2[j].handle, zh[j], ys[j], 1, streams[j])

    ke = max(6, min(400, args.steps // 4))
    e2e_ms = {}
    for nstreams in range(1, NS_E2E + 1) if not args.no_e2e else ():
        e2e_steps(6, nstreams)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e2e_steps(ke, nstreams)
        torch.cuda.synchronize()
        e2e_ms[nstreams], e2e_val = replica_summary((time.perf_counter() - t0) * 1e3 / ke, flops_step,
                                                    world, dev)
    zres = np.moveaxis(zh[(ke - 1) % NS_E2E].numpy(), -1, 0)  # the last step's result, read on the host
    ns = min(range(2, NS_E2E + 1), key=lambda k: e2e_ms[k]) if not args.no_e2e else 1
    e2e = None if args.no_e2e else {"value": round(world * flops_step / (e2e_ms[ns] * 1e-3) / 1e9, 1), "unit": "GFlop/s",
           "ms_per_step": round(e2e_ms[ns], 4), "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
           "mode": f"pipelined: {ns} handles on {ns} streams take the steps in turn, each "
                   f"holding its own packed links (and staged link blocks)",
           "streams": ns, "handles": ns,
           "ms_per_step_by_streams": {k: round(v, 4) for k, v in e2e_ms.items()},
           "one_stream_value": round(world * flops_step / (e2e_ms[1] * 1e-3) / 1e9, 1),
           "per_call_latency_ms": round(e2e_ms[1], 4),
           "per_call_note": "one handle, one stream: host->device copy, M_eo, M_eo^dag and the "
                            "device->host copy of one step back to back (the ABI's latency per step)",
           "result_finite": bool(np.isfinite(zres).all())}
    for o_ in ops2[1:]:
        o_.close()
    del ops2

    # ---- measured FMA peaks (the FP64 kernels are bound by the FP64 pipe)
    alu_peaks = {}
    try:
        alu_peaks = {"f64_tflops": round(weo.wilson_eo_alu_peak("f64") / 1e12, 3),
                     "f32_tflops": round(weo.wilson_eo_alu_peak("f32") / 1e12, 2),
                     "l2_read_gbs": round(weo.wilson_eo_l2_peak() / 1e9, 1)}
    except Exception as exc:  # pragma: no cover
        alu_peaks = {"error": repr(exc)}

    # ---- other storage formats (same workload, M_eo^dag M_eo per step)
    variants = {}
    # the side measurements (other formats, multi-RHS, batches, force, solves and
    # their oracle checks) run in single-GPU runs only: a replica run measures
    # the main step and the end-to-end step on every rank
    side = world == 1
    if not args.no_variants and side:
        Ud = torch.from_numpy(U).to(dev)
        # algo 0: two hop launches, 1: fused, 2: two staged (TMA) hop launches,
        # 3: fused staged (one TMA-fed launch)
        main = (args.prec, args.linkfmt, 2 if staged_main(args) else {2: 3}.get(args.algo, args.algo))
        for prec, fmt, algo in (("f32", 18, 0), ("f32", 18, 2), ("f32", 18, 3), ("f32", 12, 0), ("f16", 18, 0),
                                ("f16", 12, 0), ("bf16", 12, 0), ("f64", 18, 0), ("f32", 18, 1),
                                ("f32", 12, 1), ("f16", 18, 1), ("f16", 12, 1), ("bf16", 12, 1)):
            if (prec, fmt, algo) == main:
                continue
            o2 = weo.WilsonEO(DIMS, KAPPA, Ud, prec=prec, linkfmt=fmt)
            if algo == 1:
                weo.wilson_eo_set_algorithm(o2.handle, "fused", args.lookahead, 128)
            if algo == 2:
                weo.wilson_eo_set_staging(o2.handle, True)
            if algo == 3:
                weo.wilson_eo_set_algorithm(o2.handle, "fused_staged", 2)
            xv = torch.from_numpy(np.ascontiguousarray(np.moveaxis(psi, 0, -1))).to(dev) \
                if prec == "f64" else x
            yv, zv = torch.empty_like(xv), torch.empty_like(xv)
            for _ in range(3):
                weo.wilson_eo_apply(o2.handle, yv, xv, 1, stream)
                weo.wilson_eo_apply_dag(o2.handle, zv, yv, 1, stream)
            torch.cuda.synchronize()
            n = 20 if prec == "f64" else 200
            weo.wilson_eo_profile(o2.handle, True)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(n):
                weo.wilson_eo_apply(o2.handle, yv, xv, 1, stream)
                weo.wilson_eo_apply_dag(o2.handle, zv, yv, 1, stream)
            a1.record(stream)
            torch.cuda.synchronize()
            vms = a0.elapsed_time(a1) / n
            weo.wilson_eo_check(o2.handle, stream)
            vp = weo.wilson_eo_profile_read(o2.handle, reset=True)
            lab, (km, kc) = max(vp.items(), key=lambda kv: kv[1][0])
            ab = algo_bytes_per_site(lab)
            ent = {"gflops": round(flops_step / (vms * 1e-3) / 1e9, 1),
                   "hop_gflops": {k: round((1368 if "_axpy" in k else 1320) * (V // 2)
                                           / (ms_ / cnt_ * 1e-3) / 1e9, 1)
                                  for k, (ms_, cnt_) in vp.items()},
                   "ms_per_step": round(vms, 4), "dominant_kernel": lab,
                   "kernel_gbs": round(ab * V / (km / kc * 1e-3) / 1e9, 1) if ab else None,
                   "useful_work_frac": round(2 * useful_bytes_per_site(prec, fmt) * V
                                             / (vms * 1e-3) / 1e9 / peak, 4)}
            if prec == "f64" and alu_peaks.get("f64_tflops"):
                ent["fp64_alu_frac"] = round(ent["gflops"] / (alu_peaks["f64_tflops"] * 1e3), 4)
            yo = np.moveaxis(yv[:, :, torch.from_numpy(sites).to(dev)].cpu().numpy(), -1, 0) \
                if rank == 0 and check and "error" not in check else None
            if yo is not None:
                ent["meo_rel_l2_64_sites"] = float(np.linalg.norm(yo - want_y)
                                                   / np.linalg.norm(want_y))
            variants[f"{prec}_l{fmt}" + ("", "_fused", "_staged", "_fused_staged")[algo]] = ent
            o2.close()
            del xv, yv, zv
        # the same step on fully Haar-random links (seed 0): FP32 18-real staged
        # and two-launch, FP64 18-real
        import gen

        Uh = torch.from_numpy(gen.gauge_field(DIMS, "haar", seed=0)).to(dev)
        for prec, algo in (("f32", 2), ("f32", 0), ("f64", 0)):
            o2 = weo.WilsonEO(DIMS, KAPPA, Uh, prec=prec, linkfmt=18)
            if algo == 2:
                weo.wilson_eo_set_staging(o2.handle, True)
            xv = torch.from_numpy(np.ascontiguousarray(np.moveaxis(psi, 0, -1))).to(dev) \
                if prec == "f64" else x
            yv, zv = torch.empty_like(xv), torch.empty_like(xv)
            n = 20 if prec == "f64" else 200
            weo.wilson_eo_profile(o2.handle, True)
            vms = timed(lambda: (weo.wilson_eo_apply(o2.handle, yv, xv, 1, stream),
                                 weo.wilson_eo_apply_dag(o2.handle, zv, yv, 1, stream)), n, stream)
            weo.wilson_eo_check(o2.handle, stream)
            vp = weo.wilson_eo_profile_read(o2.handle, reset=True)
            variants[f"{prec}_l18" + ("", "", "_staged")[algo] + "_haar"] = {
                "gflops": round(flops_step / (vms * 1e-3) / 1e9, 1), "ms_per_step": round(vms, 4),
                "hop_gflops": {k: round((1368 if "_axpy" in k else 1320) * (V // 2)
                                        / (ms_ / cnt_ * 1e-3) / 1e9, 1)
                               for k, (ms_, cnt_) in vp.items()},
                "links": "Haar-random SU(3), seed 0"}
            o2.close()
            del xv, yv, zv
        del Uh
        # float-float M_eo (FP64-class accuracy on the FP32 pipes) on complex128 spinors
        o2 = weo.WilsonEO(DIMS, KAPPA, Ud, prec="f64")
        xv = torch.from_numpy(np.ascontiguousarray(np.moveaxis(psi, 0, -1))).to(dev)
        yv, zv = torch.empty_like(xv), torch.empty_like(xv)
        for _ in range(3):
            weo.wilson_eo_apply_ff64(o2.handle, yv, xv, 1, False, stream)
            weo.wilson_eo_apply_ff64(o2.handle, zv, yv, 1, True, stream)
        torch.cuda.synchronize()
        n = 20
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n):
            weo.wilson_eo_apply_ff64(o2.handle, yv, xv, 1, False, stream)
            weo.wilson_eo_apply_ff64(o2.handle, zv, yv, 1, True, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        vms = a0.elapsed_time(a1) / n
        ent = {"gflops": round(flops_step / (vms * 1e-3) / 1e9, 1), "ms_per_step": round(vms, 4),
               "note": "float-float arithmetic (hi + lo floats, ~48 bits), complex128 in and out"}
        if rank == 0 and check and "error" not in check:
            yo = np.moveaxis(yv[:, :, torch.from_numpy(sites).to(dev)].cpu().numpy(), -1, 0)
            ent["meo_rel_l2_64_sites"] = float(np.linalg.norm(yo - want_y) / np.linalg.norm(want_y))
        if variants.get("f64_l18"):
            ent["speedup_vs_native_f64"] = round(ent["gflops"] / variants["f64_l18"]["gflops"], 2)
        variants["ff64_l18"] = ent
        o2.close()
        del xv, yv, zv
        del Ud

    extra = {} if args.no_extras or not side else extras(U, psi, dev, stream)
    if not args.no_solve and side:
        extra["multi_rhs_solve_12"] = multi_solve_comparison(U, dev)
    solve = None if args.no_solve or not side else solve_comparison(dev, tuple(args.solve_dims),
                                                        args.solve_variants)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(U, psi)
        cpu["small_workloads"] = oracle_plan()

    if rank == 0:
        import oracle  # noqa: F401  (only for the baseline / check above)

        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "GFlop/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "float-float (2 x f32)" if args.ff else
                     {"f32": "f32", "f64": "f64", "f16": "f16-storage/f32",
                      "bf16": "bf16-storage/f32"}[args.prec],
            "data": "synthetic",
            "config": workload_config(args, world),
            "impl_config": {"algo": {1: "fused", 2: "fused staged (TMA)"}.get(args.algo) if args.algo else
                                    "two staged (TMA) hop launches" if staged_main(args)
                                    else "two hop launches",
                            "threads": args.threads,
                            "second_hop_order": "down" if args.order else "up",
                            "staged_link_blocks_mb": staged_mb,
                            "device_mb": device_mb},
            "gflops_1368_per_site": round(value * 1368 / FLOP_PER_SITE, 1),
            "site_updates_per_s": round(world * 2 * V / (ms_step * 1e-3), 0),
            "roofline": roofline, "hop_gflops": hops, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(), "check": check, "alu_peaks": alu_peaks, "variants": variants,
            "extras": extra, "solve": solve,
        }
        print(json.dumps(out), flush=True)
    op.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def replica_summary(ms_local, flops_per_rank_step, world, device=None):
    """Whole-job throughput of `world` independent replicas: the step time is the
    maximum over ranks, the work is the sum over ranks. Returns (ms, GFlop/s)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * flops_per_rank_step / (ms * 1e-3) / 1e9


def timed(fn, n, stream):
    import torch

    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(n):
        fn()
    a1.record(stream)
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / n


def extras(U, psi, dev, stream):
    """Multi-RHS, mixed-lattice batch and force forward+backward on the GPU."""
    import torch

    import gen
    import paper_2303_08609_gb300 as weo

    V = int(np.prod(DIMS))
    vh = V // 2
    out = {}
    Ud = torch.from_numpy(U).to(dev)
    # 12 spin-colour point sources at one even site (FP32, links shared per site)
    op = weo.WilsonEO(DIMS, KAPPA, Ud, prec="f32")
    site = int(np.random.default_rng(3).integers(vh))
    src = np.zeros((12, 4, 3, vh), dtype=np.complex64)
    for s_ in range(4):
        for c in range(3):
            src[3 * s_ + c, s_, c, site] = 1.0
    x = torch.from_numpy(src).to(dev)
    y, z = torch.empty_like(x), torch.empty_like(x)
    res = {}
    for rb in (1, 2, 4):
        weo.wilson_eo_set_launch(op.handle, 128, rb)
        ms = timed(lambda: (weo.wilson_eo_apply(op.handle, y, x, 12, stream),
                            weo.wilson_eo_apply_dag(op.handle, z, y, 12, stream)), 50, stream)
        res[f"rhs_per_thread_{rb}"] = {"ms_per_step": round(ms, 4),
                                       "gflops": round(12 * 2 * FLOP_PER_SITE * V / (ms * 1e-3) / 1e9, 1)}
    weo.wilson_eo_set_launch(op.handle, 128, 1)
    for nrl, rpt in ((2, 1), (4, 1), (8, 1), (2, 2), (4, 2)):
        # tiles with their links in shared memory: nrl thread groups, rpt RHS per thread
        weo.wilson_eo_set_tile_links(op.handle, nrl, rpt)
        ms = timed(lambda: (weo.wilson_eo_apply(op.handle, y, x, 12, stream),
                            weo.wilson_eo_apply_dag(op.handle, z, y, 12, stream)), 50, stream)
        res[f"tile_links_{nrl}x{rpt}"] = {"ms_per_step": round(ms, 4),
                                          "gflops": round(12 * 2 * FLOP_PER_SITE * V / (ms * 1e-3) / 1e9, 1)}
    weo.wilson_eo_set_tile_links(op.handle, 0, 1)
    t, rb, tms = weo.wilson_eo_tune(op.handle, 12, stream)
    lanes = weo.wilson_eo_get_launch(op.handle)[2]
    res["tuned"] = {"threads": t, "rhs_per_thread": rb, "rhs_lanes": lanes,
                    "tile_links": weo.wilson_eo_get_tile_links(op.handle), "ms_per_meo": round(tms, 4),
                    "gflops": round(12 * FLOP_PER_SITE * V / (tms * 1e-3) / 1e9, 1),
                    "two_pass_model_bytes": int((576 + 240 * 12) * V),
                    "two_pass_model_frac": round((576 + 240 * 12) * V / (tms * 1e-3) / 1e9
                                                 / measured_peaks()[0], 4)}
    out["multi_rhs_12_point_sources_f32"] = res
    del x, y, z
    # 16 right-hand sides: the 12 point sources and 4 Gaussian vectors (seed 9)
    g4 = np.moveaxis(gen.gaussian_spinor(DIMS, nrhs=4, seed=9), 1, -1).astype(np.complex64)
    x = torch.from_numpy(np.concatenate([src, g4])).to(dev)
    y, z = torch.empty_like(x), torch.empty_like(x)
    t, rb, tms = weo.wilson_eo_tune(op.handle, 16, stream)
    lanes = weo.wilson_eo_get_launch(op.handle)[2]
    ms = timed(lambda: (weo.wilson_eo_apply(op.handle, y, x, 16, stream),
                        weo.wilson_eo_apply_dag(op.handle, z, y, 16, stream)), 20, stream)
    out["multi_rhs_16_f32"] = {"rhs": "12 spin-colour point sources + 4 Gaussian (seed 9)",
                               "threads": t, "rhs_per_thread": rb, "rhs_lanes": lanes,
                               "tile_links": weo.wilson_eo_get_tile_links(op.handle),
                               "ms_per_step": round(ms, 4),
                               "gflops": round(16 * 2 * FLOP_PER_SITE * V / (ms * 1e-3) / 1e9, 1),
                               "two_pass_model_frac": round(2 * (576 + 240 * 16) * V / (ms * 1e-3) / 1e9
                                                            / measured_peaks()[0], 4)}
    del x, y, z
    # force: chi = M phi forward, backward M^dag g + link gradient (FP32)
    from paper_2303_08609_gb300.autograd import pseudofermion_action

    Ur = Ud.to(torch.complex64)
    opf = weo.WilsonEO(DIMS, KAPPA, Ur, prec="f32")
    Ur.requires_grad_(True)
    phi = torch.from_numpy(np.ascontiguousarray(np.moveaxis(psi, 0, -1)).astype(np.complex64)).to(dev)
    phi.requires_grad_(True)

    def fwd_bwd():
        Ur.grad = None
        phi.grad = None
        S = pseudofermion_action(phi, Ur, opf, refresh=False)
        S.backward()

    ms = timed(fwd_bwd, 20, stream)
    out["force_fwd_bwd_f32"] = {"ms_per_step": round(ms, 4),
                                "note": "S=|M_eo phi|^2: M_eo forward, M_eo^dag + link gradient backward"}
    opf.close()
    op.close()
    del Ud, Ur, phi
    # one persistent launch over 16^4, 24^3x48, 32^3x64 (independent Haar links)
    r = np.random.default_rng(5)
    ops, xs, ys, sites = [], [], [], 0
    for dims, seed in (((16, 16, 16, 16), 1), ((24, 24, 24, 48), 2), ((32, 32, 32, 64), 3)):
        Uh = gen.gauge_field(dims, "haar", seed=seed)
        ops.append(weo.WilsonEO(dims, float(r.uniform(0.12, 0.135)), torch.from_numpy(Uh).to(dev),
                                prec="f32"))
        p_ = gen.gaussian_spinor(dims, seed=seed + 20)[0]
        xs.append(torch.from_numpy(np.ascontiguousarray(np.moveaxis(p_, 0, -1)).astype(np.complex64)).to(dev))
        ys.append(torch.empty_like(xs[-1]))
        sites += int(np.prod(dims))
        del Uh
    hs = [o.handle for o in ops]
    ms_b = timed(lambda: weo.wilson_eo_apply_batch(hs, ys, xs, False, stream), 50, stream)
    ms_s = timed(lambda: [weo.wilson_eo_apply(o.handle, yy, xx, 1, stream)
                          for o, yy, xx in zip(ops, ys, xs)], 50, stream)
    out["batch_16_24_32_f32"] = {"ms_one_launch": round(ms_b, 4), "ms_separate_applies": round(ms_s, 4),
                                 "gflops_one_launch": round(FLOP_PER_SITE * sites / (ms_b * 1e-3) / 1e9, 1)}
    # the same three lattices with 4 right-hand sides each: one launch (tiles whose
    # links sit in shared memory) against one multi-RHS apply per lattice
    xs4 = [torch.cat([xx.unsqueeze(0)] * 4) for xx in xs]
    ys4 = [torch.empty_like(xx) for xx in xs4]
    ms_b4 = timed(lambda: weo.wilson_eo_apply_batch_rhs(hs, ys4, xs4, [4, 4, 4], False, stream), 20, stream)
    ms_s4 = timed(lambda: [weo.wilson_eo_apply(o.handle, yy, xx, 4, stream)
                           for o, yy, xx in zip(ops, ys4, xs4)], 20, stream)
    out["batch_16_24_32_f32_4rhs"] = {"ms_one_launch": round(ms_b4, 4), "ms_separate_applies": round(ms_s4, 4),
                                      "gflops_one_launch": round(4 * FLOP_PER_SITE * sites / (ms_b4 * 1e-3) / 1e9, 1)}
    del xs4, ys4
    for o in ops:
        o.close()
    return out


def multi_solve_comparison(U, dev):
    """12 spin-colour point sources at one even site on the benchmark lattice
    (32^3 x 64, kappa = 0.13), solved together to true residual 1e-10:
    FP16-storage mixed CG vs plain FP64 CG, both with all 12 systems in lockstep."""
    import torch

    import paper_2303_08609_gb300 as weo

    V = int(np.prod(DIMS))
    vh = V // 2
    site = int(np.random.default_rng(3).integers(vh))
    b = torch.zeros((12, 4, 3, vh), dtype=torch.complex128, device=dev)
    for s_ in range(4):
        for c in range(3):
            b[3 * s_ + c, s_, c, site] = 1.0
    Ud = torch.from_numpy(U).to(dev)
    res = {"lattice": list(DIMS), "kappa": KAPPA, "nrhs": 12, "tol": 1e-10}
    for name, prec, mixed in (("mixed_f16", "f16", True), ("mixed_f32", "f32", True),
                              ("plain_f64", "f64", False)):
        op = weo.WilsonEO(DIMS, KAPPA, Ud, prec=prec)
        # the operator's launch configuration for 12 right-hand sides, tuned
        weo.wilson_eo_tune(op.handle, nrhs=12)
        threads, rb, lanes = weo.wilson_eo_get_launch(op.handle)
        cfg = dict(weo.wilson_eo_get_algorithm(op.handle), threads=threads, rhs_per_thread=rb,
                   rhs_lanes=lanes, tile_links=weo.wilson_eo_get_tile_links(op.handle))
        try:
            x, info = op.solve(b, tol=1e-10, maxiter=20000, mixed=mixed)
            res[name] = {"seconds": round(info["seconds"], 4), "iterations": info["iterations"],
                         "reliable_updates": info["reliable_updates"],
                         "max_true_relres": max(info["true_relres"]), "converged": info["converged"],
                         "tuned": cfg}
            if name == "mixed_f16" and info["converged"]:
                # every system's residual recomputed by the FP64 oracle (not timed)
                xh = np.moveaxis(x.cpu().numpy(), -1, -3)
                bh = np.moveaxis(b.cpu().numpy(), -1, -3)
                res[name]["oracle_max_true_relres"] = max(
                    oracle_relres(U, KAPPA, xh[r], bh[r], DIMS) for r in range(12))
            del x
        except weo.WilsonEOError as exc:
            res[name] = {"error": str(exc)}
        op.close()
        torch.cuda.empty_cache()
    if res["plain_f64"].get("converged") and res["mixed_f16"].get("converged"):
        res["speedup_f16_vs_plain_f64"] = round(res["plain_f64"]["seconds"] / res["mixed_f16"]["seconds"], 2)
    return res


# solves of the default run (the others are selectable with --solve-variants)
DEFAULT_SOLVES = ("mixed_f16_fused", "mixed_bf16_fused", "mixed_f32_fused", "mixed_f16_two_pass",
                  "mixed_f16_l12_two_pass", "mixed_f16_l12_tuned", "mixed_bf16_l12_two_pass",
                  "mixed_bf16_two_pass_keep", "plain_f64")


def oracle_relres(U, kappa, x, b, dims):
    """|b - M^dag M x| / |b| recomputed by the FP64 oracle on all host cores
    (x, b in the oracle's (V/2, 4, 3) layout). A check of the GPU's answer,
    run outside every timed region."""
    import oracle

    oracle.set_threads(os.cpu_count() or 1)
    ax = oracle.meo_dag(U, kappa, oracle.meo(U, kappa, x, dims), dims)
    return float(np.linalg.norm(b - ax) / np.linalg.norm(b))


def solve_comparison(dev, dims, only=None):
    """Solve M^dag M x = b to true relative residual 1e-10 at kappa = 0.135 with
    exp(i 0.4 H) links: FP16-storage mixed CG vs plain FP64 CG, same GPU."""
    import torch

    import gen
    import paper_2303_08609_gb300 as weo

    t0 = time.perf_counter()
    U = gen.gauge_field(dims, "smooth", seed=0, eps=0.4)
    b = gen.gaussian_spinor(dims, seed=1)[0]
    gen_s = time.perf_counter() - t0
    Ud = torch.from_numpy(U).to(dev)
    bd = torch.from_numpy(np.ascontiguousarray(np.moveaxis(b, 0, -1))).to(dev)
    res = {"lattice": list(dims), "kappa": 0.135, "tol": 1e-10, "field_gen_s": round(gen_s, 1),
           "note": "fused: inner M_eo in one persistent launch (first hop 4 t-slices ahead); "
                   "two_pass: two hop launches; both keep the odd intermediate in 16-bit "
                   "for 16-bit handles and give identical iterates; reliable-update residuals "
                   "in float-float with an FP64 check before convergence, fp64res: native FP64 "
                   "residuals"}
    for name, prec, mixed, algo in (("mixed_f16_fused", "f16", True, 1),
                                    ("mixed_bf16_fused", "bf16", True, 1),
                                    ("mixed_f32_fused", "f32", True, 1),
                                    ("mixed_f16_two_pass", "f16", True, 0),
                                    ("mixed_f16_l12_two_pass", "f16", True, 0),
                                    ("mixed_f16_two_pass_fp64res", "f16", True, 0),
                                    ("mixed_f16_two_pass_delta0.03", "f16", True, 0),
                                    ("mixed_f16_l12_tuned", "f16", True, 0),
                                    ("mixed_bf16_two_pass", "bf16", True, 0),
                                    ("mixed_bf16_l12_two_pass", "bf16", True, 0),
                                    ("mixed_bf16_two_pass_keep", "bf16", True, 0),
                                    ("mixed_bf16_l12_two_pass_keep", "bf16", True, 0),
                                    ("mixed_f16_l12_restart", "f16", True, 0),
                                    ("plain_f64", "f64", False, 0),
                                    ("plain_f64_tuned", "f64", False, 0)):
        if (only and name not in only) or (not only and name not in DEFAULT_SOLVES):
            continue
        op = weo.WilsonEO(dims, 0.135, Ud, prec=prec, linkfmt=12 if "_l12" in name else 18)
        if algo:
            weo.wilson_eo_set_algorithm(op.handle, "fused", 4, 128)
        if "delta" in name:
            weo.wilson_eo_solver_config(op.handle, delta=float(name.split("delta")[1]))
        if name.endswith("fp64res"):
            weo.wilson_eo_solver_residual(op.handle, 0)
        if "restart" in name:  # defect correction: new direction at every reliable update
            weo.wilson_eo_solver_restart(op.handle, 1)
        if name.endswith("_keep"):  # directions kept across reliable updates
            weo.wilson_eo_solver_restart(op.handle, 0)
        if name.endswith("_tuned"):  # autotuned operator (tuning not timed)
            weo.wilson_eo_tune(op.handle, nrhs=1)
            res.setdefault("tuned", {})[name] = {**weo.wilson_eo_get_algorithm(op.handle),
                                                 "launch": list(weo.wilson_eo_get_launch(op.handle))}
        try:
            x, info = op.solve(bd, tol=1e-10, maxiter=20000, mixed=mixed)
            res[name] = {k: (round(v, 4) if isinstance(v, float) and k == "seconds" else v)
                         for k, v in info.items()}
            if info["converged"]:
                # the oracle's own FP64 residual of the returned x (after the timing)
                res[name]["oracle_true_relres"] = oracle_relres(
                    U, 0.135, np.moveaxis(x.cpu().numpy(), -1, 0), b, dims)
            del x
        except weo.WilsonEOError as exc:
            res[name] = {"error": str(exc)}
        op.close()
        torch.cuda.empty_cache()
    done = [(v["seconds"], k) for k, v in res.items()
            if isinstance(v, dict) and v.get("converged") and k.startswith("mixed")]
    best = min(done) if done else None
    plain = [v["seconds"] for k, v in res.items()
             if k.startswith("plain_f64") and isinstance(v, dict) and v.get("converged")]
    if plain and best:
        # against the faster of the plain FP64 solves (default and tuned operator)
        res["fastest_mixed"] = best[1]
        res["speedup_vs_plain_f64"] = round(min(plain) / best[0], 2)
    return res


def cpu_model():
    """Host CPU model as lscpu reports it (Grace reports its Neoverse core)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def slab(U, psi, T):
    """The workload's first T time slices as a periodic Lx x Ly x Lz x T lattice:
    every site does the same work as in the full lattice (only the wrap in t
    differs), so its throughput samples the full workload's."""
    lx, ly, lz, lt = DIMS
    V3 = lx * ly * lz
    Us = np.ascontiguousarray(U.reshape(4, lt, V3, 3, 3)[:, :T].reshape(4, T * V3, 3, 3))
    return Us, np.ascontiguousarray(psi[: T * V3 // 2]), (lx, ly, lz, T)


def oracle_step_seconds(U, psi, dims, reps):
    import oracle

    t0 = time.perf_counter()
    for _ in range(reps):
        yv = oracle.meo(U, KAPPA, psi, dims)
        oracle.meo_dag(U, KAPPA, yv, dims)
    return (time.perf_counter() - t0) / reps


def cpu_baseline(U, psi, reps=3):
    """The FP64 oracle on the workload step: OpenMP over all host cores on the full
    32^3 x 64 lattice, and one thread on an 8-slice sample of it."""
    import oracle

    threads = os.cpu_count() or 1
    V = int(np.prod(DIMS))
    oracle.set_threads(threads)
    dt = oracle_step_seconds(U, psi, DIMS, reps)
    used = oracle.get_threads()
    oracle.set_threads(1)
    Us, ps, sd = slab(U, psi, min(8, DIMS[3]))
    dt1 = oracle_step_seconds(Us, ps, sd, 1)
    oracle.set_threads(threads)
    return {"value": round(2 * FLOP_PER_SITE * V / dt / 1e9, 3), "unit": "GFlop/s",
            "cores": used, "kind": "oracle",
            "sample": f"{reps} full step(s) of the workload (M_eo then M_eo^dag, FP64, "
                      f"{'x'.join(map(str, DIMS))}), {dt:.2f} s each",
            "single_thread": {"value": round(2 * FLOP_PER_SITE * np.prod(sd) / dt1 / 1e9, 3),
                              "sample": f"one step on the first {sd[3]} time slices "
                                        f"({'x'.join(map(str, sd))}, periodic), {dt1:.2f} s"},
            "cpu_model": cpu_model()}


def oracle_plan(budget_s=40.0):
    """The FP64 oracle on the small workloads: M_eo and CG on M^dag M to 1e-10
    at 8^4 (kappa = 0.125, Haar links) and 16^4 (kappa = 0.13, exp(i 0.4 H)
    links), on all host cores and on one core. A one-core CG is skipped, with
    its estimate, when the all-core time says it would take over budget_s."""
    import gen
    import oracle

    cores = os.cpu_count() or 1
    out = {"cores": cores, "cpu_model": cpu_model()}
    for dims, kappa, kind in (((8, 8, 8, 8), 0.125, "haar"), ((16, 16, 16, 16), 0.13, "smooth")):
        U = gen.gauge_field(dims, kind, seed=0, eps=0.4)
        b = gen.gaussian_spinor(dims, seed=0)[0]
        V = int(np.prod(dims))
        ent = {"kappa": kappa, "links": kind}
        t_cg_all = None
        for threads in (cores, 1):
            oracle.set_threads(threads)
            key = "all_cores" if threads == cores else "one_core"
            reps, t0 = 0, time.perf_counter()
            while reps < 3 or time.perf_counter() - t0 < 0.5:
                oracle.meo(U, kappa, b, dims)
                reps += 1
            dt = (time.perf_counter() - t0) / reps
            row = {"meo_ms": round(dt * 1e3, 3),
                   "meo_gflops": round(FLOP_PER_SITE * V / dt / 1e9, 3)}
            est = None if t_cg_all is None else t_cg_all * dt / ent["all_cores"]["meo_ms"] * 1e3
            if threads == 1 and est is not None and est > budget_s:
                row["cg_skipped"] = f"estimated {est:.0f} s on one core"
            else:
                t0 = time.perf_counter()
                _, it, rr, ok = oracle.cg(U, kappa, b, dims, tol=1e-10, maxiter=20000)
                tcg = time.perf_counter() - t0
                if threads == cores:
                    t_cg_all = tcg
                row.update({"cg_seconds": round(tcg, 3), "cg_iterations": it, "cg_true_relres": rr,
                            "cg_converged": ok})
            ent[key] = row
        out["x".join(map(str, dims))] = ent
    oracle.set_threads(cores)
    return out


# wall-clock budget of a whole reference-arm run (warm-up plus timed steps)
REFERENCE_BUDGET_S = 150.0


def run_reference(args, rank, world, local):
    """Reference arm: the FP64 CPU oracle, timed on the host cores. Each step is
    M_eo then M_eo^dag on the workload's first T time slices (a periodic
    sub-lattice with the same per-site work), T chosen so that warm-up plus
    K steps stay within a few minutes; T = 64 is the whole workload."""
    if rank != 0:
        return
    import oracle

    U, psi = fields()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    lt = DIMS[3]
    # size the sample from one 2-slice step (it doubles as the first warm-up)
    Us, ps, sd = slab(U, psi, 2)
    per_slice = oracle_step_seconds(Us, ps, sd, 1) / 2
    n_steps = args.steps + max(1, args.warmup)
    T = int(REFERENCE_BUDGET_S / max(n_steps * per_slice, 1e-9))
    T = max(2, min(lt, T - T % 2))
    Us, ps, sd = slab(U, psi, T)
    for _ in range(max(1, args.warmup) - 1):
        oracle_step_seconds(Us, ps, sd, 1)
    dt = oracle_step_seconds(Us, ps, sd, args.steps)
    V = int(np.prod(sd))
    value = 2 * FLOP_PER_SITE * V / dt / 1e9
    sample = (f"each step: M_eo then M_eo^dag (FP64) on the first {T} of {lt} time slices of the "
              f"workload ({'x'.join(map(str, sd))}, periodic in t), {dt:.3f} s")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFlop/s",
           "n_gpus": world, "steps": args.steps, "warmup": max(1, args.warmup),
           "ms_per_step": round(dt * 1e3, 2), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args, world), "sample_lattice": list(sd),
           "cpu_baseline": {"value": round(value, 3), "unit": "GFlop/s",
                            "cores": oracle.get_threads(), "kind": "oracle", "sample": sample,
                            "cpu_model": cpu_model()},
           "e2e": {"value": round(value, 3), "unit": "GFlop/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def multi_rhs_only(args, local):
    """M_eo then M_eo^dag on args.only_multi_rhs Gaussian right-hand sides
    (seed 0), operator autotuned for that count (or with args.tile_links fixed);
    CUDA-event timing of args.steps steps after args.warmup."""
    import torch

    import gen
    import paper_2303_08609_gb300 as weo

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.only_multi_rhs
    U = gen.gauge_field(DIMS, "smooth", seed=0, eps=EPS)
    V = int(np.prod(DIMS))
    op = weo.WilsonEO(DIMS, KAPPA, torch.from_numpy(U).to(dev), prec=args.prec, linkfmt=args.linkfmt)
    del U
    x = torch.from_numpy(np.ascontiguousarray(np.moveaxis(gen.gaussian_spinor(DIMS, nrhs=n, seed=0), 1, -1))
                         .astype(np.complex128 if args.prec == "f64" else np.complex64)).to(dev)
    y, z = torch.empty_like(x), torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    if args.tile_links >= 0:
        weo.wilson_eo_set_tile_links(op.handle, args.tile_links, args.tile_rpt)
    else:
        weo.wilson_eo_tune(op.handle, n, stream)
    t, rb, lanes = weo.wilson_eo_get_launch(op.handle)
    tl = weo.wilson_eo_get_tile_links(op.handle)

    def step():
        weo.wilson_eo_apply(op.handle, y, x, n, stream)
        weo.wilson_eo_apply_dag(op.handle, z, y, n, stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ms = timed(step, args.steps, stream)
    op.close()
    print(json.dumps({"nrhs": n, "lattice": list(DIMS), "prec": args.prec, "linkfmt": args.linkfmt,
                      "threads": t, "rhs_per_thread": rb, "rhs_lanes": lanes, "tile_links": tl,
                      "ms_per_step": round(ms, 4),
                      "gflops": round(n * 2 * FLOP_PER_SITE * V / (ms * 1e-3) / 1e9, 1)}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.only_multi_rhs:
        multi_rhs_only(args, local)
        return
    if args.only_solve:
        import torch

        torch.cuda.set_device(local)
        print(json.dumps({"solve": solve_comparison(torch.device("cuda", local),
                                                    tuple(args.solve_dims), args.solve_variants)}),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
