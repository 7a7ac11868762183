"""Benchmark: batched mixed-precision CGNE on the 32^3 x 64 Wilson-clover workload.

One step = one call of the library's CGNE (Sec. 2: CG on the normal
equations with binary64 reset steps) that solves Dhat^dag Dhat psi = eta for
the 12 spin-colour point sources at the origin at once (eta = Dhat^dag bhat,
bhat the even part of the source), storage binary16, arithmetic binary32,
binary64 resets / solution / reductions, stopping at a binary64 relative
residual of 1e-10 for every right-hand side.

value    = algorithmic bytes of all stencil launches of the timed steps
           (each operand counted once) / wall time of those steps [GB/s]
roofline = the dominant stencil kernel: its algorithmic bytes per launch /
           its mean CUDA-event duration, against the measured HBM copy peak
e2e      = the same bytes / time of the public call with host buffers
           (pinned host -> device copy of eta, solve, device -> host psi)
tts      = time to solution of one right-hand side: binary64-only CGNE vs
           the mixed-precision solves (the "vs plain FP64 GPU" comparison)

--impl reference times the FP64 CPU oracle instead (a bounded sample: the
oracle's Dhat^dag Dhat on one right-hand side of a 4 x 32^3 slab with the
same per-site work), reporting the same metric.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dw GB/s & % of HBM roofline; CGNE/GCR time-to-1e-10 residual vs plain FP64 GPU"
DIMS = (64, 32, 32, 32)          # T x L^3
EPS, SEED, KAPPA, CSW = 0.6, 3, 0.135, 1.0
NRHS = 12
RES = 1e-10
SLAB = (4, 32, 32, 32)           # oracle sample: same spatial extent, 4 time slices
MODE_NAMES = {0: "dw_full", 1: "dw_hat_pass1_odd", 2: "dw_hat_pass2_even"}
EPI_NAMES = {0: "store", 1: "store+norm", 2: "cg_update", 3: "fp64_residual"}
PREC_NAMES = {0: "f64", 1: "f32", 2: "bf16", 3: "f16"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def traffic_for(kernel_key):
    """ncu DRAM bytes per launch recorded for this kernel, if the kernel source is unchanged since."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha256()
    for f in ("hop_impl.cuh", "oq_device.cuh", "reduce.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2202_07388_gb300", "csrc", f), "rb").read())
    if d.get("source_sha256") != h.hexdigest():
        return None
    ent = d.get("kernels", {}).get(kernel_key)
    if not ent:
        return None
    # recorded on a capture of `sites` output sites; scale to the bench launch
    return ent


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_sample_setup():
    from oracle import dirac
    from paper_2202_07388_gb300 import synth
    u = synth.make_gauge(SLAB, EPS, SEED)
    a = dirac.clover_field(u, dirac.kappa_to_m0(KAPPA), CSW)
    ainv = np.linalg.inv(a)
    eta = dirac.even_part(synth.make_source(SLAB, SEED + 1))
    return u, a, ainv, eta


def oracle_step(case):
    from oracle import dirac
    u, a, ainv, eta = case
    return dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, eta))


def algo_bytes_normal_op(ve_sites, prec_bytes, link_reals, nrhs):
    """Algorithmic bytes of one Dhat^dag Dhat (4 stencil passes) on ve_sites even sites."""
    per_pass_p1 = 48 * prec_bytes * nrhs + 8 * link_reals * 4 + 72 * 4
    per_pass_p2 = 72 * prec_bytes * nrhs + 8 * link_reals * 4 + 72 * 4
    return 2 * (per_pass_p1 + per_pass_p2) * ve_sites


def cpu_time_oracle(reps):
    """Wall and CPU time of `reps` oracle Dhat^dag Dhat applications on the slab."""
    case = oracle_sample_setup()
    oracle_step(case)  # warm-up
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(reps):
        oracle_step(case)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    ve = int(np.prod(SLAB)) // 2
    # bytes the same work would move in the GPU step's storage (f16 spinors, 12-real f32 links)
    byts = algo_bytes_normal_op(ve, 2, 12, 1) * reps
    return wall, cpu, byts


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = oracle_sample_setup()
    for _ in range(args.warmup):
        oracle_step(case)
    ve = int(np.prod(SLAB)) // 2
    per = algo_bytes_normal_op(ve, 2, 12, 1)
    times = []
    c0 = time.process_time()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = time.perf_counter()
        oracle_step(case)
        times.append(time.perf_counter() - s)
    wall = time.perf_counter() - t0
    cores = max(1, round((time.process_time() - c0) / wall))
    value = per * args.steps / wall / 1e9
    sample = (f"oracle (NumPy FP64) Dhat^dag Dhat on one rhs of a {SLAB[0]}x{SLAB[1]}^3 slab "
              f"(same per-site work as the 32^3x64 step), bytes counted as the GPU step's f16 workload")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config():
    return {"workload": "32^3x64 Wilson-clover, 12 point-source rhs, batched mixed-precision CGNE to 1e-10",
            "lattice": "x".join(str(d) for d in DIMS), "eps": EPS, "kappa": KAPPA, "csw": CSW,
            "bc_t": "antiperiodic", "nrhs": NRHS, "storage": "f16 spinors, 12-real f32 links, f32 clover",
            "resets": "f64", "res": RES, "seed": SEED,
            "l2": "inputs larger than L2 (links 403 MB, clover 1.2 GB, spinors 48 MB/rhs)"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64)).cuda()


def run_ours(args):
    import torch
    from paper_2202_07388_gb300 import oq, synth
    from paper_2202_07388_gb300 import build as _build

    ws, rank, local = dist_env()
    _build.build()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # cpu baseline first (no CUDA work in flight, rank 0 at N=1 only)
    cpu_line = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        wall, cpu, byts = cpu_time_oracle(args.cpu_reps)
        cpu_line = {"value": byts / wall / 1e9, "unit": "GB/s", "cores": max(1, round(cpu / wall)),
                    "kind": "oracle",
                    "sample": f"{args.cpu_reps} oracle (NumPy FP64) Dhat^dag Dhat on one rhs of a "
                              f"{SLAB[0]}x{SLAB[1]}^3 slab ({wall:.1f} s), bytes counted as the GPU step's "
                              f"f16 workload"}

    t_setup = time.perf_counter()
    u = synth.make_gauge(DIMS, EPS, SEED + 1000 * rank)
    h = oq.Handle(DIMS)
    ud = to_dev(u)
    del u
    h.gauge_upload(ud, oq.LINK_12)
    h.clover_build(KAPPA, CSW)
    del ud
    torch.cuda.synchronize()
    # eta = Dhat^dag bhat for the 12 point sources (bhat = b_e: the origin is even)
    src = synth.make_point_sources(DIMS)
    src_d = to_dev(src)
    del src
    pk = h.new_packed(oq.F64, oq.EVEN, nrhs=NRHS)
    pk2 = h.new_packed(oq.F64, oq.EVEN, nrhs=NRHS)
    h.pack(src_d, pk, oq.F64, oq.EVEN, nrhs=NRHS)
    h.dw_hat(pk, pk2, oq.F64, nrhs=NRHS, dagger=True)
    eta = torch.zeros_like(src_d)
    h.unpack(pk2, eta, oq.F64, oq.EVEN, nrhs=NRHS)
    del pk, pk2, src_d
    psi = torch.zeros_like(eta)
    prm = oq.SolverParams(res=RES, nmx=20000, sdtype=oq.F16)
    tuned = {}
    for pname, pc, nr in (("f16", oq.F16, NRHS), ("f64", oq.F64, NRHS)):
        tuned[f"{pname}x{nr}"] = {MODE_NAMES[m]: v for m, v in h.autotune(pc, nrhs=nr).items()}
    if not args.no_tts:
        for pname, pc in (("f64", oq.F64), ("f32", oq.F32), ("bf16", oq.BF16), ("f16", oq.F16)):
            tuned[f"{pname}x1"] = {MODE_NAMES[m]: v for m, v in h.autotune(pc, nrhs=1).items()}
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    statuses = []
    for _ in range(args.warmup):
        rc, st = h.cgne(eta, psi, prm, nrhs=NRHS)
        assert rc == oq.OK, rc
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    n0 = h.kernel_launches()
    h.profile_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            rc, st = h.cgne(eta, psi, prm, nrhs=NRHS)
            assert rc == oq.OK, rc
            statuses.append(st)
        ev1.record()
        torch.cuda.synchronize()
    prof = h.profile_stop()
    launches = h.kernel_launches() - n0
    t_ms = ev0.elapsed_time(ev1)
    if ws > 1:
        tt = torch.tensor([t_ms], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_ms = float(tt.item())
    stencil_bytes = sum(p["bytes"] for p in prof)
    total_bytes = stencil_bytes * ws
    value = total_bytes / (t_ms * 1e-3) / 1e9

    # dominant kernel
    dom = max(prof, key=lambda p: p["total_ms"])
    avg_ms = dom["total_ms"] / dom["launches"]
    achieved = (dom["bytes"] / dom["launches"]) / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    key = f"{MODE_NAMES[dom['mode']]}/{EPI_NAMES[dom['epi']]}/{PREC_NAMES[dom['prec']]}"
    tr = traffic_for(key)
    traffic = None
    if tr:
        traffic = tr["dram_bytes_per_site"] * (int(np.prod(DIMS)) // 2) * (NRHS if tr.get("per_rhs") else 1)

    # end to end through the public call with host buffers
    eta_host = eta.cpu().pin_memory()
    psi_host = torch.empty_like(eta_host).pin_memory()
    eta_dev2 = torch.empty_like(eta)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.e2e_steps):
        eta_dev2.copy_(eta_host, non_blocking=True)
        rc, _ = h.cgne(eta_dev2, psi, prm, nrhs=NRHS)
        assert rc == oq.OK
        psi_host.copy_(psi, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    e2e_value = (stencil_bytes / args.steps) / (e2e_ms * 1e-3) / 1e9

    # time to solution, one rhs: binary64 only vs mixed precision
    tts = None
    if not args.no_tts:
        eta1 = eta.view(NRHS, -1)[0:1].contiguous()
        psi1 = torch.zeros_like(eta1)
        tts = {}
        for name, sd in (("fp64", oq.F64), ("fp32", oq.F32), ("bf16", oq.BF16), ("fp16", oq.F16)):
            p1 = oq.SolverParams(res=RES, nmx=50000, sdtype=sd)
            h.cgne(eta1, psi1, p1, nrhs=1)  # warm
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            rc, st1 = h.cgne(eta1, psi1, p1, nrhs=1)
            torch.cuda.synchronize()
            tts[name] = {"s": time.perf_counter() - s0, "steps": st1[0]["steps"], "resets": st1[0]["resets"],
                         "true_rel_res": st1[0]["true_rel_res"], "converged": st1[0]["converged"]}
        tts["speedup_fp16_vs_fp64"] = tts["fp64"]["s"] / tts["fp16"]["s"]
        tts["batched_12rhs_f16_s_per_rhs"] = (t_ms * 1e-3 / args.steps) / NRHS
        tts["speedup_batched_f16_vs_fp64_per_rhs"] = tts["fp64"]["s"] / tts["batched_12rhs_f16_s_per_rhs"]

    st_last = statuses[-1]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": key,
                         "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                         "avg_launch_ms": avg_ms, "launches": dom["launches"]},
            "cpu_baseline": cpu_line,
            "e2e": {"value": e2e_value, "unit": "GB/s",
                    "h2d_bytes_per_step": int(eta.numel() * 8), "d2h_bytes_per_step": int(psi.numel() * 8),
                    "ms_per_step": e2e_ms},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "solve": {"steps": [s["steps"] for s in st_last], "resets": [s["resets"] for s in st_last],
                      "max_true_rel_res": max(s["true_rel_res"] for s in st_last)},
            "kernels": [{"kernel": f"{MODE_NAMES[p['mode']]}/{EPI_NAMES[p['epi']]}/{PREC_NAMES[p['prec']]}",
                         "launches": p["launches"], "ms": p["total_ms"],
                         "gbs": p["bytes"] / (p["total_ms"] * 1e-3) / 1e9} for p in prof],
            "tts": tts, "setup_s": setup_s, "tuned_shapes": tuned,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_profile_case(args):
    """A small case for ncu captures of the stencil kernels: 32 x 32^3 lattice
    (links + clover 0.5 GB, larger than L2), 12 rhs in F16 storage, a few Dhat and
    Dhat^dag applications with the tuned launch shapes."""
    import torch
    from paper_2202_07388_gb300 import oq, synth
    from paper_2202_07388_gb300 import build as _build
    _build.build()
    dims = (32, 32, 32, 32)
    u = synth.make_gauge(dims, EPS, SEED)
    h = oq.Handle(dims)
    h.gauge_upload(to_dev(u), oq.LINK_12)
    h.clover_build(KAPPA, CSW)
    prec = oq.PREC[args.profile_prec]
    nrhs = args.profile_nrhs
    h.autotune(prec, nrhs=nrhs)
    src = torch.randn(nrhs * int(np.prod(dims)) * 24, dtype=torch.float64, device="cuda")
    a, b = h.new_packed(prec, oq.EVEN, nrhs=nrhs), h.new_packed(prec, oq.EVEN, nrhs=nrhs)
    h.pack(src, a, prec, oq.EVEN, nrhs=nrhs)
    for _ in range(3):
        h.dw_hat(a, b, prec, nrhs=nrhs)
        h.dw_hat(b, a, prec, nrhs=nrhs, dagger=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "x".join(map(str, dims)), "prec": args.profile_prec, "nrhs": nrhs,
                      "launches": h.kernel_launches()}))
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", action="store_true")
    ap.add_argument("--profile-prec", default="fp16", choices=["fp64", "fp32", "bf16", "fp16"])
    ap.add_argument("--profile-nrhs", type=int, default=12)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-reps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tts", action="store_true")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
