"""Benchmark: batched mixed-precision CGNE on the 32^3 x 64 Wilson-clover workload.

One step = one call of the library's CGNE (Sec. 2: CG on the normal
equations with binary64 reset steps) that solves Dhat^dag Dhat psi = eta for
the 12 spin-colour point sources at the origin at once (eta = Dhat^dag bhat,
bhat the even part of the source), storage binary16, arithmetic binary32,
binary64 resets / solution / reductions, stopping at a binary64 relative
residual of 1e-10 for every right-hand side.

value    = algorithmic bytes of the stencil launches of the timed steps
           (each operand counted once; a launch's links and clover once, its
           spinors once per right-hand side live in it, as the kernels record;
           launches whose right-hand sides were all gated off by the solver
           state move nothing) / wall time of those steps [GB/s]
roofline = the dominant stencil source kernel (plain and adjoint
           instantiations summed): its algorithmic bytes per launch / its mean
           CUDA-event duration over launches that did work, against the
           measured HBM copy peak
e2e      = the same bytes / time of the public call with host buffers
           (even-site canonical fields, oq_cgne_solve_even): the pinned host
           buffers go to the solver, whose packing kernel reads the sources
           and unpacking kernel writes the solutions over the host-device
           link; copy-engine variants (pipelined on a second stream, serial,
           full-lattice fields) are reported next to it
tts      = time to solution of one right-hand side: binary64-only CGNE vs
           the mixed-precision solves (the "vs plain FP64 GPU" comparison),
           and the precision ladders (one and 12 right-hand sides)

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
FP64_PEAK_TFLOPS = 1.25          # GB300 nominal binary64 rate (no measured figure available)
# GB300 binary32 FMA rate from unit counts and clock: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12     # binary32 pipe operations (an FMA counts once)
SLAB = (4, 32, 32, 32)           # oracle sample: same spatial extent, 4 time slices
MODE_NAMES = {0: "dw_full", 1: "dw_hat_pass1_odd", 2: "dw_hat_pass2_even"}
EPI_NAMES = {0: "store", 1: "store+norm", 2: "cg_update", 3: "fp64_residual"}
PREC_NAMES = {0: "f64", 1: "f32", 2: "bf16", 3: "f16", 4: "df64"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def max_over_ranks(x, device, ws):
    """The slowest rank's value (timed regions are bracketed by barriers)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device, ws):
    """Work done by all ranks together (each rank solves its own replica)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(total_bytes, t_ms):
    """Whole-job GB/s: bytes of all ranks over the slowest rank's time."""
    return total_bytes / (t_ms * 1e-3) / 1e9


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


def kernel_key(p):
    """Name of a profiled stencil variant: pass / epilogue / storage / rhs per thread / link format
    (/dag for the adjoint instantiation)."""
    fmt = {-1: "u64", 0: "u18", 1: "u12"}[p.get("link_fmt", -1)]
    key = f"{MODE_NAMES[p['mode']]}/{EPI_NAMES[p['epi']]}/{PREC_NAMES[p['prec']]}/nr{p.get('nr', 1)}/{fmt}"
    return key + "/dag" if p.get("dag") else key


def merge_source_kernels(prof):
    """One entry per source kernel: the plain and adjoint instantiations of a
    pass (the same template, the projector sign a compile-time parameter) are
    summed; launches / total_ms / bytes / rhs_launches cover the launches with
    live right-hand sides, gated_* the launches the solver state gated off."""
    out = {}
    for p in prof:
        k = kernel_key(p)
        k = k[:-len("/dag")] if k.endswith("/dag") else k
        if k not in out:
            out[k] = dict(p, dag=0, instantiations=0)
            for f in ("launches", "total_ms", "bytes", "rhs_launches", "gated_launches", "gated_ms"):
                out[k][f] = 0
        for f in ("launches", "total_ms", "bytes", "rhs_launches", "gated_launches", "gated_ms"):
            out[k][f] += p[f]
        out[k]["instantiations"] += 1
    return [v for v in out.values() if v["launches"] > 0]


STENCIL_SOURCES = ("hop_impl.cuh", "hop_mr.cuh", "oq_device.cuh", "reduce.cuh")

# the commands whose ncu logs --write-traffic turns into profiles/traffic.json
TRAFFIC_CASE = "python bench.py --profile-case --profile-kind cgne"
TRAFFIC_COMMANDS = [
    TRAFFIC_CASE,
    "ncu --profile-from-start off -k regex:hop_mr_kernel -c 4 --metrics dram__bytes_read.sum,dram__bytes_write.sum,"
    "gpu__time_duration.sum --clock-control none --csv --log-file traffic_f16.csv " + TRAFFIC_CASE,
    "ncu --profile-from-start off -k regex:hop_kernel -c 20 --metrics dram__bytes_read.sum,dram__bytes_write.sum,"
    "gpu__time_duration.sum --clock-control none --csv --log-file traffic_reset.csv " + TRAFFIC_CASE,
    "python bench.py --write-traffic traffic_f16.csv traffic_reset.csv",
]


def code_only(text):
    """A CUDA source without its comments and with whitespace collapsed: what the compiler sees
    of it (the stencil sources hold no string literal with a comment marker)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def stencil_source_hash(read=None):
    """sha256 of the stencil sources' code (comments and layout do not count); `read(name)`
    gives a source's text (default: the working tree)."""
    import hashlib
    read = read or (lambda f: open(os.path.join(ROOT, "paper_2202_07388_gb300", "csrc", f)).read())
    h = hashlib.sha256()
    for f in STENCIL_SOURCES:
        h.update(code_only(read(f)).encode())
    return h.hexdigest()


def traffic_kernels(csvs):
    """DRAM bytes per even site of each stencil kernel variant in ncu --csv logs of the cgne
    profile case (32x32^3, 12 rhs): dram__bytes_read.sum + dram__bytes_write.sum per launch / Vh,
    averaged over the variant's launches (named as kernel_key names them, adjoint and plain
    instantiations together)."""
    import csv
    import re
    vh = 32 ** 4 // 2
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    kern = {}
    for path in csvs:
        hdr, launches = None, {}
        for r in csv.reader(open(path)):
            if not r:
                continue
            if "Kernel Name" in r:
                hdr = r
                continue
            if hdr is None or len(r) != len(hdr):
                continue
            d = dict(zip(hdr, r))
            m = launches.setdefault((int(d["ID"]), d["Kernel Name"]), {})
            m[d["Metric Name"]] = float(d["Metric Value"].replace(",", "")) * scale.get(d["Metric Unit"], 1)
        for (_, name), m in launches.items():
            targs = [int(x) for x in re.search(r"<([^>]*)>", name).group(1).split(",")]
            if "hop_mr_kernel" in name:
                prec, fmt, mode, _dag, epi, nr, _cap = targs
            else:
                prec, fmt, mode, _dag, epi = targs
                nr = 1
            lf = -1 if prec in (0, 4) else fmt
            key = kernel_key({"mode": mode, "epi": epi, "prec": prec, "nr": nr, "link_fmt": lf})
            b = (m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"]) / vh
            e = kern.setdefault(key, {"dram_bytes_per_site": 0.0, "launches": 0, "capture": os.path.basename(path)})
            e["dram_bytes_per_site"] = (e["dram_bytes_per_site"] * e["launches"] + b) / (e["launches"] + 1)
            e["launches"] += 1
    return kern


def write_traffic(csvs, path=None):
    """profiles/traffic.json (or `path`): traffic_kernels of the logs, the commands that made
    them and the hash of the stencil sources the capture was taken on."""
    kern = traffic_kernels(csvs)
    out = {"note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch / Vh, 32x32^3 lattice, 12 rhs; "
                   "bench scales by its own Vh; source_sha256: the stencil sources' code without comments",
           "commands": TRAFFIC_COMMANDS, "lattice": "32x32x32x32", "nrhs": 12, "kernels": kern,
           "source_sha256": stencil_source_hash()}
    with open(path or os.path.join(ROOT, "profiles", "traffic.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(kern, indent=1))
    return 0


def traffic_for(kernel_key):
    """ncu DRAM bytes per launch recorded for this kernel, if the kernel source is unchanged since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha256") != stencil_source_hash():
        return None
    # one entry per pass and epilogue: the adjoint instantiation moves the same bytes
    ent = d.get("kernels", {}).get(kernel_key[:-len("/dag")] if kernel_key.endswith("/dag") else kernel_key)
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


C2_CASE = ((32, 16, 16, 16), 0.5, 0.135, 2)     # 32x16^3 workload: dims, eps, kappa, seed


def _oracle_normal_seconds(dims, eps, kappa, seed, reps):
    """Seconds of one oracle Dhat^dag Dhat application (the work of one CG
    iteration on the even-odd system) on one core, mean of reps after one
    warm-up."""
    from oracle import dirac
    from paper_2202_07388_gb300 import synth
    u = synth.make_gauge(dims, eps, seed)
    a = dirac.clover_field(u, dirac.kappa_to_m0(kappa), CSW)
    ainv = np.linalg.inv(a)
    psi = dirac.even_part(synth.make_source(dims, seed + 1))
    normal = lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v))  # noqa: E731
    normal(psi)
    t0 = time.perf_counter()
    for _ in range(reps):
        normal(psi)
    return (time.perf_counter() - t0) / reps


def _pool_normal(_):
    return _oracle_normal_seconds(*C2_CASE, reps=1)


def cpu_baseline_tts():
    """The oracle's binary64 CGNE on the host cores: the 4^4 workload solved to
    1e-10 outright; the 32x16^3 and 64x32^3 workloads by their time per CG
    iteration (one normal-operator application, the 64x32^3 one scaled from
    the 32x16^3 one by the volume, 16x), to be multiplied by the step count of
    the binary64 CGNE (the GPU's, same algorithm and inputs); and all cores at
    once on independent 32x16^3 applications (a spawned process pool, the
    oracle being single-threaded NumPy)."""
    import multiprocessing as mp
    import platform
    from oracle import dirac, solvers
    from paper_2202_07388_gb300 import synth
    out = {"cpu_model": platform.processor() or platform.machine(), "nproc": os.cpu_count()}
    dims = (4, 4, 4, 4)
    u = synth.make_gauge(dims, 0.3, 1)
    a = dirac.clover_field(u, dirac.kappa_to_m0(0.13), CSW)
    ainv = np.linalg.inv(a)
    eta = dirac.even_part(synth.make_source(dims, 2))
    normal = lambda v: dirac.dw_hat_dagger(u, a, ainv, dirac.dw_hat(u, a, ainv, v))  # noqa: E731
    t0 = time.perf_counter()
    r = solvers.cgne(normal, eta, RES, 5000, "fp64")
    out["c1_4x4x4x4_cgne_fp64_s"] = time.perf_counter() - t0
    out["c1_steps"] = int(r.status)
    out["c2_32x16c_s_per_iter_1core"] = _oracle_normal_seconds(*C2_CASE, reps=2)
    out["c3_64x32c_s_per_iter_1core"] = 16.0 * out["c2_32x16c_s_per_iter_1core"]
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    workers = max(1, min(cores, 16))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        per = pool.map(_pool_normal, range(workers))
    wall = time.perf_counter() - t0
    out["all_cores"] = {"workers": workers, "cores": cores, "wall_s": wall,
                        "c2_s_per_iter_per_worker": float(np.mean(per)),
                        "c2_iters_per_s": workers / float(np.mean(per))}
    return out


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
            "resets": "double-float intermediate resets, binary64 final reset", "res": RES, "seed": SEED,
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
    cpu_tts = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu_tts = cpu_baseline_tts()
        per = cpu_tts["c2_32x16c_s_per_iter_1core"]
        ve = int(np.prod(C2_CASE[0])) // 2
        byts = algo_bytes_normal_op(ve, 2, 12, 1)
        cpu_line = {"value": byts / per / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                    "sample": f"oracle (NumPy FP64) Dhat^dag Dhat on one rhs of the 32x16^3 workload "
                              f"({per:.2f} s per application, the same per-site work as the 64x32^3 step), "
                              f"bytes counted as the GPU step's f16 workload; time-to-solution rows in tts"}

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
    for pname, pc, nr in (("f16", oq.F16, NRHS), ("f64", oq.F64, NRHS), ("df64", oq.DF64, NRHS)):
        tuned[f"{pname}x{nr}"] = {MODE_NAMES[m]: v for m, v in h.autotune(pc, nrhs=nr).items()}
    # pass 2 is tuned per epilogue: the launches the solve's norm and CG-update passes run
    tuned[f"f16x{NRHS}"]["dw_hat_pass2_even_by_epilogue"] = h.tuned_epilogues(oq.F16, NRHS)
    if not args.no_tts:
        for pname, pc in (("f64", oq.F64), ("df64", oq.DF64), ("f32", oq.F32), ("bf16", oq.BF16), ("f16", oq.F16)):
            tuned[f"{pname}x1"] = {MODE_NAMES[m]: v for m, v in h.autotune(pc, nrhs=1).items()}
        # the binary32 phase of the batched precision ladder
        tuned[f"f32x{NRHS}"] = {MODE_NAMES[m]: v for m, v in h.autotune(oq.F32, nrhs=NRHS).items()}
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    statuses = []
    # the solves (warm-up and timed) are the range an `ncu --profile-from-start off`
    # launch list covers; set-up and tuning stay outside it
    torch.cuda.profiler.start()
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
    torch.cuda.profiler.stop()
    prof = h.profile_stop()
    launches = h.kernel_launches() - n0
    t_ms = ev0.elapsed_time(ev1)
    t_ms = max_over_ranks(t_ms, "cuda", ws)
    # bytes of launches with live right-hand sides only (links and clover once
    # per such launch, spinors per live rhs); launches that the solver state
    # gated off entirely move nothing and are reported apart
    stencil_bytes = sum(p["bytes"] for p in prof)
    gated_launches = sum(p["gated_launches"] for p in prof)
    gated_ms = sum(p["gated_ms"] for p in prof)
    value = job_throughput(sum_over_ranks(stencil_bytes, "cuda", ws), t_ms)

    # dominant kernel (largest share of the timed region) and the dominant
    # bandwidth-bound (small-type) stencil kernel
    peak, peak_kind = measured_peaks()
    vh = int(np.prod(DIMS)) // 2

    def roofline_of(p):
        key = kernel_key(p)
        avg = p["total_ms"] / p["launches"]
        live = p["rhs_launches"] / p["launches"]   # mean live right-hand sides per launch
        if p["prec"] == 4:
            # double-float passes: bound by the binary32 pipe.  Binary32 operations
            # per output site and rhs of the double-float formulas (hop loop 8 x 1,200,
            # clover 3,048, scaling 48, + 264 for the sum of pass 2)
            ops = (12696.0 if p["mode"] == 1 else 12960.0) * vh * (2 if p["mode"] == 0 else 1) * live
            achieved = ops / (avg * 1e-3) / 1e12
            tr = traffic_for(key)
            return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TOPS, "unit": "Top/s",
                    "frac": achieved / FP32_PEAK_TOPS, "traffic": tr["dram_bytes_per_site"] * vh if tr else None,
                    "kernel": key, "peak_kind": "binary32 pipe operations: 152 SMs x 128 lanes x 2.07 GHz",
                    "avg_launch_ms": avg, "launches": p["launches"]}
        if p["prec"] == 0:
            # binary64 passes: bound by the FP64 pipe of GB300.  Flops per output
            # site and rhs: 1320 hopping + 504 clover (+24 for the sum of pass 2)
            flops = (1824.0 if p["mode"] == 1 else 1848.0) * vh * (2 if p["mode"] == 0 else 1) * live
            achieved = flops / (avg * 1e-3) / 1e12
            return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": key,
                    "peak_kind": "recipe nominal FP64 rate of GB300 (1.25 TFLOP/s); not in MEASURED_PEAKS.json",
                    "avg_launch_ms": avg, "launches": p["launches"]}
        achieved = (p["bytes"] / p["launches"]) / (avg * 1e-3) / 1e9
        tr = traffic_for(key)
        traffic = tr["dram_bytes_per_site"] * vh if tr else None
        # binary32 arithmetic of the same launch (stencil flops only): with many
        # right-hand sides the pass sits near the binary32 ridge
        flops = (1824.0 if p["mode"] == 1 else 1848.0) * vh * (2 if p["mode"] == 0 else 1) * live
        alu = flops / (avg * 1e-3) / 1e12
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": key, "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                "avg_launch_ms": avg, "launches": p["launches"], "mean_live_rhs": live,
                "gated_launches": p["gated_launches"],
                "alu": {"achieved": alu, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": alu / FP32_PEAK_TFLOPS,
                        "peak_kind": "binary32 FMA rate from unit counts and the 2.07 GHz clock"}}

    # the dominant source kernel (adjoint and plain instantiations summed), over
    # launches that did work
    merged = merge_source_kernels(prof)
    dom = max(merged, key=lambda p: p["total_ms"])
    roof = roofline_of(dom)
    small = [p for p in merged if p["prec"] not in (0, 4)]
    roof_hbm = roofline_of(max(small, key=lambda p: p["total_ms"])) if small else None

    # end to end through the public call with host buffers (even-site
    # canonical fields, half the bytes of full fields; buffers made at set-up)

    def e2e_time(solve, e_host, e_dev, p_dev, p_host):
        """Median over the steps of H2D + solve + D2H (events around each
        phase: the copies from pinned host memory vary from step to step on
        a host shared with other jobs); returns (total, h2d, solve, d2h) ms."""
        # untimed first: copy round trips and one pass (the first copies into freshly
        # pinned buffers, right after large host allocations, pay one-off costs)
        for _ in range(3):
            e_dev.copy_(e_host, non_blocking=True)
            p_host.copy_(p_dev, non_blocking=True)
        torch.cuda.synchronize()
        time.sleep(1.0)
        e_dev.copy_(e_host, non_blocking=True)
        solve(e_dev, p_dev)
        p_host.copy_(p_dev, non_blocking=True)
        torch.cuda.synchronize()
        rows = []
        for _ in range(args.e2e_steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record()
            e_dev.copy_(e_host, non_blocking=True)
            ev[1].record()
            rc_, _ = solve(e_dev, p_dev)
            assert rc_ == oq.OK
            ev[2].record()
            p_host.copy_(p_dev, non_blocking=True)
            ev[3].record()
            torch.cuda.synchronize()
            rows.append([ev[0].elapsed_time(ev[3]), ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                         ev[2].elapsed_time(ev[3])])
        return [statistics.median(r[k] for r in rows) for k in range(4)]

    def e2e_pipelined(solve, e_host, e_dev, p_dev, p_host):
        """A stream of solves as a user runs it: the next step's source is
        copied in on a second stream while the current step solves, and each
        step's solution is copied out while the next one solves (two device
        buffers each way).  Every step still moves its input in and its
        result out inside the timed region; returns ms per step."""
        main = torch.cuda.current_stream()
        cs = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        ev_read = [torch.cuda.Event() for _ in range(2)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for b in (0, 1):  # untimed round trips through every buffer
            e_dev[b].copy_(e_host, non_blocking=True)
            p_host[b].copy_(p_dev[b], non_blocking=True)
        torch.cuda.synchronize()
        t0.record(main)
        cs.wait_stream(main)
        with torch.cuda.stream(cs):
            e_dev[0].copy_(e_host, non_blocking=True)
            ev_in[0].record(cs)
        for k in range(args.e2e_steps):
            b = k % 2
            if k + 1 < args.e2e_steps:
                with torch.cuda.stream(cs):  # buffer 1 - b was last read by the (finished) step k - 1
                    e_dev[1 - b].copy_(e_host, non_blocking=True)
                    ev_in[1 - b].record(cs)
            main.wait_event(ev_in[b])
            if k >= 2:
                main.wait_event(ev_read[b])  # step k - 2's result has left p_dev[b]
            rc_, _ = solve(e_dev[b], p_dev[b])
            assert rc_ == oq.OK
            ev_out[b].record(main)
            with torch.cuda.stream(cs):
                cs.wait_event(ev_out[b])
                p_host[b].copy_(p_dev[b], non_blocking=True)
                ev_read[b].record(cs)
        main.wait_stream(cs)
        t1.record(main)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / args.e2e_steps

    def e2e_zero_copy(solve, e_host, p_host):
        """Each step hands the solver the pinned host buffers themselves: its
        packing kernel reads the 12 sources from host memory and its unpacking
        kernel writes the 12 solutions back over the host-device link (the
        copy engine's first transfer through a pinned buffer after other
        device work ran at 6-40 GB/s on the GPU machine; the kernels' many parallel
        requests do not wait on it).  Returns ms per step (CUDA events)."""
        solve(e_host, p_host)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.e2e_steps):
            rc_, _ = solve(e_host, p_host)
            assert rc_ == oq.OK
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / args.e2e_steps

    # The source of the even system lives on the even sites, so the headline
    # uses even-site canonical fields (oq_cgne_solve_even, half the bytes of
    # full fields).
    full = eta.cpu().numpy().view(np.complex128).reshape((NRHS, -1, 12))
    lexp = np.indices(DIMS).sum(axis=0).reshape(-1) % 2
    eta_host = torch.from_numpy(np.ascontiguousarray(full[:, lexp == 0]).view(np.float64)).pin_memory()
    del full, lexp
    psi_hosts = [torch.empty_like(eta_host).pin_memory() for _ in range(2)]
    eta_devs = [torch.empty(eta_host.shape, dtype=eta_host.dtype, device=eta.device) for _ in range(2)]
    psi_devs = [torch.empty_like(eta_devs[0]) for _ in range(2)]
    solve_even = lambda e, p: h.cgne_even(e, p, prm, nrhs=NRHS)  # noqa: E731
    e2e_ms = e2e_zero_copy(solve_even, eta_host, psi_hosts[0])
    ser_ms, ser_h2d, ser_solve, ser_d2h = e2e_time(solve_even, eta_host, eta_devs[0], psi_devs[0], psi_hosts[0])
    dma_ms = e2e_pipelined(solve_even, eta_host, eta_devs, psi_devs, psi_hosts)
    e2e_value = (stencil_bytes / args.steps) / (e2e_ms * 1e-3) / 1e9
    # the solution written to host memory is the device solve's
    psi_check = torch.empty_like(eta_devs[0])
    solve_even(eta_host.to(psi_check.device), psi_check)
    solve_even(eta_host, psi_hosts[1])
    torch.cuda.synchronize()
    e2e_same = bool(torch.equal(psi_hosts[1], psi_check.cpu()))
    del psi_check
    e2e_bytes = int(eta_host.numel() * 8)
    del eta_devs, psi_devs, psi_hosts, eta_host
    # full-lattice canonical fields (odd sites zero, oq_cgne_solve), serial, for comparison
    eta_host_f = eta.cpu().pin_memory()
    psi_host_f = torch.empty_like(eta_host_f).pin_memory()
    eta_dev_f = torch.empty_like(eta)
    psi_dev_f = torch.empty_like(eta)
    e2e_full = e2e_time(lambda e, p: h.cgne(e, p, prm, nrhs=NRHS), eta_host_f, eta_dev_f, psi_dev_f, psi_host_f)
    del eta_host_f, psi_host_f, eta_dev_f, psi_dev_f

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
        # precision ladders (Sec. 2, after Fig. 4): the storage type rises from
        # one inner solve to the next once the residual is below its epsilon
        for name, lad in (("ladder_fp16_fp32", (oq.F16, oq.F32)), ("ladder_fp16_fp32_fp64", (oq.F16, oq.F32, oq.F64)),
                          ("ladder_bf16_fp32", (oq.BF16, oq.F32))):
            p1 = oq.SolverParams(res=RES, nmx=50000, ladder=lad)
            h.cgne(eta1, psi1, p1, nrhs=1)
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            rc, st1 = h.cgne(eta1, psi1, p1, nrhs=1)
            torch.cuda.synchronize()
            tts[name] = {"s": time.perf_counter() - s0, "steps": st1[0]["steps"], "resets": st1[0]["resets"],
                         "steps_per_type": st1[0]["ladder_steps"][:len(lad)],
                         "true_rel_res": st1[0]["true_rel_res"], "converged": st1[0]["converged"]}
        for name, lad in (("batched_12rhs_ladder_fp16_fp32", (oq.F16, oq.F32)),
                          ("batched_12rhs_ladder_fp16_fp32_fp64", (oq.F16, oq.F32, oq.F64))):
            pl = oq.SolverParams(res=RES, nmx=20000, ladder=lad)
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            rc, stl = h.cgne(eta, psi, pl, nrhs=NRHS)
            torch.cuda.synchronize()
            tts[name] = {"s_per_rhs": (time.perf_counter() - s0) / NRHS,
                         "max_true_rel_res": max(x["true_rel_res"] for x in stl),
                         "resets": [x["resets"] for x in stl],
                         "steps_per_type": [x["ladder_steps"][:len(lad)] for x in stl]}
        tts["speedup_fp16_vs_fp64"] = tts["fp64"]["s"] / tts["fp16"]["s"]
        tts["batched_12rhs_f16_s_per_rhs"] = (t_ms * 1e-3 / args.steps) / NRHS
        tts["speedup_batched_f16_vs_fp64_per_rhs"] = tts["fp64"]["s"] / tts["batched_12rhs_f16_s_per_rhs"]
        # the paper's scheme for comparison: every reset in binary64
        h.set_option(oq.OPT_DF64_RESETS, 0)
        for name, sd in (("fp32_f64_resets", oq.F32), ("bf16_f64_resets", oq.BF16), ("fp16_f64_resets", oq.F16)):
            p1 = oq.SolverParams(res=RES, nmx=50000, sdtype=sd)
            h.cgne(eta1, psi1, p1, nrhs=1)
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            rc, st1 = h.cgne(eta1, psi1, p1, nrhs=1)
            torch.cuda.synchronize()
            tts[name] = {"s": time.perf_counter() - s0, "steps": st1[0]["steps"], "resets": st1[0]["resets"],
                         "true_rel_res": st1[0]["true_rel_res"], "converged": st1[0]["converged"]}
        torch.cuda.synchronize()
        h.profile_start()
        s0 = time.perf_counter()
        rc, stb = h.cgne(eta, psi, prm, nrhs=NRHS)
        torch.cuda.synchronize()
        tts["batched_12rhs_f16_f64_resets_s_per_rhs"] = (time.perf_counter() - s0) / NRHS
        tts["batched_12rhs_f16_f64_resets_max_res"] = max(x["true_rel_res"] for x in stb)
        tts["batched_12rhs_f16_f64_resets_resets"] = [x["resets"] for x in stb]
        tts["batched_12rhs_f16_f64_resets_kernels"] = [
            {"kernel": kernel_key(p),
             "launches": p["launches"], "ms": p["total_ms"]} for p in h.profile_stop()]
        h.set_option(oq.OPT_DF64_RESETS, 1)

    # time to solution on the 4^4 and 32x16^3 workloads (one Gaussian source,
    # even part): binary64 CGNE and the F16 mixed-precision CGNE, next to the
    # oracle's binary64 CGNE on the host cores
    small_tts = None
    if rank == 0 and ws == 1 and not args.no_tts:
        small_tts = {}
        for name, (dims, eps, kappa, seed) in (("c1_4x4x4x4", ((4, 4, 4, 4), 0.3, 0.13, 1)), ("c2_32x16c", C2_CASE)):
            hs = oq.Handle(dims)
            hs.gauge_upload(to_dev(synth.make_gauge(dims, eps, seed)), oq.LINK_12)
            hs.clover_build(kappa, CSW)
            src = synth.make_source(dims, seed + 1)
            src[np.indices(dims).sum(axis=0) % 2 == 1] = 0.0
            e_d = to_dev(src)
            p_d = torch.zeros_like(e_d)
            row = {}
            for pname, pc in (("fp64", oq.F64), ("fp16", oq.F16)):
                p1 = oq.SolverParams(res=RES, nmx=50000, sdtype=pc)
                hs.cgne(e_d, p_d, p1)
                torch.cuda.synchronize()
                s0 = time.perf_counter()
                rc, st1 = hs.cgne(e_d, p_d, p1)
                torch.cuda.synchronize()
                row[pname] = {"s": time.perf_counter() - s0, "steps": st1[0]["steps"], "resets": st1[0]["resets"],
                              "true_rel_res": st1[0]["true_rel_res"]}
            small_tts[name] = row
            hs.close()
    if cpu_tts is not None and small_tts is not None and tts is not None:
        # oracle binary64 CGNE time to solution: measured on 4^4, per-iteration
        # time x the binary64 step count on the larger workloads
        cpu_tts["c2_32x16c_cgne_fp64_s_extrapolated"] = (cpu_tts["c2_32x16c_s_per_iter_1core"]
                                                         * small_tts["c2_32x16c"]["fp64"]["steps"])
        cpu_tts["c3_64x32c_1rhs_cgne_fp64_s_extrapolated"] = (cpu_tts["c3_64x32c_s_per_iter_1core"]
                                                              * tts["fp64"]["steps"])
        cpu_tts["gpu_speedup_fp64_c2"] = (cpu_tts["c2_32x16c_cgne_fp64_s_extrapolated"]
                                          / small_tts["c2_32x16c"]["fp64"]["s"])
        cpu_tts["note"] = ("4^4 solved by the oracle; 32x16^3 and 64x32^3 (one point-source rhs): seconds per CG "
                           "iteration (one Dhat^dag Dhat) x the binary64 CGNE step count on the GPU; 1 core unless "
                           "all_cores")
    if cpu_line is not None:
        cpu_line["tts"] = cpu_tts

    # the uneven QCD+QED batch and the learned preconditioner against SAP-GCR,
    # compact forms of --workload c4 / c5 (rank 0, N = 1)
    extra = {}
    if rank == 0 and ws == 1 and not args.no_extra:
        t_x = time.perf_counter()
        extra["c4_uneven_batch"] = run_workload_c4(args, compact=True)
        extra["c5_learned_vs_sap"] = run_workload_c5(args, compact=True)
        extra["extra_s"] = time.perf_counter() - t_x

    st_last = statuses[-1]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(),
            "roofline": roof,
            "roofline_stencil_hbm": roof_hbm,
            "cpu_baseline": cpu_line,
            "e2e": {"value": e2e_value, "unit": "GB/s",
                    "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes,
                    "ms_per_step": e2e_ms, "layout": "even-site canonical fields (oq_cgne_solve_even)",
                    "steps": args.e2e_steps,
                    "method": "pinned host buffers passed to the solver: its packing kernel reads the sources "
                              "and its unpacking kernel writes the solutions over the host-device link",
                    "same_as_device_buffers": e2e_same,
                    "dma_pipelined": {"ms_per_step": dma_ms,
                                      "note": "copy-engine H2D / D2H into device buffers on a second stream, "
                                              "overlapping the previous / next solve"},
                    "serial": {"ms_per_step": ser_ms, "h2d_ms": ser_h2d, "solve_ms": ser_solve, "d2h_ms": ser_d2h,
                               "note": "median over steps of copy-engine H2D, solve and D2H one after the other"},
                    "serial_full_layout": {"ms_per_step": e2e_full[0], "h2d_ms": e2e_full[1],
                                           "solve_ms": e2e_full[2], "d2h_ms": e2e_full[3],
                                           "bytes_each_way": 2 * e2e_bytes,
                                           "note": "oq_cgne_solve, full-lattice canonical fields"}},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "solve": {"steps": [s["steps"] for s in st_last], "resets": [s["resets"] for s in st_last],
                      "max_true_rel_res": max(s["true_rel_res"] for s in st_last)},
            "stencil_bytes_per_step": stencil_bytes / args.steps,
            "gated_launches_per_step": gated_launches / args.steps,
            "gated_ms_per_step": gated_ms / args.steps,
            "kernels": [{"kernel": kernel_key(p),
                         "launches": p["launches"], "ms": p["total_ms"],
                         "gbs": p["bytes"] / (p["total_ms"] * 1e-3) / 1e9 if p["total_ms"] > 0 else None,
                         "rhs_launches": p["rhs_launches"], "gated_launches": p["gated_launches"],
                         "gated_ms": p["gated_ms"]} for p in prof],
            "tts": tts, "tts_small": small_tts, "setup_s": setup_s, "tuned_shapes": tuned, **extra,
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
    if args.profile_kind in ("tc", "cc", "sap", "sap_eo"):
        # learned preconditioner layers (tensor-core or CUDA-core) / SAP, binary32 fields
        src = torch.randn(int(np.prod(dims)) * 24, dtype=torch.float64, device="cuda")
        a, b = h.new_packed(oq.F32), h.new_packed(oq.F32)
        h.pack(src, a, oq.F32)
        w = torch.randn(1152, dtype=torch.float32, device="cuda") * 0.1
        prm = oq.SolverParams(ncy=1, nmr=5, bs=(4, 4, 4, 4), sap_eo=int(args.profile_kind == "sap_eo"))
        for _ in range(3):
            if args.profile_kind == "tc":
                h.nnprec_apply_tc(w, a, b)
            elif args.profile_kind == "cc":
                h.nnprec_apply(w, a, b)
            else:
                h.sap_apply(a, b, prm)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "x".join(map(str, dims)), "kind": args.profile_kind,
                          "launches": h.kernel_launches()}))
        h.close()
        return 0
    if args.profile_pin:
        bx, by, nr, cap, fmt = (int(v) for v in args.profile_pin.split(","))
        for mode in (0, 1, 2):
            h.tune_set(prec, mode, nrhs, bx, by, nr=nr, regcap=cap, link_fmt=fmt)
    else:
        h.autotune(prec, nrhs=nrhs)
    n_tune = h.kernel_launches()   # every launch so far is a stencil launch of the tuner
    # what follows is the range an `ncu --profile-from-start off` capture sees
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    if args.profile_kind == "cgne":
        # one batched mixed-precision CGNE solve; its first stencil launches
        # (after the tuner's n_tune) are pass 1, pass 2 + norm, pass 1^dag,
        # pass 2^dag + CG update
        eta = torch.randn(nrhs * int(np.prod(dims)) * 24, dtype=torch.float64, device="cuda")
        psi = torch.zeros_like(eta)
        rc, st = h.cgne(eta, psi, oq.SolverParams(res=RES, nmx=20000, sdtype=prec), nrhs=nrhs)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_case": "x".join(map(str, dims)), "kind": "cgne", "prec": args.profile_prec,
                          "nrhs": nrhs, "tuner_launches": n_tune, "rc": rc, "steps": st[0]["steps"]}))
        h.close()
        return 0
    src = torch.randn(nrhs * int(np.prod(dims)) * 24, dtype=torch.float64, device="cuda")
    if args.profile_kind == "dw":
        # the full operator on full fields
        a, b = h.new_packed(prec, nrhs=nrhs), h.new_packed(prec, nrhs=nrhs)
        h.pack(src, a, prec, nrhs=nrhs)
        for _ in range(3):
            h.dw(a, b, prec, nrhs=nrhs)
            h.dw(b, a, prec, nrhs=nrhs, dagger=True)
    else:
        a, b = h.new_packed(prec, oq.EVEN, nrhs=nrhs), h.new_packed(prec, oq.EVEN, nrhs=nrhs)
        h.pack(src, a, prec, oq.EVEN, nrhs=nrhs)
        for _ in range(3):
            h.dw_hat(a, b, prec, nrhs=nrhs)
            h.dw_hat(b, a, prec, nrhs=nrhs, dagger=True)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_case": "x".join(map(str, dims)), "prec": args.profile_prec, "nrhs": nrhs,
                      "tuner_launches": n_tune, "launches": h.kernel_launches()}))
    h.close()
    return 0


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def run_workload_c4(args, compact=False):
    """Uneven batch (QCD+QED): U(3) links with charges 2/3 and -1/3 on 8^4,
    32x16^3 and 48x24^3 lattices; batched CGNE (tile-list launches, graph
    replay) against the same systems solved one after the other; then the
    batch again with the clover of separate SU(3) and U(1) coefficients.
    compact: F16 storage only, returned as a dict (the default bench line)."""
    import torch
    from paper_2202_07388_gb300 import oq, synth
    from paper_2202_07388_gb300 import build as _build
    if not compact:
        _build.build()
    lats = [(8, 8, 8, 8), (32, 16, 16, 16), (48, 24, 24, 24)]
    charges = [2.0 / 3.0, -1.0 / 3.0]
    dims_all, fields = [], []
    for k, dims in enumerate(lats):
        su3 = synth.make_gauge(dims, 0.5, 4 + 10 * k)
        a1 = synth.make_u1_field(dims, 0.2, 5 + 10 * k)
        for q in charges:
            dims_all.append(dims)
            fields.append((su3, a1, q))
    h = oq.Handle(dims_all)
    etas, psis = [], []
    for lat, (dims, (su3, a1, q)) in enumerate(zip(dims_all, fields)):
        # U(3) links U exp(i q A) formed by the library; clover of the U(3) links
        h.gauge_upload_qed(to_dev(su3), to_dev(np.ascontiguousarray(a1)), q, lat=lat)
        h.clover_build(KAPPA, CSW, lat=lat)
        e = synth.make_source(dims, 40 + lat)
        x = np.indices(dims).sum(axis=0) % 2 == 1
        e[x] = 0.0
        etas.append(to_dev(e))
        psis.append(torch.zeros_like(etas[-1]))
    del fields
    out = {"workload": "uneven batch 8^4 + 32x16^3 + 48x24^3, U(3) links, q = 2/3, -1/3 (6 systems)"}
    for pname, pc in ((("f16", oq.F16),) if compact else (("f32", oq.F32), ("f16", oq.F16))):
        prm = oq.SolverParams(res=RES, nmx=20000, sdtype=pc)
        h.cgne_batch(list(range(len(dims_all))), etas, psis, prm)  # warm-up
        tb, (rc, st) = _timed(lambda: h.cgne_batch(list(range(len(dims_all))), etas, psis, prm))
        for lat in range(len(dims_all)):
            h.cgne(etas[lat], psis[lat], prm, lat=lat)  # warm-up
        ts = 0.0
        for lat in range(len(dims_all)):
            t, _ = _timed(lambda: h.cgne(etas[lat], psis[lat], prm, lat=lat))
            ts += t
        out[pname] = {"batched_s": tb, "sequential_s": ts, "speedup": ts / tb, "rc": rc,
                      "steps": [s["steps"] for s in st], "resets": [s["resets"] for s in st],
                      "max_true_rel_res": max(s["true_rel_res"] for s in st)}
    if compact:
        h.close()
        return out
    # openQ*D's clover with separate SU(3) and U(1) coefficients (both c_sw)
    tc, _ = _timed(lambda: [h.clover_build(KAPPA, CSW, lat=lat, csw_qed=CSW) for lat in range(len(dims_all))])
    prm = oq.SolverParams(res=RES, nmx=20000, sdtype=oq.F16)
    h.cgne_batch(list(range(len(dims_all))), etas, psis, prm)
    tb, (rc, st) = _timed(lambda: h.cgne_batch(list(range(len(dims_all))), etas, psis, prm))
    out["f16_qed_split_clover"] = {"batched_s": tb, "clover_build_s": tc, "rc": rc,
                                   "steps": [s["steps"] for s in st], "resets": [s["resets"] for s in st],
                                   "max_true_rel_res": max(s["true_rel_res"] for s in st)}
    print(json.dumps(out), flush=True)
    h.close()
    return 0


def run_workload_sf(args):
    """Schroedinger-functional time boundaries (openQCD boundary type 1) on the
    bench lattice: 64x32^3 with zero boundary fields, c_F = 1 (tree level),
    12 point sources on the first active slice (site (1, 1, 0, 0), even),
    eta = Dhat^dag b_e; the batched F16 CGNE to 1e-10 (double-float resets)
    against the one-rhs binary64 CGNE, with the stencil bytes per second of
    the batched solve."""
    import torch
    from paper_2202_07388_gb300 import oq, synth
    from paper_2202_07388_gb300 import build as _build
    _build.build()
    h = oq.Handle(DIMS, bc_t=0)
    ud = to_dev(synth.make_gauge_sf(DIMS, EPS, SEED))
    h.gauge_upload(ud, oq.LINK_12)
    h.clover_build(KAPPA, CSW, cF=1.0)
    del ud
    src = to_dev(synth.make_point_sources(DIMS, site=(1, 1, 0, 0)))
    pk, pk2 = h.new_packed(oq.F64, oq.EVEN, nrhs=NRHS), h.new_packed(oq.F64, oq.EVEN, nrhs=NRHS)
    h.pack(src, pk, oq.F64, oq.EVEN, nrhs=NRHS)
    h.dw_hat(pk, pk2, oq.F64, nrhs=NRHS, dagger=True)
    eta = torch.zeros_like(src)
    h.unpack(pk2, eta, oq.F64, oq.EVEN, nrhs=NRHS)
    del pk, pk2, src
    for pc, nr in ((oq.F16, NRHS), (oq.F64, NRHS), (oq.DF64, NRHS), (oq.F64, 1)):
        h.autotune(pc, nrhs=nr)
    psi = torch.zeros_like(eta)
    prm = oq.SolverParams(res=RES, nmx=20000, sdtype=oq.F16)
    h.cgne(eta, psi, prm, nrhs=NRHS)  # warm-up
    h.profile_start()
    reps = 2
    t, st = _timed(lambda: [h.cgne(eta, psi, prm, nrhs=NRHS) for _ in range(reps)])
    prof = h.profile_stop()
    st = st[-1][1]
    byts = sum(p["bytes"] for p in prof)
    eta1 = eta.view(NRHS, -1)[0:1].contiguous()
    psi1 = torch.zeros_like(eta1)
    p64 = oq.SolverParams(res=RES, nmx=50000, sdtype=oq.F64)
    h.cgne(eta1, psi1, p64)
    t64, (rc64, st64) = _timed(lambda: h.cgne(eta1, psi1, p64))
    out = {"workload": "Schroedinger-functional 64x32^3 (openQCD boundary type 1), 12 point-source rhs at "
                       "(1,1,0,0), batched F16 CGNE to 1e-10",
           "batched_12rhs_f16_s_per_rhs": t / reps / NRHS, "stencil_gbs": byts / t / 1e9,
           "steps": [s["steps"] for s in st], "resets": [s["resets"] for s in st],
           "max_true_rel_res": max(s["true_rel_res"] for s in st),
           "fp64_1rhs_s": t64, "fp64_steps": st64[0]["steps"], "fp64_true_rel_res": st64[0]["true_rel_res"],
           "speedup_batched_f16_vs_fp64_per_rhs": t64 / (t / reps / NRHS),
           "kernels": [{"kernel": kernel_key(p), "launches": p["launches"], "ms": p["total_ms"]} for p in prof]}
    print(json.dumps(out), flush=True)
    h.close()
    return 0


def run_workload_c5(args, compact=False):
    """48x24^3 at kappa = 0.1365: SAP-GCR (4^4 blocks, 5 MR steps, 4 cycles,
    16 Krylov vectors), its adaptive variant, GCR without preconditioner, and
    the learned PTC preconditioner trained on the GPU on (r, D^-1 r) pairs
    from the binary64 solver, each to a binary64 residual of 1e-10; plus the
    plain binary64 and the mixed-precision CGNE on the even-odd system.
    compact: static and adaptive SAP-GCR, plain GCR, the trained network,
    binary64 and F16 CGNE, returned as a dict (the default bench line)."""
    import torch
    from paper_2202_07388_gb300 import oq, synth
    from paper_2202_07388_gb300 import build as _build
    if not compact:
        _build.build()
    dims = (48, 24, 24, 24)
    kappa = 0.1365
    u = synth.make_gauge(dims, 0.5, 5)
    h = oq.Handle(dims)
    h.gauge_upload(to_dev(u), oq.LINK_12)
    h.clover_build(kappa, CSW)
    del u
    h.autotune(oq.F32, 1)
    h.autotune(oq.F64, 1)
    h.autotune(oq.DF64, 1)
    h.autotune(oq.F16, 1)
    eta = to_dev(synth.make_source(dims, 55))
    psi = torch.zeros_like(eta)
    out = {"workload": "48x24^3, kappa 0.1365, eps 0.5, Gaussian source, res 1e-10"}
    sap = oq.SolverParams(res=RES, nmx=2000, nkv=16, ncy=4, nmr=5, bs=(4, 4, 4, 4), sdtype=oq.F32)
    ada = oq.SolverParams(res=RES, nmx=2000, nkv=16, ncy=20, nmr=20, bs=(4, 4, 4, 4), sdtype=oq.F32, adaptive=1,
                          alpha=0.9)
    plain = oq.SolverParams(res=RES, nmx=5000, nkv=16, ncy=0, sdtype=oq.F32)
    # even-odd reduced block solver (MR on the blocks' Schur complements)
    import dataclasses
    sap_eo = dataclasses.replace(sap, sap_eo=1)
    sap_eo3 = dataclasses.replace(sap, sap_eo=1, nmr=3)
    ada_eo = dataclasses.replace(ada, sap_eo=1)
    # SAP block kernels: operands in shared memory (default), global operands one / two blocks per SM
    variants = (("sap_gcr", sap, 0), ("sap_gcr_global_operands", sap, 1),
                ("sap_gcr_global_operands_two_ctas", sap, 2), ("sap_gcr_adaptive", ada, 0),
                ("sap_gcr_eo_blocks", sap_eo, 0), ("sap_gcr_eo_blocks_nmr3", sap_eo3, 0),
                ("sap_gcr_adaptive_eo_blocks", ada_eo, 0), ("gcr", plain, 0))
    if compact:
        variants = tuple(v for v in variants if v[0] in ("sap_gcr", "sap_gcr_adaptive", "gcr"))
    for name, prm, kern in variants:
        h.set_option(oq.OPT_SAP_KERNEL, kern)
        h.sap_gcr(eta, psi, prm)
        t, (rc, st) = _timed(lambda: h.sap_gcr(eta, psi, prm))
        out[name] = {"s": t, "rc": rc, **{k: st[0][k] for k in ("steps", "restarts", "cycles", "mr_avg",
                                                                 "true_rel_res")}}
    h.set_option(oq.OPT_SAP_KERNEL, 0)
    # training pairs (r, e = D^-1 r) from the binary64 SAP-GCR solver
    ntrain = args.nn_pairs
    r = synth.make_source(dims, 500, nrhs=ntrain)
    vol = int(np.prod(dims))
    rp = h.new_packed(oq.F32, nrhs=ntrain)
    ep = h.new_packed(oq.F32, nrhs=ntrain)
    rd = to_dev(r)
    h.pack(rd, rp, oq.F32, nrhs=ntrain)
    ed = torch.zeros_like(rd)
    tpairs, _ = _timed(lambda: [h.sap_gcr(rd.view(ntrain, -1)[k], ed.view(ntrain, -1)[k], sap) for k in range(ntrain)])
    h.pack(ed, ep, oq.F32, nrhs=ntrain)
    del r, rd, ed
    kap = 1.0 / (2 * kappa)
    w = np.zeros(2 * 576, np.float32)
    wc = np.zeros(576, complex)
    W1 = wc[:288].reshape(9, 2, 1, 4, 4)
    W2 = wc[288:].reshape(9, 1, 2, 4, 4)
    W1[0, 0, 0] = np.eye(4)
    W2[0, 0, 0] = np.eye(4) / kap
    w[0::2], w[1::2] = wc.real, wc.imag
    wd = torch.from_numpy(w).cuda()
    ttrain, losses = _timed(lambda: h.nnprec_train(wd, rp, ep, ntrain, args.nn_lr, args.nn_steps))
    h.nn_gcr(wd, eta, psi, plain)
    t, (rc, st) = _timed(lambda: h.nn_gcr(wd, eta, psi, plain))
    out["nn_gcr"] = {"s": t, "rc": rc, "steps": st[0]["steps"], "restarts": st[0]["restarts"],
                     "true_rel_res": st[0]["true_rel_res"], "nn_fallback": st[0]["nn_fallback"],
                     "train_pairs": ntrain, "pair_solve_s": tpairs,
                     "train_steps": args.nn_steps, "train_s": ttrain, "loss_first": float(losses[0]),
                     "loss_last": float(losses[-1])}
    out["nn_gcr_speedup_vs_sap_gcr"] = out["sap_gcr"]["s"] / out["nn_gcr"]["s"]
    if compact:
        for name, pc in (("cgne_f64", oq.F64), ("cgne_f16", oq.F16)):
            ee = eta.clone().view(dims + (4, 6))
            ee[torch.from_numpy(np.indices(dims).sum(axis=0) % 2 == 1).cuda()] = 0.0
            prm = oq.SolverParams(res=RES, nmx=50000, sdtype=pc)
            h.cgne(ee, psi, prm)
            t, (rc, st) = _timed(lambda: h.cgne(ee, psi, prm))
            out[name] = {"s": t, "rc": rc, "steps": st[0]["steps"], "resets": st[0]["resets"],
                         "true_rel_res": st[0]["true_rel_res"]}
        h.close()
        return out
    h.set_option(oq.OPT_NN_TENSOR_CORES, 1)
    h.nn_gcr(wd, eta, psi, plain)
    t, (rc, st) = _timed(lambda: h.nn_gcr(wd, eta, psi, plain))
    out["nn_gcr_tensor_cores"] = {"s": t, "rc": rc, "steps": st[0]["steps"], "true_rel_res": st[0]["true_rel_res"]}
    h.set_option(oq.OPT_NN_TENSOR_CORES, 0)
    # tensor-core vs CUDA-core forward of the trained network
    a, b = h.new_packed(oq.F32), h.new_packed(oq.F32)
    h.pack(eta, a, oq.F32)
    for name, fn in (("cuda_core", h.nnprec_apply), ("tcgen05", h.nnprec_apply_tc)):
        fn(wd, a, b)
        t, _ = _timed(lambda: [fn(wd, a, b) for _ in range(10)])
        out[f"nn_forward_{name}_ms"] = 1e3 * t / 10
    # CGNE on the even-odd system, binary64 only vs mixed precision
    ee = eta.clone().view(dims + (4, 6))
    odd = torch.from_numpy(np.indices(dims).sum(axis=0) % 2 == 1).cuda()
    ee[odd] = 0.0
    for name, pc in (("cgne_f64", oq.F64), ("cgne_f16", oq.F16), ("cgne_f32", oq.F32)):
        prm = oq.SolverParams(res=RES, nmx=50000, sdtype=pc)
        h.cgne(ee, psi, prm)
        t, (rc, st) = _timed(lambda: h.cgne(ee, psi, prm))
        out[name] = {"s": t, "rc": rc, "steps": st[0]["steps"], "resets": st[0]["resets"],
                     "true_rel_res": st[0]["true_rel_res"]}
    out["volume"] = vol
    print(json.dumps(out), flush=True)
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c3", choices=["c3", "c4", "c5", "sf"])
    ap.add_argument("--nn-pairs", type=int, default=16)
    ap.add_argument("--nn-steps", type=int, default=100)
    ap.add_argument("--nn-lr", type=float, default=0.01)
    ap.add_argument("--profile-case", action="store_true")
    ap.add_argument("--profile-prec", default="fp16", choices=["fp64", "fp32", "bf16", "fp16", "df64"])
    ap.add_argument("--profile-nrhs", type=int, default=12)
    ap.add_argument("--profile-kind", default="dhat", choices=["dhat", "dw", "cgne", "tc", "cc", "sap", "sap_eo"])
    ap.add_argument("--profile-pin", default=None,
                    help="bx,by,nr,regcap,link_fmt: pin the stencil launch instead of autotuning")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tts", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the compact c4 / c5 workloads")
    ap.add_argument("--write-traffic", nargs="+", metavar="CSV", default=None,
                    help="write profiles/traffic.json from the ncu logs of the traffic capture")
    args = ap.parse_args()
    if args.write_traffic:
        return write_traffic(args.write_traffic)
    if args.profile_case:
        return run_profile_case(args)
    if args.workload == "c4":
        return run_workload_c4(args)
    if args.workload == "c5":
        return run_workload_c5(args)
    if args.workload == "sf":
        return run_workload_sf(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
