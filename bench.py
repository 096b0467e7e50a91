"""Benchmark of the batched stabilised fermion determinant on GB300.

One step = log det + G + force (forward pass with checkpoints, adjoint sweep) for one batch of
configurations.  Default workload: 256 configurations of the honeycomb L = 3 lattice (Nx = 18),
beta = 8, Nt = 64, U = 3, n_stab = 8.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec 3xtf32|tf32|fp64]
                    [--workload batch18|cold72|force72|tiny8] [--impl ours|reference]
                    [--path force|gtau|observables|bss|sparse]

--path picks what one step computes (default `force`, the headline):
  force        log det + G + force
  gtau         log det + the unequal-time G(tau, 0) for every tau (Section 4.2)
  observables  log det + fermion number + response traces tr(A G_t) at every slice (Section 4.1)
  bss          local (BSS) updates of time slice 1, every site proposed once (Section 3); the
               unit is site proposals/s, G_0 comes from an untimed FP64 log det/G call
  sparse       log det + G with the product-form slices of the intermediate-volume variant
               (Sections 8-9, n = 4 factors of the sparse hopping matrix, FP64), default
               workload sparse288; the dense FP64 path with the same E = T_4(K) is timed beside it

The headline is the mixed-precision path (slice products on tensor cores, FP64 QR/assembly);
the plain FP64 path is measured on the same inputs and reported beside it (`fp64_path`).
Prints ONE JSON line (rank 0).  `value` is configurations per second over all ranks with the
inputs resident on the device; `e2e` is the same metric through the public API with the inputs
copied from pinned host memory and the results read back inside the timed region.
The reference arm (--impl reference) times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 4 * L2_BYTES

WORKLOAD_TEXT = {
    "batch18": "honeycomb L=3 (Nx=18), kappa=1, beta=8, Nt=64, U=3, phi~N(0,delta*U), n_stab=8, "
               "256 configs",
    "cold72": "honeycomb L=6 (Nx=72), beta=64, Nt=512, U=3.5, n_stab=16, 64 configs",
    "force72": "honeycomb L=6 (Nx=72), beta=32, Nt=256, U=3, n_stab=8, 32 configs",
    "tiny8": "honeycomb L=2 (Nx=8), beta=2, Nt=16, U=2, n_stab=4, 1 config",
    "sparse288": "honeycomb L=12 (Nx=288), kappa=1, beta=8, Nt=64, U=3, n_stab=16, 152 configs",
    "uneven512": "uneven batch of 512 configs: honeycomb L in {2,3,4,5,6,7,8,12} (Nx in {8,18,32,"
                 "50,72,98,128,288}) x Nt in {32,64,128,256,512,1024}, delta=1/16 (beta=Nt/16 in "
                 "2..64), kappa=1, U=3, phi~N(0,delta*U), n_stab=16, the 48 (Nx, Nt) pairs "
                 "round-robin (first 32 pairs 11x, last 16 pairs 10x) in a seeded shuffle",
}

# what one step computes: Batch outputs, metric, and the text appended to the workload
PATHS = {
    "force": {"want": "force+green", "metric": "configs/s (log det + G + force)",
              "what": "log det + G + force"},
    "gtau": {"want": "gtau", "metric": "configs/s (log det + G(tau,0) for all tau)",
             "what": "log det + unequal-time G(tau,0), tau=0..Nt-1"},
    "observables": {"want": "nferm+response",
                    "metric": "configs/s (log det + n + tr(A G_t) for all t)",
                    "what": "log det + fermion number + response traces tr(A G_t), t=0..Nt-1"},
    "sparse": {"want": None, "metric": "configs/s (log det + G, product-form slices)",
               "what": "log det + G with every slice applied as prod_{k=1}^{4} (1 + gamma_k K) "
                       "diag(e^{i phi_t}), K = delta*kappa*A sparse (3 per row), FP64"},
    "bss": {"want": None, "metric": "site proposals/s (local updates at one time slice)",
            "what": "local (BSS) updates of slice 1, every site proposed once per step "
                    "(dphi ~ N(0, delta*U), u ~ U(0,1), w = 1), G_0 from FP64 log det/G"},
}


# ----------------------------------------------------------------------------- CPU oracle leg
def _oracle_worker(args):
    """One configuration through the CPU oracle: stabilised log det and, by path, G and the
    force, G(tau, 0) for every tau, or the fermion number and the response traces tr(A G_t).
    With `rows` (force path) only those force rows are evaluated, each a full stabilised
    evaluation on the rotated field (the oracle's force is that loop over all Nt rows); the
    times of log det + G and of the rows are returned apart so that a caller can scale the
    rows to Nt."""
    name, c, path = args[:3]
    rows = args[3] if len(args) > 3 else None
    import fd_inputs as fi
    from oracle import bss
    from oracle import force as oforce
    from oracle import observables, stable, unequal

    p = fi.workload(name, batch=1, first=c)[0]
    if path == "sparse":
        from oracle import product_form

        t0 = time.perf_counter()
        ld, G = product_form.logdet_green(p.A, p.delta, p.kappa, 4, p.phi, p.n_stab)
        return c, ld, {"G": G}, time.perf_counter() - t0
    if path == "bss":  # step 0's proposals from the G_0 of the workload's field
        dphi, u, w = (a[0] for a in fi.bss_proposals(name, 0, first=c, count=1))
        t0 = time.perf_counter()
        row, acc, total, G, _ = bss.slice_update(p.E, p.phi, p.n_stab, 1, dphi, u, w)
        return c, total, {"row": row, "acc": acc, "G": G}, time.perf_counter() - t0
    t0 = time.perf_counter()
    ld, G = stable.logdet_green(p.E, p.phi, p.n_stab)
    t_ld = time.perf_counter() - t0
    if path == "force" and rows is not None:
        t1 = time.perf_counter()
        Fr = oforce.force_rows(p.E, p.phi, p.n_stab, rows)
        t_rows = time.perf_counter() - t1
        out = {"G": G, "F_rows": Fr, "t_ld": t_ld, "t_row": t_rows / max(1, len(rows)),
               "nt": p.nt, "nx": p.nx}
        return c, ld, out, t_ld + t_rows
    if path == "force":
        out = {"G": G, "F": oforce.force(p.E, p.phi, p.n_stab)}
    elif path == "gtau":
        gt = unequal.green_tau_stable(p.E, p.phi, p.n_stab)
        out = {"Gtau": [gt[t] for t in range(p.nt)]}
    else:
        out = {"nferm": 1.0 - complex(G.trace()) / p.nx, "gmax": float(abs(G).max()),
               "R": observables.response_traces(p.E, p.phi, p.n_stab, p.A)}
    return c, ld, out, time.perf_counter() - t0


def _pool(cores):
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    pool = mp.get_context("spawn").Pool(cores)
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    return pool


def oracle_sample(pool, name, configs, path="force", rows=None):
    """Run the oracle over `configs` in the pool; rows: None, or per configuration the force rows
    to evaluate (force path only)."""
    t0 = time.perf_counter()
    if rows is None:
        work = [(name, c, path) for c in configs]
    else:
        work = [(name, c, path, r) for c, r in zip(configs, rows)]
    # longest first, so that the pool's last task is a short one
    work.sort(key=lambda a: -_oracle_cost(a))
    res = pool.map(_oracle_worker, work, chunksize=1)
    res.sort(key=lambda r: r[0])
    return res, time.perf_counter() - t0


def _oracle_cost(a):
    if a[0] != "uneven512":
        return 0
    import fd_inputs as fi

    L, nt = fi.uneven_sizes(1, a[1])[0]
    return (2 * L * L) ** 3 * nt


def uneven_sample(indices):
    """Stratified sample of an uneven batch: the first configuration of every (Nx, Nt) class
    among `indices`, with one force row (slice Nt/2) each.  Returns (configs, rows, class of
    every index)."""
    import fd_inputs as fi

    cls = {}
    first = {}
    for c in indices:
        L, nt = fi.uneven_sizes(1, c)[0]
        cls[c] = (2 * L * L, nt)
        first.setdefault(cls[c], c)
    configs = sorted(first.values())
    rows = [[cls[c][1] // 2] for c in configs]
    return configs, rows, cls


def uneven_cpu_rate(res, cls, indices, cores):
    """configs/s of the oracle on the uneven batch `indices`, extrapolated from the stratified
    sample: a configuration costs its class's log det + G time plus Nt times its class's time
    per force row, and the configurations are spread over `cores` processes."""
    per = {}
    for c, _, out, _ in res:
        per[(out["nx"], out["nt"])] = out["t_ld"] + out["nt"] * out["t_row"]
    total = sum(per[cls[c]] for c in indices)
    return len(indices) / (total / cores), total


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=parts[3],
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, label in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                               ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(label)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- helpers
KERNEL_SOURCES = ("fd_common.cuh", "fd_fp64.cuh", "fd_tc.cuh", "fd_df.cuh", "fd_qr_df.cuh",
                  "fd_bound_df.cuh", "fd_kernels_fp64.cu", "fd_kernels_mixed.cu",
                  "fd_kernels_big.cu")
# the files whose code a kernel compiles from, where that is fewer than all of them
KERNEL_SOURCES_OF = {
    "k_chain_mixed": ("fd_common.cuh", "fd_fp64.cuh", "fd_tc.cuh", "fd_kernels_mixed.cu"),
    "k_chain_big": ("fd_common.cuh", "fd_fp64.cuh", "fd_tc.cuh", "fd_df.cuh", "fd_qr_df.cuh",
                    "fd_bound_df.cuh", "fd_kernels_big.cu"),
}


def _kernel_source_hash(kernel=None):
    """Hash of the files that define a kernel's code (default: all hot-path kernels; the host
    runtime, the launcher declarations and the probes are left out: changing them does not change
    what a kernel does)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2604_02130_gb300", "csrc")
    for f in KERNEL_SOURCES_OF.get(kernel, KERNEL_SOURCES):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload, prec, step_path="force"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        db = json.load(open(path))
        key = "%s|%s|%s" % (kernel, workload, prec)
        if step_path != "force":
            key += "|" + step_path
        e = db.get(key)
        if e and e.get("source_hash") == _kernel_source_hash(kernel):
            return e["dram_bytes_per_launch"]
    except Exception:
        return None
    return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import fd_inputs as fi

    name = args.workload
    if args.path == "sparse" and name == "batch18":
        name = "sparse288"  # the same default workload as our arm of that path
    if args.path in ("sparse", "bss"):
        args.steps = max(1, min(args.steps, 10))
    cores = os.cpu_count() or 1
    pool = _pool(cores)
    if name == "uneven512":
        return _run_reference_uneven(args, pool, cores)
    batch = len(fi.workload(name, batch=None)) if name != "tiny8" else 1
    # per-step sample: about 8 configurations per core in all over 20 steps' worth of oracle
    # time, at least one per core, so that any --steps K finishes within a few minutes
    per_step = max(cores, min(8 * cores, (8 * cores * 20) // max(1, args.steps)))
    sample = list(range(min(batch, per_step)))
    for _ in range(args.warmup):
        oracle_sample(pool, name, sample[:cores], args.path)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_sample(pool, name, sample, args.path)
        times.append(dt)
    pool.close()
    total = sum(times)
    per = fi.workload(name, batch=1)[0].nx if args.path == "bss" else 1
    unit = "proposals/s" if args.path == "bss" else "configs/s"
    value = len(sample) * per * args.steps / total
    line = {
        "impl": "reference", "metric": PATHS[args.path]["metric"], "value": value,
        "unit": unit, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[name] + "; " + PATHS[args.path]["what"],
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                         "sample": "%d of the %d configurations per step, one per process"
                                   % (len(sample), batch)},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _run_reference_uneven(args, pool, cores):
    """The oracle on the uneven batch: every step runs the stratified sample (one configuration
    per (Nx, Nt) class, log det + G in full and one force row) and extrapolates to the batch."""
    if args.path != "force":
        raise SystemExit("the uneven workload is measured on the force path")
    ws = _dist()[0]
    indices = list(range(512))
    configs, rows, cls = uneven_sample(indices)
    small = [k for k, c in enumerate(configs) if cls[c][0] <= 18]
    for _ in range(args.warmup):
        oracle_sample(pool, "uneven512", [configs[k] for k in small], "force",
                      [rows[k] for k in small])
    rates, totals = [], []
    for _ in range(args.steps):
        res, _ = oracle_sample(pool, "uneven512", configs, "force", rows)
        r, tot = uneven_cpu_rate(res, cls, indices, cores)
        rates.append(r)
        totals.append(tot)
    pool.close()
    value = len(rates) / sum(1.0 / r for r in rates)  # 512 configurations per step
    sample = ("one configuration per (Nx, Nt) class (%d classes) per step: log det + G in full and "
              "one force row (a full stabilised evaluation on the rotated field), scaled to the "
              "class's Nt rows and to the 512 configurations, spread over %d processes"
              % (len(configs), cores))
    line = {
        "impl": "reference", "metric": PATHS["force"]["metric"], "value": value,
        "unit": "configs/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * 512 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["uneven512"] + "; " + PATHS["force"]["what"],
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "configs/s", "cores": cores, "kind": "oracle",
                         "sample": sample,
                         "cpu_seconds_per_512": statistics.mean(totals)},
        "e2e": {"value": value, "unit": "configs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _time_batch(batch, ctx, steps, flush, stream, barrier, sample_clocks, gpu, timing_runs=5):
    """Time `steps` calls (CUDA events on the launch stream, L2 flushed before each), then a
    separate short pass with per-launch events for the per-kernel roofline.  Per-launch events sit
    between the launches, so in that pass the phases of a size class run one after the other
    instead of overlapping (size classes still run side by side on their own streams); the timed
    steps have no events between launches."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    launches = 0
    barrier()
    clk = ClockSampler(gpu) if sample_clocks else None
    if clk:
        clk.__enter__()
    try:
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            batch.run()
            ev[k][1].record(stream)
            launches += ctx.last_launch_count()
        barrier()
    finally:
        if clk:
            clk.__exit__()
    kernel_ms = []
    ctx.set_timing(True)
    for _ in range(min(steps, timing_runs)):
        flush.zero_()
        batch.run()
        kernel_ms.append(ctx.last_kernel_ms())
    ctx.set_timing(False)
    barrier()
    return {"total_ms": sum(a.elapsed_time(b) for a, b in ev), "kernel_ms": kernel_ms,
            "launches": launches, "clocks": clk.summary() if clk else None}


def _scaled_err(a, ref):
    import numpy as np

    return float(np.abs(a - ref).max()) / max(1.0, float(np.abs(ref).max())) ** 2


def _errors(batch, res, path="force", pos=None, scale_batch=None):
    """Errors of the GPU results against the oracle's on the sampled configurations (pos maps a
    configuration index to its position in the batch; identity by default).  scale_batch: the
    FP64 path's batch, whose force rows give each row's conditioning max(1, max_x |G_t,xx|)^2
    for the scaled Im F = 1/2 invariant."""
    import numpy as np

    ld = batch.logdet_buf.cpu().numpy()
    e_ld = 0.0
    e = {}
    per_nx = {}
    for c, ldr, out, _ in res:
        k = c if pos is None else pos[c]
        g = complex(ld[k, 0], ld[k, 1])
        dim = abs(np.angle(np.exp(1j * (g.imag - ldr.imag))))
        el = max(abs(g.real - ldr.real), dim) / abs(ldr)
        e_ld = max(e_ld, el)
        if path == "force":
            eg = _scaled_err(batch.G[k].cpu().numpy(), out["G"])
            e["G_abs_over_maxG2"] = max(e.get("G_abs_over_maxG2", 0.0), eg)
            if "F_rows" in out:
                Fk = batch.F[k].cpu().numpy()
                ef = max(float(np.abs(Fk[r] - v).max()) / max(1.0, float(np.abs(v).max())) ** 2
                         for r, v in out["F_rows"].items())
                e["F_rows_abs_over_maxF2"] = max(e.get("F_rows_abs_over_maxF2", 0.0), ef)
                # Im F = 1/2 on every entry (particle-hole symmetry of the bipartite lattice),
                # relative to the conditioning of each row's G_t
                if scale_batch is not None:
                    F64 = scale_batch.F[k].cpu().numpy()
                    rs = np.maximum(1.0, np.abs(1.0 + 1j * F64).max(axis=1)) ** 2
                    e["ImF_minus_half_over_maxGt2"] = max(
                        e.get("ImF_minus_half_over_maxGt2", 0.0),
                        float((np.abs(Fk.imag - 0.5).max(axis=1) / rs).max()))
                nx = out["nx"]
                d = per_nx.setdefault(str(nx), {"logdet_rel": 0.0, "G": 0.0, "F_rows": 0.0})
                d["logdet_rel"] = max(d["logdet_rel"], el)
                d["G"] = max(d["G"], eg)
                d["F_rows"] = max(d["F_rows"], ef)
            else:
                e["F_abs_over_maxF2"] = max(e.get("F_abs_over_maxF2", 0.0),
                                            _scaled_err(batch.F[k].cpu().numpy(), out["F"]))
        elif path == "gtau":
            gt = batch.Gtau[k].cpu().numpy()
            e["Gtau_abs_over_max2"] = max(
                [e.get("Gtau_abs_over_max2", 0.0)] +
                [_scaled_err(gt[t], out["Gtau"][t]) for t in range(gt.shape[0])])
        else:
            nf = complex(*batch.nferm_buf[k].cpu().numpy())
            e["nferm_abs_over_maxG2"] = max(e.get("nferm_abs_over_maxG2", 0.0),
                                            abs(nf - out["nferm"]) / max(1.0, out["gmax"]) ** 2)
            e["R_abs_over_max"] = max(e.get("R_abs_over_max", 0.0),
                                      float(np.abs(batch.R[k].cpu().numpy() - out["R"]).max())
                                      / max(1.0, float(np.abs(out["R"]).max())))
    e.update({"logdet_rel": e_ld, "configs_checked": len(res)})
    if per_nx:
        e["per_nx"] = per_nx
    return e


PHASE_OF_KERNEL = {1: "A", 2: "B", 3: "C"}
DF_INSTR_PER_FLOP = 6
KERNEL_NAME = {0: "k_fwd_", 1: "k_chain_", 2: "k_boundary_", 3: "k_wrap_", 8: "k_merge_"}


def decode_kernel(k):
    """fd_plan_query's kernel code: (which, on the tensor cores, streamed, kernel name)."""
    which = 8 if k == 8 else k & 3
    tensor, big = bool(k & 4), bool(k & 16)
    name = KERNEL_NAME.get(which, "k_") + ("big" if big else "mixed" if tensor else "fp64")
    return which, tensor, big, name


def launch_flops(plan, probs, phase_flops):
    """Algorithmic (FP64-pipe, tensor) flops of every launch of the plan: the phase of the
    launch summed over the configurations of its size class, split by where the launch runs
    (a launch on the FP64 kernels counts its products as FP64 work; the streamed kernels' QR,
    in double-float arithmetic on the FP32 pipes, is counted with the FP64-pipe work)."""
    out = []
    for rec in plan:
        which, mixed, _, _ = decode_kernel(rec["kernel"])
        ph = PHASE_OF_KERNEL.get(which)
        f64 = tns = 0.0
        if ph:
            for p in probs:
                if p.nx == rec["nx"]:
                    pf = phase_flops(p.nx, p.nt, p.n_stab, mixed)[ph]
                    f64 += pf["fp64"]
                    tns += pf["tensor"]
        out.append((f64, tns))
    return out


def run_ours(args):
    ws, rank, local = _dist()
    import numpy as np

    import fd_inputs as fi

    name = args.workload
    uneven = name == "uneven512"
    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        pool = _pool(cores)  # spawned before the first CUDA call
    import torch

    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2604_02130_gb300 import api, shard
    from paper_2604_02130_gb300.flops import (force_phase_flops, gtau_phase_flops,
                                              response_phase_flops)

    dev = torch.device("cuda", local)
    if uneven:
        # the first 512 x ranks configurations of the uneven sequence, split by cost (LPT)
        per_rank = 512
        sizes = fi.uneven_sizes(per_rank * ws)
        mine = shard.lpt_partition([(2 * L * L) ** 3 * nt for L, nt in sizes], ws)[rank]
        probs = [fi.workload(name, batch=1, first=c)[0] for c in mine]
    else:
        per_rank = 1 if name == "tiny8" else fi.WORKLOADS[name]["batch"]
        mine = list(shard.shard_range(rank, per_rank))  # disjoint configuration indices
        probs = fi.workload(name, batch=per_rank, first=mine[0])
    n_mine = len(probs)
    n_total = per_rank * ws
    pos = {c: k for k, c in enumerate(mine)}
    # inputs resident on the device: one phi buffer for the batch (one host copy for e2e);
    # E, E^{-1} (and A, the operator of the response traces) once per lattice
    lat = {}
    for p in probs:
        if id(p.E) not in lat:
            lat[id(p.E)] = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                                 for a in (p.E, p.Einv, p.A))
    counts = [p.nt * p.nx for p in probs]
    phi_host = torch.empty(sum(counts), dtype=torch.float64).pin_memory()
    o = 0
    for p, k in zip(probs, counts):
        phi_host[o:o + k] = torch.from_numpy(np.ascontiguousarray(p.phi).ravel())
        o += k
    phi_dev = phi_host.to(dev)
    phis, o = [], 0
    for p, k in zip(probs, counts):
        phis.append(phi_dev[o:o + k].view(p.nt, p.nx))
        o += k
    spec = PATHS[args.path]
    ctx = api.Context(local)
    tuned = None
    if args.tune_nstab:
        # the QR interval of every (Nx, Nt) class from the tuner on the class's first
        # configuration: the fastest candidate within the budget against FP64
        tuned = {}
        for c, p in enumerate(probs):
            key = "%dx%d" % (p.nx, p.nt)
            if key not in tuned:
                cands = [k for k in (4, 8, 16, 32, 64) if p.nt % k == 0]
                best, errs, ms = ctx.tune_nstab((lat[id(p.E)][0], lat[id(p.E)][1], phis[c],
                                                 p.n_stab), cands, args.tune_nstab, args.prec,
                                                stats=True)
                tuned[key] = {"n_stab": best or p.n_stab, "candidates": cands, "err": errs,
                              "ms": ms}
            p.n_stab = tuned[key]["n_stab"]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    slow = uneven  # steps of seconds: fewer untimed and per-launch passes
    timing_runs = 2 if slow else 5

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def make(prec, warm):
        ops = [lat[id(p.E)][2] for p in probs] if args.path == "observables" else None
        b = api.Batch(ctx, [(lat[id(p.E)][0], lat[id(p.E)][1], phis[c], p.n_stab)
                            for c, p in enumerate(probs)], spec["want"], prec, ops)
        b.reserve()
        for _ in range(warm):
            b.run()
        barrier()
        st = b.status()
        assert all(x == 0 for x in st), "device status not OK: %s" % (
            [(c, x) for c, x in enumerate(st) if x][:8],)
        return b

    def allmax(x):
        return shard.max_over_ranks(x, dev)

    phase_flops = {"force": force_phase_flops, "gtau": gtau_phase_flops,
                   "observables": response_phase_flops}[args.path]

    # ---- headline path: device-resident timing, L2 flushed between steps
    warm = max(3, args.warmup)
    batch = make(args.prec, warm)
    plan = batch.plan()
    lf = launch_flops(plan, probs, phase_flops)
    flops_step = sum(a + b for a, b in lf)
    head = _time_batch(batch, ctx, args.steps, flush, stream, barrier, True, local, timing_runs)
    total_ms = allmax(head["total_ms"])
    value = n_total * args.steps / (total_ms * 1e-3)

    # ---- end to end through the public API: pinned host inputs in, results out
    outs = {"force": [batch.logdet_buf, batch.G_flat, batch.F_flat],
            "gtau": [batch.logdet_buf, batch.Gtau_flat],
            "observables": [batch.logdet_buf, batch.nferm_buf, batch.R_flat]}[args.path]
    hosts = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    h2d = phi_host.numel() * 8
    d2h = sum(t.numel() * t.element_size() for t in hosts)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        phi_dev.copy_(phi_host, non_blocking=True)
        batch.run()
        for h, t in zip(hosts, outs):
            h.copy_(t, non_blocking=True)
        ev2[k][1].record(stream)
    barrier()
    e2e_ms = allmax(sum(a.elapsed_time(b) for a, b in ev2))
    e2e = {"value": n_total * args.steps / (e2e_ms * 1e-3), "unit": "configs/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    launches = head["launches"]

    # ---- the plain FP64 path on the same inputs, reported beside the headline
    fp64 = None
    b64 = None
    if args.prec != "fp64" and not args.no_fp64_path:
        steps64 = 2 if slow else max(3, args.steps // 2)
        b64 = make("fp64", 1 if slow else 3)
        plan64 = b64.plan()
        r64 = _time_batch(b64, ctx, steps64, flush, stream, barrier, False, local,
                          1 if slow else 5)
        ms64 = allmax(r64["total_ms"]) / steps64
        lf64 = launch_flops(plan64, probs, phase_flops)
        km64 = [statistics.mean(k[i] for k in r64["kernel_ms"]) for i in range(len(plan64))]
        fp64 = {"value": n_total / (ms64 * 1e-3), "unit": "configs/s", "ms_per_step": ms64,
                "steps": steps64,
                "tflops": sum(a + b for a, b in lf64) * n_total / n_mine / (ms64 * 1e-3) / 1e12,
                "kernel_ms": {"%s_%d" % (decode_kernel(r["kernel"])[3], r["nx"]): m
                              for r, m in zip(plan64, km64)}}

    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    # ---- roofline of the longest launch.  Per-launch durations from CUDA events on the
    #      launch streams.
    peaks, peak_src = _measured_peaks()
    # the FP64 DFMA probe, repeated for about a second with the clocks sampled meanwhile
    clk64 = ClockSampler(local)
    clk64.__enter__()
    try:
        probe = [ctx.measure_fp64_peak() / 1e3 for _ in range(4)]
    finally:
        clk64.__exit__()
    peak_fp64 = max(probe)
    probe_clocks = clk64.summary()
    tf32_peak = peaks["bf16_tflops"] / 2.0
    # The streamed kernels' QR, boundary LU and products run in double-float on the FP32 pipes:
    # their peak is the FP32 issue rate of all SMs at the timed region's median SM clock over
    # DF_INSTR_PER_FLOP instructions per algorithmic flop (a compensated complex multiply-add,
    # 8 flops, is 4 double-float products of 12 FP32 instructions each: 48 / 8 = 6).
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = (head["clocks"] or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_df = n_sms * 128 * clk_mhz * 1e6 / DF_INSTR_PER_FLOP / 1e12
    peak_df_src = ("%d SMs x 128 FP32 lanes x %.0f MHz (median SM clock in the timed region) / "
                   "%d FP32 instructions per double-float flop" % (n_sms, clk_mhz,
                                                                  DF_INSTR_PER_FLOP))
    per_launch = [statistics.mean(k[i] for k in head["kernel_ms"]) for i in range(len(plan))]
    phases = []
    for i, rec in enumerate(plan):
        _, _, big, nm = decode_kernel(rec["kernel"])
        ms = per_launch[i]
        f64 = lf[i][0] / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
        tns = lf[i][1] / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
        ph = {"kernel": nm, "nx": rec["nx"], "configs": rec["configs"], "ms": ms}
        if big:  # double-float work on the FP32 pipes
            ph.update({"df_tflops": f64, "df_frac": f64 / peak_df})
        else:
            ph.update({"fp64_tflops": f64, "fp64_frac": f64 / peak_fp64})
        ph.update({"tensor_tflops": tns, "tensor_frac": tns / tf32_peak, "_alu": f64,
                   "_big": big})
        phases.append(ph)
    dom = max(range(len(plan)), key=lambda i: per_launch[i])
    k_ms = per_launch[dom]
    dk = decode_kernel(plan[dom]["kernel"])[0]
    what = {0: "the log det/G kernel", 1: "the chain kernel (slice products, QRs, assembly)",
            2: "the boundary kernel (boundary Green's functions: GEMMs, LU, solves)",
            3: "the wrap kernel (%s)" % ("wrap products" if args.path != "gtau"
                                         else "slice propagation of G(tau,0)")}.get(dk, "")
    what += " of the Nx=%d size class" % plan[dom]["nx"]
    P = phases[dom]
    if P["_alu"] > 0 and P["_big"]:
        roof = {"bound": "alu", "achieved": P["_alu"], "peak": peak_df, "unit": "TFLOP/s",
                "frac": P["_alu"] / peak_df,
                "what": "algorithmic QR, assembly and boundary work (FP64-class flops, computed "
                        "in double-float on the FP32 pipes) of %s per launch over its CUDA-event "
                        "duration" % what,
                "peak_source": peak_df_src}
    elif P["_alu"] > 0 or P["tensor_tflops"] == 0:
        roof = {"bound": "alu", "achieved": P["_alu"], "peak": peak_fp64,
                "unit": "TFLOP/s", "frac": P["_alu"] / peak_fp64,
                "what": "FP64 algorithmic work of %s per launch over its CUDA-event duration"
                        % what,
                "peak_source": "FP64 DFMA probe over all SMs in this run (fd_measure_fp64_peak, "
                               "best of 4), clocks during the probe: %s" % json.dumps(probe_clocks)}
    else:
        roof = {"bound": "tensor", "achieved": P["tensor_tflops"], "peak": tf32_peak,
                "unit": "TFLOP/s", "frac": P["tensor_tflops"] / tf32_peak,
                "what": "tensor-core work of %s per launch over its CUDA-event duration" % what,
                "peak_source": "%s bf16 dense x 1/2 (TF32:BF16 nominal ratio)" % peak_src}
    roof.update({"traffic": _traffic(P["kernel"], name, args.prec, args.path),
                 "kernel": P["kernel"], "kernel_ms": k_ms,
                 "kernel_ms_from": "a separate pass with CUDA events between the launches, "
                                   "every launch alone (in the timed steps the size classes run "
                                   "concurrently and the phases overlap)",
                 "fp64_issue_cycles": dict(zip(("one_lane", "full_warp", "one_of_8_warps"),
                                               ctx.measure_fp64_issue())),
                 "fp64_peak": {"value": peak_fp64, "unit": "TFLOP/s",
                               "source": "FP64 DFMA probe over all SMs (best of 4), clocks "
                                         "during the probe: %s" % json.dumps(probe_clocks)},
                 "df_peak": {"value": peak_df, "unit": "TFLOP/s", "source": peak_df_src},
                 "phases": [{k: v for k, v in ph.items() if not k.startswith("_")}
                            for ph in phases]})
    if P["tensor_tflops"] > 0 and roof["bound"] == "alu":
        roof["tensor"] = {"achieved": P["tensor_tflops"], "peak": tf32_peak,
                          "unit": "TFLOP/s", "frac": P["tensor_tflops"] / tf32_peak,
                          "what": "tensor-core work of the same kernel (a product counted once, "
                                  "not x3 for split TF32)",
                          "peak_source": "%s bf16 dense x 1/2 (TF32:BF16 nominal ratio)"
                                         % peak_src}

    # ---- CPU oracle on a bounded sample, and the errors of the GPU results on that sample
    cpu = None
    err = None
    if pool is not None:
        if uneven:
            configs, rows, cls = uneven_sample(mine)
            res, dt = oracle_sample(pool, name, configs, args.path, rows)
            rate, tot = uneven_cpu_rate(res, cls, mine, cores)
            cpu = {"value": rate, "unit": "configs/s", "cores": cores, "kind": "oracle",
                   "sample": "one configuration per (Nx, Nt) class (%d classes): log det + G in "
                             "full and one force row (a full stabilised evaluation on the "
                             "rotated field), scaled to the class's Nt rows and to the %d "
                             "configurations, spread over %d processes"
                             % (len(configs), n_mine, cores),
                   "cpu_seconds_per_step": tot, "sample_wall_s": dt}
        else:
            sample = list(range(min(n_mine, 8 * cores)))
            res, dt = oracle_sample(pool, name, sample, args.path)
            cpu = {"value": len(sample) / dt, "unit": "configs/s", "cores": cores,
                   "kind": "oracle",
                   "sample": "%d of the %d configurations (%s), one per process"
                             % (len(sample), n_mine, spec["what"])}
        pool.close()
        err = {args.prec: _errors(batch, res, args.path, pos, b64)}
        if b64 is not None:
            err["fp64"] = _errors(b64, res, args.path, pos, b64)

    line = {
        "metric": spec["metric"],
        "value": value,
        "unit": "configs/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": warm,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32+f64", "3xtf32": "3xtf32+f64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[name] + "; " + spec["what"]
                               + ("; n_stab tuned per (Nx, Nt) class within %g of FP64"
                                  % args.tune_nstab if tuned else ""),
                   "prec": args.prec, "plan": plan, "nstab_tuned": tuned,
                   "l2": "flushed between timed steps (%d MB write)" % (FLUSH_BYTES >> 20)},
        "tflops": flops_step * n_total * args.steps / n_mine / (total_ms * 1e-3) / 1e12,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": head["clocks"],
        "cpu_baseline": cpu,
        "fp64_path": fp64,
        "error_vs_oracle": err,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_bss(args):
    """--path bss: one step = one fd_bss_update call over slice 1 of every configuration of the
    shard, every site proposed once.  G_0 comes from an untimed FP64 log det/G call; the steps
    continue the Markov chain of slice 1 with fresh proposals (resident on the device, one set
    per step), so every step does the same kind of work.  A separate first call from G_0 with
    step 0's proposals is compared with the oracle."""
    ws, rank, local = _dist()
    import numpy as np

    import fd_inputs as fi

    name = args.workload
    if name == "tiny8":
        raise SystemExit("--path bss needs a batched workload")
    w_batch = fi.WORKLOADS[name]["batch"]
    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        pool = _pool(cores)  # spawned before the first CUDA call
    import torch

    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2604_02130_gb300 import api, shard

    dev = torch.device("cuda", local)
    mine = shard.shard_range(rank, w_batch)
    probs = fi.workload(name, batch=w_batch, first=mine.start)
    nx = probs[0].nx
    n_total = w_batch * ws
    ctx = api.Context(local)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # G_0 (FP64) and the field rows of slice 1, resident on the device
    phi_dev = torch.from_numpy(np.stack([p.phi for p in probs])).to(dev)
    E = torch.from_numpy(probs[0].E).to(dev)
    Einv = torch.from_numpy(probs[0].Einv).to(dev)
    g0 = api.Batch(ctx, [(E, Einv, phi_dev[c], p.n_stab) for c, p in enumerate(probs)],
                   "green", "fp64")
    g0.run()
    barrier()
    G0 = torch.stack([g.clone() for g in g0.G])
    row0 = phi_dev[:, 0, :].clone()
    warm = max(3, args.warmup)
    ntime = min(args.steps, 5)
    ncalls = 1 + warm + args.steps + ntime  # check, warm-up, timed, per-launch timing pass
    prop_host = np.stack([np.stack(fi.bss_proposals(name, s, first=mine.start, count=w_batch))
                          for s in range(ncalls)])  # (ncalls, 3, batch, nx)
    prop = torch.from_numpy(prop_host).to(dev)
    acc = torch.zeros((ncalls, w_batch, nx), dtype=torch.int32, device=dev)
    Gchk, rowchk = G0.clone(), row0.clone()
    Gs, rows = G0.clone(), row0.clone()

    def prepared(s, G, row):
        return api.BssSlices(list(G), list(row), list(prop[s, 0]), list(prop[s, 1]),
                             list(prop[s, 2]), list(acc[s]), ctx)

    calls = [prepared(0, Gchk, rowchk)] + [prepared(s, Gs, rows) for s in range(1, ncalls)]
    dld_chk = calls[0].run().clone()
    for s in range(1, 1 + warm):
        calls[s].run()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.__enter__()
    try:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            calls[1 + warm + k].run()
            ev[k][1].record(stream)
        barrier()
    finally:
        clk.__exit__()
    total_ms = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev)
    value = n_total * nx * args.steps / (total_ms * 1e-3)
    launches = args.steps  # one k_bss launch per call
    # per-launch kernel time (events around the launch alone) for the roofline
    kernel_ms = []
    ctx.set_timing(True)
    for s in range(1 + warm + args.steps, ncalls):
        flush.zero_()
        calls[s].run()
        kernel_ms.append(ctx.last_kernel_ms()[0])
    ctx.set_timing(False)
    acc_timing = int(acc[1 + warm + args.steps:].sum().item())
    acc_timed = int(acc[1 + warm:1 + warm + args.steps].sum().item())

    # end to end through the public API: the step's proposals from pinned host memory into
    # fixed device buffers, the call, decisions and the change of log det read back
    pin = torch.from_numpy(prop_host[1 + warm:1 + warm + args.steps]).pin_memory()
    buf = torch.empty((3, w_batch, nx), dtype=torch.float64, device=dev)
    acc_e = torch.empty((w_batch, nx), dtype=torch.int32, device=dev)
    e2e_call = api.BssSlices(list(Gs), list(rows), list(buf[0]), list(buf[1]), list(buf[2]),
                             list(acc_e), ctx)
    acc_h = torch.empty((w_batch, nx), dtype=torch.int32).pin_memory()
    dld_h = torch.empty((w_batch, 2), dtype=torch.float64).pin_memory()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        buf.copy_(pin[k], non_blocking=True)
        e2e_call.run()
        acc_h.copy_(acc_e, non_blocking=True)
        dld_h.copy_(e2e_call.out[:w_batch], non_blocking=True)
        ev2[k][1].record(stream)
    barrier()
    e2e_ms = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev2), dev)
    e2e = {"value": n_total * nx * args.steps / (e2e_ms * 1e-3), "unit": "proposals/s",
           "h2d_bytes_per_step": 3 * w_batch * nx * 8,
           "d2h_bytes_per_step": w_batch * nx * 4 + w_batch * 16}
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    # roofline: the rank-1 updates (8 Nx^2 real flops per accepted site) against the FP32 issue
    # bound of the double-float complex multiply-subtract (54 FP32 instructions per 8 flops on
    # 128 lanes per SM); configurations run one per SM, so only min(batch, SMs) SMs take part
    clocks = clk.summary()
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    sms = min(w_batch, torch.cuda.get_device_properties(dev).multi_processor_count)
    k_ms = statistics.mean(kernel_ms)
    achieved = 8.0 * nx * nx * acc_timing / len(kernel_ms) / (k_ms * 1e-3) / 1e12
    peak = sms * 128 * mhz * 1e6 * 8.0 / 54.0 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": _traffic("k_bss", name, "df", "bss"),
            "kernel": "k_bss", "kernel_ms": k_ms,
            "what": "rank-1 updates of G (8 Nx^2 real flops per accepted site) per launch over "
                    "the launch's CUDA-event duration",
            "peak_source": "FP32 issue bound of the double-float update: %d SMs x 128 lanes x "
                           "%.0f MHz (sampled) x 8 flops / 54 instructions" % (sms, mhz),
            "accepted_fraction": acc_timed / float(w_batch * nx * args.steps)}

    cpu = None
    err = None
    if pool is not None:
        sample = list(range(min(w_batch, cores)))
        res, dt = oracle_sample(pool, name, sample, "bss")
        pool.close()
        cpu = {"value": len(sample) * nx / dt, "unit": "proposals/s", "cores": cores,
               "kind": "oracle",
               "sample": "slice 1 of %d of the %d configurations, one per process (a stabilised "
                         "determinant per proposal)" % (len(sample), w_batch)}
        acc0 = acc[0].cpu().numpy().astype(bool)
        d0 = dld_chk.cpu().numpy()
        Gc = Gchk.cpu().numpy()
        rc = rowchk.cpu().numpy()
        e = {"decisions_differing": 0, "row_max_abs": 0.0, "G_abs_over_maxG2": 0.0,
             "dlogdet_abs": 0.0}
        for c, total, out, _ in res:
            e["decisions_differing"] += int((acc0[c] != out["acc"]).sum())
            e["row_max_abs"] = max(e["row_max_abs"], float(np.abs(rc[c] - out["row"]).max()))
            e["G_abs_over_maxG2"] = max(e["G_abs_over_maxG2"], _scaled_err(Gc[c], out["G"]))
            dd = complex(d0[c]) - total
            e["dlogdet_abs"] = max(e["dlogdet_abs"],
                                   abs(dd.real), abs(np.angle(np.exp(1j * dd.imag))))
        e["configs_checked"] = len(res)
        err = {"df": e}

    line = {
        "metric": PATHS["bss"]["metric"],
        "value": value,
        "unit": "proposals/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": warm,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 decisions, df (2 x f32) G",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[name] + "; " + PATHS["bss"]["what"],
                   "l2": "flushed between timed steps (%d MB write)" % (FLUSH_BYTES >> 20)},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "error_vs_oracle": err,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sparse(args):
    """--path sparse: one step = one fd_green_sparse call (log det + G of the shard's
    configurations with the product-form slices, n = 4).  The dense FP64 path on the same
    arithmetic (E = T_4(K) = sum_{j<=4} K^j / j!) is timed beside it.  A step of sparse288 takes
    about a second, so at most 10 steps are timed (the line reports the number)."""
    args.steps = max(1, min(args.steps, 10))
    ws, rank, local = _dist()
    import numpy as np

    import fd_inputs as fi

    name = args.workload if args.workload != "batch18" else "sparse288"
    w_batch = 1 if name == "tiny8" else fi.WORKLOADS[name]["batch"]
    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        pool = _pool(cores)  # spawned before the first CUDA call
    import torch

    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2604_02130_gb300 import api, shard
    from paper_2604_02130_gb300.flops import sparse_fwd_flops

    nfac = 4
    dev = torch.device("cuda", local)
    mine = shard.shard_range(rank, w_batch)
    probs = fi.workload(name, batch=w_batch, first=mine.start)
    p0 = probs[0]
    nx, nt, ns = p0.nx, p0.nt, p0.n_stab
    ctx = api.Context(local)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    phi_host = torch.from_numpy(np.stack([p.phi for p in probs])).pin_memory()
    phi_dev = phi_host.to(dev)
    col, val = fi.sparse_rows(p0.A)
    col_d = torch.from_numpy(col).to(dev)
    val_d = torch.from_numpy(val * (p0.delta * p0.kappa)).to(dev)
    q = col.shape[1]
    sp_probs = [(phi_dev[c], ns) for c in range(w_batch)]
    hops = [(col_d, val_d)] * w_batch

    def sparse_call():
        return api.green_sparse(sp_probs, hops, nfac=nfac, ctx=ctx)

    for _ in range(max(3, args.warmup)):
        sparse_call()
    barrier()
    assert all(s == 0 for s in ctx.status(w_batch)), "device status not OK"
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.__enter__()
    try:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            ld_s, G_s = sparse_call()
            ev[k][1].record(stream)
        barrier()
    finally:
        clk.__exit__()
    total_ms = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev)
    value = w_batch * ws * args.steps / (total_ms * 1e-3)
    ctx.set_timing(True)
    flush.zero_()
    sparse_call()
    k_ms = ctx.last_kernel_ms()[0]
    ctx.set_timing(False)
    ld_s, G_s = sparse_call()
    barrier()

    # end to end: phi from pinned host memory, log det and G read back
    G_host = torch.empty((w_batch, nx, nx), dtype=torch.complex128).pin_memory()
    ld_host = torch.empty((w_batch,), dtype=torch.complex128).pin_memory()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev2[k][0].record(stream)
        phi_dev.copy_(phi_host, non_blocking=True)
        ld_e, G_e = sparse_call()
        ld_host.copy_(ld_e, non_blocking=True)
        for c in range(w_batch):
            G_host[c].copy_(G_e[c], non_blocking=True)
        ev2[k][1].record(stream)
    barrier()
    e2e_ms = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev2), dev)
    e2e = {"value": w_batch * ws * args.steps / (e2e_ms * 1e-3), "unit": "configs/s",
           "h2d_bytes_per_step": phi_host.numel() * 8,
           "d2h_bytes_per_step": w_batch * (nx * nx + 1) * 16}

    # the dense FP64 path with the same slice matrix E = T_4(K)
    K = p0.delta * p0.kappa * p0.A.astype(np.float64)
    E4 = np.eye(nx)
    term = np.eye(nx)
    for j in range(1, nfac + 1):
        term = term @ K / j
        E4 = E4 + term
    E4_d = torch.from_numpy(E4).to(dev)
    dense = api.Batch(ctx, [(E4_d, None, phi_dev[c], ns) for c in range(w_batch)], "green",
                      "fp64")
    for _ in range(max(3, args.warmup)):
        dense.run()
    barrier()
    ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev3[k][0].record(stream)
        dense.run()
        ev3[k][1].record(stream)
    barrier()
    dense_ms = shard.max_over_ranks(sum(a.elapsed_time(b) for a, b in ev3), dev)
    dense_plan = dense.plan()
    agree = max(float((dense.logdet_buf[:, 0] - torch.view_as_real(ld_s)[:, 0]).abs().max()),
                float(max((a - b).abs().max().item() for a, b in zip(dense.G, G_s))))
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    fl = sparse_fwd_flops(nx, nt, ns, q, nfac)
    peak_fp64 = ctx.measure_fp64_peak() / 1e3
    achieved = fl["total"] * w_batch / (k_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
            "frac": achieved / peak_fp64, "traffic": None, "kernel": "k_fwd_fp64",
            "kernel_ms": k_ms,
            "what": "FP64 algorithmic work (product-form slices, QRs, assembly) per launch over "
                    "the launch's CUDA-event duration",
            "peak_source": "FP64 DFMA probe over all SMs in this run (fd_measure_fp64_peak)",
            "flops_per_config": fl}
    cpu = None
    err = None
    if pool is not None:
        sample = list(range(min(w_batch, cores)))
        res, dt = oracle_sample(pool, name, sample, "sparse")
        pool.close()
        cpu = {"value": len(sample) / dt, "unit": "configs/s", "cores": cores, "kind": "oracle",
               "sample": "%d of the %d configurations, one per process" % (len(sample), w_batch)}
        ldc = ld_s.cpu().numpy()
        e = {"logdet_rel": 0.0, "G_abs_over_maxG2": 0.0}
        for c, ldr, out, _ in res:
            d = complex(ldc[c]) - ldr
            e["logdet_rel"] = max(e["logdet_rel"], max(abs(d.real),
                                  abs(np.angle(np.exp(1j * d.imag)))) / abs(ldr))
            e["G_abs_over_maxG2"] = max(e["G_abs_over_maxG2"],
                                        _scaled_err(G_s[c].cpu().numpy(), out["G"]))
        e["configs_checked"] = len(res)
        err = {"fp64": e}
    line = {
        "metric": PATHS["sparse"]["metric"],
        "value": value,
        "unit": "configs/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[name] + "; " + PATHS["sparse"]["what"],
                   "l2": "flushed between timed steps (%d MB write)" % (FLUSH_BYTES >> 20)},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
        "dense_fp64_same_E": {"value": w_batch * ws * args.steps / (dense_ms * 1e-3),
                              "unit": "configs/s", "ms_per_step": dense_ms / args.steps,
                              "plan": dense_plan, "max_abs_difference": agree},
        "cpu_baseline": cpu,
        "error_vs_oracle": err,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5 for uneven512, else 500)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--prec", choices=("fp64", "tf32", "3xtf32"), default="3xtf32")
    ap.add_argument("--workload", choices=tuple(WORKLOAD_TEXT), default=None,
                    help="default uneven512 (force path), batch18 (other paths), sparse288 (sparse)")
    ap.add_argument("--path", choices=tuple(PATHS), default="force",
                    help="what one step computes (default: log det + G + force)")
    ap.add_argument("--tune-nstab", type=float, default=None, metavar="BUDGET",
                    help="pick n_stab per (Nx, Nt) class with the tuner (fd_tune_nstab_stats): "
                         "the fastest of 4..64 whose log det and G stay within BUDGET of FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true",
                    help="skip the FP64-path measurement reported beside the mixed path")
    args = ap.parse_args()
    if args.workload is None:
        args.workload = "uneven512" if args.path == "force" else "batch18"
    if args.steps is None:
        args.steps = 5 if args.workload == "uneven512" else 500
    if args.impl == "reference":
        return run_reference(args)
    if args.path == "bss":
        return run_bss(args)
    if args.path == "sparse":
        return run_sparse(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
