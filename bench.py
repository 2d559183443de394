"""Throughput of the pruned H.psi inside full propagation steps on one GB300.

Workload (default): 6D Henon-Heiles chain, lambda = 0.111803, HO-DVR 24 points
per mode (24^6 = 1.91e8 lattice points), coherent packet at q_k = 2, threshold
1e-6, SIL order 10, dt = 0.1, complex64 H.psi with FP64 Lanczos scalars.  A
step is one SIL step (10 H.psi) + adaption + observables.

value     active-coefficient H.psi applications per second (Gcoef/s) over the
          timed steps, inputs resident in HBM.
e2e       the same metric through the host-buffer C-ABI call pq_apply_H_host
          (copies from pinned host memory and back inside the timed region).
roofline  the pruned H.psi (all its passes) against the measured HBM copy
          bandwidth, with 20 algorithmic bytes per active coefficient
          (psi read 8 B, H.psi write 8 B, index 4 B).
cpu_baseline / --impl reference: the FP64 oracle's H.psi on a bounded sample
          of output points of the same state, on the host cores.

Replicas only: under torchrun every rank runs its own independent replica of
the workload on its own GPU; value = all ranks' coefficients / the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

BYTES_PER_COEF = {"fp32mix": 20, "fp64": 36}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def code_digest(path):
    """SHA-256 of a C++/CUDA source with its comments and whitespace removed:
    the same digest means the same tokens reach the compiler, so an edit of a
    comment keeps counters taken on the file valid.  (The sources it is used on
    have no comment markers inside string literals.)"""
    with open(path) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", " ", txt)
    txt = " ".join(txt.split())
    return hashlib.sha256(txt.encode()).hexdigest()


APPLY_SOURCES = ("apply_h.cu",)


def apply_digest(root=None):
    """Code digest of the DVR H.psi kernel sources (APPLY_SOURCES), each
    digested by code_digest, then the digests hashed together."""
    root = ROOT if root is None else root
    h = hashlib.sha256()
    for name in APPLY_SOURCES:
        p = os.path.join(root, "paper_1606_04004_gb300", "csrc", name)
        h.update((code_digest(p) if os.path.exists(p) else "absent").encode())
    return h.hexdigest()


def _traffic_record():
    """DRAM bytes per active coefficient of the H.psi kernels from the committed
    ncu summary, if it was taken on the current kernel sources (same digest)."""
    p = os.path.join(ROOT, "profiles", "apply_h_hh6d_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("apply_code_sha256") != apply_digest():
        return None
    return rec


def fibre_flops_per_coef(A, dims):
    """Algorithmic FP32 operations of one pruned DVR H.psi per active
    coefficient: 4 per active member of each of the point's D fibres (a real
    matrix element times a complex coefficient, Sec. 2.2.2) plus 4 for the
    diagonal potential times the coefficient.  Host bookkeeping on the active
    set (numpy), not part of the timed work."""
    dims = tuple(int(d) for d in dims)
    if len(A) == 0:
        return 0.0
    m = np.zeros(int(np.prod(dims)), dtype=bool)
    m[np.asarray(A, dtype=np.int64)] = True
    m = m.reshape(dims)
    total = 0
    for k in range(len(dims)):
        cnt = m.sum(axis=k, keepdims=True, dtype=np.int64)
        total += int((np.broadcast_to(cnt, m.shape) * m).sum(dtype=np.int64))
    return 4.0 * total / len(A) + 4.0


def fp32_peak_tflops():
    """FP32 FMA rate of this GPU, measured now (scalar and packed two-lane
    FMA chains, the larger of the two)."""
    import paper_1606_04004_gb300 as pq
    r1 = pq.measure_peak(pq.PEAK_FP32)
    r2 = pq.measure_peak(pq.PEAK_FP32X2)
    return max(r1["tflops"], r2["tflops"]), {"fp32_ffma": r1["tflops"], "fp32_ffma2": r2["tflops"]}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_replicas(ms, coef, dist, device):
    """Replica aggregation of the timed region: the slowest rank's time and the
    coefficients all ranks applied (value = their ratio).  dist is
    torch.distributed or None (one process)."""
    if dist is None:
        return ms, coef
    import torch
    t = torch.tensor([ms, coef], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def oracle_sample_rate(cfg, A, psi, n_sample, seed=0):
    """The FP64 oracle's pruned H.psi on n_sample output points of (A, psi):
    returns (coefficients per second, seconds, sample size)."""
    from oracle import propagate, pruned
    prob = propagate.problem_from_config(cfg)
    rng = np.random.default_rng(seed)
    pos = np.sort(rng.choice(len(A), size=min(n_sample, len(A)), replace=False))
    t0 = time.perf_counter()
    vd = prob.vdiag(A[pos])
    pruned.apply_H_at(A, psi.astype(np.complex128), prob.dims, prob.Ts, vd, pos)
    dt = time.perf_counter() - t0
    return len(pos) / dt, dt, len(pos)


_ORACLE_WORKER = {}


def _oracle_worker_init(cfg, shm_names, shapes, dtypes):
    from multiprocessing import shared_memory
    from oracle import propagate
    arrs = []
    for name, shape, dt in zip(shm_names, shapes, dtypes):
        shm = shared_memory.SharedMemory(name=name)
        arrs.append((shm, np.ndarray(shape, dtype=dt, buffer=shm.buf)))
    _ORACLE_WORKER.update(cfg=cfg, A=arrs[0][1], psi=arrs[1][1], shm=[a[0] for a in arrs],
                          prob=propagate.problem_from_config(cfg))


def _oracle_worker_apply(pos):
    from oracle import pruned
    w = _ORACLE_WORKER
    prob, A = w["prob"], w["A"]
    vd = prob.vdiag(A[pos])
    pruned.apply_H_at(A, w["psi"], prob.dims, prob.Ts, vd, pos)
    return len(pos)


def oracle_sample_rate_cores(cfg, A, psi, n_sample, cores, seed=0, reps=1):
    """The same oracle H.psi sample split over `cores` processes (spawned,
    A and psi in shared memory, the sample in one chunk per process): returns
    (coefficients per second, seconds per rep, sample size).  Only the
    parallel apply is timed (wall clock, after the workers are up)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    A = np.ascontiguousarray(A, dtype=np.int64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    shms = []
    try:
        for arr in (A, psi):
            shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
            np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)[...] = arr
            shms.append(shm)
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_oracle_worker_init,
                      initargs=(cfg, [m.name for m in shms], [A.shape, psi.shape],
                                [A.dtype, psi.dtype])) as pool:
            rng = np.random.default_rng(seed)
            pos = np.sort(rng.choice(len(A), size=min(n_sample, len(A)), replace=False))
            chunks = np.array_split(pos, cores)
            pool.map(_oracle_worker_apply, [c[: max(1, len(c) // 20)] for c in chunks])  # warm
            t0 = time.perf_counter()
            for _ in range(reps):
                pool.map(_oracle_worker_apply, chunks)
            dt = (time.perf_counter() - t0) / reps
    finally:
        for m in shms:
            m.close()
            m.unlink()
    return len(pos) / dt, dt, len(pos)


def run_reference(args, cfg):
    """--impl reference: the oracle, as it stands, on the host cores."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import propagate
    prob = propagate.problem_from_config(cfg)
    A, a, _ = propagate.initial_state(prob, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"])
    n_sample = max(1000, args.ref_sample // 4)
    cores = os.cpu_count() or 1
    secs = []
    for i in range(args.warmup + args.steps):
        r, dt, n = oracle_sample_rate_cores(cfg, A, a, n_sample * cores // 4, cores, seed=i)
        if i >= args.warmup:
            secs.append((dt, n))
    v = sum(n for _, n in secs) / sum(dt for dt, _ in secs) / 1e9
    line = {
        "impl": "reference", "metric": "pruned H.psi active-coefficient applications per second",
        "value": v, "unit": "Gcoef/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(dt for dt, _ in secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "lattice": f"{cfg['n']}^{cfg['D']}",
                   "theta": cfg["theta"], "n_active": int(len(A))},
        "cpu_baseline": {"value": v, "unit": "Gcoef/s", "cores": cores, "kind": "oracle",
                         "sample": f"{secs[-1][1]} output points of the initial {cfg['name']} "
                                   f"state per step, split over {cores} processes "
                                   f"(numpy, FP64, one thread each)"},
        "e2e": {"value": v, "unit": "Gcoef/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, cfg):
    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1606_04004_gb300 as pq

    prec = pq.FP32MIX if args.precision == "fp32mix" else pq.FP64
    b = pq.build_model(cfg)
    cap = args.capacity
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec, capacity=cap)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    K, dt, th = cfg["K"], cfg["dt"], cfg["theta"]
    # warm-up steps (untimed)
    s.propagate(K, dt, th, args.warmup, stream=sptr, reorth=args.reorth)
    n_before = len(s.observables()["n_active"])
    dims = (cfg["n"],) * cfg["D"]
    fpc_first = fibre_flops_per_coef(s.read()[0], dims) if prec == pq.FP32MIX else None
    s.set_timing(True)
    launches0 = pq.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        s.propagate(K, dt, th, args.steps, stream=sptr, reorth=args.reorth)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = pq.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    obs = s.observables()
    na = obs["n_active"]
    coef = float(np.sum(na[n_before - 1:n_before - 1 + args.steps])) * K
    tm = s.timing()
    ms_max, coef_all = aggregate_replicas(ms, coef, dist, "cuda")
    value = coef_all / (ms_max * 1e-3) / 1e9

    # roofline of the pruned H.psi (all passes), timed with CUDA events on
    # the propagation stream inside the timed region
    peak, peak_kind = _peaks()
    bpc = BYTES_PER_COEF[args.precision]
    apply_s = tm["apply_ms"] * 1e-3
    achieved = tm["coef_applied"] * bpc / apply_s / 1e9 if apply_s > 0 else 0.0
    trec = _traffic_record()
    traffic = None
    if trec and args.precision == "fp32mix" and cfg["name"] == trec.get("workload"):
        traffic = trec["dram_bytes_per_coef"] * tm["coef_applied"] / max(tm["n_apply"], 1)
    alu = None
    if fpc_first is not None and apply_s > 0:
        # FP32 ALU roofline of the same launches: algorithmic flops per coefficient
        # of the first and the last timed set, weighted by their sizes (the set
        # grows over the window)
        na_first, na_last = float(na[n_before - 1]), float(na[-1])
        fpc_last = fibre_flops_per_coef(s.read()[0], dims)
        fpc = (fpc_first * na_first + fpc_last * na_last) / (na_first + na_last)
        alu_peak, alu_parts = fp32_peak_tflops()
        alu_ach = tm["coef_applied"] * fpc / apply_s / 1e12
        alu = {"achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
               "flop_per_coef": fpc, "flop_per_coef_first_last": [fpc_first, fpc_last],
               "peak_kind": "measured in this run (FP32 FMA chains)", **alu_parts}

    # e2e: the host-buffer C-ABI call on the final state
    A_n = s.size()
    hdt = torch.complex64 if prec == pq.FP32MIX else torch.complex128
    xh = torch.randn(A_n, dtype=hdt).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    import ctypes
    lib = pq._lib
    for _ in range(2):
        lib.pq_apply_H_host(s._h, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(yh.data_ptr()),
                            prec, ctypes.c_void_p(sptr))
    reps = max(3, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        rc = lib.pq_apply_H_host(s._h, ctypes.c_void_p(xh.data_ptr()),
                                 ctypes.c_void_p(yh.data_ptr()), prec, ctypes.c_void_p(sptr))
        if rc:
            raise RuntimeError(lib.pq_last_error().decode())
    e2e_s = (time.perf_counter() - t0) / reps
    esz = 8 if prec == pq.FP32MIX else 16
    e2e = {"value": A_n / e2e_s / 1e9 * ws, "unit": "Gcoef/s",
           "h2d_bytes_per_step": A_n * esz, "d2h_bytes_per_step": A_n * esz}

    # late window: the same state propagated on (untimed) to step --late-start,
    # then args.steps steps timed the same way (the hh6d set fills the whole
    # lattice after about 100 steps and stays there for the rest of the run)
    late = None
    if args.late_start > 0 and ws == 1:
        done = len(s.observables()["n_active"]) - 1
        if args.late_start > done:
            s.set_timing(False)
            s.propagate(K, dt, th, args.late_start - done, stream=sptr, reorth=args.reorth)
        n0 = len(s.observables()["n_active"])
        s.set_timing(True)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk_late:
            g0.record(stream)
            s.propagate(K, dt, th, args.steps, stream=sptr, reorth=args.reorth)
            g1.record(stream)
            torch.cuda.synchronize()
        ms_late = g0.elapsed_time(g1)
        na_l = s.observables()["n_active"]
        coef_l = float(np.sum(na_l[n0 - 1:n0 - 1 + args.steps])) * K
        tl = s.timing()
        apply_l = tl["apply_ms"] * 1e-3   # set_timing(True) restarted the counters
        capp_l = tl["coef_applied"]
        ach_l = capp_l * bpc / apply_l / 1e9 if apply_l > 0 else 0.0
        late = {"steps": [n0 - 1, n0 - 1 + args.steps], "value": coef_l / (ms_late * 1e-3) / 1e9,
                "unit": "Gcoef/s", "ms_per_step": ms_late / args.steps,
                "n_active_first": int(na_l[n0 - 1]), "n_active_last": int(na_l[-1]),
                "lattice_points": int(cfg["n"] ** cfg["D"]),
                "apply_gcoef_s": capp_l / apply_l / 1e9 if apply_l > 0 else None,
                "achieved_gbs": ach_l, "frac": ach_l / peak, "clocks": clk_late.summary()}

    # the same early window with the other Lanczos orthogonalisation, from a
    # fresh state (same packet, warm-up and steps)
    other = None
    if ws == 1 and not args.no_fp64_compare:
        ro = 1 - args.reorth
        s2 = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec, capacity=cap)
        s2.propagate(K, dt, th, args.warmup, stream=sptr, reorth=ro)
        n2b = len(s2.observables()["n_active"])
        s2.set_timing(True)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        s2.propagate(K, dt, th, args.steps, stream=sptr, reorth=ro)
        h1.record(stream)
        torch.cuda.synchronize()
        ms2 = h0.elapsed_time(h1)
        o2 = s2.observables()
        t2 = s2.timing()
        coef2 = float(np.sum(o2["n_active"][n2b - 1:n2b - 1 + args.steps])) * K
        other = {"lanczos": "three-term recurrence" if ro == 0 else "full re-orthogonalisation",
                 "value": coef2 / (ms2 * 1e-3) / 1e9, "unit": "Gcoef/s", "ms_per_step": ms2 / args.steps,
                 "apply_gcoef_s": t2["coef_applied"] / (t2["apply_ms"] * 1e-3) / 1e9 if t2["apply_ms"] else None,
                 "max_abs_dC_vs_main": float(np.max(np.abs(o2["C"][:len(obs["C"])] - obs["C"][:len(o2["C"])])))}
        s2.free()

    line = {
        "metric": "pruned H.psi active-coefficient applications per second",
        "value": value, "unit": "Gcoef/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64" if prec == pq.FP32MIX else "c128",
        "data": "synthetic",
        "config": {"workload": f"{cfg['name']}: {cfg['D']}D Henon-Heiles chain, HO-DVR "
                               f"{cfg['n']}^{cfg['D']}, theta {cfg['theta']}, SIL K={K}, dt={dt}",
                   "precision": args.precision,
                   "lanczos": "three-term recurrence" if args.reorth == 0 else "full re-orthogonalisation",
                   "n_active_first": int(na[n_before - 1]),
                   "n_active_last": int(na[-1]), "parallelism": f"replicas{ws}",
                   "l2": "working set larger than L2 (Krylov space of 10 vectors)"},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "pruned H.psi (inner + outer fibre passes)",
                     "bytes_per_coef": bpc, "peak_kind": peak_kind,
                     "apply_gcoef_s": tm["coef_applied"] / apply_s / 1e9 if apply_s else None,
                     "alu": alu, "alu_frac": alu["frac"] if alu else None},
        "clocks": clk.summary(),
        "e2e": e2e,
        "late_window": late,
        "other_orthogonalisation": other,
    }

    if rank == 0 and ws == 1 and not args.no_fp64_compare and prec == pq.FP32MIX:
        # the same steps on the plain FP64 GPU path, from the same initial state
        s64 = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64,
                       capacity=cap)
        s64.propagate(K, dt, th, args.warmup, stream=sptr, reorth=args.reorth)
        s64.set_timing(True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.propagate(K, dt, th, args.steps, stream=sptr, reorth=args.reorth)
        f1.record(stream)
        torch.cuda.synchronize()
        o64 = s64.observables()
        ms64 = f0.elapsed_time(f1)
        coef64 = float(np.sum(o64["n_active"][n_before - 1:n_before - 1 + args.steps])) * K
        v64 = coef64 / (ms64 * 1e-3) / 1e9
        n = min(len(o64["C"]), len(obs["C"]))
        line["fp64_gpu"] = {"value": v64, "unit": "Gcoef/s", "speedup_fp32mix": value / v64,
                            "max_abs_dC": float(np.max(np.abs(o64["C"][:n] - obs["C"][:n]))),
                            "max_abs_dnorm2": float(np.max(np.abs(o64["norm2"][:n] - obs["norm2"][:n])))}
        s64.free()

    if rank == 0 and ws == 1 and not args.no_cpu:
        A, psi = s.read()
        r, secs, nsamp = oracle_sample_rate(cfg, A, psi, args.ref_sample)
        line["cpu_baseline"] = {"value": r / 1e9, "unit": "Gcoef/s", "cores": 1, "kind": "oracle",
                                "sample": f"{nsamp} output points of the final state "
                                          f"({len(A)} active), FP64 numpy, {secs:.1f} s"}
        cores = os.cpu_count() or 1
        rc_, secs_c, n_c = oracle_sample_rate_cores(cfg, A, psi, args.ref_sample * cores // 4, cores)
        line["cpu_baseline_all_cores"] = {
            "value": rc_ / 1e9, "unit": "Gcoef/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_c} output points of the final state split over {cores} processes "
                      f"(FP64 numpy, one thread each), {secs_c:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_apply(args, cfg):
    """H.psi microbenchmark: the workload's Hamiltonian on a synthetic 6D
    ellipsoid active set (realistic ragged fibres), random complex psi, an L2
    flush between launches, CUDA events on the launching stream."""
    import torch
    import paper_1606_04004_gb300 as pq
    prec = pq.FP32MIX if args.precision == "fp32mix" else pq.FP64
    if args.lattice:   # a smaller lattice of the same model (profiling captures)
        cfg = W.scaled(cfg, n=args.lattice)
    b = pq.build_model(cfg)
    r = args.radius
    A = W.ellipsoid_active_set((cfg["n"],) * cfg["D"], (r,) * cfg["D"])
    s = pq.State(b, [0.0] * cfg["D"], [0.0] * cfg["D"], [1.0] * cfg["D"], 1e30, precision=prec,
                 capacity=len(A))
    s.load(A)
    tdt = torch.complex64 if prec == pq.FP32MIX else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(len(A), dtype=tdt, device="cuda", generator=g)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        s.apply_H(x, y)
    times = []
    for _ in range(args.reps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.apply_H(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    med = statistics.median(times) * 1e-3
    peak, kind = _peaks()
    bpc = BYTES_PER_COEF[args.precision]
    fpc = fibre_flops_per_coef(A, (cfg["n"],) * cfg["D"])
    alu_peak, alu_parts = fp32_peak_tflops()
    alu = len(A) * fpc / med / 1e12
    print(json.dumps({"mode": "apply", "workload": cfg["name"], "precision": args.precision,
                      "n_active": int(len(A)), "radius": r, "median_us": med * 1e6,
                      "gcoef_s": len(A) / med / 1e9, "achieved_gbs": len(A) * bpc / med / 1e9,
                      "frac_hbm": len(A) * bpc / med / 1e9 / peak, "peak": peak,
                      "peak_kind": kind, "flop_per_coef": fpc, "alu_tflops": alu,
                      "alu_peak_tflops": alu_peak, "alu_frac": alu / alu_peak, **alu_parts,
                      "reps": args.reps}), flush=True)


TF32_NOMINAL_OVER_BF16 = 1.1 / 2.25   # dense tensor rates of the part, TF32 over BF16


def run_apply_phase_space(args, cfg):
    """H.psi microbenchmark of the 3D coupled Morse workload in projected
    Weylets (pW: nine pruned single-mode passes of dense 64 x 64 factors) or
    in pvB (H_AA on the full 64^3 grid: B, the kinetic matrix and B^dagger
    along every mode), on the workload's initial state, FP32-mix (tensor
    cores, split TF32).  Reports Gcoef/s and the tensor-core work: the MMA
    flops the passes issue (split TF32 = 3 products, fibres zero-padded to 64)
    against the TF32 dense peak (the measured BF16 peak x the nominal
    TF32 / BF16 ratio of the part), and the useful (unpadded, single-product)
    flops."""
    import torch
    import paper_1606_04004_gb300 as pq
    basis = "pvb" if args.config == "morse3d_pvb" else "pw"
    c = W.scaled(W.MORSE3D, basis=basis, q0=W.morse3d_centres(W.MORSE3D["seed"]))
    b = pq.build_model(c)
    s = pq.State(b, c["q0"], c["p0"], c["width"], c["theta"], precision=pq.FP32MIX)
    A, psi = s.read()
    x = torch.from_numpy(psi).to("cuda")
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        s.apply_H(x, y)
    launches0 = pq.launch_count()
    times = []
    for _ in range(args.reps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.apply_H(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = (pq.launch_count() - launches0) / args.reps
    med = statistics.median(times) * 1e-3
    D, n = c["D"], c["n"]
    dims = (n,) * D
    m = np.zeros(n ** D, bool)
    m[A] = True
    m = m.reshape(dims)
    if basis == "pw":
        # passes per mode: the merged single-mode factor + two pair terms
        passes = {k: 1 + (D - 1) for k in range(D)}
        tiles, useful = 0, 0.0
        for k in range(D):
            L = np.broadcast_to(m.sum(axis=k, keepdims=True), m.shape)[m]
            useful += passes[k] * 4.0 * float(L.sum())
            if k == D - 1:
                t = -(-int(m.any(axis=D - 1).sum()) // 64)          # active rows, 64 per tile
            else:
                t = int(m.any(axis=(k, D - 1)).sum())               # fibre planes
            tiles += passes[k] * t
        mma = tiles * 3 * 2.0 * 128 * 64 * 64
    else:
        ntile = (n ** D // n) // 64
        cplx = 3 * 2.0 * 128 * 128 * 64 * ntile          # a complex transform, all tiles
        real = 3 * 2.0 * 128 * 64 * 64 * ntile
        mma = 2 * D * cplx + D * real
        useful = 2 * D * 8.0 * n * n ** D + D * 4.0 * n * n ** D
    bf16 = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    tf32_peak = (bf16 if bf16 else 1900.0) * TF32_NOMINAL_OVER_BF16
    print(json.dumps({"mode": "apply", "workload": f"morse3d ({basis})", "precision": "fp32mix",
                      "n_active": int(len(A)), "median_us": med * 1e6,
                      "gcoef_s": len(A) / med / 1e9, "launches_per_apply": launches,
                      "tensor_mma_tflops": mma / med / 1e12, "useful_tflops": useful / med / 1e12,
                      "tf32_peak_tflops": tf32_peak,
                      "tf32_peak_kind": "measured BF16 burst x nominal TF32/BF16 (1.1/2.25)"
                                        if bf16 else "fallback BF16 1.9 PF x nominal ratio",
                      "tensor_frac": mma / med / 1e12 / tf32_peak, "reps": args.reps}), flush=True)


def run_snapshots(args, cfg):
    """H.psi microbenchmark on the propagation's own active sets: the hh6d run
    (FP32-mix) is stopped at the listed steps and the H.psi of its current
    (A, psi) is timed there (median of --reps, L2 flushed between launches)."""
    import torch
    import paper_1606_04004_gb300 as pq
    prec = pq.FP32MIX if args.precision == "fp32mix" else pq.FP64
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=prec, capacity=0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    tdt = torch.complex64 if prec == pq.FP32MIX else torch.complex128
    peak, kind = _peaks()
    bpc = BYTES_PER_COEF[args.precision]
    done = 0
    for step in sorted(int(v) for v in args.snapshots.split(",")):
        if step > done:
            s.propagate(cfg["K"], cfg["dt"], cfg["theta"], step - done)
            done = step
        n = s.size()
        x = torch.empty(n, dtype=tdt, device="cuda")
        x.copy_(torch.from_numpy(s.read()[1]).to("cuda"))
        y = torch.empty_like(x)
        for _ in range(3):
            s.apply_H(x, y)
        times = []
        for _ in range(args.reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.apply_H(x, y)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        med = statistics.median(times) * 1e-3
        print(json.dumps({"mode": "snapshot", "workload": cfg["name"], "precision": args.precision,
                          "step": step, "n_active": int(n), "median_us": med * 1e6,
                          "gcoef_s": n / med / 1e9, "frac_hbm": n * bpc / med / 1e9 / peak,
                          "peak": peak, "peak_kind": kind, "reps": args.reps}), flush=True)
        del x, y


def run_peaks(args):
    """Measured arithmetic peaks of this GPU: FP32 scalar and packed two-lane
    FMA chains and FP64 FMA chains (pq_measure_peak), with the SM clock sampled
    while they run."""
    import paper_1606_04004_gb300 as pq
    import torch
    torch.cuda.init()
    out = {"mode": "peaks"}
    with ClockSampler(0) as clk:
        for name, kind, iters in (("fp32_ffma", pq.PEAK_FP32, 8192), ("fp32_ffma2", pq.PEAK_FP32X2, 8192),
                                  ("fp64_dfma", pq.PEAK_FP64, 512)):
            best = max(pq.measure_peak(kind, iters)["tflops"] for _ in range(5))
            out[name + "_tflops"] = best
    out["clocks"] = clk.summary()
    print(json.dumps(out), flush=True)


def run_dwell(args):
    """Accuracy study on the paper's 2D double well (Sec. 3.1; the comparisons
    of its neighbour-radius and basis figures): the pruned FGH DVR and the
    projected Weylets built on the same FGH grids.  For each basis, neighbour
    rule and threshold, propagate to t_e = 24.6 in FP64 and report the mean
    number of basis functions used (percent of the 13365) and the infidelity,
    the Euclidean L2 distance between the C(t) series of the pruned run and of
    the unpruned FGH run (theta = 0)."""
    import paper_1606_04004_gb300 as pq

    def series(cfg, theta, rule, prec=None):
        b = pq.build_model(cfg)
        prec = pq.FP64 if prec is None else prec
        s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], theta, precision=prec, radius=rule)
        s.propagate(cfg["K"], cfg["dt"], theta, cfg["nsteps"], radius=rule)
        o = s.observables()
        s.free()
        return o

    t0 = time.perf_counter()
    nfull = int(np.prod(W.DWELL2D["n"]))
    exact = series(W.DWELL2D, 0.0, 1)
    assert int(exact["n_active"].min()) == nfull
    thetas = (3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 1e-6, 1e-8)
    # on the 2D coordinate lattice radius sqrt 2 and radius 2 add the same 8 neighbours
    plan = [(W.DWELL2D, "fgh", pq.RADIUS_1, "1"), (W.DWELL2D, "fgh", pq.RADIUS_SQRT2, "sqrt2"),
            (W.DWELL2D_PW, "pw", pq.RADIUS_1, "1"), (W.DWELL2D_PW, "pw", pq.RADIUS_SQRT2, "sqrt2"),
            (W.DWELL2D_PW, "pw", pq.RADIUS_2, "2"), (W.DWELL2D_PVB, "pvb", pq.RADIUS_1, "1")]
    # pvB is left out unless asked for: every Krylov vector needs a solve of
    # S_AA (preconditioned conjugate gradients), about 0.23 s per FP64 step and
    # 0.07 s per FP32-mix step; --dwell-pvb-fp32 runs its column in FP32-mix
    wanted = args.dwell_bases.split(",") if args.dwell_bases else ["fgh", "pw"]
    plan = [p for p in plan if p[1] in wanted]
    for cfg, basis, rule, name in plan:
        prec = pq.FP32MIX if (basis == "pvb" and args.dwell_pvb_fp32) else pq.FP64
        th_list = thetas if basis != "pvb" else (3e-2, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)
        if args.dwell_thetas:
            th_list = tuple(float(v) for v in args.dwell_thetas.split(","))
        for theta in th_list:
            o = series(cfg, theta, rule, prec)
            row = {"mode": "dwell", "basis": basis, "radius": name, "theta": theta,
                   "precision": "fp32mix" if prec == pq.FP32MIX else "fp64",
                   "mean_basis_pct": float(100.0 * o["n_active"].mean() / nfull),
                   "infidelity": float(np.linalg.norm(o["C"] - exact["C"]))}
            print(json.dumps(row), flush=True)
    print(json.dumps({"mode": "dwell", "summary": True, "t_end": W.DWELL2D["dt"] * W.DWELL2D["nsteps"],
                      "steps": W.DWELL2D["nsteps"], "K": W.DWELL2D["K"], "dt": W.DWELL2D["dt"],
                      "seconds": time.perf_counter() - t0}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="hh6d")
    ap.add_argument("--precision", default="fp32mix", choices=["fp32mix", "fp64"])
    ap.add_argument("--capacity", type=int, default=0)   # 0 = the full lattice
    ap.add_argument("--ref-sample", type=int, default=1_000_000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--mode", default="step", choices=["step", "apply", "dwell", "snapshot", "peaks"])
    ap.add_argument("--radius", type=float, default=11.2)
    ap.add_argument("--lattice", type=int, default=0)
    # Lanczos orthogonalisation of the timed runs: 1 = each Krylov vector
    # against all earlier ones, 0 = the three-term recurrence (the line also
    # reports an early window with the other one)
    ap.add_argument("--reorth", type=int, default=1)
    ap.add_argument("--late-start", type=int, default=100)   # step the late window starts at (0: none)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--snapshots", default="0,20,50,100")   # steps of --mode snapshot
    ap.add_argument("--dwell-bases", default="")   # comma list of fgh,pw,pvb (default fgh,pw)
    ap.add_argument("--dwell-pvb-fp32", action="store_true")   # the pvB column in FP32-mix
    ap.add_argument("--dwell-thetas", default="")   # comma list replacing the thresholds of --mode dwell
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("need at least 3 warm-up steps")
    if args.config in ("morse3d", "morse3d_pvb"):
        if args.mode != "apply":
            raise SystemExit("--config morse3d / morse3d_pvb: only --mode apply")
        run_apply_phase_space(args, None)
        return
    cfg = W.CONFIGS[args.config]
    if args.mode == "apply":
        run_apply(args, cfg)
    elif args.mode == "peaks":
        run_peaks(args)
    elif args.mode == "dwell":
        run_dwell(args)
    elif args.mode == "snapshot":
        run_snapshots(args, cfg)
    elif args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
