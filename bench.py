"""Benchmark of the H2*(b+t) matrix-vector product on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--storage f64|f32] [--variant h2star|h2plush|h2sqrt]

A step is one full MVP (gather, P2M, M2M, M2L far + vertex-sharing, L2L, L2P
with the near field evaluated on the fly, scatter) on the default workload:
3D 1/r, N = 262144 points uniform in [-1, 1]^3, octree with leaves of <= 64
points on average (kappa 4), NCA tolerance 1e-6, one N(0, 1) right-hand side,
fp64.  The operators (GBs) are larger than the 129 MB L2, so no flush is
needed between steps.  Prints one JSON line (rank 0).

--impl reference times the FP64 CPU oracle (exact product, sampled rows) on
the host cores instead.  Under torchrun each rank runs an independent replica
(no collective on the data path); value is the sum over ranks.
"""

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H2* MVP points·RHS/s and % HBM roofline; GMRES solve p50/p99 latency"
UNIT = "points*RHS/s"
KERNEL_NAMES = {"log2d": "log r (2D)", "invr": "1/r (3D)", "imq": "inverse multiquadric",
                "matern12": "exp(-r)"}
VARIANT_NAMES = {"h2star": "H2*(b+t)", "h2plush": "(H2+H)*", "h2sqrt": "H2_sqrt(d)(b)",
                 "h2star_t": "H2*(t)", "h2sqrt_t": "H2_sqrt(d)(t)", "h2star_b": "B2T over IL_* (naive)"}
# DRAM traffic / algorithmic bytes of the M2L block-row launch, from one ncu
# capture of the current kernel (profiles/k_rowgemv1_m2l_c2s_3d_invr_n32768.md);
# traffic grows with the stored blocks, so a full launch's traffic is this
# ratio times its algorithmic bytes.
M2L_TRAFFIC_RATIO = {"df64": 0.992, "f64": 0.995, "f32": 0.999}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- oracle legs
#: points of the sample on which the oracle's own H2* MVP is timed (its
#: construction, once per geometry, is not timed; at N = 8192 it takes ~10 s)
MVP_SAMPLE_N = 8192


def oracle_child(kind, workload, seconds):
    """Runs in a fresh single-threaded process.  kind 'rows': exact rows of
    K q by the oracle's dense definition (O1), sampled until `seconds` of
    work; kind 'mvp': the oracle's H2*(b+t) MVP (O2) on MVP_SAMPLE_N points of
    the same kernel, tolerance and leaf size, repeated until `seconds`."""
    from oracle import dense, h2
    from paper_2309_14085_gb300 import inputs
    w = inputs.workload(workload)
    nrhs = w["nrhs"]
    if kind == "rows":
        P, q = w["points"], w["q"]
        rng = np.random.default_rng(0)
        rows, t_used = 0, 0.0
        while t_used < seconds:
            idx = rng.choice(P.shape[0], 16, replace=False)
            t0 = time.perf_counter()
            dense.rows(w["kernel"], P, q, idx, chunk=16)
            t_used += time.perf_counter() - t0
            rows += 16
        out = {"units": rows, "seconds": t_used, "value": rows * nrhs / t_used}
    else:
        n = min(w["N"], MVP_SAMPLE_N)
        P = inputs.points(n, w["d"], 1000 + w["number"])
        q = inputs.rhs(n, nrhs, 2000 + w["number"])
        H = h2.H2(P, w["kernel"], n_max=w["n_max"], eps=w["eps"])
        done, t_used = 0, 0.0
        while t_used < seconds or done == 0:
            t0 = time.perf_counter()
            H.matvec(q)
            t_used += time.perf_counter() - t0
            done += 1
        out = {"units": done * n, "seconds": t_used, "value": done * n * nrhs / t_used, "n": n}
    print(json.dumps(out))


def reference_child(workload, rows, warmup, steps):
    """Runs in a fresh single-threaded process: warmup + steps exact products
    on `rows` sampled rows each; prints the time of every timed step."""
    from oracle import dense
    from paper_2309_14085_gb300 import inputs
    w = inputs.workload(workload)
    P, q = w["points"], w["q"]
    rng = np.random.default_rng(0)
    ms = []
    for i in range(warmup + steps):
        idx = rng.choice(P.shape[0], rows, replace=False)
        t0 = time.perf_counter()
        dense.rows(w["kernel"], P, q, idx, chunk=16)
        if i >= warmup:
            ms.append(1e3 * (time.perf_counter() - t0))
    print(json.dumps({"step_ms": ms}))


def run_oracle(kind, workload, seconds, procs=1):
    """The oracle leg `kind` in `procs` single-threaded processes at once (one
    independent replica per host core); value = the sum of their rates."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-child", kind, workload, str(seconds)]
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    res = []
    for p in ps:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle child failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    r = {"value": float(sum(x["value"] for x in res)), "cores": procs,
         "seconds": max(x["seconds"] for x in res)}
    if kind == "rows":
        r["sample"] = (f"{sum(x['units'] for x in res)} exact rows of K q (dense definition, "
                       f"oracle.dense.rows) of the same workload, {r['seconds']:.1f} s in {procs} "
                       f"single-threaded process(es)")
    else:
        r["sample"] = (f"oracle H2*(b+t) MVP (oracle.h2, construction not timed) on N = "
                       f"{res[0]['n']} points of the same kernel, eps and leaf size, "
                       f"{r['seconds']:.1f} s in {procs} single-threaded process(es)")
    return r


def cpu_baselines(workload, seconds):
    """The oracle on the host: its H2* MVP (O2) and its exact rows (O1), each on
    one core and on every core (os.cpu_count() processes)."""
    nproc = os.cpu_count() or 1
    legs = {}
    for kind in ("mvp", "rows"):
        for procs in (1, nproc):
            legs[f"{kind}_{'1core' if procs == 1 else 'all_cores'}"] = run_oracle(kind, workload, seconds,
                                                                                procs)
    main = legs["mvp_all_cores"]
    return {"value": main["value"], "unit": UNIT, "cores": main["cores"], "kind": "oracle",
            "sample": main["sample"], "nproc": nproc,
            "legs": {k: {"value": v["value"], "cores": v["cores"], "sample": v["sample"]}
                     for k, v in legs.items()}}


# ----------------------------------------------------------------------------- accuracy
GOLDEN = {"c2_3d_invr_n262144": "c2_3d_invr_n262144_rows.txt",
          "c3_2d_log_n1048576": "c3_2d_log_n1048576_rows.txt"}


def golden_accuracy(workload, Y):
    """Relative 2-norm error of the product Y (N x nrhs, on the device) on the
    sampled rows whose exact values an oracle-only script wrote under
    tests/golden/ (the C2 file: row, oracle K~ q, exact K q; the C3 file: row,
    exact (K Q)[row, :])."""
    name = GOLDEN.get(workload)
    if name is None:
        return None
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    t = np.loadtxt(path, comments="#", ndmin=2)
    rows = t[:, 0].astype(np.int64)
    exact = t[:, 2:3] if workload.startswith("c2") else t[:, 1:]
    import torch
    got = Y[torch.as_tensor(rows, device=Y.device)].double().cpu().numpy().reshape(len(rows), -1)
    got = got[:, :exact.shape[1]]
    re = float(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    return {"re_vs_exact": re, "rows": int(len(rows)), "rhs": int(exact.shape[1]),
            "source": f"tests/golden/{name} (exact rows written by the oracle)"}


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"h2_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- replicas
def replica_max_ms(ms_local, world, device):
    """The slowest rank's time: every rank runs an independent replica of the
    same work (no collective on the data path), so the job takes the maximum."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ms_total_local, units_per_step, steps, world, device):
    """(ms per step of the slowest rank, whole-job units per second): the units
    of all ranks over the slowest rank's time."""
    ms_step = replica_max_ms(ms_total_local, world, device) / steps
    return ms_step, world * units_per_step / (ms_step / 1e3)


# ----------------------------------------------------------------------------- our arm
def bench_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_2309_14085_gb300 import H2Matrix, inputs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    w = inputs.workload(args.workload)
    if args.nrhs:
        w["nrhs"] = args.nrhs
        w["q"] = inputs.rhs(w["N"], args.nrhs, 2000 + w["number"])
    N, nrhs = w["N"], w["nrhs"]
    t0 = time.perf_counter()
    A = H2Matrix(w["points"], w["kernel"], leaf_size=w["n_max"], tol=w["eps"],
                 variant=args.variant, storage=args.storage,
                 tensor_cores=bool(args.tensor_cores) and args.storage == "f32",
                 near="stored" if args.tensor_cores else args.near,
                 m2l="fly" if (args.m2l == "fly" and args.storage == "f32") else
                 ("device" if args.m2l == "device" else None))
    build_s = time.perf_counter() - t0
    info = A.info()
    q = torch.tensor(w["q"].reshape(N, nrhs), dtype=torch.float64, device=dev)
    Xc = q.t().contiguous().t()
    Y = torch.empty((nrhs, N), dtype=torch.float64, device=dev).t()
    stream = torch.cuda.current_stream()

    def step():
        A.matvec(Xc, out=Y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_step, value = replica_throughput(e0.elapsed_time(e1), N * nrhs, args.steps, world, dev)
    accuracy = golden_accuracy(args.workload, Y)

    # the same steps again with CUDA events between the pipeline stages (on the
    # stream the kernels run on): per-stage durations and the launch count
    A.profile(True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof_ms_step = e0.elapsed_time(e1) / args.steps
    stages, calls, launches = A.stage_times()
    A.profile(False)

    # end to end through the public API with host buffers (pinned), copies inside
    hq = torch.tensor(w["q"].reshape(N, nrhs).T.copy(), dtype=torch.float64).pin_memory()
    hy = torch.empty((nrhs, N), dtype=torch.float64).pin_memory()
    dq = torch.empty((nrhs, N), dtype=torch.float64, device=dev)
    dy = torch.empty((nrhs, N), dtype=torch.float64, device=dev)
    e_steps = max(3, min(args.steps, 50))
    for _ in range(2):
        dq.copy_(hq, non_blocking=True)
        A.matvec(dq.t(), out=dy.t())
        hy.copy_(dy, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e_steps):
        dq.copy_(hq, non_blocking=True)
        A.matvec(dq.t(), out=dy.t())
        hy.copy_(dy, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = replica_max_ms(e0.elapsed_time(e1) / e_steps, world, dev)

    # roofline of the dominant kernel (stage timed with CUDA events) among the
    # stages whose algorithmic bytes are known: M2L, the stored leaf rows, and
    # the gather / scatter between user and tree order
    per = {k: v / max(calls, 1) for k, v in stages.items()}
    # coefficient bytes (fp64, float pairs, float, float); operator entry bytes
    # are already in the stored-byte counts of h2_info
    vs = {"f64": 8, "df64": 8, "f32": 4, "bf16": 4}[args.storage]
    known = {"m2l": info["bytes_m2l"] + (info["m2l_src_coeffs"] + info["m2l_dst_coeffs"]) * vs * nrhs,
             "gather": N * nrhs * (8 + vs) + N * 8, "scatter": N * nrhs * (vs + 8) + N * 8}
    if info["near_stored"]:
        known["leaf"] = info["bytes_leaf_rows"] + (info["leaf_src_coeffs"] + N) * vs * nrhs
    dom_all = max(per, key=per.get)
    dom = dom_all if dom_all in known or dom_all == "leaf" else "m2l"
    hbm, how = _peaks()
    roof = {"kernel": dom, "dominant_stage": dom_all, "stage_ms": {k: round(v, 4) for k, v in per.items()},
            "profiled_ms_per_step": round(prof_ms_step, 4)}
    if dom == "m2l" and info["m2l_fly"] == 1:
        # M2L from the pivot coordinates: one kernel evaluation (one MUFU rsqrt /
        # lg2) per entry per RHS tile; peak 16 MUFU ops / clock / SM x 152 SMs x
        # 2.07 GHz
        sec = per[dom] / 1e3
        evals = info["m2l_entries"] * -(-nrhs // 4)
        peak = 16 * 152 * 2.07e9
        roof.update(bound="alu", achieved=round(evals / sec / 1e9, 1), peak=round(peak / 1e9, 1),
                    unit="Gevals/s", frac=round(evals / sec / peak, 4), traffic=None,
                    alg_bytes=None, peak_source="MUFU 16/clk/SM x 152 SMs x 2.07 GHz (nominal)")
    elif dom in known:
        # operators once per product, coefficients once per right-hand side
        alg = known[dom]
        sec = per[dom] / 1e3
        ach = alg / sec / 1e9
        traffic = None
        if (dom == "m2l" and args.variant == "h2star" and args.storage in M2L_TRAFFIC_RATIO
                and nrhs == 1):
            traffic = int(M2L_TRAFFIC_RATIO[args.storage] * alg)
        roof.update(bound="hbm", achieved=round(ach, 1), peak=hbm, unit="GB/s",
                    frac=round(ach / hbm, 4), traffic=traffic, alg_bytes=alg,
                    peak_source=f"{how} hbm_gbs (of measured)")
        if args.storage == "f64" and dom == "m2l":
            # one fp64 multiply-add per stored 8-byte entry: the FP64 pipe bound
            fma = info["bytes_m2l"] / 8 * nrhs / sec / 1e12
            roof["fp64_fma_tflops"] = round(2 * fma, 3)
            roof["fp64_frac_of_nominal_1.25"] = round(2 * fma / 1.25, 4)
    else:
        # near field evaluated on the fly: an ALU-bound stage
        sec = per[dom] / 1e3
        roof.update(bound="alu", achieved=round(info["near_evals"] / sec / 1e9, 2),
                    peak=None, unit="Gevals/s", frac=None, traffic=None,
                    alg_bytes=None, peak_source="kernel evaluations per second (no peak derived)")

    if nrhs == 1:
        # the whole product against the same peak: every stored operator once,
        # the near field's coordinates or blocks, the input and output vectors
        # (h2_info's algorithmic bytes), over the timed step
        wb = info["alg_bytes_per_rhs"]
        roof["whole_mvp"] = {"alg_bytes": wb, "achieved": round(wb / (ms_step / 1e3) / 1e9, 1),
                             "frac": round(wb / (ms_step / 1e3) / 1e9 / hbm, 4)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": args.storage,
        "data": "synthetic (seeded uniform points in [-1,1]^d, N(0,1) right-hand sides)",
        "config": {"workload": args.workload, "N": N, "d": w["d"],
                   "kernel": KERNEL_NAMES[w["kernel"]], "leaf_size": w["n_max"],
                   "kappa": info["kappa"], "eps": w["eps"], "variant": VARIANT_NAMES[args.variant],
                   "storage": args.storage, "nrhs": nrhs, "tensor_cores": bool(args.tensor_cores) or args.storage == "bf16",
                   "m2l": {1: "fly", 2: "stored, formed on the device"}.get(info["m2l_fly"], "stored"),
                   "near_field": "stored blocks" if info["near_stored"] else "evaluated in the product",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "operators larger than L2 (no flush)",
                   "build_seconds": round(build_s, 2),
                   "pivot_search": {"where": "device" if info["pivot_problems_device"] else "host",
                                    "seconds": round(info["pivot_seconds"], 2),
                                    "aca_problems": info["pivot_problems_device"] +
                                    info["pivot_problems_host"]},
                   "device_bytes": info["bytes_device"],
                   "autotuned_rows_per_warp": {"m2l": info["rw_m2l"], "leaf": info["rw_leaf"]},
                   "tc_persistent_ctas": info["tc_blocks"], "tc_occupancy_api": info["tc_occupancy"],
                   "ranks": info["ranks"]},
        "clocks": clk,
        "e2e": {"value": world * N * nrhs / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": N * nrhs * 8, "d2h_bytes_per_step": N * nrhs * 8},
        "gpu_launches": int(launches),   # kernels of the profiled pass = of the timed region
        "roofline": roof,
    }
    if accuracy is not None:
        out["accuracy"] = accuracy
    args._handles = getattr(args, "_handles", {})
    args._handles[args.storage] = A
    return out, w


def bench_gmres(handles, w, nsolve=10, rtol=1e-8):
    """Latency of solves (I + K~/N) x = b to rtol: plain fp64 GMRES and fp32
    iterations refined with fp64 residuals (same points, same right-hand sides)."""
    import torch
    N = w["N"]
    out = {"system": "(I + K/N) x = b, b ~ N(0,1), x0 = 0", "rtol": rtol, "solves": nsolve}
    forms = []
    if "f64" in handles:
        forms.append(("fp64", handles["f64"], None))
    if "f32" in handles and "f64" in handles:
        forms.append(("fp32_refined_fp64", handles["f32"], handles["f64"]))
    if "df64" in handles and "f64" in handles:
        forms.append(("df64_refined_fp64", handles["df64"], handles["f64"]))
    for name, A, R in forms:
        lat, its, res = [], [], []
        for k in range(nsolve + 1):
            b = torch.tensor(np.random.default_rng(5000 + k).standard_normal(N), device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, st = A.gmres(b, shift=1.0, scale=1.0 / N, rtol=rtol, restart=50, maxit=500,
                            residual=R)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if k == 0:
                continue                     # first solve allocates the Krylov workspace
            lat.append(dt)
            its.append(st["iterations"])
            res.append(st["rel_residual"])
        lat = np.array(lat)
        out[name] = {"p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
                     "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
                     "solves_per_s": round(float(len(lat) / lat.sum()), 2),
                     "iterations_median": float(np.median(its)),
                     "max_rel_residual": float(max(res))}
    return out


def bench_batched(args):
    """Batched uneven instances: the first --instances of the 512-instance
    workload (N log-uniform in [1024, 65536], 2D log r / 3D 1/r alternating,
    1 + (k mod 16) RHS, eps 1e-8, fp32, stored near field), one H2Batch."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    from paper_2309_14085_gb300 import H2Batch, H2Matrix, inputs
    inst = inputs.batched_instances(args.instances)
    t0 = time.perf_counter()
    ncpu = os.cpu_count() or 8

    def build(i):
        # large instances get more host threads; each instance goes to the device
        # at once and drops its host operators (the batch copies device to device)
        th = max(1, min(ncpu, int(ncpu * i["N"] / 65536.0) or 1))
        m = H2Matrix(i["points"], i["kernel"], leaf_size=64, tol=1e-8, storage=args.storage,
                     near="stored", threads=th, tensor_cores=args.storage == "f32")
        m.release_host()
        return m

    order = sorted(range(len(inst)), key=lambda k: -inst[k]["N"])
    mats = [None] * len(inst)
    with ThreadPoolExecutor(max(1, ncpu // 2)) as ex:
        for k, m in zip(order, ex.map(build, [inst[k] for k in order])):
            mats[k] = m
    build_s = time.perf_counter() - t0
    B = H2Batch(mats, [i["nrhs"] for i in inst])
    info = B.info()
    for m in mats:
        m.close()
    xs = [torch.tensor(i["q"], device="cuda") for i in inst]
    for _ in range(args.warmup):
        B.matvec(xs)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        B.matvec(xs)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    pts = info["points_times_rhs"]
    hbm, how = _peaks()
    # every instance's operators once per product (the bytes the method must
    # move at least; the coefficients come on top)
    ops_gbs = info["bytes_ops"] / (ms / 1e3) / 1e9
    out = {"metric": METRIC, "value": pts / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
           "config": {"workload": f"c4_batched ({args.instances} of 512 instances)",
                      "instances": args.instances, "points_times_rhs": pts,
                      "launches_per_product": info["launches_per_product"],
                      "graph": "one captured CUDA graph per batched product",
                      "host_build_seconds": round(build_s, 1),
                      "device_bytes": info["bytes_device"], "l2": "operators larger than L2"},
           "clocks": clk, "gpu_launches": info["launches_per_product"] * args.steps,
           "roofline": {"bound": "hbm", "achieved": round(ops_gbs, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(ops_gbs / hbm, 4), "traffic": None,
                        "alg_bytes": info["bytes_ops"],
                        "note": "operator bytes of all instances once per product / product time",
                        "peak_source": f"{how} hbm_gbs"},
           "tensor_cores": args.storage == "f32"}
    if args.standalone:
        print(json.dumps(out))
    return out


def bench_served(args):
    """Served RBF interpolation solves (sigma I + K) c = f, K the inverse
    multiquadric 1/sqrt(1 + (r/0.1)^2), sigma = 1e-2, on resident geometries
    (inputs.served_geometries), requests arriving as a Poisson stream.  Four
    forms on the same stream, each to the same fp64 relative residual:
      plain_fp64    one fp64 GMRES solve at a time (h2_gmres), first come first served;
      served_fp64   the continuous-batching server on the fp64 operators;
      served_df64   the server on double-float copies of the operators
                    (h2_convert; float pairs on the FP32 pipe) with fp64 residuals;
      served_f32    the server on fp32 copies with fp64 residuals; requests whose
                    shift is too small for fp32 (the server's measured rule)
                    iterate on the fp64 operator.
    value = solves/s of served_df64 over the stream (first arrival to last
    completion); latency = submit to solution on the host."""
    import queue
    import threading

    import torch

    from paper_2309_14085_gb300 import H2Matrix, H2Server, inputs
    geo = inputs.served_geometries(args.geometries)
    t0 = time.perf_counter()
    f64s = [H2Matrix(gm["points"], "imq", leaf_size=64, tol=1e-8, kparam=0.1) for gm in geo]
    f32s = [m.convert("f32") for m in f64s]
    dfs = [m.convert("df64") for m in f64s]
    build_s = time.perf_counter() - t0
    dev_bytes = sum(m.info()["bytes_device"] for m in f64s + f32s + dfs)
    arr, gid = inputs.poisson_arrivals(args.requests, args.rate, len(geo))
    sigma, rtol, restart, maxit = 1e-2, 1e-8, args.restart, 20000
    fs = [gm["f"] for gm in geo]

    def summary(lat, its, res, span, extra=None):
        lat = np.asarray(lat)
        o = {"solves_per_s": round(len(lat) / span, 3),
             "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 2),
             "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 2),
             "iterations_median": float(np.median(its)), "max_rel_residual": float(max(res)),
             "span_s": round(span, 3)}
        if extra:
            o.update(extra)
        return o

    def run_plain(arr=arr, gid=gid):
        for g, m in enumerate(f64s):          # warm-up: Krylov workspace of each geometry
            m.gmres(torch.tensor(fs[g], device="cuda"), shift=sigma, rtol=rtol, restart=restart,
                    maxit=maxit)
        torch.cuda.synchronize()
        lat, its, res = [], [], []
        start = time.perf_counter()
        for i in range(len(arr)):
            dt = start + arr[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            g = int(gid[i])
            b = torch.tensor(fs[g], device="cuda")
            x, st = f64s[g].gmres(b, shift=sigma, rtol=rtol, restart=restart, maxit=maxit)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - (start + arr[i]))
            its.append(st["iterations"])
            res.append(st["rel_residual"])
        return summary(lat, its, res, time.perf_counter() - start)

    def run_server(mats, residual, arr=arr, gid=gid):
        S = H2Server(mats, restart=restart, max_active=args.max_active, residual=residual)
        for g in range(len(mats)):            # warm-up: one request per geometry
            S.wait(S.submit(g, fs[g], shift=sigma, rtol=rtol, maxit=maxit))
        st0 = S.stats()
        q = queue.Queue()
        start = time.perf_counter()

        def submitter():
            for i in range(len(arr)):
                dt = start + arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                g = int(gid[i])
                q.put((g, S.submit(g, fs[g], shift=sigma, rtol=rtol, maxit=maxit)))

        th = threading.Thread(target=submitter)
        th.start()
        lat, its, res, qs, ops = [], [], [], [], []
        for _ in range(len(arr)):
            g, t = q.get()
            x, st = S.wait(t)
            ops.append(st["op"])
            lat.append(st["latency_seconds"])
            qs.append(st["queue_seconds"])
            its.append(st["iterations"])
            res.append(st["rel_residual"])
        span = time.perf_counter() - start
        th.join()
        st1 = S.stats()
        S.close()
        extra = {"queue_p50_ms": round(1e3 * float(np.percentile(qs, 50)), 2),
                 "max_active_seen": st1["max_active"],
                 "products": st1["products"] - st0["products"],
                 "product_columns": st1["product_columns"] - st0["product_columns"],
                 "ticks": st1["ticks"] - st0["ticks"],
                 "requests_by_operator": {"inner": ops.count(0), "fp64_by_rule": ops.count(1),
                                          "fp64_after_fallback": ops.count(2)}}
        return summary(lat, its, res, span, extra)

    forms = [f for f in args.served_forms.split(",") if f]
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    res = {}
    if "plain" in forms:
        res["plain_fp64"] = run_plain()
    if "fp64" in forms:
        res["served_fp64"] = run_server(f64s, None)
    mixed = run_server(dfs, f64s)
    res["served_df64"] = mixed
    if "f32" in forms:
        res["served_f32"] = run_server(f32s, f64s)
    if args.sub_rate > 0:
        # below saturation: latency without the queueing of the overload stream
        a2, g2 = inputs.poisson_arrivals(args.sub_requests, args.sub_rate, len(geo), seed=4998)
        res["served_df64_below_saturation"] = dict(run_server(dfs, f64s, a2, g2),
                                                    arrival_rate_per_s=args.sub_rate,
                                                    requests=args.sub_requests)
    clk = clocks.stop()
    out = {"metric": "served RBF solves/s (p50/p99 latency)", "value": mixed["solves_per_s"],
           "unit": "solves/s", "n_gpus": 1, "steps": len(arr), "warmup": len(geo),
           "ms_per_step": round(1e3 / mixed["solves_per_s"], 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "df64 operators (float pairs); f64 GMRES vectors and residuals",
           "data": "synthetic (seeded uniform points, f = sin(3 x1) cos(2 x2), Poisson arrivals)",
           "config": {"workload": "c5_served", "kernel": "inverse multiquadric, c = 0.1",
                      "sigma": sigma, "eps": 1e-8, "leaf_size": 64, "rtol": rtol,
                      "restart": restart, "max_active": args.max_active,
                      "arrival_rate_per_s": args.rate, "requests": len(arr),
                      "geometries": [{"d": gm["d"], "N": gm["N"]} for gm in geo],
                      "build_seconds": round(build_s, 1), "device_bytes": dev_bytes,
                      "l2": "operators larger than L2 (no flush)"},
           "clocks": clk}
    out.update(res)
    if args.standalone:
        print(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2_3d_invr_n262144")
    ap.add_argument("--storage", default="f64", choices=["f64", "df64", "f32", "bf16"])
    ap.add_argument("--multi-rhs", default="f32,bf16",
                    help="default workload only: also time the 64-RHS workload on the tensor "
                         "cores in these modes (comma list of f32 (3-term tf32 products of fp32 "
                         "operators), bf16; '' for none)")
    ap.add_argument("--m2l", default="device", choices=["stored", "fly", "device"],
                    help="M2L blocks: device (default: stored, formed on the device from the "
                         "pivots), stored (formed on the host and uploaded), fly (fp32: "
                         "evaluated from the pivot coordinates in each product)")
    ap.add_argument("--near", default=None, choices=["fly", "stored"],
                    help="near field: evaluated in each product (fp64: double-float arithmetic "
                         "for 1/r and the IMQ) or stored blocks; default: the storage's default")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="fp32 storage: RHS tiles of 16-64 columns on tcgen05 (tf32)")
    ap.add_argument("--variant", default="h2star", choices=list(VARIANT_NAMES))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--gmres-solves", type=int, default=10)
    ap.add_argument("--nrhs", type=int, default=0, help="override the workload's RHS count")
    ap.add_argument("--also", default="df64,f32",
                    help="other storage modes measured in the same run (comma list, '' for none)")
    ap.add_argument("--oracle-child", nargs=3, default=None)
    ap.add_argument("--reference-rows", type=int, default=256,
                    help="reference arm: exact rows of K q computed by the oracle per step")
    ap.add_argument("--instances", type=int, default=64, help="batched workload: instance count")
    ap.add_argument("--geometries", type=int, default=6, help="served workload: geometries")
    ap.add_argument("--requests", type=int, default=48, help="served workload: requests")
    ap.add_argument("--rate", type=float, default=200.0, help="served workload: arrivals per s")
    ap.add_argument("--max-active", type=int, default=16, help="served workload: active requests")
    ap.add_argument("--restart", type=int, default=1000, help="served workload: GMRES restart")
    ap.add_argument("--served-forms", default="plain,fp64,df64,f32",
                    help="served workload: forms beside the double-float server (comma list)")
    ap.add_argument("--sub-rate", type=float, default=0.0,
                    help="served workload: also a stream below saturation at this rate (req/s)")
    ap.add_argument("--sub-requests", type=int, default=12, help="requests of that stream")
    ap.add_argument("--with-batched", type=int, default=512,
                    help="default workload: also the batched workload with this many instances (0: skip)")
    ap.add_argument("--with-served", type=int, default=1,
                    help="default workload: also a bounded sample of the served workload (0: skip)")
    ap.add_argument("--with-near-fly", type=int, default=1,
                    help="default workload: also the fp64 product with the near field on the fly")
    args = ap.parse_args()
    args.standalone = False
    if args.oracle_child:
        kind, wl, arg = args.oracle_child
        if kind == "steps":
            reference_child(wl, args.reference_rows, args.warmup, args.steps)
        else:
            oracle_child(kind, wl, float(arg))
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.workload == "c5_served":
        args.standalone = True
        bench_served(args)
        return

    if args.workload == "c4_batched":
        if args.storage == "f64" and "--storage" not in sys.argv:
            args.storage = "f32"
        args.standalone = True
        bench_batched(args)
        return

    if args.impl == "reference":
        # the oracle as it stands, on this host: a step is the exact product on a
        # fixed sample of rows (--reference-rows) of the same workload, one core
        if rank != 0:
            return
        from paper_2309_14085_gb300 import inputs
        w = inputs.workload(args.workload)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", "steps",
                            args.workload, "0", "--steps", str(args.steps), "--warmup", str(args.warmup),
                            "--reference-rows", str(args.reference_rows)],
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=1800)
        if p.returncode != 0:
            raise RuntimeError("oracle child failed: " + p.stderr[-2000:])
        r = json.loads(p.stdout.strip().splitlines()[-1])
        ms = float(np.median(r["step_ms"]))
        units = args.reference_rows * w["nrhs"]
        value = units / (ms / 1e3)
        sample = (f"{args.reference_rows} exact rows of K q per step (oracle.dense.rows, dense "
                  f"definition) of the same workload, one core; median of {args.steps} steps")
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": args.workload, "N": w["N"], "d": w["d"],
                          "kernel": KERNEL_NAMES[w["kernel"]], "eps": w["eps"],
                          "rows_per_step": args.reference_rows},
               "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": sample},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out, w = bench_ours(args, rank, world)
    if args.also:
        extra = {}
        for st in [x for x in args.also.split(",") if x and x != args.storage]:
            a2 = argparse.Namespace(**vars(args))
            a2.storage = st
            a2.steps = max(3, min(args.steps, 50))
            o2, _ = bench_ours(a2, rank, world)
            args._handles = a2._handles
            r2 = o2["roofline"]
            extra[st] = {"value": o2["value"], "ms_per_step": o2["ms_per_step"],
                         "accuracy": o2.get("accuracy"),
                         "dominant": r2["kernel"], "frac": r2.get("frac"),
                         "achieved_gbs": r2.get("achieved"), "stage_ms": r2["stage_ms"],
                         "e2e": o2["e2e"]["value"], "clocks": o2["clocks"],
                         "gpu_launches": o2["gpu_launches"]}
        out["other_storage"] = extra
    if args.gmres_solves > 0:
        out["gmres"] = bench_gmres(getattr(args, "_handles", {}), w, nsolve=args.gmres_solves)
    if args.multi_rhs and args.workload == "c2_3d_invr_n262144":
        # the 64-RHS workload on the tensor cores (bf16 storage; tf32 for fp32)
        mr = {"workload": "c3_2d_log_n1048576", "nrhs": 64}
        for mode in [m for m in args.multi_rhs.split(",") if m]:
            a3 = argparse.Namespace(**vars(args))
            a3.workload, a3.nrhs, a3.steps = "c3_2d_log_n1048576", 0, 20
            a3.storage, a3.tensor_cores = ("bf16", False) if mode == "bf16" else ("f32", True)
            a3.also = ""
            a3._handles = {}
            try:
                o3, _ = bench_ours(a3, rank, world)
                r3 = o3["roofline"]
                acc = o3.get("accuracy")
                mr[mode] = {"value": o3["value"], "unit": UNIT, "ms_per_step": o3["ms_per_step"],
                            "accuracy": acc,
                            # a product whose sampled rows are off by more than 1 % carries no
                            # usable digits as an MVP (bf16 operators at eps 1e-10, 2D log r):
                            # such a mode serves as the inner operator of iterative refinement
                            "usable_as_mvp": bool(acc is not None and acc["re_vs_exact"] <= 1e-2),
                            "e2e": o3["e2e"]["value"], "dominant": r3["kernel"],
                            "frac": r3.get("frac"), "achieved_gbs": r3.get("achieved"),
                            "stage_ms": r3["stage_ms"], "clocks": o3["clocks"],
                            "gpu_launches": o3["gpu_launches"],
                            "tc_persistent_ctas": o3["config"]["tc_persistent_ctas"],
                            "build_seconds": o3["config"]["build_seconds"]}
            except Exception as e:              # report, do not lose the main line
                mr[mode] = {"error": str(e)[:300]}
            a3._handles = {}
        out["multi_rhs_tensor_cores"] = mr
    default = args.workload == "c2_3d_invr_n262144"
    if default and args.with_near_fly and args.storage == "f64":
        # the same fp64 product with the near field evaluated in double-float
        # arithmetic instead of streamed (2.3 GB less on the device)
        a6 = argparse.Namespace(**vars(args))
        a6.near, a6.steps, a6._handles = "fly", max(3, min(args.steps, 20)), {}
        o6, _ = bench_ours(a6, rank, world)
        r6 = o6["roofline"]
        out["near_on_the_fly"] = {"value": o6["value"], "ms_per_step": o6["ms_per_step"],
                                  "stage_ms": r6["stage_ms"], "m2l_frac": r6.get("frac"),
                                  "whole_mvp": r6.get("whole_mvp"),
                                  "device_bytes": o6["config"]["device_bytes"],
                                  "accuracy": o6.get("accuracy"), "clocks": o6["clocks"],
                                  "gpu_launches": o6["gpu_launches"]}
        for m in a6._handles.values():
            m.close()
    for m in getattr(args, "_handles", {}).values():
        m.close()
    args._handles = {}
    if default and args.with_batched > 0 and world == 1:
        import torch
        torch.cuda.empty_cache()
        a4 = argparse.Namespace(**vars(args))
        a4.instances, a4.storage, a4.steps, a4.warmup, a4.standalone = args.with_batched, "f32", 10, 3, False
        o4 = bench_batched(a4)
        out["batched"] = {k: o4[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "roofline",
                                             "gpu_launches", "clocks", "tensor_cores")}
    if default and args.with_served and world == 1:
        import torch
        torch.cuda.empty_cache()
        a5 = argparse.Namespace(**vars(args))
        a5.geometries, a5.requests, a5.rate, a5.served_forms = 4, 32, 200.0, "plain"
        a5.sub_rate, a5.sub_requests, a5.standalone = 1.0, 12, False
        o5 = bench_served(a5)
        out["served"] = {k: v for k, v in o5.items()
                         if k not in ("metric", "n_gpus", "warmup", "higher_is_better", "scaling",
                                      "vs_baseline", "data")}
    if rank == 0:
        out["cpu_baseline"] = cpu_baselines(args.workload, args.cpu_seconds)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
