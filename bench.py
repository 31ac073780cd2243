"""Benchmark: contraction throughput of the partitioned tensor-network engine on one GB300.

Workload (one "step"): a batch of B single amplitudes <x|C|0^n> of one 24-qubit 1D brickwork
circuit of depth 14 (seed 2), each a closed network of 569 tensors split into k = 4 partitions by
the simulated-annealing planner (DIRECTED targets, 2000 temperature iterations, seed 7, qubit-block
initial partition), with B distinct random bitstrings x.  All B contractions -- every partition's
steps and the fan-in -- run in one persistent dataflow launch, complex64 arithmetic with the FP64
final reduction.

  value  contraction TFLOP/s = (B * 8 * con_serial) / device time of the timed steps, inputs
         resident in HBM (con_serial is the plan's exact Eq. 3.2 count: 8 real flops per complex
         multiply-add).
  e2e    the same metric through the C ABI with host buffers: each step uploads the B networks'
         leaves (new bitstrings every step) from pinned host memory and reads the B results back.
  roofline  the persistent kernel against the measured HBM copy bandwidth.
  cpu_baseline / --impl reference  the oracle (complex128 C contractor) on the host cores.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contraction TFLOP/s, % roofline; amps/s, p99 latency vs plain c64 at err<=1e-4"
N_QUBITS, DEPTH, K_PARTS = 24, 14, 4
PLAN_ITERS, PLAN_SEED = 2000, 7


PRECISION_NAMES = {"c64": "complex64, FP64 final reduction",
                   "bf16": "BF16 hi/lo split on tcgen05 for dense steps (FP32 accumulation), complex64 storage, "
                           "FP64 final reduction",
                   "tf32": "TF32 hi/lo split on tcgen05 for dense steps (FP32 accumulation), complex64 storage, "
                           "FP64 final reduction",
                   "c128": "complex128"}
# relative error bound asserted against the oracle, per precision
PRECISION_TOL = {"c64": 1e-5, "tf32": 1e-5, "bf16": 1e-4, "c128": 1e-12}


def workload_config(batch, precision="c64"):
    return {"workload": f"24-qubit 1D brickwork depth {DEPTH} (seed 2), single amplitudes, "
                        f"k={K_PARTS} SA partitions (directed, {PLAN_ITERS} iterations, seed {PLAN_SEED}), "
                        f"batch of {batch} bitstrings per step",
            "n_qubits": N_QUBITS, "depth": DEPTH, "k": K_PARTS, "batch": batch,
            "precision": PRECISION_NAMES.get(precision, precision),
            "l2": "per-step working set larger than the 129 MB L2 (no flush needed)"}


def make_workload(batch, seed0=5000):
    from paper_2507_20667_gb300 import inputs as tni
    circ = tni.brickwork_1d(N_QUBITS, DEPTH, seed=2)
    xs = [tni.random_bitstring(N_QUBITS, seed0 + i) for i in range(batch)]
    nets = [tni.amplitude_tn(circ, x) for x in xs]
    return circ, xs, nets


def plan_for(tnsa, tni, net_py, net_h):
    return tnsa.tn_plan_create(net_h, k=K_PARTS, mode="directed", iterations=PLAN_ITERS, steps_per_temp=8,
                               seed=PLAN_SEED,
                               position=net_py.qubit)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    """Host cores available to this process (what nproc prints)."""
    try:
        return int(subprocess.run(["nproc"], capture_output=True, text=True, check=True).stdout.strip())
    except (OSError, ValueError, subprocess.CalledProcessError):
        return len(os.sched_getaffinity(0))


def kernel_sources_sha():
    """Hash of the engine's kernel and runtime sources: DRAM-traffic counters taken from ncu stay
    valid only while it is unchanged."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_20667_gb300", "csrc")
    for p in sorted(glob.glob(os.path.join(csrc, "*"))):
        if p.endswith((".cu", ".cuh", ".cpp", ".hpp")):
            with open(p, "rb") as f:
                h.update(os.path.basename(p).encode() + f.read())
    return h.hexdigest()[:16]


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the three contraction kernels of one
# run of the headline workload (k_warp 195.8 MB + k_local 321.9 MB + k_persist 3736.1 MB per
# launch, mean of two runs), from one ncu capture of `bench.py` at the default batch
# (profiles/traffic_brickwork24_batch2432.md); valid for the kernel sources with this hash.
TRAFFIC = {"sources_sha": "41dac86b20f80667", "batch": 2432, "bytes_per_run": 4253917056}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def oracle_tree(net):
    """The oracle's own contraction tree (its Greedy rule over the whole network) and that tree's
    exact con_serial (Eq. 3.2, big integers)."""
    from oracle import costs as ocost
    from oracle import greedy as og
    steps = og.greedy_steps(list(ocost.leaf_legs(net)), ocost.edge_dims(net))
    return steps, ocost.Tree(net, steps).con_serial()


def oracle_rate(nets, tree, budget_s, min_amps=1):
    """Whole amplitudes per second of the oracle's complex128 C contractor along `tree` on the
    host cores, over nets[0], nets[1], ... until the time budget is used."""
    from oracle import contract as oc
    t0 = time.perf_counter()
    done = 0
    while done < min_amps or (time.perf_counter() - t0 < budget_s and done < len(nets)):
        oc.contract_scalar(nets[done % len(nets)], tree)
        done += 1
    dt = time.perf_counter() - t0
    return done, dt


def oracle_sample(nets, plan_tree, plan_con_serial, budget_s=12.0):
    """The oracle as it stands on the host cores, on whole amplitudes of the same workload: along
    the engine's own simulated-annealing tree (the same tree the GPU contracts), and along the
    oracle's own serial Greedy tree."""
    cores = host_cores()
    done, dt = oracle_rate(nets, plan_tree, 0.75 * budget_s)
    own_tree, own_con = oracle_tree(nets[0])
    done2, dt2 = oracle_rate(nets, own_tree, 0.25 * budget_s)
    return {"value": done * 8 * plan_con_serial / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} whole amplitudes of the step's workload along the same SA tree as the GPU "
                      f"(con_serial {plan_con_serial}), complex128 C contractor, {dt:.1f} s",
            "amps_per_s": done / dt,
            "oracle_own_greedy_tree": {"amps_per_s": done2 / dt2, "con_serial": own_con,
                                       "tflops": done2 * 8 * own_con / dt2 / 1e12, "amplitudes": done2}}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, ws, device="cuda"):
    """Maximum of `value` over the ranks (the slowest rank's time); no-op for one rank."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, local_seconds, ws, device="cuda"):
    """Whole-job throughput of N independent replicas: all ranks' units over the slowest rank's
    time (max over ranks).  Returns (value, max_seconds)."""
    t = reduce_max(local_seconds, ws, device)
    return ws * units_per_rank / t, t


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args):
    """--impl reference: the oracle, unmodified, on the host cores (rank 0 only)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    circ, xs, nets = make_workload(max(args.steps + args.warmup, 1))
    # the tree: the configuration's simulated-annealing plan (the library's host planner, exported),
    # the same tree the GPU arm contracts; the oracle contracts along it
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa
    h = tnsa.tn_build(nets[0])
    plan = plan_for(tnsa, tni, nets[0], h)
    con_serial = tnsa.tn_plan_counts(plan)[0]
    part, psteps, _ = tnsa.tn_plan_export(plan, nets[0].n_tensors)
    tree = [(int(l), int(r)) for l, r, o in psteps]
    from oracle import contract as oc
    for i in range(args.warmup):
        oc.contract_scalar(nets[i], tree)
    t0 = time.perf_counter()
    for i in range(args.steps):  # one step = one whole amplitude (a bounded sample of the batch)
        oc.contract_scalar(nets[args.warmup + i], tree)
    dt = time.perf_counter() - t0
    value = args.steps * 8 * con_serial / dt / 1e12
    cores = host_cores()
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": workload_config(args.batch), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} whole amplitudes, one per step, complex128 C contractor "
                                       f"along the configuration's SA tree (con_serial {con_serial})"},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "amps_per_s": args.steps / dt}
    print(json.dumps(line), flush=True)


def other_configs(args, tnsa, tni, budget_s=4.0):
    """cfg1 (10-qubit brickwork depth 8, k = 1 Greedy tree) and the 4x5 depth-8 grid instance of
    cfg3 (k = 8 SA partitions): a GPU batch (complex64, CUDA events) against the oracle on the
    host cores along the same tree, with the largest plain relative error of the GPU amplitudes
    against the oracle over a sample."""
    import torch
    from oracle import contract as oc
    out = {}
    for name, (circ, x0), k in (("cfg1_brickwork10_d8", tni.cfg1(), 1), ("cfg3_grid4x5_d8", tni.cfg3(small=True), 8)):
        n = circ.n_qubits
        B = 512
        nets = [tni.amplitude_tn(circ, tni.random_bitstring(n, 8000 + i)) for i in range(B)]
        hs = [tnsa.tn_build(t) for t in nets]
        plan = tnsa.tn_plan_create(hs[0], k=k, iterations=200 if k > 1 else 0, steps_per_temp=8, seed=7,
                                   position=nets[0].qubit if k > 1 else None)
        con_serial = tnsa.tn_plan_counts(plan)[0]
        ctx = tnsa.tn_ctx_create(0)
        b = tnsa.tn_batch_create(ctx, hs, [plan] * B, "c64")
        for _ in range(3):
            tnsa.tn_batch_run(b)
        reps = 10
        for _ in range(reps):
            tnsa.tn_batch_run(b)
        ms = tnsa.tn_batch_kernel_ms(b, reps)
        mant, e2, st = tnsa.tn_batch_results(b, B)
        part, psteps, _ = tnsa.tn_plan_export(plan, nets[0].n_tensors)
        tree = [(int(l), int(r)) for l, r, o in psteps]
        done, dt = oracle_rate(nets, tree, budget_s)
        errs, mags = [], []
        for i in range(min(done, B)):
            ref = oc.contract_scalar(nets[i], tree)
            got = complex(mant[i]) * 2.0 ** int(e2[i])
            errs.append(abs(got - ref) / abs(ref))
            mags.append(abs(ref) * 2.0 ** (n / 2))
        # The parity tests' rule: an amplitude below 1e-3 of the typical 2^(-n/2) is not compared
        # by relative error (it would be redrawn there); it is counted here instead.
        kept = [e for e, m in zip(errs, mags) if m >= 1e-3]
        over = [m for e, m in zip(errs, mags) if e > 1e-5]
        b.close()
        ctx.close()
        out[name] = {"batch": B, "gpu_amps_per_s": B / (ms * 1e-3), "gpu_tflops": B * 8 * con_serial / ms / 1e9,
                     "oracle_amps_per_s": done / dt, "oracle_cores": host_cores(), "oracle_amplitudes": done,
                     "max_rel_err_c64_vs_oracle": max(kept) if kept else None, "compared": len(kept),
                     "below_1e-3_typical": len(errs) - len(kept),
                     "max_rel_err_including_those": max(errs) if errs else None,
                     "over_1e-5": len(over), "largest_|a|*2^(n/2)_over_1e-5": max(over) if over else None,
                     "con_serial": con_serial}
    return out


def run_ours(args):
    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa

    B = args.batch
    circ, xs, nets = make_workload(B, seed0=5000 + 100000 * rank)
    handles = [tnsa.tn_build(n) for n in nets]
    plan = plan_for(tnsa, tni, nets[0], handles[0])
    con_serial, con_dist, mem = tnsa.tn_plan_counts(plan)
    stream = torch.cuda.Stream()
    ctx = tnsa.tn_ctx_create(local, stream=stream.cuda_stream)
    tuning = None
    if not args.no_autotune:
        # untimed setup: the library's autotuner times its candidate configurations on this batch
        best, best_ms, cand = tnsa.tn_ctx_autotune(ctx, handles, [plan] * B, args.precision, runs=5)
        tuning = {"config": best, "ms_per_run": best_ms, "candidates_ms": cand}
    batch = tnsa.tn_batch_create(ctx, handles, [plan] * B, args.precision)
    info = tnsa.tn_batch_last_info(batch)
    flops_per_step = B * 8.0 * con_serial
    bytes_per_step = info["bytes"]  # algorithmic bytes of all B contractions

    # parity spot check of the timed configuration: a few jobs against the oracle
    tnsa.tn_batch_run(batch)
    mant, e2, st = tnsa.tn_batch_results(batch, B)
    assert (st == 0).all(), "a device wait timed out"
    if rank == 0 and not args.skip_check:
        from oracle import contract as oc
        part, steps, _ = tnsa.tn_plan_export(plan, nets[0].n_tensors)
        tree = [(int(l), int(r)) for l, r, o in steps]
        for i in sorted({0, B // 2, B - 1}):
            ref = oc.contract_scalar(nets[i], tree)
            got = complex(mant[i]) * 2.0 ** int(e2[i])
            err = abs(got - ref) / abs(ref)
            assert err <= PRECISION_TOL[args.precision], f"job {i}: relative error {err:.2e}"

    # device-resident timing: K steps bracketed by barrier + synchronize, CUDA events on the stream
    for _ in range(args.warmup):
        tnsa.tn_batch_run(batch)
    torch.cuda.synchronize()
    barrier(ws)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            tnsa.tn_batch_run(batch)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms = ev0.elapsed_time(ev1)
    kernel_ms = tnsa.tn_batch_kernel_ms(batch, min(args.steps, 256))
    class_ms = tnsa.tn_batch_kernel_times(batch, min(args.steps, 256))
    value, sec = replica_throughput(args.steps * flops_per_step / 1e12, ms * 1e-3, ws)
    ms_per_step = 1e3 * sec / args.steps

    # end to end through the C ABI with host buffers: every step B new bitstrings are written into
    # pinned host memory, copied to the device with the step, and the B results are read back
    n = N_QUBITS
    n_t = nets[0].n_tensors
    rng = np.random.default_rng(77 + rank)
    e2e_steps = max(1, min(args.steps, 20))
    jobs = np.repeat(np.arange(B, dtype=np.int32), n)
    tensors = np.tile(np.arange(n_t - n, n_t, dtype=np.int32), B)
    eye = np.eye(2, dtype=np.complex128)
    h2d = 0
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    # the host draws and stages step s + 1's bitstrings while the device runs step s (the staged
    # values reach the device in step s + 1's own copy)
    tnsa.tn_batch_set_tensors(batch, jobs, tensors, eye[rng.integers(0, 2, B * n)])
    for s in range(e2e_steps):
        tnsa.tn_batch_run(batch)
        if s + 1 < e2e_steps:
            tnsa.tn_batch_set_tensors(batch, jobs, tensors, eye[rng.integers(0, 2, B * n)])
        m2, ee, st2 = tnsa.tn_batch_results(batch, B)
    dt = reduce_max(time.perf_counter() - t0, ws)
    h2d = tnsa.tn_batch_last_info(batch)["h2d_bytes"]   # bytes copied to the device by the last step
    e2e_value = ws * e2e_steps * flops_per_step / dt / 1e12
    d2h = 32 * B

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_step / (kernel_ms * 1e-3) / 1e9
    sha = kernel_sources_sha()
    traffic = (TRAFFIC["bytes_per_run"] * B / TRAFFIC["batch"]
               if TRAFFIC["bytes_per_run"] and TRAFFIC["sources_sha"] == sha else None)
    per_kernel = {}
    for cls, key in (("warp_programs", "bytes_warp"), ("block_programs", "bytes_block"), ("tc_gemm", "bytes_tc"),
                     ("dataflow", "bytes_flow")):
        t = class_ms[cls]
        per_kernel[cls] = {"ms": t, "algorithmic_bytes": info[key],
                           "achieved_gbs": info[key] / (t * 1e-3) / 1e9 if t > 0 and info[key] > 0 else None}
    cpu = None
    if not args.skip_cpu:
        part, psteps, _ = tnsa.tn_plan_export(plan, nets[0].n_tensors)
        cpu = oracle_sample(nets, [(int(l), int(r)) for l, r, o in psteps], con_serial, budget_s=args.cpu_seconds)
    others = other_configs(args, tnsa, tni) if not args.skip_cpu else None
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision if args.precision != "bf16" else "bf16-split",
            "data": "synthetic", "config": workload_config(B, args.precision),
            "amps_per_s": ws * B / (ms_per_step * 1e-3),
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
                    "amps_per_s": ws * e2e_steps * B / dt, "steps": e2e_steps},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "contraction kernels of one run (k_warp warp programs, k_local block "
                                   "programs, k_persist dataflow steps), events around all of them",
                         "kernel_ms": kernel_ms, "peak_kind": f"{peak_kind} hbm_gbs", "sources_sha": sha,
                         "per_kernel": per_kernel},
            "gpu_launches": info["launches"] * args.steps,
            "exec": {"warp_programs": info["n_warp_progs"], "block_programs": info["n_local"],
                     "steps_in_programs": info["n_local_steps"],
                     "dyn_smem": info["dyn_smem"], "global_rows": info["n_gather"], "global_tile": info["n_tile"],
                     "global_dot": info["n_dot"]},
            "clocks": clocks.summary(),
            "plan": {"con_serial": con_serial, "con_dist": con_dist, "mem": mem},
            "tuning": tuning,
            "cpu_baseline": cpu,
            "other_configs": others}
    print(json.dumps(line), flush=True)


def _amp_model(tnsa, tni, circ, k, seed, iters):
    net = tni.amplitude_tn(circ, [0] * circ.n_qubits)
    h = tnsa.tn_build(net)
    pos = net.qubit if k > 1 else None
    plan = tnsa.tn_plan_create(h, k=k, iterations=iters, steps_per_temp=8, seed=seed, position=pos)
    return net, h, plan, tni.bra_ids(net, circ.n_qubits)


def _percentiles(lat):
    if not lat:
        return None, None
    a = np.sort(np.asarray(lat))
    return float(a[int(0.5 * (len(a) - 1))]), float(a[int(0.99 * (len(a) - 1))])


TOL = {"c128": 1e-12, "c64": 1e-5, "tf32": 1e-5, "bf16": 1e-4}


def _oracle_errors(tnsa, models, results, max_n=24, per_model=2, budget_s=60.0, prec=None):
    """Largest plain relative error of GPU amplitudes against the oracle (complex128 C contractor
    along the same plan tree), over up to `per_model` results of every model with at most `max_n`
    qubits, with the magnitude of the worst amplitude relative to the typical 2^(-n/2) and the
    number of results above the precision's bound.  results: list of (model index, bits or tensor
    data, complex amplitude)."""
    from oracle import contract as oc
    seen, errs, small, t0 = {}, [], 0, time.perf_counter()
    for mi, data, amp in results:
        net, h, plan, bras, nq = models[mi]
        if nq > max_n or seen.get(mi, 0) >= per_model or time.perf_counter() - t0 > budget_s:
            continue
        seen[mi] = seen.get(mi, 0) + 1
        part, psteps, _ = tnsa.tn_plan_export(plan, net.n_tensors)
        tree = [(int(l), int(r)) for l, r, o in psteps]
        class Q:
            pass
        q = Q()
        q.degrees, q.dims, q.edges = net.degrees, net.dims, net.edges
        d = np.asarray(net.data, np.float64).copy().view(np.complex128)
        for t, v in zip(bras, data):
            off = int(np.sum([np.prod(net.tensors[u].shape) for u in range(t)]))
            d[off:off + len(v)] = v
        q.data = d.view(np.float64)
        ref = oc.contract_scalar(q, tree)
        if abs(ref) < 1e-3 * 2.0 ** (-nq / 2):   # the parity tests redraw such a bitstring
            small += 1
            continue
        errs.append((abs(amp - ref) / abs(ref), nq, abs(ref) * 2.0 ** (nq / 2)))
    out = {"max_rel_err": max(errs)[0] if errs else None, "compared": len(errs),
           "below_1e-3_typical": small, "circuits_compared": len(seen), "max_qubits": max_n}
    if errs:
        w = max(errs)
        out["worst"] = {"n_qubits": w[1], "abs_amp_over_typical": w[2]}
    if prec is not None:
        out["bound"] = TOL[prec]
        out["over_bound"] = [{"rel_err": e, "n_qubits": q, "abs_amp_over_typical": m}
                             for e, q, m in sorted(errs, reverse=True) if e > TOL[prec]]
    return out


def run_cfg4(args):
    """Amplitude queries over 32 seeded circuits (16-36 qubits, depth 8-16, 1D and 2D, k in
    {2, 4, 8}; 16 bitstrings each, 512 queries): every feasible query in one grouped batch (all
    jobs' steps in the persistent launches of one recorded CUDA graph), BF16 split and complex64;
    the same queries through the batching server; and one query at a time through tn_contract in
    complex64.  Errors against the oracle for the circuits of at most 24 qubits."""
    import torch
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa
    ctx = tnsa.tn_ctx_create(0)
    free = torch.cuda.mem_get_info()[0]
    budget = min(int(0.6 * free), 150 << 30)
    models, reqs = [], []
    t0 = time.perf_counter()
    for i, (circ, k, xs) in enumerate(tni.cfg4_circuits()):
        net, h, plan, bras = _amp_model(tnsa, tni, circ, k, seed=7, iters=args.plan_iters)
        models.append((net, h, plan, bras, circ.n_qubits))
        for x in xs[:args.queries_per_circuit]:
            reqs.append((i, np.eye(2, dtype=np.complex128)[np.asarray(x)]))
    plan_s = time.perf_counter() - t0
    # per-query device bytes of each model (a server of the same context compiles it)
    probe = tnsa.tn_serve_create(ctx, "bf16", hbm_budget_bytes=budget, max_batch=1)
    job_bytes = [tnsa.tn_serve_model_info(probe, tnsa.tn_serve_register(probe, m[1], m[2]))[0] for m in models]
    flops_of = [tnsa.tn_serve_model_info(probe, mi)[1] for mi in range(len(models))]
    probe.close()
    # every query whose job fits the budget on its own runs; the queries are grouped, in order of
    # their per-job bytes, into as few batches as the budget allows (each batch one graph replay)
    chosen = [qi for qi, (mi, data) in enumerate(reqs) if 2 * job_bytes[mi] <= budget]
    refused = len(reqs) - len(chosen)
    chosen.sort(key=lambda qi: (job_bytes[reqs[qi][0]], qi))
    groups, cur, used = [], [], 0
    for qi in chosen:
        jb = 2 * job_bytes[reqs[qi][0]]
        if cur and used + jb > budget:
            groups.append(cur)
            cur, used = [], 0
        cur.append(qi)
        used += jb
    if cur:
        groups.append(cur)
    out = {}
    for prec in ("bf16", "c64"):
        total_ms, results, n_tc, launches = 0.0, [], 0, 0
        for grp in groups:
            hs = []
            for qi in grp:
                mi, data = reqs[qi]
                h = tnsa.tn_build(models[mi][0])
                for t, v in zip(models[mi][3], data):
                    tnsa.tn_net_set_tensor(h, t, v)
                hs.append(h)
            plans = [models[reqs[qi][0]][2] for qi in grp]
            b = tnsa.tn_batch_create(ctx, hs, plans, prec)
            tnsa.tn_batch_run(b)
            tnsa.tn_batch_results(b, len(hs))
            reps = 2
            for _ in range(reps):
                tnsa.tn_batch_run(b)
            total_ms += tnsa.tn_batch_kernel_ms(b, reps)
            mant, e2, st = tnsa.tn_batch_results(b, len(hs))
            info = tnsa.tn_batch_last_info(b)
            n_tc += info["n_tc"]
            launches += info["launches"]
            results += [(reqs[qi][0], reqs[qi][1], complex(mant[j]) * 2.0 ** int(e2[j]))
                        for j, qi in enumerate(grp) if st[j] == 0]
            b.close()
        fl = sum(flops_of[reqs[qi][0]] for qi in chosen)
        out[prec] = {"queries": len(chosen), "batches": len(groups), "ms_all_batches": total_ms,
                     "amps_per_s": len(chosen) / (total_ms * 1e-3), "tflops": fl / total_ms / 1e9,
                     "launches_per_run": launches, "graph_replay": True, "tensor_core_steps": n_tc,
                     "error_vs_oracle": _oracle_errors(tnsa, models, results, prec=prec)}
    # the same queries through the batching server (continuous batching, memory admission)
    srv = {}
    for prec in ("bf16", "c64"):
        server = tnsa.tn_serve_create(ctx, prec, hbm_budget_bytes=budget, max_batch=args.max_batch)
        mids = [tnsa.tn_serve_register(server, m[1], m[2]) for m in models]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [(qi, tnsa.tn_serve_submit(server, mids[reqs[qi][0]], models[reqs[qi][0]][3], reqs[qi][1]))
                   for qi in chosen]
        done = []
        for qi, tk in tickets:
            mant, e, lat = tnsa.tn_serve_poll(server, tk, timeout_s=600.0)
            done.append((reqs[qi][0], reqs[qi][1], complex(mant) * 2.0 ** e))
        dt = time.perf_counter() - t0
        st = tnsa.tn_serve_get_stats(server)
        srv[prec] = {"queries": len(done), "amps_per_s": len(done) / dt, "seconds": dt, "launches": st["launches"],
                     "mean_batch": st["launched_requests"] / max(st["launches"], 1),
                     "error_vs_oracle": _oracle_errors(tnsa, models, done, prec=prec)}
        server.close()
    # one query at a time, complex64, through tn_contract (each query its own launches)
    t0 = time.perf_counter()
    single = []
    for qi in sorted(chosen):   # in submission order (circuit by circuit)
        mi, data = reqs[qi]
        net, h, plan, bras, nq = models[mi]
        for q, t in enumerate(bras):
            tnsa.tn_net_set_tensor(h, t, data[q])
        m, e, _ = tnsa.tn_contract(ctx, h, plan, "c64")
        single.append((mi, data, complex(m) * 2.0 ** e))
    single_dt = time.perf_counter() - t0
    line = {"metric": METRIC, "value": out["bf16"]["amps_per_s"], "unit": "amps/s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16-split", "data": "synthetic",
            "config": {"workload": f"{len(reqs)} amplitude queries over 32 seeded circuits (16-36 qubits, depth "
                                   f"8-16, 1D/2D, k in {{2,4,8}}), {args.queries_per_circuit} per circuit; "
                                   f"{len(chosen)} feasible in {len(groups)} grouped batches under "
                                   f"{budget / 2**30:.0f} GiB, {refused} refused (one job above the budget)",
                       "queries_requested": len(reqs), "queries_run": len(chosen), "queries_refused": refused,
                       "plan_iterations": args.plan_iters, "planning_seconds": plan_s},
            "grouped_batch_bf16": out["bf16"], "grouped_batch_c64": out["c64"],
            "server_bf16": srv["bf16"], "server_c64": srv["c64"],
            "one_at_a_time_c64": {"amps_per_s": len(single) / single_dt, "seconds": single_dt, "queries": len(single),
                                  "error_vs_oracle": _oracle_errors(tnsa, models, single, prec="c64")},
            "speedup_grouped_bf16_vs_one_at_a_time_c64": out["bf16"]["amps_per_s"] / (len(single) / single_dt)}
    print(json.dumps(line), flush=True)


def run_cfg5(args):
    """Poisson arrivals (rate args.rate per s) of amplitude and <Z_i Z_j> requests on a pool of
    seeded circuits of 12-48 qubits, depth 8-20, 1D and 2D, admitted under a device-memory budget;
    p50 / p99 latency and throughput, split-BF16 against plain complex64."""
    import torch
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa
    ctx = tnsa.tn_ctx_create(0)
    free = torch.cuda.mem_get_info()[0]
    budget = min(int(0.7 * free), 150 << 30)
    rng = np.random.default_rng(5)
    pool = []
    t0 = time.perf_counter()
    for i in range(args.pool):
        n = int(rng.integers(12, 49))
        depth = int(rng.integers(8, 21))
        if rng.integers(0, 2):
            rows = int(math.floor(math.sqrt(n)))
            circ = tni.grid_2d(rows, int(round(n / rows)), depth, seed=500 + i)
        else:
            circ = tni.brickwork_1d(n, depth, seed=500 + i)
        nq = circ.n_qubits
        try:   # a plan above 2^120 operations is infeasible: its requests count as refused
            amp = _amp_model(tnsa, tni, circ, 4, seed=7, iters=args.plan_iters)
        except tnsa.TnError:
            amp = None
        znet, slots = tni.zz_slots_tn(circ)
        zh = tnsa.tn_build(znet)
        try:
            zplan = tnsa.tn_plan_create(zh, k=4, iterations=args.plan_iters, seed=7,
                                        position=znet.qubit)
            zz = (znet, zh, zplan, slots)
        except tnsa.TnError:
            zz = None
        pool.append((circ, amp, zz))
    plan_s = time.perf_counter() - t0
    models = []   # (net, handle, plan, bra or slot ids, n_qubits) as _oracle_errors expects

    def stream(prec, rate, duration, warmup_s, seed):
        server = tnsa.tn_serve_create(ctx, prec, hbm_budget_bytes=budget, max_batch=args.max_batch)
        ids = []
        for circ, amp, zz in pool:
            ids.append((tnsa.tn_serve_register(server, amp[1], amp[2]) if amp else None,
                        tnsa.tn_serve_register(server, zz[1], zz[2]) if zz else None))
        arr = np.random.default_rng(seed)
        sent = []
        unplannable = [0]

        def client():
            t_end = time.perf_counter() + warmup_s + duration
            while time.perf_counter() < t_end:
                time.sleep(arr.exponential(1.0 / rate))
                c = int(arr.integers(0, len(pool)))
                circ, amp, zz = pool[c]
                nq = circ.n_qubits
                if arr.random() < 0.5:
                    bits = arr.integers(0, 2, nq)
                    if ids[c][0] is None:
                        unplannable[0] += 1
                        continue
                    data = np.eye(2, dtype=np.complex128)[bits]
                    tk = tnsa.tn_serve_submit(server, ids[c][0], amp[3], data)
                    sent.append((time.perf_counter(), tk, ("amp", c, data)))
                else:
                    i, j = arr.choice(nq, 2, replace=False)
                    if ids[c][1] is None:
                        unplannable[0] += 1
                        continue
                    data = np.array([tni.Z_MAT if q in (i, j) else np.eye(2) for q in range(nq)], np.complex128)
                    tk = tnsa.tn_serve_submit(server, ids[c][1], zz[3], data)
                    sent.append((time.perf_counter(), tk, ("zz", c, (int(i), int(j)))))

        import threading
        th = threading.Thread(target=client)
        t_start = time.perf_counter()
        th.start()
        th.join()
        # drain: poll until every request completed or the drain deadline passed; a request still
        # open then has a latency of at least its wait so far (censored)
        t_stream_end = time.perf_counter()
        deadline = t_stream_end + args.drain_s
        lat, rejected, done, results, open_, t_last = [], 0, 0, [], 0, t_stream_end
        for ts, tk, what in sent:
            try:
                r = tnsa.tn_serve_poll(server, tk, timeout_s=max(0.0, deadline - time.perf_counter()))
            except tnsa.TnError as e:
                if e.status != tnsa.TN_EBUDGET:
                    raise
                rejected += 1
                continue
            if r is None:
                open_ += 1
                if ts - t_start >= warmup_s:
                    lat.append(float("inf"))
                continue
            t_last = time.perf_counter()
            if ts - t_start >= warmup_s:
                lat.append(r[2])
            done += 1
            results.append((what, complex(r[0]) * 2.0 ** r[1]))
        t_total = t_last - t_start
        st = tnsa.tn_serve_get_stats(server)
        server.close()
        p50, p99 = _percentiles(lat)
        fmt = lambda p: None if p is None else (1e3 * p if math.isfinite(p) else
                                                f"> {1e3 * (deadline - t_start):.0f} (censored at the drain deadline)")
        return {"rate_per_s": rate, "duration_s": duration, "requests": len(sent) + unplannable[0],
                "completed": done, "open_at_deadline": open_, "rejected_over_budget": rejected,
                "refused_plan_above_2e120": unplannable[0],
                "p50_ms": fmt(p50), "p99_ms": fmt(p99),
                "amps_per_s": done / max(t_total, 1e-9), "launches": st["launches"],
                "mean_batch": st["launched_requests"] / max(st["launches"], 1),
                "max_in_flight": st["max_in_flight"]}, results

    def errors(results, prec):
        """Amplitudes of circuits of at most 24 qubits against the oracle along the same plan;
        <Z_i Z_j> of circuits of at most 16 qubits against the state vector (error on the
        scale ||Z_i Z_j|| = 1)."""
        from oracle import statevector as sv
        amp_res, zz_errs, seen = [], [], {}
        for what, val in results:
            kind, c, data = what
            circ, amp, zz = pool[c]
            if kind == "amp" and amp is not None:
                if c not in seen:
                    seen[c] = len(models)
                    models.append((amp[0], amp[1], amp[2], amp[3], circ.n_qubits))
                amp_res.append((seen[c], data, val))
            elif kind == "zz" and circ.n_qubits <= 16 and len(zz_errs) < 40:
                zz_errs.append(abs(val - sv.zz_expectation(circ, *data)))
        e = _oracle_errors(tnsa, models, amp_res, per_model=2, budget_s=60.0, prec=prec)
        e["zz_max_abs_err"] = max(zz_errs) if zz_errs else None
        e["zz_compared"] = len(zz_errs)
        return e

    res = {}
    for prec in ("c64", "bf16"):
        r, results = stream(prec, args.rate, args.duration, args.warmup_s, 55)
        r["error_vs_oracle"] = errors(results, prec)
        # service latency without queueing: a stream at 80 % of the throughput the loaded run
        # sustained (the requested rate, if that is lower)
        sustain = max(0.5, min(args.rate, 0.8 * r["amps_per_s"]))
        r2, _ = stream(prec, sustain, min(args.duration, 20.0), min(args.warmup_s, 3.0), 56)
        r["at_sustainable_rate"] = r2
        res[prec] = r
    line = {"metric": METRIC, "value": res["bf16"]["amps_per_s"], "unit": "amps/s", "n_gpus": 1, "steps": 1,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split",
            "data": "synthetic",
            "config": {"workload": f"serving: Poisson {args.rate}/s amplitude and <Z_i Z_j> requests, "
                                   f"{args.pool} seeded circuits of 12-48 qubits depth 8-20 (1D/2D), "
                                   f"{args.duration}s stream after a {args.warmup_s}s warm-up, "
                                   f"{budget / 2**30:.0f} GiB budget",
                       "planning_seconds": plan_s, "latency_warmup_s": args.warmup_s},
            "bf16_split": res["bf16"], "c64": res["c64"]}
    print(json.dumps(line), flush=True)


def run_cfg3(args):
    """Precision sweep on the 2D grid circuit: complex128, complex64, TF32 split and BF16 split, each
    timed on a batch of amplitudes (CUDA events, after warm-up) and checked against the oracle on
    the 4x5 depth-8 instance; the 5x8 depth-12 instance is planned and its exact memory count
    reported (its contraction is infeasible with Greedy partition trees)."""
    import torch
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa
    from oracle import contract as oc
    torch.cuda.set_device(0)
    circ, x0 = tni.cfg3(small=True)
    n = circ.n_qubits
    B = min(args.batch, 256)
    xs = [x0] + [tni.random_bitstring(n, 7000 + i) for i in range(B - 1)]
    nets = [tni.amplitude_tn(circ, x) for x in xs]
    hs = [tnsa.tn_build(t) for t in nets]
    plan = tnsa.tn_plan_create(hs[0], k=8, iterations=args.plan_iters, steps_per_temp=8, seed=7,
                               position=nets[0].qubit)
    con_serial, con_dist, mem = tnsa.tn_plan_counts(plan)
    part, steps, _ = tnsa.tn_plan_export(plan, nets[0].n_tensors)
    tree = [(int(l), int(r)) for l, r, o in steps]
    check = sorted({0, B // 2, B - 1})
    refs = {i: oc.contract_scalar(nets[i], tree) for i in check}
    stream = torch.cuda.Stream()
    rows = {}
    for prec in ("c128", "c64", "tf32", "bf16"):
        ctx = tnsa.tn_ctx_create(0, stream=stream.cuda_stream)
        b = tnsa.tn_batch_create(ctx, hs, [plan] * B, prec)
        info = tnsa.tn_batch_last_info(b)
        for _ in range(max(args.warmup, 3)):
            tnsa.tn_batch_run(b)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        steps_t = max(1, min(args.steps, 50))
        for _ in range(steps_t):
            tnsa.tn_batch_run(b)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps_t
        mant, e2, st = tnsa.tn_batch_results(b, B)
        errs = []
        for i in check:
            got = complex(mant[i]) * 2.0 ** int(e2[i])
            errs.append(abs(got - refs[i]) / abs(refs[i]))
        rows[prec] = {"ms_per_step": ms, "amps_per_s": B / (ms * 1e-3), "tflops": B * 8.0 * con_serial / (ms * 1e-3) / 1e12,
                      "max_err_vs_oracle": max(errs), "status_ok": bool((st == 0).all()),
                      "tensor_core_steps": info["n_tc"], "launches": info["launches"]}
        b.close()
        ctx.close()
    # the full-size 5x8 depth-12 grid: its plan is sliced (Section 4.1) to a per-slice memory that
    # fits a batch of slices on the device; a sample of slices is contracted and timed, and the
    # time of all slices projected from it
    big = tni.amplitude_tn(tni.cfg3()[0], tni.cfg3()[1])
    bh = tnsa.tn_build(big)
    bplan = tnsa.tn_plan_create(bh, k=8, iterations=args.plan_iters, steps_per_temp=8, seed=7,
                                position=big.qubit)
    btotal, bcrit, bmem = tnsa.tn_plan_counts(bplan)
    sl = tnsa.tn_plan_slice(bh, bplan, 1 << 26, max_edges=96)
    full = {"mem_elements": bmem, "con_serial": btotal, "con_dist": bcrit, "fits_hbm_unsliced": bmem * 8 < 250e9,
            "sliced_edges": len(sl["edges"]), "n_slices": sl["n_slices"], "slice_mem_elements": sl["slice_mem"],
            "slice_con": sl["slice_con"], "total_con_sliced": sl["total_con"],
            "redundant_ops_ratio": sl["total_con"] / max(btotal, 1)}
    if sl["slice_mem"] <= (1 << 26) and sl["n_slices"] <= (1 << 40):
        ctx = tnsa.tn_ctx_create(0, stream=stream.cuda_stream)
        sample = int(min(sl["n_slices"], 64))
        try:
            tnsa.tn_contract_sliced(ctx, bh, bplan, sl["edges"], "bf16", max_jobs=32, slice_count=min(sample, 32))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tnsa.tn_contract_sliced(ctx, bh, bplan, sl["edges"], "bf16", max_jobs=32, first_slice=0,
                                    slice_count=sample)
            dt = time.perf_counter() - t0
            full.update({"timed_slices": sample, "seconds_per_slice": dt / sample,
                         "projected_seconds_all_slices": dt / sample * sl["n_slices"],
                         "sliced_tflops": sample * 8.0 * sl["slice_con"] / dt / 1e12})
        except tnsa.TnError as e:
            full["sample_error"] = str(e)
        ctx.close()
    else:
        # too many slices to sample: the projection uses the BF16 throughput of the 4x5 instance
        rate = rows["bf16"]["tflops"] * 1e12
        full.update({"timed_slices": 0, "projection_rate_tflops": rows["bf16"]["tflops"],
                     "projected_seconds_all_slices": 8.0 * sl["total_con"] / rate,
                     "projected_seconds_unsliced_if_it_fit": 8.0 * btotal / rate})
    line = {"metric": METRIC, "value": rows["bf16"]["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16-split", "data": "synthetic",
            "config": {"workload": f"2D grid 4x5 depth 8 (seed 3), k=8 SA partitions, batch of {B} amplitudes; "
                                   "precision sweep with the error against the complex128 oracle",
                       "plan": {"con_serial": con_serial, "con_dist": con_dist, "mem": mem}},
            "precisions": rows,
            "full_size_5x8_depth12": full}
    print(json.dumps(line), flush=True)


def run_permute(args):
    """TTGT permutation kernels on a 2^26-element complex64 tensor (512 MiB, 26 binary axes) --
    the largest intermediate size of the 24-qubit workload: achieved HBM bandwidth (read + write
    bytes over CUDA-event time, after warm-up; the tensor is 4x the L2) against the measured copy
    peak, for an axis reversal (shared-memory tile path) and a permutation of the outer axes that
    keeps the innermost 8 (row path)."""
    import torch
    from paper_2507_20667_gb300 import tnsa
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = tnsa.tn_ctx_create(0, stream=stream.cuda_stream)
    n_ax = 26
    dims = (2,) * n_ax
    d_in = torch.randn(1 << n_ax, 2, device="cuda")
    d_out = torch.empty_like(d_in)
    cases = {"reverse_all_axes": tuple(range(n_ax - 1, -1, -1)),
             "outer_axes_permuted_inner_8_kept": tuple([17, 3, 12, 0, 9, 5, 14, 1, 16, 7, 10, 2, 15, 4, 11, 6, 13, 8])
                                                  + tuple(range(18, 26))}
    peak, peak_kind = measured_peaks()
    res = {}
    for name, perm in cases.items():
        for _ in range(max(args.warmup, 3)):
            tnsa.tn_permute(ctx, d_in.data_ptr(), d_out.data_ptr(), 8, dims, perm)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 50))
        ev0.record(stream)
        for _ in range(reps):
            tnsa.tn_permute(ctx, d_in.data_ptr(), d_out.data_ptr(), 8, dims, perm)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        gbs = 2 * (8 << n_ax) / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "GB/s": gbs, "frac": gbs / peak}
    best = max(r["GB/s"] for r in res.values())
    line = {"metric": "TTGT permutation bandwidth", "value": best, "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "permute a 2^26-element complex64 tensor (26 binary axes), 512 MiB in and out",
                       "l2": "tensor 4x the L2"},
            "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_kind": f"{peak_kind} hbm_gbs"},
            "cases": res}
    print(json.dumps(line), flush=True)


class _TraceNet:
    """trace(A B C) as a closed network of three complex matrices (A: I x K, B: K x J, C: J x I):
    the first pairwise step A*B is a dense GEMM (M = I, N = J, K = K)."""

    def __init__(self, I, K, J, seed):
        rng = np.random.default_rng(seed)

        def rnd(*sh):
            return (rng.standard_normal(sh) + 1j * rng.standard_normal(sh)) / np.sqrt(2)
        A, B, C = rnd(I, K), rnd(K, J), rnd(J, I)
        self.degrees = np.array([2, 2, 2], np.int32)
        self.dims = np.array([I, K, K, J, J, I], np.int64)
        self.data = np.concatenate([A.ravel(), B.ravel(), C.ravel()]).view(np.float64)
        self.edges = np.array([[0, 1, 1, 0], [1, 1, 2, 0], [2, 1, 0, 0]], np.int32)


def run_tcgemm(args):
    """A dense complex GEMM step (trace(A B C), I = J = 4096, K = 1024 by default) in BF16 split,
    TF32 split (tcgen05 tensor cores) and complex64 (CUDA cores): device time of the contraction
    kernels per run, algorithmic TFLOP/s (8 M N K) and executed tensor-core TFLOP/s (24 M N K,
    three products of the 4M real form) against the measured BF16 peak."""
    from paper_2507_20667_gb300 import tnsa
    I, K, J = args.gemm
    net = _TraceNet(I, K, J, seed=1)
    h = tnsa.tn_build(net)
    plan = tnsa.tn_plan_import(h, [(0, 1), (2, 3)])
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peaks = json.load(f)
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    mnk = I * J * K
    res = {}
    for prec in ("bf16", "tf32", "c64"):
        ctx = tnsa.tn_ctx_create(0)
        tnsa.tn_ctx_set_local_budget(ctx, 0)
        b = tnsa.tn_batch_create(ctx, [h], [plan], prec)
        for _ in range(max(args.warmup, 3)):
            tnsa.tn_batch_run(b)
        reps = max(1, min(args.steps, 20))
        for _ in range(reps):
            tnsa.tn_batch_run(b)
        ms = tnsa.tn_batch_kernel_ms(b, reps)
        times = tnsa.tn_batch_kernel_times(b, reps)
        info = tnsa.tn_batch_last_info(b)
        r = {"ms": ms, "algorithmic_tflops": 8 * mnk / ms / 1e9, "tensor_core_steps": info["n_tc"],
             "kernel_ms": times}
        if prec != "c64":
            peak = bf16_peak if prec == "bf16" else bf16_peak / 2   # TF32 dense rate is half of BF16
            executed = 24 * mnk / ms / 1e9
            gemm = 24 * mnk / times["tc_gemm"] / 1e9 if times["tc_gemm"] > 0 else None
            r.update({"executed_tflops": executed, "tensor_frac": executed / peak,
                      "gemm_kernel_executed_tflops": gemm, "gemm_kernel_frac": gemm / peak if gemm else None})
        res[prec] = r
        b.close()
        ctx.close()
    line = {"metric": "dense complex GEMM step, TFLOP/s", "value": res["bf16"]["algorithmic_tflops"],
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16-split", "data": "synthetic",
            "config": {"workload": f"trace(A B C), A {I}x{K}, B {K}x{J}, C {J}x{I} complex; the A*B step"},
            "roofline": {"bound": "tensor", "peak": bf16_peak, "unit": "TFLOP/s",
                         "peak_kind": "measured bf16_tflops" if peaks else "fallback"},
            "precisions": res}
    print(json.dumps(line), flush=True)


def run_planner(args):
    """Planner quality on the 24-qubit brickwork circuit (host only): for k in a sweep, the initial
    qubit-block partition and simulated annealing in both modes (Algorithm 2, naive and directed),
    each with the exact con_dist (Eq. 3.5, the critical path) and mem (Eq. 3.1) relative to the
    serial Greedy tree (k = 1, whose con_dist is its con_serial)."""
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa
    circ = tni.brickwork_1d(N_QUBITS, DEPTH, seed=2)
    net = tni.amplitude_tn(circ, tni.random_bitstring(N_QUBITS, 1002))
    h = tnsa.tn_build(net)
    serial = tnsa.tn_plan_create(h, k=1)
    s_total, s_crit, s_mem = tnsa.tn_plan_counts(serial)
    rows = []
    for k in args.k_sweep:
        # qubit blocks need at least one qubit per part; beyond that the balanced BFS start is used
        pos = net.qubit if k <= N_QUBITS else None
        row = {"k": k, "initial": "qubit_block" if pos is not None else "bfs",
               "fanin_device": args.fanin_device if k > 4 else -1}
        for name, kw in (("initial", dict(iterations=0)),
                         ("sa_naive", dict(mode="naive", iterations=args.plan_iters)),
                         ("sa_directed", dict(mode="directed", iterations=args.plan_iters))):
            t0 = time.perf_counter()
            plan = tnsa.tn_plan_create(h, k=k, steps_per_temp=8, seed=7, position=pos,
                                       fanin_device=args.fanin_device, **kw)
            sec = time.perf_counter() - t0
            total, crit, mem = tnsa.tn_plan_counts(plan)
            row[name] = {"con_dist_ratio": crit / s_crit, "con_serial_ratio": total / s_total,
                         "mem_ratio": mem / s_mem, "seconds": sec}
        rows.append(row)
    line = {"metric": "con_dist of the k-partitioned plan relative to serial Greedy (lower is better)",
            "value": min(r["sa_directed"]["con_dist_ratio"] for r in rows), "unit": "ratio",
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": f"24-qubit brickwork depth {DEPTH}: qubit-block start (balanced BFS regions "
                                   f"for k > 24), SA naive and directed ({args.plan_iters} iterations, seed 7) "
                                   f"for k in {list(args.k_sweep)}; fan-in trees of k > 4 evaluated on "
                                   f"{'the GPU' if args.fanin_device >= 0 else 'the host'}",
                       "serial": {"con_serial": s_total, "mem": s_mem}},
            "sweep": rows}
    print(json.dumps(line), flush=True)


def run_costmodel(args):
    """Measured time against the paper's cost model: plans of the 24-qubit brickwork circuit with
    different k and SA modes, each timed on the GPU (a batch of amplitudes, CUDA events, kernel
    time per amplitude) beside its exact con_dist and con_serial; reports the Pearson correlation
    of time with each count (the paper reports 0.998 for its distributed runs)."""
    import torch
    from paper_2507_20667_gb300 import inputs as tni
    from paper_2507_20667_gb300 import tnsa
    torch.cuda.set_device(0)
    B = min(args.batch, 608)
    circ, xs, nets = make_workload(B)
    hs = [tnsa.tn_build(n) for n in nets]
    ctx = tnsa.tn_ctx_create(0)
    rows = []
    settings = [(1, "directed", 1)] + [(k, mode, iters) for k in args.k_sweep if k > 1
                                       for mode in ("naive", "directed") for iters in (30, 300, 2000)]
    for k, mode, iters in settings:
        pos = nets[0].qubit if 1 < k <= N_QUBITS else None
        plan = tnsa.tn_plan_create(hs[0], k=k, mode=mode, iterations=iters, steps_per_temp=8, seed=7,
                                   position=pos)
        total, crit, mem = tnsa.tn_plan_counts(plan)
        row = {"k": k, "mode": mode, "iterations": iters, "con_serial": total, "con_dist": crit, "mem": mem}
        if mem * 8 * B > 32e9:   # the batch's intermediates would exceed 32 GB: not timed
            rows.append(dict(row, skipped="intermediates of the batch above 32 GB"))
            continue
        try:
            b = tnsa.tn_batch_create(ctx, hs, [plan] * B, "c64")
        except tnsa.TnError as e:
            rows.append(dict(row, error=str(e)))
            continue
        for _ in range(max(args.warmup, 3)):
            tnsa.tn_batch_run(b)
        reps = max(1, min(args.steps, 20))
        for _ in range(reps):
            tnsa.tn_batch_run(b)
        ms = tnsa.tn_batch_kernel_ms(b, reps)
        rows.append(dict(row, us_per_amplitude=1e3 * ms / B))
        b.close()
    ok = [r for r in rows if "us_per_amplitude" in r]
    t = np.array([r["us_per_amplitude"] for r in ok])

    def pearson(x):
        x = np.array(x, dtype=np.float64)
        return float(np.corrcoef(x, t)[0, 1]) if len(ok) > 2 else None
    line = {"metric": "Pearson r of measured GPU time per amplitude with the plan's op counts",
            "value": pearson([r["con_serial"] for r in ok]), "unit": "r", "higher_is_better": True,
            "data": "synthetic",
            "config": {"workload": f"24-qubit brickwork depth {DEPTH}, batch of {B}, complex64; plans for k in "
                                   f"{list(args.k_sweep)}, SA naive and directed with 30, 300 and 2000 iterations"},
            "r_con_serial": pearson([r["con_serial"] for r in ok]),
            "r_con_dist": pearson([r["con_dist"] for r in ok]),
            "plans": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=2432)
    ap.add_argument("--precision", default="c64")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-check", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--workload", default="cfg2",
                    choices=["cfg2", "cfg3", "cfg4", "cfg5", "permute", "tcgemm", "planner", "costmodel"])
    ap.add_argument("--k-sweep", type=int, nargs="+", default=[1, 2, 4, 8, 16, 32, 64])
    ap.add_argument("--fanin-device", type=int, default=-1)
    ap.add_argument("--gemm", type=int, nargs=3, default=[4096, 1024, 4096], metavar=("I", "K", "J"))
    ap.add_argument("--queries-per-circuit", type=int, default=16)
    ap.add_argument("--plan-iters", type=int, default=100)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--warmup-s", type=float, default=5.0)
    ap.add_argument("--drain-s", type=float, default=60.0)
    args = ap.parse_args()
    if args.workload == "cfg3" and args.impl == "ours":
        return run_cfg3(args)
    if args.workload == "permute" and args.impl == "ours":
        return run_permute(args)
    if args.workload == "tcgemm" and args.impl == "ours":
        return run_tcgemm(args)
    if args.workload == "planner":
        return run_planner(args)
    if args.workload == "costmodel" and args.impl == "ours":
        return run_costmodel(args)
    if args.workload == "cfg4" and args.impl == "ours":
        return run_cfg4(args)
    if args.workload == "cfg5" and args.impl == "ours":
        return run_cfg5(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
