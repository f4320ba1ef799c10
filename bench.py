#!/usr/bin/env python
"""Throughput of the DG Maxwell time step on GB300, as one JSON line.

A bench "step" is one leapfrog time step (H-phase + E-phase over the whole
mesh) of the named workload.  The metric is DoF-steps/s = elements * D_e *
steps / time with D_e = 3 N3(p) + 3 N3(p-1) volume coefficients per element.

Default workload: planewave_n32_p6 (periodic unit box, n = 32, 196,608 tets,
p = 6, plane wave k = 2 pi (1,2,3)), TC16 path (fp16 tensor-core operands, fp32
state); the FP64 path is timed on the same workload and reported beside it.
The field state (330 MB in fp32) is larger than the 129 MB L2, so no L2 flush
is needed between steps.  Smaller workloads (cavity_n4_p3, pulse_n16_p4) are
L2-resident and say so in `config.l2`.  --workload batched_64 times 64 runs in
one CUDA graph; --workload adjoint_n16_p4 times the checkpointed adjoint
gradient (one bench step = one gradient over the workload's 500 time steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

For N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the method has no cross-problem exchange); value = all ranks' DoF-steps / the
max over ranks of the timed region.  --impl reference times the FP64 CPU
oracle on bounded element samples of the same workload (rank 0 only).
"""

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF-steps/s at p=4/6 (mixed vs FP64 plain, same GB300); % HBM roofline; err"
DTYPE = {"tc32": "tf32", "tc16": "f16", "tcbf16": "bf16", "tc16x2": "f16", "fp32": "f32", "fp64": "f64"}
ARITH = {"tc32": "fp32 state, TF32 tensor-core operators (tcgen05), fp32 accumulate, fp64 geometry and energy",
         "tc16": "fp32 state with fp16 operand copies, fp16 tables and trace buffers, fp16 tensor-core operators "
                 "(tcgen05 kind::f16), fp32 accumulate, fp64 geometry and energy",
         "tcbf16": "fp32 state with bf16 operand copies, bf16 tables and trace buffers, bf16 tensor-core "
                   "operators (tcgen05 kind::f16, bf16 encoding), fp32 accumulate, fp64 energy sums",
         "tc16x2": "fp32 state with fp16 operand copies, two-term fp16 tables (hi + lo, two MMAs per table "
                   "K-step), fp16 trace buffers, tcgen05 kind::f16, fp32 accumulate, fp64 energy sums",
         "fp32": "fp32 state and CUDA-core arithmetic, fp64 geometry and energy",
         "fp64": "fp64 throughout"}
UNIT = "DoF-steps/s"


def n3(q):
    return (q + 1) * (q + 2) * (q + 3) // 6 if q >= 0 else 0


def dof_per_elem(p):
    return 3 * n3(p) + 3 * n3(p - 1)


# nominal FP64 rate of one GB300: used only if the measurement below fails; the
# FP64 path is bound by FP64 arithmetic, not by HBM
FP64_NOMINAL_TFLOPS = 1.25
_FP64_PEAK = {}


def fp64_peak(device=0):
    """FP64 FMA rate of the device measured in this run (dgm_measure_fp64_peak:
    CUDA events around a kernel of independent FMA chains on every SM, best of 5)."""
    if device not in _FP64_PEAK:
        try:
            from paper_1104_4208_gb300 import _capi as capi
            _FP64_PEAK[device] = (capi.dgm_measure_fp64_peak(device, 5), "measured (FP64 FMA microbenchmark, this run)")
        except Exception as e:   # measurement failed: say so and fall back to the nominal rate
            _FP64_PEAK[device] = (FP64_NOMINAL_TFLOPS, f"nominal GB300 FP64 rate (measurement failed: {e})")
    return _FP64_PEAK[device]


def n2(q):
    return (q + 1) * (q + 2) // 2


def flops_per_elem_step(p):
    """Flops of one element and time step in the dense-operator form: curl and
    curl^T (2 x 3 x 2 N3(p-1) N3(p) mult-adds) plus traces and lifts of both
    fields on four faces (2 components x 2 x 2 N2 N3 each)."""
    return 24 * n3(p - 1) * n3(p) + 32 * (n2(p) * n3(p) + n2(p - 1) * n3(p - 1))


def phase_bytes(nt, p, b):
    """Algorithmic bytes of one H-phase and one E-phase launch over nt elements with
    b bytes per state value (g = 64 B geometry, c = 20 B topology per element): the
    H-phase reads E and H and writes H, the E-phase reads H and E and writes E."""
    NE, NH = n3(p), n3(p - 1)
    return nt * (b * (3 * NE + 6 * NH) + 64 + 20), nt * (b * (6 * NE + 3 * NH) + 64 + 20)


def executed_flops_per_elem_step(p, sparse):
    """Flops the trace-buffer CUDA-core kernels execute per element and step: curl and
    curl^T (6 N3(p-1) N3(p) mult-adds each, or 2 per nonzero of D_x, D_y, D_z with the
    sparse curl), the lifts (4 faces x 2 x N2(p-1) N) and the traces of each updated
    field (4 faces x 3 components x N2(p-1) N), N = N3(p-1) for H and N3(p) for E."""
    NE, NH, G = n3(p), n3(p - 1), n2(p - 1)
    if sparse:
        from paper_1104_4208_gb300 import _capi as capi
        curl = 2 * sum(int(np.count_nonzero(capi.dgm_reference_table(p, d))) for d in range(3))
    else:
        curl = 6 * NH * NE
    fma = 2 * curl + 8 * G * (NH + NE) + 12 * G * (NH + NE)
    return 2 * fma


def alu_roofline(w, ms_per_step, device=0, sparse=None):
    """FP64 roofline: executed flops / time against the measured FP64 rate (frac),
    and the dense-operator count of the measurement plan beside it."""
    peak, src = fp64_peak(device)
    dense_ach = w.nt * flops_per_elem_step(w.p) / (ms_per_step * 1e-3) / 1e12
    out = {"bound": "alu", "unit": "TFLOP/s", "peak": peak, "peak_source": src, "traffic": None,
           "dense_equivalent": {"flops_per_element_step": flops_per_elem_step(w.p), "achieved": dense_ach,
                                "frac": dense_ach / peak}}
    if sparse is None:   # no kernel information: the dense-operator count
        out.update(achieved=dense_ach, frac=dense_ach / peak, flops_per_element_step=flops_per_elem_step(w.p))
    else:
        fe = executed_flops_per_elem_step(w.p, sparse)
        ach = w.nt * fe / (ms_per_step * 1e-3) / 1e12
        out.update(achieved=ach, frac=ach / peak, flops_per_element_step=fe,
                   curl="sparse (exact zeros of D_x, D_y, D_z skipped)" if sparse else "dense")
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="planewave_n32_p6")
    ap.add_argument("--precision", default="tc16", choices=["tc16", "tcbf16", "tc16x2", "tc32", "fp32", "fp64"])
    ap.add_argument("--variant", type=int, default=0,
                    help="TC16: 0 resident-table kernels (default), 1 dense-operator kernels; FP64/FP32: "
                         "0 automatic (autotuned), 1 dense curl, 2 sparse curl, 3 element-group kernels (sparse curl)")
    ap.add_argument("--no-p4", action="store_true", help="skip the p = 4 sub-block of the default workload")
    ap.add_argument("--fp64-steps", type=int, default=1, help="nonzero: also run the FP64 path over the same steps")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU oracle sample")
    ap.add_argument("--cpu-procs", type=int, default=None,
                    help="single-threaded oracle processes (default: one per host core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--clocks-csv", default=None, help="keep the nvidia-smi clock samples in this file (per rank)")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="CPU budget of the whole --impl reference run (split over its steps)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def analytic(workload):
    from workloads.fields import plane_wave_fields, te110_fields, gaussian_pulse_fields
    if workload.init == "plane":
        return lambda x, t: plane_wave_fields(x, t)
    if workload.init == "te110":
        return lambda x, t: te110_fields(x, t)
    c = workload.centre
    return lambda x, t: gaussian_pulse_fields(x, c) if t == 0 else (None, None)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        # kept where --clocks-csv says (rank suffix added), else a temporary file
        self.path = (f"{path}.rank{index}" if path else f"/tmp/dgm_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if re.match(r"^[0-9.]+$", r[1])]
        smax = [float(r[2]) for r in rows if re.match(r"^[0-9.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profile_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel source (sha256 of the file that defines it,
    recorded beside the numbers)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_1104_4208_gb300", "csrc",
                       "tc2_kernels.cu" if kernel.startswith("k_tc2") else
                       "tc_kernels.cu" if kernel.startswith("k_tc") else "kernels.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel and parts[1] == sha:
                return float(parts[3])
    except OSError:
        pass
    return None


# ---------------------------------------------------------------- GPU arm
def make_solver(w, precision, variant=0):
    from paper_1104_4208_gb300.solver import Solver
    m = w.mesh
    return Solver(m.xyz, m.tets, w.p, w.eps, w.mu, vertex_key=m.vertex_key, precision=precision,
                  variant=variant if precision in ("tc16", "fp64", "fp32") else 0)


def project_initial(S, w, torch, q1d):
    from paper_1104_4208_gb300 import _capi as capi
    xh, _ = capi.dgm_quad_rule(q1d)
    maps = capi.dgm_element_maps(S.mesh, S.nt)
    F = maps[:, 3:].reshape(-1, 3, 3)
    fn = analytic(w)
    Ed = torch.empty((S.nt, xh.shape[0], 3), dtype=torch.float64, device="cuda")
    Hd = torch.empty_like(Ed)
    chunk = 16384
    for s in range(0, S.nt, chunk):
        e = min(S.nt, s + chunk)
        x = maps[s:e, None, :3] + np.einsum("tij,qj->tqi", F[s:e], xh)
        Ex, Hx = fn(x, 0.0)
        Ed[s:e].copy_(torch.from_numpy(Ex))
        Hd[s:e].copy_(torch.from_numpy(Hx))
    capi.dgm_project_device(S.prob, q1d, Ed.data_ptr(), Hd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    del Ed, Hd
    torch.cuda.empty_cache()
    return maps, xh


def l2_rel_error(S, w, torch, q1d, maps, xh, T, keep=None):
    """Relative L2 error of E against the analytic field at time T (None for the
    pulse, which has no closed form); keep: list receiving (values, weights)."""
    from paper_1104_4208_gb300 import _capi as capi
    if w.init not in ("plane", "te110") and keep is None:
        return None
    _, wq = capi.dgm_quad_rule(q1d)
    Ed = torch.empty((S.nt, xh.shape[0], 3), dtype=torch.float64, device="cuda")
    capi.dgm_eval_device(S.prob, q1d, Ed.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    Eh_all = Ed.cpu().numpy()
    del Ed
    torch.cuda.empty_cache()
    F = maps[:, 3:].reshape(-1, 3, 3)
    det = np.abs(np.linalg.det(F))
    if keep is not None:
        keep.append((Eh_all, det[:, None] * wq[None, :]))
    if w.init not in ("plane", "te110"):
        return None
    fn = analytic(w)
    err2 = ref2 = 0.0
    chunk = 16384
    for s in range(0, S.nt, chunk):
        e = min(S.nt, s + chunk)
        x = maps[s:e, None, :3] + np.einsum("tij,qj->tqi", F[s:e], xh)
        Ex, _ = fn(x, T)
        Eh = Eh_all[s:e]
        wt = det[s:e, None] * wq[None, :]
        err2 += np.einsum("tq,tqc->", wt, (Eh - Ex) ** 2)
        ref2 += np.einsum("tq,tqc->", wt, Ex ** 2)
    return float(np.sqrt(err2 / ref2))


def l2_note(state_bytes):
    import torch
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    if state_bytes > l2:
        return f"state {state_bytes / 1e6:.0f} MB larger than the {l2 / 1e6:.0f} MB L2 (no flush needed)"
    return (f"state {state_bytes / 1e6:.1f} MB fits in the {l2 / 1e6:.0f} MB L2: an L2-resident figure "
            "(the time loop reuses the state; no flush)")


def timed_run(S, torch, dt, steps, warmup):
    from paper_1104_4208_gb300 import _capi as capi
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    if warmup > 0:
        capi.dgm_run(S.prob, dt, warmup, sp)
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()
    W = np.empty(steps + 1)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = capi.dgm_run_timed(S.prob, dt, steps, sp, W)
    ev1.record(stream)
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), stats, W


_DIST = {"on": False}


def dist_barrier():
    if _DIST["on"]:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x):
    if not _DIST["on"]:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _DIST["nccl"] else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


_ORACLE_WORKER = r"""
import sys, time, json
import numpy as np
sys.path.insert(0, sys.argv[1])
from workloads.configs import make_workload
from oracle.dg import OracleDG
names = json.loads(sys.argv[2]); budget = float(sys.argv[3]); seed = int(sys.argv[4])
cache = {}
for it, name in enumerate(names):
    if name not in cache:
        w = make_workload(name)
        m = w.mesh
        dg = OracleDG(m.xyz, m.tets, w.p, w.eps, w.mu, vertex_key=m.vertex_key)
        rng0 = np.random.default_rng(seed)
        E = rng0.standard_normal(m.nt * 3 * dg.NE); H = rng0.standard_normal(m.nt * 3 * dg.NH)
        t0 = time.perf_counter(); dg.local_kick_H(E, [0], w.dt); dg.local_kick_E(H, [0], w.dt)
        per = max(time.perf_counter() - t0, 1e-3)
        cache[name] = (w, dg, E, H, per)
    w, dg, E, H, per = cache[name]
    rng = np.random.default_rng([seed, it])
    k = int(max(1, min(4096, budget / per)))
    s = rng.choice(w.nt, k, replace=False)
    t0 = time.perf_counter()
    for c in range(0, k, 16):
        dg.local_kick_H(E, s[c:c+16], w.dt); dg.local_kick_E(H, s[c:c+16], w.dt)
    t1 = time.perf_counter()
    print(json.dumps({"it": it, "elements": int(k), "seconds": t1 - t0, "dof": 3 * dg.NE + 3 * dg.NH}), flush=True)
"""


def cpu_procs():
    """Worker processes for the oracle timing: one single-threaded process per host core
    (at most 32; each holds about 1.2 GB at planewave_n32_p6)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 32))


def cpu_oracle_samples(names, seconds, procs=None):
    """The FP64 CPU oracle, as it stands, timed on bounded element samples (H- and
    E-kick of random elements) of the workloads `names` (one per step), by `procs`
    single-threaded processes running side by side, each setting up once.
    -> per step: {"elements", "dof" (element-DoF-steps), "rate" (sum of the
    processes' DoF-steps/s)}, and the process count; None if a process failed."""
    procs = procs or cpu_procs()
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    ps = [subprocess.Popen([sys.executable, "-c", _ORACLE_WORKER, ROOT, json.dumps(list(names)), str(seconds), str(q)],
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env) for q in range(procs)]
    outs = []
    for p in ps:
        try:
            o, _ = p.communicate(timeout=1800)
        except subprocess.TimeoutExpired:
            p.kill()
            return None
        if p.returncode != 0:
            return None
        outs.append([json.loads(line) for line in o.strip().splitlines() if line.startswith("{")])
    steps = []
    for it in range(len(names)):
        rows = [o[it] for o in outs]
        steps.append({"elements": sum(r["elements"] for r in rows),
                      "dof": sum(r["elements"] * r["dof"] for r in rows),
                      "rate": sum(r["elements"] * r["dof"] / r["seconds"] for r in rows),
                      "seconds": max(r["seconds"] for r in rows)})
    return steps, procs


def run_gpu(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    from workloads.configs import make_workload
    from paper_1104_4208_gb300 import _capi as capi

    w = make_workload(args.workload)
    D = dof_per_elem(w.p)
    dofs = w.nt * D
    q1d = w.p + 1
    S = make_solver(w, args.precision, args.variant)
    maps, xh = project_initial(S, w, torch, q1d)
    err0 = l2_rel_error(S, w, torch, q1d, maps, xh, 0.0)
    dt = w.dt
    tune = None
    if not args.no_autotune:   # launch configuration picked by measurement (fields unchanged)
        cfg, tms, ch = S.autotune(3)
        tune = {"per_sm": cfg, "ms_per_step": [round(x, 4) for x in tms], "chosen": cfg[ch]}

    with ClockSampler(local, args.clocks_csv) as clk:
        ms, stats, W = timed_run(S, torch, dt, args.steps, args.warmup)
    clocks = clk.summary()
    T = (args.warmup + args.steps) * dt
    kept = []
    err = l2_rel_error(S, w, torch, q1d, maps, xh, T, keep=kept if args.fp64_steps else None)
    drift = float(np.abs(W - W[0]).max() / W[0])
    ms_max = dist_max(ms)
    value = world * dofs * args.steps / (ms_max * 1e-3)

    # roofline of the dominant kernel (algorithmic bytes / CUDA-event duration)
    b = 8 if args.precision == "fp64" else 4
    bytes_H, bytes_E = phase_bytes(w.nt, w.p, b)
    tH = stats.h_phase_ms / max(stats.h_launches, 1)
    tE = stats.e_phase_ms / max(stats.e_launches, 1)
    tcp = args.precision in ("tc32", "tc16", "tcbf16", "tc16x2")
    resident = args.precision in ("tc16", "tcbf16") and args.variant == 0
    kpre = "k_tc2_phase" if resident else ("k_tc_phase" if tcp else "k_phase")
    if stats.h_phase_ms >= stats.e_phase_ms:
        kname, kbytes, kms = kpre + "_H", bytes_H, tH
    else:
        kname, kbytes, kms = kpre + "_E", bytes_E, tE
    peak, peak_src = measured_peak_hbm()
    achieved = kbytes / (kms * 1e-3) / 1e9
    sparse64 = bool(tune and tune["chosen"] >= 1000) or (not tune and args.variant in (2, 3))
    roof = alu_roofline(w, ms / args.steps, local, sparse64) if args.precision == "fp64" else \
        {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "traffic": profile_traffic(f"{kname}/{args.precision}" if tcp else f"{kname}<{'float' if b == 4 else 'double'}>"),
            "algorithmic_bytes_per_launch": kbytes, "avg_launch_ms": kms,
            "share": {kpre + "_H": stats.h_phase_ms / (stats.h_phase_ms + stats.e_phase_ms + stats.other_ms),
                      kpre + "_E": stats.e_phase_ms / (stats.h_phase_ms + stats.e_phase_ms + stats.other_ms)}}

    # FP64 plain path on the same workload, same initial data, same number of
    # steps: its throughput, and the mixed path's deviation from it at equal time
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        S.close()
        S64 = make_solver(w, "fp64")
        project_initial(S64, w, torch, q1d)
        tune64 = None
        if not args.no_autotune:   # the FP64 path in its own fastest configuration (dense or sparse curl)
            cfg64, tms64, ch64 = S64.autotune(2)
            tune64 = {"per_sm": cfg64, "ms_per_step": [round(x, 3) for x in tms64], "chosen": cfg64[ch64],
                      "note": "configurations 1000-1999: sparse curl, blocks per SM = value - 1000; >= 2000: "
                              "element-group kernels (sparse curl), blocks per SM = value - 2000"}
        ms64, st64, W64 = timed_run(S64, torch, dt, args.steps, args.warmup)
        v64 = world * dofs * args.steps / (dist_max(ms64) * 1e-3)
        kept64 = []
        err64 = l2_rel_error(S64, w, torch, q1d, maps, xh, T, keep=kept64)
        (Em, wts), (E64, _) = kept[0], kept64[0]
        dev = float(np.sqrt(np.einsum("tq,tqc->", wts, (Em - E64) ** 2) / np.einsum("tq,tqc->", wts, E64 ** 2)))
        del kept, kept64, Em, E64
        fp64 = {"value": v64, "ms_per_step": ms64 / args.steps, "speedup_of_mixed": value / v64,
                "energy_drift": float(np.abs(W64 - W64[0]).max() / W64[0]),
                "l2_rel_E_vs_analytic": err64, "mixed_minus_fp64_l2_rel": dev,
                "roofline": alu_roofline(w, ms64 / args.steps, local, bool(tune64 and tune64["chosen"] >= 1000)),
                "launch": tune64}
        S64.close()
        S = make_solver(w, args.precision, args.variant)
        project_initial(S, w, torch, q1d)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    nE, nH = S.nE, S.nH
    if args.no_e2e:
        nE = 0
    if nE:
        hE = torch.empty(nE, dtype=torch.float64, pin_memory=True).numpy()
        hH = torch.empty(nH, dtype=torch.float64, pin_memory=True).numpy()
        capi.dgm_get_fields(S.prob, hE, hH)
        torch.cuda.synchronize()
        dist_barrier()
        t0 = time.perf_counter()
        capi.dgm_set_fields(S.prob, hE, hH)
        capi.dgm_run(S.prob, dt, args.steps, None, None)
        capi.dgm_get_fields(S.prob, hE, hH)
        torch.cuda.synchronize()
        t_e2e = dist_max(time.perf_counter() - t0)
        dist_barrier()
        e2e = {"value": world * dofs * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": (nE + nH) * 8 / args.steps, "d2h_bytes_per_step": (nE + nH) * 8 / args.steps,
               "note": "one upload, K steps, one download per timed call"}
    S.close()

    p4 = None
    if args.workload == "planewave_n32_p6" and not args.no_p4:
        p4 = p4_block(args, torch, world)

    out = None
    if rank == 0:
        cpu = None
        if not args.no_cpu and world == 1:   # the oracle baseline is timed at N = 1 only
            res = cpu_oracle_samples([w.name], args.cpu_seconds, args.cpu_procs)
            if res:
                (r,), procs = res
                cpu = {"value": r["rate"], "unit": UNIT, "cores": procs, "kind": "oracle",
                       "sample": f"H- and E-kick of {r['elements']} random elements of {w.name} "
                                 f"({args.cpu_seconds:.0f} s in each of {procs} single-threaded processes)"}
        launches = int(stats.h_launches + stats.e_launches + stats.other_launches)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": DTYPE[args.precision], "data": "synthetic",
               "config": {"workload": w.name, "tets": w.nt, "p": w.p, "dof": dofs, "precision": args.precision,
                          "flux": "central", "dt": dt, "parallelism": f"replicas{world}",
                          "l2": l2_note(dofs * (8 if args.precision == "fp64" else 4)),
                          "state_mb": dofs * (8 if args.precision == 'fp64' else 4) / 1e6,
                          "arithmetic": ARITH[args.precision],
                          "kernels": ("resident-table tensor-core kernels (k_tc2)" if resident else
                                      "dense-operator tensor-core kernels (k_tc_phase)" if tcp else
                                      "CUDA-core kernels (k_phase)"),
                          "launch": ({"autotuned": tune,
                                      "unit": ("update/trace threads per element, one CTA per SM" if resident
                                               else "CTAs per SM" if tcp else "blocks per SM")}
                                     if tune else "default")},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clocks,
               "err": {"l2_rel_E_vs_analytic": err, "l2_rel_E_initial_projection": err0,
                       "energy_drift": drift},
               "fp64_plain": fp64, "p4": p4}
    return out


P4_WORKLOADS = ("pulse_n16_p4", "pulse_n32_p4")
P4_PRECISIONS = ("fp64", "fp32", "tc16")


def p4_block(args, torch, world):
    """The metric's p = 4 half, beside the p = 6 headline: pulse_n16_p4 (24,576 tets,
    state in L2) and pulse_n32_p4 (196,608 tets, state larger than L2), each in FP64,
    FP32 and TC16 (autotuned unless --no-autotune), timed like the headline (CUDA
    events around dgm_run_timed after the warm-up steps).  Per precision: DoF-steps/s,
    the dominant kernel's roofline fraction, the energy drift and the deviation of E
    from the FP64 run after the same steps in the energy norm (eps-weighted L2)."""
    from workloads.configs import make_workload
    steps = max(5, min(args.steps, 20))
    warm = max(3, args.warmup)
    out = {}
    for name in P4_WORKLOADS:
        w = make_workload(name)
        dofs = w.nt * dof_per_elem(w.p)
        rows, fields, S64 = {}, {}, None
        for prec in P4_PRECISIONS:
            S = make_solver(w, prec)
            project_initial(S, w, torch, w.p + 1)
            tuned = S.autotune(2) if not args.no_autotune else None
            ms, st, W = timed_run(S, torch, w.dt, steps, warm)
            ms = dist_max(ms)
            tH = st.h_phase_ms / max(st.h_launches, 1)
            tE = st.e_phase_ms / max(st.e_launches, 1)
            if prec == "fp64":
                sparse = bool(tuned and tuned[0][tuned[2]] >= 1000)
                roof = alu_roofline(w, ms / steps, torch.cuda.current_device(), sparse)
                frac = {"bound": "alu", "frac": roof["frac"], "achieved": roof["achieved"], "unit": "TFLOP/s",
                        "curl": roof["curl"]}
            else:
                bH, bE = phase_bytes(w.nt, w.p, 4)
                kb, kt = (bH, tH) if st.h_phase_ms >= st.e_phase_ms else (bE, tE)
                peak, _ = measured_peak_hbm()
                ach = kb / (kt * 1e-3) / 1e9
                frac = {"bound": "hbm", "frac": ach / peak, "achieved": ach, "unit": "GB/s",
                        "kernel": "H-phase" if st.h_phase_ms >= st.e_phase_ms else "E-phase"}
            rows[prec] = {"value": world * dofs * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                          "roofline": frac, "energy_drift": float(np.abs(W - W[0]).max() / W[0])}
            fields[prec] = S.get_fields()[0]
            if prec == "fp64":
                S64 = S
            else:
                S.close()
        zH = np.zeros(S64.nH)

        def enorm(X):
            S64.set_fields(X, zH)
            return np.sqrt(2.0 * S64.energy())

        n64 = enorm(fields["fp64"])
        for prec in P4_PRECISIONS:
            if prec != "fp64":
                rows[prec]["e_minus_fp64_energy_norm_rel"] = enorm(fields[prec] - fields["fp64"]) / n64
                rows[prec]["speedup_vs_fp64"] = rows[prec]["value"] / rows["fp64"]["value"]
        S64.close()
        out[name] = {"tets": w.nt, "p": w.p, "dof": dofs, "steps": steps, "warmup": warm,
                     "l2": l2_note(dofs * 4), **rows}
    return out


def run_batched(args, rank, world, local):
    """Workload batched_64: 64 independent runs (n in {8,12,16}, jitter 0.1h,
    p in {2..6}, eps ~ U[1,4], a seeded z-dipole Gaussian-derivative source each)
    in the chosen precision, each launch configuration autotuned, advanced
    together by one CUDA graph (dgm_batch_run); compared with one dgm_run call
    per run on the same problems, and with one dgm_run call per run of the
    plain FP64 path."""
    import torch
    torch.cuda.set_device(local)
    from workloads.configs import batched_runs
    from workloads.mesh import kuhn_cube_mesh
    from paper_1104_4208_gb300 import _capi as capi
    from paper_1104_4208_gb300.solver import Solver
    runs = batched_runs(64)

    def make_runs(precision, tune):
        out, dts, dofs, tuned = [], [], 0, []
        for (n, p, seed) in runs:
            m = kuhn_cube_mesh(n, jitter=0.1, seed=seed)
            rng = np.random.Generator(np.random.PCG64([seed, 1]))
            eps = rng.uniform(1, 4, m.nt)
            S = Solver(m.xyz, m.tets, p, eps, 1.0, precision=precision)
            dt = 0.2 / n / p ** 2
            tau = 500 * dt / 20
            capi.dgm_set_source(S.prob, rng.uniform(0.25, 0.75, 3), [0.0, 0.0, 1.0], 4 * tau, tau, 1.0)
            if tune:
                cfg, _, ch = S.autotune(2)
                tuned.append(cfg[ch])
            out.append(S)
            dts.append(dt)
            dofs += m.nt * dof_per_elem(p)
        return out, np.array(dts), dofs, tuned

    solvers, dts, dofs, tuned = make_runs(args.precision, not args.no_autotune)
    B = capi.dgm_batch_create(solvers[0].ctx, [S.prob for S in solvers])
    stream = torch.cuda.current_stream()
    K = args.steps
    for _ in range(max(1, args.warmup)):
        capi.dgm_batch_run(B, dts, K, stream.cuda_stream, None)   # first call captures the graph
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, args.clocks_csv) as clk:
        ev0.record(stream)
        capi.dgm_batch_run(B, dts, K, stream.cuda_stream, None)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = dist_max(ev0.elapsed_time(ev1))
    # one launch sequence per run, same problems, same steps
    torch.cuda.synchronize()
    ev0.record(stream)
    for S, dt in zip(solvers, dts):
        capi.dgm_run(S.prob, dt, K, stream.cuda_stream, None)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_seq = ev0.elapsed_time(ev1)
    W = np.empty((len(solvers), 2))
    capi.dgm_batch_run(B, dts, 1, stream.cuda_stream, W)
    capi.dgm_batch_destroy(B)
    for S in solvers:
        S.close()
    # plain FP64 path, one launch sequence per run
    s64, dts64, _, _ = make_runs("fp64", False)
    torch.cuda.synchronize()
    ev0.record(stream)
    for S, dt in zip(s64, dts64):
        capi.dgm_run(S.prob, dt, K, stream.cuda_stream, None)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms64 = ev0.elapsed_time(ev1)
    for S in s64:
        S.close()
    value = world * dofs * K / (ms * 1e-3)
    # kernels per run and step: E-phase, source, H-phase (+ the source tile's trace refresh on the
    # tensor-core path); per run once: opening trace pass and closing half kick
    per_step = 3 + (1 if args.precision in ("tc16", "tc32") else 0)
    launches = len(runs) * (per_step * K + 2)
    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
               "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": DTYPE[args.precision], "data": "synthetic",
               "config": {"workload": "batched_64", "runs": len(runs), "dof_total": dofs,
                          "precision": args.precision, "graph": "one CUDA graph, one branch per run",
                          "launch": {"autotuned_per_sm": tuned} if tuned else "default",
                          "l2": "runs small, partly L2 resident; no flush (time loop reuses state)"},
               "one_launch_sequence_per_run": {"value": world * dofs * K / (ms_seq * 1e-3), "ms": ms_seq,
                                                "batched_speedup": ms_seq / ms},
               "plain_fp64_one_launch_sequence_per_run": {"value": world * dofs * K / (ms64 * 1e-3), "ms": ms64,
                                                          "batched_speedup": ms64 / ms},
               "clocks": clk.summary(), "gpu_launches": launches}
    return out


def run_adjoint(args, rank, world, local):
    """Workload adjoint_n16_p4: J = sum of |E(x_o)|^2 over 8 seeded observation
    points and all 500 steps from the projected Gaussian pulse; one bench step is
    one dgm_adjoint_grad call (forward run with checkpoints every 50 steps,
    backward sweep recomputing each segment, dJ/d eps and dJ/d mu).  The metric
    counts the forward DoF-steps of the horizon, so value/forward-run value is
    the cost ratio of a gradient to a plain run."""
    import torch
    torch.cuda.set_device(local)
    from workloads.configs import make_workload
    from workloads.fields import random_points
    from paper_1104_4208_gb300 import _capi as capi
    w = make_workload(args.workload)
    dofs = w.nt * dof_per_elem(w.p)
    S = make_solver(w, args.precision)
    project_initial(S, w, torch, w.p + 1)
    E0, H0 = S.get_fields()
    pts = random_points(5000, 8, 0.1, 0.9)
    ckpt = 50
    tune = None
    if not args.no_autotune:
        cfg, tms, ch = S.autotune(3)
        tune = {"per_sm": cfg, "chosen": cfg[ch]}
    for _ in range(args.warmup):
        S.set_fields(E0, H0)
        capi.dgm_adjoint_grad(S.prob, w.dt, w.steps, pts, ckpt, w.nt, mu_grad=True)
    # the gradient call is synchronous (it returns host arrays): host timer around
    # K calls, after a device synchronize
    torch.cuda.synchronize()
    dist_barrier()
    t = 0.0
    with ClockSampler(local, args.clocks_csv) as clk:
        for _ in range(args.steps):
            S.set_fields(E0, H0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J, g, gm = capi.dgm_adjoint_grad(S.prob, w.dt, w.steps, pts, ckpt, w.nt, mu_grad=True)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
    t = dist_max(t)
    # a plain forward run over the same horizon, for the cost ratio
    S.set_fields(E0, H0)
    ms_fwd, _, _ = timed_run(S, torch, w.dt, w.steps, 0)
    S.close()
    value = world * dofs * w.steps * args.steps / t
    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
               "config": {"workload": w.name, "tets": w.nt, "p": w.p, "dof": dofs, "precision": args.precision,
                          "horizon_steps": w.steps, "checkpoint_every": ckpt, "observation_points": 8,
                          "step": "one dJ/d eps + dJ/d mu evaluation over the horizon",
                          "l2": l2_note(dofs * (8 if args.precision == "fp64" else 4)),
                          "launch": {"autotuned": tune} if tune else "default"},
               "forward_run": {"ms": ms_fwd, "value": world * dofs * w.steps / (ms_fwd * 1e-3),
                               "gradient_cost_in_forward_runs": 1e3 * t / args.steps / ms_fwd},
               "J": J, "grad_eps_norm": float(np.linalg.norm(g)), "grad_mu_norm": float(np.linalg.norm(gm)),
               "clocks": clk.summary(), "timer": "host clock around each synchronous gradient call"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from workloads.configs import make_workload
    batched = args.workload == "batched_64"
    # the batched workload has no single configuration: step i samples run i mod 64
    names = [f"batched_64:{i % 64}" if batched else args.workload for i in range(args.warmup + args.steps)]
    w = make_workload(names[0])
    per_step = max(0.5, args.ref_seconds / max(1, args.steps + args.warmup))
    res = cpu_oracle_samples(names, per_step, args.cpu_procs)
    if res is None:
        return {"impl": "reference", "unavailable": "CPU oracle failed to run"}
    steps, procs = res
    timed = steps[args.warmup:]
    # throughput of all processes: summed per-process rates, averaged over the timed steps
    value = sum(r["rate"] for r in timed) / len(timed)
    total_el = sum(r["elements"] for r in timed)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(r["seconds"] for r in timed) / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": ({"workload": "batched_64", "runs_sampled": min(64, args.steps), "precision": "fp64"}
                       if batched else {"workload": w.name, "tets": w.nt, "p": w.p, "precision": "fp64"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": procs,
                             "sample": f"{total_el} random elements of {args.workload} over {args.steps} steps, "
                                       f"H- and E-kick, {procs} single-threaded processes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        nccl = args.impl == "gb300" and torch.cuda.is_available()
        if nccl:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if nccl else "gloo")
        _DIST.update(on=True, nccl=nccl)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batched_64":
        out = run_batched(args, rank, world, local)
    elif args.workload == "adjoint_n16_p4":
        out = run_adjoint(args, rank, world, local)
    else:
        out = run_gpu(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if _DIST["on"]:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
