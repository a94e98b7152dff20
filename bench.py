#!/usr/bin/env python
"""Benchmark of the deterministic-NQS hot path on one B300 (or N independent replicas).

One step = one pass of the whole path over the synthetic workload of the shape of Cr2
CAS(48e,42o) (42 orbitals, 24a+24b, |S| = 2^20, backflow MLP 84-1024-1024-2016 in the mixed
BF16 form; --workload small_n16 / cr2_24e30o / tiny_n10 for the smaller shapes):
  nqs_connections  (enumerate all singles/doubles of S, look up in S, build H_SS CSR)
  nqs_energy_grad  (amplitudes, E_S, adjoint gradient)
  nqs_pt2          (emit C, radix sort, dedup, segmented reduce, EN-PT2 sums; above 30
                    orbitals over the screened set of Sec. 3.3 at eps = 1e-6, one traversal)
Metric: connections resolved per second over the step (H_SS lookups + PT2 emissions), with
E_S+grad evaluations per second reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nqs|reference] [--workload W]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2601_21310_b300 import synth  # noqa: E402

METRIC = "connections/s and E_S+grad evals/s at 1 B300; BF16 form vs FP64 at 1e-6 Ha"
UNIT = "connections/s"
WORKLOAD = "cr2_48e42o"
L2_FLUSH_BYTES = 512 << 20  # > 126 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nqs", choices=["nqs", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--eps-pt2", type=float, default=None,
                    help="PT2 screening threshold on psi normalised over S (0: the full "
                         "connected space; the paper's heat-bath value is 1e-6). Default: 0 up "
                         "to 30 orbitals, 1e-6 above (see default_eps_pt2)")
    ap.add_argument("--no-tensor-probe", action="store_true",
                    help="skip the tensor-core GEMM probe on the 42-orbital output-layer shape")
    ap.add_argument("--tensor-probe-only", default=None, metavar="M,N,K",
                    help="run only the tensor-core GEMM probe on this shape and print its line "
                         "(for profiling one GEMM form on a small case)")
    ap.add_argument("--probe-mn", action="store_true",
                    help="with --tensor-probe-only: both operands MN-major (the weight-gradient "
                         "layout: row-major [K][M] and [K][N])")
    ap.add_argument("--no-outer", action="store_true",
                    help="skip the outer-loop measurement (heat-bath set, amplitudes on T, Top-K)")
    ap.add_argument("--buckets", type=int, default=0,
                    help="PT2 hash buckets (0: the library's choice, from the free device memory)")
    ap.add_argument("--no-pt2", action="store_true",
                    help="step without PT2 (for shapes whose PT2 takes minutes); labelled in config")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the plain-FP64 comparison run (e.g. for a launch list of the step)")
    args = ap.parse_args()
    if args.eps_pt2 is None:
        args.eps_pt2 = default_eps_pt2(args.workload)
    return args


def default_eps_pt2(workload: str) -> float:
    """PT2 over all of C minus S up to 30 orbitals; above, the screened set of Sec. 3.3 at the
    paper's 1e-6 (at 42 orbitals the unscreened connected space has 2.85e11 pairs, which the
    bucketed sort would take many minutes to reduce)."""
    from paper_2601_21310_b300 import synth
    wl = synth.WORKLOADS.get(workload)
    return 1e-6 if wl is not None and wl.norb > 30 else 0.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank value over all ranks (identity on one process)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank: float, max_ms: float, world_size: int) -> float:
    """Weak scaling: every rank processes the same units; the job rate is all ranks' units over
    the slowest rank's time."""
    return world_size * units_per_rank / (max_ms / 1e3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region (read-only NVML queries)
# ------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampled every 100 ms during the timed region (read-only queries), filtered to
    this process's GPU by PCI bus id."""
    FIELDS = ["pci.bus_id", "clocks.sm", "clocks.max.sm", "power.draw",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, device_index: int):
        self.rows, self.err = [], None
        try:
            self.bus = int(torch.cuda.get_device_properties(device_index).pci_bus_id)
        except Exception:
            self.bus = None

    def __enter__(self):
        import subprocess
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:  # no nvidia-smi: report no clocks
            self.proc, self.err = None, str(e)
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [[x.strip() for x in line.split(",")] for line in out.splitlines()]
        rows = [r for r in rows if len(r) == len(self.FIELDS)]
        buses = {r[0] for r in rows}
        for r in rows:
            try:
                mine = self.bus is None or int(r[0].split(":")[1], 16) == self.bus
            except (IndexError, ValueError):
                mine = False
            if mine or len(buses) == 1:
                self.rows.append(r)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "error": self.err}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = sorted({self.REASONS[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------------------------------
# roofline bookkeeping: algorithmic work per launch of each instrumented kernel family
# ------------------------------------------------------------------------------------------
def algorithmic_work(name, wl, nS, nexc, nnz, n_emit, n_unique, net_flops, buckets=1,
                     launches=1, screened=False):
    """(bound, amount per launch, unit) - bytes for HBM-bound kernels, FLOP for GEMMs. With B
    PT2 buckets each sort and reduction launch handles one bucket: 1/B of the emitted pairs and
    unique terms; the emission runs once for all buckets or once per bucket (`launches` per
    step)."""
    kb = 4.0 if 2 * wl.norb <= 32 else (8.0 if 2 * wl.norb <= 64 else 16.0)  # PT2 key width
    if name == "pt2_emit" and not screened:  # write key+value per emission, read S and psi
        return "hbm", ((kb + 8.0) * n_emit + 24.0 * nS) / max(1, launches), "B"
    n_emit = n_emit / max(1, buckets)
    n_unique = n_unique / max(1, buckets)
    if name == "rs_scatter":   # read key+value, write key+value
        return "hbm", 2.0 * (kb + 8.0) * n_emit, "B"
    if name == "rs_hist":      # read keys
        return "hbm", kb * n_emit, "B"
    if name == "seg_reduce":   # read keys + values, write (sum, key) per run, read its run index
        return "hbm", (kb + 8.0) * n_emit + (kb + 12.0) * n_unique, "B"
    if name == "spmv":
        return "hbm", 12.0 * nnz + 8.0 * 3 * nS, "B"
    if name == "gemm":
        return "tensor", net_flops, "FLOP"
    # enumeration, probing, the CSR fill (decode + probe per hit), the screened traversal, LU and
    # the H_x'x' loop are issue-bound: no byte or FLOP roofline
    return "alu", 0.0, None


def kernel_traffic(name, wl, key="dram_bytes_per_launch"):
    """A figure of the committed ncu summary of one kernel (dram read+write bytes per launch by
    default), if the kernel source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", f"{name}_{wl}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip().split()[0]
    src = vals.get("source_file")
    sha = vals.get("source_sha256")
    tr = vals.get(key)
    if not (src and sha and tr):
        return None
    with open(os.path.join(ROOT, src), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != sha:
            return None
    return float(tr)


# ------------------------------------------------------------------------------------------
# the GPU arm
# ------------------------------------------------------------------------------------------
def run_nqs(args, ws, rank, local):
    import paper_2601_21310_b300.nqs as N
    from paper_2601_21310_b300 import build as B
    if rank == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = synth.WORKLOADS[args.workload]
    p = synth.make_problem(wl)
    dtype = N.NQS_MIXED if wl.mixed else N.NQS_FP64
    P = N.Problem(wl.norb, wl.nalpha, wl.nbeta, p.h, p.eri)
    S_host = torch.from_numpy(p.S.view(np.int64)).view(torch.uint64).pin_memory()
    dets = S_host.to(dev)
    params = N.net_tensors(p.net, dtype, device=dev)
    params_host = [t.cpu().pin_memory() for t in params]
    net = N.Net(P, params, dtype)
    nS = len(p.S)
    o_conn = N.opts(precision=dtype, validate=0)
    o_eg = N.opts(precision=dtype, validate=0)
    nexc_total = nS * synth_nexc(wl)
    buckets = args.buckets if args.buckets > 0 else 0  # 0: the library sizes the buckets
    o_pt = N.opts(precision=dtype, buckets=buckets, validate=0, eps_pt2=args.eps_pt2)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    grad = torch.empty(net.num_params(), dtype=net.grad_dtype(), device=dev)
    psi = torch.empty(nS, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev_phase = {"connections": [], "energy_grad": [], "pt2": [], "csr_free": []}

    def mark(record):
        if not record:
            return None
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def step(record=False):
        e0 = mark(record)
        csr = N.connections(P, dets, o_conn)
        e1 = mark(record)
        N.energy_grad(P, net, csr, dets, o=o_eg, out=out, grad=grad, psi=psi)
        e2 = mark(record)
        E = out[0].item()
        r = pt2_step(args, N, P, dets, psi, E, o_pt, csr)
        e3 = mark(record)
        info = dict(n_conn=csr.n_enumerated + r["n_emitted"], n_hss=csr.n_enumerated,
                    buckets=r.get("buckets", 0),
                    n_emit=r["n_emitted"], nnz=csr.nnz, n_unique=r["n_unique"], E=E,
                    ext=r["ext"], int=r["int"])
        csr.free_async()
        e4 = mark(record)
        if record:
            for k, (x, y) in zip(ev_phase, [(e0, e1), (e1, e2), (e2, e3), (e3, e4)]):
                ev_phase[k].append((x, y))
        return info

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # timed region 1: the step as a user runs it (no per-kernel instrumentation)
    launches0 = N.launch_count()
    times = []
    n_conn_total = 0
    sampler = ClockSampler(local)
    t_wall0 = time.perf_counter()
    with sampler:
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            info = step(record=True)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            n_conn_total += info["n_conn"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    launches = N.launch_count() - launches0
    phase_ms = {k: sum(x.elapsed_time(y) for x, y in v) / len(v) for k, v in ev_phase.items()}
    eg_ms = [x.elapsed_time(y) for x, y in ev_phase["energy_grad"]]
    grad_mixed = grad.clone()
    ms_step = sum(times) / len(times)
    total_ms = reduce_max_over_ranks(sum(times), dev)
    value = whole_job_rate(n_conn_total, total_ms, ws)

    # timed region 2: the same steps with every main kernel bracketed by CUDA events on its
    # launching stream (per-kernel times for the roofline; slightly slower steps)
    N.profile_reset()
    N.profile_enable(True)
    prof_times = []
    prof_steps = min(args.steps, 3)
    for _ in range(prof_steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        prof_times.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    N.profile_enable(False)
    prof = N.profile_read()
    ms_step_prof = sum(prof_times) / len(prof_times)

    # roofline of the dominant instrumented kernel
    peaks, peak_kind = load_peaks()
    net_flops_fwd = 2.0 * nS * (wl.hidden[0] * wl.hidden[1] + wl.hidden[1] * wl.norb * wl.nelec)
    total_gemm_flops = 3.0 * net_flops_fwd
    shares = {k: v[0] for k, v in prof.items() if v[1] > 0}
    nexc = synth_nexc(wl)

    def work(k):
        per_launch_flops = total_gemm_flops / max(1, prof[k][1] / prof_steps)
        return algorithmic_work(k, wl, nS, nexc, info["nnz"], info["n_emit"], info["n_unique"],
                                per_launch_flops, max(1, info["buckets"]),
                                max(1, prof[k][1] / prof_steps), args.eps_pt2 > 0)

    # the roofline is reported for the largest kernel with a byte or FLOP bound; the largest
    # kernel overall is named beside it when it is an issue-bound one
    top = max(shares, key=shares.get)
    measurable = [k for k in shares if work(k)[2] is not None]
    dom = max(measurable, key=shares.get) if measurable else top
    ms_dom, n_dom = prof[dom]
    bound, amount, unit = work(dom)
    avg_launch_s = ms_dom / n_dom / 1e3
    if unit == "B":
        achieved = amount / avg_launch_s / 1e9
        peak = peaks["hbm_gbs"]
        r_unit = "GB/s"
    else:
        achieved = amount / avg_launch_s / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1400.0)
        r_unit = "TFLOP/s"
    traffic = kernel_traffic(dom, wl.name)
    roofline = {"kernel": dom, "bound": bound, "achieved": round(achieved, 2), "peak": peak,
                "unit": r_unit, "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_per_launch": amount, "peak_source": peak_kind}
    if top != dom:
        # an issue-bound kernel: its roofline is the issue rate (one warp instruction per clock
        # per scheduler); the fraction of issue slots it used comes from its ncu summary
        roofline["largest_kernel"] = {
            "kernel": top, "bound": "alu",
            "share_of_step": round(shares[top] / sum(shares.values()), 4),
            "issue_slot_util": kernel_traffic(top, wl.name, "issue_slots_busy_frac")}
    kernels = {k: {"ms_per_step": round(v[0] / prof_steps, 4), "launches": v[1],
                   "share_of_step": round(v[0] / prof_steps / ms_step_prof, 4)}
               for k, v in prof.items() if v[1] > 0}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if wl.mixed else "f64",
        "data": "synthetic (seeded integrals, level-major S, random-init backflow MLP)",
        "config": {"workload": wl.name, "norb": wl.norb, "nalpha": wl.nalpha, "nbeta": wl.nbeta,
                   "n_S": nS, "mlp": [2 * wl.norb, *wl.hidden, wl.norb * wl.nelec],
                   "pt2_buckets": 0 if args.no_pt2 else info["buckets"],
                   "pt2_eps": args.eps_pt2,
                   "step": "connections + energy_grad" if args.no_pt2 else
                           "connections + energy_grad + pt2",
                   "l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"replicas{ws}"},
        "evals_per_s": 1e3 / (sum(eg_ms) / len(eg_ms)),
        "dets_evals_per_s": nS * 1e3 / (sum(eg_ms) / len(eg_ms)),
        "connections_per_step": info["n_conn"], "hss_nnz": info["nnz"],
        "pt2_unique": info["n_unique"], "E_S": info["E"], "dE_pt2_ext": info["ext"],
        "dE_pt2_int": info["int"], "wall_s": wall, "gpu_launches": launches,
        "roofline": roofline, "kernels": kernels, "ms_per_step_instrumented": ms_step_prof,
        "phase_ms": phase_ms,
        "clocks": sampler.summary(),
    }
    result["fp64_form"] = None if args.no_fp64_form else run_fp64_form(
        args, N, P, p, dets, dtype, out, grad_mixed, psi, info, stream)
    if result["fp64_form"]:
        result["speedup_mixed_over_fp64_form"] = (result["evals_per_s"] /
                                                  result["fp64_form"]["evals_per_s"])
    if not args.no_outer:
        result["outer_loop"] = run_outer_loop(args, N, P, net, dets, psi, dtype, stream)
    if not args.no_tensor_probe:
        result["tensor_roofline"] = run_tensor_probe(N, stream)
    if not args.no_e2e:
        result["e2e"] = run_e2e(args, N, P, net, params, params_host, S_host, dets, o_conn, o_eg,
                                o_pt, out, grad, psi, stream, ws)
    return result, p


def pt2_step(args, N, P, dets, psi, E, o_pt, csr):
    """The PT2 part of a step: over all of C minus S, or (eps_pt2 > 0) over the screened set,
    whose threshold refers to psi normalised over S."""
    if args.no_pt2:
        return dict(n_emitted=0, n_unique=0, ext=float("nan"), int=float("nan"))
    if args.eps_pt2 > 0:
        return N.pt2(P, dets, psi / torch.linalg.norm(psi), E, o=o_pt, hss=csr)
    return N.pt2(P, dets, psi, E, o=o_pt, hss=csr)


def run_fp64_form(args, N, P, p, dets, dtype, out_mixed, grad_mixed, psi_mixed, info_mixed,
                  stream):
    """The same evaluation in the plain FP64 form (FP64 parameters, FP64 GEMMs and LU): its
    E_S + gradient rate, and the mixed form's deviation from it (E_S, gradient, PT2)."""
    if dtype != N.NQS_MIXED:
        return None
    dev = dets.device
    net64 = N.Net(P, N.net_tensors(p.net, N.NQS_FP64, device=dev), N.NQS_FP64)
    o64 = N.opts(precision=N.NQS_FP64, validate=0)
    csr = N.connections(P, dets, N.opts(validate=0))
    out64 = torch.empty(4, dtype=torch.float64, device=dev)
    g64 = torch.empty(net64.num_params(), dtype=torch.float64, device=dev)
    psi64 = torch.empty(len(p.S), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    N.energy_grad(P, net64, csr, dets, o=o64, out=out64, grad=g64, psi=psi64)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    # about 30 s at most for the FP64 form (one evaluation takes ~20 s at 42 orbitals)
    reps = max(1, min(args.steps, int(30.0 / max(first_s, 1e-3))))
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        N.energy_grad(P, net64, csr, dets, o=o64, out=out64, grad=g64, psi=psi64)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    ms = sum(times) / len(times)
    # mixed-form results of the timed steps vs the FP64 form
    E64 = out64[0].item()
    r64 = (dict(ext=float("nan"), int=float("nan")) if args.no_pt2 else
           N.pt2(P, dets, psi64 / torch.linalg.norm(psi64), E64, hss=csr,
                 o=N.opts(validate=0, buckets=0, eps_pt2=args.eps_pt2)) if args.eps_pt2 > 0 else
           N.pt2(P, dets, psi64, E64, o=N.opts(validate=0, buckets=o_pt_buckets(args, p)),
                 hss=csr))
    csr.free()
    gm = grad_mixed.double()
    grel = (torch.linalg.norm(gm - g64) / torch.linalg.norm(g64)).item()
    return {"energy_grad_ms": ms, "evals_per_s": 1e3 / ms, "timed_evals": reps, "E_S": E64,
            "E_S_mixed_minus_fp64": info_mixed["E"] - E64,
            "grad_rel_l2_mixed_vs_fp64": grel,
            "dE_pt2_ext": r64["ext"], "dE_pt2_ext_mixed_minus_fp64": info_mixed["ext"] - r64["ext"],
            "dE_pt2_int_mixed_minus_fp64": info_mixed["int"] - r64["int"]}


def run_outer_loop(args, N, P, net, dets, psi, dtype, stream, eps_hb=1e-6):
    """Algorithm 1 steps 1 and 3 after the inner step: the heat-bath screened set P (Eq.
    hb_screen, eps_hb = 1e-6 as in Sec. 3.3, on psi normalised over S), amplitudes on
    T = S + P, and the Top-K selector back to |S| configurations. Each timed with CUDA events
    on the launching stream (median of the timed repetitions after one untimed run)."""
    nS = dets.shape[0]
    psi_n = psi / torch.linalg.norm(psi)
    o = N.opts(precision=dtype, validate=0)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts, r = [], None
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return sorted(ts)[len(ts) // 2], r

    reps = 3 if nS >= (1 << 20) else max(3, min(args.steps, 10))
    hb_ms, hb = timed(lambda: N.hb_select(P, dets, psi_n, eps_hb, o=o), reps)
    T = torch.cat([dets.view(torch.int64), hb["dets"].view(torch.int64)]).view(torch.uint64)
    amp_ms, (laT, _, _) = timed(lambda: N.amplitudes(P, net, T, o=o), reps)
    sel_ms, sel = timed(lambda: N.select(P, T, laT, N.SELECT_TOPK, K=nS, o=o), reps)
    kept_from_P = int((sel["index"] >= nS).sum().item())
    modes = run_modes(N, P, net, dets, T, nS, o, timed) if T.shape[0] <= MODES_MAX_T else {
        "skipped": f"|T| = {int(T.shape[0])} > {MODES_MAX_T}: the proxy Hamiltonian over T "
                   "(rows of S reach most of T) would hold billions of nonzeros"}
    return {"eps_hb": eps_hb, "n_P": int(hb["dets"].shape[0]), "n_T": int(T.shape[0]),
            "hb_pairs_kept": int(hb["n_emitted"]), "hb_candidates_tested": int(hb["n_examined"]),
            "hb_select_ms": hb_ms,
            "hb_candidates_per_s": hb["n_examined"] / (hb_ms * 1e-3),
            "amplitudes_T_ms": amp_ms, "amplitudes_T_dets_per_s": T.shape[0] / (amp_ms * 1e-3),
            "select_topk_ms": sel_ms, "select_K": nS, "kept_from_P": kept_from_P,
            "modes": modes}


def run_tensor_probe(N, stream, M=1 << 20, Nn=2016, K=1024, reps=10, mn=False):
    """The library's tcgen05 GEMM (nqs_gemm_bf16: bf16 in, FP32 out; 256-column tiles in the
    paired two-SM form) on the output-layer shape of the 42-orbital network (|S| = 2^20 rows,
    2016 outputs, width 1024), timed with CUDA events on the launching stream after warm-up.
    `achieved` is the best of `reps` single launches, each timed alone (the method of the
    measured burst peak: best of 10 timed launches), against that burst peak; `back_to_back`
    is the mean over `reps` launches in a row, which runs into the power cap, against the
    measured sustained peak. mn: both operands MN-major ([K][M] and [K][N], row-major
    activations as the weight gradients read them)."""
    if mn:
        A = torch.randn(K, M, device="cuda").to(torch.bfloat16)
        B = torch.randn(K, Nn, device="cuda").to(torch.bfloat16)
        gemm = lambda: N.gemm_bf16_ex(A, True, B, True)  # noqa: E731
    else:
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
        B = torch.randn(Nn, K, device="cuda").to(torch.bfloat16)
        gemm = lambda: N.gemm_bf16(A, B)  # noqa: E731
    for _ in range(3):
        gemm()
    torch.cuda.synchronize()
    flops = 2.0 * M * Nn * K
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    singles = []
    for a, b in ev:
        torch.cuda.synchronize()
        time.sleep(0.02)
        a.record(stream)
        gemm()
        b.record(stream)
        b.synchronize()
        singles.append(a.elapsed_time(b))
    a, b = ev[0]
    a.record(stream)
    for _ in range(reps):
        gemm()
    b.record(stream)
    b.synchronize()
    ms_b2b = a.elapsed_time(b) / reps
    ms = min(singles)
    tf = flops / (ms * 1e-3) / 1e12
    tf_b2b = flops / (ms_b2b * 1e-3) / 1e12
    peaks, kind = load_peaks()
    peak = peaks.get("bf16_tflops", 1800.0)
    peak_sus = peaks.get("bf16_tflops_sustained", 1400.0)
    del A, B
    torch.cuda.empty_cache()
    return {"kernel": "k_gemm_tc_pair", "shape": [M, Nn, K],
            "operands": "MN-major" if mn else "K-major", "bound": "tensor", "ms": ms,
            "ms_median_single": float(np.median(singles)),
            "achieved": round(tf, 1), "peak": peak, "unit": "TFLOP/s",
            "frac": round(tf / peak, 4), "peak_source": kind + " bf16 burst",
            "timing": f"best of {reps} single launches",
            "back_to_back": {"ms": ms_b2b, "achieved": round(tf_b2b, 1), "peak": peak_sus,
                             "frac": round(tf_b2b / peak_sus, 4),
                             "peak_source": kind + " bf16 sustained"}}


MODES_MAX_T = 4 << 20


def run_modes(N, P, net, dets, T, nS, o, timed):
    """The target-set modes of Sec. 2.4.1 on T = S + P and the E_diag diagnostic on S: proxy
    Hamiltonian build, E_proxy + gradient, E_asym + exact gradient, Lanczos lambda_min(H_SS)."""
    ph_ms, H = timed(lambda: N.proxy_hamiltonian(P, T, nS, o=o), 3)
    px_ms, (opx, _, _) = timed(lambda: N.energy_grad(P, net, H, T, o=o), 3)
    as_ms, (oas, _, _) = timed(lambda: N.asym_energy_grad(P, net, H, T, nS, True, o=o), 3)
    csr = N.connections(P, dets, o)
    lz_ms, (lam, iters) = timed(lambda: N.lanczos_min(csr, max_iters=300, tol=1e-12), 1)
    out, _, _ = N.energy_grad(P, net, csr, dets, o=o, with_grad=False)
    res = {"proxy_hamiltonian_ms": ph_ms, "proxy_nnz": int(H.nnz),
           "E_proxy": float(opx[0].item()), "proxy_energy_grad_ms": px_ms,
           "E_asym": float(oas[0].item()), "asym_exact_grad_ms": as_ms,
           "E_diag": lam, "lanczos_iters": iters, "lanczos_ms": lz_ms,
           "delta_opt": float(out[0].item()) - lam}
    csr.free()
    H.free()
    return res


def o_pt_buckets(args, p):
    return args.buckets if args.buckets > 0 else 0


def synth_nexc(wl):
    n, m = wl.nalpha, wl.norb - wl.nalpha
    c2 = lambda k: k * (k - 1) // 2  # noqa: E731
    return 2 * n * m + 2 * c2(n) * c2(m) + (n * m) ** 2


def run_e2e(args, N, P, net, params, params_host, S_host, dets, o_conn, o_eg, o_pt, out, grad,
            psi, stream, ws):
    """Same metric through the public API with host buffers: every step copies S and the
    parameters host->device and reads E, the gradient and the PT2 result back (up to 5 timed
    steps after up to 2 warm-up steps)."""
    grad_host = torch.empty(grad.shape, dtype=grad.dtype).pin_memory()
    out_host = torch.empty(4, dtype=torch.float64).pin_memory()
    h2d = S_host.numel() * 8 + sum(t.numel() * t.element_size() for t in params_host)
    d2h = 4 * 8 + grad.numel() * grad.element_size() + 4 * 8 + 2 * 8 * o_pt.buckets
    times, n_conn = [], 0
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dets.device)
    warm, steps = min(args.warmup, 2), min(args.steps, 5)
    for it in range(warm + steps):
        flush.zero_()  # same L2 hygiene as the device-timed steps (outside the events)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dets.copy_(S_host, non_blocking=True)
        for d, h in zip(params, params_host):
            d.copy_(h, non_blocking=True)
        csr = N.connections(P, dets, o_conn)
        N.energy_grad(P, net, csr, dets, o=o_eg, out=out, grad=grad, psi=psi)
        out_host.copy_(out, non_blocking=True)
        grad_host.copy_(grad, non_blocking=True)
        stream.synchronize()
        r = pt2_step(args, N, P, dets, psi, float(out_host[0]), o_pt, csr)
        n = csr.n_enumerated + r["n_emitted"]
        csr.free_async()
        b.record(stream)
        b.synchronize()
        if it >= warm:
            times.append(a.elapsed_time(b))
            n_conn += n
    total = reduce_max_over_ranks(sum(times), dets.device)
    return {"value": whole_job_rate(n_conn, total, ws), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": total / len(times), "steps": steps}


# ------------------------------------------------------------------------------------------
# CPU oracle (the reported baseline, and the reference arm)
# ------------------------------------------------------------------------------------------
def cpu_slices(nS: int, k: int):
    """Row blocks [0, k), [nS/2, nS/2 + k) and [nS - k, nS) of S: the bounded sample of the CPU
    oracle (the whole of S when 3k >= nS)."""
    if 3 * k >= nS:
        return [(0, nS)]
    m = nS // 2
    return [(0, k), (m, m + k), (nS - k, nS)]


def oracle_step(O, p, k, quant, with_pt2=True, eps=0.0, pt2_buckets=(0, 1), nb=64):
    """The oracle on the bounded sample of one step: H_SS rows of the three row blocks (lookups
    into all of S), E_S + gradient over the sample's own subspace, and PT2 over the sample's
    connected space for hash buckets {0, 1} of 64 (screened with eps on the sample's normalised
    amplitudes when eps > 0, like the GPU step). Returns the connections counted like the GPU
    step's (H_SS pairs resolved + PT2 pairs emitted) and the sample size."""
    wl = p.wl
    nexc = O.n_excitations(wl.norb, wl.nalpha, wl.nbeta)
    rows = cpu_slices(len(p.S), k)
    n = 0
    for a, b in rows:
        O.hss_rows(wl.norb, p.h, p.eri, p.S, a, b)
        n += (b - a) * nexc
    sample = np.concatenate([p.S[a:b] for a, b in rows])
    csr = O.hss(wl.norb, p.h, p.eri, sample)
    r = O.energy_grad(O.Net(p.net, quant=quant), sample, csr)
    if with_pt2:
        psi = r["psi"] / np.linalg.norm(r["psi"]) if eps > 0 else r["psi"]
        for bk in pt2_buckets:
            n += O.pt2(wl.norb, p.h, p.eri, sample, psi, r["E"], nb, bk, eps=eps)["n_emitted"]
    return n, len(sample)


def cpu_rows_per_block(p, budget_connections: float) -> int:
    """Rows per block so that one sample resolves about budget_connections H_SS pairs."""
    nexc = synth_nexc(p.wl)
    return int(max(1, min(4096, budget_connections // (3 * nexc))))


def cpu_baseline(p, eps, with_pt2=True):
    """The oracle as it stands on ~10-30 s of the step's work (the slices of oracle_step), with
    the full-step CPU time extrapolated from it by the number of configurations."""
    from oracle import oracle as O
    O.lib()
    k = cpu_rows_per_block(p, 3e7)
    t = time.perf_counter()
    n, ns = oracle_step(O, p, k, p.wl.mixed, with_pt2, eps)
    dt = time.perf_counter() - t
    what = "H_SS rows, E_S + gradient" + (", PT2 buckets {0, 1} of 64" if with_pt2 else "")
    return {"value": n / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"row blocks {cpu_slices(len(p.S), k)} of {len(p.S)} dets of S "
                      f"({ns} dets): {what} ({n} connections, {dt:.1f} s)",
            "extrapolated_full_step_s": dt * len(p.S) / ns}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    from oracle import oracle as O
    O.lib()
    wl = synth.WORKLOADS[args.workload]
    p = synth.make_problem(wl)
    eps = args.eps_pt2
    # each step a few seconds of oracle work, so that the whole run ends within minutes
    k = cpu_rows_per_block(p, 6e6)
    for _ in range(args.warmup):
        oracle_step(O, p, k, wl.mixed, True, eps)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.steps):
        n += oracle_step(O, p, k, wl.mixed, True, eps)[0]
    dt = time.perf_counter() - t0
    v = n / dt
    sample = (f"row blocks {cpu_slices(len(p.S), k)} of {len(p.S)} dets of S per step: H_SS rows, "
              "E_S + gradient, PT2 buckets {0, 1} of 64" + (f" (eps {eps})" if eps > 0 else ""))
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "norb": wl.norb, "nalpha": wl.nalpha, "n_S": len(p.S),
                       "mlp": [2 * wl.norb, *wl.hidden, wl.norb * wl.nelec], "pt2_eps": eps},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batched(args, ws, rank, local):
    """64 independent problems of uneven shape (norb 12-28, |S| 512-32768, width 128, BF16):
    E_S + gradient of every problem per step, timed as sequential launches on one stream, as the
    problems' pipelines on 16 side streams recorded in one CUDA graph, and in the grouped mode
    (one launch per stage over all problems, grouped tensor-core GEMMs with autotuned tile
    widths) recorded in one CUDA graph (the reported value)."""
    import paper_2601_21310_b300.nqs as N
    from paper_2601_21310_b300 import build as B
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wls = synth.batched_workloads(count=64)
    items = []
    for wl in wls:
        p = synth.make_problem(wl)
        P = N.Problem(wl.norb, wl.nalpha, wl.nbeta, p.h, p.eri)
        dets = torch.from_numpy(p.S.view(np.int64)).to(dev).view(torch.uint64)
        net = N.Net(P, N.net_tensors(p.net, N.NQS_MIXED, device=dev), N.NQS_MIXED)
        csr = N.connections(P, dets, N.opts(validate=0))
        out = torch.zeros(4, dtype=torch.float64, device=dev)
        grad = torch.zeros(net.num_params(), dtype=torch.float32, device=dev)
        items.append((P, net, csr, dets, out, grad))
    total_dets = sum(it[3].shape[0] for it in items)
    stream = torch.cuda.Stream(device=dev)
    N.set_autotune(True)
    with torch.cuda.stream(stream):
        for P, net, csr, dets, out, grad in items:
            N.energy_grad(P, net, csr, dets, out=out, grad=grad)
    N.set_autotune(False)
    torch.cuda.synchronize()
    batch = N.Batch(items, nstreams=16, mode=N.BATCH_STREAMS)
    grouped = N.Batch(items, nstreams=16, mode=N.BATCH_GROUPED)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            times = []
            for _ in range(args.steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b))
        return sum(times) / len(times)

    def sequential():
        for P, net, csr, dets, out, grad in items:
            N.energy_grad(P, net, csr, dets, out=out, grad=grad, stream=stream)

    ms_seq = timed(sequential)
    ms_conc = timed(lambda: batch.run(stream))
    batch.capture(stream)
    ms_streams_graph = timed(lambda: batch.launch(stream))
    N.set_autotune(True)  # the grouped mode tunes each GEMM stage's tile width on first use
    with torch.cuda.stream(stream):
        grouped.run(stream)
    N.set_autotune(False)
    ms_grouped_eager = timed(lambda: grouped.run(stream))
    k0 = N.launch_count()
    grouped.capture(stream)
    kernels_per_graph = N.launch_count() - k0  # kernel nodes recorded into the graph
    sampler = ClockSampler(local)
    with sampler:
        ms_graph = timed(lambda: grouped.launch(stream))
    n = len(items)
    return {
        "metric": "batched E_S+grad evals/s (64 independent problems) at 1 B300",
        "value": n * 1e3 / ms_graph, "unit": "evals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "batched_64", "problems": n, "total_dets": total_dets,
                   "norb_range": [min(w.norb for w in wls), max(w.norb for w in wls)],
                   "width": 128, "mode": "grouped (one launch per stage), CUDA graph",
                   "l2": "flushed between timed steps (512 MB write)"},
        "dets_evals_per_s": total_dets * 1e3 / ms_graph,
        "ms_per_step_sequential_launches": ms_seq,
        "ms_per_step_streams_eager": ms_conc,
        "ms_per_step_streams_graph": ms_streams_graph,
        "ms_per_step_grouped_eager": ms_grouped_eager,
        "speedup_grouped_graph_over_sequential": ms_seq / ms_graph,
        "speedup_grouped_graph_over_streams_graph": ms_streams_graph / ms_graph,
        "autotuned_gemm_shapes": len(N.autotune_entries()),
        "kernels_per_graph": kernels_per_graph,
        "gpu_launches": kernels_per_graph * args.steps,
        "clocks": sampler.summary(),
    }


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.workload == "batched":
        if rank == 0:
            print(json.dumps(run_batched(args, ws, rank, local)))
        return
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
        if res is not None:
            print(json.dumps(res))
        return
    if args.tensor_probe_only:
        M, Nn, K = (int(v) for v in args.tensor_probe_only.split(","))
        import paper_2601_21310_b300.nqs as N
        from paper_2601_21310_b300 import build as B
        B.build()
        print(json.dumps(run_tensor_probe(N, torch.cuda.current_stream(), M=M, Nn=Nn, K=K,
                                          mn=args.probe_mn)))
        return
    if ws > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    res, p = run_nqs(args, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(p, args.eps_pt2, not args.no_pt2)
        print(json.dumps(res))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
