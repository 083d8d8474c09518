#!/usr/bin/env python
"""Energy evaluations per second of the GB300 MPS-VQE hot path.

One step = one VQE energy evaluation: reset the MPS to the Hartree-Fock
state, apply the UCCSD-style circuit bound to a fresh theta, evaluate the
Jordan-Wigner Pauli-sum energy (trie of shared left environments), FP64 sum.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2|c1]
  python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)

Under torchrun each rank evaluates its own instance (independent fragments,
no collective on the data path: weak scaling); rank 0 prints one JSON line.
"""

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Concurrent evaluations run one stream each; the default of 8 hardware work
# queues would serialise streams beyond the eighth.  Read at CUDA context
# creation, so it is set before torch initialises CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

from paper_2303_03681_gb300.inputs import (MASTER_SEED, brickwork_circuit, hf_bits, jw_molecular_hamiltonian,  # noqa: E402
                                           make_rng, random_integrals, uccsd_template)
from paper_2303_03681_gb300.inputs.circuits import CircuitTemplate, uccsd_excitations  # noqa: E402

METRIC = "energy evals/s"
# accuracy target of an energy against the FP64 oracle (Ha)
ENERGY_TOL_HA = 1e-6
# derived ALU peaks (152 SMs x 2070 MHz): FP32 128 FMA/clk/SM, FP64 2 FMA/clk/SM
SM_COUNT, SM_MHZ = 152, 2070.0
ALU_PEAK_TFLOPS = {"f32": SM_COUNT * 128 * 2 * SM_MHZ * 1e6 / 1e12, "f64": SM_COUNT * 2 * 2 * SM_MHZ * 1e6 / 1e12}
# FP32 operations per flop of the double-float Jacobi sweeps (Knuth two-sum
# and fma two-product arithmetic: 144 FP32 operations for the 16 real flops
# of one stacked-column entry of a pair's Gram sums or of its rotation)
DF_OPS_PER_FLOP = 9


def build_workload(name, args, rank):
    """Seeded synthetic inputs of a named configuration."""
    if name == "c2":
        n_orb, n_e, chi = 25, 10, 128
        n_exc = args.excitations
        h, g = random_integrals(n_orb, make_rng(MASTER_SEED + 11))
        ham = jw_molecular_hamiltonian(h, g)
        tmpl = uccsd_template(2 * n_orb, n_e, max_excitations=n_exc)
        total_exc = len(uccsd_excitations(2 * n_orb, n_e))
        bits = hf_bits(2 * n_orb, n_e)
        desc = dict(workload=f"c2_uccsd_{2 * n_orb}q_chi{chi}_first{n_exc}exc",
                    n_qubits=2 * n_orb, chi_max=chi, n_terms=int(ham.n_terms),
                    excitations=f"first {n_exc} of {total_exc} (singles first)",
                    two_qubit_gates=int(tmpl.n_two_qubit), trunc_rel=args.trunc_rel,
                    hamiltonian="JW of random 25-orbital integrals, h~N(0,1), (pq|rs)~N(0,0.1^2) 8-fold",
                    theta="U[-0.05, 0.05] per excitation, new draw per step")
        return dict(ham=ham, tmpl=tmpl, bits=bits, chi=chi, trunc=args.trunc_rel, theta_scale=0.05,
                    precision=args.precision or "fp64", desc=desc)
    if name == "c1":
        h, g = random_integrals(6, make_rng(MASTER_SEED))
        ham = jw_molecular_hamiltonian(h, g)
        gl = brickwork_circuit(12, 8, make_rng(MASTER_SEED + 1))
        tmpl = CircuitTemplate.from_gates(gl)
        desc = dict(workload="c1_brickwork_12q_8layers_chi64", n_qubits=12, chi_max=64, n_terms=int(ham.n_terms),
                    two_qubit_gates=44, trunc_rel=0.0)
        return dict(ham=ham, tmpl=tmpl, bits=hf_bits(12, 6), chi=64, trunc=0.0, theta_scale=0.0,
                    precision=args.precision or "fp64", desc=desc)
    raise SystemExit(f"unknown workload {name}")


def max_over_ranks(seconds, dist, device=None):
    """The job's time: the slowest rank's (barrier-bracketed) timed region."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(seconds)
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps_per_rank, world, seconds):
    """Whole-job evals/s: every rank evaluates its own instance (weak scaling)."""
    return world * steps_per_rank / seconds


def rank_seed(rank):
    """Seed of rank r's angles: each rank evaluates a different instance."""
    return MASTER_SEED + 1000 * (rank + 1)


def thetas_for(w, count, seed):
    rng = make_rng(seed)
    n = max(1, w["tmpl"].n_params)
    return [rng.uniform(-w["theta_scale"], w["theta_scale"], n)[: w["tmpl"].n_params] for _ in range(count)]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        return False

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
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    d = os.path.join(ROOT, "paper_2303_03681_gb300", "csrc")
    hsh = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            hsh.update(open(os.path.join(d, f), "rb").read())
    return hsh.hexdigest()[:16]


def recorded_traffic(kind, workload):
    """DRAM bytes per launch from a committed ncu summary of the same kernel source, else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p))
    except ValueError:
        return None
    e = rec.get(f"{kind}:{workload}")
    if e and e.get("source_sha") == kernel_source_hash():
        return e.get("dram_bytes_per_launch")
    return None


# ---------------------------------------------------------------------------
# CPU oracle (bounded sample)
# ---------------------------------------------------------------------------

def oracle_sample(w, budget_gates_s=8.0, budget_terms_s=6.0, seed=0):
    """Times the FP64 oracle on the first gates of the step's circuit and on a
    sample of its Pauli terms; extrapolates one step linearly.  The sample's
    bond dimensions are those reached after its first gates, so the estimate is
    a lower bound on the oracle's time per step."""
    from oracle import mps as om

    theta = thetas_for(w, 1, seed)[0]
    gates = w["tmpl"].bind(theta)
    st = om.product_state(w["bits"])
    t0 = time.perf_counter()
    done = 0
    while done < gates.n_gates and time.perf_counter() - t0 < budget_gates_s:
        q = int(gates.q[done])
        if gates.arity[done] == 1:
            om.apply_1q(st, q, gates.u[done][:2, :2])
        else:
            om.apply_2q(st, q, gates.u[done], w["chi"], w["trunc"])
        done += 1
    t_g = time.perf_counter() - t0
    rng = make_rng(seed + 1)
    order = rng.permutation(w["ham"].n_terms)
    t0 = time.perf_counter()
    nt = 0
    while nt < order.size and time.perf_counter() - t0 < budget_terms_s:
        om.expect_pauli(st, w["ham"].ops[order[nt]])
        nt += 1
    t_t = time.perf_counter() - t0
    step_s = t_g / max(done, 1) * gates.n_gates + t_t / max(nt, 1) * w["ham"].n_terms
    sample = (f"oracle on the first {done} of {gates.n_gates} gates ({t_g:.1f} s, chi reached "
              f"{max(st.bond_dims())}) and {nt} of {w['ham'].n_terms} terms ({t_t:.1f} s), extrapolated linearly "
              f"to one step")
    return step_s, sample


def blas_threads():
    try:
        from threadpoolctl import threadpool_info

        return max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = build_workload(args.workload, args, 0)
    for _ in range(args.warmup):
        oracle_sample(w, 2.0, 1.0)
    times, sample = [], ""
    for k in range(args.steps):
        s, sample = oracle_sample(w, 8.0, 6.0, seed=k)
        times.append(s)
    step_s = float(np.mean(times))
    v = 1.0 / step_s
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": w["desc"],
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": blas_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2303_03681_gb300 import mps

    w = build_workload(args.workload, args, rank)
    svd_mode = {"fp32": 0, "fp64": 1, "fp64-all": 2}[args.svd]
    svd64 = svd_mode != 0
    B = args.batch
    main_stream = torch.cuda.current_stream()
    streams = [torch.cuda.Stream(device=dev) for _ in range(B)]
    ctxs = [mps.Context(local, stream=s) for s in streams]
    H = mps.Hamiltonian(ctxs[0], w["ham"])
    C = mps.Circuit(ctxs[0], w["tmpl"])
    states = [mps.State(c, w["tmpl"].n_qubits, w["bits"], chi_max=w["chi"], precision=w["precision"],
                        trunc_rel=w["trunc"], svd_fp64=svd_mode, tensor_cores=args.tensor_cores) for c in ctxs]
    n_steps = args.warmup + args.steps
    n_par = max(1, w["tmpl"].n_params)
    thetas = thetas_for(w, (n_steps + args.steps) * B, rank_seed(rank))
    th_dev = np.zeros((n_steps, B, n_par))
    for i in range(n_steps):
        for b in range(B):
            th_dev[i, b, :w["tmpl"].n_params] = thetas[i * B + b]
    d_theta = torch.tensor(th_dev, dtype=torch.float64, device=dev)
    d_energy = torch.zeros((n_steps, B), dtype=torch.float64, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def fork_join(fn):
        go = torch.cuda.Event()
        go.record(main_stream)
        for s in streams:
            s.wait_event(go)
        fn()
        for s in streams:
            done = torch.cuda.Event()
            done.record(s)
            main_stream.wait_event(done)

    def step(i):
        reqs = [(states[b], C, H, d_theta[i, b].data_ptr(), w["bits"]) for b in range(B)]
        fork_join(lambda: mps.vqe_eval_batch_async(reqs, d_energy[i].data_ptr()))

    for c in ctxs:
        c.profile(mps.KERNEL_KINDS)
    for i in range(args.warmup):
        flush.zero_()
        step(i)
    torch.cuda.synchronize()
    prof = merge_profiles([c.profile_read(reset=True) for c in ctxs])
    dominant = max(prof, key=lambda k: prof[k][2])
    for c in ctxs:
        c.profile([dominant])
    for c in ctxs:
        c.profile_read(reset=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps, outside the events
            events[k][0].record(main_stream)
            step(args.warmup + k)
            events[k][1].record(main_stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    reps = [s.report() for s in states]  # statistics of the last step
    step_ms = [a.elapsed_time(b) for a, b in events]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    kprof = merge_profiles([c.profile_read(reset=True) for c in ctxs])
    energies = d_energy.cpu().numpy()
    hbm_bytes = sum(c.bytes_allocated() for c in ctxs)

    # end to end through the C-ABI with host buffers: theta H2D, energies D2H
    e2e_times = []
    host_thetas = thetas[n_steps * B:]
    e2e_steps = min(args.steps, 3)  # the end-to-end rate needs no more samples than this
    for k in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, status = mps.vqe_eval_batch([(states[b], C, H, host_thetas[k * B + b], w["bits"]) for b in range(B)])
        e2e_times.append(time.perf_counter() - t0)
        # MPS_ENOTCONV still delivers the energy; it is counted in last_step_report
        assert all(s in (0, mps.MPS_ENOTCONV) for s in status), status
    e2e_s = max_over_ranks(sum(e2e_times), dist, dev)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = job_throughput(args.steps * B, world, total_s)
    launches_total = sum(v[0] for v in kprof.values())
    dom_launches, dom_timed, dom_ms = kprof[dominant]
    roofline = None
    if dom_timed:
        avg_s = dom_ms / 1e3 / dom_timed
        per_step = dom_timed / args.steps
        if dominant == "svd":
            # FP32 sweeps run on the FP32 FMA pipe; the FP64-accurate sweeps
            # of the mixed form (svd_mode 1) run in double-float on the same
            # pipe at DF_OPS_PER_FLOP FP32 operations per flop, those of the
            # all-FP64 form (svd_mode 2) on the FP64 units.  The roofline
            # time of a launch is the sum of both parts at their peaks.
            sw32 = sum(r["svd_sweeps_fp32"] for r in reps)
            sw64 = sum(r["svd_sweeps_fp64"] for r in reps)
            share = (sw64 / max(1, sw32 + sw64)) if svd64 else 0.0
            flops_per_launch = sum(r["svd_flops"] for r in reps) / max(1, sum(r["two_qubit_gates"] for r in reps))
            p32 = ALU_PEAK_TFLOPS["f32"]
            p64 = ALU_PEAK_TFLOPS["f64"] if svd_mode == 2 else p32 / DF_OPS_PER_FLOP
            ideal_s = ((1 - share) * flops_per_launch / p32 + share * flops_per_launch / p64) / 1e12
            achieved = flops_per_launch / avg_s / 1e12
            peak = flops_per_launch / max(ideal_s, 1e-30) / 1e12
            roofline = {"bound": "alu", "kernel": "svd (Jacobi, cluster or single CTA)", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": ideal_s / avg_s,
                        "traffic": recorded_traffic(dominant, w["desc"]["workload"]),
                        "avg_launch_us": avg_s * 1e6, "launches_per_step": per_step,
                        "peak_source": (f"derived: FP32 sweeps at the FP32 FMA peak ({SM_COUNT} SMs x 128 FMA/clk x "
                                        f"{SM_MHZ:.0f} MHz = {p32:.1f} TFLOP/s), FP64-accurate sweeps at "
                                        + (f"the FP64 peak ({p64:.2f} TFLOP/s)" if svd_mode == 2 else
                                           f"the double-float rate (FP32 peak / {DF_OPS_PER_FLOP} = {p64:.2f} TFLOP/s)")
                                        + f"; {100 * share:.0f} % of the sweeps FP64-accurate"),
                        "work": (f"Jacobi flops run per launch (sweeps x pairs x per-pair dot and rotation flops; "
                                 f"{sw32} FP32 and {sw64} FP64-accurate sweeps in the last step)"),
                        "aggregate_achieved": flops_per_launch * per_step / (total_s / args.steps) / 1e12}
        else:
            roofline = {"bound": "alu", "kernel": dominant, "achieved": None, "peak": None, "unit": "TFLOP/s",
                        "frac": None, "traffic": None, "avg_launch_us": avg_s * 1e6, "launches_per_step": per_step}
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128" if w["precision"] == "fp64" else "c64",
        "data": "synthetic",
        "config": dict(w["desc"], precision=({"fp32": "complex64 storage and contractions, ",
                                              "fp64": "complex128 storage, double-float contractions, ",
                                              "tf32x3": "complex64 storage, TF32x3 tensor-core contractions, ",
                                              "bf16x3": "complex64 storage, BF16x3 tensor-core contractions, ",
                                              "auto": "complex64 storage, TF32x3 contractions at capacity >= 256, "}
                                             [w["precision"]]
                                             + {"fp32": "FP32 Jacobi SVD",
                                                "fp64": ("FP64-accurate Jacobi SVD (FP32 sweeps, FP64 "
                                                         "re-orthonormalisation, double-float sweeps)"),
                                                "fp64-all": "FP64 Jacobi SVD"}[args.svd]
                                             + ", FP64 energy sum"),
                       contractions=contraction_label(args, w, reps),
                       batch=f"{B} concurrent evaluations per step (one stream each)",
                       l2="flushed between steps (256 MB write)", parallelism=f"replicas x{world}"),
        "e2e": {"value": job_throughput(e2e_steps * B, world, e2e_s), "unit": "evals/s", "steps": e2e_steps,
                "h2d_bytes_per_step": 8 * w["tmpl"].n_params * B, "d2h_bytes_per_step": 8 * B},
        "gpu_launches": int(launches_total),
        "roofline": roofline,
        "clocks": clocks.summary(),
        "kernel_time_share": {k: round(v[2] / max(1e-9, sum(x[2] for x in prof.values())), 4)
                              for k, v in prof.items() if v[2] > 0},
        "energies": [float(x) for x in energies[args.warmup, :min(B, 4)]],
        "last_step_report": {k: max(r[k] for r in reps) for k in ("max_chi", "discarded_weight", "svd_not_converged",
                                                                  "degenerate_cuts", "two_qubit_gates",
                                                                  "max_sweeps_used")},
        "hbm_bytes_allocated": hbm_bytes,
        "wall_s_timed_region": wall,
    }
    if not args.no_oracle_check:
        try:
            chk = oracle_check(mps, states[0], C, H, w, w["trunc"])
        except Exception as exc:  # an auxiliary field never costs the bench line
            chk = {"error": f"{type(exc).__name__}: {exc}"}
        if chk is not None:
            line["oracle_check"] = chk
    if args.serve_requests > 0:
        line["serving"] = serve_phase(mps, local, C, H, w, args, rate=0.9 * value / world)
    if not args.no_c1_phase:
        try:
            line["c1_gain_and_serving"] = c1_phase(mps, local, args)
        except Exception as exc:  # an auxiliary field never costs the bench line
            line["c1_gain_and_serving"] = {"error": f"{type(exc).__name__}: {exc}"}
    if args.contraction_chi > 0:
        try:
            line["contraction_roofline"] = [contraction_phase(mps, local, args.contraction_chi, precision=p)
                                            for p in ("tf32x3", "bf16x3")]
        except Exception as exc:  # an auxiliary field never costs the bench line
            line["contraction_roofline"] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and not args.no_cpu_baseline:
        step_s, sample = oracle_sample(w)
        line["cpu_baseline"] = {"value": 1.0 / step_s, "unit": "evals/s", "cores": blas_threads(), "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serve_phase(mps, device, C, H, w, args, rate):
    """Poisson-arriving requests (mean rate `rate`/s, about 90 % of the batched
    throughput) against a continuous-batching server with --batch slots."""
    srv = mps.Server(device, max_slots=args.batch)
    frag = srv.add_fragment(C, H, w["bits"], chi_max=w["chi"], precision=w["precision"], trunc_rel=w["trunc"],
                            svd_fp64={"fp32": 0, "fp64": 1, "fp64-all": 2}[args.svd], tensor_cores=args.tensor_cores)
    rng = make_rng(MASTER_SEED + 77)
    gaps = rng.exponential(1.0 / max(rate, 1e-6), args.serve_requests)
    thetas = thetas_for(w, args.serve_requests, MASTER_SEED + 78)
    t0 = time.perf_counter()
    tickets = []
    for k in range(args.serve_requests):
        target = t0 + float(np.sum(gaps[:k + 1]))
        delay = target - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(frag, thetas[k]))
    lat = []
    for t in tickets:
        e, l_ms = srv.poll(t, timeout_ms=-1)
        lat.append(l_ms)
    elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return {"requests": args.serve_requests, "arrival_rate_per_s": rate, "slots": args.batch,
            "throughput_evals_per_s": args.serve_requests / elapsed,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "hbm_peak_bytes": st["peak_bytes"]}


def c1_phase(mps, device, args, steps=20, batch=8, serve_requests=200):
    """The metric's comparison on the 12-qubit workload, where both forms can
    meet the 1e-6 Ha target: the plain FP32 single-instance MPS (complex64
    storage, FP32 CUDA-core contractions, FP64-accurate Jacobi SVD, one
    evaluation at a time on one stream) against the mixed-precision batched
    form (complex64 storage, TF32x3 tensor-core gate contractions, FP64 SVD and
    energy sum, `batch` evaluations overlapped on their own streams).  Each
    form's evaluations/s are timed on the device (CUDA events around the
    issued batch, warm-up first) and its energy at the stored oracle record's
    angles is compared with the record (tests/golden/c1_brickwork12_oracle.json).
    The gain is reported only when both meet 1e-6 Ha.  Then Poisson-arriving
    requests (rate 90 % of the batched throughput) go through the
    continuous-batching server in the mixed form: p50/p99 latency."""
    import torch

    w = build_workload("c1", args, 0)
    rec = json.load(open(os.path.join(ROOT, "tests", "golden", "c1_brickwork12_oracle.json")))
    dev = torch.device("cuda", device)
    out = {"workload": w["desc"]["workload"], "oracle_energy": rec["oracle_energy"]}
    forms = {"fp32_single": dict(precision="fp32", slots=1), "mixed_batched": dict(precision="tf32x3", slots=batch)}
    for name, f in forms.items():
        streams = [torch.cuda.Stream(device=dev) for _ in range(f["slots"])]
        ctxs = [mps.Context(device, stream=st) for st in streams]
        C, H = mps.Circuit(ctxs[0], w["tmpl"]), mps.Hamiltonian(ctxs[0], w["ham"])
        states = [mps.State(c, 12, w["bits"], chi_max=64, precision=f["precision"], trunc_rel=0.0, svd_fp64=1)
                  for c in ctxs]
        theta = np.zeros((max(1, w["tmpl"].n_params),))
        d_theta = torch.zeros((f["slots"], theta.size), dtype=torch.float64, device=dev)
        d_e = torch.zeros(f["slots"], dtype=torch.float64, device=dev)
        main = torch.cuda.current_stream(dev)

        def one_batch():
            go = torch.cuda.Event()
            go.record(main)
            for st in streams:
                st.wait_event(go)
            mps.vqe_eval_batch_async([(s_, C, H, d_theta[i].data_ptr(), w["bits"]) for i, s_ in enumerate(states)],
                                     d_e.data_ptr())
            for st in streams:
                done = torch.cuda.Event()
                done.record(st)
                main.wait_event(done)

        for _ in range(3):
            one_batch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        for _ in range(steps):
            one_batch()
        b.record(main)
        torch.cuda.synchronize()
        rate = steps * f["slots"] / (a.elapsed_time(b) * 1e-3)
        e, status = mps.vqe_eval_batch([(states[0], C, H, np.zeros(w["tmpl"].n_params), w["bits"])])
        err = abs(float(e[0]) - rec["oracle_energy"])
        out[name] = {"evals_per_s": rate, "streams": f["slots"], "precision": f["precision"], "abs_error_ha": err,
                     "within_tol": bool(status[0] == 0 and err <= ENERGY_TOL_HA)}
        for c in ctxs:
            c.close()
    if out["fp32_single"]["within_tol"] and out["mixed_batched"]["within_tol"]:
        out["gain_mixed_batched_over_fp32_single"] = out["mixed_batched"]["evals_per_s"] / out["fp32_single"]["evals_per_s"]
    # continuous-batching server, mixed form, Poisson arrivals
    ctx = mps.Context(device)
    C, H = mps.Circuit(ctx, w["tmpl"]), mps.Hamiltonian(ctx, w["ham"])
    srv = mps.Server(device, max_slots=batch)
    frag = srv.add_fragment(C, H, w["bits"], chi_max=64, precision="tf32x3", trunc_rel=0.0, svd_fp64=1)
    rate = 0.9 * out["mixed_batched"]["evals_per_s"]
    gaps = make_rng(MASTER_SEED + 77).exponential(1.0 / rate, serve_requests)
    t0 = time.perf_counter()
    tickets = []
    for k in range(serve_requests):
        delay = t0 + float(np.sum(gaps[:k + 1])) - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(frag, np.zeros(w["tmpl"].n_params)))
    lat, errs = [], []
    for t in tickets:
        e, l_ms = srv.poll(t, timeout_ms=-1)
        lat.append(l_ms)
        errs.append(abs(e - rec["oracle_energy"]))
    elapsed = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    ctx.close()
    out["serving"] = {"requests": serve_requests, "arrival_rate_per_s": rate, "slots": batch,
                      "throughput_evals_per_s": serve_requests / elapsed,
                      "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                      "max_abs_error_ha": float(max(errs)), "hbm_peak_bytes": stats["peak_bytes"]}
    return out


def contraction_phase(mps, device, chi=512, steps=20, warmup=3, precision="tf32x3"):
    """The theta contraction of the 100-qubit chi = 512 brickwork (2 chi = 1024
    rows, chi_m = 512, 1024 columns; random complex64 site tensors and a Haar
    SU(4) gate) through mps_contract_theta on the tensor cores, timed with CUDA
    events on the context stream with the L2 flushed before every launch.  The
    two launches of one contraction (operand split, TMA/tcgen05 GEMM) are
    timed together by the library's own CUDA events around them (the
    context's kernel profile); the whole API call, which also uploads the
    gate and the sizes, is reported beside it.  Roofline: algorithmic real
    flops 8 (2 chi) chi (2 chi) per contraction; the tensor cores execute
    three split products of each."""
    import torch

    from paper_2303_03681_gb300.inputs import haar_su4

    rng = make_rng(MASTER_SEED + 700)
    shape = (chi, 2, chi)
    bl = ((rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2 * chi)).astype(np.complex64)
    br = ((rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2 * chi)).astype(np.complex64)
    u = haar_su4(rng)
    dev = torch.device("cuda", device)
    dl, dr = torch.from_numpy(bl).to(dev), torch.from_numpy(br).to(dev)
    out = torch.empty((2 * chi, 2 * chi), dtype=torch.complex64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = mps.Context(device, stream=stream)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    ctx.profile(["theta"])
    times, call_times = [], []
    for k in range(warmup + steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mps.contract_theta(ctx, precision, chi, chi, chi, dl.data_ptr(), dr.data_ptr(), u, out.data_ptr())
            b.record(stream)
        stream.synchronize()
        launches, timed, ms = ctx.profile_read(reset=True)["theta"]
        if k >= warmup:
            call_times.append(a.elapsed_time(b) * 1e-3)
            times.append(ms * 1e-3 / max(timed, 1))
    t = float(np.median(times))
    alg = 8.0 * (2 * chi) * chi * (2 * chi)
    peaks = measured_peaks()
    dtype_peak = {"tf32x3": peaks["tf32"], "bf16x3": peaks["bf16"]}[precision]
    ctx.close()
    return {"shape": f"{2 * chi} x {chi} x {2 * chi} complex (theta of a chi={chi} bond)", "precision": precision,
            "median_us": t * 1e6, "call_median_us": float(np.median(call_times)) * 1e6,
            "launches": 2, "algorithmic_tflops": alg / t / 1e12,
            "executed_tflops": 3 * alg / t / 1e12, "dtype_peak_tflops": dtype_peak,
            "executed_frac": 3 * alg / t / 1e12 / dtype_peak, "algorithmic_frac": alg / t / 1e12 / dtype_peak,
            "peak_source": peaks["source"], "l2": "flushed before every launch (256 MB write)"}


def svd_study(mps, device, sizes=(128, 256, 512, 1024), reps=3):
    """The truncation SVD on its own against library SVDs on the same thetas
    (Results, "Speedup and Scaling": the paper's one-sided Jacobi against the
    vendor QR-based SVD).  For each 2 chi x 2 chi theta (complex128, graded
    spectrum over ten decades, seeded): this library's FP64-accurate Jacobi
    (mps_truncated_svd, svd_fp64 = 1, CUDA events on its stream), cuSOLVER
    through torch.linalg.svd on the GPU (a run-only comparator), and LAPACK
    zgesdd through numpy on the host (wall clock).  Singular values are
    checked against LAPACK's."""
    import torch

    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(device=dev)
    ctx = mps.Context(device, stream=stream)
    rows = []
    for n in sizes:
        rng = make_rng(MASTER_SEED + 800 + n)
        q1, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
        q2, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
        sv = 10.0 ** -np.linspace(0, 10, n)
        A = (q1 * sv) @ q2.conj().T
        A /= np.linalg.norm(A)
        dA = torch.from_numpy(A).to(dev)
        s_out = torch.empty(n, dtype=torch.float64, device=dev)
        vh = torch.empty((n // 2, n), dtype=torch.complex128, device=dev)
        ours, sweeps = [], None
        for r in range(reps + 1):
            with torch.cuda.stream(stream):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            k, rep, rc = mps.truncated_svd(ctx, "fp64", n, n, dA.data_ptr(), n // 2, 1e-8, 1, s_out.data_ptr(),
                                           vh.data_ptr())
            with torch.cuda.stream(stream):
                b.record(stream)
            stream.synchronize()
            if r:
                ours.append(a.elapsed_time(b) * 1e-3)
            sweeps = (rep["svd_sweeps_fp32"], rep["svd_sweeps_fp64"])
        s_ref = np.linalg.svd(A, compute_uv=False)
        err = float(np.max(np.abs(s_out.cpu().numpy()[:k] - s_ref[:k])))
        cusolver = []
        for r in range(reps + 1):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            torch.linalg.svd(dA, full_matrices=False)
            b.record()
            torch.cuda.synchronize()
            if r:
                cusolver.append(a.elapsed_time(b) * 1e-3)
        lapack = []
        for r in range(reps):
            t0 = time.perf_counter()
            np.linalg.svd(A, full_matrices=False)
            lapack.append(time.perf_counter() - t0)
        rows.append({"n": n, "ours_ms": 1e3 * min(ours), "cusolver_ms": 1e3 * min(cusolver),
                     "lapack_ms": 1e3 * min(lapack), "sweeps_fp32_fp64": sweeps, "kept": k,
                     "max_sv_error_vs_lapack": err})
    ctx.close()
    return {"what": "2chi x 2chi complex128 theta, graded spectrum (1 .. 1e-10), keep chi_max = chi at eps 1e-8",
            "ours": "FP64-accurate one-sided Jacobi (FP32 sweeps, FP64 sweeps) on a thread-block cluster",
            "cusolver": "torch.linalg.svd on the GPU (cuSOLVER, run-only comparator)",
            "lapack": f"numpy.linalg.svd on the host (zgesdd, {blas_threads()} threads)", "rows": rows}


def measured_peaks():
    """Tensor-core dtype peaks from MEASURED_PEAKS.json (measured BF16;
    TF32 = BF16 x the nominal dense ratio 1.1 / 2.25), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        rec = json.load(open(p))
        bf16, src = float(rec["bf16_tflops"]), "measured bf16 burst (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        bf16, src = 1900.0, "fallback bf16 1.9 PFLOP/s"
    return {"bf16": bf16, "tf32": bf16 * 1.1 / 2.25, "source": src + "; tf32 = bf16 x 1.1/2.25 (nominal ratio)"}


def contraction_label(args, w, reps):
    """What ran the contractions in the timed steps: the tensor-core
    environment path serves complex64 states at bond dimension >= 64 only, the
    split-product gate contractions the TF32X3 / BF16X3 / AUTO modes."""
    if w["precision"] == "fp64":
        return "CUDA cores (double-float on the FP32 units, complex128 in memory)"
    gates = {"fp32": "gates on CUDA cores (FP32)", "tf32x3": "gates on tcgen05 (TMA, TF32x3)",
             "bf16x3": "gates on tcgen05 (TMA, BF16x3)", "auto": "gates on tcgen05 (TMA, TF32x3) at capacity >= 256"}
    gates = gates[w["precision"]]
    if not args.tensor_cores and w["precision"] == "fp32":
        return gates + ", environments on CUDA cores (FP32)"
    top = max(r["max_chi"] for r in reps)
    if top < 64:
        return gates + f", environments on CUDA cores (FP32; the tcgen05 path needs bond dimension >= 64, max {top})"
    return gates + ", environments on tcgen05 (TF32 hi/lo, 4 products) at bond dimension >= 64"


def oracle_check(mps, state, C, H, w, trunc_rel):
    """|E_gpu - E_oracle| for this workload at the reference angles of a
    stored oracle energy (tests/golden/*_oracle.json, written by a committed
    script that runs only the oracle), or None when no record matches."""
    import glob

    for path in sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "*_oracle.json"))):
        rec = json.load(open(path))
        if rec.get("workload") != w["desc"]["workload"] or rec.get("trunc_rel") != trunc_rel:
            continue
        lo, hi = rec["theta_range"]
        theta = make_rng(rec["theta_seed"]).uniform(lo, hi, w["tmpl"].n_params)
        e, status = mps.vqe_eval_batch([(state, C, H, theta, w["bits"])])
        if status[0] not in (0, mps.MPS_ENOTCONV):
            return {"error": f"status {int(status[0])}"}
        err = abs(float(e[0]) - rec["oracle_energy"])
        rep = state.report()
        return {"reference": os.path.relpath(path, ROOT), "theta_seed": rec["theta_seed"],
                "energy_gpu": float(e[0]), "energy_oracle": rec["oracle_energy"],
                "abs_error_ha": err, "tolerance_ha": ENERGY_TOL_HA, "within_tol": bool(err <= ENERGY_TOL_HA),
                "svd_not_converged": int(rep["svd_not_converged"]),
                "discarded_weight_gpu": rep["discarded_weight"],
                "discarded_weight_oracle": rec["oracle_discarded_weight"]}
    return None


def merge_profiles(profs):
    out = {}
    for p in profs:
        for k, (a, b, ms) in p.items():
            x = out.get(k, (0, 0, 0.0))
            out[k] = (x[0] + a, x[1] + b, x[2] + ms)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--excitations", type=int, default=100)
    ap.add_argument("--trunc-rel", type=float, default=1e-5)
    ap.add_argument("--precision", choices=["fp32", "fp64", "tf32x3", "bf16x3", "auto"], default=None)
    ap.add_argument("--svd", choices=["fp32", "fp64", "fp64-all"], default="fp64",
                    help="Jacobi SVD: fp64 = FP64-accurate (complex64 states: FP32 sweeps, then FP64 ones), "
                         "fp64-all = every sweep in FP64, fp32 = FP32 sweeps only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the extra evaluation at the stored oracle energy's reference angles")
    ap.add_argument("--batch", type=int, default=32, help="concurrent evaluations per step")
    ap.add_argument("--tensor-cores", type=int, choices=[0, 1], default=1,
                    help="complex64 environment contractions on tcgen05 (1) or CUDA cores (0)")
    ap.add_argument("--contraction-chi", type=int, default=512,
                    help="after the timed steps, time the tensor-core theta contraction at this bond dimension "
                         "(0: skip)")
    ap.add_argument("--no-c1-phase", action="store_true",
                    help="skip the 12-qubit comparison (FP32 single vs mixed batched) and its serving run")
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="after the timed steps, serve this many Poisson-arriving requests (p50/p99 latency)")
    ap.add_argument("--svd-study", action="store_true",
                    help="time the truncation SVD against cuSOLVER and LAPACK at 2chi = 128 .. 1024 and exit")
    args = ap.parse_args()
    if args.svd_study:
        import torch

        from paper_2303_03681_gb300 import mps

        torch.cuda.set_device(0)
        print(json.dumps({"svd_study": svd_study(mps, 0)}), flush=True)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
