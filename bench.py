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
    for k in range(args.steps):
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
            dt = "f64" if svd64 else "f32"
            # the bound is the FP64 units when any sweep runs in FP64: count the FP64 sweeps' share of the flops
            sw32 = sum(r["svd_sweeps_fp32"] for r in reps)
            sw64 = sum(r["svd_sweeps_fp64"] for r in reps)
            share = (sw64 / max(1, sw32 + sw64)) if svd64 else 1.0
            flops_per_launch = share * sum(r["svd_flops"] for r in reps) / max(1, sum(r["two_qubit_gates"] for r in reps))
            achieved = flops_per_launch / avg_s / 1e12
            peak = ALU_PEAK_TFLOPS[dt]
            roofline = {"bound": "alu", "kernel": "svd (Jacobi, cluster or single CTA)", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "traffic": recorded_traffic(dominant, w["desc"]["workload"]),
                        "avg_launch_us": avg_s * 1e6, "launches_per_step": per_step,
                        "peak_source": f"derived {dt.upper()} ALU peak: {SM_COUNT} SMs x "
                                       f"{'128' if dt == 'f32' else '2'} FMA/clk x {SM_MHZ:.0f} MHz",
                        "work": (f"{dt.upper()} Jacobi flops run per launch (sweeps x pairs x per-pair dot and "
                                 f"rotation flops; {sw32} FP32 and {sw64} FP64 sweeps in the last step)"),
                        "aggregate_achieved": flops_per_launch * per_step / (total_s / args.steps) / 1e12}
        else:
            roofline = {"bound": "alu", "kernel": dominant, "achieved": None, "peak": None, "unit": "TFLOP/s",
                        "frac": None, "traffic": None, "avg_launch_us": avg_s * 1e6, "launches_per_step": per_step}
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64" if w["precision"] == "fp32" else "c128",
        "data": "synthetic",
        "config": dict(w["desc"], precision=({"fp32": "complex64", "fp64": "complex128"}[w["precision"]]
                                             + " storage and contractions, "
                                             + {"fp32": "FP32 Jacobi SVD",
                                                "fp64": ("FP64-accurate Jacobi SVD (FP32 sweeps, FP64 "
                                                         "re-orthonormalisation, FP64 sweeps)"),
                                                "fp64-all": "FP64 Jacobi SVD"}[args.svd]
                                             + ", FP64 energy sum"),
                       contractions=contraction_label(args, w, reps),
                       batch=f"{B} concurrent evaluations per step (one stream each)",
                       l2="flushed between steps (256 MB write)", parallelism=f"replicas x{world}"),
        "e2e": {"value": job_throughput(args.steps * B, world, e2e_s), "unit": "evals/s",
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


def contraction_label(args, w, reps):
    """What ran the environment contractions in the timed steps: the
    tensor-core path serves complex64 states at bond dimension >= 64 only."""
    if w["precision"] != "fp32":
        return "CUDA cores (FP64)"
    if not args.tensor_cores:
        return "CUDA cores (FP32)"
    top = max(r["max_chi"] for r in reps)
    if top < 64:
        return f"CUDA cores (FP32); tcgen05 enabled but unused (bond dimension {top} < 64)"
    return "tcgen05 TF32 hi/lo split, 4 products, at bond dimension >= 64; CUDA cores (FP32) below"


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
    ap.add_argument("--precision", choices=["fp32", "fp64"], default=None)
    ap.add_argument("--svd", choices=["fp32", "fp64", "fp64-all"], default="fp64",
                    help="Jacobi SVD: fp64 = FP64-accurate (complex64 states: FP32 sweeps, then FP64 ones), "
                         "fp64-all = every sweep in FP64, fp32 = FP32 sweeps only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the extra evaluation at the stored oracle energy's reference angles")
    ap.add_argument("--batch", type=int, default=8, help="concurrent evaluations per step")
    ap.add_argument("--tensor-cores", type=int, choices=[0, 1], default=1,
                    help="complex64 environment contractions on tcgen05 (1) or CUDA cores (0)")
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="after the timed steps, serve this many Poisson-arriving requests (p50/p99 latency)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
