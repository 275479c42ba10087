"""Benchmark of the MPS-VQE hot path on GB300 (one JSON line on stdout).

Workload (the 24-qubit configuration): 12 spatial orbitals / 24 qubits, 12
electrons, seeded random 8-fold-symmetric integrals (29 737 Jordan-Wigner Pauli
strings), UCCSD with 1818 excitations (14 112 Pauli rotations, 442 272 two-site
gates), bond cap chi = 64, mixed precision. A step is one energy evaluation
(reset to Hartree-Fock, apply the whole circuit, evaluate every string, FP64
compensated sum) with its own seeded theta, nothing skipped.

One evaluation is a strictly serial chain of 442 272 truncated SVDs, so it runs on
one SM. The K timed steps are therefore issued together, as one vqe_energy_batch
call over K slots (one thread block, i.e. one SM, per evaluation), the way the
serving loop runs independent requests; the W warm-up steps likewise. Each step's
latency is the whole call; the throughput is K over it.

  value  energy evaluations per second with inputs resident on the device, from
         CUDA events recorded by the library on its stream around its kernels
  e2e    the same metric through the C ABI call with host buffers (thetas from
         pinned host memory uploaded, energies read back inside the timed region),
         from host wall-clock time

`--impl reference` times the CPU oracle (the plain NumPy truncated-MPS code) on a
bounded, stratified sample of the same workload instead.
"""
import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS, N_ELEC, CHI, SEED = 24, 12, 64, 0
WORKLOAD = {"workload": "uccsd_24q_12e_chi64_single_eval", "qubits": N_QUBITS, "electrons": N_ELEC,
            "chi": CHI, "pauli_terms": 29737, "two_site_gates": 442272, "integral_seed": SEED,
            "theta_seed": SEED, "evals_per_call": 1}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--serve", action="store_true",
                    help="serving stream: Poisson arrivals of mixed energy/gradient requests")
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--profile-case", action="store_true",
                    help="small profiling case: 256 gates on a saturated chi=64 state + one measurement")
    ap.add_argument("--config4", action="store_true",
                    help="measurement-bound configuration: <H> of a 64-qubit chi=256 MPS, every JW string")
    ap.add_argument("--config4-tc-case", action="store_true",
                    help="small profiling case of the tensor-core GEMM: one 64-qubit chi=256 measurement of "
                         "the first --case-strings strings")
    ap.add_argument("--tc-gemm-case", action="store_true",
                    help="small profiling case: one environment-shaped tensor-core GEMM through the C ABI")
    ap.add_argument("--config3", action="store_true",
                    help="256 parameter-shift circuits of a 32-qubit chi=128 ansatz per step (one gradient)")
    ap.add_argument("--random-gates", action="store_true",
                    help="second workload: random two-site gates in brickwork order on a random chi=128 MPS")
    ap.add_argument("--circuit", default="cancel-ladders", choices=["canonical", "cancel-ladders"],
                    help="gate list of the headline workload: the ladder-cancelling compile (default: the "
                         "commuting rotations of each excitation ordered so that the CNOT ladders of "
                         "consecutive ones cancel; same unitary, 252 095 gates) or the canonical compile "
                         "(442 272 gates)")
    ap.add_argument("--case-strings", type=int, default=2000)
    ap.add_argument("--case-budget-mb", type=int, default=0,
                    help="measurement buffer budget of the tensor-core case (0: the library default)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def start(self):
        def run():
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=10).stdout.strip()
                    if out:
                        self.rows.append([c.strip() for c in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=15)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) > 8:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ inputs
def inputs():
    from paper_2207_03711_gb300 import synthetic as syn
    h, g = syn.random_integrals(N_QUBITS // 2, SEED)
    return h, g


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(h, g, budget_s=20.0):
    """Time the oracle (plain NumPy c2) on a stratified sample and extrapolate to one
    evaluation: gates from the start of the circuit (growing ranks, from the
    Hartree-Fock state) and gates from the saturated regime (a random canonical
    chi = 64 MPS), plus a sample of Pauli strings on the saturated state."""
    from oracle import circuit, mps, pauli, ucc
    from paper_2207_03711_gb300 import synthetic as syn
    rc, rp, rs, exc = ucc.uccsd_rotations(N_QUBITS, N_ELEC)
    theta = syn.random_amplitudes(len(exc), SEED)
    gates = []          # compile only as far as the sample reaches
    for code, e, sc in zip(rc, rp, rs):
        gates += circuit.two_site_gates(code, sc * theta[e], N_QUBITS)
        if len(gates) >= 30400:
            break
    n_gates = 442272
    # start of the circuit: ranks grow from 1 (the first 20 000 gates reach the cap)
    st = mps.hf_mps(N_QUBITS, N_ELEC)
    t0 = time.perf_counter()
    n_lo = 0
    while n_lo < 2000 and time.perf_counter() - t0 < budget_s * 0.3:
        b, O = gates[n_lo]
        mps.apply_two_site(st, b, O, CHI)
        n_lo += 1
    t_lo = (time.perf_counter() - t0) / n_lo
    # saturated regime: consecutive gates of the circuit's interior on a chi = 64 MPS
    r = syn.full_ranks(N_QUBITS, CHI)
    st = mps.random_canonical(N_QUBITS, r, syn.random_mps_gaussians(N_QUBITS, r, 0))
    t0 = time.perf_counter()
    n_hi = 0
    while n_hi < 400 and time.perf_counter() - t0 < budget_s * 0.5:
        b, O = gates[30000 + n_hi]
        mps.apply_two_site(st, b, O, CHI)
        n_hi += 1
    t_hi = (time.perf_counter() - t0) / n_hi
    # measurement: a sample of strings, plain left-to-right contraction
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    idx = np.random.default_rng(0).choice(len(codes), 60, replace=False)
    t0 = time.perf_counter()
    for i in idx:
        mps.expect_string(st, codes[i])
    t_term = (time.perf_counter() - t0) / len(idx)
    n_sat = max(0, n_gates - 20000)
    est = min(20000, n_gates) * t_lo + n_sat * t_hi + len(codes) * t_term
    sample = (f"{n_lo} gates from the Hartree-Fock start ({t_lo * 1e3:.2f} ms/gate) x 20000 + {n_hi} "
              f"saturated chi=64 gates ({t_hi * 1e3:.2f} ms/gate) x {n_sat} + 60 Pauli strings "
              f"({t_term * 1e3:.2f} ms/string) x {len(codes)}; extrapolated to one evaluation of the "
              f"oracle's canonical gate list")
    return 1.0 / est, sample, est


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        return max(int(i.get("num_threads", 1)) for i in threadpool_info()) or 1
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


# ------------------------------------------------------------------ reference arm
def oracle_small_eval():
    """One complete oracle evaluation of the 8-qubit, 4-electron, chi = 16 case (the
    small configuration, exactly representable), timed end to end on the host: a
    measured oracle rate beside the extrapolated 24-qubit one."""
    from oracle import circuit, mps, pauli, ucc
    from paper_2207_03711_gb300 import synthetic as syn
    n, ne, chi = 8, 4, 16
    h, g = syn.random_integrals(n // 2, SEED)
    t0 = time.perf_counter()
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    th = syn.random_amplitudes(len(exc), SEED)
    st = mps.hf_mps(n, ne)
    mps.apply_gates(st, circuit.compile_circuit(rc, rp, rs, th, n), chi)
    e, _ = mps.energy(st, codes, coeffs)
    dt = time.perf_counter() - t0
    return {"workload": "uccsd_8q_4e_chi16_single_eval", "evals_per_s": 1.0 / dt, "seconds": dt,
            "kind": "oracle", "energy_Ha": e, "pauli_terms": len(codes)}


def run_reference(args):
    """The oracle arm: each step times the oracle on a bounded, stratified sample of
    one 24-qubit evaluation (see oracle_sample) and converts it to evaluations per
    second by the extrapolation written there; ms_per_step is the measured wall time
    of a sample step, evals_per_step the fraction of an evaluation it stands for."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    h, g = inputs()
    vals, steps_s, fracs = [], [], []
    sample = ""
    budget = min(20.0, 150.0 / max(1, args.warmup + args.steps))
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, sample, est = oracle_sample(h, g, budget_s=budget)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(v)
            steps_s.append(dt)
            fracs.append(dt / est)
    value = float(np.mean(vals))
    cores = threads_used()
    line = {"impl": "reference", "metric": "VQE energy evals/s", "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(steps_s)), "evals_per_step": float(np.mean(fracs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, circuit="canonical gate list (the oracle as it stands; the same unitary as "
                                             "the ladder-cancelling compile of the other arm)"),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle-extrapolated",
                             "estimate": True, "sample": sample},
            "oracle_full_small": oracle_small_eval(),
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def accuracy_probe(G, cancel_ladders=False):
    """|dE| of both precisions on the exactly representable cases (8 qubits at chi = 16,
    10 qubits at chi = 32: the bond caps hold the state without truncation), against the
    FP64 oracle energies stored in tests/golden/exact_energies.json by the committed
    script beside it (the benchmark does not run the oracle here). cancel_ladders: the
    same through the ladder-cancelling gate list."""
    from paper_2207_03711_gb300 import synthetic as syn
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", "exact_energies.json")))
    out = {}
    for case in ref["cases"]:
        n, ne, chi = case["qubits"], case["electrons"], case["chi"]
        h, g = syn.random_integrals(n // 2, case["integral_seed"])
        H = G.ham_jw_from_integrals(h, g)
        C = G.circ_uccsd(n, ne)
        if cancel_ladders:
            G.circ_cancel_ladders(C)
        th = syn.random_amplitudes(C.n_params, case["theta_seed"])
        for name, prec in (("fp64", G.MPS_FP64), ("mixed", G.MPS_MIXED)):
            M = G.mps_create(n, chi, prec)
            out[f"abs_dE_Ha_{name}_{n}q"] = abs(G.vqe_energy(M, C, H, th) - case["energy_mps_Ha"])
            M.close()
    out["cases"] = ("8 qubits/4 electrons/chi 16 and 10 qubits/4 electrons/chi 32 (untruncated), vs the FP64 "
                    "oracle energies in tests/golden/exact_energies.json")
    return out


def alu_peaks(torch):
    """Measured CUDA-core peaks of this GPU, in this process: cuBLAS SGEMM and DGEMM at
    8192^3 with TF32 disabled (best of 5, CUDA events). The gate engine runs on the
    FP32 pipes, so SGEMM is its roofline denominator."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    try:
        for name, dt, n, reps in (("fp32", torch.float32, 8192, 5), ("fp64", torch.float64, 4096, 3)):
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            torch.matmul(a, b)
            best = 1e30
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) * 1e-3)
            out[name + "_tflops"] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "cuBLAS SGEMM 8192^3 and DGEMM 4096^3 (TF32 off), best of 5/3, CUDA events, this process"
    return out


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over the process group (the slowest
    rank sets the step time of a replicated run)."""
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_rate(world, evals_per_rank, seconds):
    """Whole-job evaluations per second: every rank ran evals_per_rank evaluations and
    the slowest rank took `seconds`."""
    return world * evals_per_rank / seconds


def run_ours(args):
    import torch
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    G.build()
    G.load_library()
    h, g = inputs()
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(N_QUBITS, N_ELEC)
    cancel = args.circuit == "cancel-ladders"
    if cancel:
        G.circ_cancel_ladders(C)
    n_gates = G.circ_num_gates(C)
    stream = torch.cuda.current_stream().cuda_stream
    K, W = args.steps, max(3, args.warmup)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if K > n_sm:
        raise SystemExit(f"--steps {K} exceeds the {n_sm} SMs: the timed steps run side by side, one SM each")
    M = G.mps_create(N_QUBITS, CHI, G.MPS_MIXED, n_slots=max(K, W), cuda_stream=stream)
    # thetas of the timed steps in pinned host memory (uploaded inside the timed call)
    th_pinned = torch.empty((K, C.n_params), dtype=torch.float64, pin_memory=True)
    th_host = th_pinned.numpy()
    th_host[:] = np.stack([syn.random_amplitudes(C.n_params, SEED + 1000 * rank + i) for i in range(K)])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2
    # warm-up: W evaluations issued together (also uploads the gate list and the trie)
    tw0 = time.perf_counter()
    G.vqe_energy_batch(M, C, H, np.stack([syn.random_amplitudes(C.n_params, 100 + i) for i in range(W)]),
                       allow_noconv=True)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - tw0
    flush.fill_(1.0)          # L2 flushed before the timed call (outside the timing)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    t0 = time.perf_counter()
    energies = G.vqe_energy_batch(M, C, H, th_host, allow_noconv=True)
    t1 = time.perf_counter()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if rank == 0 else {}
    s = G.mps_get_stats(M)
    dev_s = (s["ms_circuit"] + s["ms_measure"]) * 1e-3
    wall_s = t1 - t0
    circ_s = s["ms_circuit"] * 1e-3
    flops = s["alg_flops_call"]
    if dist:
        dev_s, wall_s, circ_s = max_over_ranks([dev_s, wall_s, circ_s], dist, "cuda")
        if rank != 0:
            dist.destroy_process_group()
            return
    peaks = alu_peaks(torch)
    # dominant kernel: the gate engine on the FP32 pipes, K thread blocks (one SM each)
    achieved = flops / circ_s / 1e12
    peak = peaks["fp32_tflops"]
    n_launch = (n_gates + 16383) // 16384
    value = replica_rate(world, K, dev_s)
    cpu_val, cpu_sample, _ = oracle_sample(h, g)
    line = {
        "metric": "VQE energy evals/s", "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * dev_s / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": dict(WORKLOAD, precision="mixed (complex64 tensors, FP32 SVD, FP64 lambda and sums)",
                       two_site_gates=n_gates, two_site_gates_canonical=442272,
                       circuit=("canonical gate list" if not cancel else
                                "ladder-cancelling compile of the same UCCSD circuit (circ_cancel_ladders): "
                                "the commuting rotations of each excitation reordered, CNOT pairs that meet "
                                "cancelled; same unitary"),
                       l2="flushed (512 MB write) before the timed call; the K steps run in that one call",
                       steps_in_flight=K,
                       warmup=f"{W} evaluations issued together, {t_warm:.1f} s wall"),
        "pauli_terms_per_s": value * 29737,
        "latency_s": {"p50": dev_s, "p99": dev_s,
                      "note": "every step is in flight for the whole call and ends with it"},
        "e2e": {"value": replica_rate(world, K, wall_s), "unit": "evals/s",
                "h2d_bytes_per_step": 8 * C.n_params + N_QUBITS, "d2h_bytes_per_step": 8},
        "gpu_launches": int(s["kernel_launches"]),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "measured: cuBLAS SGEMM in this process (FP32 CUDA cores)",
                     "kernel": "k_circuit<float,512>", "launches_per_step": n_launch,
                     "sms_busy": K * world,
                     "frac_of_busy_sms": achieved / (peak * K / n_sm),
                     "note": "achieved = algorithmic flops of all K evaluations' gate steps / circuit CUDA-event "
                             "time; traffic null until an ncu capture of the current kernel exists"},
        "alu_peaks_measured": peaks,
        "cpu_baseline": {"value": cpu_val, "unit": "evals/s", "cores": threads_used(),
                         "kind": "oracle-extrapolated", "estimate": True, "sample": cpu_sample},
        "oracle_full_small": oracle_small_eval(),
        "clocks": clocks,
        "energy_Ha": {"min": float(np.min(energies)), "max": float(np.max(energies))},
        "breakdown_ms": {"circuit": s["ms_circuit"], "measure": s["ms_measure"]},
        "svd_fallbacks_slot0": int(s["n_fallback"]),
        "svd_noconv": int(s["n_svd_noconv"]),
        "discarded_weight_slot0": s["discarded_weight"],
        "accuracy": accuracy_probe(G, cancel),
    }
    acc = line["accuracy"]
    line["accuracy_Ha"] = max(acc["abs_dE_Ha_mixed_8q"], acc["abs_dE_Ha_mixed_10q"])
    print(json.dumps(line))


C4_N, C4_CHI, C4_ORB = 64, 256, 32


def config4_inputs(G, syn, n_strings=None):
    """64 qubits / 32 spatial orbitals, seeded random integrals; every Jordan-Wigner
    string (or the first n_strings in trie order); a seeded random right-canonical MPS
    with every interior rank at min(256, 2^min(k+1, n-1-k)) (timing input: its lambda are
    not its Schmidt numbers, which the measurement does not use)."""
    h, g = syn.random_integrals(C4_ORB, SEED)
    t0 = time.perf_counter()
    H = G.ham_jw_from_integrals(h, g)
    t_jw = time.perf_counter() - t0
    if n_strings is not None:
        P, c = G.ham_get_terms(H)
        H.close()
        H = G.ham_create(P[:n_strings], c[:n_strings])
    B, lam = syn.random_right_canonical_mps(C4_N, C4_CHI, 0)
    return H, B, lam, t_jw


def tc_peak_tflops():
    """Dense TF32 tensor peak for the roofline of the compensated-TF32 GEMM: the measured
    burst BF16 figure of this pool times the nominal TF32 : BF16 ratio (1.1 : 2.25)."""
    pk = measured_peaks()
    bf16 = pk.get("bf16_tflops")
    if bf16:
        return bf16 * 1.1 / 2.25, "MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 ratio 1.1/2.25"
    return 1900.0 * 1.1 / 2.25, "fallback 1.9 PFLOP/s bf16 x nominal TF32/BF16 ratio 1.1/2.25"


def run_config4(args):
    """One step = one full measurement <H> = sum_i a_i <P_i> over all 1 542 657 strings of
    the 64-qubit Hamiltonian on the chi = 256 MPS resident in HBM (mixed precision: the
    environment contractions of levels whose bonds are both >= 128 on the tensor cores
    with compensated TF32 splits, FP64 sums). Steps run back to back; terms/s = strings x steps / time."""
    import torch
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn
    G.build()
    G.load_library()
    K, W = args.steps, max(3, args.warmup)
    H, B, lam, t_jw = config4_inputs(G, syn)
    n_terms = int(G.ham_get_terms(H)[1].size)
    stream = torch.cuda.current_stream().cuda_stream
    M = G.mps_create(C4_N, C4_CHI, G.MPS_MIXED, cuda_stream=stream)
    G.mps_set_state(M, B, lam)
    G.mps_set_kernel_timing(M, True)
    for _ in range(W):
        G.mps_energy(M, H)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    dev_ms, wall_ms, gemm_ms, gemm_fl, launches, gl, close_ms = [], [], [], [], [], [], []
    energies = []
    for _ in range(K):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        energies.append(G.mps_energy(M, H))
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        s = G.mps_get_stats(M)
        dev_ms.append(s["ms_measure"])
        gemm_ms.append(s["ms_tc_gemm"])
        close_ms.append(s["ms_close"])
        gemm_fl.append(s["tc_gemm_flops"])
        launches.append(int(s["kernel_launches"]))
        gl.append(int(s["tc_gemm_launches"]))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_dev = float(np.sum(dev_ms)) * 1e-3
    peak, peak_src = tc_peak_tflops()
    achieved = float(np.sum(gemm_fl)) / (float(np.sum(gemm_ms)) * 1e-3) / 1e12
    # CPU oracle: the plain left-to-right contraction of a bounded sample of strings
    cpu = None
    try:
        from oracle import mps as omps
        P, _ = G.ham_get_terms(H)
        idx = np.random.default_rng(0).choice(len(P), 12, replace=False)
        ranks = [b.shape[2] for b in B[:-1]]
        st = omps.MPS([np.asarray(b) for b in B], [np.asarray(l) for l in lam])
        t0 = time.perf_counter()
        for i in idx:
            omps.expect_string(st, P[i])
        dt = (time.perf_counter() - t0) / len(idx)
        cpu = {"value": 1.0 / dt, "unit": "Pauli terms/s", "cores": threads_used(), "kind": "oracle-extrapolated",
               "estimate": True, "sample": f"{len(idx)} strings of the Hamiltonian contracted one by one "
                                           f"({dt:.3f} s/string), no prefix sharing; rate per string"}
        del ranks
    except Exception as e:   # noqa: BLE001 - reported in the line
        cpu = {"error": str(e)}
    line = {
        "metric": "Pauli terms/s", "value": K * n_terms / t_dev, "unit": "terms/s", "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": 1e3 * t_dev / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 storage, tf32x3 tensor-core contractions, f64 sums", "data": "synthetic",
        "config": {"workload": "measure_64q_chi256_all_strings", "qubits": C4_N, "chi": C4_CHI,
                   "pauli_terms": n_terms, "state": "seeded random right-canonical MPS, full ranks",
                   "integral_seed": SEED, "l2": "inputs (134 MB state, 3.1 M environments per step) exceed L2"},
        "evals_per_s": K / t_dev,
        "e2e": {"value": K * n_terms / (float(np.sum(wall_ms)) * 1e-3), "unit": "terms/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * (4 + 2 * n_terms)},
        "gpu_launches": int(np.mean(launches)),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                     "kernel": "k_gemm_tf32x3 (tcgen05, 3 TF32 products per product)",
                     "launches_per_step": int(np.mean(gl)),
                     "note": "achieved = algorithmic flops (2MNK of the complex-as-real GEMMs, split products "
                             "not counted) / summed CUDA-event time of the GEMM launches; the tensor pipe "
                             "executes 3x these flops"},
        "gemm_share_of_step": float(np.sum(gemm_ms)) / float(np.sum(dev_ms)),
        "close_share_of_step": float(np.sum(close_ms)) / float(np.sum(dev_ms)),
        "cpu_baseline": cpu, "clocks": clocks, "energy_Ha": energies[-1],
        "host_jw_seconds": t_jw,
    }
    print(json.dumps(line))


def run_tc_gemm_case():
    """A fixed launch for ncu: one 43 520 x 1024 x 512 tensor-core GEMM (the GEMM-T shape of
    a 170-node chunk at D = D' = 256) through the C-ABI entry on aligned random operands,
    three calls; prints the CUDA-event time of the last call."""
    import torch
    import paper_2207_03711_gb300 as G
    G.build()
    G.load_library()
    M, N, K = 43520, 1024, 512
    g = torch.Generator(device="cuda").manual_seed(SEED)
    A = torch.randn(M, K, device="cuda", generator=g)
    B = torch.randn(N, K, device="cuda", generator=g)
    C = torch.empty(M, N, device="cuda")
    for _ in range(2):
        G.mps_tc_gemm_tf32x3(M, N, K, A.data_ptr(), K, B.data_ptr(), K, C.data_ptr(), N)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    G.mps_tc_gemm_tf32x3(M, N, K, A.data_ptr(), K, B.data_ptr(), K, C.data_ptr(), N)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"tc_gemm_case": True, "M": M, "N": N, "K": K, "ms_call": ms,
                      "tflops_algorithmic": 2.0 * M * N * K / ms / 1e9}))


def run_config4_tc_case(n_strings, budget_mb=0):
    """A short fixed workload for ncu: one chi = 256 measurement of the first n_strings
    strings of the 64-qubit Hamiltonian (mixed precision)."""
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn
    G.build()
    G.load_library()
    H, B, lam, _ = config4_inputs(G, syn, n_strings=n_strings)
    M = G.mps_create(C4_N, C4_CHI, G.MPS_MIXED)
    if budget_mb:
        G.mps_set_meas_budget(M, budget_mb << 20)
    G.mps_set_state(M, B, lam)
    e = G.mps_energy(M, H)
    s = G.mps_get_stats(M)
    print(json.dumps({"config4_tc_case": True, "strings": n_strings, "energy": e, "ms_measure": s["ms_measure"],
                      "tc_gemm_launches": s["tc_gemm_launches"], "tc_gemm_flops": s["tc_gemm_flops"]}))



def run_config3(args):
    """32 qubits / 16 electrons, chi = 128, mixed precision; ansatz = all singles and the
    first 16 doubles of the UCCSD list (13 872 two-site gates); one step = the
    parameter-shift gradient over those 16 doubles, i.e. the 256 circuits with one of
    their 128 Pauli rotations shifted by +-pi/2, each followed by a measurement of all
    strings of the 16-orbital Hamiltonian. The shifted circuits share the unshifted
    prefix up to their rotation (slot 0 runs it; 256 slots fork from it), so they run in
    one batched pass. Metric: circuits/s (256 per step)."""
    import torch
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn
    from paper_2207_03711_gb300.serve import uccsd_circuit
    G.build()
    G.load_library()
    n, ne, chi, nd = 32, 16, 128, 16
    K, W = args.steps, max(3, args.warmup)
    h, g = syn.random_integrals(n // 2, SEED)
    H = G.ham_jw_from_integrals(h, g)
    n_terms = int(G.ham_get_terms(H)[1].size)
    C = uccsd_circuit(n, ne, n_doubles=nd)
    if args.circuit == "cancel-ladders":
        G.circ_cancel_ladders(C)
    n_singles = 2 * (ne // 2) * ((n - ne) // 2)
    sel = np.arange(n_singles, n_singles + nd, dtype=np.int32)
    stream = torch.cuda.current_stream().cuda_stream
    M = G.mps_create(n, chi, G.MPS_MIXED, n_slots=257, cuda_stream=stream)
    thetas = [syn.random_amplitudes(C.n_params, 300 + i) for i in range(K + W)]
    # warm-up steps: the same kernels and slot memory over the first double only (16 of
    # the 256 circuits), so that W >= 3 warm-ups do not triple the run
    for w in range(W):
        G.vqe_gradient(M, C, H, thetas[w], sel[:1], allow_noconv=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    wall, circ_ms, meas_ms, flops, launches = [], [], [], [], []
    for k in range(K):
        t0 = time.perf_counter()
        grad = G.vqe_gradient(M, C, H, thetas[W + k], sel, allow_noconv=True)
        wall.append(time.perf_counter() - t0)
        s = G.mps_get_stats(M)
        circ_ms.append(s["ms_circuit"])
        meas_ms.append(s["ms_measure"])
        flops.append(s["alg_flops_call"])
        launches.append(int(s["kernel_launches"]))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_dev = (float(np.sum(circ_ms)) + float(np.sum(meas_ms))) * 1e-3
    peaks = alu_peaks(torch)
    achieved = float(np.sum(flops)) / (float(np.sum(circ_ms)) * 1e-3) / 1e12
    n_circ = 2 * 8 * nd
    line = {"metric": "parameter-shift circuits/s", "value": K * n_circ / t_dev, "unit": "circuits/s", "n_gpus": 1,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * t_dev / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "uccsd_32q_16e_chi128_singles_16doubles_gradient", "qubits": n, "electrons": ne,
                       "chi": chi, "two_site_gates": G.circ_num_gates(C), "circuits_per_step": n_circ,
                       "circuit": args.circuit,
                       "pauli_terms": n_terms, "slots": 257,
                       "warmup_steps": "gradient over the first double (16 circuits)"},
            "pauli_terms_per_s": K * n_circ * n_terms / t_dev,
            "e2e": {"value": K * n_circ / float(np.sum(wall)), "unit": "circuits/s",
                    "h2d_bytes_per_step": 8 * C.n_params + 4 * nd, "d2h_bytes_per_step": 8 * nd},
            "gpu_launches": int(np.mean(launches)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp32_tflops"], "traffic": None,
                         "peak_source": "measured: cuBLAS SGEMM in this process (FP32 CUDA cores)",
                         "kernel": "k_circuit<float,512> (one block per circuit)"},
            "breakdown_ms_per_step": {"circuit": float(np.mean(circ_ms)), "measure": float(np.mean(meas_ms))},
            "gradient_norm": float(np.linalg.norm(grad)), "clocks": clocks}
    print(json.dumps(line))



def run_random_gates(args):
    """The paper's second workload at the largest bond cap gates are applied at: random
    two-site unitaries on neighbouring qubits (brickwork order) applied to a seeded random
    right-canonical MPS of 32 qubits at chi = 128 (every interior rank 128 at the
    centre), mixed precision. One step = 248 gates (eight brickwork layers) through
    mps_apply_gates on one state; steps run back to back on the evolving state."""
    import torch
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn
    G.build()
    G.load_library()
    n, chi = 32, 128
    K, W = args.steps, max(3, args.warmup)
    B, lam = syn.random_right_canonical_mps(n, chi, 1)
    bonds = np.array(syn.brickwork_bonds(n, 8), dtype=np.int32)
    Us = np.array([np.linalg.qr(z)[0] for z in syn.random_gate_matrices(len(bonds) * (K + W), 4)])
    stream = torch.cuda.current_stream().cuda_stream
    M = G.mps_create(n, chi, G.MPS_MIXED, cuda_stream=stream)
    G.mps_set_state(M, B, lam)
    ng = len(bonds)
    for w in range(W):
        G.mps_apply_gates(M, bonds, Us[w * ng:(w + 1) * ng], allow_noconv=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    dev_ms, wall_ms, flops = [], [], []
    for k in range(K):
        o = (W + k) * ng
        t0 = time.perf_counter()
        G.mps_apply_gates(M, bonds, Us[o:o + ng], allow_noconv=True)
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        s = G.mps_get_stats(M)
        dev_ms.append(s["ms_circuit"])
        flops.append(s["alg_flops_call"])
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_dev = float(np.sum(dev_ms)) * 1e-3
    peaks = alu_peaks(torch)
    achieved = float(np.sum(flops)) / t_dev / 1e12
    line = {"metric": "two-site gates/s", "value": K * ng / t_dev, "unit": "gates/s", "n_gpus": 1, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * t_dev / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "random_brickwork_gates_32q_chi128", "qubits": n, "chi": chi,
                       "gates_per_step": ng, "state": "seeded random right-canonical MPS, full ranks",
                       "l2": "state (33 MB) L2-resident; the gate chain is serial"},
            "e2e": {"value": K * ng / (float(np.sum(wall_ms)) * 1e-3), "unit": "gates/s",
                    "h2d_bytes_per_step": int(ng * (4 + 256)), "d2h_bytes_per_step": 8 + 4 * 8},
            "gpu_launches": int(s["kernel_launches"]),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp32_tflops"], "traffic": None,
                         "peak_source": "measured: cuBLAS SGEMM in this process (FP32 CUDA cores)",
                         "kernel": "k_circuit<float,512> (one thread block)",
                         "frac_of_one_sm": achieved / (peaks["fp32_tflops"] / 152)},
            "ms_per_gate": 1e3 * t_dev / (K * ng), "clocks": clocks}
    print(json.dumps(line))



def run_profile_case():
    """One gate-engine launch (256 gates of the 24-qubit circuit's interior on a saturated
    chi = 64 state) and one full measurement: a short, fixed workload for ncu."""
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn
    G.build()
    G.load_library()
    h, g = inputs()
    H = G.ham_jw_from_integrals(h, g)
    paulis, coeff = G.ham_get_terms(H)
    C = G.circ_uccsd(N_QUBITS, N_ELEC)
    theta = syn.random_amplitudes(C.n_params, SEED)
    bond, U = G.circ_export_gates(C, theta)
    B, lam = syn.random_right_canonical_mps(N_QUBITS, CHI, 0)
    M = G.mps_create(N_QUBITS, CHI, G.MPS_MIXED)
    G.mps_set_state(M, B, lam)
    G.mps_apply_gates(M, bond[30000:30256], U[30000:30256], allow_noconv=True)
    s_circ = G.mps_get_stats(M)              # stats restart at every call
    vals = G.mps_expect_paulis(M, paulis)
    s = G.mps_get_stats(M)
    print(json.dumps({"profile_case": True, "gates": 256, "ms_circuit": s_circ["ms_circuit"],
                      "ms_measure": s["ms_measure"], "sum_re": float(np.sum(vals.real)),
                      "kernel_launches": s_circ["kernel_launches"] + s["kernel_launches"]}))


def run_serve(args):
    """Serving stream (scaled-down form of the mixed-size request workload): energy and
    gradient requests with qubits uniform in {12, 14, ..., 24}, chi in {16, 32, 64},
    circuit = singles + the first 32 doubles, random integrals per request. A closed-loop
    burst of 24 requests measures the saturation rate; the rest arrive as a Poisson
    stream at 0.7 of it. Prints one JSON line with throughput and p50/p99 latency."""
    import paper_2207_03711_gb300 as G
    from paper_2207_03711_gb300 import synthetic as syn
    from paper_2207_03711_gb300.serve import Request, Server
    G.build()
    G.load_library()
    rng = np.random.default_rng(SEED)
    n_doubles = 32

    def make(i):
        n = int(rng.choice(np.arange(12, 26, 2)))
        ne = n // 2
        chi = int(rng.choice([16, 32, 64]))
        h, g = syn.random_integrals(n // 2, 1000 + i)
        n_singles = 2 * (ne // 2) * ((n - ne) // 2)
        theta = syn.random_amplitudes(n_singles + n_doubles, 2000 + i)
        if rng.random() < 0.2:
            sel = n_singles + rng.choice(n_doubles, 4, replace=False)
            return Request("gradient", h, g, ne, chi, theta, sel=sel, n_slots=9, n_doubles=n_doubles, tag=i)
        return Request("energy", h, g, ne, chi, theta, n_doubles=n_doubles, tag=i)

    reqs = [make(i) for i in range(max(args.serve_requests, 30))]
    kinds = collections.Counter(r.kind for r in reqs)
    burst = reqs[:24]
    with Server(max_inflight=32) as srv:
        t0 = time.perf_counter()
        for f in [srv.submit(r) for r in burst]:
            f.result()
        sat = len(burst) / (time.perf_counter() - t0)
    rate = 0.7 * sat
    arr = np.random.default_rng(SEED + 1).exponential(1.0 / rate, size=len(reqs) - len(burst))
    with Server(max_inflight=32) as srv:
        t_next = time.perf_counter()
        futs = []
        for r, dt in zip(reqs[len(burst):], arr):
            t_next += dt
            pause = t_next - time.perf_counter()
            if pause > 0:
                time.sleep(pause)
            futs.append(srv.submit(r))
        for f in futs:
            f.result()
        st = srv.stats()
    print(json.dumps({"metric": "serving stream", "requests": len(reqs) - len(burst),
                      "kinds": dict(kinds), "saturation_req_per_s": sat, "arrival_rate_req_per_s": rate,
                      **st, "config": {"qubits": "uniform {12,...,24}", "chi": "{16, 32, 64}",
                                       "circuit": "singles + first 32 doubles", "precision": "mixed",
                                       "gradient": "4 doubles, 9 slots"}}))


def main():
    args = parse()
    if args.serve:
        run_serve(args)
        return
    if args.config4:
        run_config4(args)
    elif args.random_gates:
        run_random_gates(args)
    elif args.config3:
        run_config3(args)
    elif args.config4_tc_case:
        run_config4_tc_case(args.case_strings, args.case_budget_mb)
    elif args.tc_gemm_case:
        run_tc_gemm_case()
    elif args.profile_case:
        run_profile_case()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
