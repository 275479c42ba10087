"""Benchmark of the MPS-VQE hot path on GB300 (one JSON line on stdout).

Workload (the 24-qubit configuration): 12 spatial orbitals / 24 qubits, 12
electrons, seeded random 8-fold-symmetric integrals (29 737 Jordan-Wigner Pauli
strings), UCCSD with 1818 excitations (14 112 Pauli rotations, 442 272 two-site
gates), bond cap chi = 64, one energy evaluation per call (reset to Hartree-Fock,
apply the circuit, evaluate every string, FP64 compensated sum). A step is one
vqe_energy call in the mixed-precision mode.

  value  energy evaluations per second with inputs resident on the device, from
         CUDA events recorded by the library on its stream around its kernels
  e2e    the same metric through the C ABI call with host buffers (theta uploaded,
         energy read back inside the timed region), from host wall-clock time

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


# dram__bytes_read.sum + dram__bytes_write.sum of k_circuit in the 256-gate profile case
# (ncu capture of the current kernel; None until one exists)
TRAFFIC_PROFILE_CASE = 1.728256e6 + 0.090624e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--serve", action="store_true",
                    help="serving stream: Poisson arrivals of mixed energy/gradient requests")
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--profile-case", action="store_true",
                    help="small profiling case: 256 gates on a saturated chi=64 state + one measurement")
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
              f"({t_term * 1e3:.2f} ms/string) x {len(codes)}; extrapolated to one evaluation")
    return 1.0 / est, sample, est


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        return max(int(i.get("num_threads", 1)) for i in threadpool_info()) or 1
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    h, g = inputs()
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, sample, est = oracle_sample(h, g, budget_s=min(20.0, 150.0 / max(1, args.warmup + args.steps)))
        if i >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    cores = threads_used()
    line = {"impl": "reference", "metric": "VQE energy evals/s", "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def accuracy_probe(G):
    """|dE| of both precisions against the oracle on the exactly representable 8-qubit
    case (chi = 16 holds the state without truncation)."""
    from oracle import circuit, mps, pauli, ucc
    from paper_2207_03711_gb300 import synthetic as syn
    n, ne, chi = 8, 4, 16
    h, g = syn.random_integrals(4, 0)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    th = syn.random_amplitudes(C.n_params, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    st = mps.hf_mps(n, ne)
    mps.apply_gates(st, circuit.compile_circuit(rc, rp, rs, th, n), chi)
    e_ref = mps.energy(st, codes, coeffs)[0]
    out = {}
    for name, prec in (("fp64", G.MPS_FP64), ("mixed", G.MPS_MIXED)):
        M = G.mps_create(n, chi, prec)
        out[f"abs_dE_Ha_{name}"] = abs(G.vqe_energy(M, C, H, th) - e_ref)
        M.close()
    out["case"] = "8 qubits, 4 electrons, chi=16 (untruncated), one evaluation vs the FP64 oracle"
    return out


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over the process group (the slowest
    rank sets the step time of a replicated run)."""
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_rate(world, ms_per_step):
    """Whole-job evaluations per second of `world` replicas, one evaluation each per step."""
    return world * 1e3 / ms_per_step


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
    theta = syn.random_amplitudes(C.n_params, SEED + rank)
    stream = torch.cuda.current_stream().cuda_stream
    W = max(3, args.warmup)
    # the warm-up evaluations run together as one batch with one evaluation per SM (at
    # least W); their wall time gives the batched throughput reported beside the
    # single-evaluation metric
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    n_warm = max(W, n_sm)
    M = G.mps_create(N_QUBITS, CHI, G.MPS_MIXED, n_slots=n_warm, cuda_stream=stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 512 MB > L2
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    e_batch = G.vqe_energy_batch(M, C, H, np.stack([syn.random_amplitudes(C.n_params, 100 + i)
                                                    for i in range(n_warm)]))
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - tb0
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    dev_ms, wall_ms, energies, launches = [], [], [], []
    flops, circ_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)          # L2 flushed between timed steps (outside the timing)
        torch.cuda.synchronize()
        f0 = G.mps_get_stats(M)["alg_flops_total"]
        t0 = time.perf_counter()
        e = G.vqe_energy(M, C, H, theta)
        t1 = time.perf_counter()
        s = G.mps_get_stats(M)
        energies.append(e)
        wall_ms.append((t1 - t0) * 1e3)
        dev_ms.append(s["ms_circuit"] + s["ms_measure"])
        circ_ms.append(s["ms_circuit"])
        flops.append(s["alg_flops_total"] - f0)
        launches.append(int(s["kernel_launches"]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if rank == 0 else {}
    ms_dev, ms_wall = float(np.mean(dev_ms)), float(np.mean(wall_ms))
    if dist:
        ms_dev, ms_wall = max_over_ranks([ms_dev, ms_wall], dist, "cuda")
        if rank != 0:
            dist.destroy_process_group()
            return
    s = G.mps_get_stats(M)
    # dominant kernel: the gate engine (FP32 CUDA-core arithmetic, one block per evaluation)
    peak = 152 * 128 * 2 * 2070e6 / 1e12                 # TFLOP/s, recipe unit counts x max clock
    achieved = float(np.mean(flops)) / (float(np.mean(circ_ms)) * 1e-3) / 1e12
    n_launch = (442272 + 16383) // 16384
    value = replica_rate(world, ms_dev)
    cpu_val, cpu_sample, _ = oracle_sample(h, g)
    line = {
        "metric": "VQE energy evals/s", "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": W, "ms_per_step": ms_dev, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": dict(WORKLOAD, precision="mixed (complex64 tensors, FP32 SVD, FP64 lambda/sums)",
                       l2="flushed between timed steps (512 MB write)",
                       warmup="max(W, SM count) evaluations issued as one batch on as many slots"),
        "pauli_terms_per_s": value * 29737,
        "latency_ms": {"p50": float(np.percentile(wall_ms, 50)), "p99": float(np.percentile(wall_ms, 99))},
        "e2e": {"value": replica_rate(world, ms_wall), "unit": "evals/s", "h2d_bytes_per_step": 8 * C.n_params,
                "d2h_bytes_per_step": 8 * 4 + 8 + 16},
        "gpu_launches": int(np.mean(launches)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     # DRAM bytes per launch: the ncu capture of the 256-gate profile case
                     # (TRAFFIC_PROFILE_CASE bytes) scaled by the gates per launch; None
                     # while no capture of the current kernel exists
                     "traffic": (TRAFFIC_PROFILE_CASE / 256 * (442272 / n_launch)
                                 if TRAFFIC_PROFILE_CASE is not None else None),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 256-gate "
                                       "profile case, scaled to the mean gates per launch",
                     "kernel": "k_circuit<float,512>", "launches_per_step": n_launch,
                     "frac_of_one_sm": achieved / (peak / 152),
                     "note": "one thread block (one SM) per evaluation; peak is the whole GPU"},
        "batched": {"evals": n_warm, "evals_per_s": n_warm / t_batch, "wall_s": t_batch,
                    "pauli_terms_per_s": n_warm * 29737 / t_batch,
                    "note": "the warm-up batch: one evaluation per SM in one launch per gate chunk, "
                            "host wall time, distinct theta per evaluation",
                    "energy_spread_Ha": float(np.max(e_batch) - np.min(e_batch))},
        "cpu_baseline": {"value": cpu_val, "unit": "evals/s", "cores": threads_used(), "kind": "oracle",
                         "sample": cpu_sample},
        "clocks": clocks,
        "energy_Ha": energies[-1],
        "breakdown_ms": {"circuit": float(np.mean(circ_ms)), "measure": float(np.mean(dev_ms) - np.mean(circ_ms))},
        "svd_fallbacks_total": int(s["n_fallback"]),
        "discarded_weight": s["discarded_weight"],
        "accuracy": accuracy_probe(G),
    }
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
    if args.profile_case:
        run_profile_case()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
