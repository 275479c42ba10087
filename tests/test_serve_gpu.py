"""Serving loop on the GPU: energy and gradient requests of different sizes run side by
side under a memory budget that forces queueing, and every result equals the result
of the same request run alone (the kernels are deterministic and a request's work does
not depend on what else is in flight)."""
import numpy as np
import pytest

import paper_2207_03711_gb300 as G
from paper_2207_03711_gb300 import synthetic as syn
from paper_2207_03711_gb300.serve import Request, Server

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    specs = [("energy", 3, 2, 8, G.MPS_FP64), ("gradient", 3, 2, 8, G.MPS_FP64), ("energy", 4, 4, 8, G.MPS_MIXED),
             ("energy", 5, 4, 4, G.MPS_FP64), ("gradient", 4, 2, 4, G.MPS_MIXED), ("energy", 4, 2, 16, G.MPS_FP64),
             ("energy", 5, 6, 8, G.MPS_MIXED), ("gradient", 3, 4, 8, G.MPS_FP64), ("energy", 6, 6, 8, G.MPS_MIXED),
             ("energy", 3, 2, 4, G.MPS_MIXED)]
    for i, (kind, nsp, ne, chi, prec) in enumerate(specs):
        h, g = syn.random_integrals(nsp, 20 + i)
        n_params = G.circ_uccsd(2 * nsp, ne).n_params
        theta = syn.random_amplitudes(n_params, 30 + i) * 4
        sel = [0, n_params - 1] if kind == "gradient" else None
        out.append(Request(kind, h, g, ne, chi, theta, precision=prec, sel=sel, tag=i))
    return out


def _alone(req):
    H = G.ham_jw_from_integrals(req.h, req.eri)
    C = G.circ_uccsd(req.n_qubits, req.n_electrons)
    M = G.mps_create(req.n_qubits, req.chi, req.precision, n_slots=req.n_slots)
    if req.kind == "energy":
        return float(G.vqe_energy(M, C, H, req.theta))
    return G.vqe_gradient(M, C, H, req.theta, req.sel)


def test_results_alone_equal_results_in_the_mix():
    G.build()
    G.load_library()
    reqs = _requests()
    alone = [_alone(r) for r in reqs]
    needs = [G.mps_estimate_bytes(r.n_qubits, r.chi, r.precision, r.n_slots,
                                  G.circ_uccsd(r.n_qubits, r.n_electrons), G.ham_jw_from_integrals(r.h, r.eri))
             for r in reqs]
    budget = int(2.5 * max(needs))           # at most a few requests fit at once
    with Server(budget_bytes=budget, max_inflight=6) as srv:
        futs = [srv.submit(r) for r in reqs]
        mixed = [f.result(timeout=600) for f in futs]
        st = srv.stats()
        rec = srv.records()
    for a, b in zip(alone, mixed):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    assert st["completed"] == len(reqs)
    assert st["peak_used_bytes"] <= budget
    assert st["peak_inflight"] >= 2
    assert st["latency_p99_s"] >= st["latency_p50_s"] > 0
    # continuous, not in waves: some request started after another one and finished
    # while that one was still running (its handle came and went mid-launch)
    nested = [(a, b) for a in rec for b in rec if a[1] < b[1] and b[2] < a[2]]
    print(f"{len(nested)} nested request intervals of {len(rec)} requests")
    assert nested
