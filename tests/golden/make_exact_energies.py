"""Writes exact_energies.json: oracle energies of the untruncated cases that bench.py
checks its accuracy against (the benchmark itself never runs the oracle).

Cases: 8 qubits / 4 electrons / chi 16 and 10 qubits / 4 electrons / chi 32, seeded
random integrals (seed 0) and UCCSD amplitudes (seed 0). Both bond caps hold the exact
state, so the truncated-MPS oracle (c2) equals the statevector oracle (c1); the file
stores both and their difference. Run from the repository root:
    python tests/golden/make_exact_energies.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import circuit, mps, pauli, sv, ucc          # noqa: E402
from paper_2207_03711_gb300 import synthetic as syn      # noqa: E402


def main():
    out = {"source": "tests/golden/make_exact_energies.py (oracle c1 statevector and c2 truncated MPS, FP64)",
           "cases": []}
    for n, ne, chi in ((8, 4, 16), (10, 4, 32)):
        h, g = syn.random_integrals(n // 2, 0)
        codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
        rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
        th = syn.random_amplitudes(len(exc), 0)
        st = mps.hf_mps(n, ne)
        mps.apply_gates(st, circuit.compile_circuit(rc, rp, rs, th, n), chi)
        e2 = mps.energy(st, codes, coeffs)[0]
        e1 = sv.energy(sv.run_ansatz(n, ne, rc, rp, rs, th), codes, coeffs)[0]
        out["cases"].append({"qubits": n, "electrons": ne, "chi": chi, "integral_seed": 0, "theta_seed": 0,
                             "energy_mps_Ha": e2, "energy_statevector_Ha": e1, "abs_difference_Ha": abs(e1 - e2)})
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_energies.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
