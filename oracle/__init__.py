"""Independent CPU oracle for the MPS-VQE hot path (arXiv 2207.03711).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may use it. It shares no code with the CUDA library and takes
every random input (integrals, amplitudes, MPS tensors) as an argument.

Everything is plain NumPy in float64/complex128, written for readability:
no blocking, no fusion, no reordering beyond what the paper's definitions say.

Modules
-------
pauli      Pauli-string algebra and the Jordan-Wigner map (Eq. 1 -> Eq. 2).
fock       Brute-force Fock-space Hamiltonian and the Hartree-Fock energy
           (independent of the Pauli algebra; used to pin ``pauli``).
ucc        UCCSD excitations (Eq. 3-4) and their Pauli generators.
sv         c1: exact statevector simulation of the Trotterised ansatz.
circuit    Native-gate decomposition of each Pauli exponential and the
           fusion of single-qubit gates into two-site gates.
mps        c2: the paper's truncated right-canonical MPS algorithm
           (Eqs. 6-10) plus plain left-to-right Pauli expectations (Eq. 11).
grad       Parameter-shift gradients on top of c1 / c2.
"""
