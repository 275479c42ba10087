"""GB300 MPS-VQE hot path (arXiv 2207.03711): thin Python binding of libmpsvqe.so.

Every function here only marshals arguments into the C ABI declared in
include/mpsvqe.h and raises on a non-zero status; all arithmetic of the path runs
in the library's CUDA kernels and its host preprocessing. There is no fallback:
if the library is missing, importing the bindings raises.

Handles are wrapped in small objects whose ``close()`` (or garbage collection)
calls the matching ``*_destroy``.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmpsvqe.so")

MPS_OK, MPS_EINVAL, MPS_ENOMEM, MPS_ECUDA, MPS_ETIMEOUT, MPS_ENOCONV, MPS_ENONFINITE = 0, -1, -2, -3, -4, -5, -6
MPS_FP64, MPS_MIXED = 0, 1

# Every entry point of include/mpsvqe.h with its ctypes signature.
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)
_PI = ctypes.POINTER(ctypes.c_int)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PD = ctypes.POINTER(ctypes.c_double)


class MpsStats(ctypes.Structure):
    _fields_ = [("discarded_weight", ctypes.c_double), ("max_rank", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("n_gates", ctypes.c_int64),
                ("n_svd_noconv", ctypes.c_int64), ("ms_circuit", ctypes.c_double),
                ("ms_measure", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("cycles", ctypes.c_double * 7), ("n_fallback", ctypes.c_int64),
                ("alg_flops_total", ctypes.c_double), ("n_nonfinite", ctypes.c_int64),
                ("alg_flops_call", ctypes.c_double), ("tc_gemm_launches", ctypes.c_int64),
                ("tc_gemm_flops", ctypes.c_double), ("ms_tc_gemm", ctypes.c_double),
                ("ms_close", ctypes.c_double)]


SIGNATURES = {
    "ham_jw_from_integrals": [_I, _P, _P, _D, _PP],
    "ham_create": [_I, _I64, _P, _P, _PP],
    "ham_num_terms": [_P, _PI64],
    "ham_get_terms": [_P, _P, _P],
    "ham_destroy": [_P],
    "circ_uccsd": [_I, _I, _PP, _PI],
    "circ_create": [_I, _I64, _P, _P, _P, _PP],
    "circ_set_reference": [_P, _P],
    "circ_num_rotations": [_P, _PI64, _PI],
    "circ_get_rotations": [_P, _P, _P, _P],
    "circ_num_gates": [_P, _PI64],
    "circ_export_gates": [_P, _P, _P, _P],
    "circ_destroy": [_P],
    "mps_create": [_I, _I, _I, _I, _P, _PP],
    "mps_reset": [_P, _I, _P],
    "mps_set_svd_params": [_P, _D, _I],
    "mps_set_meas_budget": [_P, ctypes.c_size_t],
    "mps_set_kernel_timing": [_P, _I],
    "mps_apply_circuit": [_P, _P, _P, _PD],
    "mps_apply_gates": [_P, _I64, _P, _P, _PD],
    "mps_expect_paulis": [_P, _I64, _P, _P, _P],
    "mps_get_ranks": [_P, _I, _P],
    "mps_state_size": [_P, _I, _PI64, _PI64],
    "mps_get_state": [_P, _I, _P, _P],
    "mps_set_state": [_P, _I, _P, _P, _P],
    "mps_energy": [_P, _P, _PD],
    "vqe_energy": [_P, _P, _P, _P, _PD],
    "vqe_energy_batch": [_P, _P, _P, _I, _P, _P],
    "vqe_gradient": [_P, _P, _P, _P, _I, _P, _P],
    "mps_get_stats": [_P, ctypes.POINTER(MpsStats)],
    "mps_destroy": [_P],
    "circ_fuse_gates": [_P, ctypes.POINTER(ctypes.c_int64)],
    "circ_cancel_ladders": [_P, ctypes.POINTER(ctypes.c_int64)],
    "mps_estimate_bytes": [_I, _I, _I, _I, _P, _P, ctypes.POINTER(ctypes.c_size_t)],
    "mps_apply_gates_noalloc": [_I, _I, _P, _P, _P, _P, _I64, _P, _P, _P, _PD],
    "mps_tc_gemm_tf32x3": [_I, _I, _I, _P, _I64, _P, _I64, _P, _I64, _P],
    "mps_last_error": [],
}

_lib = None


def load_library(path=LIB_PATH):
    """Load libmpsvqe.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"MPS-VQE CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "mps_last_error" else ctypes.c_int
    _lib = lib
    return lib


def build(force=False):
    from .build_lib import build as _b
    return _b(force=force)


class MpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _check(rc, allow=()):
    if rc != MPS_OK and rc not in allow:
        raise MpsError(rc, load_library().mps_last_error().decode())
    return rc


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _u8(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a if shape is None else a.reshape(shape)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(load_library(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


class Ham(_Handle):
    _destroy = "ham_destroy"


class Circ(_Handle):
    _destroy = "circ_destroy"


class Mps(_Handle):
    _destroy = "mps_destroy"


# ------------------------------------------------------------------ Hamiltonian
def ham_jw_from_integrals(h, eri, e_core=0.0):
    lib = load_library()
    h, eri = _f64(h), _f64(eri)
    out = ctypes.c_void_p()
    _check(lib.ham_jw_from_integrals(h.shape[0], _ptr(h), _ptr(eri), e_core, ctypes.byref(out)))
    return _attach_n(Ham(out.value), 2 * h.shape[0])


def ham_create(paulis, coeff):
    lib = load_library()
    paulis = _u8(paulis)
    coeff = _f64(coeff)
    out = ctypes.c_void_p()
    _check(lib.ham_create(paulis.shape[1], paulis.shape[0], _ptr(paulis), _ptr(coeff), ctypes.byref(out)))
    return _attach_n(Ham(out.value), paulis.shape[1])


def ham_get_terms(ham):
    lib = load_library()
    nt = ctypes.c_int64()
    _check(lib.ham_num_terms(ham, ctypes.byref(nt)))
    paulis = np.zeros((nt.value, ham.n_qubits), dtype=np.uint8)
    coeff = np.zeros(nt.value)
    _check(lib.ham_get_terms(ham, _ptr(paulis), _ptr(coeff)))
    return paulis, coeff


def _attach_n(obj, n):
    obj.n_qubits = n
    return obj


# -------------------------------------------------------------------- circuit
def circ_uccsd(n_qubits, n_electrons):
    lib = load_library()
    out = ctypes.c_void_p()
    npar = ctypes.c_int()
    _check(lib.circ_uccsd(n_qubits, n_electrons, ctypes.byref(out), ctypes.byref(npar)))
    c = _attach_n(Circ(out.value), n_qubits)
    c.n_params = npar.value
    return c


def circ_create(paulis, param_idx, scale):
    lib = load_library()
    paulis = _u8(paulis)
    pidx = np.ascontiguousarray(param_idx, dtype=np.int32)
    scale = _f64(scale)
    out = ctypes.c_void_p()
    _check(lib.circ_create(paulis.shape[1], paulis.shape[0], _ptr(paulis), _ptr(pidx), _ptr(scale),
                           ctypes.byref(out)))
    c = _attach_n(Circ(out.value), paulis.shape[1])
    c.n_params = int(max(pidx.max() + 1, 0)) if pidx.size else 0
    return c


def circ_set_reference(circ, occ):
    _check(load_library().circ_set_reference(circ, _ptr(_u8(occ))))


def circ_get_rotations(circ):
    lib = load_library()
    nr = ctypes.c_int64()
    npar = ctypes.c_int()
    _check(lib.circ_num_rotations(circ, ctypes.byref(nr), ctypes.byref(npar)))
    paulis = np.zeros((nr.value, circ.n_qubits), dtype=np.uint8)
    pidx = np.zeros(nr.value, dtype=np.int32)
    scale = np.zeros(nr.value)
    _check(lib.circ_get_rotations(circ, _ptr(paulis), _ptr(pidx), _ptr(scale)))
    return paulis, pidx, scale


def circ_fuse_gates(circ):
    n = ctypes.c_int64(0)
    _check(load_library().circ_fuse_gates(circ, ctypes.byref(n)))
    return int(n.value)


def circ_cancel_ladders(circ):
    n = ctypes.c_int64(0)
    _check(load_library().circ_cancel_ladders(circ, ctypes.byref(n)))
    return int(n.value)


def circ_num_gates(circ):
    n = ctypes.c_int64()
    _check(load_library().circ_num_gates(circ, ctypes.byref(n)))
    return n.value


def circ_export_gates(circ, theta):
    ng = circ_num_gates(circ)
    bond = np.zeros(ng, dtype=np.int32)
    U = np.zeros((ng, 4, 4), dtype=np.complex128)
    th = _f64(theta if theta is not None else np.zeros(max(circ.n_params, 1)))
    _check(load_library().circ_export_gates(circ, _ptr(th), _ptr(bond), _ptr(U)))
    return bond, U


# ------------------------------------------------------------------ MPS state
def mps_create(n_qubits, chi, precision=MPS_FP64, n_slots=1, cuda_stream=0):
    lib = load_library()
    out = ctypes.c_void_p()
    _check(lib.mps_create(n_qubits, chi, precision, n_slots, ctypes.c_void_p(cuda_stream or None),
                          ctypes.byref(out)))
    m = _attach_n(Mps(out.value), n_qubits)
    m.chi, m.precision, m.n_slots = chi, precision, n_slots
    return m


def mps_reset(mps, occ, slot=0):
    _check(load_library().mps_reset(mps, slot, _ptr(_u8(occ))))


def mps_set_svd_params(mps, cutoff, max_sweeps):
    _check(load_library().mps_set_svd_params(mps, cutoff, max_sweeps))


def mps_set_kernel_timing(mps, on=True):
    _check(load_library().mps_set_kernel_timing(mps, 1 if on else 0))


def mps_set_meas_budget(mps, nbytes):
    _check(load_library().mps_set_meas_budget(mps, int(nbytes)))


def mps_apply_circuit(mps, circ, theta, allow_noconv=False):
    dw = ctypes.c_double()
    th = _f64(theta if theta is not None else np.zeros(max(circ.n_params, 1)))
    _check(load_library().mps_apply_circuit(mps, circ, _ptr(th), ctypes.byref(dw)),
           allow=(MPS_ENOCONV,) if allow_noconv else ())
    return dw.value


def mps_apply_gates(mps, bond, U, allow_noconv=False):
    bond = np.ascontiguousarray(bond, dtype=np.int32)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    dw = ctypes.c_double()
    _check(load_library().mps_apply_gates(mps, bond.shape[0], _ptr(bond), _ptr(U), ctypes.byref(dw)),
           allow=(MPS_ENOCONV,) if allow_noconv else ())
    return dw.value


def mps_expect_paulis(mps, paulis):
    paulis = _u8(paulis)
    re = np.zeros(paulis.shape[0])
    im = np.zeros(paulis.shape[0])
    _check(load_library().mps_expect_paulis(mps, paulis.shape[0], _ptr(paulis), _ptr(re), _ptr(im)))
    return re + 1j * im


def mps_get_ranks(mps, slot=0):
    r = np.zeros(mps.n_qubits - 1, dtype=np.int32)
    _check(load_library().mps_get_ranks(mps, slot, _ptr(r)))
    return r


def mps_get_state(mps, slot=0):
    """Returns (ranks, list of site tensors (r_{k-1}, 2, r_k) complex128, list of lambda arrays)."""
    lib = load_library()
    nb, nl = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.mps_state_size(mps, slot, ctypes.byref(nb), ctypes.byref(nl)))
    B = np.zeros(nb.value, dtype=np.complex128)
    lam = np.zeros(nl.value)
    _check(lib.mps_get_state(mps, slot, _ptr(B), _ptr(lam)))
    r = mps_get_ranks(mps, slot)
    n = mps.n_qubits
    sites, lams, o, lo = [], [], 0, 0
    for k in range(n):
        rl = 1 if k == 0 else int(r[k - 1])
        rr = 1 if k == n - 1 else int(r[k])
        sites.append(B[o:o + rl * 2 * rr].reshape(rl, 2, rr).copy())
        o += rl * 2 * rr
    for b in range(n - 1):
        lams.append(lam[lo:lo + r[b]].copy())
        lo += r[b]
    return r, sites, lams


def mps_set_state(mps, sites, lams, slot=0):
    ranks = np.array([s.shape[2] for s in sites[:-1]], dtype=np.int32)
    B = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.complex128).ravel() for s in sites]))
    lam = _f64(np.concatenate([np.asarray(l, dtype=np.float64) for l in lams]))
    _check(load_library().mps_set_state(mps, slot, _ptr(ranks), _ptr(B), _ptr(lam)))


def mps_energy(mps, ham):
    e = ctypes.c_double()
    _check(load_library().mps_energy(mps, ham, ctypes.byref(e)))
    return e.value


def vqe_energy(mps, circ, ham, theta, allow_noconv=False):
    e = ctypes.c_double()
    th = _f64(theta if theta is not None else np.zeros(max(circ.n_params, 1)))
    _check(load_library().vqe_energy(mps, circ, ham, _ptr(th), ctypes.byref(e)),
           allow=(MPS_ENOCONV,) if allow_noconv else ())
    return e.value


def vqe_energy_batch(mps, circ, ham, thetas, allow_noconv=False):
    th = _f64(thetas)
    nb = th.shape[0]
    out = np.zeros(nb)
    _check(load_library().vqe_energy_batch(mps, circ, ham, nb, _ptr(th), _ptr(out)),
           allow=(MPS_ENOCONV,) if allow_noconv else ())
    return out


def vqe_gradient(mps, circ, ham, theta, sel, allow_noconv=False):
    sel = np.ascontiguousarray(sel, dtype=np.int32)
    out = np.zeros(sel.shape[0])
    _check(load_library().vqe_gradient(mps, circ, ham, _ptr(_f64(theta)), sel.shape[0], _ptr(sel), _ptr(out)),
           allow=(MPS_ENOCONV,) if allow_noconv else ())
    return out


def mps_apply_gates_noalloc(n_qubits, chi, site_tensors, site_offsets, lambdas, ranks, n_gates, bonds, gates,
                            cuda_stream=0, allow_noconv=False):
    """Device-pointer arguments (ints); returns the discarded weight. See include/mpsvqe.h."""
    dw = ctypes.c_double()
    _check(load_library().mps_apply_gates_noalloc(n_qubits, chi, ctypes.c_void_p(site_tensors),
                                                  ctypes.c_void_p(site_offsets), ctypes.c_void_p(lambdas),
                                                  ctypes.c_void_p(ranks), n_gates, ctypes.c_void_p(bonds),
                                                  ctypes.c_void_p(gates), ctypes.c_void_p(cuda_stream or None),
                                                  ctypes.byref(dw)),
           allow=(MPS_ENOCONV,) if allow_noconv else ())
    return dw.value


def mps_tc_gemm_tf32x3(M, N, K, A, lda, B, ldb, C, ldc, cuda_stream=0):
    """Device-pointer arguments (ints): C = A . B^T on the tensor cores. See include/mpsvqe.h."""
    _check(load_library().mps_tc_gemm_tf32x3(M, N, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(B), ldb,
                                             ctypes.c_void_p(C), ldc, ctypes.c_void_p(cuda_stream or None)))


def mps_get_stats(mps):
    s = MpsStats()
    _check(load_library().mps_get_stats(mps, ctypes.byref(s)))
    out = {k: getattr(s, k) for k, _ in MpsStats._fields_}
    out["cycles"] = list(s.cycles)
    return out


def mps_estimate_bytes(n_qubits, chi, precision=MPS_FP64, n_slots=1, circ=None, ham=None):
    out = ctypes.c_size_t(0)
    _check(load_library().mps_estimate_bytes(n_qubits, chi, precision, n_slots, circ, ham, ctypes.byref(out)))
    return int(out.value)


def mps_last_error():
    return load_library().mps_last_error().decode()
