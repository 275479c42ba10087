/*
 * mpsvqe.h - C ABI of the GB300 MPS-VQE hot path (arXiv 2207.03711).
 *
 * The library applies a Trotterised UCCSD circuit of Pauli rotations to a
 * right-canonical matrix product state by two-site gate contraction and truncated
 * SVD (Sec. III-A, Eqs. 6-10), then evaluates E = <psi|H|psi> of a Jordan-Wigner
 * qubit Hamiltonian as a weighted sum of Pauli-string expectations (Eq. 2,
 * Sec. III-C), with all strings sharing left environments through a prefix trie.
 *
 * Conventions for every call:
 *   - Every function returns an int status: MPS_OK (0) or a negative MPS_E* code.
 *     No exception crosses the ABI. mps_last_error() gives a thread-local message.
 *   - Pointer arguments are caller-owned HOST memory, read during the call or
 *     written before it returns. Handles own their device memory, which is freed by
 *     the matching *_destroy.
 *   - Calls are synchronous with respect to their host outputs; device work is
 *     issued on the CUDA stream given to mps_create (NULL = legacy default stream).
 *   - Qubit q is MPS site q (site 0 leftmost) and bit q of a statevector index.
 *     Pauli strings are n_qubits bytes each, 0 = I, 1 = X, 2 = Y, 3 = Z, site 0 first.
 *   - Angles, coefficients, energies and Schmidt numbers are double.
 *   - Complex arrays are interleaved (re, im) doubles.
 */
#ifndef MPSVQE_H
#define MPSVQE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mps_s* mps_t;   /* n_slots MPS states on one GPU + workspaces  */
typedef struct ham_s* ham_t;   /* weighted Pauli sum + its prefix trie (host) */
typedef struct circ_s* circ_t; /* compiled two-site gate list                 */

enum {
  MPS_OK = 0,
  MPS_EINVAL = -1,   /* bad argument (null pointer, size out of range, ...)       */
  MPS_ENOMEM = -2,   /* device or host allocation failed                          */
  MPS_ECUDA = -3,    /* a CUDA runtime call failed (message has the CUDA error)   */
  MPS_ETIMEOUT = -4, /* a bounded device-side wait ran out                        */
  MPS_ENOCONV = -5,  /* an SVD hit its sweep cap; results are still written       */
  MPS_ENONFINITE = -6 /* a gate's M' held a NaN or Inf: that gate was skipped and    */
                      /* the state left as it was before it                          */
};

enum { MPS_FP64 = 0, MPS_MIXED = 1 };

/* ------------------------------------------------------------------ Hamiltonian */

/* Eq. (1) -> Eq. (2), Sec. II-A: Jordan-Wigner transform of the electronic
 * Hamiltonian H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs + e_core
 * with interleaved spin orbitals p = 2k + s (n_qubits = 2 n_spatial) and
 * a_p = Z_0..Z_{p-1} (X_p + i Y_p) / 2.
 *   h:   n_spatial^2 doubles, row-major, symmetric.
 *   eri: n_spatial^4 doubles, chemist order (pq|rs) at ((p*n+q)*n+r)*n+s.
 * Terms with |a| <= 1e-12 max|a| are dropped; terms are stored in trie order
 * (lexicographic over sites 0..n-1 with I < X < Y < Z). n_spatial in [1, 64].
 * Errors: MPS_EINVAL for n_spatial out of range or null pointers; MPS_EINVAL if
 * a coefficient has an imaginary part above 1e-10 (non-Hermitian input). */
int ham_jw_from_integrals(int n_spatial, const double* h, const double* eri, double e_core,
                          ham_t* out);

/* Sec. III-C: H = sum_i a_i P_i from explicit strings. paulis: n_terms x n_qubits
 * bytes; coeff: n_terms doubles. Duplicate strings are merged. The prefix trie used
 * by vqe_energy is built here (host, once; Sec. III-D keeps the measurement part
 * constant across optimisation steps). n_qubits in [2, 128], n_terms >= 1. */
int ham_create(int n_qubits, int64_t n_terms, const uint8_t* paulis, const double* coeff,
               ham_t* out);

/* Number of stored terms, and a copy of them in trie order (either output may be NULL). */
int ham_num_terms(ham_t ham, int64_t* n_terms);
int ham_get_terms(ham_t ham, uint8_t* paulis, double* coeff);
int ham_destroy(ham_t ham);

/* -------------------------------------------------------------------- circuit */

/* Eqs. (3)-(4), Sec. II-A and Sec. III-D: Trotterised UCCSD on the Hartree-Fock
 * determinant with qubits 0..n_electrons-1 occupied. Excitations are
 * spin-conserving; singles (i, a) in lexicographic order, then doubles
 * ((i < j), (a < b)) in lexicographic order; tau = a+_a a_i or a+_a a+_b a_i a_j,
 * one parameter each. Under Jordan-Wigner tau - tau+ = i sum_k c_k P_k with
 * commuting strings, applied in increasing (x-mask, z-mask) order as rotations
 * exp(-i phi_k P_k / 2), phi_k = -2 c_k theta_e. *n_params receives the number of
 * excitations. n_qubits in [2, 128], 0 < n_electrons < n_qubits. */
int circ_uccsd(int n_qubits, int n_electrons, circ_t* out, int* n_params);

/* General rotation list: rotation r is exp(-i * scale[r] * theta[param_idx[r]] / 2 * P_r),
 * applied in order r = 0, 1, ... Each rotation is compiled (Sec. III-D, Sec. III-A)
 * into nearest-neighbour two-site gates: basis change (H for X, Rx(pi/2) for Y),
 * a parity ladder lo -> hi (CNOT onto a non-identity qubit, SWAP across an identity
 * qubit), Rz(phi) on hi, the mirror ladder and basis change; single-qubit gates are
 * fused into the neighbouring two-site gates and the top hop/Rz/hop into one gate,
 * giving 2 (hi - lo) - 1 gates per rotation. param_idx[r] < 0 means a fixed angle
 * phi = scale[r]. */
int circ_create(int n_qubits, int64_t n_rot, const uint8_t* paulis, const int32_t* param_idx,
                const double* scale, circ_t* out);

/* Reference determinant used by vqe_energy* (Sec. III-D): occ is n_qubits bytes of
 * 0/1. circ_uccsd sets qubits 0..n_electrons-1; circ_create sets all zero. */
int circ_set_reference(circ_t circ, const uint8_t* occ);

/* Inspection: rotation count/list and the compiled gate list for a given theta
 * (bond: n_gates ints; U: n_gates x 4 x 4 complex, row index 2 i_b + i_{b+1}). */
int circ_num_rotations(circ_t circ, int64_t* n_rot, int* n_params);
int circ_get_rotations(circ_t circ, uint8_t* paulis, int32_t* param_idx, double* scale);
int circ_num_gates(circ_t circ, int64_t* n_gates);
int circ_export_gates(circ_t circ, const double* theta, int32_t* bond, double* U);
/* Circuit-level variant (a gate-count optimisation on top of the paper's canonical
 * list): consecutive gates on the same bond are multiplied into one, fixed gates next
 * to a parametric gate are folded into it, identity products are dropped. The state
 * is the same in exact arithmetic; truncated evaluations take fewer SVD steps and so
 * differ slightly. Rewrites circ in place; n_gates (optional) receives the new count.
 * Parameter-shift gradients stay exact (shifts act on the parametric gates only). */
int circ_fuse_gates(circ_t circ, int64_t* n_gates);
/* Circuit-level variant: ladder cancellation between consecutive exponentials. The
 * UCCSD ansatz is a first-order Trotter product over excitations (Sec. II); inside one
 * excitation the Pauli strings of its generator commute, so their exponentials can be
 * applied in any order with the same product. Inside every run of consecutive rotations
 * that share one parameter and commute pairwise, the rotations are put in ascending
 * order of their letters read from the lowest non-identity site up; consecutive
 * rotations then agree on their lowest sites, where the descending CNOT ladder of one
 * meets the ascending ladder of the next, and the gate list is recompiled and fused as
 * by circ_fuse_gates (gate fusion, Sec. III-A), which cancels those ladder segments pair
 * by pair. Same state as the canonical list in exact arithmetic (the 24-qubit,
 * 12-electron UCCSD circuit goes from 442 272 to 252 095 gates); truncated evaluations
 * take fewer SVD steps and so differ slightly. Rewrites circ in place; n_gates
 * (optional) receives the new count. Parameter-shift gradients stay exact. */
int circ_cancel_ladders(circ_t circ, int64_t* n_gates);
int circ_destroy(circ_t circ);

/* ------------------------------------------------------------------ MPS state */

/* Allocate n_slots MPS states of n_qubits sites with bond cap chi (Eq. 6) on the
 * current device, each initialised to the all-zero product state. precision:
 * MPS_FP64 (complex128 tensors, FP64 SVD and contractions) or MPS_MIXED (complex64
 * tensors, FP32 SVD with a compensated re-orthonormalisation of the kept singular
 * vectors, FP32 gate contractions, environment contractions of bonds >= 128 on the
 * tensor cores with compensated TF32 splits, FP64 Schmidt numbers and energy sums).
 * cuda_stream: a cudaStream_t (NULL = default stream). Device memory is taken and
 * returned stream-ordered on that stream. n_qubits in [2, 128], chi in [1, 256],
 * n_slots in [1, 4096]; gates are applied at chi <= 128 only (the calls that apply
 * gates return MPS_EINVAL above), larger chi serves states loaded with mps_set_state
 * and measured. Errors: MPS_EINVAL, MPS_ENOMEM, MPS_ECUDA. */
int mps_create(int n_qubits, int chi, int precision, int n_slots, void* cuda_stream, mps_t* out);

/* Sec. III-D: reset slot to the product state |occ_0 occ_1 ...> (bytes 0/1), all
 * bond ranks 1, lambda = [1]. */
int mps_reset(mps_t mps, int slot, const uint8_t* occ);

/* Truncation controls (Eq. 9): keep k = min(chi, #{sigma > cutoff * sigma_0}).
 * Defaults: cutoff 1e-13 (FP64) or 2^-20 (mixed). max_sweeps (default 60) caps the
 * sweeps of the one-sided Jacobi SVD that replaces the bidiagonal route for a gate
 * whose spectrum is numerically degenerate without a split; a gate that reaches the
 * cap is counted in n_svd_noconv and the call returns MPS_ENOCONV. */
int mps_set_svd_params(mps_t mps, double cutoff, int max_sweeps);

/* Memory of the trie measurement (Sec. III-C; no counterpart in the paper's text). The
 * prefix trie of the strings is walked depth first in chunks of consecutive nodes of one
 * level, each level keeping environment buffers (3 chi^2 complex entries per node) for
 * one chunk: bytes bounds the sum of those buffers (at least 16 nodes per level); the
 * tensor-core scratch of mixed precision then takes a quarter of bytes (at least 64 MiB).
 * 0 restores the default, 4 GiB for chi <= 128 and 48 GiB above, which mps_estimate_bytes
 * assumes. Results do not depend on the chunking. */
int mps_set_meas_budget(mps_t mps, size_t bytes);

/* Sec. III-A, Eqs. (7)-(10), for every gate of circ on slot 0 in order: contract
 * B_n B_{n+1} with the gate, scale rows by lambda_{n-1}, truncated SVD, B_{n+1} <- V,
 * B_n <- M V^+, lambda_n <- sigma. theta: n_params doubles. *discarded_weight
 * (may be NULL) receives the sum over gates of the discarded fraction
 * sum_dropped sigma^2 / sum sigma^2 (Eq. 9's monitored truncation error).
 * Returns MPS_ENOCONV if any SVD hit the sweep cap (state is still updated). */
int mps_apply_circuit(mps_t mps, circ_t circ, const double* theta, double* discarded_weight);

/* Same as mps_apply_circuit for explicit gates on slot 0: bond[g] in [0, n-2],
 * U: n_gates x 4 x 4 complex (row index 2 i_b + i_{b+1}). */
int mps_apply_gates(mps_t mps, int64_t n_gates, const int32_t* bond, const double* U,
                    double* discarded_weight);

/* Eq. (11) generalised to Pauli strings (Sec. III-C): re[i] + i im[i] =
 * <psi|P_i|psi> / <psi|psi> on slot 0, by exact transfer-matrix contraction over
 * a prefix trie (shared left environments, walked depth first in chunks) and right
 * identity environments. Returns MPS_ETIMEOUT if a bounded wait inside a tensor-core
 * GEMM ran out (mixed precision). */
int mps_expect_paulis(mps_t mps, int64_t n_terms, const uint8_t* paulis, double* re, double* im);

/* Checkpoint / inspection of one slot. ranks: n_qubits-1 bond ranks.
 * B: concatenated site tensors, site k of shape (r_{k-1}, 2, r_k) row-major complex;
 * lam: concatenated Schmidt numbers of bonds 0..n-2. mps_state_size gives the
 * number of complex entries of B and doubles of lam for the current ranks. */
int mps_get_ranks(mps_t mps, int slot, int32_t* ranks);
int mps_state_size(mps_t mps, int slot, int64_t* n_B, int64_t* n_lam);
int mps_get_state(mps_t mps, int slot, double* B, double* lam);
int mps_set_state(mps_t mps, int slot, const int32_t* ranks, const double* B, const double* lam);

/* Eq. (2), Sec. III-C: E = sum_i a_i Re<P_i> / <psi|psi> of the state slot 0 holds now
 * (no reset, no circuit), by the same trie measurement and Neumaier-compensated FP64
 * sum in trie order as vqe_energy. */
int mps_energy(mps_t mps, ham_t ham, double* energy);

/* Sec. III-C/III-D energy evaluation on slot 0: reset to the reference
 * determinant of circ (circ_set_reference), apply circ with theta, evaluate every term
 * of ham, and return E = sum_i a_i Re<P_i> / <psi|psi> (Neumaier-compensated FP64
 * sum in trie order). */
int vqe_energy(mps_t mps, circ_t circ, ham_t ham, const double* theta, double* energy);

/* n_batch independent evaluations (slots 0..n_batch-1, n_batch <= n_slots);
 * thetas: n_batch x n_params; energies: n_batch. */
int vqe_energy_batch(mps_t mps, circ_t circ, ham_t ham, int n_batch, const double* thetas,
                     double* energies);

/* Parameter-shift gradient dE/dtheta_e for the n_sel parameters sel[] (not in the
 * paper, which optimises with energies only; the rule is exact for rotations
 * exp(-i phi P / 2)): sum over the rotations k of e of
 * scale_k [E(phi_k + pi/2) - E(phi_k - pi/2)] / 2.
 * With n_slots >= 3 the shifted circuits share prefixes: slot 0 carries the unshifted
 * circuit up to rotation k's parametric gate, where its state is copied to two slots
 * that continue with phi_k +- pi/2; up to (n_slots - 1) / 2 rotations run together in
 * one batched pass. With fewer slots each shifted circuit runs from the reference
 * state in slot 0. Both routes do the same arithmetic per gate, so they agree bit for
 * bit. The contents of every slot are overwritten. Returns MPS_ENOCONV if any
 * evaluation hit the Jacobi sweep cap (grad is still written). */
int vqe_gradient(mps_t mps, circ_t circ, ham_t ham, const double* theta, int n_sel,
                 const int32_t* sel, double* grad);

/* Per-call statistics of the last apply/energy call on this handle. */
typedef struct {
  double discarded_weight; /* summed discarded fraction, slot 0                   */
  int32_t max_rank;        /* largest bond rank reached, slot 0                   */
  int32_t max_sweeps;      /* most bisection refinement passes of one gate        */
  int64_t n_gates;         /* gates applied per slot                               */
  int64_t n_svd_noconv;    /* Jacobi fallbacks that hit their sweep cap, summed    */
                           /* over the slots of the call                           */
  double ms_circuit;       /* CUDA-event time of the circuit kernels               */
  double ms_measure;       /* CUDA-event time of the measurement kernels           */
  int64_t kernel_launches; /* device kernels launched by the call                  */
  double cycles[7];        /* slot-0 SM clock cycles per gate-engine phase since   */
                           /* creation: build M', bidiagonalise, bisection,        */
                           /* twisted vectors, re-orthonormalise, back-transform,  */
                           /* site update                                          */
  int64_t n_fallback;      /* gates whose SVD fell back to one-sided Jacobi        */
                           /* (numerically degenerate Schmidt values), slot 0      */
  double alg_flops_total;  /* slot-0 algorithmic real flops of all gate steps      */
                           /* since creation (dense contraction + Golub-Reinsch    */
                           /* SVD with right vectors + site update)                */
  int64_t n_nonfinite;     /* gates skipped because M' held a NaN or Inf, summed   */
                           /* over the slots of the call                           */
  double alg_flops_call;   /* algorithmic real flops of this call's gate steps,    */
                           /* summed over every slot the call ran                  */
  int64_t tc_gemm_launches; /* tensor-core GEMMs of the call's measurements        */
  double tc_gemm_flops;    /* their algorithmic real flops (2 M N K each; the split */
                           /* products are not counted)                            */
  double ms_tc_gemm;       /* their summed CUDA-event time, when kernel timing is   */
                           /* on (mps_set_kernel_timing), else 0                   */
  double ms_close;         /* summed CUDA-event time of the close launches (<P> of  */
                           /* the strings ending at each level), same condition    */
} mps_stats_t;
int mps_get_stats(mps_t mps, mps_stats_t* stats);

/* Record CUDA events around every tensor-core GEMM launch and every close launch of
 * the measurement (on the handle's stream) and report their summed times in
 * mps_stats_t.ms_tc_gemm and ms_close; off by default (no paper counterpart: it serves
 * roofline reporting). */
int mps_set_kernel_timing(mps_t mps, int on);

/* Device bytes that a handle of these sizes would hold once it has run circ (null:
 * circuit buffers left out) and measured ham (null: measurement buffers left out).
 * No paper counterpart: serving loops use it to admit requests by device memory. The
 * figure counts the handle's own buffers (within a few KB), not allocator rounding. */
int mps_estimate_bytes(int n_qubits, int chi, int precision, int n_slots, circ_t circ, ham_t ham,
                       size_t* bytes);

int mps_destroy(mps_t mps);

/* Allocation-free gate application. The paper has no counterpart: this entry point
 * exists for callers that cannot have device memory allocated for them, such as
 * runtimes that hand out all device memory from their own pools, processes held to a
 * fixed device-memory budget, or code that may not call cudaMalloc or cudaFree at
 * this point of its run (both can synchronise the device). For them it applies
 * n_gates two-site gates (contraction with the 4x4 gate, row scaling by the Schmidt
 * numbers of the left bond, truncated SVD, site update; mixed precision) to ONE MPS
 * that lives entirely in caller-owned DEVICE memory, and allocates nothing: its
 * workspace is a 1 MiB file-scope device array inside this library, present on every
 * GPU that loads the library until the process exits. Limits: chi <= 64,
 * 2 <= n_qubits <= 128; larger sizes return MPS_EINVAL.
 *   site_tensors: complex64 (float re, im) entries; site k starts at element
 *                 site_offsets[k] and has room for cap_{k-1} x 2 x cap_k entries,
 *                 cap_b = min(chi, 2^min(b+1, n-1-b)) (cap_{-1} = cap_{n-1} = 1); the
 *                 current tensor (r_{k-1}, 2, r_k) is packed row-major at its start.
 *   site_offsets: n_qubits int64 (device). lambdas: (n_qubits-1) x chi doubles, bond b
 *                 at b * chi (device). ranks: n_qubits+1 int32, ranks[0] = ranks[n] = 1,
 *                 ranks[b+1] = rank of bond b, 1 <= ranks[b+1] <= cap_b (device). All
 *                 four are updated in place.
 *   bonds: n_gates int32 in [0, n_qubits-2] (device); gates: n_gates x 4 x 4
 *          complex128, row index 2 i_b + i_{b+1} (device). cuda_stream: stream for all
 *          work (NULL = default).
 *   discarded_weight: HOST pointer or NULL. When given, it receives the summed
 *          discarded fraction, the call waits for the stream, and problems that only
 *          the device can see are reported: MPS_EINVAL for a bond or rank outside the
 *          ranges above (the kernel checks them before indexing and stops there),
 *          MPS_ENONFINITE for a gate skipped on a NaN or Inf, MPS_ENOCONV for a Jacobi
 *          fallback that hit its sweep cap. With NULL the call does not wait and these
 *          three are not reported (out-of-range bonds and ranks are still never used).
 * The first call on each device looks up the workspace address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture. Every call
 * shares the one workspace, and each call clears the accumulators it reads, so calls
 * that overlap on the GPU (other streams or threads) race and must be serialised by the
 * caller. Returns MPS_EINVAL for null pointers or sizes beyond the limits, MPS_ECUDA if
 * a CUDA call fails. */
int mps_apply_gates_noalloc(int n_qubits, int chi, void* site_tensors, const int64_t* site_offsets,
                            double* lambdas, int32_t* ranks, int64_t n_gates, const int32_t* bonds,
                            const double* gates, void* cuda_stream, double* discarded_weight);

/* Real GEMM on the tensor cores (tcgen05, TMEM, TMA) with compensated TF32 splits:
 * C = A . B^T with A (M x K), B (N x K), C (M x N), all FP32 row-major DEVICE arrays
 * with leading dimensions lda, ldb >= K and ldc >= N. Inside the kernel each loaded
 * tile is split into hi = tf32(x) and lo = tf32(x - hi) and C is accumulated as
 * A_hi B_hi + A_hi B_lo + A_lo B_hi, each 32-wide K slice from zero, the slices summed
 * in round-to-nearest FP32 (relative error about 2^-21 of sum |a||b|, no drift with K).
 * This is the contraction primitive of the environment sweeps (Eq. 11, Sec. III-C) in
 * mixed precision, exported for tests and callers with their own operands. Takes a
 * small temporary error word, and a padded copy of any operand whose rows do not start
 * on 16-byte boundaries (lda or ldb not a multiple of 4, or a misaligned pointer), with
 * cudaMallocAsync on cuda_stream, and waits for the stream. Returns MPS_EINVAL for bad sizes or null pointers, MPS_ENOMEM,
 * MPS_ECUDA, or MPS_ETIMEOUT if a bounded pipeline wait inside the kernel ran out. */
int mps_tc_gemm_tf32x3(int M, int N, int K, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                       int64_t ldc, void* cuda_stream);

/* Thread-local description of the last error on this thread ("" if none). */
const char* mps_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MPSVQE_H */
