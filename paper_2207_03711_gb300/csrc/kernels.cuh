// Device-side entry points of the MPS-VQE engine (launchers called by api.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "host.hpp"

namespace mpsvqe {

enum { MPS_PREC_FP64 = 0, MPS_PREC_MIXED = 1 };

// Per-slot status words written by the gate engine: [0] most bisection passes of one
// gate, [1] Jacobi fallbacks that hit their sweep cap, [2] largest rank reached,
// [3] Jacobi fallbacks taken, [4] gates skipped because M' held a NaN or Inf,
// [5] set when a caller-owned bond or rank array was out of range (raw-gate launches),
// [6..7] unused.
constexpr int kStatWords = 8;

// Device view of n_slots MPS states that share one layout.
struct DevMPS {
  int n;                    // sites
  int chi;                  // bond cap
  int n_slots;
  int64_t slot_elems;       // complex entries of B per slot
  const int64_t* site_off;  // [n] entry offset of site k inside a slot
  void* B;                  // complex<R> [n_slots][slot_elems], site k = (r_{k-1}, 2, r_k) row-major
  double* lam;              // [n_slots][n-1][chi]
  int* rank;                // [n_slots][n+1]; rank[0] = rank[n] = 1, rank[b+1] = rank of bond b
  void* work_M;             // complex<R> [n_slots][(2chi)^2]  gate workspace (unscaled M)
  void* work_X;             // complex<R> [n_slots][2chi (2chi+16)]  M' when not in smem
  void* work_S;             // double [n_slots][16 chi^2]  SVD scratch (vectors, factorisations)
  double* dw;               // [n_slots] accumulated discarded weight
  int* stat;                // [n_slots][kStatWords] status words (see kStatWords)
  unsigned long long* prof; // [n_slots][8] clock cycles per gate-engine phase (thread 0)
};

struct CircDev {
  const GateRec* gates;
  int64_t n_gates;
  const double* mats;  // 32 doubles per matrix (16 complex)
  int n_params;
  const int32_t* raw_bond = nullptr;  // raw-gate launches only: bond of gate g, matrix g of mats
  // Optional per-block arrays (index blockIdx.x, i.e. slot - slot0): the first gate the
  // block applies, and a shift added to the rotation angle phi of one parametric gate
  // (parameter-shift evaluations forked from a shared prefix).
  const int64_t* start_gate = nullptr;
  const int64_t* shift_gate = nullptr;
  const double* shift_phi = nullptr;
};

// Reset slots [slot0, slot0+count) to product states; occ: [count][n] bytes (0/1).
cudaError_t launch_reset(const DevMPS& m, int prec, int slot0, int count, const uint8_t* occ_dev,
                         cudaStream_t st);

// Apply gates [g0, g1) to slots [slot0, slot0+count); theta_dev: [count][n_params].
cudaError_t launch_circuit(const DevMPS& m, int prec, const CircDev& c, int64_t g0, int64_t g1,
                           int slot0, int count, const double* theta_dev, double cutoff,
                           int max_sweeps, cudaStream_t st);

// Measurement workspace (device) for one slot at a time.
struct MeasDev {
  void* R;          // complex<R> [n+1][chi*chi] right identity environments R_k
  void* Bhat;       // complex<R> like one slot of B: B_k^i R_{k+1}
  void* Q;          // complex<R> [n][4][chi*chi]: Q_k^P = sum_ij conj(P_ij) Bhat_k^i (B_k^j)^+ per letter P
  double* vals;     // [n_terms][2] re, im of unnormalised <P>
  double* out;      // [4 + n_terms*2]: E, norm, ...
};


// Thread-local message returned by mps_last_error() (defined with the C ABI).
void set_error_message(const char* msg);

// ranks: the slot's n+1 bond ranks on the host (ranks[k] = left dimension of site k);
// site_off: the n site offsets on the host (DevMPS::site_off is the device copy).
cudaError_t launch_right_envs(const DevMPS& m, int prec, int slot, const int* ranks, const int64_t* site_off,
                              MeasDev& w, cudaStream_t st, int* launches);
// Chunked trie levels. Environment buffers: L holds node u's D_k x D_k block (row-major,
// leading dimension D_k) at u chi^2 complex entries; T holds T_j[u] = L[u] B_k^j
// (D_k x D_{k+1}, leading dimension D_{k+1}) at (2u + j) chi^2. Node indices in cnode /
// parent are absolute trie indices; node_base is the trie index of buffer entry 0.
cudaError_t launch_env_T(const DevMPS& m, int prec, int slot, int k, const void* L, void* T, int n_nodes,
                         cudaStream_t st);
cudaError_t launch_env_close(const DevMPS& m, int prec, int slot, int k, const void* L, const void* Q,
                             const int32_t* cnode, const uint8_t* cletter, const int32_t* cterm, int n_closes,
                             int node_base, double* vals, cudaStream_t st);
cudaError_t launch_env_child(const DevMPS& m, int prec, int slot, int k, const void* T, const int32_t* parent,
                             const uint8_t* edge, int n_children, int node_base, void* Lout, cudaStream_t st);
// E = sum_t coeff_t Re(vals_t) / norm + id_coeff (Neumaier, fixed order); also writes
// normalised <P_t> to out[4 + 2t], out[0] = E, out[1] = norm.
cudaError_t launch_energy_sum(const DevMPS& m, int prec, int slot, MeasDev& w, int64_t n_terms,
                              const double* coeff_dev, double id_coeff, int64_t id_term,
                              cudaStream_t st);

}  // namespace mpsvqe
