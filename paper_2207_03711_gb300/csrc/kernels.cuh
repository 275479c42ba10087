// Device-side entry points of the MPS-VQE engine (launchers called by api.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "host.hpp"

namespace mpsvqe {

enum { MPS_PREC_FP64 = 0, MPS_PREC_MIXED = 1 };

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
  int* stat;                // [n_slots][4]: bisection passes, collapsed vectors, max rank, error flag
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
  void* L[2];       // complex<R> [max_level_nodes][chi*chi] ping-pong left environments
  void* T;          // complex<R> [max_level_nodes][2][chi*chi]
  double* vals;     // [n_terms][2] re, im of unnormalised <P>
  double* out;      // [4 + n_terms*2]: E, norm, ...
};

struct TrieLevelDev {
  int32_t n_nodes;
  int32_t n_children;          // nodes at level k+1
  const int32_t* parent;       // [n_children] parent node at level k
  const uint8_t* edge;         // [n_children]
  int32_t n_closes;
  const int32_t* close_node;
  const uint8_t* close_letter;
  const int32_t* close_term;
};

// Thread-local message returned by mps_last_error() (defined with the C ABI).
void set_error_message(const char* msg);

cudaError_t launch_right_envs(const DevMPS& m, int prec, int slot, MeasDev& w, cudaStream_t st);
cudaError_t launch_level(const DevMPS& m, int prec, int slot, MeasDev& w, int k,
                         const TrieLevelDev& lv, int parity, cudaStream_t st, int* launches);
// E = sum_t coeff_t Re(vals_t) / norm + id_coeff (Neumaier, fixed order); also writes
// normalised <P_t> to out[4 + 2t], out[0] = E, out[1] = norm.
cudaError_t launch_energy_sum(const DevMPS& m, int prec, int slot, MeasDev& w, int64_t n_terms,
                              const double* coeff_dev, double id_coeff, int64_t id_term,
                              cudaStream_t st);

}  // namespace mpsvqe
