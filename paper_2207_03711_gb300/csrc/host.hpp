// Host-side structures of the MPS-VQE library: Pauli algebra, Jordan-Wigner
// Hamiltonian, UCCSD rotations, the two-site gate compiler and the prefix trie.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace mpsvqe {

using cd = std::complex<double>;
constexpr int kMaxQubits = 128;

// A Pauli operator in "XZ form": X^x Z^z = (x) X^{x_q} Z^{z_q} over qubits, with bit q
// of the masks for qubit q. Letters relate by Y = i X Z, so X^x Z^z = (-i)^{|x&z|} P.
struct XZ {
  uint64_t x[2] = {0, 0};
  uint64_t z[2] = {0, 0};
  bool operator==(const XZ& o) const {
    return x[0] == o.x[0] && x[1] == o.x[1] && z[0] == o.z[0] && z[1] == o.z[1];
  }
};
struct XZHash {
  size_t operator()(const XZ& k) const {
    uint64_t h = k.x[0] * 0x9E3779B97F4A7C15ull ^ (k.x[1] + 0x632BE59BD9B4E019ull);
    h ^= (k.z[0] + 0x85EBCA77C2B2AE63ull) * 0xC2B2AE3D27D4EB4Full;
    h ^= k.z[1] * 0x165667B19E3779F9ull;
    return (size_t)(h ^ (h >> 29));
  }
};

// Letter codes 0=I 1=X 2=Y 3=Z of an XZ key for n qubits.
void xz_to_letters(const XZ& k, int n, uint8_t* out);
XZ letters_to_xz(const uint8_t* code, int n);

struct Term {
  std::vector<uint8_t> code;
  double coeff;
};

// Weighted Pauli sum sorted in trie order plus the level structure used on device.
struct Trie {
  int n = 0;
  int n_levels = 0;                         // levels 0..n_levels-1 hold nodes
  std::vector<int32_t> level_nodes;         // nodes per level
  // node -> parent (level k+1 refers into level k) and the Pauli letter on edge
  std::vector<std::vector<int32_t>> parent;
  std::vector<std::vector<uint8_t>> edge;
  // closes at level k: (node at level k, letter at site k, term index)
  std::vector<std::vector<int32_t>> close_node;
  std::vector<std::vector<uint8_t>> close_letter;
  std::vector<std::vector<int32_t>> close_term;
  int64_t total_nodes = 0;
  int32_t max_level_nodes = 0;
  int32_t max_level_closes = 0;
};

// Strings must be in trie order (lexicographic, I < X < Y < Z). Identity strings are
// not closed in the trie (their expectation is 1).
void build_trie(int n, const std::vector<Term>& terms, Trie* trie);

// Eq. (1) -> Eq. (2) with chemist-order integrals, interleaved spin orbitals.
std::vector<Term> jordan_wigner(int n_spatial, const double* h, const double* eri, double e_core,
                                std::string* err);
// Merge duplicates, drop |a| <= rel_drop max|a|, sort in trie order.
std::vector<Term> canonical_terms(int n, std::vector<Term> terms, double rel_drop);

struct Rotation {
  std::vector<uint8_t> code;
  int32_t param;  // < 0: fixed angle phi = scale
  double scale;
};
std::vector<Rotation> uccsd_rotations(int n_qubits, int n_electrons, int* n_params);

// One compiled two-site gate. Constant gates: U = mats[m0]. Parametric gates:
// U = mats[m1] * R * mats[m0] with R = Rz(phi) on site rz_site (0: bond's left
// site, 1: right site) and phi = scale * theta[param].
struct GateRec {
  int32_t bond;
  int32_t param;
  int32_t m0;
  int32_t m1;
  double scale;
  int32_t rz_site;
  int32_t pad;
};
static_assert(sizeof(GateRec) == 32, "GateRec layout");

struct Compiled {
  int n = 0;
  int n_params = 0;
  std::vector<Rotation> rotations;
  std::vector<GateRec> gates;
  std::vector<cd> mats;          // 16 entries per matrix, row index 2 i_b + i_{b+1}
  std::vector<uint8_t> reference;
  std::vector<int64_t> rot_first_gate;  // first gate index of each rotation
};
void compile_rotations(int n, const std::vector<Rotation>& rots, Compiled* out);
// Circuit-level variant (not the paper's canonical list): consecutive gates on the same
// bond are multiplied into one, a fixed gate next to a parametric gate on the same bond
// is folded into its pre or post matrix, and products equal to the identity are
// dropped, so that the neighbours of a dropped pair meet in turn. The state is the
// same in exact arithmetic; truncated runs take fewer SVD steps. param_gate receives
// the index of each rotation's parametric gate (-1 if it has none); rot_first_gate is
// rewritten to the first gate that carries each rotation's work.
void fuse_gates(Compiled* c, std::vector<int64_t>* param_gate);
// Reorders the rotations inside every run of consecutive rotations that share one
// parameter and commute pairwise (the Pauli strings of one excitation's generator, whose
// exponentials commute, so the product is the same in any order): ascending by their
// letters read from the lowest non-identity site up. Consecutive rotations then agree on
// their lowest sites, where one's descending CNOT ladder meets the next one's ascending
// ladder, and fuse_gates cancels those ladder segments pair by pair. Returns the number
// of runs whose order changed.
int64_t order_for_ladder_cancellation(std::vector<Rotation>* rots);
// Gate of each rotation that carries its angle (-1 for a rotation without gates) in a
// list made by compile_rotations.
std::vector<int64_t> param_gates(const Compiled& c);
// Host evaluation of a gate matrix for a given theta (inspection only).
void gate_matrix(const Compiled& c, const GateRec& g, const double* theta, cd* U);

}  // namespace mpsvqe
