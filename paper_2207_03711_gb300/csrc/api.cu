// C ABI of the MPS-VQE engine: handles, device memory layout and the host-side
// orchestration of the kernels in kernels.cu. See include/mpsvqe.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mpsvqe.h"
#include "host.hpp"
#include "env_tc.cuh"
#include "kernels.cuh"

using namespace mpsvqe;

namespace {
constexpr double kHalfPi = 1.5707963267948966;
constexpr int kMaxChi = 256;        // largest bond cap of a handle (measurement)
constexpr int kMaxGateChi = 128;    // largest bond cap the gate engine applies gates at
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  return fail(MPS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CU(call)                                                 \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
  } while (0)

// Every device allocation of the library goes through dev_alloc. Allocations are
// stream-ordered (cudaMallocAsync / cudaFreeAsync from the device's memory pool) on the
// stream of the handle that owns them, so creating or destroying one handle never waits
// for work other handles have in flight on other streams (a plain cudaFree synchronises
// the whole device). Host-side fault injection for tests: with MPS_FAULT_ALLOC_AFTER=k in
// the environment, the allocations of one mps_create (or of one measurement-buffer
// set-up) after the first k fail with MPS_ENOMEM, without touching the device.
thread_local long g_alloc_count = 0;
void reset_alloc_count() { g_alloc_count = 0; }
int dev_alloc(void** p, size_t bytes, const char* what, cudaStream_t st = nullptr) {
  *p = nullptr;
  if (const char* env = std::getenv("MPS_FAULT_ALLOC_AFTER")) {
    if (g_alloc_count++ >= std::atol(env))
      return fail(MPS_ENOMEM, std::string(what) + ": device allocation failed (injected fault)");
  }
  cudaError_t e = cudaMallocAsync(p, bytes == 0 ? 1 : bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(MPS_ENOMEM, std::string(what) + ": cudaMallocAsync: " + cudaGetErrorString(e));
  }
  return MPS_OK;
}

template <class T>
int dalloc(T** p, size_t count, cudaStream_t st = nullptr) {
  void* q = nullptr;
  const int rc = dev_alloc(&q, (count == 0 ? 1 : count) * sizeof(T), "device buffer", st);
  *p = (T*)q;
  return rc;
}
#define TRY(call)              \
  do {                         \
    int r_ = (call);           \
    if (r_ != MPS_OK) return r_; \
  } while (0)

// Every call of the library has finished its device work when it returns, so a buffer
// is idle when its handle is destroyed and can go back to the pool in the order of any
// stream; the legacy stream is used for the shared circuit and Hamiltonian tables.
void dfree(void* p, cudaStream_t st = nullptr) {
  if (p) cudaFreeAsync(p, st);
}
}  // namespace

namespace mpsvqe {
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace mpsvqe

// ----------------------------------------------------------------------- handles
struct ham_s {
  int n = 0;
  std::vector<Term> terms;  // trie order
  Trie trie;
  double id_coeff = 0.0;
  int64_t id_term = -1;
  // device copies (current device at upload)
  bool uploaded = false;
  double* d_coeff = nullptr;
  std::vector<int32_t*> d_parent, d_cnode, d_cterm;
  std::vector<uint8_t*> d_edge, d_cletter;
  ~ham_s() {
    dfree(d_coeff);
    for (auto p : d_parent) dfree(p);
    for (auto p : d_cnode) dfree(p);
    for (auto p : d_cterm) dfree(p);
    for (auto p : d_edge) dfree(p);
    for (auto p : d_cletter) dfree(p);
  }
};

struct circ_s {
  Compiled comp;
  std::vector<int64_t> rot_param_gate;  // gate carrying Rz of each rotation (-1 if none)
  bool uploaded = false;
  GateRec* d_gates = nullptr;
  double* d_mats = nullptr;
  ~circ_s() {
    dfree(d_gates);
    dfree(d_mats);
  }
};

struct mps_s {
  int n = 0, chi = 0, prec = 0, n_slots = 0;
  size_t es = 0;  // bytes per complex entry
  cudaStream_t st = nullptr;
  std::vector<int> cap;            // cap of bond b at index b+1; cap[0] = cap[n] = 1
  std::vector<int64_t> site_off;
  DevMPS dm{};
  int64_t* d_site_off = nullptr;
  MeasDev w{};
  int64_t w_terms = 0;
  // chunked trie measurement: per level, environment buffers for up to lvl_cap[k] nodes
  std::vector<void*> lvl_L, lvl_T;
  std::vector<int32_t> lvl_cap;
  size_t meas_budget = 0;          // 0: the default of meas_plan
  EnvTc tc{};
  // optional per-launch timing of the tensor-core GEMMs (mps_set_kernel_timing)
  bool ktime = false;
  std::vector<cudaEvent_t> kev;
  std::vector<uint8_t> kev_kind;   // per used pair: 0 tensor-core GEMM, 1 close
  size_t kev_used = 0;
  size_t tc_floats = 0;
  double* d_theta = nullptr;
  size_t theta_cap = 0;
  uint8_t* d_occ = nullptr;
  int64_t* d_start_gate = nullptr;
  int64_t* d_shift_gate = nullptr;
  double* d_shift_val = nullptr;
  double cutoff = 1e-13;
  int max_sweeps = 60;
  mps_stats_t stats{};
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<double> h_out;
  ~mps_s() {
    dfree(dm.B, st);
    dfree(dm.lam, st);
    dfree(dm.rank, st);
    dfree(dm.work_M, st);
    dfree(dm.work_X, st);
    dfree(dm.work_S, st);
    dfree(dm.dw, st);
    dfree(dm.stat, st);
    dfree(dm.prof, st);
    dfree(d_site_off, st);
    dfree(w.R, st);
    dfree(w.Bhat, st);
    dfree(w.Q, st);
    for (void* p : lvl_L) dfree(p, st);
    for (void* p : lvl_T) dfree(p, st);
    dfree(tc.scratch, st);
    dfree(tc.err, st);
    dfree(w.vals, st);
    dfree(w.out, st);
    dfree(d_theta, st);
    dfree(d_occ, st);
    dfree(d_start_gate, st);
    dfree(d_shift_gate, st);
    dfree(d_shift_val, st);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    for (auto e : kev)
      if (e) cudaEventDestroy(e);
  }
};

// ------------------------------------------------------------------ host helpers
static int make_ham(int n, std::vector<Term> terms, ham_t* out) {
  auto h = std::make_unique<ham_s>();
  h->n = n;
  h->terms = std::move(terms);
  for (size_t t = 0; t < h->terms.size(); ++t) {
    bool id = std::all_of(h->terms[t].code.begin(), h->terms[t].code.end(), [](uint8_t c) { return c == 0; });
    if (id) {
      h->id_term = (int64_t)t;
      h->id_coeff = h->terms[t].coeff;
    }
  }
  build_trie(n, h->terms, &h->trie);
  *out = h.release();
  return MPS_OK;
}

static int upload_ham(ham_s* h) {
  if (h->uploaded) return MPS_OK;
  const int n = h->n;
  std::vector<double> co(h->terms.size());
  for (size_t t = 0; t < co.size(); ++t) co[t] = h->terms[t].coeff;
  TRY(dalloc(&h->d_coeff, co.size()));
  CU(cudaMemcpy(h->d_coeff, co.data(), co.size() * 8, cudaMemcpyHostToDevice));
  h->d_parent.assign(n, nullptr);
  h->d_edge.assign(n, nullptr);
  h->d_cnode.assign(n, nullptr);
  h->d_cletter.assign(n, nullptr);
  h->d_cterm.assign(n, nullptr);
  const Trie& t = h->trie;
  for (int k = 0; k < n; ++k) {
    if (!t.parent[k].empty()) {
      TRY(dalloc(&h->d_parent[k], t.parent[k].size()));
      TRY(dalloc(&h->d_edge[k], t.edge[k].size()));
      CU(cudaMemcpy(h->d_parent[k], t.parent[k].data(), t.parent[k].size() * 4, cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h->d_edge[k], t.edge[k].data(), t.edge[k].size(), cudaMemcpyHostToDevice));
    }
    if (!t.close_term[k].empty()) {
      TRY(dalloc(&h->d_cnode[k], t.close_node[k].size()));
      TRY(dalloc(&h->d_cletter[k], t.close_letter[k].size()));
      TRY(dalloc(&h->d_cterm[k], t.close_term[k].size()));
      CU(cudaMemcpy(h->d_cnode[k], t.close_node[k].data(), t.close_node[k].size() * 4, cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h->d_cletter[k], t.close_letter[k].data(), t.close_letter[k].size(), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h->d_cterm[k], t.close_term[k].data(), t.close_term[k].size() * 4, cudaMemcpyHostToDevice));
    }
  }
  h->uploaded = true;
  return MPS_OK;
}

static int finish_circ(int n, std::vector<Rotation> rots, int n_params, circ_t* out) {
  auto c = std::make_unique<circ_s>();
  c->comp.n_params = n_params;
  compile_rotations(n, rots, &c->comp);
  c->comp.reference.assign(n, 0);
  c->rot_param_gate = param_gates(c->comp);
  *out = c.release();
  return MPS_OK;
}

static int upload_circ(circ_s* c) {
  if (c->uploaded) return MPS_OK;
  TRY(dalloc(&c->d_gates, c->comp.gates.size()));
  TRY(dalloc(&c->d_mats, c->comp.mats.size() * 2));
  if (!c->comp.gates.empty())
    CU(cudaMemcpy(c->d_gates, c->comp.gates.data(), c->comp.gates.size() * sizeof(GateRec), cudaMemcpyHostToDevice));
  if (!c->comp.mats.empty())
    CU(cudaMemcpy(c->d_mats, c->comp.mats.data(), c->comp.mats.size() * 16, cudaMemcpyHostToDevice));
  c->uploaded = true;
  return MPS_OK;
}

static int ensure_theta(mps_s* m, size_t count) {
  if (count <= m->theta_cap) return MPS_OK;
  dfree(m->d_theta, m->st);
  m->d_theta = nullptr;
  m->theta_cap = 0;
  TRY(dalloc(&m->d_theta, count, m->st));
  m->theta_cap = count;
  return MPS_OK;
}

// Chunked measurement plan. The prefix trie is walked depth first in chunks of
// consecutive nodes of one level, so only one chunk per level is live: level k keeps
// environment buffers (L: chi^2, T: 2 chi^2 complex entries per node) for cap[k] nodes.
// cap[k] = min(nodes of level k, U) with U set by a per-handle budget (4 GiB of level
// buffers for chi <= 128, 48 GiB above) spread over the levels; in mixed precision the
// tensor-core scratch holds tc_nodes nodes (about 1 GiB for chi <= 128, 4 GiB above).
constexpr int kTcMinDim = 128;    // levels with both bonds >= 128 use the tensor cores
struct MeasPlan {
  std::vector<int32_t> cap;
  int tc_nodes = 0;
  size_t level_bytes = 0, tc_bytes = 0;
};
static MeasPlan meas_plan(const Trie& t, int chi, size_t es, bool mixed, size_t budget = 0) {
  MeasPlan p;
  const size_t chi2 = (size_t)chi * chi, node_bytes = 3 * chi2 * es;
  const bool explicit_budget = budget != 0;
  if (budget == 0) budget = (chi <= 128 ? size_t(4) : size_t(48)) << 30;
  const size_t per_level = budget / (size_t)std::max(1, t.n_levels);
  const int32_t U = (int32_t)std::max<size_t>(16, per_level / node_bytes);
  p.cap.assign(t.n, 0);
  int32_t cmax = 1;
  for (int k = 0; k < t.n_levels; ++k) {
    p.cap[k] = std::min(t.level_nodes[k], U);
    cmax = std::max(cmax, p.cap[k]);
    p.level_bytes += (size_t)p.cap[k] * node_bytes;
  }
  if (mixed && chi >= kTcMinDim) {
    const size_t per_node = 24 * chi2;    // bytes of the W rows and GEMM-C output per child
    // a quarter of an explicit budget, else 1 GiB (chi <= 128) or 4 GiB
    const size_t tc_budget = explicit_budget ? std::max<size_t>(size_t(64) << 20, budget / 4)
                                             : (chi <= 128 ? size_t(1) : size_t(4)) << 30;
    // at most 65 535 children per chunk: the W-row kernel puts one child per grid z index
    p.tc_nodes = (int)std::min<size_t>(std::min<size_t>((size_t)cmax, 65535),
                                       std::max<size_t>(32, tc_budget / per_node));
    p.tc_bytes = env_tc_scratch_floats(chi, p.tc_nodes) * sizeof(float) + 256;
  }
  return p;
}

static int ensure_meas(mps_s* m, ham_s* h) {
  const size_t chi2 = (size_t)m->chi * m->chi;
  const int64_t terms = std::max<int64_t>(1, (int64_t)h->terms.size());
  reset_alloc_count();
  if (!m->w.R) {
    void* p;
    TRY(dev_alloc(&p, (size_t)(m->n + 1) * chi2 * m->es, "right environments", m->st));
    m->w.R = p;
    TRY(dev_alloc(&p, (size_t)m->dm.slot_elems * m->es, "B-hat", m->st));
    m->w.Bhat = p;
    TRY(dev_alloc(&p, (size_t)m->n * 4 * chi2 * m->es, "per-letter right blocks", m->st));
    m->w.Q = p;
  }
  const MeasPlan plan = meas_plan(h->trie, m->chi, m->es, m->prec == MPS_MIXED, m->meas_budget);
  m->lvl_L.resize(m->n, nullptr);
  m->lvl_T.resize(m->n, nullptr);
  m->lvl_cap.resize(m->n, 0);
  for (int k = 0; k < m->n; ++k) {
    if (plan.cap[k] <= m->lvl_cap[k]) continue;
    dfree(m->lvl_L[k], m->st);
    dfree(m->lvl_T[k], m->st);
    m->lvl_L[k] = m->lvl_T[k] = nullptr;
    m->lvl_cap[k] = 0;
    TRY(dev_alloc(&m->lvl_L[k], (size_t)plan.cap[k] * chi2 * m->es, "environment buffer", m->st));
    TRY(dev_alloc(&m->lvl_T[k], (size_t)plan.cap[k] * 2 * chi2 * m->es, "T buffer", m->st));
    m->lvl_cap[k] = plan.cap[k];
  }
  if (plan.tc_nodes > m->tc.max_nodes) {
    dfree(m->tc.scratch, m->st);
    m->tc.scratch = nullptr;
    m->tc.max_nodes = 0;
    void* p;
    TRY(dev_alloc(&p, plan.tc_bytes, "tensor-core scratch", m->st));
    m->tc.scratch = (float*)p;
    if (!m->tc.err) TRY(dalloc(&m->tc.err, 1, m->st));
    m->tc.chi = m->chi;
    m->tc.max_nodes = plan.tc_nodes;
  }
  if (terms > m->w_terms) {
    dfree(m->w.vals, m->st);
    dfree(m->w.out, m->st);
    m->w.vals = m->w.out = nullptr;
    m->w_terms = 0;
    TRY(dalloc(&m->w.vals, (size_t)terms * 2, m->st));
    TRY(dalloc(&m->w.out, 4 + (size_t)terms * 2, m->st));
    m->w_terms = terms;
  }
  return MPS_OK;
}

// Sum over slots [slot0, slot0 + count) of the algorithmic flops the gate engine has
// counted since creation (profile word 7 of each slot, a double).
static int sum_slot_flops(mps_s* m, int slot0, int count, double* total) {
  std::vector<unsigned long long> pr((size_t)count * 8);
  CU(cudaMemcpy(pr.data(), m->dm.prof + (size_t)slot0 * 8, pr.size() * 8, cudaMemcpyDeviceToHost));
  double t = 0.0;
  for (int s = 0; s < count; ++s) {
    double f;
    std::memcpy(&f, &pr[(size_t)s * 8 + 7], 8);
    t += f;
  }
  *total = t;
  return MPS_OK;
}

// Apply the circuit to slots [slot0, slot0 + count) with per-slot parameters thetas
// ([count][n_params], host; null keeps the device copy). Optional per-slot host arrays:
// start (first gate), shift_gate / shift_phi (angle shift of one parametric gate).
// Gates [min start, g_end) are launched; g_end < 0 means the whole list.
static int run_circuit(mps_s* m, circ_s* c, int slot0, int count, const double* thetas,
                       const int64_t* start = nullptr, const int64_t* shift_gate = nullptr,
                       const double* shift_phi = nullptr, int64_t g_end = -1) {
  if (m->chi > kMaxGateChi)
    return fail(MPS_EINVAL, "gate application supports bond caps up to 128; a handle with a larger chi can be "
                            "loaded (mps_set_state) and measured");
  TRY(upload_circ(c));
  const int np = std::max(1, c->comp.n_params);
  TRY(ensure_theta(m, (size_t)count * np));
  if (thetas && c->comp.n_params > 0)
    CU(cudaMemcpyAsync(m->d_theta, thetas, (size_t)count * np * 8, cudaMemcpyHostToDevice, m->st));
  CircDev cd{c->d_gates, (int64_t)c->comp.gates.size(), c->d_mats, np};
  const int64_t G = g_end < 0 ? (int64_t)c->comp.gates.size() : std::min<int64_t>(g_end, c->comp.gates.size());
  int64_t g_begin = 0;
  if (start) {
    g_begin = G;
    for (int b = 0; b < count; ++b) g_begin = std::min(g_begin, start[b]);
    CU(cudaMemcpyAsync(m->d_start_gate, start, (size_t)count * 8, cudaMemcpyHostToDevice, m->st));
    cd.start_gate = m->d_start_gate;
  }
  if (shift_gate && shift_phi) {
    CU(cudaMemcpyAsync(m->d_shift_gate, shift_gate, (size_t)count * 8, cudaMemcpyHostToDevice, m->st));
    CU(cudaMemcpyAsync(m->d_shift_val, shift_phi, (size_t)count * 8, cudaMemcpyHostToDevice, m->st));
    cd.shift_gate = m->d_shift_gate;
    cd.shift_phi = m->d_shift_val;
  }
  const int64_t chunk = 16384;
  double flops0 = 0.0, flops1 = 0.0;
  TRY(sum_slot_flops(m, slot0, count, &flops0));
  CU(cudaEventRecord(m->ev[0], m->st));
  int launches = 0;
  for (int64_t g0 = g_begin; g0 < G; g0 += chunk) {
    CU(launch_circuit(m->dm, m->prec, cd, g0, std::min(G, g0 + chunk), slot0, count, m->d_theta, m->cutoff,
                      m->max_sweeps, m->st));
    ++launches;
  }
  CU(cudaEventRecord(m->ev[1], m->st));
  CU(cudaEventSynchronize(m->ev[1]));
  float ms = 0;
  CU(cudaEventElapsedTime(&ms, m->ev[0], m->ev[1]));
  m->stats.ms_circuit += ms;
  m->stats.kernel_launches += launches;
  m->stats.n_gates = (int64_t)c->comp.gates.size();
  TRY(sum_slot_flops(m, slot0, count, &flops1));
  m->stats.alg_flops_call += flops1 - flops0;
  return MPS_OK;
}

// Copy the whole state of slot src (tensors, ranks, lambda, accumulators) to slot dst.
static int copy_slot(mps_s* m, int src, int dst) {
  const size_t sb = (size_t)m->dm.slot_elems * m->es;
  CU(cudaMemcpyAsync((char*)m->dm.B + dst * sb, (char*)m->dm.B + src * sb, sb, cudaMemcpyDeviceToDevice, m->st));
  const size_t nl = (size_t)(m->n - 1) * m->chi;
  CU(cudaMemcpyAsync(m->dm.lam + dst * nl, m->dm.lam + src * nl, nl * 8, cudaMemcpyDeviceToDevice, m->st));
  const size_t nr = (size_t)m->n + 1;
  CU(cudaMemcpyAsync(m->dm.rank + dst * nr, m->dm.rank + src * nr, nr * 4, cudaMemcpyDeviceToDevice, m->st));
  CU(cudaMemcpyAsync(m->dm.dw + dst, m->dm.dw + src, 8, cudaMemcpyDeviceToDevice, m->st));
  CU(cudaMemcpyAsync(m->dm.stat + kStatWords * dst, m->dm.stat + kStatWords * src, 4 * kStatWords,
                     cudaMemcpyDeviceToDevice, m->st));
  return MPS_OK;
}

static int upload_reset(mps_s* m, int slot0, int count, const uint8_t* occ_rows) {
  CU(cudaMemcpyAsync(m->d_occ, occ_rows, (size_t)count * m->n, cudaMemcpyHostToDevice, m->st));
  CU(launch_reset(m->dm, m->prec, slot0, count, m->d_occ, m->st));
  m->stats.kernel_launches += 1;
  return MPS_OK;
}

// Depth-first walk over the prefix trie in chunks (see meas_plan). Chunk [u0, u1) of
// level k has its environments L in lvl_L[k]; T_j = L B_k^j goes to lvl_T[k], the
// strings that close at level k are evaluated from it, and the children are built and
// walked chunk by chunk. Mixed precision runs the contractions of levels whose bonds
// are both >= kTcMinDim on the tensor cores (env_tc.cu), the others on the CUDA-core
// tile kernels; both use the same buffer layouts.
struct MeasWalk {
  mps_s* m;
  ham_s* h;
  int slot;
  std::vector<int> r;   // bond ranks of the slot, r[k] = left dimension of site k
  int launches = 0;
};

// The next pair of timing events (created on first use) when kernel timing is on.
static int next_event_pair(mps_s* m, cudaEvent_t* e0, cudaEvent_t* e1, uint8_t kind = 0) {
  *e0 = *e1 = nullptr;
  if (!m->ktime) return MPS_OK;
  m->kev_kind.resize(m->kev_used / 2 + 1);
  m->kev_kind[m->kev_used / 2] = kind;
  while (m->kev.size() < m->kev_used + 2) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    m->kev.push_back(e);
  }
  *e0 = m->kev[m->kev_used];
  *e1 = m->kev[m->kev_used + 1];
  m->kev_used += 2;
  return MPS_OK;
}

static int meas_chunk(MeasWalk& c, int k, int u0, int u1) {
  mps_s* m = c.m;
  const Trie& t = c.h->trie;
  const int U = u1 - u0, D = c.r[k], Dp = c.r[k + 1];
  void* L = m->lvl_L[k];
  void* T = m->lvl_T[k];
  // the tensor-core route reads L in place as rows of 2D floats, which TMA needs 16-byte
  // aligned: levels with an odd left bond stay on the CUDA-core kernels
  const bool tc = m->prec == MPS_MIXED && m->tc.scratch && D >= kTcMinDim && Dp >= kTcMinDim && (D & 1) == 0;
  if (tc) {
    const Cx<float>* Bk = (const Cx<float>*)m->dm.B + (size_t)c.slot * m->dm.slot_elems + m->site_off[k];
    CU(env_tc_site(m->tc, Bk, D, Dp, m->st));
    ++c.launches;
    cudaEvent_t e0, e1;
    TRY(next_event_pair(m, &e0, &e1));
    CU(env_tc_T(m->tc, (const Cx<float>*)L, (Cx<float>*)T, U, D, Dp, m->st, e0, e1));
    c.launches += 1;
    m->stats.tc_gemm_launches += 1;
    m->stats.tc_gemm_flops += 2.0 * ((double)U * D) * (4.0 * Dp) * (2.0 * D);
  } else {
    CU(launch_env_T(m->dm, m->prec, c.slot, k, L, T, U, m->st));
    ++c.launches;
  }
  // strings closing at level k on this chunk's nodes
  const auto& cn = t.close_node[k];
  const int64_t cs = std::lower_bound(cn.begin(), cn.end(), u0) - cn.begin();
  const int64_t ce = std::lower_bound(cn.begin(), cn.end(), u1) - cn.begin();
  if (ce > cs) {
    cudaEvent_t e0, e1;
    TRY(next_event_pair(m, &e0, &e1, 1));
    if (e0) CU(cudaEventRecord(e0, m->st));
    CU(launch_env_close(m->dm, m->prec, c.slot, k, L, m->w.Q, c.h->d_cnode[k] + cs, c.h->d_cletter[k] + cs,
                        c.h->d_cterm[k] + cs, (int)(ce - cs), u0, m->w.vals, m->st));
    if (e1) CU(cudaEventRecord(e1, m->st));
    ++c.launches;
  }
  if (k + 1 >= t.n_levels || k + 1 >= m->n) return MPS_OK;
  const auto& par = t.parent[k + 1];
  int64_t a = std::lower_bound(par.begin(), par.end(), u0) - par.begin();
  const int64_t c1 = std::lower_bound(par.begin(), par.end(), u1) - par.begin();
  while (a < c1) {
    int64_t b = a + 1;
    while (b < c1 && b - a < m->lvl_cap[k + 1] && (!tc || b - a < m->tc.max_nodes)) ++b;
    if (tc) {
      // the shared operands of site k live in the scratch, which the deeper levels of
      // the previous sub-chunk have used for their own sites: rebuild them
      const Cx<float>* Bk = (const Cx<float>*)m->dm.B + (size_t)c.slot * m->dm.slot_elems + m->site_off[k];
      CU(env_tc_site(m->tc, Bk, D, Dp, m->st));
      ++c.launches;
      cudaEvent_t e0, e1;
      TRY(next_event_pair(m, &e0, &e1));
      const int nch = (int)(b - a);
      CU(env_tc_children(m->tc, (const Cx<float>*)T, c.h->d_parent[k + 1] + a, c.h->d_edge[k + 1] + a, nch, u0,
                         D, Dp, (Cx<float>*)m->lvl_L[k + 1], m->st, e0, e1));
      c.launches += 3;
      m->stats.tc_gemm_launches += 1;
      m->stats.tc_gemm_flops += 2.0 * (2.0 * Dp) * ((double)nch * Dp) * (4.0 * D);
    } else {
      CU(launch_env_child(m->dm, m->prec, c.slot, k, T, c.h->d_parent[k + 1] + a, c.h->d_edge[k + 1] + a,
                          (int)(b - a), u0, m->lvl_L[k + 1], m->st));
      ++c.launches;
    }
    TRY(meas_chunk(c, k + 1, (int)a, (int)b));
    a = b;
  }
  return MPS_OK;
}

// Evaluate all terms of h on one slot; out_host receives 4 + 2 T doubles.
static int run_measure(mps_s* m, ham_s* h, int slot, double* out_host, bool terms = true) {
  TRY(upload_ham(h));
  const int64_t T = (int64_t)h->terms.size();
  TRY(ensure_meas(m, h));
  MeasWalk c{m, h, slot, std::vector<int>(m->n + 1)};
  CU(cudaStreamSynchronize(m->st));
  CU(cudaMemcpy(c.r.data(), m->dm.rank + (size_t)slot * (m->n + 1), (m->n + 1) * 4, cudaMemcpyDeviceToHost));
  if (m->tc.err) CU(cudaMemsetAsync(m->tc.err, 0, sizeof(int), m->st));
  m->kev_used = 0;
  CU(cudaEventRecord(m->ev[2], m->st));
  CU(launch_right_envs(m->dm, m->prec, slot, c.r.data(), m->site_off.data(), m->w, m->st, &c.launches));
  const Trie& t = h->trie;
  if (t.n_levels > 0) {
    // root environment L_0 = [1] (one node, D_0 = 1)
    static const double one_d[2] = {1.0, 0.0};
    static const float one_f[2] = {1.0f, 0.0f};
    CU(cudaMemcpyAsync(m->lvl_L[0], m->prec == MPS_FP64 ? (const void*)one_d : (const void*)one_f, m->es,
                       cudaMemcpyHostToDevice, m->st));
    TRY(meas_chunk(c, 0, 0, t.level_nodes[0]));
  }
  CU(launch_energy_sum(m->dm, m->prec, slot, m->w, T, h->d_coeff, h->id_term >= 0 ? h->id_coeff : 0.0,
                       h->id_term, m->st));
  ++c.launches;
  CU(cudaEventRecord(m->ev[3], m->st));
  CU(cudaMemcpyAsync(out_host, m->w.out, (4 + (terms ? 2 * (size_t)T : 0)) * 8, cudaMemcpyDeviceToHost, m->st));
  int tc_err = 0;
  if (m->tc.err) CU(cudaMemcpyAsync(&tc_err, m->tc.err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  CU(cudaStreamSynchronize(m->st));
  float ms = 0;
  CU(cudaEventElapsedTime(&ms, m->ev[2], m->ev[3]));
  m->stats.ms_measure += ms;
  m->stats.kernel_launches += c.launches;
  for (size_t i = 0; i + 1 < m->kev_used; i += 2) {
    float t = 0;
    CU(cudaEventElapsedTime(&t, m->kev[i], m->kev[i + 1]));
    (m->kev_kind[i / 2] ? m->stats.ms_close : m->stats.ms_tc_gemm) += t;
  }
  if (tc_err) return fail(MPS_ETIMEOUT, "a bounded wait of the tensor-core GEMM pipeline ran out");
  return MPS_OK;
}

static void reset_stats(mps_s* m) { m->stats = mps_stats_t{}; }

// ====================================================================== C ABI
extern "C" {

const char* mps_last_error(void) { return g_err.c_str(); }

int ham_jw_from_integrals(int n_spatial, const double* h, const double* eri, double e_core, ham_t* out) {
  if (!h || !eri || !out) return fail(MPS_EINVAL, "ham_jw_from_integrals: null pointer");
  if (n_spatial < 1 || n_spatial > 64) return fail(MPS_EINVAL, "ham_jw_from_integrals: n_spatial out of [1, 64]");
  std::string err;
  std::vector<Term> terms = jordan_wigner(n_spatial, h, eri, e_core, &err);
  if (!err.empty()) return fail(MPS_EINVAL, err);
  if (terms.empty()) return fail(MPS_EINVAL, "ham_jw_from_integrals: Hamiltonian is zero");
  return make_ham(2 * n_spatial, std::move(terms), out);
}

int ham_create(int n_qubits, int64_t n_terms, const uint8_t* paulis, const double* coeff, ham_t* out) {
  if (!paulis || !coeff || !out) return fail(MPS_EINVAL, "ham_create: null pointer");
  if (n_qubits < 2 || n_qubits > kMaxQubits || n_terms < 1) return fail(MPS_EINVAL, "ham_create: bad sizes");
  std::vector<Term> terms((size_t)n_terms);
  for (int64_t t = 0; t < n_terms; ++t) {
    terms[t].code.assign(paulis + t * n_qubits, paulis + (t + 1) * n_qubits);
    for (uint8_t c : terms[t].code)
      if (c > 3) return fail(MPS_EINVAL, "ham_create: Pauli code out of {0,1,2,3}");
    terms[t].coeff = coeff[t];
  }
  return make_ham(n_qubits, canonical_terms(n_qubits, std::move(terms), 0.0), out);
}

int ham_num_terms(ham_t h, int64_t* n_terms) {
  if (!h || !n_terms) return fail(MPS_EINVAL, "ham_num_terms: null pointer");
  *n_terms = (int64_t)h->terms.size();
  return MPS_OK;
}

int ham_get_terms(ham_t h, uint8_t* paulis, double* coeff) {
  if (!h) return fail(MPS_EINVAL, "ham_get_terms: null handle");
  for (size_t t = 0; t < h->terms.size(); ++t) {
    if (paulis) std::memcpy(paulis + t * h->n, h->terms[t].code.data(), h->n);
    if (coeff) coeff[t] = h->terms[t].coeff;
  }
  return MPS_OK;
}

int ham_destroy(ham_t h) {
  delete h;
  return MPS_OK;
}

int circ_uccsd(int n_qubits, int n_electrons, circ_t* out, int* n_params) {
  if (!out) return fail(MPS_EINVAL, "circ_uccsd: null pointer");
  if (n_qubits < 2 || n_qubits > kMaxQubits || n_electrons <= 0 || n_electrons >= n_qubits)
    return fail(MPS_EINVAL, "circ_uccsd: bad sizes");
  int np = 0;
  std::vector<Rotation> rots = uccsd_rotations(n_qubits, n_electrons, &np);
  TRY(finish_circ(n_qubits, std::move(rots), np, out));
  for (int q = 0; q < n_electrons; ++q) (*out)->comp.reference[q] = 1;
  if (n_params) *n_params = np;
  return MPS_OK;
}

int circ_create(int n_qubits, int64_t n_rot, const uint8_t* paulis, const int32_t* param_idx,
                const double* scale, circ_t* out) {
  if (!paulis || !param_idx || !scale || !out) return fail(MPS_EINVAL, "circ_create: null pointer");
  if (n_qubits < 2 || n_qubits > kMaxQubits || n_rot < 0) return fail(MPS_EINVAL, "circ_create: bad sizes");
  std::vector<Rotation> rots((size_t)n_rot);
  int np = 0;
  for (int64_t r = 0; r < n_rot; ++r) {
    rots[r].code.assign(paulis + r * n_qubits, paulis + (r + 1) * n_qubits);
    for (uint8_t c : rots[r].code)
      if (c > 3) return fail(MPS_EINVAL, "circ_create: Pauli code out of {0,1,2,3}");
    rots[r].param = param_idx[r];
    rots[r].scale = scale[r];
    np = std::max(np, param_idx[r] + 1);
  }
  return finish_circ(n_qubits, std::move(rots), np, out);
}

int circ_set_reference(circ_t c, const uint8_t* occ) {
  if (!c || !occ) return fail(MPS_EINVAL, "circ_set_reference: null pointer");
  for (int q = 0; q < c->comp.n; ++q) {
    if (occ[q] > 1) return fail(MPS_EINVAL, "circ_set_reference: occupation not 0/1");
    c->comp.reference[q] = occ[q];
  }
  return MPS_OK;
}

int circ_num_rotations(circ_t c, int64_t* n_rot, int* n_params) {
  if (!c) return fail(MPS_EINVAL, "circ_num_rotations: null handle");
  if (n_rot) *n_rot = (int64_t)c->comp.rotations.size();
  if (n_params) *n_params = c->comp.n_params;
  return MPS_OK;
}

int circ_get_rotations(circ_t c, uint8_t* paulis, int32_t* param_idx, double* scale) {
  if (!c) return fail(MPS_EINVAL, "circ_get_rotations: null handle");
  const int n = c->comp.n;
  for (size_t r = 0; r < c->comp.rotations.size(); ++r) {
    if (paulis) std::memcpy(paulis + r * n, c->comp.rotations[r].code.data(), n);
    if (param_idx) param_idx[r] = c->comp.rotations[r].param;
    if (scale) scale[r] = c->comp.rotations[r].scale;
  }
  return MPS_OK;
}

int circ_num_gates(circ_t c, int64_t* n_gates) {
  if (!c || !n_gates) return fail(MPS_EINVAL, "circ_num_gates: null pointer");
  *n_gates = (int64_t)c->comp.gates.size();
  return MPS_OK;
}

int circ_export_gates(circ_t c, const double* theta, int32_t* bond, double* U) {
  if (!c) return fail(MPS_EINVAL, "circ_export_gates: null handle");
  if (!theta && c->comp.n_params > 0) return fail(MPS_EINVAL, "circ_export_gates: theta is null");
  for (size_t g = 0; g < c->comp.gates.size(); ++g) {
    if (bond) bond[g] = c->comp.gates[g].bond;
    if (U) gate_matrix(c->comp, c->comp.gates[g], theta, reinterpret_cast<cd*>(U + 32 * g));
  }
  return MPS_OK;
}

int circ_fuse_gates(circ_t c, int64_t* n_gates) {
  if (!c) return fail(MPS_EINVAL, "circ_fuse_gates: null handle");
  fuse_gates(&c->comp, &c->rot_param_gate);
  c->uploaded = false;
  dfree(c->d_gates);
  dfree(c->d_mats);
  c->d_gates = nullptr;
  c->d_mats = nullptr;
  if (n_gates) *n_gates = (int64_t)c->comp.gates.size();
  return MPS_OK;
}

int circ_cancel_ladders(circ_t c, int64_t* n_gates) {
  if (!c) return fail(MPS_EINVAL, "circ_cancel_ladders: null handle");
  std::vector<Rotation> rots = c->comp.rotations;
  order_for_ladder_cancellation(&rots);
  const int np = c->comp.n_params;
  std::vector<uint8_t> ref = c->comp.reference;
  compile_rotations(c->comp.n, rots, &c->comp);
  c->comp.n_params = np;
  c->comp.reference = ref;
  c->rot_param_gate = param_gates(c->comp);
  return circ_fuse_gates(c, n_gates);
}

int circ_destroy(circ_t c) {
  delete c;
  return MPS_OK;
}

int mps_estimate_bytes(int n_qubits, int chi, int precision, int n_slots, circ_t circ, ham_t ham,
                       size_t* bytes) {
  if (!bytes) return fail(MPS_EINVAL, "mps_estimate_bytes: null pointer");
  if (n_qubits < 2 || n_qubits > kMaxQubits || chi < 1 || chi > kMaxChi || n_slots < 1 ||
      (precision != MPS_FP64 && precision != MPS_MIXED))
    return fail(MPS_EINVAL, "mps_estimate_bytes: bad sizes");
  const int n = n_qubits;
  const size_t es = precision == MPS_FP64 ? 16 : 8, S = (size_t)n_slots, mm = 2 * (size_t)chi;
  std::vector<int64_t> cap(n + 1, 1);
  for (int b = 0; b < n - 1; ++b) {
    const int e = std::min(b + 1, n - 1 - b);
    cap[b + 1] = e >= 30 ? chi : std::min(chi, 1 << e);
  }
  size_t slot = 0;
  for (int k = 0; k < n; ++k) slot += (size_t)cap[k] * 2 * cap[k + 1];
  size_t b = S * slot * es                          // site tensors
             + S * (n - 1) * chi * 8 + S * (n + 1) * 4  // lambda, ranks
             + S * mm * mm * es + S * mm * (mm + 16) * es + S * 16 * chi * chi * 8  // workspaces
             + S * (8 + 16 + 64 + n + 24) + (size_t)n * 8;
  const size_t chi2 = (size_t)chi * chi;
  b += (size_t)(n + 1) * chi2 * es + slot * es;     // right environments, B-hat
  b += (size_t)n * 4 * chi2 * es;                   // per-letter right blocks
  if (circ) b += circ->comp.gates.size() * sizeof(GateRec) + circ->comp.mats.size() * 16 +
                 S * std::max(1, circ->comp.n_params) * 8;
  if (ham) {
    const size_t T = ham->terms.size();
    const MeasPlan plan = meas_plan(ham->trie, chi, es, precision == MPS_MIXED);
    b += plan.level_bytes + plan.tc_bytes + (4 + 4 * T) * 8;   // chunk buffers, tensor-core scratch, values
    b += T * (8 + 4 + 1 + 4) + T * (size_t)n;                  // coefficients and the trie arrays
  }
  *bytes = b;
  return MPS_OK;
}

int mps_create(int n_qubits, int chi, int precision, int n_slots, void* cuda_stream, mps_t* out) {
  if (!out) return fail(MPS_EINVAL, "mps_create: null pointer");
  if (n_qubits < 2 || n_qubits > kMaxQubits) return fail(MPS_EINVAL, "mps_create: n_qubits out of [2, 128]");
  if (chi < 1 || chi > kMaxChi) return fail(MPS_EINVAL, "mps_create: chi out of [1, 256]");
  if (precision != MPS_FP64 && precision != MPS_MIXED) return fail(MPS_EINVAL, "mps_create: bad precision");
  if (n_slots < 1 || n_slots > 4096) return fail(MPS_EINVAL, "mps_create: n_slots out of [1, 4096]");
  reset_alloc_count();
  auto m = std::make_unique<mps_s>();
  m->n = n_qubits;
  m->chi = chi;
  m->prec = precision;
  m->n_slots = n_slots;
  m->es = precision == MPS_FP64 ? 16 : 8;
  m->st = (cudaStream_t)cuda_stream;
  m->cutoff = precision == MPS_FP64 ? 1e-13 : std::ldexp(1.0, -20);
  const int n = n_qubits;
  m->cap.assign(n + 1, 1);
  for (int b = 0; b < n - 1; ++b) {
    int e = std::min(b + 1, n - 1 - b);
    m->cap[b + 1] = e >= 30 ? chi : std::min(chi, 1 << e);
  }
  m->site_off.assign(n, 0);
  int64_t off = 0;
  for (int k = 0; k < n; ++k) {
    m->site_off[k] = off;
    off += (int64_t)m->cap[k] * 2 * m->cap[k + 1];
  }
  DevMPS& d = m->dm;
  d.n = n;
  d.chi = chi;
  d.n_slots = n_slots;
  d.slot_elems = off;
  const size_t mm = 2 * (size_t)chi;
  void* p;
  TRY(dev_alloc(&p, (size_t)n_slots * off * m->es, "mps_create: B", m->st));
  d.B = p;
  TRY(dalloc(&d.lam, (size_t)n_slots * (n - 1) * chi, m->st));
  TRY(dalloc(&d.rank, (size_t)n_slots * (n + 1), m->st));
  TRY(dev_alloc(&p, (size_t)n_slots * mm * mm * m->es, "mps_create: work_M", m->st));
  d.work_M = p;
  TRY(dev_alloc(&p, (size_t)n_slots * mm * (mm + 16) * m->es, "mps_create: work_X", m->st));
  d.work_X = p;
  TRY(dev_alloc(&p, (size_t)n_slots * 16 * chi * chi * sizeof(double), "mps_create: work_S", m->st));
  d.work_S = p;
  TRY(dalloc(&d.dw, n_slots, m->st));
  TRY(dalloc(&d.stat, (size_t)n_slots * kStatWords, m->st));
  TRY(dalloc(&d.prof, (size_t)n_slots * 8, m->st));
  CU(cudaMemsetAsync(d.prof, 0, (size_t)n_slots * 8 * 8, m->st));
  TRY(dalloc(&m->d_site_off, n, m->st));
  CU(cudaMemcpyAsync(m->d_site_off, m->site_off.data(), n * 8, cudaMemcpyHostToDevice, m->st));
  d.site_off = m->d_site_off;
  TRY(dalloc(&m->d_occ, (size_t)n_slots * n, m->st));
  TRY(dalloc(&m->d_start_gate, n_slots, m->st));
  TRY(dalloc(&m->d_shift_gate, n_slots, m->st));
  TRY(dalloc(&m->d_shift_val, n_slots, m->st));
  for (auto& e : m->ev) CU(cudaEventCreate(&e));
  std::vector<uint8_t> zeros((size_t)n_slots * n, 0);
  TRY(upload_reset(m.get(), 0, n_slots, zeros.data()));
  CU(cudaStreamSynchronize(m->st));
  *out = m.release();
  return MPS_OK;
}

int mps_destroy(mps_t m) {
  if (m) cudaStreamSynchronize(m->st);
  delete m;
  return MPS_OK;
}

int mps_reset(mps_t m, int slot, const uint8_t* occ) {
  if (!m || !occ) return fail(MPS_EINVAL, "mps_reset: null pointer");
  if (slot < 0 || slot >= m->n_slots) return fail(MPS_EINVAL, "mps_reset: slot out of range");
  for (int q = 0; q < m->n; ++q)
    if (occ[q] > 1) return fail(MPS_EINVAL, "mps_reset: occupation not 0/1");
  TRY(upload_reset(m, slot, 1, occ));
  CU(cudaStreamSynchronize(m->st));
  return MPS_OK;
}

int mps_set_svd_params(mps_t m, double cutoff, int max_sweeps) {
  if (!m) return fail(MPS_EINVAL, "mps_set_svd_params: null handle");
  if (!(cutoff >= 0.0 && cutoff < 1.0) || max_sweeps < 1 || max_sweeps > 1000)
    return fail(MPS_EINVAL, "mps_set_svd_params: cutoff in [0,1), max_sweeps in [1,1000]");
  m->cutoff = cutoff;
  m->max_sweeps = max_sweeps;
  return MPS_OK;
}

// Status of slots [slot0, slot0 + count) after a circuit launch. Slot slot0's figures
// fill the per-call statistics; the counts of Jacobi caps and skipped non-finite gates
// are summed over the slots. Returns MPS_ENONFINITE if any slot skipped a gate whose M'
// held a NaN or Inf, else MPS_ENOCONV if any Jacobi fallback reached its sweep cap.
int mps_set_kernel_timing(mps_t m, int on) {
  if (!m) return fail(MPS_EINVAL, "mps_set_kernel_timing: null handle");
  m->ktime = on != 0;
  return MPS_OK;
}

int mps_set_meas_budget(mps_t m, size_t bytes) {
  if (!m) return fail(MPS_EINVAL, "mps_set_meas_budget: null handle");
  // a new budget takes effect at the next measurement; buffers are rebuilt to match
  CU(cudaStreamSynchronize(m->st));
  for (void*& p : m->lvl_L) {
    dfree(p, m->st);
    p = nullptr;
  }
  for (void*& p : m->lvl_T) {
    dfree(p, m->st);
    p = nullptr;
  }
  std::fill(m->lvl_cap.begin(), m->lvl_cap.end(), 0);
  dfree(m->tc.scratch, m->st);
  m->tc.scratch = nullptr;
  m->tc.max_nodes = 0;
  m->meas_budget = bytes;
  return MPS_OK;
}

static int finish_apply(mps_s* m, double* discarded_weight, int slot0 = 0, int count = 1) {
  std::vector<double> dws((size_t)count);
  std::vector<int> st((size_t)count * kStatWords);
  CU(cudaMemcpy(dws.data(), m->dm.dw + slot0, (size_t)count * 8, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(st.data(), m->dm.stat + (size_t)kStatWords * slot0, st.size() * 4, cudaMemcpyDeviceToHost));
  unsigned long long pr[8];
  CU(cudaMemcpy(pr, m->dm.prof + (size_t)slot0 * 8, sizeof(pr), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 7; ++i) m->stats.cycles[i] = (double)pr[i];
  double fl;
  std::memcpy(&fl, &pr[7], 8);
  m->stats.alg_flops_total = fl;
  m->stats.discarded_weight = dws[0];
  m->stats.max_sweeps = st[0];
  m->stats.max_rank = st[2];
  m->stats.n_fallback = st[3];
  int64_t noconv = 0, nonfinite = 0;
  for (int s = 0; s < count; ++s) {
    noconv += st[(size_t)s * kStatWords + 1];
    nonfinite += st[(size_t)s * kStatWords + 4];
  }
  m->stats.n_svd_noconv += noconv;
  m->stats.n_nonfinite += nonfinite;
  if (discarded_weight) *discarded_weight = dws[0];
  if (nonfinite > 0) return fail(MPS_ENONFINITE, "a gate's M' held a NaN or Inf; the gate was skipped");
  if (noconv > 0) return fail(MPS_ENOCONV, "a Jacobi SVD fallback reached its sweep cap");
  return MPS_OK;
}

int mps_apply_circuit(mps_t m, circ_t c, const double* theta, double* discarded_weight) {
  if (!m || !c) return fail(MPS_EINVAL, "mps_apply_circuit: null handle");
  if (c->comp.n != m->n) return fail(MPS_EINVAL, "mps_apply_circuit: qubit count mismatch");
  if (!theta && c->comp.n_params > 0) return fail(MPS_EINVAL, "mps_apply_circuit: theta is null");
  reset_stats(m);
  // the discarded-weight accumulator and stats of slot 0 restart at this call
  CU(cudaMemsetAsync(m->dm.dw, 0, 8, m->st));
  CU(cudaMemsetAsync(m->dm.stat, 0, 4 * kStatWords, m->st));
  TRY(run_circuit(m, c, 0, 1, theta));
  return finish_apply(m, discarded_weight);
}

int mps_apply_gates(mps_t m, int64_t n_gates, const int32_t* bond, const double* U, double* discarded_weight) {
  if (!m || (n_gates > 0 && (!bond || !U))) return fail(MPS_EINVAL, "mps_apply_gates: null pointer");
  if (n_gates < 0) return fail(MPS_EINVAL, "mps_apply_gates: negative count");
  circ_s c;
  c.comp.n = m->n;
  c.comp.n_params = 0;
  for (int64_t g = 0; g < n_gates; ++g) {
    if (bond[g] < 0 || bond[g] > m->n - 2) return fail(MPS_EINVAL, "mps_apply_gates: bond out of range");
    GateRec r{};
    r.bond = bond[g];
    r.param = -1;
    r.m0 = (int32_t)g;
    r.m1 = -1;
    c.comp.gates.push_back(r);
    for (int e = 0; e < 16; ++e) c.comp.mats.push_back(cd(U[32 * g + 2 * e], U[32 * g + 2 * e + 1]));
  }
  reset_stats(m);
  CU(cudaMemsetAsync(m->dm.dw, 0, 8, m->st));
  CU(cudaMemsetAsync(m->dm.stat, 0, 4 * kStatWords, m->st));
  TRY(run_circuit(m, &c, 0, 1, nullptr));
  return finish_apply(m, discarded_weight);
}

int mps_expect_paulis(mps_t m, int64_t n_terms, const uint8_t* paulis, double* re, double* im) {
  if (!m || !paulis || !re || !im) return fail(MPS_EINVAL, "mps_expect_paulis: null pointer");
  if (n_terms < 1) return fail(MPS_EINVAL, "mps_expect_paulis: n_terms < 1");
  const int n = m->n;
  std::vector<int64_t> order((size_t)n_terms);
  for (int64_t t = 0; t < n_terms; ++t) {
    order[t] = t;
    for (int q = 0; q < n; ++q)
      if (paulis[t * n + q] > 3) return fail(MPS_EINVAL, "mps_expect_paulis: Pauli code out of {0,1,2,3}");
  }
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return std::lexicographical_compare(paulis + a * n, paulis + a * n + n, paulis + b * n, paulis + b * n + n);
  });
  std::vector<Term> terms;
  std::vector<int64_t> uniq_of((size_t)n_terms);
  for (int64_t i = 0; i < n_terms; ++i) {
    const uint8_t* c = paulis + order[i] * n;
    if (terms.empty() || !std::equal(c, c + n, terms.back().code.begin())) terms.push_back({std::vector<uint8_t>(c, c + n), 0.0});
    uniq_of[order[i]] = (int64_t)terms.size() - 1;
  }
  ham_t h = nullptr;
  TRY(make_ham(n, std::move(terms), &h));
  std::unique_ptr<ham_s> hold(h);
  reset_stats(m);
  std::vector<double> out(4 + 2 * h->terms.size());
  TRY(run_measure(m, h, 0, out.data()));
  for (int64_t t = 0; t < n_terms; ++t) {
    re[t] = out[4 + 2 * uniq_of[t]];
    im[t] = out[5 + 2 * uniq_of[t]];
  }
  return MPS_OK;
}

int mps_get_ranks(mps_t m, int slot, int32_t* ranks) {
  if (!m || !ranks) return fail(MPS_EINVAL, "mps_get_ranks: null pointer");
  if (slot < 0 || slot >= m->n_slots) return fail(MPS_EINVAL, "mps_get_ranks: slot out of range");
  std::vector<int> r(m->n + 1);
  CU(cudaStreamSynchronize(m->st));
  CU(cudaMemcpy(r.data(), m->dm.rank + (size_t)slot * (m->n + 1), (m->n + 1) * 4, cudaMemcpyDeviceToHost));
  for (int b = 0; b < m->n - 1; ++b) ranks[b] = r[b + 1];
  return MPS_OK;
}

int mps_state_size(mps_t m, int slot, int64_t* n_B, int64_t* n_lam) {
  std::vector<int32_t> r(m ? m->n : 1);
  TRY(mps_get_ranks(m, slot, r.data()));
  int64_t nb = 0, nl = 0;
  for (int k = 0; k < m->n; ++k) {
    int rl = k == 0 ? 1 : r[k - 1], rr = k == m->n - 1 ? 1 : r[k];
    nb += (int64_t)rl * 2 * rr;
  }
  for (int b = 0; b < m->n - 1; ++b) nl += r[b];
  if (n_B) *n_B = nb;
  if (n_lam) *n_lam = nl;
  return MPS_OK;
}

int mps_get_state(mps_t m, int slot, double* B, double* lam) {
  if (!m || !B || !lam) return fail(MPS_EINVAL, "mps_get_state: null pointer");
  std::vector<int32_t> r(m->n);
  TRY(mps_get_ranks(m, slot, r.data()));
  std::vector<char> buf((size_t)m->dm.slot_elems * m->es);
  CU(cudaMemcpy(buf.data(), (char*)m->dm.B + (size_t)slot * m->dm.slot_elems * m->es, buf.size(), cudaMemcpyDeviceToHost));
  std::vector<double> lbuf((size_t)(m->n - 1) * m->chi);
  CU(cudaMemcpy(lbuf.data(), m->dm.lam + (size_t)slot * (m->n - 1) * m->chi, lbuf.size() * 8, cudaMemcpyDeviceToHost));
  int64_t o = 0;
  for (int k = 0; k < m->n; ++k) {
    int rl = k == 0 ? 1 : r[k - 1], rr = k == m->n - 1 ? 1 : r[k];
    const int64_t cnt = (int64_t)rl * 2 * rr;
    for (int64_t e = 0; e < cnt; ++e) {
      if (m->prec == MPS_FP64) {
        const double* s = (const double*)buf.data() + 2 * (m->site_off[k] + e);
        B[2 * (o + e)] = s[0];
        B[2 * (o + e) + 1] = s[1];
      } else {
        const float* s = (const float*)buf.data() + 2 * (m->site_off[k] + e);
        B[2 * (o + e)] = s[0];
        B[2 * (o + e) + 1] = s[1];
      }
    }
    o += cnt;
  }
  int64_t l = 0;
  for (int b = 0; b < m->n - 1; ++b)
    for (int t = 0; t < r[b]; ++t) lam[l++] = lbuf[(size_t)b * m->chi + t];
  return MPS_OK;
}

int mps_set_state(mps_t m, int slot, const int32_t* ranks, const double* B, const double* lam) {
  if (!m || !ranks || !B || !lam) return fail(MPS_EINVAL, "mps_set_state: null pointer");
  if (slot < 0 || slot >= m->n_slots) return fail(MPS_EINVAL, "mps_set_state: slot out of range");
  const int n = m->n;
  for (int b = 0; b < n - 1; ++b)
    if (ranks[b] < 1 || ranks[b] > m->cap[b + 1]) return fail(MPS_EINVAL, "mps_set_state: rank out of range");
  std::vector<char> buf((size_t)m->dm.slot_elems * m->es, 0);
  int64_t o = 0;
  for (int k = 0; k < n; ++k) {
    int rl = k == 0 ? 1 : ranks[k - 1], rr = k == n - 1 ? 1 : ranks[k];
    const int64_t cnt = (int64_t)rl * 2 * rr;
    for (int64_t e = 0; e < cnt; ++e) {
      if (m->prec == MPS_FP64) {
        double* d = (double*)buf.data() + 2 * (m->site_off[k] + e);
        d[0] = B[2 * (o + e)];
        d[1] = B[2 * (o + e) + 1];
      } else {
        float* d = (float*)buf.data() + 2 * (m->site_off[k] + e);
        d[0] = (float)B[2 * (o + e)];
        d[1] = (float)B[2 * (o + e) + 1];
      }
    }
    o += cnt;
  }
  std::vector<double> lbuf((size_t)(n - 1) * m->chi, 0.0);
  int64_t l = 0;
  for (int b = 0; b < n - 1; ++b)
    for (int t = 0; t < ranks[b]; ++t) lbuf[(size_t)b * m->chi + t] = lam[l++];
  std::vector<int> r(n + 1, 1);
  for (int b = 0; b < n - 1; ++b) r[b + 1] = ranks[b];
  CU(cudaStreamSynchronize(m->st));
  CU(cudaMemcpy((char*)m->dm.B + (size_t)slot * m->dm.slot_elems * m->es, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(m->dm.lam + (size_t)slot * (n - 1) * m->chi, lbuf.data(), lbuf.size() * 8, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(m->dm.rank + (size_t)slot * (n + 1), r.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
  return MPS_OK;
}

int mps_energy(mps_t m, ham_t h, double* energy) {
  if (!m || !h || !energy) return fail(MPS_EINVAL, "mps_energy: null pointer");
  if (h->n != m->n) return fail(MPS_EINVAL, "mps_energy: qubit count mismatch");
  reset_stats(m);
  m->h_out.resize(4 + 2 * h->terms.size());
  TRY(run_measure(m, h, 0, m->h_out.data(), false));
  *energy = m->h_out[0];
  return MPS_OK;
}

int vqe_energy(mps_t m, circ_t c, ham_t h, const double* theta, double* energy) {
  return vqe_energy_batch(m, c, h, 1, theta, energy);
}

int vqe_energy_batch(mps_t m, circ_t c, ham_t h, int n_batch, const double* thetas, double* energies) {
  if (!m || !c || !h || !energies) return fail(MPS_EINVAL, "vqe_energy: null pointer");
  if (!thetas && c->comp.n_params > 0) return fail(MPS_EINVAL, "vqe_energy: theta is null");
  if (c->comp.n != m->n || h->n != m->n) return fail(MPS_EINVAL, "vqe_energy: qubit count mismatch");
  if (n_batch < 1 || n_batch > m->n_slots) return fail(MPS_EINVAL, "vqe_energy_batch: n_batch out of [1, n_slots]");
  reset_stats(m);
  std::vector<uint8_t> occ((size_t)n_batch * m->n);
  for (int b = 0; b < n_batch; ++b) std::memcpy(&occ[(size_t)b * m->n], c->comp.reference.data(), m->n);
  TRY(upload_reset(m, 0, n_batch, occ.data()));
  TRY(run_circuit(m, c, 0, n_batch, thetas));
  int rc = finish_apply(m, nullptr, 0, n_batch);
  if (rc != MPS_OK && rc != MPS_ENOCONV) return rc;
  m->h_out.resize(4 + 2 * h->terms.size());
  for (int b = 0; b < n_batch; ++b) {
    TRY(run_measure(m, h, b, m->h_out.data(), false));
    energies[b] = m->h_out[0];
  }
  return rc;
}

int vqe_gradient(mps_t m, circ_t c, ham_t h, const double* theta, int n_sel, const int32_t* sel, double* grad) {
  if (!m || !c || !h || !theta || !sel || !grad) return fail(MPS_EINVAL, "vqe_gradient: null pointer");
  if (c->comp.n != m->n || h->n != m->n) return fail(MPS_EINVAL, "vqe_gradient: qubit count mismatch");
  const int np = c->comp.n_params;
  for (int i = 0; i < n_sel; ++i)
    if (sel[i] < 0 || sel[i] >= np) return fail(MPS_EINVAL, "vqe_gradient: parameter index out of range");
  // Each rotation k of parameter e contributes scale_k [E(phi_k + pi/2) - E(phi_k - pi/2)] / 2.
  // The two shifted circuits of rotation k differ from the unshifted one first at k's
  // parametric gate p_k, so they start from a copy of the unshifted state at p_k.
  struct Target {
    int sel_i;
    int64_t gate;
    double scale;
  };
  const auto& R = c->comp.rotations;
  const auto& Gs = c->comp.gates;
  std::vector<Target> tg;
  for (size_t k = 0; k < R.size(); ++k) {
    if (R[k].param < 0) continue;
    int si = -1;
    for (int i = 0; i < n_sel; ++i)
      if (sel[i] == R[k].param) si = i;
    if (si < 0) continue;
    const int64_t pk = c->rot_param_gate[k];
    if (pk < 0 || pk >= (int64_t)Gs.size() || Gs[pk].param != R[k].param)
      return fail(MPS_EINVAL, "vqe_gradient: rotation without a parametric gate");
    tg.push_back({si, pk, R[k].scale});
  }
  for (int i = 0; i < n_sel; ++i) grad[i] = 0.0;
  reset_stats(m);
  const int64_t G = (int64_t)Gs.size();
  const std::vector<uint8_t>& ref = c->comp.reference;
  m->h_out.resize(4 + 2 * h->terms.size());
  int rc_all = MPS_OK;
  auto keep = [&](int rc) {
    if (rc == MPS_ENOCONV) rc_all = MPS_ENOCONV;
    return rc == MPS_OK || rc == MPS_ENOCONV;
  };
  // a skipped non-finite gate ends the gradient with its own status
  auto stop = [&](int rc) { return rc == MPS_ENONFINITE ? rc : MPS_ECUDA; };
  if (m->n_slots < 3) {
    // one slot: every shifted circuit from the reference state
    for (const Target& t : tg) {
      double e2[2];
      for (int sgn = 0; sgn < 2; ++sgn) {
        const int64_t zero = 0, sg = t.gate;
        const double ph = sgn == 0 ? kHalfPi : -kHalfPi;
        TRY(upload_reset(m, 0, 1, ref.data()));
        TRY(run_circuit(m, c, 0, 1, theta, &zero, &sg, &ph));
        {
          const int rc = finish_apply(m, nullptr);
          if (!keep(rc)) return stop(rc);
        }
        TRY(run_measure(m, h, 0, m->h_out.data(), false));
        e2[sgn] = m->h_out[0];
      }
      grad[t.sel_i] += t.scale * (e2[0] - e2[1]) / 2.0;
    }
    return rc_all;
  }
  // slot 0 carries the unshifted prefix; each wave forks two slots per target
  const int wave = (m->n_slots - 1) / 2;
  std::vector<double> th((size_t)m->n_slots * std::max(1, np));
  for (int s = 0; s < m->n_slots; ++s)
    if (np > 0) std::memcpy(&th[(size_t)s * np], theta, (size_t)np * 8);
  TRY(upload_reset(m, 0, 1, ref.data()));
  int64_t trunk = 0;
  for (size_t w0 = 0; w0 < tg.size(); w0 += wave) {
    const int nw = (int)std::min<size_t>(wave, tg.size() - w0);
    std::vector<int64_t> start(2 * nw), sgate(2 * nw);
    std::vector<double> sphi(2 * nw);
    for (int i = 0; i < nw; ++i) {
      const Target& t = tg[w0 + i];
      if (t.gate > trunk) {
        const int64_t st0 = trunk;
        TRY(run_circuit(m, c, 0, 1, th.data(), &st0, nullptr, nullptr, t.gate));
        {
          const int rc = finish_apply(m, nullptr);
          if (!keep(rc)) return stop(rc);
        }
        trunk = t.gate;
      }
      for (int sgn = 0; sgn < 2; ++sgn) {
        TRY(copy_slot(m, 0, 1 + 2 * i + sgn));
        start[2 * i + sgn] = t.gate;
        sgate[2 * i + sgn] = t.gate;
        sphi[2 * i + sgn] = sgn == 0 ? kHalfPi : -kHalfPi;
      }
    }
    TRY(run_circuit(m, c, 1, 2 * nw, th.data() + np, start.data(), sgate.data(), sphi.data(), G));
    {
      const int rc = finish_apply(m, nullptr, 1, 2 * nw);
      if (!keep(rc)) return stop(rc);
    }
    for (int i = 0; i < nw; ++i) {
      double e2[2];
      for (int sgn = 0; sgn < 2; ++sgn) {
        TRY(run_measure(m, h, 1 + 2 * i + sgn, m->h_out.data(), false));
        e2[sgn] = m->h_out[0];
      }
      const Target& t = tg[w0 + i];
      grad[t.sel_i] += t.scale * (e2[0] - e2[1]) / 2.0;
    }
  }
  return rc_all;
}

int mps_get_stats(mps_t m, mps_stats_t* s) {
  if (!m || !s) return fail(MPS_EINVAL, "mps_get_stats: null pointer");
  *s = m->stats;
  return MPS_OK;
}

}  // extern "C"
