// Host-side preprocessing of the MPS-VQE library (runs once per Hamiltonian/ansatz).
//
//  * Jordan-Wigner map of the electronic Hamiltonian, Eq. (1) -> Eq. (2) (Sec. II-A).
//  * Trotterised UCCSD generators, Eqs. (3)-(4) (Sec. II-A).
//  * Compilation of each Pauli rotation into nearest-neighbour two-site gates with
//    single-qubit gates fused in (Sec. III-A, Sec. III-D).
//  * The prefix trie of Pauli strings that lets all strings share left environments
//    (the energy of Eq. 2 as a sum of independent expectations, Sec. III-C).
//
// Pauli operators are handled in "XZ form" X^x Z^z with bit masks; a product is
// (X^x1 Z^z1)(X^x2 Z^z2) = (-1)^{|z1 & x2|} X^{x1^x2} Z^{z1^z2}, and letters follow from
// Y = i X Z, i.e. X^x Z^z = (-i)^{|x & z|} (x) letters.
#include "host.hpp"

#include <algorithm>
#include <array>
#include <atomic>
#include <functional>
#include <thread>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>

namespace mpsvqe {

static inline int popc(uint64_t v) { return __builtin_popcountll(v); }
static inline int popc2(const uint64_t* a, const uint64_t* b) {
  return popc(a[0] & b[0]) + popc(a[1] & b[1]);
}
static inline void setbit(uint64_t* m, int q) { m[q >> 6] |= 1ull << (q & 63); }
static inline int getbit(const uint64_t* m, int q) { return (int)((m[q >> 6] >> (q & 63)) & 1ull); }

void xz_to_letters(const XZ& k, int n, uint8_t* out) {
  for (int q = 0; q < n; ++q) {
    int x = getbit(k.x, q), z = getbit(k.z, q);
    out[q] = (uint8_t)(x ? (z ? 2 : 1) : (z ? 3 : 0));
  }
}

XZ letters_to_xz(const uint8_t* code, int n) {
  XZ k;
  for (int q = 0; q < n; ++q) {
    if (code[q] == 1 || code[q] == 2) setbit(k.x, q);
    if (code[q] == 2 || code[q] == 3) setbit(k.z, q);
  }
  return k;
}

// i^e for e mod 4
static inline cd ipow(int e) {
  switch (((e % 4) + 4) % 4) {
    case 0: return cd(1, 0);
    case 1: return cd(0, 1);
    case 2: return cd(-1, 0);
    default: return cd(0, -1);
  }
}

// Jordan-Wigner ladder operator as two XZ-form terms:
//   a_p  = 1/2 Z_{<p} X_p + i/2 Z_{<p} Y_p = 1/2 X^{p} Z^{<p} - 1/2 X^{p} Z^{<=p}
//   a+_p = 1/2 X^{p} Z^{<p} + 1/2 X^{p} Z^{<=p}
struct XZTerm {
  XZ k;
  cd c;
};
static void ladder(int p, bool dagger, XZTerm out[2]) {
  XZ a, b;
  setbit(a.x, p);
  setbit(b.x, p);
  for (int q = 0; q < p; ++q) {
    setbit(a.z, q);
    setbit(b.z, q);
  }
  setbit(b.z, p);
  out[0] = {a, cd(0.5, 0)};
  out[1] = {b, cd(dagger ? 0.5 : -0.5, 0)};
}

static inline XZTerm mul(const XZTerm& l, const XZTerm& r) {
  XZTerm o;
  int sgn = popc2(l.k.z, r.k.x) & 1;
  for (int w = 0; w < 2; ++w) {
    o.k.x[w] = l.k.x[w] ^ r.k.x[w];
    o.k.z[w] = l.k.z[w] ^ r.k.z[w];
  }
  o.c = l.c * r.c * (sgn ? -1.0 : 1.0);
  return o;
}

using XZMap = std::unordered_map<XZ, cd, XZHash>;

// Accumulate weight * op_1 op_2 ... op_m (leftmost first) into acc.
static void add_ladder_product(const int* p, const bool* dag, int m, cd weight, XZMap& acc) {
  XZTerm br[4][2];
  for (int j = 0; j < m; ++j) ladder(p[j], dag[j], br[j]);
  for (int combo = 0; combo < (1 << m); ++combo) {
    XZTerm t{XZ(), weight};
    for (int j = 0; j < m; ++j) t = mul(t, br[j][(combo >> j) & 1]);
    acc[t.k] += t.c;
  }
}

// The same, each term into the map of its hash class (maps[hash % count]).
static void add_ladder_product_sharded(const int* p, const bool* dag, int m, cd weight, XZMap* maps, int count) {
  XZTerm br[4][2];
  for (int j = 0; j < m; ++j) ladder(p[j], dag[j], br[j]);
  XZHash hs;
  for (int combo = 0; combo < (1 << m); ++combo) {
    XZTerm t{XZ(), weight};
    for (int j = 0; j < m; ++j) t = mul(t, br[j][(combo >> j) & 1]);
    maps[hs(t.k) % (size_t)count][t.k] += t.c;
  }
}

// Letter-form coefficient of an accumulated XZ term.
static inline cd letter_coeff(const XZ& k, cd c) { return c * ipow(-popc2(k.x, k.z)); }

// f(0) .. f(count - 1) on up to count threads (the calls must not depend on each other).
static void parallel_for(int count, const std::function<void(int)>& f) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::min(count, hw);
  if (nt <= 1) {
    for (int i = 0; i < count; ++i) f(i);
    return;
  }
  std::atomic<int> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&] {
      for (int i = next++; i < count; i = next++) f(i);
    });
  for (auto& th : pool) th.join();
}

static bool trie_less(const std::vector<uint8_t>& a, const std::vector<uint8_t>& b) {
  return std::lexicographical_compare(a.begin(), a.end(), b.begin(), b.end());
}

std::vector<Term> canonical_terms(int n, std::vector<Term> terms, double rel_drop) {
  // trie order (lexicographic in the letters); equal strings merged in input order
  std::stable_sort(terms.begin(), terms.end(), [](const Term& a, const Term& b) { return trie_less(a.code, b.code); });
  std::vector<Term> merged;
  merged.reserve(terms.size());
  for (auto& t : terms) {
    if (!merged.empty() && merged.back().code == t.code)
      merged.back().coeff += t.coeff;
    else
      merged.push_back(std::move(t));
  }
  double mx = 0;
  for (auto& t : merged) mx = std::max(mx, std::fabs(t.coeff));
  std::vector<Term> out;
  out.reserve(merged.size());
  for (auto& t : merged)
    if (std::fabs(t.coeff) > rel_drop * mx) out.push_back(std::move(t));
  (void)n;
  return out;
}

std::vector<Term> jordan_wigner(int m, const double* h, const double* eri, double e_core,
                                std::string* err) {
  const int n = 2 * m;
  // Work is split into a fixed number of parts, whatever the machine's thread count, and
  // merged in a fixed order, so the coefficients are the same bits on every machine.
  constexpr int kParts = 16;
  // one-body: h_pq a+_p a_q, equal spins
  XZMap one;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      if ((p & 1) != (q & 1)) continue;
      double w = h[(p / 2) * m + (q / 2)];
      if (w == 0.0) continue;
      int idx[2] = {p, q};
      bool dg[2] = {true, false};
      add_ladder_product(idx, dg, 2, cd(w, 0), one);
    }
  one[XZ()] += cd(e_core, 0);
  // two-body: 1/2 (pq|rs) a+_p a+_r a_s a_q, spin(p) = spin(q), spin(r) = spin(s). The
  // operator for (r, s, p, q) is the same as for (p, q, r, s) (two swaps), so each
  // unordered pair of (p, q) and (r, s) is expanded once with both weights; r = p
  // (a+_p a+_p = 0) and s = q are skipped, so the two pairs never coincide.
  auto eri_at = [&](int p, int q, int r, int s) {
    return eri[(((size_t)(p / 2) * m + q / 2) * m + r / 2) * m + s / 2];
  };
  // part t accumulates the (p, q) pairs t, t + kParts, ... into kParts maps by key hash;
  // shard s then merges map s of every part, in part order
  std::vector<std::vector<XZMap>> part(kParts, std::vector<XZMap>(kParts));
  auto run_part = [&](int t) {
    XZMap* acc = part[t].data();
    for (int pq = t; pq < n * n; pq += kParts) {
      const int p = pq / n, q = pq % n;
      if ((p & 1) != (q & 1)) continue;
      for (int r = 0; r < n; ++r) {
        if (r == p) continue;
        for (int s = 0; s < n; ++s) {
          if ((r & 1) != (s & 1) || s == q || r * n + s < pq) continue;
          const double w = 0.5 * (eri_at(p, q, r, s) + eri_at(r, s, p, q));
          if (w == 0.0) continue;
          int idx[4] = {p, r, s, q};
          bool dg[4] = {true, true, false, false};
          add_ladder_product_sharded(idx, dg, 4, cd(w, 0), acc, kParts);
        }
      }
    }
  };
  std::vector<XZMap> shard(kParts);
  std::vector<double> shard_max(kParts, 0.0);
  auto run_shard = [&](int t) {
    XZMap& out = shard[t];
    XZHash hs;
    for (auto& kv : one)
      if (hs(kv.first) % kParts == (size_t)t) out[kv.first] += kv.second;
    for (int c = 0; c < kParts; ++c) {
      for (auto& kv : part[c][t]) out[kv.first] += kv.second;
      XZMap().swap(part[c][t]);
    }
    for (auto& kv : out) shard_max[t] = std::max(shard_max[t], std::abs(kv.second));
  };
  parallel_for(kParts, run_part);
  parallel_for(kParts, run_shard);
  const double mx = *std::max_element(shard_max.begin(), shard_max.end());
  // letters and the relative drop, per shard; concatenated in shard order
  std::vector<std::vector<Term>> found(kParts);
  std::vector<int> bad(kParts, 0);
  auto run_collect = [&](int t) {
    for (auto& kv : shard[t]) {
      cd c = letter_coeff(kv.first, kv.second);
      if (std::abs(c) <= 1e-12 * mx) continue;
      if (std::fabs(c.imag()) > 1e-10 * std::max(1.0, mx)) {
        bad[t] = 1;
        return;
      }
      Term term;
      term.code.resize(n);
      xz_to_letters(kv.first, n, term.code.data());
      term.coeff = c.real();
      found[t].push_back(std::move(term));
    }
    XZMap().swap(shard[t]);
  };
  parallel_for(kParts, run_collect);
  if (*std::max_element(bad.begin(), bad.end())) {
    if (err) *err = "Jordan-Wigner coefficient with an imaginary part: integrals not Hermitian";
    return {};
  }
  std::vector<Term> terms;
  size_t total = 0;
  for (auto& f : found) total += f.size();
  terms.reserve(total);
  for (auto& f : found)
    for (auto& t : f) terms.push_back(std::move(t));
  return canonical_terms(n, std::move(terms), 1e-12);
}

// ------------------------------------------------------------------ UCCSD rotations

static bool mask_less(const XZ& a, const XZ& b) {
  if (a.x[1] != b.x[1]) return a.x[1] < b.x[1];
  if (a.x[0] != b.x[0]) return a.x[0] < b.x[0];
  if (a.z[1] != b.z[1]) return a.z[1] < b.z[1];
  return a.z[0] < b.z[0];
}

std::vector<Rotation> uccsd_rotations(int n, int ne, int* n_params) {
  struct Exc {
    int k;
    int o[4];
  };
  std::vector<Exc> exc;
  for (int i = 0; i < ne; ++i)
    for (int a = ne; a < n; ++a)
      if ((i & 1) == (a & 1)) exc.push_back({1, {i, a, 0, 0}});
  for (int i = 0; i < ne; ++i)
    for (int j = i + 1; j < ne; ++j)
      for (int a = ne; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
          if ((i & 1) + (j & 1) == (a & 1) + (b & 1)) exc.push_back({2, {i, j, a, b}});
  std::vector<Rotation> rots;
  for (size_t e = 0; e < exc.size(); ++e) {
    XZMap acc;
    const Exc& x = exc[e];
    if (x.k == 1) {
      int i = x.o[0], a = x.o[1];
      int p1[2] = {a, i}, p2[2] = {i, a};
      bool d[2] = {true, false};
      add_ladder_product(p1, d, 2, cd(1, 0), acc);    // tau
      add_ladder_product(p2, d, 2, cd(-1, 0), acc);   // -tau+
    } else {
      int i = x.o[0], j = x.o[1], a = x.o[2], b = x.o[3];
      int p1[4] = {a, b, i, j}, p2[4] = {j, i, b, a};
      bool d[4] = {true, true, false, false};
      add_ladder_product(p1, d, 4, cd(1, 0), acc);
      add_ladder_product(p2, d, 4, cd(-1, 0), acc);
    }
    std::vector<std::pair<XZ, double>> strs;
    double mx = 0;
    for (auto& kv : acc) mx = std::max(mx, std::abs(kv.second));
    for (auto& kv : acc) {
      cd c = letter_coeff(kv.first, kv.second);  // tau - tau+ = i sum c_k P_k
      if (std::abs(c) <= 1e-12 * mx) continue;
      strs.push_back({kv.first, c.imag()});
    }
    std::sort(strs.begin(), strs.end(),
              [](const std::pair<XZ, double>& l, const std::pair<XZ, double>& r) {
                return mask_less(l.first, r.first);
              });
    for (auto& s : strs) {
      Rotation r;
      r.code.resize(n);
      xz_to_letters(s.first, n, r.code.data());
      r.param = (int32_t)e;
      r.scale = -2.0 * s.second;
      rots.push_back(std::move(r));
    }
  }
  if (n_params) *n_params = (int)exc.size();
  return rots;
}

// ------------------------------------------------------------------ gate compiler

using M2 = std::array<cd, 4>;
using M4 = std::array<cd, 16>;

static M2 eye2() { return {cd(1), cd(0), cd(0), cd(1)}; }
static M2 adj2(const M2& a) { return {std::conj(a[0]), std::conj(a[2]), std::conj(a[1]), std::conj(a[3])}; }
static M4 kron(const M2& a, const M2& b) {
  M4 o;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) o[(2 * i + j) * 4 + (2 * k + l)] = a[2 * i + k] * b[2 * j + l];
  return o;
}
static M4 mm(const M4& a, const M4& b) {
  M4 o;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd s = 0;
      for (int k = 0; k < 4; ++k) s += a[4 * i + k] * b[4 * k + j];
      o[4 * i + j] = s;
    }
  return o;
}
static M4 cnot() {
  M4 o{};
  o[0] = o[5] = o[11] = o[14] = cd(1);
  return o;
}
static M4 swp() {
  M4 o{};
  o[0] = o[6] = o[9] = o[15] = cd(1);
  return o;
}
static M2 rz2(double phi) { return {std::polar(1.0, -0.5 * phi), cd(0), cd(0), std::polar(1.0, 0.5 * phi)}; }
// Basis change B with B P B+ = Z: H for X, Rx(pi/2) = (I - iX)/sqrt2 for Y, I for Z.
static M2 basis(uint8_t c) {
  const double r = 1.0 / std::sqrt(2.0);
  if (c == 1) return {cd(r), cd(r), cd(r), cd(-r)};
  if (c == 2) return {cd(r), cd(0, -r), cd(0, -r), cd(r)};
  return eye2();
}

namespace {
struct MatTable {
  std::map<std::array<uint64_t, 32>, int32_t> index;
  std::vector<cd>* mats;
  int32_t add(const M4& m) {
    std::array<uint64_t, 32> key;
    for (int i = 0; i < 16; ++i) {
      double re = m[i].real() + 0.0, im = m[i].imag() + 0.0;  // +0.0 folds -0
      std::memcpy(&key[2 * i], &re, 8);
      std::memcpy(&key[2 * i + 1], &im, 8);
    }
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    int32_t id = (int32_t)(mats->size() / 16);
    mats->insert(mats->end(), m.begin(), m.end());
    index.emplace(key, id);
    return id;
  }
};
}  // namespace

void compile_rotations(int n, const std::vector<Rotation>& rots, Compiled* out) {
  out->n = n;
  out->rotations = rots;
  out->gates.clear();
  out->mats.clear();
  out->rot_first_gate.clear();
  MatTable tab;
  tab.mats = &out->mats;
  int np = 0;
  for (auto& r : rots) np = std::max(np, r.param + 1);
  out->n_params = std::max(out->n_params, np);
  const M2 I = eye2();
  for (const Rotation& r : rots) {
    out->rot_first_gate.push_back((int64_t)out->gates.size());
    std::vector<int> S;
    for (int q = 0; q < n; ++q)
      if (r.code[q]) S.push_back(q);
    if (S.empty()) continue;  // global phase
    auto emit = [&](int bond, const M4& pre, const M4& post, int rz_site, bool parametric) {
      GateRec g{};
      g.bond = bond;
      if (parametric && r.param >= 0) {
        g.param = r.param;
        g.scale = r.scale;
        g.m0 = tab.add(pre);
        g.m1 = tab.add(post);
        g.rz_site = rz_site;
      } else if (parametric) {  // fixed angle: fold Rz in now
        M2 z = rz2(r.scale);
        M4 R = rz_site == 0 ? kron(z, I) : kron(I, z);
        g.param = -1;
        g.m0 = tab.add(mm(post, mm(R, pre)));
        g.m1 = -1;
      } else {
        g.param = -1;
        g.m0 = tab.add(pre);
        g.m1 = -1;
      }
      out->gates.push_back(g);
    };
    if (S.size() == 1) {
      int q = S[0];
      M2 B = basis(r.code[q]);
      if (q + 1 < n)
        emit(q, kron(B, I), kron(adj2(B), I), 0, true);
      else
        emit(q - 1, kron(I, B), kron(I, adj2(B)), 1, true);
      continue;
    }
    const int lo = S.front(), hi = S.back();
    std::vector<char> inS(n, 0);
    for (int q : S) inS[q] = 1;
    auto Bq = [&](int q) { return inS[q] ? basis(r.code[q]) : I; };
    auto hop = [&](int b) { return inS[b + 1] ? cnot() : swp(); };
    for (int b = lo; b < hi - 1; ++b)  // up ladder below the top bond
      emit(b, mm(hop(b), kron(b == lo ? Bq(lo) : I, Bq(b + 1))), M4{}, 0, false);
    {  // top bond: up hop, Rz(phi) on hi, down hop
      int b = hi - 1;
      M4 pre = mm(cnot(), kron(b == lo ? Bq(lo) : I, Bq(hi)));
      M4 post = mm(kron(b == lo ? adj2(Bq(lo)) : I, adj2(Bq(hi))), cnot());
      emit(b, pre, post, 1, true);
    }
    for (int b = hi - 2; b >= lo; --b)  // down ladder
      emit(b, mm(kron(b == lo ? adj2(Bq(lo)) : I, adj2(Bq(b + 1))), hop(b)), M4{}, 0, false);
  }
}

void fuse_gates(Compiled* c, std::vector<int64_t>* param_gate) {
  const std::vector<GateRec>& G = c->gates;
  const std::vector<cd>& Mv = c->mats;
  auto get = [&](int32_t id) {
    M4 m;
    std::copy(Mv.begin() + 16 * (size_t)id, Mv.begin() + 16 * (size_t)id + 16, m.begin());
    return m;
  };
  auto is_identity = [](const M4& m) {
    for (int i = 0; i < 16; ++i)
      if (std::abs(m[i] - cd((i % 5) == 0 ? 1.0 : 0.0)) > 1e-13) return false;
    return true;
  };
  struct Item {
    bool parametric;
    M4 pre, post;  // fixed gate: pre only
    GateRec rec;
    int64_t rot;
  };
  const size_t nrot = c->rotations.size();
  std::vector<int64_t> owner(G.size(), 0);
  for (size_t r = 0; r < nrot; ++r) {
    const int64_t e = r + 1 < nrot ? c->rot_first_gate[r + 1] : (int64_t)G.size();
    for (int64_t g = c->rot_first_gate[r]; g < e; ++g) owner[g] = (int64_t)r;
  }
  std::vector<Item> out;
  for (size_t g = 0; g < G.size(); ++g) {
    Item it;
    it.parametric = G[g].param >= 0;
    it.pre = get(G[g].m0);
    if (it.parametric) it.post = get(G[g].m1);
    it.rec = G[g];
    it.rot = owner[g];
    if (!out.empty() && out.back().rec.bond == it.rec.bond) {
      Item& h = out.back();
      if (!h.parametric && !it.parametric) {  // fixed after fixed: one product
        const M4 p = mm(it.pre, h.pre);
        if (is_identity(p))
          out.pop_back();
        else
          h.pre = p;
        continue;
      }
      if (!h.parametric && it.parametric) {  // U (m1 Rz m0) after F: m0 <- m0 F
        it.pre = mm(it.pre, h.pre);
        out.back() = it;
        continue;
      }
      if (h.parametric && !it.parametric) {  // F after U: m1 <- F m1
        h.post = mm(it.pre, h.post);
        continue;
      }
    }
    out.push_back(it);
  }
  std::vector<cd> mats;
  MatTable tab;
  tab.mats = &mats;
  std::vector<GateRec> gates;
  gates.reserve(out.size());
  param_gate->assign(nrot, -1);
  std::vector<int64_t> first(nrot, (int64_t)out.size());
  for (size_t i = 0; i < out.size(); ++i) {
    GateRec rec = out[i].rec;
    rec.m0 = tab.add(out[i].pre);
    if (out[i].parametric) {
      rec.m1 = tab.add(out[i].post);
      (*param_gate)[out[i].rot] = (int64_t)i;
    } else {
      rec.param = -1;
      rec.m1 = -1;
    }
    first[out[i].rot] = std::min(first[out[i].rot], (int64_t)i);
    gates.push_back(rec);
  }
  // owners are non-decreasing along the list; a rotation without gates of its own
  // starts where the next one does
  for (size_t r = nrot; r-- > 0;)
    if (r + 1 < nrot) first[r] = std::min(first[r], first[r + 1]);
  c->gates = std::move(gates);
  c->mats = std::move(mats);
  c->rot_first_gate = std::move(first);
}

static bool pauli_commute(const std::vector<uint8_t>& a, const std::vector<uint8_t>& b) {
  int anti = 0;
  for (size_t q = 0; q < a.size(); ++q) anti += (a[q] && b[q] && a[q] != b[q]);
  return (anti & 1) == 0;
}

int64_t order_for_ladder_cancellation(std::vector<Rotation>* rots) {
  std::vector<Rotation>& R = *rots;
  int64_t changed = 0;
  size_t i = 0;
  while (i < R.size()) {
    size_t j = i + 1;
    while (j < R.size() && R[i].param >= 0 && R[j].param == R[i].param) ++j;
    bool commuting = true;
    for (size_t a = i; a < j && commuting; ++a)
      for (size_t b = a + 1; b < j && commuting; ++b) commuting = pauli_commute(R[a].code, R[b].code);
    if (j - i > 1 && commuting) {
      // the letters from the lowest non-identity site up; runs of one excitation share
      // their support, so this is a lexicographic order of the letters on it
      auto key = [](const Rotation& r) {
        size_t lo = 0;
        while (lo < r.code.size() && !r.code[lo]) ++lo;
        return std::vector<uint8_t>(r.code.begin() + (std::ptrdiff_t)lo, r.code.end());
      };
      std::vector<Rotation> run(R.begin() + (std::ptrdiff_t)i, R.begin() + (std::ptrdiff_t)j);
      std::stable_sort(run.begin(), run.end(), [&](const Rotation& x, const Rotation& y) { return key(x) < key(y); });
      bool same = true;
      for (size_t t = 0; t < run.size(); ++t) same = same && run[t].code == R[i + t].code;
      if (!same) {
        std::copy(run.begin(), run.end(), R.begin() + (std::ptrdiff_t)i);
        ++changed;
      }
    }
    i = j;
  }
  return changed;
}

std::vector<int64_t> param_gates(const Compiled& c) {
  // the single gate (one non-identity site) or the top gate of the ladder
  const auto& R = c.rotations;
  std::vector<int64_t> pg(R.size(), -1);
  for (size_t r = 0; r < R.size(); ++r) {
    int lo = -1, hi = -1, w = 0;
    for (int q = 0; q < c.n; ++q)
      if (R[r].code[q]) {
        if (lo < 0) lo = q;
        hi = q;
        ++w;
      }
    if (w == 0) continue;
    pg[r] = c.rot_first_gate[r] + (w == 1 ? 0 : (hi - lo - 1));
  }
  return pg;
}

void gate_matrix(const Compiled& c, const GateRec& g, const double* theta, cd* U) {
  M4 a;
  std::copy(c.mats.begin() + 16 * (size_t)g.m0, c.mats.begin() + 16 * (size_t)g.m0 + 16, a.begin());
  if (g.param >= 0) {
    M4 b;
    std::copy(c.mats.begin() + 16 * (size_t)g.m1, c.mats.begin() + 16 * (size_t)g.m1 + 16, b.begin());
    M2 z = rz2(g.scale * theta[g.param]);
    M4 R = g.rz_site == 0 ? kron(z, eye2()) : kron(eye2(), z);
    a = mm(b, mm(R, a));
  }
  std::copy(a.begin(), a.end(), U);
}

// ------------------------------------------------------------------ prefix trie

void build_trie(int n, const std::vector<Term>& terms, Trie* t) {
  t->n = n;
  t->level_nodes.assign(n, 0);
  t->parent.assign(n, {});
  t->edge.assign(n, {});
  t->close_node.assign(n, {});
  t->close_letter.assign(n, {});
  t->close_term.assign(n, {});
  std::vector<int32_t> cur(n + 1, -1);  // current node id per level for the current prefix
  const uint8_t* prev = nullptr;
  int max_level = -1;
  for (size_t s = 0; s < terms.size(); ++s) {
    const uint8_t* c = terms[s].code.data();
    int l = -1;
    for (int q = n - 1; q >= 0; --q)
      if (c[q]) {
        l = q;
        break;
      }
    if (l < 0) continue;  // identity string: <I> = 1, no trie path
    int lcp = 0;
    if (prev)
      while (lcp < n && prev[lcp] == c[lcp]) ++lcp;
    for (int k = lcp + 1; k <= n; ++k) cur[k] = -1;  // prefixes longer than lcp changed
    if (!prev) cur.assign(n + 1, -1);
    for (int k = 0; k <= l; ++k) {
      if (cur[k] < 0) {
        cur[k] = t->level_nodes[k]++;
        if (k > 0) {
          t->parent[k].push_back(cur[k - 1]);
          t->edge[k].push_back(c[k - 1]);
        }
      }
    }
    t->close_node[l].push_back(cur[l]);
    t->close_letter[l].push_back(c[l]);
    t->close_term[l].push_back((int32_t)s);
    max_level = std::max(max_level, l);
    prev = c;
  }
  t->n_levels = max_level + 1;
  t->total_nodes = 0;
  t->max_level_nodes = 0;
  t->max_level_closes = 0;
  for (int k = 0; k < n; ++k) {
    t->total_nodes += t->level_nodes[k];
    t->max_level_nodes = std::max(t->max_level_nodes, t->level_nodes[k]);
    t->max_level_closes = std::max(t->max_level_closes, (int32_t)t->close_term[k].size());
  }
}

}  // namespace mpsvqe
