// CPU oracle for breadth-first exploration of the configurations of a spiking
// neural P system without delays (Cabarle, Adorna, Martinez-del-Amor,
// "Simulating Spiking Neural P systems without delays using GPUs").
//
// TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
// leg of the benchmark load this library; the simulator never does.  It shares
// no code with the CUDA path.  It is deliberately plain and slow: every step is
// written as the paper states it, with no blocking, fusion or reordering.
//
// Readings of the paper that this file implements (where the paper is silent
// or ambiguous):
//  * A rule r of neuron s has E = a^i (a^j)* (j = 0: E = a^i exactly) and
//    consumes c = -M[r][s] spikes.  It is applicable to x spikes iff a^x is in
//    L(E) and x >= c (Section 2.1, rules (b-1)/(b-3)).  The paper's own rules
//    "a^k -> a" are E = a^k (a)*, i.e. "at least k spikes"; that is the only
//    reading that reproduces the printed run.
//  * General regular expressions (the paper's future work, Section 6) are
//    read as finite unions of such terms: a^x is in L(E) iff it is in the
//    language of at least one term.
//  * A neuron with no applicable rule does not fire: it contributes one
//    choice, the all-zero block, to the spiking vectors (Eq. psi with
//    max(1, |sigma_V|)).
//  * Spiking vectors are listed as the Cartesian product of the per-neuron
//    choice lists with neuron 1's choice outermost (Algorithm 2, II-3), each
//    neuron's choices in rule order (II-2).
//  * Parents are expanded first-in first-out in discovery order; a child is
//    new iff it was never produced before (Algorithm 1, step IV, second
//    stopping criterion).
//  * Truncation, absent from the paper: at most `budget` candidates are
//    examined per depth and at most `cap` new configurations are accepted per
//    depth; the depth stops at whichever comes first.  A configuration that is
//    not accepted is not remembered.
//  * max_expand >= 0: a configuration holding more than max_expand spikes in
//    some neuron is recorded but never expanded (the printed run's digit-string
//    representation stops at "109").
//
// Parity pins (tests/test_oracle_pins.py): the worked example of Algorithm 2,
// the printed children and the 48-entry allGenCk list, brute force over all
// 0/1 vectors on small systems, regex membership against Python's re, and the
// invariants of Eq. next-config.

#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <unordered_set>
#include <vector>

namespace {

struct System {
  int32_t m = 0, R = 0;
  std::vector<int32_t> rule_neuron;
  std::vector<int32_t> rule_terms;      // [R + 1]: rule r's terms are [rule_terms[r], rule_terms[r + 1])
  std::vector<int32_t> term_i, term_j;  // term t is a^term_i[t] (a^term_j[t])*
  std::vector<int32_t> M;  // R x m, row-major: rows are rules, columns neurons
};

struct VecHash {
  size_t operator()(const std::vector<int32_t>& v) const {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the bytes
    const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
    for (size_t k = 0; k < v.size() * sizeof(int32_t); ++k) {
      h ^= p[k];
      h *= 1099511628211ull;
    }
    return static_cast<size_t>(h);
  }
};

struct DepthStats {
  int64_t new_configs = 0;
  int64_t examined = 0;
  uint64_t candidates = 0;  // sum of Psi over the parents, saturating
  int32_t truncated = 0;
};

struct Result {
  int32_t m = 0;
  std::vector<int32_t> configs;  // discovery order, m per row
  std::vector<DepthStats> depths;
  int32_t depth_reached = 0;
  int32_t error = 0;
};

const uint64_t kSat = ~0ull;

uint64_t sat_mul(uint64_t a, uint64_t b) {
  if (a == 0 || b == 0) return 0;
  if (a > kSat / b) return kSat;
  return a * b;
}

uint64_t sat_add(uint64_t a, uint64_t b) { return (a > kSat - b) ? kSat : a + b; }

// Spikes consumed by rule r: the entry of M on the rule's own neuron (Definition 2).
int32_t consumed(const System& s, int r) { return -s.M[(size_t)r * s.m + s.rule_neuron[r]]; }

// Is a^x in L(a^i (a^j)*)?
bool in_language(int64_t x, int32_t i, int32_t j) {
  if (x < i) return false;
  if (j == 0) return x == i;
  return (x - i) % j == 0;
}

// Is a^x in L(E) for rule r's expression E, the union of its terms?
bool in_rule_language(const System& s, int64_t x, int r) {
  for (int t = s.rule_terms[r]; t < s.rule_terms[r + 1]; ++t)
    if (in_language(x, s.term_i[t], s.term_j[t])) return true;
  return false;
}

// Algorithm 2, II-1: rule r is applicable to configuration C.
bool applicable(const System& s, const int32_t* C, int r) {
  int64_t x = C[s.rule_neuron[r]];
  return in_rule_language(s, x, r) && x >= consumed(s, r);
}

// Algorithm 2, II-2: per neuron, the applicable rules in rule order; an empty
// list means the neuron does not fire.
std::vector<std::vector<int>> choice_lists(const System& s, const int32_t* C) {
  std::vector<std::vector<int>> lists(s.m);
  for (int r = 0; r < s.R; ++r)
    if (applicable(s, C, r)) lists[s.rule_neuron[r]].push_back(r);
  return lists;
}

// Eq. psi: the number of valid spiking vectors, prod over neurons of max(1, omega).
uint64_t psi(const std::vector<std::vector<int>>& lists) {
  uint64_t p = 1;
  for (const auto& l : lists) p = sat_mul(p, l.empty() ? 1 : l.size());
  return p;
}

// Algorithm 2, II-3 as an odometer over the per-neuron choice lists: neuron 1's
// choice is the outermost loop, the last neuron's the innermost.  Returns false
// after the last vector.
bool next_digits(const std::vector<std::vector<int>>& lists, std::vector<int>& digit) {
  for (int n = (int)lists.size() - 1; n >= 0; --n) {
    int radix = lists[n].empty() ? 1 : (int)lists[n].size();
    if (++digit[n] < radix) return true;
    digit[n] = 0;
  }
  return false;
}

// The spiking vector S (length R, entries 0/1) named by one digit per neuron.
void spiking_vector(const System& s, const std::vector<std::vector<int>>& lists,
                    const std::vector<int>& digit, std::vector<uint8_t>& S) {
  std::fill(S.begin(), S.end(), 0);
  for (int n = 0; n < s.m; ++n)
    if (!lists[n].empty()) S[lists[n][digit[n]]] = 1;
}

// Eq. next-config: C' = C + S . M, summing the rows of M that S selects.
// Returns false if an entry leaves the int32 range.
bool next_config(const System& s, const int32_t* C, const std::vector<uint8_t>& S,
                 std::vector<int64_t>& acc, std::vector<int32_t>& out) {
  for (int j = 0; j < s.m; ++j) acc[j] = C[j];
  for (int r = 0; r < s.R; ++r)
    if (S[r])
      for (int j = 0; j < s.m; ++j) acc[j] += (int64_t)S[r] * s.M[(size_t)r * s.m + j];
  for (int j = 0; j < s.m; ++j) {
    if (acc[j] < INT32_MIN || acc[j] > INT32_MAX) return false;
    out[j] = (int32_t)acc[j];
  }
  return true;
}

bool exceeds(const int32_t* C, int m, int32_t max_expand) {
  if (max_expand < 0) return false;
  for (int j = 0; j < m; ++j)
    if (C[j] > max_expand) return true;
  return false;
}

}  // namespace

extern "C" {

// Rules of the paper's form: one term a^rule_i[r] (a^rule_j[r])* per rule.
void* orc_system_create(int32_t m, int32_t R, const int32_t* rule_neuron, const int32_t* rule_i,
                        const int32_t* rule_j, const int32_t* M) {
  System* s = new System;
  s->m = m;
  s->R = R;
  s->rule_neuron.assign(rule_neuron, rule_neuron + R);
  s->rule_terms.resize(R + 1);
  for (int r = 0; r <= R; ++r) s->rule_terms[r] = r;
  s->term_i.assign(rule_i, rule_i + R);
  s->term_j.assign(rule_j, rule_j + R);
  s->M.assign(M, M + (size_t)R * m);
  return s;
}

// General rules: rule r's expression is the union of the terms
// [rule_terms[r], rule_terms[r + 1]).
void* orc_system_create_terms(int32_t m, int32_t R, const int32_t* rule_neuron, const int32_t* rule_terms,
                              const int32_t* term_i, const int32_t* term_j, const int32_t* M) {
  System* s = new System;
  s->m = m;
  s->R = R;
  s->rule_neuron.assign(rule_neuron, rule_neuron + R);
  s->rule_terms.assign(rule_terms, rule_terms + R + 1);
  s->term_i.assign(term_i, term_i + rule_terms[R]);
  s->term_j.assign(term_j, term_j + rule_terms[R]);
  s->M.assign(M, M + (size_t)R * m);
  return s;
}

void orc_system_free(void* sys) { delete static_cast<System*>(sys); }

// Per-rule applicability (Algorithm 2, II-1) for configuration C: ok[r] in {0,1}.
void orc_applicable(const void* sys, const int32_t* C, uint8_t* ok) {
  const System& s = *static_cast<const System*>(sys);
  for (int r = 0; r < s.R; ++r) ok[r] = applicable(s, C, r) ? 1 : 0;
}

// Eq. psi for configuration C (saturates at 2^64 - 1).
uint64_t orc_psi(const void* sys, const int32_t* C) {
  const System& s = *static_cast<const System*>(sys);
  return psi(choice_lists(s, C));
}

// All valid spiking vectors of C in canonical order, up to `cap` of them
// (S: cap x R bytes).  Returns Psi(C).
uint64_t orc_spiking_vectors(const void* sys, const int32_t* C, int64_t cap, uint8_t* S_out) {
  const System& s = *static_cast<const System*>(sys);
  auto lists = choice_lists(s, C);
  std::vector<int> digit(s.m, 0);
  std::vector<uint8_t> S(s.R);
  int64_t k = 0;
  do {
    if (k >= cap) break;
    spiking_vector(s, lists, digit, S);
    std::memcpy(S_out + (size_t)k * s.R, S.data(), s.R);
    ++k;
  } while (next_digits(lists, digit));
  return psi(lists);
}

// The children C + S.M of C for every valid S in canonical order, up to `cap`
// (out: cap x m).  Returns Psi(C); *err = 1 if a child left the int32 range.
uint64_t orc_step(const void* sys, const int32_t* C, int64_t cap, int32_t* out, int32_t* err) {
  const System& s = *static_cast<const System*>(sys);
  auto lists = choice_lists(s, C);
  std::vector<int> digit(s.m, 0);
  std::vector<uint8_t> S(s.R);
  std::vector<int64_t> acc(s.m);
  std::vector<int32_t> child(s.m);
  int64_t k = 0;
  *err = 0;
  do {
    if (k >= cap) break;
    spiking_vector(s, lists, digit, S);
    if (!next_config(s, C, S, acc, child)) *err = 1;
    std::memcpy(out + (size_t)k * s.m, child.data(), sizeof(int32_t) * s.m);
    ++k;
  } while (next_digits(lists, digit));
  return psi(lists);
}

// The t-th child of C (0-based, canonical order), found by writing t in the
// mixed radix of the per-neuron choice counts, the last neuron least
// significant.  Returns 0 if t >= Psi(C) or the child overflows, else 1.
int32_t orc_child(const void* sys, const int32_t* C, uint64_t t, int32_t* out) {
  const System& s = *static_cast<const System*>(sys);
  auto lists = choice_lists(s, C);
  if (t >= psi(lists)) return 0;
  std::vector<int> digit(s.m, 0);
  for (int n = s.m - 1; n >= 0; --n) {
    uint64_t radix = lists[n].empty() ? 1 : lists[n].size();
    digit[n] = (int)(t % radix);
    t /= radix;
  }
  std::vector<uint8_t> S(s.R);
  std::vector<int64_t> acc(s.m);
  std::vector<int32_t> child(s.m);
  spiking_vector(s, lists, digit, S);
  if (!next_config(s, C, S, acc, child)) return 0;
  std::memcpy(out, child.data(), sizeof(int32_t) * s.m);
  return 1;
}

// Breadth-first exploration from c0 (Algorithm 1 with the truncation rules in
// the header).  depth: number of expansions; cap, budget <= 0: unlimited.
void* orc_explore(const void* sys, const int32_t* c0, int32_t depth, int64_t cap, int64_t budget,
                  int32_t max_expand) {
  const System& s = *static_cast<const System*>(sys);
  Result* res = new Result;
  res->m = s.m;
  std::unordered_set<std::vector<int32_t>, VecHash> visited;
  std::vector<int32_t> root(c0, c0 + s.m);
  visited.insert(root);
  res->configs.insert(res->configs.end(), root.begin(), root.end());
  DepthStats d0;
  d0.new_configs = 1;
  res->depths.push_back(d0);

  size_t level_begin = 0, level_end = 1;  // rows of the current frontier
  std::vector<uint8_t> S(s.R);
  std::vector<int64_t> acc(s.m);
  std::vector<int32_t> child(s.m);
  std::vector<int32_t> parent(s.m);

  for (int d = 1; d <= depth; ++d) {
    DepthStats st;
    bool stop = false;
    for (size_t p = level_begin; p < level_end; ++p) {
      std::memcpy(parent.data(), res->configs.data() + p * s.m, sizeof(int32_t) * s.m);
      if (exceeds(parent.data(), s.m, max_expand)) continue;
      auto lists = choice_lists(s, parent.data());
      st.candidates = sat_add(st.candidates, psi(lists));
      if (stop) continue;  // keep summing Psi for the statistics
      std::vector<int> digit(s.m, 0);
      do {
        if (budget > 0 && st.examined >= budget) { stop = true; break; }
        st.examined += 1;
        spiking_vector(s, lists, digit, S);
        if (!next_config(s, parent.data(), S, acc, child)) {
          res->error = 1;
          stop = true;
          break;
        }
        if (visited.find(child) == visited.end()) {
          visited.insert(child);
          res->configs.insert(res->configs.end(), child.begin(), child.end());
          st.new_configs += 1;
          if (cap > 0 && st.new_configs >= cap) { stop = true; break; }
        }
      } while (next_digits(lists, digit));
    }
    st.truncated = ((uint64_t)st.examined < st.candidates) ? 1 : 0;
    res->depths.push_back(st);
    if (res->error) break;
    if (st.new_configs == 0) break;
    res->depth_reached = d;
    level_begin = level_end;
    level_end = res->configs.size() / s.m;
  }
  return res;
}

int64_t orc_result_count(const void* r) {
  const Result* res = static_cast<const Result*>(r);
  return (int64_t)(res->configs.size() / (res->m ? res->m : 1));
}

int32_t orc_result_ndepths(const void* r) { return (int32_t) static_cast<const Result*>(r)->depths.size(); }

int32_t orc_result_depth_reached(const void* r) { return static_cast<const Result*>(r)->depth_reached; }

int32_t orc_result_error(const void* r) { return static_cast<const Result*>(r)->error; }

// Rows [start, start + n) of the discovery-ordered list.
void orc_result_copy(const void* r, int64_t start, int64_t n, int32_t* out) {
  const Result* res = static_cast<const Result*>(r);
  std::memcpy(out, res->configs.data() + (size_t)start * res->m, sizeof(int32_t) * (size_t)n * res->m);
}

// Per-depth statistics: new, examined, candidates (saturating), truncated.
void orc_result_depth(const void* r, int32_t d, int64_t* new_configs, int64_t* examined,
                      uint64_t* candidates, int32_t* truncated) {
  const DepthStats& st = static_cast<const Result*>(r)->depths[d];
  *new_configs = st.new_configs;
  *examined = st.examined;
  *candidates = st.candidates;
  *truncated = st.truncated;
}

void orc_result_free(void* r) { delete static_cast<Result*>(r); }

}  // extern "C"
