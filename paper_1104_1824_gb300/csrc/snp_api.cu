// C ABI of the simulator (include/snp.h): handles, validation, device memory
// and the depth / chunk loop of the breadth-first exploration (Algorithm 1).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "snp_host.h"

using namespace snp;

namespace snp {

thread_local std::string g_err;
std::atomic<long long> g_alloc_countdown{0};
std::atomic<int> g_hold_root_slot{0};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// e4m3 byte of an integer v with |v| <= 16 (exact: 1 sign, 4 exponent bits
// with bias 7, 3 mantissa bits).
uint8_t e4m3_of_int(int v) {
  if (v == 0) return 0;
  const int a = std::abs(v);
  int e = 0;
  while ((2 << e) <= a) ++e;
  const int mant = ((a << 3) >> e) - 8;
  return (uint8_t)((v < 0 ? 0x80 : 0) | ((e + 7) << 3) | mant);
}

// fp8 tensor-core form: M_Pi^T in e4m3 for the tcgen05 B operand, uploaded on
// first use.  Block b holds rules 32b .. 32b + 31 (zero past R) for every
// column (zero past m, np = m rounded up to 16) as 8-column x 16-rule core
// matrices (128 contiguous bytes: 8 columns of 16 rules), the two 16-rule
// halves 128 bytes apart and the 8-column groups 256 bytes apart, so any run
// of columns starting at a multiple of 8 is one contiguous copy.
// Per-candidate hash and repeat buffers for q candidates.
int tc5_prepare(snp_system* h, uint64_t q) {
  if (!h->d_MB.p) {
    const int m = h->m, R = h->R;
    const int np = (m + 15) / 16 * 16, nblocks = (R + 31) / 32;
    std::vector<uint8_t> mb((size_t)nblocks * np * 32, 0);
    for (int b = 0; b < nblocks; ++b)
      for (int j = 0; j < m; ++j) {
        for (int k = 0; k < 32; ++k) {
          const int r = b * 32 + k;
          if (r >= R) break;
          const size_t o = ((size_t)b * np + (j & ~7)) * 32 + (size_t)((k >> 4) * 128 + (j & 7) * 16 + (k & 15));
          mb[o] = e4m3_of_int(h->M[(size_t)r * m + j]);
        }
      }
    TRY(h->d_MB.reserve(mb.size()));
    CK(cudaMemcpy(h->d_MB.p, mb.data(), mb.size(), cudaMemcpyHostToDevice));
    h->t5_np = np;
    h->t5_nblocks = nblocks;
  }
  if (h->tc_cap < q) {
    TRY(h->d_hash.reserve(sizeof(unsigned long long) * q));
    TRY(h->d_red.reserve(q));
    h->tc_cap = q;
  }
  return SNP_OK;
}

}  // namespace snp

namespace {

size_t claim_smem(int m) { return (size_t)kWarpsPerBlock * 3 * m * sizeof(int32_t); }

int check_device_errors(snp_system* h, cudaStream_t st, const char* where) {
  CK(cudaMemcpyAsync(h->pin.h, h->d_st.p, sizeof(ChunkState), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint32_t e = h->pin.h->error;
  if (!e) return SNP_OK;
  if (e & kErrOverflow) return fail(SNP_E_OVERFLOW, "%s: a spike count could leave the int32 range", where);
  if (e & kErrTimeout) return fail(SNP_E_TIMEOUT, "%s: bounded wait for a hash slot ran out", where);
  return fail(SNP_E_INTERNAL, "%s: device consistency check failed (bits 0x%x)", where, e);
}

// Per-pass buffers for chunks of up to q candidates: owners' store rows and
// the first-occurrence records (grow only; a fresh first-occurrence bitmap
// starts cleared).
int ensure_chunk_buffers(snp_system* h, uint64_t q, cudaStream_t st) {
  if (h->q_cap >= q) return SNP_OK;
  q = std::max<uint64_t>(q, std::min<uint64_t>(h->q_cap * 2, 1ull << 30));
  const uint64_t words = q / 32 + 1;
  TRY(h->d_sidx.reserve(sizeof(uint32_t) * q));
  TRY(h->d_gmin.reserve(sizeof(uint32_t) * q));
  TRY(h->d_slot_of.reserve(sizeof(uint32_t) * q));
  TRY(h->d_srow.reserve(sizeof(uint32_t) * q));
  TRY(h->d_bits.reserve(sizeof(uint32_t) * words));
  TRY(h->d_wbase.reserve(sizeof(uint32_t) * words));
  TRY(h->d_own.reserve(sizeof(uint32_t) * words));
  TRY(h->d_scan_tmp.reserve(scan_temp_bytes((int64_t)words, 4)));
  CK(cudaMemsetAsync(h->d_bits.p, 0, sizeof(uint32_t) * words, st));
  CK(cudaMemsetAsync(h->d_own.p, 0, sizeof(uint32_t) * words, st));
  h->q_cap = q;
  return SNP_OK;
}

// Tensor-core form: M_Pi^T in int8 (zero padded) and the rule maps, uploaded
// on first use; chunk buffers for up to q candidates.
int tc_prepare(snp_system* h, uint64_t q, cudaStream_t st) {
  if (!h->d_MT.p) {
    const int m = h->m, R = h->R;
    h->Rp = (R + 31) / 32 * 32;
    h->mp = (m + 3) / 4 * 4;
    h->mt_rows = (m + 127) / 128 * 128;
    std::vector<int8_t> mt((size_t)h->mt_rows * h->Rp, 0);
    for (int r = 0; r < R; ++r)
      for (int j = 0; j < m; ++j) mt[(size_t)j * h->Rp + r] = (int8_t)h->M[(size_t)r * m + j];
    std::vector<int16_t> rn(h->Rp, -1);
    std::vector<uint8_t> rk(h->Rp, 0);
    for (int r = 0; r < R; ++r) {
      rn[r] = (int16_t)h->rule_neuron[r];
      rk[r] = (uint8_t)(r - h->first_rule[h->rule_neuron[r]]);
    }
    TRY(h->d_MT.reserve(mt.size()));
    TRY(h->d_rn.reserve(sizeof(int16_t) * h->Rp));
    TRY(h->d_rk.reserve(h->Rp));
    CK(cudaMemcpy(h->d_MT.p, mt.data(), mt.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_rn.p, rn.data(), sizeof(int16_t) * h->Rp, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_rk.p, rk.data(), h->Rp, cudaMemcpyHostToDevice));
  }
  if (h->tc_cap < q) {
    TRY(h->d_loc.reserve((size_t)q * h->mp));
    TRY(h->d_pidx.reserve(sizeof(uint32_t) * q));
    TRY(h->d_rows.reserve(sizeof(int32_t) * (size_t)q * h->m));
    TRY(h->d_hash.reserve(sizeof(unsigned long long) * q));
    TRY(h->d_red.reserve(q));
    h->tc_cap = q;
  }
  return SNP_OK;
}

// Clears the table and inserts the configurations found so far (2 launches);
// row k lives in store row perm[k].
int rebuild_table(snp_system* h, uint64_t nbuckets, cudaStream_t st) {
  TRY(h->d_slots.reserve(nbuckets * kBucket * sizeof(unsigned long long)));
  h->nbuckets = nbuckets;
  const uint64_t nslots = nbuckets * kBucket;
  k_fill_u64<<<grid_for((int64_t)nslots, 256, 152 * 32), 256, 0, st>>>(h->d_slots.as<unsigned long long>(), nslots,
                                                                       kEmpty);
  CK(cudaGetLastError());
  if (h->n_rows > 0) {
    launch_insert_rows(h->dev(), h->d_pool.as<int32_t>(), h->row_w, h->d_perm.as<uint32_t>(), 0, h->n_rows, h->table(),
                       h->d_st.as<ChunkState>(), grid_for(h->n_rows, kWarpsPerBlock, 152 * 64), st);
    CK(cudaGetLastError());
  }
  return SNP_OK;
}

int validate_desc(const snp_system_desc* d) {
  if (!d) return fail(SNP_E_INVALID, "desc is NULL");
  if (d->m < 1 || d->m > 1024) return fail(SNP_E_INVALID, "m = %d outside [1, 1024]", d->m);
  if (d->R < 1) return fail(SNP_E_INVALID, "R = %d < 1", d->R);
  if (!d->rule_neuron || !d->M || !d->c0) return fail(SNP_E_INVALID, "NULL array in desc");
  const bool terms = d->rule_terms != nullptr;
  if (terms ? (!d->term_i || !d->term_j) : (!d->rule_i || !d->rule_j))
    return fail(SNP_E_INVALID, "NULL array in desc");
  if (terms && d->rule_terms[0] != 0) return fail(SNP_E_INVALID, "rule_terms[0] = %d must be 0", d->rule_terms[0]);
  int per = 0;
  for (int r = 0; r < d->R; ++r) {
    const int n = d->rule_neuron[r];
    if (n < 0 || n >= d->m) return fail(SNP_E_INVALID, "rule %d: neuron %d outside [0, m)", r, n);
    if (r > 0 && n < d->rule_neuron[r - 1])
      return fail(SNP_E_INVALID, "rule %d: rules must be grouped by neuron in increasing order", r);
    per = (r > 0 && n == d->rule_neuron[r - 1]) ? per + 1 : 1;
    if (per > 32) return fail(SNP_E_INVALID, "neuron %d has more than 32 rules", n);
    if (terms) {
      const int64_t k = (int64_t)d->rule_terms[r + 1] - d->rule_terms[r];
      if (k < 1 || k > 64) return fail(SNP_E_INVALID, "rule %d: %lld terms, expected 1 to 64", r, (long long)k);
      for (int t = d->rule_terms[r]; t < d->rule_terms[r + 1]; ++t)
        if (d->term_i[t] < 0 || d->term_j[t] < 0)
          return fail(SNP_E_INVALID, "rule %d: term a^%d(a^%d)* needs i, j >= 0", r, d->term_i[t], d->term_j[t]);
    } else if (d->rule_i[r] < 0 || d->rule_j[r] < 0) {
      return fail(SNP_E_INVALID, "rule %d: regex a^%d(a^%d)* needs i, j >= 0", r, d->rule_i[r], d->rule_j[r]);
    }
    for (int j = 0; j < d->m; ++j) {
      const int32_t v = d->M[(size_t)r * d->m + j];
      if (j == n && v > -1) return fail(SNP_E_INVALID, "rule %d: M[%d][%d] = %d must be -c with c >= 1", r, r, j, v);
      if (j != n && v < 0) return fail(SNP_E_INVALID, "rule %d: M[%d][%d] = %d must be >= 0", r, r, j, v);
    }
  }
  for (int j = 0; j < d->m; ++j)
    if (d->c0[j] < 0) return fail(SNP_E_INVALID, "c0[%d] = %d < 0", j, d->c0[j]);
  return SNP_OK;
}

}  // namespace

extern "C" {

void snp_explore_opts_init(snp_explore_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->depth = 1;
  o->transition = SNP_T_SPARSE_I32;
  o->frontier_cap = 0;
  o->candidate_budget = 0;
  o->max_expand_value = -1;
  o->record_parents = 0;
  o->chunk = 0;
  o->stream = nullptr;
}

const char* snp_last_error(void) { return g_err.c_str(); }

int snp_debug_fail_allocation(int64_t k) {
  g_alloc_countdown.store(k > 0 ? k : 0);
  return SNP_OK;
}

int snp_debug_hold_root_slot(int32_t on) {
  g_hold_root_slot.store(on ? 1 : 0);
  return SNP_OK;
}

int snp_abi_version(void) { return SNP_ABI_VERSION; }

int snp_load_system(const snp_system_desc* d, snp_handle* out) {
  g_err.clear();
  if (!out) return fail(SNP_E_INVALID, "out is NULL");
  *out = nullptr;
  TRY(validate_desc(d));
  snp_system* h = new (std::nothrow) snp_system;
  if (!h) return fail(SNP_E_NOMEM, "host allocation failed");
  CK(cudaGetDevice(&h->device));
  const int m = d->m, R = d->R;
  h->m = m;
  h->R = R;
  h->K = (m + 31) / 32;
  h->c0.assign(d->c0, d->c0 + m);
  h->M.assign(d->M, d->M + (size_t)R * m);
  h->rule_neuron.assign(d->rule_neuron, d->rule_neuron + R);
  // Rule expressions as unions of terms (one term per rule for the paper's form).
  h->rterm.assign(R + 1, 0);
  h->term.clear();
  for (int r = 0; r < R; ++r) {
    if (d->rule_terms) {
      for (int t = d->rule_terms[r]; t < d->rule_terms[r + 1]; ++t) h->term.push_back(make_int2(d->term_i[t], d->term_j[t]));
    } else {
      h->term.push_back(make_int2(d->rule_i[r], d->rule_j[r]));
    }
    h->rterm[r + 1] = (int32_t)h->term.size();
  }
  h->rule_i.resize(R);
  h->rule_j.resize(R);
  for (int r = 0; r < R; ++r) {  // the first term, for the tensor-core maps and reports
    h->rule_i[r] = h->term[h->rterm[r]].x;
    h->rule_j[r] = h->term[h->rterm[r]].y;
  }
  h->first_rule.assign(m + 1, 0);
  for (int r = 0; r < R; ++r) h->first_rule[d->rule_neuron[r] + 1]++;
  for (int n = 0; n < m; ++n) h->first_rule[n + 1] += h->first_rule[n];
  // M_Pi's nonzeros, rule by rule (Definition 2: -c on the own neuron, +p on synapse targets).
  h->rule.resize(R + 1);
  for (int r = 0; r < R; ++r) {
    const int32_t* row = &h->M[(size_t)r * m];
    h->rule[r] = make_int4(h->rule_i[r], h->rule_j[r], -row[d->rule_neuron[r]], (int)h->csr.size());
    for (int j = 0; j < m; ++j) {
      if (row[j] != 0) h->csr.push_back(make_int2(j, row[j]));
      h->max_abs_m = std::max(h->max_abs_m, std::abs(row[j]));
    }
  }
  h->rule[R] = make_int4(0, 0, 0, (int)h->csr.size());
  // gain[j]: at most one rule per neuron fires, so column j grows by at most
  // the sum over neurons of their largest positive entry in column j.
  std::vector<int64_t> g(m, 0);
  for (int n = 0; n < m; ++n)
    for (int j = 0; j < m; ++j) {
      int32_t best = 0;
      for (int r = h->first_rule[n]; r < h->first_rule[n + 1]; ++r) best = std::max(best, h->M[(size_t)r * m + j]);
      g[j] += best;
    }
  h->gain.resize(m);
  for (int j = 0; j < m; ++j) h->gain[j] = (int32_t)std::min<int64_t>(g[j], INT32_MAX);
  // Hash multipliers R[j] (odd, from the SplitMix64 finaliser) and each rule's
  // hash increment H[r] = sum_j M[r][j] * R[j] (mod 2^64).
  h->colkey.resize(m);
  for (int j = 0; j < m; ++j) {
    uint64_t z = 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    h->colkey[j] = (z ^ (z >> 31)) | 1ull;
  }
  // eqmask[r]: earlier rules of r's neuron whose row of M_Pi equals r's (same consumption and production).
  h->eqmask.assign(R + 1, 0u);
  for (int r = 0; r < R; ++r) {
    const int n = d->rule_neuron[r], r0 = h->first_rule[n];
    for (int q = r0; q < r; ++q)
      if (std::equal(&h->M[(size_t)q * m], &h->M[(size_t)q * m] + m, &h->M[(size_t)r * m])) h->eqmask[r] |= 1u << (q - r0);
  }
  h->rowkey.assign(R + 1, 0ull);
  for (int r = 0; r < R; ++r)
    for (int e = h->rule[r].w; e < h->rule[r + 1].w; ++e)
      h->rowkey[r] += (uint64_t)(int64_t)h->csr[e].y * h->colkey[h->csr[e].x];
  // Applicable rules by spike count.  Above T = 1 + the largest i or c of a
  // neuron's rule terms, a^x in L(a^i (a^j)*) reduces to (x - i) mod j == 0 for
  // the terms with j >= 1, so the entries repeat with period L = lcm of those j:
  // the table holds x = 0 .. T + L - 1.  Larger x fold onto T + (x - T) mod L
  // on the device, dividing by L as (v * magic) >> shift with
  // shift = 32 + ceil(log2 L) and magic = ceil(2^shift / L), exact for v < 2^31
  // (Granlund and Montgomery, PLDI 1994).
  h->ninfo.assign(m, snp::NeuronInfo{});
  h->atab.clear();
  for (int n = 0; n < m; ++n) {
    snp::NeuronInfo& ni = h->ninfo[n];
    ni.off = -1;
    ni.gain = h->gain[n];
    ni.colkey = h->colkey[n];
    const int r0 = h->first_rule[n], r1 = h->first_rule[n + 1];
    int64_t T = 1, L = 1;
    for (int r = r0; r < r1 && L <= 64; ++r)
      for (int t = h->rterm[r]; t < h->rterm[r + 1] && L <= 64; ++t) {
        T = std::max<int64_t>(T, 1 + std::max<int64_t>(h->term[t].x, h->rule[r].z));
        if (h->term[t].y >= 1) L = std::lcm<int64_t>(L, h->term[t].y);
      }
    if (L > 64 || T + L > 256) continue;  // evaluated from the rules on the device
    uint32_t lg = 0;
    while ((1ll << lg) < L) ++lg;
    ni.off = (int32_t)h->atab.size();
    ni.tl = (uint32_t)(T | (L << 16));
    ni.shift = 32 + lg;
    ni.magic = (((unsigned long long)1 << ni.shift) + (unsigned long long)L - 1) / (unsigned long long)L;
    for (int32_t x = 0; x < T + L; ++x) {
      uint32_t mask = 0;
      for (int r = r0; r < r1; ++r)
        if (rule_applies(x, h->rule[r], h->rterm.data(), h->term.data(), r)) mask |= 1u << (r - r0);
      uint32_t keep = mask;
      for (int k = 0; k < r1 - r0; ++k)
        if (((mask >> k) & 1u) && (h->eqmask[r0 + k] & mask)) keep &= ~(1u << k);
      snp::ApplEntry ae;
      ae.mask = mask;
      ae.keep = keep;
      ae.hfirst = mask ? h->rowkey[r0 + __builtin_ctz(mask)] : 0ull;
      h->atab.push_back(ae);
    }
  }
  // Rows of M_Pi on their neuron's support (see DevSys::rdesc): rules of one
  // neuron differ only there, so swapping one for another is one pass.
  h->rdesc.assign(R, make_int4(0, 0, 0, 0));
  h->scol.clear();
  h->rval.clear();
  for (int n = 0; n < m; ++n) {
    const int r0 = h->first_rule[n], r1 = h->first_rule[n + 1];
    std::vector<int32_t> sup;
    for (int r = r0; r < r1; ++r)
      for (int e = h->rule[r].w; e < h->rule[r + 1].w; ++e) sup.push_back(h->csr[e].x);
    std::sort(sup.begin(), sup.end());
    sup.erase(std::unique(sup.begin(), sup.end()), sup.end());
    const int off = (int)h->scol.size(), len = (int)sup.size();
    h->scol.insert(h->scol.end(), sup.begin(), sup.end());
    for (int r = r0; r < r1; ++r) {
      h->rdesc[r] = make_int4(off, len, (int)h->rval.size(), n);
      for (int i = 0; i < len; ++i) h->rval.push_back(h->M[(size_t)r * m + sup[i]]);
    }
  }
  // Direct table of small spike counts (see DevSys::dmask).
  h->dmask.assign((size_t)m * snp::kDirect, 0u);
  h->dhx.assign((size_t)m * snp::kDirect, 0ull);
  h->gain_small = 1;
  for (int n = 0; n < m; ++n) {
    if (h->gain[n] > INT32_MAX - snp::kDirect) h->gain_small = 0;
    for (int32_t x = 0; x < snp::kDirect; ++x) {
      uint32_t mask = 0;
      for (int r = h->first_rule[n]; r < h->first_rule[n + 1]; ++r)
        if (rule_applies(x, h->rule[r], h->rterm.data(), h->term.data(), r)) mask |= 1u << (r - h->first_rule[n]);
      h->dmask[(size_t)n * snp::kDirect + x] = mask;
      h->dhx[(size_t)n * snp::kDirect + x] = (unsigned long long)x * h->colkey[n] +
                                             (mask ? h->rowkey[h->first_rule[n] + __builtin_ctz(mask)] : 0ull);
    }
  }
  int rc = SNP_OK;
  auto up = [&](DevBuf& b, const void* src, size_t bytes) -> int {
    if ((rc = b.reserve(std::max<size_t>(bytes, 16))) != SNP_OK) return rc;
    CK(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
    return SNP_OK;
  };
  if ((rc = up(h->d_first_rule, h->first_rule.data(), sizeof(int32_t) * (m + 1))) ||
      (rc = up(h->d_rule, h->rule.data(), sizeof(int4) * (R + 1))) ||
      (rc = up(h->d_csr, h->csr.data(), sizeof(int2) * std::max<size_t>(h->csr.size(), 1))) ||
      (rc = up(h->d_gain, h->gain.data(), sizeof(int32_t) * m)) ||
      (rc = up(h->d_colkey, h->colkey.data(), sizeof(unsigned long long) * m)) ||
      (rc = up(h->d_rowkey, h->rowkey.data(), sizeof(unsigned long long) * (R + 1))) ||
      (rc = up(h->d_eqmask, h->eqmask.data(), sizeof(uint32_t) * (R + 1))) ||
      (rc = up(h->d_ninfo, h->ninfo.data(), sizeof(snp::NeuronInfo) * m)) ||
      (rc = up(h->d_atab, h->atab.data(), sizeof(snp::ApplEntry) * std::max<size_t>(h->atab.size(), 1))) ||
      (rc = up(h->d_dmask, h->dmask.data(), sizeof(uint32_t) * h->dmask.size())) ||
      (rc = up(h->d_rdesc, h->rdesc.data(), sizeof(int4) * std::max(R, 1))) ||
      (rc = up(h->d_scol, h->scol.data(), sizeof(int32_t) * std::max<size_t>(h->scol.size(), 1))) ||
      (rc = up(h->d_rval, h->rval.data(), sizeof(int32_t) * std::max<size_t>(h->rval.size(), 1))) ||
      (rc = up(h->d_rterm, h->rterm.data(), sizeof(int32_t) * (R + 1))) ||
      (rc = up(h->d_term, h->term.data(), sizeof(int2) * h->term.size())) ||
      (rc = up(h->d_dhx, h->dhx.data(), sizeof(unsigned long long) * h->dhx.size())) ||
      (rc = h->d_st.reserve(sizeof(ChunkState) + 64))) {
    delete h;
    return rc;
  }
  if (!h->pin.h) {
    delete h;
    return fail(SNP_E_NOMEM, "pinned host allocation failed");
  }
  CK(cudaEventCreate(&h->ev[0]));
  CK(cudaEventCreate(&h->ev[1]));
  for (auto& pair : h->evk)
    for (auto& e : pair) CK(cudaEventCreate(&e));
  for (auto& e : h->evs) CK(cudaEventCreate(&e, cudaEventDisableTiming));
  *out = h;
  return SNP_OK;
}

int snp_system_info(snp_handle h, int32_t* m, int32_t* R, int32_t* device) {
  g_err.clear();
  if (!h) return fail(SNP_E_INVALID, "handle is NULL");
  if (m) *m = h->m;
  if (R) *R = h->R;
  if (device) *device = h->device;
  return SNP_OK;
}

int snp_free(snp_handle h) {
  if (!h) return SNP_OK;
  cudaSetDevice(h->device);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& pair : h->evk)
    for (auto& e : pair)
      if (e) cudaEventDestroy(e);
  for (auto& e : h->evs)
    if (e) cudaEventDestroy(e);
  delete h;
  return SNP_OK;
}

int snp_step(snp_handle h, const int32_t* C, int64_t capacity, int32_t* out, uint64_t* psi) {
  g_err.clear();
  if (!h || !C || !psi || capacity < 0 || (capacity > 0 && !out)) return fail(SNP_E_INVALID, "bad arguments");
  CK(cudaSetDevice(h->device));
  const int m = h->m;
  std::vector<int32_t> c(m);
  CK(cudaMemcpy(c.data(), C, sizeof(int32_t) * m, cudaMemcpyDefault));
  for (int j = 0; j < m; ++j) {
    if (c[j] < 0) return fail(SNP_E_INVALID, "C[%d] = %d < 0", j, c[j]);
    if (c[j] > INT32_MAX - h->gain[j]) return fail(SNP_E_OVERFLOW, "C[%d] = %d: a child could leave int32", j, c[j]);
  }
  TRY(h->d_tmp.reserve(sizeof(int32_t) * m + 64));
  int32_t* dC = h->d_tmp.as<int32_t>();
  uint64_t* dpsi = reinterpret_cast<uint64_t*>(h->d_tmp.as<char>() + ((sizeof(int32_t) * m + 15) / 16) * 16);
  CK(cudaMemcpy(dC, c.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice));
  CK(cudaMemset(h->d_st.p, 0, sizeof(ChunkState)));
  launch_psi(h->dev(), dC, 4, nullptr, 1, -1, dpsi, nullptr, h->d_st.as<ChunkState>(), nullptr, sm_count(h->device));
  CK(cudaGetLastError());
  uint64_t ps = 0;
  CK(cudaMemcpy(&ps, dpsi, sizeof ps, cudaMemcpyDeviceToHost));
  *psi = ps;
  const uint64_t n = std::min<uint64_t>(ps, (uint64_t)capacity);
  if (n == 0) return SNP_OK;
  int32_t* dst = out;
  DevBuf tmp;
  const bool dev_out = is_device_ptr(out);
  if (!dev_out) {
    TRY(tmp.reserve(sizeof(int32_t) * m * n));
    dst = tmp.as<int32_t>();
  }
  const int blocks = grid_for((int64_t)n, kWarpsPerBlock, sm_count(h->device) * 8);
  k_step_children<<<blocks, kThreads, claim_smem(m)>>>(h->dev(), dC, n, dst);
  CK(cudaGetLastError());
  if (!dev_out) CK(cudaMemcpy(out, dst, sizeof(int32_t) * m * n, cudaMemcpyDeviceToHost));
  CK(cudaDeviceSynchronize());
  return SNP_OK;
}

}  // extern "C"

namespace {

// State a resumed exploration starts from (snp_explore_resume).
struct ResumeFrom {
  const int32_t* rows;        // [n x m] configurations in discovery order, host or device
  int64_t n;
  const snp_depth_info* stats;  // [nstats] per-depth records, depth 0 first
  int32_t nstats;
};

// Frontier rows whose Psi goes first when the last depth's Psi sum saturated.
constexpr int64_t kPsiHead = 8192;

// Bytes per spike count of a packed store.  Counts never go below 0 (a rule
// applies only to at least the spikes it consumes) and one step adds at most
// gain[j] to column j (at most one rule per neuron fires), so after `depths`
// more steps no count of column j exceeds cmax[j] + depths * gain[j].  The
// narrowest of uint8 (m % 16 == 0) and uint16 (m % 8 == 0) that holds every
// column's bound, else 4 (int32).
int packed_width(const snp_system* h, const std::vector<int64_t>& cmax, int64_t depths) {
  long double b = 0.0L;
  for (int j = 0; j < h->m; ++j)
    b = std::max(b, (long double)cmax[j] + (long double)depths * (long double)h->gain[j]);
  if (b <= 255.0L && h->m % 16 == 0) return 1;
  if (b <= 65535.0L && h->m % 8 == 0) return 2;
  return 4;
}

int explore_impl(snp_handle h, const snp_explore_opts* o, int32_t* depth_reached, int32_t* truncated_flags,
                 const ResumeFrom* rs) {
  g_err.clear();
  if (!h || !o) return fail(SNP_E_INVALID, "bad arguments");
  if (o->depth < 0) return fail(SNP_E_INVALID, "depth = %d < 0", o->depth);
  if (rs) {
    if (!rs->rows || !rs->stats || rs->nstats < 1 || rs->n < 1 || rs->n > 0x7FFFFFF0ll)
      return fail(SNP_E_INVALID, "bad checkpoint");
    int64_t sum = 0;
    for (int d = 0; d < rs->nstats; ++d) sum += rs->stats[d].new_configs;
    if (sum != rs->n || rs->stats[0].new_configs != 1)
      return fail(SNP_E_INVALID, "checkpoint: per-depth counts add up to %lld, not %lld rows", (long long)sum,
                  (long long)rs->n);
    if (o->depth < rs->nstats - 1)
      return fail(SNP_E_INVALID, "checkpoint already holds depth %d > %d", rs->nstats - 1, o->depth);
    if (o->record_parents) return fail(SNP_E_INVALID, "parent records cannot be resumed");
  }
  if (o->transition != SNP_T_SPARSE_I32 && o->transition != SNP_T_TC_I8 && o->transition != SNP_T_TC_F8)
    return fail(SNP_E_INVALID, "unknown transition %d", o->transition);
  if (o->reserved != 0) return fail(SNP_E_INVALID, "opts->reserved must be 0");
  if (o->packed != 0 && o->packed != 1) return fail(SNP_E_INVALID, "opts->packed = %d: expected 0 or 1", o->packed);
  if (o->transition == SNP_T_TC_I8 && h->max_abs_m > 127)
    return fail(SNP_E_RANGE, "int8 transition refused: |M_Pi| reaches %d > 127", h->max_abs_m);
  if (o->transition == SNP_T_TC_F8 && h->max_abs_m > 16)
    return fail(SNP_E_RANGE, "fp8 transition refused: |M_Pi| reaches %d > 16", h->max_abs_m);
  CK(cudaSetDevice(h->device));
  cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  h->explored = false;
  h->have_parents = false;
  h->stats.clear();
  h->depth_reached = 0;
  h->batch.reset();
  h->result_pool = nullptr;
  h->result_perm = nullptr;
  h->result_w = 4;
  const int m = h->m;
  const int nsm = sm_count(h->device);
  const int64_t cap = o->frontier_cap > 0 ? o->frontier_cap : 0;
  const int64_t budget = o->candidate_budget > 0 ? o->candidate_budget : 0;
  const bool tc = o->transition == SNP_T_TC_I8;
  // fp8 form: every candidate's row is written to its own store row
  const bool tc5 = o->transition == SNP_T_TC_F8;

  // Chunk size bound: 2^20 spiking vectors, or more while the rows a pass may
  // claim stay within ~512 MiB (passes of wide rows need 2^20 to keep every
  // warp of the expand kernel busy); the tensor-core form works on chunks of
  // at most 65536 spiking vectors.
  uint64_t qmax = o->chunk > 0 ? (uint64_t)o->chunk
                               : std::min<uint64_t>(1ull << 22, std::max<uint64_t>(1ull << 20, (1ull << 29) / (4ull * m)));
  // Wide rows: passes of 2^22, else 2^21 (fewer passes, so fewer task starts
  // and pass tails per candidate), the largest for which the store's reserve
  // for claims past the cap, one pass per depth, stays within 64 GiB.
  for (int lg = 22; lg >= 21 && o->chunk <= 0 && m > kWideM; --lg)
    if ((long double)(1ull << lg) * std::max(o->depth, 1) * 4.0L * m <= (long double)(64ull << 30)) {
      qmax = 1ull << lg;
      break;
    }
  qmax = std::min<uint64_t>(qmax, 1ull << 30);
  if (tc) {
    qmax = std::min<uint64_t>(qmax, 1ull << 16);
    TRY(tc_prepare(h, qmax, st));
  }
  if (tc5) {  // 2^21 while the in-place store's reserve (two passes per depth) stays within 64 GiB, else 2^20
    const bool big = (long double)(1ull << 21) * 2.0L * std::max(o->depth, 1) * 4.0L * m <= (long double)(64ull << 30);
    qmax = std::min<uint64_t>(qmax, big ? 1ull << 21 : 1ull << 20);
    TRY(tc5_prepare(h, qmax));
  }
  // Packed store: uint8 or uint16 counts where asked for, in the sparse form,
  // for rows of whole 16-byte pieces, and where the bound on every count the
  // exploration can reach allows it (packed_width); int32 otherwise.
  int W = 4;
  const int32_t* rs_rows = rs ? rs->rows : nullptr;  // a resumed exploration's rows (device copy when packed)
  if (o->packed && !tc && !tc5 && m % 8 == 0) {
    std::vector<int64_t> cmax(h->c0.begin(), h->c0.end());
    int64_t depths = o->depth;
    if (rs) {  // the checkpoint's largest count, for every column
      if (!is_device_ptr(rs->rows)) {
        TRY(h->d_tmp.reserve(sizeof(int32_t) * (size_t)m * rs->n));
        CK(cudaMemcpyAsync(h->d_tmp.p, rs->rows, sizeof(int32_t) * (size_t)m * rs->n, cudaMemcpyHostToDevice, st));
        rs_rows = h->d_tmp.as<int32_t>();
      }
      TRY(h->d_ctr.reserve(3 * sizeof(unsigned long long)));
      CK(cudaMemsetAsync(h->d_ctr.p, 0, sizeof(int32_t), st));
      launch_count_max(rs_rows, (int64_t)m * rs->n, h->d_ctr.as<int32_t>(), st);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h->pin.u64, h->d_ctr.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      cmax.assign(m, *reinterpret_cast<const int32_t*>(h->pin.u64));
      depths = o->depth - (rs->nstats - 1);
    }
    W = packed_width(h, cmax, depths);
  }
  h->row_w = W;
  h->pool_rows = (int64_t)(h->d_pool.bytes / ((size_t)W * m));  // the store's capacity in rows of this width
  // Pool: exact when capped, growing otherwise.
  int64_t rows_plan = 1 << 12;
  if (cap > 0) {
    const long double want = 1.0L + (long double)o->depth * (long double)cap;
    rows_plan = want > 2.0e9L ? (int64_t)2000000000 : (int64_t)want;
  }
  if (budget > 0 && cap == 0) {
    const long double want = 1.0L + (long double)o->depth * (long double)budget;
    if (want < 2.0e9L) rows_plan = std::max<int64_t>(rows_plan, std::min<int64_t>((int64_t)want, 1 << 20));
  }
  if (rs) {  // the rows so far, plus what the remaining depths may add
    const long double more = cap > 0 ? (long double)(o->depth - rs->nstats + 1) * (long double)cap : 4096.0L;
    rows_plan = (int64_t)std::min<long double>(2.0e9L, std::max<long double>((long double)rows_plan,
                                                                             (long double)rs->n + more));
  }
  // The store keeps every claimed row where its owner wrote it (claims past
  // the cap included, at most one pass's worth per depth); perm lists the
  // configurations in discovery order.
  if (h->perm_rows < rows_plan) {
    TRY(h->d_perm.reserve(sizeof(uint32_t) * rows_plan));
    h->perm_rows = rows_plan;
  }
  {
    // claims past the cap come from the pass that reaches it: one pass per
    // depth (the fp8 form takes a row per candidate: the pass that reaches
    // the cap and the one in flight behind it)
    const long double extra =
        (long double)qmax * (cap > 0 ? (long double)std::max(o->depth, 1) * (tc5 ? 2.0L : 1.0L) : 1.0L);
    const int64_t store_plan = (int64_t)std::min<long double>(2147483632.0L, (long double)rows_plan + extra);
    if (h->pool_rows < store_plan) {
      TRY(h->d_pool.reserve((size_t)W * m * store_plan));
      h->pool_rows = store_plan;
    }
  }

  if (o->record_parents) {
    TRY(h->d_rec_parent.reserve(sizeof(int64_t) * h->perm_rows));
    TRY(h->d_rec_index.reserve(sizeof(uint64_t) * h->perm_rows));
    h->rec_rows = h->perm_rows;
  }
  TRY(ensure_chunk_buffers(h, std::min<uint64_t>(qmax, 1 << 16), st));
  TRY(h->d_ctr.reserve(3 * sizeof(unsigned long long)));

  int64_t level_lo = 0, level_hi = 1;
  bool psi_saturated_before = false;  // the last depth's Psi sum reached 2^64 - 1
  int d_start = 1;
  if (rs) {  // the checkpoint's rows become store rows 0 .. n-1, in discovery order
    h->n_rows = rs->n;
    h->n_store = rs->n;
    if (W == 4) {
      CK(cudaMemcpyAsync(h->d_pool.p, rs->rows, sizeof(int32_t) * (size_t)m * rs->n, cudaMemcpyDefault, st));
    } else {
      launch_pack_rows(rs_rows, rs->n, m, W, h->d_pool.as<int32_t>(), st);
      CK(cudaGetLastError());
    }
    launch_iota_u32(h->d_perm.as<uint32_t>(), rs->n, st);
    CK(cudaGetLastError());
    level_hi = rs->n;
    level_lo = rs->n - rs->stats[rs->nstats - 1].new_configs;
    d_start = rs->nstats;
  } else {  // root level: C0, store row 0
    h->n_rows = 1;
    h->n_store = 1;
    if (W == 4) {
      CK(cudaMemcpyAsync(h->d_pool.p, h->c0.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    } else {  // C0 in the store's width (within range: packed_width bounds C0 too)
      std::vector<uint8_t>& b = h->c0_packed;
      b.resize((size_t)W * m);
      for (int j = 0; j < m; ++j) {
        const uint16_t v = (uint16_t)h->c0[j];
        if (W == 1) b[j] = (uint8_t)v;
        else std::memcpy(&b[2 * (size_t)j], &v, 2);
      }
      CK(cudaMemcpyAsync(h->d_pool.p, b.data(), b.size(), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(h->d_perm.p, 0, sizeof(uint32_t), st));
  }
  if (o->record_parents) {
    const int64_t rp = -1;
    const uint64_t ri = 0;
    CK(cudaMemcpyAsync(h->d_rec_parent.p, &rp, sizeof rp, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->d_rec_index.p, &ri, sizeof ri, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemsetAsync(h->d_st.p, 0, sizeof(ChunkState), st));
  {
    const uint64_t want =
        (uint64_t)((long double)(rows_plan + (int64_t)std::min<uint64_t>(qmax, 1 << 16)) * 4.0L / 3.0L / kBucket) + 1;
    TRY(rebuild_table(h, pow2_at_least(want), st));
    if (!rs && g_hold_root_slot.exchange(0)) {  // testing hook: C0's slot stays "being claimed"
      const uint64_t nslots = h->nbuckets * kBucket;
      k_hold_slot_of_row<<<grid_for((int64_t)nslots, 256, nsm * 8), 256, 0, st>>>(h->d_slots.as<unsigned long long>(),
                                                                                nslots, 0u);
      CK(cudaGetLastError());
    }
  }
  const uint64_t wait_ns = o->timeout_ms > 0 ? (uint64_t)o->timeout_ms * 1000000ull : 0ull;
  auto cancelled = [&]() { return o->cancel && *o->cancel != 0; };
  if (rs) {
    h->stats.assign(rs->stats, rs->stats + rs->nstats);
    for (int d = 0; d < rs->nstats; ++d)
      if (rs->stats[d].new_configs > 0) h->depth_reached = d;
    if (rs->stats[rs->nstats - 1].new_configs == 0) d_start = o->depth + 1;  // the exploration had ended
  } else {
    snp_depth_info s0;
    std::memset(&s0, 0, sizeof s0);
    s0.new_configs = 1;
    s0.launches = 2;  // the table build above
    h->stats.push_back(s0);
  }
  int64_t tombs = 0;
  double rate = 1.0;  // new configurations per candidate, for chunk sizing

  for (int d = d_start; d <= o->depth; ++d) {
    if (cancelled()) {
      CK(cudaStreamSynchronize(st));
      return fail(SNP_E_CANCELLED, "cancelled before depth %d", d);
    }
    snp_depth_info sd;
    std::memset(&sd, 0, sizeof sd);
    const int64_t P = level_hi - level_lo;
    sd.parents = P;
    CK(cudaEventRecord(h->ev[0], st));
    if (h->psi_cap < P + 1) {
      TRY(h->d_psi.reserve(sizeof(uint64_t) * (P + 1)));
      TRY(h->d_prec.reserve(sizeof(ParentRec) * (P + 1)));
      TRY(h->d_off.reserve(sizeof(uint64_t) * (P + 1)));
      TRY(h->d_scan_tmp.reserve(scan_temp_bytes(P + 1, 8)));
      h->psi_cap = P + 1;
    }
    const int32_t* parents = h->d_pool.as<int32_t>();            // the store (W bytes per count)
    const uint32_t* pperm = h->d_perm.as<uint32_t>() + level_lo;  // its rows of this frontier
    CK(cudaMemsetAsync(h->d_st.p, 0, sizeof(ChunkState), st));
    uint64_t* psi = h->d_psi.as<uint64_t>();
    CK(cudaMemsetAsync(psi + P, 0, sizeof(uint64_t), st));
    // When the previous depth's Psi sum saturated, the first rows alone may
    // hold 2^64 - 1 candidates: they go first, and if they do, the rest are
    // not read (no candidate and no statistic depends on them).
    const int64_t P0 = psi_saturated_before && P > 2 * kPsiHead ? kPsiHead : P;
    launch_psi(h->dev(), parents, W, pperm, P0, o->max_expand_value, psi, nullptr, h->d_st.as<ChunkState>(), st, nsm);
    if (P0 < P) {
      launch_psi_head_check(psi, P0, h->d_st.as<ChunkState>(), st);
      launch_psi(h->dev(), parents, W, pperm + P0, P - P0, o->max_expand_value, psi + P0, nullptr,
                 h->d_st.as<ChunkState>(), st, nsm);
      sd.launches += 2;
    }
    CK(cudaGetLastError());
    sd.launches += 1 + scan_u64_sat(psi, h->d_off.as<uint64_t>(), P + 1, h->d_scan_tmp.p, st);
    CK(cudaGetLastError());
    uint64_t total = 0;
    CK(cudaMemcpyAsync(h->pin.u64, h->d_off.as<uint64_t>() + P, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    TRY(check_device_errors(h, st, "applicability scan"));
    total = *h->pin.u64;
    sd.candidates = total;
    psi_saturated_before = total == ~0ull;
    // Parent records serve the batches that cross parents; with few
    // candidates per parent they are worth a second pass over the frontier.
    const bool with_records = !tc && !tc5 && P > 0 && total <= 256ull * (uint64_t)P;
    if (with_records) {
      launch_psi(h->dev(), parents, W, pperm, P, o->max_expand_value, psi, h->d_prec.as<ParentRec>(),
                 h->d_st.as<ChunkState>(), st, nsm);
      CK(cudaGetLastError());
      sd.launches += 1;
    }
    const uint64_t T = budget > 0 ? std::min<uint64_t>(total, (uint64_t)budget) : total;
    uint64_t remaining = cap > 0 ? (uint64_t)cap : ~0ull;  // as of the passes read back so far
    uint64_t g0 = 0, examined = 0;                         // g0: first candidate of the next pass
    int64_t nnew = 0;
    bool capped = false;
    // Device counters {rows, still acceptable}: the commit of a pass takes its
    // row base and limit from them, so the next pass can be enqueued before
    // this one is read back (at most two in flight; a pass that starts after
    // the depth is full does nothing).
    h->pin.ctr[0] = (unsigned long long)h->n_rows;
    h->pin.ctr[1] = remaining;
    h->pin.ctr[2] = (unsigned long long)h->n_store;
    CK(cudaMemcpyAsync(h->d_ctr.p, h->pin.ctr, 3 * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    struct Flight {
      uint64_t g0, Q, may_add;
      int slot;
    };
    Flight fl[2];
    int nfl = 0, next_slot = 0;
    uint64_t pend_add = 0, pend_q = 0;  // rows the passes in flight may add; their candidates
    auto retire = [&]() -> int {        // reads back the oldest pass in flight
      const Flight f = fl[0];
      fl[0] = fl[1];
      --nfl;
      CK(cudaEventSynchronize(h->evs[f.slot]));
      const ChunkState cs = *h->pin.slot[f.slot];
      *h->pin.h = cs;
      pend_add -= f.may_add;
      pend_q -= f.Q;
      if (cs.error) {
        const uint32_t e = cs.error;
        if (e & kErrOverflow) return fail(SNP_E_OVERFLOW, "expand/claim/commit: a spike count could leave the int32 range");
        if (e & kErrTimeout) return fail(SNP_E_TIMEOUT, "expand/claim/commit: bounded wait for a hash slot ran out");
        return fail(SNP_E_INTERNAL, "expand/claim/commit: device consistency check failed (bits 0x%x)", e);
      }
      if (capped) return SNP_OK;  // enqueued before the cap was known: did nothing
      if (o->kernel_timing) {
        float kms = 0.f;
        CK(cudaEventElapsedTime(&kms, h->evk[f.slot][0], h->evk[f.slot][1]));
        sd.expand_ms += kms;
      }
      const uint64_t acc = std::min<uint64_t>(cs.n_alloc, remaining);
      {
        // algorithmic bytes of the expand kernel (include/snp.h, snp_depth_info),
        // over the candidates examined (a pass that reaches the cap examines
        // its candidates up to the last one accepted)
        const int64_t row = (int64_t)W * m;
        const int64_t qx = cs.capped ? (int64_t)cs.last_lid + 1 : (int64_t)f.Q;
        const int64_t nparents = (int64_t)(cs.p_last - cs.p_first + 1);
        sd.expand_bytes += qx * 8 + (qx - (int64_t)acc) * row + (int64_t)acc * (row + 8) + nparents * row;
      }
      h->n_store += tc5 ? (int64_t)f.Q : (int64_t)cs.n_alloc;  // every claim (fp8 form: candidate) took a store row
      tombs += (int64_t)(cs.n_alloc - acc);
      nnew += (int64_t)acc;
      h->n_rows += (int64_t)acc;
      if (remaining != ~0ull) remaining -= acc;
      if (cs.capped) {
        examined = f.g0 + cs.last_lid + 1;
        capped = true;
      } else {
        examined = f.g0 + f.Q;
      }
      rate = std::max(1e-6, (double)cs.n_alloc / (double)f.Q);
      sd.chunks += 1;
      return SNP_OK;
    };
    for (;;) {
      if (cancelled()) {  // the passes in flight finish first
        while (nfl > 0) {
          const int rc = retire();
          if (rc != SNP_OK) return rc;
        }
        return fail(SNP_E_CANCELLED, "cancelled at depth %d", d);
      }
      // what the depth may still accept once the passes in flight are done, as expected from the last rate
      const double left = cap > 0 ? (double)remaining - rate * (double)pend_q : 1.0;
      if (nfl < 2 && g0 < T && !capped && remaining > 0 && (nfl == 0 || o->chunk > 0 || left > 0)) {
        uint64_t Q = std::min<uint64_t>(T - g0, qmax);
        if (o->chunk <= 0 && cap > 0) {
          const double want = std::max(left, 0.0) / std::max(rate, 1.0 / 1024.0) * 1.25 + 4096.0;
          if (want < (double)Q) Q = std::max<uint64_t>((uint64_t)want, std::min<uint64_t>(T - g0, 1 << 16));
        }
        // Room for every candidate of the pass being new, after those in flight.
        const uint64_t may_add = std::min<uint64_t>(Q, remaining);
        const uint64_t rows_hi = (uint64_t)h->n_rows + pend_add + may_add;  // discovery indices
        const uint64_t store_hi = (uint64_t)h->n_store + pend_q + Q;      // store rows (one per claim)
        if (rows_hi > 0x7FFFFFF0ull || store_hi > 0x7FFFFFF0ull) {
          if (nfl > 0) {  // the passes in flight may settle it
            TRY(retire());
            continue;
          }
          return fail(SNP_E_NOMEM, "more than 2^31 configurations");
        }
        if (rows_hi > (uint64_t)h->perm_rows) {
          const int64_t want = std::max<int64_t>(h->perm_rows * 2, (int64_t)rows_hi);
          TRY(h->d_perm.reserve(sizeof(uint32_t) * want, st, true));
          h->perm_rows = want;
          pperm = h->d_perm.as<uint32_t>() + level_lo;
          if (o->record_parents) {
            TRY(h->d_rec_parent.reserve(sizeof(int64_t) * want, st, true));
            TRY(h->d_rec_index.reserve(sizeof(uint64_t) * want, st, true));
            h->rec_rows = want;
          }
        }
        if (store_hi > (uint64_t)h->pool_rows) {
          // uncapped: double; capped (the plan was exact up to one pass per depth): a few passes more
          const uint64_t grow = cap > 0 ? store_hi + 2 * qmax : std::max<uint64_t>(2ull * h->pool_rows, store_hi);
          const int64_t want = (int64_t)std::min<uint64_t>(0x7FFFFFF0ull, grow);
          TRY(h->d_pool.reserve((size_t)W * m * want, st, true));
          h->pool_rows = want;
          parents = h->d_pool.as<int32_t>();
        }
        const uint64_t nslots = h->nbuckets * kBucket;
        if ((long double)(h->n_rows + tombs) + (long double)(pend_q + Q) > 0.75L * (long double)nslots) {
          if (nfl > 0) {  // a rebuild needs exact counts
            TRY(retire());
            continue;
          }
          uint64_t nb = h->nbuckets;
          while ((long double)(h->n_rows + Q) > 0.5L * (long double)(nb * kBucket)) nb *= 2;
          TRY(rebuild_table(h, nb, st));
          sd.launches += 2;
          tombs = 0;
        }
        TRY(ensure_chunk_buffers(h, Q, st));
        const int slot = next_slot;
        next_slot ^= 1;
        CK(cudaMemsetAsync(h->d_st.p, 0, sizeof(ChunkState), st));
        {
          ClaimArgs a;
          a.sys = h->dev();
          a.parents = parents;
          a.off = h->d_off.as<uint64_t>();
          a.P = P;
          a.g0 = g0;
          a.Q = (uint32_t)Q;
          a.run = 0;
          a.table = h->table();
          a.pperm = pperm;
          a.pool = h->d_pool.as<int32_t>();
          a.staging = nullptr;
          a.store_ctr = h->d_ctr.as<unsigned long long>() + 2;
          a.sidx_of = h->d_sidx.as<uint32_t>();
          a.store_cap = (uint64_t)h->pool_rows;
          a.gmin = h->d_gmin.as<uint32_t>();
          a.slot_of = h->d_slot_of.as<uint32_t>();
          a.ownbits = h->d_own.as<uint32_t>();
          a.prec = with_records ? h->d_prec.as<ParentRec>() : nullptr;
          a.ctr = h->d_ctr.as<unsigned long long>();
          a.st = h->d_st.as<ChunkState>();
          a.wait_ns = wait_ns;
          a.w = W;
          if (o->kernel_timing) CK(cudaEventRecord(h->evk[slot][0], st));
          if (tc5) {
            Tc5Args t;
            t.s = a.sys;
            t.parents = parents;
            t.pperm = pperm;
            t.off = a.off;
            t.P = P;
            t.g0 = g0;
            t.Q = (uint32_t)Q;
            t.MB = h->d_MB.as<uint8_t>();
            t.np = h->t5_np;
            t.nblocks = h->t5_nblocks;
            t.slots = tc5_slots(m, h->t5_nblocks);
            t.delta = m > kWideM ? 1 : 0;
            a.inplace = 1;
            a.inplace_base = (uint64_t)h->n_store + pend_q;
            t.out = h->d_pool.as<int32_t>() + (size_t)a.inplace_base * m;
            t.store_row0 = a.inplace_base;
            CUtensorMap map;
            std::memset(&map, 0, sizeof map);
            t.use_map = tc5_store_map(&map, h->d_pool.as<int32_t>(), m, (uint64_t)h->pool_rows) ? 1 : 0;
            t.hash = h->d_hash.as<unsigned long long>();
            t.red = h->d_red.as<uint8_t>();
            t.ctr = a.ctr;
            t.st = a.st;
            launch_tc5(t, map, st, nsm);
            launch_resolve_rows(a, t.out, t.hash, t.red, st, nsm);
            sd.launches += 2;
          } else if (tc) {
            launch_tc_digits(a.sys, parents, pperm, a.off, P, g0, (uint32_t)Q, h->d_loc.as<uint8_t>(), h->mp,
                             h->d_pidx.as<uint32_t>(), h->d_red.as<uint8_t>(), st, nsm);
            CK(cudaMemsetAsync(h->d_hash.p, 0, sizeof(unsigned long long) * Q, st));
            launch_tc_rows(a.sys, parents, h->d_loc.as<uint8_t>(), h->mp, h->d_pidx.as<uint32_t>(), (uint32_t)Q,
                           h->d_MT.as<int8_t>(), h->Rp, h->d_rn.as<int16_t>(), h->d_rk.as<uint8_t>(),
                           h->d_rows.as<int32_t>(), h->d_hash.as<unsigned long long>(), st);
            launch_resolve_rows(a, h->d_rows.as<int32_t>(), h->d_hash.as<unsigned long long>(),
                                h->d_red.as<uint8_t>(), st, nsm);
            sd.launches += 3;
          } else {
            if (m > kWideM) {
              TRY(h->d_bcache.reserve(wide_base_bytes(m)));
              a.bcache = h->d_bcache.as<int32_t>();
            }
            sd.launches += launch_expand(a, st, nsm);
          }
          CK(cudaGetLastError());
          if (o->kernel_timing) CK(cudaEventRecord(h->evk[slot][1], st));
        }
        const uint32_t nwords = (uint32_t)((Q + 31) / 32);
        k_mark<<<grid_for(nwords, 256, nsm * 8), 256, 0, st>>>(h->d_own.as<uint32_t>(), h->d_gmin.as<uint32_t>(),
                                                                 h->d_bits.as<uint32_t>(), h->d_srow.as<uint32_t>(),
                                                                 nwords, h->d_st.as<ChunkState>());
        launch_popc(h->d_bits.as<uint32_t>(), h->d_wbase.as<uint32_t>(), nwords, st);
        sd.launches += 2 + scan_u32(h->d_wbase.as<uint32_t>(), h->d_wbase.as<uint32_t>(), nwords, h->d_scan_tmp.p, st);
        CommitArgs c;
        c.sys = h->dev();
        c.nwords = nwords;
        c.bits = h->d_bits.as<uint32_t>();
        c.wbase = h->d_wbase.as<uint32_t>();
        c.srow = h->d_srow.as<uint32_t>();
        c.slot_of = h->d_slot_of.as<uint32_t>();
        c.staging = nullptr;
        c.table = h->table();
        c.pool = h->d_pool.as<int32_t>();
        c.perm = h->d_perm.as<uint32_t>();
        c.sidx_of = h->d_sidx.as<uint32_t>();
        c.row_base = 0;
        c.remaining = 0;
        c.ctr = h->d_ctr.as<unsigned long long>();
        c.rec_parent = o->record_parents ? h->d_rec_parent.as<int64_t>() : nullptr;
        c.rec_index = o->record_parents ? h->d_rec_index.as<uint64_t>() : nullptr;
        c.off = h->d_off.as<uint64_t>();
        c.P = P;
        c.parent_base = level_lo;
        c.g0 = g0;
        c.st = h->d_st.as<ChunkState>();
        k_commit<<<grid_for(nwords, 8, nsm * 16), 256, 0, st>>>(c);
        CK(cudaGetLastError());
        k_clear_bits<<<grid_for(nwords, 256, nsm * 8), 256, 0, st>>>(h->d_bits.as<uint32_t>(), nwords,
                                                                       h->d_ctr.as<unsigned long long>(),
                                                                       h->d_st.as<ChunkState>());
        CK(cudaGetLastError());
        sd.launches += 2;
        CK(cudaMemcpyAsync(h->pin.slot[slot], h->d_st.p, sizeof(ChunkState), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(h->evs[slot], st));
        fl[nfl++] = Flight{g0, Q, may_add, slot};
        pend_add += may_add;
        pend_q += Q;
        g0 += Q;
        continue;
      }
      if (nfl == 0) break;
      TRY(retire());
    }
    CK(cudaEventRecord(h->ev[1], st));
    CK(cudaEventSynchronize(h->ev[1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
    sd.ms = ms;
    sd.new_configs = nnew;
    sd.examined = (int64_t)examined;
    sd.truncated = examined < total ? 1 : 0;
    h->stats.push_back(sd);
    if (nnew == 0) break;
    h->depth_reached = d;
    level_lo = level_hi;
    level_hi = h->n_rows;
  }
  h->explored = true;
  h->result_pool = h->d_pool.as<int32_t>();
  h->result_perm = h->d_perm.as<uint32_t>();
  h->result_w = W;
  h->have_parents = o->record_parents != 0;
  if (depth_reached) *depth_reached = h->depth_reached;
  if (truncated_flags)
    for (int d = 0; d <= o->depth; ++d)
      truncated_flags[d] = d < (int)h->stats.size() ? h->stats[d].truncated : 0;
  return SNP_OK;
}

}  // namespace

extern "C" {

int snp_explore(snp_handle h, const snp_explore_opts* o, int32_t* depth_reached, int32_t* truncated_flags) {
  return explore_impl(h, o, depth_reached, truncated_flags, nullptr);
}

int snp_explore_resume(snp_handle h, const int32_t* rows, int64_t n, const snp_depth_info* stats, int32_t nstats,
                       const snp_explore_opts* o, int32_t* depth_reached, int32_t* truncated_flags) {
  const ResumeFrom rs{rows, n, stats, nstats};
  return explore_impl(h, o, depth_reached, truncated_flags, &rs);
}

int snp_reachable(snp_handle h, int32_t* out, int64_t capacity, int64_t* n, int64_t* per_depth_new) {
  g_err.clear();
  if (!h || !n) return fail(SNP_E_INVALID, "bad arguments");
  if (!h->explored) return fail(SNP_E_STATE, "no exploration to report");
  *n = h->n_rows;
  if (per_depth_new)
    for (int d = 0; d <= h->depth_reached; ++d) per_depth_new[d] = h->stats[d].new_configs;
  if (capacity < h->n_rows) return fail(SNP_E_BUFFER, "capacity %lld < %lld rows", (long long)capacity, (long long)h->n_rows);
  if (!out) return fail(SNP_E_INVALID, "out is NULL");
  CK(cudaSetDevice(h->device));
  const size_t bytes = sizeof(int32_t) * (size_t)h->m * h->n_rows;
  if (!h->result_perm && h->result_w == 4) {
    CK(cudaMemcpy(out, h->result_pool, bytes, cudaMemcpyDefault));
    return SNP_OK;
  }
  // rows in discovery order: gather from the store (into `out` when it is
  // device memory, else through a device buffer)
  int32_t* dst = out;
  if (!is_device_ptr(out)) {
    TRY(h->d_tmp.reserve(bytes));
    dst = h->d_tmp.as<int32_t>();
  }
  launch_gather_rows(h->result_pool, h->result_w, h->result_perm, h->n_rows, h->m, dst, nullptr);
  CK(cudaGetLastError());
  if (dst != out) CK(cudaMemcpy(out, dst, bytes, cudaMemcpyDeviceToHost));
  else CK(cudaDeviceSynchronize());
  return SNP_OK;
}

int snp_row_width(snp_handle h, int32_t* bytes_per_count) {
  g_err.clear();
  if (!h || !bytes_per_count) return fail(SNP_E_INVALID, "bad arguments");
  if (!h->explored) return fail(SNP_E_STATE, "no exploration to report");
  *bytes_per_count = h->result_w;
  return SNP_OK;
}

int snp_parents(snp_handle h, int64_t* parent, uint64_t* index, int64_t capacity, int64_t* n) {
  g_err.clear();
  if (!h || !n) return fail(SNP_E_INVALID, "bad arguments");
  if (!h->explored || !h->have_parents) return fail(SNP_E_STATE, "no parent records (set record_parents)");
  *n = h->n_rows;
  if (capacity < h->n_rows) return fail(SNP_E_BUFFER, "capacity %lld < %lld", (long long)capacity, (long long)h->n_rows);
  CK(cudaSetDevice(h->device));
  if (parent) CK(cudaMemcpy(parent, h->d_rec_parent.p, sizeof(int64_t) * h->n_rows, cudaMemcpyDefault));
  if (index) CK(cudaMemcpy(index, h->d_rec_index.p, sizeof(uint64_t) * h->n_rows, cudaMemcpyDefault));
  return SNP_OK;
}

int snp_depth_stats(snp_handle h, int32_t d, snp_depth_info* out) {
  g_err.clear();
  if (!h || !out) return fail(SNP_E_INVALID, "bad arguments");
  if (!h->explored) return fail(SNP_E_STATE, "no exploration");
  if (d < 0 || d >= (int)h->stats.size()) return fail(SNP_E_INVALID, "depth %d outside [0, %d)", d, (int)h->stats.size());
  *out = h->stats[d];
  return SNP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Exploration without allocation (snp_explore_static).
//
// Some callers cannot allocate device memory when they need an exploration:
// code that runs while a framework's caching allocator owns all free device
// memory, and latency-critical loops that must never block on the allocator.
// For them, snp_explore_static takes the output buffer from the caller (it
// doubles as the configuration pool) and carves every other buffer it needs
// (hash table, staging rows, first-occurrence bitmap, Psi prefix sums, scan
// temporaries, counters) out of one array compiled into this library.  It
// still launches kernels, copies counters to the host and waits on the
// caller's stream once per pass, so it cannot be called from a stream
// callback or on a stream that is being captured.
//
// The array is fixed at kStaticScratchBytes; every GPU that loads the library
// holds it until the process exits.  Calls share it and each call leaves its
// contents behind: a call clears what must start empty (table, bitmap,
// counters) before use, and two calls whose work overlaps on the GPU (other
// streams, other threads) race on it.  The first call on a device (and the
// first after the device's context was recreated) looks up the array's device
// address (cudaGetSymbolAddress) with that device current.

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;    // 64 MiB
constexpr uint64_t kStaticSlots = 1ull << 21;           // hash slots (16 MiB)
constexpr int64_t kStaticMaxRows = 1ll << 20;           // configurations per call
constexpr size_t kStaticStagingBytes = 24ull << 20;     // rows claimed per pass
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};
void* g_static_ctx[kStaticMaxDevices] = {};  // the context each address was looked up in

// The current CUDA context (cuCtxGetCurrent through the runtime's driver entry
// point), or nullptr when it cannot be told.
void* current_context() {
  using Fn = int (*)(void**);
  static Fn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<Fn>(p);
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of g_static_scratch on the current device: looked up once
// per device and context (a recreated context maps the array anew).
int static_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= kStaticMaxDevices) return fail(SNP_E_INVALID, "device %d out of range", device);
  void* ctx = current_context();
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device] || !ctx || g_static_ctx[device] != ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(SNP_E_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    g_static_addr[device] = p;
    g_static_ctx[device] = ctx;
  }
  *out = static_cast<unsigned char*>(g_static_addr[device]);
  return SNP_OK;
}

// Restores the caller's current device on scope exit.
struct DeviceRestore {
  int prev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~DeviceRestore() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct StaticLayout {
  ChunkState* st;
  unsigned long long* slots;
  uint64_t* psi;
  uint64_t* off;
  void* scan_tmp;
  int32_t* staging;
  uint32_t *gmin, *slot_of, *srow, *bits, *wbase, *own;
  uint64_t q;  // candidates per pass
};

// Carves the scratch array; every piece starts on a 256-byte boundary.
bool static_layout(unsigned char* base, int m, StaticLayout* L) {
  size_t at = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + at;
    at += (bytes + 255) & ~size_t(255);
    return p;
  };
  uint64_t q = std::min<uint64_t>(1ull << 16, kStaticStagingBytes / (4ull * m));
  q &= ~31ull;
  L->q = q;
  L->st = reinterpret_cast<ChunkState*>(take(256));
  L->slots = reinterpret_cast<unsigned long long*>(take(kStaticSlots * sizeof(unsigned long long)));
  L->psi = reinterpret_cast<uint64_t*>(take((kStaticMaxRows + 1) * sizeof(uint64_t)));
  L->off = reinterpret_cast<uint64_t*>(take((kStaticMaxRows + 1) * sizeof(uint64_t)));
  L->scan_tmp = take(std::max(scan_temp_bytes(kStaticMaxRows + 1, 8), scan_temp_bytes((int64_t)q / 32 + 1, 4)));
  L->staging = reinterpret_cast<int32_t*>(take(q * 4ull * m));
  L->gmin = reinterpret_cast<uint32_t*>(take(q * 4));
  L->slot_of = reinterpret_cast<uint32_t*>(take(q * 4));
  L->srow = reinterpret_cast<uint32_t*>(take(q * 4));
  L->bits = reinterpret_cast<uint32_t*>(take((q / 32 + 1) * 4));
  L->wbase = reinterpret_cast<uint32_t*>(take((q / 32 + 1) * 4));
  L->own = reinterpret_cast<uint32_t*>(take((q / 32 + 1) * 4));
  return at <= kStaticScratchBytes;
}

}  // namespace

extern "C" int snp_explore_static(snp_handle h, const snp_explore_opts* o, int32_t* out, int64_t capacity,
                                  int64_t* n, int32_t* depth_reached, int64_t* per_depth_new) {
  g_err.clear();
  if (!h || !o || !out || !n) return fail(SNP_E_INVALID, "bad arguments");
  if (o->depth < 0) return fail(SNP_E_INVALID, "depth = %d < 0", o->depth);
  if (o->transition != SNP_T_SPARSE_I32) return fail(SNP_E_INVALID, "only the sparse int32 transition runs here");
  if (o->record_parents) return fail(SNP_E_INVALID, "parent records need allocation; use snp_explore");
  if (capacity < 1) return fail(SNP_E_BUFFER, "capacity %lld < 1", (long long)capacity);
  if (capacity > kStaticMaxRows)
    return fail(SNP_E_INVALID, "capacity %lld exceeds the static scratch limit of %lld configurations",
                (long long)capacity, (long long)kStaticMaxRows);
  {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, out) != cudaSuccess) {
      cudaGetLastError();
      return fail(SNP_E_INVALID, "out must be device memory");
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
      return fail(SNP_E_INVALID, "out must be device memory");
    if (pa.type == cudaMemoryTypeDevice && pa.device != h->device)
      return fail(SNP_E_INVALID, "out is on device %d, the system on device %d", pa.device, h->device);
  }
  DeviceRestore keep_device;
  CK(cudaSetDevice(h->device));
  unsigned char* base = nullptr;
  TRY(static_scratch(h->device, &base));
  StaticLayout L;
  if (!static_layout(base, h->m, &L)) return fail(SNP_E_INTERNAL, "static scratch layout does not fit");
  cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  const int m = h->m;
  const int nsm = sm_count(h->device);
  const int64_t cap = o->frontier_cap > 0 ? o->frontier_cap : 0;
  const int64_t budget = o->candidate_budget > 0 ? o->candidate_budget : 0;
  const uint64_t qmax = o->chunk > 0 ? std::min<uint64_t>((uint64_t)o->chunk, L.q) : L.q;
  const DevTable table{L.slots, kStaticSlots / kBucket - 1};
  ChunkState* hst = h->pin.h;

  // Start state: C0 in row 0 of out, an empty table holding C0, a clear bitmap.
  CK(cudaMemcpyAsync(out, h->c0.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(L.st, 0, sizeof(ChunkState), st));
  CK(cudaMemsetAsync(L.bits, 0, sizeof(uint32_t) * (L.q / 32 + 1), st));
  CK(cudaMemsetAsync(L.own, 0, sizeof(uint32_t) * (L.q / 32 + 1), st));
  auto clear_and_insert = [&](int64_t rows) -> int {
    k_fill_u64<<<grid_for((int64_t)kStaticSlots, 256, nsm * 32), 256, 0, st>>>(L.slots, kStaticSlots, kEmpty);
    CK(cudaGetLastError());
    launch_insert_rows(h->dev(), out, 4, nullptr, 0, rows, table, L.st, grid_for(rows, kWarpsPerBlock, nsm * 64), st);
    CK(cudaGetLastError());
    return SNP_OK;
  };
  TRY(clear_and_insert(1));
  int64_t n_rows = 1, level_lo = 0, level_hi = 1, tombs = 0;
  int32_t reached = 0;
  if (per_depth_new) {
    per_depth_new[0] = 1;
    for (int d = 1; d <= o->depth; ++d) per_depth_new[d] = 0;
  }
  double rate = 1.0;

  for (int d = 1; d <= o->depth; ++d) {
    const int64_t P = level_hi - level_lo;
    const int32_t* parents = out + (size_t)level_lo * m;
    CK(cudaMemsetAsync(L.st, 0, sizeof(ChunkState), st));
    CK(cudaMemsetAsync(L.psi + P, 0, sizeof(uint64_t), st));
    launch_psi(h->dev(), parents, 4, nullptr, P, o->max_expand_value, L.psi, nullptr, L.st, st, nsm);
    CK(cudaGetLastError());
    scan_u64_sat(L.psi, L.off, P + 1, L.scan_tmp, st);
    CK(cudaMemcpyAsync(h->pin.u64, L.off + P, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hst, L.st, sizeof(ChunkState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hst->error & kErrOverflow) return fail(SNP_E_OVERFLOW, "a spike count could leave the int32 range");
    if (hst->error) return fail(SNP_E_INTERNAL, "device consistency check failed (bits 0x%x)", hst->error);
    const uint64_t total = *h->pin.u64;
    const uint64_t T = budget > 0 ? std::min<uint64_t>(total, (uint64_t)budget) : total;
    uint64_t remaining = cap > 0 ? (uint64_t)cap : ~0ull;
    uint64_t g0 = 0;
    int64_t nnew = 0;
    bool capped = false;
    while (g0 < T && !capped) {
      uint64_t Q = std::min<uint64_t>(T - g0, qmax);
      if (o->chunk <= 0 && cap > 0) {
        const double want = (double)remaining / std::max(rate, 1.0 / 1024.0) * 1.25 + 4096.0;
        if (want < (double)Q) Q = std::max<uint64_t>((uint64_t)want, std::min<uint64_t>(T - g0, 1 << 12));
      }
      // At most `room` more rows fit in out: the pass commits no more than that
      // and fails if it found more new configurations than fit.
      const uint64_t room = (uint64_t)(capacity - n_rows);
      const uint64_t accept = std::min<uint64_t>(remaining, room);
      const bool cap_limits = remaining <= room;  // the frontier cap, not the buffer, bounds this pass
      if ((long double)(n_rows + tombs) + (long double)Q > 0.75L * (long double)kStaticSlots) {
        TRY(clear_and_insert(n_rows));  // drops tombstones; n_rows + Q always fits
        tombs = 0;
      }
      CK(cudaMemsetAsync(L.st, 0, sizeof(ChunkState), st));
      ClaimArgs a;
      a.sys = h->dev();
      a.parents = parents;
      a.off = L.off;
      a.P = P;
      a.g0 = g0;
      a.Q = (uint32_t)Q;
      a.run = 0;
      a.table = table;
      a.pool = out;
      a.staging = L.staging;
      a.gmin = L.gmin;
      a.slot_of = L.slot_of;
      a.ownbits = L.own;
      a.prec = nullptr;
      a.ctr = nullptr;
      a.pperm = nullptr;
      a.store_ctr = nullptr;  // staging mode: rows are copied into `out` by the commit
      a.sidx_of = nullptr;
      a.store_cap = 0;
      a.st = L.st;
      a.wait_ns = o->timeout_ms > 0 ? (uint64_t)o->timeout_ms * 1000000ull : 0ull;
      launch_expand(a, st, nsm);
      CK(cudaGetLastError());
      const uint32_t nwords = (uint32_t)((Q + 31) / 32);
      k_mark<<<grid_for(nwords, 256, nsm * 8), 256, 0, st>>>(L.own, L.gmin, L.bits, L.srow, nwords, L.st);
      launch_popc(L.bits, L.wbase, nwords, st);
      scan_u32(L.wbase, L.wbase, nwords, L.scan_tmp, st);
      CommitArgs c;
      c.sys = h->dev();
      c.nwords = nwords;
      c.bits = L.bits;
      c.wbase = L.wbase;
      c.srow = L.srow;
      c.slot_of = L.slot_of;
      c.staging = L.staging;
      c.table = table;
      c.pool = out;
      c.row_base = n_rows;
      c.remaining = accept;
      c.rec_parent = nullptr;
      c.rec_index = nullptr;
      c.off = L.off;
      c.P = P;
      c.parent_base = level_lo;
      c.g0 = g0;
      c.ctr = nullptr;
      c.perm = nullptr;
      c.sidx_of = nullptr;
      c.st = L.st;
      k_commit<<<grid_for(nwords, 8, nsm * 16), 256, 0, st>>>(c);
      CK(cudaGetLastError());
      k_clear_bits<<<grid_for(nwords, 256, nsm * 8), 256, 0, st>>>(L.bits, nwords, nullptr, nullptr);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(hst, L.st, sizeof(ChunkState), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (hst->error & kErrTimeout) return fail(SNP_E_TIMEOUT, "bounded wait for a hash slot ran out");
      if (hst->error) return fail(SNP_E_INTERNAL, "device consistency check failed (bits 0x%x)", hst->error);
      if (hst->n_alloc > room && room < remaining)
        return fail(SNP_E_BUFFER, "capacity %lld reached at depth %d with new configurations left",
                    (long long)capacity, d);
      const uint64_t acc = std::min<uint64_t>(hst->n_alloc, accept);
      tombs += (int64_t)(hst->n_alloc - acc);
      nnew += (int64_t)acc;
      n_rows += (int64_t)acc;
      if (remaining != ~0ull) remaining -= acc;
      capped = hst->capped != 0 && cap_limits;
      rate = std::max(1e-6, (double)hst->n_alloc / (double)Q);
      g0 += Q;
    }
    if (per_depth_new) per_depth_new[d] = nnew;
    if (nnew == 0) break;
    reached = d;
    level_lo = level_hi;
    level_hi = n_rows;
  }
  *n = n_rows;
  if (depth_reached) *depth_reached = reached;
  return SNP_OK;
}
