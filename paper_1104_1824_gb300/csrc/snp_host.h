// Host-side state shared by the C ABI's translation units: error reporting,
// device buffers and the handle of a loaded system.
#pragma once

#include <cstdarg>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "snp.h"
#include "snp_kernels.cuh"

namespace snp {

// Message of the last failed call on this thread (snp_last_error).
extern thread_local std::string g_err;

// Records a message for snp_last_error and returns code.
int fail(int code, const char* fmt, ...);

// True for device or managed memory.
bool is_device_ptr(const void* p);

#define CK(x)                                                                                    \
  do {                                                                                           \
    cudaError_t e_ = (x);                                                                        \
    if (e_ != cudaSuccess) {                                                                     \
      if (e_ == cudaErrorMemoryAllocation) {                                                     \
        cudaGetLastError();                                                                      \
        return fail(SNP_E_NOMEM, "%s: %s", #x, cudaGetErrorString(e_));                          \
      }                                                                                          \
      return fail(SNP_E_CUDA, "%s (%s:%d): %s", #x, __FILE__, __LINE__, cudaGetErrorString(e_)); \
    }                                                                                            \
  } while (0)

#define TRY(x)              \
  do {                      \
    int r_ = (x);           \
    if (r_ != SNP_OK) return r_; \
  } while (0)

// A device allocation that grows on demand (contents are not preserved unless asked).
// Testing hook (snp_debug_fail_allocation): while positive, each device
// allocation counts it down and the one that reaches zero fails.
extern std::atomic<long long> g_alloc_countdown;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  inline int reserve(size_t want, cudaStream_t st = nullptr, bool keep = false) {
    if (want <= bytes) return SNP_OK;
    if (g_alloc_countdown.load(std::memory_order_relaxed) > 0 && g_alloc_countdown.fetch_sub(1) == 1)
      return fail(SNP_E_NOMEM, "cudaMalloc(%zu bytes): refused by the fault-injection hook", want);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SNP_E_NOMEM, "cudaMalloc(%zu bytes): %s", want, cudaGetErrorString(e));
    }
    if (keep && p && bytes) {
      e = cudaMemcpyAsync(q, p, bytes, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        cudaFree(q);
        return fail(SNP_E_CUDA, "grow copy: %s", cudaGetErrorString(e));
      }
    }
    release();
    p = q;
    bytes = want;
    return SNP_OK;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Pinned host words the depth loop reads back: chunk counters and one u64.
struct PinnedState {
  ChunkState* h = nullptr;      // counters of the last pass read back
  ChunkState* slot[2] = {nullptr, nullptr};  // counters of passes in flight
  uint64_t* u64 = nullptr;
  unsigned long long* ctr = nullptr;         // source of the device counters {rows, still acceptable}
  PinnedState() {
    void* p = nullptr;
    if (cudaMallocHost(&p, 512) == cudaSuccess) {
      char* c = static_cast<char*>(p);
      h = reinterpret_cast<ChunkState*>(c);
      u64 = reinterpret_cast<uint64_t*>(c + 128);
      slot[0] = reinterpret_cast<ChunkState*>(c + 192);
      slot[1] = reinterpret_cast<ChunkState*>(c + 256);
      ctr = reinterpret_cast<unsigned long long*>(c + 320);
    }
  }
  ~PinnedState() {
    if (h) cudaFreeHost(h);
  }
};

inline uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = kWarpsPerBlock * 32;

inline int grid_for(int64_t work_items, int per_block, int max_blocks) {
  int64_t b = (work_items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

inline int sm_count(int device) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
  return n > 0 ? n : 1;
}

struct BatchArena;

}  // namespace snp

using snp::DevBuf;
using snp::PinnedState;

struct snp_system {
  int device = 0;
  int32_t m = 0, R = 0, K = 1;
  int32_t max_abs_m = 0;
  std::vector<int32_t> c0, M, rule_neuron, rule_i, rule_j, first_rule, gain;
  std::vector<uint8_t> c0_packed;  // C0 in a packed store's width (staging of its upload)
  std::vector<int4> rule;
  std::vector<int2> csr;
  // device copies of the system
  DevBuf d_first_rule, d_rule, d_csr, d_gain, d_colkey, d_rowkey, d_eqmask, d_ninfo, d_atab, d_dmask, d_dhx, d_rdesc,
      d_scol, d_rval, d_rterm, d_term;
  std::vector<uint32_t> eqmask;
  std::vector<snp::NeuronInfo> ninfo;       // per-neuron constants of the applicability scan
  std::vector<snp::ApplEntry> atab;         // applicable rules by spike count
  std::vector<uint32_t> dmask;              // [m][kDirect] applicable masks of small counts
  std::vector<unsigned long long> dhx;      // [m][kDirect] x * R[n] + H[first applicable rule]
  int32_t gain_small = 0;
  std::vector<int4> rdesc;                  // per rule: support offset, length, value offset, neuron
  std::vector<int32_t> scol, rval;          // neuron supports; rule values on them
  std::vector<int32_t> rterm;               // [R + 1] terms of rule r: [rterm[r], rterm[r + 1])
  std::vector<int2> term;                   // {i, j} of each term a^i (a^j)*
  // tensor-core form: M_Pi^T as int8 [mt_rows][Rp], per-rule neuron and position
  DevBuf d_MT, d_rn, d_rk, d_loc, d_pidx, d_rows, d_hash, d_red;
  // fp8 tensor-core form: M_Pi^T in e4m3 (tc5_pack_mt), its column and block counts
  DevBuf d_MB;
  int32_t t5_np = 0, t5_nblocks = 0;
  int32_t Rp = 0, mp = 0, mt_rows = 0;
  uint64_t tc_cap = 0;  // candidates the tensor-core chunk buffers hold
  std::vector<unsigned long long> colkey, rowkey;
  // exploration state
  DevBuf d_pool, d_slots, d_gmin, d_slot_of, d_bits, d_wbase, d_srow, d_own, d_off, d_scan_tmp, d_st,
      d_rec_parent, d_rec_index, d_tmp,
      d_psi, d_prec, d_ctr, d_perm, d_sidx,
      d_bcache;  // wide mode: base children of each pass's largest parents
  int64_t pool_rows = 0;  // capacity in rows (of the store: every row claimed during an exploration)
  int32_t row_w = 4;      // bytes per spike count of the store's rows (4: int32; 2, 1: packed)
  int64_t perm_rows = 0;  // capacity of perm (discovery index -> store row)
  int64_t n_store = 0;    // store rows in use
  uint64_t nbuckets = 0;
  uint64_t q_cap = 0;     // staging capacity in rows
  int64_t psi_cap = 0;    // parents
  int64_t rec_rows = 0;
  PinnedState pin;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaEvent_t evk[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // around the expand kernel, per pass slot
  cudaEvent_t evs[2] = {nullptr, nullptr};   // end of a pass in flight, per slot
  // results
  bool explored = false;
  bool have_parents = false;
  int64_t n_rows = 0;
  int32_t depth_reached = 0;
  std::vector<snp_depth_info> stats;
  // After snp_explore_batch the configurations live in a shared batch arena.
  std::shared_ptr<snp::BatchArena> batch;
  const int32_t* result_pool = nullptr;  // rows snp_reachable reads (d_pool or the arena)
  const uint32_t* result_perm = nullptr;  // row k of the result is result_pool row result_perm[k] (or k)
  int32_t result_w = 4;                   // bytes per spike count of result_pool's rows

  snp::DevSys dev() const {
    snp::DevSys s;
    s.m = m;
    s.R = R;
    s.K = K;
    s.first_rule = d_first_rule.as<int32_t>();
    s.rule = d_rule.as<int4>();
    s.csr = d_csr.as<int2>();
    s.gain = d_gain.as<int32_t>();
    s.colkey = d_colkey.as<unsigned long long>();
    s.rowkey = d_rowkey.as<unsigned long long>();
    s.eqmask = d_eqmask.as<uint32_t>();
    s.ninfo = d_ninfo.as<snp::NeuronInfo>();
    s.atab = d_atab.as<snp::ApplEntry>();
    s.dmask = d_dmask.as<uint32_t>();
    s.dhx = d_dhx.as<unsigned long long>();
    s.gain_small = gain_small;
    s.rdesc = d_rdesc.as<int4>();
    s.scol = d_scol.as<int32_t>();
    s.rval = d_rval.as<int32_t>();
    s.rterm = d_rterm.as<int32_t>();
    s.term = d_term.as<int2>();
    return s;
  }
  snp::DevTable table() const { return snp::DevTable{d_slots.as<unsigned long long>(), nbuckets - 1}; }
};

namespace snp {
// fp8 tensor-core form: uploads M_Pi^T in e4m3 on first use (the operand of
// tcgen05.mma); hash and repeat buffers for q candidates (snp_api.cu).
int tc5_prepare(snp_system* h, uint64_t q);
}  // namespace snp
