// Device-side building blocks of the BFS over SNP-system configurations:
// rule applicability (Algorithm 2, II-1), mixed-radix decoding of a spiking
// vector (Eq. psi; Algorithm 2, II-2/II-3), the sparse transition
// C' = C + S . M_Pi (Eq. next-config), the column-decomposable fingerprint and
// the hash-table probe used for deduplication (Algorithm 1, step IV).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace snp {

constexpr uint64_t kSat = ~0ull;           // "at least 2^64 - 1"
constexpr unsigned long long kEmpty = ~0ull;
constexpr uint32_t kRowReserved = 0xFFFFFFFFu;
constexpr uint32_t kRowTomb = 0xFFFFFFFEu;
constexpr uint32_t kPending = 0x80000000u;  // row field names a staging row
constexpr int kBucket = 8;                  // slots per bucket (64 bytes)

// Error bits raised on the device.
constexpr uint32_t kErrTableFull = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrStaging = 4u;
constexpr uint32_t kErrOverflow = 8u;
constexpr uint32_t kErrInternal = 16u;

// Bound on the wait for a reserved slot to be published.
constexpr int kSpinLimit = 1 << 22;

// The system as the kernels see it.
struct DevSys {
  int32_t m, R, K;            // K = neurons owned by one lane = ceil(m / 32)
  const int32_t* first_rule;  // [m + 1] rules of neuron n: [first_rule[n], first_rule[n+1])
  const int4* rule;           // [R + 1] {i, j, c, csr begin}; rule[R].w = nnz
  const int2* csr;            // [nnz] {column, value}: nonzeros of M_Pi, row by row
  const int32_t* gain;        // [m] largest increase of column j in one step
  const unsigned long long* colkey;  // [m] random odd multiplier R[j] of column j
  const unsigned long long* rowkey;  // [R] H[r] = sum over row r of M_Pi of M[r][j] * R[j] (mod 2^64)
  const uint32_t* eqmask;     // [R] positions of earlier rules of the same neuron with the same row of M_Pi
  const int2* amet;           // [m] {offset into atab or -1, T | L << 16}: see appl()
  const unsigned long long* atab;  // applicable-rule masks of each neuron by spike count
};

// Rule r, chosen for a neuron whose applicable rules are `mask`, gives the
// same child as an earlier applicable rule with the same row of M_Pi: every
// candidate choosing it repeats an earlier candidate of the same parent.
__device__ __forceinline__ bool redundant_choice(const DevSys& s, uint32_t mask, int r) {
  return (mask & __ldg(s.eqmask + r)) != 0u;
}

// Per-parent summary written with Psi (step a) for batches that cross
// parents: the hash of the parent's base child (every neuron that can fire
// uses its first applicable rule) and its neurons with two or more
// applicable rules, in neuron order, as (neuron << 16) | mask.  nnt =
// kRecFull when there are more than kRecNt of them or one does not fit 16
// bits: such a parent is decoded from its row.
constexpr int kRecNt = 9;
constexpr uint32_t kRecFull = 0xFFFFFFFFu;
struct __align__(16) ParentRec {
  unsigned long long hbase;
  uint32_t nnt;
  uint32_t nt[kRecNt];
};

struct DevTable {
  unsigned long long* slots;  // [nbuckets * kBucket]: (fp32 << 32) | row
  uint64_t bmask;             // nbuckets - 1
};

// Per-chunk device counters (read back by the host after each chunk).
struct ChunkState {
  unsigned int n_alloc;       // staging rows handed out
  unsigned int error;         // kErr* bits
  unsigned int total_first;   // distinct new keys in the chunk
  unsigned int capped;        // the cap was reached inside the chunk
  unsigned int last_lid;      // chunk-local index of the last accepted first occurrence
  unsigned int pad;
  unsigned long long p_first;  // first and last frontier row the chunk's candidates come from
  unsigned long long p_last;
};

__device__ __forceinline__ uint64_t sat_mul(uint64_t a, uint64_t b) {
  if (a == 0 || b == 0) return 0;
  return __umul64hi(a, b) ? kSat : a * b;
}

__device__ __forceinline__ uint64_t sat_add(uint64_t a, uint64_t b) {
  uint64_t s = a + b;
  return s < a ? kSat : s;
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Linear hash of a configuration: h(C) = sum_j C[j] * R[j] (mod 2^64).  It is
// additive over columns (any partition of the columns can compute it) and over
// Eq. next-config: h(C + S . M_Pi) = h(C) + sum of H[r] over the rules S uses.
// The table key is mix64(h); equality is always decided by a full compare.
__device__ __forceinline__ uint64_t col_hash(const DevSys& s, int j, int32_t v) {
  return (uint64_t)(uint32_t)v * __ldg(s.colkey + j);
}

// a^x in L(a^i (a^j)*) and x >= c (Section 2.1, rule (b-1)).
__host__ __device__ __forceinline__ bool rule_applies(int32_t x, int4 rp) {
  if (x < rp.x || x < rp.z) return false;
  if (rp.y == 0) return x == rp.x;
  if (rp.y == 1) return true;
  return ((x - rp.x) % rp.y) == 0;
}

// Applicable rules of neuron n holding x spikes, from the rules themselves:
// bits 0-31 the mask (bit k = rule first_rule[n] + k), bits 32-63 the same
// mask without the rules that repeat an earlier applicable rule's row.
__device__ __forceinline__ uint64_t appl_rules(const DevSys& s, int n, int32_t x) {
  const int r0 = __ldg(s.first_rule + n), r1 = __ldg(s.first_rule + n + 1);
  uint32_t mask = 0;
  for (int r = r0; r < r1; ++r)
    if (rule_applies(x, __ldg(s.rule + r))) mask |= 1u << (r - r0);
  uint32_t keep = mask;
  for (uint32_t b = mask; b; b &= b - 1) {
    const int k = __ffs(b) - 1;
    if (__ldg(s.eqmask + r0 + k) & mask) keep &= ~(1u << k);
  }
  return (uint64_t)mask | ((uint64_t)keep << 32);
}

// appl_rules(s, n, x) by table.  Above T = 1 + the largest i or c of the
// neuron's rules every threshold holds and a^i alone never matches, so the
// masks repeat with period L = lcm of the rules' j >= 1: the table holds
// x = 0 .. T + L - 1 and larger x fold onto T + (x - T) mod L.  Neurons whose
// T + L is too large for a table (offset -1) evaluate their rules.
__device__ __forceinline__ uint64_t appl(const DevSys& s, int n, int32_t x) {
  const int2 mt = __ldg(s.amet + n);
  if (mt.x >= 0 && x >= 0) {
    const int T = mt.y & 0xFFFF, L = (int)((uint32_t)mt.y >> 16);
    int k = x;
    if (x >= T + L) k = T + ((L & (L - 1)) ? (x - T) % L : ((x - T) & (L - 1)));
    return __ldg(s.atab + mt.x + k);
  }
  return appl_rules(s, n, x);
}

// Position of the d-th set bit (0-based) of mask.
__device__ __forceinline__ int nth_set_bit(uint32_t mask, int d) {
  for (int k = 0; k < d; ++k) mask &= mask - 1;
  return __ffs(mask) - 1;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Largest p in [0, P) with off[p] <= g (off non-decreasing, off[0] = 0 <= g).
// Loads through L2: off may have been written earlier in the same kernel.
__device__ __forceinline__ int64_t warp_find_parent(const uint64_t* off, int64_t P, uint64_t g, int lane) {
  int64_t lo = 0, hi = P;
  while (hi - lo > 1) {
    int64_t n = hi - lo;
    int64_t step = (n + 31) / 32;
    int64_t idx = lo + (int64_t)lane * step;
    bool ok = idx < hi && __ldcg(off + idx) <= g;
    uint32_t b = __ballot_sync(0xffffffffu, ok);
    int L = 31 - __clz(b);
    lo = lo + (int64_t)L * step;
    hi = min(lo + step, hi);
  }
  return lo;
}

// Per-warp view of one parent configuration: its row in shared memory, the
// applicable-rule mask of every neuron and, per lane, the product of the
// choice counts of all neurons after the lane's own (mixed-radix place value).
struct WarpParent {
  int32_t* par;    // [m] spikes
  uint32_t* msk;   // [m] applicable rules of neuron n, bit k = rule first_rule[n] + k
  int32_t* buf;    // [m] child under construction
  uint64_t after;  // product of choice counts of neurons owned by later lanes (saturating)
  uint64_t psi;    // Psi of the parent (saturating)
};

// Step (a) for one parent: load the row, mark applicable rules, form the
// per-lane place values (neuron 0 most significant).
__device__ __forceinline__ void load_parent(const DevSys& s, const int32_t* __restrict__ row, WarpParent& w,
                                            int lane) {
  __syncwarp();
  for (int n = lane; n < s.m; n += 32) w.par[n] = row[n];
  __syncwarp();
  uint64_t prod = 1;
  const int n0 = lane * s.K;
  const int n1 = min(n0 + s.K, s.m);
  for (int n = n0; n < n1; ++n) {
    const uint32_t mask = (uint32_t)appl(s, n, w.par[n]);
    w.msk[n] = mask;
    prod = sat_mul(prod, mask ? (uint64_t)__popc(mask) : 1ull);
  }
  // inclusive suffix product over lanes
  uint64_t v = prod;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v = sat_mul(v, u);
  }
  w.psi = __shfl_sync(0xffffffffu, v, 0);
  uint64_t a = __shfl_down_sync(0xffffffffu, v, 1);
  w.after = (lane == 31) ? 1ull : a;
  __syncwarp();
}

// Steps (b) and (c) for candidate t of the loaded parent: decode t in the
// mixed radix of the choice counts (last neuron least significant), then
// C' = C + sum of the chosen rules' rows of M_Pi, built in w.buf.
__device__ __forceinline__ void build_child(const DevSys& s, WarpParent& w, uint64_t t, int lane) {
  for (int n = lane; n < s.m; n += 32) w.buf[n] = w.par[n];
  __syncwarp();
  const int n0 = lane * s.K;
  const int n1 = min(n0 + s.K, s.m);
  if (n0 < n1) {
    uint64_t q = (w.after > t) ? 0ull : t / w.after;
    for (int n = n1 - 1; n >= n0; --n) {
      const uint32_t mask = w.msk[n];
      if (!mask) continue;  // the neuron cannot fire: one choice
      const uint32_t radix = __popc(mask);
      uint32_t d;
      if ((q >> 32) == 0) {
        uint32_t q32 = (uint32_t)q;
        d = q32 % radix;
        q = q32 / radix;
      } else {
        d = (uint32_t)(q % radix);
        q /= radix;
      }
      const int r = __ldg(s.first_rule + n) + nth_set_bit(mask, (int)d);
      const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
      for (int e = e0; e < e1; ++e) {
        const int2 cv = __ldg(s.csr + e);
        atomicAdd(&w.buf[cv.x], cv.y);
      }
    }
  }
  __syncwarp();
}

// Table key of the configuration in buf (warp-cooperative).
__device__ __forceinline__ uint64_t fingerprint(const DevSys& s, const int32_t* buf, int lane) {
  uint64_t h = 0;
  for (int n = lane; n < s.m; n += 32) h += col_hash(s, n, buf[n]);
  return mix64(warp_sum_u64(h));
}

__device__ __forceinline__ uint32_t fp32_of(uint64_t h) {
  uint32_t f = (uint32_t)(h >> 32);
  return f == 0xFFFFFFFFu ? 0xFFFFFFFEu : f;  // keeps (fp, reserved) distinct from an empty slot
}

__device__ __forceinline__ bool rows_equal(const int32_t* buf, const int32_t* other, int m, int lane) {
  bool ok = true;
  for (int n = lane; n < m; n += 32) ok &= (__ldcg(other + n) == buf[n]);
  return __all_sync(0xffffffffu, ok);
}

}  // namespace snp
