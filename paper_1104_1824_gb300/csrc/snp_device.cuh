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

// Bound on the wait for a reserved slot to be published: this many polls,
// and (when the caller gave one) a time limit.
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Warp-uniform: true once a retry loop has run kSpinLimit polls or, with
// wait_ns > 0, wait_ns nanoseconds since its first poll (lane 0's clock).
__device__ __forceinline__ bool wait_expired(int pass, uint64_t wait_ns, uint64_t& t0) {
  if (pass >= kSpinLimit) return true;
  if (wait_ns == 0) return false;
  uint64_t now = __shfl_sync(0xffffffffu, global_ns(), 0);
  if (pass == 0) {
    t0 = now;
    return false;
  }
  return now - t0 > wait_ns;
}

// How a configuration row lies in global memory: m spike counts of type T
// (int32, or in a packed store uint16 / uint8, which the caller has shown wide
// enough for every count the exploration can reach).  VEC: m % 4 == 0 and the
// row is a whole number of 16-byte pieces (packed rows always are), so it
// moves in pieces of PER16 counts.  Rows in shared memory are int32 in every
// format.
template <typename TT, bool V>
struct RowFmt {
  using T = TT;
  static constexpr bool VEC = V;
  static constexpr int W = (int)sizeof(TT);
  static constexpr int PER16 = 16 / (int)sizeof(TT);
};
using RowI32 = RowFmt<int32_t, false>;
using RowI32V = RowFmt<int32_t, true>;
using RowU16 = RowFmt<uint16_t, true>;
using RowU8 = RowFmt<uint8_t, true>;

// Row j of a row array in format RF that the kernels' argument structs hold
// as int32_t* whatever the format.
template <class RF>
__device__ __forceinline__ typename RF::T* row_at(int32_t* base, uint64_t j, int m) {
  return reinterpret_cast<typename RF::T*>(base) + (size_t)j * m;
}
template <class RF>
__device__ __forceinline__ const typename RF::T* row_at(const int32_t* base, uint64_t j, int m) {
  return reinterpret_cast<const typename RF::T*>(base) + (size_t)j * m;
}

// Four counts (each within the row type's range) as the 4 * W bytes of the
// packed row: one 32-bit word for uint8, two for uint16.
__device__ __forceinline__ uint32_t pack4_u8(int4 v) {
  return __byte_perm(__byte_perm(v.x, v.y, 0x0040), __byte_perm(v.z, v.w, 0x0040), 0x5410);
}
__device__ __forceinline__ uint2 pack4_u16(int4 v) {
  return make_uint2(__byte_perm(v.x, v.y, 0x5410), __byte_perm(v.z, v.w, 0x5410));
}
__device__ __forceinline__ int4 unpack4_u8(uint32_t w) {
  return make_int4((int)(w & 0xFFu), (int)((w >> 8) & 0xFFu), (int)((w >> 16) & 0xFFu), (int)(w >> 24));
}
__device__ __forceinline__ int4 unpack4_u16(uint2 w) {
  return make_int4((int)(w.x & 0xFFFFu), (int)(w.x >> 16), (int)(w.y & 0xFFFFu), (int)(w.y >> 16));
}

// A row's 16-byte piece q unpacked into counts v[0 .. PER16).
template <class RF>
__device__ __forceinline__ void unpack_piece(uint4 x, int32_t* v) {
  if constexpr (RF::W == 1) {
    const int4 a = unpack4_u8(x.x), b = unpack4_u8(x.y), c = unpack4_u8(x.z), d = unpack4_u8(x.w);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    v[8] = c.x, v[9] = c.y, v[10] = c.z, v[11] = c.w, v[12] = d.x, v[13] = d.y, v[14] = d.z, v[15] = d.w;
  } else if constexpr (RF::W == 2) {
    const int4 a = unpack4_u16(make_uint2(x.x, x.y)), b = unpack4_u16(make_uint2(x.z, x.w));
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
  } else {
    v[0] = (int32_t)x.x, v[1] = (int32_t)x.y, v[2] = (int32_t)x.z, v[3] = (int32_t)x.w;
  }
}

// The 16-byte piece holding counts v[0 .. PER16) (v: int32 in shared memory,
// 16-byte aligned).
template <class RF>
__device__ __forceinline__ uint4 pack_piece(const int32_t* v) {
  const int4* v4 = reinterpret_cast<const int4*>(v);
  if constexpr (RF::W == 1) {
    return make_uint4(pack4_u8(v4[0]), pack4_u8(v4[1]), pack4_u8(v4[2]), pack4_u8(v4[3]));
  } else if constexpr (RF::W == 2) {
    const uint2 a = pack4_u16(v4[0]), b = pack4_u16(v4[1]);
    return make_uint4(a.x, a.y, b.x, b.y);
  } else {
    const int4 a = v4[0];
    return make_uint4((uint32_t)a.x, (uint32_t)a.y, (uint32_t)a.z, (uint32_t)a.w);
  }
}

struct NeuronInfo;
struct ApplEntry;

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
  const NeuronInfo* ninfo;    // [m] per-neuron constants: see appl()
  const ApplEntry* atab;      // applicable rules of each neuron by spike count
  // Direct table for spike counts below kDirect, [m][kDirect]: the applicable
  // mask, and x * R[n] + H[first applicable rule] (the neuron's share of the
  // hash of the base child).  gain_small: every column's gain is at most
  // INT32_MAX - kDirect, so counts below kDirect cannot overflow a child.
  const uint32_t* dmask;
  const unsigned long long* dhx;
  int32_t gain_small;
  // Rows of M_Pi on their neuron's support: the columns any rule of the neuron
  // touches (its own and its synapse targets).  Rule r: {offset of the support
  // in scol, its length, offset of r's values in rval, neuron}.
  const int4* rdesc;
  const int32_t* scol;
  const int32_t* rval;
  // Rule r's regular expression: the union of a^term[t].x (a^term[t].y)* over
  // t in [rterm[r], rterm[r + 1]) (one term per rule for the paper's rules).
  const int32_t* rterm;
  const int2* term;
};
constexpr int kDirect = 64;

// Per-neuron constants read together by the applicability scan.
struct __align__(16) NeuronInfo {
  int32_t off;                // first entry of the neuron in atab, or -1 (evaluate the rules)
  uint32_t tl;                // T | L << 16 (see appl)
  unsigned long long magic;   // ceil(2^shift / L): floor(v / L) = (v * magic) >> shift for v < 2^31
  int32_t gain;               // largest increase of the neuron's column in one step
  uint32_t shift;             // 32 + ceil(log2 L)
  unsigned long long colkey;  // R[n]
};

// Applicable rules of a neuron for one spike count.
struct __align__(16) ApplEntry {
  uint32_t mask;              // bit k: rule first_rule[n] + k applies
  uint32_t keep;              // mask without the rules that repeat an earlier applicable rule's row
  unsigned long long hfirst;  // H[first applicable rule], 0 if none
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
  unsigned int psi_saturated;  // Psi summed over the first parents already reached 2^64 - 1
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

// a^x in L(a^i (a^j)*) (Section 2.1; j = 0: exactly a^i).
__host__ __device__ __forceinline__ bool term_matches(int32_t x, int32_t i, int32_t j) {
  if (x < i) return false;
  if (j == 0) return x == i;
  if (j == 1) return true;
  return ((x - i) % j) == 0;
}

// Rule r applies to x spikes: x >= c (rule.z) and a^x is in the union of its
// terms (Section 2.1, rule (b-1)).
__host__ __device__ __forceinline__ bool rule_applies(int32_t x, int4 rule, const int32_t* rterm, const int2* term,
                                                      int r) {
  if (x < rule.z) return false;
  for (int t = rterm[r]; t < rterm[r + 1]; ++t)
    if (term_matches(x, term[t].x, term[t].y)) return true;
  return false;
}

// Applicable rules of neuron n holding x spikes, from the rules themselves
// (out of line, it is the rare path: it takes the arrays it reads rather than
// the whole system).
static __device__ __noinline__ ApplEntry appl_rules(const int32_t* first_rule, const int4* rule,
                                                   const int32_t* rterm, const int2* term, const uint32_t* eqmask,
                                                   const unsigned long long* rowkey, int n, int32_t x) {
  const int r0 = __ldg(first_rule + n), r1 = __ldg(first_rule + n + 1);
  uint32_t mask = 0;
  for (int r = r0; r < r1; ++r)
    if (rule_applies(x, __ldg(rule + r), rterm, term, r)) mask |= 1u << (r - r0);
  uint32_t keep = mask;
  for (uint32_t b = mask; b; b &= b - 1) {
    const int k = __ffs(b) - 1;
    if (__ldg(eqmask + r0 + k) & mask) keep &= ~(1u << k);
  }
  ApplEntry e;
  e.mask = mask;
  e.keep = keep;
  e.hfirst = mask ? __ldg(rowkey + r0 + __ffs(mask) - 1) : 0ull;
  return e;
}

// appl_rules(s, n, x) by table.  Above T = 1 + the largest i or c of the
// neuron's rules every threshold holds and a^i alone never matches, so the
// entries repeat with period L = lcm of the rules' j >= 1: the table holds
// x = 0 .. T + L - 1 and larger x fold onto T + (x - T) mod L, the quotient
// by multiply and shift (Granlund and Montgomery, PLDI 1994; exact here since
// x - T < 2^31).  Neurons whose T + L is too large for a table evaluate
// their rules.
__device__ __forceinline__ ApplEntry appl_entry(const DevSys& s, const NeuronInfo& ni, int n, int32_t x) {
  if (ni.off >= 0 && x >= 0) {
    const uint32_t T = ni.tl & 0xFFFFu, L = ni.tl >> 16;
    uint32_t k = (uint32_t)x;
    if (k >= T + L) {
      const uint32_t v = k - T;
      const uint32_t q = (uint32_t)(((unsigned long long)v * ni.magic) >> ni.shift);
      k = T + v - q * L;
    }
    const uint4 e = __ldg(reinterpret_cast<const uint4*>(s.atab + ni.off + k));
    ApplEntry r;
    r.mask = e.x;
    r.keep = e.y;
    r.hfirst = ((unsigned long long)e.w << 32) | e.z;
    return r;
  }
  return appl_rules(s.first_rule, s.rule, s.rterm, s.term, s.eqmask, s.rowkey, n, x);
}

__device__ __forceinline__ NeuronInfo neuron_info(const DevSys& s, int n) {
  const int4* p = reinterpret_cast<const int4*>(s.ninfo + n);
  const int4 a = __ldg(p), b = __ldg(p + 1);
  NeuronInfo ni;
  ni.off = a.x;
  ni.tl = (uint32_t)a.y;
  ni.magic = ((unsigned long long)(uint32_t)a.w << 32) | (uint32_t)a.z;
  ni.gain = b.x;
  ni.shift = (uint32_t)b.y;
  ni.colkey = ((unsigned long long)(uint32_t)b.w << 32) | (uint32_t)b.z;
  return ni;
}

// Bits 0-31: applicable rules of neuron n with x spikes; bits 32-63: the same
// without rules that repeat an earlier applicable rule's row.
__device__ __forceinline__ uint64_t appl(const DevSys& s, int n, int32_t x) {
  const ApplEntry e = appl_entry(s, neuron_info(s, n), n, x);
  return (uint64_t)e.mask | ((uint64_t)e.keep << 32);
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

// Table key of the configuration in buf (warp-cooperative; counts of type T).
template <typename T>
__device__ __forceinline__ uint64_t fingerprint(const DevSys& s, const T* buf, int lane) {
  uint64_t h = 0;
  for (int n = lane; n < s.m; n += 32) h += col_hash(s, n, buf[n]);
  return mix64(warp_sum_u64(h));
}

// dst[0, m) = src[0, m), read through L2, the loads issued in groups of 8 so
// that a group is in flight together (16-byte words when m % 4 == 0; both
// rows then start 16-byte aligned).
__device__ __forceinline__ void copy_row_cg(const int32_t* src, int32_t* dst, int m) {
  if ((m & 3) == 0) {
    const int4* s4 = reinterpret_cast<const int4*>(src);
    int4* d4 = reinterpret_cast<int4*>(dst);
    const int n4 = m >> 2;
    for (int j0 = 0; j0 < n4; j0 += 8) {
      int4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < n4) v[u] = __ldcg(s4 + j0 + u);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < n4) d4[j0 + u] = v[u];
    }
    return;
  }
  for (int j0 = 0; j0 < m; j0 += 8) {
    int32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (j0 + u < m) v[u] = __ldcg(src + j0 + u);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (j0 + u < m) dst[j0 + u] = v[u];
  }
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
