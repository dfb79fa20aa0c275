// The expand kernel: steps (b), (c) and (d) for one chunk of candidates.
//
// Candidates are spiking-vector indices in the mixed radix of the per-neuron
// choice counts (Eq. psi; last neuron least significant).  A warp walks a run
// of consecutive candidates in one of two ways:
//
// * block mode, while the current parent has 32 or more candidates left.  The
//   least significant neurons with two or more applicable rules, as many as
//   keep the product RL of their choice counts <= B, form a block: candidates
//   b * RL .. b * RL + RL - 1 share every other digit.  Lane k owns candidate
//   k of each block: once per parent it builds its row C' = C + S . M_Pi
//   (Eq. next-config) from the block base plus its own low digits, with the
//   linear hash of that row.  Moving to the next block changes the high
//   digits like an odometer (usually one neuron): lane 0 lists the swapped
//   rules and every lane swaps the same rows of M_Pi in its own row and their
//   H[r] in its hash.
// * crossing batches, once the parent has fewer than 32 candidates left: one
//   candidate per lane, possibly of different parents, decoded from the
//   parent's record (its multi-choice neurons and base hash) written with Psi.
//   Surviving candidates are queued in the tile and their rows built all at
//   once before they are resolved.
//
// Rows of more than kWideM neurons (k_expand_wide) are too long for a row per
// lane: lanes keep only their candidates' hashes and probe for them, and the
// whole warp builds a row in one scratch row when it has to be compared with
// a stored row or written by the lane that claimed its key; the odometer's
// swaps go into the block base itself, and the low neurons' swaps come from a
// per-parent table in shared memory.
//
// Resolving a row (step d): probe the hash table, compare full keys, and
// either find the key (seen before, or claimed earlier in this chunk: then
// lower that key's first-occurrence index) or claim an empty slot, write the
// row (to the next store row; the batch engine and the allocation-free path
// use staging row lid) and publish the slot.
#include "snp_kernels.cuh"
#include "snp_tcgen05.cuh"

namespace snp {

namespace {

struct ExpandSmem {
  int32_t* tile;              // [B][ts] block mode: row k = lane k's candidate; crossing batches: queued rows
  unsigned long long* keys;   // [B] crossing batches: table keys of the queued rows
  long long* dpc;             // [B] parent of a queued row still to be built, else -1
  unsigned long long* dt;     // [B] its index among the parent's candidates
  uint32_t* lids;             // [B] chunk-local indices of the queued rows
  int32_t* par;               // [m4] parent (not kept in the wide mode: its row is read from the store)
  int32_t* buf;               // [m4] block base child
  uint32_t* msk;              // [m4] applicable-rule masks
  uint16_t* ntl;              // [m4] neurons with two or more applicable rules, least significant first
  int2* chg;                  // [m4] (old rule, new rule) pairs of the last block step
  int* hdr;                   // [8] kNnt, kNlow, kRL, kNchg, kNred; hbase at hdr + 6
  uint8_t* dig;               // [m4] digits of the block base
  int32_t* low;               // wide mode: per low neuron (start, length), then the table of its
                              // support columns and M[rule d] - M[rule 0] on them, d = 1 .. radix - 1
};
enum { kNnt = 0, kNlow = 1, kRL = 2, kNchg = 3, kNred = 4, kLowOk = 5 };
__device__ __forceinline__ unsigned long long& hbase_of(const ExpandSmem& w) {
  return *reinterpret_cast<unsigned long long*>(w.hdr + 6);
}

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

__host__ __device__ inline size_t expand_keys_bytes(int B) { return ((size_t)B * 28 + 15) & ~size_t(15); }

__host__ __device__ inline size_t expand_warp_bytes(int m, int B, int ts) {
  const int m4 = round4(m);
  size_t b = (size_t)B * ts * 4 + expand_keys_bytes(B) + (size_t)m4 * 14 + (size_t)m4 * 8 + 32 + (size_t)m4;
  return (b + 15) & ~size_t(15);
}

// Wide rows (more than kWideM neurons): a warp keeps one scratch row instead
// of one row per lane, and queues up to 32 crossing-batch candidates.
constexpr int kWideB = 32;
constexpr int kWide = 2;        // KIND of the wide mode
constexpr int kWideWarps = 11;  // warps per CTA (one CTA per SM: 11 x 20.6 KB of shared memory at m = 1024)
// words of the low neurons' header: (start, length) per low neuron, then the
// packed low digits of the block's candidates (5 bits per neuron); then the table
constexpr int kLowDig = 16, kLowHdr = 48, kLowTab = 1024;
__host__ __device__ inline size_t expand_wide_bytes(int m) {
  const int m4 = round4(m);
  size_t b = (size_t)m4 * 4 + expand_keys_bytes(kWideB) + (size_t)m4 * 10 + 32 + (size_t)(kLowHdr + kLowTab) * 4 +
             (size_t)m4;
  return (b + 15) & ~size_t(15);
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int rule_of(const DevSys& s, const ExpandSmem& w, int n, int d) {
  return __ldg(s.first_rule + n) + nth_set_bit(w.msk[n], d);
}

// row += sign * (row r of M_Pi); the row is private to the calling lane
__device__ __forceinline__ void add_row_private(const DevSys& s, int32_t* row, int r, int sign) {
  const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
  for (int e = e0; e < e1; ++e) {
    const int2 cv = __ldg(s.csr + e);
    row[cv.x] += sign * cv.y;
  }
}

// row += M[rn] - M[ro] for two rules of one neuron (the row is private to
// the calling lane): one pass over the neuron's support.
__device__ __forceinline__ void swap_rule_private(const DevSys& s, int32_t* row, int ro, int rn) {
  const int4 dn = __ldg(s.rdesc + rn);
  const int32_t* vn = s.rval + dn.z;
  const int32_t* vo = s.rval + __ldg(&s.rdesc[ro].z);
  const int32_t* col = s.scol + dn.x;
  for (int i = 0; i < dn.y; ++i) row[__ldg(col + i)] += __ldg(vn + i) - __ldg(vo + i);
}

// row += M[r] (the row is private to the calling lane).
__device__ __forceinline__ void add_rule_private(const DevSys& s, int32_t* row, int r) {
  const int4 dr = __ldg(s.rdesc + r);
  const int32_t* v = s.rval + dr.z;
  const int32_t* col = s.scol + dr.x;
  for (int i = 0; i < dr.y; ++i) row[__ldg(col + i)] += __ldg(v + i);
}

// The batch kernel runs at its register limit: it keeps the CSR walk, which
// needs fewer live values.
template <int KIND>
__device__ __forceinline__ void swap_rule(const DevSys& s, int32_t* row, int ro, int rn) {
  if constexpr (KIND == 0) {
    swap_rule_private(s, row, ro, rn);
  } else {
    add_row_private(s, row, ro, -1);
    add_row_private(s, row, rn, 1);
  }
}

template <int KIND>
__device__ __forceinline__ void add_rule(const DevSys& s, int32_t* row, int r) {
  if constexpr (KIND == 0)
    add_rule_private(s, row, r);
  else
    add_row_private(s, row, r, 1);
}

__device__ __forceinline__ void add_row_shared(const DevSys& s, int32_t* row, int r, int sign) {
  const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
  for (int e = e0; e < e1; ++e) {
    const int2 cv = __ldg(s.csr + e);
    atomicAdd(&row[cv.x], sign * cv.y);
  }
}

// Step (a) for the parent row: masks, the multi-choice neurons (least
// significant first), the block (the least significant of them whose choice
// counts multiply to RL <= B) and, per lane, the mixed-radix place value of
// the neurons owned by later lanes (neuron 0 most significant).
template <typename T>
__device__ __forceinline__ uint64_t parent_state(const DevSys& s, const T* __restrict__ row, ExpandSmem& w, int B,
                                                 int lane) {
  __syncwarp();
  if (w.par)
    for (int n = lane; n < s.m; n += 32) w.par[n] = row[n];
  __syncwarp();
  uint64_t prod = 1;
  const int n0 = lane * s.K, n1 = min(n0 + s.K, s.m);
  for (int n = n0; n < n1; ++n) {
    const uint32_t mask = (uint32_t)appl(s, n, w.par ? w.par[n] : (int32_t)row[n]);
    w.msk[n] = mask;
    prod = sat_mul(prod, mask ? (uint64_t)__popc(mask) : 1ull);
  }
  uint64_t v = prod;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v = sat_mul(v, u);
  }
  const uint64_t a = __shfl_down_sync(0xffffffffu, v, 1);
  __syncwarp();
  int count = 0;
  for (int top = s.m - 1; top >= 0; top -= 32) {
    const int n = top - lane;
    const bool nt = n >= 0 && __popc(w.msk[n]) > 1;
    const uint32_t b = __ballot_sync(0xffffffffu, nt);
    if (nt) w.ntl[count + __popc(b & ((1u << lane) - 1u))] = (uint16_t)n;
    count += __popc(b);
  }
  __syncwarp();
  if (lane == 0) {
    int nl = 0, rl = 1;
    while (nl < count && rl * __popc(w.msk[w.ntl[nl]]) <= B) rl *= __popc(w.msk[w.ntl[nl++]]);
    w.hdr[kNnt] = count;
    w.hdr[kNlow] = nl;
    w.hdr[kRL] = rl;
  }
  __syncwarp();
  return lane == 31 ? 1ull : a;
}

// The block base becomes candidate t of the loaded parent: digits, child in
// buf, hash, and the count of neurons whose digit picks a rule that repeats an
// earlier applicable rule's row.
// (The wide mode passes the parent's row in the store as prow, there being
// no copy of it in shared memory.)
template <bool WIDE = false, typename T = int32_t>
__device__ __forceinline__ void decode_full(const DevSys& s, ExpandSmem& w, uint64_t t, uint64_t after, int lane,
                                            const T* prow = nullptr) {
  uint64_t hp = 0;
  for (int n = lane; n < s.m; n += 32) {
    const int32_t x = WIDE ? (int32_t)prow[n] : w.par[n];
    w.buf[n] = x;
    hp += col_hash(s, n, x);
  }
  __syncwarp();
  const int n0 = lane * s.K, n1 = min(n0 + s.K, s.m);
  uint64_t q = (after > t) ? 0ull : t / after;
  int red = 0;
  for (int n = n1 - 1; n >= n0; --n) {
    const uint32_t mask = w.msk[n];
    if (!mask) {
      w.dig[n] = 0;
      continue;
    }
    const uint32_t radix = __popc(mask);
    uint32_t d;
    if ((q >> 32) == 0) {
      const uint32_t q32 = (uint32_t)q;
      d = q32 % radix;
      q = q32 / radix;
    } else {
      d = (uint32_t)(q % radix);
      q /= radix;
    }
    w.dig[n] = (uint8_t)d;
    const int r = __ldg(s.first_rule + n) + nth_set_bit(mask, (int)d);
    if (WIDE) {  // long rows of M_Pi: eight loads in flight before their adds
      const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
      for (int e = e0; e < e1; e += 8) {
        int2 cv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) cv[u] = e + u < e1 ? __ldg(s.csr + e + u) : make_int2(-1, 0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (cv[u].x >= 0) atomicAdd(&w.buf[cv[u].x], cv[u].y);
      }
    } else {
      add_row_shared(s, w.buf, r, 1);
    }
    hp += __ldg(s.rowkey + r);
    red += redundant_choice(s, mask, r) ? 1 : 0;
  }
  hp = warp_sum_u64(hp);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) red += __shfl_xor_sync(0xffffffffu, red, o);
  __syncwarp();
  if (lane == 0) {
    hbase_of(w) = hp;
    w.hdr[kNred] = red;
  }
  __syncwarp();
}

template <bool VEC>
__device__ __forceinline__ void copy_row(const int32_t* src, int32_t* dst, int m) {
  if (VEC) {
    const int4* a = reinterpret_cast<const int4*>(src);
    int4* b = reinterpret_cast<int4*>(dst);
    for (int j = 0; j < (m >> 2); ++j) b[j] = a[j];
    return;
  }
  for (int j = 0; j < m; ++j) dst[j] = src[j];
}

// Full-key compare; branch-free in groups of 8 loads so that the loads of a
// group are in flight together.
template <class RF>
__device__ __forceinline__ bool row_equal_lane(const int32_t* row, const typename RF::T* other, int m) {
  if constexpr (RF::W < 4) {  // packed: the candidate is packed the same way, piece by piece
    const uint4* b = reinterpret_cast<const uint4*>(other);
    const int n16 = m / RF::PER16;
    for (int j0 = 0; j0 < n16; j0 += 8) {
      uint4 y[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < n16) y[u] = __ldcg(b + j0 + u);
      uint32_t diff = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < n16) {
          const uint4 x = pack_piece<RF>(row + (j0 + u) * RF::PER16);
          diff |= (x.x ^ y[u].x) | (x.y ^ y[u].y) | (x.z ^ y[u].z) | (x.w ^ y[u].w);
        }
      if (diff) return false;
    }
    return true;
  } else if constexpr (RF::VEC) {
    const int4* a = reinterpret_cast<const int4*>(row);
    const int4* b = reinterpret_cast<const int4*>(other);
    const int n4 = m >> 2;
    for (int j0 = 0; j0 < n4; j0 += 8) {
      int4 y[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < n4) y[u] = __ldcg(b + j0 + u);
      int diff = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < n4) {
          const int4 x = a[j0 + u];
          diff |= (x.x ^ y[u].x) | (x.y ^ y[u].y) | (x.z ^ y[u].z) | (x.w ^ y[u].w);
        }
      if (diff) return false;
    }
    return true;
  } else {
    for (int j0 = 0; j0 < m; j0 += 8) {
      int y[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < m) y[u] = __ldcg(other + j0 + u);
      int diff = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < m) diff |= row[j0 + u] ^ y[u];
      if (diff) return false;
    }
    return true;
  }
}

template <class RF>
__device__ __forceinline__ void stage_row_lane(const int32_t* row, typename RF::T* dst, int m) {
  if constexpr (RF::W < 4) {
    uint4* b = reinterpret_cast<uint4*>(dst);
    for (int j = 0; j < m / RF::PER16; ++j) __stcg(b + j, pack_piece<RF>(row + j * RF::PER16));
  } else if constexpr (RF::VEC) {
    const int4* a = reinterpret_cast<const int4*>(row);
    int4* b = reinterpret_cast<int4*>(dst);
    for (int j = 0; j < (m >> 2); ++j) __stcg(b + j, a[j]);
  } else {
    for (int j = 0; j < m; ++j) __stcg(dst + j, row[j]);
  }
}

// Step (d) for one candidate, by one lane, without waiting on any other lane:
// returns false when the key may sit in a slot that another lane or warp has
// reserved but not yet published; the caller then tries again in a later pass.
constexpr int kRetry = 0, kDone = 1, kOwner = 2;

// Frontier row p of the chunk (through the store's row map when there is one).
template <class RF>
__device__ __forceinline__ const typename RF::T* parent_row(const ClaimArgs& a, int64_t p) {
  return row_at<RF>(a.parents, a.pperm ? __ldg(a.pperm + p) : (uint64_t)p, a.sys.m);
}

template <class RF>
__device__ __forceinline__ int resolve_lane(const ClaimArgs& a, const int32_t* row, uint64_t key, uint32_t lid,
                                            unsigned long long*& owned) {
  // A bucket fills as a prefix (a slot is claimed only when every earlier
  // slot was seen taken, and slots never become empty again), so the slots
  // holding our fingerprint all precede the first empty one.  Each bucket is
  // classified branch-free; the compare and the claim then run once per lane,
  // which keeps lanes that hit different slots together.  Returns kOwner with
  // the reserved slot in `owned`; the caller does the owner's work.
  const int m = a.sys.m;
  const uint32_t fp = fp32_of(key);
  const unsigned long long mine = ((unsigned long long)fp << 32) | kRowReserved;
  uint64_t bucket = key & a.table.bmask;
  owned = nullptr;
  for (uint64_t probes = 0; probes <= a.table.bmask && !owned;) {
    unsigned long long* bs = a.table.slots + bucket * kBucket;
    const ulonglong2* b2 = reinterpret_cast<const ulonglong2*>(bs);
    uint32_t match = 0, empty = 0;
#pragma unroll
    for (int q = 0; q < kBucket / 2; ++q) {
      const ulonglong2 x = __ldcg(b2 + q);
      empty |= (x.x == kEmpty ? 1u : 0u) << (2 * q);
      empty |= (x.y == kEmpty ? 1u : 0u) << (2 * q + 1);
      match |= ((uint32_t)(x.x >> 32) == fp && (uint32_t)x.x != kRowTomb && x.x != kEmpty ? 1u : 0u) << (2 * q);
      match |= ((uint32_t)(x.y >> 32) == fp && (uint32_t)x.y != kRowTomb && x.y != kEmpty ? 1u : 0u) << (2 * q + 1);
    }
    for (; match; match &= match - 1) {
      const int j = __ffs(match) - 1;
      const unsigned long long x = __ldcg(bs + j);
      const uint32_t rf = (uint32_t)x;
      if (rf == kRowReserved) return kRetry;  // published soon: try again later
      const typename RF::T* other;
      if (rf & kPending) {
        (void)ld_acquire(bs + j);  // orders the reads of the owner's row and records after the publish
        const uint32_t o = rf & ~kPending;
        other = a.store_ctr ? row_at<RF>(a.pool, __ldcg(a.sidx_of + o), m) : row_at<RF>(a.staging, o, m);
      } else {
        other = row_at<RF>(a.pool, rf, m);
      }
      if (row_equal_lane<RF>(row, other, m)) {
        if (rf & kPending) atomicMin(a.gmin + (rf & ~kPending), lid);
        return kDone;
      }
    }
    if (empty) {
      const int j = __ffs(empty) - 1;
      if (atomicCAS(bs + j, kEmpty, mine) == kEmpty) owned = bs + j;
      continue;  // owner, or look at this bucket again
    }
    ++probes;
    bucket = (bucket + 1) & a.table.bmask;
  }
  if (!owned) {
    atomicOr(&a.st->error, kErrTableFull);
    return kDone;
  }
  return kOwner;
}

// The owner's work: its row to staging row lid, or in store mode to store
// row sidx (recorded in sidx_of), the claim records, then the publish.
template <class RF>
__device__ __forceinline__ void finish_owner(const ClaimArgs& a, const int32_t* row, uint64_t key, uint32_t lid,
                                             unsigned long long* owned, uint64_t sidx) {
  const int m = a.sys.m;
  if (a.store_ctr) {
    if (sidx >= a.store_cap) {  // the host sizes the store for every claim of the chunk
      atomicOr(&a.st->error, kErrStaging);
      return;
    }
    stage_row_lane<RF>(row, row_at<RF>(a.pool, sidx, m), m);
    a.sidx_of[lid] = (uint32_t)sidx;
  } else {
    stage_row_lane<RF>(row, row_at<RF>(a.staging, lid, m), m);
  }
  a.gmin[lid] = lid;
  a.slot_of[lid] = (uint32_t)(owned - a.table.slots);
  atomicOr(a.ownbits + (lid >> 5), 1u << (lid & 31));
  st_release(owned, ((unsigned long long)fp32_of(key) << 32) | (kPending | lid));
}

// The owner's work when its row is already in the store (row sidx, written
// there by the fp8 tensor-core form): the claim records, then the publish.
__device__ __forceinline__ void finish_owner_inplace(const ClaimArgs& a, uint64_t key, uint32_t lid,
                                                     unsigned long long* owned, uint64_t sidx) {
  if (sidx >= a.store_cap) {
    atomicOr(&a.st->error, kErrStaging);
    return;
  }
  a.sidx_of[lid] = (uint32_t)sidx;
  a.gmin[lid] = lid;
  a.slot_of[lid] = (uint32_t)(owned - a.table.slots);
  atomicOr(a.ownbits + (lid >> 5), 1u << (lid & 31));
  st_release(owned, ((unsigned long long)fp32_of(key) << 32) | (kPending | lid));
}

// Step (d) for one row per lane (lanes with todo set): passes until every
// row is resolved; a lane never waits inside a pass, so owners in this warp
// publish before anyone looks again.  KIND separates the out-of-line copies
// of the single-system kernel (0) and the batch kernel (1), whose register
// budgets differ.
template <class RF>
__device__ __forceinline__ void resolve_warp_body(const ClaimArgs& a, const int32_t* row, uint64_t key, uint32_t lid,
                                                  bool todo) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  for (int pass = 0;; ++pass) {
    unsigned long long* owned = nullptr;
    const int status = todo ? resolve_lane<RF>(a, row, key, lid, owned) : kDone;
    uint64_t sidx = 0;
    if (a.store_ctr) {  // the warp's owners take consecutive store rows with one atomic
      const uint32_t ob = __ballot_sync(0xffffffffu, status == kOwner);
      if (ob) {
        const int leader = __ffs(ob) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(a.store_ctr, (unsigned long long)__popc(ob));
        sidx = __shfl_sync(0xffffffffu, base, leader) + __popc(ob & ((1u << lane) - 1u));
      }
    }
    if (status == kOwner) finish_owner<RF>(a, row, key, lid, owned, sidx);
    todo = status == kRetry;
    if (__all_sync(0xffffffffu, !todo)) break;
    if (wait_expired(pass, a.wait_ns, t0)) {
      if (todo) atomicOr(&a.st->error, kErrTimeout);
      break;
    }
    __nanosleep(32);
  }
  __syncwarp();
}

template <class RF>
__device__ __noinline__ void resolve_warp_call(const ClaimArgs& a, const int32_t* row, uint64_t key, uint32_t lid,
                                               bool todo) {
  resolve_warp_body<RF>(a, row, key, lid, todo);
}

template <class RF, int KIND>
__device__ __forceinline__ void resolve_warp(const ClaimArgs& a, const int32_t* row, uint64_t key, uint32_t lid,
                                             bool todo) {
  if constexpr (KIND == 0)
    resolve_warp_call<RF>(a, row, key, lid, todo);
  else
    resolve_warp_body<RF>(a, row, key, lid, todo);
}

// Mixed-radix digit of a neuron with `radix` choices; q moves to the next
// more significant neuron.
__device__ __forceinline__ uint32_t next_digit(uint64_t& q, uint32_t radix) {
  if (radix <= 1) return 0;
  if ((q >> 32) == 0) {
    const uint32_t q32 = (uint32_t)q;
    q = q32 / radix;
    return q32 % radix;
  }
  const uint32_t d = (uint32_t)(q % radix);
  q /= radix;
  return d;
}

// Four counts of a row in global memory, from count 4 * j on (VEC rows).
template <class RF>
__device__ __forceinline__ int4 load4(const typename RF::T* row, int j) {
  if constexpr (RF::W == 1)
    return unpack4_u8(reinterpret_cast<const uint32_t*>(row)[j]);
  else if constexpr (RF::W == 2)
    return unpack4_u16(reinterpret_cast<const uint2*>(row)[j]);
  else
    return reinterpret_cast<const int4*>(row)[j];
}

// Calls f(n, x) for n = m - 1 down to 0 with x = row[n].
template <class RF, typename F>
__device__ __forceinline__ void for_each_neuron_desc(const typename RF::T* row, int m, F&& f) {
  if constexpr (RF::VEC) {
    for (int n4 = (m >> 2) - 1; n4 >= 0; --n4) {
      const int4 v = load4<RF>(row, n4);
      f(4 * n4 + 3, v.w);
      f(4 * n4 + 2, v.z);
      f(4 * n4 + 1, v.y);
      f(4 * n4, v.x);
    }
  } else {
    for (int n = m - 1; n >= 0; --n) f(n, (int32_t)row[n]);
  }
}

// dst[0, m) = the counts of a row in global memory (one lane; dst int32 in
// shared memory, 16-byte aligned for VEC rows).
template <class RF>
__device__ __forceinline__ void load_row(const typename RF::T* src, int32_t* dst, int m) {
  if constexpr (RF::VEC) {
    int4* b = reinterpret_cast<int4*>(dst);
    for (int j = 0; j < (m >> 2); ++j) b[j] = load4<RF>(src, j);
  } else {
    for (int j = 0; j < m; ++j) dst[j] = src[j];
  }
}

// One lane's candidate in a batch that crosses parents.
struct FlatLane {
  uint64_t o;    // end of parent p + lane (off[p + 1 + lane])
  uint64_t t;    // index of the lane's candidate among its parent's
  uint64_t h;    // linear hash of the candidate's child
  int64_t pc;    // the lane's parent
};

// Steps (b)-(c), decision half, for candidates g .. g + nf - 1 (nf <= B) of a
// batch that may cross parents: each lane finds its parent among the next 32
// (off is sorted) and decodes its spiking vector (last neuron least
// significant).  From the parent's record only the multi-choice neurons are
// visited: hash = record hash + H[chosen] - H[first applicable] for each
// neuron whose digit is not 0; a parent without a record is decoded from its
// row and the applicability table.  keep = the candidate picks no rule that
// repeats an earlier applicable rule's row.  Returns nf, which shrinks when
// parents without candidates push a parent beyond the 32 examined.
template <class RF>
__device__ __forceinline__ int flat_decode(const ClaimArgs& a, uint64_t g, int nf, int64_t p, uint64_t p_lo,
                                           int lane, FlatLane& f, bool& keep) {
  const DevSys& s = a.sys;
  const int64_t pj = p + 1 + lane;
  f.o = pj <= a.P ? __ldcg(a.off + pj) : ~0ull;
  const uint64_t o31 = __shfl_sync(0xffffffffu, f.o, 31);
  if (o31 - g < (uint64_t)nf) nf = (int)(o31 - g);  // o31 > g: parent p holds g
  const uint64_t c = g + lane;
  int k = 0;  // parents p .. p + k - 1 end at or before c
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const uint64_t v = __shfl_sync(0xffffffffu, f.o, k + step - 1);
    if (v <= c) k += step;
  }
  const uint64_t prev = __shfl_sync(0xffffffffu, f.o, k > 0 ? k - 1 : 0);
  f.pc = lane < nf ? p + k : p;
  f.t = c - (k > 0 ? prev : p_lo);
  f.h = 0;
  keep = false;
  if (lane >= nf) return nf;
  uint64_t q = f.t;
  bool red = false;
  uint32_t nnt = kRecFull;
  const ParentRec* rec = a.prec ? a.prec + f.pc : nullptr;
  if (rec) {
    const uint4 head = __ldcg(reinterpret_cast<const uint4*>(rec));
    f.h = ((unsigned long long)head.y << 32) | head.x;
    nnt = head.z;
  }
  if (nnt != kRecFull) {
    uint64_t h = f.h;
    for (int i = (int)nnt - 1; i >= 0; --i) {
      const uint32_t e = __ldcg(rec->nt + i);
      const uint32_t mask = e & 0xFFFFu;
      const uint32_t d = next_digit(q, __popc(mask));
      if (d == 0) continue;
      const int r0 = __ldg(s.first_rule + (e >> 16));
      const int rb = r0 + nth_set_bit(mask, (int)d);
      h += __ldg(s.rowkey + rb) - __ldg(s.rowkey + r0 + __ffs(mask) - 1);
      red |= (__ldg(s.eqmask + rb) & mask) != 0u;
    }
    f.h = h;
  } else {
    uint64_t h = 0;
    for_each_neuron_desc<RF>(parent_row<RF>(a, f.pc), s.m, [&](int n, int32_t x) {
      h += col_hash(s, n, x);
      const uint64_t am = appl(s, n, x);
      const uint32_t mask = (uint32_t)am;
      if (!mask) return;
      const int kb = nth_set_bit(mask, (int)next_digit(q, __popc(mask)));
      h += __ldg(s.rowkey + __ldg(s.first_rule + n) + kb);
      red |= ((am >> (32 + kb)) & 1ull) == 0;
    });
    f.h = h;
  }
  keep = !red;
  return nf;
}

// Step (c) for a candidate of a crossing batch: C' = C + the chosen rules'
// rows, built in a tile row (one lane).
template <class RF, int KIND>
__device__ __forceinline__ void flat_build(const ClaimArgs& a, int64_t pc, uint64_t t, int32_t* trow) {
  const DevSys& s = a.sys;
  const typename RF::T* prow = parent_row<RF>(a, pc);
  load_row<RF>(prow, trow, s.m);
  uint64_t q = t;
  for_each_neuron_desc<RF>(prow, s.m, [&](int n, int32_t x) {
    const uint32_t mask = (uint32_t)appl(s, n, x);
    if (!mask) return;
    const int kb = nth_set_bit(mask, (int)next_digit(q, __popc(mask)));
    add_rule<KIND>(s, trow, __ldg(s.first_rule + n) + kb);
  });
}

// Per-warp shared memory of the expand loop.
__device__ __forceinline__ ExpandSmem expand_smem(unsigned char* base, int m, int B, int ts) {
  const int m4 = round4(m);
  ExpandSmem w;
  w.tile = reinterpret_cast<int32_t*>(base);
  w.keys = reinterpret_cast<unsigned long long*>(w.tile + (size_t)B * ts);
  w.dpc = reinterpret_cast<long long*>(w.keys + B);
  w.dt = reinterpret_cast<unsigned long long*>(w.dpc + B);
  w.lids = reinterpret_cast<uint32_t*>(w.dt + B);
  w.par = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(w.keys) + expand_keys_bytes(B));
  w.buf = w.par + m4;
  w.msk = reinterpret_cast<uint32_t*>(w.buf + m4);
  w.ntl = reinterpret_cast<uint16_t*>(w.msk + m4);
  w.chg = reinterpret_cast<int2*>(w.ntl + m4);
  w.hdr = reinterpret_cast<int*>(w.chg + m4);
  w.dig = reinterpret_cast<uint8_t*>(w.hdr + 8);
  w.low = nullptr;
  return w;
}

// Per-warp shared memory of the wide mode: the scratch row, the queue of
// crossing-batch candidates, then the parent state as in expand_smem without
// the parent's row (read from the store when a task starts) and without a
// change list (the odometer's swaps go straight into the block base).
__device__ __forceinline__ ExpandSmem expand_smem_wide(unsigned char* base, int m) {
  const int m4 = round4(m);
  ExpandSmem w;
  w.tile = reinterpret_cast<int32_t*>(base);
  w.keys = reinterpret_cast<unsigned long long*>(w.tile + m4);
  w.dpc = reinterpret_cast<long long*>(w.keys + kWideB);
  w.dt = reinterpret_cast<unsigned long long*>(w.dpc + kWideB);
  w.lids = reinterpret_cast<uint32_t*>(w.dt + kWideB);
  w.par = nullptr;
  w.buf = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(w.keys) + expand_keys_bytes(kWideB));
  w.msk = reinterpret_cast<uint32_t*>(w.buf + m4);
  w.ntl = reinterpret_cast<uint16_t*>(w.msk + m4);
  w.chg = nullptr;
  w.hdr = reinterpret_cast<int*>(w.ntl + m4);
  w.low = w.hdr + 8;
  w.dig = reinterpret_cast<uint8_t*>(w.low + kLowHdr + kLowTab);
  return w;
}

// dst = src for a row in shared memory, by the whole warp.
template <bool VEC>
__device__ __forceinline__ void warp_copy_row(const int32_t* src, int32_t* dst, int m, int lane) {
  if (VEC) {
    const int4* a = reinterpret_cast<const int4*>(src);
    int4* b = reinterpret_cast<int4*>(dst);
#pragma unroll 4
    for (int j = lane; j < (m >> 2); j += 32) b[j] = a[j];
  } else {
    for (int j = lane; j < m; j += 32) dst[j] = src[j];
  }
}

// row += M[rn] - M[ro] for two rules of one neuron, by the whole warp: the
// columns of the neuron's support are distinct, so the lanes share them out.
// A lane's loads for up to three support columns are all issued before its
// updates, so that a support of up to 96 columns costs one round trip.
__device__ __forceinline__ void warp_swap_rule(const DevSys& s, int32_t* row, int ro, int rn, int lane) {
  const int4 dn = __ldg(s.rdesc + rn);
  const int32_t* vn = s.rval + dn.z;
  const int32_t* vo = s.rval + __ldg(&s.rdesc[ro].z);
  const int32_t* col = s.scol + dn.x;
  for (int i0 = 0; i0 < dn.y; i0 += 96) {
    int c[3], v[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int i = i0 + lane + 32 * u;
      c[u] = -1;
      if (i < dn.y) {
        c[u] = __ldg(col + i);
        v[u] = __ldg(vn + i) - __ldg(vo + i);
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u)
      if (c[u] >= 0) row[c[u]] += v[u];
  }
  __syncwarp();
}

// Row of candidate L of the current block in the scratch row: the block base
// with the low digits of L (all lanes decode the same digits).  cur holds the
// packed low digits of the row the scratch row already holds (kNoRow: none
// of this block): only the digits that differ are swapped, so that the
// owners of a block, taken in lane order, mostly cost one swap each.
constexpr uint32_t kNoRow = 0xFFFFFFFFu;
template <bool VEC>
__device__ __forceinline__ void build_block_row(const DevSys& s, ExpandSmem& w, int L, int nlow, int lane,
                                                uint32_t& cur) {
  uint32_t from = cur;
  const uint32_t pk = (uint32_t)w.low[kLowDig + L];
  if (from == kNoRow) {
    __syncwarp();
    warp_copy_row<VEC>(w.buf, w.tile, s.m, lane);
    __syncwarp();
    from = 0;
  }
  cur = pk;
  const bool tab = w.hdr[kLowOk] != 0;
  for (int i = 0; i < nlow; ++i) {
    const uint32_t d0 = (from >> (5 * i)) & 31u, d = (pk >> (5 * i)) & 31u;
    if (d == d0) continue;
    const int n = w.ntl[i];
    if (tab) {  // the support's columns are distinct: a lane reads its three before it writes them
      const int len = w.low[2 * i + 1];
      const int32_t* col = w.low + kLowHdr + w.low[2 * i];
      const int32_t* dv = col + (int)d * len;   // M[rule d] - M[rule 0] (d >= 1)
      const int32_t* dv0 = col + (int)d0 * len;
      for (int k0 = 0; k0 < len; k0 += 96) {
        int c[3], v[3], x[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int k = k0 + lane + 32 * u;
          c[u] = k < len ? col[k] : -1;
          v[u] = k < len ? (d ? dv[k] : 0) - (d0 ? dv0[k] : 0) : 0;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) x[u] = c[u] >= 0 ? w.tile[c[u]] : 0;
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (c[u] >= 0) w.tile[c[u]] = x[u] + v[u];
      }
      __syncwarp();
    } else {
      warp_swap_rule(s, w.tile, rule_of(s, w, n, (int)d0), rule_of(s, w, n, (int)d), lane);
    }
  }
}

// The low neurons' swap table of the loaded parent (by the whole warp): for
// low neuron i, its support columns, then for each choice d > 0 the support's
// entries of M[rule d] - M[rule 0].  Left unused (kLowOk = 0) when it does not
// fit in kLowTab words.
__device__ __forceinline__ void build_low_table(const DevSys& s, ExpandSmem& w, int lane) {
  const int nlow = w.hdr[kNlow];
  if (lane < w.hdr[kRL]) {  // RL <= 32 with every radix >= 2: at most 5 low neurons, digits < 32
    uint32_t q = (uint32_t)lane, pk = 0;
    for (int i = 0; i < nlow; ++i) {
      const uint32_t radix = __popc(w.msk[w.ntl[i]]);
      pk |= (q % radix) << (5 * i);
      q /= radix;
    }
    w.low[kLowDig + lane] = (int32_t)pk;
  }
  int at = 0;
  bool fits = true;
  for (int i = 0; fits && i < nlow; ++i) {
    const int n = w.ntl[i];
    const int radix = __popc(w.msk[n]);
    const int4 d0 = __ldg(s.rdesc + rule_of(s, w, n, 0));
    const int len = d0.y;
    if (at + len * radix > kLowTab) {
      fits = false;
      break;
    }
    int32_t* t = w.low + kLowHdr + at;
    for (int k = lane; k < len; k += 32) t[k] = __ldg(s.scol + d0.x + k);
    for (int d = 1; d < radix; ++d) {
      const int vz = __ldg(&s.rdesc[rule_of(s, w, n, d)].z);
      for (int k = lane; k < len; k += 32) t[d * len + k] = __ldg(s.rval + vz + k) - __ldg(s.rval + d0.z + k);
    }
    if (lane == 0) {
      w.low[2 * i] = at;
      w.low[2 * i + 1] = len;
    }
    at += len * radix;
  }
  __syncwarp();
  if (lane == 0) w.hdr[kLowOk] = fits ? 1 : 0;
  __syncwarp();
}

// Row of candidate t of parent pc (a crossing-batch candidate) in the scratch
// row: each lane decodes the digits of its own ceil(m / 32) neurons, whose
// place value is the product of the choice counts of the later lanes' neurons
// (last neuron least significant), and adds its chosen rules' rows.
template <class RF>
__device__ __forceinline__ void build_flat_row(const ClaimArgs& a, int32_t* row, int64_t pc, uint64_t t, int lane) {
  const DevSys& s = a.sys;
  const typename RF::T* prow = parent_row<RF>(a, pc);
  __syncwarp();
  for (int n = lane; n < s.m; n += 32) row[n] = prow[n];
  const int n0 = lane * s.K, n1 = min(n0 + s.K, s.m);
  uint64_t prod = 1;
  for (int n = n0; n < n1; ++n) {
    const uint32_t mask = (uint32_t)appl(s, n, prow[n]);
    prod = sat_mul(prod, mask ? (uint64_t)__popc(mask) : 1ull);
  }
  uint64_t v = prod;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_down_sync(0xffffffffu, v, o);
    if (lane + o < 32) v = sat_mul(v, u);
  }
  const uint64_t nxt = __shfl_down_sync(0xffffffffu, v, 1);
  const uint64_t after = lane == 31 ? 1ull : nxt;
  __syncwarp();
  uint64_t q = (after > t) ? 0ull : t / after;
  for (int n = n1 - 1; n >= n0; --n) {
    const uint32_t mask = (uint32_t)appl(s, n, prow[n]);
    if (!mask) continue;
    const int kb = nth_set_bit(mask, (int)next_digit(q, __popc(mask)));
    add_row_shared(s, row, __ldg(s.first_rule + n) + kb, 1);
  }
  __syncwarp();
}

// Full-key compare of the scratch row with a stored row, by the whole warp.
template <class RF>
__device__ __forceinline__ bool warp_rows_equal(const int32_t* row, const typename RF::T* other, int m, int lane) {
  int diff = 0;
  if constexpr (RF::W == 1) {  // lane j: counts 4j .. 4j + 3 (conflict-free 16-byte reads of the scratch row)
    const int4* a = reinterpret_cast<const int4*>(row);
    const uint32_t* b = reinterpret_cast<const uint32_t*>(other);
    for (int j = lane; j < (m >> 2); j += 32) diff |= (int)(pack4_u8(a[j]) ^ __ldcg(b + j));
  } else if constexpr (RF::W == 2) {
    const int4* a = reinterpret_cast<const int4*>(row);
    const uint2* b = reinterpret_cast<const uint2*>(other);
    for (int j = lane; j < (m >> 2); j += 32) {
      const uint2 x = pack4_u16(a[j]), y = __ldcg(b + j);
      diff |= (int)((x.x ^ y.x) | (x.y ^ y.y));
    }
  } else if constexpr (RF::VEC) {
    const int4* a = reinterpret_cast<const int4*>(row);
    const int4* b = reinterpret_cast<const int4*>(other);
    for (int j = lane; j < (m >> 2); j += 32) {
      const int4 x = a[j], y = __ldcg(b + j);
      diff |= (x.x ^ y.x) | (x.y ^ y.y) | (x.z ^ y.z) | (x.w ^ y.w);
    }
  } else {
    for (int j = lane; j < m; j += 32) diff |= row[j] ^ __ldcg(other + j);
  }
  return !__any_sync(0xffffffffu, diff != 0);
}

// The scratch row to global memory, by the whole warp (coalesced).
template <class RF>
__device__ __forceinline__ void warp_store_row(const int32_t* row, typename RF::T* dst, int m, int lane) {
  if constexpr (RF::W == 1) {
    const int4* a = reinterpret_cast<const int4*>(row);
    uint32_t* b = reinterpret_cast<uint32_t*>(dst);
#pragma unroll 4
    for (int j = lane; j < (m >> 2); j += 32) __stcg(b + j, pack4_u8(a[j]));
  } else if constexpr (RF::W == 2) {
    const int4* a = reinterpret_cast<const int4*>(row);
    uint2* b = reinterpret_cast<uint2*>(dst);
#pragma unroll 4
    for (int j = lane; j < (m >> 2); j += 32) __stcg(b + j, pack4_u16(a[j]));
  } else if constexpr (RF::VEC) {
    const int4* a = reinterpret_cast<const int4*>(row);
    int4* b = reinterpret_cast<int4*>(dst);
#pragma unroll 4
    for (int j = lane; j < (m >> 2); j += 32) __stcg(b + j, a[j]);
  } else {
    for (int j = lane; j < m; j += 32) __stcg(dst + j, row[j]);
  }
}

// Rows of int32 counts leave the scratch row by a bulk copy (cp.async.bulk,
// issued by lane 0) rather than by 16-byte stores of every lane: the lanes'
// writes to the scratch row are made visible to the async proxy before the
// copy is issued; the scratch row is written again only after the copy has
// read it; the owners publish only after every copy has completed and been
// made visible to generic loads (then the usual fence and release).
__device__ __forceinline__ void bulk_store_row(void* dst, const int32_t* scratch, uint32_t bytes, int lane) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"((uint32_t)__cvta_generic_to_shared(scratch)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
}
__device__ __forceinline__ void bulk_wait_read(int lane) {
  if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncwarp();
}
__device__ __forceinline__ void bulk_wait_all(int lane) {
  if (lane == 0) {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncwarp();
}

constexpr int kProbe = 3, kCompare = 4;

// Step (d) in the wide mode, for one key per lane (lanes with todo set).
// Lanes walk their own probe sequences as resolve_lane does; a row is built,
// by the whole warp in the scratch row, only where a stored row with the same
// fingerprint must be compared or where the lane has claimed a slot and
// writes its row.  build(L) builds lane L's row.  As in resolve_warp_body, no
// lane waits inside a pass: a lane that meets a reserved slot with its
// fingerprint starts over in a later pass, and owners publish before the pass
// ends.
template <class RF, typename Build>
__device__ __forceinline__ void resolve_warp_wide(const ClaimArgs& a, int32_t* scratch, uint64_t key, uint32_t lid,
                                                  bool todo, int lane, Build&& build) {
  const int m = a.sys.m;
  const uint32_t fp = fp32_of(key);
  const unsigned long long mine = ((unsigned long long)fp << 32) | kRowReserved;
  int st = todo ? kRetry : kDone;
  uint64_t bucket = 0, probes = 0;
  uint32_t match = 0, empty = 0;
  bool loaded = false;
  uint32_t orf = 0;
  const typename RF::T* other = nullptr;
  unsigned long long* owned = nullptr;
  uint64_t t0 = 0;
  for (int pass = 0;; ++pass) {
    if (st == kRetry) {
      st = kProbe;
      bucket = key & a.table.bmask;
      probes = 0;
      loaded = false;
    }
    for (;;) {
      // each probing lane goes on to its next compare, claim, retry or end
      while (st == kProbe) {
        unsigned long long* bs = a.table.slots + bucket * kBucket;
        if (!loaded) {
          if (probes > a.table.bmask) {
            atomicOr(&a.st->error, kErrTableFull);
            st = kDone;
            break;
          }
          const ulonglong2* b2 = reinterpret_cast<const ulonglong2*>(bs);
          match = 0;
          empty = 0;
#pragma unroll
          for (int q = 0; q < kBucket / 2; ++q) {
            const ulonglong2 x = __ldcg(b2 + q);
            empty |= (x.x == kEmpty ? 1u : 0u) << (2 * q);
            empty |= (x.y == kEmpty ? 1u : 0u) << (2 * q + 1);
            match |= ((uint32_t)(x.x >> 32) == fp && (uint32_t)x.x != kRowTomb && x.x != kEmpty ? 1u : 0u) << (2 * q);
            match |= ((uint32_t)(x.y >> 32) == fp && (uint32_t)x.y != kRowTomb && x.y != kEmpty ? 1u : 0u)
                     << (2 * q + 1);
          }
          loaded = true;
        }
        if (match) {
          const int j = __ffs(match) - 1;
          match &= match - 1;
          orf = (uint32_t)__ldcg(bs + j);
          if (orf == kRowReserved) {
            st = kRetry;
            break;
          }
          if (orf & kPending) {
            (void)ld_acquire(bs + j);
            const uint32_t o = orf & ~kPending;
            other = a.store_ctr ? row_at<RF>(a.pool, __ldcg(a.sidx_of + o), m) : row_at<RF>(a.staging, o, m);
          } else {
            other = row_at<RF>(a.pool, orf, m);
          }
          st = kCompare;
          break;
        }
        if (empty) {
          const int j = __ffs(empty) - 1;
          if (atomicCAS(bs + j, kEmpty, mine) == kEmpty) {
            owned = bs + j;
            st = kOwner;
            break;
          }
          loaded = false;  // look at this bucket again
          continue;
        }
        ++probes;
        bucket = (bucket + 1) & a.table.bmask;
        loaded = false;
      }
      // compares, one lane's row at a time
      for (uint32_t cm = __ballot_sync(0xffffffffu, st == kCompare); cm; cm &= cm - 1) {
        const int L = __ffs(cm) - 1;
        const typename RF::T* o = reinterpret_cast<const typename RF::T*>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(other), L));
        build(L);
        const bool eq = warp_rows_equal<RF>(scratch, o, m, lane);
        if (lane == L) {
          if (eq) {
            if (orf & kPending) atomicMin(a.gmin + (orf & ~kPending), lid);
            st = kDone;
          } else {
            st = kProbe;
          }
        }
      }
      // owners: consecutive store rows with one atomic, rows written by the
      // whole warp (int32 rows: by bulk copies), then each owner publishes
      // its slot
      const uint32_t ob = __ballot_sync(0xffffffffu, st == kOwner);
      if (ob) {
        uint64_t sidx = 0;
        if (a.store_ctr) {
          const int leader = __ffs(ob) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(a.store_ctr, (unsigned long long)__popc(ob));
          sidx = __shfl_sync(0xffffffffu, base, leader) + __popc(ob & ((1u << lane) - 1u));
        }
        for (uint32_t ow = ob; ow; ow &= ow - 1) {
          const int L = __ffs(ow) - 1;
          const uint64_t sl = __shfl_sync(0xffffffffu, sidx, L);
          const uint32_t ll = __shfl_sync(0xffffffffu, lid, L);
          if (a.store_ctr && sl >= a.store_cap) continue;  // reported by lane L below
          typename RF::T* dst = a.store_ctr ? row_at<RF>(a.pool, sl, m) : row_at<RF>(a.staging, ll, m);
          if constexpr (RF::W == 4 && RF::VEC) {  // m % 4 == 0: a row is whole, aligned 16-byte units
            bulk_wait_read(lane);  // the previous owner's copy has read the scratch row
            build(L);
            bulk_store_row(dst, scratch, (uint32_t)m * 4u, lane);
          } else {
            build(L);
            warp_store_row<RF>(scratch, dst, m, lane);
          }
        }
        if constexpr (RF::W == 4 && RF::VEC) bulk_wait_all(lane);
        __threadfence();
        __syncwarp();
        if (st == kOwner) {
          st = kDone;
          if (a.store_ctr) {
            if (sidx >= a.store_cap) {  // the host sizes the store for every claim of the chunk
              atomicOr(&a.st->error, kErrStaging);
              owned = nullptr;
            } else {
              a.sidx_of[lid] = (uint32_t)sidx;
            }
          }
          if (owned) {
            a.gmin[lid] = lid;
            a.slot_of[lid] = (uint32_t)(owned - a.table.slots);
            atomicOr(a.ownbits + (lid >> 5), 1u << (lid & 31));
            st_release(owned, ((unsigned long long)fp << 32) | (kPending | lid));
          }
        }
      }
      if (!__any_sync(0xffffffffu, st == kProbe)) break;
    }
    if (__all_sync(0xffffffffu, st != kRetry)) break;
    if (wait_expired(pass, a.wait_ns, t0)) {
      if (st == kRetry) atomicOr(&a.st->error, kErrTimeout);
      break;
    }
    __nanosleep(32);
  }
  __syncwarp();
}

// Resolves the queued crossing-batch candidates in the wide mode.
template <class RF>
__device__ __forceinline__ void flush_queue_wide(const ClaimArgs& a, ExpandSmem& w, int fill, int lane) {
  const bool mine = lane < fill;
  resolve_warp_wide<RF>(a, w.tile, mine ? w.keys[lane] : 0ull, mine ? w.lids[lane] : 0u, mine, lane,
                        [&](int L) { build_flat_row<RF>(a, w.tile, w.dpc[L], w.dt[L], lane); });
}

// Base children (every firing neuron on its first applicable rule) of the
// first kBaseSlots parents of a pass that hold at least kBaseMin of its
// candidates, one CTA each: the wide mode then decodes a block base as the
// cached base child plus the rows of the neurons whose digit is not 0, rather
// than C plus a chosen row of M_Pi for every firing neuron.
struct BaseSlot {
  int64_t parent;  // frontier row, or -1: slot unused in this pass
  uint64_t hash;   // linear hash of the base child (unmixed)
};
constexpr uint64_t kBaseMin = 4096;

__host__ __device__ inline size_t base_rows_offset() { return sizeof(BaseSlot) * kBaseSlots; }

template <class RF>
__global__ void __launch_bounds__(1024) k_wide_base(ClaimArgs a) {
  extern __shared__ __align__(16) int32_t brow[];  // [m]
  __shared__ int64_t s_p0;
  __shared__ unsigned long long s_h;
  const DevSys& s = a.sys;
  const int m = s.m;
  BaseSlot* hdr = reinterpret_cast<BaseSlot*>(a.bcache);
  int32_t* out = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(a.bcache) + base_rows_offset()) +
                 (size_t)blockIdx.x * round4(m);
  if (threadIdx.x == 0) {
    int64_t lo = 0, hi = a.P;  // largest p with off[p] <= g0 (off is sorted, off[0] = 0)
    while (hi - lo > 1) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (__ldg(a.off + mid) <= a.g0) lo = mid; else hi = mid;
    }
    s_p0 = lo;
    s_h = 0;
  }
  __syncthreads();
  const int64_t p = s_p0 + blockIdx.x;
  bool use = !(a.ctr && __ldcg(a.ctr + 1) == 0) && p < a.P;
  if (use) {
    const uint64_t lo = max(__ldg(a.off + p), a.g0), hi = min(__ldg(a.off + p + 1), a.g0 + a.Q);
    use = hi > lo && hi - lo >= kBaseMin;
  }
  if (!use) {
    if (threadIdx.x == 0) hdr[blockIdx.x].parent = -1;
    return;
  }
  const typename RF::T* prow = parent_row<RF>(a, p);
  for (int n = threadIdx.x; n < m; n += blockDim.x) brow[n] = (int32_t)prow[n];
  __syncthreads();
  uint64_t h = 0;
  for (int n = threadIdx.x; n < m; n += blockDim.x) {
    const int32_t x = (int32_t)prow[n];
    h += col_hash(s, n, x);
    const uint32_t mask = (uint32_t)appl(s, n, x);
    if (!mask) continue;
    const int r = __ldg(s.first_rule + n) + __ffs(mask) - 1;
    h += __ldg(s.rowkey + r);
    const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
    for (int e = e0; e < e1; e += 8) {  // eight loads in flight before their adds
      int2 cv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) cv[u] = e + u < e1 ? __ldg(s.csr + e + u) : make_int2(-1, 0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (cv[u].x >= 0) atomicAdd(&brow[cv[u].x], cv[u].y);
    }
  }
  h = warp_sum_u64(h);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_h, (unsigned long long)h);
  __syncthreads();
  for (int n = threadIdx.x; n < m; n += blockDim.x) out[n] = brow[n];
  if (threadIdx.x == 0) {
    hdr[blockIdx.x].hash = s_h;
    hdr[blockIdx.x].parent = p;
  }
}

// The block base for candidate t of the loaded parent from its cached base
// child: the neurons whose digit of t is not 0 (least significant first)
// swap their first applicable rule's row for the chosen one.  Same digits,
// base row and hash as decode_full.
__device__ __forceinline__ void decode_from_base(const DevSys& s, ExpandSmem& w, const int32_t* base, uint64_t hbase,
                                                 uint64_t t, int lane) {
  const int m4 = round4(s.m);
  const int4* b4 = reinterpret_cast<const int4*>(base);
  int4* d4 = reinterpret_cast<int4*>(w.buf);
  for (int j = lane; j < (m4 >> 2); j += 32) d4[j] = __ldcg(b4 + j);
  for (int n = lane; n < s.m; n += 32) w.dig[n] = 0;
  __syncwarp();
  uint64_t h = hbase, q = t;
  int red = 0;
  const int nnt = w.hdr[kNnt];
  for (int i = 0; i < nnt && q != 0; ++i) {
    const int n = w.ntl[i];
    const uint32_t mask = w.msk[n];
    const uint32_t d = next_digit(q, __popc(mask));
    if (d == 0) continue;
    const int r0 = rule_of(s, w, n, 0), rd = rule_of(s, w, n, (int)d);
    warp_swap_rule(s, w.buf, r0, rd, lane);
    h += __ldg(s.rowkey + rd) - __ldg(s.rowkey + r0);
    red += redundant_choice(s, mask, rd) ? 1 : 0;
    if (lane == 0) w.dig[n] = (uint8_t)d;
  }
  __syncwarp();
  if (lane == 0) {
    hbase_of(w) = h;
    w.hdr[kNred] = red;
  }
  __syncwarp();
}

// Block mode in the wide mode: lane k < RL owns candidate k of each block as
// in block_run, but keeps only its hash; rows are built on demand from the
// block base, to which the odometer applies its swaps directly.
template <class RF>
__device__ __forceinline__ uint64_t block_run_wide(const ClaimArgs& a, ExpandSmem& w, int64_t p, uint64_t p_lo,
                                                   uint64_t p_hi, uint64_t l, uint64_t lb, int64_t& cached_p,
                                                   uint64_t& after, int lane) {
  const DevSys& s = a.sys;
  const uint64_t g = a.g0 + l;
  const uint64_t gend = min(p_hi, a.g0 + lb);
  if (p != cached_p) {
    after = parent_state(s, parent_row<RF>(a, p), w, kWideB, lane);
    build_low_table(s, w, lane);
    cached_p = p;
  }
  const int RL = w.hdr[kRL], nlow = w.hdr[kNlow], nnt = w.hdr[kNnt];
  const uint64_t b = (g - p_lo) / (uint64_t)RL;
  int slot = -1;  // the parent's cached base child, if the pass has one
  if (a.bcache) {
    const BaseSlot* hs = reinterpret_cast<const BaseSlot*>(a.bcache);
    const uint32_t hit = __ballot_sync(0xffffffffu, lane < kBaseSlots && __ldcg(&hs[lane].parent) == p);
    slot = hit ? __ffs(hit) - 1 : -1;
  }
  if (slot >= 0)
    decode_from_base(s, w,
                     reinterpret_cast<const int32_t*>(reinterpret_cast<const unsigned char*>(a.bcache) +
                                                      base_rows_offset()) + (size_t)slot * round4(s.m),
                     __ldcg(&reinterpret_cast<const BaseSlot*>(a.bcache)[slot].hash), b * (uint64_t)RL, lane);
  else
    decode_full<true>(s, w, b * (uint64_t)RL, after, lane, parent_row<RF>(a, p));
  uint64_t hk = 0;
  bool redk = true;
  if (lane < RL) {
    redk = false;
    uint32_t q = (uint32_t)lane;
    for (int i = 0; i < nlow; ++i) {
      const int n = w.ntl[i];
      const uint32_t mask = w.msk[n];
      const uint32_t radix = __popc(mask);
      const uint32_t d = q % radix;
      q /= radix;
      if (d == 0) continue;
      const int r0 = rule_of(s, w, n, 0), rd = rule_of(s, w, n, (int)d);
      hk += __ldg(s.rowkey + rd) - __ldg(s.rowkey + r0);
      redk |= redundant_choice(s, mask, rd);
    }
  }
  uint64_t gb = p_lo + b * (uint64_t)RL;
  for (;;) {
    const uint64_t c = gb + lane;
    const bool todo = lane < RL && c >= g && c < gend && !redk && w.hdr[kNred] == 0;
    uint32_t cur = kNoRow;  // the scratch row holds no candidate of this block yet
    resolve_warp_wide<RF>(a, w.tile, mix64(hbase_of(w) + hk), (uint32_t)(c - a.g0), todo, lane,
                          [&](int L) { build_block_row<RF::VEC>(s, w, L, nlow, lane, cur); });
    gb += (uint64_t)RL;
    if (gb >= gend) break;
    // next block: the odometer, every lane following the same digits
    uint64_t h = hbase_of(w);
    int red = w.hdr[kNred];
    for (int i = nlow; i < nnt; ++i) {
      const int n = w.ntl[i];
      const uint32_t mask = w.msk[n];
      const int d = w.dig[n];
      const int nd = (d + 1 == __popc(mask)) ? 0 : d + 1;
      const int ro = rule_of(s, w, n, d), rn = rule_of(s, w, n, nd);
      h += __ldg(s.rowkey + rn) - __ldg(s.rowkey + ro);
      red += (redundant_choice(s, mask, rn) ? 1 : 0) - (redundant_choice(s, mask, ro) ? 1 : 0);
      warp_swap_rule(s, w.buf, ro, rn, lane);
      if (lane == 0) w.dig[n] = (uint8_t)nd;
      if (nd != 0) break;
    }
    __syncwarp();
    if (lane == 0) {
      hbase_of(w) = h;
      w.hdr[kNred] = red;
    }
    __syncwarp();
  }
  return gend - a.g0;
}

// Resolves the queued rows of crossing batches (building them first).
template <class RF, int KIND>
__device__ __forceinline__ void flush_queue(const ClaimArgs& a, ExpandSmem& w, int ts, int fill, int lane) {
  const bool mine = lane < fill;
  if (mine && w.dpc[lane] >= 0) flat_build<RF, KIND>(a, w.dpc[lane], w.dt[lane], w.tile + lane * ts);
  __syncwarp();
  resolve_warp<RF, KIND>(a, w.tile + lane * ts, mine ? w.keys[lane] : 0ull, mine ? w.lids[lane] : 0u, mine);
}

// Block mode for parent p from candidate a.g0 + l to the end of the parent or
// of the task; returns the new l.
template <class RF, int KIND>
__device__ __forceinline__ uint64_t block_run(const ClaimArgs& a, ExpandSmem& w, int B, int ts, int64_t p,
                                              uint64_t p_lo, uint64_t p_hi, uint64_t l, uint64_t lb,
                                              int64_t& cached_p, uint64_t& after, int lane) {
  const DevSys& s = a.sys;
  const int m = s.m;
  const uint64_t g = a.g0 + l;
  const uint64_t gend = min(p_hi, a.g0 + lb);
  if (p != cached_p) {  // the warp's shared memory still holds the state of cached_p
    after = parent_state(s, parent_row<RF>(a, p), w, B, lane);
    cached_p = p;
  }
  const int RL = w.hdr[kRL], nlow = w.hdr[kNlow], nnt = w.hdr[kNnt];
  uint64_t b = (g - p_lo) / (uint64_t)RL;
  decode_full(s, w, b * (uint64_t)RL, after, lane);
  // lane k < RL: candidate k of the block = base + its low digits
  int32_t* row = w.tile + lane * ts;
  uint64_t hk = 0;
  bool redk = true;
  if (lane < RL) {
    copy_row<RF::VEC>(w.buf, row, m);
    redk = false;
    uint32_t q = (uint32_t)lane;
    for (int i = 0; i < nlow; ++i) {
      const int n = w.ntl[i];
      const uint32_t mask = w.msk[n];
      const uint32_t radix = __popc(mask);
      const uint32_t d = q % radix;
      q /= radix;
      if (d == 0) continue;
      const int r0 = rule_of(s, w, n, 0), rd = rule_of(s, w, n, (int)d);
      swap_rule<KIND>(s, row, r0, rd);
      hk += __ldg(s.rowkey + rd) - __ldg(s.rowkey + r0);
      redk |= redundant_choice(s, mask, rd);
    }
  }
  uint64_t gb = p_lo + b * (uint64_t)RL;
  for (;;) {
    const uint64_t c = gb + lane;
    const bool todo = lane < RL && c >= g && c < gend && !redk && w.hdr[kNred] == 0;
    resolve_warp<RF, KIND>(a, row, mix64(hbase_of(w) + hk), (uint32_t)(c - a.g0), todo);
    gb += (uint64_t)RL;
    if (gb >= gend) break;
    // next block: the high digits move on by one (odometer, least significant first)
    if (lane == 0) {
      uint64_t h = hbase_of(w);
      int red = w.hdr[kNred], nc = 0;
      for (int i = nlow; i < nnt; ++i) {
        const int n = w.ntl[i];
        const uint32_t mask = w.msk[n];
        const int d = w.dig[n];
        const int nd = (d + 1 == __popc(mask)) ? 0 : d + 1;
        const int ro = rule_of(s, w, n, d), rn = rule_of(s, w, n, nd);
        w.chg[nc++] = make_int2(ro, rn);
        h += __ldg(s.rowkey + rn) - __ldg(s.rowkey + ro);
        red += (redundant_choice(s, mask, rn) ? 1 : 0) - (redundant_choice(s, mask, ro) ? 1 : 0);
        w.dig[n] = (uint8_t)nd;
        if (nd != 0) break;
      }
      hbase_of(w) = h;
      w.hdr[kNred] = red;
      w.hdr[kNchg] = nc;
    }
    __syncwarp();
    if (lane < RL) {
      const int nc = w.hdr[kNchg];
      for (int j = 0; j < nc; ++j) {
        const int2 rr = w.chg[j];
        swap_rule<KIND>(s, row, rr.x, rr.y);
      }
    }
  }
  return gend - a.g0;
}

template <class RF, int KIND>
__device__ __forceinline__ void flush_any(const ClaimArgs& a, ExpandSmem& w, int ts, int fill, int lane) {
  if constexpr (KIND == kWide)
    flush_queue_wide<RF>(a, w, fill, lane);
  else
    flush_queue<RF, KIND>(a, w, ts, fill, lane);
}

// Steps (b)-(d) for the tasks task0, task0 + tstride, ... of chunk a (a task
// is a run of a.run consecutive candidates), by one warp: block mode while
// the parent has 32 or more candidates left, else crossing batches.
template <class RF, int KIND>
__device__ __forceinline__ void expand_warp(const ClaimArgs& a, int B, int ts, ExpandSmem& w, uint64_t task0,
                                            uint64_t tstride, int lane) {
  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  int64_t p = -1;         // parent of the previous task's last candidate
  int64_t cached_p = -1;  // parent whose state the warp's shared memory holds
  uint64_t after = 0;     // its per-lane place values
  for (uint64_t task = task0; task < ntasks; task += tstride) {
    const uint64_t la = task * a.run;
    const uint64_t lb = min(la + a.run, (uint64_t)a.Q);
    {
      // tasks come in increasing order: look among the 32 parents from the
      // previous one first (off is sorted), else search all of them
      const uint64_t g = a.g0 + la;
      int k = 32;
      if (p >= 0) {
        const int64_t pj = p + 1 + lane;
        k = __popc(__ballot_sync(0xffffffffu, pj <= a.P && __ldcg(a.off + pj) <= g));
      }
      p = k < 32 ? p + k : warp_find_parent(a.off, a.P, g, lane);
    }
    uint64_t p_lo = __ldcg(a.off + p), p_hi = __ldcg(a.off + p + 1);
    if (task == 0 && lane == 0) a.st->p_first = (unsigned long long)p;
    uint64_t l = la;
    int fill = 0;  // rows queued by crossing batches
    for (;;) {
      const bool done = l >= lb;
      const uint64_t g = a.g0 + l;
      if (done || p_hi - g >= 32) {
        if (fill > 0) {  // the tile is about to be reused, or the task ends
          flush_any<RF, KIND>(a, w, ts, fill, lane);
          fill = 0;
        }
        if (done) break;
        if constexpr (KIND == kWide)
          l = block_run_wide<RF>(a, w, p, p_lo, p_hi, l, lb, cached_p, after, lane);
        else
          l = block_run<RF, KIND>(a, w, B, ts, p, p_lo, p_hi, l, lb, cached_p, after, lane);
        const uint64_t gn = a.g0 + l;
        if (l < lb) {
          do {
            ++p;
            p_lo = p_hi;
            p_hi = __ldcg(a.off + p + 1);
          } while (gn >= p_hi);
        }
        continue;
      }
      // crossing batch
      FlatLane f;
      bool keep = false;
      const int nb = flat_decode<RF>(a, g, (int)min((uint64_t)B, lb - l), p, p_lo, lane, f, keep);
      const uint32_t kept = __ballot_sync(0xffffffffu, keep);
      if (fill + __popc(kept) > B) {
        flush_any<RF, KIND>(a, w, ts, fill, lane);
        fill = 0;
      }
      if (keep) {
        const int slot = fill + __popc(kept & ((1u << lane) - 1u));
        w.dpc[slot] = f.pc;
        w.dt[slot] = f.t;
        w.keys[slot] = mix64(f.h);
        w.lids[slot] = (uint32_t)(l + lane);
      }
      fill += __popc(kept);
      __syncwarp();
      l += (uint64_t)nb;
      if (l >= lb) {  // keep the parent of the task's last candidate
        p = __shfl_sync(0xffffffffu, f.pc, nb - 1);
        continue;
      }
      const uint64_t gn = a.g0 + l;
      const int kn = __popc(__ballot_sync(0xffffffffu, f.o <= gn));  // parents ending at or before gn
      if (kn < 32) {
        const uint64_t lo = __shfl_sync(0xffffffffu, f.o, kn > 0 ? kn - 1 : 0);
        p_hi = __shfl_sync(0xffffffffu, f.o, kn);
        if (kn > 0) p_lo = lo;
        p += kn;
      } else {
        p = warp_find_parent(a.off, a.P, gn, lane);
        p_lo = __ldcg(a.off + p);
        p_hi = __ldcg(a.off + p + 1);
      }
    }
    if (task + 1 == ntasks && lane == 0) a.st->p_last = (unsigned long long)p;
  }
}

template <class RF>
__global__ void __launch_bounds__(256, 2) k_expand(ClaimArgs a, int B, int ts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.ctr && __ldcg(a.ctr + 1) == 0) return;  // the depth is full: a chunk enqueued ahead has nothing to do
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  ExpandSmem w = expand_smem(smem_raw + (size_t)wib * expand_warp_bytes(a.sys.m, B, ts), a.sys.m, B, ts);
  expand_warp<RF, 0>(a, B, ts, w, (uint64_t)blockIdx.x * wpb + wib, (uint64_t)gridDim.x * wpb, lane);
}

// The wide mode of k_expand (rows of more than kWideM neurons).
template <class RF>
__global__ void __launch_bounds__(kWideWarps * 32, 1) k_expand_wide(ClaimArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.ctr && __ldcg(a.ctr + 1) == 0) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  ExpandSmem w = expand_smem_wide(smem_raw + (size_t)wib * expand_wide_bytes(a.sys.m), a.sys.m);
  expand_warp<RF, kWide>(a, kWideB, 0, w, (uint64_t)blockIdx.x * wpb + wib, (uint64_t)gridDim.x * wpb, lane);
}

// Step (d) for rows already built in global memory (the tensor-core form):
// one lane per candidate, the same bounded wait-free passes as k_expand.
template <class RF>
__global__ void __launch_bounds__(256) k_resolve_rows(ClaimArgs a, const int32_t* rows,
                                                      const unsigned long long* hash, const uint8_t* redundant) {
  const int m = a.sys.m;
  if (a.ctr && __ldcg(a.ctr + 1) == 0) return;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < a.Q; base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t lid = base + threadIdx.x;
    bool done = lid >= a.Q || redundant[lid];
    const uint64_t key = done ? 0ull : mix64(hash[lid]);
    uint64_t t0 = 0;
    for (int pass = 0;; ++pass) {
      if (!done) {
        unsigned long long* owned = nullptr;
        const int status = resolve_lane<RF>(a, rows + lid * m, key, (uint32_t)lid, owned);
        if (status == kOwner) {
          if (a.inplace)
            finish_owner_inplace(a, key, (uint32_t)lid, owned, a.inplace_base + lid);
          else
            finish_owner<RF>(a, rows + lid * m, key, (uint32_t)lid, owned,
                              a.store_ctr ? atomicAdd(a.store_ctr, 1ull) : 0ull);
        }
        done = status != kRetry;
      }
      if (__all_sync(0xffffffffu, done)) break;
      if (wait_expired(pass, a.wait_ns, t0)) {
        if (!done) atomicOr(&a.st->error, kErrTimeout);
        break;
      }
      __nanosleep(32);
    }
  }
}

}  // namespace

void launch_resolve_rows(ClaimArgs a, const int32_t* rows, const unsigned long long* hash, const uint8_t* redundant,
                         cudaStream_t st, int nsm) {
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(((uint64_t)a.Q + 255) / 256, (uint64_t)nsm * 8));
  if (a.sys.m % 4 == 0)
    k_resolve_rows<RowI32V><<<blocks, 256, 0, st>>>(a, rows, hash, redundant);
  else
    k_resolve_rows<RowI32><<<blocks, 256, 0, st>>>(a, rows, hash, redundant);
}

size_t wide_base_bytes(int m) { return base_rows_offset() + (size_t)kBaseSlots * round4(m) * 4; }

int launch_expand(ClaimArgs a, cudaStream_t st, int nsm) {
  const int m = a.sys.m;
  if (m > kWideM) {
    const size_t per_warp = expand_wide_bytes(m);
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(kWideWarps, (226u << 10) / per_warp));
    const size_t smem = per_warp * wpb;
    // one task per warp: a task's first block costs a full decode (C + S . M
    // over every neuron), which wide rows make expensive
    const uint64_t warps = (uint64_t)nsm * wpb;
    a.run = (uint32_t)std::max<uint64_t>(8ull * kWideB, ((uint64_t)a.Q + warps - 1) / warps);
    const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
    const int blocks = (int)std::min<uint64_t>((ntasks + wpb - 1) / wpb, (uint64_t)nsm);
    if (a.bcache) {  // base children of the pass's largest parents
      const size_t bs = (size_t)round4(m) * 4;
      auto fb = a.w == 2 ? k_wide_base<RowU16> : a.w == 1 ? k_wide_base<RowU8>
                : (m % 4) == 0 ? k_wide_base<RowI32V> : k_wide_base<RowI32>;
      fb<<<kBaseSlots, std::min(1024, (m + 31) / 32 * 32), bs, st>>>(a);
    }
    auto fn = a.w == 2 ? k_expand_wide<RowU16> : a.w == 1 ? k_expand_wide<RowU8>
              : (m % 4) == 0 ? k_expand_wide<RowI32V> : k_expand_wide<RowI32>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<blocks > 0 ? blocks : 1, wpb * 32, smem, st>>>(a);
    return a.bcache ? 2 : 1;
  }
  const int ts = round4(m) + 4;  // tile row stride (words): 16-byte aligned, rotates banks
  const int B = (int)std::min<size_t>(32, std::max<size_t>(1, (32u << 10) / (4u * ts)));
  const size_t per_warp = expand_warp_bytes(m, B, ts);
  const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (100u << 10) / per_warp));
  const size_t smem = per_warp * wpb;
  const int per_sm = (int)std::max<size_t>(1, (220u << 10) / smem);
  // a task (run of candidates) of at least 8 tiles, and about two per warp of
  // the grid: each task pays one decode of its first block
  {
    const uint64_t two_per_warp = 2ull * nsm * per_sm * wpb;
    a.run = (uint32_t)std::max<uint64_t>(8ull * B, ((uint64_t)a.Q + two_per_warp - 1) / two_per_warp);
  }
  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  const int blocks = (int)std::min<uint64_t>((ntasks + wpb - 1) / wpb, (uint64_t)nsm * per_sm);
  auto fn = a.w == 2 ? k_expand<RowU16> : a.w == 1 ? k_expand<RowU8>
            : (m % 4) == 0 ? k_expand<RowI32V> : k_expand<RowI32>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  fn<<<blocks > 0 ? blocks : 1, wpb * 32, smem, st>>>(a, B, ts);
  return 1;
}

}  // namespace snp

// ---------------------------------------------------------------------------
// Batch engine: one launch runs depth d of every system of a batch.  A CTA
// takes systems from a work queue; for each it runs the whole depth with block
// barriers in place of the host: Psi of its frontier (Eq. psi), the saturating
// scan, then passes of up to qc candidates -- expand (the same warp code as
// k_expand), first-occurrence marks, ranks, commit -- until the frontier cap,
// the candidate budget or the candidates run out.

namespace snp {

namespace {

struct BatchScratch {
  uint64_t* psi;   // [pmax + 1]
  uint64_t* off;   // [pmax + 1]
  int32_t* staging;
  uint32_t *gmin, *slot_of, *srow, *own, *bits, *wbase;
  ChunkState* st;
  unsigned long long* hash;  // [qc] tensor-core form: linear hash of each candidate's row
  uint8_t* red;              // [qc] tensor-core form: the candidate repeats an earlier one
};

__device__ __forceinline__ BatchScratch batch_scratch(unsigned char* base, int64_t pmax, uint32_t qc, int m_max) {
  size_t at = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + at;
    at += (bytes + 255) & ~size_t(255);
    return p;
  };
  BatchScratch b;
  const int64_t npsi = (pmax + 1) > (int64_t)(qc / 32 + 1) ? (pmax + 1) : (int64_t)(qc / 32 + 1);
  b.psi = reinterpret_cast<uint64_t*>(take((size_t)npsi * 8));
  b.off = reinterpret_cast<uint64_t*>(take((pmax + 1) * 8));
  b.staging = reinterpret_cast<int32_t*>(take((size_t)qc * m_max * 4));
  b.gmin = reinterpret_cast<uint32_t*>(take(qc * 4));
  b.slot_of = reinterpret_cast<uint32_t*>(take(qc * 4));
  b.srow = reinterpret_cast<uint32_t*>(take(qc * 4));
  b.own = reinterpret_cast<uint32_t*>(take((qc / 32 + 1) * 4));
  b.bits = reinterpret_cast<uint32_t*>(take((qc / 32 + 1) * 4));
  b.wbase = reinterpret_cast<uint32_t*>(take((qc / 32 + 1) * 4));
  b.st = reinterpret_cast<ChunkState*>(take(sizeof(ChunkState)));
  b.hash = reinterpret_cast<unsigned long long*>(take((size_t)qc * 8));
  b.red = reinterpret_cast<uint8_t*>(take(qc));
  return b;
}

// Block-wide exclusive scan of v[0..n) in place (saturating u64), in tiles of blockDim.x.
__device__ void block_scan_sat(uint64_t* v, int64_t n, uint64_t* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  uint64_t carry = 0;
  for (int64_t t0 = 0; t0 < n; t0 += blockDim.x) {
    const int64_t i = t0 + tid;
    uint64_t inc = i < n ? v[i] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc = sat_add(y, inc);
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint64_t ws = lane < nw ? wsum[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws = sat_add(y, ws);
      }
      if (lane < nw) wsum[lane] = ws;
    }
    __syncthreads();
    const uint64_t before = sat_add(carry, warp > 0 ? wsum[warp - 1] : 0ull);
    uint64_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = 0;
    if (i < n) v[i] = sat_add(before, ex);
    const uint64_t tile_total = wsum[nw - 1];
    __syncthreads();
    carry = sat_add(carry, tile_total);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form of a batch pass (SNP_T_TC_F8): the rows of candidates
// g0 .. g0 + Q - 1 of the CTA's current system, C' = C_p + S . M_Pi
// (Eq. next-config) with the 0/1 spiking vector S of every firing neuron, by
// tcgen05.mma kind::f8f6f4 over tiles of 128 candidates (one thread and one
// TMEM lane per candidate), into the CTA's staging rows, with their linear
// hashes and repeat flags; the pass then resolves them like the sparse form.
// The MMA waits synchronously (the batch's CTAs overlap one another).

constexpr int kBtcSlots = 8;  // rule blocks of the left operand held at once

struct BatchTcSmem {
  uint8_t* A;          // [kBtcSlots][4096] left operand
  uint8_t* B;          // [kBtcSlots][128 * 32] M_Pi^T blocks of one 128-column chunk
  uint32_t* bitmap;    // [32] active rule blocks (at most 1024 blocks)
  uint16_t* slot_of;   // [1024]
  uint16_t* act;       // [1024]
  int* nact;
  unsigned long long* bars;  // operand arrival, MMA completion
  uint32_t* tmem_slot;
};

__host__ __device__ inline size_t batch_tc_smem_bytes() {
  return (size_t)kBtcSlots * t5::kT5ABytes * 2 + 32 * 4 + 1024 * 2 * 2 + 16 + 16 + 16 + 256;
}

__device__ __forceinline__ BatchTcSmem batch_tc_smem(unsigned char* raw) {
  unsigned char* p = reinterpret_cast<unsigned char*>(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  BatchTcSmem w;
  w.A = p;
  p += (size_t)kBtcSlots * t5::kT5ABytes;
  w.B = p;
  p += (size_t)kBtcSlots * t5::kT5ABytes;
  w.bitmap = reinterpret_cast<uint32_t*>(p);
  p += 32 * 4;
  w.slot_of = reinterpret_cast<uint16_t*>(p);
  p += 1024 * 2;
  w.act = reinterpret_cast<uint16_t*>(p);
  p += 1024 * 2;
  w.nact = reinterpret_cast<int*>(p);
  p += 16;
  w.bars = reinterpret_cast<unsigned long long*>(p);
  p += 16;
  w.tmem_slot = reinterpret_cast<uint32_t*>(p);
  return w;
}

// Chosen rule of every neuron of parent row prow for candidate t (last
// neuron least significant): f(rule or -1, mask, spikes, neuron).  Returns
// false if t is not a valid index.
template <typename F>
__device__ __forceinline__ bool batch_walk(const DevSys& s, const int32_t* prow, uint64_t t, F&& f) {
  uint64_t q = t;
  for (int n = s.m - 1; n >= 0; --n) {
    const int32_t x = prow[n];
    const uint32_t mask = (uint32_t)appl(s, n, x);
    if (!mask) {
      f(-1, 0u, x, n);
      continue;
    }
    const uint32_t radix = (uint32_t)__popc(mask);
    uint32_t d = 0;
    if (radix > 1) {
      d = (uint32_t)(q % radix);
      q /= radix;
    }
    f(__ldg(s.first_rule + n) + nth_set_bit(mask, (int)d), mask, x, n);
  }
  return q == 0;
}

// Rows of the pass by tensor core; returns false when an mbarrier wait ran
// out (the CTA then stops: products may still be in flight).
__device__ bool batch_tc_rows(const ClaimArgs& a, const BatchSys* bs, const BatchTcSmem& w, uint32_t tmem,
                              unsigned long long* hash, uint8_t* red_out, uint32_t& ph_b, uint32_t& ph_m) {
  using namespace t5;
  const DevSys& s = a.sys;
  const int m = s.m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = bs->np, nblocks = bs->nblocks;
  const int nbw = (nblocks + 31) / 32, nchunks = (np + kT5NC - 1) / kT5NC;
  const uint32_t bar_b = saddr(w.bars), bar_m = saddr(w.bars + 1);
  const uint32_t ntiles = (a.Q + kT5M - 1) / kT5M;
  for (uint32_t tile = 0; tile < ntiles; ++tile) {
    const uint32_t lid = tile * kT5M + tid;
    const bool valid = lid < a.Q;
    const uint64_t g = a.g0 + (valid ? lid : tile * kT5M);
    // parent: largest p with off[p] <= g
    int64_t lo = 0, hi = a.P;
    while (hi - lo > 1) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (__ldcg(a.off + mid) <= g) lo = mid;
      else hi = mid;
    }
    const int32_t* prow = a.parents + (size_t)lo * m;
    const uint64_t t = g - __ldcg(a.off + lo);
    for (int i = tid; i < nbw; i += kT5M) w.bitmap[i] = 0u;
    __syncthreads();
    uint64_t h = 0;
    bool red = false;
    if (valid) {
      const bool ok = batch_walk(s, prow, t, [&](int r, uint32_t mask, int32_t x, int n) {
        h += col_hash(s, n, x);
        if (r < 0) return;
        atomicOr(w.bitmap + (r >> 10), 1u << ((r >> 5) & 31));
        h += __ldg(s.rowkey + r);
        red |= redundant_choice(s, mask, r);
      });
      if (!ok) atomicOr(&a.st->error, kErrInternal);
      hash[lid] = h;
      red_out[lid] = red ? 1 : 0;
    }
    __syncthreads();
    if (warp == 0) {
      int cnt = 0;
      for (int b0 = 0; b0 < nblocks; b0 += 32) {
        const int bk = b0 + lane;
        const bool on = bk < nblocks && ((w.bitmap[bk >> 5] >> (bk & 31)) & 1u);
        const uint32_t bb = __ballot_sync(0xffffffffu, on);
        if (on) {
          const int pos = cnt + __popc(bb & ((1u << lane) - 1u));
          w.act[pos] = (uint16_t)bk;
          w.slot_of[bk] = (uint16_t)pos;
        }
        cnt += __popc(bb);
      }
      if (lane == 0) *w.nact = cnt;
    }
    __syncthreads();
    const int nact = *w.nact;
    const int ngroups = (nact + kBtcSlots - 1) / kBtcSlots;
    for (int nc = 0; nc < nchunks; ++nc) {
      const int c0 = nc * kT5NC, nc_cols = min(kT5NC, np - c0);
      for (int gi = 0; gi < ngroups; ++gi) {
        const int ga = gi * kBtcSlots, gb = min(nact, ga + kBtcSlots), gn = gb - ga;
        if (nc == 0 || ngroups > 1) {  // left operand of this group of blocks
          uint4* A4 = reinterpret_cast<uint4*>(w.A);
          for (int i = tid; i < gn * (kT5ABytes / 16); i += kT5M) A4[i] = make_uint4(0, 0, 0, 0);
          __syncthreads();
          if (valid)
            batch_walk(s, prow, t, [&](int r, uint32_t, int32_t, int) {
              if (r < 0) return;
              const int pos = w.slot_of[r >> 5];
              if (pos >= ga && pos < gb) w.A[(size_t)(pos - ga) * kT5ABytes + a_off(tid, r & 31)] = kF8PlusOne;
            });
          fence_async_smem();
          __syncthreads();
        }
        bool ok = true;
        if (tid == 0) {
          const uint32_t bytes = (uint32_t)nc_cols * kT5K;
          bar_expect_tx(bar_b, bytes * (uint32_t)gn);
          for (int k = 0; k < gn; ++k)
            bulk_g2s(saddr(w.B + (size_t)k * kT5ABytes), bs->MB + ((size_t)w.act[ga + k] * np + c0) * kT5K, bytes,
                     bar_b);
          ok = bar_wait(bar_b, ph_b);
          ph_b ^= 1u;
          fence_after_sync();
          const uint32_t id = idesc_f8(kT5M, nc_cols);
          for (int k = 0; k < gn; ++k)
            mma_f8(tmem, smem_desc(saddr(w.A + (size_t)k * kT5ABytes), 128, 256),
                   smem_desc(saddr(w.B + (size_t)k * kT5ABytes), 128, 256), id, (gi > 0 || k > 0) ? 1u : 0u);
          mma_commit(bar_m);
        }
        ok = bar_wait(bar_m, ph_m) && ok;
        ph_m ^= 1u;
        fence_after_sync();
        if (__syncthreads_or(!ok)) {
          if (tid == 0) atomicOr(&a.st->error, kErrTimeout);
          return false;
        }
      }
      // C' = C_p + D for this chunk's columns, to staging row lid
      const uint32_t acc = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c = 0; c < nc_cols; c += 32) {
        uint32_t r[32];
        const bool two = c + 32 <= nc_cols;
        if (nact == 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) r[i] = 0u;
        } else {
          if (two) tmem_ld32(acc + (uint32_t)c, r);
          else tmem_ld16(acc + (uint32_t)c, r);
          tmem_wait_ld();
        }
        const int j0 = c0 + c, cnt = min(two ? 32 : 16, m - j0);
        if (valid && !red) {
          int32_t* dst = a.staging + (size_t)lid * m + j0;
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (i < cnt) __stcg(dst + i, prow[j0 + i] + __float2int_rn(__uint_as_float(r[i])));
        }
      }
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
    }
  }
  return true;
}

}  // namespace

__global__ void k_batch_init(BatchSys* sys, const int32_t* c0, const int64_t* c0_off, int32_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    BatchSys& b = sys[i];
    const int m = b.sys.m;
    const int32_t* src = c0 + c0_off[i];
    for (int j = lane; j < m; j += 32) b.pool[j] = src[j];
    __syncwarp();
    const uint64_t h = fingerprint(b.sys, b.pool, lane);
    if (lane == 0) {
      const unsigned long long val = ((unsigned long long)fp32_of(h) << 32) | 0u;
      b.slots[(h & b.bmask) * kBucket] = val;  // the table is empty: first slot of its bucket
    }
  }
}

template <int kThreads, bool TC>
__global__ void __launch_bounds__(kThreads) k_batch_depth(BatchArgs ba) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned int s_next;
  __shared__ uint64_t s_wsum[kThreads / 32];
  __shared__ unsigned int s_cnt, s_stop, s_capped, s_last, s_broken;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kThreads / 32;
  BatchScratch sc = batch_scratch(ba.scratch + (size_t)blockIdx.x * ba.scratch_stride, ba.pmax, ba.qc, ba.m_max);
  // tensor-core form: operands in shared memory, 128 TMEM columns, two mbarriers
  BatchTcSmem tw{};
  uint32_t tmem = 0, ph_b = 0, ph_m = 0;
  if constexpr (TC) {
    tw = batch_tc_smem(smem_raw);
    if (tid == 0) {
      t5::bar_init(t5::saddr(tw.bars), 1);
      t5::bar_init(t5::saddr(tw.bars + 1), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_broken = 0;
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(t5::saddr(tw.tmem_slot)),
                   "r"((uint32_t)t5::kT5NC));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    t5::fence_before_sync();
    __syncthreads();
    t5::fence_after_sync();
    tmem = *tw.tmem_slot;
  }
  for (;;) {
    if (tid == 0) s_next = atomicAdd(ba.queue + ba.launch, 1u);
    __syncthreads();
    const int32_t si = (int32_t)s_next;
    __syncthreads();
    if (si >= ba.n) break;
    if constexpr (TC) {
      if (s_broken) break;
    }
    BatchSys* bs = ba.sys + si;
    const int32_t d = bs->cur_depth + 1;
    if (bs->done || d > bs->target_depth) continue;
    BatchDepthStat* stat = bs->stats + d;
    const int64_t cap = bs->cap, budget = bs->budget;
    const int32_t max_expand = bs->max_expand;
    const DevSys S = bs->sys;
    const int m = S.m;
    const int64_t P = bs->level_hi - bs->level_lo;
    const int32_t* parents = bs->pool + (size_t)bs->level_lo * m;
    if (tid == 0) {
      ChunkState z = {};
      *sc.st = z;
    }
    // step (a) and Psi, one thread per parent
    bool over = false;
    for (int64_t p = tid; p < P; p += kThreads) {
      const int32_t* row = parents + (size_t)p * m;
      uint64_t prod = 1;
      bool skip = false, ov = false;
      for (int n = 0; n < m; ++n) {
        const int32_t x = row[n];
        const bool small = (uint32_t)x < (uint32_t)kDirect;
        const uint32_t cnt = __popc(small ? __ldg(S.dmask + (size_t)n * kDirect + x) : (uint32_t)appl(S, n, x));
        if (cnt > 1) prod = __umul64hi(prod, cnt) ? kSat : prod * cnt;
        if (!small || !S.gain_small) ov |= x > INT32_MAX - __ldg(S.gain + n);
        skip |= max_expand >= 0 && x > max_expand;
      }
      sc.off[p] = skip ? 0ull : prod;
      over |= ov && !skip;
    }
    if (tid == 0) sc.off[P] = 0;
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(&bs->error, kErrOverflow);
    __threadfence();
    __syncthreads();
    block_scan_sat(sc.off, P + 1, s_wsum);
    __threadfence();
    __syncthreads();
    const uint64_t total = sc.off[P];
    const uint64_t T = budget > 0 ? min(total, (uint64_t)budget) : total;
    uint64_t remaining = cap > 0 ? (uint64_t)cap : ~0ull;
    uint64_t g0 = 0, examined = 0;
    int64_t nnew = 0, n_rows = bs->n_rows;
    int32_t chunks = 0;
    bool capped = false;
    ExpandSmem w = expand_smem(smem_raw + (size_t)warp * ba.warp_smem, m, ba.B, ba.ts);
    if (tid == 0) s_stop = bs->error ? 1u : 0u;
    __syncthreads();
    while (g0 < T && !capped && !s_stop) {
      const uint32_t Q = (uint32_t)min((uint64_t)ba.qc, T - g0);
      ClaimArgs a;
      a.sys = S;
      a.parents = parents;
      a.off = sc.off;
      a.P = P;
      a.g0 = g0;
      a.Q = Q;
      a.run = (uint32_t)ba.run;
      a.table = DevTable{bs->slots, bs->bmask};
      a.pool = bs->pool;
      a.staging = sc.staging;
      a.gmin = sc.gmin;
      a.slot_of = sc.slot_of;
      a.ownbits = sc.own;
      a.prec = nullptr;
      a.ctr = nullptr;
      a.pperm = nullptr;
      a.store_ctr = nullptr;
      a.sidx_of = nullptr;
      a.store_cap = 0;
      a.st = sc.st;
      if constexpr (TC) {
        if (!batch_tc_rows(a, bs, tw, tmem, sc.hash, sc.red, ph_b, ph_m)) {
          if (tid == 0) {
            s_broken = 1;
            atomicOr(&bs->error, kErrTimeout);
          }
          __syncthreads();
          break;
        }
        __threadfence();
        __syncthreads();
        // step (d) for the pass's rows, 32 candidates per warp at a time
        for (uint32_t b0 = (uint32_t)warp * 32u; b0 < Q; b0 += (uint32_t)nwarps * 32u) {
          const uint32_t lid = b0 + (uint32_t)lane;
          const bool todo = lid < Q && !sc.red[lid];
          const uint64_t key = todo ? mix64(sc.hash[lid]) : 0ull;
          const int32_t* row = sc.staging + (size_t)(lid < Q ? lid : 0) * m;
          if ((m & 3) == 0)
            resolve_warp<RowI32V, 1>(a, row, key, lid, todo);
          else
            resolve_warp<RowI32, 1>(a, row, key, lid, todo);
        }
      } else {
        if ((m & 3) == 0)
          expand_warp<RowI32V, 1>(a, ba.B, ba.ts, w, warp, nwarps, lane);
        else
          expand_warp<RowI32, 1>(a, ba.B, ba.ts, w, warp, nwarps, lane);
      }
      __threadfence();
      __syncthreads();
      // first-occurrence marks
      const uint32_t nwords = (Q + 31) / 32;
      if (tid == 0) s_cnt = 0;
      __syncthreads();
      uint32_t cnt = 0;
      for (uint32_t wd = tid; wd < nwords; wd += kThreads) {
        uint32_t word = sc.own[wd];
        if (!word) continue;
        sc.own[wd] = 0;
        cnt += __popc(word);
        while (word) {
          const uint32_t o = wd * 32u + (uint32_t)(__ffs(word) - 1);
          word &= word - 1;
          const uint32_t f = o < Q ? sc.gmin[o] : 0xFFFFFFFFu;
          if (f >= Q) {  // not a claim of this pass: record and skip
            atomicOr(&sc.st->error, kErrInternal);
            continue;
          }
          atomicOr(sc.bits + (f >> 5), 1u << (f & 31));
          sc.srow[f] = o;
        }
      }
      if (cnt) atomicAdd(&s_cnt, cnt);
      __threadfence();
      __syncthreads();
      const uint32_t n_alloc = s_cnt;
      // ranks: exclusive scan of the words' popcounts
      uint64_t* ranks = sc.psi;
      for (uint32_t wd = tid; wd < nwords; wd += kThreads) ranks[wd] = __popc(__ldcg(sc.bits + wd));
      __syncthreads();
      block_scan_sat(ranks, nwords, s_wsum);
      __threadfence();
      __syncthreads();
      // commit: warp per word, lane per set bit
      const uint64_t accept = remaining;
      for (uint32_t wd = warp; wd < nwords; wd += nwarps) {
        const uint32_t word = __ldcg(sc.bits + wd);
        if (!((word >> lane) & 1u)) continue;
        const uint32_t lid = wd * 32u + (uint32_t)lane;
        const uint64_t rank = __ldcg(ranks + wd) + __popc(word & ((1u << lane) - 1u));
        const uint32_t o = __ldcg(sc.srow + lid);
        unsigned long long* slot = bs->slots + __ldcg(sc.slot_of + o);
        const unsigned long long hi = (*slot) & 0xFFFFFFFF00000000ull;
        if (rank < accept) {
          const int64_t row = n_rows + (int64_t)rank;
          const int32_t* src = sc.staging + (size_t)o * m;
          int32_t* dst = bs->pool + (size_t)row * m;
          copy_row_cg(src, dst, m);
          *slot = hi | (uint32_t)row;
          if (rank + 1 == accept) {
            sc.st->capped = 1;
            sc.st->last_lid = lid;
          }
        } else {
          *slot = hi | kRowTomb;
        }
      }
      __threadfence();
      __syncthreads();
      const uint64_t acc = min((uint64_t)n_alloc, accept);
      nnew += (int64_t)acc;
      n_rows += (int64_t)acc;
      if (remaining != ~0ull) remaining -= acc;
      if (tid == 0) {
        s_capped = sc.st->capped;
        s_last = sc.st->last_lid;
        if (sc.st->error) atomicOr(&bs->error, sc.st->error);
        s_stop = bs->error ? 1u : 0u;
      }
      for (uint32_t wd = tid; wd < nwords; wd += kThreads) sc.bits[wd] = 0;
      __threadfence();
      __syncthreads();
      capped = s_capped != 0;
      examined = capped ? g0 + s_last + 1 : g0 + Q;
      g0 += Q;
      ++chunks;
    }
    __syncthreads();
    if (tid == 0) {
      stat->new_configs = nnew;
      stat->examined = (int64_t)examined;
      stat->candidates = total;
      stat->truncated = examined < total ? 1 : 0;
      stat->chunks = chunks;
      bs->n_rows = n_rows;
      bs->cur_depth = d;
      if (nnew == 0) {
        bs->done = 1;
      } else {
        bs->depth_reached = d;
        bs->level_lo = bs->level_hi;
        bs->level_hi = n_rows;
      }
    }
    __syncthreads();
  }
  if constexpr (TC) {
    // products of a pass whose wait ran out may still be in flight
    if (s_broken && tid == 0) (void)t5::bar_wait(t5::saddr(tw.bars + 1), ph_m ^ 1u);
    t5::fence_before_sync();
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)t5::kT5NC));
  }
}

size_t batch_tc_smem_bytes_host() { return batch_tc_smem_bytes() + 1024; }

size_t batch_scratch_bytes(int64_t pmax, uint32_t qc, int m_max) {
  auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
  return r((size_t)std::max<int64_t>(pmax + 1, qc / 32 + 1) * 8) + r((pmax + 1) * 8) + r((size_t)qc * m_max * 4) +
         3 * r(qc * 4) + 3 * r((qc / 32 + 1) * 4) +
         r(sizeof(ChunkState)) + r((size_t)qc * 8) + r(qc);
}

size_t expand_smem_bytes(int m_max, int B, int* ts) {
  *ts = round4(m_max) + 4;
  return expand_warp_bytes(m_max, B, *ts);
}

void launch_batch_depth(const BatchArgs& a, int blocks, int warps, cudaStream_t st) {
  if (a.tc) {  // four warps: the 128 TMEM lanes of a tile
    const size_t smem = batch_tc_smem_bytes_host();
    cudaFuncSetAttribute(k_batch_depth<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_depth<128, true><<<blocks, 128, smem, st>>>(a);
    return;
  }
  const size_t smem = a.warp_smem * warps;
  if (warps == 4) {
    cudaFuncSetAttribute(k_batch_depth<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_depth<128, false><<<blocks, 128, smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_batch_depth<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_depth<256, false><<<blocks, 256, smem, st>>>(a);
  }
}

}  // namespace snp
