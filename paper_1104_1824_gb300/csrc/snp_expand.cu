// The expand kernel: steps (b), (c) and (d) for one chunk of candidates.
//
// A warp takes a run of consecutive candidates of one parent (spiking-vector
// indices t0, t0 + 1, ...).  It keeps a base: the digits of t0 in the mixed
// radix of the per-neuron choice counts (Eq. psi; last neuron least
// significant), the child C' = C + S . M_Pi of t0 (Eq. next-config) and its
// linear hash.  A batch of up to 32 candidates is then built lane-parallel:
// lane k adds k to the base's digits (only the few least significant
// non-trivial neurons change), copies the base row into its own tile row and
// swaps the changed neurons' rows of M_Pi (hash: swaps their H[r]).  Lane k
// then resolves its row: it probes the hash table, compares full keys, and
// either finds the key (seen before, or staged earlier in this chunk: then it
// lowers that key's first-occurrence index) or claims an empty slot, stages
// its row and publishes the slot.  The base then moves on by the batch size.
#include "snp_kernels.cuh"

namespace snp {

namespace {

constexpr int kLowDigits = 16;  // least significant non-trivial neurons tracked per parent

struct ExpandSmem {
  int32_t* tile;              // [B][ts] rows of candidates waiting for a lookup
  unsigned long long* keys;   // [B] their table keys
  uint32_t* lids;             // [B] their chunk-local indices
  int32_t* par;               // [m4] parent
  int32_t* buf;               // [m4] base child
  uint32_t* msk;              // [m4] applicable-rule masks
  uint8_t* dig;               // [m4] base digits
  int32_t* low;               // [kLowDigits] least significant non-trivial neurons, least first
  int* nlow;                  // [1] entries of low
  uint32_t* plow;             // [1] product of their choice counts (capped at 2^31)
  uint32_t* vlow;             // [1] value of the base's digits on them (< plow)
  unsigned long long* hbase;  // [1] linear hash of the base child
  int* nred;                  // [1] neurons of the base that use a redundant rule (a later duplicate)
};

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

__host__ __device__ inline size_t expand_keys_bytes(int B) { return ((size_t)B * 12 + 15) & ~size_t(15); }

__host__ __device__ inline size_t expand_warp_bytes(int m, int B, int ts) {
  const int m4 = round4(m);
  size_t b = (size_t)B * ts * 4 + expand_keys_bytes(B) + (size_t)m4 * 12 + 96 + (size_t)m4;
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

__device__ __forceinline__ void add_row_shared(const DevSys& s, int32_t* row, int r, int sign) {
  const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
  for (int e = e0; e < e1; ++e) {
    const int2 cv = __ldg(s.csr + e);
    atomicAdd(&row[cv.x], sign * cv.y);
  }
}

// Step (a) for the parent row: masks, the list of the least significant
// non-trivial neurons, and the mixed-radix place value of the neurons owned by
// later lanes (neuron 0 most significant).
__device__ __forceinline__ uint64_t parent_state(const DevSys& s, const int32_t* __restrict__ row, ExpandSmem& w,
                                                 int lane) {
  __syncwarp();
  for (int n = lane; n < s.m; n += 32) w.par[n] = row[n];
  __syncwarp();
  uint64_t prod = 1;
  const int n0 = lane * s.K, n1 = min(n0 + s.K, s.m);
  for (int n = n0; n < n1; ++n) {
    const int32_t x = w.par[n];
    const int r0 = __ldg(s.first_rule + n), r1 = __ldg(s.first_rule + n + 1);
    uint32_t mask = 0;
    for (int r = r0; r < r1; ++r)
      if (rule_applies(x, __ldg(s.rule + r))) mask |= 1u << (r - r0);
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
  // least significant non-trivial neurons, scanning 32 neurons at a time from the end
  int count = 0;
  for (int top = s.m - 1; top >= 0 && count < kLowDigits; top -= 32) {
    const int n = top - lane;
    const bool nt = n >= 0 && __popc(w.msk[n]) > 1;
    const uint32_t b = __ballot_sync(0xffffffffu, nt);
    const int rank = __popc(b & ((1u << lane) - 1u));
    if (nt && count + rank < kLowDigits) w.low[count + rank] = n;
    count += __popc(b);
  }
  if (lane == 0) {
    const int nl = min(count, kLowDigits);
    uint64_t pl = 1;
    for (int i = 0; i < nl; ++i) {
      pl *= (uint64_t)__popc(w.msk[w.low[i]]);
      if (pl > (1ull << 31)) pl = 1ull << 31;
    }
    *w.nlow = nl;
    *w.plow = (uint32_t)pl;
  }
  __syncwarp();
  return lane == 31 ? 1ull : a;
}

// The base becomes candidate t of the loaded parent: digits, child, hash.
__device__ __forceinline__ void decode_full(const DevSys& s, ExpandSmem& w, uint64_t t, uint64_t after, int lane) {
  for (int n = lane; n < s.m; n += 32) w.buf[n] = w.par[n];
  uint64_t hp = 0;
  for (int n = lane; n < s.m; n += 32) hp += col_hash(s, n, w.par[n]);
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
    add_row_shared(s, w.buf, r, 1);
    hp += __ldg(s.rowkey + r);
    red += redundant_choice(s, mask, r) ? 1 : 0;
  }
  hp = warp_sum_u64(hp);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) red += __shfl_xor_sync(0xffffffffu, red, o);
  __syncwarp();
  if (lane == 0) {
    *w.hbase = hp;
    *w.nred = red;
    uint64_t v = 0, place = 1;
    for (int i = 0; i < *w.nlow && place < (1ull << 31); ++i) {
      const int n = w.low[i];
      v += place * w.dig[n];
      place *= __popc(w.msk[n]);
    }
    const uint64_t cap = (uint64_t)*w.plow - 1;
    *w.vlow = (uint32_t)(v < cap ? v : cap);
  }
  __syncwarp();
}

// Adds k to the base digits of the low neurons (k < the product of their
// radices); calls f(neuron, old digit, new digit) for each changed one.
template <typename F>
__device__ __forceinline__ void add_to_digits(const ExpandSmem& w, uint32_t k, F&& f) {
  const int nl = *w.nlow;
  for (int i = 0; i < nl && k; ++i) {
    const int n = w.low[i];
    const uint32_t r = __popc(w.msk[n]);
    const uint32_t d = w.dig[n];
    const uint32_t sum = d + k;
    const uint32_t nd = sum % r;
    k = sum / r;
    if (nd != d) f(n, (int)d, (int)nd);
  }
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
template <bool VEC>
__device__ __forceinline__ bool row_equal_lane(const int32_t* row, const int32_t* other, int m) {
  if (VEC) {
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
  }
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

template <bool VEC>
__device__ __forceinline__ void stage_row_lane(const int32_t* row, int32_t* dst, int m) {
  if (VEC) {
    const int4* a = reinterpret_cast<const int4*>(row);
    int4* b = reinterpret_cast<int4*>(dst);
    for (int j = 0; j < (m >> 2); ++j) __stcg(b + j, a[j]);
    return;
  }
  for (int j = 0; j < m; ++j) __stcg(dst + j, row[j]);
}

// Step (d) for one candidate, by one lane, without waiting on any other lane:
// returns false when the key may sit in a slot that another lane or warp has
// reserved but not yet published; the caller then tries again in a later pass.
template <bool VEC>
__device__ __forceinline__ bool resolve_lane(const ClaimArgs& a, const int32_t* row, uint64_t key, uint32_t lid) {
  const int m = a.sys.m;
  const uint32_t fp = fp32_of(key);
  uint64_t bucket = key & a.table.bmask;
  for (uint64_t probes = 0; probes <= a.table.bmask; ++probes, bucket = (bucket + 1) & a.table.bmask) {
    unsigned long long* bs = a.table.slots + bucket * kBucket;
    unsigned long long v[kBucket];
    const ulonglong2* b2 = reinterpret_cast<const ulonglong2*>(bs);
#pragma unroll
    for (int q = 0; q < kBucket / 2; ++q) {
      const ulonglong2 x = __ldcg(b2 + q);
      v[2 * q] = x.x;
      v[2 * q + 1] = x.y;
    }
#pragma unroll
    for (int j = 0; j < kBucket; ++j) {
      unsigned long long x = v[j];
      for (;;) {  // until slot j holds a key that is not ours, or we are done
        if (x == kEmpty) {
          const unsigned long long old = atomicCAS(bs + j, kEmpty, ((unsigned long long)fp << 32) | kRowReserved);
          if (old == kEmpty) {  // owner: stage, record, publish
            stage_row_lane<VEC>(row, a.staging + (size_t)lid * m, m);
            a.gmin[lid] = lid;
            a.slot_of[lid] = (uint32_t)(bucket * kBucket + j);
            atomicOr(a.ownbits + (lid >> 5), 1u << (lid & 31));
            st_release(bs + j, ((unsigned long long)fp << 32) | (kPending | lid));
            return true;
          }
          x = old;  // someone else took the slot: look at what is there now
          continue;
        }
        const uint32_t rf = (uint32_t)x;
        if ((uint32_t)(x >> 32) != fp || rf == kRowTomb) break;
        if (rf == kRowReserved) return false;  // published soon: try again later
        const int32_t* other;
        if (rf & kPending) {
          (void)ld_acquire(bs + j);  // orders the staged row's reads after the publish
          other = a.staging + (size_t)(rf & ~kPending) * m;
        } else {
          other = a.pool + (size_t)rf * m;
        }
        if (row_equal_lane<VEC>(row, other, m)) {
          if (rf & kPending) atomicMin(a.gmin + (rf & ~kPending), lid);
          return true;
        }
        break;
      }
    }
  }
  atomicOr(&a.st->error, kErrTableFull);
  return true;
}

// Step (d) for the fill (<= 32) rows waiting in the tile, one per lane:
// passes until every row is resolved; a lane never waits inside a pass, so
// owners in this warp publish before anyone looks again.
template <bool VEC>
__device__ __forceinline__ void flush_tile(const ClaimArgs& a, ExpandSmem& w, int ts, int fill, int lane) {
  bool todo = lane < fill;
  for (int pass = 0;; ++pass) {
    if (todo && resolve_lane<VEC>(a, w.tile + lane * ts, w.keys[lane], w.lids[lane])) todo = false;
    if (__all_sync(0xffffffffu, !todo)) break;
    if (pass >= kSpinLimit) {
      if (todo) atomicOr(&a.st->error, kErrTimeout);
      break;
    }
    __nanosleep(32);
  }
  __syncwarp();
}

// Per-warp shared memory of the expand loop.
__device__ __forceinline__ ExpandSmem expand_smem(unsigned char* base, int m, int B, int ts) {
  const int m4 = round4(m);
  ExpandSmem w;
  w.tile = reinterpret_cast<int32_t*>(base);
  w.keys = reinterpret_cast<unsigned long long*>(w.tile + (size_t)B * ts);
  w.lids = reinterpret_cast<uint32_t*>(w.keys + B);
  w.par = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(w.keys) + expand_keys_bytes(B));
  w.buf = w.par + m4;
  w.msk = reinterpret_cast<uint32_t*>(w.buf + m4);
  w.low = reinterpret_cast<int32_t*>(w.msk + m4);               // 64 bytes
  w.nlow = w.low + kLowDigits;                                    // +64
  w.plow = reinterpret_cast<uint32_t*>(w.low + kLowDigits + 1);   // +68
  w.vlow = reinterpret_cast<uint32_t*>(w.low + kLowDigits + 2);   // +72
  w.hbase = reinterpret_cast<unsigned long long*>(w.low + kLowDigits + 4);  // +80
  w.nred = w.low + kLowDigits + 6;                                // +88
  w.dig = reinterpret_cast<uint8_t*>(w.low) + 96;
  return w;
}

// Steps (b)-(d) for the tasks task0, task0 + tstride, ... of chunk a (a task
// is a run of a.run consecutive candidates), by one warp.
template <bool VEC>
__device__ __forceinline__ void expand_warp(const ClaimArgs& a, int B, int ts, ExpandSmem& w, uint64_t task0,
                                            uint64_t tstride, int lane) {
  const DevSys& s = a.sys;
  const int m = s.m;
  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  for (uint64_t task = task0; task < ntasks; task += tstride) {
    const uint64_t la = task * a.run;
    const uint64_t lb = min(la + a.run, (uint64_t)a.Q);
    int64_t p = warp_find_parent(a.off, a.P, a.g0 + la, lane);
    uint64_t p_lo = __ldcg(a.off + p), p_hi = __ldcg(a.off + p + 1);
    if (task == 0 && lane == 0) a.st->p_first = (unsigned long long)p;
    uint64_t after = parent_state(s, a.parents + (size_t)p * m, w, lane);
    decode_full(s, w, a.g0 + la - p_lo, after, lane);
    uint64_t l = la;
    int fill = 0;  // rows waiting in the tile
    while (l < lb) {
      const uint64_t g = a.g0 + l;
      // a batch never crosses a parent, nor a rollover of the tracked low digits
      const uint32_t room = *w.plow - *w.vlow;
      const int nb = (int)min(min(min((uint64_t)B, lb - l), p_hi - g), (uint64_t)room);
      if (nb <= 0) {  // cannot happen: every bound above is positive
        if (lane == 0) atomicOr(&a.st->error, kErrInternal);
        break;
      }
      // a candidate using a redundant rule repeats an earlier one: no lookup needed
      bool keep = false;
      if (lane < nb) {
        int red = *w.nred;
        add_to_digits(w, (uint32_t)lane, [&](int n, int d, int nd) {
          const uint32_t mask = w.msk[n];
          red += (redundant_choice(s, mask, rule_of(s, w, n, nd)) ? 1 : 0) -
                 (redundant_choice(s, mask, rule_of(s, w, n, d)) ? 1 : 0);
        });
        keep = red == 0;
      }
      const uint32_t kept = __ballot_sync(0xffffffffu, keep);
      if (fill + __popc(kept) > B) {  // no room for this batch's rows: resolve what waits
        flush_tile<VEC>(a, w, ts, fill, lane);
        fill = 0;
      }
      if (keep) {  // build the row in the next free tile slot
        const int slot = fill + __popc(kept & ((1u << lane) - 1u));
        int32_t* trow = w.tile + slot * ts;
        copy_row<VEC>(w.buf, trow, m);
        uint64_t h = *w.hbase;
        add_to_digits(w, (uint32_t)lane, [&](int n, int d, int nd) {
          const int r_old = rule_of(s, w, n, d), r_new = rule_of(s, w, n, nd);
          add_row_private(s, trow, r_old, -1);
          add_row_private(s, trow, r_new, 1);
          h += __ldg(s.rowkey + r_new) - __ldg(s.rowkey + r_old);
        });
        w.keys[slot] = mix64(h);
        w.lids[slot] = (uint32_t)(l + lane);
      }
      fill += __popc(kept);
      __syncwarp();
      if (fill >= B || l + nb >= lb) {
        flush_tile<VEC>(a, w, ts, fill, lane);
        fill = 0;
      }
      l += nb;
      if (l >= lb) break;
      const uint64_t gn = a.g0 + l;
      if (gn >= p_hi) {  // next parent
        do {
          ++p;
          p_lo = p_hi;
          p_hi = __ldcg(a.off + p + 1);
        } while (gn >= p_hi);
        after = parent_state(s, a.parents + (size_t)p * m, w, lane);
        decode_full(s, w, gn - p_lo, after, lane);
      } else if ((uint32_t)nb == room) {  // the low digits roll over: decode in full
        decode_full(s, w, gn - p_lo, after, lane);
      } else {  // same parent: the base moves on by nb
        if (lane == 0) {
          uint64_t h = *w.hbase;
          int red = *w.nred;
          add_to_digits(w, (uint32_t)nb, [&](int n, int d, int nd) {
            const int r_old = rule_of(s, w, n, d), r_new = rule_of(s, w, n, nd);
            add_row_private(s, w.buf, r_old, -1);
            add_row_private(s, w.buf, r_new, 1);
            h += __ldg(s.rowkey + r_new) - __ldg(s.rowkey + r_old);
            red += (redundant_choice(s, w.msk[n], r_new) ? 1 : 0) - (redundant_choice(s, w.msk[n], r_old) ? 1 : 0);
            w.dig[n] = (uint8_t)nd;
          });
          *w.hbase = h;
          *w.nred = red;
          *w.vlow += (uint32_t)nb;
        }
        __syncwarp();
      }
    }
    if (task + 1 == ntasks && lane == 0) a.st->p_last = (unsigned long long)p;
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256, 2) k_expand(ClaimArgs a, int B, int ts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  ExpandSmem w = expand_smem(smem_raw + (size_t)wib * expand_warp_bytes(a.sys.m, B, ts), a.sys.m, B, ts);
  expand_warp<VEC>(a, B, ts, w, (uint64_t)blockIdx.x * wpb + wib, (uint64_t)gridDim.x * wpb, lane);
}

// Step (d) for rows already built in global memory (the tensor-core form):
// one lane per candidate, the same bounded wait-free passes as k_expand.
template <bool VEC>
__global__ void __launch_bounds__(256) k_resolve_rows(ClaimArgs a, const int32_t* rows,
                                                      const unsigned long long* hash, const uint8_t* redundant) {
  const int m = a.sys.m;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < a.Q; base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t lid = base + threadIdx.x;
    bool done = lid >= a.Q || redundant[lid];
    const uint64_t key = done ? 0ull : mix64(hash[lid]);
    for (int pass = 0;; ++pass) {
      if (!done) done = resolve_lane<VEC>(a, rows + lid * m, key, (uint32_t)lid);
      if (__all_sync(0xffffffffu, done)) break;
      if (pass >= kSpinLimit) {
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
    k_resolve_rows<true><<<blocks, 256, 0, st>>>(a, rows, hash, redundant);
  else
    k_resolve_rows<false><<<blocks, 256, 0, st>>>(a, rows, hash, redundant);
}

int launch_expand(ClaimArgs a, cudaStream_t st, int nsm) {
  const int m = a.sys.m;
  const int ts = round4(m) + 4;  // tile row stride (words): 16-byte aligned, rotates banks
  const int B = (int)std::min<size_t>(32, std::max<size_t>(1, (32u << 10) / (4u * ts)));
  const size_t per_warp = expand_warp_bytes(m, B, ts);
  const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (100u << 10) / per_warp));
  const size_t smem = per_warp * wpb;
  a.run = (uint32_t)(8 * B);
  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  const int per_sm = (int)std::max<size_t>(1, (220u << 10) / smem);
  const int blocks = (int)std::min<uint64_t>((ntasks + wpb - 1) / wpb, (uint64_t)nsm * per_sm);
  const bool vec = (m % 4) == 0;
  auto fn = vec ? k_expand<true> : k_expand<false>;
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

template <int kThreads>
__global__ void __launch_bounds__(kThreads) k_batch_depth(BatchArgs ba) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned int s_next;
  __shared__ uint64_t s_wsum[kThreads / 32];
  __shared__ unsigned int s_cnt, s_stop, s_capped, s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kThreads / 32;
  BatchScratch sc = batch_scratch(ba.scratch + (size_t)blockIdx.x * ba.scratch_stride, ba.pmax, ba.qc, ba.m_max);
  for (;;) {
    if (tid == 0) s_next = atomicAdd(ba.queue + ba.launch, 1u);
    __syncthreads();
    const int32_t si = (int32_t)s_next;
    __syncthreads();
    if (si >= ba.n) return;
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
      int r = __ldg(S.first_rule);
      for (int n = 0; n < m; ++n) {
        const int32_t x = row[n];
        const int r1 = __ldg(S.first_rule + n + 1);
        uint32_t cnt = 0;
        for (; r < r1; ++r) cnt += rule_applies(x, __ldg(S.rule + r)) ? 1u : 0u;
        if (cnt > 1) prod = __umul64hi(prod, cnt) ? kSat : prod * cnt;
        ov |= x > INT32_MAX - __ldg(S.gain + n);
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
      a.st = sc.st;
      if ((m & 3) == 0)
        expand_warp<true>(a, ba.B, ba.ts, w, warp, nwarps, lane);
      else
        expand_warp<false>(a, ba.B, ba.ts, w, warp, nwarps, lane);
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
          for (int j = 0; j < m; ++j) dst[j] = __ldcg(src + j);
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
}

size_t batch_scratch_bytes(int64_t pmax, uint32_t qc, int m_max) {
  auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
  return r((size_t)std::max<int64_t>(pmax + 1, qc / 32 + 1) * 8) + r((pmax + 1) * 8) + r((size_t)qc * m_max * 4) +
         3 * r(qc * 4) + 3 * r((qc / 32 + 1) * 4) +
         r(sizeof(ChunkState));
}

size_t expand_smem_bytes(int m_max, int B, int* ts) {
  *ts = round4(m_max) + 4;
  return expand_warp_bytes(m_max, B, *ts);
}

void launch_batch_depth(const BatchArgs& a, int blocks, int warps, cudaStream_t st) {
  const size_t smem = a.warp_smem * warps;
  if (warps == 4) {
    cudaFuncSetAttribute(k_batch_depth<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_depth<128><<<blocks, 128, smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_batch_depth<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_depth<256><<<blocks, 256, smem, st>>>(a);
  }
}

}  // namespace snp
