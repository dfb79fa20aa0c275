// The expand kernel: steps (b), (c) and (d) for one chunk of candidates.
//
// A warp takes a run of consecutive candidates (parent p, spiking-vector
// indices t, t+1, ...).  It decodes the first index in full (mixed radix of
// the per-neuron choice counts, Eq. psi, last neuron least significant) and
// builds C' = C + S . M_Pi (Eq. next-config) in shared memory.  Each following
// index is one increment of that mixed-radix counter: only the neurons whose
// digit changes (on average fewer than two) swap the old rule's row of M_Pi
// for the new rule's row, so C' is updated, not rebuilt.  Each candidate's C'
// is copied to a per-warp tile row with its fingerprint.  Every batch of up to
// 32 tile rows is then resolved lane-parallel: lane k probes the hash table
// for row k, compares full keys, and either finds the key (seen before, or
// staged earlier in this chunk: then it lowers that key's first-occurrence
// index) or claims an empty slot, stages its row and publishes the slot.
#include "snp_kernels.cuh"

namespace snp {

namespace {

struct ExpandSmem {
  int32_t* tile;              // [B][ts] candidate rows
  unsigned long long* hk;     // [B] fingerprints
  int32_t* par;               // [m4] parent
  int32_t* buf;               // [m4] current child
  uint32_t* msk;              // [m4] applicable-rule masks
  uint8_t* dig;               // [m4] current digit per neuron
};

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

__host__ __device__ inline size_t expand_warp_bytes(int m, int B, int ts) {
  const int m4 = round4(m);
  size_t b = (size_t)B * ts * 4 + (size_t)B * 8 + (size_t)m4 * 12 + (size_t)m4;
  return (b + 15) & ~size_t(15);
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void apply_row(const DevSys& s, int32_t* buf, int r, int sign) {
  const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
  for (int e = e0; e < e1; ++e) {
    const int2 cv = __ldg(s.csr + e);
    atomicAdd(&buf[cv.x], sign * cv.y);
  }
}

// Step (a) for the parent row: masks and the mixed-radix place value of the
// neurons owned by later lanes (neuron 0 most significant).
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
  return lane == 31 ? 1ull : a;
}

// Decodes index t in full and builds C' = C + S . M_Pi in w.buf.
__device__ __forceinline__ void decode_full(const DevSys& s, ExpandSmem& w, uint64_t t, uint64_t after, int lane) {
  for (int n = lane; n < s.m; n += 32) w.buf[n] = w.par[n];
  __syncwarp();
  const int n0 = lane * s.K, n1 = min(n0 + s.K, s.m);
  uint64_t q = (after > t) ? 0ull : t / after;
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
    apply_row(s, w.buf, __ldg(s.first_rule + n) + nth_set_bit(mask, (int)d), 1);
  }
  __syncwarp();
}

// Index t -> t + 1 (t + 1 < Psi): the carry enters at the last neuron; lanes
// whose non-trivial digits are all at their maximum pass it on and wrap.
__device__ __forceinline__ void step_one(const DevSys& s, ExpandSmem& w, int lane) {
  const int n0 = lane * s.K, n1 = min(n0 + s.K, s.m);
  bool full = true;
  for (int n = n0; n < n1; ++n) {
    const int r = __popc(w.msk[n]);
    if (r > 1 && w.dig[n] != r - 1) full = false;
  }
  const uint32_t stop = __ballot_sync(0xffffffffu, !full);
  const int L = 31 - __clz(stop);
  if (lane >= L) {
    for (int n = n1 - 1; n >= n0; --n) {
      const uint32_t mask = w.msk[n];
      const int r = __popc(mask);
      if (r <= 1) continue;
      const int d = w.dig[n];
      const int nd = (d == r - 1) ? 0 : d + 1;
      const int base = __ldg(s.first_rule + n);
      apply_row(s, w.buf, base + nth_set_bit(mask, d), -1);
      apply_row(s, w.buf, base + nth_set_bit(mask, nd), 1);
      w.dig[n] = (uint8_t)nd;
      if (nd != 0) break;  // the increment is absorbed here
    }
  }
  __syncwarp();
}

template <bool VEC>
__device__ __forceinline__ bool row_equal_lane(const int32_t* row, const int32_t* other, int m) {
  if (VEC) {
    const int4* a = reinterpret_cast<const int4*>(row);
    const int4* b = reinterpret_cast<const int4*>(other);
    for (int j = 0; j < (m >> 2); ++j) {
      const int4 x = a[j], y = __ldcg(b + j);
      if (x.x != y.x || x.y != y.y || x.z != y.z || x.w != y.w) return false;
    }
    return true;
  }
  for (int j = 0; j < m; ++j)
    if (row[j] != __ldcg(other + j)) return false;
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

// Step (d) for one candidate, by one lane, independently of the other lanes
// (no warp-collective operation, so a lane may wait on another lane's slot).
template <bool VEC>
__device__ __forceinline__ void resolve_lane(const ClaimArgs& a, const int32_t* row, uint64_t h, uint32_t lid) {
  const int m = a.sys.m;
  const uint32_t fp = fp32_of(h);
  uint64_t bucket = h & a.table.bmask;
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
            return;
          }
          x = old;  // someone else took the slot: look at what is there now
          continue;
        }
        const uint32_t rf = (uint32_t)x;
        if ((uint32_t)(x >> 32) != fp || rf == kRowTomb) break;
        if (rf == kRowReserved) {  // claimed but not yet published: bounded wait
          int spins = 0;
          do {
            x = ld_acquire(bs + j);
            if ((uint32_t)x != kRowReserved) break;
            __nanosleep(64);
          } while (++spins < kSpinLimit);
          if ((uint32_t)x == kRowReserved) {
            atomicOr(&a.st->error, kErrTimeout);
            return;
          }
          continue;
        }
        const int32_t* other;
        if (rf & kPending) {
          (void)ld_acquire(bs + j);  // orders the staged row's reads after the publish
          other = a.staging + (size_t)(rf & ~kPending) * m;
        } else {
          other = a.pool + (size_t)rf * m;
        }
        if (row_equal_lane<VEC>(row, other, m)) {
          if (rf & kPending) atomicMin(a.gmin + (rf & ~kPending), lid);
          return;
        }
        break;
      }
    }
  }
  atomicOr(&a.st->error, kErrTableFull);
}

template <bool VEC>
__global__ void __launch_bounds__(256, 1) k_expand(ClaimArgs a, int B, int ts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const DevSys& s = a.sys;
  const int m = s.m, m4 = round4(m);
  ExpandSmem w;
  unsigned char* base = smem_raw + (size_t)wib * expand_warp_bytes(m, B, ts);
  w.tile = reinterpret_cast<int32_t*>(base);
  w.hk = reinterpret_cast<unsigned long long*>(base + (size_t)B * ts * 4);
  w.par = reinterpret_cast<int32_t*>(w.hk + B);
  w.buf = w.par + m4;
  w.msk = reinterpret_cast<uint32_t*>(w.buf + m4);
  w.dig = reinterpret_cast<uint8_t*>(w.msk + m4);

  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  const uint64_t nw = (uint64_t)gridDim.x * wpb;
  for (uint64_t task = (uint64_t)blockIdx.x * wpb + wib; task < ntasks; task += nw) {
    const uint64_t la = task * a.run;
    const uint64_t lb = min(la + a.run, (uint64_t)a.Q);
    int64_t p = warp_find_parent(a.off, a.P, a.g0 + la, lane);
    uint64_t p_lo = __ldg(a.off + p), p_hi = __ldg(a.off + p + 1);
    if (task == 0 && lane == 0) a.st->p_first = (unsigned long long)p;
    uint64_t after = parent_state(s, a.parents + (size_t)p * m, w, lane);
    decode_full(s, w, a.g0 + la - p_lo, after, lane);
    for (uint64_t l = la; l < lb;) {
      const int nb = (int)min((uint64_t)B, lb - l);
      for (int k = 0; k < nb; ++k) {
        int32_t* trow = w.tile + k * ts;
        uint64_t hp = 0;
        for (int n = lane; n < m; n += 32) {
          const int32_t x = w.buf[n];
          trow[n] = x;
          hp += col_hash(n, x);
        }
        hp = warp_sum_u64(hp);
        if (lane == 0) w.hk[k] = hp;
        __syncwarp();
        const uint64_t gn = a.g0 + l + k + 1;
        if (l + k + 1 < lb) {
          if (gn >= p_hi) {
            do {
              ++p;
              p_lo = p_hi;
              p_hi = __ldg(a.off + p + 1);
            } while (gn >= p_hi);
            after = parent_state(s, a.parents + (size_t)p * m, w, lane);
            decode_full(s, w, gn - p_lo, after, lane);
          } else {
            step_one(s, w, lane);
          }
        }
      }
      __syncwarp();
      if (lane < nb) resolve_lane<VEC>(a, w.tile + lane * ts, w.hk[lane], (uint32_t)(l + lane));
      __syncwarp();
      l += nb;
    }
    if (task + 1 == ntasks && lane == 0) a.st->p_last = (unsigned long long)p;
  }
}

}  // namespace

int launch_expand(ClaimArgs a, cudaStream_t st, int nsm) {
  const int m = a.sys.m;
  const int ts = round4(m) + 4;                       // tile row stride (words), 16-byte aligned
  int B = (int)std::min<size_t>(32, std::max<size_t>(4, (16u << 10) / (4u * ts)));
  const size_t per_warp = expand_warp_bytes(m, B, ts);
  int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (96u << 10) / per_warp));
  const size_t smem = per_warp * wpb;
  a.run = (uint32_t)(4 * B);
  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  const int per_sm = (int)std::max<size_t>(1, (200u << 10) / smem);
  const int blocks = (int)std::min<uint64_t>((ntasks + wpb - 1) / wpb, (uint64_t)nsm * per_sm);
  const bool vec = (m % 4) == 0;
  auto fn = vec ? k_expand<true> : k_expand<false>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  fn<<<blocks > 0 ? blocks : 1, wpb * 32, smem, st>>>(a, B, ts);
  return 1;
}

}  // namespace snp
