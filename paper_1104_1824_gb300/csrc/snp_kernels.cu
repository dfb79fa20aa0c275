// Kernels of the single-system BFS over SNP-system configurations.
//
// One depth (Algorithm 1, one round of steps II-IV) runs as:
//   k_psi      step (a) for every frontier configuration: applicable rules and
//              Psi = prod_n max(1, omega_n) (Eq. psi), saturating;
//   scan       exclusive prefix sums of Psi give each parent's first candidate;
//   per chunk of candidates [g0, g0 + Q) in canonical order:
//     k_claim  steps (b)-(d): decode the spiking vector, C' = C + S . M_Pi
//              (Eq. next-config), fingerprint, look C' up; a key never seen is
//              claimed in the table and staged, and every candidate holding a
//              staged key lowers that key's first-occurrence index;
//     k_mark   one bit per first occurrence;
//     scan     ranks of the first occurrences in candidate order;
//     k_commit the first `remaining` of them are copied, in rank order, to the
//              configuration pool and their table slots point there; the rest
//              become tombstones (the cap stops the depth).
#include "snp_kernels.cuh"

namespace snp {

namespace {

constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ void set_error(ChunkState* st, uint32_t bits) { atomicOr(&st->error, bits); }

// Looks C' (in w.buf, fingerprint h) up and, if absent, claims it for
// chunk-local candidate lid.  Writes staging rows and first-occurrence
// indices as described at the top of the file.
__device__ __forceinline__ void probe_and_claim(const ClaimArgs& a, const int32_t* buf, uint64_t h, uint32_t lid,
                                                int lane) {
  const int m = a.sys.m;
  const uint32_t fp = fp32_of(h);
  uint64_t bucket = h & a.table.bmask;
  for (uint64_t probes = 0; probes <= a.table.bmask; ++probes, bucket = (bucket + 1) & a.table.bmask) {
    unsigned long long* bs = a.table.slots + bucket * kBucket;
    for (;;) {  // re-read the bucket after a lost race
      unsigned long long v = (lane < kBucket) ? ld_acquire(bs + lane) : kEmpty;
      const bool emp = lane < kBucket && v == kEmpty;
      const bool mat = lane < kBucket && v != kEmpty && (uint32_t)(v >> 32) == fp && (uint32_t)v != kRowTomb;
      const uint32_t em = __ballot_sync(0xffffffffu, emp);
      uint32_t mm = __ballot_sync(0xffffffffu, mat);
      const int fe = em ? __ffs(em) - 1 : kBucket;
      mm &= (fe >= 32) ? 0xffffffffu : ((1u << fe) - 1u);
      while (mm) {
        const int L = __ffs(mm) - 1;
        mm &= mm - 1;
        uint32_t row = (uint32_t)__shfl_sync(0xffffffffu, v, L);
        if (row == kRowReserved) {  // claimed, not yet published: wait (bounded)
          unsigned long long w = 0;
          if (lane == 0) {
            int spins = 0;
            do {
              w = ld_acquire(bs + L);
              if ((uint32_t)w != kRowReserved) break;
              __nanosleep(64);
            } while (++spins < kSpinLimit);
          }
          w = __shfl_sync(0xffffffffu, w, 0);
          row = (uint32_t)w;
          if (row == kRowReserved) {
            if (lane == 0) set_error(a.st, kErrTimeout);
            return;
          }
          if (row == kRowTomb) continue;
        }
        __threadfence();
        const int32_t* other = (row & kPending) ? a.staging + (size_t)(row & ~kPending) * m
                                                : a.pool + (size_t)row * m;
        if (rows_equal(buf, other, m, lane)) {
          if ((row & kPending) && lane == 0) atomicMin(a.gmin + (row & ~kPending), lid);
          return;  // seen before (an earlier chunk or depth), or staged in this chunk
        }
      }
      if (fe >= kBucket) break;  // bucket full: next bucket
      unsigned long long old = 0;
      if (lane == 0)
        old = atomicCAS(bs + fe, kEmpty, ((unsigned long long)fp << 32) | kRowReserved);
      old = __shfl_sync(0xffffffffu, old, 0);
      if (old != kEmpty) continue;  // lost the race for this slot: look again
      // Owner: stage C', record the claim, then publish the slot.
      uint32_t srow = 0;
      if (lane == 0) srow = atomicAdd(&a.st->n_alloc, 1u);
      srow = __shfl_sync(0xffffffffu, srow, 0);
      if (srow >= a.Q) {
        if (lane == 0) {
          set_error(a.st, kErrStaging);
          atomicExch(bs + fe, ((unsigned long long)fp << 32) | kRowTomb);
        }
        return;
      }
      int32_t* dst = a.staging + (size_t)srow * m;
      for (int n = lane; n < m; n += 32) __stcg(dst + n, buf[n]);
      if (lane == 0) {
        a.gmin[srow] = lid;
        a.slot_of[srow] = (uint32_t)(bucket * kBucket + fe);
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicExch(bs + fe, ((unsigned long long)fp << 32) | (kPending | srow));
      return;
    }
  }
  if (lane == 0) set_error(a.st, kErrTableFull);
}

}  // namespace

// Step (a) and Eq. psi for every frontier row; flags rows whose children could
// leave int32, and gives Psi = 0 to rows not to be expanded (max_expand).
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_psi(DevSys s, const int32_t* rows, int64_t P,
                                                             int32_t max_expand, uint64_t* psi, ChunkState* st) {
  extern __shared__ int32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpParent w;
  w.par = smem + (size_t)wib * 2 * s.m;
  w.msk = reinterpret_cast<uint32_t*>(w.par + s.m);
  w.buf = nullptr;
  const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t p = (int64_t)blockIdx.x * kWarpsPerBlock + wib; p < P; p += nw) {
    const int32_t* row = rows + (size_t)p * s.m;
    load_parent(s, row, w, lane);
    bool over = false, skip = false;
    for (int n = lane; n < s.m; n += 32) {
      const int32_t x = w.par[n];
      over |= x > INT32_MAX - __ldg(s.gain + n);
      skip |= max_expand >= 0 && x > max_expand;
    }
    over = __any_sync(0xffffffffu, over);
    skip = __any_sync(0xffffffffu, skip);
    if (lane == 0) {
      psi[p] = skip ? 0ull : w.psi;
      if (over && !skip) set_error(st, kErrOverflow);
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_claim(ClaimArgs a) {
  extern __shared__ int32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int m = a.sys.m;
  WarpParent w;
  w.par = smem + (size_t)wib * 3 * m;
  w.msk = reinterpret_cast<uint32_t*>(w.par + m);
  w.buf = w.par + 2 * m;
  const uint64_t ntasks = ((uint64_t)a.Q + a.run - 1) / a.run;
  const uint64_t nw = (uint64_t)gridDim.x * kWarpsPerBlock;
  for (uint64_t task = (uint64_t)blockIdx.x * kWarpsPerBlock + wib; task < ntasks; task += nw) {
    const uint64_t la = task * a.run;
    const uint64_t lb = min(la + a.run, (uint64_t)a.Q);
    int64_t p = warp_find_parent(a.off, a.P, a.g0 + la, lane);
    uint64_t p_lo = __ldg(a.off + p), p_hi = __ldg(a.off + p + 1);
    if (task == 0 && lane == 0) a.st->p_first = (unsigned long long)p;
    load_parent(a.sys, a.parents + (size_t)p * m, w, lane);
    for (uint64_t l = la; l < lb; ++l) {
      const uint64_t g = a.g0 + l;
      if (g >= p_hi) {
        do {
          ++p;
          p_lo = p_hi;
          p_hi = __ldg(a.off + p + 1);
        } while (g >= p_hi);
        load_parent(a.sys, a.parents + (size_t)p * m, w, lane);
      }
      build_child(a.sys, w, g - p_lo, lane);
      const uint64_t h = fingerprint(a.sys, w.buf, lane);
      probe_and_claim(a, w.buf, h, (uint32_t)l, lane);
    }
    if (task + 1 == ntasks && lane == 0) a.st->p_last = (unsigned long long)p;
  }
}

// One bit per first occurrence: staging row s holds a distinct key whose
// first candidate (chunk-local) is gmin[s].
__global__ void k_mark(const uint32_t* gmin, uint32_t* bits, uint32_t* srow, uint32_t Q, ChunkState* st) {
  const uint32_t n = min(st->n_alloc, Q);
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const uint32_t lid = gmin[s];
    atomicOr(bits + (lid >> 5), 1u << (lid & 31));
    srow[lid] = s;
  }
}

__global__ void k_popc(const uint32_t* bits, uint32_t* cnt, uint32_t nwords) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += gridDim.x * blockDim.x)
    cnt[i] = __popc(bits[i]);
}

// Accepts first occurrences of rank < remaining (discovery order), rejects the
// rest.  One warp per bitmap word.
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_commit(CommitArgs a) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int m = a.sys.m;
  const uint64_t nw = (uint64_t)gridDim.x * kWarpsPerBlock;
  for (uint64_t wd = (uint64_t)blockIdx.x * kWarpsPerBlock + wib; wd < a.nwords; wd += nw) {
    const uint32_t word = a.bits[wd];
    uint32_t rest = word;
    while (rest) {
      const int b = __ffs(rest) - 1;
      rest &= rest - 1;
      const uint32_t lid = (uint32_t)wd * 32u + (uint32_t)b;
      const uint64_t rank = (uint64_t)a.wbase[wd] + __popc(word & ((1u << b) - 1u));
      const uint32_t s = a.srow[lid];
      unsigned long long* slot = a.table.slots + a.slot_of[s];
      const unsigned long long hi = (*slot) & 0xFFFFFFFF00000000ull;
      if (rank < a.remaining) {
        const int64_t row = a.row_base + (int64_t)rank;
        const int32_t* src = a.staging + (size_t)s * m;
        int32_t* dst = a.pool + (size_t)row * m;
        for (int n = lane; n < m; n += 32) dst[n] = __ldcg(src + n);
        if (lane == 0) {
          *slot = hi | (uint32_t)row;
          if (rank + 1 == a.remaining) {
            a.st->capped = 1;
            a.st->last_lid = lid;
          }
        }
        if (a.rec_parent) {
          const uint64_t g = a.g0 + lid;
          const int64_t p = warp_find_parent(a.off, a.P, g, lane);
          if (lane == 0) {
            a.rec_parent[row] = a.parent_base + p;
            a.rec_index[row] = g - a.off[p];
          }
        }
      } else if (lane == 0) {
        *slot = hi | kRowTomb;
      }
    }
  }
}

__global__ void k_clear_bits(uint32_t* bits, uint32_t nwords) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += gridDim.x * blockDim.x) bits[i] = 0;
}

// Inserts committed rows [r0, r1) (all distinct) into an empty or partly
// filled table: used for C0 and to rebuild the table when it grows.
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_insert_rows(DevSys s, const int32_t* pool, int64_t r0,
                                                                     int64_t r1, DevTable t, ChunkState* st) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t r = r0 + (int64_t)blockIdx.x * kWarpsPerBlock + wib; r < r1; r += nw) {
    const int32_t* row = pool + (size_t)r * s.m;
    uint64_t h = 0;
    for (int n = lane; n < s.m; n += 32) h += col_hash(n, row[n]);
    h = warp_sum_u64(h);
    if (lane == 0) {
      const unsigned long long val = ((unsigned long long)fp32_of(h) << 32) | (uint32_t)r;
      uint64_t b = h & t.bmask;
      bool done = false;
      for (uint64_t probes = 0; probes <= t.bmask && !done; ++probes, b = (b + 1) & t.bmask) {
        for (int k = 0; k < kBucket; ++k)
          if (atomicCAS(t.slots + b * kBucket + k, kEmpty, val) == kEmpty) {
            done = true;
            break;
          }
      }
      if (!done) set_error(st, kErrTableFull);
    }
  }
}

// All children of one configuration C in canonical order (no deduplication).
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_step_children(DevSys s, const int32_t* C, uint64_t n,
                                                                       int32_t* out) {
  extern __shared__ int32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int m = s.m;
  WarpParent w;
  w.par = smem + (size_t)wib * 3 * m;
  w.msk = reinterpret_cast<uint32_t*>(w.par + m);
  w.buf = w.par + 2 * m;
  load_parent(s, C, w, lane);
  const uint64_t nw = (uint64_t)gridDim.x * kWarpsPerBlock;
  for (uint64_t t = (uint64_t)blockIdx.x * kWarpsPerBlock + wib; t < n; t += nw) {
    build_child(s, w, t, lane);
    for (int j = lane; j < m; j += 32) out[t * m + j] = w.buf[j];
  }
}

__global__ void k_fill_u64(unsigned long long* p, uint64_t n, unsigned long long v) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ---------------------------------------------------------------------------
// Exclusive scans.

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

struct SatAdd {
  __device__ __forceinline__ uint64_t operator()(uint64_t a, uint64_t b) const { return sat_add(a, b); }
};
struct Add32 {
  __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};

template <typename T, typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const T* in, T* out, T* tile_sum, int64_t n, Op op) {
  __shared__ T wtot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T acc = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : (T)0;
    acc = op(acc, v[i]);
  }
  T x = acc;  // inclusive scan of thread totals within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = op(y, x);
  }
  if (lane == 31) wtot[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = (lane < kScanThreads / 32) ? wtot[lane] : (T)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t = op(y, t);
    }
    if (lane < kScanThreads / 32) wtot[lane] = t;
  }
  __syncthreads();
  T ex = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) ex = 0;
  T run = op(w > 0 ? wtot[w - 1] : (T)0, ex);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run = op(run, v[i]);
  }
  if (tile_sum && threadIdx.x == kScanThreads - 1) tile_sum[blockIdx.x] = run;
}

template <typename T, typename Op>
__global__ void k_scan_add(T* out, const T* tile_off, int64_t n, Op op) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = op(tile_off[i / kScanTile], out[i]);
}

// Returns the number of kernels launched.
template <typename T, typename Op>
int scan_impl(const T* in, T* out, int64_t n, T* temp, cudaStream_t st, Op op) {
  if (n <= 0) return 0;
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_scan_tile<T, Op><<<1, kScanThreads, 0, st>>>(in, out, nullptr, n, op);
    return 1;
  }
  T* sums = temp;
  k_scan_tile<T, Op><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, sums, n, op);
  const int inner = scan_impl<T, Op>(sums, sums, nb, temp + nb, st, op);
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_scan_add<T, Op><<<(unsigned)blocks, 256, 0, st>>>(out, sums, n, op);
  return inner + 2;
}

}  // namespace

size_t scan_temp_bytes(int64_t n, size_t elem) {
  size_t total = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    total += (size_t)n;
  }
  return (total + 16) * elem;
}

int scan_u64_sat(const uint64_t* in, uint64_t* out, int64_t n, void* temp, cudaStream_t st) {
  return scan_impl<uint64_t, SatAdd>(in, out, n, static_cast<uint64_t*>(temp), st, SatAdd());
}

int scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t st) {
  return scan_impl<uint32_t, Add32>(in, out, n, static_cast<uint32_t*>(temp), st, Add32());
}

void launch_popc(const uint32_t* bits, uint32_t* cnt, uint32_t nwords, cudaStream_t st) {
  const unsigned blocks = (unsigned)std::min<uint64_t>((nwords + 255) / 256, 152 * 16);
  k_popc<<<blocks ? blocks : 1, 256, 0, st>>>(bits, cnt, nwords);
}

}  // namespace snp
