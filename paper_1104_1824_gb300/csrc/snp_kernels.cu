// Kernels of the single-system BFS over SNP-system configurations.
//
// One depth (Algorithm 1, one round of steps II-IV) runs as:
//   k_psi      step (a) for every frontier configuration: applicable rules and
//              Psi = prod_n max(1, omega_n) (Eq. psi), saturating;
//   scan       exclusive prefix sums of Psi give each parent's first candidate;
//   per chunk of candidates [g0, g0 + Q) in canonical order:
//     k_expand steps (b)-(d) (snp_expand.cu): decode the spiking vector, C' = C + S . M_Pi
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

// One bit per first occurrence: every candidate lid that claimed a key
// (ownbits) names the key's first candidate gmin[lid]; clears ownbits and
// counts the claimed keys into st->n_alloc.
__global__ void k_mark(uint32_t* ownbits, const uint32_t* gmin, uint32_t* bits, uint32_t* srow, uint32_t nwords,
                       ChunkState* st) {
  uint32_t cnt = 0;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
    uint32_t word = ownbits[w];
    if (!word) continue;
    ownbits[w] = 0;
    cnt += __popc(word);
    while (word) {
      const uint32_t o = w * 32u + (uint32_t)(__ffs(word) - 1);
      word &= word - 1;
      const uint32_t f = gmin[o];
      atomicOr(bits + (f >> 5), 1u << (f & 31));
      srow[f] = o;
    }
  }
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, k);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->n_alloc, cnt);
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
