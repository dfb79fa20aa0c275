// Kernels of the single-system BFS over SNP-system configurations.
//
// One depth (Algorithm 1, one round of steps II-IV) runs as:
//   k_psi      step (a) for every frontier configuration: applicable rules and
//              Psi = prod_n max(1, omega_n) (Eq. psi), saturating (k_psi_tiled
//              for rows of a multiple of four neurons, k_psi_warp with a warp
//              per row for small frontiers; after a depth whose Psi sum
//              saturated, k_psi_head_saturated lets the rows past the first
//              8192 be skipped when those already hold 2^64 - 1 candidates);
//   scan       exclusive prefix sums of Psi give each parent's first candidate;
//   per chunk of candidates [g0, g0 + Q) in canonical order:
//     k_expand steps (b)-(d) (snp_expand.cu; k_expand_wide for rows of more
//              than kWideM neurons): decode the spiking vector, C' = C + S . M_Pi
//              (Eq. next-config), fingerprint, look C' up; a key never seen is
//              claimed in the table and its row written (to the store, or to
//              staging row lid), and every candidate holding such a pending
//              key lowers that key's first-occurrence index;
//     k_mark   one bit per first occurrence;
//     scan     ranks of the first occurrences in candidate order;
//     k_commit the first `remaining` of them get their discovery index, in
//              rank order (the row map entry; or a copy of the staged row
//              into the discovery-ordered pool), and their table slots point
//              at their rows; the rest become tombstones (the cap stops the
//              depth).
#include "snp_kernels.cuh"

namespace snp {

namespace {

constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ void set_error(ChunkState* st, uint32_t bits) { atomicOr(&st->error, bits); }

}  // namespace

// Step (a) for one configuration, neuron by neuron: Psi = prod max(1, omega)
// (saturating; four counts are multiplied in 32 bits, at most 2^20, and a
// product below 2^43 cannot overflow by such a factor), whether
// a child could leave int32, whether the row is past max_expand, and its
// ParentRec (base-child hash, multi-choice neurons in neuron order).
struct PsiAcc {
  uint64_t prod = 1, hb = 0;
  uint32_t nnt = 0, part = 1;
  int parts = 0;
  bool ov = false, skip = false;

  // prod *= part (saturating; part <= 2^20)
  __device__ __forceinline__ void flush() {
    if (part > 1) prod = (prod >> 43) ? (__umul64hi(prod, part) ? kSat : prod * part) : prod * part;
    part = 1;
    parts = 0;
  }

  template <bool REC>
  __device__ __forceinline__ void visit(const DevSys& s, int n, int32_t x, int32_t max_expand, ParentRec* rec) {
    uint32_t mask;
    uint64_t hx = 0;
    if ((uint32_t)x < (uint32_t)kDirect) {  // small count: one entry of the direct table
      const size_t k = (size_t)n * kDirect + (uint32_t)x;
      mask = __ldg(s.dmask + k);
      if (REC) hx = __ldg(s.dhx + k);
      if (!s.gain_small) ov |= x > INT32_MAX - __ldg(s.gain + n);
    } else {
      const NeuronInfo ni = neuron_info(s, n);
      const ApplEntry e = appl_entry(s, ni, n, x);
      mask = e.mask;
      if (REC) hx = (uint64_t)(uint32_t)x * ni.colkey + e.hfirst;
      ov |= x > INT32_MAX - ni.gain;
    }
    const uint32_t cnt = __popc(mask);
    part *= cnt > 1 ? cnt : 1u;  // four counts of at most 32 fit 32 bits
    if (++parts == 4) flush();
    skip |= max_expand >= 0 && x > max_expand;
    if (REC) {
      hb += hx;
      if (cnt > 1) {
        const bool fits = nnt < (uint32_t)kRecNt && n < 65536 && mask < 65536u;
        if (fits) rec->nt[nnt] = ((uint32_t)n << 16) | mask;
        nnt = fits ? nnt + 1 : kRecFull;
      }
    }
  }
  __device__ __forceinline__ uint64_t psi() {
    flush();
    return skip ? 0ull : prod;
  }
  __device__ __forceinline__ bool overflow() const { return ov && !skip; }
};

// Step (a) and Eq. psi for every frontier row, one lane per row, with the
// rows' ParentRecs when rec is given; rows not to be expanded (max_expand)
// get Psi = 0, rows whose children could leave int32 raise kErrOverflow.
// (Rows of m % 4 == 0 neurons go through k_psi_tiled instead.)
template <bool REC>
__global__ void __launch_bounds__(256) k_psi(DevSys s, const int32_t* rows, const uint32_t* perm, int64_t P,
                                             int32_t max_expand, uint64_t* psi, ParentRec* rec, ChunkState* st) {
  const int m = s.m;
  if (st && __ldcg(&st->psi_saturated)) {  // these rows lie past the last candidate: Psi is not needed
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x)
      psi[p] = 0;
    return;
  }
  bool over = false;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* row = rows + (size_t)(perm ? __ldg(perm + p) : (uint64_t)p) * m;
    PsiAcc acc;
    for (int n = 0; n < m; ++n) acc.visit<REC>(s, n, __ldg(row + n), max_expand, REC ? rec + p : nullptr);
    psi[p] = acc.psi();
    if (REC) {
      rec[p].hbase = acc.hb;
      rec[p].nnt = acc.nnt;
    }
    over |= acc.overflow();
  }
  if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) set_error(st, kErrOverflow);
}

// k_psi for small frontiers (no records): a warp per row, lane l visiting
// neurons l, l + 32, ... (coalesced), the lanes' products combined with the
// saturating product, so that a row of many neurons is not one thread's
// serial walk.
template <class RF>
__global__ void __launch_bounds__(256) k_psi_warp(DevSys s, const int32_t* rows, const uint32_t* perm, int64_t P,
                                                  int32_t max_expand, uint64_t* psi, ChunkState* st) {
  const int m = s.m;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (st && __ldcg(&st->psi_saturated)) {  // as in k_psi
    for (int64_t p = w0; p < P; p += nw)
      if (lane == 0) psi[p] = 0;
    return;
  }
  bool over = false;
  for (int64_t p = w0; p < P; p += nw) {
    const typename RF::T* row = row_at<RF>(rows, perm ? __ldg(perm + p) : (uint64_t)p, m);
    PsiAcc acc;
    for (int n = lane; n < m; n += 32) acc.visit<false>(s, n, (int32_t)__ldg(row + n), max_expand, nullptr);
    acc.flush();
    uint64_t v = acc.prod;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = sat_mul(v, __shfl_xor_sync(0xffffffffu, v, o));
    const bool skip = __any_sync(0xffffffffu, acc.skip);
    const bool ov = __any_sync(0xffffffffu, acc.ov);
    if (lane == 0) psi[p] = skip ? 0ull : v;
    over |= ov && !skip;
  }
  if (over && lane == 0) set_error(st, kErrOverflow);
}

// k_psi for rows that move in 16-byte pieces (RF::VEC) with coalesced loads:
// a block takes 256 rows at a time and moves them through shared memory 32
// columns at a time (each row's slab is 128 contiguous bytes in int32 rows,
// read by 8 consecutive threads; 64 or 32 bytes in packed rows), unpacked to
// int32; thread t then reads row t's slab at a stride of 33 words, so the 32
// lanes of a warp hit 32 different banks.
constexpr int kPsiRows = 256, kPsiSlab = 32;
template <class RF, bool REC>
__global__ void __launch_bounds__(kPsiRows) k_psi_tiled(DevSys s, const int32_t* rows, const uint32_t* perm, int64_t P,
                                                        int32_t max_expand, uint64_t* psi, ParentRec* rec,
                                                        ChunkState* st) {
  __shared__ int32_t slab[kPsiRows][kPsiSlab + 1];
  const int m = s.m;
  const int t = threadIdx.x;
  if (st && __ldcg(&st->psi_saturated)) {  // as in k_psi
    for (int64_t p = (int64_t)blockIdx.x * kPsiRows + t; p < P; p += (int64_t)gridDim.x * kPsiRows) psi[p] = 0;
    return;
  }
  bool over = false;
  for (int64_t p0 = (int64_t)blockIdx.x * kPsiRows; p0 < P; p0 += (int64_t)gridDim.x * kPsiRows) {
    const int nrows = (int)min((int64_t)kPsiRows, P - p0);
    const int64_t p = p0 + t;
    PsiAcc acc;
    for (int n0 = 0; n0 < m; n0 += kPsiSlab) {
      const int w = min(kPsiSlab, m - n0);  // columns in this slab (a multiple of RF::PER16)
      const int q4 = w / RF::PER16;         // 16-byte pieces per row
      __syncthreads();
      // rows stream through L2 only, so that they do not evict the
      // applicability table every visit reads from L1
      for (int i = t; i < nrows * q4; i += kPsiRows) {
        const int r = i / q4, q = i - r * q4;
        const uint64_t pr = perm ? __ldcg(perm + p0 + r) : (uint64_t)(p0 + r);
        const uint4 v = __ldcg(reinterpret_cast<const uint4*>(row_at<RF>(rows, pr, m) + n0) + q);
        int32_t x[RF::PER16];
        unpack_piece<RF>(v, x);
        int32_t* d = &slab[r][RF::PER16 * q];
#pragma unroll
        for (int k = 0; k < RF::PER16; ++k) d[k] = x[k];
      }
      __syncthreads();
      if (t < nrows)
        for (int j = 0; j < w; ++j) acc.visit<REC>(s, n0 + j, slab[t][j], max_expand, REC ? rec + p : nullptr);
    }
    if (t < nrows) {
      psi[p] = acc.psi();
      if (REC) {
        rec[p].hbase = acc.hb;
        rec[p].nnt = acc.nnt;
      }
      over |= acc.overflow();
    }
  }
  if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) set_error(st, kErrOverflow);
}

// st->psi_saturated = 1 when the saturating sum of psi[0 .. n) is 2^64 - 1
// (one block).
__global__ void __launch_bounds__(1024) k_psi_head_saturated(const uint64_t* psi, int64_t n, ChunkState* st) {
  __shared__ uint64_t part[32];
  uint64_t v = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v = sat_add(v, psi[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = sat_add(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = sat_add(t, part[w]);
    if (t == kSat) st->psi_saturated = 1u;
  }
}

int launch_psi_head_check(const uint64_t* psi, int64_t n, ChunkState* st, cudaStream_t stream) {
  k_psi_head_saturated<<<1, 1024, 0, stream>>>(psi, n, st);
  return 1;
}

int launch_psi(DevSys s, const int32_t* rows, int w, const uint32_t* perm, int64_t P, int32_t max_expand,
               uint64_t* psi, ParentRec* rec, ChunkState* st, cudaStream_t stream, int nsm) {
  const int threads = 256;
  const int64_t want = (P + threads - 1) / threads;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 8));
  if (!rec && P <= (int64_t)nsm * 256) {  // a warp per row
    const int wb = (int)std::max<int64_t>(1, (P + 7) / 8);
    auto fn = w == 1 ? k_psi_warp<RowU8> : w == 2 ? k_psi_warp<RowU16> : k_psi_warp<RowI32>;
    fn<<<wb, 256, 0, stream>>>(s, rows, perm, P, max_expand, psi, st);
    return 1;
  }
  if (w == 1 || w == 2 || (s.m % 4) == 0) {
    const int64_t tiles = (P + kPsiRows - 1) / kPsiRows;
    const int tb = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)nsm * 6));
    auto fn = w == 1   ? (rec ? k_psi_tiled<RowU8, true> : k_psi_tiled<RowU8, false>)
              : w == 2 ? (rec ? k_psi_tiled<RowU16, true> : k_psi_tiled<RowU16, false>)
                       : (rec ? k_psi_tiled<RowI32V, true> : k_psi_tiled<RowI32V, false>);
    fn<<<tb, kPsiRows, 0, stream>>>(s, rows, perm, P, max_expand, psi, rec, st);
    return 1;
  }
  auto fn = rec ? k_psi<true> : k_psi<false>;
  fn<<<blocks, threads, 0, stream>>>(s, rows, perm, P, max_expand, psi, rec, st);
  return 1;
}

// One bit per first occurrence: every candidate lid that claimed a key
// (ownbits) names the key's first candidate gmin[lid]; clears ownbits and
// counts the claimed keys into st->n_alloc.
__global__ void k_mark(uint32_t* ownbits, const uint32_t* gmin, uint32_t* bits, uint32_t* srow, uint32_t nwords,
                       ChunkState* st) {
  uint32_t cnt = 0;
  const uint32_t limit = nwords * 32u;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
    uint32_t word = ownbits[w];
    if (!word) continue;
    ownbits[w] = 0;
    cnt += __popc(word);
    while (word) {
      const uint32_t o = w * 32u + (uint32_t)(__ffs(word) - 1);
      word &= word - 1;
      const uint32_t f = gmin[o];
      if (f >= limit) {  // not a claim of this pass: record and skip
        atomicOr(&st->error, kErrInternal);
        continue;
      }
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

// Largest p in [0, P) with off[p] <= g, by one thread.
__device__ __forceinline__ int64_t find_parent(const uint64_t* off, int64_t P, uint64_t g) {
  int64_t lo = 0, hi = P;
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (__ldg(off + mid) <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// One first occurrence: accepted (rank < remaining: copied to its pool row in
// rank order, its slot pointed at the row) or rejected (its slot becomes a
// tombstone).
__device__ __forceinline__ void commit_one(const CommitArgs& a, uint32_t lid, uint64_t rank, int64_t row_base,
                                           uint64_t remaining) {
  const int m = a.sys.m;
  const uint32_t s = a.srow[lid];
  unsigned long long* slot = a.table.slots + a.slot_of[s];
  const unsigned long long hi = (*slot) & 0xFFFFFFFF00000000ull;
  if (rank >= remaining) {
    *slot = hi | kRowTomb;
    return;
  }
  const int64_t row = row_base + (int64_t)rank;
  if (a.perm) {  // store mode: the row stays where its owner put it
    const uint32_t sr = a.sidx_of[s];
    a.perm[row] = sr;
    *slot = hi | sr;
  } else {
    copy_row_cg(a.staging + (size_t)s * m, a.pool + (size_t)row * m, m);
    *slot = hi | (uint32_t)row;
  }
  if (rank + 1 == remaining) {
    a.st->capped = 1;
    a.st->last_lid = lid;
  }
  if (a.rec_parent) {
    const uint64_t g = a.g0 + lid;
    const int64_t p = find_parent(a.off, a.P, g);
    a.rec_parent[row] = a.parent_base + p;
    a.rec_index[row] = g - __ldg(a.off + p);
  }
}

// Commits every first occurrence of the chunk, one lane per rank: a warp
// takes ranks r0 .. r0 + 31 (st->n_alloc of them in all), finds the bitmap
// word holding r0 in the exclusive prefix sums wbase, and each lane then
// finds its own word among the next 32 and its set bit within the word.
__global__ void __launch_bounds__(256) k_commit(CommitArgs a) {
  const int lane = threadIdx.x & 31;
  const uint32_t total = *reinterpret_cast<volatile const unsigned int*>(&a.st->n_alloc);
  const int64_t row_base = a.ctr ? (int64_t)__ldcg(a.ctr) : a.row_base;
  const uint64_t remaining = a.ctr ? __ldcg(a.ctr + 1) : a.remaining;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t r0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; r0 < total;
       r0 += nwarps * 32) {
    // largest w with wbase[w] <= r0 (the word holding rank r0)
    int64_t lo = 0, hi = a.nwords;
    while (hi - lo > 1) {
      const int64_t step = (hi - lo + 31) / 32;
      const int64_t idx = lo + (int64_t)lane * step;
      const bool ok = idx < hi && a.wbase[idx] <= r0;
      const uint32_t bal = __ballot_sync(0xffffffffu, ok);
      lo += (int64_t)(31 - __clz(bal)) * step;
      hi = min(lo + step, hi);
    }
    const uint64_t r = r0 + lane;
    const int64_t wj = lo + 1 + lane;
    const uint64_t nb = wj < (int64_t)a.nwords ? a.wbase[wj] : ~0ull;  // first rank after word lo + lane
    int k = 0;  // words lo .. lo + k - 1 end at or before r
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint64_t v = __shfl_sync(0xffffffffu, nb, k + step - 1);
      if (v <= r) k += step;
    }
    const uint64_t nb31 = __shfl_sync(0xffffffffu, nb, 31);
    if (r < total) {
      uint64_t w = (uint64_t)lo + k;
      if (nb31 <= r) {  // beyond the window: a run of empty words
        int64_t l2 = lo + 32, h2 = a.nwords;
        while (h2 - l2 > 1) {
          const int64_t mid = l2 + (h2 - l2) / 2;
          if (a.wbase[mid] <= r) l2 = mid; else h2 = mid;
        }
        w = (uint64_t)l2;
      }
      const uint32_t word = a.bits[w];
      const uint32_t q = (uint32_t)(r - a.wbase[w]);
      commit_one(a, (uint32_t)w * 32u + __fns(word, 0, (int)q + 1), r, row_base, remaining);
    }
  }
}

__global__ void k_iota_u32(uint32_t* out, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (uint32_t)k;
}

void launch_iota_u32(uint32_t* out, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
  k_iota_u32<<<blocks, 256, 0, st>>>(out, n);
}

// out[k] = pool[perm[k]] (pool[k] without perm) for k < n as int32 rows, one
// warp per row (16-byte pieces of the output when m % 4 == 0; packed rows are
// widened four counts at a time).
template <class RF>
__global__ void k_gather_rows(const int32_t* pool, const uint32_t* perm, int64_t n, int m, int32_t* out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n; k += nw) {
    const typename RF::T* src = row_at<RF>(pool, perm ? __ldg(perm + k) : (uint64_t)k, m);
    int32_t* dst = out + (size_t)k * m;
    if constexpr (RF::VEC) {
      int4* d4 = reinterpret_cast<int4*>(dst);
      for (int j = lane; j < (m >> 2); j += 32) {
        if constexpr (RF::W == 1)
          d4[j] = unpack4_u8(__ldg(reinterpret_cast<const uint32_t*>(src) + j));
        else if constexpr (RF::W == 2)
          d4[j] = unpack4_u16(__ldg(reinterpret_cast<const uint2*>(src) + j));
        else
          d4[j] = __ldg(reinterpret_cast<const int4*>(src) + j);
      }
    } else {
      for (int j = lane; j < m; j += 32) dst[j] = __ldg(src + j);
    }
  }
}

void launch_gather_rows(const int32_t* pool, int w, const uint32_t* perm, int64_t n, int m, int32_t* out,
                        cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152 * 64));
  auto fn = w == 1 ? k_gather_rows<RowU8> : w == 2 ? k_gather_rows<RowU16>
            : (m & 3) == 0 ? k_gather_rows<RowI32V> : k_gather_rows<RowI32>;
  fn<<<blocks, 256, 0, st>>>(pool, perm, n, m, out);
}

// Clears the first-occurrence bitmap; with ctr, one thread then moves the
// device counters past the chunk's accepted configurations.
__global__ void k_hold_slot_of_row(unsigned long long* slots, uint64_t n, uint32_t row) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long v = slots[i];
    if (v != kEmpty && (uint32_t)v == row) slots[i] = (v & 0xFFFFFFFF00000000ull) | kRowReserved;
  }
}

__global__ void k_clear_bits(uint32_t* bits, uint32_t nwords, unsigned long long* ctr, const ChunkState* st) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += gridDim.x * blockDim.x) bits[i] = 0;
  if (ctr && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long left = ctr[1];
    const unsigned long long acc = min((unsigned long long)st->n_alloc, left);
    ctr[0] += acc;
    if (left != ~0ull) ctr[1] = left - acc;
  }
}

// Inserts committed rows [r0, r1) (all distinct) into an empty or partly
// filled table: used for C0 and to rebuild the table when it grows.
template <class RF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_insert_rows(DevSys s, const int32_t* pool,
                                                                     const uint32_t* perm, int64_t r0, int64_t r1,
                                                                     DevTable t, ChunkState* st) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t r = r0 + (int64_t)blockIdx.x * kWarpsPerBlock + wib; r < r1; r += nw) {
    const uint32_t sr = perm ? __ldg(perm + r) : (uint32_t)r;  // the row's place in the pool (the store)
    const typename RF::T* row = row_at<RF>(pool, sr, s.m);
    const uint64_t h = fingerprint(s, row, lane);
    if (lane == 0) {
      const unsigned long long val = ((unsigned long long)fp32_of(h) << 32) | sr;
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

// *out = max(*out, x[0 .. n)) (*out starts at 0; the counts are >= 0).
__global__ void k_count_max(const int32_t* x, int64_t n, int32_t* out) {
  int32_t v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v = max(v, __ldg(x + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

void launch_count_max(const int32_t* x, int64_t n, int32_t* out, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  k_count_max<<<blocks, 256, 0, st>>>(x, n, out);
}

// n int32 rows into rows of format RF (counts within its range), four counts
// per thread.
template <class RF>
__global__ void k_pack_rows(const int32_t* src, int64_t n4, int32_t* dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(src) + i);
    if constexpr (RF::W == 1)
      reinterpret_cast<uint32_t*>(dst)[i] = pack4_u8(v);
    else
      reinterpret_cast<uint2*>(dst)[i] = pack4_u16(v);
  }
}

void launch_pack_rows(const int32_t* src, int64_t n, int m, int w, int32_t* dst, cudaStream_t st) {
  const int64_t n4 = n * (m / 4);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n4 + 255) / 256, 152 * 32));
  if (w == 1)
    k_pack_rows<RowU8><<<blocks, 256, 0, st>>>(src, n4, dst);
  else
    k_pack_rows<RowU16><<<blocks, 256, 0, st>>>(src, n4, dst);
}

void launch_insert_rows(DevSys s, const int32_t* pool, int w, const uint32_t* perm, int64_t r0, int64_t r1,
                        DevTable t, ChunkState* st, int blocks, cudaStream_t stream) {
  auto fn = w == 1 ? k_insert_rows<RowU8> : w == 2 ? k_insert_rows<RowU16> : k_insert_rows<RowI32>;
  fn<<<blocks, kWarpsPerBlock * 32, 0, stream>>>(s, pool, perm, r0, r1, t, st);
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
