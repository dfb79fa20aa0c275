// Exact fp8 form of step (c) on the 5th-generation tensor core (SNP_T_TC_F8):
// C' = C + S . M_Pi (Eq. next-config) with tcgen05.mma kind::f8f6f4, operands
// staged in shared memory, the product accumulated in fp32 in tensor memory
// (TMEM) and read back with tcgen05.ld.
//
// Exactness.  Entries of M_Pi are integers with |M| <= 16 and the left
// operand holds 0, +1 or -1, all exact in e4m3.  Every output is a sum of at
// most 2 m such products, |sum| <= 2 * 16 * 1024 < 2^24, so each partial sum
// is an integer that fp32 holds exactly, whatever order the tensor core adds
// in; the int32 base row is added after the conversion back to int32.
//
// Work unit: a tile of 128 consecutive candidates (the MMA's M, one TMEM lane
// and one thread per candidate).  Two forms of the left operand:
//  * delta (rows of more than 128 neurons, tile within one parent): a CTA
//    keeps one reference candidate t_ref of the parent, its child row
//    C_ref = C + S_ref . M_Pi in shared memory, and the parent's neurons with
//    two or more applicable rules, least significant first (Eq. psi's mixed
//    radix, last neuron least significant).  Candidate t differs from t_ref
//    only in the digits where the two indices differ, so
//    C'_t = C_ref + (S_t - S_ref) . M_Pi, and S_t - S_ref has one +1 and one
//    -1 per differing neuron.  Only the 32-rule blocks holding such entries
//    take part in the product.
//  * full (rows of at most 128 neurons, or a tile that crosses parents):
//    C'_t = C_p + S_t . M_Pi with the 0/1 spiking vector S_t (Algorithm 2,
//    II-3) of every firing neuron.
// Each tile's active rule blocks are collected, the left operand is written
// in shared memory in the canonical no-swizzle K-major layout (8 x 16-byte
// core matrices), the matching blocks of M_Pi^T (prepared once per system in
// the same layout, column chunks of up to 256) arrive by cp.async.bulk, one
// thread issues the MMAs and commits to an mbarrier, and every thread turns
// its TMEM lane into C' = base + D, written to the candidate's store row (the
// rows stay where they are written: the resolve step publishes them in place).
// The linear hash h(C') = h(base) + sum of +-H[r] and whether the candidate
// repeats an earlier one through a rule with an identical row of M_Pi come
// from the digits, for the resolve step.
//
// Every wait on an mbarrier is bounded; a wait that runs out records
// SNP_E_TIMEOUT in the chunk's error word, and the CTA still frees its TMEM.
#include "snp_kernels.cuh"

namespace snp {

namespace {

constexpr int kT5M = 128;       // candidates per tile (MMA M = TMEM lanes)
constexpr int kT5NC = 256;      // columns per MMA (TMEM columns of a CTA)
constexpr int kT5K = 32;        // rules per block (K of one kind::f8f6f4 MMA)
constexpr int kT5ABytes = kT5M * kT5K;  // one block of the left operand: 4 KB
constexpr int kT5MaxSlots = 8;
constexpr uint32_t kT5SpinLimit = 1u << 24;  // mbarrier polls (with a short sleep) before a wait gives up

constexpr uint8_t kF8PlusOne = 0x38;   // e4m3 +1.0
constexpr uint8_t kF8MinusOne = 0xB8;  // e4m3 -1.0

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset between core matrices, stride byte offset between 8-row
// groups, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: D f32, A and B e4m3, both K-major.
__device__ __forceinline__ uint32_t idesc_f8(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kT5SpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 32 bits, 16 or 32 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of (row, k) in one 128 x 32 block of the left operand.
__device__ __forceinline__ uint32_t a_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 4) * 128 + (row & 7) * 16 + (k & 15));
}

struct Tc5Smem {
  uint8_t* A;          // [slots][4096]
  uint8_t* B;          // [slots][ncmax * 32]
  int32_t* ref;        // [np] reference child row (delta form)
  uint32_t* masks;     // [m] applicable rules of the cached parent
  uint16_t* list;      // [m] its neurons with >= 2 applicable rules, least significant first
  uint8_t* refd;       // [m] digits of t_ref over list
  uint32_t* bitmap;    // [nbw] active rule blocks of the tile
  uint16_t* slot_of;   // [nblocks] position of an active block in the tile's list
  uint16_t* act;       // [nblocks] active blocks in increasing order
  unsigned long long* bars;  // [2]: operand arrival, MMA completion
  uint32_t* tmem_slot;
  long long* cp;       // cached parent (frontier index), -1: none
  unsigned long long* scal;  // t_ref, h_ref, p_first
  int* iscal;          // list_len, ref_len, ref_red, nact, single
};

}  // namespace


size_t tc5_smem_bytes(int m, int nblocks, int slots) {
  const int np = (m + 15) / 16 * 16, ncmax = np < kT5NC ? np : kT5NC;
  const int nbw = (nblocks + 31) / 32;
  size_t b = 0;
  b += (size_t)slots * kT5ABytes;
  b += (size_t)slots * ncmax * kT5K;
  b += (size_t)np * 4;
  b += (size_t)((m + 3) / 4 * 4) * 4;
  b += (size_t)((m + 7) / 8 * 8) * 2;
  b += (size_t)((m + 15) / 16 * 16);
  b += (size_t)nbw * 4;
  b += (size_t)((nblocks + 7) / 8 * 8) * 2 * 2;
  b += 256;  // barriers, TMEM address, cached parent, scalars, alignment
  return (b + 1023) / 1024 * 1024 + 1024;  // + alignment of the base to 1024
}

namespace {

__device__ __forceinline__ Tc5Smem carve(unsigned char* base, int m, int np, int nblocks, int slots) {
  const int ncmax = np < kT5NC ? np : kT5NC;
  unsigned char* p = base;
  Tc5Smem w;
  w.A = p;
  p += (size_t)slots * kT5ABytes;
  w.B = p;
  p += (size_t)slots * ncmax * kT5K;
  w.ref = reinterpret_cast<int32_t*>(p);
  p += (size_t)np * 4;
  w.masks = reinterpret_cast<uint32_t*>(p);
  p += (size_t)((m + 3) / 4 * 4) * 4;
  w.list = reinterpret_cast<uint16_t*>(p);
  p += (size_t)((m + 7) / 8 * 8) * 2;
  w.refd = p;
  p += (size_t)((m + 15) / 16 * 16);
  w.bitmap = reinterpret_cast<uint32_t*>(p);
  p += (size_t)((nblocks + 31) / 32) * 4;
  p = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
  w.slot_of = reinterpret_cast<uint16_t*>(p);
  p += (size_t)((nblocks + 7) / 8 * 8) * 2;
  w.act = reinterpret_cast<uint16_t*>(p);
  p += (size_t)((nblocks + 7) / 8 * 8) * 2;
  p = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
  w.bars = reinterpret_cast<unsigned long long*>(p);
  p += 16;
  w.tmem_slot = reinterpret_cast<uint32_t*>(p);
  p += 16;
  w.cp = reinterpret_cast<long long*>(p);
  p += 8;
  w.scal = reinterpret_cast<unsigned long long*>(p);
  p += 32;
  w.iscal = reinterpret_cast<int*>(p);
  return w;
}

// Frontier row of frontier index p.
__device__ __forceinline__ const int32_t* t5_parent_row(const Tc5Args& a, int64_t p) {
  return a.parents + (size_t)(a.pperm ? __ldg(a.pperm + p) : (uint64_t)p) * a.s.m;
}

// Parent of candidate g, knowing that it is p0 or later (off is sorted; a
// window of 128 frontier rows first, then the rest).
__device__ __forceinline__ int64_t t5_find_parent(const uint64_t* off, int64_t P, int64_t p0, uint64_t g) {
  int64_t lo = p0, hi = min(P, p0 + 129);
  if (hi < P && __ldcg(off + hi) <= g) {
    lo = hi;
    hi = P;
  }
  // largest p in [lo, hi) with off[p] <= g
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (__ldcg(off + mid) <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t digit_of(uint64_t& q, uint32_t radix) {
  if ((q >> 32) == 0) {
    const uint32_t q32 = (uint32_t)q;
    q = q32 / radix;
    return q32 % radix;
  }
  const uint32_t d = (uint32_t)(q % radix);
  q /= radix;
  return d;
}

// Walks the nonzero entries of the candidate's left-operand row: f(rule, sign).
// Delta form: the neurons whose digit differs from t_ref's.  Full form: the
// chosen rule of every firing neuron of parent row prow (whose applicability
// is evaluated on the way).  Returns false if t is not a valid index.
template <typename F>
__device__ __forceinline__ bool t5_walk_delta(const DevSys& s, const Tc5Smem& w, int list_len, int ref_len, uint64_t t,
                                              F&& f) {
  uint64_t q = t;
  int e = 0;
  for (; e < list_len && (q != 0 || e < ref_len); ++e) {
    const int n = w.list[e];
    const uint32_t mask = w.masks[n];
    const uint32_t d = digit_of(q, (uint32_t)__popc(mask));
    const uint32_t dr = e < ref_len ? w.refd[e] : 0u;
    if (d != dr) {
      const int fr = __ldg(s.first_rule + n);
      f(fr + nth_set_bit(mask, (int)d), fr + nth_set_bit(mask, (int)dr), mask);
    }
  }
  return q == 0;
}

template <typename F>
__device__ __forceinline__ bool t5_walk_full(const DevSys& s, const int32_t* prow, uint64_t t, F&& f) {
  uint64_t q = t;
  for (int n = s.m - 1; n >= 0; --n) {
    const int32_t x = __ldcg(prow + n);
    const uint32_t mask = (uint32_t)appl(s, n, x);
    if (!mask) {
      f(-1, 0, x, n);
      continue;
    }
    const uint32_t radix = (uint32_t)__popc(mask);
    const uint32_t d = radix > 1 ? digit_of(q, radix) : 0u;
    f(__ldg(s.first_rule + n) + nth_set_bit(mask, (int)d), mask, x, n);
  }
  return q == 0;
}

__device__ __forceinline__ void mark_block(const Tc5Smem& w, int r) { atomicOr(w.bitmap + (r >> 10), 1u << ((r >> 5) & 31)); }

__device__ __forceinline__ void put_entry(const Tc5Smem& w, int row, int r, bool plus, int g0, int g1) {
  const int blk = r >> 5;
  const int pos = w.slot_of[blk];
  if (pos >= g0 && pos < g1) w.A[(size_t)(pos - g0) * kT5ABytes + a_off(row, r & 31)] = plus ? kF8PlusOne : kF8MinusOne;
}

// Builds the cached parent's state for the delta form: masks, the list of
// multi-choice neurons (least significant first), the digits of t_ref, the
// reference child row C_ref = C + S_ref . M_Pi and its hash and count of
// repeated-row choices.
__device__ void t5_load_parent(const Tc5Args& a, const Tc5Smem& w, int64_t p, uint64_t t_ref) {
  const DevSys& s = a.s;
  const int m = s.m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t* prow = t5_parent_row(a, p);
  __syncthreads();
  for (int n = tid; n < m; n += blockDim.x) {
    const int32_t x = __ldcg(prow + n);
    w.masks[n] = (uint32_t)appl(s, n, x);
    w.ref[n] = x;
  }
  const int np = a.np;
  for (int n = m + tid; n < np; n += blockDim.x) w.ref[n] = 0;
  if (tid == 0) {
    w.scal[1] = 0ull;  // h_ref
    w.iscal[2] = 0;    // ref_red
  }
  __syncthreads();
  if (warp == 0) {  // multi-choice neurons, last neuron first
    int cnt = 0;
    for (int base = m - 1; base >= 0; base -= 32) {
      const int n = base - lane;
      const bool mc = n >= 0 && __popc(w.masks[n]) >= 2;
      const uint32_t b = __ballot_sync(0xffffffffu, mc);
      if (mc) w.list[cnt + __popc(b & ((1u << lane) - 1u))] = (uint16_t)n;
      cnt += __popc(b);
    }
    __syncwarp();
    if (lane == 0) {  // digits of t_ref (the others are 0)
      uint64_t q = t_ref;
      int e = 0;
      for (; e < cnt && q != 0; ++e) w.refd[e] = (uint8_t)digit_of(q, (uint32_t)__popc(w.masks[w.list[e]]));
      if (q != 0) atomicOr(&a.st->error, kErrInternal);  // t_ref >= Psi
      w.iscal[0] = cnt;
      w.iscal[1] = e;
    }
  }
  __syncthreads();
  const int ref_len = w.iscal[1];
  // C_ref: every firing neuron's first applicable rule, then the swaps of the
  // neurons whose reference digit is not 0
  int red = 0;
  for (int n = tid; n < m; n += blockDim.x) {
    const uint32_t mask = w.masks[n];
    if (!mask) continue;
    const int r = __ldg(s.first_rule + n) + __ffs(mask) - 1;
    const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
    for (int e = e0; e < e1; ++e) {
      const int2 cv = __ldg(s.csr + e);
      atomicAdd(w.ref + cv.x, cv.y);
    }
  }
  for (int e = tid; e < ref_len; e += blockDim.x) {
    const uint32_t d = w.refd[e];
    if (d == 0) continue;
    const int n = w.list[e];
    const uint32_t mask = w.masks[n];
    const int fr = __ldg(s.first_rule + n);
    const int rn = fr + nth_set_bit(mask, (int)d), ro = fr + __ffs(mask) - 1;
    for (int k = __ldg(&s.rule[rn].w); k < __ldg(&s.rule[rn + 1].w); ++k) {
      const int2 cv = __ldg(s.csr + k);
      atomicAdd(w.ref + cv.x, cv.y);
    }
    for (int k = __ldg(&s.rule[ro].w); k < __ldg(&s.rule[ro + 1].w); ++k) {
      const int2 cv = __ldg(s.csr + k);
      atomicAdd(w.ref + cv.x, -cv.y);
    }
    red += redundant_choice(s, mask, rn) ? 1 : 0;
  }
  __syncthreads();
  uint64_t h = 0;
  for (int n = tid; n < m; n += blockDim.x) h += col_hash(s, n, w.ref[n]);
  h = warp_sum_u64(h);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) red += __shfl_xor_sync(0xffffffffu, red, o);
  if (lane == 0) {
    atomicAdd(w.scal + 1, (unsigned long long)h);
    atomicAdd(w.iscal + 2, red);
  }
  if (tid == 0) {
    *w.cp = p;
    w.scal[0] = t_ref;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kT5M) k_tc5_expand(Tc5Args a) {
  if (a.ctr && __ldcg(a.ctr + 1) == 0) return;  // the depth is full: nothing to do
  extern __shared__ unsigned char t5_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)t5_raw + 1023) & ~(uintptr_t)1023);
  const DevSys& s = a.s;
  const int m = s.m, np = a.np, nblocks = a.nblocks, slots = a.slots;
  const int nbw = (nblocks + 31) / 32;
  const int ncmax = np < kT5NC ? np : kT5NC;
  const int nchunks = (np + kT5NC - 1) / kT5NC;
  Tc5Smem w = carve(base, m, np, nblocks, slots);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t bar_b = saddr(w.bars), bar_m = saddr(w.bars + 1);
  if (tid == 0) {
    bar_init(bar_b, 1);
    bar_init(bar_m, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *w.cp = -1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(w.tmem_slot)),
                 "r"((uint32_t)kT5NC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *w.tmem_slot;
  uint32_t ph_b = 0, ph_m = 0;  // parities of the next phase of each barrier
  bool failed = false;

  const uint64_t ntiles = ((uint64_t)a.Q + kT5M - 1) / kT5M;
  const uint64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint64_t tile0 = (uint64_t)blockIdx.x * per, tile1 = min(ntiles, tile0 + per);
  for (uint64_t tile = tile0; tile < tile1 && !failed; ++tile) {
    const uint64_t lid0 = tile * kT5M;
    const uint32_t nrows = (uint32_t)min((uint64_t)kT5M, (uint64_t)a.Q - lid0);
    const uint64_t g_first = a.g0 + lid0, g_last = g_first + nrows - 1;
    // parent of the tile's first candidate, and whether the tile stays in it
    if (warp == 0) {
      const long long cp = *w.cp;
      int64_t p;
      if (cp >= 0 && __ldcg(a.off + cp) <= g_first && g_first < __ldcg(a.off + cp + 1)) p = cp;
      else p = warp_find_parent(a.off, a.P, g_first, lane);
      if (lane == 0) {
        w.scal[2] = (unsigned long long)p;
        w.iscal[4] = (a.delta && g_last < __ldcg(a.off + p + 1)) ? 1 : 0;
      }
    }
    for (int i = tid; i < nbw; i += blockDim.x) w.bitmap[i] = 0u;
    __syncthreads();
    const int64_t p_first = (int64_t)w.scal[2];
    const bool single = w.iscal[4] != 0;
    if (single && *w.cp != p_first) t5_load_parent(a, w, p_first, g_first - __ldcg(a.off + p_first));

    // this thread's candidate
    const uint64_t lid = lid0 + tid;
    const bool valid = tid < (int)nrows;
    const uint64_t g = a.g0 + lid;
    int64_t p = p_first;
    if (valid && !single) p = t5_find_parent(a.off, a.P, p_first, g);
    const uint64_t t = valid ? g - __ldcg(a.off + p) : 0ull;
    if (tile == 0 && tid == 0) a.st->p_first = (unsigned long long)p;
    if (tile + 1 == ntiles && tid + 1 == (int)nrows) a.st->p_last = (unsigned long long)p;
    const int32_t* prow = t5_parent_row(a, p);
    const int list_len = w.iscal[0], ref_len = w.iscal[1];

    // pass 1: active blocks, hash, repeated-row choices
    uint64_t h = 0;
    bool red = false;
    if (valid) {
      bool ok;
      if (single) {
        h = w.scal[1];
        int rc = w.iscal[2];
        ok = t5_walk_delta(s, w, list_len, ref_len, t, [&](int rn, int ro, uint32_t mask) {
          mark_block(w, rn);
          mark_block(w, ro);
          h += __ldg(s.rowkey + rn) - __ldg(s.rowkey + ro);
          rc += (redundant_choice(s, mask, rn) ? 1 : 0) - (redundant_choice(s, mask, ro) ? 1 : 0);
        });
        red = rc > 0;
      } else {
        ok = t5_walk_full(s, prow, t, [&](int r, uint32_t mask, int32_t x, int n) {
          h += col_hash(s, n, x);
          if (r < 0) return;
          mark_block(w, r);
          h += __ldg(s.rowkey + r);
          red |= redundant_choice(s, mask, r);
        });
      }
      if (!ok) atomicOr(&a.st->error, kErrInternal);
      a.hash[lid] = h;
      a.red[lid] = red ? 1 : 0;
    }
    __syncthreads();
    // active blocks in increasing order
    if (warp == 0) {
      int cnt = 0;
      for (int b0 = 0; b0 < nblocks; b0 += 32) {
        const int b = b0 + lane;
        const bool on = b < nblocks && ((w.bitmap[b >> 5] >> (b & 31)) & 1u);
        const uint32_t bb = __ballot_sync(0xffffffffu, on);
        if (on) {
          const int pos = cnt + __popc(bb & ((1u << lane) - 1u));
          w.act[pos] = (uint16_t)b;
          w.slot_of[b] = (uint16_t)pos;
        }
        cnt += __popc(bb);
      }
      if (lane == 0) w.iscal[3] = cnt;
    }
    __syncthreads();
    const int nact = w.iscal[3];
    const int ngroups = (nact + slots - 1) / slots;
    const int32_t* brow = single ? w.ref : prow;  // base row of this candidate
    int32_t* orow = a.out + (size_t)lid * m;
    const bool store = valid && !red;

    for (int nc = 0; nc < nchunks && !failed; ++nc) {
      const int c0 = nc * kT5NC;
      const int nc_cols = min(kT5NC, np - c0);
      for (int gi = 0; gi < ngroups && !failed; ++gi) {
        const int ga = gi * slots, gb = min(nact, ga + slots), gn = gb - ga;
        if (nc == 0 || ngroups > 1) {  // left operand of this group of blocks
          uint4* A4 = reinterpret_cast<uint4*>(w.A);
          for (int i = tid; i < gn * (kT5ABytes / 16); i += blockDim.x) A4[i] = make_uint4(0, 0, 0, 0);
          __syncthreads();
          if (valid) {
            if (single) {
              t5_walk_delta(s, w, list_len, ref_len, t, [&](int rn, int ro, uint32_t) {
                put_entry(w, tid, rn, true, ga, gb);
                put_entry(w, tid, ro, false, ga, gb);
              });
            } else {
              t5_walk_full(s, prow, t, [&](int r, uint32_t, int32_t, int) {
                if (r >= 0) put_entry(w, tid, r, true, ga, gb);
              });
            }
          }
          fence_async_smem();
          __syncthreads();
        }
        if (tid == 0) {  // M_Pi^T blocks of this column chunk, then the MMAs
          const uint32_t bytes = (uint32_t)nc_cols * kT5K;
          bar_expect_tx(bar_b, bytes * (uint32_t)gn);
          for (int k = 0; k < gn; ++k) {
            const uint8_t* src = a.MB + ((size_t)w.act[ga + k] * np + c0) * kT5K;
            bulk_g2s(saddr(w.B + (size_t)k * ncmax * kT5K), src, bytes, bar_b);
          }
          if (!bar_wait(bar_b, ph_b)) atomicOr(&a.st->error, kErrTimeout);
          ph_b ^= 1u;
          fence_after_sync();
          const uint32_t id = idesc_f8(kT5M, nc_cols);
          for (int k = 0; k < gn; ++k) {
            const uint64_t ad = smem_desc(saddr(w.A + (size_t)k * kT5ABytes), 128, 256);
            const uint64_t bd = smem_desc(saddr(w.B + (size_t)k * ncmax * kT5K), 128, 256);
            mma_f8(tmem, ad, bd, id, (gi > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(bar_m);
        }
        // every thread waits for the products (the operands are reused
        // next); a wait that runs out stops the CTA, all threads together
        const bool ok = bar_wait(bar_m, ph_m);
        ph_m ^= 1u;
        if (!ok) atomicOr(&a.st->error, kErrTimeout);
        fence_after_sync();
        if (__syncthreads_or(!ok)) failed = true;
      }
      if (failed) break;
      // epilogue: C' = base + D for this chunk's columns
      const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c = 0; c < nc_cols; c += 32) {
        uint32_t r[32];
        const bool two = c + 32 <= nc_cols;
        if (nact == 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) r[i] = 0u;
        } else {
          if (two) tmem_ld32(lane_addr + (uint32_t)c, r);
          else tmem_ld16(lane_addr + (uint32_t)c, r);
          tmem_wait_ld();
        }
        if (store) {
          const int j0 = c0 + c;
          const int cnt = min(two ? 32 : 16, m - j0);
          if ((m & 3) == 0) {
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              if (i < cnt) {
                const int4 b4 = *reinterpret_cast<const int4*>(brow + j0 + i);
                int4 v;
                v.x = b4.x + __float2int_rn(__uint_as_float(r[i]));
                v.y = b4.y + __float2int_rn(__uint_as_float(r[i + 1]));
                v.z = b4.z + __float2int_rn(__uint_as_float(r[i + 2]));
                v.w = b4.w + __float2int_rn(__uint_as_float(r[i + 3]));
                __stcg(reinterpret_cast<int4*>(orow + j0 + i), v);
              }
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < cnt) __stcg(orow + j0 + i, brow[j0 + i] + __float2int_rn(__uint_as_float(r[i])));
          }
        }
      }
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
    }
  }
  // the products of a failed tile may still be in flight: wait once more
  if (failed && tid == 0) (void)bar_wait(bar_m, ph_m ^ 1u);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kT5NC));
}

}  // namespace

int tc5_slots(int m, int nblocks) {
  // two CTAs per SM (each holds 256 TMEM columns): shared memory per CTA <= 113 KB
  int slots = kT5MaxSlots;
  while (slots > 1 && tc5_smem_bytes(m, nblocks, slots) > (113u << 10)) --slots;
  return slots;
}

void launch_tc5(const Tc5Args& a, cudaStream_t st, int nsm) {
  // at least 80 KB of shared memory so that no more than two CTAs (512 TMEM columns) share an SM
  const size_t smem = std::max<size_t>(tc5_smem_bytes(a.s.m, a.nblocks, a.slots), 80u << 10);
  cudaFuncSetAttribute(k_tc5_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t ntiles = ((uint64_t)a.Q + kT5M - 1) / kT5M;
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)nsm * 2));
  k_tc5_expand<<<blocks, kT5M, smem, st>>>(a);
}

}  // namespace snp
