// Exact fp8 form of step (c) on the 5th-generation tensor core (SNP_T_TC_F8):
// C' = C + S . M_Pi (Eq. next-config) with tcgen05.mma kind::f8f6f4, operands
// staged in shared memory, the product accumulated in fp32 in tensor memory
// (TMEM) and read back with tcgen05.ld.
//
// Exactness.  Entries of M_Pi are integers with |M| <= 16 and the left
// operand holds 0, +1 or -1, all exact in e4m3.  Every product sum D is an
// integer with |D| <= 2 * 16 * 1024 < 2^15, and so is every partial sum, which
// fp32 holds exactly whatever order the tensor core adds in.  The epilogue
// adds 1.5 * 2^23 in fp32 (exact: the sum stays in [2^23, 2^24), where fp32
// holds every integer), so the bits are 0x4B400000 + D, and the row is
// C' = (base - 0x4B400000) + bits in int32: two full-rate adds per entry.
//
// Work unit: a tile of 128 consecutive candidates (the MMA's M, one TMEM lane
// and one epilogue thread per candidate).  Two forms of the left operand:
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
// A CTA per SM runs a contiguous run of tiles with two roles:
//  * four epilogue warps decode the tile's candidates (hash
//    h(C') = h(base) + sum of +-H[r], repeats through rules with identical
//    rows of M_Pi, active rule blocks), write the left operand in the
//    canonical no-swizzle K-major layout (8 x 16-byte core matrices), and per
//    128-column chunk turn their TMEM lane into C' = base + D, stored to the
//    candidate's store row by TMA (128-byte swizzled staging, 32 x 32 boxes);
//  * one control thread streams the M_Pi^T blocks of each chunk into a ring
//    of shared-memory stages by cp.async.bulk, issues the MMAs into one of
//    two TMEM accumulators (128 columns each) while the epilogue drains the
//    other, and commits to the mbarriers the epilogue waits on.
// Two CTAs share an SM, so one's decode overlaps the other's stores.
// The rows stay where they are written: the resolve step publishes them in
// place.  Every mbarrier wait is bounded; a wait that runs out records
// SNP_E_TIMEOUT in the chunk's error word, stops both roles, lets copies and
// products in flight land, and the CTA still frees its TMEM.
#include <cudaTypedefs.h>

#include "snp_kernels.cuh"
#include "snp_tcgen05.cuh"

namespace snp {

using namespace t5;

namespace {

// Barrier of the four epilogue warps only (the control warp does not take part).
__device__ __forceinline__ void ew_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ bool ew_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, 128, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

constexpr int kT5Stages = 8;     // operand-B ring: one (rule block, column chunk) unit per stage
constexpr int kT5Stg = 2;        // TMA store staging buffers per epilogue warp (32 rows x 128 bytes each)
constexpr int kT5Ent = 64;       // multi-choice neurons a digit walk can reach (indices below 2^64)
constexpr int kT5Threads = 160;  // four epilogue warps (TMEM lanes 0-127) and one control warp

struct Tc5Smem {
  uint8_t* A;          // [slots][4096] left operand, one block per slot
  uint8_t* B;          // [kT5Stages][ncmax * 32] right operand ring
  uint8_t* stg;        // [4 warps][kT5Stg][4096] store staging (128-byte swizzle)
  int32_t* adj;        // [2][np] C_ref - kT5Bias (delta form): this tile's and the next tile's reference
  uint32_t* masks;     // [m] applicable rules of the cached parent
  uint16_t* list;      // [m] its neurons with >= 2 applicable rules, least significant first
  uint8_t* refd;       // [m] digits of t_ref over list
  uint4* ent;          // [kT5Ent] per list entry: {mask, repeated-row choices (bit d), first rule, radix}
  uint32_t* bitmap;    // [nbw] active rule blocks of the tile
  uint16_t* slot_of;   // [nblocks] position of an active block in the tile's list
  uint16_t* act;       // [nblocks] active blocks in increasing order
  unsigned long long* bars;  // a_full, a_empty, acc_full[2], acc_empty[2], drain, b_full[S], b_empty[S]
  uint32_t* tmem_slot;
  long long* cp;       // cached parent (frontier index), -1: none
  unsigned long long* scal;  // [0] t_ref, [1] h_ref, [2] p_first, [3] first candidate a chained tile must start at,
                             // [4] next h_ref
  int* iscal;          // [0] list_len, [1] ref buffer, [2] ref_red, [3] nact, [4] single, [5] stop, [6] next ref_red
};

}  // namespace

size_t tc5_smem_bytes(int m, int nblocks, int slots) {
  const int np = (m + 15) / 16 * 16, ncmax = np < kT5NC ? np : kT5NC;
  const int nbw = (nblocks + 31) / 32;
  size_t b = 0;
  b += (size_t)slots * kT5ABytes;
  b += (size_t)kT5Stages * ncmax * kT5K;
  b += (size_t)4 * kT5Stg * 4096;
  b += (size_t)np * 4 * 2;
  b += (size_t)((m + 3) / 4 * 4) * 4;
  b += (size_t)((m + 7) / 8 * 8) * 2;
  b += (size_t)((m + 15) / 16 * 16);
  b += (size_t)kT5Ent * 16;
  b += (size_t)nbw * 4;
  b += (size_t)((nblocks + 7) / 8 * 8) * 2 * 2;
  b += (size_t)(7 + 2 * kT5Stages) * 8 + 256;  // barriers, TMEM address, cached parent, scalars, alignment
  return (b + 1023) / 1024 * 1024 + 1024;      // + alignment of the base to 1024
}

namespace {

__device__ __forceinline__ Tc5Smem carve(unsigned char* base, int m, int np, int nblocks, int slots) {
  const int ncmax = np < kT5NC ? np : kT5NC;
  unsigned char* p = base;
  Tc5Smem w;
  w.stg = p;  // 1024-aligned (128-byte swizzle)
  p += (size_t)4 * kT5Stg * 4096;
  w.A = p;
  p += (size_t)slots * kT5ABytes;
  w.B = p;
  p += (size_t)kT5Stages * ncmax * kT5K;
  w.adj = reinterpret_cast<int32_t*>(p);
  p += (size_t)np * 4 * 2;
  w.masks = reinterpret_cast<uint32_t*>(p);
  p += (size_t)((m + 3) / 4 * 4) * 4;
  w.list = reinterpret_cast<uint16_t*>(p);
  p += (size_t)((m + 7) / 8 * 8) * 2;
  w.refd = p;
  p += (size_t)((m + 15) / 16 * 16);
  w.ent = reinterpret_cast<uint4*>(p);
  p += (size_t)kT5Ent * 16;
  w.bitmap = reinterpret_cast<uint32_t*>(p);
  p += (size_t)((nblocks + 31) / 32) * 4;
  p = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
  w.slot_of = reinterpret_cast<uint16_t*>(p);
  p += (size_t)((nblocks + 7) / 8 * 8) * 2;
  w.act = reinterpret_cast<uint16_t*>(p);
  p += (size_t)((nblocks + 7) / 8 * 8) * 2;
  p = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
  w.bars = reinterpret_cast<unsigned long long*>(p);
  p += (size_t)(7 + 2 * kT5Stages) * 8;
  w.tmem_slot = reinterpret_cast<uint32_t*>(p);
  p += 8;
  w.cp = reinterpret_cast<long long*>(p);
  p += 8;
  w.scal = reinterpret_cast<unsigned long long*>(p);
  p += 48;
  w.iscal = reinterpret_cast<int*>(p);
  return w;
}

// Barrier addresses.
struct Tc5Bars {
  uint32_t a_full, a_empty, acc_full[2], acc_empty[2], drain, b_full, b_empty;  // b_*: stage 0, 8 bytes apart
};

__device__ __forceinline__ Tc5Bars bars_of(const Tc5Smem& w) {
  Tc5Bars b;
  const uint32_t p = saddr(w.bars);
  b.a_full = p;
  b.a_empty = p + 8;
  b.acc_full[0] = p + 16;
  b.acc_full[1] = p + 24;
  b.acc_empty[0] = p + 32;
  b.acc_empty[1] = p + 40;
  b.drain = p + 48;
  b.b_full = p + 56;
  b.b_empty = p + 56 + 8 * kT5Stages;
  return b;
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

// Walks the nonzero entries of the candidate's left-operand row.  Delta form:
// f(rule of t, rule of t_ref, change in the count of repeated-row choices) for
// each neuron whose digit differs from t_ref's (t and t_ref of one parent).  Full form: f(chosen rule or -1, mask, spikes, neuron) for every
// neuron of parent row prow (applicability evaluated on the way).  Returns
// false if t is not a valid index.
template <typename F>
__device__ __forceinline__ bool t5_walk_delta(const DevSys& s, const Tc5Smem& w, int list_len, uint64_t t,
                                              uint64_t t_ref, F&& f) {
  // digits of t and t_ref, least significant first, until the remaining
  // quotients agree (every more significant digit is then the same)
  uint64_t q = t, qr = t_ref;
  const int lim = min(list_len, kT5Ent);
  for (int e = 0; e < lim && q != qr; ++e) {
    const uint4 en = w.ent[e];  // mask, repeated-row choices, first rule, radix
    const uint32_t d = digit_of(q, en.w);
    const uint32_t dr = digit_of(qr, en.w);
    if (d != dr) {
      const int fr = (int)en.z;
      f(fr + nth_set_bit(en.x, (int)d), fr + nth_set_bit(en.x, (int)dr), (int)((en.y >> d) & 1u) - (int)((en.y >> dr) & 1u));
    }
  }
  return q == qr;
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

// Builds the cached parent's state for the delta form (epilogue warps only):
// masks, the list of multi-choice neurons (least significant first), the
// digits of t_ref, the reference child row C_ref = C + S_ref . M_Pi (kept as
// C_ref - kT5Bias) and its hash and count of repeated-row choices.
__device__ void t5_load_parent(const Tc5Args& a, const Tc5Smem& w, int64_t p, uint64_t t_ref) {
  const DevSys& s = a.s;
  const int m = s.m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t* prow = t5_parent_row(a, p);
  int32_t* ref = w.adj;  // buffer 0: C_ref while it is built, then C_ref - kT5Bias
  ew_sync();
  for (int n = tid; n < m; n += kT5M) {
    const int32_t x = __ldcg(prow + n);
    w.masks[n] = (uint32_t)appl(s, n, x);
    ref[n] = x;
  }
  const int np = a.np;
  for (int n = m + tid; n < np; n += kT5M) ref[n] = 0;
  if (tid == 0) {
    w.scal[1] = 0ull;  // h_ref
    w.iscal[2] = 0;    // ref_red
  }
  ew_sync();
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
      w.iscal[6] = e;  // digits of t_ref that may be nonzero
    }
    for (int e = lane; e < min(cnt, kT5Ent); e += 32) {  // the walk's per-entry constants
      const int n = w.list[e];
      const uint32_t mask = w.masks[n];
      const int fr = __ldg(s.first_rule + n);
      uint32_t redbits = 0;
      for (int d = 0; d < __popc(mask); ++d) redbits |= (redundant_choice(s, mask, fr + nth_set_bit(mask, d)) ? 1u : 0u) << d;
      w.ent[e] = make_uint4(mask, redbits, (uint32_t)fr, (uint32_t)__popc(mask));
    }
  }
  ew_sync();
  const int ref_len = w.iscal[6];
  // C_ref: every firing neuron's first applicable rule, then the swaps of the
  // neurons whose reference digit is not 0
  int red = 0;
  for (int n = tid; n < m; n += kT5M) {
    const uint32_t mask = w.masks[n];
    if (!mask) continue;
    const int r = __ldg(s.first_rule + n) + __ffs(mask) - 1;
    const int e0 = __ldg(&s.rule[r].w), e1 = __ldg(&s.rule[r + 1].w);
    for (int e = e0; e < e1; e += 8) {  // eight loads in flight, then their adds
      int2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < e1) v[u] = __ldg(s.csr + e + u);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e + u < e1) atomicAdd(ref + v[u].x, v[u].y);
    }
  }
  for (int e = tid; e < ref_len; e += kT5M) {
    const uint32_t d = w.refd[e];
    if (d == 0) continue;
    const int n = w.list[e];
    const uint32_t mask = w.masks[n];
    const int fr = __ldg(s.first_rule + n);
    const int rn = fr + nth_set_bit(mask, (int)d), ro = fr + __ffs(mask) - 1;
    for (int k = __ldg(&s.rule[rn].w); k < __ldg(&s.rule[rn + 1].w); ++k) {
      const int2 cv = __ldg(s.csr + k);
      atomicAdd(ref + cv.x, cv.y);
    }
    for (int k = __ldg(&s.rule[ro].w); k < __ldg(&s.rule[ro + 1].w); ++k) {
      const int2 cv = __ldg(s.csr + k);
      atomicAdd(ref + cv.x, -cv.y);
    }
    red += redundant_choice(s, mask, rn) ? 1 : 0;
  }
  ew_sync();
  uint64_t h = 0;
  for (int n = tid; n < m; n += kT5M) h += col_hash(s, n, ref[n]);
  h = warp_sum_u64(h);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) red += __shfl_xor_sync(0xffffffffu, red, o);
  if (lane == 0) {
    atomicAdd(w.scal + 1, (unsigned long long)h);
    atomicAdd(w.iscal + 2, red);
  }
  ew_sync();
  for (int n = tid; n < np; n += kT5M) ref[n] = (int32_t)((uint32_t)ref[n] - kT5Bias);
  if (tid == 0) {
    *w.cp = p;
    w.scal[0] = t_ref;
    w.iscal[1] = 0;  // the reference row is in buffer 0
  }
  ew_sync();
}

// Tile schedule of a CTA: a contiguous run of tiles.
__device__ __forceinline__ void tile_range(const Tc5Args& a, uint64_t& t0, uint64_t& t1) {
  const uint64_t ntiles = ((uint64_t)a.Q + kT5M - 1) / kT5M;
  const uint64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  t0 = min(ntiles, (uint64_t)blockIdx.x * per);
  t1 = min(ntiles, t0 + per);
}

// The control warp's lane 0: for every tile and column chunk, the operand-B
// blocks by cp.async.bulk into the ring and the MMAs into the free TMEM
// buffer (which the epilogue warps filled with the bias), then the commits.
__device__ void t5_control(const Tc5Args& a, const Tc5Smem& w, const Tc5Bars& b, uint32_t tmem) {
  const int np = a.np, slots = a.slots;
  const int ncmax = np < kT5NC ? np : kT5NC;
  const int nchunks = (np + kT5NC - 1) / kT5NC;
  volatile int* stop = w.iscal + 5;
  uint64_t tile0, tile1;
  tile_range(a, tile0, tile1);
  uint32_t ph_afull = 0, ph_accempty[2] = {1u, 1u}, ph_bempty[kT5Stages], ph_bfull[kT5Stages];
  for (int i = 0; i < kT5Stages; ++i) {
    ph_bempty[i] = 1u;
    ph_bfull[i] = 0u;
  }
  uint32_t pending = 0;  // stages with a copy in flight
  int stage = 0, buf = 0;
  bool ok = true;
  for (uint64_t tile = tile0; tile < tile1 && ok; ++tile) {
    // the tile's blocks are known once its first left operand is ready
    ok = bar_wait_or_stop(b.a_full, ph_afull, stop);
    ph_afull ^= 1u;
    if (!ok) break;
    const int nact = w.iscal[3];
    const int ngroups = (nact + slots - 1) / slots;
    for (int nc = 0; nc < nchunks && ok; ++nc) {
      const int c0 = nc * kT5NC, nc_cols = min(kT5NC, np - c0);
      const uint32_t id = idesc_f8(kT5M, nc_cols), bytes = (uint32_t)nc_cols * kT5K;
      ok = bar_wait_or_stop(b.acc_empty[buf], ph_accempty[buf], stop);
      ph_accempty[buf] ^= 1u;
      if (!ok) break;
      fence_after_sync();
      const uint32_t d = tmem + (uint32_t)(buf * kT5NC);
      for (int gi = 0; gi < ngroups && ok; ++gi) {
        const int ga = gi * slots, gn = min(nact, ga + slots) - ga;
        if (ngroups > 1 && (nc > 0 || gi > 0)) {  // this group's left operand
          ok = bar_wait_or_stop(b.a_full, ph_afull, stop);
          ph_afull ^= 1u;
          if (!ok) break;
        }
        // operand B (block act[ga + k], this column chunk) runs up to a ring
        // ahead of the MMAs: a stage is refilled once the MMA that read it
        // has been issued (its commit frees the stage)
        const int st0 = stage;
        int issued = 0;
        for (int k = 0; k < gn && ok; ++k) {
          for (; issued < gn && issued < k + kT5Stages && ok; ++issued) {
            const int sL = (st0 + issued) % kT5Stages;
            ok = bar_wait_or_stop(b.b_empty + 8 * sL, ph_bempty[sL], stop);
            ph_bempty[sL] ^= 1u;
            if (!ok) break;
            bar_expect_tx(b.b_full + 8 * sL, bytes);
            bulk_g2s(saddr(w.B + (size_t)sL * ncmax * kT5K), a.MB + ((size_t)w.act[ga + issued] * np + c0) * kT5K,
                     bytes, b.b_full + 8 * sL);
            pending |= 1u << sL;
          }
          if (!ok) break;
          const int sI = (st0 + k) % kT5Stages;
          ok = bar_wait_or_stop(b.b_full + 8 * sI, ph_bfull[sI], stop);
          ph_bfull[sI] ^= 1u;
          if (!ok) break;
          pending &= ~(1u << sI);
          fence_after_sync();
          const uint64_t ad = smem_desc(saddr(w.A + (size_t)k * kT5ABytes), 128, 256);
          const uint64_t bd = smem_desc(saddr(w.B + (size_t)sI * ncmax * kT5K), 128, 256);
          mma_f8(d, ad, bd, id, (gi > 0 || k > 0) ? 1u : 0u);  // the chunk's first product overwrites
          mma_commit(b.b_empty + 8 * sI);
        }
        stage = (st0 + gn) % kT5Stages;
        if (ngroups > 1 && ok) mma_commit(b.a_empty);
      }
      if (!ok) break;
      mma_commit(b.acc_full[buf]);
      buf ^= 1;
    }
    if (ngroups <= 1 && ok) mma_commit(b.a_empty);
  }
  if (!ok) {
    atomicOr(&a.st->error, kErrTimeout);
    *stop = 1;
    // copies still in flight land before the CTA leaves
    for (int i = 0; i < kT5Stages; ++i)
      if (pending & (1u << i)) (void)bar_wait(b.b_full + 8 * i, ph_bfull[i]);
  }
  // every MMA issued completes before the TMEM is released
  mma_commit(b.drain);
  (void)bar_wait(b.drain, 0);
}

// The epilogue warps: per tile the digits (hash, repeats, active blocks), the
// left operand, then per column chunk C' = base + D from TMEM to the store.
__device__ void t5_epilogue(const Tc5Args& a, const Tc5Smem& w, const Tc5Bars& b, uint32_t tmem,
                            const CUtensorMap* map) {
  const DevSys& s = a.s;
  const int m = s.m, np = a.np, nblocks = a.nblocks, slots = a.slots;
  const int nbw = (nblocks + 31) / 32;
  const int nchunks = (np + kT5NC - 1) / kT5NC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  volatile int* stop = w.iscal + 5;
  const uint64_t ntiles = ((uint64_t)a.Q + kT5M - 1) / kT5M;
  uint64_t tile0, tile1;
  tile_range(a, tile0, tile1);
  uint32_t ph_aempty = 1u, ph_accfull[2] = {0u, 0u};
  int buf = 0, stg_i = 0;
  uint8_t* my_stg = w.stg + (size_t)warp * kT5Stg * 4096;
  const uint32_t lane_tmem = tmem + ((uint32_t)(warp * 32) << 16);
  bool ok = true;
  for (uint64_t tile = tile0; tile < tile1 && ok; ++tile) {
    const uint64_t lid0 = tile * kT5M;
    const uint32_t nrows = (uint32_t)min((uint64_t)kT5M, (uint64_t)a.Q - lid0);
    const uint64_t g_first = a.g0 + lid0, g_last = g_first + nrows - 1;
    if (warp == 0) {  // parent of the tile's first candidate, and whether the tile stays in it
      const long long cp = *w.cp;
      int64_t p;
      if (cp >= 0 && __ldcg(a.off + cp) <= g_first && g_first < __ldcg(a.off + cp + 1)) p = cp;
      else p = warp_find_parent(a.off, a.P, g_first, lane);
      if (lane == 0) {
        w.scal[2] = (unsigned long long)p;
        w.iscal[4] = (a.delta && g_last < __ldcg(a.off + p + 1)) ? 1 : 0;
      }
    }
    for (int i = tid; i < nbw; i += kT5M) w.bitmap[i] = 0u;
    ew_sync();
    const int64_t p_first = (int64_t)w.scal[2];
    const bool single = w.iscal[4] != 0;
    // The reference of a tile that follows a full tile of the same parent is
    // the candidate just before it, whose row, hash and repeat count the last
    // thread kept from that tile; otherwise the parent's state is rebuilt with
    // the tile's first candidate as reference.
    if (single && !(*w.cp == p_first && w.scal[3] == g_first))
      t5_load_parent(a, w, p_first, g_first - __ldcg(a.off + p_first));

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
    const int list_len = w.iscal[0];
    const uint64_t t_ref = w.scal[0];
    const int32_t* adj = w.adj + (size_t)w.iscal[1] * np;          // this tile's reference row - bias
    int32_t* adj_next = w.adj + (size_t)(w.iscal[1] ^ 1) * np;    // the next tile's
    const bool keep_last = single && nrows == (uint32_t)kT5M && tid == kT5M - 1;

    // pass 1: active blocks, hash, repeated-row choices
    uint64_t h = 0;
    bool red = false;
    if (valid) {
      bool good;
      if (single) {
        h = w.scal[1];
        int rc = w.iscal[2];
        good = t5_walk_delta(s, w, list_len, t, t_ref, [&](int rn, int ro, int dred) {
          mark_block(w, rn);
          mark_block(w, ro);
          h += __ldg(s.rowkey + rn) - __ldg(s.rowkey + ro);
          rc += dred;
        });
        red = rc > 0;
        if (keep_last) {  // the next tile's reference
          w.scal[4] = h;
          w.iscal[6] = rc;
        }
      } else {
        good = t5_walk_full(s, prow, t, [&](int r, uint32_t mask, int32_t x, int n) {
          h += col_hash(s, n, x);
          if (r < 0) return;
          mark_block(w, r);
          h += __ldg(s.rowkey + r);
          red |= redundant_choice(s, mask, r);
        });
      }
      if (!good) atomicOr(&a.st->error, kErrInternal);
      a.hash[lid] = h;
      a.red[lid] = red ? 1 : 0;
    }
    // the previous tile's MMAs have read the left operand and the block list
    ok = bar_wait_or_stop(b.a_empty, ph_aempty, stop);
    ph_aempty ^= 1u;
    if (ew_sync_or(!ok)) {
      ok = false;
      break;
    }
    if (warp == 0) {  // active blocks in increasing order
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
      if (lane == 0) w.iscal[3] = cnt;
    }
    ew_sync();
    const int nact = w.iscal[3];
    const int ngroups = (nact + slots - 1) / slots;
    // writes the left operand of group gi (blocks act[gi * slots ..]) and hands it to the control warp
    auto build_a = [&](int gi) {
      const int ga = gi * slots, gb = min(nact, ga + slots), gn = gb - ga;
      uint4* A4 = reinterpret_cast<uint4*>(w.A);
      for (int i = tid; i < gn * (kT5ABytes / 16); i += kT5M) A4[i] = make_uint4(0, 0, 0, 0);
      ew_sync();
      if (valid) {
        if (single) {
          t5_walk_delta(s, w, list_len, t, t_ref, [&](int rn, int ro, int) {
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
      ew_sync();
      if (tid == 0) bar_arrive(b.a_full);
    };
    if (ngroups <= 1) build_a(0);  // an empty tile hands over an empty operand

    const bool tma_rows = map != nullptr && lid0 + (uint64_t)warp * 32 + 32 <= (uint64_t)a.Q;
    const bool store = valid && !red;
    int32_t* orow = a.out + (size_t)lid * m;
    for (int nc = 0; nc < nchunks && ok; ++nc) {
      if (ngroups > 1) {
        for (int gi = 0; gi < ngroups && ok; ++gi) {
          if (nc > 0 || gi > 0) {
            ok = bar_wait_or_stop(b.a_empty, ph_aempty, stop);
            ph_aempty ^= 1u;
            if (ew_sync_or(!ok)) {
              ok = false;
              break;
            }
          }
          build_a(gi);
        }
        if (!ok) break;
      }
      ok = bar_wait_or_stop(b.acc_full[buf], ph_accfull[buf], stop);
      ph_accfull[buf] ^= 1u;
      if (ew_sync_or(!ok)) {
        ok = false;
        break;
      }
      fence_after_sync();
      const int c0 = nc * kT5NC, nc_cols = min(kT5NC, np - c0);
      const uint32_t acc = lane_tmem + (uint32_t)(buf * kT5NC);
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
        const int j0 = c0 + c;
        const int cnt = min(two ? 32 : 16, m - j0);
        if (cnt <= 0) continue;
        // bits(D + 1.5 * 2^23) = kT5Bias + D exactly (|D| < 2^22)
#pragma unroll
        for (int i = 0; i < 32; ++i) r[i] = __float_as_uint(__uint_as_float(r[i]) + 12582912.0f);
        // v = base + D = (base - bias) + bits(bias + D)
        if (single) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            if (i < cnt) {
              const int4 b4 = *reinterpret_cast<const int4*>(adj + j0 + i);
              r[i] += (uint32_t)b4.x;
              r[i + 1] += (uint32_t)b4.y;
              r[i + 2] += (uint32_t)b4.z;
              r[i + 3] += (uint32_t)b4.w;
            }
          }
          if (keep_last) {  // this row, less the bias, is the next tile's reference
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              if (i < cnt)
                *reinterpret_cast<int4*>(adj_next + j0 + i) =
                    make_int4((int)(r[i] - kT5Bias), (int)(r[i + 1] - kT5Bias), (int)(r[i + 2] - kT5Bias),
                              (int)(r[i + 3] - kT5Bias));
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (i < cnt) r[i] += (uint32_t)__ldcg(prow + j0 + i) - kT5Bias;
        }
        if (tma_rows && two) {  // 32 rows x 32 columns through the swizzled staging buffer
          uint8_t* sb = my_stg + (size_t)stg_i * 4096;
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kT5Stg - 1) : "memory");
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4*>(sb + lane * 128 + ((q ^ (lane & 7)) * 16)) =
                make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
          fence_async_smem();
          __syncwarp();
          if (lane == 0) tma_store_2d(map, j0, (int)(a.store_row0 + lid0 + (uint64_t)warp * 32), saddr(sb));
          stg_i = (stg_i + 1) % kT5Stg;
        } else if (store) {
          if ((m & 3) == 0) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              if (i < cnt)
                __stcg(reinterpret_cast<int4*>(orow + j0 + i),
                       make_int4((int)r[i], (int)r[i + 1], (int)r[i + 2], (int)r[i + 3]));
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < cnt) __stcg(orow + j0 + i, (int)r[i]);
          }
        }
      }
      // the buffer is free again
      fence_before_sync();
      __syncwarp();
      if (lane == 0) bar_arrive(b.acc_empty[buf]);
      buf ^= 1;
    }
    ew_sync();
    if (tid == 0) {  // the chain of references: the next tile may start from this one's last candidate
      if (single && nrows == (uint32_t)kT5M) {
        w.scal[3] = g_first + kT5M;
        w.scal[0] = t + (kT5M - 1);
        w.scal[1] = w.scal[4];
        w.iscal[2] = w.iscal[6];
        w.iscal[1] ^= 1;
      } else {
        w.scal[3] = ~0ull;
      }
    }
  }
  if (!ok) {
    atomicOr(&a.st->error, kErrTimeout);
    *stop = 1;
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncwarp();
}

__global__ void __launch_bounds__(kT5Threads, 2) k_tc5_expand(Tc5Args a, const __grid_constant__ CUtensorMap map) {
  if (a.ctr && __ldcg(a.ctr + 1) == 0) return;  // the depth is full: nothing to do
  extern __shared__ unsigned char t5_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)t5_raw + 1023) & ~(uintptr_t)1023);
  const int m = a.s.m, np = a.np;
  Tc5Smem w = carve(base, m, np, a.nblocks, a.slots);
  const Tc5Bars b = bars_of(w);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    bar_init(b.a_full, 1);
    bar_init(b.a_empty, 1);
    for (int i = 0; i < 2; ++i) {
      bar_init(b.acc_full[i], 1);
      bar_init(b.acc_empty[i], 4);
    }
    bar_init(b.drain, 1);
    for (int i = 0; i < kT5Stages; ++i) {
      bar_init(b.b_full + 8 * i, 1);
      bar_init(b.b_empty + 8 * i, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *w.cp = -1;
    w.scal[3] = ~0ull;
    w.iscal[5] = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(w.tmem_slot)),
                 "r"((uint32_t)(2 * kT5NC)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *w.tmem_slot;

  if (warp < 4) {
    t5_epilogue(a, w, b, tmem, a.use_map ? &map : nullptr);
  } else {
    if ((tid & 31) == 0) t5_control(a, w, b, tmem);
    __syncwarp();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * kT5NC)));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

}  // namespace

int tc5_slots(int m, int nblocks) {
  // two CTAs per SM (256 TMEM columns each): at most 113 KB of shared memory each
  int slots = kT5MaxSlots;
  while (slots > 1 && tc5_smem_bytes(m, nblocks, slots) > (113u << 10)) --slots;
  return slots;
}

bool tc5_store_map(CUtensorMap* map, int32_t* pool, int m, uint64_t rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc || (m & 3) != 0 || m < 32 || rows == 0 || rows > 0x7FFFFFFFull) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)m * 4};
  const cuuint32_t box[2] = {32, 32}, es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, pool, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_tc5(const Tc5Args& a, const CUtensorMap& map, cudaStream_t st, int nsm) {
  // more than a third of an SM's shared memory: two CTAs (256 TMEM columns each) per SM
  const size_t smem = std::max<size_t>(tc5_smem_bytes(a.s.m, a.nblocks, a.slots), 80u << 10);
  cudaFuncSetAttribute(k_tc5_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const uint64_t ntiles = ((uint64_t)a.Q + kT5M - 1) / kT5M;
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, 2ull * nsm));
  k_tc5_expand<<<blocks, kT5Threads, smem, st>>>(a, map);
}

}  // namespace snp
