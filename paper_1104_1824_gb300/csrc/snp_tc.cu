// Exact int8 tensor-core form of step (c): C' = C + S . M_Pi (Eq. next-config)
// as a dense product of the chunk's spiking vectors S (0/1, int8, Q x R) with
// M_Pi (int8, R x m), accumulated in int32 by mma.sync m16n8k32 (the int8
// tensor-core instruction sm_103a accepts).  The product is exact: each row of
// S holds at most one 1 per neuron, so every output is a sum of at most m
// entries of M_Pi, each in [-127, 127], far inside int32.
//
// Per chunk:
//   k_tc_digits  one warp per run of candidates: parent, and per neuron the
//                chosen rule's position among the neuron's rules (0xFF: none);
//   k_tc_rows    64 candidates x 128 columns per block; each 32-rule slice of
//                S is generated in shared memory from the digits, M_Pi^T comes
//                from L2, four warps issue mma.sync; the epilogue adds the
//                parent row, writes C' and accumulates its linear hash;
//   then the rows are resolved against the hash table as in the sparse path.
#include "snp_kernels.cuh"

namespace snp {

namespace {

constexpr int kTcBM = 64;        // candidates per block
constexpr int kTcBN = 128;       // columns per pass of a block
constexpr int kTcBK = 32;        // rules per k-step
constexpr int kTcAStride = 48;   // bytes per A-tile row (conflict-free fragment loads)

__device__ __forceinline__ void mma_s8(int (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

}  // namespace

// Step (b) for the chunk: per candidate its parent's row (perm[p] when the
// frontier is reached through a row map, else p) and, per neuron, the
// position of the chosen rule among the neuron's rules.
__global__ void __launch_bounds__(128) k_tc_digits(DevSys s, const int32_t* parents, const uint32_t* perm,
                                                   const uint64_t* off, int64_t P,
                                                   uint64_t g0, uint32_t Q, uint8_t* loc, int mp, uint32_t* pidx,
                                                   uint8_t* redundant) {
  extern __shared__ int32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int m = s.m;
  WarpParent w;
  w.par = smem + (size_t)wib * 2 * m;
  w.msk = reinterpret_cast<uint32_t*>(w.par + m);
  w.buf = nullptr;
  const uint32_t run = 32;
  const uint64_t ntasks = ((uint64_t)Q + run - 1) / run;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t task = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib; task < ntasks; task += nw) {
    const uint64_t la = task * run, lb = min(la + run, (uint64_t)Q);
    int64_t p = warp_find_parent(off, P, g0 + la, lane);
    uint64_t p_lo = __ldg(off + p), p_hi = __ldg(off + p + 1);
    uint32_t prow = perm ? __ldg(perm + p) : (uint32_t)p;
    load_parent(s, parents + (size_t)prow * m, w, lane);
    for (uint64_t l = la; l < lb; ++l) {
      const uint64_t g = g0 + l;
      if (g >= p_hi) {
        do {
          ++p;
          p_lo = p_hi;
          p_hi = __ldg(off + p + 1);
        } while (g >= p_hi);
        prow = perm ? __ldg(perm + p) : (uint32_t)p;
        load_parent(s, parents + (size_t)prow * m, w, lane);
      }
      const uint64_t t = g - p_lo;
      const int n0 = lane * s.K, n1 = min(n0 + s.K, m);
      uint64_t q = (w.after > t) ? 0ull : t / w.after;
      uint8_t* dst = loc + (size_t)l * mp;
      bool red = false;
      for (int n = n1 - 1; n >= n0; --n) {
        const uint32_t mask = w.msk[n];
        if (!mask) {
          dst[n] = 0xFF;
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
        const int k = nth_set_bit(mask, (int)d);
        dst[n] = (uint8_t)k;
        red |= redundant_choice(s, mask, __ldg(s.first_rule + n) + k);
      }
      red = __any_sync(0xffffffffu, red);
      if (lane == 0) {
        pidx[l] = prow;
        redundant[l] = red ? 1 : 0;
      }
      __syncwarp();
    }
  }
}

// C' = C + S . M_Pi for 64 candidates per block (all m columns, 128 per pass),
// its linear hash into hash[lid] (which must start at zero).
//   MT: M_Pi transposed, int8 [mt_rows >= round_up(m, 128)][Rp = round_up(R, 32)], zero padded.
//   rn/rk: per rule its neuron and position among the neuron's rules (Rp entries; padding rules: rn = -1).
__global__ void __launch_bounds__(128) k_tc_rows(DevSys s, const int32_t* parents, const uint8_t* loc, int mp,
                                                 const uint32_t* pidx, uint32_t Q, const int8_t* MT, int Rp,
                                                 const int16_t* rn, const uint8_t* rk, int32_t* rows,
                                                 unsigned long long* hash) {
  extern __shared__ __align__(16) unsigned char tc_smem[];
  const int m = s.m;
  uint8_t* locs = tc_smem;                                   // [64][mp]
  uint8_t* At = locs + (size_t)kTcBM * mp;                   // [64][48]
  int32_t* prow = reinterpret_cast<int32_t*>(At + kTcBM * kTcAStride);  // [64] parent index
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const uint32_t base = blockIdx.x * kTcBM;
  const int nrows = (int)((Q - base) < (uint32_t)kTcBM ? (Q - base) : (uint32_t)kTcBM);
  // stage the block's digits and parents
  for (int i = tid; i < kTcBM * (mp / 4); i += blockDim.x) {
    const int r = i / (mp / 4), c = i % (mp / 4);
    const uint32_t v = r < nrows ? reinterpret_cast<const uint32_t*>(loc + (size_t)(base + r) * mp)[c] : 0xFFFFFFFFu;
    reinterpret_cast<uint32_t*>(locs + (size_t)r * mp)[c] = v;
  }
  for (int i = tid; i < kTcBM; i += blockDim.x) prow[i] = i < nrows ? (int32_t)pidx[base + i] : 0;
  __syncthreads();

  const int row0 = warp * 16 + g, row1 = row0 + 8;
  for (int c0 = 0; c0 < m; c0 += kTcBN) {
    int acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0;
    for (int r0 = 0; r0 < Rp; r0 += kTcBK) {
      __syncthreads();
      {  // S slice: 64 rows x 32 rules, 16 bytes per thread
        const int i = tid >> 1, cb = (tid & 1) * 16;
        uint32_t word[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t wv = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = r0 + cb + q * 4 + b;
            const int n = rn[r];
            const uint32_t bit = (n >= 0 && locs[(size_t)i * mp + n] == rk[r]) ? 1u : 0u;
            wv |= bit << (8 * b);
          }
          word[q] = wv;
        }
        *reinterpret_cast<uint4*>(At + i * kTcAStride + cb) = make_uint4(word[0], word[1], word[2], word[3]);
      }
      __syncthreads();
      const uint32_t a0 = *reinterpret_cast<const uint32_t*>(At + row0 * kTcAStride + 4 * t4);
      const uint32_t a1 = *reinterpret_cast<const uint32_t*>(At + row1 * kTcAStride + 4 * t4);
      const uint32_t a2 = *reinterpret_cast<const uint32_t*>(At + row0 * kTcAStride + 16 + 4 * t4);
      const uint32_t a3 = *reinterpret_cast<const uint32_t*>(At + row1 * kTcAStride + 16 + 4 * t4);
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        const int8_t* bcol = MT + (size_t)(c0 + nt * 8 + g) * Rp + r0 + 4 * t4;
        const uint32_t b0 = __ldg(reinterpret_cast<const uint32_t*>(bcol));
        const uint32_t b1 = __ldg(reinterpret_cast<const uint32_t*>(bcol + 16));
        mma_s8(acc[nt], a0, a1, a2, a3, b0, b1);
      }
    }
    // epilogue: add the parent row, store C', accumulate the linear hash
    uint64_t h0 = 0, h1 = 0;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = c0 + nt * 8 + 2 * t4 + (e & 1);
        const int i = (e < 2) ? row0 : row1;
        if (col < m && i < nrows) {
          const int32_t v = __ldg(parents + (size_t)prow[i] * m + col) + acc[nt][e];
          rows[(size_t)(base + i) * m + col] = v;
          const uint64_t hv = (uint64_t)(uint32_t)v * __ldg(s.colkey + col);
          if (e < 2) h0 += hv; else h1 += hv;
        }
      }
    }
    h0 += __shfl_xor_sync(0xffffffffu, h0, 1);
    h0 += __shfl_xor_sync(0xffffffffu, h0, 2);
    h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
    h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
    if (t4 == 0) {
      if (row0 < nrows) atomicAdd(hash + base + row0, (unsigned long long)h0);
      if (row1 < nrows) atomicAdd(hash + base + row1, (unsigned long long)h1);
    }
  }
}

// Peak of mma.sync m16n8k32 s8 on this GPU: each warp issues `iters` rounds of
// 8 independent products; out receives a value that depends on every product.
__global__ void __launch_bounds__(128) k_tc_peak(int iters, int* out) {
  int acc[8][4];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0;
  const uint32_t a = 0x01010101u * (threadIdx.x & 3), b = 0x01010101u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) mma_s8(acc[k], a, a + it, a, a, b, b + k);
  }
  int sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += acc[k][0] + acc[k][1] + acc[k][2] + acc[k][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

void launch_tc_digits(DevSys s, const int32_t* parents, const uint32_t* perm, const uint64_t* off, int64_t P,
                      uint64_t g0, uint32_t Q,
                      uint8_t* loc, int mp, uint32_t* pidx, uint8_t* redundant, cudaStream_t st, int nsm) {
  const size_t smem = (size_t)4 * 2 * s.m * sizeof(int32_t);
  const uint64_t ntasks = ((uint64_t)Q + 31) / 32;
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((ntasks + 3) / 4, (uint64_t)nsm * 16));
  k_tc_digits<<<blocks, 128, smem, st>>>(s, parents, perm, off, P, g0, Q, loc, mp, pidx, redundant);
}

size_t tc_rows_smem(int mp) { return (size_t)kTcBM * mp + kTcBM * kTcAStride + kTcBM * sizeof(int32_t); }

void launch_tc_rows(DevSys s, const int32_t* parents, const uint8_t* loc, int mp, const uint32_t* pidx, uint32_t Q,
                    const int8_t* MT, int Rp, const int16_t* rn, const uint8_t* rk, int32_t* rows,
                    unsigned long long* hash, cudaStream_t st) {
  const size_t smem = tc_rows_smem(mp);
  if (smem > (48u << 10)) cudaFuncSetAttribute(k_tc_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned blocks = (Q + kTcBM - 1) / kTcBM;
  k_tc_rows<<<blocks, 128, smem, st>>>(s, parents, loc, mp, pidx, Q, MT, Rp, rn, rk, rows, hash);
}

}  // namespace snp

extern "C" int snp_tc_peak_tops(int32_t iters, double* tops) {
  if (!tops || iters < 1) return 1;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 4;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8, threads = 128;
  int* out = nullptr;
  if (cudaMalloc(&out, sizeof(int) * blocks * threads) != cudaSuccess) return 3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  snp::k_tc_peak<<<blocks, threads>>>(iters / 10 + 1, out);  // warm-up
  cudaEventRecord(e0);
  snp::k_tc_peak<<<blocks, threads>>>(iters, out);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return 4;
  const double ops = 2.0 * 16 * 8 * 32 * 8.0 * iters * (double)blocks * (threads / 32);
  *tops = ops / (ms * 1e-3) / 1e12;
  return 0;
}
