// Kernel entry points of the single-system BFS (declarations shared by the
// launch code in snp_api.cu and the definitions in snp_kernels.cu).
#pragma once

#include <cuda.h>

#include "snp_device.cuh"

namespace snp {

struct ClaimArgs {
  DevSys sys;
  const int32_t* parents;     // frontier rows: parents + pperm[p] * m, or parents + p * m without pperm
  const uint32_t* pperm;      // [P] store rows of the frontier, or nullptr
  const uint64_t* off;        // [P + 1] exclusive prefix sums of Psi (saturating)
  int64_t P;
  uint64_t g0;                // first candidate of the chunk
  uint32_t Q;                 // candidates in the chunk
  uint32_t run;               // consecutive candidates per warp task
  DevTable table;
  int32_t* pool;              // committed configurations (store mode: every claimed row, in claim order)
  int32_t* staging;           // [Q x m] row lid = candidate lid's configuration if lid claimed a new key
  // Store mode (store_ctr set): an owner takes the next row of the store
  // (pool) instead of staging row lid, and records it in sidx_of[lid].
  unsigned long long* store_ctr;
  uint32_t* sidx_of;          // [Q]
  uint64_t store_cap;         // rows the store holds
  uint32_t* gmin;             // [Q] per claiming lid: smallest chunk-local candidate holding its key
  uint32_t* slot_of;          // [Q] per claiming lid: its table slot
  uint32_t* ownbits;          // [Q / 32 + 1] bit lid set iff candidate lid claimed a new key
  const ParentRec* prec;      // [P] parent summaries, or nullptr (decode from the rows)
  const unsigned long long* ctr;  // device counters {rows, still acceptable} or nullptr; none left: no work
  ChunkState* st;
  // Rows already in the store (the fp8 tensor-core form writes candidate
  // lid's row to store row inplace_base + lid): an owner publishes it there.
  int32_t inplace = 0;
  uint64_t inplace_base = 0;
  uint64_t wait_ns = 0;       // > 0: time limit of a wait for a slot being claimed
  // Bytes per spike count of the rows of parents, pool and staging: 4
  // (int32), or 2 / 1 in a packed store (uint16 / uint8; m a multiple of 8 /
  // 16).  The pointers keep their int32_t type in every case.
  int32_t w = 4;
  // Wide mode: base children of the pass's largest parents (wide_base_bytes;
  // filled by the launch before each pass), or nullptr.
  int32_t* bcache = nullptr;
};

// Wide mode: base children cached per pass (headers, then rows of round4(m)).
constexpr int kBaseSlots = 8;
size_t wide_base_bytes(int m);

struct CommitArgs {
  DevSys sys;
  uint32_t nwords;            // ceil(Q / 32)
  const uint32_t* bits;       // [nwords] first-occurrence bitmap over chunk-local indices
  const uint32_t* wbase;      // [nwords] exclusive prefix of popcounts
  const uint32_t* srow;       // [Q] owner (candidate that claimed the key) of each first occurrence
  const uint32_t* slot_of;
  const int32_t* staging;
  DevTable table;
  int32_t* pool;
  // Store mode (perm set): rows stay where their owners stored them;
  // perm[row] = sidx_of[owner] records the store row of discovery index row.
  uint32_t* perm;
  const uint32_t* sidx_of;
  int64_t row_base;           // pool row of rank 0
  uint64_t remaining;         // how many more configurations the depth may accept
  const unsigned long long* ctr;  // or, when set, both from device counters {rows, still acceptable}
  // parent records (optional)
  int64_t* rec_parent;        // [rows] or nullptr
  uint64_t* rec_index;
  const uint64_t* off;
  int64_t P;
  int64_t parent_base;        // discovery index of frontier row 0
  uint64_t g0;
  ChunkState* st;
};

// ---------------------------------------------------------------------------
// Batch engine: many independent systems advance one depth per launch.

// One system of a batch (device memory; updated by the batch kernel).
struct BatchSys {
  DevSys sys;
  int32_t* pool;               // configurations, discovery order, pool_rows rows
  unsigned long long* slots;   // the system's own hash table
  uint64_t bmask;              // buckets - 1
  int64_t pool_rows;
  int64_t level_lo, level_hi;  // current frontier: pool rows [level_lo, level_hi)
  int64_t n_rows;
  int32_t done;                // a depth found nothing new: the system is finished
  uint32_t error;              // kErr* bits
  int32_t depth_reached;
  int32_t cur_depth;           // depths completed so far
  int32_t target_depth;        // depths to run
  int32_t max_expand;
  int64_t cap, budget;         // per-depth frontier cap (>= 1) and candidate budget (<= 0: none)
  struct BatchDepthStat* stats;  // [target_depth + 1]
  // fp8 tensor-core form: M_Pi^T in e4m3 (tc5_pack_mt layout), columns rounded to 16, rule blocks
  const uint8_t* MB;
  int32_t np, nblocks;
};

struct BatchDepthStat {
  int64_t new_configs;
  int64_t examined;
  uint64_t candidates;
  int32_t truncated;
  int32_t chunks;
};

// One launch advances every system by one depth (cur_depth + 1), unless it
// is finished or has run target_depth depths.
struct BatchArgs {
  BatchSys* sys;               // [n]
  int32_t n;
  int32_t launch;              // index of this launch (its work counter)
  uint32_t qc;                 // candidates per pass
  int32_t B, ts, run;          // expand tile rows, tile row stride (words), candidates per warp task
  size_t warp_smem;            // bytes of shared memory per warp
  unsigned int* queue;         // work counters, one per launch, zero before it
  unsigned char* scratch;      // per-CTA scratch
  size_t scratch_stride;
  int64_t pmax;                // largest frontier a system may have (largest cap)
  int32_t m_max;
  int32_t tc;                  // 1: rows by the fp8 tensor-core form (four warps per CTA)
};

// Bytes of per-CTA scratch for frontiers of up to pmax rows and passes of qc candidates.
size_t batch_scratch_bytes(int64_t pmax, uint32_t qc, int m_max);
// Per-warp shared memory of the expand loop for rows of up to m_max neurons.
size_t expand_smem_bytes(int m_max, int B, int* ts);
void launch_batch_depth(const BatchArgs& a, int blocks, int warps, cudaStream_t st);
// Dynamic shared memory of the batch kernel's tensor-core form.
size_t batch_tc_smem_bytes_host();
__global__ void k_batch_init(BatchSys* sys, const int32_t* c0, const int64_t* c0_off, int32_t n);

// Step (a) and Psi for P frontier rows; returns the launches made.
// rows: w bytes per spike count (4: int32; 2, 1: a packed store).
int launch_psi(DevSys s, const int32_t* rows, int w, const uint32_t* perm, int64_t P, int32_t max_expand,
               uint64_t* psi, ParentRec* rec, ChunkState* st, cudaStream_t stream, int nsm);
// Sets st->psi_saturated when Psi summed (saturating) over psi[0 .. n) is
// 2^64 - 1: later frontier rows then hold no candidate, and launch_psi with
// that st writes Psi = 0 for them without reading them.
int launch_psi_head_check(const uint64_t* psi, int64_t n, ChunkState* st, cudaStream_t stream);
// Steps (b)-(d) for the chunk's candidates (k_expand); returns the launches made.
// Rows of more than kWideM neurons go through the kernel's wide mode (one
// scratch row per warp, rows built on demand).
constexpr int kWideM = 128;
int launch_expand(ClaimArgs a, cudaStream_t st, int nsm);
// Step (d) for candidate rows already in global memory (rows[lid * m], hash[lid]).
// Candidates with redundant[lid] set repeat an earlier candidate and are skipped.
void launch_resolve_rows(ClaimArgs a, const int32_t* rows, const unsigned long long* hash, const uint8_t* redundant,
                         cudaStream_t st, int nsm);
// Tensor-core form of step (c) (snp_tc.cu).
void launch_tc_digits(DevSys s, const int32_t* parents, const uint32_t* perm, const uint64_t* off, int64_t P,
                      uint64_t g0, uint32_t Q,
                      uint8_t* loc, int mp, uint32_t* pidx, uint8_t* redundant, cudaStream_t st, int nsm);
void launch_tc_rows(DevSys s, const int32_t* parents, const uint8_t* loc, int mp, const uint32_t* pidx, uint32_t Q,
                    const int8_t* MT, int Rp, const int16_t* rn, const uint8_t* rk, int32_t* rows,
                    unsigned long long* hash, cudaStream_t st);
size_t tc_rows_smem(int mp);
// fp8 tensor-core form of step (c) on tcgen05 (snp_tc5.cu): candidate rows
// C' = C + S . M_Pi written to out[lid * m], their linear hashes and repeat flags.
struct Tc5Args {
  DevSys s;
  const int32_t* parents;     // the store (parents + pperm[p] * m) or frontier rows
  const uint32_t* pperm;
  const uint64_t* off;        // [P + 1] saturating exclusive scan of Psi
  int64_t P;
  uint64_t g0;
  uint32_t Q;
  const uint8_t* MB;          // M_Pi^T in e4m3, tc5_pack_mt layout
  int np;                     // columns rounded up to 16
  int nblocks;                // rule blocks: ceil(R / 32)
  int slots;                  // rule blocks held in shared memory at once (tc5_slots)
  int delta;                  // 1: delta form for tiles within one parent
  int32_t* out;               // [Q][m]: row lid = candidate lid's configuration (store row store_row0 + lid)
  uint64_t store_row0;        // store row of candidate 0 (the TMA store's row coordinate)
  int use_map;                // 1: rows go out through the tensor map given at launch
  unsigned long long* hash;   // [Q] linear hash h(C') of each candidate
  uint8_t* red;               // [Q] 1: repeats an earlier candidate of the same parent
  const unsigned long long* ctr;  // device counters {rows, still acceptable}: none left: no work
  ChunkState* st;
};
size_t tc5_smem_bytes(int m, int nblocks, int slots);
int tc5_slots(int m, int nblocks);
// Tensor map of the store (int32 [rows][m]) for the TMA row stores: 32 x 32
// boxes, 128-byte swizzle.  false: not available (m % 4 != 0, m < 32, or no
// driver entry point); rows are then stored by the threads.
bool tc5_store_map(CUtensorMap* map, int32_t* pool, int m, uint64_t rows);
void launch_tc5(const Tc5Args& a, const CUtensorMap& map, cudaStream_t st, int nsm);
__global__ void k_mark(uint32_t* ownbits, const uint32_t* gmin, uint32_t* bits, uint32_t* srow, uint32_t nwords,
                       ChunkState* st);
__global__ void k_commit(CommitArgs a);
void launch_iota_u32(uint32_t* out, int64_t n, cudaStream_t st);
// out[k] = row perm[k] (row k without perm) of a pool of w bytes per count, as int32.
void launch_gather_rows(const int32_t* pool, int w, const uint32_t* perm, int64_t n, int m, int32_t* out,
                        cudaStream_t st);
// Testing hook: marks the slot holding store row `row` as being claimed.
__global__ void k_hold_slot_of_row(unsigned long long* slots, uint64_t n, uint32_t row);
__global__ void k_clear_bits(uint32_t* bits, uint32_t nwords, unsigned long long* ctr, const ChunkState* st);
// *out = max(*out, x[0 .. n)) for counts x >= 0.
void launch_count_max(const int32_t* x, int64_t n, int32_t* out, cudaStream_t st);
// n int32 rows of m counts (m % 8 == 0, each count within the range of w
// bytes) into rows of w = 1 or 2 bytes per count at dst.
void launch_pack_rows(const int32_t* src, int64_t n, int m, int w, int32_t* dst, cudaStream_t st);
// Inserts rows [r0, r1) of a pool of w bytes per count into the table
// (blocks CTAs of kWarpsPerBlock warps).
void launch_insert_rows(DevSys s, const int32_t* pool, int w, const uint32_t* perm, int64_t r0, int64_t r1,
                        DevTable t, ChunkState* st, int blocks, cudaStream_t stream);
__global__ void k_step_children(DevSys s, const int32_t* C, uint64_t n, int32_t* out);
__global__ void k_fill_u64(unsigned long long* p, uint64_t n, unsigned long long v);

// Device-wide exclusive scans (n elements, in -> out; "total" gets the sum).
// Saturating for u64 (sums of Psi), plain for u32.
size_t scan_temp_bytes(int64_t n, size_t elem);
// Each returns the number of kernels it launched.
int scan_u64_sat(const uint64_t* in, uint64_t* out, int64_t n, void* temp, cudaStream_t st);
int scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* temp, cudaStream_t st);
void launch_popc(const uint32_t* bits, uint32_t* cnt, uint32_t nwords, cudaStream_t st);

}  // namespace snp
