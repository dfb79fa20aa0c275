// Batch engine, host side (snp_explore_batch, snp_batch_autotune): packs many
// loaded systems into one device arena and advances them all one depth per
// launch of k_batch_depth, the depth launches captured in one CUDA graph.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "snp_host.h"

using namespace snp;

namespace snp {

// Device memory of one batch; shared by its handles until they move on.
struct BatchArena {
  DevBuf sys, stats, pools, slots, scratch, queue, c0, c0_off;
  int32_t n = 0, depth = 0;
  // shape the buffers and the captured graph were made for
  std::vector<snp_system*> handles;
  int64_t cap = 0, budget = 0;
  int32_t max_expand = 0, blocks = 0, warps = 0, B = 0, tc = 0;
  uint32_t qc = 0;
  uint64_t nslots = 0;
  size_t scratch_stride = 0, pool_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  ~BatchArena() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

}  // namespace snp

namespace {

struct BatchPlan {
  uint32_t qc = 2048;
  int tile = 0, warps = 8;
};

int batch_setup(snp_handle* hs, int32_t n, const snp_explore_opts* o) {
  if (!hs || n < 1 || !o) return fail(SNP_E_INVALID, "bad arguments");
  if (o->depth < 0) return fail(SNP_E_INVALID, "depth = %d < 0", o->depth);
  if (o->transition == SNP_T_TC_I8)
    return fail(SNP_E_INVALID, "the batch engine's tensor-core form is SNP_T_TC_F8 (tcgen05 has no int8 kind on this GPU)");
  if (o->transition != SNP_T_SPARSE_I32 && o->transition != SNP_T_TC_F8)
    return fail(SNP_E_INVALID, "unknown transition %d", o->transition);
  if (o->record_parents) return fail(SNP_E_INVALID, "the batch engine keeps no parent records");
  if (o->frontier_cap < 1 || o->frontier_cap > (1 << 20))
    return fail(SNP_E_INVALID, "the batch engine needs 1 <= frontier_cap <= 2^20 (got %lld)", (long long)o->frontier_cap);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  for (int32_t i = 0; i < n; ++i) {
    if (!hs[i]) return fail(SNP_E_INVALID, "handle %d is NULL", i);
    if (hs[i]->device != dev) return fail(SNP_E_INVALID, "handle %d lives on device %d, not %d", i, hs[i]->device, dev);
    if (o->transition == SNP_T_TC_F8) {
      if (hs[i]->max_abs_m > 16)
        return fail(SNP_E_RANGE, "fp8 transition refused: |M_Pi| of system %d reaches %d > 16", i, hs[i]->max_abs_m);
      if ((hs[i]->R + 31) / 32 > 1024) return fail(SNP_E_INVALID, "system %d has more than 32768 rules", i);
      TRY(tc5_prepare(hs[i], 0));
    }
  }
  return SNP_OK;
}

// Runs depths 1..depth of the batch (all handles) with the given plan; fills
// the handles' results.  ms (optional) receives the device time of the depths.
int batch_run(snp_handle* hs, int32_t n, const snp_explore_opts* o, const BatchPlan& plan, int32_t* statuses,
              float* ms) {
  const int dev = hs[0]->device;
  CK(cudaSetDevice(dev));
  cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  const int nsm = sm_count(dev);
  const int64_t cap = o->frontier_cap;
  const int depth = o->depth;
  const bool tc = o->transition == SNP_T_TC_F8;
  int m_max = 1;
  for (int32_t i = 0; i < n; ++i) m_max = std::max(m_max, hs[i]->m);
  const int64_t rows_per = 1 + (int64_t)depth * cap;
  const uint64_t want_slots = (uint64_t)((long double)(rows_per + (int64_t)depth * plan.qc) * 4.0L / 3.0L) + kBucket;
  const uint64_t nslots = std::max<uint64_t>(pow2_at_least(want_slots), kBucket);
  // tile rows and warps
  int ts = 0;
  int B = plan.tile > 0 ? plan.tile : 32;  // shrunk below to what the shared memory holds
  const int warps = (tc || plan.warps == 4) ? 4 : 8;
  size_t warp_smem = expand_smem_bytes(m_max, B, &ts);
  while (B > 1 && warp_smem * warps > (200u << 10)) warp_smem = expand_smem_bytes(m_max, --B, &ts);
  if (plan.tile <= 0 && B > 16 && B < 32) {  // measured: 16 rows beat 17 (-3%) and 18 (-17%) on the batch workload
    B = 16;
    warp_smem = expand_smem_bytes(m_max, B, &ts);
  }
  if (!tc && warp_smem * warps > (220u << 10))
    return fail(SNP_E_INVALID, "rows of %d neurons do not fit the batch tile", m_max);
  int blocks_per_sm = 1;
  {
    int nb = 0;
    // one CTA per SM is always resident; two when registers and shared memory allow (the
    // tensor-core form: two CTAs of 128 TMEM columns each)
    nb = tc ? 2 : (warps == 4 && warp_smem * warps * 2 <= (200u << 10)) ? 2 : 1;
    blocks_per_sm = nb;
  }
  if (tc) B = 0;
  const int blocks = std::max(1, std::min<int>(nsm * blocks_per_sm, n));
  const size_t scratch_stride = (batch_scratch_bytes(cap, plan.qc, m_max) + 255) & ~size_t(255);

  size_t pool_bytes = 0;
  std::vector<size_t> pool_off(n);
  for (int32_t i = 0; i < n; ++i) {
    pool_off[i] = pool_bytes;
    pool_bytes += ((size_t)rows_per * hs[i]->m * sizeof(int32_t) + 255) & ~size_t(255);
  }
  // Reuse the arena (and its graph) of the previous batch over the same handles and shape.
  std::shared_ptr<BatchArena> arena = hs[0]->batch;
  bool same = arena && arena->n == n && arena->depth == depth && arena->cap == cap &&
              arena->budget == (o->candidate_budget > 0 ? o->candidate_budget : 0) &&
              arena->max_expand == o->max_expand_value && arena->blocks == blocks && arena->warps == warps &&
              arena->B == B && arena->qc == plan.qc && arena->nslots == nslots && arena->pool_bytes == pool_bytes &&
              arena->scratch_stride == scratch_stride && arena->tc == (tc ? 1 : 0);
  for (int32_t i = 0; same && i < n; ++i) same = arena->handles[i] == hs[i] && hs[i]->batch == arena;
  if (!same) {
    arena = std::make_shared<BatchArena>();
    arena->n = n;
    arena->depth = depth;
    arena->handles.assign(hs, hs + n);
    arena->cap = cap;
    arena->budget = o->candidate_budget > 0 ? o->candidate_budget : 0;
    arena->max_expand = o->max_expand_value;
    arena->blocks = blocks;
    arena->warps = warps;
    arena->B = B;
    arena->qc = plan.qc;
    arena->nslots = nslots;
    arena->pool_bytes = pool_bytes;
    arena->scratch_stride = scratch_stride;
    arena->tc = tc ? 1 : 0;
    for (int32_t i = 0; i < n; ++i) {  // release older arenas before allocating
      hs[i]->batch.reset();
      hs[i]->result_pool = nullptr;
      hs[i]->result_perm = nullptr;
      hs[i]->explored = false;
    }
  }
  TRY(arena->sys.reserve(sizeof(BatchSys) * n));
  TRY(arena->stats.reserve(sizeof(BatchDepthStat) * n * (depth + 1)));
  TRY(arena->pools.reserve(pool_bytes));
  TRY(arena->slots.reserve(sizeof(unsigned long long) * nslots * n));
  TRY(arena->scratch.reserve(scratch_stride * blocks));
  TRY(arena->queue.reserve(sizeof(unsigned int) * (depth + 1)));
  std::vector<int32_t> c0;
  std::vector<int64_t> c0_off(n);
  std::vector<BatchSys> sys(n);
  for (int32_t i = 0; i < n; ++i) {
    snp_system* h = hs[i];
    c0_off[i] = (int64_t)c0.size();
    c0.insert(c0.end(), h->c0.begin(), h->c0.end());
    BatchSys& b = sys[i];
    std::memset(&b, 0, sizeof b);
    b.sys = h->dev();
    b.pool = reinterpret_cast<int32_t*>(arena->pools.as<char>() + pool_off[i]);
    b.slots = arena->slots.as<unsigned long long>() + (size_t)i * nslots;
    b.bmask = nslots / kBucket - 1;
    b.pool_rows = rows_per;
    b.level_lo = 0;
    b.level_hi = 1;
    b.n_rows = 1;
    b.cur_depth = 0;
    b.target_depth = depth;
    b.max_expand = o->max_expand_value;
    b.cap = cap;
    b.budget = o->candidate_budget > 0 ? o->candidate_budget : 0;
    b.stats = arena->stats.as<BatchDepthStat>() + (size_t)i * (depth + 1);
    b.MB = tc ? h->d_MB.as<uint8_t>() : nullptr;
    b.np = h->t5_np;
    b.nblocks = h->t5_nblocks;
  }
  TRY(arena->c0.reserve(sizeof(int32_t) * c0.size()));
  TRY(arena->c0_off.reserve(sizeof(int64_t) * n));
  CK(cudaMemcpyAsync(arena->sys.p, sys.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(arena->c0.p, c0.data(), sizeof(int32_t) * c0.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(arena->c0_off.p, c0_off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(arena->stats.p, 0, sizeof(BatchDepthStat) * n * (depth + 1), st));
  CK(cudaMemsetAsync(arena->queue.p, 0, sizeof(unsigned int) * (depth + 1), st));
  if (!same) CK(cudaMemsetAsync(arena->scratch.p, 0, scratch_stride * blocks, st));  // bitmaps start (and stay) clear
  k_fill_u64<<<grid_for((int64_t)(nslots * n), 256, nsm * 32), 256, 0, st>>>(arena->slots.as<unsigned long long>(),
                                                                             nslots * n, kEmpty);
  CK(cudaGetLastError());
  k_batch_init<<<grid_for(n, 8, nsm * 16), 256, 0, st>>>(arena->sys.as<BatchSys>(), arena->c0.as<int32_t>(),
                                                          arena->c0_off.as<int64_t>(), n);
  CK(cudaGetLastError());

  BatchArgs a;
  std::memset(&a, 0, sizeof a);
  a.sys = arena->sys.as<BatchSys>();
  a.n = n;
  a.qc = plan.qc;
  a.B = B;
  a.ts = ts;
  a.run = 4 * B;
  a.warp_smem = warp_smem;
  a.queue = arena->queue.as<unsigned int>();
  a.scratch = arena->scratch.as<unsigned char>();
  a.scratch_stride = scratch_stride;
  a.pmax = cap;
  a.m_max = m_max;
  a.tc = tc ? 1 : 0;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
  }
  // depth launches, captured once per arena and replayed as one graph
  if (!arena->exec) {
    cudaStream_t cap_st = nullptr;
    CK(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
    for (int d = 1; d <= depth; ++d) {
      a.launch = d;
      launch_batch_depth(a, blocks, warps, cap_st);
    }
    cudaError_t ce = cudaStreamEndCapture(cap_st, &graph);
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&arena->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap_st);
    if (ce != cudaSuccess) {
      arena->exec = nullptr;
      return fail(SNP_E_CUDA, "batch graph: %s", cudaGetErrorString(ce));
    }
  }
  if (ms) CK(cudaEventRecord(e0, st));
  cudaError_t ce = cudaGraphLaunch(arena->exec, st);
  if (ms && ce == cudaSuccess) ce = cudaEventRecord(e1, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(SNP_E_CUDA, "batch run: %s", cudaGetErrorString(ce));
  if (ms) {
    CK(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  // results
  std::vector<BatchDepthStat> stats((size_t)n * (depth + 1));
  CK(cudaMemcpy(sys.data(), arena->sys.p, sizeof(BatchSys) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(stats.data(), arena->stats.p, sizeof(BatchDepthStat) * stats.size(), cudaMemcpyDeviceToHost));
  for (int32_t i = 0; i < n; ++i) {
    snp_system* h = hs[i];
    const BatchSys& b = sys[i];
    h->stats.clear();
    snp_depth_info s0;
    std::memset(&s0, 0, sizeof s0);
    s0.new_configs = 1;
    h->stats.push_back(s0);
    int64_t lo = 0, hi = 1;
    for (int d = 1; d <= depth; ++d) {
      const BatchDepthStat& x = stats[(size_t)i * (depth + 1) + d];
      if (d > 1 && h->stats.back().new_configs == 0) break;
      snp_depth_info sd;
      std::memset(&sd, 0, sizeof sd);
      sd.new_configs = x.new_configs;
      sd.parents = hi - lo;
      sd.candidates = x.candidates;
      sd.examined = x.examined;
      sd.truncated = x.truncated;
      sd.chunks = x.chunks;
      h->stats.push_back(sd);
      lo = hi;
      hi += x.new_configs;
    }
    h->n_rows = b.n_rows;
    h->depth_reached = b.depth_reached;
    h->explored = true;
    h->have_parents = false;
    h->batch = arena;
    h->result_pool = b.pool;
    h->result_perm = nullptr;
    h->result_w = 4;
    int code = SNP_OK;
    if (b.error & kErrOverflow) code = SNP_E_OVERFLOW;
    else if (b.error & kErrTimeout) code = SNP_E_TIMEOUT;
    else if (b.error) code = SNP_E_INTERNAL;
    if (statuses) statuses[i] = code;
  }
  return SNP_OK;
}

}  // namespace

extern "C" int snp_explore_batch(snp_handle* hs, int32_t n, const snp_explore_opts* o, int32_t* statuses) {
  g_err.clear();
  TRY(batch_setup(hs, n, o));
  BatchPlan plan;
  if (o->chunk > 0) plan.qc = (uint32_t)std::min<int64_t>(o->chunk, 1 << 16);
  if (o->tile > 0) plan.tile = std::min(o->tile, 32);
  if (o->warps > 0) plan.warps = o->warps;
  return batch_run(hs, n, o, plan, statuses, nullptr);
}

extern "C" int snp_batch_autotune(snp_handle* hs, int32_t n, const snp_explore_opts* o, int32_t* chunk, int32_t* tile,
                                  int32_t* warps) {
  g_err.clear();
  TRY(batch_setup(hs, n, o));
  if (!chunk || !tile || !warps) return fail(SNP_E_INVALID, "bad arguments");
  snp_explore_opts t = *o;
  t.depth = std::min(o->depth, 2);
  const uint32_t qcs[] = {1024, 2048, 4096};
  const int tiles[] = {8, 16, 32};
  const int ws[] = {4, 8};
  const bool tc = o->transition == SNP_T_TC_F8;  // the tensor-core form: tile and warps are fixed
  float best = 1e30f;
  BatchPlan bestp;
  for (uint32_t qc : qcs)
    for (int tl : tiles)
      for (int w : ws) {
        if (tc && (tl != tiles[0] || w != ws[0])) continue;
        BatchPlan p;
        p.qc = qc;
        p.tile = tl;
        p.warps = w;
        float ms = 0.f;
        TRY(batch_run(hs, n, &t, p, nullptr, &ms));
        if (ms < best) {
          best = ms;
          bestp = p;
        }
      }
  *chunk = (int32_t)bestp.qc;
  *tile = bestp.tile;
  *warps = bestp.warps;
  for (int32_t i = 0; i < n; ++i) {
    hs[i]->batch.reset();
    hs[i]->result_pool = nullptr;
    hs[i]->result_perm = nullptr;
    hs[i]->explored = false;
  }
  return SNP_OK;
}
