// Serving loop (snp_server_*): explorations submitted at any time are admitted
// while device memory allows and advanced together, one depth per tick, by
// the batch kernel.  A request that arrives while others run joins at the
// next tick (continuous batching); a finished request is copied into its
// handle, its memory is returned, and its latency (submit to result ready) is
// recorded.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "snp_host.h"

using namespace snp;

namespace {

using Clock = std::chrono::steady_clock;

__global__ void k_fill_ranges(unsigned long long* const* ptr, const uint64_t* count, int32_t n, unsigned long long v) {
  for (int32_t r = blockIdx.y; r < n; r += gridDim.y) {
    unsigned long long* p = ptr[r];
    const uint64_t c = count[r];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c; i += (uint64_t)gridDim.x * blockDim.x)
      p[i] = v;
  }
}

// First-fit allocator over [0, size), 256-byte granules.
class RangeAlloc {
 public:
  explicit RangeAlloc(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t id = 0;
  snp_system* h = nullptr;
  snp_explore_opts o{};
  Clock::time_point arrival, done;
  size_t off = 0, bytes = 0;  // arena range: pool, table, stats
  int64_t rows = 0;
  uint64_t nslots = 0;
  BatchSys bs{};
  int status = SNP_OK;
};

}  // namespace

struct snp_server {
  int device = 0;
  size_t budget = 0;
  int32_t max_active = 0;
  DevBuf arena, sys_dev, scratch, queue, c0_dev, c0_off_dev, fill_ptr, fill_cnt;
  RangeAlloc* alloc = nullptr;
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::deque<Request*> finished;
  std::thread loop;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0;
  int64_t total_new = 0;
  int64_t ticks = 0;
  double busy_ms = 0.0;
  std::vector<double> lat_ms;
  Clock::time_point first_arrival, last_done;
  bool any = false;
  size_t scratch_stride = 0;
  int loop_error = SNP_OK;
  std::string loop_msg;
};

namespace {

constexpr uint32_t kServeQc = 2048;

size_t request_bytes(const snp_system* h, const snp_explore_opts& o, int64_t* rows, uint64_t* nslots) {
  *rows = 1 + (int64_t)o.depth * o.frontier_cap;
  const uint64_t want = (uint64_t)((long double)(*rows + (int64_t)o.depth * kServeQc) * 4.0L / 3.0L) + kBucket;
  *nslots = std::max<uint64_t>(pow2_at_least(want), kBucket);
  auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
  return r((size_t)*rows * h->m * 4) + r(*nslots * 8) + r(sizeof(BatchDepthStat) * (o.depth + 1));
}

// Device state of newly admitted requests: empty tables, C0 in row 0 and in the table.
int init_requests(snp_server* S, std::vector<Request*>& fresh) {
  if (fresh.empty()) return SNP_OK;
  const int n = (int)fresh.size();
  std::vector<unsigned long long*> ptr(n);
  std::vector<uint64_t> cnt(n);
  std::vector<int32_t> c0;
  std::vector<int64_t> c0_off(n);
  std::vector<BatchSys> sys(n);
  for (int i = 0; i < n; ++i) {
    Request* r = fresh[i];
    ptr[i] = r->bs.slots;
    cnt[i] = r->nslots;
    c0_off[i] = (int64_t)c0.size();
    c0.insert(c0.end(), r->h->c0.begin(), r->h->c0.end());
    sys[i] = r->bs;
  }
  TRY(S->fill_ptr.reserve(sizeof(void*) * n));
  TRY(S->fill_cnt.reserve(sizeof(uint64_t) * n));
  TRY(S->c0_dev.reserve(sizeof(int32_t) * c0.size()));
  TRY(S->c0_off_dev.reserve(sizeof(int64_t) * n));
  TRY(S->sys_dev.reserve(sizeof(BatchSys) * std::max<size_t>(n, S->active.size() + n)));
  CK(cudaMemcpyAsync(S->fill_ptr.p, ptr.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, S->st));
  CK(cudaMemcpyAsync(S->fill_cnt.p, cnt.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, S->st));
  CK(cudaMemcpyAsync(S->c0_dev.p, c0.data(), sizeof(int32_t) * c0.size(), cudaMemcpyHostToDevice, S->st));
  CK(cudaMemcpyAsync(S->c0_off_dev.p, c0_off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, S->st));
  CK(cudaMemcpyAsync(S->sys_dev.p, sys.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice, S->st));
  dim3 grid(64, (unsigned)std::min(n, 1024));
  k_fill_ranges<<<grid, 256, 0, S->st>>>(S->fill_ptr.as<unsigned long long*>(), S->fill_cnt.as<uint64_t>(), n, kEmpty);
  CK(cudaGetLastError());
  for (int i = 0; i < n; ++i) {
    Request* r = fresh[i];
    CK(cudaMemsetAsync(r->bs.stats, 0, sizeof(BatchDepthStat) * (r->o.depth + 1), S->st));
  }
  k_batch_init<<<grid_for(n, 8, 152 * 16), 256, 0, S->st>>>(S->sys_dev.as<BatchSys>(), S->c0_dev.as<int32_t>(),
                                                             S->c0_off_dev.as<int64_t>(), n);
  CK(cudaGetLastError());
  return SNP_OK;
}

// Copies a finished request's configurations and statistics into its handle.
int retire(snp_server* S, Request* r) {
  snp_system* h = r->h;
  const BatchSys& b = r->bs;
  const int depth = r->o.depth;
  std::vector<BatchDepthStat> st(depth + 1);
  CK(cudaMemcpyAsync(st.data(), b.stats, sizeof(BatchDepthStat) * (depth + 1), cudaMemcpyDeviceToHost, S->st));
  const size_t bytes = sizeof(int32_t) * (size_t)b.n_rows * h->m;
  if (h->d_pool.reserve(bytes) != SNP_OK) {  // this request fails; the server goes on
    r->status = SNP_E_NOMEM;
    h->explored = false;
    return SNP_OK;
  }
  h->pool_rows = std::max<int64_t>(h->pool_rows, b.n_rows);
  CK(cudaMemcpyAsync(h->d_pool.p, b.pool, bytes, cudaMemcpyDeviceToDevice, S->st));
  CK(cudaStreamSynchronize(S->st));
  h->stats.clear();
  snp_depth_info s0;
  std::memset(&s0, 0, sizeof s0);
  s0.new_configs = 1;
  h->stats.push_back(s0);
  int64_t lo = 0, hi = 1;
  for (int d = 1; d <= std::min(depth, b.cur_depth); ++d) {
    const BatchDepthStat& x = st[d];
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
  h->batch.reset();
  h->result_pool = h->d_pool.as<int32_t>();
  h->result_perm = nullptr;
  h->result_w = 4;
  h->row_w = 4;
  r->status = (b.error & kErrOverflow) ? SNP_E_OVERFLOW
              : (b.error & kErrTimeout) ? SNP_E_TIMEOUT
              : b.error ? SNP_E_INTERNAL : SNP_OK;
  return SNP_OK;
}

int tick(snp_server* S) {
  const int n = (int)S->active.size();
  if (n == 0) return SNP_OK;
  int m_max = 1;
  int64_t pmax = 1;
  std::vector<BatchSys> sys(n);
  for (int i = 0; i < n; ++i) {
    sys[i] = S->active[i]->bs;
    m_max = std::max(m_max, sys[i].sys.m);
    pmax = std::max<int64_t>(pmax, sys[i].cap);
  }
  const int nsm = sm_count(S->device);
  const int warps = 8;
  int ts = 0;
  int B = 32;  // shrunk below to what the shared memory holds
  size_t warp_smem = expand_smem_bytes(m_max, B, &ts);
  while (B > 1 && warp_smem * warps > (200u << 10)) warp_smem = expand_smem_bytes(m_max, --B, &ts);
  const int blocks = std::max(1, std::min(nsm, n));
  const size_t stride = (batch_scratch_bytes(pmax, kServeQc, m_max) + 255) & ~size_t(255);
  void* before = S->scratch.p;
  TRY(S->scratch.reserve(stride * blocks));
  // The bitmaps in the scratch must start cleared (the kernel leaves them
  // cleared); a new buffer or a new layout (other stride) starts from zero.
  if (S->scratch.p != before || stride != S->scratch_stride) {
    CK(cudaMemsetAsync(S->scratch.p, 0, S->scratch.bytes, S->st));
    S->scratch_stride = stride;
  }
  TRY(S->sys_dev.reserve(sizeof(BatchSys) * n));
  TRY(S->queue.reserve(sizeof(unsigned int)));
  CK(cudaMemcpyAsync(S->sys_dev.p, sys.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice, S->st));
  CK(cudaMemsetAsync(S->queue.p, 0, sizeof(unsigned int), S->st));
  BatchArgs a;
  std::memset(&a, 0, sizeof a);
  a.sys = S->sys_dev.as<BatchSys>();
  a.n = n;
  a.launch = 0;
  a.qc = kServeQc;
  a.B = B;
  a.ts = ts;
  a.run = 4 * B;
  a.warp_smem = warp_smem;
  a.queue = S->queue.as<unsigned int>();
  a.scratch = S->scratch.as<unsigned char>();
  a.scratch_stride = stride;
  a.pmax = pmax;
  a.m_max = m_max;
  launch_batch_depth(a, blocks, warps, S->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(sys.data(), S->sys_dev.p, sizeof(BatchSys) * n, cudaMemcpyDeviceToHost, S->st));
  CK(cudaStreamSynchronize(S->st));
  for (int i = 0; i < n; ++i) S->active[i]->bs = sys[i];
  ++S->ticks;
  return SNP_OK;
}

void server_loop(snp_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Request*> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->pending.empty() && S->active.empty()) {
        if (S->stop) return;
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      while (!S->pending.empty() && (int32_t)S->active.size() < S->max_active) {
        Request* r = S->pending.front();
        size_t off = 0;
        if (!S->alloc->alloc(r->bytes, &off)) break;  // admitted when memory frees up
        S->pending.pop_front();
        r->off = off;
        auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
        unsigned char* base = S->arena.as<unsigned char>() + off;
        BatchSys& b = r->bs;
        std::memset(&b, 0, sizeof b);
        b.sys = r->h->dev();
        b.pool = reinterpret_cast<int32_t*>(base);
        b.slots = reinterpret_cast<unsigned long long*>(base + r256((size_t)r->rows * r->h->m * 4));
        b.bmask = r->nslots / kBucket - 1;
        b.stats = reinterpret_cast<BatchDepthStat*>(base + r256((size_t)r->rows * r->h->m * 4) + r256(r->nslots * 8));
        b.pool_rows = r->rows;
        b.level_lo = 0;
        b.level_hi = 1;
        b.n_rows = 1;
        b.target_depth = r->o.depth;
        b.max_expand = r->o.max_expand_value;
        b.cap = r->o.frontier_cap;
        b.budget = r->o.candidate_budget > 0 ? r->o.candidate_budget : 0;
        S->active.push_back(r);
        fresh.push_back(r);
      }
    }
    const auto t0 = Clock::now();
    int rc = init_requests(S, fresh);
    if (rc == SNP_OK) rc = tick(S);
    std::vector<Request*> done;
    if (rc == SNP_OK) {
      for (size_t i = 0; i < S->active.size();) {
        Request* r = S->active[i];
        if (r->bs.done || r->bs.cur_depth >= r->bs.target_depth || r->bs.error) {
          rc = retire(S, r);
          if (rc != SNP_OK) break;
          r->done = Clock::now();
          done.push_back(r);
          S->active.erase(S->active.begin() + i);
        } else {
          ++i;
        }
      }
    }
    S->busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc != SNP_OK && S->loop_error == SNP_OK) {
      S->loop_error = rc;
      S->loop_msg = g_err;
    }
    for (Request* r : done) {
      S->alloc->release(r->off, r->bytes);
      S->completed += 1;
      S->total_new += r->bs.n_rows - 1;
      S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->done - r->arrival).count());
      S->last_done = r->done;
      S->finished.push_back(r);
    }
    if (!done.empty() || rc != SNP_OK) S->cv_done.notify_all();
    if (rc != SNP_OK) {  // a device error ends the loop; waiting callers are released
      for (Request* r : S->active) {
        r->status = rc;
        S->finished.push_back(r);
      }
      S->active.clear();
      for (Request* r : S->pending) {
        r->status = rc;
        S->finished.push_back(r);
      }
      S->pending.clear();
      S->cv_done.notify_all();
      return;
    }
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int snp_server_create(size_t hbm_budget, int32_t max_active, void** out) {
  g_err.clear();
  if (!out || hbm_budget < (1u << 20) || max_active < 1) return fail(SNP_E_INVALID, "bad arguments");
  *out = nullptr;
  auto* S = new (std::nothrow) snp_server;
  if (!S) return fail(SNP_E_NOMEM, "host allocation failed");
  CK(cudaGetDevice(&S->device));
  S->budget = hbm_budget;
  S->max_active = max_active;
  int rc = S->arena.reserve(hbm_budget);
  if (rc != SNP_OK) {
    delete S;
    return rc;
  }
  S->alloc = new RangeAlloc(hbm_budget);
  CK(cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking));
  S->loop = std::thread(server_loop, S);
  *out = S;
  return SNP_OK;
}

int snp_server_submit(void* srv, snp_handle h, const snp_explore_opts* o, uint64_t* req_id) {
  g_err.clear();
  auto* S = static_cast<snp_server*>(srv);
  if (!S || !h || !o || !req_id) return fail(SNP_E_INVALID, "bad arguments");
  if (h->device != S->device) return fail(SNP_E_INVALID, "handle on device %d, server on %d", h->device, S->device);
  if (o->depth < 1) return fail(SNP_E_INVALID, "depth = %d < 1", o->depth);
  if (o->transition != SNP_T_SPARSE_I32 || o->record_parents)
    return fail(SNP_E_INVALID, "the server runs the sparse transition without parent records");
  if (o->frontier_cap < 1 || o->frontier_cap > (1 << 20))
    return fail(SNP_E_INVALID, "the server needs 1 <= frontier_cap <= 2^20");
  auto* r = new (std::nothrow) Request;
  if (!r) return fail(SNP_E_NOMEM, "host allocation failed");
  r->h = h;
  r->o = *o;
  r->bytes = request_bytes(h, *o, &r->rows, &r->nslots);
  if (r->bytes > S->budget) {
    delete r;
    return fail(SNP_E_NOMEM, "request needs %zu bytes, the server holds %zu", r->bytes, S->budget);
  }
  h->explored = false;
  h->batch.reset();
  h->result_pool = nullptr;
  h->result_perm = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->loop_error != SNP_OK) {
      delete r;
      return fail(S->loop_error, "server stopped: %s", S->loop_msg.c_str());
    }
    r->id = S->next_id++;
    r->arrival = Clock::now();
    if (!S->any) {
      S->first_arrival = r->arrival;
      S->any = true;
    }
    S->pending.push_back(r);
    S->submitted += 1;
    *req_id = r->id;
  }
  S->cv.notify_one();
  return SNP_OK;
}

int snp_server_poll(void* srv, uint64_t* ids, double* latency_ms, int32_t* statuses, int32_t max, int32_t* n) {
  g_err.clear();
  auto* S = static_cast<snp_server*>(srv);
  if (!S || !n || max < 0) return fail(SNP_E_INVALID, "bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  int32_t k = 0;
  while (k < max && !S->finished.empty()) {
    Request* r = S->finished.front();
    S->finished.pop_front();
    if (ids) ids[k] = r->id;
    if (latency_ms) latency_ms[k] = std::chrono::duration<double, std::milli>(r->done - r->arrival).count();
    if (statuses) statuses[k] = r->status;
    delete r;
    ++k;
  }
  *n = k;
  return SNP_OK;
}

int snp_server_wait(void* srv) {
  g_err.clear();
  auto* S = static_cast<snp_server*>(srv);
  if (!S) return fail(SNP_E_INVALID, "bad arguments");
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return (S->pending.empty() && S->active.empty()) || S->loop_error != SNP_OK; });
  if (S->loop_error != SNP_OK) return fail(S->loop_error, "server stopped: %s", S->loop_msg.c_str());
  return SNP_OK;
}

int snp_server_stats(void* srv, snp_server_info* out) {
  g_err.clear();
  auto* S = static_cast<snp_server*>(srv);
  if (!S || !out) return fail(SNP_E_INVALID, "bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof *out);
  out->submitted = (int64_t)S->submitted;
  out->completed = (int64_t)S->completed;
  out->active = (int64_t)S->active.size();
  out->pending = (int64_t)S->pending.size();
  out->new_configs = S->total_new;
  out->ticks = S->ticks;
  out->busy_ms = S->busy_ms;
  out->span_ms = S->any && S->completed ? std::chrono::duration<double, std::milli>(S->last_done - S->first_arrival).count()
                                        : 0.0;
  out->p50_ms = percentile(S->lat_ms, 0.50);
  out->p99_ms = percentile(S->lat_ms, 0.99);
  out->max_ms = percentile(S->lat_ms, 1.0);
  return SNP_OK;
}

int snp_server_destroy(void* srv) {
  auto* S = static_cast<snp_server*>(srv);
  if (!S) return SNP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->loop.joinable()) S->loop.join();
  for (Request* r : S->finished) delete r;
  for (Request* r : S->pending) delete r;
  for (Request* r : S->active) delete r;
  if (S->st) cudaStreamDestroy(S->st);
  delete S->alloc;
  delete S;
  return SNP_OK;
}

}  // extern "C"
