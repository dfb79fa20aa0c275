/* snp.h — C ABI of the GB300 simulator for spiking neural P systems without
 * delays (Cabarle, Adorna, Martinez-del-Amor, "Simulating Spiking Neural P
 * systems without delays using GPUs").
 *
 * The library explores, breadth first, every configuration reachable from the
 * initial configuration C0 (Algorithm 1).  Each depth runs four steps on one
 * GPU: (a) the rule-applicability scan of every frontier configuration
 * (Algorithm 2, II-1), (b) the enumeration of every valid spiking vector as a
 * mixed-radix index over the per-neuron choice counts (Eq. psi; Algorithm 2,
 * II-2/II-3), (c) the transition C' = C + S . M_Pi (Eq. next-config), and (d)
 * deduplication through a device hash table into the next frontier
 * (Algorithm 1, step IV).
 *
 * Conventions
 *  - Every function returns an int status (SNP_OK = 0 or an SNP_E_* code) and
 *    never throws.  snp_last_error() gives a message for the calling thread.
 *  - Arrays described as "host or device" may be either; the library infers
 *    the direction of each copy from the pointer.  Arrays described as
 *    "host" must be host memory.  The caller keeps ownership of every array
 *    it passes; the library copies what it needs before returning.
 *  - A handle owns all device memory it allocates and is bound to the CUDA
 *    device that was current when it was created.  Handles are not
 *    thread-safe: one thread at a time per handle.
 *  - Configurations are int32 rows of length m (spikes per neuron, neuron 0
 *    first); lists of configurations are row-major [n x m].
 */
#ifndef SNP_H_
#define SNP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNP_ABI_VERSION 1

/* Status codes. */
#define SNP_OK 0
#define SNP_E_INVALID 1  /* malformed system or options (shapes, signs, order, limits) */
#define SNP_E_RANGE 2    /* an entry of M_Pi is out of range for the requested transition */
#define SNP_E_NOMEM 3    /* a device or host allocation failed */
#define SNP_E_CUDA 4     /* a CUDA call or kernel failed */
#define SNP_E_TIMEOUT 5  /* a bounded device-side wait ran out */
#define SNP_E_BUFFER 6   /* caller's buffer too small: the count is set, nothing is written */
#define SNP_E_OVERFLOW 7 /* a spike count could leave the int32 range */
#define SNP_E_STATE 8    /* call out of order (e.g. results before an exploration) */
#define SNP_E_INTERNAL 9 /* a device-side consistency check failed */
#define SNP_E_CANCELLED 10 /* the caller's cancel flag was set (snp_explore_opts.cancel) */

/* Transition forms for step (c). */
#define SNP_T_SPARSE_I32 0 /* gather over M_Pi's nonzeros, int32 on the CUDA cores */
#define SNP_T_TC_I8 1      /* dense 0/1 x int8 tensor-core product (mma.sync s8), int32 accumulation */
#define SNP_T_TC_F8 2      /* e4m3 tensor-core product on tcgen05 (TMEM, fp32 accumulation, exact for |M| <= 16) */

/* Saturation value of Psi and of sums of Psi: "at least 2^64 - 1". */
#define SNP_PSI_SAT UINT64_MAX

typedef struct snp_system* snp_handle;

/* An SNP system without delays in matrix form (Definition 1, Definition 2).
 * All arrays are host memory and are copied by snp_load_system.
 *  m            neurons, 1 <= m <= 1024.
 *  R            rules, 1 <= R; the rules of one neuron are consecutive and in
 *               the system's total rule order (rule_neuron non-decreasing), at
 *               most 32 rules per neuron.
 *  rule_neuron  [R] owning neuron of each rule, in [0, m).
 *  rule_i,      [R] the rule's regular expression E = a^i (a^j)*; j = 0 means
 *  rule_j           E = a^i exactly.  i >= 0, j >= 0.  The paper's rules
 *                   a^k -> a (form (b-3)) are i = k, j = 1.
 *  M            [R * m] spiking transition matrix M_Pi, row-major, rows =
 *               rules, columns = neurons (Definition 2, Eq. snp_mat).  The
 *               entry on a rule's own neuron is -c (c >= 1 spikes consumed);
 *               every other entry is >= 0 (spikes received).
 *  c0           [m] initial configuration C0, entries >= 0.
 *  rule_terms,  optional (NULL: every rule is the single term rule_i, rule_j):
 *  term_i,      general regular expressions, the paper's future work (Section
 *  term_j       6), read as finite unions of terms a^i (a^j)*.  Rule r's
 *               expression is the union of a^term_i[t] (a^term_j[t])* over
 *               t in [rule_terms[r], rule_terms[r + 1]); rule_terms is [R + 1]
 *               with rule_terms[0] = 0, every rule has 1 to 64 terms, and
 *               term_i, term_j >= 0.  rule_i and rule_j are then ignored (may
 *               be NULL).
 * A rule is applicable to a neuron holding x spikes iff a^x is in L(E) and
 * x >= c (Section 2.1, rule (b-1)). */
typedef struct {
  int32_t m;
  int32_t R;
  const int32_t* rule_neuron;
  const int32_t* rule_i;
  const int32_t* rule_j;
  const int32_t* M;
  const int32_t* c0;
  const int32_t* rule_terms;
  const int32_t* term_i;
  const int32_t* term_j;
} snp_system_desc;

/* Options of snp_explore.  Fill with snp_explore_opts_init first.
 *  depth             number of BFS expansions (depth >= 0).  Exploration ends
 *                    earlier when a depth finds no new configuration
 *                    (Algorithm 1, stopping criteria).
 *  transition        SNP_T_SPARSE_I32, SNP_T_TC_I8 or SNP_T_TC_F8.  The
 *                    tensor-core forms compute Eq. next-config as a matrix
 *                    product: SNP_T_TC_I8 the whole product S . M_Pi with
 *                    int8 operands; SNP_T_TC_F8 tiles of 128 candidates of
 *                    one parent as C_ref + (S - S_ref) . M_Pi over the 32-rule
 *                    blocks in which S differs from a reference spiking
 *                    vector S_ref (the full S . M_Pi for tiles crossing
 *                    parents and rows of at most 128 neurons), e4m3 operands
 *                    and fp32 accumulation, exact because every partial sum
 *                    is an integer below 2^24.
 *  frontier_cap      most new configurations accepted per depth; <= 0: no cap.
 *                    The accepted ones are the first ones in candidate order.
 *  candidate_budget  most candidates (parent, spiking vector) examined per
 *                    depth; <= 0: no budget.
 *  max_expand_value  >= 0: a configuration holding more than this many spikes
 *                    in some neuron is recorded but not expanded; < 0: off.
 *  record_parents    1: remember, per configuration, its parent's discovery
 *                    index and the spiking vector's index (snp_parents).
 *  chunk             candidates per device pass; <= 0 chooses automatically:
 *                    up to 2^22 while the rows a pass may claim stay within
 *                    512 MiB, at least 2^20; 2^22 or else 2^21 for systems
 *                    of more than 128 neurons while the store's reserve for
 *                    claims past the cap (one pass per depth) stays within
 *                    64 GiB; the
 *                    last passes of a capped depth are shortened to what the
 *                    cap is expected to take; 65536 at most in the
 *                    int8 tensor-core form, 2^21 at most in the fp8 form
 *                    (2^20 when its store's reserve, two passes per depth,
 *                    would exceed 64 GiB).
 *  stream            cudaStream_t to run on, or NULL for the default stream.
 *  kernel_timing     1: time the expand kernel of every pass with CUDA events
 *                    on `stream` (snp_depth_info.expand_ms).
 *  tile              rows of a warp's candidate tile (batch engine): the most
 *                    candidates a warp builds together; <= 0: the largest
 *                    that shared memory holds.
 *  warps             warps per CTA of the batch engine (4 or 8); <= 0: automatic.
 *  timeout_ms        > 0: bound, in milliseconds, on a lane's wait for a hash
 *                    slot that another lane is claiming; past it the pass
 *                    records SNP_E_TIMEOUT (the call returns it, the handle
 *                    stays usable).  <= 0: the default bound of 2^22 polls.
 *  cancel            host int32 polled before every depth and pass (NULL:
 *                    none); once it is nonzero the passes in flight finish,
 *                    the exploration is discarded and the call returns
 *                    SNP_E_CANCELLED.
 *  packed            1: keep the configurations in the store with the
 *                    narrowest of 1, 2 or 4 bytes per spike count that holds
 *                    every count the exploration can reach (packed
 *                    configurations; exactness unchanged).  The bound: counts
 *                    never go below 0 and one step adds at most gain[j] =
 *                    sum over neurons of their largest entry in column j of
 *                    M_Pi, so no count of column j exceeds C0[j] + depth * gain[j]
 *                    (for a resumed exploration: the checkpoint's largest
 *                    count + the depths still to run times the largest
 *                    gain).  uint8 needs m % 16 == 0 and uint16 m % 8 == 0
 *                    (rows of whole 16-byte pieces); the tensor-core forms
 *                    keep int32, and so do snp_explore_batch, the server and
 *                    snp_explore_static, which ignore this field.
 *                    snp_row_width reports the width used;
 *                    snp_reachable returns int32 rows whatever it is.
 *                    0: int32 (the default).
 *  reserved          must be 0.
 * Candidate order ("canonical order"): parents in discovery order; for each,
 * its valid spiking vectors in mixed-radix order with neuron 0's choice most
 * significant and the last neuron's least; a neuron's choices are its
 * applicable rules in rule order, or "no rule" if none applies. */
typedef struct {
  int32_t depth;
  int32_t transition;
  int64_t frontier_cap;
  int64_t candidate_budget;
  int32_t max_expand_value;
  int32_t record_parents;
  int64_t chunk;
  void* stream;
  int32_t kernel_timing;
  int32_t tile;
  int32_t warps;
  int32_t timeout_ms;
  const volatile int32_t* cancel;
  int32_t packed;
  int32_t reserved;
} snp_explore_opts;

/* Statistics of one BFS depth (index 0 is the root level). */
typedef struct {
  int64_t new_configs;   /* configurations first found at this depth */
  int64_t parents;       /* frontier size expanded at this depth */
  uint64_t candidates;   /* sum of Psi over the frontier (saturating) */
  int64_t examined;      /* candidates examined before the depth stopped */
  int32_t truncated;     /* 1 iff examined < candidates */
  int32_t chunks;        /* device passes used */
  float ms;              /* device time of the depth (CUDA events) */
  float expand_ms;       /* device time of the expand kernel (kernel_timing) */
  int64_t expand_bytes;  /* algorithmic DRAM bytes of the expand kernel, over
                            the candidates examined: per candidate an 8-byte
                            slot probe, per candidate not accepted a 4m-byte
                            key compare, per accepted configuration a 4m-byte
                            row write and an 8-byte slot write, per parent a
                            4m-byte row read */
  int64_t launches;      /* kernels launched for this depth */
} snp_depth_info;

/* Fills *opts with defaults: depth 1, sparse int32, no cap, no budget,
 * max_expand_value -1, no parent records, automatic chunk, default stream,
 * no kernel timing, the default wait bound, no cancel flag. */
void snp_explore_opts_init(snp_explore_opts* opts);

/* Validates and copies a system (Definition 1, Definition 2) and uploads its
 * rule table and M_Pi to the current device.  On success *out is a new handle.
 * Errors: SNP_E_INVALID (see snp_system_desc), SNP_E_NOMEM, SNP_E_CUDA. */
int snp_load_system(const snp_system_desc* desc, snp_handle* out);

/* Shape of a loaded system (Definition 1: m neurons, R rules) and the CUDA
 * device it lives on; any pointer may be NULL.  Errors: SNP_E_INVALID. */
int snp_system_info(snp_handle h, int32_t* m, int32_t* R, int32_t* device);

/* Releases a handle and all its device memory.  NULL is accepted. */
int snp_free(snp_handle h);

/* One transition step from configuration C (Eq. next-config for every valid
 * spiking vector, Algorithm 2): writes the children C + S . M_Pi of C, in
 * canonical order and without deduplication, to out[k * m + j] for
 * k < min(Psi(C), capacity).  *psi receives Psi(C) (Eq. psi with neurons that
 * cannot fire counted once; saturating).
 *  C    [m] host or device.   out  [capacity * m] host or device.
 * Errors: SNP_E_INVALID (negative entries in C, capacity < 0),
 * SNP_E_OVERFLOW (a child would leave int32), SNP_E_CUDA. */
int snp_step(snp_handle h, const int32_t* C, int64_t capacity, int32_t* out, uint64_t* psi);

/* Breadth-first exploration from C0 (Algorithm 1): runs steps (a)-(d) for
 * depths 1..opts->depth on the device and keeps every configuration found.
 * *depth_reached = the last depth that found a new configuration.
 * truncated_flags (host, [opts->depth + 1], may be NULL) receives 1 for each
 * depth stopped by the cap or the budget.  A new call discards the previous
 * exploration.  Errors: SNP_E_INVALID, SNP_E_RANGE (SNP_T_TC_I8 with an entry
 * of M_Pi outside [-127, 127], SNP_T_TC_F8 with one outside [-16, 16]),
 * SNP_E_NOMEM, SNP_E_OVERFLOW, SNP_E_TIMEOUT,
 * SNP_E_INTERNAL, SNP_E_CUDA. */
int snp_explore(snp_handle h, const snp_explore_opts* opts, int32_t* depth_reached, int32_t* truncated_flags);

/* Resumes an exploration from a checkpoint taken at a depth boundary: the
 * configurations found so far in discovery order (snp_reachable) and the
 * per-depth records (snp_depth_stats, depth 0 first).  The paper has no
 * counterpart (it keeps no state between runs); because the exploration order
 * is canonical and the hash table holds exactly the configurations found,
 * rebuilding the table from the rows and continuing the breadth-first search
 * from depth nstats to opts->depth gives the same result as one exploration
 * to opts->depth with the same options.
 *  rows   [n * m] host or device, n = the sum of stats[d].new_configs.
 *  stats  [nstats] host, nstats >= 1 (stats[0] is C0's record).
 * The previous exploration of h, if any, is discarded; opts as for
 * snp_explore (record_parents must be 0), opts->depth >= nstats - 1.
 * Errors: as snp_explore; SNP_E_INVALID also for an inconsistent checkpoint. */
int snp_explore_resume(snp_handle h, const int32_t* rows, int64_t n, const snp_depth_info* stats, int32_t nstats,
                       const snp_explore_opts* opts, int32_t* depth_reached, int32_t* truncated_flags);

/* Every configuration found by the last snp_explore, C0 first, in discovery
 * order (depth by depth, each depth in canonical candidate order), into
 * out[capacity * m] (host or device): the set the paper's simulator collects
 * as allGenCk (Section 5; Algorithm 2 adds every new C_k to it), here as
 * int32 rows whatever the store's width.  *n receives the count.  With
 * capacity < *n nothing is written and SNP_E_BUFFER is returned (out may then
 * be NULL).  per_depth_new (host, may be NULL) receives depth_reached + 1
 * counts, index 0 being C0's level.  Errors: SNP_E_STATE, SNP_E_BUFFER, SNP_E_CUDA. */
int snp_reachable(snp_handle h, int32_t* out, int64_t capacity, int64_t* n, int64_t* per_depth_new);

/* With record_parents set in the last snp_explore: for each configuration k in
 * discovery order, parent[k] = discovery index of the parent it was first
 * produced from and index[k] = that spiking vector's position among the
 * parent's valid vectors (C0: -1 and 0).  Host or device arrays of capacity
 * entries.  Errors: SNP_E_STATE, SNP_E_BUFFER, SNP_E_CUDA. */
int snp_parents(snp_handle h, int64_t* parent, uint64_t* index, int64_t capacity, int64_t* n);

/* Statistics of depth d (0 <= d <= depth_reached + 1) of the last
 * exploration: the frontier expanded at that depth of the computation tree
 * (Section 4.1: each level's configurations are the parents of the next), the
 * sum of Psi over it (Eq. psi), the candidates examined and the new
 * configurations kept; a depth with none new is where the search stopped by
 * the second stopping criterion (Section 4.1).  Errors: SNP_E_STATE,
 * SNP_E_INVALID. */
int snp_depth_stats(snp_handle h, int32_t d, snp_depth_info* out);

/* Bytes per spike count of the store of the last exploration: 1 (uint8),
 * 2 (uint16) or 4 (int32) -- see snp_explore_opts.packed.  Errors:
 * SNP_E_STATE (no exploration), SNP_E_INVALID. */
int snp_row_width(snp_handle h, int32_t* bytes_per_count);

/* Breadth-first exploration of n independent systems at once (the batch
 * engine): every system runs exactly what snp_explore would run on it with
 * the same options, and afterwards each handle answers snp_reachable,
 * snp_depth_stats and friends for its own exploration.  All systems advance
 * together, one device launch per depth (captured in a CUDA graph); a CTA
 * takes one system at a time and runs its whole depth.
 *  hs        [n] host array of handles, all on the current device, distinct.
 *  opts      depth, frontier_cap (required: 1 <= cap <= 2^20), candidate_budget,
 *            max_expand_value, chunk (candidates per pass, <= 0: 2048),
 *            tile, warps, stream; transition must be SNP_T_SPARSE_I32 and
 *            record_parents 0.
 *  statuses  (host, [n], may be NULL) per system: SNP_OK, SNP_E_OVERFLOW,
 *            SNP_E_TIMEOUT or SNP_E_INTERNAL.
 * The systems' configurations live in one device arena shared by the handles
 * until each is freed or explored again.  Returns SNP_OK when the batch ran
 * (check statuses), else SNP_E_INVALID, SNP_E_NOMEM, SNP_E_CUDA. */
int snp_explore_batch(snp_handle* hs, int32_t n, const snp_explore_opts* opts, int32_t* statuses);

/* Chooses the batch engine's pass size, tile and warps per CTA for this batch
 * by timing the first two depths of each candidate setting (on the real
 * systems; their previous results are discarded).  *chunk, *tile and *warps
 * receive the fastest setting, for snp_explore_batch's options.  Errors as
 * snp_explore_batch. */
int snp_batch_autotune(snp_handle* hs, int32_t n, const snp_explore_opts* opts, int32_t* chunk, int32_t* tile,
                       int32_t* warps);

/* Serving: explorations submitted at any time run together on the device.
 * The paper's simulator runs one system at a time; this loop serves many.  A
 * server thread admits pending requests while its device memory allows (each
 * request needs its pool, 4m (1 + depth * cap) bytes, and its hash table),
 * then advances every admitted request by one depth per launch of the batch
 * engine, so requests that arrive while others run join at the next launch
 * (continuous batching).  A finished request's configurations are copied
 * into its handle, which then answers snp_reachable and snp_depth_stats
 * exactly as after snp_explore; its memory goes back to the server. */
typedef struct {
  int64_t submitted, completed, active, pending;
  int64_t new_configs;  /* new configurations of the completed requests */
  int64_t ticks;        /* batch launches */
  double busy_ms;       /* host time spent running launches */
  double span_ms;       /* first submit to last completion */
  double p50_ms, p99_ms, max_ms;  /* latency: submit to result ready */
} snp_server_info;

/* Creates a server on the current device with hbm_budget bytes of device
 * memory for requests and at most max_active requests on the device at once.
 * Errors: SNP_E_INVALID, SNP_E_NOMEM, SNP_E_CUDA. */
int snp_server_create(size_t hbm_budget, int32_t max_active, void** srv);

/* Queues an exploration of h with opts (depth >= 1, 1 <= frontier_cap <= 2^20,
 * SNP_T_SPARSE_I32, no parent records).  The caller must not use h until the
 * request is reported finished.  *req_id identifies it in snp_server_poll.
 * Errors: SNP_E_INVALID, SNP_E_NOMEM (larger than the server's memory). */
int snp_server_submit(void* srv, snp_handle h, const snp_explore_opts* opts, uint64_t* req_id);

/* Takes up to max finished requests: ids, latencies (ms, submit to result
 * ready) and statuses (SNP_OK or the request's error), any of them NULL. */
int snp_server_poll(void* srv, uint64_t* ids, double* latency_ms, int32_t* statuses, int32_t max, int32_t* n);

/* Blocks until no request is pending or active.  Returns SNP_OK, or the error
 * that stopped the server. */
int snp_server_wait(void* srv);

/* Counters and latency percentiles of the completed requests. */
int snp_server_stats(void* srv, snp_server_info* out);

/* Stops the server after its pending and active requests finish, and frees it. */
int snp_server_destroy(void* srv);

/* snp_explore without allocating memory: the paper has no counterpart; this
 * is for callers that may not allocate device memory at the moment they need
 * an exploration (a framework's caching allocator holds the free memory, or a
 * loop must not block on the allocator).  It runs the same search as
 * snp_explore and writes the same configurations in the same order, but
 * allocates neither device nor host memory: the configurations go straight
 * into the caller's device buffer out[capacity * m], which also serves as the
 * working pool, and every other buffer comes from one fixed 64 MiB device
 * array inside the library, held by every GPU that loads the library until
 * the process exits.  All calls share that array and each leaves its contents
 * behind; a call clears what must start empty, and calls whose work overlaps
 * on the GPU (other streams or threads) race on it.  The first call on a
 * device (and the first after its context was recreated) looks up the
 * array's address.  The call launches kernels on opts->stream and waits for
 * that stream once per pass, so it may not be made from a stream callback or
 * on a stream that is being captured.  The caller's current device is the
 * same on return.
 *  opts           as for snp_explore; transition must be SNP_T_SPARSE_I32
 *                 and record_parents 0.  Uses opts->stream.
 *  out            device memory on the handle's device, capacity rows of m
 *                 int32.
 *  capacity       1 <= capacity <= 2^20 configurations (the array's limit);
 *                 larger values are refused with SNP_E_INVALID.
 *  *n             configurations written (C0 first, discovery order).
 *  depth_reached  (host, may be NULL) as for snp_explore.
 *  per_depth_new  (host, [opts->depth + 1], may be NULL) new configurations
 *                 per depth, index 0 being C0's level.
 * The handle's exploration results are not touched (the handle's pinned
 * staging words are reused).  Errors: SNP_E_INVALID, SNP_E_BUFFER (capacity
 * reached while candidates remain), SNP_E_OVERFLOW, SNP_E_TIMEOUT,
 * SNP_E_INTERNAL, SNP_E_CUDA. */
int snp_explore_static(snp_handle h, const snp_explore_opts* opts, int32_t* out, int64_t capacity, int64_t* n,
                       int32_t* depth_reached, int64_t* per_depth_new);

/* Measures the int8 tensor-core rate of the current device (mma.sync
 * m16n8k32, s8 x s8 -> s32, the instruction SNP_T_TC_I8 uses): *tops receives
 * tera-operations per second (2 per multiply-add) over `iters` rounds of 8
 * independent products per warp on 8 blocks per SM.  A measurement utility for
 * the tensor-core roofline; the paper has no counterpart.  Allocates a small
 * device buffer.  Returns 0, or 1 (bad arguments), 3 (no memory), 4 (CUDA). */
int snp_tc_peak_tops(int32_t iters, double* tops);

/* Message for the last failed call on this thread ("" if none). */
const char* snp_last_error(void);

/* Testing hook (no counterpart in the paper): the k-th device allocation from
 * now on (k >= 1, counting every buffer the library allocates or grows) fails
 * as if the device were out of memory, so that error paths can be exercised
 * without exhausting the device; k <= 0 turns it off.  The failing call
 * returns SNP_E_NOMEM and leaves every handle usable.  Process-wide. */
int snp_debug_fail_allocation(int64_t k);

/* Testing hook (no counterpart in the paper): the next snp_explore (on any
 * handle) leaves C0's hash-table slot in the "being claimed" state instead of
 * publishing it, so a candidate equal to C0 waits until the wait bound runs
 * out and the call returns SNP_E_TIMEOUT, without any fault.  One-shot,
 * process-wide; on = 0 withdraws it. */
int snp_debug_hold_root_slot(int32_t on);

/* SNP_ABI_VERSION of the loaded library. */
int snp_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SNP_H_ */
