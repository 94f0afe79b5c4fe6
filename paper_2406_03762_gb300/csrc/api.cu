// api.cu -- host orchestration behind the C ABI (include/cortex.h): planning of the indegree
// sub-graph decomposition (targets per block, warps per block), device memory, the builder waves,
// the step loop (persistent cooperative launches replayed from a CUDA graph, or split update /
// delivery launches), and the data accessors.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cortex.h"
#include "cortex_internal.cuh"

using namespace cortex;

namespace {

// NVTX range around a public call (visible in a profiler's timeline; free when no tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) { return cortex::record_error(code, msg.c_str()); }

#define CUDA_TRY(expr)                                                                                         \
  do {                                                                                                         \
    cudaError_t e_ = (expr);                                                                                   \
    if (e_ != cudaSuccess) {                                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? CORTEX_ERR_OOM : CORTEX_ERR_CUDA,                          \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                                         \
    }                                                                                                          \
  } while (0)

constexpr size_t kKeyBudget = size_t(4) << 30;  // builder scratch per wave (keys)

}  // namespace

struct cortex_net {
  cudaStream_t stream = nullptr;
  int device = 0;
  int n_nets = 0;
  std::vector<cortex_params> params;
  std::vector<uint64_t> seeds;
  std::vector<NetDev> nets_h;
  std::vector<BlockWork> work_h;
  NetDev* nets_d = nullptr;
  BlockWork* work_d = nullptr;
  int wdtype = 0;
  int64_t n_total = 0, total_syn = 0, total_ring = 0, total_hdr = 0, total_raster = 0;
  // device arrays
  void* rec_w = nullptr;
  uint16_t* rec_meta = nullptr;
  uint4* hdr = nullptr;
  unsigned long long* row_base = nullptr;
  float* V = nullptr;
  float* I = nullptr;
  int32_t* R = nullptr;
  float* ring = nullptr;
  uint32_t* pub_ids = nullptr;
  uint32_t* pub_cnt = nullptr;
  unsigned long long* pub_flag = nullptr;
  unsigned long long* mbox = nullptr;
  int32_t* raster_step = nullptr;
  int32_t* raster_id = nullptr;
  unsigned long long* raster_count = nullptr;
  unsigned long long* events = nullptr;
  int32_t* err = nullptr;
  long long* step_counter = nullptr;
  uint32_t* max_seg = nullptr;
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  // plan
  int n_warps = 14, threads = 448, n_blocks = 0, n_sm = 0;
  int w_max = 1, w_split = 1;
  bool ring_smem = false;
  bool ring_red = false;  // global ring adds by the L2 reduction unit (exact for the weights)
  bool exact = false;     // every partial sum of a ring cell is exact: order-free adds
  bool helper_warp = false;  // ring kernel: one more warp per block builds the piece descriptors
  bool no_auto_helper = false;  // the automatic helper warp was dropped (blocks not co-resident)
  cortex_options build_opts = {};  // the build's options (a later switch to the ordered fold redoes the layout)
  int e_min = 0;          // exact: every weight is an integer multiple of 2^e_min
  double exact_bound = 0; // exact: largest |partial sum| of a cell, in units of 2^e_min
  cudaAccessPolicyWindow apw = {};  // the global ring, persisting in L2 (num_bytes 0: none)
  // delay-ordered delivery
  int delivery = CORTEX_DELIVERY_RING;
  int d_threads = 1024;   // threads per block of the delay-ordered kernel
  size_t d_smem = 0;      // its dynamic shared memory
  uint16_t* dtgt = nullptr;
  void* dw = nullptr;
  uint16_t* dtbl = nullptr;
  uint32_t* hist_ids = nullptr;
  uint32_t* hist_cnt = nullptr;
  unsigned long long* bar_count = nullptr;
  int hist_max = 0;
  int64_t total_tbl = 0;
  int64_t h2d_bytes = 0;  // host -> device bytes the build copied (network and block tables)
  uint32_t* stamps = nullptr;            // ownership check: writer warp per ring cell
  unsigned long long* viol = nullptr;    // ownership check: violations, first bad cell + 1
  bool l2_user = false;   // this handle raised the process's persisting-L2 limit
  int mode = CORTEX_MODE_PERSISTENT;
  int stage_bytes = 0, batch = 32;  // largest staging area, fewest spikes per round (stats)
  size_t smem = 0;
  int steps_per_launch = 1000;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  long long timeout_ns = 2000000000ll;
  int32_t withhold_block = -1;
  bool timed_out = false;  // a device wait gave up: the barrier epochs are inconsistent
  bool no_layout = false;  // the switch to the ordered fold found no shared-memory layout: no launches
  std::vector<uint32_t> max_seg_len;  // longest (source, block) piece of each network
  size_t smem_cap = 0;                 // dynamic shared memory a block may use
  // bookkeeping
  int64_t step = 0;
  int64_t spikes_cleared = 0;
  double build_ms = 0, sim_ms = 0;
  int64_t sim_steps = 0, sim_events = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  template <class T>
  cudaError_t alloc(T** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    device_bytes += bytes;
    *p = reinterpret_cast<T*>(q);
    return cudaSuccess;
  }

  ~cortex_net();
  void destroy() {
    if (graph) cudaGraphExecDestroy(graph);
    for (void* p : allocs) cudaFree(p);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

namespace {

// The persisting-L2 limit is a property of the process's CUDA context: handles that keep a global
// ring resident raise it, and the last of them to be freed puts back the value found before.
std::mutex g_l2_mu;
int g_l2_users = 0;
size_t g_l2_saved = 0;

void l2_persist_acquire(cortex_net* h, int64_t ring_bytes) {
  int maxp = 0, maxw = 0;
  if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, h->device) != cudaSuccess || maxp <= 0 ||
      maxw <= 0 || ring_bytes <= 0) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_l2_mu);
  size_t cur = 0;
  if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (g_l2_users == 0) g_l2_saved = cur;
  const size_t want = std::min<size_t>((size_t)ring_bytes, (size_t)maxp);
  if (cur < want) {
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess ||
        cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  }
  ++g_l2_users;
  h->l2_user = true;
  const size_t win = std::min<size_t>((size_t)ring_bytes, (size_t)maxw);
  h->apw.base_ptr = h->ring;
  h->apw.num_bytes = win;
  h->apw.hitRatio = (float)std::min(1.0, (double)cur / (double)win);
  h->apw.hitProp = cudaAccessPropertyPersisting;
  h->apw.missProp = cudaAccessPropertyStreaming;
}

void l2_persist_release(cortex_net* h) {
  if (!h->l2_user) return;
  std::lock_guard<std::mutex> lk(g_l2_mu);
  h->l2_user = false;
  if (--g_l2_users == 0) {
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_saved);
    cudaGetLastError();
  }
}

// w = m * 2^e with m an odd integer (w finite and nonzero); false otherwise
bool weight_grid(float w, int& e) {
  if (w == 0.0f || !std::isfinite(w)) return false;
  int x = 0;
  const double f = std::frexp((double)w, &x);  // |f| in [0.5, 1)
  long long m = std::llround(std::ldexp(f, 24));  // exact: a float has 24 significant bits
  e = x - 24;
  while ((m & 1) == 0) {
    m /= 2;
    ++e;
  }
  return true;
}

// Whether every partial sum of every ring cell is exactly representable in FP32.  A cell receives
// at most one add per incoming synapse of its target (a synapse's successive arrivals land at
// different steps, and the cell is cleared when its step consumes it): at most k_exc adds of w_exc
// and k_inh of w_inh.  With every weight an integer multiple of 2^e_min, every partial sum is an
// integer multiple of 2^e_min of magnitude at most k_exc |w_exc| + k_inh |w_inh|; when that is at
// most 2^24 * 2^e_min (and 2^e_min is a normal number) every partial sum is a float, no add rounds,
// and the order of the adds does not change the result.
bool prove_exact(const std::vector<NetDev>& nets, int& e_min, double& bound) {
  e_min = INT_MAX;
  for (const NetDev& d : nets)
    for (int q = 0; q < 2; ++q) {
      const float w = q ? d.w_inh : d.w_exc;
      const int k = q ? d.k_inh : d.k_exc;
      int e = 0;
      if (k == 0 || w == 0.0f) continue;
      if (!weight_grid(w, e)) return false;
      e_min = std::min(e_min, e);
    }
  if (e_min == INT_MAX) {  // no nonzero weight: every sum is zero
    e_min = 0;
    bound = 0;
    return true;
  }
  if (e_min < -126 || e_min + 24 > 127) return false;
  bound = 0;
  for (const NetDev& d : nets) {
    const double b = (double)d.k_exc * std::fabs((double)d.w_exc) + (double)d.k_inh * std::fabs((double)d.w_inh);
    bound = std::max(bound, std::ldexp(b, -e_min));
  }
  return bound <= 16777216.0;
}

int validate_params(const cortex_params& p, std::string& why) {
  if (p.n_exc < 0 || p.n_inh < 0 || (int64_t)p.n_exc + p.n_inh <= 0) return why = "neuron counts", CORTEX_ERR_ARG;
  if ((int64_t)p.n_exc + p.n_inh > (1ll << 31) - 1) return why = "too many neurons", CORTEX_ERR_UNSUPPORTED;
  if (p.k_exc < 0 || p.k_inh < 0) return why = "in-degree", CORTEX_ERR_ARG;
  if ((p.k_exc > 0 && p.n_exc == 0) || (p.k_inh > 0 && p.n_inh == 0)) return why = "in-degree from an empty population", CORTEX_ERR_ARG;
  if ((int64_t)p.k_exc + p.k_inh > 65535) return why = "in-degree above 65535", CORTEX_ERR_UNSUPPORTED;
  if (p.d_min < 1 || p.d_max < p.d_min) return why = "delays must satisfy 1 <= d_min <= d_max", CORTEX_ERR_ARG;
  if (p.d_max > 255) return why = "d_max above 255", CORTEX_ERR_UNSUPPORTED;
  if (!(p.tau_m > 0) || !(p.tau_syn > 0) || !(p.c_m > 0) || !(p.dt > 0) || !(p.t_ref >= 0))
    return why = "time constants, capacitance, dt and t_ref must be positive", CORTEX_ERR_ARG;
  if (p.tau_m == p.tau_syn) return why = "tau_m == tau_syn (singular propagator)", CORTEX_ERR_UNSUPPORTED;
  if (std::llround((double)p.t_ref / (double)p.dt) > 32767)
    return why = "t_ref / dt above 32767 steps (16-bit refractory counter)", CORTEX_ERR_UNSUPPORTED;
  if (!(p.nu_ext_hz >= 0)) return why = "nu_ext_hz", CORTEX_ERR_ARG;
  if (p.weight_dtype != CORTEX_F32 && p.weight_dtype != CORTEX_BF16) return why = "weight_dtype", CORTEX_ERR_ARG;
  if (p.e_l != 0.0f) return why = "only E_L = 0 is supported (potentials relative to rest)", CORTEX_ERR_UNSUPPORTED;
  return CORTEX_OK;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// The most targets one block of network p may own: its shared-memory layout (ring in global
// memory) must leave staging for two spikes per round, with the expected piece of a source
// (t K / N records for uniformly drawn sources) plus six standard deviations.
int64_t max_block_targets(const cortex_params& p, int wsz, int n_warps, size_t smem_cap) {
  const int64_t n = (int64_t)p.n_exc + p.n_inh, k = std::max<int64_t>(1, (int64_t)p.k_exc + p.k_inh);
  auto fits = [&](int64_t t) {
    const double lam = (double)t * (double)k / (double)n;
    int cw = 0, cm = 0;
    step_staging_caps((int)std::ceil(lam + 6.0 * std::sqrt(lam) + 16.0), wsz, &cw, &cm);
    const size_t fixed = step_smem_bytes((int)t, p.d_max + 1, p.d_min + 1, (int)ceil_div(n, t), false, 0, n_warps, true);
    return fixed + (size_t)2 * kStages * (cw + cm) <= smem_cap;
  };
  int64_t lo = std::min<int64_t>(n, 32ll * n_warps), hi = std::min<int64_t>(n, 65535);
  if (fits(hi)) return hi;
  while (hi - lo > 1) {  // fits(lo) is assumed: the smallest block always fits
    const int64_t mid = (lo + hi) / 2;
    (fits(mid) ? lo : hi) = mid;
  }
  return lo;
}

// Targets per block for every network so that all blocks are co-resident (one per SM).  Every
// network is cut into equal blocks.  A budget common to all networks sets the size of their
// blocks: balance 0, targets (T per block); balance 1, synapses (a network of in-degree K gets
// about budget / K targets per block), so that blocks of a batch with uneven in-degrees carry
// similar delivery work; balance 2, work (a network whose targets cost w each per step gets about
// budget / w), so that blocks of networks with uneven firing rates finish their steps together.
// No block exceeds max_block_targets.  The budget grows until the blocks fit on the SMs and is
// then bisected down to the smallest budget that still fits.
int plan_blocks(cortex_net* h, const cortex_options& o, std::vector<int32_t>& tb) {
  const int cap = h->n_sm;  // one block per SM
  const int64_t tmin = 32ll * h->n_warps;
  const int wsz = h->wdtype == CORTEX_BF16 ? 2 : 4;
  const bool fixed_t = o.targets_per_block > 0;
  const int mode = fixed_t ? 0 : o.balance;
  std::vector<int64_t> tcap(h->n_nets);
  std::vector<double> cost(h->n_nets);  // budget units per target of each network
  int64_t n_total = 0;
  double total = 0.0, cmax = 0.0;
  for (int b = 0; b < h->n_nets; ++b) {
    const cortex_params& p = h->params[b];
    const int64_t n = (int64_t)p.n_exc + p.n_inh, k = std::max<int64_t>(1, (int64_t)p.k_exc + p.k_inh);
    tcap[b] = max_block_targets(p, wsz, h->n_warps, h->smem_cap);
    cost[b] = mode == 0 ? 1.0 : mode == 1 ? (double)k : (double)o.net_work[b];
    n_total += n;
    total += (double)n * cost[b];
    cmax = std::max(cmax, cost[b]);
  }
  double S = mode == 0 ? (double)std::max<int64_t>(tmin, ceil_div(n_total, cap))
                       : std::max((double)tmin * cmax, std::ceil(total / cap));
  if (fixed_t) S = std::min<double>(S, o.targets_per_block);
  // the plan of budget S: targets per block of every network; returns the block count, and
  // whether every network is at its largest block already (a larger budget changes nothing)
  auto plan_for = [&](double S, std::vector<int32_t>& out, bool& capped) -> int64_t {
    int64_t blocks = 0;
    capped = true;
    out.assign(h->n_nets, 0);
    for (int b = 0; b < h->n_nets; ++b) {
      const int64_t n = (int64_t)h->params[b].n_exc + h->params[b].n_inh;
      int64_t t = std::min<int64_t>(n, std::max<int64_t>(tmin, (int64_t)(S / cost[b])));
      capped = capped && (t >= n || (!fixed_t && t >= tcap[b]));
      if (!fixed_t) t = std::min(t, tcap[b]);
      // balance the blocks of one network
      const int64_t nb = ceil_div(n, t);
      t = ceil_div(n, nb);
      out[b] = (int32_t)std::min<int64_t>(t, 1 << 30);
      blocks += nb;
    }
    return blocks;
  };
  auto too_wide = [&](const std::vector<int32_t>& t) {
    for (int32_t x : t)
      if (x > 65535) return fail(CORTEX_ERR_UNSUPPORTED, "targets per block above 65535 (network too large for one GPU plan)");
    return CORTEX_OK;
  };
  bool capped = false;
  int64_t blocks = plan_for(S, tb, capped);
  if (too_wide(tb) != CORTEX_OK) return CORTEX_ERR_UNSUPPORTED;
  if (blocks <= cap || fixed_t) return CORTEX_OK;
  // grow the budget until the blocks fit on the SMs (the block count never grows with the budget),
  // then bisect between the last budget that did not fit and the first that did: the smallest
  // budget that fits gives the smallest largest block
  double lo = S;
  for (int iter = 0;; ++iter) {
    if (capped)
      return fail(CORTEX_ERR_UNSUPPORTED, "the networks need " + std::to_string(blocks) + " blocks of at most the " +
                                              "targets shared memory allows, more than the " + std::to_string(cap) +
                                              " SMs (too large for one GPU plan)");
    if (iter == 10000) return fail(CORTEX_ERR_UNSUPPORTED, "could not plan the blocks");
    lo = S;
    S += std::max(1.0, std::floor(S / 16));
    blocks = plan_for(S, tb, capped);
    if (too_wide(tb) != CORTEX_OK) return CORTEX_ERR_UNSUPPORTED;
    if (blocks <= cap) break;
  }
  std::vector<int32_t> trial;
  for (int it = 0; it < 64 && S - lo > (mode == 0 ? 1.0 : 1e-9 * S); ++it) {
    const double mid = mode == 0 ? std::floor((lo + S) / 2) : (lo + S) / 2;
    bool c2 = false;
    if (plan_for(mid, trial, c2) <= cap) {
      S = mid;
      tb.swap(trial);
    } else {
      lo = mid;
    }
  }
  return CORTEX_OK;
}

// parameters of every network and the options, checked before anything is allocated
int check_inputs(const cortex_params* params, int32_t n_nets, const cortex_options& o) {
  for (int b = 0; b < n_nets; ++b) {
    std::string why;
    int rc = validate_params(params[b], why);
    if (rc != CORTEX_OK) return fail(rc, "network " + std::to_string(b) + ": " + why);
    if (params[b].weight_dtype != params[0].weight_dtype)
      return fail(CORTEX_ERR_UNSUPPORTED, "all networks of a batch must use the same weight_dtype");
  }
  if (o.warps_per_block < 0) return fail(CORTEX_ERR_ARG, "warps_per_block must be >= 0");
  if (o.mode != CORTEX_MODE_PERSISTENT && o.mode != CORTEX_MODE_SPLIT) return fail(CORTEX_ERR_ARG, "mode");
  if (o.ring < 0 || o.ring > 2) return fail(CORTEX_ERR_ARG, "ring");
  if (o.balance < 0 || o.balance > 2) return fail(CORTEX_ERR_ARG, "balance");
  if (o.balance == 2) {
    if (!o.net_work) return fail(CORTEX_ERR_ARG, "balance 2 needs net_work");
    for (int b = 0; b < n_nets; ++b)
      if (!(o.net_work[b] > 0.0f) || !std::isfinite(o.net_work[b])) return fail(CORTEX_ERR_ARG, "net_work must be finite and > 0");
  }
  if (o.spikes_per_round < 0 || o.spikes_per_round > kSpikeBatch) return fail(CORTEX_ERR_ARG, "spikes_per_round must be 0..32");
  if (o.fold < CORTEX_FOLD_AUTO || o.fold > CORTEX_FOLD_EXACT) return fail(CORTEX_ERR_ARG, "fold must be 0..2");
  if (o.l2_persist < -1 || o.l2_persist > 1) return fail(CORTEX_ERR_ARG, "l2_persist must be -1, 0 or 1");
  if (o.delivery != CORTEX_DELIVERY_RING && o.delivery != CORTEX_DELIVERY_DELAY) return fail(CORTEX_ERR_ARG, "delivery");
  if (o.check_ownership < 0 || o.check_ownership > 1) return fail(CORTEX_ERR_ARG, "check_ownership must be 0 or 1");
  if (o.helper_warp < -1 || o.helper_warp > 1) return fail(CORTEX_ERR_ARG, "helper_warp must be -1, 0 or 1");
  if (o.helper_warp > 0 && o.warps_per_block >= kMaxWarps)
    return fail(CORTEX_ERR_ARG, "helper_warp needs warps_per_block <= 15 (the helper is one more warp)");
  if (o.check_ownership && o.delivery == CORTEX_DELIVERY_DELAY)
    return fail(CORTEX_ERR_UNSUPPORTED, "the ownership check stamps ring cells: ring delivery only");
  if (o.delivery == CORTEX_DELIVERY_DELAY) {
    if (o.mode == CORTEX_MODE_SPLIT) return fail(CORTEX_ERR_UNSUPPORTED, "delay-ordered delivery runs in persistent mode only");
    if (o.warps_per_block < 0 || o.warps_per_block > kDMaxWarps) return fail(CORTEX_ERR_ARG, "warps_per_block must be 1..32");
  } else if (o.warps_per_block > kMaxWarps) {
    return fail(CORTEX_ERR_ARG, "warps_per_block must be 1..16");
  }
  return CORTEX_OK;
}

}  // namespace

cortex_net::~cortex_net() {
  l2_persist_release(this);
  destroy();
}

namespace {

int check_err(cortex_net* h, const char* where) {
  int32_t e = 0;
  CUDA_TRY(cudaMemcpyAsync(&e, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (e & kErrTimeout) {
    h->timed_out = true;
    return fail(CORTEX_ERR_TIMEOUT, std::string(where) + ": a device wait timed out");
  }
  if (e & kErrBuild) return fail(CORTEX_ERR_CUDA, std::string(where) + ": builder consistency check failed");
  if (e & kErrSegment) return fail(CORTEX_ERR_UNSUPPORTED, std::string(where) + ": a sub-graph segment exceeds the staging capacity");
  if (e & kErrRaster) return fail(CORTEX_ERR_OVERFLOW, std::string(where) + ": raster capacity exceeded");
  if (h->viol) {
    unsigned long long v[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(v, h->viol, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (v[0])
      return fail(CORTEX_ERR_CHECK, std::string(where) + ": ownership check: " + std::to_string(v[0]) +
                                        " ring cell writes by a second warp (first: global ring cell " +
                                        std::to_string((long long)v[1] - 1) + ")");
  }
  return CORTEX_OK;
}

StepArgs make_args(cortex_net* h) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.nets = h->nets_d;
  a.work = h->work_d;
  a.n_blocks = h->n_blocks;
  a.w_max = h->w_max;
  a.n_total = h->n_total;
  a.rec_w = h->rec_w;
  a.rec_meta = h->rec_meta;
  a.hdr = h->hdr;
  a.row_base = h->row_base;
  a.V = h->V;
  a.I = h->I;
  a.R = h->R;
  a.ring = h->ring;
  a.pub_ids = h->pub_ids;
  a.pub_cnt = h->pub_cnt;
  a.pub_flag = h->pub_flag;
  a.mbox = h->mbox;
  a.raster_step = h->raster_step;
  a.raster_id = h->raster_id;
  a.raster_count = h->raster_count;
  a.events = h->events;
  a.err = h->err;
  a.step_counter = h->step_counter;
  a.timeout_ns = h->timeout_ns;
  a.ring_red = h->ring_red ? 1 : 0;
  a.exact = h->exact ? 1 : 0;
  a.helper_warp = h->helper_warp ? 1 : 0;
  a.bf16 = h->wdtype == CORTEX_BF16 ? 1 : 0;
  a.withhold_block = h->withhold_block;
  a.t_fixed = -1;
  a.dtgt = h->dtgt;
  a.dw = h->dw;
  a.dtbl = h->dtbl;
  a.hist_ids = h->hist_ids;
  a.hist_cnt = h->hist_cnt;
  a.hist_max = h->hist_max;
  a.bar_count = h->bar_count;
  a.stamps = h->stamps;
  a.viol = h->viol;
  return a;
}

cudaError_t launch_persistent(cortex_net* h, int n_steps, cudaStream_t s) {
  StepArgs a = make_args(h);
  a.n_steps = n_steps;
  a.phases = kPhaseUpdate | kPhaseDeliver | kPhaseBarrier;
  a.ring_smem = h->ring_smem ? 1 : 0;
  if (h->delivery == CORTEX_DELIVERY_DELAY) return launch_dstep(a, h->n_blocks, h->d_threads, h->d_smem, s);
  return launch_step(a, h->n_blocks, h->threads, h->smem, true, s, &h->apw);
}

cudaError_t launch_split_window(cortex_net* h, int wn, cudaStream_t s) {
  StepArgs a = make_args(h);
  a.n_steps = wn;
  a.ring_smem = 0;
  a.phases = kPhaseUpdate;
  cudaError_t e = launch_step(a, h->n_blocks, h->threads, h->smem, false, s, &h->apw);
  if (e != cudaSuccess) return e;
  a.phases = kPhaseDeliver;
  a.ring_smem = h->ring_smem ? 1 : 0;  // the delivery launch stages its ring slice in shared memory
  e = launch_step(a, h->n_blocks, h->threads, h->smem, false, s, &h->apw);
  if (e != cudaSuccess) return e;
  return launch_advance_split(a, h->n_nets, wn, s);
}

// Capture one chunk of the step loop in a CUDA graph (persistent: one cooperative launch of
// steps_per_launch steps; split: as many windows as fit in the same number of steps).
int ensure_graph(cortex_net* h) {
  if (h->graph) return CORTEX_OK;
  // capture on a private stream (the legacy default stream cannot be captured); the graph is
  // then launched on the handle's stream
  cudaStream_t cs = nullptr;
  CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    cudaGetLastError();
    h->use_graph = false;
    return CORTEX_OK;
  }
  if (h->mode == CORTEX_MODE_PERSISTENT) {
    e = launch_persistent(h, h->steps_per_launch, cs);
  } else {
    for (int s = 0; s + h->w_split <= h->steps_per_launch && e == cudaSuccess; s += h->w_split)
      e = launch_split_window(h, h->w_split, cs);
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    h->use_graph = false;  // fall back to direct launches
    return CORTEX_OK;
  }
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->graph = nullptr;
    h->use_graph = false;
    return CORTEX_OK;
  }
  h->graph_steps = (h->mode == CORTEX_MODE_PERSISTENT) ? h->steps_per_launch
                                                       : (h->steps_per_launch / h->w_split) * h->w_split;
  return CORTEX_OK;
}

int build_network(cortex_net* h, int b, const std::vector<int32_t>& tb) {
  const NetDev& nd = h->nets_h[b];
  const int64_t n = nd.n;
  const int nbk = nd.n_blocks;
  cudaStream_t st = h->stream;
  // 1. counts of every (block, source) and the rows of the CSR by source
  uint32_t *cnt_all = nullptr, *off_all = nullptr, *rowcnt = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&cnt_all, (size_t)nbk * n * 4, st));
  CUDA_TRY(cudaMallocAsync((void**)&off_all, (size_t)nbk * n * 4, st));
  CUDA_TRY(cudaMallocAsync((void**)&rowcnt, (size_t)n * 4, st));
  CUDA_TRY(cudaMemsetAsync(cnt_all, 0, (size_t)nbk * n * 4, st));
  CUDA_TRY(launch_build_count_net(h->nets_d, b, (int32_t)n, 0, nbk, tb[b], cnt_all, st));
  CUDA_TRY(launch_build_rows(cnt_all, nbk, (int32_t)n, off_all, rowcnt, h->row_base + nd.row_off, st));
  // 2. waves of blocks (keys scratch bounded): scan, fill, finalize
  const int64_t keys_per_block = (int64_t)tb[b] * nd.k;
  int per_wave = (int)std::max<int64_t>(1, std::min<int64_t>(nbk, (int64_t)(kKeyBudget / 4) / std::max<int64_t>(1, keys_per_block)));
  uint32_t *cursor = nullptr, *keys = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&cursor, (size_t)per_wave * n * 4, st));
  CUDA_TRY(cudaMallocAsync((void**)&keys, (size_t)std::max<int64_t>(1, per_wave * keys_per_block) * 4, st));
  int rc = CORTEX_OK;
  for (int g0 = 0; g0 < nbk && rc == CORTEX_OK; g0 += per_wave) {
    const int ng = std::min(per_wave, nbk - g0);
    uint32_t* cnt = cnt_all + (size_t)g0 * n;
    cudaError_t e = launch_scan_groups(cnt, cursor, ng, (int32_t)n, nullptr, st);
    if (e == cudaSuccess) e = launch_build_fill_net(h->nets_d, b, (int32_t)n, g0, ng, tb[b], cursor, keys, st);
    if (e == cudaSuccess)
      e = launch_build_finalize_net(h->nets_d, h->work_d, b, g0, ng, h->n_warps, cnt, cursor, keys, off_all,
                                    h->row_base, h->rec_w, h->rec_meta, h->hdr, h->err, h->max_seg + b, st);
    if (e != cudaSuccess) rc = fail(CORTEX_ERR_CUDA, std::string("builder: ") + cudaGetErrorString(e));
  }
  cudaFreeAsync(cnt_all, st);
  cudaFreeAsync(off_all, st);
  cudaFreeAsync(rowcnt, st);
  cudaFreeAsync(cursor, st);
  cudaFreeAsync(keys, st);
  return rc;
}

// Shared-memory layout of each network: state for its blocks' targets, and staging bytes per
// spike from its own longest piece.  Each network's rounds hold as many spikes (up to 32) as fit
// next to its state; the launch reserves the largest layout.  The ring goes to shared memory when
// every network still gets rounds of at least 16 spikes next to it.
int choose_stage_and_ring(cortex_net* h, const cortex_options& o) {
  const int wsz = h->wdtype == CORTEX_BF16 ? 2 : 4;
  const int cap_round = o.spikes_per_round > 0 ? o.spikes_per_round : kSpikeBatch;
  const int nn = h->n_nets;
  std::vector<int> cw(nn), cm(nn);
  std::vector<size_t> per(nn);  // staging bytes per spike of a round (kStages rounds in flight)
  // the helper warp (it fetches the piece headers and builds the descriptors while the others
  // fold): as asked, else automatic for the persistent kernel with the ring in global memory (where
  // it measured faster; with the ring in shared memory it measured slower)
  auto helper_for = [&](bool ring) {
    if (h->delivery != CORTEX_DELIVERY_RING || h->n_warps >= kMaxWarps) return false;
    if (o.helper_warp != 0) return o.helper_warp > 0;
    return !h->no_auto_helper && h->mode == CORTEX_MODE_PERSISTENT && !ring;
  };
  auto layout = [&](int b, bool ring, size_t stage) {
    const NetDev& d = h->nets_h[b];
    return step_smem_bytes(h->work_h[d.first_block].nt, d.depth, d.window, d.n_blocks, ring, (int)stage, h->n_warps,
                           !h->exact);
  };
  auto room = [&](int b, bool ring) -> size_t {  // staging bytes that fit next to the rest
    const size_t fixed = layout(b, ring, 0);
    return fixed >= h->smem_cap ? 0 : (h->smem_cap - fixed) / 16 * 16;
  };
  size_t fit_smem = SIZE_MAX, fit_glob = SIZE_MAX;  // fewest spikes per round over the networks
  for (int b = 0; b < nn; ++b) {
    step_staging_caps((int)std::max<uint32_t>(h->max_seg_len[b], 1u), wsz, &cw[b], &cm[b]);
    per[b] = (size_t)kStages * (cw[b] + cm[b]);
    fit_smem = std::min(fit_smem, room(b, true) / per[b]);
    fit_glob = std::min(fit_glob, room(b, false) / per[b]);
  }
  bool smem_ring;
  if (o.ring == CORTEX_RING_SMEM) smem_ring = true;
  else if (o.ring == CORTEX_RING_GLOBAL) smem_ring = false;
  else smem_ring = fit_smem >= 16;
  if ((smem_ring ? fit_smem : fit_glob) < 1)
    return fail(CORTEX_ERR_UNSUPPORTED, std::string("shared memory too small for this plan (ring in ") +
                                            (smem_ring ? "shared" : "global") + " memory)");
  h->ring_smem = smem_ring;
  h->helper_warp = helper_for(smem_ring);
  h->threads = 32 * (h->n_warps + (h->helper_warp ? 1 : 0));
  {
    // reductions flush subnormals: allowed when every weight is 0 or >= 2^-102 in magnitude (with
    // margin for bf16 rounding), so that no partial sum of a cell can be subnormal
    bool ok = true;
    for (const auto& p : h->params)
      for (float w : {p.j_exc, p.j_inh})
        ok = ok && (w == 0.0f || std::fabs(w) >= std::ldexp(1.0f, -102));
    h->ring_red = ok && !smem_ring;
  }
  h->smem = 0;
  h->stage_bytes = 0;
  h->batch = kSpikeBatch;
  for (int b = 0; b < nn; ++b) {
    const int bb = (int)std::min<size_t>((size_t)cap_round, room(b, smem_ring) / per[b]);
    NetDev& d = h->nets_h[b];
    d.batch = bb;
    d.cap_w = cw[b];
    d.cap_m = cm[b];
    d.stage_bytes = (int32_t)(per[b] * bb);
    h->smem = std::max(h->smem, layout(b, smem_ring, (size_t)d.stage_bytes));
    h->stage_bytes = std::max(h->stage_bytes, d.stage_bytes);
    h->batch = std::min(h->batch, bb);
  }
  CUDA_TRY(step_kernel_attributes(h->smem));
  if (h->helper_warp && o.helper_warp == 0 && step_occupancy(h->threads, h->smem, h->ring_smem) * h->n_sm < h->n_blocks) {
    h->no_auto_helper = true;  // the automatic helper would keep the blocks from being co-resident
    return choose_stage_and_ring(h, o);
  }
  CUDA_TRY(cudaMemcpyAsync(h->nets_d, h->nets_h.data(), sizeof(NetDev) * nn, cudaMemcpyHostToDevice, h->stream));
  h->h2d_bytes += (int64_t)(sizeof(NetDev) * nn);
  return CORTEX_OK;
}

// The layout again, after the handle switched from the order-free to the ordered fold (its shared
// memory then holds the duplicate-detection tags): stage, ring placement and helper warp as at the
// build, and split launches if the persistent kernel's blocks are no longer co-resident.
int relayout_for_fold(cortex_net* h) {
  int rc = choose_stage_and_ring(h, h->build_opts);
  if (rc != CORTEX_OK) return rc;
  if (h->mode == CORTEX_MODE_PERSISTENT && h->delivery == CORTEX_DELIVERY_RING &&
      step_occupancy(h->threads, h->smem, h->ring_smem) * h->n_sm < h->n_blocks) {
    h->mode = CORTEX_MODE_SPLIT;
    rc = choose_stage_and_ring(h, h->build_opts);
  }
  return rc;
}

}  // namespace

extern "C" {

const char* cortex_strerror(int code) {
  switch (code) {
    case CORTEX_OK: return "ok";
    case CORTEX_ERR_ARG: return "invalid argument";
    case CORTEX_ERR_OOM: return "out of memory";
    case CORTEX_ERR_CUDA: return "CUDA error";
    case CORTEX_ERR_TIMEOUT: return "device wait timed out";
    case CORTEX_ERR_UNSUPPORTED: return "unsupported size or configuration";
    case CORTEX_ERR_OVERFLOW: return "buffer too small";
    case CORTEX_ERR_CHECK: return "ownership check failed";
    default: return "unknown status";
  }
}

const char* cortex_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace cortex {
int record_error(int code, const char* msg) {
  g_last_error = msg;
  return code;
}
}  // namespace cortex

extern "C" {

void cortex_free(cortex_net* net) {
  if (!net) return;
  if (net->stream) cudaStreamSynchronize(net->stream);
  delete net;
}

int cortex_build_batch(const cortex_params* params, const uint64_t* seeds, int32_t n_nets, const cortex_options* opts,
                       void* stream, cortex_net** out) {
  NvtxRange nvtx_range("cortex_build");
  if (!out) return fail(CORTEX_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!params || !seeds || n_nets <= 0) return fail(CORTEX_ERR_ARG, "params, seeds, n_nets");
  cortex_options o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  int rc = check_inputs(params, n_nets, o);
  if (rc != CORTEX_OK) return rc;

  cortex_net* h = new (std::nothrow) cortex_net();
  if (!h) return fail(CORTEX_ERR_OOM, "handle");
  auto bail = [&](int rc) {
    delete h;
    return rc;
  };
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->build_opts = o;
  if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(CORTEX_ERR_UNSUPPORTED, "no CUDA device"));
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return bail(fail(CORTEX_ERR_CUDA, "device properties"));
  if (prop.major < 10) return bail(fail(CORTEX_ERR_UNSUPPORTED, "needs a Blackwell GPU (sm_103a build)"));
  h->n_sm = prop.multiProcessorCount;
  h->smem_cap = (size_t)prop.sharedMemPerBlockOptin - 1024;  // room for static shared memory
  h->n_nets = n_nets;
  h->params.assign(params, params + n_nets);
  h->seeds.assign(seeds, seeds + n_nets);
  h->wdtype = params[0].weight_dtype;
  h->delivery = o.delivery;
  if (h->delivery == CORTEX_DELIVERY_DELAY) {
    // the delay-ordered kernel runs up to 32 warps; the records are first built in the ring layout,
    // whose piece headers describe at most 16 warps
    h->d_threads = 32 * (o.warps_per_block ? o.warps_per_block : kDMaxWarps);
    h->n_warps = std::min(o.warps_per_block ? o.warps_per_block : 14, kMaxWarps);
  } else {
    h->n_warps = o.warps_per_block ? o.warps_per_block : 14;
  }
  h->helper_warp = o.helper_warp > 0 && h->delivery == CORTEX_DELIVERY_RING;
  h->threads = 32 * (h->n_warps + (h->helper_warp ? 1 : 0));
  h->mode = o.mode;
  h->steps_per_launch = o.steps_per_launch > 0 ? o.steps_per_launch : 1000;
  h->use_graph = o.use_graph >= 0;
  if (o.barrier_timeout_ms > 0) h->timeout_ns = (long long)(o.barrier_timeout_ms * 1e6);
  h->withhold_block = o.test_withhold_block > 0 ? o.test_withhold_block - 1 : -1;

  std::vector<int32_t> tb;
  rc = plan_blocks(h, o, tb);
  if (rc != CORTEX_OK) return bail(rc);

  // networks and the work table
  h->w_max = 1;
  h->w_split = 1 << 30;
  int64_t neuron_base = 0, rec = 0, hdr = 0, ring = 0, raster = 0;
  for (int b = 0; b < n_nets; ++b) {
    const cortex_params& p = params[b];
    NetDev d;
    memset(&d, 0, sizeof(d));
    d.n_exc = p.n_exc;
    d.n_inh = p.n_inh;
    d.n = p.n_exc + p.n_inh;
    d.k_exc = p.k_exc;
    d.k_inh = p.k_inh;
    d.k = p.k_exc + p.k_inh;
    d.d_min = p.d_min;
    d.d_max = p.d_max;
    d.depth = p.d_max + 1;   // the persistent window leaves one slot pending across its barrier
    d.window = p.d_min + 1;  // persistent window (split launches use at most d_min steps)
    d.dbits = 0;
    while ((1 << d.dbits) < p.d_max - p.d_min + 1) ++d.dbits;
    d.seed_lo = (uint32_t)seeds[b];
    d.seed_hi = (uint32_t)(seeds[b] >> 32);
    d.wdtype = p.weight_dtype;
    d.v_th = p.v_th;
    d.v_reset = p.v_reset;
    d.j_ext = p.j_ext;
    d.tau_m = p.tau_m;
    d.c_m = p.c_m;
    d.tau_syn = p.tau_syn;
    d.t_ref = p.t_ref;
    d.dt = p.dt;
    d.nu_ext_hz = p.nu_ext_hz;
    d.j_exc_in = p.j_exc;
    d.j_inh_in = p.j_inh;
    d.neuron_base = neuron_base;
    d.row_off = neuron_base;
    d.rec_base = rec;
    d.hdr_base = hdr;
    const int nbk = (int)ceil_div(d.n, tb[b]);
    d.first_block = (int)h->work_h.size();
    d.n_blocks = nbk;
    const int64_t rcap = o.raster_capacity > 0 ? o.raster_capacity : std::max<int64_t>(1 << 20, 16ll * d.n);
    d.raster_base = raster;
    d.raster_cap = rcap;
    raster += rcap;
    d.tbl_stride = (p.d_max - p.d_min + 2) * nbk;  // per block: one offset per delay and the piece end
    d.tbl_base = h->total_tbl;
    d.hist_depth = p.d_max + d.window + 1;
    if (h->delivery == CORTEX_DELIVERY_DELAY) {
      if ((p.d_max + 1) * (nbk + 2) > kDCntCap)
        return bail(fail(CORTEX_ERR_UNSUPPORTED, "delay-ordered delivery: (d_max + 1) * (blocks + 2) of a network above " +
                                                     std::to_string(kDCntCap)));
      h->total_tbl += (int64_t)d.n * d.tbl_stride;
      h->hist_max = std::max(h->hist_max, d.hist_depth);
    }
    const int32_t tw = (int32_t)ceil_div(tb[b], h->n_warps);  // targets per warp
    if ((int64_t)tw > (1ll << (16 - d.dbits)))
      return bail(fail(CORTEX_ERR_UNSUPPORTED, "targets per delivery warp (" + std::to_string(tw) +
                                                   ") do not fit the 16-bit record with " + std::to_string(d.dbits) +
                                                   " delay bits; use more warps per block"));
    for (int g = 0; g < nbk; ++g) {
      BlockWork w;
      memset(&w, 0, sizeof(w));
      w.net = b;
      w.group = g;
      w.t0 = g * tb[b];
      w.nt = std::min<int32_t>(tb[b], d.n - w.t0);
      w.tw = tw;
      w.n_src = d.n;
      w.rec_base = rec;
      w.hdr_base = hdr;
      w.ring_base = ring;
      w.pub_base = neuron_base + w.t0;
      rec += (int64_t)w.nt * d.k;
      hdr += d.n;
      ring += (int64_t)d.depth * w.nt;
      h->work_h.push_back(w);
    }
    h->w_max = std::max(h->w_max, d.window);
    h->w_split = std::min(h->w_split, d.d_min);
    neuron_base += d.n;
    h->nets_h.push_back(d);
  }
  h->n_blocks = (int)h->work_h.size();
  h->n_total = neuron_base;
  h->total_syn = rec;
  h->total_hdr = hdr;
  h->total_ring = ring;
  h->total_raster = raster;

  cudaStream_t s = h->stream;
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
    return bail(fail(CORTEX_ERR_CUDA, "events"));
  auto A = [&](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return CORTEX_OK;
    return fail(e == cudaErrorMemoryAllocation ? CORTEX_ERR_OOM : CORTEX_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
#define TRY(e, what)                 \
  do {                               \
    int r_ = A((e), (what));         \
    if (r_ != CORTEX_OK) return bail(r_); \
  } while (0)

  const size_t wsz = h->wdtype == CORTEX_BF16 ? 2 : 4;
  TRY(h->alloc(&h->nets_d, sizeof(NetDev) * n_nets), "alloc nets");
  TRY(h->alloc(&h->work_d, sizeof(BlockWork) * h->n_blocks), "alloc work");
  TRY(h->alloc(&h->rec_w, wsz * h->total_syn + 64), "alloc weights");
  TRY(h->alloc(&h->rec_meta, 2 * h->total_syn + 64), "alloc record meta");
  TRY(h->alloc(&h->hdr, 32 * h->total_hdr), "alloc headers");
  TRY(h->alloc(&h->row_base, 8 * h->n_total), "alloc rows");
  TRY(h->alloc(&h->V, 4 * h->n_total), "alloc V");
  TRY(h->alloc(&h->I, 4 * h->n_total), "alloc I");
  TRY(h->alloc(&h->R, 4 * h->n_total), "alloc R");
  TRY(h->alloc(&h->ring, 4 * h->total_ring), "alloc ring");
  TRY(h->alloc(&h->pub_ids, 4 * (size_t)2 * h->w_max * h->n_total), "alloc spike lists");
  TRY(h->alloc(&h->pub_cnt, 4 * (size_t)2 * h->w_max * h->n_blocks), "alloc spike counts");
  TRY(h->alloc(&h->pub_flag, 8 * (size_t)h->n_blocks), "alloc flags");
  TRY(h->alloc(&h->mbox, 8 * 2 * (size_t)kMboxWords * h->n_blocks), "alloc mailboxes");
  TRY(h->alloc(&h->raster_step, 4 * h->total_raster), "alloc raster");
  TRY(h->alloc(&h->raster_id, 4 * h->total_raster), "alloc raster");
  TRY(h->alloc(&h->raster_count, 8 * (size_t)n_nets), "alloc counters");
  TRY(h->alloc(&h->events, 8 * (size_t)n_nets), "alloc counters");
  TRY(h->alloc(&h->err, 16), "alloc err");
  TRY(h->alloc(&h->step_counter, 16), "alloc step");
  TRY(h->alloc(&h->max_seg, 4 * (size_t)n_nets), "alloc max_seg");
  if (o.check_ownership) {
    TRY(h->alloc(&h->stamps, 4 * h->total_ring + 16), "alloc ownership stamps");
    TRY(h->alloc(&h->viol, 16), "alloc ownership counters");
    TRY(cudaMemsetAsync(h->stamps, 0, 4 * h->total_ring + 16, s), "memset stamps");
    TRY(cudaMemsetAsync(h->viol, 0, 16, s), "memset ownership counters");
  }
  if (h->delivery == CORTEX_DELIVERY_DELAY) {
    // BF16: one packed u32 per record (target, weight); FP32: u16 targets and float weights
    TRY(h->alloc(&h->dtgt, h->wdtype == CORTEX_BF16 ? 64 : 2 * h->total_syn + 64), "alloc delay-ordered targets");
    TRY(h->alloc(&h->dw, 4 * h->total_syn + 64), "alloc delay-ordered records");
    TRY(h->alloc(&h->dtbl, 2 * h->total_tbl + 64), "alloc delay tables");
    TRY(h->alloc(&h->hist_ids, 4 * (size_t)h->hist_max * h->n_total), "alloc spike buffer");
    TRY(h->alloc(&h->hist_cnt, 4 * (size_t)h->hist_max * h->n_blocks), "alloc spike buffer counts");
    TRY(h->alloc(&h->bar_count, 8 * (size_t)n_nets), "alloc barrier counters");
  }

  TRY(cudaEventRecord(h->ev0, s), "event");
  TRY(cudaMemcpyAsync(h->nets_d, h->nets_h.data(), sizeof(NetDev) * n_nets, cudaMemcpyHostToDevice, s), "upload nets");
  TRY(cudaMemcpyAsync(h->work_d, h->work_h.data(), sizeof(BlockWork) * h->n_blocks, cudaMemcpyHostToDevice, s), "upload work");
  h->h2d_bytes += (int64_t)(sizeof(NetDev) * n_nets + sizeof(BlockWork) * h->n_blocks);
  TRY(cudaMemsetAsync(h->err, 0, 16, s), "memset");
  TRY(cudaMemsetAsync(h->max_seg, 0, 4 * (size_t)n_nets, s), "memset");
  TRY(cudaMemsetAsync(h->step_counter, 0, 16, s), "memset");
  TRY(launch_props(h->nets_d, n_nets, s), "propagators");
  TRY(cudaMemcpyAsync(h->nets_h.data(), h->nets_d, sizeof(NetDev) * n_nets, cudaMemcpyDeviceToHost, s), "download nets");
  TRY(cudaStreamSynchronize(s), "sync");
  for (int b = 0; b < n_nets; ++b)
    if (h->nets_h[b].n_thr < 1) return bail(fail(CORTEX_ERR_UNSUPPORTED, "Poisson rate too high for the threshold table"));

  for (int b = 0; b < n_nets; ++b) {
    rc = build_network(h, b, tb);
    if (rc != CORTEX_OK) return bail(rc);
    TRY(launch_init_state(&h->nets_h[b], h->nets_d, b, h->V, h->I, h->R, s), "init state");
    if (h->delivery == CORTEX_DELIVERY_DELAY) {
      // the delay-ordered layout reads every piece header: only once the builder has written them
      // all (a piece over the staging cap or a row over 65,535 records leaves headers unwritten
      // or truncated)
      rc = check_err(h, "build");
      if (rc != CORTEX_OK) return bail(rc);
      TRY(launch_delay_layout(h->nets_d, &h->nets_h[b], h->work_d, b, h->n_warps, h->hdr, h->row_base, h->rec_w,
                              h->rec_meta, h->dtbl, h->dtgt, h->dw, h->err, s),
          "delay-ordered layout");
    }
  }
  if (h->delivery == CORTEX_DELIVERY_DELAY) {
    TRY(cudaMemsetAsync(h->hist_cnt, 0, 4 * (size_t)h->hist_max * h->n_blocks, s), "memset spike buffer");
    TRY(cudaMemsetAsync(h->bar_count, 0, 8 * (size_t)n_nets, s), "memset barrier");
  }
  TRY(cudaMemsetAsync(h->ring, 0, 4 * h->total_ring, s), "memset ring");
  TRY(cudaMemsetAsync(h->pub_flag, 0, 8 * (size_t)h->n_blocks, s), "memset flags");
  TRY(cudaMemsetAsync(h->mbox, 0, 8 * 2 * (size_t)kMboxWords * h->n_blocks, s), "memset mailboxes");
  TRY(cudaMemsetAsync(h->pub_cnt, 0, 4 * (size_t)2 * h->w_max * h->n_blocks, s), "memset counts");
  TRY(cudaMemsetAsync(h->raster_count, 0, 8 * (size_t)n_nets, s), "memset");
  TRY(cudaMemsetAsync(h->events, 0, 8 * (size_t)n_nets, s), "memset");
  h->max_seg_len.assign(n_nets, 0u);
  TRY(cudaMemcpyAsync(h->max_seg_len.data(), h->max_seg, 4 * (size_t)n_nets, cudaMemcpyDeviceToHost, s), "download");
  TRY(cudaEventRecord(h->ev1, s), "event");
  rc = check_err(h, "build");
  if (rc != CORTEX_OK) return bail(rc);
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->build_ms = ms;

  {
    // the fold: order-free adds when every partial sum of a cell is proven exact
    const bool proven = prove_exact(h->nets_h, h->e_min, h->exact_bound);
    if (o.fold == CORTEX_FOLD_EXACT && !proven)
      return bail(fail(CORTEX_ERR_UNSUPPORTED, "fold EXACT: the weights do not make every partial sum of a ring cell exact"));
    h->exact = proven && o.fold != CORTEX_FOLD_ORDERED;
  }
  rc = choose_stage_and_ring(h, o);
  if (rc != CORTEX_OK) return bail(rc);
  if (h->mode == CORTEX_MODE_PERSISTENT && h->delivery == CORTEX_DELIVERY_RING) {
    const int occ = step_occupancy(h->threads, h->smem, h->ring_smem);
    if (occ * h->n_sm < h->n_blocks) {
      if (o.mode == CORTEX_MODE_PERSISTENT && opts && opts->mode == CORTEX_MODE_PERSISTENT && o.ring == CORTEX_RING_SMEM)
        return bail(fail(CORTEX_ERR_UNSUPPORTED, "blocks cannot all be resident for the persistent kernel"));
      h->mode = CORTEX_MODE_SPLIT;  // not co-resident: fall back to split launches
      rc = choose_stage_and_ring(h, o);
      if (rc != CORTEX_OK) return bail(rc);
    }
  }
  if (h->delivery == CORTEX_DELIVERY_DELAY) {
    if (h->mode != CORTEX_MODE_PERSISTENT)
      return bail(fail(CORTEX_ERR_UNSUPPORTED, "delay-ordered delivery: the blocks cannot all be resident"));
    h->d_smem = 0;
    for (const NetDev& d : h->nets_h)
      h->d_smem = std::max(h->d_smem, dstep_smem_bytes(h->work_h[d.first_block].nt, d.window, d.n_blocks, d.d_max,
                                                       h->d_threads / 32, h->exact));
    if (h->d_smem > h->smem_cap)
      return bail(fail(CORTEX_ERR_UNSUPPORTED, "delay-ordered delivery: the accumulators and state of a block need " +
                                                   std::to_string(h->d_smem) + " bytes of shared memory"));
    TRY(dstep_kernel_attributes(h->d_smem), "delay kernel attributes");
    if (dstep_occupancy(h->d_threads, h->d_smem) * h->n_sm < h->n_blocks)
      return bail(fail(CORTEX_ERR_UNSUPPORTED, "delay-ordered delivery: the blocks cannot all be resident"));
  } else if (!h->ring_smem && o.l2_persist > 0) {
    l2_persist_acquire(h, 4 * h->total_ring);
  }
#undef TRY
  *out = h;
  return CORTEX_OK;
}

int cortex_plan(const cortex_params* params, int32_t n_nets, const cortex_options* opts, int32_t n_sm,
                int64_t smem_per_block, int32_t* targets_out, int32_t* n_blocks_out) {
  if (!params || n_nets <= 0 || n_sm <= 0 || smem_per_block <= 1024 || !targets_out)
    return fail(CORTEX_ERR_ARG, "cortex_plan: arguments");
  cortex_options o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  int rc = check_inputs(params, n_nets, o);
  if (rc != CORTEX_OK) return rc;
  cortex_net h;  // host fields only: nothing is allocated on the device
  h.n_sm = n_sm;
  h.smem_cap = (size_t)smem_per_block - 1024;  // as the build: room for static shared memory
  h.n_nets = n_nets;
  h.params.assign(params, params + n_nets);
  h.wdtype = params[0].weight_dtype;
  h.n_warps = o.warps_per_block ? o.warps_per_block : 14;
  std::vector<int32_t> tb;
  rc = plan_blocks(&h, o, tb);
  if (rc != CORTEX_OK) return rc;
  int64_t blocks = 0;
  for (int b = 0; b < n_nets; ++b) {
    targets_out[b] = tb[b];
    blocks += ceil_div((int64_t)params[b].n_exc + params[b].n_inh, tb[b]);
  }
  if (n_blocks_out) *n_blocks_out = (int32_t)blocks;
  return CORTEX_OK;
}

int cortex_build(const cortex_params* params, uint64_t seed, const cortex_options* opts, void* stream,
                 cortex_net** out) {
  return cortex_build_batch(params, &seed, 1, opts, stream, out);
}

int cortex_autotune(const cortex_params* params, const uint64_t* seeds, int32_t n_nets, const cortex_options* base,
                    int32_t trial_steps, void* stream, cortex_options* best, double* best_ms_per_step,
                    int32_t* n_tried, float* net_work_out) {
  NvtxRange nvtx_range("cortex_autotune");
  if (!params || !seeds || n_nets <= 0 || trial_steps <= 0 || !best) return fail(CORTEX_ERR_ARG, "cortex_autotune: arguments");
  cortex_options b0;
  memset(&b0, 0, sizeof(b0));
  if (base) b0 = *base;
  // candidates: warps per block (the width of the per-warp sub-graphs) x block plan; the plans of
  // balance 2 charge a target of network b its measured events per step plus a fixed update cost
  struct Cand {
    int balance, warps;
    float update_cost;
  };
  const int warps[] = {8, 10, 12, 14, 16};
  std::vector<Cand> cands;
  for (int bal = 0; bal <= 1; ++bal)
    for (int w : warps) cands.push_back({bal, w, 0.0f});
  if (net_work_out && n_nets > 1)
    for (float cu : {0.5f, 2.0f, 8.0f})
      for (int w : warps) cands.push_back({2, w, cu});
  std::vector<double> events_per_target;  // per network, from the first candidate that ran
  std::vector<float> work(n_nets), best_work;
  double best_ms = -1.0;
  int tried = 0, last_rc = CORTEX_ERR_UNSUPPORTED;
  for (const Cand& c : cands) {
    cortex_options o = b0;
    o.warps_per_block = c.warps;
    o.balance = c.balance;
    o.net_work = nullptr;
    if (c.balance == 2) {
      if (events_per_target.empty()) continue;
      for (int b = 0; b < n_nets; ++b) work[b] = (float)events_per_target[b] + c.update_cost;
      o.net_work = work.data();
    }
    cortex_net* h = nullptr;
    int rc = cortex_build_batch(params, seeds, n_nets, &o, stream, &h);
    if (rc == CORTEX_OK) rc = cortex_simulate(h, std::min<int64_t>(trial_steps, h->steps_per_launch));  // warm-up
    double ms = 0.0;
    if (rc == CORTEX_OK) {
      rc = cortex_simulate(h, trial_steps);
      ms = h->sim_ms;
    }
    if (rc == CORTEX_OK && events_per_target.empty()) {
      std::vector<unsigned long long> e(n_nets);
      if (cudaMemcpyAsync(e.data(), h->events, 8 * (size_t)n_nets, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        rc = CORTEX_ERR_CUDA;
      events_per_target.resize(n_nets);
      for (int b = 0; b < n_nets; ++b)
        events_per_target[b] = (double)e[b] / ((double)h->nets_h[b].n * (double)std::max<int64_t>(h->step, 1));
    }
    if (h) cortex_free(h);
    if (rc == CORTEX_ERR_CUDA || rc == CORTEX_ERR_TIMEOUT) return rc;  // not a property of the plan
    if (rc != CORTEX_OK) {
      last_rc = rc;
      continue;
    }
    ++tried;
    if (best_ms < 0.0 || ms < best_ms) {
      best_ms = ms;
      *best = o;
      best_work = c.balance == 2 ? work : std::vector<float>();
    }
  }
  if (n_tried) *n_tried = tried;
  if (best_ms < 0.0) return fail(last_rc, "cortex_autotune: no candidate plan could be built");
  if (best->balance == 2) {
    std::copy(best_work.begin(), best_work.end(), net_work_out);
    best->net_work = net_work_out;
  }
  if (best_ms_per_step) *best_ms_per_step = best_ms / trial_steps;
  return CORTEX_OK;
}

int cortex_autotune_cached(const cortex_params* params, const uint64_t* seeds, int32_t n_nets, const cortex_options* base,
                           int32_t trial_steps, void* stream, const char* cache_path, cortex_options* best,
                           double* best_ms_per_step, int32_t* n_tried, float* net_work_out, int32_t* hit) {
  if (hit) *hit = 0;
  if (!cache_path)
    return cortex_autotune(params, seeds, n_nets, base, trial_steps, stream, best, best_ms_per_step, n_tried,
                           net_work_out);
  if (!params || !seeds || n_nets <= 0 || trial_steps <= 0 || !best)
    return fail(CORTEX_ERR_ARG, "cortex_autotune_cached: arguments");
  cortex_options b0;
  memset(&b0, 0, sizeof(b0));
  if (base) b0 = *base;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return fail(CORTEX_ERR_CUDA, "cortex_autotune_cached: device properties");
  // FNV-1a 64 over the fields that decide the tuned plan
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) key = (key ^ c[i]) * 1099511628211ull;
  };
  mix(prop.name, strnlen(prop.name, sizeof(prop.name)));
  mix(&prop.multiProcessorCount, sizeof(int));
  mix(&prop.sharedMemPerBlockOptin, sizeof(size_t));
  mix(&n_nets, sizeof(n_nets));
  for (int b = 0; b < n_nets; ++b) {
    mix(&params[b], sizeof(cortex_params));
    mix(&seeds[b], sizeof(uint64_t));
  }
  const int32_t shape[7] = {b0.ring, b0.mode, b0.targets_per_block, b0.steps_per_launch, b0.spikes_per_round, b0.fold,
                            b0.delivery};
  mix(shape, sizeof(shape));
  mix(&trial_steps, sizeof(trial_steps));
  char khex[17];
  snprintf(khex, sizeof(khex), "%016llx", (unsigned long long)key);
  // lookup: "cortex-autotune-1 <key> <warps> <balance> <ms_per_step> <n_nets> <work_0> ... <work_{n-1}>"
  if (FILE* f = fopen(cache_path, "r")) {
    char line[65536];
    bool found = false;
    int w = 0, bal = 0, nn = 0;
    double ms = 0;
    std::vector<float> work;
    while (fgets(line, sizeof(line), f)) {
      char tag[32], k[32];
      int used = 0;
      int w2 = 0, b2 = 0, n2 = 0;
      double ms2 = 0;
      if (sscanf(line, "%31s %31s %d %d %lf %d%n", tag, k, &w2, &b2, &ms2, &n2, &used) != 6) continue;
      if (strcmp(tag, "cortex-autotune-1") != 0 || strcmp(k, khex) != 0 || n2 != n_nets || b2 < 0 || b2 > 2 || w2 < 1 ||
          w2 > kDMaxWarps)
        continue;
      std::vector<float> wk(n_nets, 0.0f);
      const char* q = line + used;
      bool ok = true;
      for (int b = 0; b < n_nets && ok; ++b) {
        int u = 0;
        ok = sscanf(q, "%f%n", &wk[b], &u) == 1;
        q += u;
      }
      if (!ok) continue;
      found = true;
      w = w2;
      bal = b2;
      ms = ms2;
      nn = n2;
      work.swap(wk);
    }
    fclose(f);
    if (found && nn == n_nets && (bal != 2 || net_work_out)) {
      *best = b0;
      best->warps_per_block = w;
      best->balance = bal;
      best->net_work = nullptr;
      if (bal == 2) {
        std::copy(work.begin(), work.end(), net_work_out);
        best->net_work = net_work_out;
      }
      if (best_ms_per_step) *best_ms_per_step = ms;
      if (n_tried) *n_tried = 0;
      if (hit) *hit = 1;
      return CORTEX_OK;
    }
  }
  double ms = 0;
  int32_t tried = 0;
  const int rc = cortex_autotune(params, seeds, n_nets, base, trial_steps, stream, best, &ms, &tried, net_work_out);
  if (rc != CORTEX_OK) return rc;
  if (best_ms_per_step) *best_ms_per_step = ms;
  if (n_tried) *n_tried = tried;
  FILE* f = fopen(cache_path, "a");
  if (!f) return fail(CORTEX_ERR_ARG, std::string("cortex_autotune_cached: cannot append to ") + cache_path);
  std::string line = std::string("cortex-autotune-1 ") + khex + " " + std::to_string(best->warps_per_block) + " " +
                     std::to_string(best->balance) + " ";
  char num[64];
  snprintf(num, sizeof(num), "%.9g %d", ms, n_nets);
  line += num;
  for (int b = 0; b < n_nets; ++b) {
    snprintf(num, sizeof(num), " %.9g", best->balance == 2 && best->net_work ? (double)best->net_work[b] : 0.0);
    line += num;
  }
  line += "\n";
  const bool wrote = fputs(line.c_str(), f) >= 0;
  fclose(f);
  if (!wrote) return fail(CORTEX_ERR_ARG, std::string("cortex_autotune_cached: cannot append to ") + cache_path);
  return CORTEX_OK;
}

int cortex_simulate(cortex_net* h, int64_t n_steps) {
  NvtxRange nvtx_range("cortex_simulate");
  if (!h || n_steps < 0) return fail(CORTEX_ERR_ARG, "cortex_simulate: handle / n_steps");
  if (h->timed_out) return fail(CORTEX_ERR_TIMEOUT, "cortex_simulate: an earlier device wait timed out; free the handle");
  if (h->no_layout)
    return fail(CORTEX_ERR_UNSUPPORTED, "cortex_simulate: the restored ring needs the ordered fold, whose layout does not fit");
  unsigned long long ev_before = 0;
  {
    std::vector<unsigned long long> e(h->n_nets);
    CUDA_TRY(cudaMemcpyAsync(e.data(), h->events, 8 * h->n_nets, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (auto x : e) ev_before += x;
  }
  CUDA_TRY(cudaMemsetAsync(h->err, 0, 4, h->stream));
  CUDA_TRY(cudaEventRecord(h->ev0, h->stream));
  int64_t left = n_steps;
  if (h->use_graph && left >= h->steps_per_launch) {
    int rc = ensure_graph(h);
    if (rc != CORTEX_OK) return rc;
  }
  while (left > 0) {
    if (h->use_graph && h->graph && left >= h->graph_steps && h->graph_steps > 0) {
      CUDA_TRY(cudaGraphLaunch(h->graph, h->stream));
      left -= h->graph_steps;
      continue;
    }
    if (h->mode == CORTEX_MODE_PERSISTENT) {
      const int n = (int)std::min<int64_t>(left, h->steps_per_launch);
      CUDA_TRY(launch_persistent(h, n, h->stream));
      left -= n;
    } else {
      const int wn = (int)std::min<int64_t>(left, h->w_split);
      CUDA_TRY(launch_split_window(h, wn, h->stream));
      left -= wn;
    }
  }
  CUDA_TRY(cudaEventRecord(h->ev1, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  h->sim_ms = ms;
  h->sim_steps = n_steps;
  h->step += n_steps;
  unsigned long long ev_after = 0;
  {
    std::vector<unsigned long long> e(h->n_nets);
    CUDA_TRY(cudaMemcpy(e.data(), h->events, 8 * h->n_nets, cudaMemcpyDeviceToHost));
    for (auto x : e) ev_after += x;
  }
  h->sim_events = (int64_t)(ev_after - ev_before);
  return check_err(h, "simulate");
}

int cortex_spikes(cortex_net* h, int32_t net_idx, int64_t* n_inout, int32_t* steps, int32_t* ids) {
  NvtxRange nvtx_range("cortex_spikes");
  if (!h || !n_inout || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_spikes: arguments");
  unsigned long long c = 0;
  CUDA_TRY(cudaMemcpyAsync(&c, h->raster_count + net_idx, 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  const NetDev& d = h->nets_h[net_idx];
  const int64_t n = std::min<int64_t>((int64_t)c, d.raster_cap);
  if (*n_inout < n) {
    *n_inout = n;
    return fail(CORTEX_ERR_OVERFLOW, "cortex_spikes: capacity too small");
  }
  *n_inout = n;
  if (n == 0) return CORTEX_OK;
  if (!steps || !ids) return fail(CORTEX_ERR_ARG, "cortex_spikes: NULL output");
  CUDA_TRY(cudaMemcpyAsync(steps, h->raster_step + d.raster_base, 4 * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(ids, h->raster_id + d.raster_base, 4 * n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CORTEX_OK;
}

int cortex_clear_spikes(cortex_net* h) {
  if (!h) return fail(CORTEX_ERR_ARG, "handle");
  std::vector<unsigned long long> c(h->n_nets);
  CUDA_TRY(cudaMemcpyAsync(c.data(), h->raster_count, 8 * h->n_nets, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (auto x : c) h->spikes_cleared += (int64_t)x;
  CUDA_TRY(cudaMemsetAsync(h->raster_count, 0, 8 * h->n_nets, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CORTEX_OK;
}

int cortex_stats(cortex_net* h, cortex_stats_t* st) {
  if (!h || !st) return fail(CORTEX_ERR_ARG, "cortex_stats: arguments");
  memset(st, 0, sizeof(*st));
  std::vector<unsigned long long> c(h->n_nets), e(h->n_nets);
  CUDA_TRY(cudaMemcpyAsync(c.data(), h->raster_count, 8 * h->n_nets, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(e.data(), h->events, 8 * h->n_nets, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  st->n_nets = h->n_nets;
  st->n_neurons = h->n_total;
  st->n_synapses = h->total_syn;
  st->step = h->step;
  st->spikes = h->spikes_cleared;
  for (auto x : c) st->spikes += (int64_t)x;
  for (auto x : e) st->events += (int64_t)x;
  st->build_ms = h->build_ms;
  st->simulate_ms = h->sim_ms;
  st->simulate_steps = h->sim_steps;
  st->simulate_events = h->sim_events;
  st->n_blocks = h->n_blocks;
  st->threads_per_block = h->threads;
  st->helper_warp = h->helper_warp ? 1 : 0;
  st->ring_in_smem = h->ring_smem ? 1 : 0;
  st->mode = h->mode;
  st->device_bytes = (int64_t)h->device_bytes;
  st->spikes_per_round = h->batch;
  st->smem_bytes = (int32_t)h->smem;
  st->exact_fold = h->exact ? 1 : 0;
  st->l2_persist_bytes = (int64_t)h->apw.num_bytes;
  st->delivery = h->delivery;
  st->build_h2d_bytes = h->h2d_bytes;
  if (h->delivery == CORTEX_DELIVERY_DELAY) {
    st->threads_per_block = h->d_threads;
    st->smem_bytes = (int32_t)h->d_smem;
    st->ring_in_smem = 0;
  }
  return CORTEX_OK;
}

int cortex_get_state(cortex_net* h, int32_t net_idx, float* v, float* i_syn, int32_t* refr) {
  if (!h || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_get_state: arguments");
  const NetDev& d = h->nets_h[net_idx];
  if (v) CUDA_TRY(cudaMemcpyAsync(v, h->V + d.neuron_base, 4ull * d.n, cudaMemcpyDeviceToHost, h->stream));
  if (i_syn) CUDA_TRY(cudaMemcpyAsync(i_syn, h->I + d.neuron_base, 4ull * d.n, cudaMemcpyDeviceToHost, h->stream));
  if (refr) CUDA_TRY(cudaMemcpyAsync(refr, h->R + d.neuron_base, 4ull * d.n, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CORTEX_OK;
}

int cortex_get_ring(cortex_net* h, int32_t net_idx, float* ring) {
  if (!h || !ring || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_get_ring: arguments");
  if (h->delivery == CORTEX_DELIVERY_DELAY)
    return fail(CORTEX_ERR_UNSUPPORTED, "cortex_get_ring: delay-ordered delivery keeps a spike buffer, not a ring");
  const NetDev& d = h->nets_h[net_idx];
  // each block holds [D][T_b] floats of its targets; the host array is [D][n]
  for (int g = 0; g < d.n_blocks; ++g) {
    const BlockWork& w = h->work_h[d.first_block + g];
    CUDA_TRY(cudaMemcpy2DAsync(ring + w.t0, 4 * (size_t)d.n, h->ring + w.ring_base, 4 * (size_t)w.nt,
                               4 * (size_t)w.nt, (size_t)d.depth, cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CORTEX_OK;
}

int cortex_get_stamps(cortex_net* h, int32_t net_idx, uint32_t* stamps) {
  if (!h || !stamps || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_get_stamps: arguments");
  if (!h->stamps) return fail(CORTEX_ERR_ARG, "cortex_get_stamps: the handle was built without check_ownership");
  const NetDev& d = h->nets_h[net_idx];
  for (int g = 0; g < d.n_blocks; ++g) {
    const BlockWork& w = h->work_h[d.first_block + g];
    CUDA_TRY(cudaMemcpy2DAsync(stamps + w.t0, 4 * (size_t)d.n, h->stamps + w.ring_base, 4 * (size_t)w.nt,
                               4 * (size_t)w.nt, (size_t)d.depth, cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CORTEX_OK;
}

int cortex_check_stamps(int32_t n, int32_t depth, int32_t targets_per_block, int32_t warps, int32_t first_block,
                        const uint32_t* stamps, int64_t* n_bad, int64_t* first_bad) {
  if (n <= 0 || depth <= 0 || targets_per_block <= 0 || warps <= 0 || warps > kMaxWarps || first_block < 0 ||
      !stamps || !n_bad || !first_bad)
    return fail(CORTEX_ERR_ARG, "cortex_check_stamps: arguments");
  const int64_t tw = ceil_div(targets_per_block, warps);
  int64_t bad = 0, first = -1;
  for (int64_t s = 0; s < depth; ++s)
    for (int64_t i = 0; i < n; ++i) {
      const uint32_t st = stamps[s * n + i];
      if (st == 0) continue;
      const int64_t g = i / targets_per_block, local = i - g * targets_per_block;
      const uint32_t owner = (uint32_t)((first_block + g) * kMaxWarps + local / tw) + 1u;
      if (st != owner) {
        if (first < 0) first = s * n + i;
        ++bad;
      }
    }
  *n_bad = bad;
  *first_bad = first;
  return CORTEX_OK;
}

int cortex_set_state(cortex_net* h, int32_t net_idx, const float* v, const float* i_syn, const int32_t* refr,
                     const float* ring) {
  if (!h || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_set_state: arguments");
  if (h->delivery == CORTEX_DELIVERY_DELAY)
    return fail(CORTEX_ERR_UNSUPPORTED, "cortex_set_state: delay-ordered delivery keeps a spike buffer, not a ring");
  if (h->timed_out) return fail(CORTEX_ERR_TIMEOUT, "cortex_set_state: an earlier device wait timed out; free the handle");
  const NetDev& d = h->nets_h[net_idx];
  if (refr)
    for (int32_t i = 0; i < d.n; ++i)
      if (refr[i] < 0 || refr[i] > d.n_ref) return fail(CORTEX_ERR_ARG, "cortex_set_state: refractory count outside 0..n_ref");
  if (ring && h->exact) {
    // order-free adds stay exact only from cells that are themselves integer multiples of
    // 2^e_min with room below 2^24 * 2^e_min for a full cell's adds; otherwise the handle
    // returns to the ordered fold (same results, whatever the restored values)
    bool ok = true;
    for (int64_t q = 0; q < (int64_t)d.depth * d.n && ok; ++q) {
      const double x = std::ldexp((double)ring[q], -h->e_min);
      ok = std::isfinite(x) && x == std::nearbyint(x) && std::fabs(x) + h->exact_bound <= 16777216.0;
    }
    if (!ok) {
      h->exact = false;
      if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
      }
      if (h->delivery == CORTEX_DELIVERY_RING) {
        const int rc = relayout_for_fold(h);
        if (rc != CORTEX_OK) {
          h->no_layout = true;  // the order-free layout holds no tags for the ordered fold
          return rc;
        }
      }
    }
  }
  if (v) CUDA_TRY(cudaMemcpyAsync(h->V + d.neuron_base, v, 4ull * d.n, cudaMemcpyHostToDevice, h->stream));
  if (i_syn) CUDA_TRY(cudaMemcpyAsync(h->I + d.neuron_base, i_syn, 4ull * d.n, cudaMemcpyHostToDevice, h->stream));
  if (refr) CUDA_TRY(cudaMemcpyAsync(h->R + d.neuron_base, refr, 4ull * d.n, cudaMemcpyHostToDevice, h->stream));
  if (ring)
    for (int g = 0; g < d.n_blocks; ++g) {
      const BlockWork& w = h->work_h[d.first_block + g];
      CUDA_TRY(cudaMemcpy2DAsync(h->ring + w.ring_base, 4 * (size_t)w.nt, ring + w.t0, 4 * (size_t)d.n,
                                 4 * (size_t)w.nt, (size_t)d.depth, cudaMemcpyHostToDevice, h->stream));
    }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return CORTEX_OK;
}

int cortex_set_step(cortex_net* h, int64_t step) {
  if (!h || step < 0) return fail(CORTEX_ERR_ARG, "cortex_set_step: arguments");
  if (h->delivery == CORTEX_DELIVERY_DELAY)
    return fail(CORTEX_ERR_UNSUPPORTED, "cortex_set_step: delay-ordered delivery keeps a spike buffer, not a ring");
  if (h->timed_out) return fail(CORTEX_ERR_TIMEOUT, "cortex_set_step: an earlier device wait timed out; free the handle");
  const long long st = (long long)step;
  CUDA_TRY(cudaMemcpyAsync(h->step_counter, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->step = step;
  return CORTEX_OK;
}

int cortex_constants(cortex_net* h, int32_t net_idx, float* out6, uint32_t* thr, int32_t* n_thr, int32_t* n_ref) {
  if (!h || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_constants: arguments");
  const NetDev& d = h->nets_h[net_idx];
  if (out6) {
    out6[0] = d.p11;
    out6[1] = d.p21;
    out6[2] = d.p22m1;
    out6[3] = d.w_exc;
    out6[4] = d.w_inh;
    out6[5] = d.j_ext;
  }
  if (thr)
    for (int k = 0; k < d.n_thr; ++k) thr[k] = d.thr[k];
  if (n_thr) *n_thr = d.n_thr;
  if (n_ref) *n_ref = d.n_ref;
  return CORTEX_OK;
}

int cortex_export_synapses(cortex_net* h, int32_t net_idx, int32_t t_begin, int32_t t_end, int64_t* n_inout,
                           int32_t* src, int32_t* tgt, int32_t* delay, float* weight) {
  if (!h || !n_inout || net_idx < 0 || net_idx >= h->n_nets) return fail(CORTEX_ERR_ARG, "cortex_export_synapses: arguments");
  const NetDev& d = h->nets_h[net_idx];
  if (t_begin < 0 || t_end > d.n || t_begin > t_end) return fail(CORTEX_ERR_ARG, "cortex_export_synapses: target range");
  const int64_t need = (int64_t)(t_end - t_begin) * d.k;
  if (*n_inout < need) {
    *n_inout = need;
    return fail(CORTEX_ERR_OVERFLOW, "cortex_export_synapses: capacity too small");
  }
  *n_inout = need;
  if (need == 0) return CORTEX_OK;
  int32_t *ds = nullptr, *dt = nullptr, *dd = nullptr;
  float* dw = nullptr;
  unsigned long long* cnt = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&ds, 4 * need, h->stream));
  CUDA_TRY(cudaMallocAsync((void**)&dt, 4 * need, h->stream));
  CUDA_TRY(cudaMallocAsync((void**)&dd, 4 * need, h->stream));
  CUDA_TRY(cudaMallocAsync((void**)&dw, 4 * need, h->stream));
  CUDA_TRY(cudaMallocAsync((void**)&cnt, 8, h->stream));
  CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, h->stream));
  for (int g = 0; g < d.n_blocks; ++g) {
    const BlockWork& w = h->work_h[d.first_block + g];
    if (w.t0 + w.nt <= t_begin || w.t0 >= t_end) continue;
    CUDA_TRY(launch_export(h->nets_d, h->work_d, d.first_block + g, h->n_warps, h->rec_w, d.wdtype, h->rec_meta,
                           h->hdr, h->row_base, d.n, t_begin, t_end, cnt, ds, dt, dd, dw, need, h->stream));
  }
  unsigned long long got = 0;
  std::vector<int32_t> hs(need), ht(need), hd(need);
  std::vector<float> hw(need);
  CUDA_TRY(cudaMemcpyAsync(&got, cnt, 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(hs.data(), ds, 4 * need, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(ht.data(), dt, 4 * need, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(hd.data(), dd, 4 * need, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaMemcpyAsync(hw.data(), dw, 4 * need, cudaMemcpyDeviceToHost, h->stream));
  cudaFreeAsync(ds, h->stream);
  cudaFreeAsync(dt, h->stream);
  cudaFreeAsync(dd, h->stream);
  cudaFreeAsync(dw, h->stream);
  cudaFreeAsync(cnt, h->stream);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if ((int64_t)got != need) return fail(CORTEX_ERR_CUDA, "cortex_export_synapses: synapse count mismatch");
  // canonical order: (target, source, delay)
  std::vector<int64_t> idx(need);
  for (int64_t q = 0; q < need; ++q) idx[q] = q;
  std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
    if (ht[x] != ht[y]) return ht[x] < ht[y];
    if (hs[x] != hs[y]) return hs[x] < hs[y];
    return hd[x] < hd[y];
  });
  for (int64_t q = 0; q < need; ++q) {
    if (src) src[q] = hs[idx[q]];
    if (tgt) tgt[q] = ht[idx[q]];
    if (delay) delay[q] = hd[idx[q]];
    if (weight) weight[q] = hw[idx[q]];
  }
  return CORTEX_OK;
}

int cortex_deliver(cortex_net* h, int32_t net_idx, const int32_t* ids, int64_t n, int64_t t_emit, int32_t reps,
                   double* ms_out, int64_t* events_out) {
  if (!h || net_idx < 0 || net_idx >= h->n_nets || n < 0 || (n > 0 && !ids) || t_emit < 0 || reps < 1)
    return fail(CORTEX_ERR_ARG, "cortex_deliver: arguments");
  if (h->delivery == CORTEX_DELIVERY_DELAY)
    return fail(CORTEX_ERR_UNSUPPORTED, "cortex_deliver: measures the ring delivery only");
  if (h->no_layout)
    return fail(CORTEX_ERR_UNSUPPORTED, "cortex_deliver: the restored ring needs the ordered fold, whose layout does not fit");
  const NetDev& d = h->nets_h[net_idx];
  std::vector<int32_t> v(ids, ids + n);
  for (int32_t x : v)
    if (x < 0 || x >= d.n) return fail(CORTEX_ERR_ARG, "cortex_deliver: neuron id out of range");
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  // publication slots (parity 0, window step 0): ids of each block's range, counts per block
  std::vector<uint32_t> cnt(h->n_blocks, 0);
  const int32_t tb = h->work_h[d.first_block].nt;
  std::vector<uint32_t> slots(d.n, 0);
  for (int32_t x : v) {
    const int g = x / tb;
    slots[(int64_t)g * tb + cnt[d.first_block + g]] = (uint32_t)x;
    cnt[d.first_block + g] += 1;
  }
  CUDA_TRY(cudaMemcpyAsync(h->pub_cnt, cnt.data(), 4 * h->n_blocks, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->pub_ids + d.neuron_base, slots.data(), 4ull * d.n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemsetAsync(h->err, 0, 4, h->stream));
  unsigned long long e0 = 0, e1 = 0;
  CUDA_TRY(cudaMemcpyAsync(&e0, h->events + net_idx, 8, cudaMemcpyDeviceToHost, h->stream));
  StepArgs a = make_args(h);
  a.n_steps = 1;
  a.phases = kPhaseDeliver;
  a.ring_smem = h->ring_smem ? 1 : 0;
  a.raster_step = nullptr;
  a.raster_id = nullptr;
  a.t_fixed = t_emit;
  CUDA_TRY(cudaEventRecord(h->ev0, h->stream));
  for (int r = 0; r < reps; ++r) CUDA_TRY(launch_step(a, h->n_blocks, h->threads, h->smem, false, h->stream, &h->apw));
  CUDA_TRY(cudaEventRecord(h->ev1, h->stream));
  CUDA_TRY(cudaMemcpyAsync(&e1, h->events + net_idx, 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  if (ms_out) *ms_out = ms / reps;
  if (events_out) *events_out = (int64_t)((e1 - e0) / (unsigned long long)reps);
  return check_err(h, "deliver");
}

int cortex_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(CORTEX_ERR_ARG, "cortex_philox: arguments");
  if (n == 0) return CORTEX_OK;
  uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
  CUDA_TRY(cudaMalloc(&dc, 16 * n));
  CUDA_TRY(cudaMalloc(&dk, 8 * n));
  CUDA_TRY(cudaMalloc(&dout, 16 * n));
  CUDA_TRY(cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice));
  CUDA_TRY(launch_philox(dc, dk, n, dout, nullptr));
  CUDA_TRY(cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost));
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return CORTEX_OK;
}

}  // extern "C"
