// cortex_internal.cuh -- device-side data layout and helpers shared by the library's kernels.
//
// Layout in HBM (one handle, possibly many networks):
//   records   two streams, one entry per synapse: w (f32 or bf16) and meta (u16) =
//             (target index relative to its delivery warp << dbits) | (delay - d_min).  Sorted by
//             (source, block, target, draw): the CSR by source of the whole network, in which the
//             synapses of one source are grouped by owning block and, inside a block, by target --
//             so each delivery warp's target sub-range is a contiguous piece of its block's piece.
//             All blocks read adjacent pieces of one spiking source's row (shared pages and rows).
//   row_base  u64 per source: first record of the source's row, relative to the network's base.
//   headers   one 32-byte header per (source, block), stored source-major: word 0 = first record of
//             the block's piece relative to the row (low 16 bits; the high half is reserved), then
//             sixteen 12-bit fields end[w] for the delivery warps w = 0..15 (entries of warps
//             0..w; the fields of absent warps repeat the total) -- see hdr_end.
//   state     V (f32), I (f32), refractory counter (i32) per neuron.
//   ring      per block [D][T_b] floats, D = d_max + 1: cell (slot, j) holds the input due at the
//             step t with t mod D == slot for local target j.
//   pub       spike lists published per window: ids[(parity*W_max + ws) * n_total + pub_base + k],
//             counts[(parity*W_max + ws) * n_blocks + block] (read by split launches, and by the
//             persistent kernel only beyond a mailbox line's capacity);
//             mailbox[parity][block][16] u64 words = (window tag << 48) | payload;
//             windows[block] = windows completed (kept across launches).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace cortex {

constexpr int kPoissonCap = 64;     // Poisson threshold table entries
constexpr int kMaxWarps = 16;       // warps per block, all of them delivery warps (one 12-bit end each in the header)
constexpr int kNarrowWarps = 14;    // blocks of up to this many warps run a kernel built for them
                                     // (448 threads: up to 146 registers a thread instead of 128)
constexpr uint32_t kMaxPiece = 4095;  // entries of one (source, block) piece: the ends are 12-bit fields

// The 32-byte header of a (source, block) piece, as eight 32-bit words: bits 0-15 of word 0 are
// the piece's offset in the source's row; from bit 32 on, sixteen 12-bit fields hold end[w], the
// end (exclusive, in entries from the piece start) of delivery warp w's sub-range; the fields of
// warps the block does not have hold the piece length, so end[kMaxWarps - 1] is the length.
__host__ __device__ inline uint32_t hdr_end(const uint32_t* words, int w) {
  const int p = 32 + 12 * w, i = p >> 5, s = p & 31;  // i + 1 <= 7 for w < 16
  const unsigned long long x = ((unsigned long long)words[i + 1] << 32) | words[i];
  return (uint32_t)(x >> s) & 0xfffu;
}
constexpr int kSpikeBatch = 32;     // spikes staged per delivery round (at most)
constexpr int kStages = 4;          // delivery rounds in flight per block
constexpr int kHdrSlots = 4;       // rounds of fetched piece headers held in shared memory (two pairs)
constexpr int kIdCap = 2048;        // spike ids of a window kept in shared memory
constexpr int kMboxWords = 16;      // 64-bit words of a block's mailbox line (128 bytes)
constexpr int kInlMax = 3 * (kMboxWords - 1);  // spike ids a mailbox line carries (one count word)

// delay-ordered delivery: (emission step, block) spike counts and spike ids a block keeps in shared
// memory while it folds a window
constexpr int kDCntCap = 6400;
constexpr int kDIdCap = 4096;
constexpr int kDMaxWarps = 32;      // warps per block of the delay-ordered kernel

constexpr uint32_t kStreamConn = 1u;
constexpr uint32_t kStreamV0 = 2u;
constexpr uint32_t kStreamPoisson = 3u;

// device error word values
constexpr int kErrTimeout = 1;
constexpr int kErrRaster = 2;
constexpr int kErrSegment = 4;
constexpr int kErrBuild = 8;

struct NetDev {
  int32_t n, n_exc, n_inh, k_exc, k_inh, k;
  int32_t d_min, d_max, depth, window;        // depth D = d_max + 1, window W = d_min + 1
  int32_t dbits;                               // bits of (delay - d_min) in a record's meta
  uint32_t seed_lo, seed_hi;
  int32_t wdtype;                              // 0 f32, 1 bf16
  int32_t first_block, n_blocks;               // blocks of this network in the work table
  int32_t n_ref, n_thr;
  float p11, p21, p22m1;                       // FP32 propagators (from FP64 on the device); P22 - 1
  float v_th, v_reset, j_ext;
  float w_exc, w_inh;                          // stored weights (bf16-rounded when wdtype = 1)
  int32_t batch, cap_w, cap_m;                 // spikes per delivery round, staging bytes per spike
  int32_t stage_bytes;                         // staging area of a block (shared-memory layout)
  // host-provided inputs for the propagator kernel
  float tau_m, c_m, tau_syn, t_ref, dt, nu_ext_hz, j_exc_in, j_inh_in;
  int64_t neuron_base;                         // offset of this network in V / I / R
  int64_t rec_base;                            // first record of this network
  int64_t hdr_base;                            // first header of this network (source-major)
  int64_t row_off;                             // offset of this network in row_base
  int64_t raster_base, raster_cap;             // offset and capacity in the raster arrays
  // delay-ordered delivery (records sorted by source, delay, block, target, draw)
  int64_t tbl_base;                            // first table word of this network
  int32_t tbl_stride;                          // table words per source: (n_delays + 1) * n_blocks
  int32_t hist_depth;                          // steps of spike history kept: d_max + window + 1
  uint32_t thr[kPoissonCap];
};

struct BlockWork {
  int32_t net;        // network index
  int32_t group;      // block index within the network
  int32_t t0;         // first target (network-local id)
  int32_t nt;         // targets owned (T_b)
  int32_t tw;         // targets per warp (T_w)
  int32_t n_src;      // sources of the network (headers per block)
  int64_t rec_base;   // first record of the block
  int64_t hdr_base;   // first header of the block (in headers)
  int64_t ring_base;  // first ring cell of the block (floats): D * T_b cells
  int64_t pub_base;   // first publication slot of the block
};

struct StepArgs {
  const NetDev* nets;
  const BlockWork* work;
  int32_t n_blocks;
  int32_t w_max;                  // largest window over the networks
  int64_t n_total;                // neurons over all networks (publication stride)
  const void* rec_w;
  const uint16_t* rec_meta;
  const uint4* hdr;               // 2 x uint4 per header
  const unsigned long long* row_base;
  float* V;
  float* I;
  int32_t* R;
  float* ring;
  uint32_t* pub_ids;
  uint32_t* pub_cnt;
  unsigned long long* pub_flag;   // per block: windows completed (kept across launches)
  unsigned long long* mbox;       // [2][n_blocks][kMboxWords] self-tagged mailbox lines
  int32_t* raster_step;
  int32_t* raster_id;
  unsigned long long* raster_count;   // per network: spikes emitted so far
  unsigned long long* events;         // per network: synaptic events so far
  int32_t* err;
  long long* step_counter;            // current step (device resident, graph friendly)
  int32_t n_steps;                    // steps this launch
  int32_t phases;                     // kPhaseUpdate | kPhaseDeliver
  int32_t ring_smem;                  // 1: ring slice in shared memory
  int32_t bf16;                       // 1: weights stored as bf16 (all networks of a handle)
  int32_t ring_red;                   // 1: adds into a global ring use the L2 reduction unit
  int32_t exact;                      // 1: every partial sum of a ring cell is exact (order-free adds)
  int32_t helper_warp;                // 1: the block's last warp builds descriptors, does not fold
  long long timeout_ns;
  int32_t withhold_block;             // test hook: this block never publishes (-1: none)
  // delivery-only launches (cortex_deliver): fixed emission step
  long long t_fixed;
  // delay-ordered delivery
  const uint16_t* dtgt;               // block-local target of every record (delay-ordered rows)
  const void* dw;                     // weight of every record (f32), or the packed record (bf16: target | w << 16)
  const uint16_t* dtbl;               // per source and block: offsets in the row of the delay pieces
  uint32_t* hist_ids;                 // [hist slot][n_total]: ids a block emitted at a step
  uint32_t* hist_cnt;                 // [hist slot][n_blocks]: how many
  int32_t hist_max;                   // slots of the history arrays (largest hist_depth)
  unsigned long long* bar_count;      // per network: window arrivals of its blocks (monotonic)
  // ownership check (debug): per ring cell the id of the warp that wrote it; violations
  uint32_t* stamps;
  unsigned long long* viol;           // [0] cells written by a second warp, [1] first such cell + 1
};

constexpr int kPhaseUpdate = 1;
constexpr int kPhaseDeliver = 2;
constexpr int kPhaseBarrier = 4;    // persistent: grid barrier between the phases

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 products with
// the round multipliers, the high words xor-ed with the other counter words and the round key,
// the key advanced by the Weyl constants after each round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = c.x, b = c.z;
    const uint32_t lo0 = 0xD2511F53u * a, hi0 = __umulhi(0xD2511F53u, a);
    const uint32_t lo1 = 0xCD9E8D57u * b, hi1 = __umulhi(0xCD9E8D57u, b);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// floor(u * n / 2^32): maps a uniform 32-bit word onto 0..n-1
__device__ __forceinline__ uint32_t scale32(uint32_t u, uint32_t n) { return __umulhi(u, n); }

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// bring [p, p + bytes) into L2 (p and bytes multiples of 16), no completion tracking
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// position of the n-th (0-based) set bit of m; m has more than n set bits
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const int c = __popc(m & ((1u << s) - 1u));
    if (n >= c) {
      n -= c;
      m >>= s;
      pos += s;
    }
  }
  return pos;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- asynchronous copies global -> shared ------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy global -> shared (L2 only), tracked per thread
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// 8-byte asynchronous copy global -> shared (through L1), tracked per thread
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace cortex

// host launch wrappers (defined in build.cu and step.cu)
namespace cortex {
// sets the calling thread's cortex_last_error() text and returns code (api.cu)
int record_error(int code, const char* msg);
cudaError_t launch_props(NetDev* nets, int n_nets, cudaStream_t s);
cudaError_t launch_build_count_net(const NetDev* nets_dev, int net_idx, int32_t n, int first_group, int n_groups,
                                   int32_t tb, uint32_t* cnt, cudaStream_t s);
cudaError_t launch_scan_groups(uint32_t* cnt, uint32_t* cursor, int n_groups, int32_t n_src, uint32_t* tmp,
                               cudaStream_t s);
cudaError_t launch_build_rows(const uint32_t* cnt_all, int nb, int32_t n, uint32_t* off_all, uint32_t* rowcnt,
                              unsigned long long* row_base, cudaStream_t s);
cudaError_t launch_build_fill_net(const NetDev* nets_dev, int net_idx, int32_t n, int first_group, int n_groups,
                                  int32_t tb, uint32_t* cursor, uint32_t* keys, cudaStream_t s);
cudaError_t launch_build_finalize_net(const NetDev* nets_dev, const BlockWork* work_dev, int net_idx, int first_group,
                                      int n_groups, int n_warps_blk, const uint32_t* cnt, const uint32_t* seg_end,
                                      const uint32_t* keys, const uint32_t* off_all,
                                      const unsigned long long* row_base, void* rec_w, uint16_t* rec_meta,
                                      uint4* hdr, int32_t* err, uint32_t* max_seg, cudaStream_t s);
cudaError_t launch_init_state(const NetDev* net_host, const NetDev* net_dev, int net_idx, float* V, float* I,
                              int32_t* R, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, cudaStream_t s);
cudaError_t launch_delay_layout(const NetDev* nets_dev, const NetDev* net_host, const BlockWork* work_dev, int net_idx,
                                int n_dw, const uint4* hdr, const unsigned long long* row_base, const void* rec_w,
                                const uint16_t* rec_meta, uint16_t* dtbl, uint16_t* dtgt, void* dw, int32_t* err,
                                cudaStream_t s);
cudaError_t launch_dstep(const StepArgs& a, int grid, int threads, size_t smem, cudaStream_t s);
size_t dstep_smem_bytes(int nt, int window, int nb, int d_max, int n_warps, bool exact);
cudaError_t dstep_kernel_attributes(size_t smem);
int dstep_occupancy(int threads, size_t smem);
// apw: optional access-policy window of the launch (the ring kept resident in L2), NULL for none
cudaError_t launch_step(const StepArgs& a, int grid, int threads, size_t smem, bool cooperative, cudaStream_t s,
                        const cudaAccessPolicyWindow* apw = nullptr);
cudaError_t launch_advance_split(const StepArgs& a, int n_nets, int wn, cudaStream_t s);
// dynamic shared memory of a block of a network: nt targets per block (its largest block),
// ring depth, window steps, nb blocks, staging bytes
size_t step_smem_bytes(int nt, int depth, int window, int nb, bool ring_smem, int stage_bytes, int n_warps,
                       bool ordered);
void step_staging_caps(int max_seg_len, int wsz, int* cap_w, int* cap_m);
cudaError_t step_kernel_attributes(size_t smem);
int step_occupancy(int threads, size_t smem, bool ring_smem);

cudaError_t launch_export(const NetDev* nets_dev, const BlockWork* work_dev, int block, int n_dw, const void* rec_w,
                          int wdtype, const uint16_t* rec_meta, const uint4* hdr, const unsigned long long* row_base,
                          int32_t n_src, int32_t t_begin, int32_t t_end, unsigned long long* counter, int32_t* src,
                          int32_t* tgt, int32_t* dly, float* w, int64_t cap, cudaStream_t s);
}  // namespace cortex
