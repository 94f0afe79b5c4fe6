// step.cu -- the per-step hot path: neuron update, spike compaction, spike publication, grid
// barrier, and spike delivery over the indegree sub-graphs.
//
// Every block owns a contiguous range of post-synaptic neurons and all of their incoming synapses
// (Eq. 5, Eq. 9-10).  Inside the block every warp owns a contiguous sub-range of those neurons
// (Sec. III-B, "each synaptic interaction and its post-synaptic neuron should be accessed by a
// specific thread only").  A spike from source s is read as the block's (s) segment -- contiguous
// records sorted by target -- and each warp folds its own piece of it into the ring buffer of its
// neurons.  Different warps never touch the same ring cell; inside a warp, equal cells are added in
// lane order.  So every cell receives its weights in the order (emission step, source id, draw
// index) with no atomics and no locks (Eq. 12-14).
//
// One step (Sec. II-B, Eq. 1-3) has two halves.  The V half updates the membrane potential from
// V and I of the previous step, applies the refractory clamp and the threshold: it decides the
// step's spikes.  The I half decays I and adds the ring slot of the step and the Poisson drive.
// A spike emitted at step t arrives at slot t + d (d >= d_min) and so first changes I at t + d and
// a spike decision at t + d + 1.  The persistent kernel therefore runs windows of W = d_min + 1
// steps between grid barriers: inside a window every V half and every I half but the last only
// read slots that earlier windows completed, and the last step's I half waits until the window's
// spikes have been delivered (it runs at the start of the next window, or in the epilogue).  The
// blocks of a network meet at one barrier per window, publish the window's spikes and deliver
// them; the ring has D = d_max + 1 slots so that no delivery reaches the pending slot.  Launches
// without the barrier (split mode) run whole steps, at most d_min per window.
//
// Publication and barrier: each block writes one 128-byte mailbox line per window whose 64-bit
// words all carry the window's tag (step counts, then up to 45 spike ids), and bulk-prefetches
// into L2 the header rows of its first spiking neurons (with the ring in shared memory, their record
// rows too); reading every line of the network with the tag is the barrier.  Every thread first makes the next window's Poisson draws (they need nothing from the
// other blocks), then the threads of the polls read the lines.
//
// Delivery runs in rounds of up to kSpikeBatch spikes (per network: as many as its staging
// layout holds), taken in pairs behind one block barrier.  Headers (and row starts) are copied into
// shared memory a pair ahead of their use; one lane per spike turns them into a piece descriptor
// (global addresses and 16-byte chunk counts for the copy, spike-minor offsets and per-warp ends
// for the fold); all warps stage the records of the next pair with 16-byte cp.async copies (each
// spike has a fixed-size region of its slot), then fold the current pair while those land.
#include <type_traits>

#include "cortex_internal.cuh"
#include "step_common.cuh"

namespace cortex {

// delivery rounds whose descriptors are kept: the pair being folded, the pair being copied and the
// pair being described
constexpr uint32_t kDescSlots = 6;

struct SmemLayout {
  uint32_t ring, sv, si, sr, thr, cnt, woffs, wcnt, wlist, ids, mbl, mbi, mbc, pk, hdr, desc, dsoa, perm, tags, stage, total;
};

__host__ __device__ inline uint32_t align_to(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }


// ordered: the fold orders equal cells (duplicate-detection tags); the order-free fold has none
__host__ __device__ inline SmemLayout make_layout(int nt, int depth, int window, int nb, bool ring_smem,
                                                  int stage_bytes, int n_warps, bool ordered) {
  SmemLayout L;
  uint32_t o = 0;
  L.ring = o;
  o += ring_smem ? (uint32_t)(depth * nt * 4) : 0u;
  o = align_to(o, 16);
  L.sv = o;
  o += nt * 4;
  L.si = o;
  o += nt * 4;
  L.sr = o;    // refractory counters (32 bit; 16 bit when the ring is global, to leave room for staging)
  o += nt * (ring_smem ? 4 : 2);
  o = align_to(o, 16);
  L.thr = o;
  o += kPoissonCap * 4;
  L.cnt = o;
  o += (uint32_t)(window * (nb + 1) * 4);
  o = align_to(o, 16);
  L.woffs = o;
  o += (uint32_t)((window + 1) * 4);
  o = align_to(o, 16);
  L.wcnt = o;
  o += (kMaxWarps + 2) * 4;
  o = align_to(o, 16);
  L.wlist = o;  // per-warp spike lists of a step (local ids; 32 bit, 16 bit when the ring is global)
  o += nt * (ring_smem ? 4 : 2);
  o = align_to(o, 16);
  L.ids = o;
  o += kIdCap * 4;
  L.mbi = o;   // the block's first spike ids of the window (local, u16), for its mailbox line
  o += align_to(kInlMax * 2, 16);
  L.mbc = o;   // the block's spike count of every step of the window
  o += align_to((uint32_t)(window * 4), 16);
  L.pk = o;    // Poisson counts of the window's I halves, [step][target] (persistent kernel)
  o += align_to((uint32_t)(window * nt), 16);
  L.hdr = o;   // fetched headers: kHdrSlots rounds of (32-byte header, 8-byte row start, pad) per spike
  o += kHdrSlots * kSpikeBatch * 48;
  L.desc = o;  // piece descriptors, kDescSlots rounds: 32 bytes per spike (copy), then per round
  o += kDescSlots * kSpikeBatch * 32;  //   u32 aux[spike] and u16 end[warp][spike] (fold; from the 12-bit fields)
  L.dsoa = o;
  o += kDescSlots * kSpikeBatch * (4 + 2 * kMaxWarps);
  L.perm = o;  // per delivery warp, the compaction of the non-empty pieces of a round (two rounds)
  o += kMaxWarps * 64;
  o = align_to(o, 16);
  L.tags = o;
  o += !ordered ? 0u : ring_smem ? align_to((uint32_t)(depth * nt), 16) : (uint32_t)(n_warps * kTagHash);
  o = align_to(o, 128);
  L.mbl = o;   // mailbox lines read at the barrier: one per block of the network
  o += (uint32_t)(nb * kMboxWords * 8);
  o = align_to(o, 128);
  L.stage = o;
  o += (uint32_t)stage_bytes;
  L.total = o;
  return L;
}

// Fold N (1..4) consecutive chunks with one tag array, software-pipelined: chunk u + 1 writes its
// tags as soon as chunk u's tags have been read (its ballot has consumed them), so that the tag
// round trip of chunk u + 1 overlaps the ring updates of chunk u.  The __syncwarp that ends
// chunk u's updates also orders chunk u + 1's tag writes before its tag reads, and chunk u's ring
// updates before chunk u + 1's.
template <bool kRingSmem, int N>
__device__ __forceinline__ void fold_n(float* ring, uint8_t* wtags, const uint32_t* key, const float* w, int lane,
                                       bool red) {
  if constexpr (N == 1) {
    fold_one<kRingSmem>(ring, wtags, key[0], w[0], lane, red);
  } else {
    auto tag_of = [&](uint32_t k) -> uint8_t* {
      return kRingSmem ? wtags + (k != 0xffffffffu ? k : 0u) : wtags + (k & (uint32_t)(kTagHash - 1));
    };
    uint8_t* tg = tag_of(key[0]);
    if (key[0] != 0xffffffffu) *tg = (uint8_t)lane;
    __syncwarp();
    uint32_t t = key[0] != 0xffffffffu ? (uint32_t)*tg : (uint32_t)lane;
    uint32_t losers = __ballot_sync(0xffffffffu, key[0] != 0xffffffffu && t != (uint32_t)lane);
#pragma unroll
    for (int u = 0; u < N; ++u) {
      uint8_t* tgn = nullptr;
      if (u + 1 < N) {
        tgn = tag_of(key[u + 1]);
        if (key[u + 1] != 0xffffffffu) *tgn = (uint8_t)lane;
      }
      fold_apply<kRingSmem>(ring, key[u], w[u], t, losers, lane, red);  // ends with __syncwarp
      if (u + 1 < N) {
        t = key[u + 1] != 0xffffffffu ? (uint32_t)*tgn : (uint32_t)lane;
        losers = __ballot_sync(0xffffffffu, key[u + 1] != 0xffffffffu && t != (uint32_t)lane);
      }
    }
  }
}

// Ownership check (debug mode, Sec. IV-A "Verification": a synaptic interaction or post-synaptic
// neuron touched by two threads is an error).  Every ring cell a delivery warp writes is stamped
// with the warp's id (block * 16 + warp + 1) in a global array laid out like the global ring; a cell
// found stamped by another warp is counted (viol[0]) and the first one recorded (viol[1] = cell + 1).
// Nothing traps: the host reads the counters after the launch.  Out of line: debug mode only, and
// the fold it sits in is inlined for every chunk of every group size.
__device__ __noinline__ void stamp_cell(const StepArgs& a, int64_t ring_base, uint32_t key, uint32_t writer) {
  if (key == 0xffffffffu) return;
  const int64_t cell = ring_base + key;
  const uint32_t old = atomicCAS(a.stamps + cell, 0u, writer);
  if (old != 0u && old != writer) {
    atomicAdd(a.viol, 1ull);
    atomicCAS(a.viol + 1, 0ull, (unsigned long long)cell + 1ull);
  }
}

// ---- the step kernel ---------------------------------------------------------------------------
// phases: kPhaseUpdate, kPhaseDeliver, and kPhaseBarrier for the persistent form (both phases and
// a barrier per window inside one cooperative launch of n_steps steps).  kRingSmem: the block's
// ring slice lives in shared memory for the whole launch (loaded in the prologue, written back
// in the epilogue); otherwise it is updated in place in global memory.  kExact: the adds of the
// delivery need no order (ring_add_exact), so the fold skips the sharing test.
template <bool kRingSmem, bool kBf16, bool kWide, bool kExact>
__global__ void __launch_bounds__((kWide ? kMaxWarps : kNarrowWarps) * 32, 1) k_step(const StepArgs a) {
  constexpr uint32_t kWsz = kBf16 ? 2u : 4u;  // bytes per stored weight
  // neuron chunks per update iteration: a global ring is read from L2, so several reads are kept
  // in flight (8: one L2 round trip per step for about 250 targets per warp; measured 1% faster than
  // 4 on the 500,000- and 1e6-neuron networks); a shared ring is read with low latency and small
  // per-warp ranges favour one
  constexpr int kUpd = kRingSmem ? 1 : 8;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
  // delivery warps own the target sub-ranges of the layout; with a helper warp (the last one), that
  // warp fetches the piece headers and builds the descriptors while the others fold
  const int n_fold = n_warps - (a.helper_warp ? 1 : 0);
  const int desc_tid = a.helper_warp ? tid - 32 * n_fold : tid;  // 0..31: the threads that do that work
  const int blk = blockIdx.x;
  const BlockWork wk = a.work[blk];
  const NetDev& ndg = a.nets[wk.net];
  NeuronConst nd;
  nd.p11 = ndg.p11;
  nd.p21 = ndg.p21;
  nd.p22m1 = ndg.p22m1;
  nd.v_th = ndg.v_th;
  nd.v_reset = ndg.v_reset;
  nd.j_ext = ndg.j_ext;
  nd.n_ref = ndg.n_ref;
  nd.n_thr = ndg.n_thr;
  const uint32_t seed_lo = ndg.seed_lo, seed_hi = ndg.seed_hi;
  const int nb = ndg.n_blocks, first_block = ndg.first_block, window = ndg.window;
  const int d_min = ndg.d_min, dbits = ndg.dbits;
  const uint32_t dmask = (1u << dbits) - 1u;
  const int64_t neuron_base = ndg.neuron_base, raster_base = ndg.raster_base, raster_cap = ndg.raster_cap;
  const int64_t rec_net = ndg.rec_base, hdr_net = ndg.hdr_base, row_off = ndg.row_off;
  const int D = ndg.depth;
  const int nt = wk.nt, tw = wk.tw;
  const int tb_full = a.work[first_block].nt;  // targets of the network's full blocks
  const bool persistent = (a.phases & kPhaseBarrier) != 0;
  const bool ring_red = a.ring_red != 0;
  const bool do_update = (a.phases & kPhaseUpdate) != 0;
  const bool do_deliver = (a.phases & kPhaseDeliver) != 0;
  // round size and staging bytes per spike of this block's network (its longest piece sets them)
  const uint32_t B = (uint32_t)ndg.batch, cap_w = (uint32_t)ndg.cap_w, cap = (uint32_t)(ndg.cap_w + ndg.cap_m);

  // the network's own layout (its blocks' targets, depth, window and block count)
  const SmemLayout L = make_layout(tb_full, D, window, nb, kRingSmem, ndg.stage_bytes, n_fold, !kExact);
  float* ring_s = reinterpret_cast<float*>(smem + L.ring);
  float* sV = reinterpret_cast<float*>(smem + L.sv);
  float* sI = reinterpret_cast<float*>(smem + L.si);
  using RefT = typename std::conditional<kRingSmem, int32_t, int16_t>::type;
  using ListT = typename std::conditional<kRingSmem, uint32_t, uint16_t>::type;
  RefT* sR = reinterpret_cast<RefT*>(smem + L.sr);
  uint32_t* thr = reinterpret_cast<uint32_t*>(smem + L.thr);
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + L.cnt);
  uint32_t* woffs = reinterpret_cast<uint32_t*>(smem + L.woffs);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + L.wcnt);
  ListT* wlist = reinterpret_cast<ListT*>(smem + L.wlist);
  uint32_t* ids_s = reinterpret_cast<uint32_t*>(smem + L.ids);
  unsigned long long* mbl = reinterpret_cast<unsigned long long*>(smem + L.mbl);
  uint16_t* mbi = reinterpret_cast<uint16_t*>(smem + L.mbi);
  uint32_t* mbc = reinterpret_cast<uint32_t*>(smem + L.mbc);
  uint8_t* pk = smem + L.pk;
  unsigned char* hdr_s = smem + L.hdr;
  uint4* desc_s = reinterpret_cast<uint4*>(smem + L.desc);
  unsigned char* dsoa_s = smem + L.dsoa;
  uint8_t* perm = smem + L.perm + warp * 64;
  uint8_t* tags = smem + L.tags;
  unsigned char* stage = smem + L.stage;

  float* ring_g = a.ring + wk.ring_base;
  float* ring = kRingSmem ? ring_s : ring_g;
  const int64_t nbase = neuron_base + wk.t0;

  // ---- prologue: state, thresholds, ring slice ----
  for (int q = tid; q < kPoissonCap; q += blockDim.x) thr[q] = ndg.thr[q];
  if (do_update) {
    for (int j = tid; j < nt; j += blockDim.x) {
      sV[j] = a.V[nbase + j];
      sI[j] = a.I[nbase + j];
      sR[j] = (RefT)a.R[nbase + j];
    }
  }
  if (kRingSmem) {
    for (int q = tid; q < D * nt; q += blockDim.x) ring_s[q] = ring_g[q];
  }
  const long long t_start = (a.t_fixed >= 0) ? a.t_fixed : *a.step_counter;
  uint32_t epoch = persistent ? (uint32_t)__ldcg(a.pub_flag + blk) : 0u;
  unsigned long long raster_total = a.raster_count[wk.net];
  unsigned long long my_events = 0;
  bool aborted = false;
  __syncthreads();

  // Poisson counts of steps tfirst .. tfirst + ns - 1 for every owned target.  One generator call
  // gives the drive of four consecutive neurons (network-local ids 4g .. 4g + 3) at one step; the
  // work items are (step, group of four) pairs q0, q0 + dq, ...
  const int pq_g0 = wk.t0 >> 2, pq_ng = ((wk.t0 + nt + 3) >> 2) - pq_g0;  // groups of four targets
  auto poisson_fill = [&](long long tfirst, int ns, int q0, int qend, int dq) {
    const int g0 = pq_g0, ng = pq_ng;
    const int tot = min(ns * ng, qend);
    for (int q = q0; q < tot; q += dq) {
      const int sidx = q / ng, g = g0 + (q - sidx * ng);
      const uint4 rr = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(tfirst + sidx), kStreamPoisson, 0u),
                                     seed_lo, seed_hi);
      const uint32_t wd[4] = {rr.x, rr.y, rr.z, rr.w};
      // the four inversions side by side: threshold k is read once for all words still above it
      int kk[4] = {0, 0, 0, 0};
      for (int k = 0; k < nd.n_thr - 1; ++k) {
        const uint32_t th = thr[k];
        bool any = false;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const bool up = kk[w] == k && wd[w] >= th;
          kk[w] += up ? 1 : 0;
          any = any || up;
        }
        if (!any) break;
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int j = 4 * g + w - wk.t0;
        if (j >= 0 && j < nt) pk[sidx * nt + j] = (uint8_t)kk[w];
      }
    }
  };
  const bool defer = persistent;  // V/I halves with the window's last I half after the barrier
  bool pend = false;               // the I half of the previous window's last step is due
  const int W = persistent ? window : min(window, a.n_steps);
  if (persistent && do_update) {
    // the first window's table: pk[s] holds step t_start - 1 + s (the I half run before V half s)
    poisson_fill(t_start - 1, min(W, a.n_steps), tid, 1 << 30, blockDim.x);
    __syncthreads();
  }
  const int tw_u = (nt + n_warps - 1) / n_warps;  // update split over the warps
  int done = 0;
  while (done < a.n_steps) {
    const int Wn = min(W, a.n_steps - done);
    const long long t0 = t_start + done;
    const int tm0 = (int)(t0 % D);  // ring slot of the window's first step
    const uint32_t par = persistent ? ((epoch + 1u) & 1u) : 0u;
    const int n_cw = (Wn + 2) / 3;                          // count words of a mailbox line
    const uint32_t inl = (uint32_t)(3 * (kMboxWords - n_cw));  // ids a mailbox line carries

    // ================= update + compaction + publication =================
    if (do_update) {
      uint32_t win_total = 0;  // spikes of the block so far in this window
      for (int ws = 0; ws < Wn; ++ws) {
        const long long t = t0 + ws;
        const int slot = (tm0 + ws) % D;
        const int pslot = (tm0 + ws + D - 1) % D;    // slot of step t - 1
        const bool prev = defer && (ws > 0 || pend);  // the I half of step t - 1 is still due
        float* rs = ring + (int64_t)(defer ? pslot : slot) * nt;
        const uint32_t tu = (uint32_t)(defer ? t - 1 : t);
        const int lo = warp * tw_u, hi = min(lo + tw_u, nt);
        uint32_t cw = 0;
        if constexpr (kUpd == 1) {
          for (int c = lo; c < hi; c += 32) {
            const int j = c + lane;
            bool spk = false;
            if (j < hi) {
              float v = sV[j], cur = sI[j];
              int32_t r = sR[j];
              if (defer) {
                if (prev) {
                  const float in = ring_read<kRingSmem>(rs + j);
                  rs[j] = 0.0f;
                  i_half_k(cur, in, pk[ws * nt + j], nd);
                }
                spk = v_half(v, cur, r, nd);
              } else {
                const float in = ring_read<kRingSmem>(rs + j);
                rs[j] = 0.0f;
                const uint32_t gi = (uint32_t)(wk.t0 + j);
                const uint4 rr = philox4x32_10(make_uint4(gi >> 2, tu, kStreamPoisson, 0u), seed_lo, seed_hi);
                spk = v_half(v, cur, r, nd);
                i_half(cur, in, philox_word(rr, gi & 3u), nd, thr);
              }
              sV[j] = v;
              sI[j] = cur;
              sR[j] = (RefT)r;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, spk);
            if (spk) wlist[lo + cw + __popc(bal & lanemask_lt())] = (ListT)j;
            cw += __popc(bal);
          }
        } else {
          for (int c = lo; c < hi; c += kUpd * 32) {
            // kUpd 32-neuron chunks: their loads are issued together, then updated, then compacted
            // in ascending order
            float v[kUpd], cur[kUpd], in[kUpd];
            int32_t r[kUpd];
            int kp[kUpd];
#pragma unroll
            for (int u = 0; u < kUpd; ++u) {
              const int j = c + 32 * u + lane;
              in[u] = 0.0f;
              kp[u] = 0;
              if (j < hi) {
                v[u] = sV[j];
                cur[u] = sI[j];
                r[u] = sR[j];
                if (!defer || prev) in[u] = ring_read<kRingSmem>(rs + j);
                if (defer && prev) kp[u] = pk[ws * nt + j];
              }
            }
            bool spk[kUpd];
#pragma unroll
            for (int u = 0; u < kUpd; ++u) {
              const int j = c + 32 * u + lane;
              spk[u] = false;
              if (j < hi) {
                if (defer) {
                  if (prev) {
                    rs[j] = 0.0f;
                    i_half_k(cur[u], in[u], kp[u], nd);
                  }
                  spk[u] = v_half(v[u], cur[u], r[u], nd);
                } else {
                  rs[j] = 0.0f;
                  const uint32_t gi = (uint32_t)(wk.t0 + j);
                  const uint4 rr = philox4x32_10(make_uint4(gi >> 2, tu, kStreamPoisson, 0u), seed_lo, seed_hi);
                  spk[u] = v_half(v[u], cur[u], r[u], nd);
                  i_half(cur[u], in[u], philox_word(rr, gi & 3u), nd, thr);
                }
                sV[j] = v[u];
                sI[j] = cur[u];
                sR[j] = (RefT)r[u];
              }
            }
#pragma unroll
            for (int u = 0; u < kUpd; ++u) {
              const uint32_t bal = __ballot_sync(0xffffffffu, spk[u]);
              if (spk[u]) wlist[lo + cw + __popc(bal & lanemask_lt())] = (ListT)(c + 32 * u + lane);
              cw += __popc(bal);
            }
          }
        }
        if (lane == 0) wcnt[warp] = cw;
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int q = 0; q < n_warps; ++q) {
          const uint32_t x = wcnt[q];
          if (q < warp) before += x;
          total += x;
        }
        uint32_t* dst = a.pub_ids + ((int64_t)(par * a.w_max + ws) * a.n_total + neuron_base + wk.t0);
        for (uint32_t q = lane; q < cw; q += 32) {
          const uint32_t id = (uint32_t)wk.t0 + wlist[lo + q];
          dst[before + q] = id;
          const uint32_t pw = win_total + before + q;
          if (persistent && pw < inl) mbi[pw] = (uint16_t)(id - (uint32_t)wk.t0);
        }
        if (tid == 0) {
          a.pub_cnt[(int64_t)(par * a.w_max + ws) * a.n_blocks + blk] = total;
          mbc[ws] = total;
        }
        win_total += total;
        __syncthreads();
      }
      pend = defer;
      if (persistent) {
        // Publication: the block's mailbox line for this window.  Every 64-bit word carries the
        // window's tag in its top 16 bits, so a reader that sees the tag in a word sees that word's
        // payload: count words (three u16 step counts each), then id words (three u16 local ids
        // each).  When the window's spikes overflow the line, the count words are release
        // stores: they order the global id lists (read by others only beyond the line's capacity)
        // before them.  Otherwise a reader needs nothing but the line, and every word is a
        // relaxed store (a release costs the block a fence on the barrier's critical path).  A
        // reader accepts a word only with the tag it waits for, and the line is rewritten (two
        // windows later) only after every block of the network has published the next window's
        // line, which a block does after its polls of this line have returned.
        const unsigned long long tag = (unsigned long long)(((epoch + 1u) & 0x7fffu) | 0x8000u) << 48;
        const uint32_t nin = min(win_total, inl);
        if (tid < kMboxWords && blk != a.withhold_block) {
          unsigned long long pay = 0;
          for (int f = 0; f < 3; ++f) {
            if (tid < n_cw) {
              const int ws = 3 * tid + f;
              if (ws < Wn) pay |= (unsigned long long)mbc[ws] << (16 * f);
            } else {
              const uint32_t pq = 3u * (uint32_t)(tid - n_cw) + (uint32_t)f;
              if (pq < nin) pay |= (unsigned long long)mbi[pq] << (16 * f);
            }
          }
          unsigned long long* dst = a.mbox + ((size_t)par * a.n_blocks + blk) * kMboxWords + tid;
          if (tid < n_cw && win_total > inl) st_release_u64(dst, tag | pay);  // after the global id lists
          else st_relaxed_u64(dst, tag | pay);
        }
        // L2 prefetch of the spiking rows (every block of the network reads them after the
        // barrier): the header row, and with the ring in shared memory the record rows of the
        // window's first spikes (with a ring in global memory, the burst of record rows evicted ring
        // lines from L2 and measured slower: 1e6 neurons 6%, 500,000 neurons 1.7%)
        const int pq = tid - (int)(blockDim.x - kInlMax);
        if (pq >= 0 && (uint32_t)pq < nin) {
          const uint32_t id = (uint32_t)wk.t0 + mbi[pq];
          prefetch_l2_bulk(a.hdr + 2 * (hdr_net + (int64_t)id * nb), (uint32_t)nb * 32u);
          if (kRingSmem && (int)id + 1 < ndg.n) {
            const unsigned long long r0 = (unsigned long long)rec_net + __ldg(a.row_base + row_off + id);
            const unsigned long long r1 = (unsigned long long)rec_net + __ldg(a.row_base + row_off + id + 1);
            const unsigned long long spans[2][2] = {{r0 * kWsz, r1 * kWsz}, {r0 * 2ull, r1 * 2ull}};
            const unsigned char* bases[2] = {reinterpret_cast<const unsigned char*>(a.rec_w),
                                             reinterpret_cast<const unsigned char*>(a.rec_meta)};
            for (int st = 0; st < 2; ++st) {
              unsigned long long b0 = spans[st][0] & ~15ull;
              const unsigned long long b1 = (spans[st][1] + 15ull) & ~15ull;
              while (b0 < b1) {
                const uint32_t len = (uint32_t)min(b1 - b0, 16384ull);
                prefetch_l2_bulk(bases[st] + b0, len);
                b0 += len;
              }
            }
          }
        }
      }
    }

    // ================= grid barrier among the blocks of this network =================
    // Each block of the network has published its line; reading every line with this window's
    // tag in every needed word is the barrier, and gives the counts and the first spike ids.
    if (persistent) {
      epoch += 1u;
      const unsigned long long want = (unsigned long long)((epoch & 0x7fffu) | 0x8000u);
      int fail = 0;
      auto poll = [&](const unsigned long long* p, unsigned long long w) -> unsigned long long {
        if ((w >> 48) == want) return w;
        const long long tb0 = global_ns();
        uint32_t spins = 0;
        do {
          if ((++spins & 255u) == 0 && (global_ns() - tb0 > a.timeout_ns || *(volatile int32_t*)a.err != 0)) {
            fail = 1;
            return 0ull;
          }
          w = ld_relaxed_u64(p);
        } while ((w >> 48) != want);
        return w;
      };
      // First the next window's Poisson table (its first entry is this window's last step, whose I
      // half runs after the delivery), by every thread: it needs nothing from the other blocks,
      // whose lines arrive meanwhile.  (Filling it in the warps that do not poll, alongside the
      // polls, left the warp holding both kinds of lanes on the critical path.)
      if (do_update) poisson_fill(t0 + Wn - 1, max(min(W, a.n_steps - done - Wn), 1), tid, 1 << 30, blockDim.x);
      for (int b = tid; b < nb && !fail; b += blockDim.x) {
        const unsigned long long* line = a.mbox + ((size_t)par * a.n_blocks + first_block + b) * kMboxWords;
        unsigned long long* ml = mbl + (size_t)b * kMboxWords;
        unsigned long long w[kMboxWords];
#pragma unroll
        for (int j = 0; j < kMboxWords; ++j)  // count words and the first id word, loads in flight together
          if (j <= n_cw) w[j] = ld_relaxed_u64(line + j);
        uint32_t tot = 0;
#pragma unroll
        for (int j = 0; j < kMboxWords; ++j) {
          if (j <= n_cw && !fail) {
            w[j] = poll(line + j, w[j]);
            ml[j] = w[j];
            if (j < n_cw)
              for (int f = 0; f < 3; ++f) {
                const int ws = 3 * j + f;
                if (ws < Wn) {
                  const uint32_t c = (uint32_t)(w[j] >> (16 * f)) & 0xffffu;
                  cnt_s[ws * nb + b] = c;
                  tot += c;
                }
              }
          }
        }
        const int n_idw = (int)((min(tot, inl) + 2u) / 3u);
        for (int j = n_cw + 1; j < n_cw + n_idw && !fail; ++j) ml[j] = poll(line + j, ld_relaxed_u64(line + j));
        if (tot > inl) __threadfence();  // the block's further ids are read from its global list
      }
      if (__syncthreads_or(fail)) {
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        aborted = true;
        break;
      }
    }

    // ================= delivery =================
    if (do_deliver) {
      // counts of every (window step, block) of this network, flat (step-major), turned in place
      // into exclusive prefixes: cnt_s[ws * nb + b] = window position of block b's first spike of
      // step ws; cnt_s[Wn * nb] = spikes of the window
      const int E = Wn * nb;
      if (!persistent)
        for (int q = tid; q < E; q += blockDim.x)
          cnt_s[q] = __ldcg(a.pub_cnt + (int64_t)(par * a.w_max + q / nb) * a.n_blocks + first_block + q % nb);
      __syncthreads();
      {
        const int per = (E + (int)blockDim.x - 1) / (int)blockDim.x;
        const int e0 = min(tid * per, E), e1 = min(e0 + per, E);
        uint32_t loc = 0;
        for (int e = e0; e < e1; ++e) loc += cnt_s[e];
        uint32_t x = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) wcnt[warp] = x;
        __syncthreads();
        if (warp == 0) {
          uint32_t v = (lane < n_warps) ? wcnt[lane] : 0u;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
          }
          if (lane < n_warps) wcnt[lane] = v;
        }
        __syncthreads();
        uint32_t run = (warp ? wcnt[warp - 1] : 0u) + x - loc;
        for (int e = e0; e < e1; ++e) {
          const uint32_t c = cnt_s[e];
          cnt_s[e] = run;
          run += c;
        }
        if (tid == 0) cnt_s[E] = wcnt[n_warps - 1];
        __syncthreads();
        for (int ws = tid; ws <= Wn; ws += blockDim.x) woffs[ws] = cnt_s[ws * nb];
        __syncthreads();
      }
      const uint32_t S_tot = woffs[Wn];
      if (persistent && S_tot > (uint32_t)kIdCap) {
        // ids beyond the shared list are read from the global lists: order them after the lines
        if (tid < nb) __threadfence();
        __syncthreads();
      }
      // spike ids of the window into shared memory (window order: step, then id); raster.  One
      // thread per (window step, block): the ids come from the block's mailbox line (persistent
      // kernel, first ids of its window) or from its global list.  The same thread starts the
      // header copy (32-byte header, 8-byte row start) of every spike of the first kStages rounds.
      const uint32_t B0 = B;
      for (int e = tid; e < E; e += blockDim.x) {
        const uint32_t o = cnt_s[e], c = cnt_s[e + 1] - o;
        if (c == 0) continue;
        const int ws = e / nb, b = e - ws * nb;
        const uint32_t* src = a.pub_ids + (int64_t)(par * a.w_max + ws) * a.n_total + neuron_base + (int64_t)b * tb_full;
        const bool mine = (b == wk.group) && a.raster_step != nullptr;
        uint32_t p0 = 0;  // position of the step's first id in block b's list for the window
        if (persistent)
          for (int w2 = 0; w2 < ws; ++w2) p0 += cnt_s[w2 * nb + b + 1] - cnt_s[w2 * nb + b];
        const unsigned long long* ml = mbl + (size_t)b * kMboxWords + n_cw;
        for (uint32_t q = 0; q < c; ++q) {
          const bool need = (o + q < (uint32_t)kIdCap) || mine;
          if (!need) break;
          const uint32_t pw = p0 + q;
          const uint32_t id = (persistent && pw < inl)
                                  ? (uint32_t)b * (uint32_t)tb_full + ((uint32_t)(ml[pw / 3u] >> (16u * (pw % 3u))) & 0xffffu)
                                  : __ldcg(src + q);
          if (o + q < (uint32_t)kIdCap) ids_s[o + q] = id;
          if (o + q < (uint32_t)kStages * B0) {
            const uint32_t x = (o + q) / B0, k = (o + q) - x * B0;
            unsigned char* h = hdr_s + ((x % kHdrSlots) * kSpikeBatch + k) * 48u;
            const uint4* hp = a.hdr + 2 * (hdr_net + (int64_t)id * nb + wk.group);
            cp_async16(h, hp);
            cp_async16(h + 16, hp + 1);
            cp_async8(h + 32, a.row_base + row_off + id);
          }
          if (mine) {
            const unsigned long long pos = raster_total + o + q;
            if ((long long)pos < raster_cap) {
              a.raster_step[raster_base + pos] = (int32_t)(t0 + ws);
              a.raster_id[raster_base + pos] = (int32_t)id;
            } else {
              atomicOr(a.err, kErrRaster);
            }
          }
        }
      }
      raster_total += S_tot;
      cp_async_commit();
      cp_async_wait<0>();  // the header copies of the first kStages rounds
      __syncthreads();

      const uint32_t R = (S_tot + B - 1) / B;  // delivery rounds of this window
      // spike id of window index g (shared list, or the published global lists beyond it)
      auto spike_id = [&](uint32_t g) -> uint32_t {
        if (g < (uint32_t)kIdCap) return ids_s[g];
        int lo2 = 0, hi2 = E;  // the last (step, block) whose first window position is <= g
        while (hi2 - lo2 > 1) {
          const int mid = (lo2 + hi2) >> 1;
          if (cnt_s[mid] <= g) lo2 = mid;
          else hi2 = mid;
        }
        const int ws = lo2 / nb, b = lo2 - ws * nb;
        return __ldcg(a.pub_ids + (int64_t)(par * a.w_max + ws) * a.n_total + neuron_base + (int64_t)b * tb_full +
                      (g - cnt_s[lo2]));
      };
      // header (32 B) and row start of the block's piece of spike g, fetched asynchronously into
      // the header slot of its round
      auto fetch_hdr = [&](uint32_t x, uint32_t k) {
        const uint32_t id = spike_id(x * B + k);
        unsigned char* h = hdr_s + ((x % kHdrSlots) * kSpikeBatch + k) * 48u;
        const uint4* hp = a.hdr + 2 * (hdr_net + (int64_t)id * nb + wk.group);
        cp_async16(h, hp);
        cp_async16(h + 16, hp + 1);
        cp_async8(h + 32, a.row_base + row_off + id);
      };
      // Descriptors of round x, built by the 32 lanes of one warp (lane k: spike k of the round).
      // For the copy: [0] 16-byte-aligned global addresses of the weight and meta pieces, [1].x
      // weight chunks | meta chunks << 16.  For the fold (read by lane k of a warp, so stored
      // spike-minor to keep the lanes on distinct banks): aux[k] = weight offset | meta offset << 8 |
      // emission slot << 16, and the header's end[w][k].
      auto desc_slot = [&](uint32_t x) { return desc_s + (x % kDescSlots) * (2 * kSpikeBatch); };
      auto aux_slot = [&](uint32_t x) {
        return reinterpret_cast<uint32_t*>(dsoa_s + (x % kDescSlots) * kSpikeBatch * (4 + 2 * kMaxWarps));
      };
      auto ends_slot = [&](uint32_t x) { return reinterpret_cast<uint16_t*>(aux_slot(x) + kSpikeBatch); };
      auto store_desc = [&](uint32_t x) {
        const uint32_t k = (uint32_t)lane, g = x * B + k;
        const bool valid = k < B && g < S_tot;
        uint32_t nw = 0, nm = 0;
        if (valid) {
          const unsigned char* h = hdr_s + ((x % kHdrSlots) * kSpikeBatch + k) * 48u;
          const uint4 h0 = *reinterpret_cast<const uint4*>(h), h1 = *reinterpret_cast<const uint4*>(h + 16);
          const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
          const unsigned long long row = *reinterpret_cast<const unsigned long long*>(h + 32);
          int ws = 0;
          while (ws + 1 < Wn && woffs[ws + 1] <= g) ++ws;
          const uint32_t len = hdr_end(hw, kMaxWarps - 1);
          const unsigned long long r0 = (unsigned long long)rec_net + row + (h0.x & 0xffffu);
          const unsigned long long wbyte = r0 * kWsz, mbyte = r0 * 2ull;
          const uint32_t wal = (uint32_t)(wbyte & 15u), mal = (uint32_t)(mbyte & 15u);
          nw = len ? (wal + len * kWsz + 15u) >> 4 : 0u;
          nm = len ? (mal + len * 2u + 15u) >> 4 : 0u;
          const unsigned long long gw = reinterpret_cast<unsigned long long>(a.rec_w) + (wbyte & ~15ull);
          const unsigned long long gm = reinterpret_cast<unsigned long long>(a.rec_meta) + (mbyte & ~15ull);
          desc_slot(x)[2 * k] = make_uint4((uint32_t)gw, (uint32_t)(gw >> 32), (uint32_t)gm, (uint32_t)(gm >> 32));
          aux_slot(x)[k] = wal | (mal << 8) | ((uint32_t)((tm0 + ws) % D) << 16);
          uint16_t* en = ends_slot(x) + k;
#pragma unroll
          for (int q = 0; q < kMaxWarps; ++q)
            if (q < n_fold) en[q * kSpikeBatch] = (uint16_t)hdr_end(hw, q);
        }
        if (valid) desc_slot(x)[2 * k + 1] = make_uint4(nw | (nm << 16), 0u, 0u, 0u);
      };
      // stage the records of round x: delivery warp w copies spikes w, w + n_fold, ...; lane c
      // copies the 16-byte chunk c of the weight piece followed by the meta piece
      auto issue_round = [&](uint32_t x) {
        if (x >= R || warp >= n_fold) return;
        const uint4* ds = desc_slot(x);
        const uint32_t n = min(B, S_tot - x * B);
        unsigned char* sb = stage + (x % kStages) * (B * cap);
        for (uint32_t k = warp; k < n; k += n_fold) {
          const uint4 d0 = ds[2 * k];
          const uint32_t cnt = ds[2 * k + 1].x;
          const uint32_t nw = cnt & 0xffffu, nt2 = nw + (cnt >> 16);
          const unsigned char* gw = reinterpret_cast<const unsigned char*>(((unsigned long long)d0.y << 32) | d0.x);
          const unsigned char* gm = reinterpret_cast<const unsigned char*>(((unsigned long long)d0.w << 32) | d0.z);
          unsigned char* dst = sb + k * cap;
          for (uint32_t c = lane; c < nt2; c += 32) {
            const bool isw = c < nw;
            const uint32_t o = 16u * (isw ? c : c - nw);
            cp_async16(dst + (isw ? 0u : cap_w) + o, (isw ? gw : gm) + o);
          }
        }
      };
      const uint32_t lanes_lt = lanemask_lt();
      // Pipeline: rounds in pairs, one block barrier per pair.  Iteration of pair (r0, r0 + 1): wait
      // for the thread's copies (the pair's records and the headers of rounds r0 + 4, r0 + 5, all
      // issued in the previous iteration) and meet at the barrier; build the descriptors of rounds
      // r0 + 4 and r0 + 5 and fetch the headers of rounds r0 + 6 and r0 + 7 (header slots of rounds
      // r0 + 2 and r0 + 3, whose descriptors were built in the previous iteration); issue the
      // records of rounds r0 + 2 and r0 + 3 into the staging slots of rounds r0 - 2 and r0 - 1, which
      // every warp folded before this barrier; then fold rounds r0 and r0 + 1, during which those
      // copies land.  Descriptor slots: six rounds (the pair being folded, the pair being copied,
      // the pair being described).  The fold has one call site (code size: a second inlined copy of
      // it measured slower), and the window's last folds meet the update at the barrier after the
      // loop.
      if (R > 0) {
        // descriptors of the first kStages rounds (their headers were copied with the ids), then the
        // headers of rounds 4 and 5 and the records of the first pair
        for (uint32_t x = (uint32_t)warp; x < min(R, (uint32_t)kStages); x += (uint32_t)n_warps) store_desc(x);
        __syncthreads();
        for (uint32_t i = tid; i < 2u * B; i += blockDim.x) {
          const uint32_t x = 4u + i / B, k = i % B;
          if (x < R && x * B + k < S_tot) fetch_hdr(x, k);
        }
        issue_round(0u);
        issue_round(1u);
        cp_async_commit();
      }
      const uint32_t wbase_t = (uint32_t)(warp * tw);
      const uint32_t writer = (uint32_t)(blk * kMaxWarps + warp) + 1u;  // ownership check: this warp's stamp
      uint8_t* wtags = kRingSmem ? tags : tags + (size_t)warp * kTagHash;
      // The chunks of one round for this delivery warp, given its segments: per lane, the first
      // entry of segment `lane` in the warp's stream of the round (c_start), the staging addresses
      // of entry 0 as if the segment started there (c_wadj, c_madj), the emission slot + d_min;
      // n_ne segments, total entries.
      auto fold_chunks = [&](const uint32_t c_start, const uint32_t c_wadj, const uint32_t c_madj, const uint32_t c_sb,
                             const int n_ne, const uint32_t total) {
        if (lane == 0) my_events += total;
        int cur = -1;  // segment of the entry before the next chunk
        // the warp's chunks of 32 entries, up to four at a time.  Keys (ring cells, 0xffffffff:
        // no entry) and weights of all of a group's chunks are found step by step across the
        // chunks (segment starts, segment of each lane's entry, its staging addresses, its
        // record), so that the chunks' dependency chains overlap; then their ring updates run
        // in chunk order.
        uint32_t e = 0;
        auto fold_group = [&](auto nc) {
          constexpr int N = decltype(nc)::value;
          uint32_t key[N], sm[N], wa[N], ma[N], sbv[N];
          int sl[N];
          float wv[N];
#pragma unroll
          for (int u = 0; u < N; ++u) {
            const uint32_t cb = e + 32u * u;
            sm[u] = __reduce_or_sync(0xffffffffu, (lane < n_ne && c_start - cb < 32u) ? (1u << (c_start - cb)) : 0u);
          }
#pragma unroll
          for (int u = 0; u < N; ++u) {
            sl[u] = (cur + __popc(sm[u] & (lanes_lt | (1u << lane)))) & 31;
            cur += __popc(sm[u]);
          }
#pragma unroll
          for (int u = 0; u < N; ++u) wa[u] = __shfl_sync(0xffffffffu, c_wadj, sl[u]);
#pragma unroll
          for (int u = 0; u < N; ++u) ma[u] = __shfl_sync(0xffffffffu, c_madj, sl[u]);
#pragma unroll
          for (int u = 0; u < N; ++u) sbv[u] = __shfl_sync(0xffffffffu, c_sb, sl[u]);
#pragma unroll
          for (int u = 0; u < N; ++u) {
            const uint32_t q = e + 32u * u + lane;
            key[u] = 0xffffffffu;
            wv[u] = 0.0f;
            if (q < total) {
              const uint32_t meta = *reinterpret_cast<const uint16_t*>(stage + ma[u] + 2u * q);
              if constexpr (kBf16) wv[u] = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(stage + wa[u] + 2u * q));
              else wv[u] = *reinterpret_cast<const float*>(stage + wa[u] + 4u * q);
              uint32_t slot = sbv[u] + (meta & dmask);
              if (slot >= (uint32_t)D) slot -= (uint32_t)D;
              key[u] = slot * (uint32_t)nt + wbase_t + (meta >> dbits);
            }
          }
          if (a.stamps != nullptr)
#pragma unroll
            for (int u = 0; u < N; ++u) stamp_cell(a, wk.ring_base, key[u], writer);
          if constexpr (kExact) {
#pragma unroll
            for (int u = 0; u < N; ++u)
              if (key[u] != 0xffffffffu) ring_add_exact<kRingSmem>(ring, key[u], wv[u]);
          } else {
            fold_n<kRingSmem, N>(ring, wtags, key, wv, lane, ring_red);
          }
          e += 32u * N;
        };
        if constexpr (kExact) {
          // order-free adds: pairs of chunks (the second may be empty), one instantiation of the
          // group (smaller code measured faster than groups of one to four here)
          while (e < total) fold_group(std::integral_constant<int, 2>());
        } else {
          while (e < total) {
            const uint32_t left = (total - e + 31u) >> 5;
            if (left >= 4u) fold_group(std::integral_constant<int, 4>());
            else if (left == 3u) fold_group(std::integral_constant<int, 3>());
            else if (left == 2u) fold_group(std::integral_constant<int, 2>());
            else fold_group(std::integral_constant<int, 1>());
          }
        }
      };
      // the warp's segments of round r (spikes with entries in its sub-range), in spike order;
      // empty pieces are dropped so that segment starts are distinct
      auto segments_in = [&](const uint32_t r, uint32_t& len_k, uint32_t& wb_k, uint32_t& mb_k, uint32_t& sb_k) {
        len_k = wb_k = mb_k = sb_k = 0u;
        const uint32_t* aux_r = aux_slot(r);
        const uint16_t* ends_r = ends_slot(r);
        const uint32_t n = min(B, S_tot - r * B);
        if ((uint32_t)lane < n) {
          const uint32_t e1 = ends_r[warp * kSpikeBatch + lane];
          const uint32_t e0 = warp ? ends_r[(warp - 1) * kSpikeBatch + lane] : 0u;
          const uint32_t aux = aux_r[lane];
          len_k = e1 - e0;
          const uint32_t pk = (r % kStages) * (B * cap) + (uint32_t)lane * cap;
          wb_k = pk + (aux & 15u) + e0 * kWsz;
          mb_k = pk + cap_w + ((aux >> 8) & 15u) + e0 * 2u;
          sb_k = (aux >> 16) + (uint32_t)d_min;
        }
      };
      // ---- fold round r: each delivery warp, its target sub-range of every staged piece, in spike order
      auto fold_round = [&](const uint32_t r) {
        if (warp >= n_fold) return;
        uint32_t len_k, wb_k, mb_k, sb_k;
        segments_in(r, len_k, wb_k, mb_k, sb_k);
        const uint32_t ne = __ballot_sync(0xffffffffu, len_k > 0);
        const int n_ne = __popc(ne);
        uint32_t c_len = len_k, c_wb = wb_k, c_mb = mb_k, c_sb = sb_k;
        if (ne != (0xffffffffu >> (32 - max(n_ne, 1))) || n_ne == 0) {
          if (len_k > 0) perm[__popc(ne & lanes_lt)] = (uint8_t)lane;
          __syncwarp();
          const int src_lane = (lane < n_ne) ? (int)perm[lane] : 0;
          c_len = __shfl_sync(0xffffffffu, len_k, src_lane);
          c_wb = __shfl_sync(0xffffffffu, wb_k, src_lane);
          c_mb = __shfl_sync(0xffffffffu, mb_k, src_lane);
          c_sb = __shfl_sync(0xffffffffu, sb_k, src_lane);
          if (lane >= n_ne) c_len = 0;
          __syncwarp();
        }
        uint32_t c_end = c_len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, c_end, o);
          if (lane >= o) c_end += y;
        }
        const uint32_t c_start = c_end - c_len;
        fold_chunks(c_start, c_wb - c_start * kWsz, c_mb - c_start * 2u, c_sb, n_ne, __shfl_sync(0xffffffffu, c_end, 31));
      };
      // ---- fold rounds r0 and r0 + 1 with the two rounds' segment setups side by side (their chains
      // overlap), then each round's chunks (the ring in global memory with the ordered fold, where it
      // measured faster than one round at a time)
      auto fold_pair = [&](const uint32_t r0) {
        if (warp >= n_fold) return;
        const uint32_t nr = min(2u, R - r0);
        uint32_t len_k[2], wb_k[2], mb_k[2], sb_k[2], ne[2];
        int nne[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          len_k[k] = wb_k[k] = mb_k[k] = sb_k[k] = 0u;
          if ((uint32_t)k < nr) segments_in(r0 + (uint32_t)k, len_k[k], wb_k[k], mb_k[k], sb_k[k]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          ne[k] = __ballot_sync(0xffffffffu, len_k[k] > 0);
          nne[k] = __popc(ne[k]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (len_k[k] > 0) perm[k * 32 + __popc(ne[k] & lanes_lt)] = (uint8_t)lane;
        __syncwarp();
        uint32_t c_len[2], c_wb[2], c_mb[2], c_sbk[2], c_end[2], tot[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int src_lane = (lane < nne[k]) ? (int)perm[k * 32 + lane] : 0;
          c_len[k] = __shfl_sync(0xffffffffu, len_k[k], src_lane);
          c_wb[k] = __shfl_sync(0xffffffffu, wb_k[k], src_lane);
          c_mb[k] = __shfl_sync(0xffffffffu, mb_k[k], src_lane);
          c_sbk[k] = __shfl_sync(0xffffffffu, sb_k[k], src_lane);
          if (lane >= nne[k]) c_len[k] = 0;
          c_end[k] = c_len[k];
        }
        __syncwarp();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, c_end[k], o);
            if (lane >= o) c_end[k] += y;
          }
#pragma unroll
        for (int k = 0; k < 2; ++k) tot[k] = __shfl_sync(0xffffffffu, c_end[k], 31);
#pragma unroll 1
        for (uint32_t k = 0; k < nr; ++k) {
          const uint32_t c_start = k ? c_end[1] - c_len[1] : c_end[0] - c_len[0];
          fold_chunks(c_start, (k ? c_wb[1] : c_wb[0]) - c_start * kWsz, (k ? c_mb[1] : c_mb[0]) - c_start * 2u,
                      k ? c_sbk[1] : c_sbk[0], k ? nne[1] : nne[0], k ? tot[1] : tot[0]);
        }
      };
      for (uint32_t r0 = 0; r0 < R; r0 += 2u) {
        cp_async_wait<0>();
        __syncthreads();
        if (desc_tid >= 0 && desc_tid < 32) {  // the helper, else warp 0
          if (r0 + 4u < R) store_desc(r0 + 4u);
          if (r0 + 5u < R) store_desc(r0 + 5u);
        }
        if (desc_tid >= 0 && desc_tid < (int)B)
          for (uint32_t xh = r0 + 6u; xh < r0 + 8u; ++xh)
            if (xh < R && xh * B + desc_tid < S_tot) fetch_hdr(xh, (uint32_t)desc_tid);
        issue_round(r0 + 2u);
        issue_round(r0 + 3u);
        cp_async_commit();
        if constexpr (!kRingSmem && !kExact) {
          fold_pair(r0);
        } else {
#pragma unroll 1
          for (uint32_t r = r0; r < min(r0 + 2u, R); ++r) fold_round(r);
        }
      }
      cp_async_wait<0>();
      __syncthreads();
    }
    done += Wn;
  }

  // ---- epilogue: the pending I half of the last step, then write back state and ring ----
  __syncthreads();
  if (pend && !aborted) {
    const long long tl = t_start + a.n_steps - 1;
    float* rs = ring + (int64_t)(tl % D) * nt;
    for (int j = tid; j < nt; j += blockDim.x) {
      const float in = ring_read<kRingSmem>(rs + j);
      rs[j] = 0.0f;
      float cur = sI[j];
      i_half_k(cur, in, pk[j], nd);  // filled at the last barrier for step tl
      sI[j] = cur;
    }
    __syncthreads();
  }
  if (do_update) {
    for (int j = tid; j < nt; j += blockDim.x) {
      a.V[nbase + j] = sV[j];
      a.I[nbase + j] = sI[j];
      a.R[nbase + j] = sR[j];
    }
  }
  if (kRingSmem) {
    for (int q = tid; q < D * nt; q += blockDim.x) ring_g[q] = ring_s[q];
  }
  if (lane == 0 && my_events) atomicAdd(a.events + wk.net, my_events);
  if (persistent && do_deliver && wk.group == 0 && tid == 0 && a.raster_step != nullptr)
    a.raster_count[wk.net] = raster_total;
  if (persistent && blk == 0 && tid == 0 && a.t_fixed < 0 && !aborted) *a.step_counter = t_start + a.n_steps;
  if (persistent && tid == 0 && !aborted) a.pub_flag[blk] = epoch;  // windows completed, for the next launch
}

// split mode: advance the step counter and the per-network spike totals after a window
__global__ void k_advance(const StepArgs a, int n_nets, int wn) {
  const int net = blockIdx.x * blockDim.x + threadIdx.x;
  if (net < n_nets) {
    const NetDev& nd = a.nets[net];
    unsigned long long s = 0;
    for (int ws = 0; ws < wn; ++ws)
      for (int b = 0; b < nd.n_blocks; ++b) s += a.pub_cnt[(int64_t)ws * a.n_blocks + nd.first_block + b];
    a.raster_count[net] += s;
  }
  if (net == 0) *a.step_counter += wn;
}

// the kernel variant for a launch: ring placement, weight type, whether the block is wider than
// kNarrowWarps warps, and whether the adds need an order
using StepKernel = void (*)(StepArgs);
template <bool kRingSmem, bool kBf16, bool kWide>
StepKernel step_kernel_x(bool exact) {
  return exact ? k_step<kRingSmem, kBf16, kWide, true> : k_step<kRingSmem, kBf16, kWide, false>;
}
template <bool kRingSmem, bool kBf16>
StepKernel step_kernel_w(bool wide, bool exact) {
  return wide ? step_kernel_x<kRingSmem, kBf16, true>(exact) : step_kernel_x<kRingSmem, kBf16, false>(exact);
}
StepKernel step_kernel(bool ring_smem, bool bf16, int threads, bool exact) {
  const bool wide = threads > kNarrowWarps * 32;
  if (ring_smem) return bf16 ? step_kernel_w<true, true>(wide, exact) : step_kernel_w<true, false>(wide, exact);
  return bf16 ? step_kernel_w<false, true>(wide, exact) : step_kernel_w<false, false>(wide, exact);
}

cudaError_t launch_step(const StepArgs& a, int grid, int threads, size_t smem, bool cooperative, cudaStream_t s,
                        const cudaAccessPolicyWindow* apw) {
  StepKernel kern = step_kernel(a.ring_smem != 0, a.bf16 != 0, threads, a.exact != 0);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (cooperative) {
    // all blocks must be co-resident: they wait on each other at the window barrier
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  if (apw != nullptr && apw->num_bytes > 0) {
    // the global ring is marked persisting in L2, so the streamed records do not evict it
    attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[na].val.accessPolicyWindow = *apw;
    ++na;
  }
  cfg.attrs = na ? attr : nullptr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_advance_split(const StepArgs& a, int n_nets, int wn, cudaStream_t s) {
  k_advance<<<(n_nets + 127) / 128, 128, 0, s>>>(a, n_nets, wn);
  return cudaGetLastError();
}

size_t step_smem_bytes(int nt, int depth, int window, int nb, bool ring_smem, int stage_bytes, int n_warps,
                       bool ordered) {
  return make_layout(nt, depth, window, nb, ring_smem, stage_bytes, n_warps, ordered).total;
}

// staging bytes per spike: a segment of up to max_seg_len records, widened to 16-byte boundaries
void step_staging_caps(int max_seg_len, int wsz, int* cap_w, int* cap_m) {
  *cap_w = (int)align_to((uint32_t)(max_seg_len * wsz + 32), 16);
  *cap_m = (int)align_to((uint32_t)(max_seg_len * 2 + 32), 16);
}

cudaError_t step_kernel_attributes(size_t smem) {
  for (int v = 0; v < 16; ++v) {
    const StepKernel k = step_kernel((v & 1) != 0, (v & 2) != 0, (v & 4) ? kMaxWarps * 32 : 32, (v & 8) != 0);
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int step_occupancy(int threads, size_t smem, bool ring_smem) {
  int n = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel(ring_smem, false, threads, false), threads, smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace cortex
