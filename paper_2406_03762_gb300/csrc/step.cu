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
// Delivery runs in rounds of up to kSpikeBatch spikes.  All warps stage the record segments of
// round r + kStages - 1 into shared memory with 16-byte cp.async copies (each spike has a
// fixed-size region of its slot), then fold round r; the headers of round r + kStages load into
// registers meanwhile.  So kStages - 1 rounds of records are always in flight.
#include "cortex_internal.cuh"

namespace cortex {

struct SpikeInfo {    // one staged spike of a delivery round
  uint32_t woff;     // staging byte offset of record 0 of the block's piece, weight stream
  uint32_t moff;     // ... meta stream
  uint32_t endw[7];  // header words 1..7: u16 end[w] of the delivery warps
  uint32_t tm;       // emission step mod D
};

struct SmemLayout {
  uint32_t ring, sv, si, sr, thr, cnt, woffs, wcnt, wlist, ids, hdr, rowb, info, perm, tags, stage, total;
};

__host__ __device__ inline uint32_t align_to(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// duplicate-detection tags: one byte per ring cell when the ring is in shared memory, else a
// hashed table of kTagHash bytes per warp
constexpr int kTagHash = 2048;

__host__ __device__ inline SmemLayout make_layout(int max_nt, int max_depth, int w_max, int max_nb, bool ring_smem,
                                                  int stage_bytes) {
  SmemLayout L;
  uint32_t o = 0;
  L.ring = o;
  o += ring_smem ? (uint32_t)(max_depth * max_nt * 4) : 0u;
  o = align_to(o, 16);
  L.sv = o;
  o += max_nt * 4;
  L.si = o;
  o += max_nt * 4;
  L.sr = o;
  o += max_nt * 4;
  o = align_to(o, 16);
  L.thr = o;
  o += kPoissonCap * 4;
  L.cnt = o;
  o += (uint32_t)(w_max * (max_nb + 1) * 4);
  o = align_to(o, 16);
  L.woffs = o;
  o += (uint32_t)((w_max + 1) * 4);
  o = align_to(o, 16);
  L.wcnt = o;
  o += (kMaxWarps + 2) * 4;
  o = align_to(o, 16);
  L.wlist = o;
  o += max_nt * 4;
  o = align_to(o, 16);
  L.ids = o;
  o += kIdCap * 4;
  L.hdr = o;
  o += (kStages + 1) * kSpikeBatch * 32;
  L.rowb = o;
  o += (kStages + 1) * kSpikeBatch * 8;
  L.info = o;
  o += kStages * kSpikeBatch * (uint32_t)sizeof(SpikeInfo);
  L.perm = o;
  o += kMaxWarps * 32;
  o = align_to(o, 16);
  L.tags = o;
  o += ring_smem ? align_to((uint32_t)(max_depth * max_nt), 16) : (uint32_t)(kMaxWarps * kTagHash);
  o = align_to(o, 128);
  L.stage = o;
  o += (uint32_t)stage_bytes;
  L.total = o;
  return L;
}

// ---- one neuron, one step (Eq. 1-3, exact integration) --------------------------------------
//   V half: refractory: V = V_reset, counter - 1;  else V = V + fma(P22 - 1, V, P21 * I) with
//           the I of the previous step;  V >= V_th: spike, V = V_reset, counter = n_ref (Eq. 2)
//   I half: in = ring cell of the step (cleared); k = Poisson draw; ext = k * J_ext;
//           I = fma(P11, I, in); I = I + ext
struct NeuronConst {
  float p11, p21, p22m1, v_th, v_reset, j_ext;
  int32_t n_ref, n_thr;
};

__device__ __forceinline__ bool v_half(float& v, float cur, int32_t& r, const NeuronConst& nd) {
  if (r > 0) {
    v = nd.v_reset;
    r -= 1;
  } else {
    v = __fadd_rn(v, __fmaf_rn(nd.p22m1, v, __fmul_rn(nd.p21, cur)));
  }
  const bool spk = v >= nd.v_th;
  if (spk) {
    v = nd.v_reset;
    r = nd.n_ref;
  }
  return spk;
}

__device__ __forceinline__ void i_half(float& cur, float in, uint32_t u, const NeuronConst& nd, const uint32_t* thr) {
  int k = 0;
  while (k < nd.n_thr - 1 && u >= thr[k]) ++k;
  const float ext = __fmul_rn((float)k, nd.j_ext);
  cur = __fmaf_rn(nd.p11, cur, in);
  cur = __fadd_rn(cur, ext);
}

// Add the weights of one 32-lane chunk to their ring cells (key = cell, 0xffffffff = no entry).
// Lanes hold entries in stream order.  Lanes whose cell no other lane of the chunk touches add at
// once; lanes that share a cell add one by one in lane order, so every cell folds its weights in
// stream order.  Sharing is found by writing the lane id into a tag per cell and reading it back.
template <bool kRingSmem>
__device__ __forceinline__ void fold_chunk(float* ring, uint8_t* wtags, uint32_t key, float w, int lane) {
  const bool valid = key != 0xffffffffu;
  // shared ring: one tag per cell (warps own disjoint cells); global ring: the warp's hashed table
  uint8_t* tg = kRingSmem ? wtags + (valid ? key : 0u) : wtags + (key & (uint32_t)(kTagHash - 1));
  if (valid) *tg = (uint8_t)lane;
  __syncwarp();
  const uint32_t t = valid ? (uint32_t)*tg : (uint32_t)lane;
  const bool loser = valid && t != (uint32_t)lane;
  const uint32_t losers = __ballot_sync(0xffffffffu, loser);
  if (losers == 0) {
    if (valid) ring[key] = __fadd_rn(ring[key], w);
  } else {
    const uint32_t winners = __reduce_or_sync(0xffffffffu, loser ? (1u << t) : 0u);
    const uint32_t dup = losers | winners;
    if (valid && !((dup >> lane) & 1u)) ring[key] = __fadd_rn(ring[key], w);
    __syncwarp();
    uint32_t m = dup;
    while (m) {
      const int first = __ffs(m) - 1;
      if (lane == first) ring[key] = __fadd_rn(ring[key], w);
      __syncwarp();
      m &= m - 1u;
    }
  }
  __syncwarp();
}

// ---- the step kernel ---------------------------------------------------------------------------
// phases: kPhaseUpdate, kPhaseDeliver, and kPhaseBarrier for the persistent form (both phases and
// a barrier per window inside one cooperative launch of n_steps steps).  kRingSmem: the block's
// ring slice lives in shared memory for the whole launch (loaded in the prologue, written back
// in the epilogue); otherwise it is updated in place in global memory.
template <bool kRingSmem>
__global__ void __launch_bounds__(kMaxWarps * 32) k_step(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
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
  const bool do_update = (a.phases & kPhaseUpdate) != 0;
  const bool do_deliver = (a.phases & kPhaseDeliver) != 0;
  const bool bf16 = ndg.wdtype == 1;
  const uint32_t wsz = bf16 ? 2u : 4u;
  const uint32_t B = (uint32_t)a.batch, cap_w = (uint32_t)a.cap_w, cap = (uint32_t)(a.cap_w + a.cap_m);

  const SmemLayout L = make_layout(a.max_nt, a.max_depth, a.w_max, a.max_nb, kRingSmem, a.stage_bytes);
  float* ring_s = reinterpret_cast<float*>(smem + L.ring);
  float* sV = reinterpret_cast<float*>(smem + L.sv);
  float* sI = reinterpret_cast<float*>(smem + L.si);
  int32_t* sR = reinterpret_cast<int32_t*>(smem + L.sr);
  uint32_t* thr = reinterpret_cast<uint32_t*>(smem + L.thr);
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + L.cnt);
  uint32_t* woffs = reinterpret_cast<uint32_t*>(smem + L.woffs);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + L.wcnt);
  uint32_t* wlist = reinterpret_cast<uint32_t*>(smem + L.wlist);
  uint32_t* ids_s = reinterpret_cast<uint32_t*>(smem + L.ids);
  uint4* hdr_s = reinterpret_cast<uint4*>(smem + L.hdr);
  unsigned long long* rowb_s = reinterpret_cast<unsigned long long*>(smem + L.rowb);
  SpikeInfo* info = reinterpret_cast<SpikeInfo*>(smem + L.info);
  uint8_t* perm = smem + L.perm + warp * 32;
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
      sR[j] = a.R[nbase + j];
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

  const bool defer = persistent;  // V/I halves with the window's last I half after the barrier
  bool pend = false;               // the I half of the previous window's last step is due
  const int W = persistent ? window : min(window, a.n_steps);
  const int tw_u = (nt + n_warps - 1) / n_warps;  // update split over the warps
  int done = 0;
  while (done < a.n_steps) {
    const int Wn = min(W, a.n_steps - done);
    const long long t0 = t_start + done;
    const int tm0 = (int)(t0 % D);  // ring slot of the window's first step
    const uint32_t par = persistent ? ((epoch + 1u) & 1u) : 0u;

    // ================= update + compaction + publication =================
    if (do_update) {
      for (int ws = 0; ws < Wn; ++ws) {
        const long long t = t0 + ws;
        const int slot = (tm0 + ws) % D;
        const int pslot = (tm0 + ws + D - 1) % D;    // slot of step t - 1
        const bool prev = defer && (ws > 0 || pend);  // the I half of step t - 1 is still due
        float* rs = ring + (int64_t)(defer ? pslot : slot) * nt;
        const uint32_t tu = (uint32_t)(defer ? t - 1 : t);
        const int lo = warp * tw_u, hi = min(lo + tw_u, nt);
        uint32_t cw = 0;
        for (int c = lo; c < hi; c += 32) {
          const int j = c + lane;
          bool spk = false;
          if (j < hi) {
            float v = sV[j], cur = sI[j];
            int32_t r = sR[j];
            if (defer) {
              if (prev) {
                const float in = rs[j];
                rs[j] = 0.0f;
                const uint4 rr = philox4x32_10(make_uint4((uint32_t)(wk.t0 + j), tu, kStreamPoisson, 0u), seed_lo, seed_hi);
                i_half(cur, in, rr.x, nd, thr);
              }
              spk = v_half(v, cur, r, nd);
            } else {
              const float in = rs[j];
              rs[j] = 0.0f;
              const uint4 rr = philox4x32_10(make_uint4((uint32_t)(wk.t0 + j), tu, kStreamPoisson, 0u), seed_lo, seed_hi);
              spk = v_half(v, cur, r, nd);
              i_half(cur, in, rr.x, nd, thr);
            }
            sV[j] = v;
            sI[j] = cur;
            sR[j] = r;
          }
        const uint32_t bal = __ballot_sync(0xffffffffu, spk);
          if (spk) wlist[lo + cw + __popc(bal & lanemask_lt())] = (uint32_t)(wk.t0 + j);
          cw += __popc(bal);
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
        for (uint32_t q = lane; q < cw; q += 32) dst[before + q] = wlist[lo + q];
        if (tid == 0) {
          a.pub_cnt[(int64_t)(par * a.w_max + ws) * a.n_blocks + blk] = total;
          if (ws == 0) wcnt[kMaxWarps] = total;
        }
        __syncthreads();
      }
      pend = defer;
      if (persistent && tid == 0 && blk != a.withhold_block) {
        // the release store orders every write of the block before it (bar.sync + cumulativity)
        st_release_u64(a.pub_flag + blk, (unsigned long long)(epoch + 1u) | ((unsigned long long)wcnt[kMaxWarps] << 32));
      }
    }

    // ================= grid barrier among the blocks of this network =================
    if (persistent) {
      epoch += 1u;
      int fail = 0;
      for (int b = tid; b < nb; b += blockDim.x) {
        const unsigned long long* f = a.pub_flag + first_block + b;
        unsigned long long m = ld_acquire_u64(f);
        if ((int32_t)((uint32_t)m - epoch) < 0) {
          const long long tb0 = global_ns();
          uint32_t spins = 0;
          do {
            if ((++spins & 255u) == 0 &&
                (global_ns() - tb0 > a.timeout_ns || *(volatile int32_t*)a.err != 0)) {
              fail = 1;
              break;
            }
            m = ld_acquire_u64(f);
          } while ((int32_t)((uint32_t)m - epoch) < 0);
        }
        cnt_s[b] = (uint32_t)(m >> 32);  // count of the window's first step
      }
      if (__syncthreads_or(fail)) {
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        aborted = true;
        break;
      }
    }

    // ================= delivery =================
    if (do_deliver) {
      // counts of every block of this network, then exclusive prefixes per window step
      for (int q = tid; q < Wn * nb; q += blockDim.x) {
        const int ws = q / nb, b = q % nb;
        if (!persistent || ws > 0)
          cnt_s[ws * (nb + 1) + b] =
              __ldcg(a.pub_cnt + (int64_t)(par * a.w_max + ws) * a.n_blocks + first_block + b);
      }
      __syncthreads();
      for (int ws = warp; ws < Wn; ws += n_warps) {
        uint32_t* c = cnt_s + ws * (nb + 1);
        uint32_t carry = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
          const int b = b0 + lane;
          const uint32_t v = (b < nb) ? c[b] : 0u;
          uint32_t x = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
          }
          if (b < nb) c[b] = carry + x - v;
          carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) c[nb] = carry;
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t o = 0;
        for (int ws = 0; ws < Wn; ++ws) {
          woffs[ws] = o;
          o += cnt_s[ws * (nb + 1) + nb];
        }
        woffs[Wn] = o;
      }
      __syncthreads();
      const uint32_t S_tot = woffs[Wn];
      // spike ids of the window into shared memory (window order: step, then id); raster
      for (int task = warp; task < Wn * nb; task += n_warps) {
        const int ws = task / nb, b = task % nb;
        const uint32_t* pref = cnt_s + ws * (nb + 1);
        const uint32_t c = pref[b + 1] - pref[b];
        if (c == 0) continue;
        const uint32_t* src = a.pub_ids + (int64_t)(par * a.w_max + ws) * a.n_total + neuron_base + (int64_t)b * tb_full;
        const uint32_t o = woffs[ws] + pref[b];
        const bool mine = (b == wk.group) && a.raster_step != nullptr;
        for (uint32_t q = lane; q < c; q += 32) {
          const bool need = (o + q < (uint32_t)kIdCap) || mine;
          if (!need) continue;
          const uint32_t id = __ldcg(src + q);
          if (o + q < (uint32_t)kIdCap) ids_s[o + q] = id;
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
      __syncthreads();

      const uint32_t R = (S_tot + B - 1) / B;  // delivery rounds of this window
      // spike id of window index g (shared list, or the published global lists beyond it)
      auto spike_id = [&](uint32_t g) -> uint32_t {
        if (g < (uint32_t)kIdCap) return ids_s[g];
        int ws = 0;
        while (ws + 1 < Wn && woffs[ws + 1] <= g) ++ws;
        const uint32_t* pref = cnt_s + ws * (nb + 1);
        const uint32_t qq = g - woffs[ws];
        int lo2 = 0, hi2 = nb;
        while (hi2 - lo2 > 1) {
          const int mid = (lo2 + hi2) >> 1;
          if (pref[mid] <= qq) lo2 = mid;
          else hi2 = mid;
        }
        return __ldcg(a.pub_ids + (int64_t)(par * a.w_max + ws) * a.n_total + neuron_base + (int64_t)lo2 * tb_full +
                      (qq - pref[lo2]));
      };
      // header (32 B) and row start of the block's piece of spike g
      auto load_hdr = [&](uint32_t g, uint4& h0, uint4& h1, unsigned long long& row) {
        const uint32_t id = spike_id(g);
        const uint4* hp = a.hdr + 2 * (hdr_net + (int64_t)id * nb + wk.group);
        h0 = __ldg(hp);
        h1 = __ldg(hp + 1);
        row = __ldg(a.row_base + row_off + id);
      };
      auto hdr_slot = [&](uint32_t x) { return hdr_s + (x % (kStages + 1)) * (2 * kSpikeBatch); };
      auto rowb_slot = [&](uint32_t x) { return rowb_s + (x % (kStages + 1)) * kSpikeBatch; };
      // stage the records of round x: warp w copies spikes w, w + n_warps, ... (lanes over 16-byte
      // chunks) and records where each piece landed
      auto issue_round = [&](uint32_t x) {
        if (x >= R) return;
        const uint4* hs = hdr_slot(x);
        const unsigned long long* rb = rowb_slot(x);
        const uint32_t n = min(B, S_tot - x * B);
        const uint32_t sb = (x % kStages) * (B * cap);
        SpikeInfo* inf = info + (x % kStages) * kSpikeBatch;
        for (uint32_t k = warp; k < n; k += n_warps) {
          const uint4 h0 = hs[2 * k], h1 = hs[2 * k + 1];
          const uint32_t len = h1.w >> 16;
          const uint64_t r0 = (uint64_t)rec_net + rb[k] + (h0.x & 0xffffu);
          const uint32_t d = sb + k * cap;
          if (lane == 0) {
            const uint32_t g = x * B + k;
            int ws = 0;
            while (ws + 1 < Wn && woffs[ws + 1] <= g) ++ws;
            SpikeInfo si;
            si.woff = d + (uint32_t)((r0 * wsz) & 15u);
            si.moff = d + cap_w + (uint32_t)((r0 * 2u) & 15u);
            si.endw[0] = h0.y; si.endw[1] = h0.z; si.endw[2] = h0.w;
            si.endw[3] = h1.x; si.endw[4] = h1.y; si.endw[5] = h1.z; si.endw[6] = h1.w;
            si.tm = (uint32_t)((tm0 + ws) % D);
            inf[k] = si;
          }
          if (len == 0) continue;
          const uint64_t wb0 = (r0 * wsz) & ~15ull, wb1 = ((r0 + len) * wsz + 15) & ~15ull;
          const uint64_t mb0 = (r0 * 2u) & ~15ull, mb1 = ((r0 + len) * 2u + 15) & ~15ull;
          const unsigned char* gw = reinterpret_cast<const unsigned char*>(a.rec_w) + wb0;
          const unsigned char* gm = reinterpret_cast<const unsigned char*>(a.rec_meta) + mb0;
          const uint32_t nw = (uint32_t)((wb1 - wb0) >> 4), nm = (uint32_t)((mb1 - mb0) >> 4);
          for (uint32_t c = lane; c < nw; c += 32) cp_async16(stage + d + 16u * c, gw + 16u * c);
          for (uint32_t c = lane; c < nm; c += 32) cp_async16(stage + d + cap_w + 16u * c, gm + 16u * c);
        }
      };

      if (R > 0) {
        // headers of the first kStages rounds, then the records of the first kStages - 1 rounds
        for (uint32_t i = tid; i < min(R, (uint32_t)kStages) * B; i += blockDim.x) {
          const uint32_t x = i / B, k = i % B;
          if (x * B + k < S_tot) {
            uint4 h0, h1;
            unsigned long long row;
            load_hdr(x * B + k, h0, h1, row);
            hdr_slot(x)[2 * k] = h0;
            hdr_slot(x)[2 * k + 1] = h1;
            rowb_slot(x)[k] = row;
          }
        }
        __syncthreads();
        for (int x = 0; x < kStages - 1; ++x) {
          issue_round((uint32_t)x);
          cp_async_commit();
        }
      }
      const uint32_t wbase_t = (uint32_t)(warp * tw);
      uint8_t* wtags = kRingSmem ? tags : tags + (size_t)warp * kTagHash;
      for (uint32_t r = 0; r < R; ++r) {
        issue_round(r + kStages - 1);
        cp_async_commit();
        // header of round r + kStages into registers (stored after the fold)
        uint4 nh0 = make_uint4(0, 0, 0, 0), nh1 = nh0;
        unsigned long long nrow = 0;
        const uint32_t xn = r + kStages;
        const bool have_next = tid < (int)B && xn < R && xn * B + tid < S_tot;
        if (have_next) load_hdr(xn * B + tid, nh0, nh1, nrow);
        cp_async_wait<kStages - 1>();
        __syncthreads();

        // ---- fold round r: each warp, its target sub-range of every staged piece, in spike order
        {
          const SpikeInfo* inf = info + (r % kStages) * kSpikeBatch;
          const uint32_t n = min(B, S_tot - r * B);
          uint32_t len_k = 0, wb_k = 0, mb_k = 0, tm_k = 0;
          if ((uint32_t)lane < n) {
            const uint16_t* ends = reinterpret_cast<const uint16_t*>(inf[lane].endw);
            const uint32_t e0 = warp ? ends[warp - 1] : 0u, e1 = ends[warp];
            len_k = e1 - e0;
            wb_k = inf[lane].woff + e0 * wsz;
            mb_k = inf[lane].moff + e0 * 2u;
            tm_k = inf[lane].tm;
          }
          // compact the non-empty pieces (their order is the spike order)
          const uint32_t ne = __ballot_sync(0xffffffffu, len_k > 0);
          const int n_ne = __popc(ne);
          if (len_k > 0) perm[__popc(ne & lanemask_lt())] = (uint8_t)lane;
          __syncwarp();
          const int src_lane = (lane < n_ne) ? (int)perm[lane] : 0;
          const uint32_t c_wb = __shfl_sync(0xffffffffu, wb_k, src_lane);
          const uint32_t c_mb = __shfl_sync(0xffffffffu, mb_k, src_lane);
          const uint32_t c_tm = __shfl_sync(0xffffffffu, tm_k, src_lane);
          uint32_t c_len = __shfl_sync(0xffffffffu, len_k, src_lane);
          if (lane >= n_ne) c_len = 0;
          uint32_t c_end = c_len;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, c_end, o);
            if (lane >= o) c_end += y;
          }
          const uint32_t c_start = c_end - c_len;
          const uint32_t total = __shfl_sync(0xffffffffu, c_end, 31);
          if (lane == 0) my_events += total;
          int cur = -1;
          // key and weight of the lane's entry in the chunk starting at cb (0xffffffff: none)
          auto chunk_key = [&](uint32_t cb, float& wv) -> uint32_t {
            const uint32_t bits = (lane < n_ne && c_start >= cb && c_start < cb + 32) ? (1u << (c_start - cb)) : 0u;
            const uint32_t sm = __reduce_or_sync(0xffffffffu, bits);
            const int seg = cur + __popc(sm & (0xffffffffu >> (31 - lane)));
            cur += __popc(sm);
            const uint32_t q = cb + lane;
            const int sl = seg & 31;
            const uint32_t swb = __shfl_sync(0xffffffffu, c_wb, sl);
            const uint32_t smb = __shfl_sync(0xffffffffu, c_mb, sl);
            const uint32_t scs = __shfl_sync(0xffffffffu, c_start, sl);
            const uint32_t stm = __shfl_sync(0xffffffffu, c_tm, sl);
            wv = 0.0f;
            if (q >= total) return 0xffffffffu;
            const uint32_t m = q - scs;
            const uint32_t meta = *reinterpret_cast<const uint16_t*>(stage + smb + 2u * m);
            wv = bf16 ? __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(stage + swb + 2u * m))
                      : *reinterpret_cast<const float*>(stage + swb + 4u * m);
            int slot = (int)stm + d_min + (int)(meta & dmask);
            if (slot >= D) slot -= D;
            return (uint32_t)slot * (uint32_t)nt + wbase_t + (meta >> dbits);
          };
          uint32_t e = 0;
          for (; e + 3 * 32 < total; e += 4 * 32) {  // four chunks at a time while they are all used
            uint32_t key[4];
            float wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) key[u] = chunk_key(e + 32u * u, wv[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) fold_chunk<kRingSmem>(ring, wtags, key[u], wv[u], lane);
          }
          for (; e < total; e += 32) {
            float wv;
            const uint32_t key = chunk_key(e, wv);
            fold_chunk<kRingSmem>(ring, wtags, key, wv, lane);
          }
        }
        if (have_next) {
          hdr_slot(xn)[2 * tid] = nh0;
          hdr_slot(xn)[2 * tid + 1] = nh1;
          rowb_slot(xn)[tid] = nrow;
        }
        __syncthreads();
      }
      cp_async_wait<0>();
    }
    done += Wn;
  }

  // ---- epilogue: the pending I half of the last step, then write back state and ring ----
  __syncthreads();
  if (pend && !aborted) {
    const long long tl = t_start + a.n_steps - 1;
    float* rs = ring + (int64_t)(tl % D) * nt;
    for (int j = tid; j < nt; j += blockDim.x) {
      const float in = rs[j];
      rs[j] = 0.0f;
      const uint4 rr = philox4x32_10(make_uint4((uint32_t)(wk.t0 + j), (uint32_t)tl, kStreamPoisson, 0u), seed_lo, seed_hi);
      float cur = sI[j];
      i_half(cur, in, rr.x, nd, thr);
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

cudaError_t launch_step(const StepArgs& a, int grid, int threads, size_t smem, bool cooperative, cudaStream_t s) {
  void (*kern)(StepArgs) = a.ring_smem ? k_step<true> : k_step<false>;
  if (cooperative) {
    // all blocks must be co-resident: they wait on each other at the window barrier
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
  }
  kern<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_advance_split(const StepArgs& a, int n_nets, int wn, cudaStream_t s) {
  k_advance<<<(n_nets + 127) / 128, 128, 0, s>>>(a, n_nets, wn);
  return cudaGetLastError();
}

size_t step_smem_bytes(int max_nt, int max_depth, int w_max, int max_nb, bool ring_smem, int stage_bytes) {
  return make_layout(max_nt, max_depth, w_max, max_nb, ring_smem, stage_bytes).total;
}

// staging bytes per spike: a segment of up to max_seg_len records, widened to 16-byte boundaries
void step_staging_caps(int max_seg_len, int wsz, int* cap_w, int* cap_m) {
  *cap_w = (int)align_to((uint32_t)(max_seg_len * wsz + 32), 16);
  *cap_m = (int)align_to((uint32_t)(max_seg_len * 2 + 32), 16);
}

cudaError_t step_kernel_attributes(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_step<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int step_occupancy(int threads, size_t smem, bool ring_smem) {
  int n = 0;
  cudaError_t e = ring_smem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<true>, threads, smem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<false>, threads, smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace cortex
