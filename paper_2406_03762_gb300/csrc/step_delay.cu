// step_delay.cu -- the per-step hot path with delay-ordered delivery (Sec. III-B "Varied Synaptic
// Delays": the synapses of a source are reordered by delay and processed as steps pass; Sec. III-C:
// a spike buffer holds the spiking pre-neurons until all their delays have elapsed).
//
// Ownership is the same as in the ring kernel (step.cu): every block owns a contiguous range of
// post-synaptic neurons and all their incoming synapses (Eq. 5, Eq. 9-10).  What changes is when a
// synapse is read.  The ring kernel reads a spike's synapses once, at emission, and adds each weight
// into a ring of future input (D = d_max + 1 slots per neuron).  Here the synapses of delay d of a
// source that spiked at step e are read at step e + d, when they arrive, and added into an
// accumulator of that arrival step only.  So a block needs the input of the steps of one window
// (W = d_min + 1 accumulators per neuron, in shared memory) instead of a D-deep ring, and needs the
// spikes of the last d_max steps: the spike buffer, kept in HBM (hist_ids / hist_cnt, d_max + W + 1
// steps deep).
//
// Records (built once by k_delay_layout): each (source, block) piece of a row sorted by (delay,
// target, draw), with a table of u16 offsets of its delay pieces.  At arrival step T a block reads,
// for every delay d and every source s that spiked at T - d, the piece (s, block, d).  The pieces
// of one spike for the W arrival steps of a window (consecutive delays) are adjacent, and so are
// their table entries: the lanes that hold them share cache lines.
//
// Summation order of an accumulator cell (T, target): emission step ascending (= delay descending),
// then source id ascending, then draw index -- the order of the oracle and of the ring kernel, so
// the results are the same bits.  The block walks the emission steps in ascending order and their
// spikes in ascending id; the arrival steps of a window are independent cells.  Two folds:
//   ordered: one warp per arrival step folds that step's pieces in stream order, lanes sharing a
//            cell in lane order (fold_one, tags per cell);
//   exact:   when the build has proven every partial sum exact (see ring_add_exact), every warp
//            folds any piece with shared-memory reductions, in any order.
//
// Window structure (as in the ring kernel): W = d_min + 1 steps per window.  Update: for each step
// t of the window, the I half of t - 1 (accumulator of arrival step t - 1, Poisson drive) then the
// V half of t; the spikes of t go to the spike buffer.  Then the grid barrier of the network.  Then
// the delivery of the next window's arrival steps t_last .. t_last + W - 1 (t_last the window's
// last step): they need spikes up to t_last + W - 1 - d_min = t_last, all published.
#include <type_traits>

#include "cortex_internal.cuh"
#include "step_common.cuh"

namespace cortex {

struct DLayout {
  uint32_t acc, sv, si, sr, pk, thr, wcnt, wlist, ecnt, ids, ide, tags, total;
};

// (emission step, block) counts a delivery of a network needs, plus the raster's prefix pairs
__host__ __device__ inline int dcount_words(int d_max, int nb) { return (d_max + 1) * (nb + 2); }

__host__ __device__ inline uint32_t dalign(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline DLayout make_dlayout(int nt, int window, int n_warps, bool exact, int ncnt) {
  DLayout L;
  uint32_t o = 0;
  L.acc = o;  // window x nt accumulators: the input of the window's arrival steps
  o += (uint32_t)(window * nt * 4);
  L.sv = o;
  o += nt * 4;
  L.si = o;
  o += nt * 4;
  L.sr = o;  // refractory counters, 16 bit
  o = dalign(o + nt * 2, 16);
  L.pk = o;  // Poisson counts of the window's I halves, [step][target]
  o = dalign(o + (uint32_t)(window * nt), 16);
  L.thr = o;
  o += kPoissonCap * 4;
  L.wcnt = o;  // per-warp counts and scan scratch
  o += (kDMaxWarps + 2) * 4;
  L.wlist = o;  // the step's spikes of each warp's sub-range (local ids, 16 bit)
  o = dalign(o + nt * 2, 16);
  L.ecnt = o;  // (emission step, block) spike counts of the window's delivery, then their prefixes
  o = dalign(o + (uint32_t)(ncnt + 1) * 4, 16);
  L.ids = o;  // spike ids of the current chunk of emission steps
  o += kDIdCap * 4;
  L.ide = o;  // their emission step, relative to the first
  o += kDIdCap * 2;
  L.tags = o;  // ordered fold: one tag byte per cell for each folding warp
  o = dalign(o + (exact ? 0u : (uint32_t)(min(window, n_warps) * nt)), 16);
  L.total = o;
  return L;
}

template <bool kBf16, bool kExact, bool kWide>
__global__ void __launch_bounds__(kWide ? kDMaxWarps * 32 : 16 * 32, 1) k_dstep(const StepArgs a) {
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
  const int nb = ndg.n_blocks, first_block = ndg.first_block, W = ndg.window;
  const int d_min = ndg.d_min, d_max = ndg.d_max, H = ndg.hist_depth;
  const int64_t neuron_base = ndg.neuron_base, raster_base = ndg.raster_base, raster_cap = ndg.raster_cap;
  const int64_t rec_net = ndg.rec_base, row_off = ndg.row_off, tbl_net = ndg.tbl_base;
  const int tbl_stride = ndg.tbl_stride, tbl_last = tbl_stride - 1;  // last word: the row length
  const int n_del1 = d_max - d_min + 2;  // table words per block: one per delay, and the piece end
  const int nt = wk.nt;
  const int tb_full = a.work[first_block].nt;

  const int ncnt = dcount_words(d_max, nb);  // <= kDCntCap (checked by the build)
  const DLayout L = make_dlayout(tb_full, W, n_warps, kExact, ncnt);
  float* acc = reinterpret_cast<float*>(smem + L.acc);
  float* sV = reinterpret_cast<float*>(smem + L.sv);
  float* sI = reinterpret_cast<float*>(smem + L.si);
  int16_t* sR = reinterpret_cast<int16_t*>(smem + L.sr);
  uint8_t* pk = smem + L.pk;
  uint32_t* thr = reinterpret_cast<uint32_t*>(smem + L.thr);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + L.wcnt);
  uint16_t* wlist = reinterpret_cast<uint16_t*>(smem + L.wlist);
  uint32_t* ecnt = reinterpret_cast<uint32_t*>(smem + L.ecnt);
  uint32_t* ids_s = reinterpret_cast<uint32_t*>(smem + L.ids);
  uint16_t* ide_s = reinterpret_cast<uint16_t*>(smem + L.ide);
  uint8_t* tags = smem + L.tags;

  const int64_t nbase = neuron_base + wk.t0;
  for (int q = tid; q < kPoissonCap; q += blockDim.x) thr[q] = ndg.thr[q];
  for (int j = tid; j < nt; j += blockDim.x) {
    sV[j] = a.V[nbase + j];
    sI[j] = a.I[nbase + j];
    sR[j] = (int16_t)a.R[nbase + j];
  }
  const long long t_start = *a.step_counter;
  uint32_t epoch = (uint32_t)__ldcg(a.pub_flag + blk);  // windows this network completed
  unsigned long long raster_total = a.raster_count[wk.net];
  unsigned long long my_events = 0;
  bool aborted = false;
  __syncthreads();

  // Poisson counts of steps tfirst .. tfirst + ns - 1 of every owned target: one generator call per
  // (step, group of four consecutive neurons), word i mod 4 for neuron i (as the oracle draws)
  const int pq_g0 = wk.t0 >> 2, pq_ng = ((wk.t0 + nt + 3) >> 2) - pq_g0;
  auto poisson_fill = [&](long long tfirst, int ns) {
    const int tot = ns * pq_ng;
    for (int q = tid; q < tot; q += blockDim.x) {
      const int sidx = q / pq_ng, g = pq_g0 + (q - sidx * pq_ng);
      const uint4 rr = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(tfirst + sidx), kStreamPoisson, 0u),
                                     seed_lo, seed_hi);
      const uint32_t wd[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int j = 4 * g + w - wk.t0;
        if (j >= 0 && j < nt) pk[sidx * nt + j] = (uint8_t)poisson_k(wd[w], nd, thr);
      }
    }
  };

  // record r of the delay-ordered rows: block-local target and weight (BF16: one packed u32)
  auto load_record = [&](unsigned long long r, bool ok, uint32_t& key, float& wv) {
    key = 0xffffffffu;
    wv = 0.0f;
    if (!ok) return;
    if constexpr (kBf16) {
      const uint32_t x = reinterpret_cast<const uint32_t*>(a.dw)[r];
      key = x & 0xffffu;
      wv = __bfloat162float(__ushort_as_bfloat16((unsigned short)(x >> 16)));
    } else {
      key = a.dtgt[r];
      wv = reinterpret_cast<const float*>(a.dw)[r];
    }
  };

  // ================= delivery of arrival steps Ta .. Ta + Wd - 1 into acc[0 .. Wd) =================
  auto deliver = [&](const long long Ta, const int Wd) {
    for (int q = tid; q < Wd * nt; q += blockDim.x) acc[q] = 0.0f;
    // emission steps whose spikes arrive in the window: e = T - d, d in [d_min, d_max]
    const long long e_lo = Ta - d_max, e_hi = Ta + Wd - 1 - d_min;
    const int n_e = (int)(e_hi - e_lo + 1);
    const int E = n_e * nb;  // < ncnt
    for (int q = tid; q < E; q += blockDim.x) {
      const long long e = e_lo + q / nb;
      ecnt[q] = e >= 0 ? __ldcg(a.hist_cnt + (int64_t)(e % H) * a.n_blocks + first_block + (q % nb)) : 0u;
    }
    __syncthreads();
    {
      // exclusive prefix of the counts in (emission step, block) order: ecnt[q] = position of the
      // first spike of (step, block) q in the window's list, ecnt[E] = spikes of the list
      const int per = (E + (int)blockDim.x - 1) / (int)blockDim.x;
      const int q0 = min(tid * per, E), q1 = min(q0 + per, E);
      uint32_t loc = 0;
      for (int q = q0; q < q1; ++q) loc += ecnt[q];
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
      for (int q = q0; q < q1; ++q) {
        const uint32_t c = ecnt[q];
        ecnt[q] = run;
        run += c;
      }
      if (tid == 0) ecnt[E] = wcnt[n_warps - 1];
      __syncthreads();
    }
    const uint32_t S_tot = ecnt[E];
    const int n_fold = min(Wd, n_warps);  // ordered fold: warps folding one arrival step each

    // the spike list in chunks of kDIdCap ids (ascending emission step, then id)
    for (uint32_t g0 = 0; g0 < S_tot; g0 += (uint32_t)kDIdCap) {
      const uint32_t g1 = min(S_tot, g0 + (uint32_t)kDIdCap), n_ids = g1 - g0;
      for (int q = tid; q < E; q += blockDim.x) {
        const uint32_t o = ecnt[q], c = ecnt[q + 1] - o;
        if (o >= g1 || o + c <= g0) continue;
        const int ei = q / nb, b = q - ei * nb;
        const long long e = e_lo + ei;
        const uint32_t* src = a.hist_ids + (int64_t)(e % H) * a.n_total + neuron_base + (int64_t)b * tb_full;
        const uint32_t k0 = o < g0 ? g0 - o : 0u, k1 = min(c, g1 - o);
        for (uint32_t k = k0; k < k1; ++k) {
          const uint32_t id = __ldcg(src + k);
          ids_s[o + k - g0] = id;
          ide_s[o + k - g0] = (uint16_t)ei;
        }
      }
      __syncthreads();

      // Order-free fold: the loads of a piece (its table entries and row start).  Lanes hold the
      // pieces of a spike for consecutive arrival steps, i.e. consecutive delays, whose
      // table entries are adjacent: a piece's end is the next lane's start, unless the next lane is
      // another spike, the next group, or past d_max (then the lane loads it too).
      struct PieceLoad {
        uint32_t lo, hi;
        unsigned long long row;
        bool in, own_end;
        int ti;
      };
      auto piece_issue = [&](uint32_t gq, int ti, bool valid) {
        PieceLoad pl;
        pl.lo = pl.hi = 0;
        pl.row = 0;
        pl.in = pl.own_end = false;
        pl.ti = ti;
        if (valid) {
          const uint32_t s = ids_s[gq];
          const long long e = e_lo + ide_s[gq];
          const int dly = (int)(Ta + ti - e);
          if (dly >= d_min && dly <= d_max) {
            pl.in = true;
            pl.own_end = ti == Wd - 1 || lane == 31 || dly == d_max;
            const int64_t tb = tbl_net + (int64_t)s * tbl_stride + (int64_t)wk.group * n_del1 + (dly - d_min);
            pl.lo = a.dtbl[tb];
            if (pl.own_end) pl.hi = a.dtbl[tb + 1];
            pl.row = __ldg(a.row_base + row_off + s);
          }
        }
        return pl;
      };

      // One group of up to 32 pieces per warp pass: lane p holds piece p (its first record, length
      // and arrival step index); the nonempty pieces are packed to the low lanes and their lengths
      // scanned; then 32-entry chunks of the concatenated pieces, each lane finding its piece from
      // the starts that fall inside the chunk.
      auto fold_run = [&](uint32_t len, unsigned long long rec, int tix, float* acc_t_fixed, uint8_t* wtags) {
        const uint32_t ne = __ballot_sync(0xffffffffu, len > 0);
        const int n_ne = __popc(ne);
        if (n_ne == 0) return;
        const int src_lane = lane < n_ne ? nth_set_bit(ne, lane) : 0;
        uint32_t c_len = __shfl_sync(0xffffffffu, len, src_lane);
        const unsigned long long c_rec = __shfl_sync(0xffffffffu, rec, src_lane);
        const int c_ti = __shfl_sync(0xffffffffu, tix, src_lane);
        if (lane >= n_ne) c_len = 0;
        uint32_t c_end = c_len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, c_end, o);
          if (lane >= o) c_end += y;
        }
        const uint32_t c_start = c_end - c_len;
        const uint32_t total = __shfl_sync(0xffffffffu, c_end, 31);
        const uint32_t lanes_le = lanemask_lt() | (1u << lane);
        int cur = -1;
        // the segment of lane entry cb + lane: pieces starting inside the chunk [cb, cb + 32) are
        // marked in one word; the lane's piece is the last one starting at or before it
        auto segment = [&](uint32_t cb, uint32_t& st, unsigned long long& rb, int& sti) {
          const uint32_t bits = (lane < n_ne && c_start - cb < 32u) ? (1u << (c_start - cb)) : 0u;
          const uint32_t sm = __reduce_or_sync(0xffffffffu, bits);
          const int seg = (cur + __popc(sm & lanes_le)) & 31;
          cur += __popc(sm);
          st = __shfl_sync(0xffffffffu, c_start, seg);
          rb = __shfl_sync(0xffffffffu, c_rec, seg);
          sti = __shfl_sync(0xffffffffu, c_ti, seg);
        };
        if constexpr (kExact) {
          // four chunks at a time: every record load of the four is issued before the first add
          for (uint32_t cb0 = 0; cb0 < total; cb0 += 128) {
            unsigned long long r[4];
            int sti[4];
            bool ok[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t cb = cb0 + 32u * (uint32_t)u;
              ok[u] = false;
              r[u] = 0;
              sti[u] = 0;
              if (cb < total) {  // warp-uniform
                uint32_t st;
                unsigned long long rb;
                segment(cb, st, rb, sti[u]);
                const uint32_t q = cb + lane;
                ok[u] = q < total;
                r[u] = rb + (q - st);
              }
            }
            uint32_t key[4];
            float wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              load_record(r[u], ok[u], key[u], wv[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (key[u] == 0xffffffffu) continue;
              if (key[u] >= (uint32_t)nt) {  // not a target of this block: a layout error, recorded
                atomicOr(a.err, kErrBuild);
                continue;
              }
              ring_add_exact<true>(acc + sti[u] * nt, key[u], wv[u]);
            }
          }
        } else {
          for (uint32_t cb = 0; cb < total; cb += 32) {
            uint32_t st;
            unsigned long long rb;
            int sti;
            segment(cb, st, rb, sti);
            const uint32_t q = cb + lane;
            uint32_t key = 0xffffffffu;
            float wv = 0.0f;
            if (q < total) {
              const unsigned long long r = rb + (q - st);
              load_record(r, true, key, wv);
              if (key >= (uint32_t)nt) {  // not a target of this block: a layout error, recorded
                atomicOr(a.err, kErrBuild);
                key = 0xffffffffu;
              }
            }
            fold_one<true>(acc_t_fixed, wtags, key, wv, lane, false);
          }
        }
      };

      if constexpr (kExact) {
        // every (spike, arrival step) piece, in any order, by every warp
        const uint32_t n_pc = n_ids * (uint32_t)Wd;
        for (uint32_t p0 = (uint32_t)warp * 32u; p0 < n_pc; p0 += (uint32_t)n_warps * 32u) {
          const uint32_t p = p0 + (uint32_t)lane;
          const PieceLoad pl = piece_issue(p / (uint32_t)Wd, (int)(p % (uint32_t)Wd), p < n_pc);
          const uint32_t lo_next_lane = __shfl_down_sync(0xffffffffu, pl.lo, 1);
          const uint32_t len = pl.in ? (pl.own_end ? pl.hi : lo_next_lane) - pl.lo : 0u;
          const unsigned long long rec = pl.in ? (unsigned long long)rec_net + pl.row + pl.lo : 0ull;
          fold_run(len, rec, pl.ti, nullptr, nullptr);
        }
      } else {
        // warp f folds arrival steps ti = f, f + n_fold, ...: its pieces in stream order
        if (warp < n_fold) {
          for (int ti = warp; ti < Wd; ti += n_fold) {
            float* acc_t = acc + ti * nt;
            uint8_t* wtags = tags + (size_t)warp * tb_full;
            for (uint32_t p0 = 0; p0 < n_ids; p0 += 32u) {
              const uint32_t gq = p0 + (uint32_t)lane;
              uint32_t len = 0;
              unsigned long long rec = 0;
              if (gq < n_ids) {
                const uint32_t s = ids_s[gq];
                const long long e = e_lo + ide_s[gq];
                const int dly = (int)(Ta + ti - e);
                if (dly >= d_min && dly <= d_max) {
                  const int64_t tb = tbl_net + (int64_t)s * tbl_stride + (int64_t)wk.group * n_del1 + (dly - d_min);
                  const uint32_t lo = a.dtbl[tb], hi = a.dtbl[tb + 1];
                  len = hi - lo;
                  rec = (unsigned long long)rec_net + __ldg(a.row_base + row_off + s) + lo;
                }
              }
              fold_run(len, rec, ti, acc_t, wtags);
            }
          }
        }
      }
      __syncthreads();
    }
  };

  const int tw_u = (nt + n_warps - 1) / n_warps;  // update split over the warps
  bool pend = false;  // the I half of the previous window's last step is due
  poisson_fill(t_start - 1, min(W, a.n_steps));
  // the first window's I halves (steps t_start .. t_start + W - 2; acc[0], step t_start - 1, was
  // completed by the previous launch and is not used) need spikes up to t_start - 1 only
  __syncthreads();
  deliver(t_start - 1, min(W, a.n_steps));
  int done = 0;
  while (done < a.n_steps) {
    const int Wn = min(W, a.n_steps - done);
    const long long t0 = t_start + done;

    // ================= update + compaction + spike buffer =================
    for (int ws = 0; ws < Wn; ++ws) {
      const long long t = t0 + ws;
      const bool prev = ws > 0 || pend;  // the I half of step t - 1 is due
      const int lo = warp * tw_u, hi = min(lo + tw_u, nt);
      const float* in_t = acc + ws * nt;
      uint32_t cw = 0;
      for (int c = lo; c < hi; c += 32) {
        const int j = c + lane;
        bool spk = false;
        if (j < hi) {
          float v = sV[j], cur = sI[j];
          int32_t r = sR[j];
          if (prev) i_half_k(cur, in_t[j], pk[ws * nt + j], nd);
          spk = v_half(v, cur, r, nd);
          sV[j] = v;
          sI[j] = cur;
          sR[j] = (int16_t)r;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, spk);
        if (spk) wlist[lo + cw + __popc(bal & lanemask_lt())] = (uint16_t)j;
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
      const int slot = (int)(t % H);
      uint32_t* dst = a.hist_ids + (int64_t)slot * a.n_total + neuron_base + (int64_t)wk.group * tb_full;
      for (uint32_t q = lane; q < cw; q += 32) {
        const uint32_t id = (uint32_t)wk.t0 + wlist[lo + q];
        dst[before + q] = id;
        my_events += a.dtbl[tbl_net + (int64_t)id * tbl_stride + tbl_last];  // out-degree of the spike
      }
      if (tid == 0) a.hist_cnt[(int64_t)slot * a.n_blocks + blk] = total;
      __syncthreads();
    }
    pend = true;

    // ================= grid barrier among the blocks of this network =================
    // Every thread's spike-buffer writes are ordered before thread 0's fence by the block barrier;
    // the fence makes them visible to the GPU before the arrival is counted.  Readers load the
    // spike buffer bypassing L1 (__ldcg), so they see them after observing the count.
    const int remaining = a.n_steps - done - Wn;
    const int Wd = max(1, min(W, remaining));  // arrival steps to deliver: the next window's I halves
    {
      if (tid == 0 && blk != a.withhold_block) {
        __threadfence();
        atomicAdd(a.bar_count + wk.net, 1ull);
      }
      // the next window's Poisson table (its first entry is this window's last step) needs nothing
      // from the other blocks
      poisson_fill(t0 + Wn - 1, Wd);
      int fail = 0;
      if (tid == 0) {
        const unsigned long long want = (unsigned long long)(epoch + 1u) * (unsigned long long)nb;
        const long long tb0 = global_ns();
        uint32_t spins = 0;
        while (ld_acquire_u64(a.bar_count + wk.net) < want) {
          if ((++spins & 255u) == 0 && (global_ns() - tb0 > a.timeout_ns || *(volatile int32_t*)a.err != 0)) {
            fail = 1;
            break;
          }
        }
      }
      if (__syncthreads_or(fail)) {
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        aborted = true;
        break;
      }
      epoch += 1u;
    }

    // ================= raster: the block's own spikes of the window =================
    if (a.raster_step != nullptr) {
      for (int q = tid; q < Wn * nb; q += blockDim.x) {
        const int ws = q / nb, b = q - ws * nb;
        ecnt[q] = __ldcg(a.hist_cnt + (int64_t)((t0 + ws) % H) * a.n_blocks + first_block + b);
      }
      __syncthreads();
      // warp ws: the spikes of step t0 + ws in blocks before this one, and in all blocks
      for (int ws = warp; ws < Wn; ws += n_warps) {
        uint32_t before = 0, tot = 0;
        for (int b = lane; b < nb; b += 32) {
          const uint32_t x = ecnt[ws * nb + b];
          before += b < wk.group ? x : 0u;
          tot += x;
        }
        before = __reduce_add_sync(0xffffffffu, before);
        tot = __reduce_add_sync(0xffffffffu, tot);
        if (lane == 0) {
          ecnt[ncnt - 2 * (ws + 1)] = before;  // past the counts (Wn * nb + 2 Wn <= ncnt)
          ecnt[ncnt - 2 * (ws + 1) + 1] = tot;
        }
      }
      __syncthreads();
      unsigned long long pos0 = raster_total;
      for (int ws = 0; ws < Wn; ++ws) {
        const uint32_t before = ecnt[ncnt - 2 * (ws + 1)], tot = ecnt[ncnt - 2 * (ws + 1) + 1];
        const uint32_t mine = ecnt[ws * nb + wk.group];
        const uint32_t* src = a.hist_ids + (int64_t)((t0 + ws) % H) * a.n_total + neuron_base + (int64_t)wk.group * tb_full;
        for (uint32_t q = tid; q < mine; q += blockDim.x) {
          const unsigned long long p = pos0 + before + q;
          if ((long long)p < raster_cap) {
            a.raster_step[raster_base + p] = (int32_t)(t0 + ws);
            a.raster_id[raster_base + p] = (int32_t)__ldcg(src + q);
          } else {
            atomicOr(a.err, kErrRaster);
          }
        }
        pos0 += tot;
      }
      raster_total = pos0;
      __syncthreads();
    }

    deliver(t0 + Wn - 1, Wd);
    done += Wn;
  }

  // ---- epilogue: the pending I half of the last step (accumulator 0), then write back ----
  __syncthreads();
  if (pend && !aborted) {
    for (int j = tid; j < nt; j += blockDim.x) {
      float cur = sI[j];
      i_half_k(cur, acc[j], pk[j], nd);  // pk[0] holds the last step (filled at the last barrier)
      sI[j] = cur;
    }
    __syncthreads();
  }
  for (int j = tid; j < nt; j += blockDim.x) {
    a.V[nbase + j] = sV[j];
    a.I[nbase + j] = sI[j];
    a.R[nbase + j] = sR[j];
  }
  if (my_events) atomicAdd(a.events + wk.net, my_events);
  if (wk.group == 0 && tid == 0 && a.raster_step != nullptr && !aborted) a.raster_count[wk.net] = raster_total;
  if (blk == 0 && tid == 0 && !aborted) *a.step_counter = t_start + a.n_steps;
  if (tid == 0 && !aborted) a.pub_flag[blk] = epoch;  // windows completed, for the next launch
}

using DStepKernel = void (*)(StepArgs);
DStepKernel dstep_kernel(bool bf16, bool exact, int threads) {
  const bool wide = threads > 16 * 32;
  if (wide)
    return bf16 ? (exact ? k_dstep<true, true, true> : k_dstep<true, false, true>)
                : (exact ? k_dstep<false, true, true> : k_dstep<false, false, true>);
  return bf16 ? (exact ? k_dstep<true, true, false> : k_dstep<true, false, false>)
              : (exact ? k_dstep<false, true, false> : k_dstep<false, false, false>);
}

cudaError_t launch_dstep(const StepArgs& a, int grid, int threads, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // the blocks of a network wait on each other
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, dstep_kernel(a.bf16 != 0, a.exact != 0, threads), a);
}

size_t dstep_smem_bytes(int nt, int window, int nb, int d_max, int n_warps, bool exact) {
  return make_dlayout(nt, window, n_warps, exact, dcount_words(d_max, nb)).total;
}

cudaError_t dstep_kernel_attributes(size_t smem) {
  for (int v = 0; v < 8; ++v) {
    const DStepKernel k = dstep_kernel((v & 1) != 0, (v & 2) != 0, (v & 4) ? kDMaxWarps * 32 : 32);
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int dstep_occupancy(int threads, size_t smem) {
  int n = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dstep_kernel(false, false, threads), threads, smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace cortex
