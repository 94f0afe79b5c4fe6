// step.cu -- the per-step hot path: neuron update, spike compaction, spike publication, grid
// barrier, and spike delivery over the indegree sub-graphs.
//
// Every block owns a contiguous range of post-synaptic neurons and all of their incoming synapses
// (Eq. 5, Eq. 9-10).  Inside the block every warp owns a contiguous sub-range of those neurons
// (Sec. III-B, "each synaptic interaction and its post-synaptic neuron should be accessed by a
// specific thread only").  A spike from source s is read as the block's (s) segment -- contiguous
// records sorted by target -- and each warp folds its own piece of it into the ring buffer of its
// neurons.  Different warps never touch the same ring cell; inside a warp, equal cells are added
// in lane order.  So every cell receives its weights in the order (emission step, source id,
// draw index) with no atomics and no locks (Eq. 12-14).
//
// One step (Sec. II-B): update all owned neurons (consuming the ring slot of this step), compact
// the spikes into the block's ascending list, publish it; every W = d_min steps (the window) the
// blocks of a network meet at a barrier and deliver the window's spikes, which land at least d_min
// steps later and so never in a slot the window still reads.
#include "cortex_internal.cuh"

namespace cortex {

struct SmemLayout {
  uint32_t bar, ring, sv, si, sr, thr, cnt, own, wcnt, wlist, sp, stage, total;
};

struct SpikeSlots {
  uint32_t woff[kSpikeBatch];   // staging byte offset of record 0 of the spike's segment, w stream
  uint32_t toff[kSpikeBatch];   // ... target stream
  uint32_t doff[kSpikeBatch];   // ... delay stream
  uint16_t end[kSpikeBatch][kMaxWarps];
  uint32_t n_take;
  uint32_t pad[3];
};

__host__ __device__ inline uint32_t align_to(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout make_layout(int max_nt, int max_depth, int w_max, int max_nb, bool ring_smem,
                                                  int stage_bytes) {
  SmemLayout L;
  uint32_t o = 0;
  L.bar = o;
  o += 16;
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
  L.own = o;
  o += (uint32_t)(w_max * 4);
  o = align_to(o, 16);
  L.wcnt = o;
  o += (kMaxWarps + 2) * 4;
  o = align_to(o, 16);
  L.wlist = o;
  o += max_nt * 4;
  o = align_to(o, 16);
  L.sp = o;
  o += sizeof(SpikeSlots);
  o = align_to(o, 128);
  L.stage = o;
  o += stage_bytes;
  L.total = o;
  return L;
}

// ---- one neuron, one step (Eq. 1-3, exact integration) --------------------------------------
//   in = ring cell of this step (cleared); k = Poisson draw; ext = k * J_ext
//   refractory: V = V_reset, counter - 1;  else V = fma(P22, V, P21 * I) with the old I
//   I = fma(P11, I, in); I = I + ext
//   V >= V_th: spike, V = V_reset, counter = n_ref (Eq. 2)
struct NeuronConst {
  float p11, p21, p22, v_th, v_reset, j_ext;
  int32_t n_ref, n_thr;
};

__device__ __forceinline__ bool update_neuron(float& v, float& cur, int32_t& r, float in, uint32_t u,
                                              const NeuronConst& nd, const uint32_t* thr) {
  int k = 0;
  while (k < nd.n_thr - 1 && u >= thr[k]) ++k;
  const float ext = __fmul_rn((float)k, nd.j_ext);
  if (r > 0) {
    v = nd.v_reset;
    r -= 1;
  } else {
    v = __fmaf_rn(nd.p22, v, __fmul_rn(nd.p21, cur));
  }
  cur = __fmaf_rn(nd.p11, cur, in);
  cur = __fadd_rn(cur, ext);
  const bool spk = v >= nd.v_th;
  if (spk) {
    v = nd.v_reset;
    r = nd.n_ref;
  }
  return spk;
}

__device__ __forceinline__ uint32_t floor16(uint64_t x) { return (uint32_t)(x & 15u); }

// ---- the step kernel ---------------------------------------------------------------------------
// phases: kPhaseUpdate, kPhaseDeliver, and kPhaseBarrier for the persistent form (both phases and
// a barrier per window inside one cooperative launch of n_steps steps).
__global__ void __launch_bounds__(kMaxWarps * 32) k_step(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n_warps = blockDim.x >> 5;
  const int blk = blockIdx.x;
  const BlockWork wk = a.work[blk];
  const NetDev& ndg = a.nets[wk.net];
  NeuronConst nd;
  nd.p11 = ndg.p11; nd.p21 = ndg.p21; nd.p22 = ndg.p22;
  nd.v_th = ndg.v_th; nd.v_reset = ndg.v_reset; nd.j_ext = ndg.j_ext;
  nd.n_ref = ndg.n_ref; nd.n_thr = ndg.n_thr;
  const uint32_t seed_lo = ndg.seed_lo, seed_hi = ndg.seed_hi;
  const int nb = ndg.n_blocks, first_block = ndg.first_block, window = ndg.window;
  const int64_t neuron_base = ndg.neuron_base, raster_base = ndg.raster_base, raster_cap = ndg.raster_cap;
  const int D = ndg.depth;
  const int nt = wk.nt, tw = wk.tw;
  const bool persistent = (a.phases & kPhaseBarrier) != 0;
  const bool do_update = (a.phases & kPhaseUpdate) != 0;
  const bool do_deliver = (a.phases & kPhaseDeliver) != 0;
  const bool ring_smem = a.ring_smem != 0;
  const bool bf16 = ndg.wdtype == 1;
  const uint32_t wsz = bf16 ? 2u : 4u;

  // same layout arithmetic as the host (maxima passed through stage_bytes and the work table)
  const SmemLayout L = make_layout(a.max_nt, a.max_depth, a.w_max, a.max_nb, ring_smem, a.stage_bytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  float* ring_s = reinterpret_cast<float*>(smem + L.ring);
  float* sV = reinterpret_cast<float*>(smem + L.sv);
  float* sI = reinterpret_cast<float*>(smem + L.si);
  int32_t* sR = reinterpret_cast<int32_t*>(smem + L.sr);
  uint32_t* thr = reinterpret_cast<uint32_t*>(smem + L.thr);
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + L.cnt);
  uint32_t* own_cnt = reinterpret_cast<uint32_t*>(smem + L.own);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + L.wcnt);
  uint32_t* wlist = reinterpret_cast<uint32_t*>(smem + L.wlist);
  SpikeSlots* sp = reinterpret_cast<SpikeSlots*>(smem + L.sp);
  unsigned char* stage = smem + L.stage;

  float* ring_g = a.ring + wk.ring_base;
  const int64_t nbase = neuron_base + wk.t0;

  // ---- prologue: state, thresholds, ring slice, barrier object ----
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int q = tid; q < kPoissonCap; q += blockDim.x) thr[q] = ndg.thr[q];
  if (do_update) {
    for (int j = tid; j < nt; j += blockDim.x) {
      sV[j] = a.V[nbase + j];
      sI[j] = a.I[nbase + j];
      sR[j] = a.R[nbase + j];
    }
  }
  if (ring_smem) {
    for (int q = tid; q < D * nt; q += blockDim.x) ring_s[q] = ring_g[q];
  }
  const long long t_start = (a.t_fixed >= 0) ? a.t_fixed : *a.step_counter;
  uint32_t epoch = persistent ? ld_cg_u32(a.pub_flag + blk) : 0u;
  unsigned long long raster_total = a.raster_count[wk.net];
  unsigned long long my_events = 0;
  uint32_t mbar_phase = 0;
  bool aborted = false;
  __shared__ int s_abort;
  if (tid == 0) s_abort = 0;
  __syncthreads();

  const int W = persistent ? window : min(window, a.n_steps);
  int done = 0;
  while (done < a.n_steps && !aborted) {
    const int Wn = min(W, a.n_steps - done);
    const long long t0 = t_start + done;
    const uint32_t par = persistent ? ((epoch + 1u) & 1u) : 0u;

    // ================= update + compaction + publication =================
    if (do_update) {
      for (int ws = 0; ws < Wn; ++ws) {
        const long long t = t0 + ws;
        const int slot = (int)(t % D);
        float* rs = ring_smem ? ring_s + slot * nt : ring_g + (int64_t)slot * nt;
        const int lo = warp * tw, hi = min(lo + tw, nt);
        uint32_t cw = 0;
        for (int c = lo; c < hi; c += 32) {
          const int j = c + lane;
          bool spk = false;
          if (j < hi) {
            const float in = rs[j];
            rs[j] = 0.0f;
            const uint4 rr = philox4x32_10(make_uint4((uint32_t)(wk.t0 + j), (uint32_t)t, kStreamPoisson, 0u),
                                           seed_lo, seed_hi);
            float v = sV[j], cur = sI[j];
            int32_t r = sR[j];
            spk = update_neuron(v, cur, r, in, rr.x, nd, thr);
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
        if (tid == 0) own_cnt[ws] = total;
        __syncthreads();
      }
      if (tid < Wn) a.pub_cnt[(int64_t)(par * a.w_max + tid) * a.n_blocks + blk] = own_cnt[tid];
      __syncthreads();
      if (persistent && tid == 0) {
        __threadfence();
        st_release_u32(a.pub_flag + blk, epoch + 1u);
      }
    }

    // ================= grid barrier among the blocks of this network =================
    if (persistent) {
      epoch += 1u;
      if (warp == 0) {
        const long long t_begin = global_ns();
        bool ok = true;
        for (int b = lane; b < nb && ok; b += 32) {
          const uint32_t* f = a.pub_flag + first_block + b;
          uint32_t spins = 0;
          while ((int32_t)(ld_acquire_u32(f) - epoch) < 0) {
            if ((++spins & 255u) == 0) {
              if (global_ns() - t_begin > a.timeout_ns || *(volatile int32_t*)a.err != 0) {
                ok = false;
                break;
              }
            }
          }
        }
        const bool all_ok = __all_sync(0xffffffffu, ok);
        if (!all_ok && lane == 0) {
          atomicOr(a.err, kErrTimeout);
          s_abort = 1;
        }
      }
      __syncthreads();
      if (s_abort) {
        aborted = true;
        break;
      }
    }

    // ================= delivery =================
    if (do_deliver) {
      // counts of every block of this network for the window, then exclusive prefixes
      for (int q = tid; q < Wn * nb; q += blockDim.x) {
        const int ws = q / nb, b = q % nb;
        cnt_s[ws * (nb + 1) + b] = ld_cg_u32(a.pub_cnt + (int64_t)(par * a.w_max + ws) * a.n_blocks + first_block + b);
      }
      __syncthreads();
      if (warp < Wn) {
        uint32_t* c = cnt_s + warp * (nb + 1);
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

      for (int ws = 0; ws < Wn; ++ws) {
        const long long t_emit = t0 + ws;
        const int tm = (int)(t_emit % D);
        const uint32_t* pref = cnt_s + ws * (nb + 1);
        const uint32_t S = pref[nb];
        const uint32_t* ids = a.pub_ids + (int64_t)(par * a.w_max + ws) * a.n_total + neuron_base;
        // raster: this block's own spikes, at (spikes so far) + (spikes of lower blocks this step)
        if (a.raster_step != nullptr) {
          const uint32_t mine = pref[wk.group + 1] - pref[wk.group];
          const unsigned long long pos0 = raster_total + pref[wk.group];
          for (uint32_t q = tid; q < mine; q += blockDim.x) {
            const unsigned long long pos = pos0 + q;
            if ((long long)pos < raster_cap) {
              a.raster_step[raster_base + pos] = (int32_t)t_emit;
              a.raster_id[raster_base + pos] = (int32_t)ld_cg_u32(ids + wk.t0 + q);
            } else if (q == 0) {
              atomicOr(a.err, kErrRaster);
            }
          }
        }
        raster_total += S;

        for (uint32_t sb = 0; sb < S;) {
          // -- warp 0: fetch the headers of up to 32 spikes and stage their record segments --
          if (warp == 0) {
            const uint32_t q = sb + lane;
            uint32_t hw[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            uint32_t seg_len = 0;
            if (q < S) {
              int lo = 0, hi = nb;  // last block b with pref[b] <= q
              while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pref[mid] <= q) lo = mid;
                else hi = mid;
              }
              const int64_t tb = a.work[first_block].nt;
              const uint32_t src = ld_cg_u32(ids + lo * tb + (q - pref[lo]));
              const uint4* hp = a.hdr + 2 * (wk.hdr_base + src);
              const uint4 h0 = __ldg(hp), h1 = __ldg(hp + 1);
              hw[0] = h0.x; hw[1] = h0.y; hw[2] = h0.z; hw[3] = h0.w;
              hw[4] = h1.x; hw[5] = h1.y; hw[6] = h1.z; hw[7] = h1.w;
              seg_len = hw[7] >> 16;
            }
            const uint64_t r0 = (uint64_t)wk.rec_base + hw[0];
            // byte ranges of the three streams, widened to 16-byte boundaries
            const uint64_t wb0 = r0 * wsz, wb1 = (r0 + seg_len) * wsz;
            const uint64_t tb0 = r0 * 2u, tb1 = (r0 + seg_len) * 2u;
            const uint64_t db0 = r0, db1 = r0 + seg_len;
            const uint32_t wsz16 = seg_len ? (uint32_t)(((wb1 + 15) & ~15ull) - (wb0 & ~15ull)) : 0u;
            const uint32_t tsz16 = seg_len ? (uint32_t)(((tb1 + 15) & ~15ull) - (tb0 & ~15ull)) : 0u;
            const uint32_t dsz16 = seg_len ? (uint32_t)(((db1 + 15) & ~15ull) - (db0 & ~15ull)) : 0u;
            const uint32_t need = wsz16 + tsz16 + dsz16;
            uint32_t incl = need;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= o) incl += y;
            }
            // the staged spikes are the longest prefix whose segments fit (incl grows with the
            // lane, so the fitting lanes are lanes 0..n_fit-1).  The host sizes the staging area to
            // hold the longest segment, so n_fit >= 1; if not, the spike is skipped and flagged.
            const uint32_t fits = __ballot_sync(0xffffffffu, q < S && incl <= (uint32_t)a.stage_bytes);
            const uint32_t n_fit = (uint32_t)__popc(fits);
            const uint32_t n_valid = n_fit ? n_fit : 1u;
            const bool oversize = (n_fit == 0);
            if (oversize && lane == 0) atomicOr(a.err, kErrSegment);
            if (lane < (int)n_valid) {
              const uint32_t off = incl - need;
              sp->woff[lane] = off + floor16(wb0);
              sp->toff[lane] = off + wsz16 + floor16(tb0);
              sp->doff[lane] = off + wsz16 + tsz16 + floor16(db0);
#pragma unroll
              for (int w = 0; w < kMaxWarps; ++w) {
                const uint32_t word = hw[1 + (w >> 1)];
                sp->end[lane][w] = oversize ? (uint16_t)0 : (uint16_t)((w & 1) ? (word >> 16) : (word & 0xffffu));
              }
              if (seg_len && !oversize) {
                fence_proxy_async_smem();
                const unsigned char* gw = reinterpret_cast<const unsigned char*>(a.rec_w) + (wb0 & ~15ull);
                const unsigned char* gt = reinterpret_cast<const unsigned char*>(a.rec_tgt) + (tb0 & ~15ull);
                const unsigned char* gd = reinterpret_cast<const unsigned char*>(a.rec_dly) + (db0 & ~15ull);
                bulk_g2s(stage + off, gw, wsz16, bar);
                bulk_g2s(stage + off + wsz16, gt, tsz16, bar);
                bulk_g2s(stage + off + wsz16 + tsz16, gd, dsz16, bar);
              }
            }
            const uint32_t total_bytes = oversize ? 0u : __shfl_sync(0xffffffffu, incl, (int)n_valid - 1);
            if (lane == 0) {
              mbar_arrive_expect_tx(bar, total_bytes);
              sp->n_take = n_valid;
            }
          }
          __syncthreads();
          const uint32_t n_take = sp->n_take;
          // -- everyone waits for the staged records --
          {
            const long long tw0 = global_ns();
            uint32_t spins = 0;
            while (!mbar_try_wait(bar, mbar_phase)) {
              if ((++spins & 1023u) == 0 && global_ns() - tw0 > a.timeout_ns) {
                if (lane == 0) atomicOr(a.err, kErrTimeout);
                break;
              }
            }
            mbar_phase ^= 1u;
          }
          // -- every warp folds its own target sub-range of each staged segment, in spike order --
          {
            uint32_t lo_k = 0, len_k = 0;
            if (lane < (int)n_take) {
              const uint32_t e1 = sp->end[lane][warp];
              const uint32_t e0 = warp ? sp->end[lane][warp - 1] : 0u;
              lo_k = e0;
              len_k = e1 - e0;
            }
            const uint32_t ne = __ballot_sync(0xffffffffu, len_k > 0);
            const int n_ne = __popc(ne);
            // compacted position c (0..n_ne-1) -> spike slot
            const int src_lane = (lane < n_ne) ? (int)__fns(ne, 0, lane + 1) : 0;
            const uint32_t c_lo = __shfl_sync(0xffffffffu, lo_k, src_lane);
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
            my_events += (lane == 0) ? total : 0u;
            int cur = -1;
            for (uint32_t e = 0; e < total; e += 32) {
              const uint32_t bits = (lane < n_ne && c_start >= e && c_start < e + 32) ? (1u << (c_start - e)) : 0u;
              const uint32_t startmask = __reduce_or_sync(0xffffffffu, bits);
              const int seg = cur + __popc(startmask & (0xffffffffu >> (31 - lane)));
              cur += __popc(startmask);
              const uint32_t q = e + lane;
              const bool valid = q < total;
              const int sl = seg & 31;
              const int sk = __shfl_sync(0xffffffffu, src_lane, sl);
              const uint32_t sstart = __shfl_sync(0xffffffffu, c_start, sl);
              const uint32_t slo = __shfl_sync(0xffffffffu, c_lo, sl);
              uint32_t key = 0xffffffffu;
              float wv = 0.0f;
              if (valid) {
                const uint32_t m = slo + (q - sstart);
                const uint32_t tgt = *reinterpret_cast<const uint16_t*>(stage + sp->toff[sk] + 2u * m);
                const uint32_t dl = stage[sp->doff[sk] + m];
                wv = bf16 ? __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(stage + sp->woff[sk] + 2u * m))
                          : *reinterpret_cast<const float*>(stage + sp->woff[sk] + 4u * m);
                int slot = tm + (int)dl;
                if (slot >= D) slot -= D;
                key = (uint32_t)slot * (uint32_t)nt + tgt;
              }
              const uint32_t peers = __match_any_sync(0xffffffffu, key);
              const int rank = __popc(peers & lanemask_lt());
              const int maxrank = __reduce_max_sync(0xffffffffu, valid ? rank : 0);
              for (int rr = 0; rr <= maxrank; ++rr) {
                if (valid && rank == rr) {
                  float* cell = ring_smem ? ring_s + key : ring_g + key;
                  *cell = __fadd_rn(*cell, wv);
                }
                __syncwarp();
              }
            }
          }
          __syncthreads();
          sb += n_take;
        }
      }
    }
    done += Wn;
  }

  // ---- epilogue: write back state and ring, counters ----
  __syncthreads();
  if (do_update) {
    for (int j = tid; j < nt; j += blockDim.x) {
      a.V[nbase + j] = sV[j];
      a.I[nbase + j] = sI[j];
      a.R[nbase + j] = sR[j];
    }
  }
  if (ring_smem) {
    for (int q = tid; q < D * nt; q += blockDim.x) ring_g[q] = ring_s[q];
  }
  // warp sums of events -> one atomic per block
  if (lane == 0 && my_events) atomicAdd(a.events + wk.net, my_events);
  if (persistent && do_deliver && wk.group == 0 && tid == 0 && a.raster_step != nullptr)
    a.raster_count[wk.net] = raster_total;
  if (persistent && blk == 0 && tid == 0 && a.t_fixed < 0 && !aborted) *a.step_counter = t_start + a.n_steps;
}

// split mode: advance the step counter and the per-network spike totals after a window
__global__ void k_advance(const StepArgs a, int n_nets, int wn) {
  const int net = blockIdx.x * blockDim.x + threadIdx.x;
  if (net < n_nets) {
    const NetDev nd = a.nets[net];
    unsigned long long s = 0;
    for (int ws = 0; ws < wn; ++ws)
      for (int b = 0; b < nd.n_blocks; ++b) s += a.pub_cnt[(int64_t)ws * a.n_blocks + nd.first_block + b];
    a.raster_count[net] += s;
  }
  if (net == 0) *a.step_counter += wn;
}

cudaError_t launch_step(const StepArgs& a, int grid, int threads, size_t smem, bool cooperative, cudaStream_t s) {
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
    return cudaLaunchKernelEx(&cfg, k_step, a);
  }
  k_step<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_advance_split(const StepArgs& a, int n_nets, int wn, cudaStream_t s) {
  k_advance<<<(n_nets + 127) / 128, 128, 0, s>>>(a, n_nets, wn);
  return cudaGetLastError();
}

size_t step_smem_bytes(int max_nt, int max_depth, int w_max, int max_nb, bool ring_smem, int stage_bytes) {
  return make_layout(max_nt, max_depth, w_max, max_nb, ring_smem, stage_bytes).total;
}

cudaError_t step_kernel_attributes(size_t smem) {
  return cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int step_occupancy(int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step, threads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace cortex
