// build.cu -- one-time device work: propagators (FP64), initial state, and the network builder
// that turns Philox draws into per-block sub-graphs stored as CSR by source (Eq. 5, Eq. 9-10,
// Sec. III-B: each block owns a contiguous range of post-synaptic neurons and all of their
// incoming synapses; inside the block the synapses of one source are contiguous and sorted by
// target, hence by owning warp).
//
// Builder passes for a wave of blocks of one network:
//   count     every (target, draw) increments cnt[block][source]              (integer atomics)
//   scan      cursor[block][*] = exclusive prefix of cnt[block][*]
//   fill      key = (local target << 16 | draw) placed at cursor[block][source]++
//   finalize  one warp per (block, source) segment: sort the keys, regenerate source and delay
//             from Philox, write the SoA records and the segment header
#include <algorithm>
#include "cortex_internal.cuh"

namespace cortex {

// ---- propagators and Poisson thresholds (FP64, once) ----------------------------------------
// Exact integration of Eq. 1 with an exponential current (Eq. 3 as a current synapse):
//   P22 = exp(-h/tau_m), P11 = exp(-h/tau_syn), P21 = tau_m tau_syn / (C (tau_syn - tau_m)) (P11 - P22)
// The neuron update uses P22 - 1 = expm1(-h/tau_m) (V + ((P22 - 1) V + P21 I)): P22 is within 1% of 1,
// so P22 itself would carry a float rounding that the stationary potential amplifies by 1/(1 - P22).
// Poisson(lambda = nu_ext dt) thresholds thr[k] = floor(2^32 P(X <= k)), saturating at 2^32 - 1.
__global__ void k_props(NetDev* nets, int n_nets) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_nets) return;
  NetDev& d = nets[b];
  const double h = (double)d.dt, tm = (double)d.tau_m, ts = (double)d.tau_syn, c = (double)d.c_m;
  const double p22 = exp(-h / tm);
  const double p11 = exp(-h / ts);
  const double p21 = tm * ts / (c * (ts - tm)) * (p11 - p22);
  d.p11 = (float)p11;
  d.p21 = (float)p21;
  d.p22m1 = (float)expm1(-h / tm);
  d.n_ref = (int32_t)llround((double)d.t_ref / h);
  const double lam = (double)d.nu_ext_hz * (double)d.dt / 1000.0;
  double pmf = exp(-lam), cdf = pmf;
  int n = -1;
  for (int k = 0; k < kPoissonCap; ++k) {
    if (k > 0) {
      pmf = pmf * lam / (double)k;
      cdf = cdf + pmf;
    }
    const double x = cdf * 4294967296.0;
    if (x >= 4294967295.0) {
      d.thr[k] = 0xffffffffu;
      n = k + 1;
      break;
    }
    d.thr[k] = (uint32_t)floor(x);
  }
  d.n_thr = n;  // -1: table did not saturate (rejected by the host)
  if (d.wdtype == 1) {
    d.w_exc = __bfloat162float(__float2bfloat16_rn(d.j_exc_in));
    d.w_inh = __bfloat162float(__float2bfloat16_rn(d.j_inh_in));
  } else {
    d.w_exc = d.j_exc_in;
    d.w_inh = d.j_inh_in;
  }
}

cudaError_t launch_props(NetDev* nets, int n_nets, cudaStream_t s) {
  k_props<<<(n_nets + 63) / 64, 64, 0, s>>>(nets, n_nets);
  return cudaGetLastError();
}

// ---- draws ---------------------------------------------------------------------------------
// Draw j of target i: Philox(ctr = (i, j/2, 1, 0), key = seed) gives two draws per call; words
// (x, y) for even j, (z, w) for odd j.  Source from the first word (E for j < K_E, else I),
// delay d_min + floor(word2 * (d_max - d_min + 1) / 2^32).
struct Draw2 {
  uint32_t src[2];
  uint32_t dly[2];
};

__device__ __forceinline__ Draw2 draw_pair(const NetDev& d, uint32_t i, uint32_t pair) {
  const uint4 r = philox4x32_10(make_uint4(i, pair, kStreamConn, 0u), d.seed_lo, d.seed_hi);
  Draw2 out;
  const uint32_t nd = (uint32_t)(d.d_max - d.d_min + 1);
  const uint32_t j0 = 2u * pair, j1 = j0 + 1u;
  out.src[0] = (j0 < (uint32_t)d.k_exc) ? scale32(r.x, (uint32_t)d.n_exc) : (uint32_t)d.n_exc + scale32(r.x, (uint32_t)d.n_inh);
  out.dly[0] = (uint32_t)d.d_min + scale32(r.y, nd);
  out.src[1] = (j1 < (uint32_t)d.k_exc) ? scale32(r.z, (uint32_t)d.n_exc) : (uint32_t)d.n_exc + scale32(r.z, (uint32_t)d.n_inh);
  out.dly[1] = (uint32_t)d.d_min + scale32(r.w, nd);
  return out;
}

// Targets of a wave: [t_lo, t_hi) of the network; block of target i = i / tb.
__global__ void k_count(const NetDev* __restrict__ nets, int net_idx, int32_t t_lo, int32_t t_hi, int32_t tb,
                        int first_group, uint32_t* __restrict__ cnt) {
  const NetDev& d = nets[net_idx];
  const int64_t pairs = (d.k + 1) / 2;
  const int64_t total = (int64_t)(t_hi - t_lo) * pairs;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(t_lo + q / pairs);
    const uint32_t p = (uint32_t)(q % pairs);
    const Draw2 dr = draw_pair(d, i, p);
    const int64_t g = (int64_t)(i / tb) - first_group;
    atomicAdd(&cnt[g * d.n + dr.src[0]], 1u);
    if (2 * p + 1 < (uint32_t)d.k) atomicAdd(&cnt[g * d.n + dr.src[1]], 1u);
  }
}

cudaError_t launch_build_count_net(const NetDev* nets_dev, int net_idx, int32_t n, int first_group, int n_groups,
                                   int32_t tb, uint32_t* cnt, cudaStream_t s) {
  const int32_t t_lo = first_group * tb;
  const int32_t t_hi = min(n, (first_group + n_groups) * tb);
  k_count<<<152 * 8, 256, 0, s>>>(nets_dev, net_idx, t_lo, t_hi, tb, first_group, cnt);
  return cudaGetLastError();
}

// ---- per-block exclusive scan over the sources -------------------------------------------
__global__ void k_scan(const uint32_t* __restrict__ cnt, uint32_t* __restrict__ cursor, int32_t n_src) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  const int64_t base = (int64_t)blockIdx.x * n_src;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int64_t off = 0; off < n_src; off += blockDim.x) {
    const int64_t s = off + threadIdx.x;
    const uint32_t v = (s < n_src) ? cnt[base + s] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = (lane < nwarps) ? warp_sum[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nwarps) warp_sum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0u) + x - v;
    if (s < n_src) cursor[base + s] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nwarps - 1];
    __syncthreads();
  }
}

cudaError_t launch_scan_groups(uint32_t* cnt, uint32_t* cursor, int n_groups, int32_t n_src, uint32_t*, cudaStream_t s) {
  k_scan<<<n_groups, 1024, 0, s>>>(cnt, cursor, n_src);
  return cudaGetLastError();
}

// ---- rows of the CSR by source: per-block offsets inside each row, row starts -------------------
// off[b][s] = sum over blocks b' < b of cnt[b'][s]; rowcnt[s] = sum over all blocks
__global__ void k_colscan(const uint32_t* __restrict__ cnt_all, int nb, int32_t n, uint32_t* __restrict__ off_all,
                          uint32_t* __restrict__ rowcnt) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    uint32_t acc = 0;
    for (int b = 0; b < nb; ++b) {
      off_all[(int64_t)b * n + s] = acc;
      acc += cnt_all[(int64_t)b * n + s];
    }
    rowcnt[s] = acc;
  }
}

// row_base[s] = exclusive prefix of rowcnt over the sources (64-bit), one block
__global__ void k_rowscan(const uint32_t* __restrict__ rowcnt, int32_t n, unsigned long long* __restrict__ row_base) {
  __shared__ unsigned long long warp_sum[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int64_t off = 0; off < n; off += blockDim.x) {
    const int64_t s = off + threadIdx.x;
    const unsigned long long v = (s < n) ? rowcnt[s] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = (lane < nwarps) ? warp_sum[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nwarps) warp_sum[lane] = w;
    }
    __syncthreads();
    if (s < n) row_base[s] = carry + (warp > 0 ? warp_sum[warp - 1] : 0ull) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nwarps - 1];
    __syncthreads();
  }
}

cudaError_t launch_build_rows(const uint32_t* cnt_all, int nb, int32_t n, uint32_t* off_all, uint32_t* rowcnt,
                              unsigned long long* row_base, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(4096, ((int64_t)n + 255) / 256);
  k_colscan<<<std::max(blocks, 1), 256, 0, s>>>(cnt_all, nb, n, off_all, rowcnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rowscan<<<1, 1024, 0, s>>>(rowcnt, n, row_base);
  return cudaGetLastError();
}

// ---- fill: scatter keys into their (block, source) segments --------------------------------
__global__ void k_fill(const NetDev* __restrict__ nets, int net_idx, int32_t t_lo, int32_t t_hi, int32_t tb,
                       int first_group, uint32_t* __restrict__ cursor, uint32_t* __restrict__ keys) {
  const NetDev& d = nets[net_idx];
  const int64_t pairs = (d.k + 1) / 2;
  const int64_t total = (int64_t)(t_hi - t_lo) * pairs;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(t_lo + q / pairs);
    const uint32_t p = (uint32_t)(q % pairs);
    const Draw2 dr = draw_pair(d, i, p);
    const int64_t g = (int64_t)(i / tb) - first_group;
    const uint32_t local = i - (uint32_t)((g + first_group) * tb);
    const int64_t kbase = g * (int64_t)tb * d.k;  // keys of block g start here (all blocks but the last hold tb targets)
    {
      const uint32_t pos = atomicAdd(&cursor[g * d.n + dr.src[0]], 1u);
      keys[kbase + pos] = (local << 16) | (2u * p);
    }
    if (2 * p + 1 < (uint32_t)d.k) {
      const uint32_t pos = atomicAdd(&cursor[g * d.n + dr.src[1]], 1u);
      keys[kbase + pos] = (local << 16) | (2u * p + 1u);
    }
  }
}

cudaError_t launch_build_fill_net(const NetDev* nets_dev, int net_idx, int32_t n, int first_group, int n_groups,
                                  int32_t tb, uint32_t* cursor, uint32_t* keys, cudaStream_t s) {
  const int32_t t_lo = first_group * tb;
  const int32_t t_hi = min(n, (first_group + n_groups) * tb);
  k_fill<<<152 * 8, 256, 0, s>>>(nets_dev, net_idx, t_lo, t_hi, tb, first_group, cursor, keys);
  return cudaGetLastError();
}

// ---- finalize: sort each segment, write records and headers --------------------------------
// Record of synapse (source s -> local target j, delay d): weight w and
//   meta = ((j - wd * tw) << dbits) | (d - d_min),   wd = j / tw the delivery warp owning j.
constexpr int kSegCap = 2048;  // keys sorted in shared memory per warp
static_assert(kSegCap <= (int)kMaxPiece, "piece ends are 12-bit header fields");

// Bitonic sort, ascending, of the 32 E keys of a warp held in registers: key v[e] of lane l has
// index l + 32 e.  Compare-exchange partners at distance jj < 32 are in lane l ^ jj (shuffle), at
// distance >= 32 in the same lane; the result is the sorted sequence in the same index order.
template <int E>
__device__ __forceinline__ void warp_bitonic_sort(uint32_t (&v)[E], int lane) {
  constexpr int P = 32 * E;
#pragma unroll
  for (int kk = 2; kk <= P; kk <<= 1) {
#pragma unroll
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      if (jj >= 32) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int pe = e ^ (jj >> 5);
          if (pe > e) {
            const bool up = (((uint32_t)lane + 32u * (uint32_t)e) & (uint32_t)kk) == 0u;
            const uint32_t x = v[e], y = v[pe];
            if ((x > y) == up) {
              v[e] = y;
              v[pe] = x;
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t y = __shfl_xor_sync(0xffffffffu, v[e], jj);
          const bool up = (((uint32_t)lane + 32u * (uint32_t)e) & (uint32_t)kk) == 0u;
          const bool lower = (lane & jj) == 0;
          v[e] = (lower == up) ? min(v[e], y) : max(v[e], y);
        }
      }
    }
  }
}

// keys [key0, key0 + len) sorted into buf[0, len) by one warp in registers (len <= 32 E)
template <int E>
__device__ __forceinline__ void warp_sort_keys(const uint32_t* __restrict__ keys, int64_t key0, uint32_t len,
                                               uint32_t* buf, int lane) {
  uint32_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t q = (uint32_t)lane + 32u * (uint32_t)e;
    v[e] = q < len ? keys[key0 + q] : 0xffffffffu;
  }
  warp_bitonic_sort<E>(v, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) buf[(uint32_t)lane + 32u * (uint32_t)e] = v[e];
}

__global__ void __launch_bounds__(256) k_finalize(const NetDev* __restrict__ nets, const BlockWork* __restrict__ work,
                                                  int net_idx, int first_group, int n_groups, int n_dw,
                                                  const uint32_t* __restrict__ cnt,
                                                  const uint32_t* __restrict__ seg_end,
                                                  const uint32_t* __restrict__ keys,
                                                  const uint32_t* __restrict__ off_all,
                                                  const unsigned long long* __restrict__ row_base,
                                                  void* __restrict__ rec_w, uint16_t* __restrict__ rec_meta,
                                                  uint4* __restrict__ hdr, int32_t* __restrict__ err,
                                                  uint32_t* __restrict__ max_seg) {
  extern __shared__ uint32_t sk[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* buf = sk + wib * kSegCap;
  const NetDev& d = nets[net_idx];
  const int32_t n = d.n, n_exc = d.n_exc, k = d.k, d_min = d.d_min, dbits = d.dbits, wdtype = d.wdtype;
  const int32_t nbk = d.n_blocks;
  const int64_t rec_net = d.rec_base, hdr_net = d.hdr_base, row_off = d.row_off;
  const float w_exc = d.w_exc, w_inh = d.w_inh;
  const int64_t n_seg = (int64_t)n_groups * n;
  const int64_t warp_global = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t warp_stride = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t tb_full = work[d.first_block].nt;
  for (int64_t sg = warp_global; sg < n_seg; sg += warp_stride) {
    const int64_t g = sg / n;
    const uint32_t src = (uint32_t)(sg % n);
    const BlockWork w = work[d.first_block + first_group + g];
    const uint32_t len = cnt[sg];
    const uint32_t end = seg_end[sg];
    const uint32_t start = end - len;
    // keys of block g start at g * tb * K (all blocks but the last hold tb targets)
    const int64_t key0 = g * tb_full * k + start;
    if (len > kSegCap || len > 65535u) {
      if (lane == 0) atomicOr(err, kErrSegment);
      continue;
    }
    if (lane == 0 && len) atomicMax(max_seg, len);
    uint32_t p2 = 32;
    while (p2 < len) p2 <<= 1;
    // sort ascending by (local target, draw): in registers up to 128 keys, else in shared memory
    if (p2 <= 32) {
      warp_sort_keys<1>(keys, key0, len, buf, lane);
    } else if (p2 <= 64) {
      warp_sort_keys<2>(keys, key0, len, buf, lane);
    } else if (p2 <= 128) {
      warp_sort_keys<4>(keys, key0, len, buf, lane);
    } else {
      for (uint32_t q = lane; q < p2; q += 32) buf[q] = (q < len) ? keys[key0 + q] : 0xffffffffu;
      __syncwarp();
      for (uint32_t kk = 2; kk <= p2; kk <<= 1) {
        for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
          for (uint32_t q = lane; q < p2; q += 32) {
            const uint32_t l = q ^ jj;
            if (l > q) {
              const uint32_t x = buf[q], y = buf[l];
              const bool up = (q & kk) == 0;
              if ((x > y) == up) {
                buf[q] = y;
                buf[l] = x;
              }
            }
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
    // the block's piece of the source's row (CSR by source, blocks in ascending order)
    const uint32_t piece = off_all[(int64_t)(first_group + g) * n + src];
    const int64_t r0 = rec_net + (int64_t)row_base[row_off + src] + piece;
    for (uint32_t q = lane; q < len; q += 32) {
      const uint32_t key = buf[q];
      const uint32_t local = key >> 16, j = key & 0xffffu;
      const Draw2 dr = draw_pair(d, (uint32_t)w.t0 + local, j >> 1);
      const uint32_t s2 = dr.src[j & 1u], dl = dr.dly[j & 1u];
      if (s2 != src) atomicOr(err, kErrBuild);
      const float wv = (src < (uint32_t)n_exc) ? w_exc : w_inh;
      if (wdtype == 1) reinterpret_cast<__nv_bfloat16*>(rec_w)[r0 + q] = __float2bfloat16_rn(wv);
      else reinterpret_cast<float*>(rec_w)[r0 + q] = wv;
      const uint32_t wd = local / (uint32_t)w.tw;
      const uint32_t rel = local - wd * (uint32_t)w.tw;
      rec_meta[r0 + q] = (uint16_t)((rel << dbits) | (dl - (uint32_t)d_min));
    }
    // header: base, then for delivery warp wd the number of entries with local target < (wd + 1) * tw
    uint32_t e_w = len;
    if (lane < n_dw) {
      const uint32_t bound = min((uint32_t)((lane + 1) * w.tw), (uint32_t)w.nt);
      uint32_t lo = 0, hi = len;  // first q with (buf[q] >> 16) >= bound
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((buf[mid] >> 16) < bound) lo = mid + 1;
        else hi = mid;
      }
      e_w = lo;
    }
    // (a cell repeated inside a piece -- a source drawn twice by one target with one delay -- needs
    // no mark: the delivery orders equal cells of a chunk by lane, i.e. in record order)
    if (piece + len > 0xffffu && lane == 0) atomicOr(err, kErrSegment);  // rows longer than 65535
    uint32_t words[8] = {piece & 0xffffu, 0u, 0u, 0u, 0u, 0u, 0u, 0u};  // high half of word 0 reserved
#pragma unroll
    for (int q = 0; q < kMaxWarps; ++q) {  // end[q] as the 12-bit field at bit 32 + 12 q
      const uint32_t x = __shfl_sync(0xffffffffu, e_w, q);
      const uint32_t e = (q < n_dw) ? x : len;
      const int p = 32 + 12 * q, i = p >> 5, sh = p & 31;
      words[i] |= e << sh;
      if (sh > 20) words[i + 1] |= e >> (32 - sh);
    }
    if (lane == 0) {
      const int64_t h = hdr_net + (int64_t)src * nbk + (first_group + g);
      hdr[2 * h] = make_uint4(words[0], words[1], words[2], words[3]);
      hdr[2 * h + 1] = make_uint4(words[4], words[5], words[6], words[7]);
    }
    __syncwarp();
  }
}

cudaError_t launch_build_finalize_net(const NetDev* nets_dev, const BlockWork* work_dev, int net_idx, int first_group,
                                      int n_groups, int n_dw, const uint32_t* cnt, const uint32_t* seg_end,
                                      const uint32_t* keys, const uint32_t* off_all,
                                      const unsigned long long* row_base, void* rec_w, uint16_t* rec_meta,
                                      uint4* hdr, int32_t* err, uint32_t* max_seg, cudaStream_t s) {
  const size_t smem = 8 * kSegCap * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_finalize<<<152 * 4, 256, smem, s>>>(nets_dev, work_dev, net_idx, first_group, n_groups, n_dw, cnt, seg_end, keys,
                                        off_all, row_base, rec_w, rec_meta, hdr, err, max_seg);
  return cudaGetLastError();
}

// ---- delay-ordered layout (Sec. III-B "Varied Synaptic Delays": synapses reordered by delay) ---
// From the CSR by source (row of source s grouped by block, by target inside a block), a second
// copy of the records in which every (source, block) piece is sorted by (delay, target, draw), and
// per source a table of u16 offsets in its row: tbl[b * (n_delays + 1) + k] = first record of
// block b's piece of delay d_min + k, tbl[b * (n_delays + 1) + n_delays] = the end of block b's
// piece (for the last block: the row length).  A block's pieces of consecutive delays, and their
// table entries, are adjacent, so the few pieces a spike contributes to one window share cache
// lines.  A record keeps its block-local target and its weight (BF16: packed as one u32, target in
// the low half; FP32: a u16 target array and a float weight array); the delay is the piece's.
// Every delay piece is a stable subsequence of the block's piece, so it stays in (target, draw)
// order.  One warp per source: per block, count the delays, scan, scatter (ranks of equal delays
// inside a 32-entry chunk by __match_any_sync).
__global__ void __launch_bounds__(128) k_delay_layout(const NetDev* __restrict__ nets,
                                                      const BlockWork* __restrict__ work, int net_idx, int n_dw,
                                                      const uint4* __restrict__ hdr,
                                                      const unsigned long long* __restrict__ row_base,
                                                      const void* __restrict__ rec_w,
                                                      const uint16_t* __restrict__ rec_meta,
                                                      uint16_t* __restrict__ dtbl, uint16_t* __restrict__ dtgt,
                                                      void* __restrict__ dw, int32_t* __restrict__ err) {
  __shared__ uint32_t dl_cnt[4][256 + 1];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* c = dl_cnt[wib];
  const NetDev& d = nets[net_idx];
  const int nb = d.n_blocks, n_del = d.d_max - d.d_min + 1;
  const uint32_t dmask = (1u << d.dbits) - 1u;
  const int64_t warp_global = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t warp_stride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = warp_global; s < d.n; s += warp_stride) {
    const int64_t r0 = d.rec_base + (int64_t)row_base[d.row_off + s];
    for (int b = 0; b < nb; ++b) {
      const BlockWork wk = work[d.first_block + b];
      const int64_t hi = d.hdr_base + s * nb + b;
      const uint4 h0 = hdr[2 * hi], h1 = hdr[2 * hi + 1];
      const uint32_t words[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
      const uint32_t off = words[0] & 0xffffu, len = hdr_end(words, kMaxWarps - 1);
      // 1. entries per delay of the piece
      for (int q = lane; q <= n_del; q += 32) c[q] = 0u;
      __syncwarp();
      for (uint32_t q = lane; q < len; q += 32) atomicAdd(&c[rec_meta[r0 + off + q] & dmask], 1u);
      __syncwarp();
      // 2. exclusive scan over the delays -> the block's table row (offsets in the row)
      uint32_t run = off;
      uint16_t* trow = dtbl + d.tbl_base + s * d.tbl_stride + (int64_t)b * (n_del + 1);
      for (int q0 = 0; q0 < n_del; q0 += 32) {
        const int q = q0 + lane;
        const uint32_t v = q < n_del ? c[q] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (q < n_del) {
          c[q] = run + x - v;
          trow[q] = (uint16_t)(run + x - v);
        }
        run += __shfl_sync(0xffffffffu, x, 31);
      }
      if (lane == 0) {
        trow[n_del] = (uint16_t)run;
        if (run > 0xffffu || run != off + len) atomicOr(err, kErrSegment);
      }
      __syncwarp();
      // 3. scatter, stable inside every delay piece
      for (uint32_t q0 = 0; q0 < len; q0 += 32) {
        const uint32_t q = q0 + lane;
        const bool valid = q < len;
        uint32_t key = 0xffffffffu, local = 0;
        float w = 0.0f;
        if (valid) {
          const uint32_t meta = rec_meta[r0 + off + q];
          key = meta & dmask;
          uint32_t wd = 0;  // delivery warp of entry q: the number of warp ends at or below q
          for (int k = 0; k < n_dw; ++k) wd += (hdr_end(words, k) <= q) ? 1u : 0u;
          local = wd * (uint32_t)wk.tw + (meta >> d.dbits);
          w = d.wdtype == 1 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(rec_w)[r0 + off + q])
                            : reinterpret_cast<const float*>(rec_w)[r0 + off + q];
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        const uint32_t base = valid ? c[key] : 0u;
        __syncwarp();
        if (valid) {
          const int64_t pos = r0 + base + rank;
          if (d.wdtype == 1) {
            const __nv_bfloat16 wb = __float2bfloat16_rn(w);
            reinterpret_cast<uint32_t*>(dw)[pos] = local | ((uint32_t)__bfloat16_as_ushort(wb) << 16);
          } else {
            dtgt[pos] = (uint16_t)local;
            reinterpret_cast<float*>(dw)[pos] = w;
          }
          if (rank == 0) c[key] = base + (uint32_t)__popc(peers);
        }
        __syncwarp();
      }
    }
  }
}

cudaError_t launch_delay_layout(const NetDev* nets_dev, const NetDev* net_host, const BlockWork* work_dev, int net_idx,
                                int n_dw, const uint4* hdr, const unsigned long long* row_base, const void* rec_w,
                                const uint16_t* rec_meta, uint16_t* dtbl, uint16_t* dtgt, void* dw, int32_t* err,
                                cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(152 * 8, (net_host->n + 3) / 4);
  k_delay_layout<<<std::max(blocks, 1), 128, 0, s>>>(nets_dev, work_dev, net_idx, n_dw, hdr, row_base, rec_w,
                                                     rec_meta, dtbl, dtgt, dw, err);
  return cudaGetLastError();
}

// ---- initial state ------------------------------------------------------------------------
// V0 = V_reset + (V_th - V_reset) * ((u >> 8) 2^-24), u = word 0 of Philox(ctr = (i, 0, 2, 0));
// each operation rounded to float.  I = 0, refractory counter = 0.
__global__ void k_init_state(const NetDev* __restrict__ nets, int net_idx, float* __restrict__ V,
                             float* __restrict__ I, int32_t* __restrict__ R) {
  const NetDev& d = nets[net_idx];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0u, kStreamV0, 0u), d.seed_lo, d.seed_hi);
    const float frac = __fmul_rn((float)(r.x >> 8), 0x1p-24f);
    const float span = __fsub_rn(d.v_th, d.v_reset);
    V[d.neuron_base + i] = __fadd_rn(d.v_reset, __fmul_rn(span, frac));
    I[d.neuron_base + i] = 0.0f;
    R[d.neuron_base + i] = 0;
  }
}

cudaError_t launch_init_state(const NetDev* net_host, const NetDev* net_dev, int net_idx, float* V, float* I,
                              int32_t* R, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(4096, (net_host->n + 255) / 256);
  k_init_state<<<max(blocks, 1), 256, 0, s>>>(net_dev, net_idx, V, I, R);
  return cudaGetLastError();
}

// ---- Philox check kernel ---------------------------------------------------------------------
__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key, int64_t n,
                         uint32_t* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4(ctr[4 * q], ctr[4 * q + 1], ctr[4 * q + 2], ctr[4 * q + 3]), key[2 * q],
                                  key[2 * q + 1]);
    out[4 * q] = r.x;
    out[4 * q + 1] = r.y;
    out[4 * q + 2] = r.z;
    out[4 * q + 3] = r.w;
  }
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(1024, (n + 255) / 256);
  k_philox<<<max(blocks, 1), 256, 0, s>>>(ctr, key, n, out);
  return cudaGetLastError();
}

// ---- export of the incoming synapses of a target range (connectivity checks) ------------------
__global__ void k_export(const NetDev* __restrict__ nets, const BlockWork* __restrict__ work, int block, int n_dw,
                         const void* __restrict__ rec_w, int wdtype, const uint16_t* __restrict__ rec_meta,
                         const uint4* __restrict__ hdr, const unsigned long long* __restrict__ row_base,
                         int32_t n_src, int32_t t_begin, int32_t t_end,
                         unsigned long long* counter, int32_t* o_src, int32_t* o_tgt, int32_t* o_dly, float* o_w,
                         int64_t cap) {
  const BlockWork w = work[block];
  const NetDev& d = nets[w.net];
  const uint32_t dmask = (1u << d.dbits) - 1u;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_src; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t hi = d.hdr_base + s * d.n_blocks + w.group;
    const uint4 h0 = hdr[2 * hi];
    const uint4 h1 = hdr[2 * hi + 1];
    const uint32_t words[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
    const uint32_t base = words[0] & 0xffffu;
    uint32_t e0 = 0;
    for (int wd = 0; wd < n_dw; ++wd) {
      const uint32_t e1 = hdr_end(words, wd);
      for (uint32_t q = e0; q < e1; ++q) {
        const int64_t r = d.rec_base + (int64_t)row_base[d.row_off + s] + base + q;
        const uint32_t meta = rec_meta[r];
        const int32_t tgt = w.t0 + wd * w.tw + (int32_t)(meta >> d.dbits);
        if (tgt < t_begin || tgt >= t_end) continue;
        const unsigned long long pos = atomicAdd(counter, 1ull);
        if ((int64_t)pos >= cap) continue;
        o_src[pos] = (int32_t)s;
        o_tgt[pos] = tgt;
        o_dly[pos] = d.d_min + (int32_t)(meta & dmask);
        o_w[pos] = wdtype == 1 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(rec_w)[r])
                               : reinterpret_cast<const float*>(rec_w)[r];
      }
      e0 = e1;
    }
  }
}

cudaError_t launch_export(const NetDev* nets_dev, const BlockWork* work_dev, int block, int n_dw, const void* rec_w,
                          int wdtype, const uint16_t* rec_meta, const uint4* hdr, const unsigned long long* row_base,
                          int32_t n_src, int32_t t_begin, int32_t t_end, unsigned long long* counter, int32_t* src,
                          int32_t* tgt, int32_t* dly, float* w, int64_t cap, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(1024, (n_src + 255) / 256);
  k_export<<<std::max(blocks, 1), 256, 0, s>>>(nets_dev, work_dev, block, n_dw, rec_w, wdtype, rec_meta, hdr,
                                               row_base, n_src, t_begin, t_end, counter, src, tgt, dly, w, cap);
  return cudaGetLastError();
}

}  // namespace cortex
