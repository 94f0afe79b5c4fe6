// noalloc.cu -- the incoming sub-graph of a target range, built without allocating device memory.
//
// Some callers cannot allocate device memory at the time they need connectivity: code that runs
// while a framework owns the whole device pool, or inside a driver loop that must never call the
// allocator.  cortex_subgraph_noalloc() gives them the same Philox connectivity the network
// builder produces, for targets [t_begin, t_end), as a CSR by source in buffers the caller passes.
// Its working memory (per-source counters and the sort keys) is the file-scope array below, which
// every GPU that loads the library keeps until the process exits.
#include <mutex>

#include "cortex.h"
#include "cortex_internal.cuh"

namespace cortex {

// 8 MiB of working memory: (n_src + 1) counters followed by (t_end - t_begin) * K sort keys
constexpr size_t kNoAllocWords = size_t(2) << 20;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kNaSegCap = 2048;  // synapses of one source inside the range (sorted in shared memory)

struct NaParams {
  uint32_t seed_lo, seed_hi;
  int32_t n, n_exc, n_inh, k_exc, k, d_min, d_max;
  int32_t t_begin, t_end;
  float w_exc, w_inh;
  int32_t bf16;
};

__device__ __forceinline__ void na_draw(const NaParams& p, uint32_t i, uint32_t j, uint32_t& src, uint32_t& dly) {
  const uint4 r = philox4x32_10(make_uint4(i, j >> 1, kStreamConn, 0u), p.seed_lo, p.seed_hi);
  const uint32_t a = (j & 1u) ? r.z : r.x, b = (j & 1u) ? r.w : r.y;
  src = (j < (uint32_t)p.k_exc) ? scale32(a, (uint32_t)p.n_exc) : (uint32_t)p.n_exc + scale32(a, (uint32_t)p.n_inh);
  dly = (uint32_t)p.d_min + scale32(b, (uint32_t)(p.d_max - p.d_min + 1));
}

__global__ void k_na_clear(uint32_t* w, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) w[q] = 0u;
}

__global__ void k_na_count(NaParams p, uint32_t* cnt) {
  const int64_t total = (int64_t)(p.t_end - p.t_begin) * p.k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t s, d;
    na_draw(p, (uint32_t)(p.t_begin + q / p.k), (uint32_t)(q % p.k), s, d);
    atomicAdd(&cnt[s], 1u);
  }
}

// one block: exclusive prefix of the counters -> row_ptr (output) and the fill cursors (in place)
__global__ void k_na_scan(NaParams p, uint32_t* cnt, int32_t* row_ptr) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int64_t off = 0; off < p.n; off += blockDim.x) {
    const int64_t s = off + threadIdx.x;
    const uint32_t v = (s < p.n) ? cnt[s] : 0u;
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
      if (lane < nwarps) warp_sum[lane] = w;
    }
    __syncthreads();
    const uint32_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0u) + x - v;
    if (s < p.n) {
      row_ptr[s] = (int32_t)before;
      cnt[s] = before;  // becomes the fill cursor
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nwarps - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) row_ptr[p.n] = (int32_t)carry;
}

__global__ void k_na_fill(NaParams p, uint32_t* cursor, uint32_t* keys) {
  const int64_t total = (int64_t)(p.t_end - p.t_begin) * p.k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t local = (uint32_t)(q / p.k), j = (uint32_t)(q % p.k);
    uint32_t s, d;
    na_draw(p, (uint32_t)p.t_begin + local, j, s, d);
    keys[atomicAdd(&cursor[s], 1u)] = (local << 16) | j;
  }
}

// one warp per source: sort its keys by (target, draw), write the synapses in that order
__global__ void __launch_bounds__(256) k_na_rows(NaParams p, const int32_t* row_ptr, const uint32_t* keys,
                                                 int32_t* tgt, int32_t* delay, float* weight, int32_t* err) {
  extern __shared__ uint32_t sk[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* buf = sk + wib * kNaSegCap;
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; s < p.n; s += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    const uint32_t b = (uint32_t)row_ptr[s], len = (uint32_t)row_ptr[s + 1] - b;
    if (len > (uint32_t)kNaSegCap) {
      if (lane == 0) atomicOr(err, 1);
      continue;
    }
    uint32_t p2 = 32;
    while (p2 < len) p2 <<= 1;
    for (uint32_t q = lane; q < p2; q += 32) buf[q] = (q < len) ? keys[b + q] : 0xffffffffu;
    __syncwarp();
    for (uint32_t kk = 2; kk <= p2; kk <<= 1) {
      for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
        for (uint32_t q = lane; q < p2; q += 32) {
          const uint32_t l = q ^ jj;
          if (l > q) {
            const uint32_t x = buf[q], y = buf[l];
            if ((x > y) == ((q & kk) == 0)) {
              buf[q] = y;
              buf[l] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    for (uint32_t q = lane; q < len; q += 32) {
      const uint32_t local = buf[q] >> 16, j = buf[q] & 0xffffu;
      uint32_t s2, d;
      na_draw(p, (uint32_t)p.t_begin + local, j, s2, d);
      if (s2 != (uint32_t)s) atomicOr(err, 2);
      tgt[b + q] = p.t_begin + (int32_t)local;
      delay[b + q] = (int32_t)d;
      const float w = (s < p.n_exc) ? p.w_exc : p.w_inh;
      weight[b + q] = p.bf16 ? __bfloat162float(__float2bfloat16_rn(w)) : w;
    }
    __syncwarp();
  }
}

namespace {
std::mutex g_na_mutex;
void* g_na_ptr[256] = {};  // device address of g_noalloc_scratch, per device ordinal
}  // namespace

}  // namespace cortex

using namespace cortex;

extern "C" int cortex_subgraph_noalloc(const cortex_params* params, uint64_t seed, int32_t t_begin, int32_t t_end,
                                       void* stream, int32_t* row_ptr, int32_t* tgt, int32_t* delay, float* weight) {
  if (!params || !row_ptr || t_begin < 0 || t_end < t_begin)
    return record_error(CORTEX_ERR_ARG, "cortex_subgraph_noalloc: params / row_ptr NULL or bad target range");
  const cortex_params& c = *params;
  const int64_t n = (int64_t)c.n_exc + c.n_inh, k = (int64_t)c.k_exc + c.k_inh;
  if (c.n_exc < 0 || c.n_inh < 0 || n <= 0 || c.k_exc < 0 || c.k_inh < 0 || k > 65535 || t_end > n ||
      (c.k_exc > 0 && c.n_exc == 0) || (c.k_inh > 0 && c.n_inh == 0) || c.d_min < 1 || c.d_max < c.d_min ||
      (c.weight_dtype != CORTEX_F32 && c.weight_dtype != CORTEX_BF16))
    return record_error(CORTEX_ERR_ARG, "cortex_subgraph_noalloc: invalid network parameters or t_end > n");
  const int64_t nnz = (t_end - t_begin) * k;
  if (nnz > 0 && (!tgt || !delay || !weight))
    return record_error(CORTEX_ERR_ARG, "cortex_subgraph_noalloc: NULL output buffer");
  if (t_end - t_begin > 65536)  // local target in 16 bits
    return record_error(CORTEX_ERR_UNSUPPORTED, "cortex_subgraph_noalloc: more than 65536 targets in the range");
  if ((size_t)(n + 1) + (size_t)nnz > kNoAllocWords)  // scratch limit
    return record_error(CORTEX_ERR_UNSUPPORTED,
                        "cortex_subgraph_noalloc: (n + 1) + targets * K above the 2^21 words of the static array");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return record_error(CORTEX_ERR_CUDA, "cortex_subgraph_noalloc: no current CUDA device");
  void* base = nullptr;
  {
    // set-up, once per device (with that device current): the device address of the array
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      if (cudaGetSymbolAddress(&g_na_ptr[dev], g_noalloc_scratch) != cudaSuccess) {
        g_na_ptr[dev] = nullptr;
        return record_error(CORTEX_ERR_CUDA, "cortex_subgraph_noalloc: cudaGetSymbolAddress of the static array failed");
      }
    }
    base = g_na_ptr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base);  // n + 1 counters (the last word: error flags)
  uint32_t* keys = cnt + (n + 1);
  NaParams p;
  p.seed_lo = (uint32_t)seed;
  p.seed_hi = (uint32_t)(seed >> 32);
  p.n = (int32_t)n;
  p.n_exc = c.n_exc;
  p.n_inh = c.n_inh;
  p.k_exc = c.k_exc;
  p.k = (int32_t)k;
  p.d_min = c.d_min;
  p.d_max = c.d_max;
  p.t_begin = t_begin;
  p.t_end = t_end;
  p.w_exc = c.j_exc;
  p.w_inh = c.j_inh;
  p.bf16 = c.weight_dtype == CORTEX_BF16;
  const int grid = 152 * 4;
  k_na_clear<<<grid, 256, 0, s>>>(cnt, n + 1);  // the array keeps the previous call's contents
  if (nnz > 0) {
    k_na_count<<<grid, 256, 0, s>>>(p, cnt);
    k_na_scan<<<1, 1024, 0, s>>>(p, cnt, row_ptr);
    k_na_fill<<<grid, 256, 0, s>>>(p, cnt, keys);
    const size_t smem = 8 * kNaSegCap * sizeof(uint32_t);
    if (cudaFuncSetAttribute(k_na_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return record_error(CORTEX_ERR_CUDA, "cortex_subgraph_noalloc: kernel attribute");
    k_na_rows<<<grid, 256, smem, s>>>(p, row_ptr, keys, tgt, delay, weight, reinterpret_cast<int32_t*>(cnt + n));
  } else {
    k_na_scan<<<1, 1024, 0, s>>>(p, cnt, row_ptr);
  }
  if (cudaGetLastError() != cudaSuccess) return record_error(CORTEX_ERR_CUDA, "cortex_subgraph_noalloc: kernel launch");
  uint32_t flags = 0;
  if (cudaMemcpyAsync(&flags, cnt + n, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return record_error(CORTEX_ERR_CUDA, "cortex_subgraph_noalloc: stream synchronisation");
  if (flags & 1u)  // found on the device, after the outputs were partly written
    return record_error(CORTEX_ERR_UNSUPPORTED,
                        "cortex_subgraph_noalloc: a source has more than 2048 synapses in the range (outputs undefined)");
  if (flags & 2u) return record_error(CORTEX_ERR_CUDA, "cortex_subgraph_noalloc: device consistency check failed");
  return CORTEX_OK;
}
