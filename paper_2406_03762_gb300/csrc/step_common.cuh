// step_common.cuh -- device code shared by the two step kernels (ring delivery in step.cu,
// delay-ordered delivery in step_delay.cu): the exact-integration neuron update (Eq. 1-3) and the
// ordered fold of a 32-lane chunk of synaptic entries into accumulator cells.
#pragma once
#include "cortex_internal.cuh"

namespace cortex {

// duplicate-detection tags: one byte per ring cell when the ring is in shared memory, else a
// hashed table of kTagHash bytes per warp.  (Finding the sharing of several chunks ahead of their
// ring updates, in separate tables, measured slower with reductions into a global ring.)
constexpr int kTagHash = 2048;

// ---- one neuron, one step (Eq. 1-3, exact integration) --------------------------------------
//   V half: refractory: V = V_reset, counter - 1;  else V = V + fma(P22 - 1, V, P21 * I) with
//           the I of the previous step;  V >= V_th: spike, V = V_reset, counter = n_ref (Eq. 2)
//   I half: in = ring cell of the step (cleared); k = Poisson draw (neuron i, step t: word i mod 4
//           of Philox(counter = (i / 4, t, 3, 0))); ext = k * J_ext;
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

// word w (0..3) of a generator output
__device__ __forceinline__ uint32_t philox_word(const uint4& r, uint32_t w) {
  return w == 0u ? r.x : (w == 1u ? r.y : (w == 2u ? r.z : r.w));
}

// Poisson count of the external drive by inversion: the smallest k with u < thr[k]
__device__ __forceinline__ int poisson_k(uint32_t u, const NeuronConst& nd, const uint32_t* thr) {
  int k = 0;
  while (k < nd.n_thr - 1 && u >= thr[k]) ++k;
  return k;
}

__device__ __forceinline__ void i_half_k(float& cur, float in, int k, const NeuronConst& nd) {
  const float ext = __fmul_rn((float)k, nd.j_ext);
  cur = __fmaf_rn(nd.p11, cur, in);
  cur = __fadd_rn(cur, ext);
}

__device__ __forceinline__ void i_half(float& cur, float in, uint32_t u, const NeuronConst& nd, const uint32_t* thr) {
  i_half_k(cur, in, poisson_k(u, nd, thr), nd);
}

// One ring cell += w.  A ring in shared memory: load, add, store.  A ring in global memory: the
// same, or (red) an add performed by the L2 reduction unit, which rounds to nearest even like the
// load-add-store but flushes subnormal operands and results to zero.  The host selects red only
// when every weight is zero or at least 2^-103 in magnitude: every partial sum of a cell is then an
// integer multiple of the smallest weight's ulp (>= 2^-126), so no operand or result is subnormal
// and both forms give the same bits.  Lanes that add to one cell are ordered by __syncwarp, which
// orders their memory operations.
template <bool kRingSmem>
__device__ __forceinline__ void ring_add(float* ring, uint32_t key, float w, bool red) {
  if (!kRingSmem && red) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(ring + key), "f"(w) : "memory");
  } else {
    ring[key] = __fadd_rn(ring[key], w);
  }
}

// One ring cell += w when the build has shown that every partial sum of a cell is exact (every
// weight an integer multiple of 2^e, e >= -126, and the sum of |w| / 2^e over a target's in-degree
// below 2^24): the FP32 adds then round nothing, so any order gives the bits of the ordered fold,
// and lanes that share a cell need no ordering.  Shared ring: a shared-memory reduction; global
// ring: an L2 reduction.  Both flush subnormals, and none occurs (every nonzero partial sum is at
// least 2^e >= 2^-126 in magnitude).
template <bool kRingSmem>
__device__ __forceinline__ void ring_add_exact(float* ring, uint32_t key, float w) {
  if constexpr (kRingSmem) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(smem_addr(ring + key)), "f"(w) : "memory");
  } else {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(ring + key), "f"(w) : "memory");
  }
}

// a ring cell read by the update: a global ring bypasses L1 (reductions are performed in L2)
template <bool kRingSmem>
__device__ __forceinline__ float ring_read(const float* p) {
  if (kRingSmem) return *p;
  return __ldcg(p);
}

// Ring updates of one 32-lane chunk (key = cell, 0xffffffff = no entry) whose sharing is known:
// t = the lane id read back from the cell's tag, losers = lanes whose tag names another lane (a
// group of lanes with one cell has one recorded writer; the others are losers).  Lanes hold
// entries in stream order, and every cell must receive its weights in lane order:
//   - no sharing: all lanes add at once;
//   - every group a pair (one loser, one writer): the lower lane of each pair adds with the
//     unshared lanes, then the higher lanes add;
//   - otherwise: unshared lanes at once, then the shared lanes one by one in lane order.
// With hashed tags two lanes of different cells may be taken for a pair: they are then merely
// ordered, which is always allowed.  The general case is rare and kept out of line
// (fold_apply_serial): the fold is inlined into every chunk of every group size, and its code size
// measured in the step time.
template <bool kRingSmem>
__device__ __noinline__ void fold_apply_serial(float* ring, uint32_t key, float w, uint32_t dup, int lane, bool red) {
  const bool valid = key != 0xffffffffu;
  const bool isdup = (dup >> lane) & 1u;
  if (valid && !isdup) ring_add<kRingSmem>(ring, key, w, red);
  __syncwarp();
  uint32_t m = dup;
  while (m) {
    const int f = __ffs(m) - 1;
    if (lane == f) ring_add<kRingSmem>(ring, key, w, red);
    __syncwarp();
    m &= m - 1u;
  }
}

template <bool kRingSmem>
__device__ __forceinline__ void fold_apply(float* ring, uint32_t key, float w, uint32_t t, uint32_t losers, int lane,
                                           bool red) {
  const bool valid = key != 0xffffffffu;
  if (losers == 0) {
    if (valid) ring_add<kRingSmem>(ring, key, w, red);
    __syncwarp();
    return;
  }
  const bool loser = (losers >> lane) & 1u;
  const uint32_t winners = __reduce_or_sync(0xffffffffu, loser ? (1u << t) : 0u);
  const uint32_t wfirst = __reduce_or_sync(0xffffffffu, (loser && (uint32_t)lane > t) ? (1u << t) : 0u);
  const uint32_t dup = losers | winners;
  const bool isdup = (dup >> lane) & 1u;
  if (__popc(losers) == __popc(winners)) {
    const bool first = !isdup || (loser ? ((uint32_t)lane < t) : ((wfirst >> lane) & 1u));
    if (valid && first) ring_add<kRingSmem>(ring, key, w, red);
    __syncwarp();
    if (valid && !first) ring_add<kRingSmem>(ring, key, w, red);
    __syncwarp();
    return;
  }
  fold_apply_serial<kRingSmem>(ring, key, w, dup, lane, red);
}

// Fold one chunk: every lane writes its lane id into the tag of its cell and reads it back, which
// finds the lanes that share a cell (shared ring: one tag per cell, since warps own disjoint cells;
// global ring: a hashed tag array of kTagHash bytes per warp), then the ring updates run in lane
// order.
template <bool kRingSmem>
__device__ __forceinline__ void fold_one(float* ring, uint8_t* wtags, uint32_t key, float w, int lane, bool red) {
  const bool valid = key != 0xffffffffu;
  uint8_t* tg = kRingSmem ? wtags + (valid ? key : 0u) : wtags + (key & (uint32_t)(kTagHash - 1));
  if (valid) *tg = (uint8_t)lane;
  __syncwarp();
  const uint32_t t = valid ? (uint32_t)*tg : (uint32_t)lane;
  const uint32_t losers = __ballot_sync(0xffffffffu, valid && t != (uint32_t)lane);
  fold_apply<kRingSmem>(ring, key, w, t, losers, lane, red);
}

}  // namespace cortex
