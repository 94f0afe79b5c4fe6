/*
 * cortex.h -- C ABI of the GB300 spike-delivery library (CORTEX, arXiv 2406.03762).
 *
 * The library simulates spiking networks of leaky integrate-and-fire neurons (Eq. 1) with
 * threshold, reset and refractory period (Eq. 2) and an exponentially decaying synaptic current
 * (Eq. 3, read as a current-based synapse: an arriving spike adds its weight to the current).
 * Connectivity is a fixed in-degree random graph G = (V, E) (Sec. II-A, Eq. 4).  Each thread
 * block owns a contiguous range of post-synaptic neurons together with all of their incoming
 * synapses -- the indegree sub-graph inS(V_i) of Eq. 5 and Eq. 9-10 -- so delivery into a
 * neuron's delay ring buffer needs no atomics (Eq. 14, Sec. III-B "Avoid Data Racing").
 * One simulation step follows Sec. II-B: spikes act on their targets after the synaptic delay,
 * then every neuron updates and produces the next spikes.
 *
 * Conventions
 *   - Every call returns CORTEX_OK (0) or a negative CORTEX_ERR_* code; no exception, abort or
 *     exit crosses the ABI.  cortex_last_error() describes the most recent failure of the
 *     calling thread.
 *   - All device memory is allocated and owned by the library inside the cortex_net handle and
 *     released by cortex_free().  Host buffers passed in are owned by the caller; the library
 *     never keeps a pointer to them after the call returns.
 *   - Work is issued on the CUDA stream passed at build time (a cudaStream_t given as void*;
 *     NULL is the legacy default stream).  Calls on one handle must not overlap; calls that
 *     return data to the host synchronise that stream.
 *   - Time is counted in steps of dt.  Delays are integers d_min..d_max steps (d_min >= 1).
 */
#ifndef CORTEX_H
#define CORTEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CORTEX_OK 0
#define CORTEX_ERR_ARG (-1)          /* invalid argument or size; nothing was changed */
#define CORTEX_ERR_OOM (-2)          /* device or host allocation failed */
#define CORTEX_ERR_CUDA (-3)         /* a CUDA runtime call failed (see cortex_last_error) */
#define CORTEX_ERR_TIMEOUT (-4)      /* a device-side wait gave up; the CUDA context stays usable */
#define CORTEX_ERR_UNSUPPORTED (-5)  /* sizes outside the supported range, or no capable GPU */
#define CORTEX_ERR_OVERFLOW (-6)     /* an output buffer was too small (needed size returned) */
#define CORTEX_ERR_CHECK (-7)        /* ownership check: a ring cell was written by two warps */

/* synaptic weight storage */
#define CORTEX_F32 0                 /* float weights: 6 stored bytes per synapse (weight, u16 target/delay) */
#define CORTEX_BF16 1                /* bfloat16 weights, round-to-nearest-even: 4 stored bytes */

/* ring-buffer placement (cortex_options.ring) */
#define CORTEX_RING_AUTO 0
#define CORTEX_RING_SMEM 1           /* each block keeps its targets' ring in shared memory */
#define CORTEX_RING_GLOBAL 2         /* the ring stays in global memory (owner-exclusive) */

/* delivery fold (cortex_options.fold).  Every ring cell receives its weights in the order
 * (emission step, source id, draw index), which fixes the FP32 sum.  When the build proves that
 * every partial sum of a cell is exact -- every weight an integer multiple of 2^e with e >= -126,
 * and k_exc |j_exc| + k_inh |j_inh| below 2^24 * 2^e (as stored, e.g. bfloat16 weights) -- no add
 * rounds, so any order gives the same bits and the fold needs no ordering (EXACT). */
#define CORTEX_FOLD_AUTO 0           /* EXACT when proven, else ORDERED */
#define CORTEX_FOLD_ORDERED 1        /* lanes sharing a cell add in stream order (always valid) */
#define CORTEX_FOLD_EXACT 2          /* order-free adds; the build fails (UNSUPPORTED) unless proven */

/* delivery schemes (cortex_options.delivery) */
#define CORTEX_DELIVERY_RING 0       /* a spike's synapses are read at emission and added into a ring
                                        of future input, D = d_max + 1 slots per neuron */
#define CORTEX_DELIVERY_DELAY 1      /* delay-ordered (Sec. III-B "Varied Synaptic Delays", Sec. III-C
                                        spike buffer): each block's piece of a row sorted by
                                        (delay, target); the
                                        synapses of delay d of a spike at step e are read at step
                                        e + d into an accumulator of that step (d_min + 1 per neuron,
                                        in shared memory); the spikes of the last d_max steps are
                                        kept in a spike buffer.  Same results as RING, bit for bit.
                                        Persistent mode only; no ring to export or restore
                                        (cortex_get_ring, cortex_set_state, cortex_set_step and
                                        cortex_deliver return CORTEX_ERR_UNSUPPORTED).  Needs
                                        (d_max + 1) * (blocks + 2) <= 6400 for a network's
                                        blocks. */

/* step-loop modes (cortex_options.mode) */
#define CORTEX_MODE_PERSISTENT 0     /* one cooperative kernel per chunk, grid barrier inside */
#define CORTEX_MODE_SPLIT 1          /* an update kernel and a delivery kernel per window */

/* One network.  Units: ms, pF, mV, pA, Hz.  Neurons 0..n_exc-1 are excitatory, the rest
 * inhibitory.  Each neuron receives exactly k_exc excitatory and k_inh inhibitory synapses,
 * drawn with replacement (multapses and autapses allowed, Sec. II-A "x != y can be ignored").
 * Weights: j_exc for excitatory sources, j_inh for inhibitory ones; external drive: a Poisson
 * process of rate nu_ext_hz per neuron, each event adding j_ext to the synaptic current. */
typedef struct cortex_params {
  int32_t n_exc, n_inh, k_exc, k_inh;
  float tau_m, c_m, tau_syn, v_th, v_reset, e_l, t_ref, dt;
  float j_exc, j_inh;
  int32_t d_min, d_max;
  float nu_ext_hz, j_ext;
  int32_t weight_dtype;              /* CORTEX_F32 or CORTEX_BF16 */
} cortex_params;

/* Tuning overrides; zero-initialise for automatic choices. */
typedef struct cortex_options {
  int32_t ring;                      /* CORTEX_RING_* */
  int32_t mode;                      /* CORTEX_MODE_* */
  int32_t warps_per_block;           /* 0 = auto (14); 1..16 */
  int32_t targets_per_block;         /* 0 = auto; upper bound on targets owned by one block */
  int32_t steps_per_launch;          /* 0 = auto; steps per persistent launch (graph node) */
  int32_t use_graph;                 /* 0 = auto (on), 1 = on, -1 = off */
  int64_t raster_capacity;           /* 0 = auto; spikes kept on the device per network */
  double barrier_timeout_ms;         /* 0 = 2000 ms; device waits give up after this */
  int32_t spikes_per_round;          /* 0 = auto (the largest that fits, at most 32); else 1..32 */
  int32_t balance;                   /* block plan of a batch: 0 = equal targets per block,
                                        1 = equal synapses per block (targets x in-degree),
                                        2 = equal work per block, with net_work[b] the cost of one
                                        target of network b per step (needs net_work) */
  int32_t test_withhold_block;       /* test hook, 0 = off.  b + 1: block b of the persistent
                                        kernel never publishes its spikes, so every block's bounded
                                        wait at the window barrier runs out and cortex_simulate
                                        returns CORTEX_ERR_TIMEOUT (error path of the barrier) */
  const float* net_work;             /* balance 2: n_nets finite costs > 0 (any common unit), read
                                        by the build only; caller-owned; NULL otherwise */
  int32_t fold;                      /* CORTEX_FOLD_*: how delivery adds into a ring cell */
  int32_t l2_persist;                /* ring in global memory: 0 = auto (off), 1 = on, -1 = off.
                                        On: the launches mark the ring as persisting in L2 (an
                                        access-policy window), and the build raises the process's
                                        persisting-L2 limit (cudaLimitPersistingL2CacheSize) to the
                                        ring's size, at most the device maximum; the previous limit
                                        is restored when the last handle that raised it is freed.
                                        Off by default: the limit is process-wide state, and the
                                        window changes the step time by about 1% */
  int32_t delivery;                  /* CORTEX_DELIVERY_* */
  int32_t check_ownership;           /* debug mode, 0 = off.  1: the ownership check of Sec. IV-A
                                        ("Verification": a synapse or post-synaptic neuron touched
                                        by two threads is an error).  Every ring cell a delivery warp
                                        writes is stamped with the warp's id; a cell written by a
                                        second warp makes cortex_simulate return CORTEX_ERR_CHECK
                                        (no trap).  Ring delivery only (CORTEX_ERR_UNSUPPORTED with
                                        delay-ordered delivery); slower, and 4 more bytes per cell */
  int32_t helper_warp;               /* ring delivery: 1 = every block runs one more warp, which
                                        fetches the piece headers and builds the copy and fold
                                        descriptors of the coming rounds while the delivery warps
                                        fold (warps_per_block stays the number of delivery warps, at
                                        most 15); -1 = off; 0 = auto: on when the ring is in global
                                        memory, in persistent mode.  Same results. */
} cortex_options;

typedef struct cortex_stats_t {
  int64_t n_nets;
  int64_t n_neurons;                 /* over all networks */
  int64_t n_synapses;                /* over all networks */
  int64_t step;                      /* steps simulated so far */
  int64_t spikes;                    /* spikes emitted so far, all networks */
  int64_t events;                    /* synaptic events: sum over spikes of the out-degree */
  double build_ms;                   /* device time of the last build */
  double simulate_ms;                /* device time of the last cortex_simulate call */
  int64_t simulate_steps;            /* steps of the last cortex_simulate call */
  int64_t simulate_events;           /* events delivered during the last cortex_simulate */
  int32_t n_blocks;                  /* thread blocks (indegree sub-graphs) of the step kernel */
  int32_t threads_per_block;
  int32_t ring_in_smem;              /* 1 if the ring lives in shared memory */
  int32_t mode;                      /* CORTEX_MODE_* in use */
  int64_t device_bytes;              /* device memory held by the handle */
  int32_t spikes_per_round;          /* spikes staged per delivery round (fewest over a batch) */
  int32_t smem_bytes;                /* dynamic shared memory per block of the step kernel
                                        (the largest network layout of a batch) */
  int32_t exact_fold;                /* 1 if the delivery uses order-free adds (CORTEX_FOLD_EXACT) */
  int64_t l2_persist_bytes;          /* bytes of the ring in the persisting L2 window (0: none) */
  int32_t delivery;                  /* CORTEX_DELIVERY_* in use */
  int64_t build_h2d_bytes;           /* host -> device bytes the build copied (its inputs: the
                                        network parameters and the block plan) */
  int32_t helper_warp;               /* 1 if the ring kernel runs a helper warp per block */
} cortex_stats_t;

typedef struct cortex_net cortex_net;

/* Build one network on the device from its parameters and a 64-bit seed (Sec. II-B "problem
 * description" -> "domain decomposition").  Propagators are computed once in FP64 on the GPU
 * and rounded to FP32; connectivity is drawn by Philox4x32-10 per (target, draw) and sorted into
 * per-block sub-graphs, CSR by source inside each block (Eq. 5, Eq. 9-10, Sec. III-B).
 * stream: cudaStream_t or NULL.  opts may be NULL.  On success *out owns all device memory.
 * Errors: CORTEX_ERR_ARG (invalid parameters), CORTEX_ERR_UNSUPPORTED (sizes beyond the
 * layout limits: in-degree or targets per block > 65535, d_max > 255, more than 2,048 synapses
 * from one source into one block, a source's row (its out-degree) above 65,535 synapses, no block
 * plan within the SMs and their shared memory),
 * CORTEX_ERR_OOM, CORTEX_ERR_CUDA.  On error *out is NULL and nothing is leaked. */
int cortex_build(const cortex_params* params, uint64_t seed, const cortex_options* opts,
                 void* stream, cortex_net** out);

/* Build n_nets independent networks (params[n], seeds[n]) in one handle; they are stepped
 * together by one persistent kernel (each block owns a target range of one network).  Same
 * errors as cortex_build. */
int cortex_build_batch(const cortex_params* params, const uint64_t* seeds, int32_t n_nets,
                       const cortex_options* opts, void* stream, cortex_net** out);

/* The block plan cortex_build_batch makes (the domain decomposition of Sec. II-B: targets per
 * block, Eq. 9-10), computed on the host alone with no device call: for a GPU with n_sm SMs and
 * smem_per_block bytes of opt-in dynamic shared memory per block, targets_out[b] receives the
 * targets per block of network b (its last block may hold fewer) and *n_blocks_out (may be NULL)
 * the block count.  Same options and errors as the build's planning step: CORTEX_ERR_ARG,
 * CORTEX_ERR_UNSUPPORTED (no plan fits the SMs). */
int cortex_plan(const cortex_params* params, int32_t n_nets, const cortex_options* opts,
                int32_t n_sm, int64_t smem_per_block, int32_t* targets_out, int32_t* n_blocks_out);

/* Autotuner (the paper has no counterpart: its partition is fixed by processes and threads).
 * Builds the network(s) of params / seeds with each candidate plan -- warps per block, i.e. the
 * number and width of the per-warp indegree sub-graphs (Sec. III-B), in {8, 10, 12, 14, 16}, times the
 * block plan -- simulates trial_steps > 0 steps after one untimed launch, frees it, and returns
 * in *best the options of the fastest candidate (the other fields copied from base, which may be
 * NULL).  Block plans: balance 0 and 1, and, when net_work_out is not NULL and n_nets > 1,
 * balance 2 with each network's cost per target and step taken from the first candidate's
 * trial: the synaptic events it delivered per target and step, plus a fixed cost of one target
 * update (three values tried).  net_work_out: NULL or n_nets floats, caller-owned; when a
 * balance-2 candidate wins, it receives that candidate's costs and best->net_work points to it,
 * so it must outlive every build made with *best.  The simulation results do not depend on the
 * plan (the summation order is fixed by emission step, source and draw); only the time does.
 * best_ms_per_step and n_tried (candidates that could be built) may be NULL.  Candidates that
 * exceed the layout limits are skipped.  Errors: CORTEX_ERR_ARG, CORTEX_ERR_UNSUPPORTED (no
 * candidate could be built), CORTEX_ERR_CUDA, CORTEX_ERR_TIMEOUT, CORTEX_ERR_OOM. */
int cortex_autotune(const cortex_params* params, const uint64_t* seeds, int32_t n_nets,
                    const cortex_options* base, int32_t trial_steps, void* stream,
                    cortex_options* best, double* best_ms_per_step, int32_t* n_tried,
                    float* net_work_out);

/* cortex_autotune with a cache file (text, one line per tuned case, appended).  The key hashes
 * (FNV-1a 64) the GPU's name, SM count and shared memory per block, every network's parameters and
 * seed, the base options that shape a plan (ring, mode, targets_per_block, steps_per_launch,
 * spikes_per_round, fold, delivery) and trial_steps.  On a hit the cached plan is returned without
 * building anything (*hit = 1, *n_tried = 0, *best_ms_per_step the cached time); on a miss the
 * candidates are tried as cortex_autotune does and the winner is appended (*hit = 0).  cache_path
 * NULL: no cache.  hit may be NULL.  A line that does not parse is skipped; the last line with the
 * key wins.  Same errors as cortex_autotune, plus CORTEX_ERR_ARG when the file cannot be written. */
int cortex_autotune_cached(const cortex_params* params, const uint64_t* seeds, int32_t n_nets,
                           const cortex_options* base, int32_t trial_steps, void* stream,
                           const char* cache_path, cortex_options* best, double* best_ms_per_step,
                           int32_t* n_tried, float* net_work_out, int32_t* hit);

/* Advance every network by n_steps >= 0 steps from the current step (Sec. II-B loop: deliver,
 * update, compact spikes).  Continuing in pieces gives the same result as one call.
 * Synchronises the stream.  Errors: CORTEX_ERR_ARG, CORTEX_ERR_TIMEOUT (a grid-barrier or copy
 * wait gave up; the simulation state is undefined, later cortex_simulate calls on the handle
 * return CORTEX_ERR_TIMEOUT at once, and the handle can still be freed), CORTEX_ERR_CUDA.  If the
 * device raster is full, spikes keep being simulated and counted but no longer recorded, and
 * the call returns CORTEX_ERR_OVERFLOW after finishing all steps. */
int cortex_simulate(cortex_net* net, int64_t n_steps);

/* Copy the recorded spikes of network net_idx, ordered by (step, neuron id), into caller-owned
 * host arrays.  *n_inout: capacity on input, number of spikes on output.  If the capacity is too
 * small, nothing is copied, *n_inout receives the needed count and CORTEX_ERR_OVERFLOW is
 * returned.  steps/ids may be NULL when *n_inout is 0 (size query). */
int cortex_spikes(cortex_net* net, int32_t net_idx, int64_t* n_inout, int32_t* steps,
                  int32_t* ids);

/* Forget the recorded spikes (the simulation state is unchanged). */
int cortex_clear_spikes(cortex_net* net);

/* Counters and timings (see cortex_stats_t). */
int cortex_stats(cortex_net* net, cortex_stats_t* out);

/* Incoming synapses of targets [t_begin, t_end) of network net_idx, for connectivity checks:
 * for each synapse its source, target, delay (steps) and stored weight (as float).  Order:
 * by target block, then source, then target.  *n_inout as in cortex_spikes. */
int cortex_export_synapses(cortex_net* net, int32_t net_idx, int32_t t_begin, int32_t t_end,
                           int64_t* n_inout, int32_t* src, int32_t* tgt, int32_t* delay,
                           float* weight);

/* Neuron state of network net_idx (host arrays of its n neurons): membrane potential (mV),
 * synaptic current (pA), remaining refractory steps.  Any pointer may be NULL. */
int cortex_get_state(cortex_net* net, int32_t net_idx, float* v, float* i_syn, int32_t* refr);

/* Ring of future synaptic input of network net_idx (the delay buffer of Sec. III-B): D = d_max
 * + 1 slots per neuron, slot-major host array of D * n floats.  ring[s * n + i] is the summed
 * input neuron i takes in at the one step t' in [t, t + D) with t' mod D == s, t being the
 * current step (the next one cortex_simulate runs). */
int cortex_get_ring(cortex_net* net, int32_t net_idx, float* ring);

/* Checkpoint restore for network net_idx: V, I, refractory counts (each in 0..n_ref) and the ring
 * (layout as cortex_get_ring), host arrays of its n neurons.  Any pointer may be NULL to leave
 * that part unchanged.  Everything else a step reads is fixed by (params, seed, step): the
 * connectivity and the counter-based Poisson drive.  So a handle built from the same params and
 * seeds, given the state of every network and the step (cortex_set_step), continues a
 * checkpointed simulation bit for bit (Sec. II-B loop).  The recorded raster and the counters
 * are not part of the state.  A ring whose values are not sums of the network's weights on the
 * grid that made the order-free fold exact (exact_fold in cortex_stats) returns the handle to
 * the ordered fold, with a new shared-memory layout (same results).  Errors: CORTEX_ERR_ARG
 * (index, or a refractory count outside 0..n_ref; nothing is changed), CORTEX_ERR_TIMEOUT (an
 * earlier device wait of the handle timed out), CORTEX_ERR_UNSUPPORTED (the ordered fold's layout
 * does not fit; the handle then refuses cortex_simulate and cortex_deliver), CORTEX_ERR_CUDA. */
int cortex_set_state(cortex_net* net, int32_t net_idx, const float* v, const float* i_syn,
                     const int32_t* refr, const float* ring);

/* Set the current step of every network of the handle (the first step the next cortex_simulate
 * runs), step >= 0.  Errors: CORTEX_ERR_ARG, CORTEX_ERR_TIMEOUT, CORTEX_ERR_CUDA. */
int cortex_set_step(cortex_net* net, int64_t step);

/* The FP32 constants network net_idx uses, as computed on the device: out6 = {P11, P21,
 * P22 - 1 (= expm1(-h/tau_m), the form the update uses), w_exc, w_inh, j_ext}; thr = Poisson thresholds (up to 64 words), *n_thr their count,
 * *n_ref the refractory steps. */
int cortex_constants(cortex_net* net, int32_t net_idx, float* out6, uint32_t* thr,
                     int32_t* n_thr, int32_t* n_ref);

/* Deliver a given list of spikes of network net_idx, emitted at step t_emit, with the delivery
 * kernel alone (measurement of the delivery path, Sec. III-B).  ids: host array of n neuron
 * ids, any order, duplicates ignored.  The weights are added to the ring buffers exactly as in
 * a simulation step, so the network's future input changes.  reps: number of times the launch
 * is repeated (timing); *ms_out receives the mean device time of one launch (may be NULL);
 * *events_out the synaptic events of one launch (may be NULL). */
int cortex_deliver(cortex_net* net, int32_t net_idx, const int32_t* ids, int64_t n,
                   int64_t t_emit, int32_t reps, double* ms_out, int64_t* events_out);

/* Philox4x32-10 on the device for n counters (ctr: 4n words, key: 2n words, out: 4n words;
 * host arrays).  Used to check the device generator against its published definition. */
int cortex_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out);

/* The incoming synapses of targets [t_begin, t_end) of the network described by params and seed
 * -- the same Philox connectivity cortex_build draws -- as a CSR by source, computed WITHOUT
 * allocating any device memory.  The paper has no counterpart: this exists for callers that cannot
 * call the device allocator when they need connectivity (for example while another framework owns
 * the whole device memory pool).  All output pointers are DEVICE pointers owned by the caller:
 * row_ptr[n + 1] (n = n_exc + n_inh; synapses of source s are entries row_ptr[s]..row_ptr[s+1]-1,
 * ordered by target), tgt/delay/weight[(t_end - t_begin) * (k_exc + k_inh)] (delay in steps,
 * weight as stored: bfloat16-rounded when weight_dtype is CORTEX_BF16).  Work is issued on stream
 * and the call synchronises it.
 * Working memory is one static 8 MiB device array per GPU: (n + 1) + (t_end - t_begin) * K must be
 * at most 2^21 words and t_end - t_begin at most 65536; larger sizes return CORTEX_ERR_UNSUPPORTED
 * without launching anything.  No source may have more than 2048 synapses in the range: that is
 * found on the device, after the outputs were partly written, and returns CORTEX_ERR_UNSUPPORTED
 * with the outputs undefined.  Every call copies a status word to pageable host memory and
 * synchronises the stream, so a call cannot be captured in a CUDA graph.  The first call on a
 * device looks up the array's device address (with that device current).  Every call reuses the same array (it is cleared
 * at the start of each call), so calls that overlap on the GPU -- on different streams or host
 * threads -- race and must be serialised by the caller.  Errors: CORTEX_ERR_ARG (bad parameters
 * or NULL outputs), CORTEX_ERR_UNSUPPORTED (size limits), CORTEX_ERR_CUDA. */
int cortex_subgraph_noalloc(const cortex_params* params, uint64_t seed, int32_t t_begin, int32_t t_end,
                            void* stream, int32_t* row_ptr, int32_t* tgt, int32_t* delay, float* weight);

/* Ownership stamps of network net_idx (built with check_ownership = 1): for every ring cell, the
 * id of the warp that wrote it during the simulation, block * 16 + warp + 1 (block: the index in
 * the handle's block list, the blocks of network b following those of networks 0..b-1), 0 if
 * no delivery wrote it.  Host array of D * n words, slot-major like cortex_get_ring.  Errors:
 * CORTEX_ERR_ARG (no stamps: check mode off), CORTEX_ERR_CUDA. */
int cortex_get_stamps(cortex_net* net, int32_t net_idx, uint32_t* stamps);

/* Host-only check of ownership stamps against the block plan (no device call): a network of n
 * neurons cut into blocks of targets_per_block targets (the last may hold fewer), whose first block
 * has index first_block, each block split into `warps` delivery sub-ranges of ceil(T_b / warps)
 * targets.  The owner of target i is warp (i mod T_b) / ceil(T_b / warps) of block first_block +
 * i / T_b; every nonzero stamp of a cell of target i (stamps: D * n words, slot-major) must name
 * it.  *n_bad receives the number of cells stamped by another warp, *first_bad the index of the
 * first of them (-1 if none).  Errors: CORTEX_ERR_ARG. */
int cortex_check_stamps(int32_t n, int32_t depth, int32_t targets_per_block, int32_t warps,
                        int32_t first_block, const uint32_t* stamps, int64_t* n_bad,
                        int64_t* first_bad);

/* Release everything the handle owns.  NULL is allowed. */
void cortex_free(cortex_net* net);

/* Text of a status code; and of the calling thread's last error (empty if none). */
const char* cortex_strerror(int code);
const char* cortex_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CORTEX_H */
