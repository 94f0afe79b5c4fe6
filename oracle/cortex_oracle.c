/*
 * cortex_oracle.c -- plain, slow CPU reference simulator (single-threaded, or target-partitioned
 * over threads with bitwise-identical results).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark load this file.  The CUDA library never links or calls it, and it shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it computes (paper: CORTEX, arXiv 2406.03762):
 *   - LIF neurons, Eq. 1, with threshold / reset / refractory period, Eq. 2;
 *   - exponentially decaying synaptic current, Eq. 3, read as a current-based synapse: an
 *     arriving spike adds its weight W_ji (pA) to the synaptic current I_syn,i;
 *   - the simulation loop of Sec. II-B: spikes of the pre-synaptic neurons act on their
 *     post-synaptic neurons after the synaptic delay, then every neuron updates its state and
 *     produces the next spikes.
 * The paper names no integrator, no random-number layout and no Poisson method.  The readings
 * taken here (exact integration, Philox4x32-10 counters, inversion sampling with 32-bit
 * thresholds, the fixed FP32 operation sequence) are listed in the design notes of the repo.
 *
 * Precision modes:
 *   ORACLE_FP32: every state variable, propagator and weight is a float, and the update uses
 *                exactly the float operations written in step_neuron_f32() (fmaf where written,
 *                nothing else fused: compile with -ffp-contract=off).
 *   ORACLE_FP64: the same sequence in double, from the double parameters (error reference).
 *
 * Connectivity (fixed in-degree, Sec. IV-A "number of incoming synaptic interactions per neuron
 * is fixed"): target i draws K_E excitatory and K_I inhibitory sources with replacement, each
 * with an integer delay, from Philox4x32-10 (Salmon et al., SC'11).  The outgoing lists are
 * sorted by (source, target, draw index), so delivery adds weights to a target's ring cell in
 * the order: emission step, source id, draw index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_OOM (-2)

#define ORACLE_FP32 0
#define ORACLE_FP64 1

#define STREAM_CONN 1u
#define STREAM_V0 2u
#define STREAM_POISSON 3u

#define POISSON_TABLE_CAP 64

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",  */
/* SC'11).  Ten rounds of the 4x32 Philox S-box: two 32x32->64 multiplications by the round  */
/* multipliers, the high halves xor-ed with the other counter words and the round key, and a  */
/* Weyl-sequence key schedule.                                                                  */
/* ------------------------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;   /* round multipliers */
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;   /* key-schedule increments */
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)mult0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)mult1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += weyl0;
    k1 += weyl1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t scale_u32(uint32_t u, uint32_t n) {           /* floor(u * n / 2^32) */
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------------------------ */
/* Parameters                                                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct oracle_params {
  int32_t n_exc, n_inh, k_exc, k_inh;
  double tau_m, c_m, tau_syn, v_th, v_reset, e_l, t_ref, dt; /* ms, pF, mV */
  double j_exc, j_inh;                                       /* pA */
  int32_t d_min, d_max;                                      /* delays in steps, inclusive */
  double nu_ext_hz, j_ext;                                   /* external Poisson drive */
  double i_e;              /* constant bias current in pA; 0 for every network configuration */
  int32_t precision;       /* ORACLE_FP32 or ORACLE_FP64 */
  int32_t bf16_weights;    /* FP32 mode: recurrent weights rounded to bfloat16 first */
  int32_t poisson_on;      /* 0 switches the external drive off (closed-form tests) */
} oracle_params;

/* bfloat16 round-to-nearest-even of a float, returned as float. */
float oracle_round_bf16(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  if ((b & 0x7f800000u) == 0x7f800000u) return x;           /* inf / nan unchanged */
  uint32_t lsb = (b >> 16) & 1u;
  b += 0x7fffu + lsb;
  b &= 0xffff0000u;
  float y;
  memcpy(&y, &b, 4);
  return y;
}

/* Exact-integration propagators for Eq. 1 with an exponential current (Eq. 3 read as a current
 * synapse), R = tau_m / C_m, u_rest = E_L:
 *   I(t+h) = P11 I(t)                    P11 = exp(-h/tau_syn)
 *   V(t+h) = P22 V(t) + P21 I(t) + P20 I_e
 *            P22 = exp(-h/tau_m)
 *            P21 = tau_m tau_syn / (C (tau_syn - tau_m)) (P11 - P22)
 *            P20 = tau_m / C (1 - P22)
 * V is measured relative to E_L.  n_ref = round(t_ref / h) steps of clamping (Eq. 2).
 * The update is evaluated as V + ((P22 - 1) V + P21 I) with P22 - 1 = expm1(-h/tau_m): the same
 * map, but P22 lies within 1% of 1, and its float rounding, divided by 1 - P22 in the stationary
 * potential, would bias V by up to ~3e-6 relative; P22 - 1 rounds with 6e-8 relative error. */
typedef struct { double p11, p21, p22, p20, p22m1; int32_t n_ref; } props64;

static props64 compute_props(double tau_m, double c_m, double tau_syn, double t_ref, double h) {
  props64 q;
  q.p22 = exp(-h / tau_m);
  q.p22m1 = expm1(-h / tau_m);
  q.p11 = exp(-h / tau_syn);
  q.p21 = tau_m * tau_syn / (c_m * (tau_syn - tau_m)) * (q.p11 - q.p22);
  q.p20 = tau_m / c_m * (1.0 - q.p22);
  q.n_ref = (int32_t)llround(t_ref / h);
  return q;
}

/* FP32 mode takes its parameters as the float values a float parameter record would hold. */
static double as_f(double x) { return (double)(float)x; }

void oracle_propagators(const oracle_params* p, double out64[5], float out32[5], int32_t* n_ref) {
  props64 q = compute_props(p->tau_m, p->c_m, p->tau_syn, p->t_ref, p->dt);
  out64[0] = q.p11; out64[1] = q.p21; out64[2] = q.p22; out64[3] = q.p20; out64[4] = q.p22m1;
  props64 f = compute_props(as_f(p->tau_m), as_f(p->c_m), as_f(p->tau_syn), as_f(p->t_ref),
                            as_f(p->dt));
  out32[0] = (float)f.p11; out32[1] = (float)f.p21; out32[2] = (float)f.p22; out32[3] = (float)f.p20;
  out32[4] = (float)f.p22m1;
  *n_ref = (p->precision == ORACLE_FP32) ? f.n_ref : q.n_ref;
}

/* Poisson(lambda) by inversion: thr[k] = floor(2^32 * P(X <= k)), saturated at 2^32-1, where the
 * table stops.  A draw u (uint32) gives k = the smallest k with u < thr[k], capped at n-1.
 * pmf_0 = exp(-lambda), pmf_k = pmf_{k-1} * lambda / k, both in double.
 * Returns the table length, or -1 if the table does not saturate within the cap. */
int oracle_poisson_table(double lambda, uint32_t* thr, int cap) {
  if (!(lambda >= 0.0) || cap < 1) return -1;
  double pmf = exp(-lambda);
  double cdf = pmf;
  for (int k = 0; k < cap; ++k) {
    if (k > 0) {
      pmf = pmf * lambda / (double)k;
      cdf = cdf + pmf;
    }
    double x = cdf * 4294967296.0;
    if (x >= 4294967295.0) {
      thr[k] = 0xffffffffu;
      return k + 1;
    }
    thr[k] = (uint32_t)floor(x);
  }
  return -1;
}

int oracle_poisson_sample(uint32_t u, const uint32_t* thr, int n) {
  int k = 0;
  while (k < n - 1 && u >= thr[k]) ++k;
  return k;
}

/* Draw j of target i (fixed in-degree, with replacement):
 *   r = Philox(ctr = (i, j/2, STREAM_CONN, 0), key = (seed_lo, seed_hi)); words (2(j%2), 2(j%2)+1)
 *   j <  K_E: source = floor(a N_E / 2^32)          (excitatory population 0..N_E-1)
 *   j >= K_E: source = N_E + floor(a N_I / 2^32)    (inhibitory population N_E..N-1)
 *   delay = d_min + floor(b (d_max - d_min + 1) / 2^32) */
void oracle_draw(uint64_t seed, int32_t n_exc, int32_t n_inh, int32_t k_exc, int32_t d_min,
                 int32_t d_max, int64_t i, int64_t j, int32_t* src, int32_t* delay) {
  uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(j >> 1), STREAM_CONN, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  oracle_philox4x32_10(ctr, key, r);
  uint32_t a = r[2 * (j & 1)], b = r[2 * (j & 1) + 1];
  if (j < k_exc) *src = (int32_t)scale_u32(a, (uint32_t)n_exc);
  else *src = n_exc + (int32_t)scale_u32(a, (uint32_t)n_inh);
  *delay = d_min + (int32_t)scale_u32(b, (uint32_t)(d_max - d_min + 1));
}

/* Initial membrane potential: V0 = V_reset + (V_th - V_reset) * frac, frac = (u >> 8) 2^-24 with
 * u = word 0 of Philox(ctr = (i, 0, STREAM_V0, 0)).  In FP32 mode each operation rounds to float. */
static uint32_t v0_word(uint64_t seed, int64_t i) {
  uint32_t ctr[4] = {(uint32_t)i, 0u, STREAM_V0, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  oracle_philox4x32_10(ctr, key, r);
  return r[0];
}

/* External drive of neuron i at step t: word (i mod 4) of Philox(ctr = (floor(i / 4), t,
 * STREAM_POISSON, 0)); one generator call serves four consecutive neurons at one step. */
static uint32_t poisson_word(uint64_t seed, int64_t i, int64_t t) {
  uint32_t ctr[4] = {(uint32_t)(i >> 2), (uint32_t)t, STREAM_POISSON, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  oracle_philox4x32_10(ctr, key, r);
  return r[i & 3];
}

/* ------------------------------------------------------------------------------------------ */
/* Network                                                                                     */
/* ------------------------------------------------------------------------------------------ */
typedef struct oracle_net {
  oracle_params p;
  uint64_t seed;
  int64_t n;                 /* neurons */
  int32_t depth;             /* ring depth D = d_max + 1 */
  /* outgoing lists (CSR by source), sorted by (source, target, draw index) */
  int64_t* row;              /* [n + 1] */
  int32_t* out_tgt;          /* [n_syn] */
  uint8_t* out_dly;          /* [n_syn] delay in steps (< 256) */
  double* out_w;             /* [n_syn] only for hand-built graphs; NULL: weight by population */
  int64_t n_syn;
  /* state */
  int64_t step;
  float* v32; float* i32; float* ring32;       /* FP32 mode, ring [n][D] */
  double* v64; double* i64; double* ring64;    /* FP64 mode */
  int32_t* refr;
  /* constants */
  float p11f, p21f, p22f, p20f, p22m1f, vthf, vresetf, wexf, winf, jextf, ief;
  double p11, p21, p22, p20, p22m1;
  int32_t n_ref;
  uint32_t thr[POISSON_TABLE_CAP];
  int n_thr;
  /* outputs */
  int64_t raster_n, raster_cap;
  int64_t* raster_step;
  int32_t* raster_id;
  int64_t events;            /* sum over emitted spikes of the source's out-degree */
  int32_t* count_ring;       /* optional [n][D] event counter (delivery invariant tests) */
  int64_t* consumed_events;  /* optional [n] events consumed per target */
  double* consumed_weight;   /* optional [n] weight consumed per target (double sum) */
  double* weight_ring;       /* optional [n][D] double shadow of the ring for the above */
  /* target-partitioned form (oracle_build_par): part k owns targets [part_lo[k], part_lo[k+1])
   * and keeps its own CSR by source of their incoming synapses, sorted by (source, target, draw) */
  int32_t n_part;            /* 0: the single lists above */
  int32_t sim_threads;       /* threads that step the parts (any number gives the same bits) */
  int64_t* part_lo;          /* [n_part + 1] */
  int64_t** prow;            /* [n_part][n + 1] */
  int32_t** ptgt;            /* [n_part][synapses of the part] */
  uint8_t** pdly;
} oracle_net;

static void* xcalloc(size_t n, size_t sz) { return (n == 0) ? calloc(1, 1) : calloc(n, sz); }

static int validate(const oracle_params* p) {
  if (p->n_exc < 0 || p->n_inh < 0 || p->n_exc + p->n_inh <= 0) return 0;
  if (p->k_exc < 0 || p->k_inh < 0) return 0;
  if (p->k_exc > 0 && p->n_exc == 0) return 0;
  if (p->k_inh > 0 && p->n_inh == 0) return 0;
  if (p->d_min < 1 || p->d_max < p->d_min || p->d_max > 255) return 0;
  if (!(p->tau_m > 0) || !(p->tau_syn > 0) || !(p->c_m > 0) || !(p->dt > 0)) return 0;
  if (p->tau_m == p->tau_syn) return 0;
  if (!(p->t_ref >= 0)) return 0;
  return 1;
}

static int init_common(oracle_net* net, const oracle_params* p, uint64_t seed) {
  net->p = *p;
  net->seed = seed;
  net->n = (int64_t)p->n_exc + p->n_inh;
  net->depth = p->d_max + 1;
  double o64[5]; float o32[5]; int32_t nref;
  oracle_propagators(p, o64, o32, &nref);
  net->p11 = o64[0]; net->p21 = o64[1]; net->p22 = o64[2]; net->p20 = o64[3]; net->p22m1 = o64[4];
  net->p11f = o32[0]; net->p21f = o32[1]; net->p22f = o32[2]; net->p20f = o32[3]; net->p22m1f = o32[4];
  net->n_ref = nref;
  net->vthf = (float)p->v_th; net->vresetf = (float)p->v_reset;
  net->wexf = (float)p->j_exc; net->winf = (float)p->j_inh;
  if (p->bf16_weights) { net->wexf = oracle_round_bf16(net->wexf); net->winf = oracle_round_bf16(net->winf); }
  net->jextf = (float)p->j_ext; net->ief = (float)p->i_e;
  /* lambda = nu_ext[Hz] * dt[ms] / 1000 (expected external spikes per step) */
  double lam = (p->precision == ORACLE_FP32) ? as_f(p->nu_ext_hz) * as_f(p->dt) / 1000.0
                                             : p->nu_ext_hz * p->dt / 1000.0;
  net->n_thr = oracle_poisson_table(lam, net->thr, POISSON_TABLE_CAP);
  if (p->poisson_on && net->n_thr < 1) return ORACLE_ERR_ARG;
  size_t n = (size_t)net->n, nd = n * (size_t)net->depth;
  net->refr = (int32_t*)xcalloc(n, sizeof(int32_t));
  if (p->precision == ORACLE_FP32) {
    net->v32 = (float*)xcalloc(n, sizeof(float));
    net->i32 = (float*)xcalloc(n, sizeof(float));
    net->ring32 = (float*)xcalloc(nd, sizeof(float));
    if (!net->v32 || !net->i32 || !net->ring32) return ORACLE_ERR_OOM;
  } else {
    net->v64 = (double*)xcalloc(n, sizeof(double));
    net->i64 = (double*)xcalloc(n, sizeof(double));
    net->ring64 = (double*)xcalloc(nd, sizeof(double));
    if (!net->v64 || !net->i64 || !net->ring64) return ORACLE_ERR_OOM;
  }
  if (!net->refr) return ORACLE_ERR_OOM;
  /* initial potentials */
  for (int64_t i = 0; i < net->n; ++i) {
    uint32_t u = v0_word(seed, i);
    uint32_t m = u >> 8;
    if (p->precision == ORACLE_FP32) {
      float frac = (float)m * 0x1p-24f;
      float span = net->vthf - net->vresetf;
      float prod = span * frac;
      net->v32[i] = net->vresetf + prod;
    } else {
      double frac = (double)m * 0x1p-24;
      net->v64[i] = p->v_reset + (p->v_th - p->v_reset) * frac;
    }
  }
  net->raster_cap = 1024;
  net->raster_step = (int64_t*)malloc(sizeof(int64_t) * (size_t)net->raster_cap);
  net->raster_id = (int32_t*)malloc(sizeof(int32_t) * (size_t)net->raster_cap);
  if (!net->raster_step || !net->raster_id) return ORACLE_ERR_OOM;
  return ORACLE_OK;
}

void oracle_free(oracle_net* net) {
  if (!net) return;
  free(net->row); free(net->out_tgt); free(net->out_dly); free(net->out_w);
  free(net->v32); free(net->i32); free(net->ring32);
  free(net->v64); free(net->i64); free(net->ring64);
  free(net->refr); free(net->raster_step); free(net->raster_id);
  free(net->count_ring); free(net->consumed_events); free(net->consumed_weight);
  free(net->weight_ring);
  for (int32_t k = 0; k < net->n_part; ++k) {
    if (net->prow) free(net->prow[k]);
    if (net->ptgt) free(net->ptgt[k]);
    if (net->pdly) free(net->pdly[k]);
  }
  free(net->part_lo); free(net->prow); free(net->ptgt); free(net->pdly);
  free(net);
}

/* Fixed in-degree network from Philox draws.  Two passes over the draws (count, then fill);
 * the fill visits targets in ascending order and draws in ascending order, so every source's
 * list comes out sorted by (target, draw index) without a separate sort. */
int oracle_build(const oracle_params* p, uint64_t seed, oracle_net** out) {
  *out = NULL;
  if (!validate(p)) return ORACLE_ERR_ARG;
  oracle_net* net = (oracle_net*)calloc(1, sizeof(oracle_net));
  if (!net) return ORACLE_ERR_OOM;
  int rc = init_common(net, p, seed);
  if (rc != ORACLE_OK) { oracle_free(net); return rc; }
  int64_t n = net->n, k = (int64_t)p->k_exc + p->k_inh;
  net->n_syn = n * k;
  net->row = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  net->out_tgt = (int32_t*)xcalloc((size_t)net->n_syn, sizeof(int32_t));
  net->out_dly = (uint8_t*)xcalloc((size_t)net->n_syn, sizeof(uint8_t));
  int64_t* cursor = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  if (!net->row || !net->out_tgt || !net->out_dly || !cursor) {
    free(cursor); oracle_free(net); return ORACLE_ERR_OOM;
  }
  int32_t s, d;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < k; ++j) {
      oracle_draw(seed, p->n_exc, p->n_inh, p->k_exc, p->d_min, p->d_max, i, j, &s, &d);
      net->row[s + 1] += 1;
    }
  for (int64_t q = 0; q < n; ++q) net->row[q + 1] += net->row[q];
  for (int64_t q = 0; q < n; ++q) cursor[q] = net->row[q];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < k; ++j) {
      oracle_draw(seed, p->n_exc, p->n_inh, p->k_exc, p->d_min, p->d_max, i, j, &s, &d);
      int64_t pos = cursor[s]++;
      net->out_tgt[pos] = (int32_t)i;
      net->out_dly[pos] = (uint8_t)d;
    }
  free(cursor);
  *out = net;
  return ORACLE_OK;
}

/* Hand-built graph (brute-force tests): explicit edges with their own weights.  Edges are kept
 * in the order given within each source (the caller lists them in the intended order). */
int oracle_build_edges(const oracle_params* p, uint64_t seed, int64_t n_edges, const int32_t* src,
                       const int32_t* tgt, const int32_t* delay, const double* w, oracle_net** out) {
  *out = NULL;
  if (!validate(p)) return ORACLE_ERR_ARG;
  oracle_net* net = (oracle_net*)calloc(1, sizeof(oracle_net));
  if (!net) return ORACLE_ERR_OOM;
  int rc = init_common(net, p, seed);
  if (rc != ORACLE_OK) { oracle_free(net); return rc; }
  int64_t n = net->n;
  for (int64_t e = 0; e < n_edges; ++e)
    if (src[e] < 0 || src[e] >= n || tgt[e] < 0 || tgt[e] >= n || delay[e] < p->d_min ||
        delay[e] > p->d_max) { oracle_free(net); return ORACLE_ERR_ARG; }
  net->n_syn = n_edges;
  net->row = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  net->out_tgt = (int32_t*)xcalloc((size_t)n_edges, sizeof(int32_t));
  net->out_dly = (uint8_t*)xcalloc((size_t)n_edges, sizeof(uint8_t));
  net->out_w = (double*)xcalloc((size_t)n_edges, sizeof(double));
  int64_t* cursor = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  if (!net->row || !net->out_tgt || !net->out_dly || !net->out_w || !cursor) {
    free(cursor); oracle_free(net); return ORACLE_ERR_OOM;
  }
  for (int64_t e = 0; e < n_edges; ++e) net->row[src[e] + 1] += 1;
  for (int64_t q = 0; q < n; ++q) net->row[q + 1] += net->row[q];
  for (int64_t q = 0; q < n; ++q) cursor[q] = net->row[q];
  for (int64_t e = 0; e < n_edges; ++e) {
    int64_t pos = cursor[src[e]]++;
    net->out_tgt[pos] = tgt[e];
    net->out_dly[pos] = (uint8_t)delay[e];
    net->out_w[pos] = w[e];
  }
  free(cursor);
  *out = net;
  return ORACLE_OK;
}

/* Turn on the per-target delivery bookkeeping (event counts and double weight sums). */
int oracle_enable_accounting(oracle_net* net) {
  size_t n = (size_t)net->n, nd = n * (size_t)net->depth;
  net->count_ring = (int32_t*)xcalloc(nd, sizeof(int32_t));
  net->weight_ring = (double*)xcalloc(nd, sizeof(double));
  net->consumed_events = (int64_t*)xcalloc(n, sizeof(int64_t));
  net->consumed_weight = (double*)xcalloc(n, sizeof(double));
  if (!net->count_ring || !net->weight_ring || !net->consumed_events || !net->consumed_weight)
    return ORACLE_ERR_OOM;
  return ORACLE_OK;
}

static int push_spike(oracle_net* net, int64_t t, int32_t id) {
  if (net->raster_n == net->raster_cap) {
    int64_t cap = net->raster_cap * 2;
    int64_t* s = (int64_t*)realloc(net->raster_step, sizeof(int64_t) * (size_t)cap);
    if (!s) return ORACLE_ERR_OOM;
    net->raster_step = s;
    int32_t* d = (int32_t*)realloc(net->raster_id, sizeof(int32_t) * (size_t)cap);
    if (!d) return ORACLE_ERR_OOM;
    net->raster_id = d;
    net->raster_cap = cap;
  }
  net->raster_step[net->raster_n] = t;
  net->raster_id[net->raster_n] = id;
  net->raster_n += 1;
  return ORACLE_OK;
}

/* One neuron, one step, FP32 (Eq. 1-3 with exact integration).  Returns 1 on a spike.
 *   1. in  = ring[i][t mod D]; the cell is cleared.
 *   2. k   = Poisson draw; ext = k * J_ext.
 *   3. refractory: V = V_reset and the counter counts down; otherwise
 *      V = V + fma(P22 - 1, V, P21 * I) with the old I (+ P20 * I_e when a bias current is set).
 *   4. I = fma(P11, I, in); I = I + ext.
 *   5. V >= V_th: spike, V = V_reset, counter = n_ref (Eq. 2). */
static int step_neuron_f32(oracle_net* net, int64_t i, int64_t t) {
  size_t cell = (size_t)i * (size_t)net->depth + (size_t)(t % net->depth);
  float in = net->ring32[cell];
  net->ring32[cell] = 0.0f;
  float v = net->v32[i], cur = net->i32[i];
  if (net->refr[i] > 0) {
    v = net->vresetf;
    net->refr[i] -= 1;
  } else {
    float pi = net->p21f * cur;
    float dv = fmaf(net->p22m1f, v, pi);
    v = v + dv;
    if (net->ief != 0.0f) v = v + net->p20f * net->ief;
  }
  cur = fmaf(net->p11f, cur, in);
  if (net->p.poisson_on) {
    int k = oracle_poisson_sample(poisson_word(net->seed, i, t), net->thr, net->n_thr);
    float ext = (float)k * net->jextf;
    cur = cur + ext;
  }
  int spiked = 0;
  if (v >= net->vthf) {
    spiked = 1;
    v = net->vresetf;
    net->refr[i] = net->n_ref;
  }
  net->v32[i] = v;
  net->i32[i] = cur;
  return spiked;
}

static int step_neuron_f64(oracle_net* net, int64_t i, int64_t t) {
  size_t cell = (size_t)i * (size_t)net->depth + (size_t)(t % net->depth);
  double in = net->ring64[cell];
  net->ring64[cell] = 0.0;
  double v = net->v64[i], cur = net->i64[i];
  if (net->refr[i] > 0) {
    v = net->p.v_reset;
    net->refr[i] -= 1;
  } else {
    double pi = net->p21 * cur;
    v = v + fma(net->p22m1, v, pi);
    if (net->p.i_e != 0.0) v = v + net->p20 * net->p.i_e;
  }
  cur = fma(net->p11, cur, in);
  if (net->p.poisson_on) {
    int k = oracle_poisson_sample(poisson_word(net->seed, i, t), net->thr, net->n_thr);
    double ext = (double)k * net->p.j_ext;
    cur = cur + ext;
  }
  int spiked = 0;
  if (v >= net->p.v_th) {
    spiked = 1;
    v = net->p.v_reset;
    net->refr[i] = net->n_ref;
  }
  net->v64[i] = v;
  net->i64[i] = cur;
  return spiked;
}

/* Deliver the spike of source s emitted at step t: every outgoing synapse (tgt, d, w) adds w to
 * ring[tgt][(t + d) mod D], in list order (target, draw index). */
static void deliver(oracle_net* net, int32_t s, int64_t t) {
  const int64_t b = net->row[s], e = net->row[s + 1];
  const int is_exc = s < net->p.n_exc;
  net->events += e - b;
  for (int64_t q = b; q < e; ++q) {
    size_t cell = (size_t)net->out_tgt[q] * (size_t)net->depth +
                  (size_t)((t + net->out_dly[q]) % net->depth);
    if (net->p.precision == ORACLE_FP32) {
      float w = net->out_w ? (float)net->out_w[q] : (is_exc ? net->wexf : net->winf);
      net->ring32[cell] = net->ring32[cell] + w;
    } else {
      double w = net->out_w ? net->out_w[q] : (is_exc ? net->p.j_exc : net->p.j_inh);
      net->ring64[cell] = net->ring64[cell] + w;
    }
    if (net->count_ring) {
      net->count_ring[cell] += 1;
      net->weight_ring[cell] += net->out_w ? net->out_w[q] : (is_exc ? net->p.j_exc : net->p.j_inh);
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Target-partitioned form (Sec. III-B "Avoid Data Racing": each thread owns a set of post-      */
/* synaptic neurons and the synapses into them, so no two threads write the same ring cell).     */
/* ------------------------------------------------------------------------------------------ */
/* Part k builds the incoming synapses of its target range exactly as oracle_build does for all
 * targets (ascending targets, ascending draws), so the part's list of a source is the global list
 * of that source restricted to the part's targets, in the same (target, draw) order.  Every ring
 * cell therefore receives the same adds in the same order as in the single-list form: the results
 * are the same bits, whatever the number of parts. */
int oracle_build_par(const oracle_params* p, uint64_t seed, int32_t n_part, oracle_net** out) {
  *out = NULL;
  if (!validate(p) || n_part < 1) return ORACLE_ERR_ARG;
  oracle_net* net = (oracle_net*)calloc(1, sizeof(oracle_net));
  if (!net) return ORACLE_ERR_OOM;
  int rc = init_common(net, p, seed);
  if (rc != ORACLE_OK) { oracle_free(net); return rc; }
  const int64_t n = net->n, k = (int64_t)p->k_exc + p->k_inh;
  if (n_part > n) n_part = (int32_t)n;
  net->n_syn = n * k;
  net->part_lo = (int64_t*)xcalloc((size_t)n_part + 1, sizeof(int64_t));
  net->prow = (int64_t**)xcalloc((size_t)n_part, sizeof(int64_t*));
  net->ptgt = (int32_t**)xcalloc((size_t)n_part, sizeof(int32_t*));
  net->pdly = (uint8_t**)xcalloc((size_t)n_part, sizeof(uint8_t*));
  if (!net->part_lo || !net->prow || !net->ptgt || !net->pdly) { oracle_free(net); return ORACLE_ERR_OOM; }
  net->n_part = n_part;
  net->sim_threads = n_part;
  for (int32_t q = 0; q <= n_part; ++q) net->part_lo[q] = n * q / n_part;
  int failed = 0;
#pragma omp parallel for num_threads(n_part) schedule(static, 1) reduction(| : failed)
  for (int32_t q = 0; q < n_part; ++q) {
    const int64_t lo = net->part_lo[q], hi = net->part_lo[q + 1];
    int64_t* row = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
    int64_t* cursor = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
    int32_t* tgt = (int32_t*)xcalloc((size_t)((hi - lo) * k), sizeof(int32_t));
    uint8_t* dly = (uint8_t*)xcalloc((size_t)((hi - lo) * k), sizeof(uint8_t));
    net->prow[q] = row; net->ptgt[q] = tgt; net->pdly[q] = dly;
    if (!row || !cursor || !tgt || !dly) { free(cursor); failed |= 1; continue; }
    int32_t s, d;
    for (int64_t i = lo; i < hi; ++i)
      for (int64_t j = 0; j < k; ++j) {
        oracle_draw(seed, p->n_exc, p->n_inh, p->k_exc, p->d_min, p->d_max, i, j, &s, &d);
        row[s + 1] += 1;
      }
    for (int64_t x = 0; x < n; ++x) row[x + 1] += row[x];
    for (int64_t x = 0; x < n; ++x) cursor[x] = row[x];
    for (int64_t i = lo; i < hi; ++i)
      for (int64_t j = 0; j < k; ++j) {
        oracle_draw(seed, p->n_exc, p->n_inh, p->k_exc, p->d_min, p->d_max, i, j, &s, &d);
        int64_t pos = cursor[s]++;
        tgt[pos] = (int32_t)i;
        dly[pos] = (uint8_t)d;
      }
    free(cursor);
  }
  if (failed) { oracle_free(net); return ORACLE_ERR_OOM; }
  *out = net;
  return ORACLE_OK;
}

/* Threads that step the parts of a target-partitioned network (1 .. n_part). */
int oracle_set_threads(oracle_net* net, int32_t threads) {
  if (net->n_part < 1 || threads < 1) return ORACLE_ERR_ARG;
  net->sim_threads = threads < net->n_part ? threads : net->n_part;
  return ORACLE_OK;
}

/* Deliver the spike of source s emitted at step t onto the targets of part q (its own list). */
static void deliver_part(oracle_net* net, int32_t q, int32_t s, int64_t t) {
  const int64_t* row = net->prow[q];
  const int is_exc = s < net->p.n_exc;
  for (int64_t e = row[s]; e < row[s + 1]; ++e) {
    size_t cell = (size_t)net->ptgt[q][e] * (size_t)net->depth + (size_t)((t + net->pdly[q][e]) % net->depth);
    if (net->p.precision == ORACLE_FP32) {
      float w = is_exc ? net->wexf : net->winf;
      net->ring32[cell] = net->ring32[cell] + w;
    } else {
      double w = is_exc ? net->p.j_exc : net->p.j_inh;
      net->ring64[cell] = net->ring64[cell] + w;
    }
  }
}

/* The simulation loop of oracle_simulate with the target ranges stepped by their own threads:
 * every part updates its neurons; the spikes are recorded in ascending id (one thread); every part
 * delivers every spike, in ascending source order, onto its own targets. */
static int simulate_par(oracle_net* net, int64_t n_steps) {
  char* emitted = (char*)xcalloc((size_t)net->n, 1);
  if (!emitted) return ORACLE_ERR_OOM;
  int rc = ORACLE_OK;
  const int32_t n_part = net->n_part;
#pragma omp parallel num_threads(net->sim_threads)
  {
    for (int64_t step = 0; step < n_steps; ++step) {
      const int64_t t = net->step + step;
#pragma omp for schedule(static, 1)
      for (int32_t q = 0; q < n_part; ++q)
        for (int64_t i = net->part_lo[q]; i < net->part_lo[q + 1]; ++i)
          emitted[i] = (char)((net->p.precision == ORACLE_FP32) ? step_neuron_f32(net, i, t) : step_neuron_f64(net, i, t));
#pragma omp single
      for (int64_t i = 0; i < net->n; ++i) {
        if (!emitted[i]) continue;
        if (push_spike(net, t, (int32_t)i) != ORACLE_OK) rc = ORACLE_ERR_OOM;
        for (int32_t q = 0; q < n_part; ++q) net->events += net->prow[q][i + 1] - net->prow[q][i];
      }
#pragma omp for schedule(static, 1)
      for (int32_t q = 0; q < n_part; ++q)
        for (int64_t i = 0; i < net->n; ++i)
          if (emitted[i]) deliver_part(net, q, (int32_t)i, t);
    }
  }
  net->step += n_steps;
  free(emitted);
  return rc;
}

/* Advance n_steps from the current step.  Forced spikes (test hook, sorted by step) are emitted
 * in addition to the neurons' own spikes, without touching their state. */
int oracle_simulate(oracle_net* net, int64_t n_steps, int64_t n_forced, const int64_t* forced_step,
                    const int32_t* forced_id, int64_t n_trace, const int32_t* trace_ids,
                    double* v_trace) {
  if (net->n_part > 0) {
    if (n_forced > 0 || n_trace > 0 || net->count_ring) return ORACLE_ERR_ARG;  /* single-list form only */
    return simulate_par(net, n_steps);
  }
  int64_t fq = 0;
  char* emitted = (char*)xcalloc((size_t)net->n, 1);
  if (!emitted) return ORACLE_ERR_OOM;
  for (int64_t step = 0; step < n_steps; ++step) {
    int64_t t = net->step;
    if (net->count_ring) {
      for (int64_t i = 0; i < net->n; ++i) {
        size_t cell = (size_t)i * (size_t)net->depth + (size_t)(t % net->depth);
        net->consumed_events[i] += net->count_ring[cell];
        net->consumed_weight[i] += net->weight_ring[cell];
        net->count_ring[cell] = 0;
        net->weight_ring[cell] = 0.0;
      }
    }
    for (int64_t i = 0; i < net->n; ++i) {
      int sp = (net->p.precision == ORACLE_FP32) ? step_neuron_f32(net, i, t) : step_neuron_f64(net, i, t);
      emitted[i] = (char)sp;
    }
    while (fq < n_forced && forced_step[fq] < t) ++fq;
    while (fq < n_forced && forced_step[fq] == t) {
      if (forced_id[fq] >= 0 && forced_id[fq] < net->n) emitted[forced_id[fq]] = 1;
      ++fq;
    }
    for (int64_t i = 0; i < net->n; ++i) {
      if (!emitted[i]) continue;
      if (push_spike(net, t, (int32_t)i) != ORACLE_OK) { free(emitted); return ORACLE_ERR_OOM; }
      deliver(net, (int32_t)i, t);
    }
    if (n_trace > 0 && v_trace) {
      for (int64_t q = 0; q < n_trace; ++q) {
        int32_t id = trace_ids[q];
        v_trace[step * n_trace + q] = (net->p.precision == ORACLE_FP32) ? (double)net->v32[id] : net->v64[id];
      }
    }
    net->step = t + 1;
  }
  free(emitted);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Accessors                                                                                   */
/* ------------------------------------------------------------------------------------------ */
int64_t oracle_n(const oracle_net* net) { return net->n; }
int64_t oracle_n_syn(const oracle_net* net) { return net->n_syn; }
int64_t oracle_step(const oracle_net* net) { return net->step; }
int64_t oracle_events(const oracle_net* net) { return net->events; }
int32_t oracle_depth(const oracle_net* net) { return net->depth; }
int64_t oracle_raster_size(const oracle_net* net) { return net->raster_n; }

void oracle_raster(const oracle_net* net, int64_t* steps, int32_t* ids) {
  memcpy(steps, net->raster_step, sizeof(int64_t) * (size_t)net->raster_n);
  memcpy(ids, net->raster_id, sizeof(int32_t) * (size_t)net->raster_n);
}

/* State widened to double (exact for FP32 mode). */
void oracle_state(const oracle_net* net, double* v, double* cur, int32_t* refr) {
  for (int64_t i = 0; i < net->n; ++i) {
    if (net->p.precision == ORACLE_FP32) { v[i] = net->v32[i]; cur[i] = net->i32[i]; }
    else { v[i] = net->v64[i]; cur[i] = net->i64[i]; }
    refr[i] = net->refr[i];
  }
}

/* Ring as [n][D], cell (i, s) holding the input due at the step t with t mod D == s. */
void oracle_ring(const oracle_net* net, double* ring) {
  size_t nd = (size_t)net->n * (size_t)net->depth;
  for (size_t c = 0; c < nd; ++c)
    ring[c] = (net->p.precision == ORACLE_FP32) ? (double)net->ring32[c] : net->ring64[c];
}

void oracle_out_row(const oracle_net* net, int64_t* row) {
  memcpy(row, net->row, sizeof(int64_t) * (size_t)(net->n + 1));
}

void oracle_out_edges(const oracle_net* net, int32_t* tgt, int32_t* dly) {
  for (int64_t q = 0; q < net->n_syn; ++q) { tgt[q] = net->out_tgt[q]; dly[q] = net->out_dly[q]; }
}

void oracle_accounting(const oracle_net* net, int64_t* events, double* weight) {
  for (int64_t i = 0; i < net->n; ++i) { events[i] = net->consumed_events[i]; weight[i] = net->consumed_weight[i]; }
}

/* Float constants the FP32 mode uses (for comparison with a float parameter record). */
void oracle_constants_f32(const oracle_net* net, float* out8, uint32_t* thr, int32_t* n_thr, int32_t* n_ref) {
  out8[0] = net->p11f; out8[1] = net->p21f; out8[2] = net->p22m1f; out8[3] = net->p20f;
  out8[4] = net->wexf; out8[5] = net->winf; out8[6] = net->jextf; out8[7] = net->vthf;
  for (int k = 0; k < net->n_thr; ++k) thr[k] = net->thr[k];
  *n_thr = net->n_thr;
  *n_ref = net->n_ref;
}

uint32_t oracle_v0_word(uint64_t seed, int64_t i) { return v0_word(seed, i); }
uint32_t oracle_poisson_word(uint64_t seed, int64_t i, int64_t t) { return poisson_word(seed, i, t); }

/* Overwrite the neuron state (closed-form tests start from a chosen V, I, refractory count). */
void oracle_set_state(oracle_net* net, const double* v, const double* cur, const int32_t* refr) {
  for (int64_t i = 0; i < net->n; ++i) {
    if (net->p.precision == ORACLE_FP32) { net->v32[i] = (float)v[i]; net->i32[i] = (float)cur[i]; }
    else { net->v64[i] = v[i]; net->i64[i] = cur[i]; }
    net->refr[i] = refr[i];
  }
}

/* Overwrite the ring, [n][D] as oracle_ring gives it (checkpoint tests). */
void oracle_set_ring(oracle_net* net, const double* ring) {
  size_t nd = (size_t)net->n * (size_t)net->depth;
  for (size_t c = 0; c < nd; ++c) {
    if (net->p.precision == ORACLE_FP32) net->ring32[c] = (float)ring[c];
    else net->ring64[c] = ring[c];
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Replay of a few targets                                                                     */
/* ------------------------------------------------------------------------------------------ */
/* The trajectory of a neuron depends only on its own incoming synapses and on the spikes their
 * sources emitted (Eq. 1-3: the input at step t is the sum of the weights whose spikes arrive at
 * t).  So a given raster of the whole network -- every (step, id) emitted, sorted by step then id
 * -- determines each target's input exactly, and one target can be simulated alone.
 *
 * oracle_replay() does that for the ascending, distinct targets[0..n_t): each target draws its
 * K_E + K_I incoming synapses as oracle_build() does; the synapses onto the chosen targets are
 * kept as outgoing lists sorted by (source, target, draw index); for t = 0 .. n_steps-1 every
 * chosen target is updated (step_neuron_f32 / _f64, consuming ring slot t), then every raster
 * spike of step t is delivered onto the chosen targets (deliver(), same order as the full
 * simulation).  The targets' own spikes are written to out_step/out_id (up to cap; *out_n is the
 * count, which may exceed cap) and their final V, I, refractory counts to v/cur/refr (widened to
 * double); v_trace (optional, [n_steps][n_t]) receives every target's V after every step.  The raster is taken as given: a target's own replayed spikes are not fed back, so a
 * run of the full oracle replays to itself exactly, and a raster from another simulator is
 * checked one target at a time. */
int oracle_replay(const oracle_params* p, uint64_t seed, int64_t n_t, const int32_t* targets,
                  int64_t n_steps, int64_t n_spk, const int64_t* spk_step, const int32_t* spk_id,
                  int64_t cap, int64_t* out_step, int32_t* out_id, int64_t* out_n,
                  double* v, double* cur, int32_t* refr, double* v_trace) {
  if (!validate(p) || n_t < 0 || n_steps < 0 || n_spk < 0 || cap < 0 || !out_n) return ORACLE_ERR_ARG;
  const int64_t n = (int64_t)p->n_exc + p->n_inh;
  for (int64_t q = 0; q < n_t; ++q)
    if (targets[q] < 0 || targets[q] >= n || (q > 0 && targets[q] <= targets[q - 1])) return ORACLE_ERR_ARG;
  for (int64_t e = 0; e < n_spk; ++e) {
    if (spk_id[e] < 0 || spk_id[e] >= n || spk_step[e] < 0) return ORACLE_ERR_ARG;
    if (e > 0 && (spk_step[e] < spk_step[e - 1] || (spk_step[e] == spk_step[e - 1] && spk_id[e] <= spk_id[e - 1])))
      return ORACLE_ERR_ARG;
  }
  oracle_net* net = (oracle_net*)calloc(1, sizeof(oracle_net));
  if (!net) return ORACLE_ERR_OOM;
  int rc = init_common(net, p, seed);
  if (rc != ORACLE_OK) { oracle_free(net); return rc; }
  const int64_t k = (int64_t)p->k_exc + p->k_inh;
  net->n_syn = n_t * k;
  net->row = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  net->out_tgt = (int32_t*)xcalloc((size_t)net->n_syn, sizeof(int32_t));
  net->out_dly = (uint8_t*)xcalloc((size_t)net->n_syn, sizeof(uint8_t));
  int64_t* cursor = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  if (!net->row || !net->out_tgt || !net->out_dly || !cursor) { free(cursor); oracle_free(net); return ORACLE_ERR_OOM; }
  int32_t s, d;
  for (int64_t q = 0; q < n_t; ++q)
    for (int64_t j = 0; j < k; ++j) {
      oracle_draw(seed, p->n_exc, p->n_inh, p->k_exc, p->d_min, p->d_max, targets[q], j, &s, &d);
      net->row[s + 1] += 1;
    }
  for (int64_t x = 0; x < n; ++x) net->row[x + 1] += net->row[x];
  for (int64_t x = 0; x < n; ++x) cursor[x] = net->row[x];
  for (int64_t q = 0; q < n_t; ++q)  /* ascending targets, ascending draws: (source, target, draw) order */
    for (int64_t j = 0; j < k; ++j) {
      oracle_draw(seed, p->n_exc, p->n_inh, p->k_exc, p->d_min, p->d_max, targets[q], j, &s, &d);
      int64_t pos = cursor[s]++;
      net->out_tgt[pos] = targets[q];
      net->out_dly[pos] = (uint8_t)d;
    }
  free(cursor);
  int64_t e = 0, got = 0;
  for (int64_t t = 0; t < n_steps; ++t) {
    for (int64_t q = 0; q < n_t; ++q) {
      int sp = (p->precision == ORACLE_FP32) ? step_neuron_f32(net, targets[q], t) : step_neuron_f64(net, targets[q], t);
      if (sp) {
        if (got < cap) { out_step[got] = t; out_id[got] = targets[q]; }
        ++got;
      }
      if (v_trace)
        v_trace[t * n_t + q] = (p->precision == ORACLE_FP32) ? (double)net->v32[targets[q]] : net->v64[targets[q]];
    }
    while (e < n_spk && spk_step[e] < t) ++e;
    while (e < n_spk && spk_step[e] == t) { deliver(net, spk_id[e], t); ++e; }
  }
  *out_n = got;
  for (int64_t q = 0; q < n_t; ++q) {
    int32_t i = targets[q];
    if (v) v[q] = (p->precision == ORACLE_FP32) ? (double)net->v32[i] : net->v64[i];
    if (cur) cur[q] = (p->precision == ORACLE_FP32) ? (double)net->i32[i] : net->i64[i];
    if (refr) refr[q] = net->refr[i];
  }
  oracle_free(net);
  return ORACLE_OK;
}
