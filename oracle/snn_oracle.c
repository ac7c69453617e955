/*
 * snn_oracle.c -- plain, slow, FP64 CPU oracle for spike delivery in a
 * time-driven simulation of a balanced random network of current-based
 * leaky integrate-and-fire neurons with alpha-shaped synaptic currents.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * What it computes, and where the paper (arXiv 2109.12855, "Routing brain
 * traffic through the von Neumann bottleneck") defines it:
 *   - Spike delivery, Section 3.2, Algorithm REF: every spike entry addresses
 *     the target segment of its source; each synapse of the segment adds its
 *     weight into its target neuron's spike ring buffer at position
 *     (emission step + delay).  The latency-hiding variants of Section 4
 *     (bwRB*, lagRB, bwTS, bwTSRB*) reorder the same additions and are kept
 *     here only as order-preserving self-checks of REF.
 *   - Connection store, Section 3.1 / Fig. 3: synapses live in source-specific
 *     target segments; here one source-major array with row offsets.
 *   - Simulation cycle, Section 1 and Section 2.1: neurons are updated on a
 *     0.1 ms grid; spikes are exchanged and delivered once per min-delay
 *     interval.
 *   - Neuron update, Section 1 and Section 2.1: linear subthreshold dynamics
 *     integrated exactly with a precomputed propagator matrix (the paper
 *     cites Rotter & Diesmann 1999), threshold, reset and refractoriness.
 * The paper defers the model parameters to an external table; the values
 * come from the caller.  Where the paper is silent (order of operations in
 * one step, ring-buffer slot arithmetic, connection rule details, random
 * streams) the reading used is stated at each function.
 *
 * Random numbers: one counter-based generator, Philox4x32-10, written from
 * its published definition (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).
 *
 * Pins: the paper prints no worked example (its model numbers live in a
 * cited external table), so no function here can be checked against numbers
 * it prints; every function is pinned by closed forms, library routines,
 * brute force or invariants in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Section 3: the Philox S-box with two 32x32->64     */
/* multiplications per round and a Weyl sequence for the round keys).      */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_MUL_A 0xD2511F53u
#define ORC_PHILOX_MUL_B 0xCD9E8D57u
#define ORC_PHILOX_WEYL_A 0x9E3779B9u
#define ORC_PHILOX_WEYL_B 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: add the Weyl constants */
      k0 += ORC_PHILOX_WEYL_A;
      k1 += ORC_PHILOX_WEYL_B;
    }
    uint64_t pa = (uint64_t)ORC_PHILOX_MUL_A * x0;
    uint64_t pb = (uint64_t)ORC_PHILOX_MUL_B * x2;
    uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
    uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
    uint32_t y0 = pb_hi ^ x1 ^ k0;
    uint32_t y1 = pb_lo;
    uint32_t y2 = pa_hi ^ x3 ^ k1;
    uint32_t y3 = pa_lo;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout used by every random draw of the model (a reading: the
 * paper does not say how its benchmark draws random numbers).
 *   stream 0: connection (target, k)      -> words: source, delay, 2 normal
 *   stream 1: initial membrane potential  (neuron, 0)
 *   stream 2: Poisson drive               (neuron, step / 4), word step % 4 */
static void orc_draw(uint64_t seed, uint32_t a, uint64_t b, uint32_t stream,
                     uint32_t out[4]) {
  uint32_t ctr[4] = {a, (uint32_t)b, (uint32_t)(b >> 32), stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* floor(u * n / 2^32): a uniform integer in [0, n). */
static uint32_t orc_scale_u32(uint32_t u, uint32_t n) {
  return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Weight storage rounding, used to model what the store keeps.            */
/* ------------------------------------------------------------------------ */
double orc_round_f32(double x) { return (double)(float)x; }

/* Round to the nearest bfloat16 (8 significant bits, float's exponent
 * range), ties to even, in one step from FP64.  Written from the definition:
 * x = m * 2^e with m in [0.5, 1); keep 8 bits of m. */
double orc_round_bf16(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  double m = frexp(x, &e);
  double r = nearbyint(ldexp(m, 8)); /* default rounding mode: ties to even */
  return ldexp(r, e - 8);
}

/* ------------------------------------------------------------------------ */
/* Neuron model: iaf_psc_alpha with resting potential 0.                    */
/*   dV/dt  = -V/tau_m + I/C                                                */
/*   dI/dt  = -I/tau_s + J          (J is the auxiliary state "dI")         */
/*   dJ/dt  = -J/tau_s                                                      */
/* A presynaptic spike of weight w (pA) adds (e/tau_s) w to J, so that the  */
/* current peaks at w after tau_s.                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  double h;       /* ms */
  double tau_m;   /* ms */
  double c_m;     /* pF */
  double v_th;    /* mV */
  double v_reset; /* mV */
  double t_ref;   /* ms */
  double tau_syn; /* ms */
} orc_neuron;

/* g(x) = 1 - e^{-x} (1 + x), the alpha-kernel factor of the membrane
 * response.  For small x the two terms cancel, so there the Taylor series
 * g(x) = sum_{m>=2} (-1)^m (m-1) x^m / m! is summed instead. */
static double orc_one_minus_exp_1px(double x) {
  if (fabs(x) >= 0.5) return 1.0 - exp(-x) * (1.0 + x);
  double term = x * x / 2.0, sum = 0.0; /* m = 2 term is x^2/2 */
  for (int m = 2; m < 40; ++m) {
    sum += term; /* term = (-1)^m (m-1) x^m / m! */
    term *= -x * (double)m / ((double)(m - 1) * (double)(m + 1));
  }
  return sum;
}

/* Exact propagator P = expm(A h) for y = (J, I, V), entries in closed form.
 * out = {P11, P21, P22, P31, P32, P33}:  J' = P11 J;  I' = P21 J + P22 I;
 * V' = P31 J + P32 I + P33 V.  Requires tau_syn != tau_m. */
void orc_propagators(const orc_neuron* nm, double out[6]) {
  double h = nm->h, a = 1.0 / nm->tau_syn, b = 1.0 / nm->tau_m, C = nm->c_m;
  double ea = exp(-a * h), eb = exp(-b * h);
  double c = a - b;
  out[0] = ea;                /* P11 */
  out[1] = h * ea;            /* P21 */
  out[2] = ea;                /* P22 */
  /* V response to J(0)=1: (1/C) e^{-bh} (1 - e^{-ch}(1 + ch)) / c^2 */
  out[3] = eb * orc_one_minus_exp_1px(c * h) / (c * c) / C; /* P31 */
  /* V response to I(0)=1: (1/C) (e^{-bh} - e^{-ah}) / (a - b)
   *                     = (1/C) e^{-bh} (1 - e^{-ch}) / c */
  out[4] = -eb * expm1(-c * h) / c / C; /* P32 */
  out[5] = eb;                /* P33 */
}

/* Membrane response V(t) to one PSC of weight 1 pA arriving at t = 0. */
double orc_psp_unit(const orc_neuron* nm, double t) {
  double a = 1.0 / nm->tau_syn, b = 1.0 / nm->tau_m, c = a - b;
  if (t <= 0.0) return 0.0;
  return (M_E / nm->tau_syn) / nm->c_m * exp(-b * t) *
         orc_one_minus_exp_1px(c * t) / (c * c);
}

/* Peak of orc_psp_unit: the response rises to a single maximum and decays,
 * so the zero of its slope is bracketed by [0, 20 tau_m] and found by
 * bisection on the sign of a central difference (plain and robust). */
double orc_psp_peak(const orc_neuron* nm, double* t_peak) {
  double lo = 1e-9, hi = 20.0 * nm->tau_m;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double dt = 1e-7 * (1.0 + mid);
    double slope = orc_psp_unit(nm, mid + dt) - orc_psp_unit(nm, mid - dt);
    if (slope > 0.0) lo = mid; else hi = mid;
  }
  double tp = 0.5 * (lo + hi);
  if (t_peak) *t_peak = tp;
  return orc_psp_unit(nm, tp);
}

/* Refractory period in steps: nearest integer to t_ref / h. */
int orc_refractory_steps(const orc_neuron* nm) {
  return (int)floor(nm->t_ref / nm->h + 0.5);
}

/* ------------------------------------------------------------------------ */
/* Poisson drive: count = min{k : u < T_k} with T_k = floor(F_k 2^32), F_k   */
/* the Poisson(lambda) CDF and u the raw 32-bit Philox word (inversion).    */
/* The table ends at the first k whose threshold reaches 2^32 - 1 (the FP64 */
/* CDF may never reach 1 exactly); that last threshold is set to 2^32, so    */
/* the tail beyond it (mass below 2^-31) is folded into the last outcome.  */
/* ------------------------------------------------------------------------ */
int orc_poisson_table(double lambda, uint64_t* thr, int cap) {
  double p = exp(-lambda), F = p;
  int n = 0;
  for (int k = 0; k < cap; ++k) {
    double T = floor(F * 4294967296.0);
    if (T >= 4294967295.0) {
      thr[n++] = 4294967296ull;
      return n;
    }
    thr[n++] = (uint64_t)T;
    p *= lambda / (double)(k + 1);
    F += p;
  }
  thr[n - 1] = 4294967296ull; /* cap reached: close the table */
  return n;
}

static int orc_poisson_from_u32(uint32_t u, const uint64_t* thr, int n) {
  int k = 0;
  while (k < n - 1 && (uint64_t)u >= thr[k]) ++k;
  return k;
}

/* One Philox call yields four words; the drive of neuron i at step t uses
 * word (t mod 4) of the call at counter (i, floor(t / 4)) on stream 2. */
int orc_poisson_count(uint64_t seed, uint32_t neuron, int64_t step,
                      const uint64_t* thr, int n) {
  uint32_t r[4];
  int64_t block = step >= 0 ? step / 4 : -((-step + 3) / 4);
  orc_draw(seed, neuron, (uint64_t)block, 2u, r);
  return orc_poisson_from_u32(r[(int)(step - 4 * block)], thr, n);
}

/* Initial potential: V0 = V_reset + (V_th - V_reset) u, u = x 2^-32. */
void orc_init_v(const orc_neuron* nm, uint32_t n, uint64_t seed, double* V) {
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t r[4];
    orc_draw(seed, i, 0, 1u, r);
    V[i] = nm->v_reset + (nm->v_th - nm->v_reset) * ((double)r[0] * 0x1p-32);
  }
}

/* ------------------------------------------------------------------------ */
/* Connectivity: fixed in-degree (the benchmark model's rule).             */
/* Target j draws K_E sources from [0, N_E) and K_I from [N_E, N_E + N_I),  */
/* uniformly with replacement (multapses and autapses allowed); draw k of   */
/* target j uses Philox stream 0 at counter (j, k):                         */
/*   word 0 -> source, word 1 -> delay d_lo + floor(u (d_hi-d_lo+1) 2^-32),  */
/*   words 2, 3 -> a Box-Muller normal when a weight spread is requested.   */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n_e, n_i, k_e, k_i;
  double w_e, w_i;   /* mean weights, pA */
  double sd_e, sd_i; /* standard deviations, pA (0: fixed weight) */
  int32_t d_lo, d_hi;
  uint64_t seed;
  int32_t clip_e; /* E weights clipped at >= 0 */
  int32_t clip_i; /* I weights clipped at <= 0 */
  int32_t wfmt;   /* 0: keep FP64, 1: round to FP32, 2: round to BF16 */
} orc_conn;

void orc_draw_synapse(const orc_conn* cp, uint32_t tgt, uint32_t k,
                      uint32_t* src, int32_t* delay, double* w) {
  uint32_t r[4];
  orc_draw(cp->seed, tgt, (uint64_t)k, 0u, r);
  int exc = k < cp->k_e;
  *src = exc ? orc_scale_u32(r[0], cp->n_e)
             : cp->n_e + orc_scale_u32(r[0], cp->n_i);
  *delay = cp->d_lo + (int32_t)orc_scale_u32(r[1], (uint32_t)(cp->d_hi - cp->d_lo + 1));
  double mean = exc ? cp->w_e : cp->w_i, sd = exc ? cp->sd_e : cp->sd_i;
  double x = mean;
  if (sd != 0.0) {
    double u1 = ((double)r[2] + 1.0) * 0x1p-32; /* (0, 1] */
    double u2 = (double)r[3] * 0x1p-32;         /* [0, 1) */
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    x = mean + sd * z;
  }
  if (exc && cp->clip_e && x < 0.0) x = 0.0;
  if (!exc && cp->clip_i && x > 0.0) x = 0.0;
  if (cp->wfmt == 1) x = orc_round_f32(x);
  else if (cp->wfmt == 2) x = orc_round_bf16(x);
  *w = x;
}

/* The K_E + K_I incoming synapses of one target, in draw order k. */
void orc_incoming(const orc_conn* cp, uint32_t tgt, uint32_t* src,
                  int32_t* delay, double* w) {
  uint32_t kk = cp->k_e + cp->k_i;
  for (uint32_t k = 0; k < kk; ++k)
    orc_draw_synapse(cp, tgt, k, &src[k], &delay[k], &w[k]);
}

/* Full source-major store.  Segments are ordered by (delay, target, k):
 * targets are visited in increasing order and k increasing, which leaves
 * each segment sorted by (target, k); a stable counting pass by delay then
 * gives (delay, target, k).  Arrays tgt/delay/w hold N (K_E+K_I) entries;
 * row_ptr holds N+1. */
int orc_build_fixed_indegree(const orc_conn* cp, uint64_t* row_ptr,
                             uint32_t* tgt, int32_t* delay, double* w) {
  uint32_t n = cp->n_e + cp->n_i, kk = cp->k_e + cp->k_i;
  uint64_t total = (uint64_t)n * kk;
  int nd = cp->d_hi - cp->d_lo + 1;
  uint64_t* cnt = calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t* s_src = malloc(total * sizeof(uint32_t) + 1);
  int32_t* s_d = malloc(total * sizeof(int32_t) + 1);
  double* s_w = malloc(total * sizeof(double) + 1);
  if (!cnt || !s_src || !s_d || !s_w) {
    free(cnt); free(s_src); free(s_d); free(s_w);
    return -1;
  }
  uint64_t e = 0;
  for (uint32_t j = 0; j < n; ++j)
    for (uint32_t k = 0; k < kk; ++k, ++e) {
      orc_draw_synapse(cp, j, k, &s_src[e], &s_d[e], &s_w[e]);
      cnt[s_src[e] + 1]++;
    }
  for (uint32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  memcpy(row_ptr, cnt, ((size_t)n + 1) * sizeof(uint64_t));
  /* fill each row in (target, k) order, then stable-partition by delay */
  uint64_t* fill = malloc(((size_t)n + 1) * sizeof(uint64_t));
  memcpy(fill, cnt, ((size_t)n + 1) * sizeof(uint64_t));
  uint32_t* t_tmp = malloc(total * sizeof(uint32_t) + 1);
  int32_t* d_tmp = malloc(total * sizeof(int32_t) + 1);
  double* w_tmp = malloc(total * sizeof(double) + 1);
  e = 0;
  for (uint32_t j = 0; j < n; ++j)
    for (uint32_t k = 0; k < kk; ++k, ++e) {
      uint64_t pos = fill[s_src[e]]++;
      t_tmp[pos] = j;
      d_tmp[pos] = s_d[e];
      w_tmp[pos] = s_w[e];
    }
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t pos = row_ptr[i];
    for (int dd = 0; dd < nd; ++dd)
      for (uint64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
        if (d_tmp[q] == cp->d_lo + dd) {
          tgt[pos] = t_tmp[q];
          delay[pos] = d_tmp[q];
          w[pos] = w_tmp[q];
          ++pos;
        }
  }
  free(cnt); free(fill); free(s_src); free(s_d); free(s_w);
  free(t_tmp); free(d_tmp); free(w_tmp);
  return 0;
}

/* Store restricted to the targets [tgt_lo, tgt_hi): the segments a NEST
 * thread owning those targets would hold (Section 2.1: synapses live with
 * their target).  Same ordering rule as orc_build_fixed_indegree.  Output
 * arrays hold (tgt_hi - tgt_lo)(K_E + K_I) entries; row_ptr holds N+1. */
int orc_build_fixed_indegree_targets(const orc_conn* cp, uint32_t tgt_lo,
                                     uint32_t tgt_hi, uint64_t* row_ptr,
                                     uint32_t* tgt, int32_t* delay,
                                     double* w) {
  uint32_t n = cp->n_e + cp->n_i, kk = cp->k_e + cp->k_i;
  uint64_t total = (uint64_t)(tgt_hi - tgt_lo) * kk;
  int nd = cp->d_hi - cp->d_lo + 1;
  uint64_t* cnt = calloc((size_t)n + 1, sizeof(uint64_t));
  uint64_t* fill = malloc(((size_t)n + 1) * sizeof(uint64_t));
  uint32_t* t_tmp = malloc(total * sizeof(uint32_t) + 1);
  int32_t* d_tmp = malloc(total * sizeof(int32_t) + 1);
  double* w_tmp = malloc(total * sizeof(double) + 1);
  if (!cnt || !fill || !t_tmp || !d_tmp || !w_tmp) {
    free(cnt); free(fill); free(t_tmp); free(d_tmp); free(w_tmp);
    return -1;
  }
  for (uint32_t j = tgt_lo; j < tgt_hi; ++j)
    for (uint32_t k = 0; k < kk; ++k) {
      uint32_t s; int32_t d; double x;
      orc_draw_synapse(cp, j, k, &s, &d, &x);
      cnt[s + 1]++;
    }
  for (uint32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  memcpy(row_ptr, cnt, ((size_t)n + 1) * sizeof(uint64_t));
  memcpy(fill, cnt, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint32_t j = tgt_lo; j < tgt_hi; ++j)
    for (uint32_t k = 0; k < kk; ++k) {
      uint32_t s; int32_t d; double x;
      orc_draw_synapse(cp, j, k, &s, &d, &x);
      uint64_t pos = fill[s]++;
      t_tmp[pos] = j; d_tmp[pos] = d; w_tmp[pos] = x;
    }
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t pos = row_ptr[i];
    for (int dd = 0; dd < nd; ++dd)
      for (uint64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
        if (d_tmp[q] == cp->d_lo + dd) {
          tgt[pos] = t_tmp[q]; delay[pos] = d_tmp[q]; w[pos] = w_tmp[q];
          ++pos;
        }
  }
  free(cnt); free(fill); free(t_tmp); free(d_tmp); free(w_tmp);
  return 0;
}

/* Store from an explicit edge list.  Edge e = (src[e], tgt[e], delay[e],
 * w[e]); each segment is ordered by (delay, target, e).  Built by counting
 * rows, then for every row an insertion of its edges in e order followed by
 * a stable insertion sort on (delay, target): plain and obviously stable. */
int orc_build_edges(uint32_t n, uint64_t n_edges, const uint32_t* src,
                    const uint32_t* tg, const int32_t* dl, const double* wt,
                    uint64_t* row_ptr, uint32_t* tgt, int32_t* delay,
                    double* w) {
  memset(row_ptr, 0, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint64_t e = 0; e < n_edges; ++e) {
    if (src[e] >= n || tg[e] >= n) return -2;
    row_ptr[src[e] + 1]++;
  }
  for (uint32_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
  uint64_t* fill = malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!fill) return -1;
  memcpy(fill, row_ptr, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint64_t e = 0; e < n_edges; ++e) {
    uint64_t pos = fill[src[e]]++;
    tgt[pos] = tg[e]; delay[pos] = dl[e]; w[pos] = wt[e];
  }
  free(fill);
  for (uint32_t i = 0; i < n; ++i) {
    for (uint64_t q = row_ptr[i] + 1; q < row_ptr[i + 1]; ++q) {
      uint32_t t0 = tgt[q]; int32_t d0 = delay[q]; double w0 = w[q];
      uint64_t p = q;
      while (p > row_ptr[i] &&
             (delay[p - 1] > d0 || (delay[p - 1] == d0 && tgt[p - 1] > t0))) {
        tgt[p] = tgt[p - 1]; delay[p] = delay[p - 1]; w[p] = w[p - 1];
        --p;
      }
      tgt[p] = t0; delay[p] = d0; w[p] = w0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Spike delivery.                                                          */
/* Ring buffer rb[slot][neuron] with n_slots slots (a power of two); step u */
/* uses slot u mod n_slots.  "AddValue(delay, weight)" of a spike emitted   */
/* at step t adds the weight at step t + delay.  Optional instruments:      */
/* cnt[slot][neuron] counts additions; absw[slot][neuron] accumulates |w|.  */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n;       /* neurons */
  int32_t n_slots;  /* ring-buffer slots */
  const uint64_t* row_ptr;
  const uint32_t* tgt;
  const int32_t* delay;
  const double* w;
} orc_store;

static int64_t orc_slot(int64_t step, int32_t n_slots) {
  int64_t s = step % n_slots;
  return s < 0 ? s + n_slots : s;
}

static void orc_add_value(const orc_store* st, double* rb, uint32_t* cnt,
                          double* absw, uint32_t target, int64_t step,
                          double weight) {
  size_t cell = (size_t)orc_slot(step, st->n_slots) * st->n + target;
  rb[cell] += weight;
  if (cnt) cnt[cell] += 1;
  if (absw) absw[cell] += fabs(weight);
}

/* Algorithm REF (Section 3.2): for each spike entry walk its target
 * segment; for each synapse read (target, delay, weight), then add the
 * weight into the target's ring buffer at the delay.  An empty segment
 * delivers nothing (a source without local targets). */
uint64_t orc_deliver_ref(const orc_store* st, uint64_t n_sp,
                         const uint32_t* sp_src, const int64_t* sp_t,
                         double* rb, uint32_t* cnt, double* absw) {
  uint64_t events = 0;
  for (uint64_t s = 0; s < n_sp; ++s) {
    uint32_t src = sp_src[s];
    for (uint64_t lcid = st->row_ptr[src]; lcid < st->row_ptr[src + 1];
         ++lcid) {
      orc_add_value(st, rb, cnt, absw, st->tgt[lcid], sp_t[s] + st->delay[lcid],
                    st->w[lcid]);
      ++events;
    }
  }
  return events;
}

/* bwRB (Section 4.1): synapse reads fill auxiliary arrays of size b_rb
 * across segment boundaries; when full, all b_rb ring-buffer additions are
 * performed in order; leftovers are added at the end.  Same additions, same
 * order per ring-buffer cell as REF. */
uint64_t orc_deliver_bwrb(const orc_store* st, uint64_t n_sp,
                          const uint32_t* sp_src, const int64_t* sp_t,
                          double* rb, int b_rb) {
  uint32_t* a_tgt = malloc(sizeof(uint32_t) * (size_t)b_rb);
  int64_t* a_step = malloc(sizeof(int64_t) * (size_t)b_rb);
  double* a_w = malloc(sizeof(double) * (size_t)b_rb);
  int i = 0;
  uint64_t events = 0;
  for (uint64_t s = 0; s < n_sp; ++s) {
    uint32_t src = sp_src[s];
    for (uint64_t lcid = st->row_ptr[src]; lcid < st->row_ptr[src + 1];
         ++lcid) {
      a_tgt[i] = st->tgt[lcid];
      a_step[i] = sp_t[s] + st->delay[lcid];
      a_w[i] = st->w[lcid];
      ++i;
      if (i == b_rb) {
        for (int q = 0; q < b_rb; ++q)
          orc_add_value(st, rb, NULL, NULL, a_tgt[q], a_step[q], a_w[q]);
        events += (uint64_t)b_rb;
        i = 0;
      }
    }
  }
  for (int q = 0; q < i; ++q)
    orc_add_value(st, rb, NULL, NULL, a_tgt[q], a_step[q], a_w[q]);
  events += (uint64_t)i;
  free(a_tgt); free(a_step); free(a_w);
  return events;
}

/* lagRB (Section 4.2): synapse reads run b_rb entries ahead of ring-buffer
 * additions through circular auxiliary arrays of size b_rb + 1; the first
 * b_rb reads only fill, afterwards each read is followed by the addition of
 * the entry read b_rb reads earlier; the tail is drained at the end. */
uint64_t orc_deliver_lagrb(const orc_store* st, uint64_t n_sp,
                           const uint32_t* sp_src, const int64_t* sp_t,
                           double* rb, int b_rb) {
  int cap = b_rb + 1;
  uint32_t* a_tgt = malloc(sizeof(uint32_t) * (size_t)cap);
  int64_t* a_step = malloc(sizeof(int64_t) * (size_t)cap);
  double* a_w = malloc(sizeof(double) * (size_t)cap);
  int wr = 0, rd = 0;
  uint64_t filled = 0, events = 0;
  for (uint64_t s = 0; s < n_sp; ++s) {
    uint32_t src = sp_src[s];
    for (uint64_t lcid = st->row_ptr[src]; lcid < st->row_ptr[src + 1];
         ++lcid) {
      a_tgt[wr] = st->tgt[lcid];
      a_step[wr] = sp_t[s] + st->delay[lcid];
      a_w[wr] = st->w[lcid];
      wr = (wr + 1) % cap;
      ++filled;
      if (filled > (uint64_t)b_rb) { /* pipeline is primed */
        orc_add_value(st, rb, NULL, NULL, a_tgt[rd], a_step[rd], a_w[rd]);
        rd = (rd + 1) % cap;
        ++events;
      }
    }
  }
  while (rd != wr) {
    orc_add_value(st, rb, NULL, NULL, a_tgt[rd], a_step[rd], a_w[rd]);
    rd = (rd + 1) % cap;
    ++events;
  }
  free(a_tgt); free(a_step); free(a_w);
  return events;
}

/* bwTS (Section 4.3): spike entries are taken in batches of b_ts: first the
 * segment starts of the batch are gathered, then the segment sizes, then
 * each segment is walked with a fixed-count loop; the last, partial batch
 * is handled the same way with fewer entries.  With b_rb > 0 the additions
 * inside the fixed-count loop are batched as in bwRB (bwTSRB*, Section 4.4). */
uint64_t orc_deliver_bwts(const orc_store* st, uint64_t n_sp,
                          const uint32_t* sp_src, const int64_t* sp_t,
                          double* rb, int b_ts, int b_rb) {
  uint64_t* lcid = malloc(sizeof(uint64_t) * (size_t)b_ts);
  uint64_t* ts_size = malloc(sizeof(uint64_t) * (size_t)b_ts);
  int use_rb = b_rb > 0;
  int cap = use_rb ? b_rb : 1;
  uint32_t* a_tgt = malloc(sizeof(uint32_t) * (size_t)cap);
  int64_t* a_step = malloc(sizeof(int64_t) * (size_t)cap);
  double* a_w = malloc(sizeof(double) * (size_t)cap);
  int i = 0;
  uint64_t events = 0;
  for (uint64_t l = 0; l < n_sp; l += (uint64_t)b_ts) {
    int nb = (int)((n_sp - l) < (uint64_t)b_ts ? (n_sp - l) : (uint64_t)b_ts);
    for (int k = 0; k < nb; ++k) lcid[k] = st->row_ptr[sp_src[l + k]];
    for (int k = 0; k < nb; ++k)
      ts_size[k] = st->row_ptr[sp_src[l + k] + 1] - st->row_ptr[sp_src[l + k]];
    for (int k = 0; k < nb; ++k) {
      for (uint64_t r = 0; r < ts_size[k]; ++r) {
        uint64_t q = lcid[k]++;
        if (!use_rb) {
          orc_add_value(st, rb, NULL, NULL, st->tgt[q], sp_t[l + k] + st->delay[q],
                        st->w[q]);
          ++events;
        } else {
          a_tgt[i] = st->tgt[q];
          a_step[i] = sp_t[l + k] + st->delay[q];
          a_w[i] = st->w[q];
          if (++i == b_rb) {
            for (int p = 0; p < b_rb; ++p)
              orc_add_value(st, rb, NULL, NULL, a_tgt[p], a_step[p], a_w[p]);
            events += (uint64_t)b_rb;
            i = 0;
          }
        }
      }
    }
  }
  for (int p = 0; p < i; ++p)
    orc_add_value(st, rb, NULL, NULL, a_tgt[p], a_step[p], a_w[p]);
  events += (uint64_t)i;
  free(lcid); free(ts_size); free(a_tgt); free(a_step); free(a_w);
  return events;
}

/* ------------------------------------------------------------------------ */
/* Neuron update over n_steps grid steps starting at step t0.               */
/* Order inside one step t (a reading; the paper does not spell it out):    */
/*  1. if not refractory: V <- P31 J + P32 I + P33 V, else count down;      */
/*  2. I <- P21 J + P22 I;  J <- P11 J;                                     */
/*  3. J += (e/tau_s) (rb[t] + w_ext * Poisson count(i, t)); rb[t] <- 0;    */
/*  4. if V >= V_th: V <- V_reset, refractory for round(t_ref/h) steps,     */
/*     emit (i, t).                                                         */
/* Spikes are written in step-major, neuron-minor order.  Returns the number */
/* of spikes (which may exceed cap; only cap are stored).                   */
/* ------------------------------------------------------------------------ */
/* The same update for the neurons [lo, hi) of a population of n (state and
 * ring-buffer arrays indexed globally; the drive is keyed by the global
 * index): a thread that owns those neurons runs exactly these steps. */
uint64_t orc_update_range(const orc_neuron* nm, uint32_t lo, uint32_t hi,
                          uint32_t n, int32_t n_slots, double* V, double* I,
                          double* J, int32_t* refr, double* rb, int64_t t0,
                          int32_t n_steps, double nu_ext_hz, double w_ext,
                          uint64_t seed, uint32_t* sp_src, int64_t* sp_t,
                          uint64_t cap) {
  double P[6];
  orc_propagators(nm, P);
  double psc = M_E / nm->tau_syn;
  int ref_steps = orc_refractory_steps(nm);
  uint64_t thr[256];
  int nthr = orc_poisson_table(nu_ext_hz * nm->h * 1e-3, thr, 256);
  uint64_t ns = 0;
  for (int32_t s = 0; s < n_steps; ++s) {
    int64_t t = t0 + s;
    size_t row = (size_t)orc_slot(t, n_slots) * n;
    for (uint32_t i = lo; i < hi; ++i) {
      if (refr[i] == 0)
        V[i] = P[3] * J[i] + P[4] * I[i] + P[5] * V[i];
      else
        refr[i] -= 1;
      I[i] = P[1] * J[i] + P[2] * I[i];
      J[i] = P[0] * J[i];
      double in = rb[row + i];
      rb[row + i] = 0.0;
      int c = (w_ext != 0.0 && nu_ext_hz > 0.0)
                  ? orc_poisson_count(seed, i, t, thr, nthr) : 0;
      J[i] += psc * (in + w_ext * (double)c);
      if (V[i] >= nm->v_th) {
        V[i] = nm->v_reset;
        refr[i] = ref_steps;
        if (ns < cap) { sp_src[ns] = i; sp_t[ns] = t; }
        ++ns;
      }
    }
  }
  return ns;
}

uint64_t orc_update(const orc_neuron* nm, uint32_t n, int32_t n_slots,
                    double* V, double* I, double* J, int32_t* refr, double* rb,
                    int64_t t0, int32_t n_steps, double nu_ext_hz, double w_ext,
                    uint64_t seed, uint32_t* sp_src, int64_t* sp_t,
                    uint64_t cap) {
  return orc_update_range(nm, 0, n, n, n_slots, V, I, J, refr, rb, t0, n_steps,
                          nu_ext_hz, w_ext, seed, sp_src, sp_t, cap);
}

/* ------------------------------------------------------------------------ */
/* Simulation cycle (Section 1, Section 2.1): repeat {update the neurons for */
/* one min-delay interval; deliver that interval's spikes with REF} until   */
/* n_steps are done.  A final interval may be shorter.  Because every delay */
/* is at least the interval length, nothing delivered in an interval is due */
/* inside it.  Returns the number of spikes (stored up to cap).             */
/* ------------------------------------------------------------------------ */
uint64_t orc_simulate(const orc_neuron* nm, const orc_store* st,
                      int32_t interval, double* V, double* I, double* J,
                      int32_t* refr, double* rb, int64_t t0, int64_t n_steps,
                      double nu_ext_hz, double w_ext, uint64_t seed,
                      uint32_t* sp_src, int64_t* sp_t, uint64_t cap,
                      uint64_t* events_out) {
  uint64_t total = 0, events = 0;
  uint64_t iv_cap = (uint64_t)st->n * (uint64_t)interval;
  uint32_t* iv_src = malloc(sizeof(uint32_t) * (iv_cap ? iv_cap : 1));
  int64_t* iv_t = malloc(sizeof(int64_t) * (iv_cap ? iv_cap : 1));
  for (int64_t t = t0; t < t0 + n_steps; t += interval) {
    int32_t m = (int32_t)((t0 + n_steps - t) < interval ? (t0 + n_steps - t)
                                                        : interval);
    uint64_t k = orc_update(nm, st->n, st->n_slots, V, I, J, refr, rb, t, m,
                            nu_ext_hz, w_ext, seed, iv_src, iv_t, iv_cap);
    events += orc_deliver_ref(st, k, iv_src, iv_t, rb, NULL, NULL);
    for (uint64_t q = 0; q < k; ++q, ++total)
      if (total < cap) { sp_src[total] = iv_src[q]; sp_t[total] = iv_t[q]; }
  }
  free(iv_src); free(iv_t);
  if (events_out) *events_out = events;
  return total;
}

/* ------------------------------------------------------------------------ */
/* Spike-timing dependent plasticity of E->E synapses, evaluated at          */
/* delivery.  The paper's discussion (Section 6) describes the class of      */
/* plasticity rules it has in view: an update scheme driven by presynaptic   */
/* spikes in which a weight is computed only when the spike becomes visible  */
/* at the target, so the weight arithmetic becomes part of delivery; it      */
/* cites the pair-based power-law rule of Morrison, Aertsen & Diesmann       */
/* (2007).  Readings (the paper gives no formulas):                          */
/*  - a synapse i->j with delay d sees a presynaptic spike of i at its       */
/*    emission step t_e and a postsynaptic spike of j at t_p + d (the whole  */
/*    delay is dendritic);                                                   */
/*  - every pre/post pair interacts (all-to-all) with                        */
/*    D = (t_p + d - t_e) h:  D > 0 potentiates by                           */
/*    lambda w0^(1-mu) w^mu exp(-D / tau_plus),  D <= 0 depresses by         */
/*    lambda alpha w exp(D / tau_minus);                                     */
/*  - at a presynaptic spike t_e the synapse first applies, in time order,   */
/*    the potentiation owed to the post spikes seen since the previous pre   */
/*    spike (t_prev < t_p + d <= t_e; each against all earlier pre spikes),  */
/*    then the depression of the pairs (t_e, t_p) with t_p + d <= t_e, and   */
/*    delivers the resulting weight; weights stay in [0, w_max].             */
/* The traces are summed here directly over the full spike history.         */
/* ------------------------------------------------------------------------ */
typedef struct {
  double h, tau_plus, tau_minus, lambda, alpha, mu, w0, w_max;
  uint32_t n_exc;  /* synapse i->j is plastic iff i < n_exc and j < n_exc */
} orc_stdp;

typedef struct {
  uint32_t n, cap;  /* neurons, spike times kept per neuron */
  int64_t* t;       /* [n][cap], increasing per neuron */
  uint32_t* count;  /* [n] */
} orc_hist;

/* Append spikes (in any neuron order, increasing time per neuron).  Returns
 * -1 if a neuron's history is full. */
int orc_hist_add(orc_hist* hs, uint64_t n_sp, const uint32_t* src,
                 const int64_t* t) {
  for (uint64_t s = 0; s < n_sp; ++s) {
    uint32_t i = src[s];
    if (i >= hs->n || hs->count[i] >= hs->cap) return -1;
    hs->t[(size_t)i * hs->cap + hs->count[i]] = t[s];
    hs->count[i] += 1;
  }
  return 0;
}

/* sum over spikes t' of neuron i with t' < before of exp(-(at - t') h / tau) */
static double orc_trace_before(const orc_hist* hs, uint32_t i, int64_t before,
                               int64_t at, double h, double tau) {
  double k = 0.0;
  const int64_t* ts = hs->t + (size_t)i * hs->cap;
  for (uint32_t q = 0; q < hs->count[i]; ++q)
    if (ts[q] < before) k += exp(-(double)(at - ts[q]) * h / tau);
  return k;
}

uint64_t orc_deliver_stdp(const orc_store* st, double* w, const orc_stdp* p,
                          const orc_hist* hs, uint64_t n_sp,
                          const uint32_t* sp_src, const int64_t* sp_t,
                          double* rb, double* absw) {
  uint64_t events = 0;
  const double c_pot = p->lambda * pow(p->w0, 1.0 - p->mu);
  const double c_dep = p->lambda * p->alpha;
  for (uint64_t s = 0; s < n_sp; ++s) {
    const uint32_t i = sp_src[s];
    const int64_t te = sp_t[s];
    /* latest presynaptic spike before t_e */
    int has_prev = 0;
    int64_t tprev = 0;
    const int64_t* ti = hs->t + (size_t)i * hs->cap;
    for (uint32_t q = 0; q < hs->count[i]; ++q)
      if (ti[q] < te && (!has_prev || ti[q] > tprev)) { tprev = ti[q]; has_prev = 1; }
    for (uint64_t lcid = st->row_ptr[i]; lcid < st->row_ptr[i + 1]; ++lcid) {
      const uint32_t j = st->tgt[lcid];
      const int64_t d = st->delay[lcid];
      double wt = w[lcid];
      if (i < p->n_exc && j < p->n_exc) {
        const int64_t* tj = hs->t + (size_t)j * hs->cap;
        if (has_prev) {
          for (uint32_t q = 0; q < hs->count[j]; ++q) {
            const int64_t tp = tj[q];
            if (tp + d > tprev && tp + d <= te) {
              /* pre trace at t_p + d over all pre spikes before t_e */
              double kp = orc_trace_before(hs, i, te, tp + d, p->h, p->tau_plus);
              wt += c_pot * pow(wt, p->mu) * kp;
              if (wt > p->w_max) wt = p->w_max;
            }
          }
        }
        /* post trace at t_e over post spikes seen at t_p + d <= t_e */
        double km = orc_trace_before(hs, j, te - d + 1, te - d, p->h, p->tau_minus);
        wt -= c_dep * wt * km;
        if (wt < 0.0) wt = 0.0;
        w[lcid] = wt;
      }
      orc_add_value(st, rb, NULL, absw, j, te + d, wt);
      ++events;
    }
  }
  return events;
}

/* ------------------------------------------------------------------------ */
/* Thread-parallel form (Section 2.1: NEST's thread model).  Every thread    */
/* owns a contiguous range of neurons and holds the target segments of all  */
/* sources restricted to its targets (synapses live with their target).     */
/* Per interval each thread updates its own neurons; the threads' spikes    */
/* are merged into one list in step-major, neuron-minor order (the order of */
/* orc_update over the whole population); each thread then walks the whole  */
/* list with Algorithm REF onto its own targets.  A ring-buffer cell is     */
/* written by one thread only, and its additions come in the same order as  */
/* in orc_simulate (spikes in list order, synapses in segment order), so    */
/* the results are bitwise those of the single-thread form.  Used for      */
/* timing on all host cores and for whole-network runs of large nets.       */
/* ------------------------------------------------------------------------ */
#include <pthread.h>

typedef struct {
  uint32_t lo, hi;   /* owned neurons */
  uint64_t m;        /* synapses onto them */
  uint64_t* row_ptr; /* [N+1] */
  uint32_t* tgt;
  int32_t* delay;
  double* w;
  /* per-interval scratch */
  uint32_t* sp_src;
  int64_t* sp_t;
  uint64_t n_sp, events;
} orc_part;

typedef struct orc_mt {
  uint32_t n;
  int32_t n_slots;
  int n_threads;
  orc_part* part;
  /* merged interval list */
  uint32_t* m_src;
  int64_t* m_t;
  uint64_t m_n;
  pthread_barrier_t bar;
  /* the job of the current call */
  int job; /* 0 build, 1 simulate, 2 deliver, 3 update */
  const orc_conn* cp;
  const orc_neuron* nm;
  int32_t interval;
  double *V, *I, *J, *rb;
  int32_t* refr;
  int64_t t0, n_steps;
  double nu, w_ext;
  uint64_t seed;
  uint32_t* out_src;
  int64_t* out_t;
  uint64_t cap, total;
  const uint32_t* d_src;
  const int64_t* d_t;
  int status;
} orc_mt;

typedef struct {
  orc_mt* mt;
  int k;
} orc_mt_arg;

static void orc_mt_free_part(orc_part* p) {
  free(p->row_ptr); free(p->tgt); free(p->delay); free(p->w);
  free(p->sp_src); free(p->sp_t);
  memset(p, 0, sizeof(*p));
}

/* Thread k's share of one call. */
static void* orc_mt_worker(void* a) {
  orc_mt* mt = ((orc_mt_arg*)a)->mt;
  const int k = ((orc_mt_arg*)a)->k;
  orc_part* p = &mt->part[k];
  const orc_store st = {mt->n, mt->n_slots, p->row_ptr, p->tgt, p->delay, p->w};
  if (mt->job == 0) { /* the segments of the owned targets */
    const uint32_t kk = mt->cp->k_e + mt->cp->k_i;
    p->m = (uint64_t)(p->hi - p->lo) * kk;
    p->row_ptr = malloc(((size_t)mt->n + 1) * sizeof(uint64_t));
    p->tgt = malloc(p->m * sizeof(uint32_t) + 1);
    p->delay = malloc(p->m * sizeof(int32_t) + 1);
    p->w = malloc(p->m * sizeof(double) + 1);
    if (!p->row_ptr || !p->tgt || !p->delay || !p->w ||
        orc_build_fixed_indegree_targets(mt->cp, p->lo, p->hi, p->row_ptr,
                                         p->tgt, p->delay, p->w) != 0)
      p->events = 1; /* failure flag of the build */
    return NULL;
  }
  if (mt->job == 3) { /* the owned neurons' update; their spikes dropped */
    p->n_sp = orc_update_range(mt->nm, p->lo, p->hi, mt->n, mt->n_slots,
                               mt->V, mt->I, mt->J, mt->refr, mt->rb, mt->t0,
                               (int32_t)mt->n_steps, mt->nu, mt->w_ext,
                               mt->seed, NULL, NULL, 0);
    return NULL;
  }
  if (mt->job == 2) { /* one list onto the owned targets */
    p->events = orc_deliver_ref(&st, mt->m_n, mt->d_src, mt->d_t, mt->rb,
                                NULL, NULL);
    return NULL;
  }
  /* job 1: the time-driven cycle */
  p->events = 0;
  for (int64_t t = mt->t0; t < mt->t0 + mt->n_steps; t += mt->interval) {
    const int32_t m = (int32_t)((mt->t0 + mt->n_steps - t) < mt->interval
                                    ? (mt->t0 + mt->n_steps - t)
                                    : mt->interval);
    p->n_sp = orc_update_range(mt->nm, p->lo, p->hi, mt->n, mt->n_slots,
                               mt->V, mt->I, mt->J, mt->refr, mt->rb, t, m,
                               mt->nu, mt->w_ext, mt->seed, p->sp_src, p->sp_t,
                               (uint64_t)(p->hi - p->lo) * (uint64_t)m);
    pthread_barrier_wait(&mt->bar);
    if (k == 0) { /* merge: step by step, threads in neuron order */
      uint64_t q = 0;
      uint64_t* at = calloc((size_t)mt->n_threads, sizeof(uint64_t));
      for (int32_t s = 0; s < m; ++s)
        for (int r = 0; r < mt->n_threads; ++r) {
          const orc_part* pr = &mt->part[r];
          while (at[r] < pr->n_sp && pr->sp_t[at[r]] == t + s) {
            mt->m_src[q] = pr->sp_src[at[r]];
            mt->m_t[q] = pr->sp_t[at[r]];
            ++q;
            ++at[r];
          }
        }
      free(at);
      mt->m_n = q;
      for (uint64_t e = 0; e < q; ++e, ++mt->total)
        if (mt->total < mt->cap) {
          mt->out_src[mt->total] = mt->m_src[e];
          mt->out_t[mt->total] = mt->m_t[e];
        }
    }
    pthread_barrier_wait(&mt->bar);
    p->events += orc_deliver_ref(&st, mt->m_n, mt->m_src, mt->m_t, mt->rb,
                                 NULL, NULL);
  }
  return NULL;
}

static void orc_mt_run(orc_mt* mt) {
  pthread_t* th = malloc(sizeof(pthread_t) * (size_t)mt->n_threads);
  orc_mt_arg* args = malloc(sizeof(orc_mt_arg) * (size_t)mt->n_threads);
  for (int k = 0; k < mt->n_threads; ++k) {
    args[k].mt = mt;
    args[k].k = k;
    pthread_create(&th[k], NULL, orc_mt_worker, &args[k]);
  }
  for (int k = 0; k < mt->n_threads; ++k) pthread_join(th[k], NULL);
  free(th);
  free(args);
}

void orc_mt_destroy(orc_mt* mt) {
  if (!mt) return;
  for (int k = 0; k < mt->n_threads; ++k) orc_mt_free_part(&mt->part[k]);
  free(mt->part);
  free(mt->m_src);
  free(mt->m_t);
  pthread_barrier_destroy(&mt->bar);
  free(mt);
}

/* Build the per-thread stores of the fixed in-degree rule for n_threads
 * threads that split the neurons [tgt_lo, tgt_hi) evenly in order (the
 * whole population: 0, N); rows of every source, only the owned targets.
 * NULL if memory runs out or the range is invalid. */
orc_mt* orc_mt_create(const orc_conn* cp, int n_threads, int32_t n_slots,
                      uint32_t tgt_lo, uint32_t tgt_hi) {
  const uint32_t n = cp->n_e + cp->n_i;
  if (tgt_hi > n || tgt_lo > tgt_hi) return NULL;
  const uint32_t span = tgt_hi - tgt_lo;
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > span && span > 0) n_threads = (int)span;
  orc_mt* mt = calloc(1, sizeof(orc_mt));
  if (!mt) return NULL;
  mt->n = n;
  mt->n_slots = n_slots;
  mt->n_threads = n_threads;
  mt->part = calloc((size_t)n_threads, sizeof(orc_part));
  pthread_barrier_init(&mt->bar, NULL, (unsigned)n_threads);
  if (!mt->part) { free(mt); return NULL; }
  for (int k = 0; k < n_threads; ++k) {
    mt->part[k].lo = tgt_lo + (uint32_t)((uint64_t)span * (uint64_t)k /
                                         (uint64_t)n_threads);
    mt->part[k].hi = tgt_lo + (uint32_t)((uint64_t)span * (uint64_t)(k + 1) /
                                         (uint64_t)n_threads);
  }
  mt->job = 0;
  mt->cp = cp;
  orc_mt_run(mt);
  int bad = 0;
  for (int k = 0; k < n_threads; ++k) bad |= mt->part[k].events != 0;
  if (bad) { orc_mt_destroy(mt); return NULL; }
  return mt;
}

int orc_mt_threads(const orc_mt* mt) { return mt->n_threads; }

/* Bounds of thread k's neurons. */
void orc_mt_range(const orc_mt* mt, int k, uint32_t* lo, uint32_t* hi) {
  *lo = mt->part[k].lo;
  *hi = mt->part[k].hi;
}

/* orc_simulate on all threads: same arguments and results (bitwise), with
 * the store given by orc_mt_create.  Returns the number of spikes (stored
 * up to cap), or UINT64_MAX if memory runs out. */
uint64_t orc_mt_simulate(orc_mt* mt, const orc_neuron* nm, int32_t interval,
                         double* V, double* I, double* J, int32_t* refr,
                         double* rb, int64_t t0, int64_t n_steps,
                         double nu_ext_hz, double w_ext, uint64_t seed,
                         uint32_t* sp_src, int64_t* sp_t, uint64_t cap,
                         uint64_t* events_out) {
  if (mt->part[0].lo != 0 || mt->part[mt->n_threads - 1].hi != mt->n)
    return UINT64_MAX; /* a closed network needs every neuron */
  const uint64_t iv_cap = (uint64_t)mt->n * (uint64_t)interval;
  free(mt->m_src);
  free(mt->m_t);
  mt->m_src = malloc(sizeof(uint32_t) * (iv_cap ? iv_cap : 1));
  mt->m_t = malloc(sizeof(int64_t) * (iv_cap ? iv_cap : 1));
  int bad = !mt->m_src || !mt->m_t;
  for (int k = 0; k < mt->n_threads && !bad; ++k) {
    orc_part* p = &mt->part[k];
    const uint64_t c = (uint64_t)(p->hi - p->lo) * (uint64_t)interval;
    free(p->sp_src);
    free(p->sp_t);
    p->sp_src = malloc(sizeof(uint32_t) * (c ? c : 1));
    p->sp_t = malloc(sizeof(int64_t) * (c ? c : 1));
    bad |= !p->sp_src || !p->sp_t;
  }
  if (bad) return UINT64_MAX;
  mt->job = 1;
  mt->nm = nm;
  mt->interval = interval;
  mt->V = V; mt->I = I; mt->J = J; mt->refr = refr; mt->rb = rb;
  mt->t0 = t0;
  mt->n_steps = n_steps;
  mt->nu = nu_ext_hz;
  mt->w_ext = w_ext;
  mt->seed = seed;
  mt->out_src = sp_src;
  mt->out_t = sp_t;
  mt->cap = cap;
  mt->total = 0;
  orc_mt_run(mt);
  uint64_t events = 0;
  for (int k = 0; k < mt->n_threads; ++k) events += mt->part[k].events;
  if (events_out) *events_out = events;
  return mt->total;
}

/* Algorithm REF of one spike list onto every thread's targets (rb [S][N]);
 * returns the events.  Bitwise equal to orc_deliver_ref on the full store. */
uint64_t orc_mt_deliver(orc_mt* mt, uint64_t n_sp, const uint32_t* sp_src,
                        const int64_t* sp_t, double* rb) {
  mt->job = 2;
  mt->m_n = n_sp;
  mt->d_src = sp_src;
  mt->d_t = sp_t;
  mt->rb = rb;
  orc_mt_run(mt);
  uint64_t events = 0;
  for (int k = 0; k < mt->n_threads; ++k) events += mt->part[k].events;
  return events;
}

/* orc_update_range of every thread's neurons for n_steps steps from t0
 * (state and rb indexed globally, [S][N]); the spikes are counted, not
 * kept.  Returns the number of spikes. */
uint64_t orc_mt_update(orc_mt* mt, const orc_neuron* nm, double* V, double* I,
                       double* J, int32_t* refr, double* rb, int64_t t0,
                       int32_t n_steps, double nu_ext_hz, double w_ext,
                       uint64_t seed) {
  mt->job = 3;
  mt->nm = nm;
  mt->V = V; mt->I = I; mt->J = J; mt->refr = refr; mt->rb = rb;
  mt->t0 = t0;
  mt->n_steps = n_steps;
  mt->nu = nu_ext_hz;
  mt->w_ext = w_ext;
  mt->seed = seed;
  orc_mt_run(mt);
  uint64_t spikes = 0;
  for (int k = 0; k < mt->n_threads; ++k) spikes += mt->part[k].n_sp;
  return spikes;
}
