/*
 * snn_oracle.c -- plain, slow, single-threaded CPU simulator of the DPSNN-style
 * cortical grid (Pastorelli et al. 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header or table generator with the CUDA path; both are written from
 * the paper and from the step contract below.
 *
 * The simulation runs on the calling thread.  The tests may let several
 * threads generate the synapse rows a step needs (orc_configure_rows): a row
 * is a pure function of (seed, source), so this changes no result.
 *
 * Compile with -O2 -ffp-contract=off and no fast-math: every float operation
 * below is one IEEE-754 binary32 operation rounded to nearest, in the order
 * written, with no fused multiply-add.
 *
 * Model (Sec. 2.2):
 *   - grid of gx*gy modules of K = 1250 neurons, populations F (local index
 *     0..249), B (250..999), I (1000..1249); neuron n = module*K + local.
 *   - Eq. 2: dV/dt = -(V-E)/tau_m - g_c c/C_m + sum J delta(...) + sum J_ext delta(...),
 *            dc/dt = -c/tau_c + alpha_c sum delta(t - t_spike);
 *     threshold V_theta (crossed when V > V_theta), reset to V_r held for
 *     tau_arp, c += alpha_c on firing; inhibitory neurons have no adaptation.
 *   - Eq. 1: excitatory projections fall off as exp(-d/lambda) with the
 *     inter-module distance d, open boundaries; inhibitory projections stay
 *     in the source module; every neuron has out-degree M (0.9 K = 1125).
 *   - efficacies Gaussian with mean J and SD dJ_frac*|J|; external input a
 *     Poisson process of rate N_ext*nu_ext with Gaussian amplitudes (Sec. 2.1,
 *     Sec. 2.2, Table S1).
 *
 * Step contract (time-driven, dt = 0.1 ms, D = n_delay + 1 ring slots):
 *   for each neuron n (population p) at step t, slot st = t mod D:
 *     I = ring[st][n]; ring[st][n] = 0
 *     w = word (n mod 4) of Philox4x32-10(key = seed, ctr = (n div 4, t, 1, 0))
 *     k_ext = #{k < 16 : (w >> 12) >= T_p[k]}  (Poisson CDF thresholds, 2^20 scale)
 *     I += amp_p[z-index of external event e] for e < k_ext: event 0 takes
 *          w & 0xFFF, event e >= 1 the top 12 bits of 16-bit half (e-1) mod 8
 *          of Philox(key = seed, ctr = (n, t, 3, (e-1) div 8))
 *     if ref > 0: ref -= 1, V = V_r                      (input discarded)
 *     else: V = fl(fl(E + fl(fl(P_VV*fl(V-E)) + fl(P_Vc*c))) + fl(I*2^-16))
 *           if V > V_theta: spike, V = V_r, ref = n_arp
 *     c = fl(P_cc*c) (+ alpha, rounded, when the neuron fired)
 *   then every spike of step t adds its row's fixed-point weights into
 *   ring[(t + d) mod D][target].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define ORC_K 1250
#define ORC_ZTAB 4096
#define ORC_KMAX 16
#define ORC_FMT_F32 0
#define ORC_FMT_I16 1
#define ORC_ROW_BATCH 16384   /* spikes whose rows are generated together */

typedef struct {
  int32_t gx, gy;
  float lambda;
  float p_local;        /* >= 0: share of excitatory out-degree kept local; < 0: pure Eq. 1 */
  int32_t out_degree;
  int32_t n_delay;
  int32_t min_delay;    /* delays uniform on min_delay..n_delay (0 is read as 1) */
  float dt_ms;
  int32_t record_format;
  int32_t bin_steps;
  float tau_m[3], C_m[3], E_L[3], V_th[3], V_r[3], tau_arp[3], alpha_c[3], tau_c[3], g_c[3];
  float J[3][3];        /* [target population][source population], mV */
  float dJ_frac;
  float J_ext[3];
  float dJ_ext_frac;
  float nu_ext[3];      /* Hz per external train */
  float N_ext[3];       /* external trains per neuron */
} orc_params;

typedef struct {
  float pvv, pvc, pcc, el, vth, vr, alpha;
  int32_t narp;
  uint64_t thr[ORC_KMAX];
  int32_t amp[ORC_ZTAB];
} orc_pop;

typedef struct {
  orc_params p;
  uint32_t k0, k1;          /* Philox key = seed */
  int32_t G, N, M, D;
  float ztab[ORC_ZTAB];
  orc_pop pop[3];
  uint32_t *cdf;            /* [G][G-1] module thresholds */
  float *V, *c;
  int32_t *ref;
  int32_t *ring;            /* [D][N] */
  uint32_t **row_key;       /* lazily generated rows (pure functions of seed, source) */
  float **row_w;
  int32_t row_threads;      /* threads that generate a step's missing rows (1 = this thread) */
  int32_t keep_rows;        /* 1: rows stay cached after use; 0: freed after the step's delivery */
  uint32_t t;
  /* records */
  uint32_t *rs_t, *rs_n;
  size_t rs_len, rs_cap;
  uint32_t *rates;          /* [bin][G][3] */
  size_t rates_bins;
  uint64_t n_spikes, n_ext_events, n_rec_events;
  double row_build_seconds;   /* wall time spent generating rows on first use */
  /* optional per-step input trace for tiny tests: recurrent and external input */
  int32_t *trace_rec, *trace_ext;
  uint32_t trace_t0, trace_steps;
} orc_net;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32 */
/* multiplications with the Weyl-sequence key schedule.                       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], uint32_t key0, uint32_t key1, uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key0, k1 = key1;
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod1;
    uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void orc_rng(const orc_net *net, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  orc_philox4x32_10(ctr, net->k0, net->k1, out);
}

static int orc_pop_of(int32_t local) { return local < 250 ? 0 : (local < 1000 ? 1 : 2); }

/* ------------------------------------------------------------------------ */
/* Tables                                                                    */
/* ------------------------------------------------------------------------ */

/* Standard normal CDF written through erfc. */
static double orc_phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Inverse standard normal CDF by bisection on orc_phi (monotone), run until
 * the bracket cannot shrink any further in double precision. */
double orc_inv_phi(double p) {
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 2000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_phi(mid) < p) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

static float orc_keep_sign(float w, float mean) {
  if (mean > 0.0f && w < 0.0f) return 0.0f;
  if (mean < 0.0f && w > 0.0f) return 0.0f;
  return w;
}

/* Exact propagators of the linear part of Eq. 2 over one step. */
static void orc_build_pop(orc_net *net, int p) {
  const orc_params *P = &net->p;
  orc_pop *q = &net->pop[p];
  double dt = (double)P->dt_ms;
  double tm = (double)P->tau_m[p];
  double tc = (double)P->tau_c[p];
  double gc = (double)P->g_c[p] / (double)P->C_m[p];     /* nS / pF = 1/ms */
  double em = exp(-dt / tm);
  double ec = exp(-dt / tc);
  double pvc;
  if (tc != tm) pvc = -(gc * (tm * tc / (tc - tm))) * (ec - em);
  else pvc = -(gc * dt) * em;
  q->pvv = (float)em;
  q->pcc = (float)ec;
  q->pvc = (float)pvc;
  q->el = P->E_L[p];
  q->vth = P->V_th[p];
  q->vr = P->V_r[p];
  q->alpha = P->alpha_c[p];
  q->narp = (int32_t)lround((double)P->tau_arp[p] / dt);
  /* Poisson count of the superposed external trains: rate N_ext*nu_ext. */
  double lam = (double)P->N_ext[p] * (double)P->nu_ext[p] * (double)P->dt_ms / 1000.0;
  double pmf = exp(-lam), cum = pmf;
  for (int k = 0; k < ORC_KMAX; ++k) {
    if (k > 0) { pmf = (pmf * lam) / (double)k; cum = cum + pmf; }
    q->thr[k] = (uint64_t)floor(cum * 1048576.0);
  }
  /* external amplitude table: J_ext + sigma*z in 2^-16 mV */
  float sig = P->dJ_ext_frac * fabsf(P->J_ext[p]);
  for (int i = 0; i < ORC_ZTAB; ++i) {
    float prod = sig * net->ztab[i];
    float w = P->J_ext[p] + prod;
    w = orc_keep_sign(w, P->J_ext[p]);
    float scaled = w * 65536.0f;
    q->amp[i] = (int32_t)lrintf(scaled);
  }
}

/* Thresholds of the target-module distribution of one source module: the
 * exponential decay with distance of Eq. 1 (Sec. 2.2), either as the pure
 * kernel over all modules or with a fixed local share. */
static void orc_build_cdf_row(orc_net *net, int32_t ms, uint32_t *T) {
  const orc_params *P = &net->p;
  int32_t G = net->G, gx = P->gx;
  int32_t sx = ms % gx, sy = ms / gx;
  double lam = (double)P->lambda;
  double pl = (double)P->p_local;
  double S = 0.0;
  for (int32_t m = 0; m < G; ++m) {
    if (pl >= 0.0 && m == ms) continue;
    double dx = (double)(m % gx - sx), dy = (double)(m / gx - sy);
    double d = sqrt(dx * dx + dy * dy);
    S = S + exp(-(d / lam));
  }
  double cum = 0.0;
  for (int32_t m = 0; m < G - 1; ++m) {
    double dx = (double)(m % gx - sx), dy = (double)(m / gx - sy);
    double d = sqrt(dx * dx + dy * dy);
    double e = exp(-(d / lam));
    double prob;
    if (pl >= 0.0) prob = (m == ms) ? pl : ((1.0 - pl) * e) / S;
    else prob = e / S;
    cum = cum + prob;
    double f = floor(cum * 4294967296.0);
    T[m] = f >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)f;
  }
}

/* ------------------------------------------------------------------------ */
/* Construction of one outgoing row                                          */
/* ------------------------------------------------------------------------ */

/* Target module: first m < G-1 with u < T[m], else G-1 (binary search). */
static int32_t orc_pick_module(const uint32_t *T, int32_t G, uint32_t u) {
  int32_t lo = 0, hi = G - 1;       /* answer in [lo, hi] */
  while (lo < hi) {
    int32_t mid = lo + (hi - lo) / 2;
    if (u < T[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* Synapse j of source s: target module (Eq. 1), target neuron uniform in the
 * module, delay uniform on min_delay..n_delay steps (the paper fixes only the
 * minimum delay, Sec. 2.1.1), and efficacy Gaussian around J (Sec. 2.2), from
 * one Philox call. */
void orc_synapse(const orc_net *net, uint32_t s, uint32_t j, uint32_t *key, float *w) {
  const orc_params *P = &net->p;
  uint32_t r[4];
  orc_rng(net, s, j, 0u, 0u, r);
  int32_t ms = (int32_t)(s / ORC_K), sl = (int32_t)(s % ORC_K);
  int sp = orc_pop_of(sl);
  int32_t mt;
  if (sp == 2 || net->G == 1) mt = ms;
  else mt = orc_pick_module(net->cdf + (size_t)ms * (size_t)(net->G - 1), net->G, r[0]);
  uint32_t lt = (uint32_t)(((uint64_t)r[1] * (uint64_t)ORC_K) >> 32);
  uint32_t tgt = (uint32_t)mt * ORC_K + lt;
  uint32_t dmin = P->min_delay < 1 ? 1u : (uint32_t)P->min_delay;
  uint32_t d = dmin + (uint32_t)(((uint64_t)r[2] * (uint64_t)(P->n_delay - (int32_t)dmin + 1)) >> 32);
  int tp = orc_pop_of((int32_t)lt);
  float J = P->J[tp][sp];
  float sig = P->dJ_frac * fabsf(J);
  float prod = sig * net->ztab[r[3] >> 20];
  float wv = J + prod;
  *w = orc_keep_sign(wv, J);
  *key = (d << 24) | tgt;
}

/* One drawn synapse before ordering: its record key and its draw index j. */
typedef struct {
  uint32_t key;
  int32_t j;
} orc_rec;

static int orc_rec_cmp(const void *a, const void *b) {
  const orc_rec *x = (const orc_rec *)a, *y = (const orc_rec *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->j > y->j) - (x->j < y->j);
}

/* Row of source s: its M synapses ordered by key (delay << 24 | target), i.e.
 * grouped by delay (Sec. 2.1) and by target within a delay, synapses with the
 * same delay and target in draw order.  The order is a storage choice: the
 * delivered sums do not depend on it. */
void orc_build_row(const orc_net *net, uint32_t s, uint32_t *key_out, float *w_out) {
  int32_t M = net->M;
  orc_rec *r = (orc_rec *)malloc(sizeof(orc_rec) * (size_t)M);
  float *w = (float *)malloc(sizeof(float) * (size_t)M);
  for (int32_t j = 0; j < M; ++j) {
    orc_synapse(net, s, (uint32_t)j, &r[j].key, &w[j]);
    r[j].j = j;
  }
  qsort(r, (size_t)M, sizeof(orc_rec), orc_rec_cmp);
  for (int32_t p = 0; p < M; ++p) {
    key_out[p] = r[p].key;
    w_out[p] = w[r[p].j];
  }
  free(w);
  free(r);
}

static double orc_now(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void orc_make_row(orc_net *net, uint32_t s) {
  net->row_key[s] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)net->M);
  net->row_w[s] = (float *)malloc(sizeof(float) * (size_t)net->M);
  orc_build_row(net, s, net->row_key[s], net->row_w[s]);
}

/* Rows of a list of sources generated by several threads.  A row is a pure
 * function of (seed, source) and each thread writes only its own sources'
 * slots, so the result does not depend on how the list is split. */
typedef struct {
  orc_net *net;
  const uint32_t *src;
  int32_t n, first, stride;
} orc_row_job;

static void *orc_row_worker(void *arg) {
  orc_row_job *job = (orc_row_job *)arg;
  for (int32_t i = job->first; i < job->n; i += job->stride) orc_make_row(job->net, job->src[i]);
  return NULL;
}

static void orc_make_rows(orc_net *net, const uint32_t *src, int32_t n) {
  double t_in = orc_now();
  int32_t T = net->row_threads;
  if (T > 64) T = 64;
  if (T > n) T = n;
  if (T <= 1) {
    for (int32_t i = 0; i < n; ++i) orc_make_row(net, src[i]);
  } else {
    pthread_t th[64];
    orc_row_job jobs[64];
    int32_t started = 0;
    for (int32_t k = 0; k < T; ++k) {
      jobs[k].net = net; jobs[k].src = src; jobs[k].n = n; jobs[k].first = k; jobs[k].stride = T;
      if (pthread_create(&th[k], NULL, orc_row_worker, &jobs[k]) != 0) break;
      ++started;
    }
    /* whatever could not be handed to a thread is generated here */
    for (int32_t k = started; k < T; ++k) orc_row_worker(&jobs[k]);
    for (int32_t k = 0; k < started; ++k) pthread_join(th[k], NULL);
  }
  net->row_build_seconds += orc_now() - t_in;
}

static void orc_drop_row(orc_net *net, uint32_t s) {
  free(net->row_key[s]); free(net->row_w[s]);
  net->row_key[s] = NULL; net->row_w[s] = NULL;
}

double orc_row_build_seconds(const orc_net *net) { return net->row_build_seconds; }

/* Test-harness setting, no effect on results: how many threads generate the
 * rows a step needs, and whether rows stay cached (a 5M-neuron grid needs
 * ~46 GB to cache every row). */
void orc_configure_rows(orc_net *net, int32_t threads, int32_t keep) {
  net->row_threads = threads < 1 ? 1 : threads;
  net->keep_rows = keep ? 1 : 0;
}

/* Fixed-point weight (2^-16 mV) delivered by one record. */
static int32_t orc_wfix(const orc_net *net, float w) {
  if (net->p.record_format == ORC_FMT_I16) {
    long q = lrintf(w * 1024.0f);
    if (q > 32767) q = 32767;
    if (q < -32768) q = -32768;
    return (int32_t)q * 64;
  }
  return (int32_t)lrintf(w * 65536.0f);
}

/* ------------------------------------------------------------------------ */
/* Neuron update (Eq. 2 over one step)                                       */
/* ------------------------------------------------------------------------ */
int orc_neuron_update(const orc_pop *q, float *V, float *c, int32_t *ref, int32_t I) {
  int spike = 0;
  float c_old = *c;
  if (*ref > 0) {
    *ref -= 1;
    *V = q->vr;
  } else {
    float a = *V - q->el;
    float b = q->pvv * a;
    float e = q->pvc * c_old;
    float f = b + e;
    float g = q->el + f;
    float x = (float)I * (1.0f / 65536.0f);
    float vn = g + x;
    if (vn > q->vth) { spike = 1; vn = q->vr; *ref = q->narp; }
    *V = vn;
  }
  float cn = q->pcc * c_old;
  if (spike) cn = cn + q->alpha;
  *c = cn;
  return spike;
}

/* Gaussian-table index (12 bits) of external event e of neuron n at step t
 * (external Poisson drive with Gaussian efficacies, Sec. 2.1 and Table S1);
 * `w` is the neuron's 32-bit word of the step's shared draw. */
static uint32_t orc_ext_index(const orc_net *net, uint32_t w, uint32_t n, uint32_t t, int32_t e) {
  if (e == 0) return w & 0xFFFu;
  uint32_t r[4];
  int32_t i = (e - 1) % 8;
  orc_rng(net, n, t, 3u, (uint32_t)((e - 1) / 8), r);
  uint32_t word = r[i / 2];
  uint32_t half = (i & 1) ? (word >> 16) : (word & 0xFFFFu);
  return half >> 4;
}

/* ------------------------------------------------------------------------ */
/* Public API                                                                */
/* ------------------------------------------------------------------------ */
void orc_destroy(orc_net *net) {
  if (!net) return;
  if (net->row_key) {
    for (int32_t s = 0; s < net->N; ++s) { free(net->row_key[s]); free(net->row_w[s]); }
  }
  free(net->row_key); free(net->row_w);
  free(net->cdf); free(net->V); free(net->c); free(net->ref); free(net->ring);
  free(net->rs_t); free(net->rs_n); free(net->rates);
  free(net->trace_rec); free(net->trace_ext);
  free(net);
}

orc_net *orc_create(const orc_params *P, uint64_t seed) {
  if (P->gx < 1 || P->gy < 1 || P->out_degree < 1 || P->n_delay < 1 || P->n_delay > 255 ||
      P->min_delay < 0 || P->min_delay > P->n_delay ||
      P->bin_steps < 1 || !(P->dt_ms > 0.0f) || !(P->lambda > 0.0f))
    return NULL;
  orc_net *net = (orc_net *)calloc(1, sizeof(orc_net));
  net->p = *P;
  net->k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  net->k1 = (uint32_t)(seed >> 32);
  net->G = P->gx * P->gy;
  net->N = net->G * ORC_K;
  net->M = P->out_degree;
  net->D = P->n_delay + 1;
  for (int i = 0; i < ORC_ZTAB; ++i) net->ztab[i] = (float)orc_inv_phi(((double)i + 0.5) / (double)ORC_ZTAB);
  for (int p = 0; p < 3; ++p) orc_build_pop(net, p);
  if (net->G > 1) {
    net->cdf = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)net->G * (size_t)(net->G - 1));
    for (int32_t m = 0; m < net->G; ++m) orc_build_cdf_row(net, m, net->cdf + (size_t)m * (size_t)(net->G - 1));
  }
  size_t N = (size_t)net->N;
  net->V = (float *)malloc(sizeof(float) * N);
  net->c = (float *)calloc(N, sizeof(float));
  net->ref = (int32_t *)calloc(N, sizeof(int32_t));
  net->ring = (int32_t *)calloc(N * (size_t)net->D, sizeof(int32_t));
  net->row_key = (uint32_t **)calloc(N, sizeof(uint32_t *));
  net->row_w = (float **)calloc(N, sizeof(float *));
  net->row_threads = 1;
  net->keep_rows = 1;
  /* initial membrane potential uniform on [0, V_theta) from stream 2 */
  for (int32_t n = 0; n < net->N; ++n) {
    uint32_t r[4];
    orc_rng(net, (uint32_t)n, 0u, 2u, 0u, r);
    float u = (float)(r[0] >> 8) * (1.0f / 16777216.0f);
    net->V[n] = net->pop[orc_pop_of(n % ORC_K)].vth * u;
  }
  return net;
}

/* Record a spike: raster entry and its (5 ms bin, module, population) count
 * (Sec. 2.3). */
static void orc_push_spike(orc_net *net, uint32_t t, uint32_t n) {
  if (net->rs_len == net->rs_cap) {
    net->rs_cap = net->rs_cap ? 2 * net->rs_cap : 4096;
    net->rs_t = (uint32_t *)realloc(net->rs_t, sizeof(uint32_t) * net->rs_cap);
    net->rs_n = (uint32_t *)realloc(net->rs_n, sizeof(uint32_t) * net->rs_cap);
  }
  net->rs_t[net->rs_len] = t;
  net->rs_n[net->rs_len] = n;
  net->rs_len++;
  size_t bin = t / (uint32_t)net->p.bin_steps;
  size_t per_bin = (size_t)net->G * 3;
  if (bin >= net->rates_bins) {
    size_t nb = bin + 1 > 2 * net->rates_bins ? bin + 1 : 2 * net->rates_bins;
    net->rates = (uint32_t *)realloc(net->rates, sizeof(uint32_t) * nb * per_bin);
    memset(net->rates + net->rates_bins * per_bin, 0, sizeof(uint32_t) * (nb - net->rates_bins) * per_bin);
    net->rates_bins = nb;
  }
  net->rates[bin * per_bin + (n / ORC_K) * 3 + (size_t)orc_pop_of((int32_t)(n % ORC_K))] += 1;
}

/* Advance `steps` time steps: every neuron in index order (Eq. 2 with its
 * input and external drive), then every spike of the step delivered through
 * its row into the delay ring, sources in ascending order (Sec. 2.1.1). */
int orc_run(orc_net *net, uint32_t steps) {
  int32_t N = net->N, M = net->M, D = net->D;
  uint32_t *spk = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
  uint32_t *miss = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ORC_ROW_BATCH);
  for (uint32_t it = 0; it < steps; ++it) {
    uint32_t t = net->t;
    int32_t st = (int32_t)(t % (uint32_t)D);
    int32_t *slot = net->ring + (size_t)st * (size_t)N;
    int tracing = net->trace_rec && t >= net->trace_t0 && t - net->trace_t0 < net->trace_steps;
    int32_t nsp = 0;
    for (int32_t n = 0; n < N; ++n) {
      int p = orc_pop_of(n % ORC_K);
      const orc_pop *q = &net->pop[p];
      int32_t I = slot[n];
      slot[n] = 0;
      uint32_t r[4];
      orc_rng(net, (uint32_t)n / 4u, t, 1u, 0u, r);
      uint32_t w = r[n % 4];
      int32_t kext = 0;
      while (kext < ORC_KMAX && (uint64_t)(w >> 12) >= q->thr[kext]) kext++;
      int32_t Iext = 0;
      for (int32_t e = 0; e < kext; ++e) Iext += q->amp[orc_ext_index(net, w, (uint32_t)n, t, e)];
      net->n_ext_events += (uint64_t)kext;
      if (tracing) {
        size_t o = (size_t)(t - net->trace_t0) * (size_t)N + (size_t)n;
        net->trace_rec[o] = I;
        net->trace_ext[o] = Iext;
      }
      I += Iext;
      if (orc_neuron_update(q, &net->V[n], &net->c[n], &net->ref[n], I)) {
        spk[nsp++] = (uint32_t)n;
        orc_push_spike(net, t, (uint32_t)n);
      }
    }
    /* delivery of this step's spikes in ascending source order, in batches
     * whose missing rows are generated first */
    for (int32_t b0 = 0; b0 < nsp; b0 += ORC_ROW_BATCH) {
      int32_t b1 = b0 + ORC_ROW_BATCH < nsp ? b0 + ORC_ROW_BATCH : nsp;
      int32_t nmiss = 0;
      for (int32_t i = b0; i < b1; ++i)
        if (!net->row_key[spk[i]]) miss[nmiss++] = spk[i];
      if (nmiss) orc_make_rows(net, miss, nmiss);
      for (int32_t i = b0; i < b1; ++i) {
        uint32_t s = spk[i];
        const uint32_t *rk = net->row_key[s];
        const float *rw = net->row_w[s];
        for (int32_t j = 0; j < M; ++j) {
          uint32_t d = rk[j] >> 24, tgt = rk[j] & 0xFFFFFFu;
          int32_t sl = (int32_t)((t + d) % (uint32_t)D);
          net->ring[(size_t)sl * (size_t)N + tgt] += orc_wfix(net, rw[j]);
        }
      }
      if (!net->keep_rows)
        for (int32_t i = b0; i < b1; ++i) orc_drop_row(net, spk[i]);
    }
    net->n_spikes += (uint64_t)nsp;
    net->n_rec_events += (uint64_t)nsp * (uint64_t)M;
    net->t = t + 1;
  }
  free(miss);
  free(spk);
  return 0;
}

/* ---- accessors used by the tests ---------------------------------------- */
uint32_t orc_time(const orc_net *net) { return net->t; }
int32_t orc_n(const orc_net *net) { return net->N; }
size_t orc_raster_len(const orc_net *net) { return net->rs_len; }
void orc_raster(const orc_net *net, uint32_t *t_out, uint32_t *n_out) {
  memcpy(t_out, net->rs_t, sizeof(uint32_t) * net->rs_len);
  memcpy(n_out, net->rs_n, sizeof(uint32_t) * net->rs_len);
}
size_t orc_rates_bins(const orc_net *net) {
  if (net->t == 0) return 0;
  return (size_t)((net->t + (uint32_t)net->p.bin_steps - 1) / (uint32_t)net->p.bin_steps);
}
void orc_rates(const orc_net *net, uint32_t *out) {
  size_t nb = orc_rates_bins(net), per = (size_t)net->G * 3;
  memset(out, 0, sizeof(uint32_t) * nb * per);
  size_t have = nb < net->rates_bins ? nb : net->rates_bins;
  if (have) memcpy(out, net->rates, sizeof(uint32_t) * have * per);
}
void orc_state(const orc_net *net, float *V, float *c, int32_t *ref) {
  size_t N = (size_t)net->N;
  memcpy(V, net->V, sizeof(float) * N);
  memcpy(c, net->c, sizeof(float) * N);
  memcpy(ref, net->ref, sizeof(int32_t) * N);
}
void orc_ring(const orc_net *net, int32_t *out) {
  memcpy(out, net->ring, sizeof(int32_t) * (size_t)net->N * (size_t)net->D);
}
void orc_counters(const orc_net *net, uint64_t out[3]) {
  out[0] = net->n_spikes; out[1] = net->n_rec_events; out[2] = net->n_ext_events;
}
void orc_ztab(const orc_net *net, float *out) { memcpy(out, net->ztab, sizeof(net->ztab)); }
/* per population: pvv, pvc, pcc (float), narp (int), thresholds (u64[16]), amp (i32[4096]) */
void orc_pop_tables(const orc_net *net, int p, float prop[3], int32_t *narp, uint64_t *thr, int32_t *amp) {
  const orc_pop *q = &net->pop[p];
  prop[0] = q->pvv; prop[1] = q->pvc; prop[2] = q->pcc;
  *narp = q->narp;
  memcpy(thr, q->thr, sizeof(q->thr));
  memcpy(amp, q->amp, sizeof(q->amp));
}
void orc_cdf_row(const orc_net *net, int32_t ms, uint32_t *out) {
  if (net->G > 1) memcpy(out, net->cdf + (size_t)ms * (size_t)(net->G - 1), sizeof(uint32_t) * (size_t)(net->G - 1));
}
int orc_enable_trace(orc_net *net, uint32_t t0, uint32_t steps) {
  size_t n = (size_t)steps * (size_t)net->N;
  free(net->trace_rec); free(net->trace_ext);
  net->trace_rec = (int32_t *)calloc(n, sizeof(int32_t));
  net->trace_ext = (int32_t *)calloc(n, sizeof(int32_t));
  net->trace_t0 = t0;
  net->trace_steps = steps;
  return (net->trace_rec && net->trace_ext) ? 0 : -1;
}
void orc_trace(const orc_net *net, int32_t *rec, int32_t *ext) {
  size_t n = (size_t)net->trace_steps * (size_t)net->N;
  memcpy(rec, net->trace_rec, sizeof(int32_t) * n);
  memcpy(ext, net->trace_ext, sizeof(int32_t) * n);
}

/* Single-neuron driver for closed-form checks: runs the same update as the
 * network with a given per-step input (2^-16 mV) and no external drive. */
int orc_neuron_trace(const orc_params *P, int32_t pop, float V0, float c0, uint32_t steps,
                     const int32_t *I, float *V_out, float *c_out, uint8_t *spike_out) {
  orc_net tmp;
  memset(&tmp, 0, sizeof(tmp));
  tmp.p = *P;
  for (int i = 0; i < ORC_ZTAB; ++i) tmp.ztab[i] = 0.0f;
  orc_build_pop(&tmp, pop);
  const orc_pop *q = &tmp.pop[pop];
  float V = V0, c = c0;
  int32_t ref = 0;
  for (uint32_t s = 0; s < steps; ++s) {
    int sp = orc_neuron_update(q, &V, &c, &ref, I[s]);
    V_out[s] = V; c_out[s] = c; spike_out[s] = (uint8_t)sp;
  }
  return 0;
}
