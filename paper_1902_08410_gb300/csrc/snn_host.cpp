// snn_host.cpp -- host runtime of the C ABI declared in include/snn.h.
//
// Responsibilities: validate parameters, build the small FP64 tables the
// kernels consume (Eq. 2 propagators, Poisson thresholds, Gaussian quantiles,
// Eq. 1 module thresholds), own each network's device arena, capture windows
// of time steps into CUDA graphs, and drain spike records and rate counts to
// host memory after every window.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/snn.h"
#include "snn_internal.h"
#include "snn_raster.h"

using namespace snn;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

int snn_fail(int code, const std::string &msg);
static int fail(int code, const std::string &msg) { return snn_fail(code, msg); }
int snn_fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

#define CU_TRY(expr)                                                                          \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess) return fail(SNN_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

extern "C" const char *snn_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
struct AllocFns {
  snn_alloc_fn alloc = nullptr;
  snn_free_fn free_fn = nullptr;
  void *ctx = nullptr;
};
static std::mutex g_alloc_mu;
static AllocFns g_alloc;

extern "C" int snn_set_allocator(snn_alloc_fn alloc, snn_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(SNN_ERR_ARG, "alloc and free must both be set or both be NULL");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free_fn = free_fn;
  g_alloc.ctx = ctx;
  return SNN_OK;
}

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  AllocFns fns;
  void release() {
    if (!p) return;
    if (fns.free_fn) fns.free_fn(p, fns.ctx);
    else cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

static int dev_alloc(DevBuf &b, size_t bytes) {
  AllocFns fns;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    fns = g_alloc;
  }
  void *p = nullptr;
  if (fns.alloc) {
    p = fns.alloc(bytes, fns.ctx);
    if (!p) return fail(SNN_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? SNN_ERR_OOM : SNN_ERR_CUDA,
                  "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
    if (fns.free_fn) fns.free_fn(p, fns.ctx); else cudaFree(p);
    return fail(SNN_ERR_ARG, "allocator returned memory that is not 256-byte aligned");
  }
  b.p = p;
  b.bytes = bytes;
  b.fns = fns;
  return SNN_OK;
}

// ---------------------------------------------------------------------------
// host tables (FP64, rounded once)
// ---------------------------------------------------------------------------
namespace snn {

double std_normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Inverse of the standard normal CDF: a coarse bracket by halving, then
// Newton steps on Phi(x) - p until the correction vanishes.
double inverse_normal_cdf(double p) {
  double a = -12.0, b = 12.0;
  for (int i = 0; i < 48; ++i) {
    const double c = 0.5 * (a + b);
    if (std_normal_cdf(c) < p) a = c; else b = c;
  }
  double x = 0.5 * (a + b);
  const double inv_sqrt_2pi = 0.3989422804014327;
  for (int i = 0; i < 8; ++i) {
    const double dens = inv_sqrt_2pi * std::exp(-0.5 * x * x);
    const double step = (std_normal_cdf(x) - p) / dens;
    const double xn = x - step;
    if (xn == x) break;
    x = xn;
  }
  // settle on the smallest double with Phi(x) >= p
  for (int i = 0; i < 256 && std_normal_cdf(x) < p; ++i) x = std::nextafter(x, 1e300);
  for (int i = 0; i < 256; ++i) {
    const double dn = std::nextafter(x, -1e300);
    if (std_normal_cdf(dn) >= p) x = dn; else break;
  }
  return x;
}

struct PopTables {
  float pvv, pvc, pcc;
  int32_t narp;
  unsigned long long thr[kPoisMax];
};

PopTables pop_tables(const snn_params &p, int q) {
  PopTables t{};
  const double dt = (double)p.dt_ms, tm = (double)p.tau_m[q], tc = (double)p.tau_c[q];
  const double g_over_c = (double)p.g_c[q] / (double)p.C_m[q];
  const double decay_m = std::exp(-dt / tm);
  const double decay_c = std::exp(-dt / tc);
  // V(dt) picks up -(g/C) * int_0^dt exp(-(dt-s)/tau_m) c(0) exp(-s/tau_c) ds
  double coupling;
  if (tc == tm) coupling = -(g_over_c * dt) * decay_m;
  else coupling = -(g_over_c * (tm * tc / (tc - tm))) * (decay_c - decay_m);
  t.pvv = (float)decay_m;
  t.pcc = (float)decay_c;
  t.pvc = (float)coupling;
  t.narp = (int32_t)std::lround((double)p.tau_arp[q] / dt);
  const double lam = (double)p.N_ext[q] * (double)p.nu_ext[q] * (double)p.dt_ms / 1000.0;
  double pk = std::exp(-lam), acc = pk;
  for (int k = 0; k < kPoisMax; ++k) {
    if (k) {
      pk = (pk * lam) / (double)k;
      acc = acc + pk;
    }
    t.thr[k] = (unsigned long long)std::floor(acc * 1048576.0);   // compared with a 20-bit uniform
  }
  return t;
}

float sign_kept(float w, float mean) {
  if (mean > 0.0f && w < 0.0f) return 0.0f;
  if (mean < 0.0f && w > 0.0f) return 0.0f;
  return w;
}

// Thresholds T[0..G-2] of the target-module distribution of every source
// module (Eq. 1), built from one table of kernel values per displacement.
// Eq. 1 thresholds T[src][m] = floor(2^32 * sum_{m' <= m} P(m' | src)) for
// every source module, in FP64 with the sums taken in module index order.
// Rows are independent and computed in parallel over host threads; the
// arithmetic of every row is the same sequence as a serial loop.
void module_thresholds(const snn_params &p, std::vector<uint32_t> &out) {
  const int gx = p.gx, gy = p.gy, G = gx * gy;
  out.assign((size_t)G * (size_t)(G - 1), 0u);
  if (G < 2) return;
  const double lam = (double)p.lambda, pl = (double)p.p_local;
  std::vector<double> kern((size_t)gx * gy);   // kernel value for |dx|, |dy|
  for (int ay = 0; ay < gy; ++ay)
    for (int ax = 0; ax < gx; ++ax) {
      const double dx = (double)ax, dy = (double)ay;
      kern[(size_t)ay * gx + ax] = std::exp(-(std::sqrt(dx * dx + dy * dy) / lam));
    }
  auto rows = [&](int src0, int src1) {
    for (int src = src0; src < src1; ++src) {
      const int sx = src % gx, sy = src / gx;
      double total = 0.0;
      for (int my = 0, m = 0; my < gy; ++my) {
        const double *krow = kern.data() + (size_t)std::abs(my - sy) * gx;
        for (int mx = 0; mx < gx; ++mx, ++m) {
          if (pl >= 0.0 && m == src) continue;
          total = total + krow[std::abs(mx - sx)];
        }
      }
      double acc = 0.0;
      uint32_t *T = out.data() + (size_t)src * (size_t)(G - 1);
      for (int my = 0, m = 0; my < gy; ++my) {
        const double *krow = kern.data() + (size_t)std::abs(my - sy) * gx;
        for (int mx = 0; mx < gx && m + 1 < G; ++mx, ++m) {
          const double k = krow[std::abs(mx - sx)];
          double pm;
          if (pl >= 0.0) pm = (m == src) ? pl : ((1.0 - pl) * k) / total;
          else pm = k / total;
          acc = acc + pm;
          const double f = std::floor(acc * 4294967296.0);
          T[m] = f >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)f;
        }
      }
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int parts = (int)std::min<long long>(std::min<unsigned>(hw, 16u), std::max<long long>(1, (long long)G * G / (1 << 16)));
  if (parts <= 1) {
    rows(0, G);
    return;
  }
  std::vector<std::thread> th;
  for (int q = 0; q < parts; ++q) th.emplace_back(rows, (int)((long long)G * q / parts), (int)((long long)G * (q + 1) / parts));
  for (auto &t : th) t.join();
}

// The table depends on nothing but its size: computed once per process
// (~250k erfc evaluations), then copied.
void gaussian_table(std::vector<float> &ztab) {
  static const std::vector<float> table = [] {
    std::vector<float> z(kZTab);
    for (int i = 0; i < kZTab; ++i) z[i] = (float)inverse_normal_cdf(((double)i + 0.5) / (double)kZTab);
    return z;
  }();
  ztab = table;
}

void build_inputs(const snn_params &p, BuildDev &bd) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      bd.J[a][b] = p.J[a][b];
      bd.sig[a][b] = p.dJ_frac * std::fabs(p.J[a][b]);
    }
  bd.n_delay = (uint32_t)p.n_delay;
  bd.min_delay = (uint32_t)(p.min_delay < 1 ? 1 : p.min_delay);
  bd.p_local_mode = p.p_local >= 0.0f ? 1 : 0;
}

}  // namespace snn

// ---------------------------------------------------------------------------
// network object
// ---------------------------------------------------------------------------
// Device arena of one network, in this order: V, c, ref, the input buffers of
// the next min_delay + 1 steps, the spike counts and spike lists of the last
// n_delay + min_delay steps (everything a run modifies), synapse rows, their
// delay-group table, amplitude table, two windows, two recording blocks
// (header, external-event slots, rate window: one contiguous copy per window),
// two raster entry buffers.  Windows alternate between the two buffer sets, so
// the host drains one window's records while the GPU runs the next.
struct Layout {
  size_t off_V, off_c, off_ref, off_acc, off_cnt, off_hist, off_rows, off_offs, off_amp;
  size_t off_win[2], off_rec[2], off_ext[2], off_rates[2], off_entries[2];
  size_t rec_block;   // bytes of one recording block
  size_t total;
  uint32_t N, N_pad, G, M, M_pad, D, row_bytes, os, kmin, nbuf;
  uint32_t window, rates_bins, rec_cap, n_ext_slots;
};

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int snn_validate_params(const snn_params &p);
static int validate(const snn_params &p) { return snn_validate_params(p); }
int snn_validate_params(const snn_params &p) {
  if (p.gx < 1 || p.gy < 1) return fail(SNN_ERR_ARG, "grid must be at least 1x1");
  if (!(p.lambda > 0.0f) || !std::isfinite(p.lambda)) return fail(SNN_ERR_ARG, "lambda must be > 0");
  if (!std::isfinite(p.p_local) || p.p_local > 1.0f) return fail(SNN_ERR_ARG, "p_local must be <= 1");
  if (p.out_degree < 1) return fail(SNN_ERR_ARG, "out_degree must be >= 1");
  if (p.out_degree > 2048) return fail(SNN_ERR_LIMIT, "out_degree above 2048");
  if (p.n_delay < 1 || p.n_delay > 254) return fail(SNN_ERR_ARG, "n_delay must be in 1..254");
  if (p.min_delay < 0 || p.min_delay > p.n_delay) return fail(SNN_ERR_ARG, "min_delay must be in 0..n_delay");
  if (!(p.dt_ms > 0.0f)) return fail(SNN_ERR_ARG, "dt_ms must be > 0");
  if (p.record_format != SNN_REC_F32 && p.record_format != SNN_REC_I16) return fail(SNN_ERR_ARG, "unknown record_format");
  if (p.bin_steps < 1) return fail(SNN_ERR_ARG, "bin_steps must be >= 1");
  for (int q = 0; q < 3; ++q) {
    if (!(p.tau_m[q] > 0.0f) || !(p.tau_c[q] > 0.0f) || !(p.C_m[q] > 0.0f))
      return fail(SNN_ERR_ARG, "tau_m, tau_c, C_m must be > 0");
    if (p.tau_arp[q] < 0.0f || p.N_ext[q] < 0.0f || p.nu_ext[q] < 0.0f)
      return fail(SNN_ERR_ARG, "tau_arp, N_ext, nu_ext must be >= 0");
    const double narp = std::lround((double)p.tau_arp[q] / (double)p.dt_ms);
    if (narp > 255) return fail(SNN_ERR_LIMIT, "refractory period above 255 steps");
  }
  const uint64_t N = (uint64_t)p.gx * (uint64_t)p.gy * (uint64_t)kK;
  if (N >= (1ull << 24)) return fail(SNN_ERR_LIMIT, "N >= 2^24 neurons (24-bit target index)");
  return SNN_OK;
}

static Layout make_layout(const snn_params &p) {
  Layout L{};
  L.G = (uint32_t)(p.gx * p.gy);
  L.N = L.G * (uint32_t)kK;
  L.N_pad = (uint32_t)align_up(L.N, kNeuronAlign);
  L.M = (uint32_t)p.out_degree;
  L.M_pad = (uint32_t)align_up(L.M, 8);
  L.kmin = (uint32_t)(p.min_delay < 1 ? 1 : p.min_delay);
  L.nbuf = 2u * L.kmin;   // >= kmin + 1; windows of one graph start at the same t0 mod nbuf
  L.D = (uint32_t)p.n_delay + L.kmin;
  L.row_bytes = L.M_pad * 4u + L.M_pad * (p.record_format == SNN_REC_I16 ? 2u : 4u);
  L.os = offs_stride((uint32_t)p.n_delay);
  L.n_ext_slots = L.N_pad / 128u;
  int narp_min = 255;
  for (int q = 0; q < 3; ++q)
    narp_min = std::min(narp_min, (int)std::lround((double)p.tau_arp[q] / (double)p.dt_ms));
  // A neuron fires at most once per narp_min + 1 steps, so a window of W steps
  // holds at most N * ceil(W / (narp_min + 1)) raster entries: size the window
  // so that this bound fits the entry budget, and the raster can never overflow.
  const size_t budget = std::min<size_t>(192ull << 20, std::max<size_t>(8ull << 20, (size_t)L.N * 256u));
  const size_t per_step = (size_t)L.N * 8u / (size_t)(narp_min + 1) + 8u;
  L.window = (uint32_t)std::max<size_t>(16, std::min<size_t>(1024, budget / per_step));
  L.rec_cap = (uint32_t)std::min<uint64_t>(0xFFFFFFF0ull,
                                           (uint64_t)L.N * ((L.window + narp_min) / (narp_min + 1) + 1));
  L.rates_bins = L.window / (uint32_t)p.bin_steps + 2u;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.off_V = take((size_t)L.N_pad * 4);
  L.off_c = take((size_t)L.N_pad * 4);
  L.off_ref = take((size_t)L.N_pad);
  L.off_acc = take((size_t)L.nbuf * L.N_pad * 4);
  L.off_cnt = take((size_t)L.D * 4);
  L.off_hist = take((size_t)L.D * L.N_pad * 4);
  L.off_rows = take((size_t)L.N * L.row_bytes);
  L.off_offs = take((size_t)L.N * L.os * 2);
  L.off_amp = take((size_t)kNPop * kZTab * 4);
  for (int b = 0; b < 2; ++b) L.off_win[b] = take(sizeof(NetWin));
  const size_t ext_at = 256;
  const size_t rates_at = align_up(ext_at + (size_t)L.n_ext_slots * 8, 256);
  L.rec_block = align_up(rates_at + (size_t)L.rates_bins * L.G * 3 * 4, 256);
  for (int b = 0; b < 2; ++b) {
    L.off_rec[b] = take(L.rec_block);
    L.off_ext[b] = L.off_rec[b] + ext_at;
    L.off_rates[b] = L.off_rec[b] + rates_at;
  }
  for (int b = 0; b < 2; ++b) L.off_entries[b] = take((size_t)L.rec_cap * 8);
  L.total = o;
  return L;
}

struct snn_net {
  snn_params p{};
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t cap_stream = nullptr; // private stream used for graph capture
  DevBuf arena;
  Layout L{};
  NetDev hd{};                       // static descriptor (kernel parameter), buffer set 0
  NetWin *pinned_win = nullptr;      // pinned staging of the two windows
  uint8_t *pinned_rec = nullptr;     // pinned copies of the two recording blocks
  unsigned long long *pinned_entries = nullptr;
  size_t pinned_entries_cap = 0;
  cudaStream_t copy_stream = nullptr;   // raster entry copies while the next window runs
  cudaEvent_t ev_block[2] = {nullptr, nullptr};   // recording block b copied to the host
  snn_launch cfg{};
  // window graphs of the two-kernel path, per buffer set and phase of the
  // window's first step (t0 % nbuf, which fixes its input buffers and its
  // position in the exchange period), captured lazily
  std::vector<cudaGraphExec_t> exec[2];
  std::vector<uint32_t> exec_kernels[2];   // kernels launched by each graph
  uint32_t exec_window = 0;
  snn_launch exec_cfg{};
  float exec_l2_ratio = -1.0f;       // hit ratio baked into the captured graphs
  // host records
  uint64_t t = 0;
  std::vector<unsigned long long> raster;   // (step << 32 | id), non-decreasing in step
  size_t raster_sorted = 0;
  std::vector<uint32_t> rates;              // [bin][G][3]
  uint64_t spikes = 0, ext_events = 0;
  double build_ms = 0.0;
  bool broken = false;
  int sm_count = 0;
  uint64_t h2d = 0, d2h = 0, launches = 0;
  bool l2_held = false;                      // holds a reference on the persisting set-aside
};

// ---------------------------------------------------------------------------
// Persisting L2 set-aside of the CUDA context.  While at least one network
// runs with l2_persist, the set-aside is raised to the device maximum; when
// the last such network is freed, persisting lines are reset to normal and the
// limit the context had before is restored.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_l2_mu;
int g_l2_refs = 0;
size_t g_l2_prev = 0;
size_t g_l2_setaside = 0;
}  // namespace

static int l2_acquire(snn_net *h) {
  if (h->l2_held) return SNN_OK;
  std::lock_guard<std::mutex> lk(g_l2_mu);
  if (g_l2_refs == 0) {
    int dev = 0, max_persist = 0;
    CU_TRY(cudaGetDevice(&dev));
    CU_TRY(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev));
    CU_TRY(cudaDeviceGetLimit(&g_l2_prev, cudaLimitPersistingL2CacheSize));
    if ((size_t)max_persist > g_l2_prev) CU_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)max_persist));
    CU_TRY(cudaDeviceGetLimit(&g_l2_setaside, cudaLimitPersistingL2CacheSize));
  }
  ++g_l2_refs;
  h->l2_held = true;
  return SNN_OK;
}

static void l2_release(snn_net *h) {
  if (!h->l2_held) return;
  std::lock_guard<std::mutex> lk(g_l2_mu);
  h->l2_held = false;
  if (--g_l2_refs == 0) {
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_prev);
  }
}

// Bytes of the persisting window at the start of the arena: V, c, ref, the
// input buffers and the spike counts when they fit the set-aside together,
// else V, c and ref alone.  The spike lists (sparse: only the ids of recent
// spikes are touched) are never part of it.
static size_t l2_window_bytes(const snn_net *h) {
  int dev = 0, max_win = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t all = h->L.off_hist, state = h->L.off_acc;
  return std::min<size_t>(all <= g_l2_setaside ? all : state, (size_t)max_win);
}

// The persisting window of network h.  Networks that run at the same time
// keep their full hit ratio: splitting the set-aside between two 24x24
// networks (ratio 0.63 each) was 10% slower than letting their persisting
// lines compete.
static int l2_window(snn_net *h, L2Window *out) {
  *out = L2Window{};
  if (!h->cfg.l2_persist) return SNN_OK;
  int rc = l2_acquire(h);
  if (rc) return rc;
  const size_t bytes = l2_window_bytes(h);
  if (bytes == 0 || g_l2_setaside == 0) return SNN_OK;
  out->base = h->arena.p;
  out->bytes = bytes;
  out->hit_ratio = (float)std::min(1.0, (double)g_l2_setaside / (double)bytes);
  return SNN_OK;
}

static int sm_count_cached() {
  static int v = 0;
  if (!v) v = device_sm_count();
  return v;
}

// Delivery grid: deliver_blocks blocks per SM (every warp takes segments).
static int deliver_grid(const snn_net *h);

static void default_launch(snn_net *h) {
  h->cfg.path = 0;
  h->cfg.update_block = 256;
  h->cfg.deliver_warps = 16;
  h->cfg.fused_block = 128;
  h->cfg.fused_items_per_sm = 8;
  h->cfg.window_steps = (int32_t)h->L.window;
  h->cfg.deliver_lanes = 32;
  h->cfg.update_groups = 1;
  h->cfg.l2_persist = 1;
  h->cfg.deliver_blocks = 3;   // three 16-warp blocks per SM (40 registers)
  h->cfg.overlap = 1;
}

extern "C" int snn_footprint(const snn_params *p, size_t *bytes_out) {
  if (!p || !bytes_out) return fail(SNN_ERR_ARG, "null argument");
  int rc = validate(*p);
  if (rc) return rc;
  *bytes_out = make_layout(*p).total;
  return SNN_OK;
}

static int deliver_grid(const snn_net *h) {
  const int sms = h->sm_count > 0 ? h->sm_count : 148;
  return std::max(1, sms * h->cfg.deliver_blocks);
}

static void free_net(snn_net *h) {
  if (!h) return;
  l2_release(h);
  for (int b = 0; b < 2; ++b) {
    for (auto e : h->exec[b])
      if (e) cudaGraphExecDestroy(e);
    if (h->ev_block[b]) cudaEventDestroy(h->ev_block[b]);
  }
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->pinned_win) cudaFreeHost(h->pinned_win);
  if (h->pinned_rec) cudaFreeHost(h->pinned_rec);
  if (h->pinned_entries) cudaFreeHost(h->pinned_entries);
  h->arena.release();
  delete h;
}

extern "C" void snn_free(snn_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_net(h);
}

static void set_buffers(NetDev &d, const snn_net *h, int b);

static void fill_descriptor(snn_net *h) {
  const Layout &L = h->L;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  NetDev &d = h->hd;
  std::memset(&d, 0, sizeof(d));
  d.N = L.N;
  d.N_pad = L.N_pad;
  d.G = L.G;
  d.gx = (uint32_t)h->p.gx;
  d.M = L.M;
  d.M_pad = L.M_pad;
  d.D = L.D;
  d.fmt = (uint32_t)h->p.record_format;
  d.row_bytes = L.row_bytes;
  d.bin_steps = (uint32_t)h->p.bin_steps;
  d.key0 = (uint32_t)(h->seed & 0xFFFFFFFFu);
  d.key1 = (uint32_t)(h->seed >> 32);
  d.slot = 0;
  d.rec_cap = L.rec_cap;
  d.rates_bins = L.rates_bins;
  d.n_delay = (uint32_t)h->p.n_delay;
  d.os = L.os;
  d.kmin = L.kmin;
  d.nbuf = L.nbuf;
  for (int q = 0; q < 3; ++q) {
    const PopTables t = pop_tables(h->p, q);
    d.pvv[q] = t.pvv;
    d.pvc[q] = t.pvc;
    d.pcc[q] = t.pcc;
    d.el[q] = h->p.E_L[q];
    d.vth[q] = h->p.V_th[q];
    d.vr[q] = h->p.V_r[q];
    d.alpha[q] = h->p.alpha_c[q];
    d.narp[q] = t.narp;
    for (int k = 0; k < kPoisMax; ++k) d.thr[q][k] = (uint32_t)t.thr[k];   // <= 2^20
  }
  d.V = reinterpret_cast<float *>(base + L.off_V);
  d.c = reinterpret_cast<float *>(base + L.off_c);
  d.ref = base + L.off_ref;
  d.acc = reinterpret_cast<int32_t *>(base + L.off_acc);
  d.cnt = reinterpret_cast<uint32_t *>(base + L.off_cnt);
  d.hist = reinterpret_cast<uint32_t *>(base + L.off_hist);
  d.rows = base + L.off_rows;
  d.offs = reinterpret_cast<const uint16_t *>(base + L.off_offs);
  d.amp = reinterpret_cast<const int32_t *>(base + L.off_amp);
  set_buffers(d, h, 0);
}

// The descriptor of buffer set b: same network, window and recording of set b.
static void set_buffers(NetDev &d, const snn_net *h, int b) {
  const Layout &L = h->L;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  d.win = reinterpret_cast<const NetWin *>(base + L.off_win[b]);
  d.rec = reinterpret_cast<RecHeader *>(base + L.off_rec[b]);
  d.ext_acc = reinterpret_cast<unsigned long long *>(base + L.off_ext[b]);
  d.rates = reinterpret_cast<uint32_t *>(base + L.off_rates[b]);
  d.rec_entries = reinterpret_cast<unsigned long long *>(base + L.off_entries[b]);
}

static NetDev descriptor(const snn_net *h, int b) {
  NetDev d = h->hd;
  set_buffers(d, h, b);
  return d;
}

extern "C" int snn_build_network(const snn_params *p, uint64_t seed, void *cuda_stream, snn_handle *out) {
  if (!p || !out) return fail(SNN_ERR_ARG, "null argument");
  *out = nullptr;
  int rc = validate(*p);
  if (rc) return rc;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(SNN_ERR_CUDA, "no CUDA device available");
  }
  const auto t_start = std::chrono::steady_clock::now();
  std::unique_ptr<snn_net, void (*)(snn_net *)> h(new snn_net(), free_net);
  h->p = *p;
  h->seed = seed;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->L = make_layout(*p);
  h->sm_count = sm_count_cached();
  CU_TRY(prepare_kernels());
  CU_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CU_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b) CU_TRY(cudaEventCreateWithFlags(&h->ev_block[b], cudaEventDisableTiming));
  rc = dev_alloc(h->arena, h->L.total);
  if (rc) return rc;
  fill_descriptor(h.get());
  default_launch(h.get());
  const Layout &L = h->L;
  cudaStream_t s = h->stream;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);

  // tables for construction and the external drive
  std::vector<float> ztab;
  gaussian_table(ztab);
  std::vector<int32_t> amp((size_t)kNPop * kZTab);
  for (int q = 0; q < 3; ++q) {
    const float sig = p->dJ_ext_frac * std::fabs(p->J_ext[q]);
    for (int i = 0; i < kZTab; ++i) {
      const float spread = sig * ztab[i];
      const float w = sign_kept(p->J_ext[q] + spread, p->J_ext[q]);
      amp[(size_t)q * kZTab + i] = (int32_t)std::lrintf(w * 65536.0f);
    }
  }
  std::vector<uint32_t> cdf;
  module_thresholds(*p, cdf);
  BuildDev bd{};
  build_inputs(*p, bd);
  DevBuf tmp;
  const size_t cdf_bytes = std::max<size_t>(cdf.size() * 4, 16);
  rc = dev_alloc(tmp, align_up(cdf_bytes, 256) + kZTab * 4);
  if (rc) return rc;
  struct TmpGuard {
    DevBuf *b;
    cudaStream_t s;
    ~TmpGuard() {
      cudaStreamSynchronize(s);
      b->release();
    }
  } guard{&tmp, s};
  uint32_t *d_cdf = static_cast<uint32_t *>(tmp.p);
  float *d_z = reinterpret_cast<float *>(static_cast<uint8_t *>(tmp.p) + align_up(cdf_bytes, 256));
  if (!cdf.empty()) CU_TRY(cudaMemcpyAsync(d_cdf, cdf.data(), cdf.size() * 4, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemcpyAsync(d_z, ztab.data(), kZTab * 4, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemcpyAsync(base + L.off_amp, amp.data(), amp.size() * 4, cudaMemcpyHostToDevice, s));
  h->h2d += cdf.size() * 4 + kZTab * 4 + amp.size() * 4;
  h->launches += 2;
  bd.cdf = d_cdf;
  bd.ztab = d_z;
  CU_TRY(cudaMemsetAsync(base + L.off_acc, 0, L.off_hist - L.off_acc, s));   // inputs, spike counts
  CU_TRY(cudaMemsetAsync(base + L.off_win[0], 0, L.off_entries[0] - L.off_win[0], s));   // windows, blocks
  CU_TRY(cudaMallocHost(&h->pinned_win, 2 * sizeof(NetWin)));
  std::memset(h->pinned_win, 0, 2 * sizeof(NetWin));
  CU_TRY(launch_build_rows(h->hd, bd, s));
  CU_TRY(launch_init_state(h->hd, s));
  CU_TRY(cudaMallocHost(&h->pinned_rec, 2 * L.rec_block));
  CU_TRY(cudaStreamSynchronize(s));
  h->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  *out = h.release();
  return SNN_OK;
}

// ---------------------------------------------------------------------------
// windows of steps
// ---------------------------------------------------------------------------
// Window of steps [t0, t_end) as the kernels read it.
static void set_window(const snn_net *h, NetWin *w, uint64_t t0, uint64_t t_end) {
  std::memset(w, 0, sizeof(NetWin));
  w->t0 = (uint32_t)t0;
  w->t_end = (uint32_t)t_end;
  w->bin0 = (uint32_t)(t0 / (uint64_t)h->p.bin_steps);
  w->t0_slot = (uint32_t)(t0 % h->L.D);
}

// Drop the cached window graphs unless they were captured for this window
// length, launch shape and L2 window.
static int prepare_graphs(snn_net *h, uint32_t window) {
  L2Window l2;   // set-aside changes are not allowed while a capture is open
  int rc = l2_window(h, &l2);
  if (rc) return rc;
  if (h->exec_window == window && h->exec_l2_ratio == l2.hit_ratio &&
      std::memcmp(&h->exec_cfg, &h->cfg, sizeof(snn_launch)) == 0 && h->exec[0].size() == h->L.nbuf)
    return SNN_OK;
  for (int b = 0; b < 2; ++b) {
    for (auto e : h->exec[b])
      if (e) cudaGraphExecDestroy(e);
    h->exec[b].assign(h->L.nbuf, nullptr);
    h->exec_kernels[b].assign(h->L.nbuf, 0u);
  }
  h->exec_window = window;
  h->exec_cfg = h->cfg;
  h->exec_l2_ratio = l2.hit_ratio;
  return SNN_OK;
}

// Capture the steps k = 0..steps-1 of a window starting at a step with
// phase = t0 % nbuf: the update of every step, the delivery pass after every
// step t with (t + 1) % kmin == 0.  With `ev`, event record nodes bracket every
// kernel (ev[4k..4k+3]: update start/end, delivery start/end) and the kernels
// do not overlap.
static int capture_steps(snn_net *h, const NetDev &d, uint32_t steps, uint32_t phase, const L2Window &l2,
                         cudaEvent_t *ev, cudaGraphExec_t *out, uint32_t *kernels) {
  const snn_launch &c = h->cfg;
  cudaStream_t cs = h->cap_stream;
  CU_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  uint32_t n = 0;
  // programmatic dependent launch between an update and the delivery pass
  // after it and between a pass and the next update, unless event nodes
  // separate the kernels (each kernel timed alone); an update that follows an
  // update (inside an exchange period) waits for it to finish
  const bool pdl = c.overlap && !ev;
  for (uint32_t k = 0; k < steps && err == cudaSuccess; ++k) {
    if (ev) err = cudaEventRecordWithFlags(ev[4 * k + 0], cs, cudaEventRecordExternal);
    const bool after_pass = k > 0 && (phase + k) % h->L.kmin == 0u;   // a pass follows step t0 + k - 1
    const bool pdl_u = pdl && after_pass;
    const StepMod km{k % h->L.D, (phase + k) % h->L.nbuf, pdl_u ? 1u : 0u};
    if (err == cudaSuccess) err = launch_update(d, k, km, c.update_block, c.update_groups, l2, pdl_u, cs);
    ++n;
    if (ev && err == cudaSuccess) err = cudaEventRecordWithFlags(ev[4 * k + 1], cs, cudaEventRecordExternal);
    if ((phase + k + 1u) % h->L.kmin == 0u) {
      if (ev && err == cudaSuccess) err = cudaEventRecordWithFlags(ev[4 * k + 2], cs, cudaEventRecordExternal);
      if (err == cudaSuccess)
        err = launch_deliver(d, k, km, (uint32_t)c.deliver_lanes, c.deliver_warps, deliver_grid(h), l2, pdl, cs);
      ++n;
      if (ev && err == cudaSuccess) err = cudaEventRecordWithFlags(ev[4 * k + 3], cs, cudaEventRecordExternal);
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(SNN_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(err != cudaSuccess ? err : e2));
  }
  cudaError_t e3 = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) return fail(SNN_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
  if (kernels) *kernels = n;
  return SNN_OK;
}

// The window graph of buffer set b for windows starting at phase `phase`.
static int window_graph(snn_net *h, int b, uint32_t phase, cudaGraphExec_t *out, uint32_t *kernels) {
  if (!h->exec[b][phase]) {
    L2Window l2;
    int rc = l2_window(h, &l2);
    if (rc) return rc;
    rc = capture_steps(h, descriptor(h, b), h->exec_window, phase, l2, nullptr, &h->exec[b][phase],
                       &h->exec_kernels[b][phase]);
    if (rc) return rc;
  }
  *out = h->exec[b][phase];
  *kernels = h->exec_kernels[b][phase];
  return SNN_OK;
}

// Draining a finished window's records of buffer set b: (1) copy the recording
// block (header, external-event slots, rates) to pinned memory, enqueued right
// behind the window's kernels, with an event; (2) once that event completes,
// check the status and copy the raster entries (side stream); (3) append them
// on the host and reset the device block on the run stream, ahead of the
// window that reuses the set.
static uint8_t *pinned_block(snn_net *h, int b) { return h->pinned_rec + (size_t)b * h->L.rec_block; }

static int drain_copy_block(snn_net *h, int b, cudaStream_t s) {
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  CU_TRY(cudaMemcpyAsync(pinned_block(h, b), base + h->L.off_rec[b], h->L.rec_block, cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaEventRecord(h->ev_block[b], s));
  h->d2h += h->L.rec_block;
  return SNN_OK;
}

static int drain_copy_entries(snn_net *h, int b, cudaStream_t s, uint32_t *n_out) {
  const Layout &L = h->L;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  const RecHeader *rh = reinterpret_cast<const RecHeader *>(pinned_block(h, b));
  *n_out = 0;
  if (rh->status & kStatusRasterOverflow) {
    h->broken = true;
    return fail(SNN_ERR_LIMIT, "spike record window overflowed");
  }
  const uint32_t n_rec = std::min(rh->cursor, L.rec_cap);
  if (n_rec) {
    if (h->pinned_entries_cap < n_rec) {
      if (h->pinned_entries) cudaFreeHost(h->pinned_entries);
      h->pinned_entries = nullptr;
      size_t cap = std::max<size_t>(n_rec, h->pinned_entries_cap * 2);
      cap = std::min<size_t>(cap, L.rec_cap);
      CU_TRY(cudaMallocHost(&h->pinned_entries, cap * 8));
      h->pinned_entries_cap = cap;
    }
    CU_TRY(cudaMemcpyAsync(h->pinned_entries, base + L.off_entries[b], (size_t)n_rec * 8, cudaMemcpyDeviceToHost, s));
    h->d2h += (uint64_t)n_rec * 8;
  }
  *n_out = n_rec;
  return SNN_OK;
}

static int drain_absorb(snn_net *h, int b, uint64_t t0, uint32_t n_rec, cudaStream_t run_stream) {
  const Layout &L = h->L;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  const uint8_t *blk = pinned_block(h, b);
  h->spikes += n_rec;
  const unsigned long long *ext = reinterpret_cast<const unsigned long long *>(blk + (L.off_ext[b] - L.off_rec[b]));
  for (uint32_t i = 0; i < L.n_ext_slots; ++i) h->ext_events += ext[i];
  if (n_rec) {
    const size_t old = h->raster.size();
    h->raster.resize(old + n_rec);
    for (uint32_t i = 0; i < n_rec; ++i) {
      const unsigned long long e = h->pinned_entries[i];
      const uint64_t k = (e >> 32) & 0xFFFFu;
      h->raster[old + i] = ((t0 + k) << 32) | (e & 0xFFFFFFFFull);
    }
  }
  // rates of the window, bins from t0 / bin_steps
  const uint32_t *rw = reinterpret_cast<const uint32_t *>(blk + (L.off_rates[b] - L.off_rec[b]));
  const uint64_t bin0 = t0 / (uint64_t)h->p.bin_steps;
  const size_t per_bin = (size_t)L.G * 3;
  const size_t need = (size_t)(bin0 + L.rates_bins) * per_bin;
  if (h->rates.size() < need) h->rates.resize(need, 0u);
  for (size_t i = 0; i < (size_t)L.rates_bins * per_bin; ++i) h->rates[bin0 * per_bin + i] += rw[i];
  CU_TRY(cudaMemsetAsync(base + L.off_rec[b], 0, L.rec_block, run_stream));
  return SNN_OK;
}

// Wait for buffer set b's block copy, then fetch and absorb its entries.
static int drain_finish(snn_net *h, int b, uint64_t t0, cudaStream_t run_stream) {
  CU_TRY(cudaEventSynchronize(h->ev_block[b]));
  uint32_t n_rec = 0;
  int rc = drain_copy_entries(h, b, h->copy_stream, &n_rec);
  if (rc) return rc;
  if (n_rec) CU_TRY(cudaStreamSynchronize(h->copy_stream));
  return drain_absorb(h, b, t0, n_rec, run_stream);
}

// Copy a finished window's records of buffer set b to host memory and reset them.
static int drain_window(snn_net *h, int b, uint64_t t0, cudaStream_t s) {
  int rc = drain_copy_block(h, b, s);
  if (rc) return rc;
  return drain_finish(h, b, t0, s);
}

// The same for every network of a batch, with two host waits in total.
static int drain_batch(snn_net *const *hs, int b, const uint64_t *t0s, const uint64_t *adv, int32_t n,
                       cudaEvent_t block_done, cudaStream_t copy_stream, cudaStream_t run_stream) {
  CU_TRY(cudaEventSynchronize(block_done));
  std::vector<uint32_t> n_rec(n, 0);
  bool any = false;
  int first_err = SNN_OK;
  for (int i = 0; i < n; ++i)
    if (adv[i]) {
      int rc = drain_copy_entries(hs[i], b, copy_stream, &n_rec[i]);
      if (rc && first_err == SNN_OK) first_err = rc;
      any |= n_rec[i] != 0;
    }
  if (any) CU_TRY(cudaStreamSynchronize(copy_stream));
  if (first_err) return first_err;
  for (int i = 0; i < n; ++i)
    if (adv[i]) {
      int rc = drain_absorb(hs[i], b, t0s[i], n_rec[i], run_stream);
      if (rc) return rc;
    }
  return SNN_OK;
}

// Windows of one network on the two-kernel path.  They alternate between the
// two buffer sets; up to two are in flight, and the host drains the older one
// while the GPU runs the newer.
struct PlainRunner {
  struct Pending {
    int b;
    uint64_t t0, n;
  };
  snn_net *h = nullptr;
  uint32_t window = 0;
  uint64_t steps = 0, issued = 0, t_issue = 0;
  Pending q[2];
  int nq = 0, next_b = 0;
  bool can_issue() const { return issued < steps && nq < 2; }
  bool busy() const { return issued < steps || nq > 0; }
};

static uint32_t plain_window(const snn_net *h) {
  return (uint32_t)std::max(1, std::min<int32_t>(h->cfg.window_steps, (int32_t)h->L.window));
}

static int runner_issue(PlainRunner &r) {
  snn_net *h = r.h;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  const uint64_t t0 = r.t_issue;
  const uint64_t n = std::min<uint64_t>(r.window, r.steps - r.issued);
  if (t0 + n > 0xFFFFFFFFull) return fail(SNN_ERR_LIMIT, "step counter beyond 2^32");
  const int b = r.next_b;
  NetWin *pw = h->pinned_win + b;   // free: the copy of its last use finished before that drain
  set_window(h, pw, t0, t0 + n);
  cudaGraphExec_t gx = nullptr;
  uint32_t kernels = 0;
  int rc = window_graph(h, b, (uint32_t)(t0 % h->L.nbuf), &gx, &kernels);
  if (rc) return rc;
  CU_TRY(cudaMemcpyAsync(base + h->L.off_win[b], pw, sizeof(NetWin), cudaMemcpyHostToDevice, h->stream));
  CU_TRY(cudaGraphLaunch(gx, h->stream));
  h->h2d += sizeof(NetWin);
  h->launches += kernels;
  rc = drain_copy_block(h, b, h->stream);
  if (rc) return rc;
  r.q[r.nq++] = PlainRunner::Pending{b, t0, n};
  r.next_b ^= 1;
  r.issued += n;
  r.t_issue += n;
  return SNN_OK;
}

static int runner_drain(PlainRunner &r) {
  const PlainRunner::Pending p = r.q[0];
  r.q[0] = r.q[1];
  --r.nq;
  int rc = drain_finish(r.h, p.b, p.t0, r.h->stream);
  if (rc == SNN_OK) r.h->t = p.t0 + p.n;
  return rc;
}

static int run_plain(snn_net *h, uint64_t steps) {
  PlainRunner r;
  r.h = h;
  r.window = plain_window(h);
  r.steps = steps;
  r.t_issue = h->t;
  int rc = prepare_graphs(h, r.window);
  if (rc) return rc;
  int status = SNN_OK;
  while (status == SNN_OK && r.busy()) status = r.can_issue() ? runner_issue(r) : runner_drain(r);
  if (status != SNN_OK) cudaStreamSynchronize(h->stream);   // nothing left in flight
  return status;
}

// Several networks on the two-kernel path, each on its own stream: their
// windows are issued and drained round robin from this thread, so the kernels
// of different networks overlap on the GPU.
static int run_plain_many(snn_net *const *hs, const uint64_t *steps, int32_t n) {
  std::vector<PlainRunner> rs((size_t)n);
  for (int i = 0; i < n; ++i) {
    rs[i].h = hs[i];
    rs[i].window = plain_window(hs[i]);
    rs[i].steps = steps[i];
    rs[i].t_issue = hs[i]->t;
    if (steps[i]) {
      int rc = prepare_graphs(hs[i], rs[i].window);
      if (rc) return rc;
    }
  }
  int status = SNN_OK;
  bool any = true;
  while (status == SNN_OK && any) {
    any = false;
    for (int i = 0; i < n && status == SNN_OK; ++i)
      while (status == SNN_OK && rs[i].can_issue()) status = runner_issue(rs[i]);
    for (int i = 0; i < n && status == SNN_OK; ++i)
      if (rs[i].nq > 0) status = runner_drain(rs[i]);
    for (int i = 0; i < n; ++i) any |= rs[i].busy();
  }
  if (status != SNN_OK)
    for (int i = 0; i < n; ++i) cudaStreamSynchronize(hs[i]->stream);
  return status;
}

// ---------------------------------------------------------------------------
// fused path over a set of networks
// ---------------------------------------------------------------------------
struct BatchCtx {
  DevBuf nets[2];              // NetDev[cap] per buffer set
  DevBuf wins[2];              // NetWin[cap] per buffer set
  DevBuf items;                // FusedItem[item_cap]
  DevBuf n_items_dev;          // u32 item count read by the kernel
  size_t cap = 0, item_cap = 0;
  NetDev *pinned_nets = nullptr;   // [2][cap]
  NetWin *pinned_wins = nullptr;   // [2][cap]
  FusedItem *pinned_items = nullptr;
  cudaStream_t cap_stream = nullptr, copy_stream = nullptr;
  cudaEvent_t ev_block[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  uint32_t exec_window = 0, exec_items = 0, exec_lanes = 0, exec_chunks = 0;
  uint32_t pinned_count = 0;   // staging of the item count (copied before the replays)
  int exec_block = 0, exec_blocks = 0;
  void drop_graphs() {
    for (auto &e : exec)
      if (e) {
        cudaGraphExecDestroy(e);
        e = nullptr;
      }
  }
  ~BatchCtx() {
    drop_graphs();
    for (auto e : ev_block)
      if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (pinned_nets) cudaFreeHost(pinned_nets);
    if (pinned_wins) cudaFreeHost(pinned_wins);
    if (pinned_items) cudaFreeHost(pinned_items);
    for (int b = 0; b < 2; ++b) {
      nets[b].release();
      wins[b].release();
    }
    items.release();
    n_items_dev.release();
  }
};
static thread_local std::unique_ptr<BatchCtx> g_batch;

static int run_fused(snn_net *const *hs, const uint64_t *steps, int32_t n) {
  if (!g_batch) g_batch.reset(new BatchCtx());
  BatchCtx &B = *g_batch;
  const snn_launch &cfg = hs[0]->cfg;
  const int block = cfg.fused_block;
  const uint32_t npi = 4u * (uint32_t)block;
  const uint32_t lanes = (uint32_t)cfg.deliver_lanes;
  size_t n_items = 0;
  uint32_t window = 0xFFFFFFFFu;
  for (int i = 0; i < n; ++i) {
    n_items += (hs[i]->L.N_pad + npi - 1) / npi;
    window = std::min<uint32_t>(window, hs[i]->L.window);
  }
  window = std::max<uint32_t>(1, std::min<uint32_t>(window, (uint32_t)std::max(1, cfg.window_steps)));
  if ((size_t)n > B.cap) {
    for (int b = 0; b < 2; ++b) {
      B.nets[b].release();
      B.wins[b].release();
    }
    if (B.pinned_nets) cudaFreeHost(B.pinned_nets);
    if (B.pinned_wins) cudaFreeHost(B.pinned_wins);
    B.pinned_nets = nullptr;
    B.pinned_wins = nullptr;
    const size_t cap = std::max<size_t>((size_t)n, 2 * B.cap);
    B.cap = 0;
    B.drop_graphs();
    for (int b = 0; b < 2; ++b) {
      int rc = dev_alloc(B.nets[b], cap * sizeof(NetDev));
      if (rc) return rc;
      rc = dev_alloc(B.wins[b], cap * sizeof(NetWin));
      if (rc) return rc;
    }
    CU_TRY(cudaMallocHost(&B.pinned_nets, 2 * cap * sizeof(NetDev)));
    CU_TRY(cudaMallocHost(&B.pinned_wins, 2 * cap * sizeof(NetWin)));
    B.cap = cap;
  }
  if (n_items > B.item_cap) {
    B.items.release();
    if (B.pinned_items) cudaFreeHost(B.pinned_items);
    B.pinned_items = nullptr;
    const size_t cap = std::max<size_t>(n_items, 2 * B.item_cap);
    B.item_cap = 0;
    B.drop_graphs();
    int rc = dev_alloc(B.items, cap * sizeof(FusedItem));
    if (rc) return rc;
    CU_TRY(cudaMallocHost(&B.pinned_items, cap * sizeof(FusedItem)));
    B.item_cap = cap;
  }
  if (!B.cap_stream) CU_TRY(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking));
  if (!B.copy_stream) CU_TRY(cudaStreamCreateWithFlags(&B.copy_stream, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b)
    if (!B.ev_block[b]) CU_TRY(cudaEventCreateWithFlags(&B.ev_block[b], cudaEventDisableTiming));
  if (!B.n_items_dev.p) {
    int rc = dev_alloc(B.n_items_dev, 256);
    if (rc) return rc;
  }
  cudaStream_t s = hs[0]->stream;
  // all networks of the batch are ordered on the first network's stream
  for (int i = 0; i < n; ++i)
    if (hs[i]->stream != s) CU_TRY(cudaStreamSynchronize(hs[i]->stream));
  size_t it = 0;
  for (int i = 0; i < n; ++i) {
    // items of network i: consecutive neuron ranges, each knowing its index
    // among the network's items (its share of the network's delivery)
    const uint32_t I = (hs[i]->L.N_pad + npi - 1) / npi;
    for (uint32_t j = 0; j < I; ++j) B.pinned_items[it++] = FusedItem{(uint32_t)i, j * npi, j, I};
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < n; ++i) {
      NetDev d = descriptor(hs[i], b);
      d.slot = (uint32_t)i;
      d.win = static_cast<const NetWin *>(B.wins[b].p) + i;
      B.pinned_nets[(size_t)b * B.cap + i] = d;
    }
  uint32_t max_delay = 1;
  for (int i = 0; i < n; ++i) max_delay = std::max<uint32_t>(max_delay, (uint32_t)hs[i]->p.n_delay);
  const uint32_t chunks = pre_chunks(max_delay);   // delay chunks of the largest delay in the batch
  const int sms = hs[0]->sm_count > 0 ? hs[0]->sm_count : 148;
  const int per_sm = std::min(cfg.fused_items_per_sm, fused_blocks_per_sm(block, chunks));
  const int blocks = sms * per_sm;   // fixed grid: the same graphs serve any set of networks
  if (!B.exec[0] || !B.exec[1] || B.exec_window != window || B.exec_block != block || B.exec_blocks != blocks ||
      B.exec_lanes != lanes || B.exec_chunks != chunks) {
    B.drop_graphs();
    for (int b = 0; b < 2; ++b) {
      FusedTable tab{static_cast<const NetDev *>(B.nets[b].p), static_cast<const FusedItem *>(B.items.p),
                     static_cast<const uint32_t *>(B.n_items_dev.p), lanes, chunks};
      CU_TRY(cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t err = cudaSuccess;
      for (uint32_t k = 0; k < window && err == cudaSuccess; ++k)
        err = launch_fused(tab, k, block, blocks, B.cap_stream);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(B.cap_stream, &g);
      if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(SNN_ERR_CUDA, std::string("fused launch during capture: ") + cudaGetErrorString(err));
      }
      if (e2 != cudaSuccess) return fail(SNN_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e2));
      cudaError_t e3 = cudaGraphInstantiate(&B.exec[b], g, 0);
      cudaGraphDestroy(g);
      if (e3 != cudaSuccess) return fail(SNN_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
    }
    B.exec_window = window;
    B.exec_items = (uint32_t)n_items;
    B.exec_block = block;
    B.exec_blocks = blocks;
    B.exec_lanes = lanes;
    B.exec_chunks = chunks;
  }
  CU_TRY(cudaMemcpyAsync(B.items.p, B.pinned_items, n_items * sizeof(FusedItem), cudaMemcpyHostToDevice, s));
  B.pinned_count = (uint32_t)n_items;
  CU_TRY(cudaMemcpyAsync(B.n_items_dev.p, &B.pinned_count, 4, cudaMemcpyHostToDevice, s));
  for (int b = 0; b < 2; ++b)
    CU_TRY(cudaMemcpyAsync(B.nets[b].p, B.pinned_nets + (size_t)b * B.cap, (size_t)n * sizeof(NetDev),
                           cudaMemcpyHostToDevice, s));
  for (int i = 0; i < n; ++i) hs[i]->h2d += 2 * sizeof(NetDev);

  // windows alternate between the two buffer sets, two in flight at most
  struct Pending {
    int b;
    std::vector<uint64_t> t0s, adv;
  };
  Pending q[2];
  int nq = 0, next_b = 0;
  std::vector<uint64_t> left(steps, steps + n), t_issue(n);
  for (int i = 0; i < n; ++i) t_issue[i] = hs[i]->t;
  int status = SNN_OK;
  while (status == SNN_OK) {
    uint64_t most = 0;
    for (int i = 0; i < n; ++i) most = std::max(most, left[i]);
    if (most > 0 && nq < 2) {
      const int b = next_b;
      NetWin *pw = B.pinned_wins + (size_t)b * B.cap;
      Pending p{b, std::vector<uint64_t>(n), std::vector<uint64_t>(n)};
      for (int i = 0; i < n; ++i) {
        const uint64_t adv = std::min<uint64_t>(window, left[i]);
        if (t_issue[i] + adv > 0xFFFFFFFFull) {
          status = fail(SNN_ERR_LIMIT, "step counter beyond 2^32");
          break;
        }
        set_window(hs[i], pw + i, t_issue[i], t_issue[i] + adv);
        p.t0s[i] = t_issue[i];
        p.adv[i] = adv;
      }
      if (status != SNN_OK) break;
      CU_TRY(cudaMemcpyAsync(B.wins[b].p, pw, (size_t)n * sizeof(NetWin), cudaMemcpyHostToDevice, s));
      CU_TRY(cudaGraphLaunch(B.exec[b], s));
      hs[0]->launches += window;   // one fused kernel per step for the whole batch
      for (int i = 0; i < n; ++i) {
        hs[i]->h2d += sizeof(NetWin);
        if (p.adv[i]) {
          int rc = drain_copy_block(hs[i], b, s);
          if (rc) return rc;
        }
        t_issue[i] += p.adv[i];
        left[i] -= p.adv[i];
      }
      CU_TRY(cudaEventRecord(B.ev_block[b], s));
      q[nq++] = std::move(p);
      next_b ^= 1;
      continue;
    }
    if (nq == 0) break;
    Pending p = std::move(q[0]);
    q[0] = std::move(q[1]);
    --nq;
    status = drain_batch(hs, p.b, p.t0s.data(), p.adv.data(), n, B.ev_block[p.b], B.copy_stream, s);
    if (status == SNN_OK)
      for (int i = 0; i < n; ++i) hs[i]->t = p.t0s[i] + p.adv[i];
  }
  if (status != SNN_OK) cudaStreamSynchronize(s);
  return status;
}

// ---------------------------------------------------------------------------
// public run calls
// ---------------------------------------------------------------------------
extern "C" int snn_run(snn_handle h, uint64_t steps) {
  if (!h) return fail(SNN_ERR_ARG, "null handle");
  if (h->broken) return fail(SNN_ERR_STATE, "network is invalid after an earlier failure");
  if (steps == 0) return SNN_OK;
  if (h->cfg.path == 1) {
    snn_net *one[1] = {h};
    return run_fused(one, &steps, 1);
  }
  return run_plain(h, steps);
}

extern "C" int snn_run_batch(const snn_handle *hs, const uint64_t *steps, int32_t n) {
  if (!hs || !steps || n < 1) return fail(SNN_ERR_ARG, "empty batch");
  if (n > 65535) return fail(SNN_ERR_LIMIT, "more than 65535 networks in one batch");
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(SNN_ERR_ARG, "null handle in batch");
    if (hs[i]->broken) return fail(SNN_ERR_STATE, "network is invalid after an earlier failure");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(SNN_ERR_ARG, "a network appears twice in the batch");
  }
  return run_fused(hs, steps, n);
}

extern "C" int snn_run_concurrent(const snn_handle *hs, const uint64_t *steps, int32_t n) {
  if (!hs || !steps || n < 1) return fail(SNN_ERR_ARG, "no networks");
  if (n > 1024) return fail(SNN_ERR_LIMIT, "more than 1024 networks in one call");
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(SNN_ERR_ARG, "null handle");
    if (hs[i]->broken) return fail(SNN_ERR_STATE, "network is invalid after an earlier failure");
    if (hs[i]->cfg.path != 0) return fail(SNN_ERR_ARG, "snn_run_concurrent runs the two-kernel path (launch path 0)");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(SNN_ERR_ARG, "a network appears twice");
  }
  return run_plain_many(hs, steps, n);
}

// ---------------------------------------------------------------------------
// reads
// ---------------------------------------------------------------------------
extern "C" int snn_read_spikes(snn_handle h, uint64_t t0, uint64_t t1, uint32_t *step_out, uint32_t *id_out,
                               size_t cap, size_t *n_out) {
  if (!h || !n_out) return fail(SNN_ERR_ARG, "null argument");
  if (h->raster_sorted < h->raster.size()) {
    // records are appended window by window, so only the new tail needs ordering
    order_raster(h->raster, h->raster_sorted);
    h->raster_sorted = h->raster.size();
  }
  auto a = t0 > 0xFFFFFFFFull ? h->raster.end()
                              : std::lower_bound(h->raster.begin(), h->raster.end(), (unsigned long long)(t0 << 32));
  auto b = t1 > 0xFFFFFFFFull ? h->raster.end()
                              : std::lower_bound(a, h->raster.end(), (unsigned long long)(t1 << 32));
  if (t1 <= t0) b = a;
  const size_t n = (size_t)(b - a);
  *n_out = n;
  if (n > cap) return fail(SNN_ERR_BUFFER, "spike buffer too small");
  if (n && (!step_out || !id_out)) return fail(SNN_ERR_ARG, "null output buffer");
  if (n) split_raster(&*a, n, step_out, id_out);
  return SNN_OK;
}

extern "C" int snn_rates(snn_handle h, uint32_t *counts_out, size_t cap, size_t *n_out) {
  if (!h || !n_out) return fail(SNN_ERR_ARG, "null argument");
  const size_t per_bin = (size_t)h->L.G * 3;
  const uint64_t bins = (h->t + (uint64_t)h->p.bin_steps - 1) / (uint64_t)h->p.bin_steps;
  const size_t n = (size_t)bins * per_bin;
  *n_out = n;
  if (n > cap) return fail(SNN_ERR_BUFFER, "rate buffer too small");
  if (n && !counts_out) return fail(SNN_ERR_ARG, "null output buffer");
  for (size_t i = 0; i < n; ++i) counts_out[i] = i < h->rates.size() ? h->rates[i] : 0u;
  return SNN_OK;
}

extern "C" int snn_read_state(snn_handle h, float *V_out, float *c_out, int32_t *ref_out, size_t n) {
  if (!h) return fail(SNN_ERR_ARG, "null handle");
  const uint32_t N = h->L.N;
  if (n < N) return fail(SNN_ERR_BUFFER, "state buffers shorter than N");
  std::vector<uint8_t> ref(N);
  if (V_out) CU_TRY(cudaMemcpyAsync(V_out, h->hd.V, (size_t)N * 4, cudaMemcpyDeviceToHost, h->stream));
  if (c_out) CU_TRY(cudaMemcpyAsync(c_out, h->hd.c, (size_t)N * 4, cudaMemcpyDeviceToHost, h->stream));
  CU_TRY(cudaMemcpyAsync(ref.data(), h->hd.ref, N, cudaMemcpyDeviceToHost, h->stream));
  CU_TRY(cudaStreamSynchronize(h->stream));
  if (ref_out)
    for (uint32_t i = 0; i < N; ++i) ref_out[i] = ref[i];
  return SNN_OK;
}

extern "C" int snn_read_row(snn_handle h, uint32_t s, uint32_t *keys_out, float *w_out, size_t cap) {
  if (!h) return fail(SNN_ERR_ARG, "null handle");
  if (s >= h->L.N) return fail(SNN_ERR_ARG, "source index out of range");
  if (cap < h->L.M) return fail(SNN_ERR_BUFFER, "row buffers shorter than M");
  std::vector<uint8_t> row(h->L.row_bytes);
  CU_TRY(cudaMemcpyAsync(row.data(), h->hd.rows + (size_t)s * h->L.row_bytes, h->L.row_bytes,
                         cudaMemcpyDeviceToHost, h->stream));
  CU_TRY(cudaStreamSynchronize(h->stream));
  const uint32_t M = h->L.M, Mp = h->L.M_pad;
  if (keys_out) std::memcpy(keys_out, row.data(), (size_t)M * 4);
  if (w_out) {
    if (h->p.record_format == SNN_REC_I16) {
      const int16_t *q = reinterpret_cast<const int16_t *>(row.data() + (size_t)Mp * 4);
      for (uint32_t j = 0; j < M; ++j) w_out[j] = (float)q[j] * (1.0f / 1024.0f);
    } else {
      std::memcpy(w_out, row.data() + (size_t)Mp * 4, (size_t)M * 4);
    }
  }
  return SNN_OK;
}

extern "C" int snn_get_stats(snn_handle h, snn_stats *out) {
  if (!h || !out) return fail(SNN_ERR_ARG, "null argument");
  out->t = h->t;
  out->spikes = h->spikes;
  out->rec_events = h->spikes * (uint64_t)h->L.M;
  out->ext_events = h->ext_events;
  out->n_neurons = h->L.N;
  out->n_synapses = (uint64_t)h->L.N * h->L.M;
  out->device_bytes = h->arena.bytes;
  out->record_bytes = (uint64_t)h->L.N * h->L.row_bytes;
  out->build_ms = h->build_ms;
  out->h2d_bytes = h->h2d;
  out->d2h_bytes = h->d2h;
  out->kernel_launches = h->launches;
  return SNN_OK;
}

extern "C" int snn_time_kernels(snn_handle h, uint32_t steps, double *ms_out) {
  if (!h || !ms_out) return fail(SNN_ERR_ARG, "null argument");
  if (h->broken) return fail(SNN_ERR_STATE, "network is invalid after an earlier failure");
  if (steps == 0 || steps > h->L.window) return fail(SNN_ERR_ARG, "steps must be in 1..window");
  const uint64_t t0 = h->t;
  if (t0 + steps > 0xFFFFFFFFull) return fail(SNN_ERR_LIMIT, "step counter beyond 2^32");
  const Layout &L = h->L;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  cudaStream_t s = h->stream;
  L2Window l2;
  int rc = l2_window(h, &l2);
  if (rc) return rc;
  std::vector<cudaEvent_t> ev(4 * (size_t)steps + 2, nullptr);
  for (auto &e : ev) CU_TRY(cudaEventCreate(&e));
  struct Guard {
    std::vector<cudaEvent_t> *v;
    cudaGraphExec_t gx[2] = {nullptr, nullptr};
    DevBuf snap;
    cudaStream_t s;
    ~Guard() {
      cudaStreamSynchronize(s);
      for (auto e : *v)
        if (e) cudaEventDestroy(e);
      for (auto g : gx)
        if (g) cudaGraphExecDestroy(g);
      snap.release();
    }
  } guard{&ev};
  guard.s = s;
  const uint32_t phase = (uint32_t)(t0 % L.nbuf);
  uint32_t kernels = 0;
  rc = capture_steps(h, descriptor(h, 0), steps, phase, l2, nullptr, &guard.gx[0], &kernels);
  if (rc) return rc;
  rc = capture_steps(h, descriptor(h, 0), steps, phase, l2, ev.data(), &guard.gx[1], nullptr);
  if (rc) return rc;
  rc = dev_alloc(guard.snap, L.off_rows);   // V, c, ref, input buffers, spike history
  if (rc) return rc;
  set_window(h, h->pinned_win, t0, t0 + steps);
  CU_TRY(cudaMemcpyAsync(base + L.off_win[0], h->pinned_win, sizeof(NetWin), cudaMemcpyHostToDevice, s));
  // (1) the steps as snn_run runs them, from a snapshot that is restored after
  CU_TRY(cudaMemcpyAsync(guard.snap.p, base, L.off_rows, cudaMemcpyDeviceToDevice, s));
  cudaEvent_t a = ev[4 * (size_t)steps], b = ev[4 * (size_t)steps + 1];
  CU_TRY(cudaGraphUpload(guard.gx[0], s));   // keep the first launch's upload out of the timed span
  CU_TRY(cudaGraphUpload(guard.gx[1], s));
  CU_TRY(cudaEventRecord(a, s));
  CU_TRY(cudaGraphLaunch(guard.gx[0], s));
  CU_TRY(cudaEventRecord(b, s));
  CU_TRY(cudaMemcpyAsync(base, guard.snap.p, L.off_rows, cudaMemcpyDeviceToDevice, s));
  CU_TRY(cudaMemsetAsync(base + L.off_rec[0], 0, L.rec_block, s));
  // (2) the same steps with event nodes around every kernel; these results stay
  CU_TRY(cudaGraphLaunch(guard.gx[1], s));
  h->launches += 2ull * kernels;
  rc = drain_window(h, 0, t0, s);
  if (rc) return rc;
  h->t = t0 + steps;
  double up = 0, dl = 0;
  uint32_t n_dl = 0;
  for (uint32_t k = 0; k < steps; ++k) {
    float x = 0, y = 0;
    CU_TRY(cudaEventElapsedTime(&x, ev[4 * k + 0], ev[4 * k + 1]));
    up += x;
    if ((phase + k + 1u) % L.kmin == 0u) {
      CU_TRY(cudaEventElapsedTime(&y, ev[4 * k + 2], ev[4 * k + 3]));
      dl += y;
      ++n_dl;
    }
  }
  float whole = 0;
  CU_TRY(cudaEventElapsedTime(&whole, a, b));
  ms_out[0] = up / steps;
  ms_out[1] = n_dl ? dl / n_dl : 0.0;
  ms_out[2] = (double)whole / steps;
  return SNN_OK;
}

// ---------------------------------------------------------------------------
// batch tuner: fused-kernel shapes timed on the whole batch from snapshots of
// every network, restored after each trial
// ---------------------------------------------------------------------------
// Snapshots of several networks for the multi-network tuners: state (V, c,
// ref, input buffers, spike history), counters, records and launch shape,
// restored after every trial so that the networks' results are unchanged.
// Copies are ordered on the first network's stream; the others wait for it.
struct MultiSnapshot {
  struct Saved {
    DevBuf snap;
    uint64_t t, spikes, ext;
    size_t raster, sorted;
    std::vector<uint32_t> rates;
    snn_launch cfg;
  };
  const snn_handle *hs = nullptr;
  int n = 0;
  cudaStream_t s = nullptr;
  std::vector<Saved> sv;
  ~MultiSnapshot() {
    if (s) cudaStreamSynchronize(s);
    for (auto &x : sv) x.snap.release();
  }
  int take(const snn_handle *hs_, int n_) {
    hs = hs_;
    n = n_;
    s = hs[0]->stream;
    for (int i = 0; i < n; ++i)
      if (hs[i]->stream != s) CU_TRY(cudaStreamSynchronize(hs[i]->stream));
    sv.resize((size_t)n);
    for (int i = 0; i < n; ++i) {
      snn_net *h = hs[i];
      int rc = dev_alloc(sv[i].snap, h->L.off_rows);   // V, c, ref, input buffers, spike history
      if (rc) return rc;
      CU_TRY(cudaMemcpyAsync(sv[i].snap.p, h->arena.p, h->L.off_rows, cudaMemcpyDeviceToDevice, s));
      sv[i].t = h->t;
      sv[i].spikes = h->spikes;
      sv[i].ext = h->ext_events;
      sv[i].raster = h->raster.size();
      sv[i].sorted = h->raster_sorted;
      sv[i].rates = h->rates;
      sv[i].cfg = h->cfg;
    }
    return SNN_OK;
  }
  int restore() {
    for (int i = 0; i < n; ++i) {
      snn_net *h = hs[i];
      uint8_t *base = static_cast<uint8_t *>(h->arena.p);
      CU_TRY(cudaMemcpyAsync(base, sv[i].snap.p, h->L.off_rows, cudaMemcpyDeviceToDevice, s));
      CU_TRY(cudaMemsetAsync(base + h->L.off_rec[0], 0, h->L.off_entries[0] - h->L.off_rec[0], s));   // both blocks
      h->t = sv[i].t;
      h->spikes = sv[i].spikes;
      h->ext_events = sv[i].ext;
      h->raster.resize(sv[i].raster);
      h->raster_sorted = std::min(sv[i].sorted, sv[i].raster);
      h->rates = sv[i].rates;
    }
    CU_TRY(cudaStreamSynchronize(s));   // every network's stream may use its state next
    return SNN_OK;
  }
};

static int check_multi(const snn_handle *hs, int32_t n, uint32_t trial_steps, int32_t max_n) {
  if (!hs || n < 1) return fail(SNN_ERR_ARG, "no networks");
  if (n > max_n) return fail(SNN_ERR_LIMIT, "too many networks in one call");
  if (trial_steps == 0) return fail(SNN_ERR_ARG, "trial_steps must be > 0");
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(SNN_ERR_ARG, "null handle");
    if (hs[i]->broken) return fail(SNN_ERR_STATE, "network is invalid after an earlier failure");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(SNN_ERR_ARG, "a network appears twice");
  }
  return SNN_OK;
}

extern "C" int snn_autotune_batch(const snn_handle *hs, int32_t n, uint32_t trial_steps) {
  int rc = check_multi(hs, n, trial_steps, 65535);
  if (rc) return rc;
  MultiSnapshot snap;
  rc = snap.take(hs, n);
  if (rc) return rc;
  cudaStream_t s = snap.s;
  cudaEvent_t e0, e1;
  CU_TRY(cudaEventCreate(&e0));
  CU_TRY(cudaEventCreate(&e1));
  std::vector<uint64_t> steps((size_t)n, trial_steps);
  // one shape on the whole batch: the first pass captures the graphs, the
  // shape's time is the best of the next `reps` passes
  auto trial = [&](const snn_launch &c, int reps, float *ms_out) -> int {
    for (int i = 0; i < n; ++i) hs[i]->cfg = c;
    *ms_out = 1e30f;
    for (int rep = 0; rep <= reps; ++rep) {
      int r = snap.restore();
      if (r) return r;
      CU_TRY(cudaEventRecord(e0, s));
      r = run_fused(hs, steps.data(), n);
      if (r) return r;
      CU_TRY(cudaEventRecord(e1, s));
      CU_TRY(cudaEventSynchronize(e1));
      float ms = 0;
      CU_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) *ms_out = std::min(*ms_out, ms);
    }
    return SNN_OK;
  };
  snn_launch orig = hs[0]->cfg;
  orig.path = 1;
  float orig_ms = 1e30f, best_ms = 1e30f;
  snn_launch best = orig;
  int status = trial(orig, 2, &orig_ms);
  for (int fb : {128, 256, 512})
    for (int ips : {2, 4, 8, 16})
      for (int ln : {8, 16, 32}) {
        if (status != SNN_OK) break;
        snn_launch c = orig;
        c.fused_block = fb;
        c.fused_items_per_sm = ips;
        c.deliver_lanes = ln;
        float ms = 0;
        status = trial(c, 1, &ms);
        if (status == SNN_OK && ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rr = snap.restore();
  const bool replace = status == SNN_OK && best_ms < 0.97f * orig_ms;   // the incumbent unless clearly slower
  for (int i = 0; i < n; ++i) hs[i]->cfg = (status == SNN_OK) ? (replace ? best : orig) : snap.sv[i].cfg;
  return status != SNN_OK ? status : rr;
}

extern "C" int snn_autotune_concurrent(const snn_handle *hs, int32_t n, uint32_t trial_steps) {
  int rc = check_multi(hs, n, trial_steps, 1024);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    if (hs[i]->cfg.path != 0) return fail(SNN_ERR_ARG, "snn_autotune_concurrent tunes the two-kernel path (launch path 0)");
  MultiSnapshot snap;
  rc = snap.take(hs, n);
  if (rc) return rc;
  // events: the start on the first stream (the others wait for it), the end on every stream
  std::vector<cudaEvent_t> ev((size_t)n + 1, nullptr);
  struct EvGuard {
    std::vector<cudaEvent_t> *v;
    ~EvGuard() {
      for (auto e : *v)
        if (e) cudaEventDestroy(e);
    }
  } eg{&ev};
  for (auto &e : ev) CU_TRY(cudaEventCreate(&e));
  std::vector<uint64_t> steps((size_t)n, trial_steps);
  // one assignment of shapes (per network) run concurrently: the first pass
  // captures the graphs, the time is the best of the next `reps` passes
  auto trial = [&](const std::vector<snn_launch> &cs, int reps, float *ms_out) -> int {
    for (int i = 0; i < n; ++i) hs[i]->cfg = cs[(size_t)i];
    *ms_out = 1e30f;
    for (int rep = 0; rep <= reps; ++rep) {
      int r = snap.restore();
      if (r) return r;
      CU_TRY(cudaEventRecord(ev[0], hs[0]->stream));
      for (int i = 1; i < n; ++i) CU_TRY(cudaStreamWaitEvent(hs[i]->stream, ev[0], 0));
      r = run_plain_many(hs, steps.data(), n);
      if (r) return r;
      for (int i = 0; i < n; ++i) CU_TRY(cudaEventRecord(ev[(size_t)i + 1], hs[i]->stream));
      float ms = 0;
      for (int i = 0; i < n; ++i) {
        CU_TRY(cudaEventSynchronize(ev[(size_t)i + 1]));
        float x = 0;
        CU_TRY(cudaEventElapsedTime(&x, ev[0], ev[(size_t)i + 1]));
        ms = std::max(ms, x);
      }
      if (rep > 0) *ms_out = std::min(*ms_out, ms);
    }
    return SNN_OK;
  };
  std::vector<snn_launch> orig((size_t)n);
  for (int i = 0; i < n; ++i) orig[(size_t)i] = hs[i]->cfg;
  float orig_ms = 1e30f;
  int status = trial(orig, 3, &orig_ms);
  // candidates: one update and delivery shape for every network (the
  // networks' other settings kept); all timed once, the four fastest again
  std::vector<std::vector<snn_launch>> cands;
  const int dwb[][2] = {{16, 3}, {16, 2}, {8, 4}, {8, 3}, {8, 6}, {4, 8}};
  for (int ub : {128, 256})
    for (const auto &w : dwb)
      for (int ln : {16, 32}) {
        std::vector<snn_launch> cs = orig;
        for (auto &c : cs) {
          c.update_block = ub;
          c.update_groups = 1;
          c.deliver_warps = w[0];
          c.deliver_blocks = w[1];
          c.deliver_lanes = ln;
        }
        cands.push_back(cs);
      }
  std::vector<std::pair<float, size_t>> timed;
  for (size_t i = 0; i < cands.size() && status == SNN_OK; ++i) {
    float ms = 0;
    status = trial(cands[i], 1, &ms);
    timed.emplace_back(ms, i);
  }
  std::sort(timed.begin(), timed.end());
  float best_ms = 1e30f;
  size_t best = 0;
  for (size_t r = 0; r < timed.size() && r < 4 && status == SNN_OK; ++r) {
    float ms = 0;
    status = trial(cands[timed[r].second], 3, &ms);
    if (status == SNN_OK && ms < best_ms) {
      best_ms = ms;
      best = timed[r].second;
    }
  }
  int rr = snap.restore();
  const bool replace = status == SNN_OK && best_ms < 0.97f * orig_ms;   // the incumbents unless clearly slower
  for (int i = 0; i < n; ++i)
    hs[i]->cfg = (status == SNN_OK) ? (replace ? cands[best][(size_t)i] : orig[(size_t)i]) : snap.sv[(size_t)i].cfg;
  return status != SNN_OK ? status : rr;
}

extern "C" int snn_get_launch(snn_handle h, snn_launch *out) {
  if (!h || !out) return fail(SNN_ERR_ARG, "null argument");
  *out = h->cfg;
  return SNN_OK;
}

extern "C" int snn_set_launch(snn_handle h, const snn_launch *cfg) {
  if (!h || !cfg) return fail(SNN_ERR_ARG, "null argument");
  const snn_launch &c = *cfg;
  if (c.path != 0 && c.path != 1) return fail(SNN_ERR_ARG, "path must be 0 or 1");
  if (c.update_block != 64 && c.update_block != 128 && c.update_block != 256 && c.update_block != 512)
    return fail(SNN_ERR_ARG, "update_block must be 64, 128, 256 or 512");
  if (c.update_block == 64 && c.update_groups != 1) return fail(SNN_ERR_ARG, "update_block 64 takes update_groups 1");
  if (c.deliver_warps < 1 || c.deliver_warps > 16) return fail(SNN_ERR_ARG, "deliver_warps must be in 1..16");
  if (c.fused_block < 128 || c.fused_block > 512 || c.fused_block % 32)
    return fail(SNN_ERR_ARG, "fused_block must be a multiple of 32 in 128..512");
  if (c.fused_items_per_sm < 1 || c.fused_items_per_sm > 32) return fail(SNN_ERR_ARG, "fused_items_per_sm in 1..32");
  if (c.window_steps < 1 || c.window_steps > 4096) return fail(SNN_ERR_ARG, "window_steps in 1..4096");
  if (c.deliver_lanes != 4 && c.deliver_lanes != 8 && c.deliver_lanes != 16 && c.deliver_lanes != 32)
    return fail(SNN_ERR_ARG, "deliver_lanes must be 4, 8, 16 or 32");
  if (c.update_groups != 1 && c.update_groups != 2 && c.update_groups != 4)
    return fail(SNN_ERR_ARG, "update_groups must be 1, 2 or 4");
  if (c.update_block == 512 && c.update_groups == 4)
    return fail(SNN_ERR_ARG, "update_groups 4 needs update_block <= 256");
  if (c.l2_persist != 0 && c.l2_persist != 1) return fail(SNN_ERR_ARG, "l2_persist must be 0 or 1");
  if (c.deliver_blocks < 1 || c.deliver_blocks > 32) return fail(SNN_ERR_ARG, "deliver_blocks must be in 1..32");
  if (c.overlap != 0 && c.overlap != 1) return fail(SNN_ERR_ARG, "overlap must be 0 or 1");
  h->cfg = c;
  return SNN_OK;
}


// ---------------------------------------------------------------------------
// autotuner: time candidate shapes from a snapshot of the state, restore the
// snapshot after each trial, so the network's results are unchanged.
// ---------------------------------------------------------------------------
// path_only: -1 = both launch paths, 0 = two-kernel path only, 1 = fused only.
static int autotune_impl(snn_net *h, uint32_t trial_steps, int path_only) {
  if (!h) return fail(SNN_ERR_ARG, "null handle");
  if (h->broken) return fail(SNN_ERR_STATE, "network is invalid after an earlier failure");
  if (trial_steps == 0) return fail(SNN_ERR_ARG, "trial_steps must be > 0");
  if (path_only < -1 || path_only > 1) return fail(SNN_ERR_ARG, "path must be -1, 0 or 1");
  const Layout &L = h->L;
  uint8_t *base = static_cast<uint8_t *>(h->arena.p);
  const size_t state_bytes = L.off_rows;   // V, c, ref, input buffers, spike history
  DevBuf snap;
  int rc = dev_alloc(snap, state_bytes);
  if (rc) return rc;
  struct G {
    DevBuf *b;
    cudaStream_t s;
    ~G() {
      cudaStreamSynchronize(s);
      b->release();
    }
  } guard{&snap, h->stream};
  cudaStream_t s = h->stream;
  CU_TRY(cudaMemcpyAsync(snap.p, base, state_bytes, cudaMemcpyDeviceToDevice, s));
  const uint64_t t_saved = h->t, spikes_saved = h->spikes, ext_saved = h->ext_events;
  const size_t raster_saved = h->raster.size(), sorted_saved = h->raster_sorted;
  const std::vector<uint32_t> rates_saved = h->rates;
  const snn_launch saved_cfg = h->cfg;
  snn_launch orig = h->cfg;   // the incumbent, on the allowed path
  if (path_only >= 0) orig.path = path_only;

  // stage 1: update shapes with the current delivery shape, and the fused path
  std::vector<snn_launch> cands;
  for (int ub : {64, 128, 256})
    for (int ug : {1, 2, 4}) {
      if (ub == 64 && ug != 1) continue;
      if (path_only == 1) continue;
      snn_launch c = orig;
      c.path = 0;
      c.update_block = ub;
      c.update_groups = ug;
      cands.push_back(c);
    }
  for (int fb : {128, 256})
    for (int ips : {4, 8, 16})
      for (int ln : {8, 16}) {
        if (path_only == 0) continue;
        snn_launch c = orig;
        c.path = 1;
        c.fused_block = fb;
        c.fused_items_per_sm = ips;
        c.deliver_lanes = ln;
        cands.push_back(c);
      }
  cudaEvent_t e0, e1;
  CU_TRY(cudaEventCreate(&e0));
  CU_TRY(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  snn_launch best = orig;
  // time one shape from the snapshot: the first pass captures the graphs, the
  // shape's time is the best of the next `reps` passes
  auto trial = [&](const snn_launch &c, int reps, float *ms_out) -> int {
    h->cfg = c;
    *ms_out = 1e30f;
    for (int rep = 0; rep <= reps; ++rep) {
      CU_TRY(cudaMemcpyAsync(base, snap.p, state_bytes, cudaMemcpyDeviceToDevice, s));
      h->t = t_saved;
      CU_TRY(cudaEventRecord(e0, s));
      int r = snn_run(h, trial_steps);
      if (r) return r;
      CU_TRY(cudaEventRecord(e1, s));
      CU_TRY(cudaEventSynchronize(e1));
      float ms = 0;
      CU_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) *ms_out = std::min(*ms_out, ms);
    }
    return SNN_OK;
  };
  int status = SNN_OK;
  // every candidate timed once, then the four fastest again (best of three),
  // so that one lucky trial does not pick the shape
  auto run_cands = [&]() {
    std::vector<std::pair<float, size_t>> timed;
    for (size_t i = 0; i < cands.size(); ++i) {
      float ms = 0;
      status = trial(cands[i], 1, &ms);
      if (status != SNN_OK) return;
      timed.emplace_back(ms, i);
    }
    std::sort(timed.begin(), timed.end());
    for (size_t r = 0; r < timed.size() && r < 4; ++r) {
      float ms = 0;
      status = trial(cands[timed[r].second], 3, &ms);
      if (status != SNN_OK) return;
      if (ms < best_ms) {
        best_ms = ms;
        best = cands[timed[r].second];
      }
    }
  };
  // the incumbent shape, timed like the L2 switch below; a challenger must be
  // at least 3% faster to replace it (trial times of near-equal shapes differ
  // by noise)
  float orig_ms = 1e30f;
  status = trial(orig, 3, &orig_ms);
  if (status == SNN_OK) run_cands();
  if (status == SNN_OK && best.path == 0) {
    // stage 2: delivery shapes with the best update shape
    cands.clear();
    for (int dw : {4, 8, 16})
      for (int ln : {8, 16, 32})
        for (int db : {2, 3, 4, 6, 8}) {
          snn_launch c = best;
          c.deliver_warps = dw;
          c.deliver_lanes = ln;
          c.deliver_blocks = db;
          cands.push_back(c);
        }
    run_cands();
  }
  // on/off switches on the best shape (the persisting L2 window, then the
  // overlap of the kernels): both settings timed again, and a switch is
  // turned off only when that is clearly faster
  auto switch_trial = [&](int32_t snn_launch::*field) {
    snn_launch on = best, off = best;
    on.*field = 1;
    off.*field = 0;
    float ms_on = 0, ms_off = 0;
    status = trial(on, 3, &ms_on);
    if (status == SNN_OK) status = trial(off, 3, &ms_off);
    if (status == SNN_OK) {
      const bool use_off = ms_off < 0.97f * ms_on;
      best = use_off ? off : on;
      best_ms = use_off ? ms_off : ms_on;
    }
  };
  if (status == SNN_OK && best.path == 0) switch_trial(&snn_launch::l2_persist);
  if (status == SNN_OK && best.path == 0) switch_trial(&snn_launch::overlap);
  if (status == SNN_OK && !(best_ms < 0.97f * orig_ms)) best = orig;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the network exactly as it was
  CU_TRY(cudaMemcpyAsync(base, snap.p, state_bytes, cudaMemcpyDeviceToDevice, s));
  CU_TRY(cudaMemsetAsync(base + L.off_rec[0], 0, L.off_entries[0] - L.off_rec[0], s));   // both blocks
  CU_TRY(cudaStreamSynchronize(s));
  h->t = t_saved;
  h->spikes = spikes_saved;
  h->ext_events = ext_saved;
  h->raster.resize(raster_saved);
  h->raster_sorted = std::min(sorted_saved, raster_saved);
  h->rates = rates_saved;
  h->cfg = (status == SNN_OK) ? best : saved_cfg;
  return status;
}

extern "C" int snn_autotune(snn_handle h, uint32_t trial_steps) { return autotune_impl(h, trial_steps, -1); }

extern "C" int snn_autotune_path(snn_handle h, uint32_t trial_steps, int32_t path) {
  return autotune_impl(h, trial_steps, path);
}
