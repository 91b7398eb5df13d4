/*
 * snn.h -- C ABI of the GB300 (sm_103a) simulator of a DPSNN-style cortical grid.
 *
 * Model (Pastorelli et al. 2019, Sec. 2.2): a gx x gy grid of modules of
 * K = 1250 leaky integrate-and-fire neurons with spike-frequency adaptation
 * (Eq. 2), populations F / B / I = local indices 0..249 / 250..999 / 1000..1249;
 * neuron id = module * 1250 + local, module = y * gx + x.  Each neuron projects
 * M (1125 = 0.9 K) synapses; excitatory targets fall off with module distance as
 * exp(-d/lambda) (Eq. 1), inhibitory targets stay in the source module;
 * efficacies are Gaussian (mean J, SD dJ_frac*|J|); every neuron also receives a
 * Poisson drive of N_ext trains at nu_ext with Gaussian amplitudes (Sec. 2.1,
 * Table S1).  The simulation is time driven with dt = dt_ms, delays of
 * min_delay..n_delay steps, and synaptic input accumulated in int32 fixed point of
 * 2^-16 mV, so spike rasters do not depend on delivery order.
 *
 * Conventions:
 *   - Every call returns 0 (SNN_OK) or a negative SNN_ERR_* code; the message of
 *     the last failure on the calling thread is available from snn_last_error().
 *   - The library owns all device memory of a network (allocated through the
 *     allocator installed with snn_set_allocator, cudaMalloc otherwise) and the
 *     caller owns every host buffer passed in.  Pointers named *_out are host
 *     pointers written by the call.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns SNN_ERR_CUDA.
 *   - A network is not thread safe; distinct networks may be used from
 *     distinct threads.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNN_OK 0
#define SNN_ERR_ARG -1       /* invalid argument or parameter set */
#define SNN_ERR_OOM -2       /* device or host allocation failed */
#define SNN_ERR_CUDA -3      /* CUDA runtime error or no device */
#define SNN_ERR_BUFFER -5    /* caller buffer too small; *n_out holds the required count */
#define SNN_ERR_LIMIT -6     /* size beyond an implementation limit (e.g. N >= 2^24 neurons) */
#define SNN_ERR_STATE -7     /* call not valid in the current state */

#define SNN_REC_F32 0        /* synapse record: u32 (delay << 24 | target) + f32 weight (8 B) */
#define SNN_REC_I16 1        /* synapse record: u32 (delay << 24 | target) + i16 weight in 2^-10 mV (6 B) */

#define SNN_K 1250           /* neurons per module (Sec. 2.2) */

/* Model parameters.  Arrays indexed [population] use F = 0, B = 1, I = 2. */
typedef struct snn_params {
  int32_t gx, gy;          /* grid of modules */
  float lambda;            /* Eq. 1 decay length, in inter-module distances */
  float p_local;           /* >= 0: share of excitatory out-degree kept in the source
                              module, the rest over the other modules ~ exp(-d/lambda);
                              < 0: pure Eq. 1 kernel over all modules, source included */
  int32_t out_degree;      /* M, synapses per neuron (1125) */
  int32_t n_delay;         /* largest delay in steps (1..254) */
  int32_t min_delay;       /* smallest delay in steps (1..n_delay; 0 is read as 1): delays are
                              uniform on min_delay..n_delay.  The spikes of min_delay
                              consecutive steps are delivered in one pass (Sec. 2.1.1: the
                              exchange step equals the minimum delay) */
  float dt_ms;             /* time step (0.1 ms) */
  int32_t record_format;   /* SNN_REC_F32 or SNN_REC_I16 */
  int32_t bin_steps;       /* steps per rate bin (50 = 5 ms, Sec. 2.3) */
  float tau_m[3];          /* membrane time constant, ms (Table S1) */
  float C_m[3];            /* capacitance, pF */
  float E_L[3];            /* resting potential, mV */
  float V_th[3];           /* threshold, mV; a spike when V > V_th */
  float V_r[3];            /* reset, mV, held for tau_arp */
  float tau_arp[3];        /* absolute refractory period, ms */
  float alpha_c[3];        /* adaptation jump per spike, mV (0 = no adaptation) */
  float tau_c[3];          /* adaptation time constant, ms */
  float g_c[3];            /* adaptation conductance, nS (g_c/C_m in 1/ms) */
  float J[3][3];           /* mean efficacy J[target population][source population], mV */
  float dJ_frac;           /* efficacy SD as a fraction of |J| (0.25) */
  float J_ext[3];          /* mean external efficacy, mV */
  float dJ_ext_frac;       /* external efficacy SD as a fraction of |J_ext| (0.25) */
  float nu_ext[3];         /* rate per external train, Hz */
  float N_ext[3];          /* external trains per neuron (400) */
} snn_params;

typedef struct snn_net *snn_handle;

/* Counters of one network. */
typedef struct snn_stats {
  uint64_t t;              /* steps simulated so far */
  uint64_t spikes;         /* spikes emitted */
  uint64_t rec_events;     /* recurrent synaptic events delivered (= spikes * M) */
  uint64_t ext_events;     /* external (Poisson) events drawn */
  uint64_t n_neurons;
  uint64_t n_synapses;     /* recurrent synapses stored */
  uint64_t device_bytes;   /* device memory held by the network */
  uint64_t record_bytes;   /* of which synapse records */
  double build_ms;         /* wall time of snn_build_network */
  uint64_t h2d_bytes;      /* host-to-device bytes copied by the library for this network */
  uint64_t d2h_bytes;      /* device-to-host bytes copied by the library for this network */
  uint64_t kernel_launches;/* kernels launched on this network's behalf (graph nodes included) */
} snn_stats;

/* Launch shapes; chosen by snn_autotune or set explicitly. */
typedef struct snn_launch {
  int32_t path;            /* 0 = two kernels per step (update, deliver); 1 = fused step kernel */
  int32_t update_block;    /* threads per update block: 64 (update_groups 1 only), 128, 256 or 512 */
  int32_t deliver_warps;   /* warps per delivery block: 1..16 */
  int32_t fused_block;     /* threads per fused-step block: 128..512 */
  int32_t fused_items_per_sm; /* fused blocks per SM to launch (1..32, capped by occupancy) */
  int32_t window_steps;    /* steps per captured CUDA graph (1..4096) */
  int32_t deliver_lanes;   /* lanes that share one (spike, delay) segment of records: 4, 8, 16, 32 */
  int32_t update_groups;   /* groups of 4 neurons per update thread: 1, 2 or 4
                              (512-thread blocks: 1 or 2) */
  int32_t l2_persist;      /* two-kernel path: 1 = the neuron state and input buffers are
                              given a persisting L2 access-policy window (the CUDA
                              context's persisting set-aside is raised to the device
                              maximum while any such network lives, then restored);
                              0 = normal caching */
  int32_t deliver_blocks;  /* delivery blocks per SM: 1..32 (the grid is SMs x deliver_blocks;
                              every warp takes (spike, delay) segments of the pass) */
  int32_t overlap;         /* two-kernel path: 1 = the kernels of consecutive steps overlap
                              (programmatic dependent launch: a delivery pass starts on the
                              spikes of earlier steps while the update still runs, and the
                              next update computes its external drive while the pass
                              finishes); 0 = every kernel starts after the previous one ends */
} snn_launch;

typedef void *(*snn_alloc_fn)(size_t bytes, void *ctx);
typedef void (*snn_free_fn)(void *ptr, void *ctx);

/* Install the device allocator used for all later allocations (e.g. PyTorch's
 * caching allocator).  NULL functions restore cudaMalloc/cudaFree.  Memory
 * must be device memory of the current device, 256-byte aligned.  Networks
 * keep the functions that allocated them. */
int snn_set_allocator(snn_alloc_fn alloc, snn_free_fn free_fn, void *ctx);

/* Device bytes a network with these parameters will hold once built
 * (synapse records and their delay-group table, neuron state, 2 max(1, min_delay)
 * input buffers, spike history of the last n_delay + max(1, min_delay) steps,
 * tables, recording buffers). */
int snn_footprint(const snn_params *p, size_t *bytes_out);

/* Build a network on the device (Sec. 2.1 initialisation; Eq. 1 connectivity,
 * Sec. 2.2 efficacies).  Synapse j of source neuron s is a pure function of
 * (seed, s, j) drawn from Philox4x32-10, each outgoing row is stored grouped
 * by delay (the paper's delay-ordered synapse lists, Sec. 2.1) and by target
 * within a delay (ties in draw order), with the end of each delay group kept
 * in a table, and the initial V is uniform on [0, V_th).
 * `cuda_stream` (a cudaStream_t, or NULL for the legacy default stream) is the
 * stream every later call of this network is ordered on.  The call returns
 * when the network is ready.  Errors: SNN_ERR_ARG (bad parameters),
 * SNN_ERR_LIMIT (N >= 2^24 neurons or M > 4096), SNN_ERR_OOM, SNN_ERR_CUDA. */
int snn_build_network(const snn_params *p, uint64_t seed, void *cuda_stream, snn_handle *out);

/* Advance the network by `steps` time steps (Eq. 2 update with Poisson drive,
 * spike detection, delivery of each spike's records to their targets d steps
 * later, Sec. 2.1.1) and record spikes and rate counts (Sec. 2.3).  Returns
 * after the steps completed and their records reached host memory.  Errors:
 * SNN_ERR_LIMIT (spike record window overflowed: cannot happen with a
 * refractory period of at least one step), SNN_ERR_CUDA. */
int snn_run(snn_handle h, uint64_t steps);

/* Advance n networks together by steps[i] each with one fused kernel per time
 * step over all of them (networks that reach their count stop early).  Each
 * network's results are identical to snn_run on it alone.  The networks must
 * share one device; the call is ordered on the first network's stream.
 * Errors as snn_run, plus SNN_ERR_ARG (a network twice or NULL) and
 * SNN_ERR_LIMIT (more than 65535 networks).  The paper has no counterpart:
 * batching independent networks is a systems pattern of this library. */
int snn_run_batch(const snn_handle *hs, const uint64_t *steps, int32_t n);

/* Advance n networks by steps[i] each on the two-kernel path (launch path 0
 * for all of them, else SNN_ERR_ARG), every network on its own stream: the
 * windows of the networks are issued round robin, so kernels of different
 * networks run at the same time when their streams differ (networks sharing a
 * stream run one after the other).  Each network's results
 * are identical to snn_run on it alone.  Returns after all steps completed and
 * their records reached host memory.  n in 1..1024.  The paper has no
 * counterpart (one MPI job simulates one network). */
int snn_run_concurrent(const snn_handle *hs, const uint64_t *steps, int32_t n);

/* The spike raster (Sec. 2.3: the spikes every analysis starts from): spikes
 * with t0 <= step < t1, ordered by (step, id), as two parallel host arrays of
 * capacity `cap` owned by the caller (either may be NULL when cap is 0, to
 * query the count).  *n_out receives the count; if it exceeds cap nothing is
 * written and SNN_ERR_BUFFER is returned.  The raster is held in host memory
 * by the library, so the call does not touch the device. */
int snn_read_spikes(snn_handle h, uint64_t t0, uint64_t t1, uint32_t *step_out, uint32_t *id_out,
                    size_t cap, size_t *n_out);

/* Spike counts per (bin, module, population) for all completed steps, layout
 * [bin][module][F, B, I], bin = step / bin_steps (Sec. 2.3: population rates
 * in 5 ms bins; Hz = count / (population size * bin_steps * dt)).  The bin
 * width is the network's parameter bin_steps, fixed at build: the counts are
 * accumulated on the device while the steps run (other widths: bin the raster
 * of snn_read_spikes).  *n_out = bins * G * 3; SNN_ERR_BUFFER when cap is
 * smaller (nothing written). */
int snn_rates(snn_handle h, uint32_t *counts_out, size_t cap, size_t *n_out);

/* Copy the neuron state of Eq. 2 (V in mV, c in mV, remaining refractory
 * steps) of all N neurons to caller-owned host arrays of length n >= N (any of
 * them may be NULL).  Refractory counters are stored as 8-bit values on the
 * device and widened to int32 here.  Synchronises the network's stream. */
int snn_read_state(snn_handle h, float *V_out, float *c_out, int32_t *ref_out, size_t n);

/* Copy the stored outgoing row of source neuron s (Eq. 1 construction,
 * Sec. 2.2 efficacies): M record keys (delay << 24 | target) in stored order
 * and weights in mV (for SNN_REC_I16, q * 2^-10) into caller arrays of
 * capacity cap >= M.  Synchronises the network's stream. */
int snn_read_row(snn_handle h, uint32_t s, uint32_t *keys_out, float *w_out, size_t cap);

/* Counters of the network (host memory; no device access).  Events follow the
 * paper's equivalent-event count (Sec. 2.4) when multiplied by M + N_ext. */
int snn_get_stats(snn_handle h, snn_stats *out);

/* Launch shapes (results never depend on them). */
int snn_get_launch(snn_handle h, snn_launch *out);
int snn_set_launch(snn_handle h, const snn_launch *cfg);

/* Time candidate launch shapes on this network for `trial_steps` steps each
 * and keep the fastest; the network's state, counters and records are
 * restored afterwards, so results are unchanged.  Stages: update shapes (and
 * fused-path shapes), then delivery shapes for the best update shape, each
 * stage timing every candidate once and its four fastest again (best of
 * three); then the L2 window and the kernel overlap switched off only when
 * that is at least 3% faster.  The result replaces the current shape only if
 * at least 3% faster.  Synchronises the network's stream. */
int snn_autotune(snn_handle h, uint32_t trial_steps);

/* The same with the launch path fixed: path 0 tunes the two-kernel path only
 * (the shapes snn_run_concurrent can run), 1 the fused path only, -1 both
 * (= snn_autotune).  The paper has no counterpart of the tuners. */
int snn_autotune_path(snn_handle h, uint32_t trial_steps, int32_t path);

/* The same for a batch advanced by snn_run_batch: fused-kernel shapes (block
 * size, blocks per SM, delivery chunk) are timed on the whole batch for
 * `trial_steps` steps each, from snapshots of every network (state, counters
 * and records restored afterwards, so results are unchanged); the fastest
 * shape replaces the first network's current shape only if at least 3%
 * faster, and is set on every network with launch path 1.  The networks must
 * share one device; the call is ordered on the first network's stream.
 * Allocates a temporary copy of each network's neuron state, input buffers and
 * spike history. */
int snn_autotune_batch(const snn_handle *hs, int32_t n, uint32_t trial_steps);

/* The same for networks advanced together by snn_run_concurrent (launch path
 * 0 on every network): candidate update and delivery shapes, one shape for
 * all networks, are timed running concurrently on the networks' own streams
 * for `trial_steps` steps each (every candidate once, the four fastest again,
 * best of three), from snapshots of every network (state, counters and
 * records restored afterwards, so results are unchanged).  The fastest
 * replaces the networks' current shapes only if at least 3% faster than them
 * running together.  Shapes that are best for a network alone can be slower
 * when networks share the GPU (two 24x24 networks: ~4%).  At most 1024
 * networks; synchronises their streams.  The paper has no counterpart. */
int snn_autotune_concurrent(const snn_handle *hs, int32_t n, uint32_t trial_steps);

/* Measure the two-kernel path on the next `steps` (1..window) steps, then
 * advance the network by them.  The steps run twice from the same state on the
 * network's stream: once captured into one CUDA graph as snn_run runs them
 * (ms_out[2] = mean time per step in milliseconds, CUDA events around the
 * graph; the state is then restored from a device snapshot), and once with an
 * event record node before and after every kernel, each kernel then running
 * alone, without the overlap of consecutive kernels (ms_out[0] / ms_out[1] =
 * mean span of one update / one delivery launch; event nodes lengthen each
 * span, so their ratio is the reliable part).  ms_out holds 3 doubles.
 * Results are identical to snn_run; the call exists to measure kernels without
 * a profiler.  Allocates a temporary copy of the neuron state, input buffers
 * and spike history. */
int snn_time_kernels(snn_handle h, uint32_t steps, double *ms_out);

/* Build the synapse rows of a network (the same construction and the same
 * bytes as snn_build_network) into device memory the caller owns, with no
 * device allocation by the library.  The paper has no counterpart of this
 * call; it exists for callers that cannot let a library call cudaMalloc (a
 * program whose device memory is all handed out by its own pool allocator, a
 * real-time loop that cannot take cudaMalloc's latency and synchronisation,
 * a process that has reserved nearly all device memory).
 *   rows_out:   device pointer, 16-byte aligned, receives N rows of
 *               row_bytes = 4 * M_pad + (4 or 2) * M_pad bytes (M_pad = M rounded
 *               up to 8): M_pad record keys (delay << 24 | target), then M_pad
 *               weights (f32 mV, or i16 in 2^-10 mV for SNN_REC_I16), records in
 *               delay order, padding records zero.  NULL queries the size.
 *   rows_bytes: in: bytes available at rows_out; out: bytes required.
 *   cuda_stream: stream the copies and the kernel are ordered on; the call
 *               returns once they are enqueued.
 * Scratch (module thresholds, Gaussian table) lives in one static device array
 * of about 4.2 MB that every GPU loading the library holds until exit, so the
 * grid may have at most 1024 modules (SNN_ERR_LIMIT beyond).  The first call
 * on a device (the size query included) looks up that array's address, which
 * loads the library's device code and places the array on the device: make a
 * size query before reserving the rest of the device's memory.  The call
 * uploads its tables from host memory it frees on return, so it refuses a
 * stream that is being captured (SNN_ERR_ARG).  All calls share the array:
 * calls whose work overlaps on the GPU race and must be ordered by the caller
 * (for example on one stream).
 * Errors: SNN_ERR_ARG, SNN_ERR_LIMIT, SNN_ERR_BUFFER (rows_bytes too small),
 * SNN_ERR_CUDA. */
int snn_build_rows_static(const snn_params *p, uint64_t seed, void *rows_out, size_t *rows_bytes,
                          void *cuda_stream);

/* Release the network and its device memory. */
void snn_free(snn_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char *snn_last_error(void);


#ifdef __cplusplus
}
#endif
#endif /* SNN_H */
