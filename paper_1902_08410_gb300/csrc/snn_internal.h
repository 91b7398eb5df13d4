// snn_internal.h -- device descriptors shared by the host runtime (snn_host.cpp)
// and the kernels (snn_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace snn {

constexpr int kK = 1250;          // neurons per module (Sec. 2.2)
constexpr int kNPop = 3;          // F, B, I
constexpr int kZTab = 4096;       // Gaussian quantile table size (12-bit index)
constexpr int kPoisMax = 16;      // external events per neuron and step are capped at 16
constexpr int kMaxM = 4096;       // out-degree limit
constexpr int kNeuronAlign = 128; // neuron arrays padded to a multiple of 128

// status bits written by kernels
constexpr uint32_t kStatusRasterOverflow = 2u;

// Time window of one graph replay (device memory, rewritten by the host
// before every replay so that captured graphs stay valid).
struct alignas(16) NetWin {
  uint32_t t0;          // absolute step of the window's first step
  uint32_t t_end;       // exclusive absolute step at which the network stops
  uint32_t bin0;        // first rate bin of the window (t0 / bin_steps)
  uint32_t t0_slot;     // t0 mod D
  uint32_t pad[4];
};

// Baked into the kernels of step k of a window when the window is captured
// (windows of one graph all start at the same t0 mod nbuf): k mod D, from
// which a kernel finds the slot of step t0 + k with the window's t0_slot and
// no division, and the input buffer of step t0 + k itself, known before the
// window is read.
struct StepMod {
  uint32_t slot;        // k mod D
  uint32_t buf;         // (t0 + k) mod nbuf
  uint32_t overlapped;  // update of step t0 + k: launched to overlap the delivery pass before it
                        // (programmatic dependent launch; its input buffer is read after griddepcontrol.wait)
};

// Recording header of a network (device memory, zeroed at every window start).
struct alignas(16) RecHeader {
  uint32_t cursor;        // raster entries appended in this window
  uint32_t status;        // kStatus* bits
  uint32_t pad[2];
};

// Static description of a network.  Passed by value as a kernel parameter on
// the single-network path and stored in a device table on the fused path.
struct alignas(16) NetDev {
  // --- sizes
  uint32_t N;           // neurons
  uint32_t N_pad;       // padded to kNeuronAlign
  uint32_t G, gx;       // modules, grid width
  uint32_t M;           // out-degree
  uint32_t M_pad;       // padded to a multiple of 8
  uint32_t D;           // spike-history slots = n_delay + kmin
  uint32_t fmt;         // 0 = f32 weights, 1 = i16 weights
  uint32_t row_bytes;   // bytes of one row: M_pad keys then M_pad weights
  uint32_t bin_steps;
  uint32_t key0, key1;  // Philox key (seed)
  uint32_t slot;        // index of this network in a batch
  uint32_t rec_cap;     // raster entries per window
  uint32_t rates_bins;  // bins in the rate window
  uint32_t n_delay;     // largest delay in steps
  uint32_t os;          // u16 entries per row of the delay-group table (multiple of 8)
  uint32_t kmin;        // smallest delay: steps per exchange period (delivery after steps t with (t + 1) % kmin == 0)
  uint32_t nbuf;        // input buffers = 2 kmin (the input of step t is buffer t % nbuf)
  uint32_t pad1;

  // --- per population constants (Eq. 2 propagators, Table S1)
  float pvv[kNPop], pvc[kNPop], pcc[kNPop];
  float el[kNPop], vth[kNPop], vr[kNPop], alpha[kNPop];
  int32_t narp[kNPop];
  uint32_t pad0[2];
  uint32_t thr[kNPop][kPoisMax];   // Poisson CDF thresholds, scaled by 2^20

  // --- device arrays
  float *V;             // [N_pad]
  float *c;             // [N_pad]
  uint8_t *ref;         // [N_pad]
  // Synaptic input of step t (2^-16 mV): acc[t % nbuf][n], accumulated by
  // reductions during the delivery pass before step t, cleared by the update.
  int32_t *acc;         // [nbuf][N_pad]
  uint32_t *cnt;        // [D] spikes of the step with slot t mod D
  uint32_t *hist;       // [D][N_pad] their ids, in the order they were appended
  uint8_t *rows;        // [N][row_bytes]
  const uint16_t *offs; // [N][os] delay groups: records with delay <= d end at offs[s * os + d]
  const int32_t *amp;   // [3][kZTab] external amplitudes, 2^-16 mV
  const NetWin *win;    // current window
  RecHeader *rec;       // recording header
  unsigned long long *rec_entries;  // [rec_cap] (slot << 48 | k << 32 | id)
  uint32_t *rates;      // [rates_bins][G][3] window counts
  unsigned long long *ext_acc;      // [N_pad / 128] external events per 128-neuron group
};

// Construction-time inputs.
struct BuildDev {
  const uint32_t *cdf;  // [G][G-1] module thresholds
  const float *ztab;    // [kZTab]
  float J[kNPop][kNPop];
  float sig[kNPop][kNPop];
  uint32_t n_delay;     // delays uniform on min_delay..n_delay
  uint32_t min_delay;
  int32_t p_local_mode; // 1 when p_local >= 0 (local bucket shortcut valid), 0 otherwise
};

// Work item of the fused step kernel: a range of one network's neurons to
// update; the item's index among its network's items also selects its share
// of the network's delivery work.
struct FusedItem {
  uint32_t net;         // index into the NetDev table
  uint32_t n_begin;     // first neuron (multiple of 4)
  uint32_t index;       // index of the item among its network's items
  uint32_t count;       // items of the network
};

struct FusedTable {
  const NetDev *nets;
  const FusedItem *items;
  const uint32_t *n_items;  // item count in device memory (the graph outlives any one batch)
  uint32_t lanes;           // lanes per delivery segment
  uint32_t chunks;          // register prefix chunks of 32 delays: 1 or kMaxPreChunks (largest n_delay of the table)
};

// ---- launchers (snn_kernels.cu) -------------------------------------------
cudaError_t prepare_kernels();
cudaError_t launch_build_rows(const NetDev &h_nd, const BuildDev &bd, cudaStream_t s);
cudaError_t launch_init_state(const NetDev &nd, cudaStream_t s);
// Persisting L2 access-policy window attached to a launch (bytes == 0: none).
struct L2Window {
  void *base = nullptr;
  size_t bytes = 0;
  float hit_ratio = 0.0f;
};
// pdl: launched with programmatic stream serialization (overlaps the previous kernel).
cudaError_t launch_update(const NetDev &nd, uint32_t k, StepMod km, int block, int groups, const L2Window &l2,
                          bool pdl, cudaStream_t s);
cudaError_t launch_deliver(const NetDev &nd, uint32_t k, StepMod km, uint32_t lanes, int warps, int blocks,
                           const L2Window &l2, bool pdl, cudaStream_t s);
cudaError_t launch_fused(const FusedTable &tab, uint32_t k, int block, int blocks, cudaStream_t s);
int fused_blocks_per_sm(int block, uint32_t chunks);   // resident fused blocks per SM
// Delivery keeps each warp's segment prefix in registers, in chunks of 32
// delays: one chunk up to n_delay 32, else kMaxPreChunks (n_delay <= 256).
constexpr uint32_t kMaxPreChunks = 8;
inline uint32_t pre_chunks(uint32_t n_delay) { return n_delay <= 32u ? 1u : kMaxPreChunks; }
// u16 entries per row of the delay-group table
inline uint32_t offs_stride(uint32_t n_delay) { return (n_delay + 1u + 7u) & ~7u; }
int device_sm_count();

}  // namespace snn

// ---- host helpers shared by the host translation units (snn_host.cpp) ----
#include <string>
#include <vector>
struct snn_params;
namespace snn {
void module_thresholds(const snn_params &p, std::vector<uint32_t> &out);   // Eq. 1 thresholds [G][G-1]
void gaussian_table(std::vector<float> &ztab);                             // Phi^-1((i + 0.5) / 4096)
void build_inputs(const snn_params &p, BuildDev &bd);                      // efficacy means and spreads
}  // namespace snn
int snn_validate_params(const snn_params &p);   // SNN_OK or an error code (message set)
int snn_fail(int code, const std::string &msg);  // set the thread's last error, return code
