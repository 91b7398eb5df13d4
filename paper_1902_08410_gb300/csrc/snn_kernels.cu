// snn_kernels.cu -- sm_103a kernels of the DPSNN-style grid simulation.
//
// Arithmetic contract (identical on every path, no FMA contraction: the
// dynamics use explicit __fmul_rn/__fadd_rn and the file is built with
// -fmad=false):
//   Eq. 2 over one step for neuron n at step t:
//     I  = synaptic input of step t (int32, 2^-16 mV), cleared once read
//     w  = word (n mod 4) of Philox4x32-10(key = seed, ctr = (n div 4, t, 1, 0))
//     k  = #{j < 16 : (w >> 12) >= thr[pop][j]}     (Poisson count, Sec. 2.1)
//     I += amp[pop][z_e] for the k external events: z_0 = w & 0xFFF, z_e (e >= 1)
//          = top 12 bits of half (e-1) mod 8 of Philox(seed, (n, t, 3, (e-1) div 8))
//     ref > 0 : ref -= 1, V = V_r                    (refractory clamp, Sec. 2.2)
//     else    : V = (E + (P_VV*(V-E) + P_Vc*c)) + I*2^-16; spike if V > V_th
//     c = P_cc*c (+ alpha when the neuron fired)
//   Delivery (Sec. 2.1.1): a spike of source s at step t reaches the target of
//   each record (d, target, w) of s's row at step t + d: the record's
//   fixed-point weight is added to the target's input of step t + d (int32
//   reductions, so the sum does not depend on order).
//
// Delay-major delivery.  A row is stored grouped by delay (Sec. 2.1), with the
// end of each delay group in a small table (offs).  Delays run from kmin to
// n_delay.  A delivery pass follows every kmin-th step t (the paper's exchange
// step equals the minimum delay): it produces the inputs of steps t + 1 ..
// t + kmin, for each of them adding, for d = kmin..n_delay, the delay-d group
// of every spike of step T - d.  Every record handled lands in one of the
// next kmin steps, so the input needs only kmin + 1 int32 buffers per neuron
// (the one being read is never written); 2 kmin are kept, so that windows
// starting at the same step mod 2 kmin share one captured graph, instead of a
// ring of n_delay + 1 slots.  They stay in L2.  The spikes of the last
// n_delay + kmin steps are kept per step slot in `hist`.
#include <algorithm>
#include <cstdint>

#include "snn_internal.h"

namespace snn {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ int pop_of_local(uint32_t local) { return local < 250u ? 0 : (local < 1000u ? 1 : 2); }

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Fire-and-forget prefetch of [src, src + bytes) into L2 (16-byte aligned
// address, size a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Prefetch the byte range [p, p + bytes) widened to 16-byte boundaries; the
// caller guarantees the widened range lies inside one allocation.
__device__ __forceinline__ void prefetch_range_l2(const uint8_t *p, uint32_t bytes) {
  if (bytes == 0) return;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15);
  const uintptr_t a1 = (reinterpret_cast<uintptr_t>(p) + bytes + 15u) & ~uintptr_t(15);
  bulk_prefetch_l2(reinterpret_cast<const void *>(a0), (uint32_t)(a1 - a0));
}

// Programmatic dependent launch: wait for the previous kernel in the stream
// (no-op when launched without the attribute), then let the next one launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Fire-and-forget global reductions (no value returned, no scoreboard wait).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_add_s32(int32_t *addr, int32_t v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u32(uint32_t *addr, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u64(unsigned long long *addr, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(addr), "l"(v) : "memory");
}

// L2-only loads (never served from L1) of data that other kernels of the
// stream write: the neuron state and input buffers, and the spike lists and
// counts, which the update of a step appends to while an overlapping delivery
// pass reads older slots of the same arrays.  L1 stays for the amplitude table.
__device__ __forceinline__ float4 ld_cg_f4(const float4 *p) {
  float4 v;
  asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ld_cg_i4(const int4 *p) {
  int4 v;
  asm volatile("ld.global.cg.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// Read-only loads of synapse records, not kept in L1 (each is used once).
__device__ __forceinline__ uint32_t ld_rec_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_rec_f32(const float *p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int32_t ld_rec_s16(const int16_t *p) {
  int16_t v;
  asm volatile("ld.global.nc.L1::no_allocate.s16 %0, [%1];" : "=h"(v) : "l"(p));
  return (int32_t)v;
}

// ---------------------------------------------------------------------------
// Neuron update (Eq. 2 over one step, Poisson drive) of 4 consecutive neurons.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t poisson_count(const NetDev &nd, int pop, uint32_t w) {
  const uint32_t u = w >> 12;   // 20-bit uniform
  uint32_t k = 0;
  while (k < (uint32_t)kPoisMax && u >= nd.thr[pop][k]) ++k;
  return k;
}

// Amplitudes of external events e0..k-1 of neuron n at step t (2^-16 mV), one
// Philox draw per 8 events; only the rare tail e0 = 9 comes through here.
__device__ __noinline__ int32_t extra_amplitudes(const NetDev &nd, int pop, uint32_t e0, uint32_t k, uint32_t n,
                                                 uint32_t t) {
  const int32_t *ap = nd.amp + pop * kZTab;
  int32_t I = 0;
  uint4 q = make_uint4(0, 0, 0, 0);
  for (uint32_t e = e0; e < k; ++e) {
    const uint32_t i = (e - 1u) & 7u;
    if (e == e0 || i == 0) q = philox4x32_10(n, t, 3u, (e - 1u) >> 3, nd.key0, nd.key1);
    const uint32_t w = i >> 1;
    const uint32_t word = (w == 0) ? q.x : ((w == 1) ? q.y : ((w == 2) ? q.z : q.w));
    const uint32_t half = (i & 1u) ? (word >> 16) : (word & 0xFFFFu);
    I += __ldg(ap + (half >> 4));
  }
  return I;
}

// Amplitudes of events 1..k-1 (k >= 2) of neuron n: events 1..8 come from the
// halves of one draw and their table loads are independent.
__device__ __forceinline__ int32_t extra_sum(const NetDev &nd, int pop, uint32_t k, uint32_t n, uint32_t t) {
  const int32_t *ap = nd.amp + pop * kZTab;
  const uint4 R = philox4x32_10(n, t, 3u, 0u, nd.key0, nd.key1);
  const uint32_t h[8] = {R.x & 0xFFFFu, R.x >> 16, R.y & 0xFFFFu, R.y >> 16,
                         R.z & 0xFFFFu, R.z >> 16, R.w & 0xFFFFu, R.w >> 16};
  int32_t I = 0;
#pragma unroll
  for (uint32_t j = 0; j < 8u; ++j)
    if (j + 1u < k) I += __ldg(ap + (h[j] >> 4));
  if (k > 9u) I += extra_amplitudes(nd, pop, 9u, k, n, t);
  return I;
}

// Events 1..k-1 of every neuron of the warp's 128-neuron tile that received
// more than one external event this step (about 1.4% of neurons at 0.18
// expected events).  The pending (lane, q) pairs are numbered q-major by
// ballots and lane i serves pair i, so a warp pays one draw and one table
// round trip instead of one per neuron and event; sums return by shuffle.
// Called by whole warps (all 32 lanes).
__device__ __forceinline__ void extra_events_warp(const NetDev &nd, uint32_t n0, uint32_t t, const uint32_t (&kx)[4],
                                                  int32_t (&Iv)[4]) {
  if (!__any_sync(0xFFFFFFFFu, kx[0] > 1u || kx[1] > 1u || kx[2] > 1u || kx[3] > 1u)) return;   // most warps
  const uint32_t lane = lane_id(), lt = (1u << lane) - 1u;
  uint32_t bal[4], idx[4], cnt[4], total = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    bal[q] = __ballot_sync(0xFFFFFFFFu, kx[q] > 1u);
    idx[q] = total + __popc(bal[q] & lt);
    cnt[q] = total;
    total += __popc(bal[q]);
  }
  if (total == 0u) return;
  const uint32_t packed = kx[0] | (kx[1] << 8) | (kx[2] << 16) | (kx[3] << 24);   // each count <= 16
  const uint32_t tile0 = n0 - lane * 4u;
  for (uint32_t s = 0; s < total; s += 32u) {
    const uint32_t i = s + lane;
    uint32_t q = 0, owner = 0;
    if (i < total) {
      q = (i >= cnt[1] ? 1u : 0u) + (i >= cnt[2] ? 1u : 0u) + (i >= cnt[3] ? 1u : 0u);
      uint32_t b = (q == 0u) ? bal[0] : ((q == 1u) ? bal[1] : ((q == 2u) ? bal[2] : bal[3]));
      const uint32_t base = (q == 0u) ? 0u : ((q == 1u) ? cnt[1] : ((q == 2u) ? cnt[2] : cnt[3]));
      for (uint32_t r = base; r < i; ++r) b &= b - 1u;   // drop the lower set bits: rank i - base
      owner = (uint32_t)(__ffs(b) - 1);
    }
    const uint32_t pk = __shfl_sync(0xFFFFFFFFu, packed, owner);
    int32_t acc = 0;
    if (i < total) {
      const uint32_t n = tile0 + owner * 4u + q;
      acc = extra_sum(nd, pop_of_local(n % (uint32_t)kK), (pk >> (8u * q)) & 0xFFu, n, t);
    }
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const int32_t v = __shfl_sync(0xFFFFFFFFu, acc, idx[qq] & 31u);
      if (kx[qq] > 1u && idx[qq] - s < 32u) Iv[qq] += v;
    }
  }
}


__device__ __forceinline__ bool neuron_step(const NetDev &nd, int pop, float &V, float &c, uint32_t &ref, int32_t I) {
  bool spike = false;
  const float c_old = c;
  if (ref > 0u) {
    ref -= 1u;
    V = nd.vr[pop];
  } else {
    const float el = nd.el[pop];
    const float a = __fsub_rn(V, el);
    const float b = __fmul_rn(nd.pvv[pop], a);
    const float e = __fmul_rn(nd.pvc[pop], c_old);
    const float f = __fadd_rn(b, e);
    const float g = __fadd_rn(el, f);
    const float x = __fmul_rn(__int2float_rn(I), 1.0f / 65536.0f);
    float vn = __fadd_rn(g, x);
    if (vn > nd.vth[pop]) {
      spike = true;
      vn = nd.vr[pop];
      ref = (uint32_t)nd.narp[pop];
    }
    V = vn;
  }
  float cn = __fmul_rn(nd.pcc[pop], c_old);
  if (spike) cn = __fadd_rn(cn, nd.alpha[pop]);
  c = cn;
  return spike;
}

// State of 4 consecutive neurons n0..n0+3 (n0 % 4 == 0, n0 < N_pad).
struct Group4 {
  float4 V, c;
  uint32_t ref;   // 4 x u8
  int4 I;         // synaptic input of the step
};

__device__ __forceinline__ void load_state4(const NetDev &nd, uint32_t n0, Group4 &g) {
  const uint32_t i4 = n0 >> 2;
  g.V = ld_cg_f4(reinterpret_cast<const float4 *>(nd.V) + i4);
  g.c = ld_cg_f4(reinterpret_cast<const float4 *>(nd.c) + i4);
  g.ref = ld_cg_u32(reinterpret_cast<const uint32_t *>(nd.ref) + i4);
}

// Input buffer of the step (buffer `buf` = t % nbuf).  It is cleared by integrate4
// after the neuron state is stored: a store right behind the load to the same
// address held every later load of the warp back.
__device__ __forceinline__ void load_input4(const NetDev &nd, uint32_t n0, uint32_t buf, Group4 &g) {
  g.I = ld_cg_i4(reinterpret_cast<const int4 *>(nd.acc + (size_t)buf * nd.N_pad) + (n0 >> 2));
}

// External drive of 4 neurons at step t (Poisson counts from one
// counter-based draw, word n mod 4 each; amplitudes from the table): adds the
// drive to I and the number of external events of the live neurons to n_ext.
// Reads only the parameters and the amplitude table.
__device__ __forceinline__ void drive4(const NetDev &nd, uint32_t n0, uint32_t t, int32_t (&I)[4], uint32_t &n_ext) {
  const uint4 R = philox4x32_10(n0 >> 2, t, 1u, 0u, nd.key0, nd.key1);
  const uint32_t Wv[4] = {R.x, R.y, R.z, R.w};
  uint32_t local = n0 % (uint32_t)kK;
  int pops[4];
  uint32_t kx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    pops[q] = pop_of_local(local);
    kx[q] = poisson_count(nd, pops[q], Wv[q]);
    local = (local + 1u == (uint32_t)kK) ? 0u : local + 1u;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)   // first external event: independent table loads
    if (kx[q]) I[q] += __ldg(nd.amp + pops[q] * kZTab + (Wv[q] & 0xFFFu));
  extra_events_warp(nd, n0, t, kx, I);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (n0 + q < nd.N) n_ext += kx[q];
}

// Advance the 4 neurons of g by one step (Eq. 2) with total input I (the
// external drive plus the buffer g.I), store the state and clear input buffer
// `buf`; returns the 4-bit spike mask.  Integer input: the order in which the
// drive and the buffer are summed does not change the result.
__device__ __forceinline__ uint32_t integrate4(const NetDev &nd, uint32_t n0, uint32_t buf, const Group4 &g,
                                               const int32_t (&I)[4]) {
  const int32_t Iv[4] = {I[0] + g.I.x, I[1] + g.I.y, I[2] + g.I.z, I[3] + g.I.w};
  float Vv[4] = {g.V.x, g.V.y, g.V.z, g.V.w};
  float cv[4] = {g.c.x, g.c.y, g.c.z, g.c.w};
  uint32_t rv[4] = {g.ref & 0xFFu, (g.ref >> 8) & 0xFFu, (g.ref >> 16) & 0xFFu, g.ref >> 24};
  uint32_t mask = 0;
  uint32_t local = n0 % (uint32_t)kK;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (n0 + q < nd.N && neuron_step(nd, pop_of_local(local), Vv[q], cv[q], rv[q], Iv[q])) mask |= 1u << q;
    local = (local + 1u == (uint32_t)kK) ? 0u : local + 1u;
  }
  if (n0 < nd.N) {
    const uint32_t i4 = n0 >> 2;
    reinterpret_cast<float4 *>(nd.V)[i4] = make_float4(Vv[0], Vv[1], Vv[2], Vv[3]);
    reinterpret_cast<float4 *>(nd.c)[i4] = make_float4(cv[0], cv[1], cv[2], cv[3]);
    reinterpret_cast<uint32_t *>(nd.ref)[i4] = rv[0] | (rv[1] << 8) | (rv[2] << 16) | (rv[3] << 24);
    reinterpret_cast<int4 *>(nd.acc + (size_t)buf * nd.N_pad)[i4] = make_int4(0, 0, 0, 0);
  }
  return mask;
}

// One step of 4 neurons: the state and input loads are issued first and are
// in flight while the drive is computed.
__device__ __forceinline__ uint32_t update4(const NetDev &nd, uint32_t n0, uint32_t t, uint32_t buf, uint32_t &n_ext) {
  Group4 g;
  load_state4(nd, n0, g);
  load_input4(nd, n0, buf, g);
  int32_t I[4] = {0, 0, 0, 0};
  drive4(nd, n0, t, I, n_ext);
  return integrate4(nd, n0, buf, g, I);
}

// Slot (t mod D) of step t = t0 + k from the window's residue and the step's,
// without a division.
__device__ __forceinline__ uint32_t step_slot(const NetDev &nd, const NetWin &w, StepMod km) {
  const uint32_t tm = w.t0_slot + km.slot;
  return tm >= nd.D ? tm - nd.D : tm;
}

// Warp-level recording of the warp's spikes over G groups (all 32 lanes
// active; in group g lane L owns neurons n0[g]..n0[g]+3, and the warp's 32
// lanes cover one aligned 128-neuron tile).  Appends raster entries and the
// step's spike list (`hist`) with one returning atomic each per warp, counts
// rates with fire-and-forget reductions, adds each tile's external events to
// that tile's slot and prefetches into L2 the delay-group table and the first
// records of every spiking neuron's row.  When `smem_list` is given the ids
// are also appended there (block-local list for the fused step).
template <int G>
__device__ __forceinline__ void record_warp(const NetDev &nd, const uint32_t (&mask)[G], const uint32_t (&n0)[G],
                                            const uint32_t (&n_ext)[G], uint32_t t, uint32_t slot, uint32_t k,
                                            uint32_t bin0, uint32_t *smem_list, uint32_t *smem_count) {
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t before[G], wtot = 0;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    before[g] = wtot;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t b = __ballot_sync(0xFFFFFFFFu, (mask[g] >> q) & 1u);
      before[g] += __popc(b & lt);
      wtot += __popc(b);
    }
    uint32_t ext = n_ext[g];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ext += __shfl_xor_sync(0xFFFFFFFFu, ext, o);
    const uint32_t tile = __shfl_sync(0xFFFFFFFFu, n0[g], 0) >> 7;
    if (lane == 0 && ext) red_add_u64(nd.ext_acc + tile, ext);   // slot owned by this warp
  }
  if (wtot == 0) return;
  uint32_t gbase = 0, hbase = 0, sbase = 0;
  if (lane == 0) {
    gbase = atomicAdd(&nd.rec->cursor, wtot);
    hbase = atomicAdd(nd.cnt + slot, wtot);
    if (smem_list) sbase = atomicAdd(smem_count, wtot);
  }
  gbase = __shfl_sync(0xFFFFFFFFu, gbase, 0);
  hbase = __shfl_sync(0xFFFFFFFFu, hbase, 0);
  sbase = __shfl_sync(0xFFFFFFFFu, sbase, 0);
  if (lane == 0 && gbase + wtot > nd.rec_cap) atomicOr(&nd.rec->status, kStatusRasterOverflow);
  const unsigned long long tag = ((unsigned long long)nd.slot << 48) | ((unsigned long long)k << 32);
  const uint32_t bin = t / nd.bin_steps - bin0;
  const uint32_t wb = nd.fmt ? 2u : 4u;
  const uint32_t pre_keys = min(256u, nd.M_pad * 4u), pre_w = min(256u, nd.M_pad * wb);
  uint32_t *hist = nd.hist + (size_t)slot * nd.N_pad;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    uint32_t pos = before[g];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if ((mask[g] >> q) & 1u) {
        const uint32_t id = n0[g] + q;
        // the delivery reads this row's delay groups over the next steps
        const uint8_t *row = nd.rows + (size_t)id * nd.row_bytes;
        bulk_prefetch_l2(nd.offs + (size_t)id * nd.os, nd.os * 2u);
        bulk_prefetch_l2(row, pre_keys);
        bulk_prefetch_l2(row + (size_t)nd.M_pad * 4u, pre_w);
        if (gbase + pos < nd.rec_cap) nd.rec_entries[gbase + pos] = tag | id;
        hist[hbase + pos] = id;
        if (smem_list) smem_list[sbase + pos] = id;
        const uint32_t m = id / (uint32_t)kK;
        red_add_u32(nd.rates + ((size_t)bin * nd.G + m) * 3u + pop_of_local(id - m * (uint32_t)kK), 1u);
        ++pos;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Delay-major delivery (Sec. 2.1.1).  A delivery pass follows the update of
// every step t with (t + 1) % kmin == 0 (kmin = the smallest delay: the spikes
// of kmin consecutive steps are delivered together, the paper's exchange step
// equal to the minimum delay).  It produces the inputs of the next kmin steps
// T = t + 1 .. t + kmin: for each T, the delay-d group (kmin <= d <= n_delay)
// of every spike of step T - d, one segment per (spike, d).  Segments are
// spread over all warps of the grid, `lanes` lanes per segment, and their
// records are reduced straight into the input buffer of T.
// ---------------------------------------------------------------------------
// Slot of step T - d, Tm = T mod D, 1 <= d < D.
__device__ __forceinline__ uint32_t slot_back(uint32_t Tm, uint32_t d, uint32_t D) { return Tm >= d ? Tm - d : Tm + D - d; }

// Segment prefix of one target step, held in registers across the warp:
// lane l of chunk c stands for delay d = 32 c + l + 1, with incl[c] = the
// spikes of steps T - d' summed over kmin <= d' <= d (0 below kmin; past
// n_delay it stays at the total) and base[c] = the sum below the chunk.
// NCH = chunks of 32 delays (n_delay <= 32 NCH).  No shared memory.
template <int NCH>
struct WarpPrefix {
  uint32_t incl[NCH];
  uint32_t base[NCH];
  uint32_t total;
};

// T = t + 1 + j with Tm = T mod D; the spikes of step t itself are left out
// when skip_current.  The count loads of all chunks are issued first.
template <int NCH>
__device__ __forceinline__ void warp_prefix(const NetDev &nd, WarpPrefix<NCH> &P, uint32_t Tm, uint32_t j,
                                            bool skip_current) {
  const uint32_t lane = lane_id();
  const uint32_t D = nd.D, dmax = nd.n_delay, kmin = nd.kmin;
  uint32_t v[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const uint32_t d = 32u * c + lane + 1u;
    const bool use = d >= kmin && d <= dmax && !(skip_current && d == j + 1u);
    v[c] = use ? ld_cg_u32(nd.cnt + slot_back(Tm, d, D)) : 0u;
  }
  uint32_t run = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    uint32_t x = v[c];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    P.base[c] = run;
    P.incl[c] = x + run;
    run = __shfl_sync(0xFFFFFFFFu, P.incl[c], 31);
  }
  P.total = run;
}

// The delay d of segment g of this lane's group (smallest d with prefix > g)
// and the prefix below it; d = 0 when g >= the total.  Called by whole warps:
// every group's g is tested against a chunk with one ballot.
template <int NCH>
__device__ __forceinline__ void find_delay(const WarpPrefix<NCH> &P, uint32_t g, uint32_t lanes, uint32_t &d,
                                           uint32_t &below) {
  const uint32_t lane = lane_id(), grp = lane / lanes, gpw = 32u / lanes;
  d = 0;
  below = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    uint32_t first = 32u;   // this group's first lane of the chunk with prefix > g
    for (uint32_t q = 0; q < gpw; ++q) {
      const uint32_t gq = __shfl_sync(0xFFFFFFFFu, g, q * lanes);
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, P.incl[c] > gq);
      if (grp == q && bal) first = (uint32_t)(__ffs(bal) - 1);
    }
    const uint32_t prev = __shfl_sync(0xFFFFFFFFu, P.incl[c], (first - 1u) & 31u);
    if (d == 0 && first < 32u) {
      d = 32u * c + first + 1u;
      below = first ? prev : P.base[c];
    }
  }
}

// Prefetch into L2 the next delay group (after record b) of source s's row.
__device__ __forceinline__ void prefetch_next_group(const NetDev &nd, uint32_t s, const uint16_t *o, uint32_t d,
                                                    uint32_t b) {
  if (d >= nd.n_delay) return;
  const uint32_t c2 = o[d + 1u];
  if (c2 <= b) return;
  const uint32_t wb = nd.fmt ? 2u : 4u;
  const uint8_t *row = nd.rows + (size_t)s * nd.row_bytes;
  prefetch_range_l2(row + (size_t)b * 4u, (c2 - b) * 4u);
  prefetch_range_l2(row + (size_t)nd.M_pad * 4u + (size_t)b * wb, (c2 - b) * wb);
}

// Reduce the records [a, b) of source s's row into `acc_T`, `lanes` lanes
// (this lane is `sub`), the loads of four records per lane issued first.
__device__ __forceinline__ void add_records(const NetDev &nd, int32_t *acc_T, uint32_t s, uint32_t a, uint32_t b,
                                            uint32_t sub, uint32_t lanes) {
  const uint8_t *row = nd.rows + (size_t)s * nd.row_bytes;
  const uint32_t *keys = reinterpret_cast<const uint32_t *>(row);
  const uint8_t *wrow = row + (size_t)nd.M_pad * 4u;
  for (uint32_t r = a + sub; r < b; r += 4u * lanes) {
    uint32_t kk[4];
    int32_t vv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t rr = r + (uint32_t)u * lanes;
      kk[u] = 0u;
      vv[u] = 0;
      if (rr < b) {
        kk[u] = ld_rec_u32(keys + rr);
        vv[u] = nd.fmt ? ld_rec_s16(reinterpret_cast<const int16_t *>(wrow) + rr) * 64
                       : __float2int_rn(__fmul_rn(ld_rec_f32(reinterpret_cast<const float *>(wrow) + rr), 65536.0f));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r + (uint32_t)u * lanes < b) red_add_s32(acc_T + (kk[u] & 0xFFFFFFu), vv[u]);
  }
}

// Segments of the target step with slot Tm (prefix P): the warp takes
// segments wbase .. wbase + 32 / lanes - 1, then the same plus stride, ...,
// one per group of `lanes` lanes (this lane is `sub` of group grp).
template <int NCH>
__device__ __forceinline__ void deliver_segments(const NetDev &nd, const WarpPrefix<NCH> &P, uint32_t Tm,
                                                 int32_t *acc_T, uint32_t wbase, uint32_t stride, uint32_t lanes) {
  const uint32_t D = nd.D;
  const uint32_t lane = lane_id(), grp = lane / lanes, sub = lane % lanes;
  for (uint32_t gb = wbase; gb < P.total; gb += stride) {   // warp-uniform
    const uint32_t g = gb + grp;
    uint32_t d, below;
    find_delay<NCH>(P, g, lanes, d, below);
    if (d == 0) continue;   // g past the total (last round)
    const uint32_t s = ld_cg_u32(nd.hist + (size_t)slot_back(Tm, d, D) * nd.N_pad + (g - below));
    const uint16_t *o = nd.offs + (size_t)s * nd.os;
    add_records(nd, acc_T, s, o[d - 1u], o[d], sub, lanes);
  }
}

// Fused step, delivery pass after step t: the delay-kmin records of the
// block's own spikes of step t, reduced into the input of step t + kmin (the
// step's spike list is not complete while other blocks still update).
__device__ void deliver_own(const NetDev &nd, const uint32_t *ids, uint32_t cnt, uint32_t t, uint32_t lanes) {
  const uint32_t tid = threadIdx.x;
  const uint32_t grp = tid / lanes, sub = tid % lanes, ngrp = blockDim.x / lanes;
  const uint32_t kmin = nd.kmin;
  uint32_t b = t % nd.nbuf + kmin;
  b = b >= nd.nbuf ? b - nd.nbuf : b;
  int32_t *acc_T = nd.acc + (size_t)b * nd.N_pad;
  for (uint32_t j = grp; j < cnt; j += ngrp) {
    const uint32_t s = ids[j];
    const uint16_t *o = nd.offs + (size_t)s * nd.os;
    const uint32_t a = o[kmin - 1u], b = o[kmin];
    if (sub == 0) prefetch_next_group(nd, s, o, kmin, b);
    add_records(nd, acc_T, s, a, b, sub, lanes);
  }
}

// The counts of the slots the next kmin steps append to (none of them read by
// the pass after step t).
__device__ __forceinline__ void clear_next_counts(const NetDev &nd, uint32_t t) {
  for (uint32_t i = threadIdx.x; i < nd.kmin; i += blockDim.x) nd.cnt[(t + 1u + i) % nd.D] = 0u;
}

// Target step T = t + 1 + j of the pass after step t: its slot T mod D and its
// input buffer T mod nbuf, from tm = t mod D and tb = t mod nbuf (j < kmin < D,
// kmin < nbuf = 2 kmin: one wrap at most).
__device__ __forceinline__ void target_of(const NetDev &nd, uint32_t tm, uint32_t tb, uint32_t j, uint32_t &Tm,
                                          int32_t *&acc_T) {
  Tm = tm + 1u + j;
  Tm = Tm >= nd.D ? Tm - nd.D : Tm;
  uint32_t b = tb + 1u + j;
  b = b >= nd.nbuf ? b - nd.nbuf : b;
  acc_T = nd.acc + (size_t)b * nd.N_pad;
}

// ---------------------------------------------------------------------------
// Kernel: initial state (V uniform on [0, V_th) from Philox stream 2).
// ---------------------------------------------------------------------------
__global__ void k_init_state(const __grid_constant__ NetDev nd) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nd.N_pad) return;
  float v = 0.0f;
  if (n < nd.N) {
    const uint4 r = philox4x32_10(n, 0u, 2u, 0u, nd.key0, nd.key1);
    const float u = __fmul_rn(__uint2float_rn(r.x >> 8), 1.0f / 16777216.0f);
    v = __fmul_rn(nd.vth[pop_of_local(n % (uint32_t)kK)], u);
  }
  nd.V[n] = v;
  nd.c[n] = 0.0f;
  nd.ref[n] = 0;
}

// ---------------------------------------------------------------------------
// Kernel: synapse rows (Eq. 1 module choice, uniform target within the module,
// uniform delay, Gaussian efficacy), each row ordered by key (delay << 24 |
// target), records with equal keys in draw order: grouped by delay and sorted
// by target within a delay, so that the lanes of one delivery instruction
// often update the same 32-byte sector of the input buffer.
// Grid (G, 5): block (m, y) builds rows of module m, local indices
// [250 y, 250 y + 250).  One warp per row at a time.  A warp keeps, per draw,
// the key and the 12-bit quantile index of its efficacy (the weight is formed
// again when the row is written), so that up to 16 warps share the SM.
// ---------------------------------------------------------------------------
constexpr int kBuildWarpsMax = 16;

// Shared memory of one building warp: keys (u32), 256 counters (u32), then
// quantile indices and two permutations (u16), rounded up to 16 bytes.
__host__ __device__ inline uint32_t build_warp_bytes(uint32_t M_pad) {
  return (M_pad * 10u + 256u * 4u + 15u) & ~15u;
}

// Bytes of shared memory before the staged CDF: the quantile table, then the
// efficacy means and spreads (s_js[0] = J, s_js[1] = sigma, [target][source]).
constexpr uint32_t kBuildTableBytes = kZTab * 4u + 128u;

// Efficacy of a synapse from a population-sp source with key `key` and
// quantile index z: J + sigma * z-quantile, clamped so it keeps J's sign.
__device__ __forceinline__ float synapse_weight(const float *s_js, const float *s_z, int sp, uint32_t key,
                                                uint32_t z) {
  const uint32_t tgt = key & 0xFFFFFFu;
  const int tp = pop_of_local(tgt % (uint32_t)kK);
  const float J = s_js[tp * kNPop + sp];
  float w = __fadd_rn(J, __fmul_rn(s_js[kNPop * kNPop + tp * kNPop + sp], s_z[z]));
  if (J > 0.0f && w < 0.0f) w = 0.0f;
  if (J < 0.0f && w > 0.0f) w = 0.0f;
  return w;
}

__global__ void __launch_bounds__(kBuildWarpsMax * 32) k_build_rows(const __grid_constant__ NetDev nd,
                                                                  const __grid_constant__ BuildDev bd, uint32_t cdf_in_smem) {
  extern __shared__ __align__(128) uint8_t smem[];
  float *s_z = reinterpret_cast<float *>(smem);                       // kZTab
  float *s_js = s_z + kZTab;                                          // J, sigma
  uint32_t *s_cdf = reinterpret_cast<uint32_t *>(smem + kBuildTableBytes);   // G-1 (if staged)
  const uint32_t Gm1 = nd.G - 1u;
  const uint32_t cdf_words = cdf_in_smem ? ((Gm1 + 3u) & ~3u) : 0u;
  uint8_t *warp_base = reinterpret_cast<uint8_t *>(s_cdf + cdf_words);
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t per_warp = build_warp_bytes(nd.M_pad);
  uint32_t *w_key = reinterpret_cast<uint32_t *>(warp_base + (size_t)warp * per_warp);
  uint32_t *w_cnt = w_key + nd.M_pad;                                  // 256 counters
  uint16_t *w_z = reinterpret_cast<uint16_t *>(w_cnt + 256);          // quantile index per draw
  uint16_t *w_perm_a = w_z + nd.M_pad;
  uint16_t *w_perm_b = w_perm_a + nd.M_pad;

  const uint32_t m = blockIdx.x;
  for (uint32_t i = threadIdx.x; i < (uint32_t)kZTab; i += blockDim.x) s_z[i] = bd.ztab[i];
  if (threadIdx.x < (uint32_t)(kNPop * kNPop)) {
    s_js[threadIdx.x] = bd.J[threadIdx.x / kNPop][threadIdx.x % kNPop];
    s_js[kNPop * kNPop + threadIdx.x] = bd.sig[threadIdx.x / kNPop][threadIdx.x % kNPop];
  }
  const uint32_t *cdf_row = bd.cdf + (size_t)m * Gm1;
  if (cdf_in_smem)
    for (uint32_t i = threadIdx.x; i < Gm1; i += blockDim.x) s_cdf[i] = cdf_row[i];
  __syncthreads();
  const uint32_t *T = cdf_in_smem ? s_cdf : cdf_row;
  // local bucket of the source module: [T[m-1], T[m])
  const unsigned long long lo_loc = (m == 0u) ? 0ull : (unsigned long long)T[m - 1u];
  const unsigned long long hi_loc = (m == Gm1) ? (1ull << 32) : (unsigned long long)T[m];

  const uint32_t M = nd.M, Mp = nd.M_pad, nd_del = bd.n_delay;
  const uint32_t n_warps = blockDim.x >> 5;
  for (uint32_t l = blockIdx.y * 250u + warp; l < blockIdx.y * 250u + 250u; l += n_warps) {
    const uint32_t s = m * (uint32_t)kK + l;
    const int sp = pop_of_local(l);
    // 1. draw the M synapses of row s
    for (uint32_t j = lane; j < M; j += 32u) {
      const uint4 r = philox4x32_10(s, j, 0u, 0u, nd.key0, nd.key1);
      uint32_t mt;
      if (sp == 2 || nd.G == 1u) {
        mt = m;
      } else if ((unsigned long long)r.x >= lo_loc && (unsigned long long)r.x < hi_loc) {
        mt = m;
      } else {
        uint32_t lo = 0, hi = Gm1;
        while (lo < hi) {
          const uint32_t mid = lo + ((hi - lo) >> 1);
          if (r.x < T[mid]) hi = mid; else lo = mid + 1u;
        }
        mt = lo;
      }
      const uint32_t lt = __umulhi(r.y, (uint32_t)kK);
      const uint32_t tgt = mt * (uint32_t)kK + lt;
      const uint32_t d = bd.min_delay + __umulhi(r.z, nd_del - bd.min_delay + 1u);
      w_key[j] = (d << 24) | tgt;
      w_z[j] = (uint16_t)(r.w >> 20);
    }
    __syncwarp();
    // 2. stable LSD radix sort of the draws by key, one byte per pass: after
    //    pass b the order is by the key's low b + 1 bytes, equal keys in draw
    //    order; passes whose byte is the same for every draw leave it as is
    uint16_t *perm_in = w_perm_a, *perm_out = w_perm_b;
    for (uint32_t i = lane; i < M; i += 32u) perm_in[i] = (uint16_t)i;
    for (uint32_t sh = 0; sh < 32u; sh += 8u) {
      for (uint32_t i = lane; i < 256u; i += 32u) w_cnt[i] = 0u;
      __syncwarp();
      for (uint32_t i = lane; i < M; i += 32u) atomicAdd(&w_cnt[(w_key[i] >> sh) & 0xFFu], 1u);
      __syncwarp();
      // exclusive scan of the 256 counts (8 per lane); skip a pass with one bucket
      uint32_t v[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        v[q] = w_cnt[lane * 8 + q];
        sum += v[q];
      }
      const bool one_bucket = __any_sync(0xFFFFFFFFu, v[0] == M || v[1] == M || v[2] == M || v[3] == M ||
                                                          v[4] == M || v[5] == M || v[6] == M || v[7] == M);
      if (one_bucket) continue;
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      uint32_t acc = incl - sum;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        w_cnt[lane * 8 + q] = acc;
        acc += v[q];
      }
      __syncwarp();
      // stable placement, draws visited in the current order
      for (uint32_t i0 = 0; i0 < M; i0 += 32u) {
        const uint32_t i = i0 + lane;
        const bool valid = i < M;
        const uint32_t e = valid ? perm_in[i] : 0u;
        const uint32_t dg = valid ? ((w_key[e] >> sh) & 0xFFu) : (0x100u + lane);
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dg);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid) perm_out[w_cnt[dg] + rank] = (uint16_t)e;
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == (int)lane) w_cnt[dg] += __popc(peers);
        __syncwarp();
      }
      uint16_t *tmp = perm_in;
      perm_in = perm_out;
      perm_out = tmp;
    }
    const uint16_t *w_perm = perm_in;
    // 4. write the row: keys then weights, padding records zero
    uint8_t *row = nd.rows + (size_t)s * nd.row_bytes;
    uint32_t *okey = reinterpret_cast<uint32_t *>(row);
    for (uint32_t p = lane; p < Mp; p += 32u) okey[p] = p < M ? w_key[w_perm[p]] : 0u;
    if (nd.fmt) {
      int16_t *ow = reinterpret_cast<int16_t *>(row + (size_t)Mp * 4u);
      for (uint32_t p = lane; p < Mp; p += 32u) {
        int q = 0;
        if (p < M) {
          const uint32_t e = w_perm[p];
          q = __float2int_rn(__fmul_rn(synapse_weight(s_js, s_z, sp, w_key[e], w_z[e]), 1024.0f));
          q = q > 32767 ? 32767 : (q < -32768 ? -32768 : q);
        }
        ow[p] = (int16_t)q;
      }
    } else {
      float *ow = reinterpret_cast<float *>(row + (size_t)Mp * 4u);
      for (uint32_t p = lane; p < Mp; p += 32u) {
        float w = 0.0f;
        if (p < M) {
          const uint32_t e = w_perm[p];
          w = synapse_weight(s_js, s_z, sp, w_key[e], w_z[e]);
        }
        ow[p] = w;
      }
    }
    // 5. delay groups of the row: records with delay <= d end at offs[d]
    //    (binary search of the sorted keys, one delay per lane)
    if (nd.offs) {
      uint16_t *orow = const_cast<uint16_t *>(nd.offs) + (size_t)s * nd.os;
      for (uint32_t d = lane; d < nd.os; d += 32u) {
        uint32_t lo = 0, hi = M;
        if (d < nd_del) {
          while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((w_key[w_perm[mid]] >> 24) <= d) lo = mid + 1u; else hi = mid;
          }
        } else {
          lo = M;
        }
        orow[d] = (uint16_t)lo;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Kernel: neuron update + recording (two-kernel path).  No block barrier:
// spikes are appended per warp.
// ---------------------------------------------------------------------------
// Each thread advances G groups of 4 neurons; group g of block b covers the
// neuron range ((b * G + g) * BLOCK + thread) * 4, so every warp owns whole
// aligned 128-neuron tiles.
// The neuron state is final when the kernel starts: either the kernel before
// it has finished, or (km.overlapped) it is a delivery pass launched after the
// previous update, which it waited for before letting this kernel start.  The
// state loads are issued first, then the external drive (which reads no state)
// is computed; without overlap the input buffer is loaded with the state, with
// it only after griddepcontrol.wait (the pass writes that buffer).  The trigger
// that follows the wait lets the delivery pass after this step start on older
// spikes.
// One group per thread is capped at 48 registers (40 resident warps per SM), so
// that a 720k-neuron grid (37 warps per SM) runs in a single wave.
template <int BLOCK, int G>
__global__ void __launch_bounds__(BLOCK, G == 1 ? 1280 / BLOCK : 1) k_update(const __grid_constant__ NetDev nd,
                                                                           uint32_t k, StepMod km) {
  uint32_t n0[G];
  bool live[G];
  bool any = false;
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const uint32_t tile0 = ((blockIdx.x * G + g) * BLOCK + (threadIdx.x & ~31u)) * 4u;
    n0[g] = ((blockIdx.x * G + g) * BLOCK + threadIdx.x) * 4u;
    live[g] = tile0 < nd.N_pad;     // whole warps: N_pad is a multiple of 128
    any |= live[g];
  }
  if (!any) return;
  const NetWin w = *nd.win;   // written before the window's first kernel
  const uint32_t t = w.t0 + k;
  if (t >= w.t_end) return;
  Group4 st4[G];
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (live[g]) {
      load_state4(nd, n0[g], st4[g]);
      if (!km.overlapped) load_input4(nd, n0[g], km.buf, st4[g]);
    }
  int32_t I[G][4];
  uint32_t n_ext[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    I[g][0] = I[g][1] = I[g][2] = I[g][3] = 0;
    n_ext[g] = 0;
    if (live[g]) drive4(nd, n0[g], t, I[g], n_ext[g]);
  }
  pdl_wait();      // the previous kernel (and everything before it) is complete
  pdl_trigger();
  const uint32_t slot = step_slot(nd, w, km), buf = km.buf;
  uint32_t mask[G];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    mask[g] = 0;
    if (live[g] && km.overlapped) load_input4(nd, n0[g], buf, st4[g]);
  }
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (live[g]) mask[g] = integrate4(nd, n0[g], buf, st4[g], I[g]);
  // record per group whose tile is live (warp-uniform)
  if (live[G - 1]) {
    record_warp<G>(nd, mask, n0, n_ext, t, slot, k, w.bin0, nullptr, nullptr);
  } else {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (live[g]) {
        const uint32_t m1[1] = {mask[g]}, a1[1] = {n0[g]}, e1[1] = {n_ext[g]};
        record_warp<1>(nd, m1, a1, e1, t, slot, k, w.bin0, nullptr, nullptr);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel: delivery pass after step t (two-kernel path).  Every warp takes
// segments of every target step of the pass.  Launched with programmatic
// dependent launch after the update of step t: the segments of older spikes
// (steps before t, complete before that update started) are delivered first,
// while the update may still run; after griddepcontrol.wait the step's own
// spikes (their delay-kmin group, into the input of step t + kmin).  The
// trigger after the wait lets the next update load its state and compute its
// drive while the pass finishes.
// ---------------------------------------------------------------------------
// One prefix chunk (n_delay <= 32) fits in 40 registers: three 512-thread
// blocks per SM.
template <int NCH>
__global__ void __launch_bounds__(512, NCH == 1 ? 3 : 2) k_deliver(const __grid_constant__ NetDev nd, uint32_t k, StepMod km,
                                                  uint32_t lanes) {
  const NetWin w = *nd.win;   // written before the window's first kernel
  const uint32_t t = w.t0 + k;
  if (t >= w.t_end) return;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint32_t gpw = 32u / lanes, grp = lane / lanes, sub = lane % lanes;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + warp;
  const uint32_t first = gw * gpw + grp, stride = nwarps * gpw;
  const uint32_t tm = step_slot(nd, w, km), tb = km.buf;
  for (uint32_t j = 0; j < nd.kmin; ++j) {
    uint32_t Tm;
    int32_t *acc_T;
    target_of(nd, tm, tb, j, Tm, acc_T);
    WarpPrefix<NCH> P;   // each warp its own prefix, in registers
    warp_prefix<NCH>(nd, P, Tm, j, true);
    deliver_segments<NCH>(nd, P, Tm, acc_T, gw * gpw, stride, lanes);
  }
  pdl_wait();       // the update of step t is complete: its spike list is final
  pdl_trigger();
  {
    const uint32_t kmin = nd.kmin;
    uint32_t Tm;
    int32_t *acc_T;
    target_of(nd, tm, tb, kmin - 1u, Tm, acc_T);
    const uint32_t *ids = nd.hist + (size_t)tm * nd.N_pad;
    // the list's first entry of this group is loaded together with the count
    // (entries past the count are stale ids, in bounds and unused)
    const uint32_t s0 = first < nd.N_pad ? ld_cg_u32(ids + first) : 0u;
    const uint32_t n = ld_cg_u32(nd.cnt + tm);
    for (uint32_t i = first; i < n; i += stride) {
      const uint32_t s = i == first ? s0 : ld_cg_u32(ids + i);
      const uint16_t *o = nd.offs + (size_t)s * nd.os;
      const uint32_t a = o[kmin - 1u], b = o[kmin];
      if (sub == 0) prefetch_next_group(nd, s, o, kmin, b);
      add_records(nd, acc_T, s, a, b, sub, lanes);
    }
  }
  if (blockIdx.x == 0) clear_next_counts(nd, t);
}

// ---------------------------------------------------------------------------
// Kernel: fused step over a table of networks.  A block takes work items
// (network, 4*blockDim neurons): update and recording with a block-local spike
// list and, after the last step of an exchange period, the delay-kmin records
// of those spikes and the item's share of the rest of the network's pass.
// Update reads input buffer t % nbuf and delivery writes the buffers of steps
// t + 1 .. t + kmin (nbuf = 2 kmin > kmin: never the one being read), so
// blocks need no grid-wide barrier; many small blocks per SM let one block's
// update overlap another's delivery.  Launched with programmatic dependent
// launch: the prologue (descriptor copy, window read) runs while the previous
// step drains.
// ---------------------------------------------------------------------------
template <int NCH>
__global__ void __launch_bounds__(512) k_fused(const __grid_constant__ FusedTable tab, uint32_t k) {
  extern __shared__ __align__(128) uint8_t smem[];   // the item's spike ids (4 * blockDim)
  __shared__ NetDev nd;
  __shared__ NetWin s_win;
  __shared__ uint32_t s_count;
  __shared__ uint32_t s_net;
  uint32_t *s_ids = reinterpret_cast<uint32_t *>(smem);
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  if (threadIdx.x == 0) s_net = 0xFFFFFFFFu;
  bool waited = false;
  const uint32_t n_items = *tab.n_items;
  for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const FusedItem item = tab.items[it];
    __syncthreads();   // the previous item is done with shared memory
    if (s_net != item.net) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(tab.nets + item.net);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&nd);
      for (uint32_t i = threadIdx.x; i < sizeof(NetDev) / 4; i += blockDim.x) dst[i] = src[i];
      if (threadIdx.x == 0) s_win = *reinterpret_cast<const NetWin *>(tab.nets[item.net].win);
    }
    if (threadIdx.x == 0) s_count = 0u;
    __syncthreads();
    if (threadIdx.x == 0) s_net = item.net;
    const uint32_t t = s_win.t0 + k;
    if (t >= s_win.t_end) continue;
    if (!waited) {     // everything below reads what the previous step wrote
      pdl_wait();
      pdl_trigger();
      waited = true;
    }
    const uint32_t n0 = item.n_begin + threadIdx.x * 4u;
    const uint32_t warp_first = item.n_begin + warp * 128u;
    const uint32_t tm = t % nd.D, tb = t % nd.nbuf;
    if (warp_first < nd.N_pad) {
      uint32_t n_ext[1] = {0};
      const uint32_t mask[1] = {update4(nd, n0, t, tb, n_ext[0])};
      const uint32_t a1[1] = {n0};
      record_warp<1>(nd, mask, a1, n_ext, t, tm, k, s_win.bin0, s_ids, &s_count);
    }
    __syncthreads();
    if ((t + 1u) % nd.kmin == 0u) {   // the last step of an exchange period: delivery pass
      const uint32_t lanes = tab.lanes;
      deliver_own(nd, s_ids, s_count, t, lanes);
      // the item's share of the pass: its network's segments are dealt over
      // all groups of all the network's items
      const uint32_t gpb = blockDim.x / lanes, gpw = 32u / lanes;
      const uint32_t wbase = item.index * gpb + warp * gpw, stride = item.count * gpb;
      for (uint32_t j = 0; j < nd.kmin; ++j) {
        uint32_t Tm;
        int32_t *acc_T;
        target_of(nd, tm, tb, j, Tm, acc_T);
        WarpPrefix<NCH> P;
        warp_prefix<NCH>(nd, P, Tm, j, true);
        deliver_segments<NCH>(nd, P, Tm, acc_T, wbase, stride, lanes);
      }
      if (item.index == 0) clear_next_counts(nd, t);
    }
  }
  if (!waited) {
    pdl_wait();
    pdl_trigger();
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

static bool valid_lanes(uint32_t lanes) { return lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32; }
static size_t fused_smem_bytes(int block) { return (size_t)block * 16u; }

// Dynamic shared memory of one construction block: the device's opt-in
// maximum per block (227 KB on sm_103), never above 227 KB.
static size_t build_smem_budget() {
  static size_t cached = 0;
  if (cached) return cached;
  int dev = 0, optin = 0;
  size_t b = 200u * 1024u;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && optin > 0)
    b = std::min<size_t>((size_t)optin, 227u * 1024u);
  cached = b;
  return b;
}

cudaError_t prepare_kernels() {
  return cudaFuncSetAttribute(k_build_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem_budget());
}

cudaError_t launch_init_state(const NetDev &nd, cudaStream_t s) {
  const uint32_t threads = 256;
  const uint32_t blocks = (nd.N_pad + threads - 1) / threads;
  k_init_state<<<blocks, threads, 0, s>>>(nd);
  return cudaGetLastError();
}

cudaError_t launch_build_rows(const NetDev &h_nd, const BuildDev &bd, cudaStream_t s) {
  const uint32_t Gm1 = h_nd.G - 1u;
  const uint32_t cdf_in_smem = (Gm1 <= 12288u) ? 1u : 0u;
  const size_t per_warp = build_warp_bytes(h_nd.M_pad);
  const size_t fixed = (size_t)kBuildTableBytes + (cdf_in_smem ? (((size_t)Gm1 + 3u) & ~(size_t)3u) * 4u : 0u);
  const size_t budget = build_smem_budget();
  if (fixed + per_warp > budget) return cudaErrorInvalidValue;
  const int warps = (int)std::min<size_t>(kBuildWarpsMax, (budget - fixed) / per_warp);
  const size_t smem = fixed + per_warp * (size_t)warps;
  dim3 grid(h_nd.G, 5);
  k_build_rows<<<grid, warps * 32, smem, s>>>(h_nd, bd, cdf_in_smem);
  return cudaGetLastError();
}

// Launch with an optional persisting L2 access-policy window.
// Launch with an optional persisting L2 access-policy window and, with `pdl`,
// programmatic stream serialization (the kernel may start once every block of
// the previous kernel has passed griddepcontrol.launch_dependents).
template <typename... Args>
static cudaError_t launch_ex(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem, const L2Window &l2,
                             bool pdl, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  unsigned n = 0;
  if (pdl) {
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  if (l2.bytes) {
    attr[n].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[n].val.accessPolicyWindow.base_ptr = l2.base;
    attr[n].val.accessPolicyWindow.num_bytes = l2.bytes;
    attr[n].val.accessPolicyWindow.hitRatio = l2.hit_ratio;
    attr[n].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[n].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    ++n;
  }
  cfg.attrs = n ? attr : nullptr;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_update(const NetDev &nd, uint32_t k, StepMod km, int block, int groups, const L2Window &l2,
                          bool pdl, cudaStream_t s) {
  const uint32_t per_block = (uint32_t)block * 4u * (uint32_t)groups;
  const uint32_t blocks = (nd.N_pad + per_block - 1) / per_block;
#define SNN_UPD(B, G) \
  if (block == B && groups == G) return launch_ex(k_update<B, G>, dim3(blocks), dim3(B), 0, l2, pdl, s, nd, k, km);
  SNN_UPD(64, 1) SNN_UPD(128, 1) SNN_UPD(128, 2) SNN_UPD(128, 4)
  SNN_UPD(256, 1) SNN_UPD(256, 2) SNN_UPD(256, 4)
  SNN_UPD(512, 1) SNN_UPD(512, 2)
#undef SNN_UPD
  return cudaErrorInvalidValue;
}

cudaError_t launch_deliver(const NetDev &nd, uint32_t k, StepMod km, uint32_t lanes, int warps, int blocks,
                           const L2Window &l2, bool pdl, cudaStream_t s) {
  if (warps < 1 || warps > 16 || blocks < 1 || !valid_lanes(lanes)) return cudaErrorInvalidValue;
  if (pre_chunks(nd.n_delay) == 1u)
    return launch_ex(k_deliver<1>, dim3((unsigned)blocks), dim3(warps * 32), 0, l2, pdl, s, nd, k, km, lanes);
  if (nd.n_delay <= 32u * kMaxPreChunks)
    return launch_ex(k_deliver<kMaxPreChunks>, dim3((unsigned)blocks), dim3(warps * 32), 0, l2, pdl, s, nd, k, km,
                     lanes);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused(const FusedTable &tab, uint32_t k, int block, int blocks, cudaStream_t s) {
  if (block < 128 || block > 512 || (block % 32) || !valid_lanes(tab.lanes)) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = fused_smem_bytes(block);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (tab.chunks == 1u) return cudaLaunchKernelEx(&cfg, k_fused<1>, tab, k);
  if (tab.chunks == kMaxPreChunks) return cudaLaunchKernelEx(&cfg, k_fused<kMaxPreChunks>, tab, k);
  return cudaErrorInvalidValue;
}

int fused_blocks_per_sm(int block, uint32_t chunks) {
  int n = 0;
  cudaError_t e = chunks == 1u
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<1>, block, fused_smem_bytes(block))
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<kMaxPreChunks>, block,
                                                                      fused_smem_bytes(block));
  if (e != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace snn
