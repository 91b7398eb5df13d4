#!/usr/bin/env python
"""Benchmark: equivalent synaptic events/s of the 24x24 grid on one GB300.

Workload: two 24x24-module networks (720k neurons, 0.81G recurrent synapses
each, lambda = 1.0 module spacing, f32 synapse records), one in the slow-wave
(SWA) regime and one in the asynchronous (AW) regime.  One bench step advances
both networks by one simulated second (10,000 steps of 0.1 ms) through the
library's public API.  Events follow the paper's equivalent-event count
(Sec. 2.4): every spike counts its recurrent plus external synapses (1125 +
400).

The two networks run concurrently, each on its own CUDA stream
(`run_concurrent`: their kernels overlap on the GPU); `--sequential` runs them
one after the other.

The JSON line reports the device-resident throughput (`value`), an end-to-end
number through the C ABI with host buffers (`e2e`), the roofline of the
dominant kernel measured with CUDA events, SM clocks sampled during the timed
region, and the CPU oracle timed on a bounded sample (`cpu_baseline`).
`--impl reference` times the oracle alone on the host cores.

Multi-GPU (torchrun): every rank simulates its own independent pair of
networks (replicas; the path has no data exchange), `value` is the sum over
ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "synaptic events/s"
UNIT = "events/s"
EQUIV_PER_SPIKE = W.OUT_DEGREE + 400          # recurrent + external synapses per neuron
STEPS_PER_BENCH_STEP = 10_000                 # 1 s simulated per network per bench step
WORKLOAD = ("grid24x24 x2 (SWA + AW): 720k neurons and 0.81G recurrent synapses each, lambda 1.0, "
            "f32 records, 1 s simulated per network per step")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--sim-steps", type=int, default=STEPS_PER_BENCH_STEP,
                    help="0.1 ms steps per network per bench step")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--launch", type=str, default="{}",
                    help="grid mode with --no-tune: launch fields as JSON, e.g. '{\"deliver_blocks\": 8}'")
    ap.add_argument("--sequential", action="store_true",
                    help="run the two networks one after the other instead of concurrently")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="grid mode: skip the compact 64x64, 256-network batch and serving points")
    ap.add_argument("--mode", choices=["grid", "batch", "serve", "grid64", "profile", "table_s1", "min_delay"],
                    default="grid",
                    help="grid: 24x24 SWA+AW (default); batch: 256-network SWA->AW sweep; serve: request "
                         "stream; grid64: 64x64 lambda sweep with f32 vs i16 records")
    ap.add_argument("--grid64-steps", type=int, default=50_000)
    ap.add_argument("--s1-steps", type=int, default=50_000,
                    help="table_s1 and min_delay modes: measured steps per run")
    # --mode profile: one network, fixed launch shape (the target of ncu captures)
    ap.add_argument("--grid", type=int, default=24)
    ap.add_argument("--regime", choices=["SWA", "AW"], default="AW")
    ap.add_argument("--fmt", choices=["f32", "i16"], default="f32")
    ap.add_argument("--path", type=int, choices=[0, 1], default=0)
    ap.add_argument("--warm-steps", type=int, default=1024)
    ap.add_argument("--run-steps", type=int, default=64)
    ap.add_argument("--window", type=int, default=64)
    ap.add_argument("--update-block", type=int, default=256)
    ap.add_argument("--update-groups", type=int, default=1)
    ap.add_argument("--deliver-warps", type=int, default=16)
    ap.add_argument("--deliver-lanes", type=int, default=32)
    ap.add_argument("--deliver-blocks", type=int, default=3)
    ap.add_argument("--l2-persist", type=int, choices=[0, 1], default=1,
                    help="persisting L2 window (profile mode, and grid mode with --no-tune)")
    ap.add_argument("--overlap", type=int, choices=[0, 1], default=1,
                    help="profile mode: kernels of consecutive steps overlap (programmatic dependent launch)")
    ap.add_argument("--grid64-lambdas", type=str, default="0.4,1.0,2.0")
    ap.add_argument("--batch-nets", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=20_000)
    ap.add_argument("--plain-steps", type=int, default=2_000)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=0.0, help="requests/s; 0 = 0.8 x measured capacity")
    ap.add_argument("--duration-scale", type=float, default=1.0)
    ap.add_argument("--chunk-steps", type=int, default=1000)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def reduce(self, value: float, op: str) -> float:
        if not self.pg:
            return value
        import torch
        dev = f"cuda:{self.local_rank}" if torch.cuda.is_available() and self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def job_throughput(dist: Dist, units_local: float, seconds_local: float) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units of all ranks over
    the slowest rank's time.  Returns (throughput, slowest time)."""
    t_max = dist.reduce(seconds_local, "max")
    units_all = dist.reduce(float(units_local), "sum")
    return units_all / t_max, t_max


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[3:7]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_selector(local_rank: int) -> str:
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        return str(local_rank)


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------
def measured_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    with open(os.path.join(ROOT, "paper_1902_08410_gb300", "csrc", "snn_kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def committed_traffic(kernel: str) -> float | None:
    """DRAM bytes per launch from the committed ncu capture, if the kernel source is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    k = t.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_launch"])


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(regimes=("SWA", "AW"), warm_steps=30, timed_steps=100, nets=None):
    """Time the oracle on the same 24x24 networks: `warm_steps` untimed steps
    (the initial volley, during which most rows are generated), then
    `timed_steps` timed steps per network.  Returns (events, seconds, nets)."""
    import oracle
    if nets is None:
        nets = []
        for reg in regimes:
            wl = W.grid_24x24(reg)
            o = oracle.OracleNet(wl["params"], wl["seed"])
            o.run(warm_steps)
            nets.append(o)
    events, secs = 0, 0.0
    for o in nets:
        s0 = o.counters()["spikes"]
        t0 = time.perf_counter()
        o.run(timed_steps)
        secs += time.perf_counter() - t0
        events += (o.counters()["spikes"] - s0) * EQUIV_PER_SPIKE
    return events, secs, nets


def _oracle_core_worker(spec: dict, warm_steps: int, seconds: float, barrier, out) -> None:
    """One host core: one oracle network of the sweep, `warm_steps` untimed
    steps, then 100-step chunks until `seconds` have passed."""
    sys.path.insert(0, ROOT)
    import oracle
    o = oracle.OracleNet(spec["params"], spec["seed"])
    o.run(warm_steps)
    barrier.wait(timeout=900)
    s0 = o.counters()["spikes"]
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.run(100)
        steps += 100
    sec = time.perf_counter() - t0
    out.put(((o.counters()["spikes"] - s0) * EQUIV_PER_SPIKE, sec, steps))
    o.close()


def oracle_all_cores(specs: list[dict], warm_steps: int = 100, seconds: float = 10.0) -> dict | None:
    """The oracle on every host core at once (spawned processes, one independent
    network of `specs` each, started together): aggregate events/s, or None if
    a worker failed."""
    import multiprocessing as mp
    import queue
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")   # never fork a process that has a CUDA context
    barrier = ctx.Barrier(cores)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_core_worker, args=(specs[i % len(specs)], warm_steps, seconds, barrier, out))
             for i in range(cores)]
    for p in procs:
        p.start()
    res = []
    deadline = time.time() + seconds + 900
    while len(res) < len(procs):
        try:
            res.append(out.get(timeout=5))
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs) or time.time() > deadline:
                for p in procs:   # our own children, by handle
                    if p.is_alive():
                        p.terminate()
                return None
    for p in procs:
        p.join(timeout=60)
    ev = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": ev / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle (plain C) on all {cores} host cores at once, one independent network of the sweep "
                      f"per core (networks 0..{min(cores, len(specs)) - 1}), {warm_steps} untimed steps, then "
                      f"~{seconds:.0f} s of 100-step chunks each; value = all cores' events / the slowest core's time",
            "steps_per_core": [r[2] for r in res]}


def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return
    timed_per_step = 10
    _, _, nets = oracle_sample(warm_steps=30, timed_steps=0)
    for _ in range(args.warmup):
        oracle_sample(timed_steps=timed_per_step, nets=nets)
    ev_tot, sec_tot = 0, 0.0
    for _ in range(args.steps):
        ev, sec, _ = oracle_sample(timed_steps=timed_per_step, nets=nets)
        ev_tot += ev
        sec_tot += sec
    value = ev_tot / sec_tot
    sample = (f"oracle (plain C, 1 thread) on the same two 24x24 networks after 30 untimed steps; each bench step "
              f"= {timed_per_step} time steps of each network (rows generated lazily, as the oracle stands)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_steps_per_network": timed_per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
def run_gb300(args, dist: Dist):
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    if dist.rank == 0:
        snn.build()
    dist.barrier()
    snn.lib()
    stream = torch.cuda.current_stream()

    # every network on its own stream: snn_run_concurrent overlaps their kernels
    nets, names, streams = [], [], []
    for reg in ("SWA", "AW"):
        wl = W.grid_24x24(reg)
        streams.append(torch.cuda.Stream())
        nets.append(snn.Network(wl["params"], wl["seed"] + 7919 * dist.rank, stream=streams[-1].cuda_stream))
        names.append(reg)
    # Two ways to advance the pair: "concurrent" (two-kernel path, each network
    # tuned alone, then the pair tuned running together, each on its own
    # stream) and "batch" (both networks in one fused kernel per step, shape
    # tuned on the pair).  After the initial volley both are tuned and timed on
    # alternating stretches of the same run; the faster one is benchmarked.
    form, form_trial = ("sequential" if args.sequential else "concurrent"), None
    if not args.no_tune:
        for n in nets:
            n.run(2000)
            n.autotune(400, path=0)
        cfg_conc = [n.launch for n in nets]
        cfg_batch = None
        if not args.sequential:
            cfg_conc = snn.autotune_concurrent(nets, 400)
            cfg_batch = snn.autotune_batch(nets, 200)
            form_trial = {"concurrent_ms": 0.0, "batch_ms": 0.0, "steps_each": 3 * 700}
            for _ in range(3):
                for f in ("concurrent", "batch"):
                    for n, c in zip(nets, cfg_conc if f == "concurrent" else [cfg_batch] * len(nets)):
                        n.launch = c
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    a.record(stream)
                    for st in streams:
                        st.wait_event(a)
                    if f == "batch":
                        snn.run_batch(nets, [700] * len(nets))
                    else:
                        snn.run_concurrent(nets, 700)
                    for st in streams:
                        stream.wait_stream(st)
                    b.record(stream)
                    torch.cuda.synchronize()
                    form_trial[f + "_ms"] += a.elapsed_time(b)
            form = "batch" if form_trial["batch_ms"] < form_trial["concurrent_ms"] else "concurrent"
        chosen = [cfg_batch] * len(nets) if form == "batch" else cfg_conc
        for n, c in zip(nets, chosen):
            n.launch = c
    else:
        for n in nets:
            n.launch = {"l2_persist": args.l2_persist, **json.loads(args.launch)}
        if nets[0].launch["path"] == 1 and not args.sequential:
            form = "batch"
    steps = args.sim_steps

    def advance(group, n_steps):
        if form == "sequential":
            for n in group:
                n.run(n_steps)
        elif form == "batch":
            snn.run_batch(group, [n_steps] * len(group))
        else:
            snn.run_concurrent(group, n_steps)

    def bench_step():
        advance(nets, steps)

    for _ in range(args.warmup):
        bench_step()
    st0 = [n.stats() for n in nets]
    sampler = ClockSampler(gpu_selector(dist.local_rank))
    dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    # device-side timing: e0 on the current stream, which the networks' streams
    # wait for; at the end the current stream waits for both and records e1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in streams:
        st.wait_event(e0)
    for i in range(args.steps):
        bench_step()
    for st in streams:
        stream.wait_stream(st)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = sampler.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    st1 = [n.stats() for n in nets]
    spikes = [b["spikes"] - a["spikes"] for a, b in zip(st0, st1)]
    ext = [b["ext_events"] - a["ext_events"] for a, b in zip(st0, st1)]
    launches = sum(b["kernel_launches"] - a["kernel_launches"] for a, b in zip(st0, st1))
    events_local = sum(spikes) * EQUIV_PER_SPIKE
    value, t_max = job_throughput(dist, events_local, elapsed)
    sim_s = args.steps * steps * W.DT_MS * 1e-3

    # ---- roofline of the dominant kernel (CUDA events on the launching stream)
    # snn_time_kernels runs the next steps twice from the same state: as a plain
    # graph (step time, CUDA events on the network's stream) and with event
    # nodes around every kernel (the kernels' shares of the step: event nodes
    # lengthen each span, so only their ratio is used).  A kernel's launch
    # duration = step time x its share, both from the same steps, so launch
    # gaps are charged to the kernels and `achieved` is a lower bound.  Four
    # samples 1500 steps apart per network cover the slow oscillation of the
    # SWA network (a single sample may fall in a Down state).  The algorithmic
    # bytes per launch use the spike rate of the timed region itself.
    peak, peak_kind = measured_peaks()
    n_samples, gap = 4, 1500
    per_net = []
    for j, n in enumerate(nets):
        tk_steps = max(1, min(351, n.launch["window_steps"]))
        t_upd = t_dl = t_step = 0.0
        spk = 0
        for i in range(n_samples):
            if i:
                n.run(gap)
            s_a = n.stats()["spikes"]
            tk = n.time_kernels(tk_steps)
            spk += n.stats()["spikes"] - s_a
            sh_u = tk["update_ms"] / (tk["update_ms"] + tk["deliver_ms"])
            t_step += tk["step_ms"] * tk_steps
            t_upd += tk["step_ms"] * sh_u * tk_steps
            t_dl += tk["step_ms"] * (1.0 - sh_u) * tk_steps
        ns = n_samples * tk_steps
        rec_bytes = 8 if n.params["record_format"] == W.REC_F32 else 6
        timed_spk_per_step = spikes[j] / float(args.steps * steps)
        per_net.append({"step_ms": t_step / ns, "update_ms": t_upd / ns, "deliver_ms": t_dl / ns,
                        "update_bytes": 26.0 * n.N,
                        "deliver_bytes": timed_spk_per_step * (n.M * rec_bytes + 8),
                        "timed_spikes_per_step": timed_spk_per_step, "sampled_spikes_per_step": spk / ns})
    upd_ms = sum(x["update_ms"] for x in per_net) / len(per_net)
    dl_ms = sum(x["deliver_ms"] for x in per_net) / len(per_net)
    upd_b = sum(x["update_bytes"] for x in per_net) / len(per_net)
    dl_b = sum(x["deliver_bytes"] for x in per_net) / len(per_net)
    kernels = {
        "k_update": {"ms_per_launch": upd_ms, "algorithmic_bytes": upd_b,
                     "achieved_gbs": upd_b / (upd_ms * 1e-3) / 1e9},
        "k_deliver": {"ms_per_launch": dl_ms, "algorithmic_bytes": dl_b,
                      "achieved_gbs": dl_b / (dl_ms * 1e-3) / 1e9},
    }
    dom = "k_update" if upd_ms >= dl_ms else "k_deliver"
    share = {k: v["ms_per_launch"] / (upd_ms + dl_ms) for k, v in kernels.items()}
    method = (f"launch duration = ms per time step of the network alone ({n_samples} samples of 351 steps, {gap} "
              f"steps apart, each as a graph timed with CUDA events) x the kernel's share of the same steps run "
              f"again with event nodes; delivery bytes = timed-region spikes per step x (M x record bytes + 8)")
    if form == "batch":
        # the timed region ran one fused kernel per step for both networks:
        # its launch duration is the timed region's time per step
        fu_ms = 1e3 * elapsed / (args.steps * steps)
        fu_b = sum(x["update_bytes"] + x["deliver_bytes"] for x in per_net)
        kernels["k_fused"] = {"ms_per_launch": fu_ms, "algorithmic_bytes": fu_b,
                              "achieved_gbs": fu_b / (fu_ms * 1e-3) / 1e9}
        share["k_fused"] = 1.0
        dom = "k_fused"
        method = ("k_fused: one launch per step for both networks in the timed region; launch duration = timed "
                  "region / steps (CUDA events on the launching stream), bytes = both networks' neuron state + "
                  "timed-region spikes per step x (M x record bytes + 8).  k_update / k_deliver: the two-kernel "
                  "path of each network alone, for reference (" + method + ")")
    ach = kernels[dom]["achieved_gbs"]
    # the whole step, the unit a user sees: algorithmic bytes of a step (neuron
    # state + every record delivered) over the step time, per network alone,
    # and over the timed region for the job (both networks concurrently)
    job_bytes = sum(26.0 * n.N * args.steps * steps for n in nets) + sum(
        spikes[j] * (nets[j].M * (8 if nets[j].params["record_format"] == W.REC_F32 else 6) + 8)
        for j in range(len(nets)))
    step_frac = {names[j]: (x["update_bytes"] + x["deliver_bytes"]) / (x["step_ms"] * 1e-3) / 1e9 / peak
                 for j, x in enumerate(per_net)}
    step_frac["job"] = job_bytes / elapsed / 1e9 / peak
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": peak_kind, "traffic": committed_traffic(dom),
                "share_of_step": share[dom],
                "method": method,
                "step_ms": {names[j]: x["step_ms"] for j, x in enumerate(per_net)},
                "step_frac": step_frac,
                "per_network": {names[j]: x for j, x in enumerate(per_net)},
                "kernels": {k: {**v, "frac": v["achieved_gbs"] / peak, "share": share[k]} for k, v in kernels.items()}}

    # ---- activity of the simulated networks (host analysis of the binned rates, Sec. 2.3)
    from paper_1902_08410_gb300 import analysis
    bin_s = W.BIN_STEPS * W.DT_MS * 1e-3
    activity = []
    for n in nets:
        r = n.rates()
        activity.append({"slow_oscillation_hz": analysis.dominant_frequency(r, bin_s),
                         "slow_waves": analysis.slow_wave_speeds(r, 24, 24, bin_s, imd=IMD_MM, skip_s=1.0)})

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e_steps = 5000
        h2d = d2h = 0
        ev = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_nets = []
        for j, reg in enumerate(("SWA", "AW")):
            wl = W.grid_24x24(reg)
            e2e_nets.append(snn.Network(wl["params"], wl["seed"] + 104729 + 7919 * dist.rank,
                                        stream=streams[j].cuda_stream))
        for n, c in zip(e2e_nets, [n.launch for n in nets]):
            n.launch = c
        advance(e2e_nets, e2e_steps)
        for n in e2e_nets:
            st_, ids = n.spikes()
            rates = n.rates()
            s = n.stats()
            h2d += s["h2d_bytes"]
            d2h += s["d2h_bytes"]
            ev += s["spikes"] * EQUIV_PER_SPIKE
            n.close()
        torch.cuda.synchronize()
        e2e_value, t_e2e = job_throughput(dist, ev, time.perf_counter() - t0)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "step": "build both 24x24 networks from host parameters, 0.5 s simulated each, read spikes "
                       "and rates into host arrays, free", "seconds_per_step": t_e2e}

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1)
    cpu = None
    if not args.no_cpu_baseline and dist.world == 1:
        ev, sec, onets = oracle_sample(warm_steps=30, timed_steps=100)
        for o in onets:
            o.close()
        cpu = {"value": ev / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "oracle (plain C, 1 thread) on the same two 24x24 networks: 30 untimed steps, then 100 "
                         "timed steps of each (0.01 s simulated each)", "seconds": sec}

    launch_cfgs = [n.launch for n in nets]
    for n in nets:
        n.close()
    # ---- compact points of the other configurations, each with its own clocks
    extras = None
    if not args.no_extras and dist.world == 1:
        extras = {
            "grid64x64_aw_i16_lambda1": measure_grid64(snn, torch, dist, "AW", 1.0, W.REC_I16, timed=5000,
                                                       transient=5000, trial_steps=100, analyse=False),
        }
        res, _, bnets = measure_batch(snn, torch, dist, n_nets=256, warm=2000, timed=5000, plain_timed=1000)
        for n in bnets:
            n.close()
        extras["batch256"] = res
        extras["serve200"] = measure_serve(snn, torch, dist, n_req=200, duration_scale=0.25, chunk_steps=1000)

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "networks_per_gpu": 2, "neurons_per_gpu": sum(n.N for n in nets),
                       "recurrent_synapses_per_gpu": sum(n.N * n.M for n in nets),
                       "sim_seconds_per_step_per_network": steps * W.DT_MS * 1e-3,
                       "l2": "inputs larger than L2 (2 x 6.5 GB synapse records); the neuron state and input "
                             "buffers of each network (~12 MB) stay in L2 across time steps by design",
                       "launch": launch_cfgs, "parallelism": f"replicas x{dist.world}",
                       "networks_run": {"sequential": "one after the other",
                                        "concurrent": "concurrently, one CUDA stream each, two-kernel path "
                                                      "(snn_run_concurrent), shapes tuned with both running "
                                                      "(snn_autotune_concurrent)",
                                        "batch": "together, one fused kernel per step for both networks "
                                                 "(snn_run_batch)"}[form],
                       "form_trial": form_trial},
            "sim_seconds_per_wall_second": sim_s * len(nets) * dist.world / t_max,
            "per_regime": {names[i]: {"spikes": spikes[i], "rate_hz": spikes[i] / (nets[i].N * sim_s),
                                      "recurrent_events": spikes[i] * W.OUT_DEGREE, "external_events": ext[i],
                                      **activity[i]}
                           for i in range(len(nets))},
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clocks,
            "paper_context": "2.3e9-4.1e9 equivalent synaptic events/s on up to 1024 Haswell cores (Abstract)",
            "extra_configs": extras,
        }
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched sweep: one fused kernel per step over all networks vs one network per launch
# ---------------------------------------------------------------------------
def measure_batch(snn, torch, dist: Dist, n_nets: int, warm: int, timed: int, plain_timed: int,
                  plain_nets: int | None = None) -> tuple[dict, list, list]:
    """The batched sweep: `n_nets` networks on the fused path (one kernel per
    step for all of them, shape from the batch tuner after `warm` steps), then
    `timed` steps timed; beside it one network per launch (two kernels per
    step, each network alone) on fresh copies of the first `plain_nets`
    networks: their first `warm` steps compared with the batch's rasters, the
    next `plain_timed` steps timed.  Returns (result, specs, batch networks)."""
    import numpy as np
    specs = W.batched_sweep(n_nets=n_nets, steps=timed)
    t0 = time.perf_counter()
    nets = [snn.Network(sp["params"], sp["seed"] + 7919 * dist.rank) for sp in specs]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    for n in nets:
        n.launch = {"path": 1}
    stream = torch.cuda.current_stream()
    # the first steps (the initial volley) untimed, then the fused shape tuned
    # on the whole batch (state restored after the trials)
    snn.run_batch(nets, [warm] * len(nets))
    tuned = snn.autotune_batch(nets, 200)
    st0 = sum(n.stats()["spikes"] for n in nets)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_selector(dist.local_rank))
    sampler.start()
    e0.record(stream)
    snn.run_batch(nets, [timed] * len(nets))
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_batch = e0.elapsed_time(e1) / 1e3
    ev_batch = (sum(n.stats()["spikes"] for n in nets) - st0) * EQUIV_PER_SPIKE
    plain_nets = len(nets) if plain_nets is None else min(plain_nets, len(nets))
    ev_plain, t_plain, same, ev_batch_sub = 0, 0.0, 0, 0
    for sp, bn in zip(specs[:plain_nets], nets[:plain_nets]):
        n = snn.Network(sp["params"], sp["seed"] + 7919 * dist.rank)
        n.launch = {"path": 0}
        n.run(warm)
        ps, pi = n.spikes()
        bs, bi = bn.spikes(0, warm)
        same += int(np.array_equal(ps, bs) and np.array_equal(pi, bi))
        s0 = n.stats()["spikes"]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        n.run(plain_timed)
        b.record(stream)
        torch.cuda.synchronize()
        t_plain += a.elapsed_time(b) / 1e3
        ev_plain += (n.stats()["spikes"] - s0) * EQUIV_PER_SPIKE
        n.close()
    res = {
        "workload": f"{len(nets)} networks, sides U{{2..8}}, g_c on a 16-point SWA->AW grid, nu_ext U[2, 8] Hz, "
                    f"i16 records",
        "neurons": sum(n.N for n in nets), "recurrent_synapses": sum(n.N * n.M for n in nets),
        "batched": {"events_per_s": ev_batch / t_batch, "seconds": t_batch, "steps": timed,
                    "us_per_step": 1e6 * t_batch / timed},
        "one_network_per_launch": {"events_per_s": ev_plain / t_plain, "seconds": t_plain, "steps": plain_timed,
                                   "networks": plain_nets},
        "speedup": (ev_batch / t_batch) / (ev_plain / t_plain),
        "identical_rasters": f"{same}/{plain_nets} networks (first {warm} steps, batched vs one per launch)",
        "fused_launch": {k: tuned[k] for k in ("fused_block", "fused_items_per_sm", "deliver_lanes", "window_steps")},
        "timing": f"both forms timed after the first {warm} steps of each network",
        "build_seconds": build_s, "clocks": clocks,
    }
    return res, specs, nets


def run_batch_mode(args, dist: Dist):
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    snn.build()
    res, specs, nets = measure_batch(snn, torch, dist, args.batch_nets, args.plain_steps, args.batch_steps,
                                     args.plain_steps)
    for n in nets:
        n.close()
    batch_value, _ = job_throughput(dist, res["batched"]["events_per_s"] * res["batched"]["seconds"],
                                    res["batched"]["seconds"])
    cpu = None
    if not args.no_cpu_baseline and dist.world == 1:
        cpu = oracle_all_cores(specs)
    line = {"metric": METRIC, "mode": "batch", "value": batch_value, "unit": UNIT, "n_gpus": dist.world,
            "higher_is_better": True, "data": "synthetic", "dtype": "f32+i32",
            "config": {"workload": res["workload"] + f", {args.batch_steps} steps each", "neurons": res["neurons"],
                       "recurrent_synapses": res["recurrent_synapses"]},
            **{k: v for k, v in res.items() if k not in ("workload", "neurons", "recurrent_synapses")},
            "cpu_baseline": cpu}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: Poisson-arrival stream of requests, continuous batching
# ---------------------------------------------------------------------------
def measure_serve(snn, torch, dist: Dist, n_req: int, duration_scale: float, chunk_steps: int,
                  rate: float = 0.0) -> dict:
    """Serve a Poisson-arrival stream of `n_req` requests (continuous batching,
    admission by device-memory footprint); arrivals at `rate` requests/s, or at
    0.8 x the batched capacity measured on the first requests after their
    initial transient."""
    import numpy as np
    from paper_1902_08410_gb300.serve import Server
    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.8)
    reqs = W.serving_requests(n_req=n_req, rate_hz=1.0)
    for r in reqs:
        r["steps"] = max(1, int(round(r["steps"] * duration_scale)))
    if rate <= 0:
        # capacity: neuron-steps per second of the batched path on the first
        # requests, timed after their initial transient (the first steps fire a
        # synchronous volley that would make the capacity look far lower)
        sample = reqs[:min(128, len(reqs))]
        nets = [snn.Network(r["params"], r["seed"]) for r in sample]
        snn.run_batch(nets, [1000] * len(nets))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        snn.run_batch(nets, [2000] * len(nets))
        torch.cuda.synchronize()
        rate_ns = sum(n.N for n in nets) * 2000 / (time.perf_counter() - t0)
        for n in nets:
            n.close()
        work = np.mean([W.n_neurons(r["params"]) * r["steps"] for r in reqs])
        rate = 0.8 * rate_ns / work
    # arrivals: unit-rate stream rescaled to the chosen rate
    srv = Server(memory_budget=budget, chunk_steps=chunk_steps, realtime=True)
    for r in reqs:
        srv.submit(r["params"], r["seed"], r["steps"], arrival_s=r["arrival_s"] / rate)
    sampler = ClockSampler(gpu_selector(dist.local_rank))
    sampler.start()
    out = srv.run()
    clocks = sampler.stop()
    lat = np.array([x.latency_s for x in out["results"]])
    return {"p50_latency_s": out["p50_latency_s"], "p99_latency_s": out["p99_latency_s"],
            "mean_latency_s": float(lat.mean()), "events_per_s": out["events_per_s"], "unit": UNIT,
            "requests": len(reqs), "rate_per_s": rate, "wall_s": out["wall_s"], "chunks": out["chunks"],
            "workload": f"{len(reqs)} requests, sides round(2^U(1,4)), durations U[0.5, 10] s x {duration_scale}, "
                        f"SWA/AW 50/50, i16 records, Poisson arrivals",
            "memory_budget_bytes": budget, "chunk_steps": chunk_steps, "clocks": clocks}


def run_serve_mode(args, dist: Dist):
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    snn.build()
    res = measure_serve(snn, torch, dist, args.requests, args.duration_scale, args.chunk_steps, args.rate)
    line = {"metric": "serving latency and aggregate synaptic events/s", "mode": "serve",
            **{k: v for k, v in res.items() if k not in ("workload", "memory_budget_bytes", "chunk_steps")},
            "config": {"workload": res["workload"], "memory_budget_bytes": res["memory_budget_bytes"],
                       "chunk_steps": res["chunk_steps"]},
            "data": "synthetic", "n_gpus": dist.world}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# 64x64 grid: lambda sweep, SWA and AW, f32 vs packed i16 records
# ---------------------------------------------------------------------------
IMD_MM = 0.4    # inter-module distance in mm (Sec. 3.3.2)


def run_table_s1_mode(args, dist: Dist):
    """Table S1's three parameter states (recurrent and external efficacies per
    population, pure Eq. 1 kernel) on the 24x24 grid at lambda 0.4 and 0.6: mean
    rates per population against the paper's 3.1 / 2.8 / 8.8 Hz, the dominant
    slow-oscillation frequency, the slow-wave speed (Eq. 4, mm/s at 0.4 mm per
    module; Fig. 7A: faster at larger lambda), and the throughput on the same
    kernels."""
    import numpy as np
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    from paper_1902_08410_gb300 import analysis
    snn.build()
    bin_s = W.BIN_STEPS * W.DT_MS * 1e-3
    warm = 10_000
    runs = []
    for lam in (0.4, 0.6):
        for state, target_hz in (("SW_3.1Hz", 3.1), ("AW_2.8Hz", 2.8), ("AW_8.8Hz", 8.8)):
            p = W.table_s1_params(24, 24, lam, state)
            net = snn.Network(p, 1)
            net.run(warm)
            st0 = net.stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            net.run(args.s1_steps)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            st1 = net.stats()
            rates = net.rates()[warm // W.BIN_STEPS:]
            dur = args.s1_steps * W.DT_MS * 1e-3
            pop_hz = (rates.sum(axis=(0, 1)).astype(np.float64) / (np.array(W.POP_SIZES) * net.G * dur)).tolist()
            spikes = st1["spikes"] - st0["spikes"]
            run = {"state": state, "lambda": lam, "paper_rate_hz": target_hz,
                   "rate_hz": spikes / (net.N * dur), "exc_rate_hz": (pop_hz[0] * 250 + pop_hz[1] * 750) / 1000,
                   "pop_rate_hz": pop_hz,
                   "slow_oscillation_hz": analysis.dominant_frequency(rates, bin_s),
                   "slow_waves": analysis.slow_wave_speeds(rates, 24, 24, bin_s, imd=IMD_MM),
                   "events_per_s": spikes * EQUIV_PER_SPIKE / sec, "us_per_step": 1e6 * sec / args.s1_steps}
            runs.append(run)
            net.close()
            if dist.rank == 0:
                print(json.dumps(run), flush=True)
    if dist.rank == 0:
        print(json.dumps({"metric": METRIC, "mode": "table_s1", "unit": UNIT, "runs": len(runs), "data": "synthetic",
                          "config": {"workload": f"24x24 grid, Table S1 efficacies, pure Eq. 1 kernel, {warm} "
                                                 f"warm-up steps then {args.s1_steps} measured steps, seed 1"}}),
              flush=True)


def measure_grid64(snn, torch, dist: Dist, regime: str, lam: float, fmt: int, timed: int, transient: int = 5000,
                   trial_steps: int = 300, analyse: bool = True) -> dict:
    """One 64x64 network (5.12M neurons, 5.76G synapses): `transient` steps,
    the tuner (trials of `trial_steps`), then `timed` steps timed with CUDA
    events (clocks sampled meanwhile)."""
    import numpy as np
    from paper_1902_08410_gb300 import analysis
    wl = W.grid_64x64(regime, lam, fmt)
    t0 = time.perf_counter()
    net = snn.Network(wl["params"], wl["seed"])
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    net.run(transient)              # past the initial transient, where the tuner's choice would not hold
    cfg = net.autotune(trial_steps)
    st0 = net.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_selector(dist.local_rank))
    sampler.start()
    e0.record()
    net.run(timed)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    sec = e0.elapsed_time(e1) / 1e3
    st1 = net.stats()
    spikes = st1["spikes"] - st0["spikes"]
    sim_s = timed * W.DT_MS * 1e-3
    rec_bytes = 8 if fmt == W.REC_F32 else 6
    peak, _ = measured_peaks()
    step_bytes = 26.0 * net.N + spikes / timed * (net.M * rec_bytes + 8)
    out = {"format": "f32" if fmt == W.REC_F32 else "i16", "regime": regime, "lambda": lam,
           "events_per_s": spikes * EQUIV_PER_SPIKE / sec, "sim_seconds_per_wall_second": sim_s / sec,
           "us_per_step": 1e6 * sec / timed, "steps_timed": timed, "rate_hz": spikes / (net.N * sim_s),
           "step_frac": step_bytes / (sec / timed) / 1e9 / peak,
           "bytes_per_recurrent_synapse": st1["device_bytes"] / st1["n_synapses"],
           "build_seconds": build_s, "launch": cfg, "clocks": clocks,
           "timing": f"after {transient} steps and the tuner; {timed} steps, CUDA events"}
    if analyse:
        rates = net.rates()
        pop = rates.sum(axis=(0, 1)).astype(np.float64)
        dur = st1["t"] * W.DT_MS * 1e-3
        out["pop_rate_hz"] = (pop / (np.array(W.POP_SIZES) * net.G * dur)).tolist()
        out["swa_frequency_hz"] = analysis.dominant_frequency(rates, W.BIN_STEPS * W.DT_MS * 1e-3)
        out["slow_waves"] = analysis.slow_wave_speeds(rates, 64, 64, W.BIN_STEPS * W.DT_MS * 1e-3, imd=IMD_MM,
                                                      skip_s=0.5)
    net.close()
    return out


def run_grid64_mode(args, dist: Dist):
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    snn.build()
    runs = []
    for lam in [float(x) for x in args.grid64_lambdas.split(",")]:
        for reg in ("SWA", "AW"):
            f = measure_grid64(snn, torch, dist, reg, lam, W.REC_F32, args.grid64_steps)
            q = measure_grid64(snn, torch, dist, reg, lam, W.REC_I16, args.grid64_steps)
            runs.append({"lambda": lam, "regime": reg, "f32": f, "i16": q,
                         "i16_vs_f32": {"rate_delta_rel": q["rate_hz"] / f["rate_hz"] - 1.0,
                                        "swa_frequency_delta_hz": (None if f["swa_frequency_hz"] is None
                                                                   or q["swa_frequency_hz"] is None
                                                                   else q["swa_frequency_hz"] - f["swa_frequency_hz"]),
                                        "speedup": q["events_per_s"] / f["events_per_s"]}})
            if dist.rank == 0:
                print(json.dumps(runs[-1]), flush=True)
    if dist.rank == 0:
        print(json.dumps({"metric": METRIC, "mode": "grid64", "unit": UNIT, "steps_per_run": args.grid64_steps,
                          "runs": len(runs), "data": "synthetic",
                          "config": {"workload": "64x64 grid, 5.12M neurons, 5.76G recurrent synapses"}}),
              flush=True)


def run_min_delay_mode(args, dist: Dist):
    """The paper's exchange step (Sec. 2.1.1): a 24x24 AW network with delays
    of 10..20 steps (minimum delay 1 ms), delivered once per 10 steps, beside
    the benchmark form with delays of 1..20 steps delivered every step.  Both
    on the two-kernel path, tuned after their first 5000 steps; events/s, time
    per step and kernel launches per simulated millisecond."""
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    snn.build()
    out = []
    for kmin in (1, 10):
        p = W.base_params(24, 24, 1.0, "AW")
        p["min_delay"] = kmin
        net = snn.Network(p, 1)
        net.run(5000)
        cfg = net.autotune(300, path=0)   # both forms on the two-kernel path: one pass launch per exchange
        st0 = net.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(gpu_selector(dist.local_rank))
        sampler.start()
        e0.record()
        net.run(args.s1_steps)
        e1.record()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        sec = e0.elapsed_time(e1) / 1e3
        st1 = net.stats()
        spikes = st1["spikes"] - st0["spikes"]
        sim_ms = args.s1_steps * W.DT_MS
        out.append({"min_delay": kmin, "delays": f"{kmin}..{p['n_delay']} steps",
                    "events_per_s": spikes * EQUIV_PER_SPIKE / sec, "us_per_step": 1e6 * sec / args.s1_steps,
                    "rate_hz": spikes / (net.N * sim_ms * 1e-3),
                    "launches_per_sim_ms": (st1["kernel_launches"] - st0["kernel_launches"]) / sim_ms,
                    "launch": cfg, "clocks": clocks})
        net.close()
        if dist.rank == 0:
            print(json.dumps(out[-1]), flush=True)
    if dist.rank == 0:
        print(json.dumps({"metric": METRIC, "mode": "min_delay", "unit": UNIT, "data": "synthetic",
                          "config": {"workload": f"24x24 AW grid, lambda 1.0, f32 records, {args.s1_steps} "
                                                 f"timed steps after 5000 and the tuner, seed 1"},
                          "launches_ratio": out[1]["launches_per_sim_ms"] / out[0]["launches_per_sim_ms"],
                          "speedup": out[1]["events_per_s"] / out[0]["events_per_s"]}), flush=True)


def run_profile_mode(args, dist: Dist):
    """One network, fixed launch shape: `warm-steps` steps, then `run-steps`
    steps in windows of `window` steps (the kernels an ncu capture targets)."""
    import torch
    torch.cuda.set_device(dist.local_rank)
    import paper_1902_08410_gb300 as snn
    snn.build()
    fmt = W.REC_F32 if args.fmt == "f32" else W.REC_I16
    net = snn.Network(W.base_params(args.grid, args.grid, 1.0, args.regime, record_format=fmt), 1)
    net.launch = {"path": args.path, "window_steps": args.window, "update_block": args.update_block,
                  "update_groups": args.update_groups, "deliver_warps": args.deliver_warps,
                  "deliver_lanes": args.deliver_lanes, "l2_persist": args.l2_persist,
                  "deliver_blocks": args.deliver_blocks, "overlap": args.overlap}
    net.run(args.warm_steps)
    net.run(args.run_steps)
    torch.cuda.synchronize()
    if dist.rank == 0:
        print(json.dumps({"mode": "profile", "grid": args.grid, "regime": args.regime, "format": args.fmt,
                          "launch": net.launch, "stats": net.stats()}), flush=True)
    net.close()


def main():
    args = parse_args()
    if args.mode in ("batch", "serve", "grid64", "profile", "table_s1", "min_delay"):
        dist = Dist("nccl")
        try:
            {"batch": run_batch_mode, "serve": run_serve_mode, "grid64": run_grid64_mode, "table_s1": run_table_s1_mode,
             "profile": run_profile_mode, "min_delay": run_min_delay_mode}[args.mode](args, dist)
        finally:
            dist.close()
        return
    if args.impl == "reference":
        dist = Dist("gloo")
        try:
            run_reference(args, dist)
        finally:
            dist.close()
        return
    dist = Dist("nccl")
    try:
        run_gb300(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
