"""Benchmark of the mechanics hot path: agent-steps/s on the large mechanics + diffusion workload
(10^8 spheres at 0.3 volume fraction, 512^3 FP32 substance grid co-stepped, FP32 forces / FP64
positions), one JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--agents N]

A step is one pass of the whole hot path: grid rebuild (bounds, box ids + histogram, scan, scatter,
canonical gather), force + capped update, and one FTCS diffusion step with its FP64 mass total.
Timed on the device with CUDA events on the library's stream; inputs (12+ GB of agent state) are far
larger than L2.  Under torchrun each rank runs an independent replica (the path is not sharded across
GPUs), value = agents x steps x ranks / max-over-ranks time.

`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2006_06775_gb300 import synth  # noqa: E402

WORKLOAD = "large_mechanics: 1e8 spheres (d~U[8,12] um, 0.3 volume fraction, 5662 um cube) + 512^3 FP32 FTCS grid"
METRIC = "agent-steps/s"

# Algorithmic bytes (compulsory traffic: every input read once, every output written once) per agent
# of each kernel of the mixed-precision step; the box-array terms scale with boxes per agent (B).
KERNEL_BYTES = {
    "key_hist": lambda B: 24 + 8 + 8 * B,        # FP64 centres in; key + rank out; histogram r/w
    "scan_box": lambda B: 12 * B,                # counts in, starts out, counts cleared
    "scatter": lambda B: 12 + 4 + 4 * B,         # key + rank in, starts, perm out
    "gather": lambda B: 44 + 48 + 4 * B,         # perm, key, payload (32) in; payload + skey + p4 out
    "force_mixed": lambda B: 44 + 28 + 4 * B,    # p4, FP64 centre, skey in; centre + count out
    "force_list": lambda m: 96 + 4 * m,          # list (4 B per entry) + count, own p4, FP64 centre
                                                 # and move in; centre, p4, move and neighbour count
                                                 # out (the update is fused)
}
STEP_BYTES_PER_AGENT = lambda B: 4 * 32 + 8 * B  # rebuild + force + update, agent state S = 32 B
# Algorithmic FP32 work of the force kernel: 9 FLOP per candidate pair of the 27-box search (3 sub,
# 3 mul, 2 add, 1 compare; 27 B candidates per agent) + 13 per agent for the capped update.
FORCE_FLOP_PER_AGENT = lambda B: 9 * 27 * B + 13
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
TUNED_PATH = os.path.join(ROOT, "paper_2006_06775_gb300", "tuned.json")


def measured_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` from the committed ncu record, or None when the kernel's
    sources changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_agent"] * n
    except (OSError, KeyError, ValueError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_uuid:
            cmd += ["-i", gpu_uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for name, v in zip(names, r[4:8]):
                    if v.strip() == "Active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_over_ranks(elapsed_ms, agents, steps, world, device=None):
    """Whole-job throughput: agents x steps x ranks over the maximum time of any rank (one
    all-reduce; every rank gets the same result).  Works with NCCL (device tensors) and gloo."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return agents * steps * world / (elapsed_ms * 1e-3), elapsed_ms


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_workload(n, seed):
    params, inp = synth.large_mechanics(n=n, seed=seed, grid_side=synth.large_side(n))
    return params, inp


# ------------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample of the same workload
# ------------------------------------------------------------------------------------------------
class OracleSample:
    """The FP64 oracle on a bounded sample of the workload: n_sample agents at the same density in a
    proportionally smaller cube, with a grid of the same voxel size."""

    def __init__(self, n_sample, seed=2):
        import oracle
        self.oracle = oracle
        self.n = n_sample
        self.gn = max(8, int(round(512 * (n_sample / 1e8) ** (1.0 / 3.0))))
        params, inp = synth.large_mechanics(n=n_sample, seed=seed, grid_n=self.gn)
        self.sim = oracle.OracleSim(params)
        self.sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        self.sim.set_grid(inp["grid"])

    def time_steps(self, steps):
        t0 = time.perf_counter()
        self.sim.step(steps)
        return time.perf_counter() - t0

    def describe(self, steps, secs):
        return ("%d step(s) of %d agents at the workload's density with a %d^3 grid of the same "
                "voxel size, FP64 oracle, OpenMP over agents; %.1f s" % (steps, self.n, self.gn, secs))


def oracle_baseline(n_sample, steps=1):
    s = OracleSample(n_sample)
    secs = s.time_steps(steps)
    return {"value": n_sample * steps / secs, "unit": METRIC, "cores": s.oracle.num_threads(),
            "kind": "oracle", "sample": s.describe(steps, secs)}


def neurite_oracle_baseline(n_sample=20_000):
    """The FP64 neurite oracle as it stands (every pair, no grid) for one step of a neuron forest of
    n_sample agents at the benchmark's density and cell size."""
    import oracle
    scale = n_sample / 9_000_000
    neurons = max(1, int(round(5000 * scale)))
    side = 2000.0 * scale ** (1.0 / 3.0)
    params, inp = synth.neuron_forest(neurons, n_sample, side=side)
    t0 = time.perf_counter()
    oracle.neurite_step(inp["x"], inp["y"], inp["z"], inp["diameter"], inp["rest"], inp["mother"],
                        inp["ox"], inp["oy"], inp["oz"], params["dt"], params["repulsion"],
                        params["attraction"], params["max_displacement"], params["spring"])
    secs = time.perf_counter() - t0
    return {"value": n_sample / secs, "unit": "agent-steps/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "1 step of a %d-agent forest at the same density (%d neurons, %.0f um cube), "
                      "FP64 oracle over all pairs, OpenMP over agents; %.2f s"
                      % (n_sample, neurons, side, secs)}


def sir_oracle_baseline(runs=2, steps=20):
    """The FP64/integer SIR oracle as it stands on `runs` runs of the ensemble, `steps` steps each."""
    import oracle
    ens = synth.sir_ensemble()[:runs]
    secs, agents = 0.0, 0
    for p, inp in ens:
        sim = oracle.OracleSim(dict(p, sir_boxes=32))
        sim.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        t0 = time.perf_counter()
        sim.step(steps)
        secs += time.perf_counter() - t0
        agents += len(inp["x"])
    return {"value": agents * steps / secs, "unit": "agent-steps/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "%d runs x %d persons of the ensemble, %d steps each, 32 boxes per axis, "
                      "oracle (integer positions, one run at a time); %.2f s"
                      % (runs, agents // max(1, runs), steps, secs)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    s = OracleSample(args.cpu_sample)
    s.time_steps(args.warmup)
    secs = s.time_steps(args.steps)
    value = s.n * args.steps / secs
    cpu = {"value": value, "unit": METRIC, "cores": s.oracle.num_threads(), "kind": "oracle",
           "sample": s.describe(args.steps, secs)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "agents": int(1e8), "grid": 512,
                       "sample_agents": s.n},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_2006_06775_gb300 import bdm
    import paper_2006_06775_gb300.build as libbuild

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()
    bdm.load(build_if_missing=False)
    n = args.agents
    params, inp = make_workload(n, seed=2 + rank)
    from paper_2006_06775_gb300 import tune
    cache = tune.TuneCache(TUNED_PATH)
    knobs = None
    if args.tune:  # drop the cached choices of this GPU so that they are measured again
        mine = cache.data.get(tune.gpu_name(), {})
        mine.pop(tune.workload_signature(params, n, inp["side"] ** 3), None)
        for sig in [k for k in mine if k.startswith("sir-batch/")]:
            mine.pop(sig)
        knobs = tune.tune_mechanics(params, inp, inp["side"] ** 3, cache=cache)
    else:
        knobs = cache.get(tune.workload_signature(params, n, inp["side"] ** 3), tune.gpu_name())
    if args.skin is not None:  # explicit sort cadence (neighbour-list skin, um) instead of the tuned one
        knobs = dict(knobs or {"box_factor": 1.0, "force_variant": 0}, skin=args.skin)
    if knobs:
        params = tune.mechanics_params(params, inp, knobs)
    stream = torch.cuda.Stream()
    sim = bdm.Sim(params, stream=stream)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.set_grid(inp["grid"])

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    st0 = sim.get_state(fields=())
    nbox = int(np.prod(st0["grid_dims"]))
    boxes_per_agent = nbox / n

    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    time.sleep(0.3)
    sim.profile(True)
    launches0 = bdm.bdm_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = bdm.bdm_launch_count() - launches0
    ktimes = sim.kernel_times()
    sim.profile(False)
    clk = clocks.stop()
    # max over ranks
    value, elapsed_ms = aggregate_over_ranks(elapsed_ms, n, args.steps, world, device="cuda")
    ms_per_step = elapsed_ms / args.steps

    peak, peak_kind = load_peaks()
    per_launch = {k: v[1] / max(v[0], 1) for k, v in ktimes.items()}
    share = {k: v[1] for k, v in ktimes.items()}
    dom = max(share, key=lambda k: share[k])
    # Roofline of the dominant kernel: its algorithmic intensity (~0.6 FLOP per algorithmic byte with
    # a skin, ~1.3 without) is far below the machine balance of ~12 FLOP/B (FP32 peak over the
    # measured copy bandwidth), so its roofline is HBM bandwidth.  The kernel does not reach it
    # because it is issue-bound (ncu: ~63 % issue active, DRAM ~37 %); the FP32 view of the same
    # launch is reported beside it.  With a skin the dominant kernel evaluates neighbour lists
    # (9 FLOP per listed pair + 13 per agent).
    st1 = sim.get_state(fields=())
    skin = float(params.get("skin", 0.0))
    rebuilds_timed = int(st1["grid_rebuilds"]) - int(st0["grid_rebuilds"])
    if skin > 0.0:
        fkernel = "force_list"
        per_agent = st1["list_entries"] / n
        flop_pa = 9.0 * per_agent + 13.0
        bytes_pa = KERNEL_BYTES["force_list"](per_agent)
    else:
        fkernel = "force_mixed"
        flop_pa = FORCE_FLOP_PER_AGENT(boxes_per_agent)
        bytes_pa = KERNEL_BYTES["force_mixed"](boxes_per_agent)
    force_ms = per_launch.get(fkernel, float("nan"))
    flops = flop_pa * n
    achieved_tf = flops / (force_ms * 1e-3) / 1e12
    alg_bytes = bytes_pa * n
    achieved_gb = alg_bytes / (force_ms * 1e-3) / 1e9
    mech_ms = sum(v[1] for k, v in ktimes.items() if k != "ftcs") / args.steps
    # The step's algorithmic bytes count the per-step rebuild the method defines (box = interaction
    # radius R, the largest diameter), whatever cadence runs: 4 S + 8 B_R per agent + 8 per voxel.
    R = float(np.max(inp["diameter"]))
    dims_R = [int(np.floor((float(np.max(inp[a])) - float(np.min(inp[a]))) / R)) + 1 for a in "xyz"]
    boxes_per_agent_R = float(np.prod(dims_R, dtype=np.float64)) / n
    step_bpa = STEP_BYTES_PER_AGENT(boxes_per_agent_R)
    step_bytes = step_bpa * n + 8.0 * 512 ** 3
    step_achieved = step_bytes / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": fkernel, "achieved": achieved_gb, "peak": peak,
                "unit": "GB/s", "frac": achieved_gb / peak, "traffic": measured_traffic(fkernel, n),
                "peak_kind": peak_kind, "alg_bytes_per_agent": bytes_pa,
                "alg_flop_per_byte": flop_pa / bytes_pa,
                "dominant_kernel_by_time": dom, "kernel_ms": force_ms,
                "step_ms": ms_per_step, "step_alg_bytes": step_bytes,
                "step_bytes_per_agent": step_bpa, "step_frac": step_achieved / peak,
                "fp32": {"achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved_tf / FP32_PEAK_TFLOPS, "alg_flop_per_agent": flop_pa,
                         "peak_kind": "derived (152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz)"}}

    diffusion = None
    if "ftcs" in per_launch:
        vox = 512 ** 3
        dms = per_launch["ftcs"]
        diffusion = {"grid": "512^3 FP32, FTCS + FP64 mass, co-stepped", "ms_per_step": dms,
                     "voxel_steps_per_s": vox / (dms * 1e-3), "alg_bytes_per_voxel": 8,
                     "achieved": 8 * vox / (dms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": 8 * vox / (dms * 1e-3) / 1e9 / peak}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(sim, inp, n, args.e2e_steps, stream)

    sim.close()
    ensemble = serving = plain = spheroid = stationary = oncology = neurite = mech_pool = None
    if rank == 0 and args.neurite_agents > 0:
        neurite = bench_neurite(args.neurite_agents, skin=args.neurite_skin)
    if rank == 0 and not args.no_small:
        plain = bench_plain()
        spheroid = bench_spheroid()
        oncology = bench_oncology()
        stationary = bench_stationary()
        mech_pool = bench_mech_pool()
    if rank == 0 and not args.no_ensemble:
        ensemble = bench_ensemble(args.ensemble_steps, args.ensemble_baseline_runs)
    if rank == 0 and args.serve_requests > 0:
        serving = bench_serving(args.serve_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(args.cpu_sample, 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 forces, f64 positions",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "agents": n, "grid": 512, "precision": "mixed",
                       "boxes_per_agent": round(boxes_per_agent, 4),
                       "tuned": ({"box_factor": knobs["box_factor"],
                                  "force_variant": knobs["force_variant"],
                                  "skin": knobs.get("skin", 0.0)} if knobs else None),
                       "sort_cadence": {"skin_um": skin,
                                        "grid_rebuilds_in_timed_steps": rebuilds_timed,
                                        "list_entries_per_agent": (st1["list_entries"] / n
                                                                   if skin > 0.0 else None)},
                       "skin_um": skin, "grid_rebuilds_timed": rebuilds_timed,
                       "list_entries_per_agent": (st1["list_entries"] / n if skin > 0.0 else 0.0),
                       "boxes_per_agent_R": round(boxes_per_agent_R, 4),
                       "cache": "inputs larger than L2 (agent state ~12 GB)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "step_roofline": {"bytes_per_agent_step": step_bpa,
                              "diffusion_bytes_per_step": 8 * 512 ** 3,
                              "achieved": step_achieved, "peak": peak, "unit": "GB/s",
                              "frac": step_achieved / peak, "nominal_peak": 7900.0,
                              "frac_of_nominal": step_achieved / 7900.0,
                              "mechanics_ms_per_step": mech_ms},
            "kernels_ms_per_launch": {k: round(v, 4) for k, v in per_launch.items()},
            "diffusion": diffusion,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
            "plain": plain, "spheroid": spheroid, "oncology": oncology, "stationary": stationary,
            "neurite": neurite, "ensemble": ensemble, "mech_pool": mech_pool,
            "serving": serving,
        }
        if mech_pool:
            line["mech_pool_ms_per_step"] = mech_pool["pool_ms_per_step"]
            line["mech_pool_alone_ms_per_step"] = mech_pool["alone_ms_per_step"]
        if serving:
            for key, arm in (("served", "served"), ("no_pool", "served_no_pool"),
                             ("alone", "one_at_a_time"), ("alone_plain", "one_at_a_time_plain")):
                line["serve_%s_sims_per_s" % key] = serving[arm]["sims_per_s"]
                line["serve_%s_p99_s" % key] = serving[arm]["p99_s"]
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_ensemble(steps, baseline_runs):
    """Batched SIR ensemble (256 runs x 20,000 persons, one persistent launch per step) against the
    same runs advanced one at a time with the single-run kernels (a sample of runs, scaled)."""
    import torch
    from paper_2006_06775_gb300 import bdm
    from paper_2006_06775_gb300 import tune
    ens = synth.sir_ensemble()
    choice = tune.tune_sir_batch([p for p, _ in ens], [inp for _, inp in ens],
                                 cache=tune.TuneCache(TUNED_PATH))
    ens = [(dict(p, sir_boxes=choice["sir_boxes"]), inp) for p, inp in ens]
    batch = bdm.Batch([p for p, _ in ens], history_steps=steps)
    for k, (_, inp) in enumerate(ens):
        batch.add_agents(k, inp["x"], inp["y"], inp["z"], inp["sir_state"])
    batch.step(3)  # warm-up (builds the device layout, captures the graph)
    batch.sync()
    t0 = time.perf_counter()
    batch.step(steps)
    batch.sync()
    t_batch = time.perf_counter() - t0
    agents = sum(len(inp["x"]) for _, inp in ens)
    # one at a time: the first `baseline_runs` runs, each alone, then scaled to all runs
    t_single = 0.0
    for k in range(baseline_runs):
        p, inp = ens[k]
        sim = bdm.Sim(p)
        sim.add_agents(inp["x"], inp["y"], inp["z"], sir_state=inp["sir_state"])
        sim.step(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(steps)
        sim.get_state(fields=())
        t_single += time.perf_counter() - t0
        sim.close()
    t_single *= len(ens) / baseline_runs
    batch.close()
    return {"workload": "256 SIR runs x 20,000 persons, 1000 um periodic cube",
            "steps": steps, "sir_boxes_per_axis": choice["sir_boxes"], "agent_steps_per_s": agents * steps / t_batch,
            "sims_per_s": len(ens) / t_batch, "ms_per_step": 1e3 * t_batch / steps,
            "one_at_a_time_agent_steps_per_s": agents * steps / t_single,
            "speedup_vs_one_at_a_time": t_single / t_batch,
            "one_at_a_time_sample_runs": baseline_runs,
            "cpu_baseline": sir_oracle_baseline()}


def _event_time_ms(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def bench_mech_pool(slots=64, steps=25, seed0=300):
    """Batched mechanics: 64 served-size simulations (1e3..32,768 agents, log-uniform like the
    pooled part of the served stream) advanced together in the slot pool, one graph replay of
    `steps` steps, against the same simulations stepped one after another on their own handles
    (one stream, each a `steps`-step graph replay).  Both rebuild the grid every step and give
    bit-identical states."""
    import math
    import torch
    from paper_2006_06775_gb300 import bdm
    g = np.random.default_rng(seed0)
    sizes = np.exp(g.uniform(math.log(1e3), math.log(32768), slots)).astype(np.int64)
    cases = [synth.served_mechanics(int(n), seed0 + k) for k, n in enumerate(sizes)]
    stream = torch.cuda.Stream()
    pool = bdm.MechBatch("mixed", slots=slots, slot_capacity=32768, stream=stream)
    for sl, (params, inp) in enumerate(cases):
        pool.load_sim(sl, params, inp["x"], inp["y"], inp["z"], inp["diameter"], 1 << 30)
    pool.step(steps)
    ms_pool = _event_time_ms(stream, lambda: pool.step(steps)) / steps
    pool.close()
    sims = []
    for params, inp in cases:
        sim = bdm.Sim(dict(params, skin=0.0), stream=stream)
        sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        sim.step(steps)
        sims.append(sim)

    def alone():
        for sim in sims:
            sim.step(steps)
    ms_alone = _event_time_ms(stream, alone) / steps
    for sim in sims:
        sim.close()
    agents = int(sizes.sum())
    return {"simulations": slots, "agents": agents, "steps": steps,
            "pool_ms_per_step": ms_pool, "alone_ms_per_step": ms_alone,
            "pool_agent_steps_per_s": agents / (ms_pool * 1e-3),
            "alone_agent_steps_per_s": agents / (ms_alone * 1e-3),
            "speedup": ms_alone / ms_pool, "pool_launches_per_step": 9}


def bench_plain(steps=10, reps=50):
    """Plain mechanics (4096 spheres in a 160 um cube): the FP64 check path and the mixed path,
    `steps`-step graph replays after one untimed replay."""
    from paper_2006_06775_gb300 import bdm
    params, inp = synth.plain_mechanics()
    out = {"workload": "plain mechanics: 4096 spheres, 160 um cube, d~U[8,12] um",
           "steps_per_replay": steps, "replays": reps}
    for prec in ("fp64", "mixed"):
        sim = bdm.Sim(dict(params, precision=prec))
        sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        sim.step(steps)

        def run():
            for _ in range(reps):
                sim.step(steps)
        ms = _event_time_ms(sim.stream, run)
        st = sim.get_state(fields=("neighbour_count",))
        sim.close()
        out[prec] = {"agent_steps_per_s": 4096 * steps * reps / (ms * 1e-3),
                     "ms_per_step": ms / (steps * reps)}
        if prec == "fp64":
            # the FP64 path is bound by GB300's FP64 arithmetic: its algorithmic FP64 work (9 per
            # candidate pair of the 27-box search, ~25 per contact) against the FP64 peak measured here
            nbox = int(np.prod(st["grid_dims"]))
            flop_pa = 9.0 * 27.0 * 4096 / nbox + 25.0 * float(st["neighbour_count"].mean())
            peak = fp64_peak_tflops()
            achieved = 4096 * flop_pa / (out[prec]["ms_per_step"] * 1e-3) / 1e12
            out[prec]["roofline"] = {"bound": "fp64", "alg_flop_per_agent": flop_pa,
                                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                     "frac": achieved / peak,
                                     "peak_kind": "measured: cuBLAS DGEMM 4096^3 on this GPU"}
    return out


def fp64_peak_tflops(n=4096, reps=5):
    """FP64 arithmetic peak of this GPU as cuBLAS reaches it (DGEMM), in TFLOP/s."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    stream = torch.cuda.current_stream()
    ms = _event_time_ms(stream, lambda: [torch.matmul(a, b) for _ in range(reps)])
    return 2.0 * n ** 3 * reps / (ms * 1e-3) / 1e12


def bench_oncology(steps=100, p_apoptosis=0.02, sigma=0.5):
    """The tumour spheroid with the oncology behaviours (apoptosis at step start, Brownian migration
    after the update) and secretion into the co-stepped 128^3 grid: `steps` steps after one
    warm-up step, timed on the device."""
    from paper_2006_06775_gb300 import bdm
    params, inp = synth.spheroid()
    params = dict(params, capacity=1 << 21, p_apoptosis=p_apoptosis, brownian_sigma=sigma)
    sim = bdm.Sim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(1)
    n0 = int(sim.get_state(fields=())["n"])
    ms = _event_time_ms(sim.stream, lambda: sim.step(steps))
    n1 = int(sim.get_state(fields=())["n"])
    sim.close()
    return {"workload": "tumour spheroid (512 cells) with apoptosis p = %g per step and Brownian "
                        "migration sigma = %g um, growth, division and secretion into a 128^3 grid"
                        % (p_apoptosis, sigma),
            "steps": steps, "agents_start": n0, "agents_end": n1, "ms_per_step": ms / steps}


NEURITE_BYTES_PER_AGENT = 92  # state read once (position 24, diameter 8, rest 8, mother 4,
                              # offset 24) + position written (24)
NEURITE_FORCE_BYTES_PER_AGENT = 92  # own record (40) + spring and bound (16) + key (4) read,
                                    # output record (32) written
# with neighbour lists the force kernel reads its own records (16 + 32), spring and bound (16), list
# length (4) and 4 B per listed entry, and writes the output record (32)
NEURITE_LIST_BYTES_PER_AGENT = lambda m: 100 + 4 * m
NEURITE_SKIN = 1.0  # neighbour-list skin (um) of the neuron-forest benchmark


def bench_neurite(n_agents=9_000_000, neurons=5000, steps=10, warmup=3, fp64_steps=2,
                  oracle_sample=20_000, skin=NEURITE_SKIN):
    """Neurite mechanics on the neuron forest (somata with apical and basal dendrite trees, the
    large pyramidal-cell run's 5000 cells and 9e6 agents), mixed precision: `steps` steps after
    `warmup`, timed on the device; per-kernel times from a separately profiled step; the FP64 check
    path timed over `fp64_steps` steps for comparison; the oracle on a bounded sample beside it."""
    from paper_2006_06775_gb300 import bdm
    # other sizes keep the density and the cells' size: neurons and cube side scale with n
    scale = n_agents / 9_000_000
    neurons = max(1, int(round(neurons * scale)))
    side = 2000.0 * scale ** (1.0 / 3.0)
    params, inp = synth.neuron_forest(neurons, n_agents, side=side)
    n = len(inp["x"])
    out = {"workload": "neuron forest: %d somata (10 um) with 1 apical + 3 basal dendrite trees, "
                       "%d agents, %.0f um cube, branching 0.038 / 0.006 per generation"
                       % (neurons, n, side),
           "agents": n, "steps": steps, "warmup": warmup, "precision": "mixed", "skin_um": skin}
    params = dict(params, capacity=n, box_capacity=4 * n + 4096)
    sim = bdm.Neurite(dict(params, precision="mixed", skin=skin))
    sim.set_agents(inp)
    sim.step(warmup)
    rb0 = sim.list_info()[0]
    ms = _event_time_ms(sim.stream, lambda: sim.step(steps))
    rb1, entries = sim.list_info()
    st = sim.get_state()
    # per-kernel times over as many steps as were timed (list and rebuild steps in their mix)
    sim.profile(True)
    sim.step(steps)
    kt = sim.kernel_times()
    sim.profile(False)
    sim.close()
    per = {k: v[1] / v[0] for k, v in kt.items()}
    peak, peak_kind = load_peaks()
    if skin > 0.0:
        fkernel = "nr_force_list"
        fbytes = NEURITE_LIST_BYTES_PER_AGENT(entries / n)
        out.update({"rebuilds_in_timed_steps": rb1 - rb0, "list_entries_per_agent": entries / n})
    else:
        fkernel, fbytes = "nr_force", NEURITE_FORCE_BYTES_PER_AGENT
    fms = per.get(fkernel, float("nan"))
    achieved = fbytes * n / (fms * 1e-3) / 1e9
    step_achieved = NEURITE_BYTES_PER_AGENT * n / (ms / steps * 1e-3) / 1e9
    out.update({"ms_per_step": ms / steps, "agent_steps_per_s": n * steps / (ms * 1e-3),
                "neighbours_per_agent": float(np.mean(st["neighbour_count"])),
                "L_um": st["L"],
                "kernels_ms_per_launch": {k: round(v, 4) for k, v in per.items()},
                "roofline": {"bound": "hbm", "kernel": fkernel, "achieved": achieved,
                             "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "peak_kind": peak_kind, "kernel_ms": fms,
                             "alg_bytes_per_agent": fbytes,
                             "traffic": measured_traffic(fkernel, n)},
                "step_roofline": {"bytes_per_agent_step": NEURITE_BYTES_PER_AGENT,
                                  "achieved": step_achieved, "peak": peak, "unit": "GB/s",
                                  "frac": step_achieved / peak}})
    if fp64_steps > 0:
        sim = bdm.Neurite(dict(params, precision="fp64"))
        sim.set_agents(inp)
        sim.step(1)
        ms64 = _event_time_ms(sim.stream, lambda: sim.step(fp64_steps))
        sim.close()
        out["fp64_ms_per_step"] = ms64 / fp64_steps
    if oracle_sample > 0:
        out["cpu_baseline"] = neurite_oracle_baseline(oracle_sample)
    return out


def bench_stationary(n=10_000_000, steps=10, warmup=3, skin=2.5):
    """A settled lattice around a relaxing ball (10% of 10^7 agents), neighbour lists with a 2.5 um
    skin: steps with stationary warps skipped against the same steps evaluating every agent (the
    results are identical).  `skipped_per_list_step` is the fraction of agents skipped on a list
    step; `list_kernel_ms_per_list_step` times the list kernel (with the skip, plus the kernel that
    picks the warps) on list steps alone, from a separately profiled run."""
    from paper_2006_06775_gb300 import bdm
    params, inp = synth.settled_mechanics(n, 0.1)
    R = float(np.max(inp["diameter"]))
    params = dict(params, interaction_radius=R, skin=skin)
    out = {"workload": "settled lattice (spacing 14 um) around a ball of overlapping agents at 0.3 "
                       "volume fraction holding 10%% of %d agents; skin %.1f um" % (n, skin),
           "steps": steps, "warmup": warmup}
    for key, skip in (("skip", 1), ("evaluate_all", 0)):
        sim = bdm.Sim(dict(params, skip_stationary=skip))
        sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
        sim.step(warmup)
        s0 = sim.get_state(fields=())
        ms = _event_time_ms(sim.stream, lambda: sim.step(steps))
        s1 = sim.get_state(fields=())
        # the list kernel on list steps alone (events around each kernel, one step at a time)
        sim.profile(True)
        prev, list_ms, list_steps = {}, 0.0, 0
        for _ in range(steps):
            r0 = int(sim.get_state(fields=())["grid_rebuilds"])
            sim.step(1)
            r1 = int(sim.get_state(fields=())["grid_rebuilds"])
            cur = {k: v[1] for k, v in sim.kernel_times().items()}
            d = {k: cur[k] - prev.get(k, 0.0) for k in cur}
            prev = cur
            if r1 == r0:
                list_ms += d.get("force_list", 0.0) + d.get("still_warps", 0.0)
                list_steps += 1
        sim.profile(False)
        sim.close()
        rebuilds = int(s1["grid_rebuilds"]) - int(s0["grid_rebuilds"])
        skipped = int(s1["stationary_skipped"]) - int(s0["stationary_skipped"])
        out[key] = {"ms_per_step": ms / steps, "agent_steps_per_s": n * steps / (ms * 1e-3),
                    "grid_rebuilds": rebuilds,
                    "skipped_per_list_step": skipped / max(1, n * (steps - rebuilds)),
                    "list_kernel_ms_per_list_step": list_ms / max(1, list_steps)}
    out["speedup"] = out["evaluate_all"]["ms_per_step"] / out["skip"]["ms_per_step"]
    out["list_step_kernel_speedup"] = (out["evaluate_all"]["list_kernel_ms_per_list_step"] /
                                       out["skip"]["list_kernel_ms_per_list_step"])
    return out


def bench_spheroid(max_agents=1_000_000, max_steps=160):
    """Tumour spheroid: 512 cells growing and dividing to about 10^6, each secreting into a 128^3
    grid co-stepped by FTCS.  The agent count of every step is recorded in an untimed run; the same
    seeded run is then timed step by step (one graph replay per step) after one warm-up step."""
    from paper_2006_06775_gb300 import bdm
    params, inp = synth.spheroid()
    params = dict(params, capacity=1 << 21)
    counts = []
    sim = bdm.Sim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    while len(counts) < max_steps:
        sim.step(1)
        counts.append(int(sim.get_state(fields=())["n"]))
        if counts[-1] >= max_agents:
            break
    sim.close()
    import torch
    sim = bdm.Sim(params)
    sim.add_agents(inp["x"], inp["y"], inp["z"], inp["diameter"])
    sim.step(1)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(len(counts))]

    def run():
        marks[0].record(sim.stream)
        for k in range(1, len(counts)):
            sim.step(1)
            marks[k].record(sim.stream)
    ms = _event_time_ms(sim.stream, run)
    st = sim.get_state(fields=())
    sim.close()
    assert int(st["n"]) == counts[-1], (st["n"], counts[-1])
    step_ms = [marks[k - 1].elapsed_time(marks[k]) for k in range(1, len(counts))]
    by_n = {}
    for k in range(1, len(counts)):
        by_n.setdefault(counts[k], []).append(step_ms[k - 1])
    # closed-form mass: secretion q per agent, then decay (zero-flux walls conserve the rest)
    keep = 1.0 - params["decay"] * params["dt_diffusion"]
    mass = 0.0
    for n in counts:
        mass = keep * (mass + params["secretion"] * n)
    agent_steps = float(sum(counts[1:]))
    return {"workload": "tumour spheroid: 512 cells, growth 100 um^3/step, division at 14 um, "
                        "secretion into a 128^3 FTCS grid",
            "steps": len(counts) - 1, "agents_after_first_step": counts[0],
            "agents_final": counts[-1], "agent_steps": agent_steps,
            "agent_steps_per_s": agent_steps / (ms * 1e-3), "ms_per_step": ms / (len(counts) - 1),
            "by_agents": [{"agents": n, "steps": len(v), "ms_per_step": sum(v) / len(v),
                           "agent_steps_per_s": n * len(v) / (sum(v) * 1e-3)}
                          for n, v in sorted(by_n.items())],
            "mass_total": st["mass_total"], "mass_closed_form": mass,
            "mass_rel_error": abs(st["mass_total"] - mass) / mass}


def bench_serving(count):
    """Served request stream (Poisson 200/s, sizes log-uniform 1e3..1e6, 50..500 steps, 70%
    mechanics / 30% SIR, 150 GB budget).  Arms on the same trace:
      served            mechanics up to 32,768 agents in a 64-slot pool (one launch sequence per
                        step for all of them), larger ones and SIR on own handles over 16 streams,
                        mechanics handles with 2.5 um neighbour lists
      served_no_pool    the same without the pool (every request on its own handle)
      one_at_a_time     FIFO, one simulation at a time, mechanics with the same 2.5 um lists
      one_at_a_time_plain   the same with the plain kernels (grid rebuilt every step)"""
    from paper_2006_06775_gb300 import serve
    reqs = synth.request_stream(count=count)
    payloads = {r.rid: serve.payload(r) for r in reqs}
    warm = [synth.Request(10 ** 6 + k, 0.0, kind, 2000, 10, 7 + k) for k, kind in
            enumerate(("mechanics", "sir", "mechanics"))]
    warm[2] = synth.Request(10 ** 6 + 2, 0.0, "mechanics", 200_000, 10, 9)
    wp = {r.rid: serve.payload(r) for r in warm}
    serve.run_one_at_a_time(serve.GpuExecutor(1), warm, lambda r: wp[r.rid])
    serve.run_one_at_a_time(serve.GpuExecutor(1, mechanics_skin=2.5), warm, lambda r: wp[r.rid])
    pool_slots, pool_cap, chunk = 64, 32768, 25

    def served_arm(pool):
        ex = serve.GpuExecutor(streams=16, mechanics_skin=2.5, pool_slots=pool_slots if pool else 0,
                               pool_capacity=pool_cap, pool_chunk=chunk)
        if pool:
            ex.warm_pool(wp[warm[0].rid], 2 * chunk)
        jobs = serve.Server(ex, budget_bytes=150e9, max_active=64, chunk=chunk).run(
            reqs, lambda r: payloads[r.rid])
        ex.shutdown()
        return jobs

    served = served_arm(True)
    out = {"trace": "all %d requests of the Poisson stream (seed 4)" % count,
           "served": serve.summarize(served)}
    out["served"]["pooled_requests"] = sum(j.pooled for j in served)
    out["served"]["pool"] = {"slots": pool_slots, "slot_capacity": pool_cap, "chunk_steps": chunk,
                             "launches_per_step": 9}
    out["served_no_pool"] = serve.summarize(served_arm(False))
    out["one_at_a_time"] = serve.summarize(serve.run_one_at_a_time(
        serve.GpuExecutor(streams=1, mechanics_skin=2.5), reqs, lambda r: payloads[r.rid]))
    out["one_at_a_time_plain"] = serve.summarize(serve.run_one_at_a_time(
        serve.GpuExecutor(streams=1), reqs, lambda r: payloads[r.rid]))
    out["mechanics_skin_um"] = 2.5
    out["streams"] = 16
    return out


def run_e2e(sim, inp, n, steps, stream):
    """End to end through the C ABI: pinned host inputs -> add agents + grid -> `steps` steps ->
    positions and mass back to pinned host memory, per job."""
    import torch
    from paper_2006_06775_gb300 import bdm

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t

    hx, hy, hz = pinned(inp["x"]), pinned(inp["y"]), pinned(inp["z"])
    hd = pinned(inp["diameter"])
    hg = pinned(inp["grid"].reshape(-1))
    outs = {a: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy() for a in ("x", "y", "z")}
    h2d = n * (3 * 8 + 4) + hg.numel() * 4
    d2h = n * 3 * 8 + 8
    times = []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.reset()
        sim.add_agents(hx.numpy(), hy.numpy(), hz.numpy(), hd.numpy())
        sim.set_grid(hg.numpy())
        sim.step(steps)
        st = sim.get_state(fields=("x", "y", "z"), out=outs)
        times.append(time.perf_counter() - t0)
        assert st["n"] == n
    t = min(times)
    return {"value": n * steps / t, "unit": METRIC, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "steps_per_job": steps,
            "job_seconds": t}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--agents", type=int, default=100_000_000)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-sample", type=int, default=20_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", action="store_true",
                    help="re-measure the tunable knobs on this workload and cache the choice")
    ap.add_argument("--skin", type=float, default=None,
                    help="neighbour-list skin in um (0: grid rebuilt every step); default: tuned")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the plain-mechanics and tumour-spheroid sub-benchmarks")
    ap.add_argument("--ensemble-steps", type=int, default=1000)
    ap.add_argument("--ensemble-baseline-runs", type=int, default=16)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--neurite-agents", type=int, default=9_000_000,
                    help="agents of the neuron-forest sub-benchmark (0: skip it)")
    ap.add_argument("--neurite-skin", type=float, default=NEURITE_SKIN,
                    help="neighbour-list skin (um) of the neuron-forest sub-benchmark (0: rebuild every step)")
    ap.add_argument("--neurite-only", action="store_true",
                    help="run only the neuron-forest sub-benchmark and print its object")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.neurite_only:
        print(json.dumps({"neurite": bench_neurite(args.neurite_agents, steps=args.steps,
                                                   warmup=args.warmup, skin=args.neurite_skin)}),
              flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
