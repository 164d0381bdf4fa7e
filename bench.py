"""Benchmark: SPH pair interactions per second (density + force) of the
sorted cell-pair path on one GB300, with the FP32 roofline fraction of the
dominant sweep kernel and the forward+adjoint / forward time ratio.

One step = the whole path on one batch: decomposition build (Morton sort,
octree, tasks, 13-direction sorts), density with the smoothing-length
solve, ghost, force, and the adjoint of L = sum (rho - 1)^2 + sum |a|^2.
Units per step = directed density interactions (r < h_i, self included) +
unordered force pairs (r < max(h_i, h_j)), both at the solved h.

Default workload: the large clustered box, 256^3 particles drawn from a
lognormal density field (h spans ~1300x), the largest single-GPU
configuration.  The line also carries the plain-FP32 forward (no
compensated sums) on the same GPU, a small full-oracle parity check with
per-quantity errors (h, rho, a, du/dt, and the three gradients), short
timings of the other workloads, the naive-versus-sorted ablation and the
viscous force (both on the 128^3 multi-resolution box).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH pair interactions/s (density+force), % of FP32 roofline; fwd+adj/fwd time"
UNIT = "interactions/s"
# canonical FP32-pipe instructions per unit: density and d2rho/dh2 per
# directed interaction, force and the two adjoints per unordered pair
# counted once (the first and third as fixed for this path; the others
# derived the same way from the minimal arithmetic of each pair term)
INSTR = {0: 18.0, 1: 24.0, 2: 40.0, 3: 100.0, 4: 65.0}
# the kernels behind each phase: the density and force phases sweep the
# sorted cell pairs (the force sweep also records the pair lists); the later
# phases over the force pairs read those lists (a masked sweep takes the
# particles whose list overflowed)
PHASE_KERNELS = {0: "k_sweep<PDensity>", 1: "k_listeval<PDensityD2>", 2: "k_sweep<PForce>",
                 3: "k_listeval<PForceAdj>", 4: "k_listeval<PDensityAdj>"}
BUILD_STAGES = ["morton_order", "h_estimate", "octree", "pair_tasks", "blocks_and_block_sorts",
                "list_merge", "interaction_lists", "node_h_max"]
PHASE_NAMES = {0: "density", 1: "density_d2", 2: "force", 3: "force_adjoint", 4: "density_adjoint"}
LANES = 128  # FP32 lanes per SM (four sub-partitions of 32)


def workload(name):
    """The synthetic workloads (synth/configs.py); batched ones carry
    'offsets' / 'boxes' for sph_build_batch."""
    import synth.configs as C
    if name == "multires128":
        return C.multires(128, seed=2)
    if name == "multires64":
        return C.multires(64, seed=2)
    if name == "lattice16":
        return C.uniform_lattice(16, seed=1)
    if name == "sinusoid64":
        return C.sinusoid(64, seed=4)
    if name == "batch64":
        return C.concat_boxes(C.batch_boxes(64, seed=3))
    if name == "lognormal256":
        return C.lognormal(256, seed=5, sigma=4.0)
    if name == "lognormal128":  # the same field law at 1/8 of the particles (profiling case)
        return C.lognormal(128, seed=5, sigma=4.0)
    if name == "zeldovich256":
        return C.zeldovich(256, seed=5, amp=8.0)
    raise SystemExit(f"unknown workload {name}")


def profiled_traffic(phase_name, units_per_launch):
    """DRAM bytes per launch of a sweep phase: the bytes per accepted unit
    from the committed ncu summary of a smaller case of the same field law
    (dram__bytes_read.sum + dram__bytes_write.sum over all the phase's
    launches of one step, divided by the units those launches accepted),
    times this run's units per launch; None when the sweep kernel source
    changed since that capture."""
    import hashlib
    import re
    src = os.path.join(ROOT, "paper_1404_2303_gb300", "csrc", "sweep.cu")
    summ = os.path.join(ROOT, "profiles", "traffic_sweeps_lognormal128.md")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        text = open(summ).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256: ([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_unit\[" + re.escape(phase_name) + r"\]: ([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != sha:
        return None
    return float(t.group(1)) * units_per_launch


def build_rate(st, n, pk, pk_kind):
    """One decomposition build against the HBM copy bandwidth: algorithmic
    bytes n (24 + 12 + 8) (positions in, keys, FP32 relative positions and
    permutation out) + 2 x 13 x 8 n (the 13 sorted lists of (key, index)
    written and read once) over the mean build time of the profiled pass
    (stages timed with a stream synchronisation at each boundary)."""
    builds = max(1, int(st.get("builds", 0)))
    ms = sum(st["build_ms"]) / builds
    alg = float(n) * (24 + 12 + 8) + 2.0 * 13 * 8 * float(n)
    gbs = alg / (ms / 1e3) / 1e9 if ms > 0 else None
    peak = float(pk.get("hbm_gbs", 6800.0))
    return {"ms_per_build": ms, "builds_in_profiled_pass": builds, "algorithmic_bytes": alg,
            "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak if gbs else None,
            "peak_source": f"hbm_gbs of {pk_kind} peaks"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _subcube(x, rng, side=0.375, inner=0.125):
    """Indices of the particles inside a cube of the given side around a
    random centre, positions translated (periodically) so that the cube is
    centred in the unit box, and the indices of those in the concentric
    inner cube.  Every quantity of an inner particle depends only on
    particles within twice the largest smoothing length of it, so with
    (side - inner)/2 >= 2 h_max the oracle run on the cube alone gives the
    whole box's values there."""
    c = rng.random(3)
    y = np.mod(x - c + 0.5, 1.0)
    lo, hi = 0.5 - side / 2, 0.5 + side / 2
    inside = np.all((y >= lo) & (y < hi), axis=1)
    idx = np.nonzero(inside)[0]
    ilo, ihi = 0.5 - inner / 2, 0.5 + inner / 2
    core = np.all((y[idx] >= ilo) & (y[idx] < ihi), axis=1)
    return idx, y[idx], np.nonzero(core)[0]


def oracle_sample_rate(d, seed=0, sample=None, cube_above=2_500_000):
    """Time the FP64 oracle on a bounded random sample of the workload:
    units of the sampled particles (their directed density interactions
    plus half their force partners) per second of oracle time.  Above
    cube_above particles the oracle runs on a cube of side 3/8 of the box
    around a random centre (its neighbour structures over the whole set
    alone would take minutes) and the sample is drawn from the concentric
    cube of side 1/8, whose values the larger cube determines exactly while
    h_max <= 1/16."""
    from oracle import sph_oracle as O
    rng = np.random.default_rng(seed)
    S = sample or 256
    x, m, u, v = d["x"], d["m"], d["u"], d["v"]
    base = 0
    gidx = None
    if "offsets" in d:  # independent boxes: sample inside one of them
        off = d["offsets"]
        b = int(rng.integers(len(off) - 1))
        sl = slice(off[b], off[b + 1])
        x, m, u, v = x[sl], m[sl], u[sl], v[sl]
        base = int(off[b])
    if x.shape[0] > cube_above:
        gidx, xc, core = _subcube(x, rng)
        x, m, u, v = xc, m[gidx], u[gidx], v[gidx]
        pool = core
    else:
        pool = np.arange(x.shape[0])
    S = min(S, pool.size)
    idx = np.sort(rng.choice(pool, S, replace=False))
    t0 = time.perf_counter()
    r = O.evaluate_sample(x, m, u, idx, v=v)
    dt = time.perf_counter() - t0
    units = float(np.sum(r["count"]) + 0.5 * np.sum(r["force_count"]))
    glob = base + (gidx[idx] if gidx is not None else idx)
    where = (f"a cube of side 3/8 ({x.shape[0]} particles) around a random centre, sample "
             "from its central cube of side 1/8" if gidx is not None else "the whole set")
    return dict(value=units / dt, seconds=dt, sample=int(S), units=units, ref=r, index=glob,
                where=where)


def max_over_ranks(x, device=None):
    """The largest of every rank's x (all ranks get it); x itself on one rank.
    The timed region of a step ends when the slowest replica ends."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_per_step):
    """Whole-job throughput of `world` replicas that each process
    units_per_rank per step, the step lasting ms_per_step (max over ranks)."""
    return units_per_rank * world / (ms_per_step / 1e3)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    d = workload(args.workload)
    S = args.ref_sample
    vals, secs = [], []
    where = ""
    for k in range(args.warmup + args.steps):
        r = oracle_sample_rate(d, seed=k, sample=S)
        where = r["where"]
        if k >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
    v = float(np.mean(vals))
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "particles": int(d["x"].shape[0]),
                   "sample_per_step": S},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{S} random particles of {args.workload} per step ({where}), "
                                   "evaluated from scratch (h solve of the sample and its force "
                                   "partners, density, force); units = their density "
                                   "interactions + half their force partners"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _t(a, dev, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a), device=dev)
    return t.to(dtype) if dtype is not None else t


def _step_fn(sph, d, stream, ev=None, adjoint=True):
    """One step of the path on workload d through the public API; with ev,
    CUDA events on the launch stream mark the forward / adjoint split."""
    import torch
    batched = "offsets" in d

    def step(pos, m, u, vel):
        if ev is not None:
            ev.setdefault("f0", []).append(torch.cuda.Event(enable_timing=True))
            ev["f0"][-1].record(stream)
        if batched:
            sph.build_batch(pos, d["offsets"], d["boxes"])
        else:
            sph.build(pos)
        den = sph.density(m)
        acc, dudt, _ = sph.force(u, vel)
        if ev is not None:
            ev.setdefault("f1", []).append(torch.cuda.Event(enable_timing=True))
            ev["f1"][-1].record(stream)
        if not adjoint:
            return den, acc, dudt, None, None, None
        g_pos, g_m, g_u = sph.adjoint(2.0 * (den["rho"] - 1.0), 2.0 * acc, None)
        if ev is not None:
            ev.setdefault("a1", []).append(torch.cuda.Event(enable_timing=True))
            ev["a1"][-1].record(stream)
        return den, acc, dudt, g_pos, g_m, g_u
    return step


def _count_units(sph, m, u, vel, h):
    sph.density_fixed_h(m, h, count=True)
    sph.force(u, vel, count=True)
    st = sph.stats()
    return st["density_interactions"], st["force_pairs"]


def other_workload(name, dev, params, warmup=2, steps=3):
    """Short timing of another configuration: full steps (build, density with
    the h solve, force, adjoint) between device events."""
    import torch
    from paper_1404_2303_gb300 import SPH
    d = workload(name)
    pos, m = _t(d["x"], dev, torch.float64), _t(d["m"], dev)
    u, vel = _t(d["u"], dev), _t(d["v"], dev)
    sph = SPH(**params)
    stream = torch.cuda.current_stream()
    step = _step_fn(sph, d, stream)
    for _ in range(warmup):
        out = step(pos, m, u, vel)
    torch.cuda.synchronize()
    dens, fp = _count_units(sph, m, u, vel, out[0]["h"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(pos, m, u, vel)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = sph.stats()
    sph.close()
    return {"particles": int(d["x"].shape[0]), "ms_per_step": ms, "value": (dens + fp) / (ms / 1e3),
            "units_per_step": int(dens + fp), "newton_iters": st["newton_iters"],
            "rebuilds": st["rebuilds"], "steps": steps}


def small_parity(dev, n=4096, seed=29):
    """Full-oracle parity of one small clumped box with random velocities:
    per-quantity errors of h, rho, a, du/dt and of the gradients of
    L = sum (rho - 1)^2 + sum |a|^2 + sum w du/dt."""
    import torch
    from oracle import sph_oracle as O
    from paper_1404_2303_gb300 import SPH
    import synth.configs as C
    d = C.random_box(n, seed, "clumped", v_sigma=0.1)
    sph = SPH()
    sph.build(_t(d["x"], dev, torch.float64))
    den = sph.density(_t(d["m"], dev))
    acc, dudt, _ = sph.force(_t(d["u"], dev), _t(d["v"], dev))
    w = np.random.default_rng(3).normal(size=n).astype(np.float32)
    g = sph.adjoint(2.0 * (den["rho"] - 1.0), 2.0 * acc, _t(w, dev))
    torch.cuda.synchronize()
    ref = O.evaluate(d["x"], d["m"], d["u"], v=d["v"], h_guess=0.1)
    f64 = lambda t: t.double().cpu().numpy()
    gref = O.gradient(ref, d["x"], d["m"], d["u"], d["v"].astype(np.float64),
                      2.0 * (f64(den["rho"]) - 1.0), 2.0 * f64(acc), w.astype(np.float64))
    rms = lambda a: float(np.sqrt(np.mean(np.sum(np.atleast_2d(a.T).T ** 2, axis=-1)))) \
        if a.ndim > 1 else float(np.sqrt(np.mean(a ** 2)))
    out = {"particles": n, "config": "uniform + Gaussian clumps, velocities N(0, 0.1^2)",
           "max_rel_err_h": float(np.max(np.abs(f64(den["h"]) / ref["h"] - 1))),
           "max_rel_err_rho": float(np.max(np.abs(f64(den["rho"]) / ref["rho"] - 1))),
           "max_err_acc_over_rms": float(np.max(np.linalg.norm(f64(acc) - ref["a"], axis=1))
                                         / rms(ref["a"])),
           "max_err_dudt_over_rms": float(np.max(np.abs(f64(dudt) - ref["dudt"])) / rms(ref["dudt"]))}
    for name, got, want in (("x", g[0], gref["g_x"]), ("m", g[1], gref["g_m"]), ("u", g[2], gref["g_u"])):
        gg = f64(got).reshape(want.shape)
        r = float(np.sqrt(np.mean(want ** 2)))
        out[f"grad_{name}_rel_l2"] = float(np.linalg.norm(gg - want) / np.linalg.norm(want))
        out[f"grad_{name}_max_elem"] = float(np.max(np.abs(gg - want) / (r + np.abs(want))))
    out["tolerances"] = {"h": 1e-5, "rho": 1e-5, "acc": 1e-4, "dudt": 1e-4, "grad_rel_l2": 1e-3,
                         "grad_elem": 1e-3}
    sph.close()
    return out


def _oracle_box(name):
    import synth.configs as C
    if name == "lattice16":
        return C.uniform_lattice(16, seed=1), "the whole 16^3 jittered lattice (4096 particles)"
    return C.sinusoid(64, seed=4), "the whole 64^3 sinusoid box (262,144 particles)"


def oracle_full_rate(name="lattice16"):
    """The oracle on a whole box (its neighbour queries on all host cores):
    units (directed density interactions + unordered force pairs) per
    second, tree build included."""
    from oracle import sph_oracle as O
    d, what = _oracle_box(name)
    t0 = time.perf_counter()
    O.Neighbours(d["x"], 1.0)  # the neighbour tree alone, timed apart
    t_tree = time.perf_counter() - t0
    t0 = time.perf_counter()
    f = O.evaluate(d["x"], d["m"], d["u"], h_guess=d["h_guess"])
    dt = time.perf_counter() - t0
    units = float(f["count"].sum() + 0.5 * f["force_count"].sum())
    return {"value": units / dt, "seconds": dt, "units": units, "sample": what + ", tree build included",
            "tree_build_seconds": t_tree,
            "value_without_tree_build": units / max(dt - t_tree, 1e-9)}


def _one_core_rate(name, q):
    os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    q.put(oracle_full_rate(name))


def oracle_full_rate_one_core(name="lattice16"):
    """The same on one host core: a spawned process pinned to one CPU (the
    neighbour-query threads then share it)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_one_core_rate, args=(name, q))
    pr.start()
    r = q.get(timeout=600)
    pr.join()
    r["cores"] = 1
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="lognormal256")
    ap.add_argument("--side-workload", default="multires128",
                    help="workload of the naive-versus-sorted ablation and the viscous force")
    ap.add_argument("--others", default="multires128,batch64,sinusoid64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--oracle-c4", action="store_true",
                    help="also time the oracle on the whole 64^3 sinusoid box, all cores and one")
    ap.add_argument("--kahan", type=int, default=1)
    ap.add_argument("--block-max", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ablation, the viscous force, the other workloads and the small "
                         "full-oracle parity check")
    ap.add_argument("--profile-step", action="store_true",
                    help="for kernel profilers: run --warmup steps, then one step with the h "
                         "iteration as a host loop (every sweep a separate launch), and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import __graft_entry__ as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    g.build()
    from paper_1404_2303_gb300 import SPH

    d = workload(args.workload)
    n = d["x"].shape[0]
    dev = torch.device("cuda", local)
    # inputs resident in HBM
    pos = _t(d["x"], dev, torch.float64)
    m, u, vel = _t(d["m"], dev), _t(d["u"], dev), _t(d["v"], dev)
    params = {"kahan": args.kahan}
    if args.block_max:
        params["block_max"] = args.block_max
    if args.warps:
        params["warps_per_cta"] = args.warps
    stream = torch.cuda.current_stream()
    if args.profile_step:
        sp = SPH(use_graph=0, **params)
        step = _step_fn(sp, d, stream)
        for _ in range(args.warmup + 1):
            den = step(pos, m, u, vel)[0]
        torch.cuda.synchronize()
        print(json.dumps({"profile_step": args.workload, "iters": den["iters"]}), flush=True)
        return 0
    sph = SPH(**params)

    # sweep launch shape from the project's autotuner, timed on this workload
    tuned = None
    if not args.no_tune:
        from paper_1404_2303_gb300.autotune import tune
        shape, timings = tune(pos, m, u, vel, offsets=d.get("offsets"), boxes=d.get("boxes"),
                              use_cache=False, **params)
        sph.set_sweep_config(**shape)
        tuned = {"shape": shape, "candidates": len(timings)}
    else:
        shape = None

    ev = {}
    step = _step_fn(sph, d, stream, ev)
    for _ in range(args.warmup):
        out = step(pos, m, u, vel)
    ev.clear()
    torch.cuda.synchronize()
    # units per step (counted at the solved h, outside the timed region)
    den = out[0]
    dens_units, force_units = _count_units(sph, m, u, vel, den["h"])
    units = dens_units + force_units

    def timed(profile, steps):
        """steps full steps between a barrier + synchronize on both sides."""
        ev.clear()
        sph.profile(profile)
        launches0 = sph.launch_count()
        clk = ClockSampler(local)
        clk.start()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            step(pos, m, u, vel)
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = clk.stop()
        launches = sph.launch_count() - launches0
        ms = t0.elapsed_time(t1) / steps
        fwd = float(np.mean([a.elapsed_time(b) for a, b in zip(ev["f0"], ev["f1"])]))
        adj = float(np.mean([a.elapsed_time(b) for a, b in zip(ev["f1"], ev["a1"])]))
        stats = sph.stats()
        sph.profile(False)
        ms = max_over_ranks(ms, dev)
        return dict(ms=ms, fwd=fwd, adj=adj, launches=launches, stats=stats, clocks=clocks,
                    steps=steps)

    # production pass: device-side graphs for the h iteration, no profiling
    prod = timed(False, args.steps)
    # profiled pass: every sweep launch bracketed by CUDA events on its stream
    prof = timed(True, max(1, min(args.steps, 3)))
    ms, fwd_ms, adj_ms, launches, clocks = (prod["ms"], prod["fwd"], prod["adj"], prod["launches"],
                                            prod["clocks"])
    st = prof["stats"]
    value = job_rate(units, world, ms)

    # ---- the plain-FP32 forward (no compensated sums) on the same GPU
    sp32 = SPH(**dict(params, kahan=0))
    if shape:
        sp32.set_sweep_config(**shape)
    step32 = _step_fn(sp32, d, stream, adjoint=False)
    step32(pos, m, u, vel)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out32 = step32(pos, m, u, vel)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd32_ms = e0.elapsed_time(e1) / args.steps
    rho_k, rho_p = den["rho"].double(), out32[0]["rho"].double()
    plain32 = {"fwd_ms": fwd32_ms, "value": units / (fwd32_ms / 1e3),
               "compensated_fwd_ms": fwd_ms,
               "max_rel_diff_rho_vs_compensated": float(((rho_p - rho_k).abs() / rho_k).max())}
    sp32.close()

    # ---- end to end through the public API: pinned host inputs, host outputs
    hpos = torch.tensor(d["x"], dtype=torch.float64).pin_memory()
    hm = torch.tensor(d["m"]).pin_memory()
    hu = torch.tensor(d["u"]).pin_memory()
    hv = torch.tensor(d["v"]).pin_memory()
    outs_host = None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_e2e = _step_fn(sph, d, stream)
    e0.record(stream)
    for _ in range(args.steps):
        dp = hpos.to(dev, non_blocking=True)
        dm = hm.to(dev, non_blocking=True)
        du_ = hu.to(dev, non_blocking=True)
        dv = hv.to(dev, non_blocking=True)
        den2, acc, dudt, g_pos, g_m, g_u = step_e2e(dp, dm, du_, dv)
        outs_host = [t.to("cpu", non_blocking=True)
                     for t in (den2["rho"], den2["h"], acc, dudt, g_pos, g_m, g_u)]
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    h2d = sum(t.numel() * t.element_size() for t in (hpos, hm, hu, hv))
    d2h = sum(t.numel() * t.element_size() for t in outs_host)

    # ---- roofline of the dominant sweep kernel
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_alu = sms * LANES * sm_max * 1e6  # FP32 lane-instructions/s at the maximum SM clock
    phase_ms = st["sweep_ms"]
    dom = int(np.argmax(phase_ms[:5]))
    kernels = {}
    for ph in range(5):
        if st["sweep_launches"][ph] == 0:
            continue
        L = st["sweep_launches"][ph]
        u_ph = st["sweep_units"][ph]
        if ph >= 2:
            u_ph = u_ph / 2.0  # ordered -> unordered pairs
        kernels[PHASE_NAMES[ph]] = {
            "kernel": PHASE_KERNELS[ph],
            "launches_per_step": L / prof["steps"], "ms_per_launch": phase_ms[ph] / L,
            "units_per_launch": u_ph / L,
            "share_of_step": phase_ms[ph] / prof["steps"] / prof["ms"],
            "frac_fp32": (u_ph / L) * INSTR[ph] / (phase_ms[ph] / L / 1e3) / peak_alu,
        }
    roof = None
    dname = PHASE_NAMES[dom]
    if dom in INSTR and st["sweep_launches"][dom] > 0:
        k = kernels[dname]
        achieved = k["units_per_launch"] * INSTR[dom] / (k["ms_per_launch"] / 1e3)
        roof = {"kernel": PHASE_KERNELS[dom], "bound": "alu", "achieved": achieved / 1e12,
                "peak": peak_alu / 1e12, "unit": "T FP32-instr/s",
                "frac": achieved / peak_alu, "traffic": profiled_traffic(dname, k["units_per_launch"]),
                "peak_source": f"{sms} SMs (device attribute) x {LANES} FP32 lanes x "
                               f"{sm_max:.0f} MHz (sm_max_mhz of {pk_kind} peaks)",
                "instr_per_unit": INSTR[dom]}

    extras = {}
    if rank == 0 and not args.no_extras:
        side = workload(args.side_workload)
        spos = _t(side["x"], dev, torch.float64)
        sm_, su, sv = _t(side["m"], dev), _t(side["u"], dev), _t(side["v"], dev)
        sb = "offsets" in side
        hs = SPH(**params)
        if sb:
            hs.build_batch(spos, side["offsets"], side["boxes"])
        else:
            hs.build(spos)
        h_sol = hs.density(sm_)["h"]
        # ---- ablation of the sorting (Section 3.3): the naive cell-pair loop
        # over the same tasks, one density and one force sweep at the solved h
        ablation = {"workload": args.side_workload}
        for mode, name in ((1, "sorted"), (0, "naive")):
            sa = SPH(sorted_sweep=mode, pair_list_cap=0, **params)
            if sb:
                sa.build_batch(spos, side["offsets"], side["boxes"], h_guess=h_sol)
            else:
                sa.build(spos, h_guess=h_sol)
            sa.density_fixed_h(sm_, h_sol)
            sa.force(su, sv)
            torch.cuda.synchronize()
            sa.profile(True)
            for _ in range(3):
                sa.density_fixed_h(sm_, h_sol)
                sa.force(su, sv)
            torch.cuda.synchronize()
            sst = sa.stats()
            sa.profile(False)
            ablation[name] = {
                "density_ms": sst["sweep_ms"][0] / 3, "force_ms": sst["sweep_ms"][2] / 3,
                "density_accepted_fraction": sst["sweep_units"][0] / max(1, sst["sweep_candidates"][0]),
                "force_accepted_fraction": sst["sweep_units"][2] / max(1, sst["sweep_candidates"][2])}
            sa.close()
        ablation["sorting_speedup"] = {
            k: ablation["naive"][k] / ablation["sorted"][k] for k in ("density_ms", "force_ms")}
        extras["ablation_naive_vs_sorted"] = ablation
        # ---- next row: the force with artificial viscosity and the Eq. (dt)
        # time step (Section 4.1): velocity-derivative and viscous force sweeps
        hs.force_viscous(su, sv)
        torch.cuda.synchronize()
        hs.profile(True)
        for _ in range(3):
            hs.force_viscous(su, sv)
        torch.cuda.synchronize()
        vst = hs.stats()
        hs.profile(False)
        extras["viscous_force"] = {
            "workload": args.side_workload,
            "velocity_derivatives_ms": vst["sweep_ms"][5] / 3,
            "viscous_force_ms": vst["sweep_ms"][6] / 3,
            "force_pairs_per_s": vst["sweep_units"][6] / 2 / (vst["sweep_ms"][6] / 1e3),
            "kernels": ["k_sweep<PVelDeriv>", "k_sweep<PForceVisc>"]}
        hs.close()
        del spos, sm_, su, sv
        # ---- the other configurations, briefly
        others = {}
        for name in [x for x in args.others.split(",") if x and x != args.workload]:
            try:
                others[name] = other_workload(name, dev, params)
            except Exception as e:  # noqa: BLE001
                others[name] = {"failed": str(e)}
        extras["other_workloads"] = others
        try:
            extras["parity_small_full_oracle"] = small_parity(dev)
        except Exception as e:  # noqa: BLE001
            extras["parity_small_full_oracle"] = {"failed": str(e)}

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            r = oracle_sample_rate(d, sample=args.ref_sample)
            cpu = {"value": r["value"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{r['sample']} random particles of {args.workload} ({r['where']}), "
                             f"evaluated from scratch in {r['seconds']:.1f} s (h solve of the "
                             "sample and its force partners, density, force; neighbour trees "
                             "included)"}
            try:
                cpu["whole_small_box"] = oracle_full_rate()
                cpu["whole_small_box_one_core"] = oracle_full_rate_one_core()
                if args.oracle_c4:  # minutes of CPU time: on request only
                    cpu["whole_sinusoid64"] = oracle_full_rate("sinusoid64")
                    cpu["whole_sinusoid64_one_core"] = oracle_full_rate_one_core("sinusoid64")
            except Exception as e:  # noqa: BLE001
                cpu["whole_small_box"] = {"failed": str(e)}
            # the oracle's values of that sample against this run's results
            try:
                gi, ref = r["index"], r["ref"]
                gh = den["h"].double().cpu().numpy()[gi]
                grho = den["rho"].double().cpu().numpy()[gi]
                ga = out[1].double().cpu().numpy()[gi]
                arms = float(np.sqrt(np.mean(np.sum(ref["a"] ** 2, axis=1))))
                hmax = float(den["h"].max())
                parity = {"particles": int(len(gi)), "where": r["where"],
                          "h_max_vs_cube_margin": hmax / 0.125,
                          "max_rel_err_h": float(np.max(np.abs(gh / ref["h"] - 1.0))),
                          "max_rel_err_rho": float(np.max(np.abs(grho / ref["rho"] - 1.0))),
                          "max_err_acc_over_rms": float(np.max(np.linalg.norm(ga - ref["a"], axis=1))
                                                        / arms) if arms > 0 else None,
                          "tolerances": {"h": 1e-5, "rho": 1e-5, "acc": 1e-4}}
            except Exception as e:  # noqa: BLE001
                parity = {"failed": str(e)}
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {e}"}
    if rank == 0:
        ratio = (fwd_ms + adj_ms) / fwd_ms
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "particles": n,
                       "units_per_step": units, "density_interactions": dens_units,
                       "force_pairs": force_units,
                       "step": "build+density(h-solve)+ghost+force+adjoint",
                       "l2": "working set per step > L2 (sorted lists alone ~%d MB)"
                             % (st["sorted_entries"] * 8 // 2**20),
                       "kahan": args.kahan, "parallelism": f"replicas x{world}",
                       "h_iteration": "CUDA graph, device-side while loop",
                       "fwd_adj_over_fwd": ratio,
                       "plain_fp32_fwd_ms": fwd32_ms, "compensated_fwd_ms": fwd_ms},
            "fwd_ms": fwd_ms, "adj_ms": adj_ms, "fwd_adj_over_fwd": ratio,
            "fwd_value": units / (fwd_ms / 1e3),
            "plain_fp32_forward": plain32,
            "clocks": clocks,
            "e2e": {"value": job_rate(units, world, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "profiled_pass": {"ms_per_step": prof["ms"], "steps": prof["steps"],
                              "gpu_launches": int(prof["launches"]), "clocks": prof["clocks"],
                              "note": "roofline and kernels come from this pass (host-loop h "
                                      "iteration, CUDA events around every sweep launch)"},
            "autotune": tuned,
            "roofline": roof,
            "kernels": kernels,
            "decomposition": {k: prod["stats"][k] for k in ("ncell", "nleaf", "nblock", "nself", "npair",
                                                            "ndt", "max_depth", "newton_iters",
                                                            "rebuilds")},
            "h_iteration_active": [x for x in prod["stats"]["newton_active"] if x],
            "sampled_parity": parity,
            "build_stages_ms": {BUILD_STAGES[k]: st["build_ms"][k] / prof["steps"] for k in range(8)},
            "build": build_rate(st, n, pk, pk_kind),
            "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
