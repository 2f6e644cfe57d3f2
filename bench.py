"""Benchmark of the fused anisotropic Cahn-Hilliard MRT-LBM step on GB300.

Workload: the 8192x8192 periodic spinodal field (phi0 = U[-0.05, 0.05], seed 0,
alpha = 0.3, Eq. 39 parameters), FP32 arithmetic. One benchmark step = 100 lattice
time steps (one fused kernel launch each) followed by the logged diagnostics, total
mass and free energy (FP64 reductions on the GPU); --steps 20 covers the
workload's 2000 time steps. Inputs (9 x 8192^2 populations, 2.4 GB per buffer)
are far larger than L2, so no flush is needed between steps.

Prints one JSON line. The metric is MLUPS (million lattice-node updates per
second), with the step kernel's HBM roofline fraction for FP32 storage and, as
variants, the BF16- and FP16-deviation storages. Beside it: the 64^2 droplet
(single launches and graph replay), the 256^2 spinodal run of 20000 steps in every
storage with its energy law and error against the FP64 oracle, the error of every
storage against the oracle per workload, the batched sweep, the D3Q15 cube, the
learned leap with its online judge, and the oracle's own rates on the host cores.

--impl reference times the FP64 CPU oracle (the test suite's reference) on the
host cores instead, on a 2048x2048 sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N = 8192
ALPHA = 0.3
SEED = 0
NOISE = 0.05
INNER = 100  # lattice steps per benchmark step
WORKLOAD = "spinodal-8192x8192"
METRIC = "MLUPS (lattice-node updates/s, 1e6)"
STEP_KERNEL_SOURCES = ("paper_2501_03759_gb300/csrc/lbch_step.cuh",
                       "paper_2501_03759_gb300/csrc/lbch_lattice.cuh",
                       "paper_2501_03759_gb300/csrc/lbch_f2.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N, help="grid edge (default: the 8192^2 workload)")
    ap.add_argument("--no-variants", action="store_true", help="skip the 16-bit storage variants")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-field parameter-sweep batch")
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--no-3d", action="store_true", help="skip the D3Q15 measurement")
    ap.add_argument("--n3", type=int, default=256, help="edge of the D3Q15 spinodal cube (default 256)")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-leap time-to-t measurement")
    ap.add_argument("--no-small-configs", action="store_true",
                    help="skip the 64^2 droplet and 256^2 spinodal legs and the oracle comparisons")
    ap.add_argument("--config2-steps", type=int, default=20000,
                    help="steps of the 256^2 spinodal run (a multiple of 100, at least 1000: the oracle "
                         "comparison reads phi at step 1000)")
    ap.add_argument("--log-dir", default=os.environ.get("LBCH_LOG_DIR"),
                    help="write the 256^2 run's mass and energy every 100 steps as CSV into this folder "
                         "(default: $LBCH_LOG_DIR; none if unset)")
    ap.add_argument("--storage", choices=["f32", "bf16_dev", "f16_dev"], default="f32",
                    help="population storage of the main timed line")
    args = ap.parse_args()
    if args.config2_steps < 1000 or args.config2_steps % 100:
        ap.error("--config2-steps must be a multiple of 100 and at least 1000")
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(storage_name: str):
    """DRAM bytes per node update of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"step_kernel_{storage_name}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_node_update"])
    except (KeyError, ValueError):
        return None


def max_over_ranks(dist, v: float) -> float:
    """Maximum of a per-rank scalar over the process group (identity without one)."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput of independent replicas: all units over the slowest rank's time."""
    return world * units_per_rank / max_seconds


NOMINAL_HBM_GBS = 8000.0  # the GB300's nominal HBM3e bandwidth, about 8 TB/s


def sig(v, digits: int = 4):
    """Rounds floats (also inside dicts and lists) to a few significant digits, so the JSON
    line stays short."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}") if np.isfinite(v) else v
    if isinstance(v, dict):
        return {k: sig(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [sig(x, digits) for x in v]
    return v


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def time_storage(lbch, torch, phi0, n, storage, steps, warmup, with_launch_events=True):
    """Runs warmup + timed benchmark steps on one storage; returns timings (seconds)."""
    solver = lbch.Solver(lbch.make_params(n, n, alpha=ALPHA, storage=storage))
    solver.init_field(phi0)
    stream = solver.stream
    mass, energy = [], []
    for _ in range(warmup):
        solver.step(INNER)
        solver.mass()
        solver.free_energy()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(steps):
        ev[k][0].record(stream)
        solver.step(INNER)
        ev[k][1].record(stream)
        mass.append(solver.mass())
        energy.append(solver.free_energy())
    stop.record(stream)
    torch.cuda.synchronize()
    total = start.elapsed_time(stop) / 1e3
    step_kernels = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    solver.close()
    del solver
    torch.cuda.empty_cache()
    return {"total_s": total, "kernel_s_per_launch": step_kernels / (steps * INNER),
            "mass_first": mass[0], "mass_last": mass[-1], "energy_first": energy[0],
            "energy_last": energy[-1]}


def run_e2e(lbch, torch, phi0, n, steps, warmup):
    """Same metric through the public API from pinned host buffers: every step copies phi0
    in, runs INNER lattice steps, reads mass and energy, and copies phi back out."""
    solver = lbch.Solver(lbch.make_params(n, n, alpha=ALPHA))
    h_in = torch.from_numpy(phi0).pin_memory()
    h_out = torch.empty((n, n), dtype=torch.float64).pin_memory()

    def one():
        solver.init_field(h_in)
        solver.step(INNER)
        solver.mass()
        solver.free_energy()
        solver.field(h_out)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    solver.close()
    return {"lu": steps * INNER * n * n, "unit": "MLUPS",
            "h2d_bytes_per_step": int(h_in.numel() * 8), "d2h_bytes_per_step": int(h_out.numel() * 8 + 16),
            "wall_s": dt}


def run_batch_sweep(lbch, torch, steps: int, count: int = 512, seed: int = 0, storage: str = "f32"):
    """The parameter-sweep workload: count fields (edges from {64, 128, 256, 512}, alpha in
    [0, 0.5], droplets and spinodal fields) stepped together in the given storage."""
    import workloads

    specs = workloads.batch_sweep_specs(count, seed)
    n = [sp["n"] for sp in specs]
    sites = sum(v * v for v in n)
    codes = {"f32": lbch.STORE_F32, "bf16_dev": lbch.STORE_BF16_DEV, "f16_dev": lbch.STORE_F16_DEV}
    b = lbch.Batch(lbch.make_params(8, 8, storage=codes[storage]), n, n, [sp["alpha"] for sp in specs])
    for i, sp in enumerate(specs):
        b.init_field(i, workloads.batch_field(sp))
    b.step(64)  # warm-up (one graph replay)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    out = {"value": steps * sites / sec / 1e6, "unit": "MLUPS", "fields": count, "nodes": sites,
           "steps": steps, "ms_per_step": sec / steps * 1e3, "rows_per_warp": b.rows_target,
           "storage": storage, "launch": "one kernel per step for all fields, CUDA graphs of 64 steps"}
    b.close()
    return out


def run_3d(lbch, torch, n: int, steps: int):
    """The D3Q15 path on an n^3 periodic spinodal field (alpha 0.3, noise 0.05), FP32."""
    rng = np.random.default_rng(SEED)
    s = lbch.Solver3(lbch.make_params3(n, n, n, alpha=ALPHA))
    s.init_field(rng.uniform(-NOISE, NOISE, (n, n, n)))
    s.step(5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    s.close()
    mlups = steps * n ** 3 / sec / 1e6
    peak_bw = measured_peaks()[0]
    return {"value": mlups, "unit": "MLUPS", "workload": f"spinodal-{n}^3 D3Q15", "steps": steps,
            "ms_per_step": sec / steps * 1e3, "algorithmic_bytes_per_lu": 120,
            "roofline_frac_algorithmic": 120 * mlups * 1e6 / (peak_bw * 1e9),
            "launch": "three kernels per step (phi; mu_alpha and mu_beta by a z-sweep; collide and store)"}


def run_config1(lbch, torch, steps: int = 2000):
    """The 64^2 droplet workload (radius 20, profile tanh((R - r)/(sqrt(2) 1.5)), alpha 0.3),
    FP32: the time per step with one launch per lbch_step call and with the context's graph
    replay (launch-bound: 4096 nodes per step, labelled, not a roofline number), and phi
    after `steps` steps in every storage for the oracle comparison."""
    import workloads

    n = 64
    phi0 = workloads.droplet_workload(n)
    out, fields = {"workload": f"droplet-{n}x{n} alpha {ALPHA}", "steps": steps}, {}
    s = lbch.Solver(lbch.make_params(n, n, alpha=ALPHA))
    for mode in ("single", "graph"):
        s.init_field(phi0)
        s.step(32)
        s.init_field(phi0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        if mode == "single":
            for _ in range(steps):
                s.step(1)
        else:
            s.step(steps)
        e1.record(s.stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        out[f"us_per_step_{mode}"] = sec / steps * 1e6
        out[f"mlups_{mode}"] = steps * n * n / sec / 1e6
    fields["f32"] = s.field()
    s.close()
    for name, st in (("bf16_dev", lbch.STORE_BF16_DEV), ("f16_dev", lbch.STORE_F16_DEV)):
        v = lbch.Solver(lbch.make_params(n, n, alpha=ALPHA, storage=st))
        v.init_field(phi0)
        v.step(steps)
        fields[name] = v.field()
        v.close()
    out["bound"] = "launch/latency (L2-resident, 4096 nodes per step)"
    return out, fields


def run_config2(lbch, torch, steps: int = 20000, every: int = 100, alpha: float = 0.2, n: int = 256):
    """The 256^2 spinodal workload (U[-0.05, 0.05], seed 0, alpha 0.2): `steps` steps in each
    storage with mass and free energy logged every `every` steps on the device (read back
    once), phi at 1000 and at `steps` steps. Returns per storage the MLUPS of the whole
    logged run, the logs and the two fields."""
    import workloads

    phi0 = workloads.noise(n, n, NOISE, SEED)
    res = {}
    for name, st in (("f32", lbch.STORE_F32), ("bf16_dev", lbch.STORE_BF16_DEV), ("f16_dev", lbch.STORE_F16_DEV)):
        s = lbch.Solver(lbch.make_params(n, n, alpha=alpha, storage=st))
        s.init_field(phi0)
        s.step(64)  # warm-up: the graph is captured, clocks up
        s.init_field(phi0)
        k = steps // every
        log = torch.zeros((k + 1, 2), dtype=torch.float64, device=s.device)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.mass_device(log[0, 0:1])
        s.free_energy_device(log[0, 1:2])
        phi1000 = None
        for j in range(1, k + 1):
            s.step(every)
            s.mass_device(log[j, 0:1])
            s.free_energy_device(log[j, 1:2])
            if j * every == 1000:
                phi1000 = s.phi_device().clone()
        e1.record(s.stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        res[name] = {"mlups": steps * n * n / sec / 1e6, "us_per_step": sec / steps * 1e6,
                     "log": log.cpu().numpy(), "phi1000": phi1000.cpu().numpy().astype(np.float64),
                     "phi_end": s.field()}
        s.close()
    return res


def energy_law(E, rise_tol: float = 1e-4, trend: float = 0.9):
    """The energy gate of the small-noise spinodal at alpha > 0: rises between samples of at
    most rise_tol |E| (Eq. 15 is the exact gradient flow only at an interface) and a falling
    trend (the last sample below trend times the first)."""
    E = np.asarray(E, dtype=np.float64)
    rise = float(np.max(np.diff(E) / np.abs(E[:-1])))
    ok = bool(rise <= rise_tol and E[-1] < trend * E[0])
    return {"max_rise_rel": rise, "end_over_start": float(E[-1] / E[0]), "gate": f"rise<={rise_tol:g}, end<{trend:g} start",
            "pass": ok}


def full_size_window_errors(lbch, phi0, n: int, steps: int = 5, wsz: int = 32):
    """max |phi - phi_oracle| of each storage on the 8192^2 workload after `steps` steps, on
    eight windows (corners, the periodic seam, strip and segment boundaries), the oracle
    running each window with a halo of the steps' footprint (exact on the window)."""
    import oracle

    p = oracle.Params(n, n, alpha=ALPHA)
    corners = [(0, 0), (n - wsz, n - wsz), (n - wsz, 0), (0, n - wsz), (4000, 4090), (116, 7000),
               (120 * 34 - 16, 482 * 9 - 16), (8150, 470)]
    refs = [oracle.run_window(p, phi0, x0, y0, wsz, wsz, steps) for (x0, y0) in corners]
    out = {}
    for name, st in (("f32", lbch.STORE_F32), ("bf16_dev", lbch.STORE_BF16_DEV), ("f16_dev", lbch.STORE_F16_DEV)):
        s = lbch.Solver(lbch.make_params(n, n, alpha=ALPHA, storage=st))
        s.init_field(phi0)
        s.step(steps)
        g = s.field()
        s.close()
        out[name] = max(float(np.abs(g[y0:y0 + wsz, x0:x0 + wsz] - r).max()) for (x0, y0), r in zip(corners, refs))
        del g
    return out


def timed_oracle(p, f, steps: int, threads: int):
    """Runs the oracle `steps` steps on `threads` host threads; returns (state, seconds)."""
    import oracle

    oracle.set_threads(threads)
    t0 = time.perf_counter()
    g = oracle.step(p, f, steps)
    return g, time.perf_counter() - t0


def oracle_legs(c1_fields, c2, full_windows, c1_steps: int = 2000, c2_steps: int = 20000):
    """The FP64 oracle on the host cores: the reference results of the 64^2 droplet (2000
    steps) and of the 256^2 spinodal run (1000 and 20000 steps), with the errors of every
    storage against them, and the oracle's own rates single-threaded and on all cores
    (configs 1 and 2 in full on all cores; single-threaded samples of 300 and 1000 steps;
    the 8192^2 workload from a 2048^2 sample)."""
    import oracle
    import workloads

    cores = os.cpu_count() or 1
    rates = {}
    # 64^2 droplet, alpha 0.3
    p1 = oracle.Params(64, 64, alpha=ALPHA)
    f1 = oracle.init(p1, workloads.droplet_workload(64))
    g1, dt = timed_oracle(p1, f1, c1_steps, cores)
    rates["droplet64"] = {"all_cores": c1_steps * 64 * 64 / dt / 1e6}
    _, dt = timed_oracle(p1, f1, c1_steps, 1)
    rates["droplet64"]["one_core"] = c1_steps * 64 * 64 / dt / 1e6
    ref1 = oracle.phi(p1, g1)
    # 256^2 spinodal, alpha 0.2
    p2 = oracle.Params(256, 256, alpha=0.2)
    f2 = oracle.init(p2, workloads.noise(256, 256, NOISE, SEED))
    _, dt = timed_oracle(p2, f2, 300, 1)
    rates["spinodal256"] = {"one_core": 300 * 256 * 256 / dt / 1e6, "one_core_sample_steps": 300}
    g2a, dta = timed_oracle(p2, f2, 1000, cores)
    g2b, dtb = timed_oracle(p2, g2a, c2_steps - 1000, cores)
    rates["spinodal256"]["all_cores"] = c2_steps * 256 * 256 / (dta + dtb) / 1e6
    ref2a, ref2b = oracle.phi(p2, g2a), oracle.phi(p2, g2b)
    e2_end = oracle.energy(p2, g2b)
    # 8192^2 workload: per-node rate from a 2048^2 sample
    p4 = oracle.Params(2048, 2048, alpha=ALPHA)
    f4 = oracle.init(p4, workloads.noise(2048, 2048, NOISE, SEED))
    _, dt = timed_oracle(p4, f4, 1, 1)
    rates["spinodal8192_from_2048_sample"] = {"one_core": 2048 * 2048 / dt / 1e6}
    oracle.set_threads(cores)
    errs = {}
    for name in ("f32", "bf16_dev", "f16_dev"):
        errs[name] = {
            f"droplet64_{c1_steps}": float(np.abs(c1_fields[name] - ref1).max()),
            "spinodal256_1000": float(np.abs(c2[name]["phi1000"] - ref2a).max()),
            f"spinodal256_{c2_steps}": float(np.abs(c2[name]["phi_end"] - ref2b).max()),
            "spinodal8192_5_windows": full_windows[name],
        }
    return {"errors": errs, "rates": rates, "cores": cores, "energy_oracle_spinodal256_end": e2_end}


SURROGATE_THETA = os.path.join(ROOT, "paper_2501_03759_gb300", "weights", "leap512_k500.npy")


def run_surrogate(alphas=(0.1, 0.3, 0.45), seed: int = 777, more_seeds=(2024, 31337)):
    """Time-to-t of the learned leap against the plain LBM on a held-out 512^2 spinodal field
    to t = 50000 (500 LBM steps, then 90 x (one 500-step leap + 50 LBM steps)), with the
    committed trained parameters, for each anisotropy strength; None if they are absent."""
    if not os.path.exists(SURROGATE_THETA):
        return None
    from paper_2501_03759_gb300 import surrogate

    theta = np.load(SURROGATE_THETA)
    gates = {"phi_rel_l2_max": 5e-2, "energy_rel_diff_max": 1e-2, "speedup_min": 5.0}
    runs = []
    single = [surrogate.evaluate(theta, a, seed, turns=1)["phi_rel_l2"] for a in alphas]
    # further held-out fields (none among the training seeds): phi error per alpha and the
    # smallest speedup, compactly
    more = [[surrogate.evaluate(theta, a, sd) for a in alphas] for sd in more_seeds]
    for a in alphas:
        r = surrogate.evaluate(theta, a, seed)
        j = r["judge"]
        runs.append({"alpha": a, "phi_rel_l2": r["phi_rel_l2"], "energy_rel_diff": r["energy_rel_diff"],
                     "mass_drift_abs": r["mass_drift_abs"], "s_plain": r["seconds_plain"],
                     "s_leap": r["seconds_leap"], "speedup": r["speedup"],
                     "judge": [j["accepted"], j["rejected"], j["rejected_energy"], j["rejected_mass"],
                               j["rejected_nonfinite"]],
                     "max_rise": [j["max_leap_rise"], j["max_corr_rise"]],
                     "pass": bool(r["phi_rel_l2"] <= gates["phi_rel_l2_max"] and
                                  r["energy_rel_diff"] <= gates["energy_rel_diff_max"] and
                                  r["speedup"] >= gates["speedup_min"])})
    return {"workload": "spinodal-512^2 K=500 leap + 50 LBM steps to t=50000, held-out seed 777, judged; "
                        f"each leap averaged over {surrogate.TURNS} quarter turns of the field",
            "phi_rel_l2_one_turn": single,
            "more_held_out": {"seeds": list(more_seeds),
                              "phi_rel_l2": [[r["phi_rel_l2"] for r in rs] for rs in more],
                              "energy_rel_diff_max": max(r["energy_rel_diff"] for rs in more for r in rs),
                              "speedup_min": min(r["speedup"] for rs in more for r in rs),
                              "rejected": sum(r["judge"]["rejected"] for rs in more for r in rs)},
            "judge": f"lbnop_leap_run_judged: energy_rtol {surrogate.JUDGE['energy_rtol']:g}, "
                     f"mass_atol {surrogate.JUDGE['mass_atol']:g}/node; judge = [accepted, rejected, "
                     "by energy, by mass, non-finite]; max_rise = largest relative energy rise across a "
                     "leap and across its 50 correction steps",
            "network": "96/64/96/96 channels, 826,096 parameters: wider than the configured 32 base "
                       "channels (~0.5M), which left the rollout error 2-4x above the gate",
            "gates": gates, "by_alpha": runs, "speedup": min(r["speedup"] for r in runs),
            "kernels": surrogate.time_kernels(theta),
            "conv_level0_b16": conv_with_roofline(surrogate.time_conv(16))}


def conv_with_roofline(c):
    """The tcgen05 convolution's throughput against the measured bf16 peaks: the sustained one
    (a kernel inside a long step) and the burst one."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        sus, burst, kind = float(d["bf16_tflops_sustained"]), float(d["bf16_tflops"]), "measured"
    else:
        sus, burst, kind = 1700.0, 1900.0, "fallback"
    c = dict(c)
    c["frac_of_sustained"] = c["tflops"] / sus
    c["frac_of_burst"] = c["tflops"] / burst
    c["peak_kind"] = kind
    return c


def host_cpu() -> str:
    """The host CPU's model name (lscpu), for the oracle timings; 'unknown' if unavailable."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:  # noqa: BLE001 - a label only, never fatal
        pass
    return platform.machine() or "unknown"


def cpu_oracle_rate(target_s: float = 8.0, n_sample: int = 2048):
    """The FP64 oracle, as it stands, on the host cores: MLUPS on an n_sample^2 spinodal
    sample of the workload (alpha 0.3, noise 0.05, seed 0)."""
    import oracle
    import workloads

    cores = oracle.set_threads(os.cpu_count() or 1)
    p = oracle.Params(n_sample, n_sample, alpha=ALPHA)
    f = oracle.init(p, workloads.noise(n_sample, n_sample, NOISE, SEED))
    t0 = time.perf_counter()
    f = oracle.step(p, f, 1)
    one = time.perf_counter() - t0
    k = max(1, int(target_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    oracle.step(p, f, k)
    dt = time.perf_counter() - t0
    return {"value": k * n_sample * n_sample / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{k} FP64 oracle steps on a {n_sample}x{n_sample} spinodal field "
                      f"(alpha {ALPHA}, noise {NOISE}, seed {SEED}), OpenMP over rows",
            "seconds": dt}


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    import workloads

    n_sample = 2048
    cores = oracle.set_threads(os.cpu_count() or 1)
    p = oracle.Params(n_sample, n_sample, alpha=ALPHA)
    f = oracle.init(p, workloads.noise(n_sample, n_sample, NOISE, SEED))
    f = oracle.step(p, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.step(p, f, args.steps)  # one call: the oracle allocates its field passes once
    dt = time.perf_counter() - t0
    value = args.steps * n_sample * n_sample / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{n_sample}x{n_sample}", "alpha": ALPHA, "noise": NOISE,
                   "seed": SEED, "lattice_steps_per_step": 1, "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "host": host_cpu(),
                         "sample": f"each step: 1 FP64 oracle step on a {n_sample}x{n_sample} spinodal field"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch

    from paper_2501_03759_gb300 import lbch
    import workloads

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("gloo")
    n = args.n
    phi0 = workloads.noise(n, n, NOISE, SEED)
    lbch.load()

    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else None

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    storages = {"f32": lbch.STORE_F32, "bf16_dev": lbch.STORE_BF16_DEV, "f16_dev": lbch.STORE_F16_DEV}
    main_st = storages[args.storage]
    barrier()
    with ClockSampler(gpu_id) as clk:
        r32 = time_storage(lbch, torch, phi0, n, main_st, args.steps, args.warmup)
    barrier()
    total = max_over_ranks(dist, r32["total_s"])
    per_launch = max_over_ranks(dist, r32["kernel_s_per_launch"])
    lu_per_rank = args.steps * INNER * n * n
    value = job_rate(world, lu_per_rank, total) / 1e6

    peak, peak_kind = measured_peaks()

    def roofline_of(st, name, launch_s):
        b = lbch.ALGORITHMIC_BYTES_PER_LU[st]
        ach = b * n * n / launch_s / 1e9
        tr = profiled_traffic(name)
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "frac_of_nominal_8tbs": ach / NOMINAL_HBM_GBS,
                "traffic": None if tr is None else tr * n * n, "peak_kind": peak_kind,
                "kernel": f"lbch::step_kernel<{name}, vec, fast rates>", "algorithmic_bytes_per_launch": b * n * n,
                "launch_ms": launch_s * 1e3}

    roofline = roofline_of(main_st, args.storage, per_launch)

    variants = {}
    if not args.no_variants:
        for name, st in storages.items():
            if st == main_st:
                continue
            r = time_storage(lbch, torch, phi0, n, st, args.steps, args.warmup)
            pl = max_over_ranks(dist, r["kernel_s_per_launch"])
            rf = roofline_of(st, name, pl)
            variants[name] = {"value": job_rate(world, lu_per_rank, max_over_ranks(dist, r["total_s"])) / 1e6,
                              "launch_ms": pl * 1e3, "frac": rf["frac"], "frac_of_nominal_8tbs": rf["frac_of_nominal_8tbs"],
                              "traffic": rf["traffic"],
                              "mass_drift_rel": abs(r["mass_last"] - r["mass_first"]) / max(1e-300, abs(r["mass_first"]))}

    e2e = None
    if not args.no_e2e:
        e = run_e2e(lbch, torch, phi0, n, args.steps, args.warmup)
        barrier()
        e2e = {"value": job_rate(world, e["lu"], max_over_ranks(dist, e["wall_s"])) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": e["h2d_bytes_per_step"], "d2h_bytes_per_step": e["d2h_bytes_per_step"],
               "lattice_steps_per_step": INNER}

    batch = None
    if not args.no_batch:
        batch = run_batch_sweep(lbch, torch, args.batch_steps)
        peak_bw = measured_peaks()[0]
        batch["roofline_frac"] = 72 * batch["value"] * 1e6 / (peak_bw * 1e9)
        batch["value"] = job_rate(world, batch["value"], 1.0)  # replicas: rates add
        batch.pop("launch", None)
        if not args.no_variants:
            bv = run_batch_sweep(lbch, torch, args.batch_steps, storage="bf16_dev")
            batch["bf16_dev"] = {"value": job_rate(world, bv["value"], 1.0), "ms_per_step": bv["ms_per_step"],
                                 "rows_per_warp": bv["rows_per_warp"],
                                 "roofline_frac": 48 * bv["value"] * 1e6 / (peak_bw * 1e9)}

    d3 = None
    if not args.no_3d:
        d3 = run_3d(lbch, torch, args.n3, 50)
        d3["paper_100"] = run_3d(lbch, torch, 100, 200)["value"]
        d3.pop("launch", None)

    leap = None
    if not args.no_surrogate and rank == 0:
        leap = run_surrogate()

    cfg1 = cfg2 = errors = cpu_rates = None
    if rank == 0 and world == 1 and not args.no_small_configs:
        cfg1, c1_fields = run_config1(lbch, torch)
        c2 = run_config2(lbch, torch, args.config2_steps)
        windows = full_size_window_errors(lbch, phi0, n) if not args.no_cpu_baseline else None
        cfg2 = {"workload": "spinodal-256x256 alpha 0.2", "steps": args.config2_steps,
                "log_every": 100}
        for name, r in c2.items():
            cfg2[name] = {"mlups": r["mlups"], "us_per_step": r["us_per_step"],
                          "energy_law": energy_law(r["log"][:, 1]),
                          "mass_drift_per_node": float(abs(r["log"][-1, 0] - r["log"][0, 0]) / (256 * 256))}
        if args.log_dir:  # mass and energy every 100 steps, both storages
            os.makedirs(args.log_dir, exist_ok=True)
            csv = os.path.join(args.log_dir, "config2_spinodal256_mass_energy.csv")
            with open(csv, "w") as fh:
                fh.write("step," + ",".join(f"mass_{k},energy_{k}" for k in c2) + "\n")
                for j in range(c2["f32"]["log"].shape[0]):
                    fh.write(f"{j * 100}," + ",".join(f"{c2[k]['log'][j, 0]:.12e},{c2[k]['log'][j, 1]:.12e}"
                                                        for k in c2) + "\n")
            cfg2["csv"] = csv
        if not args.no_cpu_baseline:
            o = oracle_legs(c1_fields, c2, windows, c2_steps=args.config2_steps)
            errors = o["errors"]
            cpu_rates = o["rates"]
            cpu_rates["cores"] = o["cores"]
            cpu_rates["host"] = host_cpu()
            cfg2["energy_end_vs_oracle_rel"] = {
                k: abs(float(c2[k]["log"][-1, 1]) - o["energy_oracle_spinodal256_end"]) /
                abs(o["energy_oracle_spinodal256_end"]) for k in c2}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if n == N else f"spinodal-{n}x{n}", "nx": n, "ny": n, "alpha": ALPHA,
                       "noise": NOISE, "seed": SEED, "storage": args.storage, "lattice_steps_per_step": INNER,
                       "diagnostics_per_step": ["mass", "free_energy"],
                       "l2": "inputs larger than L2 (2.4 GB per population buffer), no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline,
            "kernel_only_mlups": world * n * n / per_launch / 1e6,
            "oracle_error_bounds": {"f32": "1e-6 after 1 step, 1e-4 after 1000 steps (gated in tests)",
                                    "bf16_dev/f16_dev": "reported; tests hold measured maxima x2"},
            "cpu_oracle_rates_mlups": cpu_rates,
            "batch_sweep": batch,
            "d3q15": d3,
            "surrogate": leap,
            "config1_droplet64": cfg1,
            "config2_spinodal256": cfg2,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": args.steps * (INNER + 5),
            "mass_drift_rel": abs(r32["mass_last"] - r32["mass_first"]) / max(1e-300, abs(r32["mass_first"])),
            "energy_first_last": [r32["energy_first"], r32["energy_last"]],
            # last, so that a reader keeping only the end of the output still sees the 16-bit
            # storages' rates, roofline fractions and errors against the FP64 oracle
            "max_abs_dphi_vs_fp64_oracle": errors,
            "variants": variants,
        }
        line = {k: (sig(v, 6) if k in ("value", "ms_per_step", "energy_first_last") else sig(v))
                for k, v in line.items()}
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
