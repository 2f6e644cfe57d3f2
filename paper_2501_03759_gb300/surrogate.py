"""The learned leap's workflow: generate LBM trajectories, train the network, and run
and check the leap/LBM alternation against the plain LBM.

  python -m paper_2501_03759_gb300.surrogate train --out DIR   # data + training, writes DIR/leap_theta.npy
  python -m paper_2501_03759_gb300.surrogate eval --theta FILE  # gates against a held-out plain run
  python -m paper_2501_03759_gb300.surrogate time --theta FILE  # device time of a forward and a step
  python -m paper_2501_03759_gb300.surrogate conv               # device time of one 3x3 convolution

Data: periodic n x n spinodal runs of the scheme (phi0 = U[-0.05, 0.05], seeded; alpha of
Eq. 6 spread over [0, 0.5]; the other parameters of Eq. 39), stepped together by the
batched lbch path; phi is copied on the device every `every` steps. A training pair is
(phi(t), phi(t + leap)) for any stored t.

Evaluation: from a held-out initial field, the plain LBM runs T = warmup + cycles (leap + corr)
steps; the surrogate run takes the same warmup LBM steps (the white noise of phi0 decays),
then alternates one leap (K = leap steps) with corr LBM steps, cycles times.
Reported: relative L2 error of phi at T, relative free-energy difference, mass drift, and
the time-to-T of both runs (CUDA events on the shared stream).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import lbch, lbnop

LEAP = 500        # steps per leap (K)
EVERY = 50        # snapshot spacing
CORR = 50         # LBM correction steps after each leap
SCALE = 0.01      # phi_out = phi + SCALE sig (D - mean D), sig the field's rms
T_END = 50000
WARMUP = 500      # plain LBM steps before the first leap (the noise of phi0 decays first)
TURNS = 4         # leaps average the network over the field's four quarter turns
CLIP = 3.0        # training clips each gradient to CLIP x the median norm of recent steps
CLIP_WINDOW = 200
CLIP_START = 20
# (c_in, c_out) of the network's layers, in the order of include/lbnop.h
LAYERS = [(16, 96), (96, 96), (96, 64), (64, 64), (64, 96), (96, 96), (96, 96), (96, 96),
          (96, 96), (96, 64), (64, 64), (64, 96), (96, 96), (96, 16), (16, 16), (16, 16)]
OUT = 13  # the output layer; the two after it are the linear path


def make_runs(count: int, seed: int = 1000):
    """(alpha, seed) of each training run: alphas evenly over [0, 0.5], shuffled."""
    r = np.random.default_rng(seed)
    alphas = r.permutation(np.linspace(0.0, 0.5, count))
    return [(float(a), seed + 1 + k) for k, a in enumerate(alphas)]


def init_theta(seed: int, out_scale: float = 0.1) -> np.ndarray:
    """Initial parameters (flat layout of include/lbnop.h): He-normal 3 x 3 weights
    (std sqrt(2 / (9 c_in))), the output layer's scaled by out_scale so that training
    starts near the identity leap, a zero linear path, zero biases and conditioning vector."""
    r = np.random.default_rng(seed)
    parts = []
    for k, (ci, co) in enumerate(LAYERS):
        w = r.normal(0.0, (2.0 / (9 * ci)) ** 0.5, 9 * co * ci) * (out_scale if k == OUT else 1.0)
        if k > OUT:
            w[:] = 0.0
        parts += [w, np.zeros(co)]
        if k == 0:
            parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def spinodal(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-0.05, 0.05, (n, n))


def generate(runs, n: int = 512, t_end: int = T_END, every: int = EVERY):
    """Device tensor [len(runs), t_end / every + 1, n, n] (FP32) of phi snapshots."""
    import torch

    count = len(runs)
    snaps = t_end // every + 1
    data = torch.empty((count, snaps, n, n), dtype=torch.float32, device="cuda")
    b = lbch.Batch(lbch.make_params(8, 8), [n] * count, [n] * count, [a for a, _ in runs])
    for i, (_, seed) in enumerate(runs):
        b.init_field(i, spinodal(n, seed))
    for k in range(snaps):
        if k:
            b.step(every)
        for i in range(count):
            b.phi_device(i, data[i, k])
    torch.cuda.synchronize()
    b.close()
    return data


def d4(t, k: int, flip: bool):
    """One element of the square's symmetry group on a batch of periodic fields [B][n][n]: a
    rotation by k quarter turns, then a reflection x -> -x if flip."""
    import torch

    t = torch.rot90(t, k, dims=(1, 2)) if k else t
    return (torch.flip(t, dims=(2,)) if flip else t).contiguous()


def train(data, alphas, iters: int, batch: int = 16, lr: float = 1e-3, lr_end: float = 1e-5, seed: int = 0,
          theta0=None, log_every: int = 200, clip: float = CLIP, augment: bool = True, alpha_weight: float = 0.0):
    """Adam on the leap error over random (run, t) pairs, each pair weighted by the inverse of
    its own mean squared change (so that the identity map scores 1 on every pair and small
    late-time changes count as much as the early decay of the noise); cosine learning rate.

    With augment, each batch is turned by a random element of the square's symmetry group
    (rotations by quarter turns, reflections). The scheme commutes with all eight: the
    D2Q9 velocities and weights, gamma(n) of Eq. 6 and the relaxation rates (s_3 = s_5) are
    invariant under them, so a turned pair is another exact pair of the same dynamics.

    With alpha_weight > 0, run i is drawn with probability proportional to
    1 + alpha_weight alpha_i (uniform otherwise).

    With clip > 0, each step's gradient is clipped to `clip` times the median global norm
    of the last CLIP_WINDOW steps (from step CLIP_START on): a rare batch whose gradient is
    orders of magnitude above the rest otherwise moves every weight by about 30 lr through
    Adam's momentum, and the second-moment estimate it inflates then stalls learning for
    thousands of steps."""
    import torch

    count, snaps, n, _ = data.shape
    gap = LEAP // EVERY
    s = lbnop.Surrogate(n, n, max_batch=batch, scale=SCALE)
    s.set_params(init_theta(seed) if theta0 is None else theta0)
    r = np.random.default_rng(seed + 17)
    x = torch.empty((batch, n, n), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    alphas = np.asarray(alphas, dtype=np.float64)
    log = []
    norms = []
    clipped = 0
    t0 = time.perf_counter()
    p_run = None
    if alpha_weight > 0:
        p_run = 1.0 + alpha_weight * alphas
        p_run = p_run / p_run.sum()
    for it in range(iters):
        ri = r.integers(0, count, batch) if p_run is None else r.choice(count, size=batch, p=p_run)
        ki = r.integers(WARMUP // EVERY, snaps - gap, batch)
        ri_t, ki_t = torch.from_numpy(ri).cuda(), torch.from_numpy(ki).cuda()
        torch.index_select(data.view(count * snaps, n, n), 0, ri_t * snaps + ki_t, out=x)
        torch.index_select(data.view(count * snaps, n, n), 0, ri_t * snaps + ki_t + gap, out=y)
        xs, ys = x, y
        if augment:
            k, flip = int(r.integers(0, 4)), bool(r.integers(0, 2))
            xs, ys = d4(x, k, flip), d4(y, k, flip)
        rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * it / max(1, iters - 1)))
        want = (it % log_every == 0) or it == iters - 1
        change = ((ys - xs) ** 2).mean(dim=(1, 2)).double().cpu().numpy()
        weight = 1.0 / np.maximum(change, 1e-30)
        limit = clip * float(np.median(norms[-CLIP_WINDOW:])) if clip > 0 and len(norms) >= CLIP_START else 0.0
        s.set_clip(limit)
        loss = s.train_step(xs, alphas[ri], ys, rate, want_loss=want, weight=weight)
        norms.append(s.grad_norm())
        clipped += int(0.0 < limit < norms[-1])
        if want:
            log.append({"iter": it, "relative_loss": loss, "lr": rate, "grad_norm": norms[-1], "clip": limit,
                        "clipped_so_far": clipped, "seconds": time.perf_counter() - t0})
    torch.cuda.synchronize()
    theta = s.params_host()
    s.close()
    return theta, log


# The online judge of the leap runs (lbnop_leap_run_judged): a leap, or the correction steps
# after it, may raise the free energy by at most 1e-4 of |E| (the size of the rises between
# samples that the small-noise spinodal shows at alpha > 0, where Eq. 15 is not the exact
# gradient flow), and may move the mass by at most 1e-6 per node.
JUDGE = dict(energy_rtol=1e-4, mass_atol=1e-6)


def evaluate(theta, alpha: float, seed: int, n: int = 512, cycles: int = 90, leap: int = LEAP, corr: int = CORR,
             warmup: int = WARMUP, judged: bool = True, audit_every: int = 0, phi_rtol: float = 1e-2,
             turns: int = TURNS):
    """Plain LBM versus (warmup LBM steps, then cycles of one leap and corr LBM steps) from
    the same held-out field, to T = warmup + cycles (leap + corr) steps (50000 by default).
    With judged=True every leap is checked on the device by the plain scheme's mass and
    energy (and every audit_every-th against K plain steps) and replaced by plain steps if it
    fails. turns = 4 averages each leap over the field's four quarter turns
    (lbnop_set_leap_turns). Returns the gates, the judge's counts and timings."""
    import torch

    steps = warmup + cycles * (leap + corr)
    phi0 = spinodal(n, seed)
    s = lbnop.Surrogate(n, n, max_batch=max(1, turns), scale=SCALE)
    s.set_params(theta)
    s.set_leap_turns(turns)
    plain = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    lept = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    # warm-up (kernels loaded, clocks up), then timed runs from fresh initial states
    plain.init_field(phi0)
    plain.step(200)
    judge = lbnop.make_judge(leap_steps=leap, audit_every=audit_every, phi_rtol=phi_rtol, **JUDGE)

    def run_leaps(k):
        if judged:
            return s.leap_run_judged(lept, alpha, k, corr, judge)
        s.leap_run(lept, alpha, k, corr)
        return None

    lept.init_field(phi0)
    run_leaps(2)
    plain.init_field(phi0)
    lept.init_field(phi0)
    m0 = plain.mass()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(s.stream)
    plain.step(steps)
    ev[1].record(s.stream)
    lept.step(warmup)
    stats = run_leaps(cycles)
    ev[2].record(s.stream)
    torch.cuda.synchronize()
    t_plain = ev[0].elapsed_time(ev[1]) / 1e3
    t_leap = ev[1].elapsed_time(ev[2]) / 1e3
    a, b = plain.field(), lept.field()
    e_plain, e_leap = plain.free_energy(), lept.free_energy()
    m_leap = lept.mass()
    out = {
        "alpha": alpha, "seed": seed, "n": n, "steps": steps, "warmup": warmup, "cycles": cycles, "leap": leap,
        "corr": corr,
        "phi_rel_l2": float(np.linalg.norm(b - a) / np.linalg.norm(a)),
        "energy_rel_diff": float(abs(e_leap - e_plain) / abs(e_plain)),
        "energy_plain": e_plain, "energy_leap": e_leap,
        "mass_drift_rel": float(abs(m_leap - m0) / max(abs(m0), 1e-300)),
        "mass_drift_abs": float(abs(m_leap - m0)),
        "seconds_plain": t_plain, "seconds_leap": t_leap, "speedup": t_plain / t_leap,
        "phi_rms_plain": float(np.sqrt(np.mean(a * a))),
        "judge": stats, "steps_taken": lept.steps_taken, "turns": turns,
    }
    plain.close()
    lept.close()
    s.close()
    return out


def time_kernels(theta, n: int = 512, batch: int = 16, reps: int = 20):
    """Mean device time (CUDA events) of one leap forward of a single field and of one
    training step on `batch` fields, both n x n."""
    import torch

    s = lbnop.Surrogate(n, n, max_batch=batch, scale=SCALE)
    s.set_params(theta)
    r = np.random.default_rng(0)
    x1 = torch.from_numpy(r.uniform(-0.05, 0.05, (1, n, n)).astype(np.float32)).cuda()
    xb = torch.from_numpy(r.uniform(-0.05, 0.05, (batch, n, n)).astype(np.float32)).cuda()
    out1 = torch.empty_like(x1)

    def clock(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(k):
            fn()
        e1.record(s.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k * 1e3

    fwd = clock(lambda: s.forward(x1, [0.3], out1), reps)
    step = clock(lambda: s.train_step(xb, [0.3] * batch, xb, 0.0), max(1, reps // 4))
    s.close()
    return {"n": n, "forward_batch1_us": fwd, "train_step_us": step, "train_batch": batch}


def time_conv(batch: int = 16, n0: int = 128, ci: int = 96, co: int = 96, reps: int = 20):
    """Device time (CUDA events) and FP32-accumulated BF16 tensor throughput of one periodic
    3 x 3 convolution of batch x n0 x n0 pixels, c_in -> c_out (the finest level of a 512^2
    field at n0 = 128; rows of 128 pixels take the tcgen05 path). FLOPs: 2 * 9 * c_in * c_out per
    pixel."""
    import torch

    r = np.random.default_rng(1)
    x = torch.from_numpy(r.integers(-64, 65, (batch, n0, n0, ci)).astype(np.float32) / 64).cuda()
    w = torch.from_numpy(r.integers(-64, 65, (9, co, ci)).astype(np.float32) / 256).cuda()
    xb, wb = x.to(torch.bfloat16), w.to(torch.bfloat16)
    y = torch.empty((batch, n0, n0, co), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    tc0 = lbnop.lbnop_tc_launches()
    # weights packed once for the tensor-core path, as the network keeps them between refreshes
    pk = torch.empty(lbnop.lbnop_conv3x3_packed_bytes(ci, co), dtype=torch.uint8, device="cuda")
    lbnop.lbnop_conv3x3_pack(wb.data_ptr(), ci, co, pk.data_ptr(), stream.cuda_stream)

    def run():
        lbnop.lbnop_conv3x3_packed(xb.data_ptr(), wb.data_ptr(), pk.data_ptr(), None, batch, n0, n0, ci, co,
                                   y.data_ptr(), stream.cuda_stream)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / reps * 1e3
    flop = 2.0 * 9 * ci * co * batch * n0 * n0
    return {"batch": batch, "pixels": batch * n0 * n0, "c_in": ci, "c_out": co, "us": us,
            "tflops": flop / us / 1e6, "tensor_core_path": lbnop.lbnop_tc_launches() > tc0}


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", required=True)
    t.add_argument("--runs", type=int, default=32)
    t.add_argument("--n", type=int, default=512)
    t.add_argument("--iters", type=int, default=48000)
    t.add_argument("--batch", type=int, default=32)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--lr-end", type=float, default=1e-5, help="learning rate at the end of the cosine schedule")
    t.add_argument("--init", help="start from these weights (.npy) instead of a fresh initialisation")
    t.add_argument("--clip", type=float, default=CLIP, help="clip factor over the median recent norm; 0: off")
    t.add_argument("--no-augment", action="store_true", help="train without the symmetry-group turns")
    t.add_argument("--alpha-weight", type=float, default=0.0, help="draw run i with weight 1 + this * alpha_i")
    e = sub.add_parser("eval")
    e.add_argument("--theta", required=True)
    e.add_argument("--alpha", type=float, nargs="+", default=[0.3])
    e.add_argument("--seed", type=int, default=777)
    e.add_argument("--turns", type=int, default=TURNS, choices=[1, 4])
    k = sub.add_parser("time")
    k.add_argument("--theta", required=True)
    k.add_argument("--reps", type=int, default=20)
    cb = sub.add_parser("conv", help="time one 3x3 convolution (the tcgen05 path for rows of 128 pixels)")
    cb.add_argument("--batch", type=int, default=16)
    cb.add_argument("--n0", type=int, default=128)
    cb.add_argument("--ci", type=int, default=96)
    cb.add_argument("--co", type=int, default=96)
    cb.add_argument("--reps", type=int, default=20)
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    if args.cmd == "train":
        os.makedirs(args.out, exist_ok=True)
        runs = make_runs(args.runs)
        t0 = time.perf_counter()
        data = generate(runs, args.n)
        t_gen = time.perf_counter() - t0
        theta0 = np.load(args.init) if args.init else None
        theta, log = train(data, [a for a, _ in runs], args.iters, args.batch, args.lr, lr_end=args.lr_end,
                           theta0=theta0, clip=args.clip, augment=not args.no_augment,
                           alpha_weight=args.alpha_weight)
        t_train = time.perf_counter() - t0 - t_gen
        np.save(os.path.join(args.out, "leap_theta.npy"), theta.astype(np.float32))
        report = {"runs": runs, "n": args.n, "iters": args.iters, "batch": args.batch, "lr": args.lr,
                  "lr_end": args.lr_end, "init": os.path.basename(args.init) if args.init else None,
                  "clip": args.clip, "augment": not args.no_augment, "alpha_weight": args.alpha_weight,
                  "leap": LEAP, "every": EVERY, "scale": SCALE, "t_end": T_END,
                  "seconds_generate": t_gen, "seconds_train": t_train, "log": log}
        with open(os.path.join(args.out, "train_report.json"), "w") as fh:
            json.dump(report, fh, indent=1)
        for row in log:
            print(json.dumps(row))
        del data
    elif args.cmd == "time":
        print(json.dumps(time_kernels(np.load(args.theta), reps=args.reps)))
    elif args.cmd == "conv":
        print(json.dumps(time_conv(args.batch, args.n0, args.ci, args.co, args.reps)))
    else:
        theta = np.load(args.theta)
        for a in args.alpha:
            print(json.dumps(evaluate(theta, a, args.seed, turns=args.turns)))


if __name__ == "__main__":
    main()
