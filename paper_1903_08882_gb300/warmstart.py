"""Learned warm start of the steady side-heated cell.

Pipeline (all lattice work in the CUDA library, all network work in the
kernels of include/lbm_nn.h; this module sequences them):
  1. steady fields of the side-heated cell for seeded (Ra, Pr) draws, on a
     coarse (33^3) and a fine (65^3) lattice, solved by the lattice Boltzmann
     library itself (batched cells, steady criterion on the hot-wall Nu);
  2. the 3D U-Net (unet.py) trained on them with Adam: input log10(Ra), Pr and
     the coarse (u/U, v/U, w/U, T, (rho - 1)/U^2) trilinearly upsampled; target
     the fine ones.  The density deviation is part of the prediction because a
     start with the wrong density excites acoustic modes that the bulk
     viscosity damps only over ~1e5 steps;
  3. evaluation on held-out draws: steps to the steady state, at the same
     criterion, from rest, from the network's prediction, from the upsampled
     coarse solution alone, and through the judged warm start (run_judged):
     the network's and the coarse start each advance a short probe, the start
     whose fields changed least continues, and if even that one is far from
     steady the run falls back to a cold start.
Training fields are solved from the upsampled coarse solution, which reaches
the same steady state sooner.

  python -m paper_1903_08882_gb300.warmstart --train 400 --test 32 --out report.json
  python -m paper_1903_08882_gb300.warmstart --load paper_1903_08882_gb300/warmstart_unet_65.npz --test 32
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import drivers, inputs
from . import lbm as L

COARSE, FINE = 33, 65
U = 0.1


def _norm_inputs(Ra, Pr):
    return (np.log10(Ra) - 6.0), (Pr - 3.75) / 3.25


def steady_set(pairs, N, stream, group=32, every=1000, tol=1e-7, max_steps=300_000, storage="fp32", starts=None):
    """Steady fields (5, N, N, N) float32 [u/U, v/U, w/U, T, (rho-1)/U^2] for each (Ra, Pr),
    solved in batched groups, from rest or from the given start fields (the
    steady state does not depend on the start).  Returns (fields, steps,
    converged, Nu_hot); a cell that diverges gets fields None."""
    out_f, out_s, out_c, out_nu = [], [], [], []
    for g0 in range(0, len(pairs), group):
        chunk = pairs[g0:g0 + group]
        lats = [L.Lattice(N, N, N, L.walls_side_heated(), Ra=Ra, Pr=Pr, U=U, storage=storage, stream=stream)
                for Ra, Pr in chunk]
        if starts is not None:
            for k, lat in enumerate(lats):
                s0 = starts[g0 + k]
                if s0 is not None:
                    lat.set_fields(1.0 + s0[4].astype(np.float64) * U**2, s0[:3].astype(np.float64) * U,
                                   s0[3].astype(np.float64))
        prev = [None] * len(lats)
        done = [None] * len(lats)
        steps = 0
        with L.Batch(lats, stream=stream) as b:
            b.set_schedule(block_size=128, blocks_per_sm=3, steps_per_launch=100, graph_chunk=every)
            while steps < max_steps and any(d is None for d in done):
                b.step(every)
                steps += every
                for k, lat in enumerate(lats):
                    if done[k] is not None:
                        continue
                    lat.sample()
                    d = lat.diagnostics(reset=True, raise_on_diverged=False)
                    nu = d["Nu_face"][0]
                    if d["diverged"] or not np.isfinite(nu):
                        done[k] = ("diverged", steps, np.nan)
                    elif prev[k] is not None and abs(nu - prev[k]) <= tol * abs(nu):
                        done[k] = ("converged", steps, nu)
                    prev[k] = nu
        for k, lat in enumerate(lats):
            state = done[k] if done[k] is not None else ("max_steps", steps, prev[k])
            if state[0] == "diverged":
                out_f.append(None)
            else:
                rho, u3, T = lat.moments()
                out_f.append(np.concatenate([u3 / U, T[None], (rho[None] - 1.0) / U**2]).astype(np.float32))
            out_s.append(state[1])
            out_c.append(state[0] == "converged")
            out_nu.append(state[2])
            lat.close()
    return out_f, out_s, out_c, out_nu


def upsample(coarse):
    """Coarse fields (5, n, n, n) -> (5, FINE, FINE, FINE) on the GPU (trilinear kernel)."""
    import torch

    from .unet import trilinear

    y = torch.empty((5, FINE, FINE, FINE), device="cuda")
    trilinear(torch.from_numpy(coarse).cuda(), y)
    return y


class Trainer:
    def __init__(self, seed=0):
        import torch

        from .unet import UNet

        self.torch = torch
        self.net = UNet((FINE, FINE, FINE), seed=seed)

    # per-channel scale of the five field channels (inputs and targets alike):
    # the inverse standard deviation of each fine field over the training set
    scale = np.ones(5, dtype=np.float32)

    def upsample(self, coarse):
        return upsample(coarse)

    def make_input(self, coarse, Ra, Pr):
        torch = self.torch
        x = torch.empty((7, FINE, FINE, FINE), device="cuda")
        a, b = _norm_inputs(Ra, Pr)
        x[0].fill_(a)
        x[1].fill_(b)
        x[2:7] = self.upsample(coarse) * torch.from_numpy(self.scale).cuda().view(5, 1, 1, 1)
        return x

    def set_scale(self, fine_list):
        acc = np.zeros(5)
        for f in fine_list:
            acc += (f.astype(np.float64) ** 2).mean(axis=(1, 2, 3))
        self.scale = (1.0 / np.sqrt(acc / len(fine_list) + 1e-30)).astype(np.float32)

    def target(self, fine):
        return self.torch.from_numpy(fine * self.scale.reshape(5, 1, 1, 1)).cuda()

    def fit(self, xs, ys, epochs=60, lr=2e-3, lr_min=2e-5, batch=8, seed=0, log=None):
        """Adam with a cosine learning-rate decay from lr to lr_min."""
        rng = np.random.default_rng(seed)
        net = self.net
        hist = []
        for ep in range(epochs):
            lr_ep = lr_min + 0.5 * (lr - lr_min) * (1 + np.cos(np.pi * ep / max(epochs - 1, 1)))
            order = rng.permutation(len(xs))
            tot = 0.0
            for k0 in range(0, len(order), batch):
                net.zero_grad()
                for k in order[k0:k0 + batch]:
                    net.forward(xs[k])
                    tot += net.backward(xs[k], ys[k]).item()
                # the accumulated gradient is a sum over the batch
                net.adam_step(lr_ep / batch)
            hist.append(tot / len(xs))
            if log:
                log(f"epoch {ep} loss {hist[-1]:.3e}")
        return hist

    def predict(self, x):
        out = self.net.forward(x)
        return out.detach().cpu().numpy() / self.scale.reshape(5, 1, 1, 1)

    def save(self, path):
        np.savez_compressed(path, scale=self.scale,
                            **{k: p["wb"].cpu().numpy() for k, p in self.net.params.items()},
                            **{k + "_b": p["b"].cpu().numpy() for k, p in self.net.params.items()})

    def load(self, path):
        torch = self.torch
        z = np.load(path)
        self.scale = z["scale"].astype(np.float32)
        for k, p in self.net.params.items():
            p["wb"].copy_(torch.from_numpy(z[k]))
            p["b"].copy_(torch.from_numpy(z[k + "_b"]))


def start_fields(fields):
    """(rho, u3, T) of a predicted or interpolated start.  The lattice
    Boltzmann step conserves mass exactly, so the density deviation is
    shifted to zero mean: the start then holds the mass of the cold start
    (rho0 = 1 everywhere) and converges to the same steady state."""
    drho = fields[4].astype(np.float64)
    return 1.0 + (drho - drho.mean()) * U**2, fields[:3].astype(np.float64) * U, fields[3].astype(np.float64)


def run_from(Ra, Pr, fields, stream, tol=1e-7, fallback_tol=None, max_steps=400_000):
    """Steps to the steady state from `fields` (None: from rest)."""
    with L.Lattice(FINE, FINE, FINE, L.walls_side_heated(), Ra=Ra, Pr=Pr, U=U, stream=stream) as lat:
        fell_back = False
        if fields is not None:
            lat.set_fields(*start_fields(fields))
            if fallback_tol is not None:
                lat.sample()
                nu0 = lat.diagnostics()["Nu_face"][0]
                lat.step(1000)
                lat.sample()
                nu1 = lat.diagnostics()["Nu_face"][0]
                if not np.isfinite(nu1) or abs(nu1 - nu0) > fallback_tol * abs(nu1):
                    fell_back = True
                    lat.set_fields(1.0, np.zeros(3), 0.0)
        r = drivers.run_to_steady(lat, every=1000, tol=tol, max_steps=max_steps)
        extra = 1000 if (fields is not None and fallback_tol is not None) else 0
        return dict(steps=r["steps"] + extra, converged=r["converged"], Nu=float(r["Nu"]), fell_back=fell_back)


def _residual(a, b):
    """Sec. 3 steady residuals between two moment sets (rho, u3, T): the
    relative change of the velocity (sum of |du|_2) and of T (L1)."""
    du, dT = drivers.field_residuals(a[1], b[1], a[2], b[2])
    return max(du, dT)


def run_judged(Ra, Pr, pred, coarse_up, stream, probe=2000, fallback=0.5, tol=1e-7, max_steps=400_000):
    """Warm start with a judge: both candidate starts (the network's
    prediction and the upsampled coarse solution) advance `probe` steps; the
    one whose fields changed least continues to the steady state.  When even
    that change exceeds `fallback` (a start that is plainly wrong: the fields
    change by half their size in the probe) the run restarts from rest.
    Every step taken counts in the returned total."""
    lats, res = [], []
    try:
        for fields in (pred, coarse_up):
            lat = L.Lattice(FINE, FINE, FINE, L.walls_side_heated(), Ra=Ra, Pr=Pr, U=U, stream=stream)
            lat.set_fields(*start_fields(fields))
            m0 = lat.moments()
            lat.step(probe)
            res.append(_residual(lat.moments(), m0))
            lats.append(lat)
        best = int(np.argmin(res))
        chosen = ["network", "coarse"][best]
        lat = lats[best]
        spent = 2 * probe
        if not np.isfinite(res[best]) or res[best] > fallback:
            chosen = "cold"
            lat.set_fields(1.0, np.zeros(3), 0.0)
        r = drivers.run_to_steady(lat, every=1000, tol=tol, max_steps=max_steps)
        return dict(steps=r["steps"] + spent, converged=r["converged"], Nu=float(r["Nu"]), chosen=chosen,
                    residuals=[float(x) for x in res])
    finally:
        for lat in lats:
            lat.close()


def evaluate(trainer, test_pairs, coarse, stream, log, starts=("network", "coarse", "judged")):
    """Steps to the steady state from rest and from each requested start."""
    results = []
    for k, (Ra, Pr) in enumerate(test_pairs):
        c = coarse[k]
        if c is None:
            results.append(dict(Ra=Ra, Pr=Pr, skipped="coarse solve diverged"))
            continue
        x = trainer.make_input(c, Ra, Pr)
        pred = trainer.predict(x)
        up = upsample(c).cpu().numpy()
        cold = run_from(Ra, Pr, None, stream)
        r = dict(Ra=Ra, Pr=Pr, cold=cold)
        if "network" in starts:
            r["network"] = run_from(Ra, Pr, pred, stream)
            r["speedup_network"] = cold["steps"] / max(r["network"]["steps"], 1)
        if "coarse" in starts:
            r["upsampled_coarse"] = run_from(Ra, Pr, up, stream)
            r["speedup_coarse"] = cold["steps"] / max(r["upsampled_coarse"]["steps"], 1)
        if "judged" in starts:
            r["judged"] = run_judged(Ra, Pr, pred, up, stream)
            r["speedup_judged"] = cold["steps"] / max(r["judged"]["steps"], 1)
        results.append(r)
        log(f"test {k}: Ra {Ra:.3g} Pr {Pr:.2f} cold {cold['steps']} Nu {cold['Nu']:.5f} " +
            " ".join(f"{key} {r[key]['steps']} (Nu {r[key]['Nu']:.5f})"
                     for key in ("network", "upsampled_coarse", "judged") if key in r))
    return results


def summarize(results):
    out = {}
    for key in ("speedup_network", "speedup_judged", "speedup_coarse"):
        v = np.array([r[key] for r in results if key in r])
        if len(v):
            out[key] = dict(median=float(np.median(v)), mean=float(v.mean()), geomean=float(np.exp(np.log(v).mean())),
                            frac_ge_3=float((v >= 3).mean()), n=int(len(v)))
    return out


def main():
    global FINE
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--seed", type=int, default=190308882)
    ap.add_argument("--out", default="warmstart_report.json")
    ap.add_argument("--weights", default=None, help="save the trained BF16 weights (npz)")
    ap.add_argument("--load", default=None, help="evaluate stored weights instead of training")
    ap.add_argument("--fine", type=int, default=FINE, help="edge of the fine lattice (the network's output)")
    ap.add_argument("--starts", default="network,coarse,judged",
                    help="warm starts to evaluate against the cold start (comma-separated)")
    args = ap.parse_args()
    FINE = args.fine
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.1f}s] {m}", flush=True)  # noqa: E731
    stream = torch.cuda.Stream()
    report = {"coarse": COARSE, "fine": FINE, "U": U}
    with torch.cuda.stream(stream):
        pairs = inputs.warmstart_pairs(args.seed, args.train + args.test + 64)
        # the held-out set ends with the case the FP64 oracle has a steady state for
        test_pairs = pairs[args.train:args.train + args.test - 1] + [(1e6, 0.71)]
        train_pairs = pairs[:args.train]
        if args.load:
            cf, _, _, _ = steady_set(test_pairs, COARSE, stream)
            trainer = Trainer(seed=1)
            trainer.load(args.load)
            report["weights"] = args.load
            results = evaluate(trainer, test_pairs, cf, stream, log, starts=args.starts.split(","))
        else:
            log(f"coarse solves: {len(train_pairs) + len(test_pairs)}")
            cf, cs, cc, _ = steady_set(train_pairs + test_pairs, COARSE, stream)
            log(f"coarse done: converged {sum(cc)}, diverged {sum(f is None for f in cf)}")
            tr = [i for i in range(len(train_pairs)) if cf[i] is not None]
            starts = [upsample(cf[i]).cpu().numpy() for i in tr]
            ff, fs, fc, fnu = steady_set([train_pairs[i] for i in tr], FINE, stream, starts=starts)
            del starts
            log(f"fine training solves done: converged {sum(fc)}, mean steps {np.mean(fs):.0f}")
            keep = [j for j in range(len(tr)) if ff[j] is not None]
            trainer = Trainer(seed=1)
            trainer.set_scale([ff[j] for j in keep])
            report["channel_scale"] = trainer.scale.tolist()
            xs = [trainer.make_input(cf[tr[j]], *train_pairs[tr[j]]) for j in keep]
            ys = [trainer.target(ff[j]) for j in keep]
            report["train_samples"] = len(xs)
            report["loss_history"] = trainer.fit(xs, ys, epochs=args.epochs, log=log)
            del xs, ys
            if args.weights:
                trainer.save(args.weights)
            results = evaluate(trainer, test_pairs, cf[len(train_pairs):], stream, log,
                               starts=args.starts.split(","))
        report["tests"] = results
        report["summary"] = summarize(results)
        report["wall_seconds"] = round(time.time() - t0, 1)
    with open(args.out, "w") as fh:
        json.dump(report, fh, indent=1)
    log(f"summary {json.dumps(report['summary'])}")


if __name__ == "__main__":
    main()
