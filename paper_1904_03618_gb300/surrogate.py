"""Learned surrogate of droplet impact: (density ratio, viscosity ratio,
Weber, Reynolds, contact angle) -> spreading-factor series D(t)/D0.

The solver generates its own training data: every sampled parameter set
becomes one case of a batched run (a red drop falling onto a bounce-back
floor with the contact-angle wetting rule), and the wetted footprint on the
floor -- the cells of the first fluid layer where rho^N > 0, counted by
lbm_batch_footprint -- gives D = 2 sqrt(area / pi) at K sample times.  The
network (dense tanh layers, BF16 tensor-core GEMMs with FP32 accumulation,
Adam on MSE; lbm_mlp_*) is trained on the GPU by the library's own forward
and backward kernels.  The solver stays the fallback and the reference:
the held-out error is measured against solver runs the network never saw.

The paper has no counterpart; it fixes only the step that produces the data.

Dimensionless groups (drop = red, density rho_d = lambda, gas density 1,
drop diameter D0 = 2 R, impact speed U0, all in lattice units):
  We = rho_d U0^2 D0 / sigma,  Re = rho_d U0 D0 / mu_d,
  lambda = rho_d / rho_g,      M = mu_d / mu_g,
with mu_k = rho_k nu_k and nu_k = (c_s^k)^2 (tau_k - 1/2) (below Eq. 52),
sigma = 2 (A_R + A_B) / 9 and alpha_R from the pressure balance of Eq. 13.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lbm
from . import params as P

# sampled box of the five inputs (log-uniform for the first four)
RANGES = {"density_ratio": (1.0, 20.0), "viscosity_ratio": (1.0, 50.0),
          "weber": (10.0, 100.0), "reynolds": (20.0, 200.0), "theta_deg": (60.0, 150.0)}
TAU_MIN, TAU_MAX = 0.51, 3.0
ALPHA_B = 0.2


@dataclass
class ImpactSetup:
    radius: int = 8            # drop radius R (D0 = 2R)
    box: tuple = (64, 64, 32)  # nx, ny, nz; floor wall at z = 0 (walls in z)
    speed: float = 0.04        # impact speed U0
    t_end: float = 4.0         # last sample time in units of D0 / U0
    samples: int = 16          # K sample times t_k = k t_end / K, k = 1..K
    gap: int = 2               # gas layers between floor and drop at t = 0
    storage: str = "f32"
    beta: float = 0.7

    @property
    def steps(self) -> int:
        return int(round(self.t_end * 2 * self.radius / self.speed))

    @property
    def sample_steps(self) -> list:
        return [int(round(self.steps * (k + 1) / self.samples)) for k in range(self.samples)]


def relaxation_times(s: dict, setup: ImpactSetup):
    lam, M, Re = s["density_ratio"], s["viscosity_ratio"], s["reynolds"]
    D0 = 2.0 * setup.radius
    alpha_R = P.alpha_R_from_balance(lam, 1.0, ALPHA_B)
    nu_d = setup.speed * D0 / Re              # mu_d / rho_d
    nu_g = nu_d * lam / M                     # mu_g / rho_g with rho_g = 1
    return (P.tau_from_nu(nu_d, alpha_R), P.tau_from_nu(nu_g, ALPHA_B), alpha_R)


def sample_impacts(n: int, setup: ImpactSetup, seed: int = 2024, ranges: dict = None) -> list:
    """n parameter sets drawn from `ranges` (default RANGES), keeping those
    whose relaxation times lie in [TAU_MIN, TAU_MAX] (the stable window of
    the solver)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        s = {}
        for k, (lo, hi) in (ranges or RANGES).items():
            if k == "theta_deg":
                s[k] = float(rng.uniform(lo, hi))
            else:
                s[k] = float(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        tR, tB, _ = relaxation_times(s, setup)
        if TAU_MIN <= tR <= TAU_MAX and TAU_MIN <= tB <= TAU_MAX:
            out.append(s)
    return out


def impact_params(s: dict, setup: ImpactSetup):
    """lbm_params of one impact."""
    nx, ny, nz = setup.box
    R, U0 = setup.radius, setup.speed
    lam = s["density_ratio"]
    tR, tB, alpha_R = relaxation_times(s, setup)
    sigma = lam * U0 * U0 * 2 * R / s["weber"]
    A = P.A_from_sigma(sigma)
    return lbm.make_params(nx, ny, nz, wall=(0, 0, 1), improved=True, storage=setup.storage,
                           rho_in_R=lam, rho_in_B=1.0, alpha_R=alpha_R, alpha_B=ALPHA_B,
                           tau_R=tR, tau_B=tB, A_R=A, A_B=A, beta=setup.beta, delta=0.98,
                           wetting=True, contact_angle_deg=s["theta_deg"],
                           ref_R=0.0, ref_B=1.0)


def impact_fields(s: dict, setup: ImpactSetup):
    """Initial fields (rho_R, rho_B, u) of one impact, float32 (z, y, x): a
    sphere of radius R, `gap` layers above the floor, moving at -U0 in z.
    The sphere test runs on broadcast coordinates (integers and halves,
    exact in float32), so a 256 x 256 x 160 box costs its three fields and
    no coordinate grids."""
    nx, ny, nz = setup.box
    R, U0 = setup.radius, setup.speed
    lam = s["density_ratio"]
    c = ((nx - 1) / 2.0, (ny - 1) / 2.0, setup.gap + R)
    x = np.arange(nx, dtype=np.float32)[None, None, :]
    y = np.arange(ny, dtype=np.float32)[None, :, None]
    z = np.arange(nz, dtype=np.float32)[:, None, None]
    inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= R * R
    rho_R = np.where(inside, np.float32(lam), np.float32(0.0))
    rho_B = np.where(inside, np.float32(0.0), np.float32(1.0))
    u = np.zeros((3, nz, ny, nx), dtype=np.float32)
    u[2][inside] = -U0
    return rho_R, rho_B, u


def impact_case(s: dict, setup: ImpactSetup):
    """lbm_params and initial fields (rho_R, rho_B, u) of one impact."""
    return impact_params(s, setup), impact_fields(s, setup)


@dataclass
class ImpactRuns:
    samples: list
    series: np.ndarray            # (n, K) D(t_k) / D0, NaN for unstable cases
    valid: np.ndarray             # (n,) bool
    seconds: float                # solver wall time (all cases)
    cell_updates: float           # lattice cell updates performed
    setup: ImpactSetup = field(default_factory=ImpactSetup)

    @property
    def seconds_per_case(self) -> float:
        return self.seconds / max(len(self.samples), 1)


def run_impacts(samples: list, setup: ImpactSetup, chunk: int = 512, device=None,
                log=None) -> ImpactRuns:
    """Runs every sample through the batched solver and records D(t)/D0."""
    dev = torch.device(device or "cuda")
    K = setup.samples
    series = np.full((len(samples), K), np.nan)
    valid = np.zeros(len(samples), dtype=bool)
    D0 = 2.0 * setup.radius
    total = 0.0
    cells = 0.0
    for c0 in range(0, len(samples), chunk):
        part = samples[c0:c0 + chunk]
        stream = torch.cuda.Stream(dev)
        b = lbm.Batch([impact_params(s, setup) for s in part], device=dev, stream=stream)
        try:
            # fields built one case at a time: a chunk of full-size boxes
            # would otherwise hold tens of GB of host arrays
            for k, s in enumerate(part):
                b.init_fields(k, *impact_fields(s, setup))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            done = 0
            for j, st in enumerate(setup.sample_steps):
                b.step(st - done)
                done = st
                area = b.footprint(axis=2, index=0).astype(np.float64)
                series[c0:c0 + len(part), j] = 2.0 * np.sqrt(area / math.pi) / D0
            torch.cuda.synchronize(dev)
            total += time.perf_counter() - t0
            cells += float(np.prod(setup.box)) * len(part) * done
            for k in range(len(part)):
                d = b.diagnostics(k, raise_unstable=False)
                valid[c0 + k] = d[5] == 0 and d[6] == 0
        finally:
            b.close()
        if log:
            log("impacts %d-%d: %.1f s so far" % (c0, c0 + len(part) - 1, total))
    series[~valid] = np.nan
    return ImpactRuns(samples, series, valid, total, cells, setup)


def features(samples: list) -> np.ndarray:
    """Inputs scaled to [-1, 1]: logs of the four ratios, the angle linearly."""
    X = np.zeros((len(samples), 5))
    for i, s in enumerate(samples):
        for j, k in enumerate(RANGES):
            lo, hi = RANGES[k]
            v, a, b = (s[k], lo, hi) if k == "theta_deg" else \
                (math.log(s[k]), math.log(lo), math.log(hi))
            X[i, j] = 2.0 * (v - a) / (b - a) - 1.0
    return X


class Surrogate:
    """Dense tanh network on the tensor cores with standardised outputs."""

    def __init__(self, n_out: int, width: int = 256, depth: int = 4, max_batch: int = 1 << 16,
                 seed: int = 7, device=None):
        self.n_in, self.n_out, self.width, self.depth = 5, n_out, width, depth
        self.dev = torch.device(device or "cuda")
        self.max_batch = max_batch
        with torch.cuda.device(self.dev):
            self.stream = torch.cuda.Stream(self.dev)
            self.m = lbm.lbm_mlp_create(self.n_in, width, depth, n_out, max_batch,
                                        self.stream.cuda_stream)
        rng = np.random.default_rng(seed)
        dims = [self.n_in] + [width] * depth + [n_out]
        parts = []
        for a, b in zip(dims[:-1], dims[1:]):
            parts.append(rng.uniform(-1, 1, a * b) * math.sqrt(6.0 / (a + b)))
            parts.append(np.zeros(b))
        theta = np.concatenate(parts).astype(np.float32)
        assert theta.size == lbm.lbm_mlp_num_params(self.m)
        lbm.lbm_mlp_set_params(self.m, theta)
        self.y_mean = np.zeros(n_out)
        self.y_std = np.ones(n_out)

    def fit(self, X: np.ndarray, Y: np.ndarray, steps: int = 3000, lr: float = 1e-3,
            batch: int = 256, seed: int = 0, lr_final: float = 1e-5) -> list:
        """Adam on minibatches drawn with replacement; cosine learning-rate
        decay from lr to lr_final.  Returns the loss every 100 steps."""
        self.y_mean = Y.mean(axis=0)
        self.y_std = Y.std(axis=0) + 1e-6
        Yn = (Y - self.y_mean) / self.y_std
        Xd = torch.as_tensor(X, dtype=torch.float32, device=self.dev)
        Yd = torch.as_tensor(Yn, dtype=torch.float32, device=self.dev)
        n = X.shape[0]
        batch = min(batch, n, self.max_batch)
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        losses = []
        with torch.cuda.stream(self.stream):
            idx_all = torch.randint(0, n, (steps, batch), device=self.dev, generator=g)
            xb = torch.empty((batch, self.n_in), device=self.dev)
            yb = torch.empty((batch, self.n_out), device=self.dev)
            for it in range(steps):
                torch.index_select(Xd, 0, idx_all[it], out=xb)
                torch.index_select(Yd, 0, idx_all[it], out=yb)
                rate = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / steps))
                want = (it % 100 == 0) or it == steps - 1
                loss = lbm.lbm_mlp_train_step(self.m, xb, yb, batch, rate, want_loss=want)
                if want:
                    losses.append(loss)
        self.stream.synchronize()
        return losses

    def predict_device(self, Xd: torch.Tensor) -> torch.Tensor:
        """Normalised-space forward pass of device inputs, de-standardised."""
        n = Xd.shape[0]
        out = torch.empty((n, self.n_out), device=self.dev)
        with torch.cuda.stream(self.stream):
            for s in range(0, n, self.max_batch):
                e = min(n, s + self.max_batch)
                lbm.lbm_mlp_forward(self.m, Xd[s:e].contiguous(), e - s, out[s:e])
        self.stream.synchronize()
        return out

    def predict(self, X: np.ndarray) -> np.ndarray:
        Xd = torch.as_tensor(X, dtype=torch.float32, device=self.dev)
        Yn = self.predict_device(Xd).cpu().double().numpy()
        return Yn * self.y_std + self.y_mean

    def close(self):
        if self.m is not None:
            lbm.lbm_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def split(n: int, holdout: float = 0.2, seed: int = 99):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    k = int(round(n * holdout))
    return perm[k:], perm[:k]


def evaluate(Y_true: np.ndarray, Y_pred: np.ndarray) -> dict:
    err = Y_pred - Y_true
    return {"rmse": float(np.sqrt(np.mean(err ** 2))),
            "mae": float(np.mean(np.abs(err))),
            "max_abs": float(np.max(np.abs(err))),
            "rel_l2": float(np.linalg.norm(err) / np.linalg.norm(Y_true))}


def screen(Y_true: np.ndarray, Y_pred: np.ndarray, quantile: float = 0.8,
           flag_fraction: float = 0.3) -> dict:
    """Sweep screening: find the cases whose maximum spreading factor lies in
    the top (1 - quantile) of the solver's own results.  The surrogate flags
    the top `flag_fraction` of its predictions; only those would be re-run
    with the solver.  Returns the recall of the true top cases and the share
    of solver runs saved."""
    true_max = Y_true.max(axis=1)
    pred_max = Y_pred.max(axis=1)
    thr = np.quantile(true_max, quantile)
    top = true_max >= thr
    nflag = int(math.ceil(flag_fraction * len(pred_max)))
    flagged = np.zeros(len(pred_max), dtype=bool)
    flagged[np.argsort(-pred_max)[:nflag]] = True
    return {"recall": float((top & flagged).sum() / max(top.sum(), 1)),
            "solver_runs_saved": float(1.0 - flagged.mean()),
            "top_cases": int(top.sum()), "flagged": int(nflag)}


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Generate impact data with the solver, train "
                                             "the tensor-core surrogate, report held-out error")
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--radius", type=int, default=8)
    ap.add_argument("--box", type=int, nargs=3, default=[64, 64, 32])
    ap.add_argument("--speed", type=float, default=0.04)
    ap.add_argument("--t-end", type=float, default=4.0)
    ap.add_argument("--steps", type=int, default=4000, help="training steps")
    ap.add_argument("--chunk", type=int, default=512)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--series", type=int, default=16, help="sample times K per run")
    ap.add_argument("--density-max", type=float, default=RANGES["density_ratio"][1])
    ap.add_argument("--reynolds", type=float, nargs=2, default=list(RANGES["reynolds"]))
    ap.add_argument("--out", default=None, help="write the report (JSON) here")
    args = ap.parse_args(argv)
    setup = ImpactSetup(radius=args.radius, box=tuple(args.box), speed=args.speed,
                        t_end=args.t_end, samples=args.series)
    ranges = dict(RANGES, density_ratio=(RANGES["density_ratio"][0], args.density_max),
                  reynolds=tuple(args.reynolds))
    samples = sample_impacts(args.samples, setup, seed=args.seed, ranges=ranges)
    runs = run_impacts(samples, setup, chunk=args.chunk,
                       log=lambda m: print(m, flush=True))
    rep = report(runs, train_steps=args.steps)
    print(json.dumps(rep))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(rep, fh, indent=1)


def report(runs: ImpactRuns, train_steps: int = 4000, width: int = 256, depth: int = 4) -> dict:
    """Trains on the stable runs, evaluates on the held-out split and times
    the surrogate against the solver."""
    ok = np.flatnonzero(runs.valid)
    X = features([runs.samples[i] for i in ok])
    Y = runs.series[ok]
    tr, te = split(len(ok))
    sur = Surrogate(Y.shape[1], width=width, depth=depth)
    try:
        t0 = time.perf_counter()
        losses = sur.fit(X[tr], Y[tr], steps=train_steps)
        t_train = time.perf_counter() - t0
        pred = sur.predict(X[te])
        # inference throughput on a large synthetic sweep (inputs on the device)
        sweep = torch.rand((1 << 16, 5), device=sur.dev) * 2 - 1
        sur.predict_device(sweep)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 5
        for _ in range(reps):
            sur.predict_device(sweep)
        torch.cuda.synchronize()
        t_inf = (time.perf_counter() - t0) / (reps * sweep.shape[0])
    finally:
        sur.close()
    mean_pred = np.broadcast_to(Y[tr].mean(axis=0), Y[te].shape)
    # linear least squares on the same inputs: the cheapest learned baseline
    A = np.hstack([X[tr], np.ones((len(tr), 1))])
    coef, *_ = np.linalg.lstsq(A, Y[tr], rcond=None)
    lin_pred = np.hstack([X[te], np.ones((len(te), 1))]) @ coef
    lo_hi = lambda k: [min(sm[k] for sm in runs.samples), max(sm[k] for sm in runs.samples)]  # noqa: E731
    return {
        "sampled_ranges": {k: lo_hi(k) for k in RANGES},
        "setup": {"radius": runs.setup.radius, "box": list(runs.setup.box),
                  "speed": runs.setup.speed, "steps": runs.setup.steps,
                  "sample_steps": runs.setup.sample_steps, "storage": runs.setup.storage},
        "cases": len(runs.samples), "stable": int(runs.valid.sum()),
        "train": int(len(tr)), "held_out": int(len(te)),
        "solver_seconds": runs.seconds, "solver_seconds_per_case": runs.seconds_per_case,
        "solver_mlups": runs.cell_updates / runs.seconds / 1e6 if runs.seconds > 0 else None,
        "train_seconds": t_train, "train_steps": train_steps, "loss_trace": losses,
        "surrogate_seconds_per_case": t_inf,
        "speedup_vs_solver": runs.seconds_per_case / t_inf,
        "held_out_error": evaluate(Y[te], pred),
        "mean_predictor_error": evaluate(Y[te], mean_pred),
        "linear_fit_error": evaluate(Y[te], lin_pred),
        "screening": screen(Y[te], pred),
    }


if __name__ == "__main__":
    main()
