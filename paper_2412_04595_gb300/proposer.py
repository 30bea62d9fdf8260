"""Learned proposal of the near-field neighbour count n_nb, and hence of the
cutoff r_c and of everything the analytic selection (Sec. 4.3) derives from
it: mid grid, window support, split index m, Chebyshev order.

The analytic selection sizes each part for the tolerance; n_nb only moves
work between the near field and the spectral parts.  The best n_nb depends
on the system (size, aspect ratio, density, z structure) and on the GPU, so
it is learned from timings of the library itself: each training system is
timed at several candidate n_nb, and the network (sog_mlp_* in the C ABI,
trained by its own kernels) learns the log evaluation time from the
features of sog_features and the work that the analytic parameters of the
candidate imply (near-field pairs, grid points, spreading work).  The
proposal is the candidate of least predicted time; outside the range the
model was trained on, without a trained network, or when the predicted
saving is small, the proposal falls back to the analytic default.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B

CANDIDATES = (40.0, 60.0, 80.0, 100.0, 120.0, 160.0, 220.0)
DEFAULT_NNB = 120.0
NNB_RANGE = (30.0, 300.0)


def time_eval(N, L, tol, q, r, n_nb, precision=B.SOG_PREC_MIXED, reps=5):
    """Median device time (ms) of one evaluation of energy and forces with
    the analytic parameters for n_nb, or None if no feasible plan exists."""
    import torch
    try:
        plan = B.Plan(N, L, tol, precision=precision, n_nb=n_nb)
    except B.SogError:
        return None
    dev = q.device
    phi = torch.empty(N, dtype=q.dtype, device=dev)
    F = torch.empty(N, 3, dtype=q.dtype, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(2):
        plan.eval(q, r, phi, E, F)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.eval(q, r, phi, E, F)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ok = plan.check() == 0
    plan.close()
    return float(np.median(times)) if ok else None


N_INPUTS = B.N_FEATURES + 5


def cand_features(sys_feat, N, L, tol, n_nb):
    """Inputs of the cost model for one candidate n_nb: the system features
    and log10 of the work the analytic parameters for n_nb imply: near-field
    pairs, mid grid points, mid spreading work N P^3, long-range proxy grid
    points P_cheb I_long^2 and long-range spreading work N P_cheb P_long^2.
    None if n_nb has no feasible parameter set."""
    try:
        p = B.sog_select_params(N, *L, tol, n_nb=n_nb)
    except B.SogError:
        return None
    rho = N / (L[0] * L[1] * L[2])
    pairs = N * 4.0 / 3.0 * math.pi * p["rc"] ** 3 * rho
    mid = p["m"] >= 0
    mid_pts = p["I"][0] * p["I"][1] * p["I"][2] if mid else 1
    mid_work = N * p["P_win"] ** 3 if mid else 1
    long_ = p["m"] < p["M"]
    long_pts = p["P_cheb"] * p["I_long"][0] * p["I_long"][1] if long_ else 1
    long_work = N * p["P_cheb"] * p["P_long"] ** 2 if long_ else 1
    return list(sys_feat) + [math.log10(max(v, 1.0)) for v in
                             (pairs, mid_pts, mid_work, long_pts, long_work)]


def measure(systems, tol, precision=B.SOG_PREC_MIXED, candidates=CANDIDATES, reps=5):
    """For a list of systems [(q, r, L)] (NumPy): cost-model inputs Z and
    log evaluation times Y (ms) of every feasible (system, candidate), and
    the table of times [n_systems x len(candidates)] (NaN where infeasible)."""
    import torch
    dt = torch.float64 if precision == B.SOG_PREC_FP64 else torch.float32
    Z, Y, tab = [], [], []
    for q, r, L in systems:
        N = q.size
        qt = torch.tensor(q, dtype=dt, device="cuda")
        rt = torch.tensor(r, dtype=dt, device="cuda")
        feat = B.sog_features(N, L, tol, rt)
        row = []
        for c in candidates:
            z = cand_features(feat, N, L, tol, c)
            t = time_eval(N, L, tol, qt, rt, c, precision, reps) if z is not None else None
            row.append(t if t is not None else float("nan"))
            if t is not None:
                Z.append(z)
                Y.append(math.log(t))
        tab.append(row)
    return np.array(Z, dtype=np.float64), np.array(Y, dtype=np.float64), np.array(tab)


class Proposer:
    """A learned cost model: log evaluation time from the system features and
    the work implied by the analytic parameters of a candidate n_nb.  The
    proposal is the candidate of least predicted time; the analytic default
    is kept unless the predicted saving is at least `margin`."""

    def __init__(self, n_hidden=32, seed=0, margin=0.03):
        self.mlp = B.MLP(N_INPUTS, n_hidden, seed)
        self.trained = False
        self.margin = margin

    def fit(self, Z, Y, iters=3000, lr=1e-2, candidates=CANDIDATES):
        import torch
        Z = np.asarray(Z, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.z_mu, self.z_sd = Z.mean(0), Z.std(0) + 1e-6
        self.y_mu, self.y_sd = Y.mean(), Y.std() + 1e-6
        self.z_lo, self.z_hi = Z.min(0), Z.max(0)
        self.candidates = tuple(candidates)
        Zn = torch.tensor((Z - self.z_mu) / self.z_sd, dtype=torch.float32, device="cuda")
        Yn = torch.tensor((Y - self.y_mu) / self.y_sd, dtype=torch.float32, device="cuda")
        loss = self.mlp.train(Zn, Yn, iters, lr)
        self.trained = True
        return loss

    def covers(self, z):
        """True when every input lies in the training range widened by a
        quarter of its span."""
        z = np.asarray(z, dtype=np.float64)
        span = self.z_hi - self.z_lo
        return bool(np.all(z >= self.z_lo - 0.25 * span - 1e-9) and
                    np.all(z <= self.z_hi + 0.25 * span + 1e-9))

    def predict(self, Z):
        """Predicted log time (ms) for rows of cost-model inputs."""
        import torch
        Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))
        Zt = torch.tensor((Z - self.z_mu) / self.z_sd, dtype=torch.float32, device="cuda")
        return self.mlp.forward(Zt).double().cpu().numpy() * self.y_sd + self.y_mu

    def propose(self, feat, N, L, tol):
        """(n_nb, source) for a system with features `feat`."""
        if not self.trained:
            return DEFAULT_NNB, "analytic"
        cands, Z = [], []
        for c in self.candidates:
            z = cand_features(feat, N, L, tol, c)
            if z is not None and self.covers(z):
                cands.append(c)
                Z.append(z)
        if DEFAULT_NNB not in cands:
            return DEFAULT_NNB, "analytic"
        pred = self.predict(Z)
        base = pred[cands.index(DEFAULT_NNB)]
        k = int(np.argmin(pred))
        if pred[k] > base + math.log(1.0 - self.margin):
            return DEFAULT_NNB, "analytic"
        return float(cands[k]), "mlp"

    def plan(self, N, L, tol, r, precision=B.SOG_PREC_MIXED):
        """A plan for the system with positions r (CUDA tensor) and its
        proposed n_nb; falls back to the analytic default if the proposal has
        no feasible plan."""
        n_nb, src = self.propose(B.sog_features(N, L, tol, r), N, L, tol)
        try:
            return B.Plan(N, L, tol, precision=precision, n_nb=n_nb), n_nb, src
        except B.SogError:
            return B.Plan(N, L, tol, precision=precision, n_nb=DEFAULT_NNB), DEFAULT_NNB, "analytic"


def training_systems(n, seed=0, nmin=5000, nmax=200000):
    """Synthetic systems for the proposer: uniform neutral charges with N
    log-uniform in [nmin, nmax], aspect ratio Lz/Lx log-uniform in [0.1, 10],
    density log-uniform in [0.03, 0.3]; every fourth one an electric double
    layer instead of uniform."""
    from . import workloads
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        N += N % 2
        a = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        rho = math.exp(rng.uniform(math.log(0.03), math.log(0.3)))
        Lx = (N / (rho * a)) ** (1.0 / 3.0)
        L = (Lx, Lx, a * Lx)
        s = int(rng.integers(1 << 31))
        if k % 4 == 3:
            q, r = workloads.edl_neutral(N, L, s, decay=max(0.5, 0.02 * L[2]))
        else:
            q, r = workloads.uniform_neutral(N, L, s)
        out.append((q, r.astype(np.float32).astype(np.float64), L))
    return out
