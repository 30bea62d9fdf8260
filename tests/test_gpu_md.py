"""Repeated evaluation for molecular dynamics (sog_md_step): velocity-Verlet
steps with the library's forces, the plan reused across steps and the
particles re-sorted into cell order every few steps.

* Ten steps on the GPU (FP64 plan) follow the same integrator driven by the
  FP64 oracle's forces (Eq. 2.28, Algorithms 1-2) to 1e-9.
* Over 400 steps the total energy (the evaluation's energy plus the kinetic
  energy) stays constant to the integrator's accuracy: the SOG split is C^1
  at the cutoff (Sec. 2.2, Eq. 2.23-2.24) and the forces are the gradient of
  the computed energy.
* Runs with and without re-sorting agree once mapped back by `order`."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L = (12.0, 12.0, 12.0)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def _gas(N, seed, dmin=0.8):
    """Neutral +-1 charges at random positions at least dmin apart (minimum
    image in x, y), Gaussian velocities of variance 0.09."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < N:
        p = np.array([rng.uniform(-L[0] / 2, L[0] / 2), rng.uniform(-L[1] / 2, L[1] / 2),
                      rng.uniform(-L[2] / 2 + 0.5, L[2] / 2 - 0.5)])
        ok = True
        for o in pts:
            d = p - o
            d[:2] -= np.array(L[:2]) * np.round(d[:2] / np.array(L[:2]))
            if d @ d < dmin * dmin:
                ok = False
                break
        if ok:
            pts.append(p)
    r = np.array(pts)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    v = rng.normal(0.0, 0.3, size=(N, 3))
    return q, r, v


def _verlet_oracle(osog, prm, q, r, v, dt, nsteps):
    """The integrator of sog_md_step with the oracle's forces, unit masses."""
    r, v = r.copy(), v.copy()
    F = osog.sog_eval(prm, q, r)["F"]
    for _ in range(nsteps):
        v += 0.5 * dt * F
        r += dt * v
        for d in (0, 1):
            r[:, d] = np.where(r[:, d] >= L[d] / 2, r[:, d] - L[d], r[:, d])
            r[:, d] = np.where(r[:, d] < -L[d] / 2, r[:, d] + L[d], r[:, d])
        hz = L[2] / 2
        hi, lo = r[:, 2] > hz, r[:, 2] < -hz
        r[hi, 2] = 2 * hz - r[hi, 2]
        r[lo, 2] = -2 * hz - r[lo, 2]
        v[hi | lo, 2] *= -1.0
        F = osog.sog_eval(prm, q, r)["F"]
        v += 0.5 * dt * F
    return r, v


def _setup(B, prm, q, r, v, N):
    dev = torch.device("cuda:0")
    plan = B.Plan(N, L, 1e-8, precision=B.SOG_PREC_FP64, manual=prm)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev).contiguous()
    qt, rt, vt = t(q), t(r), t(v)
    F = torch.empty(N, 3, dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, None, E, F)
    order = torch.arange(N, dtype=torch.int32, device=dev)
    return plan, qt, rt, vt, F, E, order


def test_md_follows_oracle_verlet(B, oracle_mod):
    N, dt, steps = 300, 1e-3, 10
    q, r, v = _gas(N, 3)
    prm = oracle_mod.select_params(N, *L, 1e-8, n_nb=60)
    plan, qt, rt, vt, F, E, order = _setup(B, prm, q, r, v, N)
    md = B.MD(plan)
    md.step(qt, rt, vt, F, dt, nsteps=steps, E=E)
    torch.cuda.synchronize()
    assert plan.check() == 0
    r_ref, v_ref = _verlet_oracle(oracle_mod, prm, q, r, v, dt, steps)
    dr = rt.cpu().numpy() - r_ref
    for d in (0, 1):  # a wrap may differ by one period at the boundary
        dr[:, d] -= L[d] * np.round(dr[:, d] / L[d])
    assert np.abs(dr).max() <= 1e-9 * max(L)
    assert np.abs(vt.cpu().numpy() - v_ref).max() <= 1e-9 * np.abs(v_ref).max()
    md.close()
    plan.close()


def test_md_conserves_energy_and_sorting_is_transparent(B, oracle_mod):
    N, dt = 500, 1e-3
    q, r, v = _gas(N, 4)
    prm = oracle_mod.select_params(N, *L, 1e-8, n_nb=60)
    finals = {}
    for sort_every in (0, 10):
        plan, qt, rt, vt, F, E, order = _setup(B, prm, q, r, v, N)
        md = B.MD(plan)
        H = []
        for chunk in range(20):
            md.step(qt, rt, vt, F, dt, nsteps=20, E=E, sort_every=sort_every, order=order)
            torch.cuda.synchronize()
            H.append(E.item() + 0.5 * float((vt * vt).sum()))
        assert plan.check() == 0
        ke = 0.5 * float((vt * vt).sum())
        drift = max(abs(h - H[0]) for h in H)
        # the oracle-driven integrator drifts by 6e-6 of this scale on the same run
        assert drift <= 5e-5 * (abs(H[0]) + ke), (sort_every, drift, H[0], ke)
        o = order.cpu().numpy()
        rr = np.empty((N, 3))
        vv = np.empty((N, 3))
        rr[o] = rt.cpu().numpy()
        vv[o] = vt.cpu().numpy()
        qq = np.empty(N)
        qq[o] = qt.cpu().numpy()
        assert np.array_equal(qq, q)
        finals[sort_every] = (rr, vv)
        md.close()
        plan.close()
    dr = finals[10][0] - finals[0][0]
    for d in (0, 1):
        dr[:, d] -= L[d] * np.round(dr[:, d] / L[d])
    assert np.abs(dr).max() <= 1e-8 * max(L)
    assert np.abs(finals[10][1] - finals[0][1]).max() <= 1e-8


def test_md_mixed_precision_runs(B):
    """The FP32 path through the same integrator: 50 steps with re-sorting,
    no data error, finite state, order a permutation."""
    N, dt = 2000, 1e-3
    rng = np.random.default_rng(5)
    from paper_2412_04595_gb300 import workloads
    q, r = workloads.uniform_neutral(N, (30.0, 30.0, 10.0), 5, dtype=np.float32)
    dev = torch.device("cuda:0")
    plan = B.Plan(N, (30.0, 30.0, 10.0), 1e-6, precision=B.SOG_PREC_MIXED)
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    vt = torch.tensor(rng.normal(0, 0.1, (N, 3)).astype(np.float32), device=dev)
    F = torch.empty(N, 3, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, None, E, F)
    order = torch.arange(N, dtype=torch.int32, device=dev)
    md = B.MD(plan)
    md.step(qt, rt, vt, F, 1e-4, nsteps=50, E=E, sort_every=5, order=order)
    torch.cuda.synchronize()
    assert plan.check() == 0
    assert torch.isfinite(rt).all() and torch.isfinite(vt).all()
    assert int(order.sort().values.eq(torch.arange(N, device=dev, dtype=torch.int32)).all()) == 1
    md.close()
    plan.close()
