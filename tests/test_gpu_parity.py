"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Element-by-element comparisons on seeded inputs; FP64 plans must agree with
the oracle to rounding (same parameters, same discrete steps), mixed
precision plans within the tolerance the FP32 arithmetic allows.
"""
import math

import numpy as np
import pytest

from tests.conftest import uniform_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def run_gpu(B, prm, q, r, precision, parts=False):
    N = q.size
    dt = torch.float64 if precision == B.SOG_PREC_FP64 else torch.float32
    dev = torch.device("cuda:0")
    plan = B.Plan(N, prm["L"], 1e-6, precision=precision, manual=prm)
    qt = torch.tensor(q, dtype=dt, device=dev)
    rt = torch.tensor(r, dtype=dt, device=dev)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, phi, E, F)
    out = dict(phi=phi.double().cpu().numpy(), F=F.double().cpu().numpy(), E=E.item())
    if parts:
        pp = torch.empty(4, N, dtype=torch.float64, device=dev)
        pg = torch.empty(4, N, 3, dtype=torch.float64, device=dev)
        plan.eval_components(qt, rt, pp, pg)
        out["pp"] = pp.cpu().numpy()
        out["pg"] = pg.cpu().numpy()
    torch.cuda.synchronize()
    out["status"] = plan.check()
    plan.close()
    return out


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def compare(out, ref, q):
    relE = abs(out["E"] - ref["E"]) / abs(ref["E"])
    rmsF = math.sqrt(np.mean(np.sum((out["F"] - ref["F"]) ** 2, 1)) / np.mean(np.sum(ref["F"] ** 2, 1)))
    linf = rel_max(out["phi"], ref["phi"])
    return relE, rmsF, linf


CASES = {
    "cube10": (1000, (10.0, 10.0, 10.0), 1e-6, 60),
    "box_rect": (700, (9.0, 11.0, 7.0), 1e-6, 40),
    "slab": (600, (24.0, 24.0, 2.0), 1e-6, 40),
    "tol1e-4": (800, (10.0, 10.0, 10.0), 1e-4, 60),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, oracle_mod):
    N, L, tol, nnb = CASES[request.param]
    q, r = uniform_system(N, L, 21)
    prm = oracle_mod.select_params(N, *L, tol, n_nb=nnb)
    ref = oracle_mod.sog_eval(prm, q, r)
    return request.param, q, r, prm, ref


def test_fp64_parts_match_oracle(B, case):
    name, q, r, prm, ref = case
    out = run_gpu(B, prm, q, r, B.SOG_PREC_FP64, parts=True)
    assert out["status"] == 0
    for k, key in enumerate(("near", "mid", "long", "k0")):
        rp, rg = ref["parts"][key]
        if np.max(np.abs(rp)) == 0.0:
            assert np.max(np.abs(out["pp"][k])) == 0.0
            continue
        assert rel_max(out["pp"][k], rp) < 1e-11, (name, key, rel_max(out["pp"][k], rp))
        assert rel_max(out["pg"][k], rg) < 1e-10, (name, key, rel_max(out["pg"][k], rg))
    relE, rmsF, linf = compare(out, ref, q)
    assert relE < 1e-11 and rmsF < 1e-10 and linf < 1e-11, (name, relE, rmsF, linf)


def test_mixed_matches_oracle(B, case):
    name, q, r, prm, ref = case
    q32, r32 = q.astype(np.float32), r.astype(np.float32)
    out = run_gpu(B, prm, q32, r32, B.SOG_PREC_MIXED, parts=True)
    assert out["status"] == 0
    relE, rmsF, linf = compare(out, ref, q)
    # the FP32 inputs move particles by up to 6e-8 relative; the oracle is
    # evaluated on the exact FP64 positions, so part of this is input rounding
    assert relE < 1e-5 and rmsF < 1e-4 and linf < 1e-4, (name, relE, rmsF, linf)


def test_mixed_matches_oracle_on_rounded_inputs(B, oracle_mod):
    """FP32 plan vs the oracle evaluated on the same float32-rounded inputs.
    At N = 1000 the FP32 rounding of ~1e-7 per term leaves the energy within
    2e-6 and the RMS force within 1e-5 (the energy error falls like 1/sqrt(N);
    see the full-size test)."""
    N, L = 1000, (10.0, 10.0, 10.0)
    q, r = uniform_system(N, L, 31)
    q32, r32 = q.astype(np.float32), r.astype(np.float32)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=60)
    ref = oracle_mod.sog_eval(prm, q32.astype(np.float64), r32.astype(np.float64))
    out = run_gpu(B, prm, q32, r32, B.SOG_PREC_MIXED)
    relE, rmsF, linf = compare(out, ref, q)
    assert relE < 2e-6 and rmsF < 1e-5, (relE, rmsF, linf)


def test_full_size_bench_workload(B, oracle_mod):
    """The 1e5 cube workload (N = 1e5 neutral +-1 charges in a 100^3 box,
    tol 1e-6, mixed precision, the launch configuration of
    `bench.py --workload c2`): energy and RMS force against the FP64 oracle
    on the same rounded inputs and parameters, and phi element-wise on 2000
    sampled particles."""
    N, L, tol = 100000, (100.0, 100.0, 100.0), 1e-6
    from paper_2412_04595_gb300 import workloads
    q32, r32 = workloads.uniform_neutral(N, L, 1, dtype=np.float32)
    prm = oracle_mod.select_params(N, *L, tol, n_nb=120)
    out = run_gpu(B, prm, q32, r32, B.SOG_PREC_MIXED)
    assert out["status"] == 0
    ref = oracle_mod.sog_eval(prm, q32.astype(np.float64), r32.astype(np.float64))
    relE, rmsF, linf = compare(out, ref, q32)
    assert relE < 1e-6 and rmsF < 1e-5 and linf < 3e-6, (relE, rmsF, linf)
    idx = np.random.default_rng(0).choice(N, 2000, replace=False)
    scale = np.max(np.abs(ref["phi"]))
    assert np.max(np.abs(out["phi"][idx] - ref["phi"][idx])) < 3e-6 * scale


def test_fp64_vs_ewald2d(B, oracle_mod):
    N, L = 500, (10.0, 10.0, 10.0)
    q, r = uniform_system(N, L, 41)
    pe, ge = oracle_mod.ewald2d(q, r, L)
    Ee = 0.5 * math.fsum(q * pe)
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_FP64, n_nb=60)
    dev = torch.device("cuda:0")
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    phi = torch.empty(N, dtype=torch.float64, device=dev)
    F = torch.empty(N, 3, dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, phi, E, F)
    torch.cuda.synchronize()
    assert abs(E.item() - Ee) / abs(Ee) < 1e-6
    Fe = -q[:, None] * ge
    Fg = F.cpu().numpy()
    assert math.sqrt(np.mean(np.sum((Fg - Fe) ** 2, 1)) / np.mean(np.sum(Fe**2, 1))) < 1e-5
    plan.close()


def test_selection_matches_oracle(B, oracle_mod):
    for (N, L, tol) in [(1000, (10, 10, 10), 1e-6), (100000, (100, 100, 100), 1e-6),
                        (100000, (100, 100, 100), 1e-4), (1000000, (50, 50, 2000), 1e-6),
                        (4000000, (400, 400, 100), 1e-5)]:
        a = B.sog_select_params(N, *map(float, L), tol, n_nb=120)
        b = oracle_mod.select_params(N, *map(float, L), tol, n_nb=120)
        for k in ("M", "m", "I", "P_win", "I_long", "P_long", "P_cheb"):
            assert tuple(np.atleast_1d(a[k])) == tuple(np.atleast_1d(b[k])), (k, a[k], b[k])
        for k in ("b", "r0", "omega", "sigma", "rc", "hz", "shape", "shape_long"):
            assert abs(a[k] - b[k]) <= 1e-13 * max(1.0, abs(b[k])), (k, a[k], b[k])


def test_status_errors(B):
    N, L = 200, (10.0, 10.0, 10.0)
    q, r = uniform_system(N, L, 51)
    dev = torch.device("cuda:0")
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_FP64, n_nb=40)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    # z outside the box
    r2 = r.copy()
    r2[5, 2] = 7.0
    plan.eval(torch.tensor(q, device=dev), torch.tensor(r2, device=dev), None, E, None)
    assert plan.check() == 3
    # non-neutral
    q2 = q.copy()
    q2[0] += 1.0
    plan.eval(torch.tensor(q2, device=dev), torch.tensor(r, device=dev), None, E, None)
    assert plan.check() == 2
    # NaN coordinate: flagged, no fault, finite outputs elsewhere
    r3 = r.copy()
    r3[3, 0] = float("nan")
    plan.eval(torch.tensor(q, device=dev), torch.tensor(r3, device=dev), None, E, None)
    assert plan.check() == 3
    # recovered: a good call is clean again
    plan.eval(torch.tensor(q, device=dev), torch.tensor(r, device=dev), None, E, None)
    assert plan.check() == 0
    # x, y wrapped by one period give the same result
    phi_a = torch.empty(N, dtype=torch.float64, device=dev)
    phi_b = torch.empty(N, dtype=torch.float64, device=dev)
    plan.eval(torch.tensor(q, device=dev), torch.tensor(r, device=dev), phi_a, None, None)
    r4 = r.copy()
    r4[::3, 0] += L[0]
    r4[1::3, 1] -= L[1]
    plan.eval(torch.tensor(q, device=dev), torch.tensor(r4, device=dev), phi_b, None, None)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(phi_a - phi_b)).item() < 1e-12
    plan.close()
    # argument errors
    with pytest.raises(B.SogError):
        B.Plan(1, L, 1e-6)
    with pytest.raises(B.SogError):
        B.Plan(N, (10.0, -1.0, 10.0), 1e-6)


def test_host_entry_point_matches_device(B, oracle_mod):
    N, L = 300, (8.0, 8.0, 8.0)
    q, r = uniform_system(N, L, 61)
    prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=40)
    out = run_gpu(B, prm, q, r, B.SOG_PREC_FP64)
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_FP64, manual=prm)
    phi = np.empty(N)
    F = np.empty((N, 3))
    E = np.empty(1)
    st = plan.eval_host(np.ascontiguousarray(q), np.ascontiguousarray(r), phi, E, F)
    assert st == 0
    assert np.max(np.abs(phi - out["phi"])) < 1e-12
    assert np.max(np.abs(F - out["F"])) < 1e-12
    assert abs(E[0] - out["E"]) < 1e-10
    plan.close()


def test_small_and_ragged(B, oracle_mod):
    """N = 2, and an odd N with one zero charge; tiles and cells mostly empty."""
    for N, L in [(2, (6.0, 6.0, 6.0)), (37, (7.0, 5.0, 4.0))]:
        q, r = uniform_system(N, L, 71)
        prm = oracle_mod.select_params(N, *L, 1e-6, n_nb=2)
        ref = oracle_mod.sog_eval(prm, q, r)
        out = run_gpu(B, prm, q, r, B.SOG_PREC_FP64)
        assert out["status"] == 0
        assert rel_max(out["phi"], ref["phi"]) < 1e-10
        assert rel_max(out["F"], ref["F"]) < 1e-9


def long_variants(oracle_mod, prm, tol):
    """The same parameters with the long range by direct sums (Algorithm 3)
    and by window gridding and FFTs (Algorithm 2), mode counts and grids
    sized for |k| <= K_long as the selection does."""
    w, s = oracle_mod.sog_weights(prm["b"], prm["sigma"], prm["omega"], prm["M"])
    Kl = 2.0 * math.sqrt(math.log(1.0 / (0.3 * tol))) / s[prm["m"] + 1]
    Lx, Ly, _ = prm["L"]
    Kx, Ky = math.ceil(Kl * Lx / (2 * math.pi)), math.ceil(Kl * Ly / (2 * math.pi))
    grid = tuple(oracle_mod._fft_size(max(math.ceil(Kl * Ld / math.pi), prm["P_win"] + 4))
                 for Ld in (Lx, Ly))
    common = dict(L=prm["L"], b=prm["b"], r0=prm["r0"], omega=prm["omega"], rc=prm["rc"],
                  M=prm["M"], m=prm["m"], I=prm["I"], hz=prm["hz"], P_win=prm["P_win"],
                  P_cheb=prm["P_cheb"], window=prm["window"], shape=prm["shape"])
    out = {"grid": oracle_mod.make_params(I_long=grid, P_long=prm["P_win"], long_direct=False,
                                          **common)}
    if Ky + Kx * (2 * Ky + 1) <= 256 and (Ky + Kx * (2 * Ky + 1)) * prm["P_cheb"] <= 8192:
        out["direct"] = oracle_mod.make_params(I_long=(2 * Kx + 1, 2 * Ky + 1),
                                               P_long=prm["P_win"], long_direct=True, **common)
    return out


@pytest.mark.parametrize("name", ["cube10", "box_rect"])
def test_fp64_long_range_both_algorithms(B, oracle_mod, name):
    """Algorithms 2 and 3 on the same system: each matches the oracle's own
    evaluation of that algorithm to rounding, and the two long ranges agree
    with each other to the tolerance."""
    N, L, tol, nnb = CASES[name]
    q, r = uniform_system(N, L, 21)
    prm = oracle_mod.select_params(N, *L, tol, n_nb=nnb)
    assert prm["m"] < prm["M"]
    variants = long_variants(oracle_mod, prm, tol)
    assert "direct" in variants
    longs = {}
    for kind, pv in variants.items():
        ref = oracle_mod.sog_eval(pv, q, r)
        out = run_gpu(B, pv, q, r, B.SOG_PREC_FP64, parts=True)
        assert out["status"] == 0
        rp, rg = ref["parts"]["long"]
        assert rel_max(out["pp"][2], rp) < 1e-11, (name, kind, rel_max(out["pp"][2], rp))
        assert rel_max(out["pg"][2], rg) < 1e-10, (name, kind, rel_max(out["pg"][2], rg))
        longs[kind] = out["pp"][2]
    # both approximate the same long-range potential within the tolerance
    scale = np.max(np.abs(longs["grid"]))
    assert np.max(np.abs(longs["direct"] - longs["grid"])) < 10 * tol * max(scale, 1.0)


@pytest.mark.parametrize("window", ["kb", "gauss"])
def test_other_windows_match_oracle(B, oracle_mod, window):
    """The Kaiser-Bessel and Gaussian windows (Remark 3.4): FP64 parts against
    the oracle to rounding, mixed precision within the FP32 tolerance."""
    N, L, tol, nnb = CASES["cube10"]
    q, r = uniform_system(N, L, 21)
    prm = oracle_mod.select_params(N, *L, tol, n_nb=nnb, window=window)
    assert prm["window"] == window and prm["m"] >= 0
    ref = oracle_mod.sog_eval(prm, q, r)
    out = run_gpu(B, prm, q, r, B.SOG_PREC_FP64, parts=True)
    assert out["status"] == 0
    for k, key in enumerate(("near", "mid", "long", "k0")):
        rp, rg = ref["parts"][key]
        if np.max(np.abs(rp)) == 0.0:
            continue
        assert rel_max(out["pp"][k], rp) < 1e-11, (window, key, rel_max(out["pp"][k], rp))
        assert rel_max(out["pg"][k], rg) < 1e-10, (window, key, rel_max(out["pg"][k], rg))
    q32, r32 = q.astype(np.float32), r.astype(np.float32)
    outm = run_gpu(B, prm, q32, r32, B.SOG_PREC_MIXED)
    assert outm["status"] == 0
    relE, rmsF, linf = compare(outm, ref, q)
    assert relE < 1e-5 and rmsF < 1e-4 and linf < 1e-4, (window, relE, rmsF, linf)


def test_forces_are_the_gradient_of_the_energy(B, oracle_mod):
    """The forces are the exact gradient of the energy the plan computes
    (spread and gather share the window, the near table is C1 at r_c): central
    differences of the FP64 energy in a few coordinates match -F."""
    N, L, tol, nnb = CASES["cube10"]
    q, r = uniform_system(N, L, 21)
    prm = oracle_mod.select_params(N, *L, tol, n_nb=nnb)
    base = run_gpu(B, prm, q, r, B.SOG_PREC_FP64)
    assert base["status"] == 0
    Fmax = np.max(np.abs(base["F"]))
    h = 1e-5
    rng = np.random.default_rng(3)
    for i in rng.choice(N, 4, replace=False):
        for d in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, d] += h
            rm[i, d] -= h
            Ep = run_gpu(B, prm, q, rp, B.SOG_PREC_FP64)["E"]
            Em = run_gpu(B, prm, q, rm, B.SOG_PREC_FP64)["E"]
            fd = -(Ep - Em) / (2 * h)
            assert abs(fd - base["F"][i, d]) < 1e-6 * Fmax, (i, d, fd, base["F"][i, d])


@pytest.mark.parametrize("name", ["cube10", "slab"])
@pytest.mark.parametrize("window", ["es", "kb"])
def test_polynomial_windows_match_oracle(B, oracle_mod, name, window):
    """Polynomial windows (win_poly = nu, Sec. 3.4, 5.1) on the mid grid, the
    small one-tile long-range grid (cube10, Algorithm 2 variant) and the tiled
    long-range grid (slab): FP64 parts against the oracle's evaluation of the
    same polynomials to rounding; mixed precision within the FP32 tolerance;
    and the energy within 1e-7 of the exact windows'."""
    N, L, tol, nnb = CASES[name]
    q, r = uniform_system(N, L, 21)
    prm = oracle_mod.select_params(N, *L, tol, n_nb=nnb, window=window)
    if name == "cube10":
        prm = long_variants(oracle_mod, prm, tol)["grid"]
    prm = dict(prm, win_poly=10)
    ref = oracle_mod.sog_eval(prm, q, r)
    out = run_gpu(B, prm, q, r, B.SOG_PREC_FP64, parts=True)
    assert out["status"] == 0
    for k, key in enumerate(("mid", "long")):
        rp, rg = ref["parts"][key]
        if np.max(np.abs(rp)) == 0.0:
            continue
        assert rel_max(out["pp"][k + 1], rp) < 1e-11, (window, key, rel_max(out["pp"][k + 1], rp))
        assert rel_max(out["pg"][k + 1], rg) < 1e-10, (window, key, rel_max(out["pg"][k + 1], rg))
    assert abs(out["E"] - ref["E"]) <= 1e-11 * abs(ref["E"])
    exact = oracle_mod.sog_eval(dict(prm, win_poly=0), q, r)
    assert abs(ref["E"] - exact["E"]) <= 1e-7 * abs(exact["E"])
    q32, r32 = q.astype(np.float32), r.astype(np.float32)
    outm = run_gpu(B, prm, q32, r32, B.SOG_PREC_MIXED)
    assert outm["status"] == 0
    relE, rmsF, linf = compare(outm, ref, q)
    assert relE < 1e-5 and rmsF < 1e-4 and linf < 1e-4, (window, relE, rmsF, linf)
