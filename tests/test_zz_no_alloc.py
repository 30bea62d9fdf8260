"""sog_assemble_noalloc: the plan-free, allocation-free assembly of Phi, U and
F from the four parts of the potential, through the C ABI.

Its results must match those of sog_eval on the same charges (the parts come
from sog_eval_components of the same plan), on two calls in a row, and the
second call must repeat the first exactly (the energy partials live in a
fixed device array that every call overwrites)."""
import ctypes

import numpy as np
import pytest

from paper_2412_04595_gb300 import workloads

torch = pytest.importorskip("torch")

SOG_OK, SOG_ERR_ARG = 0, 1  # sog_status values of include/sog.h


def _lib():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    return binding


def test_argument_errors_without_device_work():
    B = _lib()
    L = B.load()
    prm = B.SogParams.from_dict(B.sog_select_params(1000, 10.0, 10.0, 10.0, 1e-6))
    dummy = ctypes.c_void_p(16)
    for N, prec, params, q, pp in ((0, 1, ctypes.byref(prm), dummy, dummy),
                                   (715827883, 1, ctypes.byref(prm), dummy, dummy),
                                   (10, 7, ctypes.byref(prm), dummy, dummy),
                                   (10, 1, None, dummy, dummy),
                                   (10, 1, ctypes.byref(prm), None, dummy),
                                   (10, 1, ctypes.byref(prm), dummy, None)):
        assert L.sog_assemble_noalloc(N, prec, params, q, pp, None, None, None, None, None) == \
            SOG_ERR_ARG
    # forces asked for without their gradient parts
    assert L.sog_assemble_noalloc(10, 1, ctypes.byref(prm), dummy, dummy, None, None, None,
                                  dummy, None) == SOG_ERR_ARG
    # parameters a plan would reject: omega <= 0 or not finite, sigma <= 0, b <= 1
    for field, value in (("omega", 0.0), ("omega", -1.0), ("omega", float("nan")),
                         ("sigma", 0.0), ("b", 1.0), ("b", float("inf"))):
        bad = B.SogParams.from_dict(B.sog_select_params(1000, 10.0, 10.0, 10.0, 1e-6))
        setattr(bad, field, value)
        assert L.sog_assemble_noalloc(10, 1, ctypes.byref(bad), dummy, dummy, None, None, None,
                                      None, None) == SOG_ERR_ARG, (field, value)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,N", [("fp64", 20000), ("mixed", 20000), ("mixed", 100000)])
def test_matches_sog_eval_on_two_calls_in_a_row(precision, N):
    """N = 1e5 needs more blocks than the assembly launches (two per SM), so
    the grid-stride loop and the full set of energy partials are used."""
    B = _lib()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fp64 = precision == "fp64"
    dt = torch.float64 if fp64 else torch.float32
    prec = B.SOG_PREC_FP64 if fp64 else B.SOG_PREC_MIXED
    L = (30.0 * (N / 20000) ** (1.0 / 3.0),) * 3
    q, r = workloads.uniform_neutral(N, L, seed=11, dtype=np.float64)
    dev = torch.device("cuda:0")
    qt = torch.tensor(q, dtype=dt, device=dev)
    rt = torch.tensor(r, dtype=dt, device=dev)
    plan = B.Plan(N, L, 1e-6, precision=prec)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, phi, E, F)
    pp = torch.empty(4, N, dtype=torch.float64, device=dev)
    pg = torch.empty(4, N, 3, dtype=torch.float64, device=dev)
    plan.eval_components(qt, rt, pp, pg)
    torch.cuda.synchronize()
    assert plan.check() == SOG_OK
    outs = []
    for _ in range(2):
        phi_a = torch.full((N,), float("nan"), dtype=dt, device=dev)
        F_a = torch.full((N, 3), float("nan"), dtype=dt, device=dev)
        E_a = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        B.sog_assemble_noalloc(plan.params, qt, pp, pg, phi_a, E_a, F_a)
        outs.append((phi_a, E_a, F_a))
    torch.cuda.synchronize()
    plan.close()
    # the parts of the second evaluation differ from those inside sog_eval
    # only by the order of floating-point atomics in the grid spreading
    tol_phi, tol_E = (1e-12, 1e-12) if fp64 else (2e-6, 2e-6)
    ref_phi = phi.double()
    ref_F = F.double()
    scale_phi = ref_phi.abs().max().item()
    scale_F = ref_F.abs().max().item()
    for phi_a, E_a, F_a in outs:
        assert torch.isfinite(phi_a).all() and torch.isfinite(F_a).all()
        assert (phi_a.double() - ref_phi).abs().max().item() <= tol_phi * scale_phi
        assert (F_a.double() - ref_F).abs().max().item() <= 10 * tol_phi * scale_F
        assert abs(E_a.item() - E.item()) <= tol_E * abs(E.item())
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][2], outs[1][2])
    assert outs[0][1].item() == outs[1][1].item()


@pytest.mark.gpu
def test_energy_only_call():
    """phi and F left out (NULL): only the energy is written, and it equals
    the energy of sog_eval."""
    B = _lib()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N, L = 30000, (40.0, 40.0, 40.0)
    q, r = workloads.uniform_neutral(N, L, seed=12, dtype=np.float64)
    dev = torch.device("cuda:0")
    qt = torch.tensor(q, dtype=torch.float64, device=dev)
    rt = torch.tensor(r, dtype=torch.float64, device=dev)
    plan = B.Plan(N, L, 1e-6, precision=B.SOG_PREC_FP64)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, None, E, None)
    pp = torch.empty(4, N, dtype=torch.float64, device=dev)
    plan.eval_components(qt, rt, pp, None)
    torch.cuda.synchronize()
    assert plan.check() == SOG_OK
    for _ in range(2):
        E_a = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        B.sog_assemble_noalloc(plan.params, qt, pp, None, None, E_a, None)
        torch.cuda.synchronize()
        assert abs(E_a.item() - E.item()) <= 1e-12 * abs(E.item())
    plan.close()
