"""Argument checks of the Python binding (CPU only): a tensor of the wrong
dtype or element count must raise ValueError before its pointer reaches the
C ABI, where it would be read or written out of bounds."""
import pytest

torch = pytest.importorskip("torch")

from paper_2412_04595_gb300 import binding as B  # noqa: E402


def _plan(N, precision):
    # a Plan object without a device plan: only the checks before the C call run
    p = B.Plan.__new__(B.Plan)
    p.N = N
    p.precision = precision
    p._h = None
    p._lib = None
    return p


@pytest.mark.parametrize("precision", [B.SOG_PREC_FP64, B.SOG_PREC_MIXED])
def test_eval_rejects_wrong_sizes_and_dtypes(precision):
    N = 10
    p = _plan(N, precision)
    dt = p.dtype
    q, r = torch.zeros(N, dtype=dt), torch.zeros(N, 3, dtype=dt)
    phi, F = torch.zeros(N, dtype=dt), torch.zeros(N, 3, dtype=dt)
    E = torch.zeros(1, dtype=torch.float64)
    bad = [
        dict(q=torch.zeros(N - 1, dtype=dt)),
        dict(r=torch.zeros(N, 2, dtype=dt)),
        dict(phi=torch.zeros(N + 1, dtype=dt)),
        dict(F=torch.zeros(N, dtype=dt)),
        dict(E=torch.zeros(0, dtype=torch.float64)),
        dict(E=torch.zeros(1, dtype=torch.float32)),
        dict(q=torch.zeros(N, dtype=torch.float16)),
        dict(F=torch.zeros(3 * N, dtype=dt)[::1].reshape(N, 3).t()),  # not contiguous
    ]
    for kw in bad:
        args = dict(q=q, r=r, phi=phi, E=E, F=F)
        args.update(kw)
        with pytest.raises(ValueError) as ei:
            p.eval(**args)
        assert "CUDA" not in str(ei.value), (kw, str(ei.value))
    # right sizes on the host: rejected only for not being on the device
    with pytest.raises(ValueError, match="CUDA"):
        p.eval(q, r, phi, E, F)


@pytest.mark.parametrize("precision", [B.SOG_PREC_FP64, B.SOG_PREC_MIXED])
def test_eval_components_checks_parts(precision):
    N = 7
    p = _plan(N, precision)
    dt = p.dtype
    q, r = torch.zeros(N, dtype=dt), torch.zeros(N, 3, dtype=dt)
    for pp, pg in ((torch.zeros(4, N, dtype=torch.float32), None),   # parts must be float64
                   (torch.zeros(3, N, dtype=torch.float64), None),
                   (None, torch.zeros(4, N, dtype=torch.float64)),
                   (None, torch.zeros(4, N, 3, dtype=torch.float32))):
        with pytest.raises(ValueError) as ei:
            p.eval_components(q, r, pp, pg)
        assert "CUDA" not in str(ei.value)


def test_eval_host_checks_sizes():
    N = 5
    p = _plan(N, B.SOG_PREC_FP64)
    import numpy as np
    q, r = np.zeros(N), np.zeros((N, 3))
    with pytest.raises(ValueError):
        p.eval_host(q, r, phi=np.zeros(N - 1))
    with pytest.raises(ValueError):
        p.eval_host(q, r, F=np.zeros((N, 3), dtype=np.float32))
    with pytest.raises(ValueError):
        p.eval_host(q, np.zeros((N + 1, 3)))


def test_assemble_noalloc_checks_sizes():
    N = 6
    q = torch.zeros(N, dtype=torch.float32)
    pp, pg = torch.zeros(4, N, dtype=torch.float64), torch.zeros(4, N, 3, dtype=torch.float64)
    prm = {"L": (1.0, 1.0, 1.0), "b": 1.3, "r0": 4.0, "omega": 1.0, "sigma": 0.5, "rc": 2.0,
           "M": 10, "m": -1, "I": (0, 0, 0), "hz": 0.0, "P_win": 4, "shape": 1.0,
           "I_long": (8, 8), "P_long": 4, "shape_long": 1.0, "P_cheb": 4}
    bad = [
        dict(phi_parts=torch.zeros(4, N, dtype=torch.float32)),   # FP32 parts from a mixed plan
        dict(phi_parts=torch.zeros(3, N, dtype=torch.float64)),
        dict(grad_parts=torch.zeros(4, N, dtype=torch.float64)),
        dict(phi=torch.zeros(N + 1, dtype=torch.float32)),
        dict(F=torch.zeros(N, 2, dtype=torch.float32)),
        dict(F=torch.zeros(N, 3, dtype=torch.float64)),
        dict(E=torch.zeros(0, dtype=torch.float64)),
        dict(grad_parts=None, F=torch.zeros(N, 3, dtype=torch.float32)),
    ]
    for kw in bad:
        args = dict(phi_parts=pp, grad_parts=pg, phi=None, E=None, F=None)
        args.update(kw)
        with pytest.raises(ValueError) as ei:
            B.sog_assemble_noalloc(prm, q, **args)
        assert "CUDA" not in str(ei.value), (kw, str(ei.value))
    with pytest.raises(ValueError, match="CUDA"):
        B.sog_assemble_noalloc(prm, q, pp, pg)
