"""Edge cases of the method against the oracle, element by element.

One neutral system in a 50 x 50 x 8 box (parameters with both a mid grid
and the gridded long range of Algorithm 2) holds, besides uniform charges:

* charges exactly on the walls z = -Lz/2 and z = +Lz/2 (inside the box);
* charges at x = +Lx/2 and y = +Ly/2, which wrap to -Lx/2, -Ly/2 (Sec. 2.1);
* charges on every mid-grid and long-grid line in x, y and z, hence on every
  tile boundary of the spreading and gathering, and on the near-field cell
  boundaries (cells of edge L / floor(L / r_c), Sec. 2.2);
* opposite-charge pairs at distance 1e-3 r_c (the near-field table near
  r = 0, Eq. 2.28) and at r_c (1 - 1e-6), r_c (1 + 1e-6) (the cutoff where
  the near field hands the pair to the far field);
* a dense layer of charges within 0.02 of each wall (the double-layer case).

FP64 plans must match the oracle to 1e-10 and mixed plans (inputs rounded to
FP32 once for both sides) to 1e-5: potentials relative to the largest
potential of the group, forces as an RMS over the group.  The close pairs are
their own group, since their potentials and forces are orders of magnitude
larger than the others'."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L = (50.0, 50.0, 8.0)
TOL = 1e-6
N_NB = 60


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_2412_04595_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def _edge_system(prm):
    """Positions (n x 3, float64), charges and the indices of the close-pair
    particles.  Charges alternate in sign within every group of even size."""
    rng = np.random.default_rng(2024)
    Lx, Ly, Lz = L
    pts = []

    def add(p):
        pts.append(np.asarray(p, dtype=np.float64))

    def rnd(n):
        return np.column_stack([rng.uniform(-Lx / 2, Lx / 2, n), rng.uniform(-Ly / 2, Ly / 2, n),
                                rng.uniform(-Lz / 2, Lz / 2, n)])

    # uniform background
    for p in rnd(2400):
        add(p)
    # walls and wrapping edges
    for z in (-Lz / 2, Lz / 2):
        for p in rnd(10):
            add((p[0], p[1], z))
    for p in rnd(6):
        add((Lx / 2, p[1], p[2]))
        add((p[0], Ly / 2, p[2]))
    add((Lx / 2, Ly / 2, Lz / 2))
    add((Lx / 2, Ly / 2, -Lz / 2))
    # grid lines (tile boundaries) of the mid grid, the long grid, and the
    # near-field cell boundaries
    Ix, Iy, Iz = prm["I"]
    hz = prm["hz"]
    lines_x = [-Lx / 2 + j * Lx / Ix for j in range(Ix)]
    lines_y = [-Ly / 2 + j * Ly / Iy for j in range(Iy)]
    Ilx, Ily = prm["I_long"]
    lines_x += [-Lx / 2 + j * Lx / Ilx for j in range(Ilx)]
    lines_y += [-Ly / 2 + j * Ly / Ily for j in range(Ily)]
    rc = prm["rc"]
    ncx, ncy = int(Lx // rc), int(Ly // rc)
    lines_x += [-Lx / 2 + k * Lx / ncx for k in range(ncx)]
    lines_y += [-Ly / 2 + k * Ly / ncy for k in range(ncy)]
    Lzs = Iz * hz
    lines_z = [-Lzs / 2 + g * hz for g in range(Iz) if abs(-Lzs / 2 + g * hz) <= Lz / 2]
    for x in lines_x:
        p = rnd(1)[0]
        add((x, p[1], p[2]))
    for y in lines_y:
        p = rnd(1)[0]
        add((p[0], y, p[2]))
    for z in lines_z:
        p = rnd(1)[0]
        add((p[0], p[1], z))
    # a corner on all three sets of lines at once
    add((lines_x[8], lines_y[8], lines_z[len(lines_z) // 2]))
    # dense layers at the walls
    for p in rnd(200):
        add((p[0], p[1], -Lz / 2 + 0.02 * rng.random()))
        add((p[0] + 0.37, p[1] - 0.21, Lz / 2 - 0.02 * rng.random()))
    n_plain = len(pts)
    # close pairs: distance 1e-3 rc, rc (1 - 1e-6), rc (1 + 1e-6)
    close = []
    for d in (1e-3 * rc, 1e-3 * rc, rc * (1 - 1e-6), rc * (1 + 1e-6)):
        for _ in range(4):
            c = rnd(1)[0]
            c[2] *= 0.5
            if d < 1e-2 * rc:
                u = rng.normal(size=3)
                u /= np.linalg.norm(u)
            else:        # in the xy plane, so that the partner stays inside in z
                t = rng.uniform(0.0, 2.0 * math.pi)
                u = np.array([math.cos(t), math.sin(t), 0.0])
            close.append(len(pts))
            add(c)
            close.append(len(pts))
            add(c + d * u)
    r = np.array(pts)
    if n_plain % 2:          # keep the plain part of even size
        r = np.insert(r, n_plain, rnd(1)[0], axis=0)
        close = [i + 1 for i in close]
    q = np.where(np.arange(r.shape[0]) % 2 == 0, 1.0, -1.0)
    return q, r, np.array(close[::1], dtype=np.int64)


def _errors(phi, F, ref_phi, ref_F, idx):
    e_phi = np.max(np.abs(phi[idx] - ref_phi[idx])) / np.max(np.abs(ref_phi[idx]))
    e_F = math.sqrt(np.sum((F[idx] - ref_F[idx]) ** 2) / np.sum(ref_F[idx] ** 2))
    return e_phi, e_F


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases_match_oracle(B, oracle_mod, precision):
    prm = oracle_mod.select_params(4000, *L, TOL, n_nb=N_NB)
    assert prm["m"] >= 0 and prm["m"] < prm["M"] and not prm["long_direct"]
    q, r, close = _edge_system(prm)
    N = q.size
    assert abs(q.sum()) == 0.0
    fp64 = precision == "fp64"
    if not fp64:
        r = r.astype(np.float32).astype(np.float64)
    # the points on +Lx/2 and +Ly/2 are passed as they are: the library wraps them
    assert np.any(r[:, 0] == L[0] / 2) and np.any(r[:, 1] == L[1] / 2)
    assert np.any(r[:, 2] == L[2] / 2) and np.any(r[:, 2] == -L[2] / 2)
    ref = oracle_mod.sog_eval(prm, q, r)
    dt = torch.float64 if fp64 else torch.float32
    prec = B.SOG_PREC_FP64 if fp64 else B.SOG_PREC_MIXED
    dev = torch.device("cuda:0")
    plan = B.Plan(N, L, TOL, precision=prec, manual=prm)
    qt = torch.tensor(q, dtype=dt, device=dev)
    rt = torch.tensor(r, dtype=dt, device=dev)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    plan.eval(qt, rt, phi, E, F)
    torch.cuda.synchronize()
    assert plan.check() == 0
    plan.close()
    phi = phi.double().cpu().numpy()
    F = F.double().cpu().numpy()
    bound = 1e-10 if fp64 else 1e-5
    rest = np.setdiff1d(np.arange(N), close)
    for name, idx in (("plain", rest), ("close pairs", close)):
        e_phi, _ = _errors(phi, F, ref["phi"], ref["F"], idx)
        assert e_phi <= bound, (name, e_phi)
    # Forces.  The ES window's derivative is unbounded at the edge of its
    # support (it goes as 1/sqrt(1 - |v|), with the small factor beta
    # e^-beta), and a charge exactly on a grid line puts a window point
    # exactly on that edge: its force then depends on the last bit of the
    # grid coordinate.  FP64 plans compute that coordinate as the oracle
    # does, bit for bit, so every charge is compared.  Mixed plans compute it
    # in float pairs: the charges whose FP32 position lies on a grid line
    # (to 1e-9 grid spacings) are compared in potential only.
    on_line = np.zeros(N, dtype=bool)
    if not fp64:
        Lzs = prm["I"][2] * prm["hz"]
        axes = [(0, L[0] / prm["I"][0], L[0] / 2), (1, L[1] / prm["I"][1], L[1] / 2),
                (2, prm["hz"], Lzs / 2), (0, L[0] / prm["I_long"][0], L[0] / 2),
                (1, L[1] / prm["I_long"][1], L[1] / 2)]
        for d, h, off in axes:
            t = (r[:, d] + off) / h
            on_line |= np.abs(t - np.round(t)) < 1e-9
        assert 0 < on_line.sum() < 200
    for name, idx in (("plain", np.setdiff1d(rest, np.nonzero(on_line)[0])), ("close pairs", close)):
        _, e_F = _errors(phi, F, ref["phi"], ref["F"], idx)
        assert e_F <= bound, (name, e_F)
    assert abs(E.item() - ref["E"]) <= bound * abs(ref["E"])
