"""Host logic of the learned parameter proposer, without a GPU: the cost-model
inputs of a candidate neighbour count and the decision rule (the analytic
default unless the model covers the inputs and predicts a real saving)."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def P():
    from paper_2412_04595_gb300 import _build
    _build.build()
    from paper_2412_04595_gb300 import proposer
    return proposer


def test_candidate_features_follow_the_analytic_parameters(P):
    from paper_2412_04595_gb300 import binding as B
    N, L, tol = 100000, (100.0, 100.0, 100.0), 1e-6
    feat = [0.0] * B.N_FEATURES
    z = P.cand_features(feat, N, L, tol, 120.0)
    prm = B.sog_select_params(N, *L, tol, n_nb=120.0)
    assert len(z) == P.N_INPUTS
    rho = N / (L[0] * L[1] * L[2])
    pairs = N * 4.0 / 3.0 * math.pi * prm["rc"] ** 3 * rho
    assert abs(z[B.N_FEATURES] - math.log10(pairs)) < 1e-12
    assert abs(z[B.N_FEATURES + 1] - math.log10(np.prod(prm["I"]))) < 1e-12
    # more neighbours: more pairs, a coarser mid grid
    z2 = P.cand_features(feat, N, L, tol, 220.0)
    assert z2[B.N_FEATURES] > z[B.N_FEATURES] and z2[B.N_FEATURES + 1] <= z[B.N_FEATURES + 1]


def _stub(P, pred, lo=-1e9, hi=1e9, margin=0.03):
    """A proposer whose cost model returns pred[c] for candidate c."""
    prop = object.__new__(P.Proposer)
    prop.trained = True
    prop.margin = margin
    prop.candidates = tuple(sorted(pred))
    prop.z_lo = np.full(P.N_INPUTS, lo)
    prop.z_hi = np.full(P.N_INPUTS, hi)
    order = list(prop.candidates)

    def predict(Z):
        # rows arrive in candidate order (feasible, covered candidates only)
        return np.array([math.log(pred[c]) for c in order[:len(Z)]])
    prop.predict = predict
    return prop


def test_proposal_needs_a_real_predicted_saving(P):
    N, L, tol = 100000, (100.0, 100.0, 100.0), 1e-6
    feat = [0.0] * 8
    # 1 % cheaper than the default: below the margin, the default stays
    prop = _stub(P, {100.0: 0.99, 120.0: 1.0, 160.0: 1.2})
    assert prop.propose(feat, N, L, tol) == (P.DEFAULT_NNB, "analytic")
    # 10 % cheaper: proposed
    prop = _stub(P, {100.0: 0.9, 120.0: 1.0, 160.0: 1.2})
    assert prop.propose(feat, N, L, tol) == (100.0, "mlp")


def test_untrained_or_uncovered_model_keeps_the_default(P):
    N, L, tol = 100000, (100.0, 100.0, 100.0), 1e-6
    feat = [0.0] * 8
    prop = _stub(P, {100.0: 0.5, 120.0: 1.0})
    prop.trained = False
    assert prop.propose(feat, N, L, tol) == (P.DEFAULT_NNB, "analytic")
    # inputs outside the training range (widened by a quarter span): default
    prop = _stub(P, {100.0: 0.5, 120.0: 1.0}, lo=1e3, hi=1e3 + 1.0)
    assert prop.propose(feat, N, L, tol) == (P.DEFAULT_NNB, "analytic")
