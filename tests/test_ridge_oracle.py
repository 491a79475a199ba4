"""The oracle's ridge regression from aggregates (Section 3, linear regression) pinned without
the oracle's own join: on a star join whose dimension keys are unique and always present,
every fact row is one joined tuple, so the design matrix is formed by direct indexing and the
minimiser of J(theta) = 1/(2|D|) |X theta - y|^2 + lambda/2 |theta|^2 comes from
numpy.linalg.lstsq on the augmented system [X; sqrt(|D| lambda) I] theta = [y; 0]."""
import numpy as np

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from tests.test_cart_tree_oracle import joined_columns

FEATS = ["f1", "f2", "x1", "x2", "x3", "z1", "z2"]


def setup():
    rels = W.star_schema(n_fact=3000, seed=11)
    q = W.ridge_batch(["y"] + FEATS, [])[0]
    res = O.evaluate(rels, [q])[0]
    cols = joined_columns(rels)
    X = np.column_stack([np.ones(3000)] + [cols[f].astype(np.float64) for f in FEATS])
    y = cols["y"].astype(np.float64)
    return res, q, X, y


def test_closed_form_equals_lstsq_on_the_joined_rows():
    res, q, X, y = setup()
    A, b, syy = O.ridge_system(res, q, "y", FEATS)
    n = len(y)
    for lam in (0.0, 0.3):
        th = O.ridge_closed_form(A, b, lam)
        Xa = np.vstack([X, np.sqrt(n * lam) * np.eye(X.shape[1])])
        ya = np.concatenate([y, np.zeros(X.shape[1])])
        ref, *_ = np.linalg.lstsq(Xa, ya, rcond=None)
        np.testing.assert_allclose(th, ref, rtol=1e-8, atol=1e-10)


def test_objective_and_gradient_descent():
    res, q, X, y = setup()
    A, b, syy = O.ridge_system(res, q, "y", FEATS)
    n, lam = len(y), 0.2
    th = np.random.default_rng(0).standard_normal(X.shape[1])
    direct = 0.5 / n * np.sum((X @ th - y) ** 2) + 0.5 * lam * th @ th
    assert abs(O.ridge_objective(A, b, syy, lam, th) - direct) <= 1e-10 * abs(direct)
    # the first step from zero is step * b; with a step below 2 / lambda_max the iteration
    # contracts to the closed form
    step = 0.5
    np.testing.assert_allclose(O.ridge_bgd(A, b, lam, 1, step), step * b, rtol=1e-12)
    lmax = np.linalg.eigvalsh(A + lam * np.eye(len(b))).max()
    assert step < 2 / lmax
    np.testing.assert_allclose(O.ridge_bgd(A, b, lam, 3000, step), O.ridge_closed_form(A, b, lam), rtol=1e-7,
                               atol=1e-9)
