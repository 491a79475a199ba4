"""Ridge regression fitted on the device from the batch's aggregates (lmfao_ridge_fit) against
the oracle's fit from its own aggregates: closed form and batch gradient descent, FP64 and
FP32 passes; a query without the needed aggregates is refused."""
import numpy as np
import pytest

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.lmfao import ERR_ARG, Engine, LmfaoError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["star", "retailer"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ridge_fit_matches_the_oracle(which, precision):
    if which == "star":
        rels, qs, feats = W.star_schema(n_fact=200_000), W.star_batch(), ["f1", "f2", "x1", "x2", "x3", "z1", "z2"]
    else:
        rels, qs = W.retailer_schema(n_fact=300_000, seed=9), W.retailer_batch()
        feats = [a for a in W.RETAILER_CONTS if a != "y"]
    ref = O.evaluate(rels, qs[:1])[0]
    A, b, syy = O.ridge_system(ref, qs[0], "y", feats)
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        e.add_queries(qs)
        e.plan(precision=precision)
        e.run()
        lam = 0.1
        th, J, gn = e.ridge_fit(0, "y", feats, lam)
        want = O.ridge_closed_form(A, b, lam)
        tol = 1e-9 if precision == "fp64" else 1e-4
        np.testing.assert_allclose(th, want, rtol=tol, atol=tol * np.abs(want).max())
        assert abs(J - O.ridge_objective(A, b, syy, lam, want)) <= tol * abs(J) and gn <= 1e-6 * (1 + abs(J))
        step = 1.0 / np.linalg.eigvalsh(A + lam * np.eye(len(b))).max()
        thb, Jb, _ = e.ridge_fit(0, "y", feats, lam, method="bgd", iters=200, step=step)
        np.testing.assert_allclose(thb, O.ridge_bgd(A, b, lam, 200, step), rtol=tol, atol=tol * np.abs(want).max())
        with pytest.raises(LmfaoError) as ei:
            e.ridge_fit(1, "y", feats, lam)  # a grouped query
        assert ei.value.code == ERR_ARG
        with pytest.raises(LmfaoError) as ei:
            e.ridge_fit(0, "y", feats + ["no_such"], lam)
        assert ei.value.code == ERR_ARG and "no SUM" in str(ei.value)
    finally:
        e.close()
