"""Comparison of engine results with the oracle (shared by the GPU tests and smoke())."""
import numpy as np

# FP aggregates: |engine - oracle| <= RTOL * sum of |terms| (+ ATOL for all-zero terms).
RTOL = 1e-5
ATOL = 1e-9


def integral_aggs(q):
    return [len(a) == 0 for a in q["aggs"]]


def compare(q, got, ref, rtol=RTOL, where=""):
    """Group keys and COUNTs bit-exact; integral aggregates exact; FP within tolerance."""
    np.testing.assert_array_equal(got["keys"], ref["keys"], err_msg=f"group keys differ {where}")
    np.testing.assert_array_equal(got["counts"], ref["counts"], err_msg=f"counts differ {where}")
    integ = integral_aggs(q)
    for j, exact in enumerate(integ):
        g, r, a = got["sums"][:, j], ref["sums"][:, j], ref["abs"][:, j]
        if exact:
            np.testing.assert_array_equal(g, r, err_msg=f"integral aggregate {j} differs {where}")
        else:
            err = np.abs(g - r)
            bad = err > rtol * a + ATOL
            if bad.any():
                i = int(np.argmax(err - rtol * a))
                raise AssertionError(f"aggregate {j} group {i} {where}: engine {g[i]!r} oracle {r[i]!r} "
                                     f"|terms| {a[i]!r} rel.err {err[i] / max(a[i], 1e-300):.3e}")


def max_rel_error(qs, gots, refs):
    worst = 0.0
    for q, g, r in zip(qs, gots, refs):
        if len(g["keys"]) != len(r["keys"]):
            return float("inf")
        for j, exact in enumerate(integral_aggs(q)):
            if exact:
                continue
            a = r["abs"][:, j]
            e = np.abs(g["sums"][:, j] - r["sums"][:, j])
            nz = a > 0
            if nz.any():
                worst = max(worst, float((e[nz] / a[nz]).max()))
    return worst
