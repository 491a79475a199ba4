"""The allocation-free CART entry point (lmfao_cart_variances_noalloc) returns what the
allocating one (lmfao_cart_variances) returns, on two calls in a row (the second on a
stream of its own), and the device's free memory does not change during those calls.

Callers that cannot allocate device memory when they evaluate splits (a fixed device
budget owned by their framework's caching allocator, or a loop that must avoid the
synchronisation of cudaMalloc / cudaFree) use the no-allocation variant; its descriptors
live in a fixed device array shared by all calls. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.lmfao import ERR_ARG, Engine, LmfaoError
from tests.parity import ATOL, RTOL

pytestmark = pytest.mark.gpu


def test_noalloc_cart_variances_match_allocating_entry_point():
    import torch
    rels = W.retailer_schema(n_fact=100_000, seed=1)
    qs, _splits, thr = W.dt_level_batch(rels, seed=1)
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs)
    e.plan(precision="fp32")
    e.run()
    nb = max(len(t) for t in thr.values()) + 1
    ids = [i for i, q in enumerate(qs) if len(q["groupby"][0][2]) + 1 == nb]
    assert len(ids) > 100
    ref = torch.zeros((len(ids), nb - 1, 2), dtype=torch.float64, device="cuda")
    e.cart_variances(ids, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    outs = [torch.full((len(ids), nb - 1, 2), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    side = torch.cuda.Stream()
    e.cart_variances_noalloc(ids, outs[2])  # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call, order in enumerate((ids, ids[::-1])):
        out = outs[call]
        if call == 1:  # the second call on a stream of its own
            side.wait_stream(torch.cuda.current_stream())
            e.cart_variances_noalloc(order, out, stream=side)
            side.synchronize()
        else:
            e.cart_variances_noalloc(order, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "device memory changed during the call"
        got = out.cpu().numpy()
        want = ref if call == 0 else ref[::-1]
        np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL, err_msg=f"call {call}")
    with pytest.raises(LmfaoError) as ei:
        e.cart_variances_noalloc(list(range(4097)), torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert ei.value.code == ERR_ARG and "at most 4096" in str(ei.value)
    e.close()
