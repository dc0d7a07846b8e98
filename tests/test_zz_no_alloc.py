"""The allocation-free estimator entry point against the pooled one.

pb_recip_estimates_noalloc serves callers that cannot allocate device memory
while they run (engines that reserve all device memory up front, processes
whose allocations another runtime caps or pools, latency-critical code that
cannot take cudaMalloc's implicit synchronisation). Given the entries of an
iteration's pool in (light path, vertex) order it must return the same
reciprocal estimates as pb_iteration, twice in a row on the same (shared,
reused) scratch. This file sorts last so that a run stopping at the first
failure has run every other test before it.
"""

import numpy as np
import pytest

import oracle as O
from paper_2503_23412_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_noalloc_estimates_match_pooled_estimator():
    torch = pytest.importorskip("torch")
    from paper_2503_23412_gb300 import build
    build.build()
    from paper_2503_23412_gb300 import native as N

    sc = scenes.cornell(16, 16)
    o = O.Oracle(sc)
    p = O.params(M=1500, M_p=600, max_depth=6)
    tri, bary = o.light_pass(p, 11)
    ents, _ = o.entries(p, tri, bary)
    n = len(ents)
    assert n > 20
    # one B for every cell keeps both paths on the same bound: 1.5 x the
    # largest f/q of 64 draws over all entries
    mx = 0.0
    for k, e in enumerate(ents):
        f, q = o.entry_fq(e, 64, a=3, b=k)
        r = np.where(q > 0, f / np.where(q > 0, q, 1.0), 0.0)
        mx = max(mx, float(r.max()))
    tab = scenes.random_tables(sc, KT=8, KS=8, KSp=4, KC=2, B=1.5 * mx, mis=1.0)
    r = N.Renderer(sc, tab)
    cfg = N.config(M=1500, M_p=600, max_depth=6, repeats=5, pilot_max=-1)   # table B, no per-entry pilot
    ref = r.iteration(cfg, 11, tri, bary)
    assert len(ref["rhat"]) == n

    dev = torch.device("cuda", 0)
    d_tri = torch.tensor([[e.y_tri, e.h_tri] for e in ents], dtype=torch.int32, device=dev)
    d_bary = torch.tensor([[e.y_b1, e.y_b2, e.h_b1, e.h_b2] for e in ents], dtype=torch.float32, device=dev)
    d_info = torch.tensor([e.u | (e.type << 3) | (e.back << 30) for e in ents], dtype=torch.int32, device=dev)
    d_B = torch.full((n,), 1.5 * mx, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    for call in range(2):
        d_rhat = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
        d_nodes = torch.zeros(n, dtype=torch.float32, device=dev)
        r.recip_estimates_noalloc(cfg, 11, n, d_tri.data_ptr(), d_bary.data_ptr(), d_info.data_ptr(),
                                  d_B.data_ptr(), d_rhat.data_ptr(), d_nodes.data_ptr())
        got = d_rhat.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_array_equal(d_nodes.cpu().numpy(), ref["entry_nodes"])
        np.testing.assert_allclose(got, ref["rhat"], rtol=1e-4)
    with pytest.raises(N.PBError) as e:
        r.recip_estimates_noalloc(cfg, 11, 1 << 20, d_tri.data_ptr(), d_bary.data_ptr(), d_info.data_ptr(),
                                  d_B.data_ptr(), d_rhat.data_ptr())
    assert e.value.status == N.PB_ERR_ARG
    r.close()
