"""The allocation-free estimator entry point against the pooled one and the oracle.

pb_recip_estimates_noalloc serves callers that cannot allocate device memory
while they run (engines that reserve all device memory up front, processes
whose allocations another runtime caps or pools, latency-critical code that
cannot take cudaMalloc's implicit synchronisation). Given the entries of an
iteration's pool in (light path, vertex) order it must return the same
reciprocal estimates as pb_iteration, and the oracle's within the parity
tolerance, twice in a row on the same (shared, reused) scratch, without
changing the device's free memory. This file sorts last so that a run
stopping at the first failure has run every other test before it.
"""

import numpy as np
import pytest

import oracle as O
from paper_2503_23412_gb300 import scenes

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    from paper_2503_23412_gb300 import build
    build.build()
    from paper_2503_23412_gb300 import native as N

    sc = scenes.cornell(16, 16)
    o = O.Oracle(sc)
    p = O.params(M=1500, M_p=600, max_depth=6)
    tri, bary = o.light_pass(p, 11)
    ents, _ = o.entries(p, tri, bary)
    assert len(ents) > 20
    # one B for every cell keeps both paths on the same bound: 1.5 x the
    # largest f/q of 64 draws over all entries
    mx = 0.0
    for k, e in enumerate(ents):
        f, q = o.entry_fq(e, 64, a=3, b=k)
        r = np.where(q > 0, f / np.where(q > 0, q, 1.0), 0.0)
        mx = max(mx, float(r.max()))
    tab = scenes.random_tables(sc, KT=8, KS=8, KSp=4, KC=2, B=1.5 * mx, mis=1.0)
    r = N.Renderer(sc, tab)
    dev = torch.device("cuda", 0)
    d = dict(
        tri=torch.tensor([[e.y_tri, e.h_tri] for e in ents], dtype=torch.int32, device=dev),
        bary=torch.tensor([[e.y_b1, e.y_b2, e.h_b1, e.h_b2] for e in ents], dtype=torch.float32, device=dev),
        info=torch.tensor([e.u | (e.type << 3) | (e.back << 30) for e in ents], dtype=torch.int32, device=dev),
        B=torch.full((len(ents),), 1.5 * mx, dtype=torch.float32, device=dev))
    yield dict(torch=torch, N=N, sc=sc, o=o, tri=tri, bary=bary, ents=ents, tab=tab, r=r, d=d, dev=dev)
    r.close()


def _outputs(s):
    torch = s["torch"]
    return (torch.full((len(s["ents"]),), float("nan"), dtype=torch.float32, device=s["dev"]),
            torch.zeros(len(s["ents"]), dtype=torch.float32, device=s["dev"]))


def _call(s, cfg, n=None, B=None, out=None):
    """One call on device buffers; the outputs are allocated here unless given."""
    d = s["d"]
    n = len(s["ents"]) if n is None else n
    rhat, nodes = _outputs(s) if out is None else out
    ntr = s["r"].recip_estimates_noalloc(cfg, 11, n, d["tri"].data_ptr(), d["bary"].data_ptr(), d["info"].data_ptr(),
                                         (d["B"] if B is None else B).data_ptr(), rhat.data_ptr(), nodes.data_ptr())
    return rhat, nodes, ntr


@pytest.mark.parametrize("side_in", [0.0, 0.9])
def test_noalloc_estimates_match_pooled_estimator_and_oracle(setup, side_in):
    """Two calls in a row equal pb_iteration's estimates (node counts
    exactly), match the oracle's FP64 estimates within the parity tolerance,
    report the pooled run's truncation count, and leave the device's free
    memory unchanged. side_in = 0.9 moves the dielectric sphere's cosine
    draws toward the dropped vertex (Sec. 5.3); both paths read it."""
    s = setup
    N, torch, r = s["N"], s["torch"], s["r"]
    cfg = N.config(M=1500, M_p=600, max_depth=6, repeats=5, pilot_max=-1, side_in=side_in)   # table B, no pilot
    ref = r.iteration(cfg, 11, s["tri"], s["bary"])
    n = len(s["ents"])
    assert len(ref["rhat"]) == n
    orc = s["o"].iteration(O.params(M=1500, M_p=600, max_depth=6, pilot_max=0, side_in=side_in),
                           s["o"].tables(s["tab"]), 11, s["tri"], s["bary"], pix_lo=0, pix_hi=0)
    outs = [_outputs(s) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        free0 = torch.cuda.mem_get_info()[0]
        rhat, nodes, ntr = _call(s, cfg, out=outs[call])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        got, nodes = rhat.cpu().numpy(), nodes.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_array_equal(nodes, ref["entry_nodes"])
        np.testing.assert_allclose(got, ref["rhat"], rtol=REL)
        assert ntr == ref["stats"]["n_truncated"]
        np.testing.assert_array_equal(nodes, orc["entry_nodes"])
        np.testing.assert_allclose(got, orc["rhat"], rtol=REL)


def test_noalloc_truncation_count_matches_pooled_run(setup):
    """A 24-node cap truncates many chains: the call reports as many entries
    with a truncated repeat as the pooled estimator does."""
    s = setup
    N = s["N"]
    cfg = N.config(M=1500, M_p=600, max_depth=6, repeats=5, pilot_max=-1, trial_cap=24)
    ref = s["r"].iteration(cfg, 11, s["tri"], s["bary"])
    assert ref["stats"]["n_truncated"] > 0
    for call in range(2):
        rhat, _, ntr = _call(s, cfg)
        assert ntr == ref["stats"]["n_truncated"]
        assert np.isfinite(rhat.cpu().numpy()).all()


def test_noalloc_rejects_bad_bounds_and_sizes(setup):
    """An entry whose B is not positive gets NaN and an error status, while
    the others are still estimated; sizes beyond the array's capacity and an
    out-of-range side_in are rejected before any work."""
    s = setup
    N, torch = s["N"], s["torch"]
    cfg = N.config(M=1500, M_p=600, max_depth=6, repeats=5, pilot_max=-1)
    good = _call(s, cfg)[0].cpu().numpy()
    B = s["d"]["B"].clone()
    B[3] = 0.0
    with pytest.raises(N.PBError) as e:
        _call(s, cfg, B=B)
    assert e.value.status == N.PB_ERR_ARG
    rhat = torch.full((len(s["ents"]),), float("nan"), dtype=torch.float32, device=s["dev"])
    d = s["d"]
    with pytest.raises(N.PBError):
        s["r"].recip_estimates_noalloc(cfg, 11, len(s["ents"]), d["tri"].data_ptr(), d["bary"].data_ptr(),
                                       d["info"].data_ptr(), B.data_ptr(), rhat.data_ptr())
    got = rhat.cpu().numpy()
    assert np.isnan(got[3])
    keep = np.arange(len(got)) != 3
    np.testing.assert_allclose(got[keep], good[keep], rtol=REL)
    with pytest.raises(N.PBError) as e:
        _call(s, cfg, n=1 << 20)
    assert e.value.status == N.PB_ERR_ARG
    with pytest.raises(N.PBError) as e:
        _call(s, N.config(M=1500, M_p=600, max_depth=6, repeats=5, pilot_max=-1, side_in=1.0))
    assert e.value.status == N.PB_ERR_ARG
