"""Host check of the block walk's schedule for the reciprocal estimator
(Alg. I~ in pre-order): walking the top region of the stack (the current node
and the frames that share its weight) with pending counts over runs of nodes
with g >= 0, moving to the pending node below when the region is exhausted,
and walking only negative-g nodes and short runs on the full stack, must
take the same nodes, sum the same terms and leave the same stack as the
sequential walk. This restates, in Python, the schedule k_wf_walk_long runs
on the device; the GPU parity tests compare the device's schedules with each
other and with the oracle."""

import copy

import numpy as np


def _children(g, u):
    r = abs(g)
    n = int(np.floor(r))
    return n + 1 if u < r - n else n


def _seq(G, U, st, start, cnt, cap=48):
    """the sequential walk: frames [weight, pending] with merging on equal weight"""
    s, taken = 0.0, 0
    for j in range(start, start + cnt):
        g, u = G[j], U[j]
        n = _children(g, u)
        s += st["w"] * g
        taken += 1
        cw = st["w"] * (1.0 if g > 0 else -1.0)
        fr = st["fr"]
        if n >= 1:
            if fr and fr[-1][0] == cw:
                fr[-1][1] += n
            else:
                if len(fr) >= cap:
                    return taken, 2, s
                fr.append([cw, n])
        if not fr:
            return taken, 1, s
        st["w"] = fr[-1][0]
        fr[-1][1] -= 1
        if fr[-1][1] == 0:
            fr.pop()
    return taken, 0, s


def _take_top(st):
    w, pend = st["w"], 1
    while st["fr"] and st["fr"][-1][0] == w:
        pend += st["fr"].pop()[1]
    return pend, w


def _put_top(st, pend, w):
    st["w"] = w
    if pend - 1 > 0:
        st["fr"].append([w, pend - 1])


def _pop_below(st):
    if not st["fr"]:
        return False
    st["w"] = st["fr"][-1][0]
    st["fr"][-1][1] -= 1
    if st["fr"][-1][1] == 0:
        st["fr"].pop()
    return True


def _regions(G, U, st, start, cnt, tile=1024, short=64):
    s, nxt, done = 0.0, start, 0
    pend, w = _take_top(st)
    j0 = start
    while j0 < start + cnt and not done:
        c = min(tile, start + cnt - j0)
        pos = 0
        while pos < c and not done:
            gs, us = G[j0:j0 + c], U[j0:j0 + c]
            neg = [jj for jj in range(pos, c) if gs[jj] < 0]
            b = neg[0] if neg else c
            if b < c and b - pos < short:
                _put_top(st, pend, w)
                t, done, ss = _seq(G, U, st, j0 + pos, b - pos + 1)
                s += ss
                nxt += t
                if not done:
                    pend, w = _take_top(st)
                pos = b + 1
                continue
            p, end = pend, c
            for jj in range(pos, b):   # the block scan of (children - 1)
                p = p - 1 + _children(gs[jj], us[jj])
                if p <= 0:
                    end = jj
                    break
            stop = min(b, end + 1)
            s += sum(w * gs[jj] for jj in range(pos, stop))
            nxt += stop - pos
            if end < b:
                if not _pop_below(st):
                    done = 1
                else:
                    pend, w = _take_top(st)
                pos = end + 1
            else:
                pend = p
                if b < c:
                    _put_top(st, pend, w)
                    t, done, ss = _seq(G, U, st, j0 + b, 1)
                    s += ss
                    nxt += t
                    if not done:
                        pend, w = _take_top(st)
                pos = b + 1 if b < c else c
        j0 += c
    if not done:
        _put_top(st, pend, w)
    return nxt - start, done, s


def test_top_region_walk_equals_sequential_walk():
    rng = np.random.default_rng(5)
    ended = 0
    for trial in range(60):
        N = int(rng.integers(1500, 6000))
        pneg = [0.0, 0.002, 0.02, 0.1][trial % 4]
        G = np.where(rng.random(N) < pneg, -0.9 * rng.random(N), rng.random(N) ** 0.05)
        U = rng.random(N)
        st0 = {"w": 1.0 if rng.random() < 0.5 else -1.0, "fr": []}
        for f in range(int(rng.integers(0, 5))):
            wv = 1.0 if f % 2 == 0 else -1.0
            st0["fr"].append([wv, int(rng.integers(1, 5))])
        a, b = copy.deepcopy(st0), copy.deepcopy(st0)
        ta, da, sa = _seq(G, U, a, 0, N)
        tb, db, sb = _regions(G, U, b, 0, N)
        assert (ta, da) == (tb, db), (trial, ta, tb, da, db)
        assert abs(sa - sb) <= 1e-9 * max(1.0, abs(sa)), (trial, sa, sb)
        if not da:
            assert a == b, trial
        ended += da == 1
    assert ended > 5   # both chains that end inside the window and chains that go on are covered
