"""Host check of the lane-refill loop of the persistent traversal kernels
(k_wf_trace_pt, k_eye_occ_pt): warps of 32 lanes take queries from one
counter with a ballot (the lanes that need work take consecutive indices),
advance each busy lane by up to PT_STEPS node visits per trip, and leave
when no lane is busy and every lane has seen the counter run out. With warps
scheduled in an arbitrary interleaving and traversals of random length, every
query must be answered exactly once and every warp must leave: each trip
either advances a busy lane's traversal or takes or refuses a query."""

import numpy as np

PT_STEPS = 8


def _run(n, steps_of, n_warps, rng):
    counter = [0]
    answered = np.zeros(n, np.int64)
    warps = [dict(q=[-1] * 32, left=[0] * 32, drained=[False] * 32, done=False, trips=0) for _ in range(n_warps)]
    live = list(range(n_warps))
    while live:
        w = warps[live[rng.integers(len(live))]]   # any warp may run its next trip
        w["trips"] += 1
        need = [w["q"][l] < 0 and not w["drained"][l] for l in range(32)]
        if any(need):
            base = counter[0]
            counter[0] += sum(need)
            rank = 0
            for l in range(32):
                if need[l]:
                    k = base + rank
                    rank += 1
                    if k < n:
                        w["q"][l] = k
                        w["left"][l] = steps_of[k]
                    else:
                        w["drained"][l] = True
        if not any(q >= 0 for q in w["q"]):
            if all(w["drained"]):
                w["done"] = True
                live = [i for i in live if not warps[i]["done"]]
            continue
        for l in range(32):
            if w["q"][l] >= 0:
                w["left"][l] -= min(PT_STEPS, w["left"][l])
                if w["left"][l] == 0:
                    answered[w["q"][l]] += 1
                    w["q"][l] = -1
    return answered, warps


def test_every_query_is_answered_once_and_every_warp_leaves():
    rng = np.random.default_rng(3)
    for n, n_warps in ((0, 3), (1, 4), (31, 1), (1000, 7), (5000, 24)):
        steps_of = rng.integers(1, 200, n) if n else np.zeros(0, np.int64)
        answered, warps = _run(n, steps_of, n_warps, rng)
        assert np.all(answered == 1)
        # a trip that finds no work and no busy lane only happens once per lane before it leaves
        work_trips = int(np.sum(-(-steps_of // PT_STEPS))) if n else 0
        for w in warps:
            assert w["done"]
            assert w["trips"] <= work_trips + n + 33, (w["trips"], n)
