// Loading one incomplete light sub-path of the pool as an estimator entry
// (shared by the estimator's warp/block kernels and its wavefront kernels).
#pragma once

#include "pb_kernels.h"
#include "pb_estimator.cuh"

// Entry k of slot `slot`: y_{s-1} (Y), h_c = y_0 (H), the side of y_{s-2}
// relative to Y's normal, u, the type, and the S' and C labels.
__device__ __forceinline__ Entry load_entry(const DScene &S, const KParams &P, const Pool &B, int slot, int k,
                                            int &Sp, int &C) {
    size_t o = (size_t)slot * B.ML;
    int fixed = B.ent_idx[o + k];
    int l = fixed / P.L, e = fixed % P.L;
    size_t gb = o + (size_t)l * P.L;
    Entry E;
    E.Y = vertex_at(S, B.gtri[gb + e], B.gbary[gb + e].x, B.gbary[gb + e].y);
    E.H = vertex_at(S, B.gtri[gb], B.gbary[gb].x, B.gbary[gb].y);
    Vtx Yp = vertex_at(S, B.gtri[gb + e - 1], B.gbary[gb + e - 1].x, B.gbary[gb + e - 1].y);
    E.back = dot(E.Y.n, Yp.p - E.Y.p) < 0.0f ? 1 : 0;
    E.pin = P.side_in;
    int info = B.einfo[o + fixed];
    E.u = info & 7;
    E.type = (info >> 3) & 1;
    C = info >> 4;
    Sp = B.elabel[o + fixed];
    return E;
}
