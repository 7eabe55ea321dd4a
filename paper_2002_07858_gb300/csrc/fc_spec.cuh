// fc_spec.cuh -- where a grid's spectra come from: stored rows, or the
// oscillation shape model evaluated where a row is read.
//
// The paper's kernels recompute the prediction S(q) from the physics model for
// every evaluation rather than caching it (§3, Table 2).  A grid loaded from a
// shape model may be kept the same way: none of its binary64 spectra, their
// centred, binary32 or double-float copies is stored, and every kernel that
// reads a row asks this header for it.  The model is
//     s_i(p) = b_i + sum_t amp_t(p) sin^2(1.27 dm2_t(p) L_i / E_i) f_ti
// and its sine depends only on the value of the term's dm2 axis and the bin,
// so it is tabulated once per (axis value, bin); a spectrum element then costs
// three multiplies and an add per term.  The same evaluation fills a stored
// grid, so a grid gives the same bits stored or recomputed.
// (SpecModel, FullSrc and GridSpec themselves are declared in fc_internal.cuh.)
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fc_df.cuh"
#include "fc_internal.cuh"

namespace fcdev {

// one grid point of the model: each term's amplitude and sine-table row
struct ModelRow {
    double amp[kMaxOscTerms];
    const double* sn[kMaxOscTerms];
};

__device__ __forceinline__ ModelRow model_row(const SpecModel& m, int64_t g) {
    int idx[kMaxOscAxes];
    int64_t rem = g;
    for (int a = m.D - 1; a >= 0; --a) {
        const int64_t len = m.axis_len[a];
        idx[a] = (int)(rem % len);
        rem /= len;
    }
    ModelRow r;
#pragma unroll
    for (int t = 0; t < kMaxOscTerms; ++t) {
        if (t < m.n_terms) {
            r.amp[t] = m.axis_val[m.axis_off[m.amp_ax[t]] + idx[m.amp_ax[t]]];
            r.sn[t] = m.sinT + (int64_t)(m.sin_off[t] + idx[m.dm2_ax[t]]) * m.nf;
        } else {
            r.amp[t] = 0.0;
            r.sn[t] = nullptr;
        }
    }
    return r;
}

// full bin i: b_i, then each term's amp (sn sn) f added in order t = 0, 1, ...
// (every operation separately rounded)
__device__ __forceinline__ double model_full(const SpecModel& m, const ModelRow& r, int i) {
    double v = m.b[i];
#pragma unroll
    for (int t = 0; t < kMaxOscTerms; ++t) {
        if (t < m.n_terms) {
            const double sn = r.sn[t][i];
            v = __dadd_rn(v, __dmul_rn(__dmul_rn(r.amp[t], __dmul_rn(sn, sn)), m.f[t * m.nf + i]));
        }
    }
    return v;
}

// fit bin j: its full bins summed in increasing order from 0 (the collapse of
// a stored grid, k_collapse)
__device__ __forceinline__ double model_fit(const SpecModel& m, const ModelRow& r, int j) {
    if (m.mem_off == nullptr) return __dadd_rn(0.0, model_full(m, r, j));
    double acc = 0.0;
    for (int k = m.mem_off[j]; k < m.mem_off[j + 1]; ++k) acc = __dadd_rn(acc, model_full(m, r, m.mem[k]));
    return acc;
}

// Row g of a full-bin source into out[0 .. nf) by every thread of the CTA,
// followed by a barrier.
__device__ __forceinline__ void stage_full_row(const FullSrc& src, int nf, int64_t g, double* out) {
    if (src.S) {
        for (int i = threadIdx.x; i < nf; i += blockDim.x) out[i] = src.S[g * nf + i];
    } else {
        const ModelRow r = model_row(src.m, g);
        for (int i = threadIdx.x; i < nf; i += blockDim.x) out[i] = model_full(src.m, r, i);
    }
    __syncthreads();
}

// one row of a GridSpec: a stored row, or the model's row
struct FitRow {
    int64_t g;
    ModelRow mr;
};

__device__ __forceinline__ FitRow fit_row(const GridSpec& gs, int64_t g) {
    FitRow r;
    r.g = g;
    if (gs.S_fit == nullptr) r.mr = model_row(gs.m, g);
    return r;
}

__device__ __forceinline__ double row_fit(const GridSpec& gs, const FitRow& r, int j) {
    return gs.S_fit ? gs.S_fit[r.g * gs.nfit + j] : model_fit(gs.m, r.mr, j);
}

__device__ __forceinline__ double row_sc(const GridSpec& gs, const FitRow& r, int j) {
    return gs.Sc ? gs.Sc[r.g * gs.nfit + j] : __dsub_rn(row_fit(gs, r, j), gs.centre[j]);
}

__device__ __forceinline__ float row_sc32(const GridSpec& gs, const FitRow& r, int j) {
    return gs.Sc32 ? gs.Sc32[r.g * gs.nfit + j] : (float)__dsub_rn(row_fit(gs, r, j), gs.centre[j]);
}

__device__ __forceinline__ float2 row_df(const GridSpec& gs, const FitRow& r, int j) {
    return gs.Sdf ? gs.Sdf[r.g * gs.nfit + j] : df_from(row_fit(gs, r, j));
}

// A row of s as double-float for the residual routines: a stored row (p), or
// the model's row.  Held by value: every routine that takes one is inlined, so
// the copy folds away and no kernel parameter has its address taken.
struct DfRow {
    const float2* p;  // stored row or nullptr
    GridSpec gs;
    FitRow r;
    __device__ __forceinline__ float2 operator[](int j) const { return p ? p[j] : row_df(gs, r, j); }
};

// row g of S as double-float (g = -1: the centre)
__device__ __forceinline__ DfRow df_row_of(const GridSpec& gs, const float2* centre_df, int64_t g) {
    DfRow d;
    d.gs = gs;
    if (g < 0) {
        d.p = centre_df;
    } else if (gs.Sdf) {
        d.p = gs.Sdf + g * gs.nfit;
    } else {
        d.p = nullptr;
        d.r = fit_row(gs, g);
    }
    return d;
}

}  // namespace fcdev
