// fc_kernels.cu -- CUDA kernels of the Feldman-Cousins grid fit (all steps but
// the tensor-core screen, which lives in fc_screen.cu).
//
// Method (§2, Algorithm 1, Algorithm 2, Eq. 1): per universe, fluctuate the
// true point's spectrum, scan every grid spectrum with chi2 = r^T A r
// (r = s_g - d, A = M^-1), keep the first minimum, refit M at the minimum and
// rescan until the minimum repeats, then dchi2 = chi2(p) - chi2_min under the
// last scan's A.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>
#include <cstdint>

#include "fc_df.cuh"
#include "fc_internal.cuh"
#include "fc_sampler.cuh"
#include "fc_spec.cuh"

namespace fcdev {

namespace {

constexpr int kThreads = 256;
constexpr int kResolveMaxN = 64;  // a fit-space matrix is staged in shared memory up to this N_fit

inline unsigned blocks_for(int64_t n, int t = kThreads) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 2147483647LL) b = 2147483647LL;
    return (unsigned)b;
}

// (value, index) lexicographic minimum across a warp
__device__ __forceinline__ void warp_argmin(double& v, int32_t& g) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int32_t og = __shfl_xor_sync(0xffffffffu, g, o);
        if (ov < v || (ov == v && og < g)) {
            v = ov;
            g = og;
        }
    }
}

// The plain path's residual form ||W r||^2 (r = s - d, A = W^T W, W lower
// triangular) in binary64, spread over a warp: lanes form the row dot products
// t_i = sum_{j<=i} W_ij r_j (each summed over j in increasing order with fma),
// lane 0 sums t_i^2 in row order with fma.
// r and t are this warp's shared-memory vectors; the result is lane 0's.
__device__ double resid_chi2_warp(const double* __restrict__ W, int n, const double* r, double* t, int lane) {
    for (int i = lane; i < n; i += 32) {
        const double* Wi = W + i * n;
        double x = 0.0;
        for (int j = 0; j <= i; ++j) x = fma(Wi[j], r[j], x);
        t[i] = x;
    }
    __syncwarp();
    double acc = 0.0;
    if (lane == 0)
        for (int i = 0; i < n; ++i) acc = fma(t[i], t[i], acc);
    __syncwarp();
    return acc;
}

// The mixed path's residual chi2 = |W (s - d)|^2 in double-float (fc_df.cuh):
// r_j = s_j - d_j, t_i = sum_j W_ij r_j (df_row), chi2 = sum_i t_i^2 in
// increasing i.  Every mixed-path kernel evaluates
// it in this order, so a universe's result has the same bits whichever
// certified round decided it.  W and s are double-float copies of the
// binary64 arrays; the value is returned as binary64.
// Row i of W r: four interleaved partial sums (j = 0, 1, 2, 3 mod 4, each in
// increasing j) so that four double-float chains run side by side, combined
// as (p0 + p1) + (p2 + p3) and renormalised.  A row runs over whole blocks of
// four columns, j < min(4 ceil((i + 1) / 4), N_fit): W is lower triangular
// with exact zeros above the diagonal (k_build_cov), so the columns past the
// diagonal add exact zeros and every kernel takes the same blocks.
__device__ __forceinline__ float2 df_row(const float2* __restrict__ Wi, const float2* __restrict__ r, int len, int n) {
    float2 p0 = make_float2(0.0f, 0.0f), p1 = p0, p2 = p0, p3 = p0;
    for (int j = 0; j < len; j += 4) {
        p0 = df_fma(p0, Wi[j], r[j]);
        if (j + 1 < n) p1 = df_fma(p1, Wi[j + 1], r[j + 1]);
        if (j + 2 < n) p2 = df_fma(p2, Wi[j + 2], r[j + 2]);
        if (j + 3 < n) p3 = df_fma(p3, Wi[j + 3], r[j + 3]);
    }
    const float2 a = df_add(df_norm(p0.x, p0.y), df_norm(p1.x, p1.y));
    const float2 b = df_add(df_norm(p2.x, p2.y), df_norm(p3.x, p3.y));
    return df_add(a, b);
}

// Four consecutive entries W[k .. k+3] of a W row: two 16-byte loads when
// rows start on 16 bytes at multiple-of-4 columns (even N_fit), else four.
template <bool EVEN>
__device__ __forceinline__ void w_load4(const float2* __restrict__ Wk, float2 (&w)[4]) {
    if constexpr (EVEN) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(Wk));
        const float4 b = __ldg(reinterpret_cast<const float4*>(Wk) + 1);
        w[0] = make_float2(a.x, a.y);
        w[1] = make_float2(a.z, a.w);
        w[2] = make_float2(b.x, b.y);
        w[3] = make_float2(b.z, b.w);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = __ldg(Wk + c);
    }
}

// The residual chi2 computed four rows at a time: each group of four columns
// of r is loaded once per block of rows i0 .. i0+3 (i0 a multiple of 4) and
// meets the four rows' W entries.  Row i keeps df_row's four chains (column j
// on chain j mod 4, each chain in increasing j) and the rows are squared and
// summed in increasing i, so every operation and its order are df_row's and
// the row loop's: the bits are the same, with a quarter of the loads of r.
// In the last block, rows past N_fit read row N_fit - 1 and are dropped.
template <bool EVEN, class SRow>
__device__ __forceinline__ double resid_df_blk(const float2* __restrict__ W, int n, const SRow& s,
                                               const float* __restrict__ du) {
    __align__(16) float2 r[kMaxBins + 4];
    for (int j = 0; j < n; ++j) r[j] = df_sub_f(s[j], du[j]);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int i0 = 0; i0 < n; i0 += 4) {
        float2 p[4][4];
        const float2* Wb[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            Wb[b] = W + (i0 + b < n ? i0 + b : n - 1) * n;
#pragma unroll
            for (int c = 0; c < 4; ++c) p[b][c] = make_float2(0.0f, 0.0f);
        }
        // columns 0 .. i0-1: every row of the block takes all four of each group
#pragma unroll 1
        for (int j = 0; j < i0; j += 4) {
            const float4 ra = *reinterpret_cast<const float4*>(&r[j]);
            const float4 rb = *reinterpret_cast<const float4*>(&r[j + 2]);
            const float2 rv[4] = {make_float2(ra.x, ra.y), make_float2(ra.z, ra.w), make_float2(rb.x, rb.y),
                                  make_float2(rb.z, rb.w)};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float2 w[4];
                w_load4<EVEN>(Wb[b] + j, w);
#pragma unroll
                for (int c = 0; c < 4; ++c) p[b][c] = df_fma(p[b][c], w[c], rv[c]);
            }
        }
        // columns i0 .. i0+3 (those below N_fit): the whole block for every row of the block
        // (W is zero above the diagonal)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (i0 + c < n) {
                const float2 rc = r[i0 + c];
#pragma unroll
                for (int b = 0; b < 4; ++b) p[b][c] = df_fma(p[b][c], Wb[b][i0 + c], rc);
            }
        }
        const int nb = (n - i0 < 4) ? n - i0 : 4;  // rows of this block that exist
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (b < nb) {
                const float2 x = df_add(df_norm(p[b][0].x, p[b][0].y), df_norm(p[b][1].x, p[b][1].y));
                const float2 y = df_add(df_norm(p[b][2].x, p[b][2].y), df_norm(p[b][3].x, p[b][3].y));
                const float2 t = df_add(x, y);
                acc = df_fma(acc, t, t);
            }
        }
    }
    return df_to(df_norm(acc.x, acc.y));
}

// s: the row s_g as double-float (a stored row, or a DfRow that may evaluate the shape model)
template <class SRow>
__device__ double resid_df(const float2* __restrict__ W, int n, const SRow& s, const float* __restrict__ du) {
    return (n % 2 == 0) ? resid_df_blk<true>(W, n, s, du) : resid_df_blk<false>(W, n, s, du);
}

// resid_df with the residual vector in registers, for N_fit <= NR: every index
// of r is a compile-time constant (the column loop is unrolled in blocks of
// four and a block runs only when the row reaches it, a branch that is uniform
// across the warp because all its lanes walk the same rows).  The operations
// and their order are resid_df's, term for term, so the bits are the same;
// what changes is that no per-thread array lives in local memory.
template <int NR, class SRow>
__device__ __forceinline__ double resid_df_reg(const float2* __restrict__ W, int n, const SRow& s,
                                               const float* __restrict__ du) {
    static_assert(NR % 4 == 0, "NR is a multiple of 4");
    float2 r[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) r[j] = (j < n) ? df_sub_f(s[j], du[j]) : make_float2(0.0f, 0.0f);
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
        const float2* Wi = W + i * n;
        const int len = i + 1;
        float2 p0 = make_float2(0.0f, 0.0f), p1 = p0, p2 = p0, p3 = p0;
#pragma unroll
        for (int j = 0; j < NR; j += 4) {
            if (j < len) {  // whole blocks (df_row)
                p0 = df_fma(p0, Wi[j], r[j]);
                if (j + 1 < n) p1 = df_fma(p1, Wi[j + 1], r[j + 1]);
                if (j + 2 < n) p2 = df_fma(p2, Wi[j + 2], r[j + 2]);
                if (j + 3 < n) p3 = df_fma(p3, Wi[j + 3], r[j + 3]);
            }
        }
        const float2 a = df_add(df_norm(p0.x, p0.y), df_norm(p1.x, p1.y));
        const float2 b = df_add(df_norm(p2.x, p2.y), df_norm(p3.x, p3.y));
        const float2 t = df_add(a, b);
        acc = df_fma(acc, t, t);
    }
    return df_to(df_norm(acc.x, acc.y));
}

// The mixed path's residual chi2 for a compile-time bound NR on N_fit (0 = any N_fit).
template <int NR, class SRow>
__device__ __forceinline__ double resid_mixed(const float2* __restrict__ W, int n, const SRow& s,
                                              const float* __restrict__ du) {
    if constexpr (NR > 0)
        return resid_df_reg<NR>(W, n, s, du);
    else
        return resid_df(W, n, s, du);
}

// resid_df spread over a warp with the same bits: r_j = s_j - d_j is formed in
// this warp's shared vector r, lanes form the rows t_i into t, lane 0 sums
// t_i^2 in row order.  The result is lane 0's.
template <class SRow>
__device__ double resid_df_warp(const float2* __restrict__ W, int n, const SRow& s, const float* __restrict__ du,
                                float2* r, float2* t, int lane) {
    for (int j = lane; j < n; j += 32) r[j] = df_sub_f(s[j], du[j]);
    __syncwarp();
    for (int i = lane; i < n; i += 32) t[i] = df_row(W + i * n, r, i + 1, n);
    __syncwarp();
    float2 acc = make_float2(0.0f, 0.0f);
    if (lane == 0)
        for (int i = 0; i < n; ++i) acc = df_fma(acc, t[i], t[i]);
    __syncwarp();
    return df_to(df_norm(acc.x, acc.y));
}

// Row g of s for the residual routines (g = -1: the centre).  The kernels that
// score residuals are instantiated twice: MODEL = false reads the stored
// double-float rows through a plain pointer, MODEL = true (a recomputed grid)
// evaluates the shape model through a DfRow.  Both feed the same routines, so
// the bits agree and the stored path carries none of the model's registers.
template <bool MODEL>
__device__ __forceinline__ auto srow(const GridSpec& gs, const float2* centre_df, int64_t g) {
    if constexpr (MODEL)
        return df_row_of(gs, centre_df, g);
    else
        return (g < 0) ? centre_df : gs.Sdf + g * gs.nfit;
}

// double-float copies of W for a list of slots
__global__ void k_wdf(const double* __restrict__ W64, const int32_t* __restrict__ slots, int nfit,
                      float2* __restrict__ Wdf) {
    const size_t base = (size_t)slots[blockIdx.x] * nfit * nfit;
    for (int e = threadIdx.x; e < nfit * nfit; e += blockDim.x) Wdf[base + e] = df_from(W64[base + e]);
}

__global__ void k_to_df(const double* __restrict__ x, int64_t n, float2* __restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = df_from(x[i]);
}

// ---------------------------------------------------------------- ingest ---

__global__ void k_collapse(const double* __restrict__ S, int64_t G, int nf, const int32_t* __restrict__ coll,
                           int nfit, double* __restrict__ out) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= G) return;
    double acc[kMaxBins];
    for (int j = 0; j < nfit; ++j) acc[j] = 0.0;
    for (int i = 0; i < nf; ++i) {
        const int j = coll ? coll[i] : i;
        acc[j] = __dadd_rn(acc[j], S[g * nf + i]);
    }
    for (int j = 0; j < nfit; ++j) out[g * nfit + j] = acc[j];
}

// Sine table of an oscillation shape model: for each term t and each value k
// of its dm2 axis, sin(1.27 dm2_k L_i / E_i) for every full bin i, with the
// products and the quotient in that order.
__global__ void k_osc_sin(SpecModel m, int rows, const double* __restrict__ L, const double* __restrict__ E,
                          double* __restrict__ sinT) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * m.nf) return;
    const int row = (int)(e / m.nf), i = (int)(e % m.nf);
    int t = 0;
    while (t + 1 < m.n_terms && row >= m.sin_off[t + 1]) ++t;
    const int a = m.dm2_ax[t];
    const double dm2 = m.axis_val[m.axis_off[a] + (row - m.sin_off[t])];
    sinT[e] = sin(__ddiv_rn(__dmul_rn(__dmul_rn(1.27, dm2), L[i]), E[i]));
}

// Grid spectra from an oscillation shape model, one thread per (grid point,
// full bin): s_i(p) = b_i + sum_t amp_t(p) sin^2(1.27 dm2_t(p) L_i / E_i) f_ti,
// the terms added in order t = 0, 1, ... to b_i (model_full).  Grid point p is
// the row-major index over the axes (axis 0 slowest); term t reads its
// amplitude from axis amp_ax[t] and its dm2 from axis dm2_ax[t].  S null: the
// spectra are only checked.  bad counts entries that are not finite and >= 0.
__global__ void k_osc_spectra(SpecModel m, int64_t G, double* __restrict__ S, int* __restrict__ bad) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= G * m.nf) return;
    const int64_t g = e / m.nf;
    const int i = (int)(e % m.nf);
    const double v = model_full(m, model_row(m, g), i);
    if (S) S[e] = v;
    if (!(v >= 0.0) || !isfinite(v)) atomicAdd(bad, 1);
}

// Approximate per-bin median of the grid spectra by two rounds of a 4096-bucket
// histogram; it only chooses the centring vector of the screen, any value works.
__global__ void k_centre(GridSpec gs, int64_t G, double* __restrict__ centre) {
    constexpr int NB = 4096;
    __shared__ unsigned hist[NB];
    __shared__ double red_lo[kThreads / 32], red_hi[kThreads / 32];
    __shared__ double s_lo, s_hi;
    __shared__ int64_t s_rank;
    __shared__ int s_bucket;
    const int j = blockIdx.x;
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int64_t g = threadIdx.x; g < G; g += blockDim.x) {
        const double x = row_fit(gs, fit_row(gs, g), j);
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red_lo[threadIdx.x >> 5] = lo;
        red_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = red_lo[0], b = red_hi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a = fmin(a, red_lo[w]);
            b = fmax(b, red_hi[w]);
        }
        s_lo = a;
        s_hi = b;
        s_rank = (G - 1) / 2;
    }
    __syncthreads();
    double blo = s_lo, bhi = s_hi;
    for (int round = 0; round < 2; ++round) {
        for (int b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const double w = (bhi - blo) / NB;
        for (int64_t g = threadIdx.x; g < G; g += blockDim.x) {
            const double x = row_fit(gs, fit_row(gs, g), j);
            if (x < blo || x > bhi) continue;
            int b = (w > 0.0) ? (int)((x - blo) / w) : 0;
            b = b < 0 ? 0 : (b >= NB ? NB - 1 : b);
            atomicAdd(&hist[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t acc = 0;
            int b = 0;
            for (; b < NB; ++b) {
                if (acc + hist[b] > s_rank) break;
                acc += hist[b];
            }
            if (b >= NB) b = NB - 1;
            s_bucket = b;
            s_rank -= acc;
        }
        __syncthreads();
        const double nlo = blo + w * s_bucket;
        const double nhi = (s_bucket == NB - 1) ? bhi : blo + w * (s_bucket + 1);
        __syncthreads();
        blo = nlo;
        bhi = nhi;
    }
    if (threadIdx.x == 0) centre[j] = 0.5 * (blo + bhi);
}

__device__ __forceinline__ int64_t btile_offset(int64_t g, int c, int K) {
    // B-operand image of one BN-row tile: [2K/8 chunks][BN/8 row groups][8 rows][8 cols] bf16
    const int64_t t = g / kBN;
    const int r = (int)(g % kBN);
    return t * (int64_t)(2 * K * kBN) + (int64_t)(c >> 3) * (kBN * 8) + (r >> 3) * 64 + (r & 7) * 8 + (c & 7);
}

// The screen's bf16 hi/lo image of s~ = s - centre and the norms of its split,
// one thread per grid point; the binary64 and binary32 centred rows are stored
// when Sc / Sc32 are given.
__global__ void k_centred(GridSpec gs, int64_t G, int K, double* __restrict__ Sc, float* __restrict__ Sc32,
                          float4* __restrict__ gnorm, uint16_t* __restrict__ Bt) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int nfit = gs.nfit;
    const FitRow fr = fit_row(gs, g);
    double ss = 0.0, sl = 0.0, sr = 0.0;
    for (int j = 0; j < nfit; ++j) {
        const double x = __dsub_rn(row_fit(gs, fr, j), gs.centre[j]);
        if (Sc) Sc[g * nfit + j] = x;
        if (Sc32) Sc32[g * nfit + j] = (float)x;
        ss = fma(x, x, ss);
        const __nv_bfloat16 h = __double2bfloat16(x);
        const double rem = x - (double)__bfloat162float(h);
        const __nv_bfloat16 l = __double2bfloat16(rem);
        const double lo = (double)__bfloat162float(l);
        const double res = rem - lo;  // r_S: what hi + lo leave out
        sl = fma(lo, lo, sl);
        sr = fma(res, res, sr);
        Bt[btile_offset(g, j, K)] = __bfloat16_as_ushort(h);
        Bt[btile_offset(g, K + j, K)] = __bfloat16_as_ushort(l);
    }
    // norms rounded up (double sqrt, then float), carried by the spare columns of the lo half
    const float n = __double2float_ru(__dsqrt_ru(ss) * (1.0 + 1e-12));
    const float nl = __double2float_ru(__dsqrt_ru(sl) * (1.0 + 1e-12));
    const float nr = __double2float_ru(__dsqrt_ru(sr) * (1.0 + 1e-12));
    gnorm[g] = make_float4(n, nl, nr, 0.0f);
    Bt[btile_offset(g, K + nfit, K)] = __bfloat16_as_ushort(__float2bfloat16_ru(n));
    Bt[btile_offset(g, K + nfit + 1, K)] = __bfloat16_as_ushort(__float2bfloat16_ru(nl));
    Bt[btile_offset(g, K + nfit + 2, K)] = __bfloat16_as_ushort(__float2bfloat16_ru(nr));
}

// ------------------------------------------------------------ covariances ---

// The systematic factor is staged in shared memory as a packed lower triangle
// (element (i, j), j <= i, at i(i+1)/2 + j) up to this N_full: 98 KB at 155,
// 33 KB at N_full = 90, so six true points share an SM.
constexpr int kCholPackN = 155;

// e -> (a, b) with 0 <= b <= a and e = a(a+1)/2 + b
__device__ __forceinline__ void tri_decode(int e, int& a, int& b) {
    a = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    while (a * (a + 1) / 2 > e) --a;
    b = e - a * (a + 1) / 2;
}

template <bool PACKED>
__device__ __forceinline__ int lidx(int i, int j, int n) {
    return PACKED ? i * (i + 1) / 2 + j : i * n + j;
}

// Cholesky in place on the lower triangle (packed, or row-major n x n with the
// upper triangle zeroed at the end; shared or global memory); every element's
// sum runs k = 0..j-1 with separately rounded multiply and subtract, so the
// factor is reproducible bit for bit.
template <bool PACKED>
__device__ bool chol_inplace(double* L, int n) {
    // Right-looking form: after column k is final, every trailing element
    // (i >= j > k) subtracts L_ik L_jk.  Each element therefore still sees its
    // terms in increasing k with a separately rounded multiply and subtract --
    // the same sequence as the left-looking sum -- while the dependency chain
    // shrinks to one step per column.
    __shared__ double s_d;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            double acc = L[lidx<PACKED>(k, k, n)];
            if (!(acc > 0.0)) {
                s_bad = 1;
                acc = 1.0;
            }
            s_d = __dsqrt_rn(acc);
            L[lidx<PACKED>(k, k, n)] = s_d;
        }
        __syncthreads();
        const double dk = s_d;
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
            L[lidx<PACKED>(i, k, n)] = __ddiv_rn(L[lidx<PACKED>(i, k, n)], dk);
        __syncthreads();
        // trailing update of the lower triangle, rows i > k, columns k < j <= i
        const int m = n - k - 1;
        const int cnt = m * (m + 1) / 2;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            int a, b;
            tri_decode(e, a, b);
            const int i = k + 1 + a, jj = k + 1 + b;
            L[lidx<PACKED>(i, jj, n)] =
                __dsub_rn(L[lidx<PACKED>(i, jj, n)], __dmul_rn(L[lidx<PACKED>(i, k, n)], L[lidx<PACKED>(jj, k, n)]));
        }
        __syncthreads();
    }
    if (!PACKED) {
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, c = e % n;
            if (c > i) L[e] = 0.0;
        }
        __syncthreads();
    }
    return s_bad == 0;
}

__global__ void k_chol_sys(FullSrc src, int nf, const double* __restrict__ F, const int64_t* __restrict__ ps,
                           int gauss, double* __restrict__ L64, float* __restrict__ L32, float* __restrict__ s32,
                           int* __restrict__ status) {
    extern __shared__ double sL[];
    __shared__ double s_row[kMaxBins];
    const int ip = blockIdx.x;
    stage_full_row(src, nf, ps[ip], s_row);
    const double* s = s_row;
    double* Lg = L64 + (size_t)ip * nf * nf;
    float* Lf = L32 + (size_t)ip * nf * nf;
    // element (i, j), j <= i, of diag(s) F diag(s) (+ diag(s) in the Gaussian mode)
    auto msys = [&](int i, int j) {
        double v = __dmul_rn(__dmul_rn(s[i], F[i * nf + j]), s[j]);
        if (gauss && i == j) v = __dadd_rn(v, s[i]);
        return v;
    };
    bool ok;
    if (nf <= kCholPackN) {
        // packed in shared memory (the dependent sums run at shared-memory latency)
        const int np = nf * (nf + 1) / 2;
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            int i, j;
            tri_decode(e, i, j);
            sL[e] = msys(i, j);
        }
        __syncthreads();
        ok = chol_inplace<true>(sL, nf);
        for (int e = threadIdx.x; e < nf * nf; e += blockDim.x) {
            const int i = e / nf, j = e % nf;
            const double v = (j <= i) ? sL[i * (i + 1) / 2 + j] : 0.0;
            Lg[e] = v;
            Lf[e] = __double2float_rn(v);
        }
    } else {
        for (int e = threadIdx.x; e < nf * nf; e += blockDim.x) {
            const int i = e / nf, j = e % nf;
            if (j <= i) Lg[e] = msys(i, j);
        }
        __syncthreads();
        ok = chol_inplace<false>(Lg, nf);
        for (int e = threadIdx.x; e < nf * nf; e += blockDim.x) Lf[e] = __double2float_rn(Lg[e]);
    }
    if (!ok && threadIdx.x == 0) atomicOr(status, kDevNotSpd);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) s32[(size_t)ip * nf + i] = __double2float_rn(s[i]);
}

// One CTA per (slot, q): M(q) = C [diag(s) F diag(s) + diag(s)] C^T, L = chol(M),
// W = L^-1, A = W^T W.  The binary64 pipe of this GPU is narrow, so every
// phase spreads its elements over all threads of the CTA (a phase with a few
// busy lanes would hold the pipe for whole warps) and a column's divisions
// become one reciprocal and multiplies.  These factors feed the fit, not the
// fake data, so they need not repeat the oracle's rounding bit for bit.
__global__ void k_build_cov(FullSrc src, int nf, int nfit, const int32_t* __restrict__ coll,
                            const double* __restrict__ F, const int32_t* __restrict__ q_list,
                            const int32_t* __restrict__ slot_list, int cov_mode, double* __restrict__ A64,
                            double* __restrict__ W64, float* __restrict__ A32, float* __restrict__ rho,
                            double* __restrict__ work, int* __restrict__ status) {
    extern __shared__ double sLW[];
    __shared__ int s_moff[kMaxBins + 1], s_mem[kMaxBins], s_cur[kMaxBins];
    __shared__ double s_inv[kMaxBins];
    __shared__ int s_bad;
    const int e0 = blockIdx.x;
    const int q = q_list[e0];
    const int slot = slot_list[e0];
    const int n = nfit;
    const bool staged = (n <= kResolveMaxN);
    double* L = staged ? sLW : work + (size_t)e0 * n * n;
    double* Wg = W64 + (size_t)slot * n * n;
    double* W = staged ? sLW + n * n : Wg;
    double* A = A64 + (size_t)slot * n * n;
    __shared__ double s_row[kMaxBins];
    stage_full_row(src, nf, q, s_row);
    const double* s = s_row;
    if (cov_mode == 2) {  // identity test mode
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const double v = (e / n == e % n) ? 1.0 : 0.0;
            Wg[e] = v;
            A[e] = v;
            A32[(size_t)slot * n * n + e] = (float)v;
        }
        if (threadIdx.x == 0) rho[slot] = 1.0f;
        return;
    }
    // full bins of each fit bin, in increasing order (counting sort by one thread)
    if (threadIdx.x == 0) {
        s_bad = 0;
        if (coll) {
            for (int j = 0; j <= n; ++j) s_moff[j] = 0;
            for (int i = 0; i < nf; ++i) ++s_moff[coll[i] + 1];
            for (int j = 0; j < n; ++j) s_moff[j + 1] += s_moff[j];
            for (int j = 0; j < n; ++j) s_cur[j] = s_moff[j];
            for (int i = 0; i < nf; ++i) s_mem[s_cur[coll[i]]++] = i;
        }
    }
    __syncthreads();
    // 1. M in fit space (lower triangle; upper zero): element (j, l) sums (s_a F_ab) s_b (+ s_a when a == b)
    //    over full bins a -> j, b -> l in increasing (a, b)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int j = e / n, l = e % n;
        double v = 0.0;
        if (l <= j) {
            if (coll == nullptr) {
                v = (s[j] * F[j * nf + l]) * s[l];
                if (j == l) v += s[j];
            } else {
                for (int ia = s_moff[j]; ia < s_moff[j + 1]; ++ia) {
                    const int a = s_mem[ia];
                    for (int ib = s_moff[l]; ib < s_moff[l + 1]; ++ib) {
                        const int b = s_mem[ib];
                        double t = (s[a] * F[a * nf + b]) * s[b];
                        if (a == b) t += s[a];
                        v += t;
                    }
                }
            }
        }
        L[e] = v;
    }
    __syncthreads();
    // 2. Cholesky, right-looking; column k is scaled by the reciprocal of its pivot
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            double d = L[k * n + k];
            if (!(d > 0.0)) {
                s_bad = 1;
                d = 1.0;
            }
            const double sd = __dsqrt_rn(d);
            L[k * n + k] = sd;
            s_inv[k] = 1.0 / sd;
        }
        __syncthreads();
        const double ik = s_inv[k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) L[i * n + k] *= ik;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int a = e / m, b = e % m;
            if (b > a) continue;
            const int i = k + 1 + a, jj = k + 1 + b;
            L[i * n + jj] -= L[i * n + k] * L[jj * n + k];
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) atomicOr(status, kDevNotSpd);
        return;
    }
    // 3. W = L^-1 by elimination on [L | I]: at step k row k of W is scaled by 1/L_kk and
    //    final; every row i > k then subtracts L_ik times it (columns c <= k)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) W[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double ik = s_inv[k];
        for (int c = threadIdx.x; c <= k; c += blockDim.x) W[k * n + c] *= ik;
        __syncthreads();
        const int m = n - k - 1, w = k + 1;
        for (int e = threadIdx.x; e < m * w; e += blockDim.x) {
            const int i = k + 1 + e / w, c = e % w;
            W[i * n + c] -= L[i * n + k] * W[k * n + c];
        }
        __syncthreads();
    }
    // A = W^T W: A_ij = sum_{k >= max(i,j)} W_ki W_kj
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (j > i) continue;
        double acc = 0.0;
        for (int k = i; k < n; ++k) acc = fma(W[k * n + i], W[k * n + j], acc);
        A[i * n + j] = acc;
        A[j * n + i] = acc;
    }
    if (staged)
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) Wg[e] = W[e];
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A32[(size_t)slot * n * n + e] = (float)A[e];
    // rho = max_i sum_j |A_ij| (an upper bound of the spectral norm of |A|), rounded up
    __shared__ double s_rho;
    if (threadIdx.x == 0) s_rho = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += fabs(A[i * n + j]);
        atomicMax((unsigned long long*)&s_rho, (unsigned long long)__double_as_longlong(r));
    }
    __syncthreads();
    if (threadIdx.x == 0) rho[slot] = __double2float_ru(s_rho * (1.0 + 1e-9));
}

// q_g = s~_g^T A s~_g in binary64, one thread per g
// q_g = s~_g^T A s~_g = |W s~_g|^2 (A = W^T W, W lower triangular): t_i = sum_{j<=i}
// W_ij s~_j and q = sum_i t_i^2, each an fma chain in increasing index, so
// N (N + 3) / 2 DFMA per point instead of the N^2 + N of s~^T (A s~).
__global__ void k_qvec64(GridSpec gs, int64_t G, int nfit, const double* __restrict__ W64,
                         const int32_t* __restrict__ slots, int64_t ldq, double* __restrict__ Q64) {
    const int slot = slots[blockIdx.y];
    const double* W = W64 + (size_t)slot * nfit * nfit;
    double sl[kMaxBins];  // the row, when it is recomputed rather than stored
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
        const double* s = gs.Sc ? gs.Sc + g * nfit : sl;
        if (!gs.Sc) {
            const FitRow fr = fit_row(gs, g);
            for (int j = 0; j < nfit; ++j) sl[j] = row_sc(gs, fr, j);
        }
        double q = 0.0;
        for (int i = 0; i < nfit; ++i) {
            const double* Wi = W + i * nfit;
            double t = 0.0;
            for (int j = 0; j <= i; ++j) t = fma(Wi[j], s[j], t);
            q = fma(t, t, q);
        }
        Q64[(size_t)slot * ldq + g] = q;
    }
}

// binary32 q_g with its rounding bound; s~_g held in registers (NMAX >= nfit,
// NMAX a multiple of 4), A staged in shared memory with rows padded to NMAX.
template <int NMAX>
__global__ void k_qvec32(GridSpec gs, const float4* __restrict__ gnorm, int64_t G, int64_t G_pad,
                         int nfit, const float* __restrict__ A32, const float* __restrict__ rho,
                         const int32_t* __restrict__ slots, float* __restrict__ Qc, float* __restrict__ Qb,
                         uint16_t* __restrict__ Qb3) {
    __shared__ __align__(16) float sA[NMAX * NMAX];
    const int slot = slots[blockIdx.y];
    const float* A = A32 + (size_t)slot * nfit * nfit;
    for (int e = threadIdx.x; e < NMAX * NMAX; e += blockDim.x) {
        const int i = e / NMAX, j = e % NMAX;
        sA[e] = (i < nfit && j < nfit) ? A[i * nfit + j] : 0.0f;
    }
    __syncthreads();
    const float r = rho[slot];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G_pad; g += (int64_t)gridDim.x * blockDim.x) {
        float qc = 0.0f, qb = 3.0e38f;
        if (g < G) {
            float s[NMAX];
            if (gs.Sc32) {
#pragma unroll
                for (int j = 0; j < NMAX; ++j) s[j] = (j < nfit) ? gs.Sc32[g * nfit + j] : 0.0f;
            } else {
                const FitRow fr = fit_row(gs, g);
#pragma unroll
                for (int j = 0; j < NMAX; ++j) s[j] = (j < nfit) ? row_sc32(gs, fr, j) : 0.0f;
            }
            float q = 0.0f;
#pragma unroll
            for (int i = 0; i < NMAX; ++i) {
                const float4* Ai = reinterpret_cast<const float4*>(sA + i * NMAX);
                float t = 0.0f;
#pragma unroll
                for (int j4 = 0; j4 < NMAX / 4; ++j4) {
                    const float4 a4 = Ai[j4];
                    t = fmaf(a4.x, s[4 * j4 + 0], t);
                    t = fmaf(a4.y, s[4 * j4 + 1], t);
                    t = fmaf(a4.z, s[4 * j4 + 2], t);
                    t = fmaf(a4.w, s[4 * j4 + 3], t);
                }
                q = fmaf(s[i], t, q);
            }
            const float n = gnorm[g].x;
            // |q^ - q| <= (nfit+4) 2^-24 rho |s|^2 + 2^-23 |q^|   (A rounded to binary32, dot products, final rounding)
            const float beta = 1.02f * ((float)(nfit + 4) * 5.9604645e-08f * r * n * n + q_rel_slack(nfit) * fabsf(q));
            qc = q;
            qb = __fsub_rd(q, beta);
        }
        Qc[(size_t)slot * G_pad + g] = qc;
        Qb[(size_t)slot * G_pad + g] = qb;
        store_qb3(Qb3 + ((size_t)slot * G_pad + g) * 8, qb);
    }
}

__global__ void k_qvec32_generic(GridSpec gs, const float4* __restrict__ gnorm, int64_t G,
                                 int64_t G_pad, int nfit, const float* __restrict__ A32, const float* __restrict__ rho,
                                 const int32_t* __restrict__ slots, float* __restrict__ Qc, float* __restrict__ Qb,
                                 uint16_t* __restrict__ Qb3) {
    const int slot = slots[blockIdx.y];
    const float* A = A32 + (size_t)slot * nfit * nfit;
    const float r = rho[slot];
    float sl[kMaxBins];  // the row, when it is recomputed rather than stored
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G_pad; g += (int64_t)gridDim.x * blockDim.x) {
        float qc = 0.0f, qb = 3.0e38f;
        if (g < G) {
            const float* s = gs.Sc32 ? gs.Sc32 + g * nfit : sl;
            if (!gs.Sc32) {
                const FitRow fr = fit_row(gs, g);
                for (int j = 0; j < nfit; ++j) sl[j] = row_sc32(gs, fr, j);
            }
            float q = 0.0f;
            for (int i = 0; i < nfit; ++i) {
                float t = 0.0f;
                for (int j = 0; j < nfit; ++j) t = fmaf(A[i * nfit + j], s[j], t);
                q = fmaf(s[i], t, q);
            }
            const float n = gnorm[g].x;
            const float beta = 1.02f * ((float)(nfit + 4) * 5.9604645e-08f * r * n * n + q_rel_slack(nfit) * fabsf(q));
            qc = q;
            qb = __fsub_rd(q, beta);
        }
        Qc[(size_t)slot * G_pad + g] = qc;
        Qb[(size_t)slot * G_pad + g] = qb;
        store_qb3(Qb3 + ((size_t)slot * G_pad + g) * 8, qb);
    }
}

// -------------------------------------------------------------- fake data ---

// One thread per universe: z from Philox/Box-Muller, lam_i = max(0, s_i +
// sum_{j<=i} L_ij z_j) accumulated with fma in j order, n_i = Poisson(lam_i)
// from bin i's own stream, fit bin = sum of its full bins in i order.
__global__ void __launch_bounds__(128) k_fake_data(const float* __restrict__ L32, const float* __restrict__ s32,
                                                    int nf, const int32_t* __restrict__ coll, int nfit,
                                                    const int64_t* __restrict__ ps, int U, uint32_t k0,
                                                    uint32_t k1, int gauss, float* __restrict__ d) {
    const int ip = blockIdx.y;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const uint32_t p = (uint32_t)ps[ip];
    const float* L = L32 + (size_t)ip * nf * nf;
    const float* s = s32 + (size_t)ip * nf;
    float z[kMaxBins + 4];
    for (int j = 0; 4 * j < nf; ++j) {
        float zz[4];
        normal_block((uint32_t)j, (uint32_t)u, p, k0, k1, zz);
#pragma unroll
        for (int h = 0; h < 4; ++h) z[4 * j + h] = zz[h];
    }
    float dfit[kMaxBins];
    for (int j = 0; j < nfit; ++j) dfit[j] = 0.0f;
    for (int i = 0; i < nf; ++i) {
        const float* Li = L + (size_t)i * nf;
        float acc = 0.0f;
        for (int j = 0; j <= i; ++j) acc = __fmaf_rn(__ldg(Li + j), z[j], acc);
        float lam = __fadd_rn(__ldg(s + i), acc);
        float v;
        if (gauss) {
            v = lam;
        } else {
            if (!(lam > 0.0f)) lam = 0.0f;
            UniformStream st;
            st.init(k0, k1, (uint32_t)u, p, (uint32_t)i);
            v = (float)poisson(lam, st);
        }
        const int jf = coll ? coll[i] : i;
        dfit[jf] = __fadd_rn(dfit[jf], v);
    }
    float* o = d + ((size_t)ip * U + u) * nfit;
    for (int j = 0; j < nfit; ++j) o[j] = dfit[j];
}

// ------------------------------------------------------- bookkeeping -------

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_iota_i32(int32_t* p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

__global__ void k_mark_used(const int32_t* __restrict__ active, int64_t n, const int32_t* __restrict__ cur,
                            uint8_t* __restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[cur[active[i]]] = 1;
}

__global__ void k_compact_flags(uint8_t* __restrict__ flag, int64_t G, int32_t* __restrict__ list,
                                int32_t* __restrict__ count) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= G) return;
    if (flag[g]) {
        flag[g] = 0;
        list[atomicAdd(count, 1)] = (int32_t)g;
    }
}

__global__ void k_lookup_slots(const int32_t* __restrict__ active, int64_t n, const int32_t* __restrict__ cur,
                               const int32_t* __restrict__ slot_of, int32_t* __restrict__ uslot) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) uslot[i] = slot_of[cur[active[i]]];
}

__global__ void k_set_slots(const int32_t* __restrict__ q, const int32_t* __restrict__ s, int n,
                            int32_t* __restrict__ slot_of) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot_of[q[i]] = s[i];
}

// ------------------------------------------------------ plain fp64 scan -----

// Plain binary64 scan: chi2_g - c = q_g - 2 y.s~_g with y = A (d - v) for every
// g, the first minimum in index order.  The y.s~ products of 32 universes x 64
// grid points are a small dense contraction on the FP64 pipe: y and a tile of
// s~ (transposed to [j][g]) sit in shared memory and every thread keeps a 4 x 2
// block of dot products in registers (the binary64 pipe is narrow, so operand
// loads are never the limit; 16 universes per CTA keep enough CTAs for the
// later scans, which hold fewer universes).  Every dot product is one fma chain
// over j in increasing order, as in a per-pair loop, so the minimum found does
// not depend on the blocking.
constexpr int kS64U = 16;   // universes per CTA
constexpr int kS64G = 64;   // grid points per staged tile
constexpr int kS64LdS = kS64G + 2;  // row stride of the staged tile (fewer bank conflicts, 16-byte rows)
constexpr int kS64Threads = 128;

__global__ void __launch_bounds__(kS64Threads) k_scan64(const int32_t* __restrict__ list, int64_t n,
                                                         const int32_t* __restrict__ uslot,
                                                         const float* __restrict__ d, GridSpec gs, int64_t G,
                                                         int nfit, const double* __restrict__ A64,
                                                         const double* __restrict__ Q64, int64_t ldq,
                                                         int32_t* __restrict__ best) {
    extern __shared__ double2 sm64v[];
    double* sy = reinterpret_cast<double*>(sm64v);   // [nfit][kS64U]
    double* ss = sy + (size_t)nfit * kS64U;          // [nfit][kS64LdS]
    __shared__ double s_bv[kS64Threads / 4][kS64U];
    __shared__ int32_t s_bg[kS64Threads / 4][kS64U];
    __shared__ int s_slot[kS64U];
    const int tid = threadIdx.x;
    const int64_t u0 = (int64_t)blockIdx.x * kS64U;
    const int nu = (int)((n - u0) < kS64U ? (n - u0) : kS64U);
    if (tid < kS64U) s_slot[tid] = (tid < nu) ? uslot[u0 + tid] : 0;
    // d - v of the CTA's universes, [j][u] (in the tile buffer, free until the first tile)
    for (int e = tid; e < nfit * kS64U; e += kS64Threads) {
        const int j = e / kS64U, uu = e - (e / kS64U) * kS64U;
        ss[e] = (uu < nu) ? (double)d[(size_t)list[u0 + uu] * nfit + j] - gs.centre[j] : 0.0;
    }
    __syncthreads();
    // y_r = sum_j A_rj (d - v)_j, one fma chain in j order
    for (int e = tid; e < nfit * kS64U; e += kS64Threads) {
        const int r = e / kS64U, uu = e - (e / kS64U) * kS64U;
        double t = 0.0;
        if (uu < nu) {
            const double* A = A64 + (size_t)s_slot[uu] * nfit * nfit + (size_t)r * nfit;
            for (int j = 0; j < nfit; ++j) t = fma(A[j], ss[j * kS64U + uu], t);
        }
        sy[r * kS64U + uu] = t;
    }
    const int tu = tid & 3, tg = tid >> 2;  // universes 4 tu .. 4 tu + 3, tile points 2 tg, 2 tg + 1
    double bv[4];
    int32_t bg[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        bv[a] = DBL_MAX;
        bg[a] = INT32_MAX;
    }
    for (int64_t g0 = 0; g0 < G; g0 += kS64G) {
        __syncthreads();  // y complete / the previous tile's readers done
        if (gs.Sc) {
            for (int e = tid; e < kS64G * nfit; e += kS64Threads) {
                const int gg = e / nfit, j = e - (e / nfit) * nfit;
                const int64_t g = g0 + gg;
                ss[j * kS64LdS + gg] = (g < G) ? gs.Sc[g * nfit + j] : 0.0;
            }
        } else {
            // recomputed rows: one point per thread, decoded once
            for (int gg = tid; gg < kS64G; gg += kS64Threads) {
                const int64_t g = g0 + gg;
                if (g < G) {
                    const FitRow fr = fit_row(gs, g);
                    for (int j = 0; j < nfit; ++j) ss[j * kS64LdS + gg] = row_sc(gs, fr, j);
                } else {
                    for (int j = 0; j < nfit; ++j) ss[j * kS64LdS + gg] = 0.0;
                }
            }
        }
        __syncthreads();
        double acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) acc[a][b] = 0.0;
        for (int j = 0; j < nfit; ++j) {
            const double2 y01 = *reinterpret_cast<const double2*>(sy + j * kS64U + 4 * tu);
            const double2 y23 = *reinterpret_cast<const double2*>(sy + j * kS64U + 4 * tu + 2);
            const double2 s01 = *reinterpret_cast<const double2*>(ss + j * kS64LdS + 2 * tg);
            const double y[4] = {y01.x, y01.y, y23.x, y23.y};
            const double sv[2] = {s01.x, s01.y};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) acc[a][b] = fma(y[a], sv[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int uu = 4 * tu + a;
            if (uu >= nu) continue;
            const double* Q = Q64 + (size_t)s_slot[uu] * ldq;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int64_t g = g0 + 2 * tg + b;
                if (g >= G) continue;
                const double v = fma(-2.0, acc[a][b], Q[g]);
                if (v < bv[a] || (v == bv[a] && (int32_t)g < bg[a])) {
                    bv[a] = v;
                    bg[a] = (int32_t)g;
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        s_bv[tg][4 * tu + a] = bv[a];
        s_bg[tg][4 * tu + a] = bg[a];
    }
    __syncthreads();
    if (tid < nu) {
        double v = DBL_MAX;
        int32_t g = INT32_MAX;
        for (int k = 0; k < kS64Threads / 4; ++k) {
            const double x = s_bv[k][tid];
            const int32_t xg = s_bg[k][tid];
            if (x < v || (x == v && xg < g)) {
                v = x;
                g = xg;
            }
        }
        best[list[u0 + tid]] = g;
    }
}

// Exact residual-form scan (Algorithm 2 for every g) of the universes in
// `list`, used when all certified screen rounds failed, so it never needs
// binary64 q-vectors.  Grid (universe, split): each CTA stages W of the
// universe's covariance in shared memory and scans every split-th grid point;
// k_scan_resid_reduce takes the first minimum over the splits.
template <bool MODEL>
__global__ void __launch_bounds__(256) k_scan_resid(const int32_t* __restrict__ list, const int32_t* __restrict__ uslot,
                                                     const float* __restrict__ d, GridSpec gs,
                                                     int64_t G, int nfit, const float2* __restrict__ Wdf,
                                                     double* __restrict__ part_v, int32_t* __restrict__ part_g) {
    extern __shared__ float2 sWd[];
    __shared__ double rv[8];
    __shared__ int32_t rg[8];
    const int i = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y;
    const int u = list[i];
    const float2* Wg = Wdf + (size_t)uslot[i] * nfit * nfit;
    const bool staged = (nfit <= kResolveMaxN);
    if (staged)
        for (int e = threadIdx.x; e < nfit * nfit; e += blockDim.x) sWd[e] = Wg[e];
    __syncthreads();
    const float2* W = staged ? sWd : Wg;
    const float* du = d + (size_t)u * nfit;
    double bv = DBL_MAX;
    int32_t bg = INT32_MAX;
    for (int64_t g = (int64_t)sp * blockDim.x + threadIdx.x; g < G; g += (int64_t)nsp * blockDim.x) {
        const double c = resid_df(W, nfit, srow<MODEL>(gs, nullptr, g), du);
        if (c < bv) {
            bv = c;
            bg = (int32_t)g;
        }
    }
    warp_argmin(bv, bg);
    if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = bv;
        rg[threadIdx.x >> 5] = bg;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        bv = threadIdx.x < (blockDim.x >> 5) ? rv[threadIdx.x] : DBL_MAX;
        bg = threadIdx.x < (blockDim.x >> 5) ? rg[threadIdx.x] : INT32_MAX;
        warp_argmin(bv, bg);
        if (threadIdx.x == 0) {
            part_v[(size_t)i * nsp + sp] = bv;
            part_g[(size_t)i * nsp + sp] = bg;
        }
    }
}

__global__ void k_scan_resid_reduce(const int32_t* __restrict__ list, int64_t n, int nsp,
                                    const double* __restrict__ part_v, const int32_t* __restrict__ part_g,
                                    int32_t* __restrict__ best) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double bv = DBL_MAX;
    int32_t bg = INT32_MAX;
    for (int sp = 0; sp < nsp; ++sp) {
        const double v = part_v[i * nsp + sp];
        const int32_t g = part_g[i * nsp + sp];
        if (v < bv || (v == bv && g < bg)) {
            bv = v;
            bg = g;
        }
    }
    best[list[i]] = bg;
}

// ------------------------------------------------------ mixed: grouping -----

// Universes of one job sit next to each other and mostly share a slot, so the
// lanes of a warp that hold the same slot add their count with one atomic.
__global__ void k_count_slots(const int32_t* __restrict__ uslot, int64_t n, int32_t* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const unsigned act = __ballot_sync(0xffffffffu, i < n);
    if (i >= n) return;
    const int s = uslot[i];
    const unsigned peers = __match_any_sync(act, s);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[s], __popc(peers));
}

// exclusive scan of ceil(cnt / 32) over slots (single CTA): each slot's first
// quadrant in base[s], the quadrant total in base[n_slots], the tile count
// (quadrants rounded up to whole tiles) in *n_tiles
__global__ void k_tile_scan(const int32_t* __restrict__ cnt, int n_slots, int slot_rows, int32_t* __restrict__ base,
                            int32_t* __restrict__ n_tiles) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int start = 0; start < n_slots; start += blockDim.x) {
        const int s = start + threadIdx.x;
        // quadrants of the slot: its rows in granules of slot_rows (32: a quadrant, 128: a tile)
        const int32_t v = (s < n_slots) ? (cnt[s] + slot_rows - 1) / slot_rows * (slot_rows / kQuadRows) : 0;
        int32_t x = v;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int32_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int32_t excl = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - v;
        if (s < n_slots) base[s] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        base[n_slots] = carry;
        *n_tiles = (carry + kQuads - 1) / kQuads;
    }
}

// quadrant -> slot; the quadrants that pad the last tile take the slot of the
// last used quadrant, so a tile whose used quadrants share a slot stays uniform
__global__ void k_tile_slots(const int32_t* __restrict__ cnt, const int32_t* __restrict__ base, int n_slots,
                             const int32_t* __restrict__ n_tiles, int32_t* __restrict__ quad_slot) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int nq = base[s + 1] - base[s];
    for (int q = 0; q < nq; ++q) quad_slot[base[s] + q] = s;
    // the slot that owns the last used quadrant also pads the last tile
    const int used = base[n_slots];
    if (nq > 0 && base[s] + nq == used)
        for (int q = used; q < *n_tiles * kQuads; ++q) quad_slot[q] = s;
}

__global__ void k_scatter_tiles(const int32_t* __restrict__ active, int64_t n, const int32_t* __restrict__ uslot,
                                const int32_t* __restrict__ base, int32_t* __restrict__ fill,
                                int32_t* __restrict__ tile_univ) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const unsigned act = __ballot_sync(0xffffffffu, i < n);
    if (i >= n) return;
    const int s = uslot[i];
    // one atomic per slot per warp; the lanes of a slot take consecutive positions
    const unsigned peers = __match_any_sync(act, s);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int first = 0;
    if (lane == leader) first = atomicAdd(&fill[s], __popc(peers));
    first = __shfl_sync(peers, first, leader);
    const int pos = first + __popc(peers & ((1u << lane) - 1u));
    // quadrant base[s] + pos / 32, row pos % 32 of it: rows are numbered quadrant * 32 + row
    tile_univ[(int64_t)(base[s] + pos / kQuadRows) * kQuadRows + pos % kQuadRows] = active[i];
}

// ---------------------------------------------------------- mixed: y prep ---

__device__ __forceinline__ int64_t ytile_offset(int64_t t, int r, int c, int K) {
    // A-operand image of one BM-row tile: [2K/8 chunks][BM/8 row groups][8 rows][8 cols] bf16
    return t * (int64_t)(2 * K * kBM) + (int64_t)(c >> 3) * (kBM * 8) + (r >> 3) * 64 + (r & 7) * 8 + (c & 7);
}

// One CTA per tile, one thread per row (its quadrant's covariance slot): y^ = A (d - v) in binary32, Y = -2 y^
// split into bf16 hi + lo, and the error-bound coefficient alpha in the spare
// column so that the screen directly yields a lower bound of chi2_g - c_u.
// It also evaluates the row's screen value at its own covariance point q
// (= cur[u]) with an upper bound UB_q: no grid point with LB >= UB_q can be the
// minimum, so tau0 = UB_q seeds the screen's top-k threshold.
// NR > 0: N_fit <= NR and the row's d - v lives in registers (every index a
// compile-time constant, the loops unrolled to NR with the columns past N_fit
// skipped); NR = 0: any N_fit, with d - v in a per-thread array.  Same
// operations in the same order either way.
template <int NR>
__global__ void __launch_bounds__(kBM) k_yprep(const int32_t* __restrict__ quad_slot,
                                                const int32_t* __restrict__ tile_univ, const float* __restrict__ d,
                                                const double* __restrict__ centre, int nfit, int K,
                                                const float* __restrict__ A32, const float* __restrict__ rho,
                                                const int32_t* __restrict__ cur, GridSpec gs,
                                                const float4* __restrict__ gnorm, const float* __restrict__ Qc,
                                                const float* __restrict__ Qb, int64_t G_pad,
                                                uint16_t* __restrict__ Yt, float4* __restrict__ alpha,
                                                float* __restrict__ tau0, int32_t* __restrict__ tile_j0,
                                                bool stage_all) {
    extern __shared__ float sA[];
    const int64_t t = blockIdx.x;
    const int r = threadIdx.x;
    const int slot = quad_slot[t * kQuads + r / kQuadRows];
    // each distinct covariance of the tile's quadrants is staged once (up to four where they fit;
    // otherwise the tile's first slot is staged and rows of other slots read theirs)
    int qs[kQuads], first[kQuads];  // first[k]: the first quadrant holding qs[k]
#pragma unroll
    for (int k = 0; k < kQuads; ++k) {
        qs[k] = quad_slot[t * kQuads + k];
        first[k] = k;
        for (int k2 = k - 1; k2 >= 0; --k2)
            if (qs[k2] == qs[k]) first[k] = k2;
    }
    const int nn = nfit * nfit;
    for (int k = 0; k < kQuads; ++k) {
        if (first[k] != k || (!stage_all && k > 0)) continue;
        for (int e = threadIdx.x; e < nn; e += blockDim.x) sA[k * nn + e] = A32[(size_t)qs[k] * nn + e];
    }
    __syncthreads();
    const int myq = r / kQuadRows;
    const float* Arow = (stage_all || qs[myq] == qs[0]) ? sA + first[myq] * nn : A32 + (size_t)slot * nn;
    const int u = tile_univ[t * kBM + r];
    // the screen walks this tile's grid tiles starting at the one holding row 0's q
    if (r == 0) tile_j0[t] = (u >= 0) ? cur[u] / kBN : 0;
    if (u < 0) {
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int c8 = 0; c8 < 2 * K / 8; ++c8) *reinterpret_cast<uint4*>(Yt + ytile_offset(t, r, c8 * 8, K)) = z;
        alpha[t * kBM + r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        tau0[t * kBM + r] = -FLT_MAX;  // padding rows keep no candidate
        return;
    }
    const int q = cur[u];
    float sql[kMaxBins];  // the probe row, when it is recomputed rather than stored
    const float* sq = gs.Sc32 ? gs.Sc32 + (int64_t)q * nfit : sql;
    if (!gs.Sc32) {
        const FitRow fr = fit_row(gs, q);
        for (int j = 0; j < nfit; ++j) sql[j] = row_sc32(gs, fr, j);
    }

    float dt[NR > 0 ? NR : kMaxBins];
    float dn2 = 0.0f;
    if (NR > 0) {
#pragma unroll
        for (int j = 0; j < (NR > 0 ? NR : 1); ++j) {
            dt[j] = 0.0f;
            if (j < nfit) {
                dt[j] = (float)((double)d[(size_t)u * nfit + j] - centre[j]);
                dn2 = fmaf(dt[j], dt[j], dn2);
            }
        }
    } else {
        for (int j = 0; j < nfit; ++j) {
            dt[j] = (float)((double)d[(size_t)u * nfit + j] - centre[j]);
            dn2 = fmaf(dt[j], dt[j], dn2);
        }
    }
    float yn2 = 0.0f, yl2 = 0.0f, yhl2 = 0.0f, ry2 = 0.0f, dot = 0.0f, adot = 0.0f;
    // the row's A-image entries in runs of 8 columns (one 16-byte core-matrix row per half)
    for (int c8 = 0; c8 < K / 8; ++c8) {
        uint32_t vh[4] = {0u, 0u, 0u, 0u}, vl[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
            const int i = c8 * 8 + ii;
            if (i < nfit) {
                float y = 0.0f;
                const float* Ai = Arow + i * nfit;
                if (NR > 0) {
#pragma unroll
                    for (int j = 0; j < (NR > 0 ? NR : 1); ++j)
                        if (j < nfit) y = fmaf(Ai[j], dt[j], y);
                } else {
                    for (int j = 0; j < nfit; ++j) y = fmaf(Ai[j], dt[j], y);
                }
                const float Y = -2.0f * y;
                yn2 = fmaf(Y, Y, yn2);
                dot = fmaf(Y, sq[i], dot);
                adot = fmaf(fabsf(Y), fabsf(sq[i]), adot);
                const __nv_bfloat16 h = __float2bfloat16_rn(Y);
                const float rem = Y - __bfloat162float(h);           // exact
                const __nv_bfloat16 l = __float2bfloat16_rn(rem);
                const float lo = __bfloat162float(l), hl = __bfloat162float(h) + lo;
                const float ry = rem - lo;                            // exact: r_Y = Y - hi - lo
                yl2 = fmaf(lo, lo, yl2);
                yhl2 = fmaf(hl, hl, yhl2);
                ry2 = fmaf(ry, ry, ry2);
                vh[ii >> 1] |= (uint32_t)__bfloat16_as_ushort(h) << (16 * (ii & 1));
                vl[ii >> 1] |= (uint32_t)__bfloat16_as_ushort(l) << (16 * (ii & 1));
            }
        }
        *reinterpret_cast<uint4*>(Yt + ytile_offset(t, r, c8 * 8, K)) = make_uint4(vh[0], vh[1], vh[2], vh[3]);
        *reinterpret_cast<uint4*>(Yt + ytile_offset(t, r, K + c8 * 8, K)) = make_uint4(vl[0], vl[1], vl[2], vl[3]);
    }
    // -2 y.s~_g - (hi*hi + lo*hi + hi*lo products)  =  -2 (y - y^).s~ + Y_lo.S_lo + (Y_hi + Y_lo).r_S + r_Y.s~
    // and the binary32 accumulation of the 3K products (each add bounded as truncated, Sum|products| <= 1.02 |Y||s~|):
    //   |error| <= [2 |y - y^| + |r_Y| + (3K+2) 1.02 2^-23 |Y|] |s~| + |Y_lo| |S_lo| + |Y_hi+Y_lo| |r_S|
    // with |y - y^| <= (nfit+2) 2^-24 rho |d~| (A and d~ rounded to binary32, binary32 dot products).
    const float dn = sqrtf(dn2) * 1.0001f, yn = sqrtf(yn2) * 1.0001f;
    const float a_acc = 1.02f * (2.0f * (float)(nfit + 2) * 5.9604645e-08f * rho[slot] * dn +
                                 (float)(3 * K + 2) * 1.1920929e-07f * 1.02f * yn + sqrtf(ry2));
    const float4 al = make_float4(a_acc, 1.0001f * sqrtf(yl2), 1.0001f * sqrtf(yhl2), 0.0f);
    alpha[t * kBM + r] = al;
    // the spare columns nfit .. nfit+2 of the hi half (written as zero above; same thread, program order)
    Yt[ytile_offset(t, r, nfit, K)] = __bfloat16_as_ushort(__float2bfloat16_rd(-al.x));
    Yt[ytile_offset(t, r, nfit + 1, K)] = __bfloat16_as_ushort(__float2bfloat16_rd(-al.y));
    Yt[ytile_offset(t, r, nfit + 2, K)] = __bfloat16_as_ushort(__float2bfloat16_rd(-al.z));
    // probe at q: sigma^ = q^_q + Y.s~_q (binary32), |sigma^ - sigma| <= 2|y - y^||s~_q| + |q^ - q|
    //   + (nfit+1) 2^-24 (sum |Y_i s~_i| + |q^|) + 2^-24 |sigma^|   (all inside eps below)
    const int64_t qi = (int64_t)slot * G_pad + q;
    const float qc = Qc[qi];
    const float sig = qc + dot;
    const float eps = bound_dot(al, gnorm[q]) + (qc - Qb[qi]) +
                      (float)(nfit + 2) * 5.9604645e-08f * (adot + fabsf(qc)) + 1.1920929e-07f * (fabsf(sig) + 1.0f);
    tau0[t * kBM + r] = (sig + 2.0f * eps) * 1.0000005f + 1.0e-6f + 4.7683716e-07f * fabsf(sig);
}

// ------------------------------------------------------- mixed: resolution --

constexpr int kItemCu = kMaxTopK;     // item codes beyond the candidates
constexpr int kItemP = kMaxTopK + 1;
constexpr int kItemMin = kMaxTopK + 2;
constexpr int kItemCodes = kMaxTopK + 3;

// Resolution of a top-k round, as five flat launches (launch_resolve): the
// residuals are the work, and a tile's rows need very different numbers of
// them, so they are evaluated from flat lists that keep every lane busy
// instead of inside the tile's CTA (where the lanes of rows with few residuals
// waited at barriers for the rows with many).
//  k_resolve_emit     per row: the screen certificate (decide_row); the
//                     residual items the row needs, appended in tile order;
//  k_resid_items      every item's double-float residual chi2 (W of the row's
//                     covariance slot; the residual vector in registers);
//  k_resolve_conclude per row: the same decision again, then the rescored
//                     minimum and its certificate; finish (dchi2) / advance /
//                     hand on, exactly as one kernel did before; rescored rows
//                     that finish with p != best list their chi2_p;
//  k_resid_items      those chi2_p;
//  k_resolve_tail     their dchi2.
// Decision per row (§2 steps 3-4 with the screen's certificate):
//  1. from the screen's lower bounds LB and upper bounds UB = LB + 2 eps of
//     its candidates, accept the first candidate when it is the only one that
//     can still be the minimum and its UB is below every outside bound tau;
//  2. otherwise the residual-form chi2 of every candidate that can still be
//     the minimum (and c_u = |W (d - v)|^2 when the certificate needs it):
//     the first minimum, certified against tau, else the universe is handed
//     to the next round;
//  3. universes whose minimum repeats their covariance index (or that used
//     their last scan) finish with dchi2 = chi2_p - chi2_min; the others
//     move their covariance index to the minimum.
struct RowDecision {
    int state;  // 0 padding, 1 certified by the bounds, 2 rescoring, 3 nothing below the seed
    bool full;
    float tau, min_ub;
    int ncodes;                      // residual items of the row, in emission order
    uint8_t code[kMaxTopK + 1];      // candidate j < topk, kItemCu, kItemP, kItemMin
    int32_t g[kMaxTopK];
    float lb[kMaxTopK];
};

__device__ __forceinline__ void decide_row(const ResolveArgs& a, int64_t row, int slot, int u, RowDecision& D) {
    const int topk = a.topk;
    D.state = 0;
    D.ncodes = 0;
    D.full = false;
    D.tau = FLT_MAX;
    D.min_ub = FLT_MAX;
    if (u < 0) return;
    const float4 al = a.alpha[row];
    float ub[kMaxTopK];
    int nvalid = 0;
    for (int j = 0; j < topk; ++j) {
        const int32_t gj = a.cidx[row * topk + j];
        D.g[j] = gj;
        D.lb[j] = a.cval[row * topk + j];
        ub[j] = FLT_MAX;
        if (gj < 0) continue;
        ++nvalid;
        const int64_t q = (int64_t)slot * a.G_pad + gj;
        const float eps = bound_dot(al, a.gnorm[gj]) + (a.Qc[q] - a.Qb[q]);
        ub[j] = D.lb[j] + 2.0f * eps + 4.7683716e-07f * (fabsf(D.lb[j]) + fabsf(a.Qc[q]) + 1.0f);
        D.min_ub = fminf(D.min_ub, ub[j]);
    }
    // every grid point outside the list has LB >= the k-th kept value; an empty slot holds the
    // seed tau0 = UB of the row's probe, so a list that is not full holds every point that can
    // be the minimum
    D.full = (nvalid == topk);
    D.tau = D.lb[topk - 1] - 4.7683716e-07f * (fabsf(D.lb[topk - 1]) + 1.0f);
    int nR = 0;
    for (int j = 0; j < topk; ++j)
        if (D.g[j] >= 0 && D.lb[j] <= D.min_ub) ++nR;
    if (nvalid == 0) {
        D.state = 3;  // nothing below the seed: only possible with non-finite data
    } else if (nR == 1 && ub[0] < D.tau) {
        D.state = 1;
        // a universe that finishes on this certificate needs chi2_p and chi2_min in residual form
        if (D.g[0] == a.cur[u] || a.nscan[u] + 1 >= a.maxit[u]) {
            if (a.pt[u] != D.g[0]) D.code[D.ncodes++] = (uint8_t)kItemP;
            D.code[D.ncodes++] = (uint8_t)kItemMin;
        }
    } else {
        D.state = 2;
        for (int j = 0; j < topk; ++j)
            if (D.g[j] >= 0 && D.lb[j] <= D.min_ub) D.code[D.ncodes++] = (uint8_t)j;
        if (D.full && !(D.min_ub < D.tau)) D.code[D.ncodes++] = (uint8_t)kItemCu;
    }
}

// exclusive prefix sum of v over a CTA of kBM threads; *total receives the sum
__device__ __forceinline__ int block_excl_scan(int v, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int before = 0, sum = 0;
    for (int w = 0; w < kBM / 32; ++w) {
        before += (w < warp) ? s_warp[w] : 0;
        sum += s_warp[w];
    }
    *total = sum;
    return before + x - v;
}

__global__ void __launch_bounds__(kBM) k_resolve_emit(ResolveArgs a) {
    __shared__ int s_warp[kBM / 32];
    __shared__ int s_base;
    const int64_t t = blockIdx.x;
    const int64_t row = t * kBM + threadIdx.x;
    const int slot = a.quad_slot[row / kQuadRows];
    const int u = a.tile_univ[row];
    RowDecision D;
    decide_row(a, row, slot, u, D);
    int total = 0;
    const int off = block_excl_scan(D.ncodes, s_warp, &total);
    if (threadIdx.x == 0) {
        s_base = total ? atomicAdd(&a.counts[0], total) : 0;
        // a warp is a quadrant (one covariance): its rows' items are one contiguous range
        int q0 = s_base;
        for (int w = 0; w < kQuads; ++w) {
            a.tile_items[t * kQuads + w] = make_int2(q0, s_warp[w]);
            q0 += s_warp[w];
        }
        if (total) atomicAdd(a.n_resid, (unsigned long long)total);
    }
    __syncthreads();
    const int base = s_base + off;
    a.item_base[row] = base;
    for (int k = 0; k < D.ncodes; ++k) {
        const int c = D.code[k];
        const int32_t g = (c < kMaxTopK) ? D.g[c] : (c == kItemCu ? -1 : (c == kItemP ? a.pt[u] : D.g[0]));
        a.items[base + k] = make_int2((int32_t)row, g);
    }
}

// Residual chi2 of one tile's items.  The items of each quadrant are a
// contiguous range (tile_items[4t + w]) and the tile's quadrants follow each
// other; a run of quadrants with one covariance slot shares one W, staged in
// shared memory (every lane reads the same element at once), and the lanes
// stride over the run's items with no barrier but the staging's.  A tile
// whose quadrants share one slot stages once.  Small CTAs (two warps) keep the
// last, partly filled round of a run cheap.
constexpr int kResidThreads = 64;

template <int NR>
__global__ void __launch_bounds__(kResidThreads, 6) k_resid_tiles(const ResolveArgs a, const int2* __restrict__ items,
                                                                 const int2* __restrict__ tile_items,
                                                                 double* __restrict__ res) {
    extern __shared__ float2 sWd[];
    const int n = a.nfit;
    const int64_t t = blockIdx.x;
    int w0 = 0;
    while (w0 < kQuads) {  // every bound below is the same for all lanes
        const int slot = a.quad_slot[t * kQuads + w0];
        int w1 = w0 + 1;
        while (w1 < kQuads && a.quad_slot[t * kQuads + w1] == slot) ++w1;
        const int64_t i0 = tile_items[t * kQuads + w0].x;
        const int2 last = tile_items[t * kQuads + w1 - 1];
        const int64_t i1 = (int64_t)last.x + last.y;
        w0 = w1;
        if (i1 <= i0) continue;
        const float2* Wg = a.Wdf + (size_t)slot * n * n;
        const float2* W = Wg;
        if constexpr (NR > 0) {  // staged where it fits (N_fit <= 64)
            __syncthreads();      // the previous run's reads of sWd are done
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) sWd[e] = Wg[e];
            __syncthreads();
            W = sWd;
        }
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int2 it = items[i];
            const int u = a.tile_univ[it.x];
            res[i] = resid_mixed<NR>(W, n, srow<false>(a.gs, a.centre_df, it.y), a.d + (size_t)u * n);
        }
    }
}

// N_fit > 64: W is not staged, so the items are scored flat, one thread per
// item, grid-stride over the device count.  A row's items follow each other and
// the rows of a tile quadrant share a slot, so a warp's lanes mostly read the
// same W element at once.
template <bool MODEL>
__global__ void __launch_bounds__(256) k_resid_flat(const ResolveArgs a, const int2* __restrict__ items,
                                                    const int32_t* __restrict__ count, double* __restrict__ res) {
    const int n = a.nfit;
    const int64_t total = *count;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 it = items[i];
        const int u = a.tile_univ[it.x];
        const float2* W = a.Wdf + (size_t)a.quad_slot[it.x / kQuadRows] * n * n;
        res[i] = resid_df(W, n, srow<MODEL>(a.gs, a.centre_df, it.y), a.d + (size_t)u * n);
    }
}

__global__ void __launch_bounds__(kBM) k_resolve_conclude(ResolveArgs a) {
    __shared__ int s_nnext, s_nfb, s_n2[kQuads], s_cnt[3];
    __shared__ int s_base_next, s_base_fb, s_base2;
    const int64_t t = blockIdx.x;
    const int r = threadIdx.x;
    const int64_t row = t * kBM + r;
    const int slot = a.quad_slot[row / kQuadRows];
    const int u = a.tile_univ[row];
    if (r == 0) {
        s_nnext = 0;
        s_nfb = 0;
        for (int w = 0; w < kQuads; ++w) s_n2[w] = 0;
        s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    }
    __syncthreads();
    RowDecision D;
    decide_row(a, row, slot, u, D);
    const int base = a.item_base[row];
    const int topk = a.topk;
    int state = D.state;
    int32_t g_best = -1;
    double chi2_min = 0.0, chi2_p = 0.0;
    bool have_min = false, have_p = false;
    if (state == 1) {
        g_best = D.g[0];
        for (int k = 0; k < D.ncodes; ++k) {
            if (D.code[k] == kItemMin) {
                chi2_min = a.res[base + k];
                have_min = true;
            } else if (D.code[k] == kItemP) {
                chi2_p = a.res[base + k];
                have_p = true;
            }
        }
        atomicAdd(&s_cnt[0], 1);
    } else if (state == 2) {
        double bchi = DBL_MAX, cu = 0.0;
        int32_t bg = INT32_MAX;
        for (int k = 0; k < D.ncodes; ++k) {
            const int c = D.code[k];
            const double v = a.res[base + k];
            if (c == kItemCu) {
                cu = v;
            } else if (v < bchi || (v == bchi && D.g[c] < bg)) {
                bchi = v;
                bg = D.g[c];
            }
        }
        bool ok = !D.full || (D.min_ub < D.tau);
        if (!ok) ok = (double)D.tau > (bchi - cu) + 1e-9 * (fabs(bchi) + fabs(cu));
        if (ok) {
            state = 1;
            g_best = bg;
            chi2_min = bchi;
            have_min = true;
            atomicAdd(&s_cnt[1], 1);
        } else {
            state = 3;
            atomicAdd(&s_cnt[2], 1);
            // every grid point that can still be the minimum has LB <= sigma* = chi2_min - c_u of the
            // best candidate found: a list screen seeded with sigma* (rounded up) lists all of them
            if (a.thr) {
                const double sig = (bchi - cu) + 1e-9 * (fabs(bchi) + fabs(cu));
                a.thr[u] = __double2float_ru(sig) + 4.7683716e-07f * (fabsf((float)sig) + 1.0f);
            }
        }
    } else if (state == 3) {
        atomicAdd(&s_cnt[2], 1);
        if (a.thr) a.thr[u] = FLT_MAX;
    }
    (void)topk;
    if (state == 1 && a.rmask)
        a.rmask[u] |= a.round_bit ? a.round_bit : (D.state == 2 ? kDecidedRescored : kDecidedCert);
    // finish converged / exhausted universes, advance the others
    bool finishing = false, tail = false;
    int32_t p = -1;
    if (state == 1) {
        a.best[u] = g_best;
        finishing = (g_best == a.cur[u]) || (a.nscan[u] + 1 >= a.maxit[u]);
        if (finishing) {
            p = a.pt[u];
            // a rescored row that finishes still needs chi2_p (the certified ones listed it already)
            tail = (p != g_best) && !have_p;
        } else {
            a.cur[u] = g_best;
            a.nscan[u] = (int8_t)(a.nscan[u] + 1);
        }
    }
    const bool to_next = (state == 1 && !finishing);
    const int my_next = to_next ? atomicAdd(&s_nnext, 1) : -1;
    const int my_fb = (state == 3) ? atomicAdd(&s_nfb, 1) : -1;
    // chi2_p items stay grouped by quadrant (one W per residual CTA)
    const int quad = r / kQuadRows;
    const int my_2 = tail ? atomicAdd(&s_n2[quad], 1) : -1;
    __syncthreads();
    if (r == 0) {
        s_base_next = s_nnext ? atomicAdd(a.n_next, s_nnext) : 0;
        s_base_fb = s_nfb ? atomicAdd(a.n_fb, s_nfb) : 0;
        const int n2 = s_n2[0] + s_n2[1] + s_n2[2] + s_n2[3];
        s_base2 = n2 ? atomicAdd(&a.counts[1], n2) : 0;
        int q0 = s_base2;
        for (int w = 0; w < kQuads; ++w) {
            a.tile_items2[t * kQuads + w] = make_int2(q0, s_n2[w]);
            q0 += s_n2[w];
        }
        if (n2) atomicAdd(a.n_resid, (unsigned long long)n2);
        if (s_cnt[0]) atomicAdd(&a.counters[0], (unsigned long long)s_cnt[0]);
        if (s_cnt[1]) atomicAdd(&a.counters[1], (unsigned long long)s_cnt[1]);
        if (s_cnt[2]) atomicAdd(&a.counters[2], (unsigned long long)s_cnt[2]);
    }
    __syncthreads();
    if (to_next) a.next[s_base_next + my_next] = u;
    if (state == 3) a.fb[s_base_fb + my_fb] = u;
    if (tail) {
        int pos = s_base2 + my_2;
        for (int w = 0; w < quad; ++w) pos += s_n2[w];
        a.items2[pos] = make_int2((int32_t)row, p);
        a.cmin2[pos] = chi2_min;
    } else if (finishing) {
        a.dchi2[u] = (p == g_best) ? 0.0 : chi2_p - chi2_min;
        if (a.chi2min) a.chi2min[u] = chi2_min;
        a.nscan[u] = (int8_t)(a.nscan[u] + 1);
        atomicSub(&a.job_left[a.job_of[u]], 1);
    }
}

__global__ void k_resolve_tail(ResolveArgs a) {
    const int64_t total = a.counts[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int u = a.tile_univ[a.items2[i].x];
        const double cmin = a.cmin2[i];
        a.dchi2[u] = a.res2[i] - cmin;
        if (a.chi2min) a.chi2min[u] = cmin;
        a.nscan[u] = (int8_t)(a.nscan[u] + 1);
        atomicSub(&a.job_left[a.job_of[u]], 1);
    }
}

// List rounds: every grid point whose screen lower bound is at or below the
// row's seed (an upper bound of the minimum) is listed, so the residual-form
// minimum over a complete list is the minimum of the scan.  A row's list is
// cut into chunks of kListChunk points, one per lane of a warp, so a long list
// spreads over many warps.  k_list_plan checks each listed row (rows[] holds
// the round's occupied tile rows) and reserves its chunks; rows whose list
// overflowed go to the exact scan (their counts size the next, exact-size list
// round).
__global__ void k_list_plan(ResolveArgs a, const int32_t* __restrict__ cand_count, const int32_t* __restrict__ rows,
                            int64_t n_rows, const int32_t* __restrict__ n_rows_dev, ListPlan lp) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= n_rows || w >= *n_rows_dev) return;
    const int64_t row = rows[w];
    const int u = a.tile_univ[row];
    const int n0 = cand_count[row * 2], n1 = cand_count[row * 2 + 1];
    bool complete;
    if (a.list_off) {
        const int2 want = a.list_n[u];
        complete = (n0 == want.x && n1 == want.y);
    } else {
        complete = (n0 >= 0 && n1 >= 0 && n0 <= kListCap && n1 <= kListCap);
    }
    lp.row_nc[w] = 0;
    if (complete && n0 + n1 > 0) {
        const int nc = (n0 + n1 + kListChunk - 1) / kListChunk;
        const int base = atomicAdd(lp.n_chunk, nc);
        if ((int64_t)base + nc <= lp.max_chunks) {
            lp.row_base[w] = base;
            lp.row_done[w] = 0;
            lp.row_nc[w] = nc;
            for (int k = 0; k < nc; ++k) lp.chunk[base + k] = make_int2((int32_t)w, k);
            return;
        }
        // no room (the host's bound makes this unreachable): void the reservation, take the exact scan
        for (int64_t k = base; k < lp.max_chunks && k < (int64_t)base + nc; ++k) lp.chunk[k] = make_int2(-1, 0);
    }
    if (a.lcount) a.lcount[u] = (n0 >= 0 && n1 >= 0) ? make_int2(n0, n1) : make_int2(-1, -1);
    a.fb[atomicAdd(a.n_fb, 1)] = u;
    atomicAdd(&a.counters[1], 1ull);
}

// One warp per chunk (grid-stride over the device count): lane l scores listed
// point k * kListChunk + l with the canonical residual, the warp takes the
// first minimum (lowest index among equal values) and publishes it.  The warp
// that completes a row's last chunk takes the first minimum over the row's
// chunks and finishes (dchi2) or advances the row.
template <bool MODEL>
__global__ void __launch_bounds__(256) k_list_chunks(ResolveArgs a, const int32_t* __restrict__ cand_count,
                                                     const int32_t* __restrict__ rows, ListPlan lp) {
    const int n = a.nfit;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ float2 s_r[8][kMaxBins], s_t[8][kMaxBins];
    const int64_t total = *lp.n_chunk < lp.max_chunks ? (int64_t)*lp.n_chunk : lp.max_chunks;
    const int64_t stride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; e < total; e += stride) {
        const int2 ck = lp.chunk[e];
        if (ck.x < 0) continue;
        const int w = ck.x;
        const int64_t row = rows[w];
        const int u = a.tile_univ[row];
        // W of the row's quadrant (double-float, read through L1: the warp's lanes read the same element)
        const float2* W = a.Wdf + (size_t)a.quad_slot[row / kQuadRows] * n * n;
        const int n0 = cand_count[row * 2], n1 = cand_count[row * 2 + 1];
        int64_t base0, base1;
        if (a.list_off) {
            base0 = a.list_off[u];
            base1 = base0 + a.list_n[u].x;
        } else {
            base0 = row * 2 * (int64_t)kListCap;
            base1 = base0 + kListCap;
        }
        const float* du = a.d + (size_t)u * n;
        double bv = DBL_MAX;
        int32_t bg = INT32_MAX;
        const int k = ck.y * kListChunk + lane;
        if (k < n0 + n1) {
            const int32_t g = a.cidx[(k < n0) ? base0 + k : base1 + (k - n0)];
            bv = resid_df(W, n, srow<MODEL>(a.gs, nullptr, g), du);
            bg = g;
        }
        warp_argmin(bv, bg);
        int last = 0;
        if (lane == 0) {
            const int pos = lp.row_base[w] + ck.y;
            lp.pv[pos] = bv;
            lp.pg[pos] = bg;
            __threadfence();
            last = (atomicAdd(&lp.row_done[w], 1) == lp.row_nc[w] - 1);
        }
        if (!__shfl_sync(0xffffffffu, last, 0)) continue;
        __threadfence();
        bv = DBL_MAX;
        bg = INT32_MAX;
        const int nc = lp.row_nc[w], rb = lp.row_base[w];
        for (int j = lane; j < nc; j += 32) {
            const double v = __ldcg(&lp.pv[rb + j]);
            const int32_t gg = __ldcg(&lp.pg[rb + j]);
            if (v < bv || (v == bv && gg < bg)) {
                bv = v;
                bg = gg;
            }
        }
        warp_argmin(bv, bg);
        if (lane == 0 && a.rmask) a.rmask[u] |= a.round_bit;
        if (lane == 0 && a.n_resid) atomicAdd(a.n_resid, (unsigned long long)(n0 + n1));
        const int32_t cur_u = a.cur[u];
        const bool finishing = (bg == cur_u) || (a.nscan[u] + 1 >= a.maxit[u]);
        if (finishing) {
            const int p = a.pt[u];
            double cp = 0.0;
            if (p != bg) {
                // chi2_p in residual form (row dot products over the lanes, the bits of resid_df)
                cp = resid_df_warp(W, n, srow<MODEL>(a.gs, nullptr, p), du, s_r[warp], s_t[warp], lane);
                if (lane == 0 && a.n_resid) atomicAdd(a.n_resid, 1ull);
            }
            if (lane == 0) {
                a.best[u] = bg;
                a.dchi2[u] = (p == bg) ? 0.0 : cp - bv;
                if (a.chi2min) a.chi2min[u] = bv;
                a.nscan[u] = (int8_t)(a.nscan[u] + 1);
                atomicSub(&a.job_left[a.job_of[u]], 1);
                atomicAdd(&a.counters[0], 1ull);
            }
        } else if (lane == 0) {
            a.best[u] = bg;
            a.cur[u] = bg;
            a.nscan[u] = (int8_t)(a.nscan[u] + 1);
            a.next[atomicAdd(a.n_next, 1)] = u;
            atomicAdd(&a.counters[0], 1ull);
        }
    }
}

__global__ void k_or_mask(const int32_t* __restrict__ list, int64_t n, uint8_t bit, uint8_t* __restrict__ rmask) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) rmask[list[i]] |= bit;
}

__global__ void k_min_tau(const int32_t* __restrict__ tile_univ, int64_t n_rows, const float* __restrict__ thr,
                          float* __restrict__ tau0) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    const int u = tile_univ[i];
    if (u >= 0) tau0[i] = fminf(tau0[i], thr[u]);
}

// ---------------------------------------------------------- finishing -------

// One warp per finishing universe: chi2_p and chi2_min in residual form under
// the last scan's covariance (A = W^T W), dchi2 = chi2_p - chi2_min.
template <bool MODEL>
__global__ void __launch_bounds__(128) k_finish(const int32_t* __restrict__ list, int64_t n,
                                                 const int32_t* __restrict__ uslot, const int32_t* __restrict__ best,
                                                 UniverseState us, const float* __restrict__ d, GridSpec gs,
                                                 int nfit, const double* __restrict__ W64,
                                                 const float2* __restrict__ Wdf, double* __restrict__ dchi2,
                                                 double* __restrict__ chi2min) {
    __shared__ double rp[4][kMaxBins], rm[4][kMaxBins], tt[4][kMaxBins];
    __shared__ float2 fr[4][kMaxBins], ft[4][kMaxBins];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = blockIdx.x * 4LL + w;
    if (i >= n) return;
    const int u = list[i];
    const int slot = uslot[i];
    const int p = us.pt[u];
    const int g = best[u];
    const float* du = d + (size_t)u * nfit;
    double cp = 0.0, cm = 0.0;
    if (Wdf) {
        // mixed path: the double-float residual of every other mixed-path kernel
        const float2* W = Wdf + (size_t)slot * nfit * nfit;
        cp = (p == g) ? 0.0 : resid_df_warp(W, nfit, srow<MODEL>(gs, nullptr, p), du, fr[w], ft[w], lane);
        cm = resid_df_warp(W, nfit, srow<MODEL>(gs, nullptr, g), du, fr[w], ft[w], lane);
    } else {
        // plain path: binary64, in the summation order of resid_chi2_warp
        const FitRow rowp = fit_row(gs, p), rowg = fit_row(gs, g);
        for (int j = lane; j < nfit; j += 32) {
            rp[w][j] = __dsub_rn(row_fit(gs, rowp, j), (double)du[j]);
            rm[w][j] = __dsub_rn(row_fit(gs, rowg, j), (double)du[j]);
        }
        __syncwarp();
        const double* W = W64 + (size_t)slot * nfit * nfit;
        cp = (p == g) ? 0.0 : resid_chi2_warp(W, nfit, rp[w], tt[w], lane);
        cm = resid_chi2_warp(W, nfit, rm[w], tt[w], lane);
    }
    if (lane == 0) {
        dchi2[u] = (p == g) ? 0.0 : cp - cm;
        if (chi2min) chi2min[u] = cm;
        atomicSub(&us.job_left[us.job_of[u]], 1);
    }
}

// exact-path bookkeeping: a universe finishes when its minimum repeats its
// covariance index or it used its last scan; the others move on
__global__ void k_advance(const int32_t* __restrict__ active, int64_t n, const int32_t* __restrict__ best,
                          UniverseState us, int32_t* __restrict__ next_active, int32_t* __restrict__ n_next,
                          int32_t* __restrict__ fin, int32_t* __restrict__ n_fin) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int u = active[i];
    const int done = us.nscan[u] + 1;
    us.nscan[u] = (int8_t)done;
    if (best[u] == us.cur[u] || done >= us.maxit[u]) {
        fin[atomicAdd(n_fin, 1)] = u;
    } else {
        us.cur[u] = best[u];
        next_active[atomicAdd(n_next, 1)] = u;
    }
}

// ---------------------------------------------------------- quantiles -------

// One CTA per row: counts[row] += #{u < n : x[row][u] < thr[row]} (the empirical
// distribution of the row's dchi2 at the data's value).
__global__ void k_count_below(const double* __restrict__ x, int n, const double* __restrict__ thr,
                              int64_t* __restrict__ counts) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const double t = thr[blockIdx.x];
    const double* xr = x + (size_t)blockIdx.x * n;
    int c = 0;
    for (int u = threadIdx.x; u < n; u += blockDim.x) c += (xr[u] < t) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] += s_cnt;
}


// One CTA per row: bitonic sort in shared memory, then numpy's "linear" rule.
__global__ void k_quantiles(const double* __restrict__ x, int n, int npow2, const double* __restrict__ probs,
                            int nq, double* __restrict__ out) {
    extern __shared__ double sx[];
    const int row = blockIdx.x;
    for (int i = threadIdx.x; i < npow2; i += blockDim.x) sx[i] = (i < n) ? x[(size_t)row * n + i] : DBL_MAX;
    __syncthreads();
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = ((i & k) == 0);
                    const double a = sx[i], b = sx[ixj];
                    if ((a > b) == up) {
                        sx[i] = b;
                        sx[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const double h = (double)(n - 1) * probs[q];
        int lo = (int)floor(h);
        if (lo < 0) lo = 0;
        if (lo > n - 1) lo = n - 1;
        const int hi = lo + 1 < n ? lo + 1 : n - 1;
        const double f = h - lo;
        out[(size_t)row * nq + q] = sx[lo] + f * (sx[hi] - sx[lo]);
    }
}

}  // namespace

// ---------------------------------------------------------- peak probes -----

namespace {

// Eight independent fma chains per thread, x <- x a + b with |a| < 1 (values
// stay normal): 16 flops per iteration, no memory traffic.
template <typename T>
__global__ void k_fma_peak(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += x[k];
    if (sum == (T)-1) out[blockIdx.x] = sum;  // never true; keeps the chains live
}

}  // namespace

// TFLOP/s of one fma probe: best of three timed launches after a warm-up.
template <typename T>
static double fma_peak_tflops(int n_sm, int iters, cudaStream_t st) {
    T* out = nullptr;
    if (cudaMalloc(&out, 4096 * sizeof(T)) != cudaSuccess) return 0.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const unsigned blocks = (unsigned)n_sm * 8;
    const int threads = 256;
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        k_fma_peak<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999999, (T)1e-3);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 16.0 * iters * (double)blocks * threads;
        if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return best;
}

bool measure_fma_peaks(int n_sm, double* fp64_tflops, double* fp32_tflops, cudaStream_t st) {
    count_launch(8);
    *fp64_tflops = fma_peak_tflops<double>(n_sm, 20000, st);
    *fp32_tflops = fma_peak_tflops<float>(n_sm, 400000, st);
    return cudaGetLastError() == cudaSuccess && *fp64_tflops > 0.0 && *fp32_tflops > 0.0;
}

// ------------------------------------------------------------- launchers ----

void launch_collapse(const double* S, int64_t G, int nf, const int32_t* coll, int nfit, double* out,
                     cudaStream_t st) {
    count_launch();
    k_collapse<<<blocks_for(G, 128), 128, 0, st>>>(S, G, nf, coll, nfit, out);
}

void launch_centre(const GridSpec& gs, int64_t G, double* centre, cudaStream_t st) {
    count_launch();
    k_centre<<<gs.nfit, kThreads, 0, st>>>(gs, G, centre);
}

void launch_centred(const GridSpec& gs, int64_t G, int64_t G_pad, int K, double* Sc, float* Sc32, float4* gnorm,
                    uint16_t* Bt, cudaStream_t st) {
    cudaMemsetAsync(Bt, 0, (size_t)G_pad * 2 * K * sizeof(uint16_t), st);
    count_launch();
    k_centred<<<blocks_for(G, 128), 128, 0, st>>>(gs, G, K, Sc, Sc32, gnorm, Bt);
}

void launch_chol_sys(const FullSrc& src, int nf, const double* F, const int64_t* ps, int P, int gauss, double* L64,
                     float* L32, float* s32, double*, int* status, cudaStream_t st) {
    if (P <= 0) return;
    count_launch();
    const size_t smem = nf <= kCholPackN ? (size_t)nf * (nf + 1) / 2 * sizeof(double) : 0;
    // the attribute belongs to the current device, so it is set at every launch (a cheap host call)
    cudaFuncSetAttribute(k_chol_sys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kCholPackN * (kCholPackN + 1) / 2 * (int)sizeof(double));
    k_chol_sys<<<P, 256, smem, st>>>(src, nf, F, ps, gauss, L64, L32, s32, status);
}

void launch_build_cov(const FullSrc& src, int nf, int nfit, const int32_t* coll, const double* F, const int32_t* q_list,
                      const int32_t* slot_list, int n, int cov_mode, double* A64, double* W64, float* A32,
                      float* rho, double* work, int* status, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    const size_t smem = nfit <= kResolveMaxN ? 2 * (size_t)nfit * nfit * sizeof(double) : 0;
    cudaFuncSetAttribute(k_build_cov, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * kResolveMaxN * kResolveMaxN * (int)sizeof(double));
    k_build_cov<<<n, 256, smem, st>>>(src, nf, nfit, coll, F, q_list, slot_list, cov_mode, A64, W64, A32, rho,
                                      work, status);
}

void launch_qvec64(const GridSpec& gs, int64_t G, int nfit, const double* W64, const int32_t* slots, int n,
                   int64_t ldq, double* Q64, cudaStream_t st) {
    // blockIdx.y is the slot within a launch: chunks of at most gridDim.y's limit
    for (int s0 = 0; s0 < n; s0 += 65535) {
        const int ns = n - s0 < 65535 ? n - s0 : 65535;
        dim3 grid(blocks_for(G, 128) < 64 ? blocks_for(G, 128) : 64, ns);
        count_launch();
        k_qvec64<<<grid, 128, 0, st>>>(gs, G, nfit, W64, slots + s0, ldq, Q64);
    }
}

void launch_qvec32(const GridSpec& gs, const float4* gnorm, int64_t G, int64_t G_pad, int nfit, const float* A32,
                   const float* rho, const int32_t* slots, int n, float* Qc, float* Qb, uint16_t* Qb3,
                   cudaStream_t st) {
    if (n <= 0) return;
    if (n > 65535) {
        // blockIdx.y is the slot within a launch: chunks of at most gridDim.y's limit
        for (int s0 = 0; s0 < n; s0 += 65535)
            launch_qvec32(gs, gnorm, G, G_pad, nfit, A32, rho, slots + s0, n - s0 < 65535 ? n - s0 : 65535, Qc, Qb,
                          Qb3, st);
        return;
    }
    // ~16 grid points per thread so each block's staging of A is amortised
    unsigned gx = blocks_for(G_pad, 128 * 16);
    if (gx > 128) gx = 128;
    dim3 grid(gx, n);
    count_launch();
    if (nfit <= 16)
        k_qvec32<16><<<grid, 128, 0, st>>>(gs, gnorm, G, G_pad, nfit, A32, rho, slots, Qc, Qb, Qb3);
    else if (nfit <= 32)
        k_qvec32<32><<<grid, 128, 0, st>>>(gs, gnorm, G, G_pad, nfit, A32, rho, slots, Qc, Qb, Qb3);
    else if (nfit <= 48)
        k_qvec32<48><<<grid, 128, 0, st>>>(gs, gnorm, G, G_pad, nfit, A32, rho, slots, Qc, Qb, Qb3);
    else if (nfit <= 64)
        k_qvec32<64><<<grid, 128, 0, st>>>(gs, gnorm, G, G_pad, nfit, A32, rho, slots, Qc, Qb, Qb3);
    else
        k_qvec32_generic<<<grid, 128, 0, st>>>(gs, gnorm, G, G_pad, nfit, A32, rho, slots, Qc, Qb, Qb3);
}

void launch_fake_data(const float* L32, const float* s32, int nf, const int32_t* coll, int nfit, const int64_t* ps,
                      int P, int U, uint64_t seed, int gauss, float* d, cudaStream_t st) {
    if (P <= 0 || U <= 0) return;
    // blockIdx.y is the point within a launch; more points than gridDim.y allows take several launches
    constexpr int kMaxGridY = 65535;
    for (int p0 = 0; p0 < P; p0 += kMaxGridY) {
        const int np = P - p0 < kMaxGridY ? P - p0 : kMaxGridY;
        dim3 grid((U + 127) / 128, np);
        count_launch();
        k_fake_data<<<grid, 128, 0, st>>>(L32 + (size_t)p0 * nf * nf, s32 + (size_t)p0 * nf, nf, coll, nfit, ps + p0,
                                           U, (uint32_t)seed, (uint32_t)(seed >> 32), gauss,
                                           d + (size_t)p0 * U * nfit);
    }
}

void launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t st) {
    if (n <= 0) return;
    unsigned b = blocks_for(n);
    if (b > 4096) b = 4096;
    count_launch();
    k_fill_i32<<<b, kThreads, 0, st>>>(p, n, v);
}

void launch_iota_i32(int32_t* p, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    unsigned b = blocks_for(n);
    if (b > 4096) b = 4096;
    count_launch();
    k_iota_i32<<<b, kThreads, 0, st>>>(p, n);
}

void launch_mark_used(const int32_t* active, int64_t n, const int32_t* cur, uint8_t* flag, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_mark_used<<<blocks_for(n), kThreads, 0, st>>>(active, n, cur, flag);
}

void launch_compact_flags(uint8_t* flag, int64_t G, int32_t* list, int32_t* count, cudaStream_t st) {
    count_launch();
    k_compact_flags<<<blocks_for(G), kThreads, 0, st>>>(flag, G, list, count);
}

void launch_lookup_slots(const int32_t* active, int64_t n, const int32_t* cur, const int32_t* slot_of,
                         int32_t* uslot, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_lookup_slots<<<blocks_for(n), kThreads, 0, st>>>(active, n, cur, slot_of, uslot);
}

void launch_set_slots(const int32_t* q, const int32_t* s, int n, int32_t* slot_of, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_set_slots<<<blocks_for(n), kThreads, 0, st>>>(q, s, n, slot_of);
}

void launch_scan64(const int32_t* list, int64_t n, const int32_t* uslot, const float* d, const GridSpec& gs,
                   int64_t G, int nfit, const double* A64, const double* Q64, int64_t ldq, int32_t* best,
                   cudaStream_t st) {
    if (n <= 0) return;
    const size_t smem = (size_t)nfit * (kS64U + kS64LdS) * sizeof(double);
    cudaFuncSetAttribute(k_scan64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    k_scan64<<<(unsigned)((n + kS64U - 1) / kS64U), kS64Threads, smem, st>>>(list, n, uslot, d, gs, G, nfit, A64,
                                                                            Q64, ldq, best);
}

void launch_scan_resid(const int32_t* list, int64_t n, const int32_t* uslot, const float* d, const GridSpec& gs,
                       int64_t G, int nfit, const float2* Wdf, double* part_v, int32_t* part_g, int nsp,
                       int32_t* best, cudaStream_t st) {
    if (n <= 0) return;
    const size_t smem = nfit <= kResolveMaxN ? (size_t)nfit * nfit * sizeof(float2) : 0;
    count_launch(2);
    const dim3 grid((unsigned)n, (unsigned)nsp);
    if (gs.Sdf)
        k_scan_resid<false><<<grid, 256, smem, st>>>(list, uslot, d, gs, G, nfit, Wdf, part_v, part_g);
    else
        k_scan_resid<true><<<grid, 256, smem, st>>>(list, uslot, d, gs, G, nfit, Wdf, part_v, part_g);
    k_scan_resid_reduce<<<blocks_for(n), kThreads, 0, st>>>(list, n, nsp, part_v, part_g, best);
}

void launch_group(const int32_t* active, int64_t n, const int32_t* uslot, int n_slots, int32_t* cnt,
                  int32_t* tile_base, int32_t* fill, int32_t* n_tiles_dev, int32_t* quad_slot, int32_t* tile_univ,
                  int64_t max_tiles, int slot_rows, cudaStream_t st) {
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n_slots, st);
    cudaMemsetAsync(fill, 0, sizeof(int32_t) * (size_t)n_slots, st);
    launch_fill_i32(tile_univ, max_tiles * kBM, -1, st);
    if (n > 0) {
        count_launch();
        k_count_slots<<<blocks_for(n), kThreads, 0, st>>>(uslot, n, cnt);
    }
    count_launch();
    k_tile_scan<<<1, 1024, 0, st>>>(cnt, n_slots, slot_rows, tile_base, n_tiles_dev);
    count_launch();
    k_tile_slots<<<blocks_for(n_slots), kThreads, 0, st>>>(cnt, tile_base, n_slots, n_tiles_dev, quad_slot);
    if (n > 0) {
        count_launch();
        k_scatter_tiles<<<blocks_for(n), kThreads, 0, st>>>(active, n, uslot, tile_base, fill, tile_univ);
    }
}

void launch_yprep(const int32_t* quad_slot, const int32_t* tile_univ, int64_t n_tiles, const float* d,
                  const double* centre, int nfit, int K, const float* A32, const float* rho, const int32_t* cur,
                  const GridSpec& gs, const float4* gnorm, const float* Qc, const float* Qb, int64_t G_pad,
                  uint16_t* Yt, float4* alpha, float* tau0, int32_t* tile_j0, cudaStream_t st) {
    if (n_tiles <= 0) return;
    // the A of every quadrant's slot up to N_fit = 64 (64 KB); beyond, the tile's first slot
    const bool stage_all = nfit <= kResolveMaxN;
    const size_t smem = (size_t)(stage_all ? kQuads : 1) * nfit * nfit * sizeof(float);
    auto kern = nfit <= 48 ? k_yprep<48> : k_yprep<0>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    kern<<<(unsigned)n_tiles, kBM, smem, st>>>(quad_slot, tile_univ, d, centre, nfit, K, A32, rho, cur, gs, gnorm, Qc,
                                               Qb, G_pad, Yt, alpha, tau0, tile_j0, stage_all);
}

void launch_or_mask(const int32_t* list, int64_t n, uint8_t bit, uint8_t* rmask, cudaStream_t st) {
    if (n <= 0 || !rmask) return;
    count_launch();
    k_or_mask<<<blocks_for(n), kThreads, 0, st>>>(list, n, bit, rmask);
}

void launch_min_tau(const int32_t* tile_univ, int64_t n_tiles, const float* thr, float* tau0, cudaStream_t st) {
    if (n_tiles <= 0) return;
    count_launch();
    k_min_tau<<<blocks_for(n_tiles * kBM), kThreads, 0, st>>>(tile_univ, n_tiles * kBM, thr, tau0);
}

// rows[] <- the indices t * BM + r of the tile rows that hold a universe (any order)
__global__ void k_list_rows(const int32_t* __restrict__ tile_univ, int64_t n, int32_t* __restrict__ rows,
                            int32_t* __restrict__ n_rows) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool have = e < n && tile_univ[e] >= 0;
    const unsigned m = __ballot_sync(0xffffffffu, have);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int first = 0;
    if (lane == leader) first = atomicAdd(n_rows, __popc(m));
    first = __shfl_sync(0xffffffffu, first, leader);
    if (have) rows[first + __popc(m & ((1u << lane) - 1u))] = (int32_t)e;
}

void launch_resolve_list(const ResolveArgs& a, const int32_t* cand_count, int64_t n_tiles, int64_t n_rows,
                         int32_t* rows, int32_t* n_rows_dev, const ListPlan& lp, cudaStream_t st) {
    if (n_tiles <= 0 || n_rows <= 0) return;
    cudaMemsetAsync(n_rows_dev, 0, 4, st);
    cudaMemsetAsync(lp.n_chunk, 0, 4, st);
    count_launch();
    k_list_rows<<<blocks_for(n_tiles * kBM), kThreads, 0, st>>>(a.tile_univ, n_tiles * kBM, rows, n_rows_dev);
    count_launch();
    k_list_plan<<<blocks_for(n_rows), kThreads, 0, st>>>(a, cand_count, rows, n_rows, n_rows_dev, lp);
    // eight warps a CTA, grid-stride over the chunks the plan reserved
    const int64_t want = (lp.max_chunks + 7) / 8, cap = (int64_t)a.n_sm * 8;
    count_launch();
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(want, cap));
    if (a.gs.Sdf)
        k_list_chunks<false><<<grid, 256, 0, st>>>(a, cand_count, rows, lp);
    else
        k_list_chunks<true><<<grid, 256, 0, st>>>(a, cand_count, rows, lp);
}

void launch_resolve(const ResolveArgs& a, int64_t n_tiles, cudaStream_t st) {
    if (n_tiles <= 0) return;
    cudaMemsetAsync(a.counts, 0, 2 * sizeof(int32_t), st);
    // the tail loops over its device-side count
    const unsigned g3 = (unsigned)std::min<int64_t>(n_tiles, (int64_t)a.n_sm * 8);
    const size_t smem = (a.nfit <= 64 ? (size_t)a.nfit * a.nfit : 0) * sizeof(float2);
    auto resid = [&](const int2* items, const int2* tile_items, const int32_t* count, int64_t max_items, double* res) {
        if (a.nfit > 64 || !a.gs.Sdf) {  // recomputed rows: the flat form for every N_fit
            const int64_t want = (max_items + 255) / 256, cap = (int64_t)a.n_sm * 4;
            const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(want, cap));
            if (a.gs.Sdf)
                k_resid_flat<false><<<grid, 256, 0, st>>>(a, items, count, res);
            else
                k_resid_flat<true><<<grid, 256, 0, st>>>(a, items, count, res);
            return;
        }
        auto run = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * (int)sizeof(float2));
            kern<<<(unsigned)n_tiles, kResidThreads, smem, st>>>(a, items, tile_items, res);
        };
        if (a.nfit <= 16)
            run(k_resid_tiles<16>);
        else if (a.nfit <= 32)
            run(k_resid_tiles<32>);
        else if (a.nfit <= 48)
            run(k_resid_tiles<48>);
        else
            run(k_resid_tiles<64>);
    };
    count_launch(5);
    k_resolve_emit<<<(unsigned)n_tiles, kBM, 0, st>>>(a);
    resid(a.items, a.tile_items, a.counts, n_tiles * kBM * (a.topk + 1), a.res);
    k_resolve_conclude<<<(unsigned)n_tiles, kBM, 0, st>>>(a);
    resid(a.items2, a.tile_items2, a.counts + 1, n_tiles * kBM, a.res2);
    k_resolve_tail<<<g3, 256, 0, st>>>(a);
}

void launch_finish(const int32_t* list, int64_t n, const int32_t* uslot, const int32_t* best, const UniverseState& us,
                   const float* d, const GridSpec& gs, int nfit, const double* W64, const float2* Wdf, double* dchi2,
                   double* chi2min, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    const unsigned grid = (unsigned)((n + 3) / 4);
    if (gs.Sdf || !Wdf)
        k_finish<false><<<grid, 128, 0, st>>>(list, n, uslot, best, us, d, gs, nfit, W64, Wdf, dchi2, chi2min);
    else
        k_finish<true><<<grid, 128, 0, st>>>(list, n, uslot, best, us, d, gs, nfit, W64, Wdf, dchi2, chi2min);
}

void launch_wdf(const double* W64, const int32_t* slots, int n, int nfit, float2* Wdf, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_wdf<<<n, 256, 0, st>>>(W64, slots, nfit, Wdf);
}

void launch_to_df(const double* x, int64_t n, float2* y, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_to_df<<<blocks_for(n), kThreads, 0, st>>>(x, n, y);
}

void launch_advance(const int32_t* active, int64_t n, const int32_t* best, const UniverseState& us,
                    int32_t* next_active, int32_t* n_next, int32_t* fin, int32_t* n_fin, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_advance<<<blocks_for(n), kThreads, 0, st>>>(active, n, best, us, next_active, n_next, fin, n_fin);
}

void launch_count_below(const double* x, int rows, int n, const double* thr, int64_t* counts, cudaStream_t st) {
    if (rows <= 0 || n <= 0) return;
    count_launch();
    k_count_below<<<rows, 256, 0, st>>>(x, n, thr, counts);
}

void launch_osc_sin(const SpecModel& m, int rows, const double* L, const double* E, double* sinT, cudaStream_t st) {
    const int64_t n = (int64_t)rows * m.nf;
    if (n <= 0) return;
    count_launch();
    k_osc_sin<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, rows, L, E, sinT);
}

void launch_osc_spectra(const SpecModel& m, int64_t G, double* S, int* bad, cudaStream_t st) {
    const int64_t n = G * m.nf;
    if (n <= 0) return;
    count_launch();
    k_osc_spectra<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, G, S, bad);
}

void launch_quantiles(double* x, int rows, int n, const double* probs, int nq, double* out, cudaStream_t st) {
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    const size_t smem = (size_t)p2 * sizeof(double);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_quantiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    k_quantiles<<<rows, 512, smem, st>>>(x, n, p2, probs, nq, out);
}

}  // namespace fcdev
