// fc_sampler.cuh -- device random numbers for the fake data (§2 step 2).
//
// The paper only says "fluctuation of s"; this library draws
//   d_i = Poisson(max(0, s_i + sum_{j<=i} L_ij z_j)),  L = chol(diag(s) F diag(s)),
// with z standard normal.  Every quantity is a binary32 value produced by
// correctly rounded IEEE operations written as explicit intrinsics (so nvcc
// cannot contract a multiply and an add), in a fixed order; the counts are
// therefore a pure function of (seed, point, universe, bin).
//
//   Philox4x32-10 ......... Salmon, Moraes, Dror, Shaw, SC'11
//   normals ............... Box-Muller on consecutive uniform pairs
//   Poisson, lam < 10 ..... inversion by sequential search
//   Poisson, lam >= 10 .... Hormann (1993) transformed rejection with squeeze
//   log-pmf ............... Loader (2000) deviance bd0 + Stirling remainder
//   log / exp / sin / cos . own range reductions + Taylor / atanh series
#pragma once
#include <cstdint>

namespace fcdev {

struct Philox4 {
    uint32_t x[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t m0 = 0xD2511F53u * c0, h0 = __umulhi(0xD2511F53u, c0);
        const uint32_t m1 = 0xCD9E8D57u * c2, h1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = h1 ^ c1 ^ k0;
        const uint32_t n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = m1;
        c2 = n2;
        c3 = m0;
    }
    Philox4 o;
    o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

// ((x >> 9) + 1/2) * 2^-23: exact, in [2^-24, 1 - 2^-24]
__device__ __forceinline__ float unit_uniform(uint32_t x) {
    return __fmul_rn(__fadd_rn(__uint2float_rn(x >> 9), 0.5f), 1.1920928955078125e-07f);
}

constexpr float kLn2Hi = 0.693145751953125f;       // 15 significant bits: n * kLn2Hi is exact
constexpr float kLn2Lo = 1.428606765330187e-06f;
constexpr float kSqrt2 = 1.41421353816986083984375f;

// natural log of a positive normal binary32
__device__ __forceinline__ float ln32(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > kSqrt2) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float p = __fmaf_rn(t2, 0.111111111111111111f, 0.142857142857142857f);
    p = __fmaf_rn(t2, p, 0.2f);
    p = __fmaf_rn(t2, p, 0.333333333333333333f);
    const float tt = __fadd_rn(t, t);
    const float lnm = __fmaf_rn(__fmul_rn(tt, t2), p, tt);
    const float fe = __int2float_rn(e);
    return __fmaf_rn(fe, kLn2Hi, __fmaf_rn(fe, kLn2Lo, lnm));
}

// e^x, |x| <= 87
__device__ __forceinline__ float exp32(float x) {
    const float kf = rintf(__fmul_rn(x, 1.44269502162933349609375f));
    float r = __fmaf_rn(-kf, kLn2Hi, x);
    r = __fmaf_rn(-kf, kLn2Lo, r);
    float p = __fmaf_rn(r, 2.48015873015873015873e-05f, 1.98412698412698412698e-04f);
    p = __fmaf_rn(r, p, 1.38888888888888888889e-03f);
    p = __fmaf_rn(r, p, 8.33333333333333333333e-03f);
    p = __fmaf_rn(r, p, 4.16666666666666666667e-02f);
    p = __fmaf_rn(r, p, 1.66666666666666666667e-01f);
    p = __fmaf_rn(r, p, 0.5f);
    p = __fmaf_rn(r, p, 1.0f);
    p = __fmaf_rn(r, p, 1.0f);
    const int n = (int)kf;
    return __fmul_rn(p, __uint_as_float((uint32_t)(n + 127) << 23));
}

// (sin, cos) of 2*pi*u, u in (0,1)
__device__ __forceinline__ void sincos_2pi(float u, float& s_out, float& c_out) {
    const float w = __fmul_rn(u, 4.0f);
    const float jf = rintf(w);
    const float f = __fsub_rn(w, jf);
    const float x = __fmul_rn(f, 1.57079637050628662109375f);
    const float x2 = __fmul_rn(x, x);
    float ps = __fmaf_rn(x2, 2.75573192239858906526e-06f, -1.98412698412698412698e-04f);
    ps = __fmaf_rn(x2, ps, 8.33333333333333333333e-03f);
    ps = __fmaf_rn(x2, ps, -1.66666666666666666667e-01f);
    const float s = __fmaf_rn(__fmul_rn(x2, x), ps, x);
    float pc = __fmaf_rn(x2, -2.75573192239858906526e-07f, 2.48015873015873015873e-05f);
    pc = __fmaf_rn(x2, pc, -1.38888888888888888889e-03f);
    pc = __fmaf_rn(x2, pc, 4.16666666666666666667e-02f);
    pc = __fmaf_rn(x2, pc, -0.5f);
    const float c = __fmaf_rn(x2, pc, 1.0f);
    switch (((int)jf) & 3) {
        case 0: c_out = c; s_out = s; break;
        case 1: c_out = -s; s_out = c; break;
        case 2: c_out = -c; s_out = -s; break;
        default: c_out = s; s_out = -c; break;
    }
}

constexpr uint32_t kTagNormal = 0u;
constexpr uint32_t kTagPoisson = 0x80000000u;

// Normals 4j..4j+3 of universe (p, u): Box-Muller on (w0,w1) and (w2,w3).
__device__ __forceinline__ void normal_block(uint32_t j, uint32_t u, uint32_t p, uint32_t k0, uint32_t k1,
                                             float z[4]) {
    const Philox4 r = philox4x32_10(j, u, p, kTagNormal, k0, k1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float ua = unit_uniform(r.x[2 * h]);
        const float ub = unit_uniform(r.x[2 * h + 1]);
        const float R = __fsqrt_rn(__fmul_rn(ln32(ua), -2.0f));
        float sn, cs;
        sincos_2pi(ub, sn, cs);
        z[2 * h] = __fmul_rn(R, cs);
        z[2 * h + 1] = __fmul_rn(R, sn);
    }
}

// A bin's private uniform stream: counter (block, u, p, kTagPoisson | bin).
struct UniformStream {
    uint32_t k0, k1, u, p, tag, blk;
    uint32_t buf[4];
    int pos;
    __device__ __forceinline__ void init(uint32_t key0, uint32_t key1, uint32_t uu, uint32_t pp, uint32_t bin) {
        k0 = key0; k1 = key1; u = uu; p = pp; tag = kTagPoisson | bin; blk = 0; pos = 4;
    }
    __device__ __forceinline__ float next() {
        if (pos == 4) {
            const Philox4 r = philox4x32_10(blk, u, p, tag, k0, k1);
            buf[0] = r.x[0]; buf[1] = r.x[1]; buf[2] = r.x[2]; buf[3] = r.x[3];
            blk += 1;
            pos = 0;
        }
        return unit_uniform(buf[pos++]);
    }
};

// ln k! for k <= 9 by summing logs
__device__ __forceinline__ float lnfact_small(float k) {
    float s = 0.0f;
    for (float j = 2.0f; j <= k; j = __fadd_rn(j, 1.0f)) s = __fadd_rn(s, ln32(j));
    return s;
}

// ln k! - (k ln k - k + ln(2 pi k)/2), k >= 10
__device__ __forceinline__ float stirling_rem(float k) {
    const float ik = __fdiv_rn(1.0f, k);
    const float ik2 = __fmul_rn(ik, ik);
    float p = __fmaf_rn(-ik2, 7.93650793650793650794e-04f, 2.77777777777777777778e-03f);
    p = __fmaf_rn(-ik2, p, 8.33333333333333333333e-02f);
    return __fmul_rn(ik, p);
}

// k ln(k/lam) + lam - k without cancellation near k = lam
__device__ __forceinline__ float deviance_bd0(float k, float lam) {
    const float diff = __fsub_rn(k, lam);
    const float sum = __fadd_rn(k, lam);
    if (fabsf(diff) < __fmul_rn(0.1f, sum)) {
        const float v = __fdiv_rn(diff, sum);
        float s = __fmul_rn(diff, v);
        float ej = __fmul_rn(__fadd_rn(k, k), v);
        const float v2 = __fmul_rn(v, v);
#pragma unroll
        for (int j = 1; j <= 6; ++j) {
            ej = __fmul_rn(ej, v2);
            s = __fadd_rn(s, __fdiv_rn(ej, (float)(2 * j + 1)));
        }
        return s;
    }
    const float t = __fmul_rn(k, ln32(__fdiv_rn(k, lam)));
    return __fsub_rn(__fadd_rn(t, lam), k);
}

__device__ __forceinline__ float log_pmf(float k, float lam, float loglam) {
    if (k < 10.0f) return __fsub_rn(__fsub_rn(__fmul_rn(k, loglam), lam), lnfact_small(k));
    const float t1 = deviance_bd0(k, lam);
    const float t2 = __fmul_rn(ln32(__fmul_rn(6.28318548202514648438f, k)), 0.5f);
    const float t3 = stirling_rem(k);
    return __fsub_rn(__fsub_rn(-t1, t2), t3);
}

__device__ __forceinline__ int32_t poisson(float lam, UniformStream& st) {
    if (!(lam > 0.0f)) return 0;
    if (lam < 10.0f) {
        float pk = exp32(-lam);
        float cdf = pk;
        int32_t k = 0;
        const float u = st.next();
        while (u > cdf && k < 64) {
            k += 1;
            pk = __fdiv_rn(__fmul_rn(pk, lam), __int2float_rn(k));
            cdf = __fadd_rn(cdf, pk);
        }
        return k;
    }
    const float slam = __fsqrt_rn(lam);
    const float loglam = ln32(lam);
    const float b = __fmaf_rn(2.53f, slam, 0.931f);
    const float a = __fmaf_rn(0.02483f, b, -0.059f);
    const float twoa = __fadd_rn(a, a);
    const float inv_alpha = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fsub_rn(b, 3.4f)));
    const float v_r = __fsub_rn(0.9277f, __fdiv_rn(3.6224f, __fsub_rn(b, 2.0f)));
    for (int it = 0; it < 64; ++it) {
        const float U = __fsub_rn(st.next(), 0.5f);
        const float V = st.next();
        const float us = __fsub_rn(0.5f, fabsf(U));
        float t = __fdiv_rn(twoa, us);
        t = __fadd_rn(t, b);
        t = __fmul_rn(t, U);
        t = __fadd_rn(t, lam);
        t = __fadd_rn(t, 0.43f);
        const float kf = floorf(t);
        if (us >= 0.07f && V <= v_r) return (int32_t)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        const float den = __fadd_rn(__fdiv_rn(a, __fmul_rn(us, us)), b);
        const float lhs = ln32(__fdiv_rn(__fmul_rn(V, inv_alpha), den));
        if (lhs <= log_pmf(kf, lam, loglam)) return (int32_t)kf;
    }
    return (int32_t)floorf(lam);
}

}  // namespace fcdev
