// fc_qvec.cu -- q_g = s~_g^T A s~_g for every grid point on the tensor cores.
//
// The screen (fc_screen.cu) needs, per inverse covariance A = M^-1, the
// vector q_g of Eq. 1 expanded around the centre v (s~_g = s_g - v).  With
// A = W^T W (W = L^-1, lower triangular, from the Cholesky factor of M),
//
//     q_g = || W s~_g ||^2 ,
//
// so q is the row-wise squared norm of the G x K x K product T = S~ W^T.  One
// CTA tile is 128 grid points; the tile's S~ rows (the screen's own B image,
// bf16 hi + lo) and the W image (bf16 hi + lo) meet on tcgen05 as
// hi*hi + lo*hi + hi*lo with binary32 accumulation in TMEM, and the epilogue
// squares and sums each row.  Every term left out is bounded from the
// realized norms of the split parts:
//
//     T - T^ = W_lo S_lo + r_W s~ + (W_hi + W_lo) r_S + accumulation error
//     ||T - T^||_2 <= E_g = |W_lo|_F |S_lo| + |r_W|_F |s~| + |W_hl|_F |r_S|
//                          + (3K+2) 1.02 2^-23 |W|_F |s~|
//
// so q_g lies in [(|T^| - E_g)^2, (|T^| + E_g)^2] with |T^| from the binary32
// sum of squares (relative error <= (K+2) 2^-24).  The stored pair is
// Qc = that sum and Qb = Qc - delta - q_rel_slack |Qc|, delta the larger
// distance to either end, so q >= Qb and q <= Qc + (Qc - Qb) as the screen
// and the probes require.
//
// Roles (192 threads, one CTA per SM, persistent over (slot, 128-point tile)
// items in slot-major order):
//   warp 0      bulk-async copies: the slot's W image when the slot changes,
//               then the S~ rows of each tile into a stage ring
//   warp 1      TMEM allocation; one lane issues tcgen05.mma
//   warps 2..5  epilogue, one TMEM lane quadrant each: tcgen05.ld of the row,
//               sum of squares, certified bound, Qc / Qb / Qb3 stores
// Waits are bounded as in the screen (kDevTimeout, abort flag, TMEM freed).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <float.h>

#include <cstdint>

#include "fc_internal.cuh"
#include "fc_tc.cuh"

namespace fcdev {
namespace {

using namespace tc;

constexpr int kQM = 128;                 // grid points per tile (TMEM lanes)
constexpr uint32_t kQSlab = kQM * 16u;   // one 8-column slab of a tile's S~ rows
constexpr int kQTmemCols = 512;          // two accumulators of up to 256 columns
constexpr uint32_t kQSmemMax = 232448u;

__device__ __forceinline__ int64_t wimg_offset(int i, int c, int K) {
    // [2K/8 slabs][K rows][8 cols] bf16, hi columns 0..K-1, lo columns K..2K-1
    return (int64_t)(c >> 3) * (K * 8) + (i >> 3) * 64 + (i & 7) * 8 + (c & 7);
}

// W image of a slot: W = W_hi + W_lo + r_W split of the binary64 factor, and
// the Frobenius norms (rounded up) of W, W_lo, r_W and W_hi + W_lo.
__global__ void __launch_bounds__(256) k_wimage(const double* __restrict__ W64, const int32_t* __restrict__ slots,
                                                int nfit, int K, uint16_t* __restrict__ Wimg,
                                                float4* __restrict__ wnorm) {
    const int slot = slots[blockIdx.x];
    const double* W = W64 + (size_t)slot * nfit * nfit;
    uint16_t* img = Wimg + (size_t)slot * 2 * K * K;
    double sw = 0.0, sl = 0.0, sr = 0.0, sh = 0.0;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, j = e % K;
        const double w = (i < nfit && j < nfit) ? W[i * nfit + j] : 0.0;
        const __nv_bfloat16 h = __double2bfloat16(w);
        const double rem = w - (double)__bfloat162float(h);
        const __nv_bfloat16 l = __double2bfloat16(rem);
        const double lo = (double)__bfloat162float(l);
        const double hl = (double)__bfloat162float(h) + lo;
        const double r = rem - lo;
        sw = fma(w, w, sw);
        sl = fma(lo, lo, sl);
        sr = fma(r, r, sr);
        sh = fma(hl, hl, sh);
        img[wimg_offset(i, j, K)] = __bfloat16_as_ushort(h);
        img[wimg_offset(i, K + j, K)] = __bfloat16_as_ushort(l);
    }
    __shared__ double red[4][8];
    for (int o = 16; o > 0; o >>= 1) {
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
        sl += __shfl_xor_sync(0xffffffffu, sl, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sh += __shfl_xor_sync(0xffffffffu, sh, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = sw;
        red[1][warp] = sl;
        red[2][warp] = sr;
        red[3][warp] = sh;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[k] += red[k][w];
        auto up = [](double x) { return __double2float_ru(__dsqrt_ru(x) * (1.0 + 1e-12)); };
        wnorm[slot] = make_float4(up(t[0]), up(t[1]), up(t[2]), up(t[3]));
    }
}

// A group of up to m = 256 / K slots shares each S~ tile: their W images sit
// side by side as one B operand of N = m K columns, so one MMA chain gives the
// T tiles of every slot in the group and the tile is read once per group.
// S~ rows stream through a ring of stages that hold either a whole tile (2K
// columns) or, when that does not fit beside the W images, one 16-column K
// slice of it (two hi slabs, two lo slabs).
struct QvecLayout {
    int K, m, stages, sliced;
    uint32_t w_bytes, s_bytes, off_s, off_bar, bytes;
};

constexpr int kQNumBars(int stages) { return 2 * stages + 2 + 2 + 2 + 1; }
constexpr int kQEpiWarps = 8;  // two per TMEM lane quadrant, splitting the group's slots

inline QvecLayout qvec_layout(int K, int m, int stages, int sliced) {
    QvecLayout l{};
    l.K = K;
    l.m = m;
    l.stages = stages;
    l.sliced = sliced;
    l.w_bytes = (uint32_t)m * 2u * K * K * 2u;
    l.s_bytes = sliced ? 4u * kQSlab : 2u * K * kQM * 2u;
    l.off_s = l.w_bytes;
    l.off_bar = l.off_s + stages * l.s_bytes;
    l.bytes = l.off_bar + kQNumBars(stages) * 8 + 16 + 1024;
    return l;
}

// Items are (group, 128-point tile) pairs.  Groups run in waves of gridDim.x;
// a full wave gives every CTA one group whose tiles it walks in order, so all
// CTAs read the same region of the S~ image at about the same time and it is
// fetched from DRAM about once per wave.  A partial wave splits its items
// evenly.  Every role walks the same sequence; f returns false to stop.
template <class F>
__device__ __forceinline__ void qvec_items(int64_t n_groups, int64_t n_tq, F&& f) {
    for (int64_t v0 = 0; v0 < n_groups; v0 += gridDim.x) {
        const int64_t wg = (n_groups - v0 < (int64_t)gridDim.x) ? n_groups - v0 : (int64_t)gridDim.x;
        const int64_t tot = wg * n_tq;
        const int64_t ch = (tot + gridDim.x - 1) / gridDim.x;
        const int64_t a = (int64_t)blockIdx.x * ch;
        const int64_t b = (a + ch < tot) ? a + ch : tot;
        for (int64_t it = a; it < b; ++it)
            if (!f(v0 + it / n_tq, it % n_tq)) return;
    }
}

__global__ void __launch_bounds__(64 + 32 * kQEpiWarps, 1)
    k_qvec_tc(const uint16_t* __restrict__ Bt, const uint16_t* __restrict__ Wimg, const float4* __restrict__ wnorm,
              const float4* __restrict__ gnorm, const int32_t* __restrict__ slots, int n_slots, int64_t G,
              int64_t G_pad, int nfit, float* __restrict__ Qc, float* __restrict__ Qb, uint16_t* __restrict__ Qb3,
              int* __restrict__ status, QvecLayout lay) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_addr(smem);
    const int K = lay.K, M = lay.m, STAGES = lay.stages;
    uint64_t* bars = (uint64_t*)(smem + lay.off_bar);
    uint32_t* tmem_holder = (uint32_t*)(smem + lay.off_bar + kQNumBars(STAGES) * 8);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
    auto bar = [&](int i) { return smem_addr(&bars[i]); };
    const int S_FULL = 0, S_EMPTY = STAGES, W_FULL = 2 * STAGES, W_EMPTY = 2 * STAGES + 1,
              T_FULL = 2 * STAGES + 2, T_EMPTY = 2 * STAGES + 4, DONE = 2 * STAGES + 6;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar(S_FULL + s), 1);
            mbar_init(bar(S_EMPTY + s), 1);
        }
        mbar_init(bar(W_FULL), 1);
        mbar_init(bar(W_EMPTY), 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(T_FULL + i), 1);
            mbar_init(bar(T_EMPTY + i), kQEpiWarps);
        }
        mbar_init(bar(DONE), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_holder)),
                     "r"(kQTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const int64_t n_tq = G_pad / kQM;
    const int64_t n_groups = (n_slots + M - 1) / M;
    auto group_size = [&](int64_t grp) {
        const int64_t r = n_slots - grp * M;
        return (int)(r < M ? r : M);
    };
    const uint32_t tile_elems = 2u * K * kBN;      // bf16 elements of one 256-row B-image tile
    const int NC = lay.sliced ? K / 16 : 1;        // stages per tile
    const uint32_t wslab = (uint32_t)M * K * 16u;  // one 8-column slab of the group's B operand

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        int s_par[16];
        for (int s = 0; s < STAGES; ++s) s_par[s] = -1;
        int w_par = -1, w_loads = 0, s = 0;
        int64_t cur = -1;
        uint32_t ph = 0;
        bool ok = true;
        qvec_items(n_groups, n_tq, [&](int64_t grp, int64_t t) {
            if (grp != cur) {
                if (w_loads > 0 && !mbar_wait(bar(W_EMPTY), (uint32_t)((w_loads - 1) & 1), abort_flag)) {
                    ok = false;
                    return false;
                }
                const int mg = group_size(grp);
                mbar_expect_tx(bar(W_FULL), (uint32_t)mg * 2u * K * K * 2u);
                // slab j of slot i of the group lands at slab j's row block i
                for (int i = 0; i < mg; ++i) {
                    const uint16_t* w = Wimg + (size_t)slots[grp * M + i] * 2 * K * K;
                    for (int j = 0; j < 2 * K / 8; ++j)
                        bulk_g2s(sbase + j * wslab + i * (K * 16u), w + (size_t)j * K * 8, K * 16u, bar(W_FULL));
                }
                w_par = w_loads & 1;
                ++w_loads;
                cur = grp;
            }
            // rows (t & 1) * 128 .. +127 of B-image tile t / 2: one 2 KB run per 8-column slab
            const uint16_t* src = Bt + (t >> 1) * (int64_t)tile_elems + (t & 1) * (kQM * 8);
            for (int c = 0; c < NC; ++c) {
                if (!mbar_wait(bar(S_EMPTY + s), ph ^ 1, abort_flag)) {
                    ok = false;
                    return false;
                }
                mbar_expect_tx(bar(S_FULL + s), lay.s_bytes);
                const uint32_t dst = sbase + lay.off_s + s * lay.s_bytes;
                if (lay.sliced) {
                    // hi slabs 2c, 2c+1 and lo slabs K/8 + 2c, K/8 + 2c + 1
                    for (int k = 0; k < 4; ++k) {
                        const int sl = (k < 2 ? 2 * c + k : K / 8 + 2 * c + k - 2);
                        bulk_g2s(dst + k * kQSlab, src + (int64_t)sl * (kBN * 8), kQSlab, bar(S_FULL + s));
                    }
                } else {
                    for (int sl = 0; sl < 2 * K / 8; ++sl)
                        bulk_g2s(dst + sl * kQSlab, src + (int64_t)sl * (kBN * 8), kQSlab, bar(S_FULL + s));
                }
                s_par[s] = (int)ph;
                if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
            return true;
        });
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, kDevTimeout);
            if (w_par >= 0) mbar_wait(bar(W_FULL), (uint32_t)w_par, nullptr);
            for (int s = 0; s < STAGES; ++s)
                if (s_par[s] >= 0) mbar_wait(bar(S_FULL + s), (uint32_t)s_par[s], nullptr);
        }
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------------------- MMA
        int w_uses = 0, s = 0, ab = 0;
        int64_t cur = -1;
        uint32_t ph = 0, aph = 0, idesc = 0;
        bool ok = true;
        qvec_items(n_groups, n_tq, [&](int64_t grp, int64_t) {
            if (grp != cur) {
                // the previous group's W images stay until every MMA issued so far has completed
                if (w_uses > 0) mma_commit(bar(W_EMPTY));
                if (!mbar_wait(bar(W_FULL), (uint32_t)(w_uses & 1), abort_flag)) {
                    ok = false;
                    return false;
                }
                ++w_uses;
                cur = grp;
                idesc = idesc_bf16(kQM, group_size(grp) * K);
            }
            if (!mbar_wait(bar(T_EMPTY + ab), aph ^ 1, abort_flag)) {
                ok = false;
                return false;
            }
            const uint32_t d = tmem_base + (uint32_t)(ab * 256);
            for (int c = 0; c < NC; ++c) {
                if (!mbar_wait(bar(S_FULL + s), ph, abort_flag)) {
                    ok = false;
                    return false;
                }
                tc_fence_after();
                const uint32_t a0 = sbase + lay.off_s + s * lay.s_bytes;
                const int k_lo = lay.sliced ? c : 0, k_hi = lay.sliced ? c + 1 : K / 16;
                // first K step's descriptors, advanced by adding the slab offset to the address field
                uint64_t a_hi = smem_desc(lay.sliced ? a0 : a0 + (2 * k_lo) * kQSlab, kQSlab, 128);
                uint64_t a_lo = smem_desc(lay.sliced ? a0 + 2 * kQSlab : a0 + (K / 8 + 2 * k_lo) * kQSlab, kQSlab, 128);
                uint64_t b_hi = smem_desc(sbase + (2 * k_lo) * wslab, wslab, 128);
                uint64_t b_lo = smem_desc(sbase + (K / 8 + 2 * k_lo) * wslab, wslab, 128);
                const uint64_t a_step = lay.sliced ? 0 : (2 * kQSlab) >> 4, b_step = (uint64_t)(2 * wslab) >> 4;
#pragma unroll 4
                for (int kk = k_lo; kk < k_hi; ++kk) {
                    mma_bf16(d, a_hi, b_hi, idesc, kk > 0 ? 1u : 0u);
                    mma_bf16(d, a_lo, b_hi, idesc, 1u);
                    mma_bf16(d, a_hi, b_lo, idesc, 1u);
                    a_hi += a_step;
                    a_lo += a_step;
                    b_hi += b_step;
                    b_lo += b_step;
                }
                mma_commit(bar(S_EMPTY + s));
                if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
            mma_commit(bar(T_FULL + ab));
            if (++ab == 2) { ab = 0; aph ^= 1u; }
            return true;
        });
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, kDevTimeout);
        }
        mma_commit(bar(DONE));
        mbar_wait(bar(DONE), 0, nullptr);
    } else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;  // slots half, half + 2, ... of each group
        const int row = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const float gam = (float)(K + 2) * 5.9604645e-08f;
        const float acc = (float)(3 * K + 2) * 1.02f * 1.1920929e-07f;
        const float slack = q_rel_slack(nfit);
        int ab = 0;
        uint32_t aph = 0;
        qvec_items(n_groups, n_tq, [&](int64_t grp, int64_t t) {
            const bool w_ok = mbar_wait(bar(T_FULL + ab), aph, abort_flag);
            if (!__all_sync(0xffffffffu, w_ok)) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicOr(status, kDevTimeout);
                }
                return false;
            }
            tc_fence_after();
            const uint32_t tb = tmem_base + lane_base + (uint32_t)(ab * 256);
            const int mg = group_size(grp);
            const int64_t g = t * kQM + row;
            const float4 gn = g < G ? gnorm[g] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int i = half; i < mg; i += 2) {
                // sum of squares of the slot's K columns in column order
                float q = 0.0f;
                for (int c0 = i * K; c0 < (i + 1) * K; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tb + c0, r);
                    tmem_wait(r);
#pragma unroll
                    for (int k = 0; k < 16; ++k) q = fmaf(__uint_as_float(r[k]), __uint_as_float(r[k]), q);
                }
                const int slot = slots[grp * M + i];
                float qc = 0.0f, qb = 3.0e38f;
                if (g < G) {
                    const float4 wn = wnorm[slot];
                    const float E =
                        1.0001f * fmaf(wn.y, gn.y, fmaf(wn.z, gn.x, fmaf(wn.w, gn.z, acc * wn.x * gn.x)));
                    const float tlo = __fsqrt_rd(__fmul_rd(q, __fsub_rd(1.0f, gam)));
                    const float thi = __fsqrt_ru(__fmul_ru(q, __fadd_ru(1.0f, gam)));
                    const float lo = fmaxf(0.0f, __fsub_rd(tlo, E));
                    const float hi = __fadd_ru(thi, E);
                    const float delta = fmaxf(__fsub_ru(q, __fmul_rd(lo, lo)), __fsub_ru(__fmul_ru(hi, hi), q));
                    qc = q;
                    qb = __fsub_rd(__fsub_rd(q, delta), slack * q);
                }
                const size_t o = (size_t)slot * G_pad + g;
                Qc[o] = qc;
                Qb[o] = qb;
                store_qb3(Qb3 + o * 8, qb);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(T_EMPTY + ab));
            if (++ab == 2) { ab = 0; aph ^= 1u; }
            return true;
        });
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kQTmemCols)
                     : "memory");
    }
}

}  // namespace

bool qvec_tc_supported(int K) { return K >= 16 && K <= kMaxScreenK && K % 16 == 0; }

void launch_wimage(const double* W64, const int32_t* slots, int n, int nfit, int K, uint16_t* Wimg, float4* wnorm,
                   cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_wimage<<<n, 256, 0, st>>>(W64, slots, nfit, K, Wimg, wnorm);
}

// Widest group whose W images leave room for at least two stages: whole-tile
// stages when two fit beside the images, else K slices.
static bool qvec_pick_layout(int K, int n, QvecLayout* out) {
    int m = 256 / K;
    if (m > n) m = n;
    for (; m >= 1; --m) {
        for (int sliced = 0; sliced < 2; ++sliced) {
            const QvecLayout one = qvec_layout(K, m, 1, sliced);
            if (one.bytes > kQSmemMax) continue;
            int stages = 1 + (int)((kQSmemMax - one.bytes) / (one.s_bytes + 16u));
            const int cap = sliced ? 8 : 4;
            stages = stages > cap ? cap : stages;
            if (stages < 2) continue;
            *out = qvec_layout(K, m, stages, sliced);
            return true;
        }
    }
    return false;
}

bool launch_qvec_tc(const uint16_t* Bt, const uint16_t* Wimg, const float4* wnorm, const float4* gnorm,
                    const int32_t* slots, int n, int64_t G, int64_t G_pad, int nfit, int K, float* Qc, float* Qb,
                    uint16_t* Qb3, int* status, int n_sm, cudaStream_t st) {
    if (n <= 0) return true;
    if (!qvec_tc_supported(K)) return false;
    QvecLayout lay{};
    if (!qvec_pick_layout(K, n, &lay)) return false;
    cudaFuncSetAttribute(k_qvec_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes);
    const int64_t groups = (n + lay.m - 1) / lay.m;
    const int64_t items = groups * (G_pad / kQM);
    const int grid = (int)(items < n_sm ? items : n_sm);
    count_launch();
    k_qvec_tc<<<grid, 64 + 32 * kQEpiWarps, lay.bytes, st>>>(Bt, Wimg, wnorm, gnorm, slots, n, G, G_pad, nfit, Qc,
                                                              Qb, Qb3, status, lay);
    return true;
}

}  // namespace fcdev
