// fc_screen.cu -- tensor-core chi2 screen (§2 steps 3-4 over the whole grid).
//
// For a tile of BM = 128 universes that share one inverse covariance A and a
// tile of BN = 256 grid points, the screen value
//
//     LB_{u,g} = qb_g + sum_k Y_{u,k} S_{g,k}
//              ~ (q_g - 2 y_u . s~_g) - alpha_u |s~_g| - beta_g   <=  chi2_g - c_u
//
// is a lower bound of chi2_g(d_u) minus a per-universe constant, where
// y_u = A (d_u - v), s~_g = s_g - v, q_g = s~_g^T A s~_g, c_u = (d_u - v)^T A (d_u - v)
// (Eq. 1 expanded around the centre v).  Y = -2 y and s~ are split into BF16
// hi + lo parts and multiplied as hi*hi + lo*hi + hi*lo on tcgen05 (kind::f16,
// FP32 accumulation in TMEM); one spare K column carries -alpha_u x |s~_g|,
// the error bound of that product.  A first K-step multiplies a constant
// operand [1, 1, 1, 0...] with [qb_hi, qb_mid, qb_lo, 0...] (q_g lowered by its
// rounding bound, split in three BF16) so the accumulator starts at qb_g and
// the epilogue reads finished lower bounds.  It keeps, per universe, the TOPK
// smallest (LB, g) pairs with the lowest index first among equal values --
// the strict "<" of Algorithm 1.  The U x G score matrix never leaves the SM.
//
// Roles (one CTA per SM, persistent over universe tiles):
//   warp 0      bulk-async (TMA) copies: Y tile, then S~ tile + qb rows per stage
//   warp 1      TMEM allocation; one lane issues tcgen05.mma and commits
//   warps 2..9  epilogue: two warps per TMEM lane quadrant, each owning half of
//               the BN columns; tcgen05.ld double-buffered in registers, running
//               top-k, the two halves merged through shared memory per tile row
// Every mbarrier wait is bounded (about 2 s of %globaltimer); on timeout the
// kernel records kDevTimeout, waits for its own copies and MMAs, frees TMEM
// and returns.
#include <cuda_runtime.h>
#include <float.h>

#include <cstdint>

#include "fc_internal.cuh"
#include "fc_spec.cuh"
#include "fc_tc.cuh"

namespace fcdev {
namespace {

using namespace tc;

// kind::f16 instruction descriptor of the screen: D f32, A/B bf16, both K-major, M = BM, N = BN
constexpr uint32_t kIdesc = idesc_bf16(kBM, kBN);

// Minimum of 32 accumulator values as a depth-4 tree of three-input minima
// (min.f32 with three sources, sm_100+).  A minimum is exact, so the result
// does not depend on the order; the tree keeps the dependency chain short and
// needs 17 instructions instead of 31.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float min32(const uint32_t (&r)[32]) {
    float m[11];
#pragma unroll
    for (int i = 0; i < 10; ++i)
        m[i] = fmin3(__uint_as_float(r[3 * i]), __uint_as_float(r[3 * i + 1]), __uint_as_float(r[3 * i + 2]));
    m[10] = fminf(__uint_as_float(r[30]), __uint_as_float(r[31]));
    const float a = fmin3(m[0], m[1], m[2]), b = fmin3(m[3], m[4], m[5]), c = fmin3(m[6], m[7], m[8]);
    return fmin3(a, b, fminf(c, fminf(m[9], m[10])));
}

// (value, index) insertion into a list sorted in lexicographic order, the
// last entry dropping out.  Every position compares with the new pair at once
// (the outcomes are monotone in t because the list is sorted), then each entry
// takes its left neighbour, the new pair or itself: a few dependent steps
// instead of a chain through all TOPK positions, for an epilogue that waits on
// latency, not on issue slots.
template <int TOPK>
__device__ __forceinline__ void topk_insert(float (&vals)[TOPK], int32_t (&idx)[TOPK], float x, int32_t g) {
    bool c[TOPK];
#pragma unroll
    for (int t = 0; t < TOPK; ++t) c[t] = x < vals[t] || (x == vals[t] && g < idx[t]);
#pragma unroll
    for (int t = TOPK - 1; t >= 1; --t) {
        vals[t] = c[t - 1] ? vals[t - 1] : (c[t] ? x : vals[t]);
        idx[t] = c[t - 1] ? idx[t - 1] : (c[t] ? g : idx[t]);
    }
    vals[0] = c[0] ? x : vals[0];
    idx[0] = c[0] ? g : idx[0];
}

// Bit i set when value i of the chunk is at or below tau: four independent
// 8-bit groups, combined at the end (a short dependency chain).
__device__ __forceinline__ uint32_t below_mask(const uint32_t (&r)[32], float tau) {
    uint32_t q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        q[k] = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) q[k] |= (__uint_as_float(r[8 * k + i]) <= tau ? 1u : 0u) << i;
    }
    return (q[0] | (q[1] << 8)) | ((q[2] << 16) | (q[3] << 24));
}

// 32 lower bounds of one row (columns g0..g0+31): running top-k.  Fast path:
// a min over the 32 values and one compare.  If exactly one value is at or
// below the current k-th one it is that minimum and is inserted directly;
// with several, they are parked in this warp's shared scratch ([i][lane]) and
// inserted in a rolled loop (small code for the instruction cache).
template <int TOPK>
__device__ __forceinline__ void topk_chunk(float (&vals)[TOPK], int32_t (&idx)[TOPK], const uint32_t (&r)[32],
                                           float m, int64_t g0, int64_t G, float* scratch, int lane) {
    if (m <= vals[TOPK - 1]) {
        const float tau = vals[TOPK - 1];
        uint32_t mask = below_mask(r, tau);
        const int64_t lim = G - g0;
        if (lim < 32) mask &= (lim <= 0) ? 0u : ((1u << lim) - 1u);
        if (__popc(mask) == 1) {
            topk_insert<TOPK>(vals, idx, m, (int32_t)(g0 + __ffs(mask) - 1));
        } else if (mask) {
#pragma unroll
            for (int i = 0; i < 32; ++i) scratch[i * 32 + lane] = __uint_as_float(r[i]);
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                topk_insert<TOPK>(vals, idx, scratch[i * 32 + lane], (int32_t)(g0 + i));
            }
        }
    }
}

// Screen modes: kModeMin (first pass) uses only the hi*hi products and keeps
// each row's minimum index, which k_min_seed then turns into a certified upper
// bound that tightens the row's seed tau0 in place; kModeTopK keeps the full top-k; kModeList lists
// every grid point whose lower bound is at or below the seed (kListCap per
// half row, the count says whether the list overflowed).
struct ProbeArgs {
    const float* Qc;
    const float* Qb;
    const float4* gnorm;
    const float4* alpha;
    GridSpec gs;  // the probe rows s~_g (binary32)
    int nfit;
};

constexpr int kModeTopK = 0;
constexpr int kModeMin = 1;
constexpr int kModeList = 2;

// List mode: append every value at or below the seed (and its grid index).
__device__ __forceinline__ void list_chunk(int32_t& n, int32_t cap, float* __restrict__ lval, int32_t* __restrict__ lidx,
                                           float seed, const uint32_t (&r)[32], float m, int64_t g0, int64_t G) {
    if (m <= seed) {
        uint32_t mask = below_mask(r, seed);
        const int64_t lim = G - g0;
        if (lim < 32) mask &= (lim <= 0) ? 0u : ((1u << lim) - 1u);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            if (n < cap) {
                lidx[n] = (int32_t)(g0 + i);
                lval[n] = m;  // a lower bound of the entry (the chunk minimum); only the index is used
            }
            ++n;
        }
    }
}

// First pass: running minimum of a row.  The index is recovered only when the
// chunk improves the minimum (rare after the first tiles).
__device__ __forceinline__ void min_chunk(float& bv, int32_t& bi, const uint32_t (&r)[32], float m, int64_t g0,
                                          int64_t G) {
    if (m < bv) {
        int ii = 31;
#pragma unroll
        for (int i = 31; i >= 0; --i) ii = (__uint_as_float(r[i]) == m) ? i : ii;
        if (g0 + ii < G) {
            bv = m;
            bi = (int32_t)(g0 + ii);
        }
    }
}

__device__ __forceinline__ int64_t ytile_elem(int64_t t, int r, int c, int K) {
    return t * (int64_t)(2 * K * kBM) + (int64_t)(c >> 3) * (kBM * 8) + (r >> 3) * 64 + (r & 7) * 8 + (c & 7);
}

// Certified upper bound of sigma_g = chi2_g - c_u for one row at grid point g:
// sigma^ = q^_g + Y.s~_g in binary32 with Y = hi + lo from the row's A image
// (|Y_hl - Y| <= 2^-16 |Y|, inside alpha), plus every error term of the screen.
__device__ float probe_upper_bound(const uint16_t* __restrict__ Yt, int64_t item, int row, int slot, int32_t g,
                                   int64_t G_pad, const ProbeArgs& pa) {
    const int n = pa.nfit;
    const int K = screen_k(n);
    const FitRow fr = fit_row(pa.gs, g);
    float dot = 0.0f, adot = 0.0f;
    for (int i = 0; i < n; ++i) {
        const float h = __uint_as_float((uint32_t)Yt[ytile_elem(item, row, i, K)] << 16);
        const float l = __uint_as_float((uint32_t)Yt[ytile_elem(item, row, K + i, K)] << 16);
        const float y = h + l;
        const float sgi = row_sc32(pa.gs, fr, i);
        dot = fmaf(y, sgi, dot);
        adot = fmaf(fabsf(y), fabsf(sgi), adot);
    }
    const int64_t qi = (int64_t)slot * G_pad + g;
    const float qc = pa.Qc[qi];
    const float sig = qc + dot;
    const float eps = bound_dot(pa.alpha[item * kBM + row], pa.gnorm[g]) + (qc - pa.Qb[qi]) +
                      (float)(n + 2) * 5.9604645e-08f * (adot + fabsf(qc)) + 1.1920929e-07f * (fabsf(sig) + 1.0f);
    return (sig + 2.0f * eps) * 1.0000005f + 1.0e-6f + 4.7683716e-07f * fabsf(sig);
}

// After a min-only pass: tau0 <- min(tau0, certified upper bound at the row's
// minimum index bidx), one thread per row (bidx = INT32_MAX: no minimum).
__global__ void k_min_seed(const uint16_t* __restrict__ Yt, const int32_t* __restrict__ quad_slot,
                           const int32_t* __restrict__ bidx, float* __restrict__ tau0, int64_t n_rows, int64_t G,
                           int64_t G_pad, ProbeArgs pa, const int* __restrict__ status) {
    const int64_t orow = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (orow >= n_rows) return;
    // an aborted min pass leaves rows it never reached unwritten: use nothing of it
    if (*status & kDevTimeout) return;
    const int32_t bi = bidx[orow];
    const float seed = tau0[orow];
    if (bi < 0 || bi >= G || !(seed > -FLT_MAX)) return;
    const int64_t item = orow / kBM;
    const int row = (int)(orow % kBM);
    tau0[orow] = fminf(seed, probe_upper_bound(Yt, item, row, quad_slot[orow / kQuadRows], bi, G_pad, pa));
}

constexpr int kTmemCols = 2 * kBN;  // two accumulator buffers
constexpr int kEpiWarps = 8;
constexpr int kHalfCols = kBN / 2;
constexpr uint32_t kAChunk = kBM * 16u;  // one 8-column slab of the A image
constexpr uint32_t kBChunk = kBN * 16u;  // one 8-column slab of the B image
constexpr uint32_t kQBytes = kBN * 16u;  // one 8-column slab of q-step rows
constexpr uint32_t kSmemMax = 232448u;   // dynamic shared memory per CTA
constexpr uint32_t kSmemAlign = 128u;     // alignment of the plan's base (16 bytes would do for every operand)

// Shared-memory plan of one screen launch.  A pipeline stage holds either a
// whole B tile (2K columns x BN rows, for K <= 64) or, with kchunk, one
// 16-column K slice of it (two hi slabs, two lo slabs) so that large K still
// gets a deep pipeline; the stage's q-step slab follows its B part.  A tile
// whose quadrants hold different covariances takes one more stage per grid
// tile: the four slots' q-step slabs, in the B part.
struct ScreenLayout {
    int K, stages, ybuf, kchunk;
    uint32_t y_bytes;       // one A-image tile: 2K columns x BM rows, bf16
    uint32_t bpart_bytes;   // B part of a stage
    uint32_t stage_bytes;   // B part + q slab
    uint32_t off_b, off_ones, off_zero, off_sel, off_scratch, off_bar, bytes;
};

constexpr int kNumBars(int stages) { return 2 + 2 + stages + stages + 2 + 2 + 1; }

inline ScreenLayout screen_layout(int K, int stages, int ybuf, int kchunk) {
    ScreenLayout l{};
    l.K = K;
    l.stages = stages;
    l.ybuf = ybuf;
    l.kchunk = kchunk;
    l.y_bytes = 2u * K * kBM * 2u;
    l.bpart_bytes = kchunk ? 4u * kBChunk : 2u * K * kBN * 2u;
    l.stage_bytes = l.bpart_bytes + kQBytes;
    l.off_b = ybuf * l.y_bytes;
    l.off_ones = l.off_b + stages * l.stage_bytes;  // A slab of the q-step: [1,1,1,0..] per row
    l.off_zero = l.off_ones + kAChunk;               // second slab of the q-step, all zero
    // selector slabs of a mixed tile's q-step, one per quadrant: [1,1,1,0..] in that quadrant's rows
    l.off_sel = l.off_zero + kBChunk;
    // per epilogue warp 4 KB: slow-path scratch inside a tile, top-k hand-over at the end of a row tile
    l.off_scratch = l.off_sel + kQuads * kAChunk;
    l.off_bar = l.off_scratch + kEpiWarps * 4096;
    // after the barriers: TMEM address, abort flag, pair flags [4][2]; then the alignment slack
    l.bytes = l.off_bar + kNumBars(stages) * 8 + 48 + kSmemAlign;
    return l;
}

template <int TOPK, int MODE, bool KCHUNK>
__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1)
    k_screen(const uint16_t* __restrict__ Yt, const uint16_t* __restrict__ Bt, const uint16_t* __restrict__ Qb3,
             const int32_t* __restrict__ quad_slot, float* __restrict__ tau0, const int32_t* __restrict__ tile_j0,
             int64_t n_tiles, int64_t G, int64_t G_pad, float* __restrict__ cand_val, int32_t* __restrict__ cand_idx,
             int32_t* __restrict__ cand_count, int* __restrict__ status, ProbeArgs pa, ScreenLayout lay,
             ListArgs la, WaitTest wt) {
    static_assert(2 * TOPK * 32 * 4 <= 4096, "top-k hand-over exceeds the warp scratch");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + (kSmemAlign - 1)) & ~(uintptr_t)(kSmemAlign - 1));
    const uint32_t sbase = smem_addr(smem);
    const int K = lay.K, STAGES = lay.stages, YBUF = lay.ybuf;
    uint64_t* bars = (uint64_t*)(smem + lay.off_bar);
    uint32_t* tmem_holder = (uint32_t*)(smem + lay.off_bar + kNumBars(STAGES) * 8);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
    // per TMEM lane quadrant, whether each epilogue half finished the current item
    volatile int* pair_ok = (volatile int*)(tmem_holder + 2);
    auto bar = [&](int i) { return smem_addr(&bars[i]); };
    const int Y_FULL = 0, Y_EMPTY = 2, B_FULL = 4, B_EMPTY = 4 + STAGES, T_FULL = 4 + 2 * STAGES,
              T_EMPTY = 6 + 2 * STAGES, DONE = 8 + 2 * STAGES;
    // pipeline steps per grid tile: one whole tile, or K/16 slices
    const int NC = KCHUNK ? K / 16 : 1;
    // min mode multiplies only the hi halves, so only they are copied
    constexpr bool kLo = (MODE != kModeMin);
    const uint32_t tile_elems = 2u * K * kBN;  // bf16 elements of one B tile

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // constant q-step operand slabs (generic-proxy writes, fenced for the tensor core below)
    {
        uint32_t* ones = (uint32_t*)(smem + lay.off_ones);
        for (int i = threadIdx.x; i < (int)(kAChunk / 4); i += blockDim.x) {
            const int w = i & 3;  // 4 words per 16-byte row: bf16 pairs (1,1), (1,0), (0,0), (0,0)
            ones[i] = (w == 0) ? 0x3F803F80u : (w == 1 ? 0x00003F80u : 0u);
        }
        uint32_t* zero = (uint32_t*)(smem + lay.off_zero);
        for (int i = threadIdx.x; i < (int)(kBChunk / 4); i += blockDim.x) zero[i] = 0u;
        // selector slab k: the ones row of the q-step in the rows of quadrant k (16 bytes per row)
        uint32_t* sel = (uint32_t*)(smem + lay.off_sel);
        for (int i = threadIdx.x; i < (int)(kQuads * kAChunk / 4); i += blockDim.x) {
            const int k = i / (int)(kAChunk / 4), row = (i % (int)(kAChunk / 4)) >> 2, w = i & 3;
            const bool on = (row / kQuadRows) == k;
            sel[i] = !on ? 0u : ((w == 0) ? 0x3F803F80u : (w == 1 ? 0x00003F80u : 0u));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(Y_FULL + i), 1);
            mbar_init(bar(Y_EMPTY + i), 1);
            mbar_init(bar(T_FULL + i), 1);
            mbar_init(bar(T_EMPTY + i), kEpiWarps);
        }
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar(B_FULL + s), 1);
            mbar_init(bar(B_EMPTY + s), 1);
        }
        mbar_init(bar(DONE), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_holder)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const int n_gt = (int)(G_pad / kBN);
    // limit of the pipeline waits (the drain and completion waits keep the built-in limit)
    const uint64_t wlim = wt.wait_ns ? wt.wait_ns : kWaitNs;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        int y_par[2] = {-1, -1};
        int b_par[16];
        for (int s = 0; s < STAGES; ++s) b_par[s] = -1;
        bool ok = true, stopped = false;
        int64_t issued = 0;  // pipeline stages issued (for the test hook wt.stop_after)
        // ring positions and phases advance by counting (no division in the issue loop)
        int yb = 0, s = 0;
        uint32_t yph = 0, ph = 0;
        for (int64_t item = blockIdx.x; ok && !stopped && item < n_tiles; item += gridDim.x) {
            if (!mbar_wait(bar(Y_EMPTY + yb), yph ^ 1, abort_flag, wlim)) { ok = false; break; }
            mbar_expect_tx(bar(Y_FULL + yb), lay.y_bytes);
            bulk_g2s(sbase + yb * lay.y_bytes, Yt + item * (int64_t)(lay.y_bytes / 2), lay.y_bytes,
                     bar(Y_FULL + yb));
            y_par[yb] = (int)yph;
            if (++yb == YBUF) { yb = 0; yph ^= 1u; }
            const int32_t* qs = quad_slot + item * kQuads;
            const bool mixed = qs[1] != qs[0] || qs[2] != qs[0] || qs[3] != qs[0];
            const uint16_t* qrow = Qb3 + (int64_t)qs[0] * G_pad * 8;
            int j = ((tile_j0[item] % n_gt) + n_gt) % n_gt;
            for (int jj = 0; ok && !stopped && jj < n_gt; ++jj) {
                const uint16_t* btile = Bt + (int64_t)j * tile_elems;
                if (mixed) {
                    // an extra stage: the q-step slabs of the four quadrants' slots, side by side
                    if (wt.stop_after >= 0 && issued >= wt.stop_after) { stopped = true; break; }
                    ++issued;
                    if (!mbar_wait(bar(B_EMPTY + s), ph ^ 1, abort_flag, wlim)) { ok = false; break; }
                    const uint32_t st0 = sbase + lay.off_b + s * lay.stage_bytes;
                    mbar_expect_tx(bar(B_FULL + s), kQuads * kQBytes);
                    for (int k = 0; k < kQuads; ++k)
                        bulk_g2s(st0 + k * kQBytes, Qb3 + ((int64_t)qs[k] * G_pad + (int64_t)j * kBN) * 8, kQBytes,
                                 bar(B_FULL + s));
                    b_par[s] = (int)ph;
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
                for (int c = 0; c < NC; ++c) {
                    if (wt.stop_after >= 0 && issued >= wt.stop_after) { stopped = true; break; }
                    ++issued;
                    if (!mbar_wait(bar(B_EMPTY + s), ph ^ 1, abort_flag, wlim)) { ok = false; break; }
                    const uint32_t st0 = sbase + lay.off_b + s * lay.stage_bytes;
                    const uint32_t hi_bytes = KCHUNK ? 2u * kBChunk : lay.bpart_bytes / 2u;
                    const uint32_t bytes = (kLo ? 2u * hi_bytes : hi_bytes) + (c == 0 && !mixed ? kQBytes : 0u);
                    mbar_expect_tx(bar(B_FULL + s), bytes);
                    if (KCHUNK) {
                        // hi slabs 2c, 2c+1 and lo slabs K/8 + 2c, K/8 + 2c + 1 of the tile
                        bulk_g2s(st0, btile + (int64_t)(2 * c) * (kBChunk / 2), hi_bytes, bar(B_FULL + s));
                        if (kLo)
                            bulk_g2s(st0 + hi_bytes, btile + (int64_t)(K / 8 + 2 * c) * (kBChunk / 2), hi_bytes,
                                     bar(B_FULL + s));
                    } else {
                        bulk_g2s(st0, btile, kLo ? lay.bpart_bytes : hi_bytes, bar(B_FULL + s));
                    }
                    if (c == 0 && !mixed)
                        bulk_g2s(st0 + lay.bpart_bytes, qrow + (int64_t)j * kBN * 8, kQBytes, bar(B_FULL + s));
                    b_par[s] = (int)ph;
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
                if (++j == n_gt) j = 0;
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, kDevTimeout);
        }
        if (!ok || stopped) {
            // let every copy this thread issued land before the CTA can exit (the consumers of a
            // stopped producer time out on the stages that never come)
            for (int i = 0; i < YBUF; ++i)
                if (y_par[i] >= 0) mbar_wait(bar(Y_FULL + i), (uint32_t)y_par[i], nullptr);
            for (int s = 0; s < STAGES; ++s)
                if (b_par[s] >= 0) mbar_wait(bar(B_FULL + s), (uint32_t)b_par[s], nullptr);
        }
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------------------- MMA
        bool ok = true;
        const uint64_t a_q = smem_desc(sbase + lay.off_ones, lay.off_zero - lay.off_ones, 128);
        // selector pairs of a mixed tile: quadrants 0 and 1 in K columns 0-7 and 8-15, then 2 and 3
        const uint64_t a_s01 = smem_desc(sbase + lay.off_sel, kAChunk, 128);
        const uint64_t a_s23 = smem_desc(sbase + lay.off_sel + 2 * kAChunk, kAChunk, 128);
        int yb = 0, s = 0, ab = 0;
        uint32_t yph = 0, ph = 0, aph = 0;
        for (int64_t item = blockIdx.x; ok && item < n_tiles; item += gridDim.x) {
            if (!mbar_wait(bar(Y_FULL + yb), yph, abort_flag, wlim)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a0 = sbase + yb * lay.y_bytes;
            const int32_t* qs = quad_slot + item * kQuads;
            const bool mixed = qs[1] != qs[0] || qs[2] != qs[0] || qs[3] != qs[0];
            for (int jj = 0; ok && jj < n_gt; ++jj) {
                if (!mbar_wait(bar(T_EMPTY + ab), aph ^ 1, abort_flag, wlim)) { ok = false; break; }
                const uint32_t d = tmem_base + (uint32_t)(ab * kBN);
                if (mixed) {
                    // q-step stage: accumulator <- q_g of each row's own covariance (two selector MMAs;
                    // a row takes its quadrant's slab and exact zeros from the other three)
                    if (!mbar_wait(bar(B_FULL + s), ph, abort_flag, wlim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t q0 = sbase + lay.off_b + s * lay.stage_bytes;
                    mma_bf16(d, a_s01, smem_desc(q0, kQBytes, 128), kIdesc, 0u);
                    mma_bf16(d, a_s23, smem_desc(q0 + 2 * kQBytes, kQBytes, 128), kIdesc, 1u);
                    mma_commit(bar(B_EMPTY + s));
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
                for (int c = 0; c < NC; ++c) {
                    if (!mbar_wait(bar(B_FULL + s), ph, abort_flag, wlim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t b0 = sbase + lay.off_b + s * lay.stage_bytes;
                    if (c == 0 && !mixed) {
                        // q-step: accumulator <- qb_g
                        const uint32_t qoff = lay.off_b + s * lay.stage_bytes + lay.bpart_bytes;
                        mma_bf16(d, a_q, smem_desc(sbase + qoff, lay.off_zero - qoff, 128), kIdesc, 0u);
                    }
                    // descriptors of the first K step; a step of 16 columns moves the start address by
                    // two slabs, i.e. adds (2 slab bytes) >> 4 to the descriptor's address field
                    const int k_lo = KCHUNK ? c : 0, k_hi = KCHUNK ? c + 1 : K / 16;
                    uint64_t a_hi = smem_desc(a0 + (2 * k_lo) * kAChunk, kAChunk, 128);
                    uint64_t a_lo = smem_desc(a0 + (K / 8 + 2 * k_lo) * kAChunk, kAChunk, 128);
                    uint64_t b_hi = smem_desc(KCHUNK ? b0 : b0 + (2 * k_lo) * kBChunk, kBChunk, 128);
                    uint64_t b_lo = smem_desc(KCHUNK ? b0 + 2 * kBChunk : b0 + (K / 8 + 2 * k_lo) * kBChunk,
                                              kBChunk, 128);
                    constexpr uint64_t kAStep = (2 * kAChunk) >> 4, kBStep = (2 * kBChunk) >> 4;
#pragma unroll 4
                    for (int kk = k_lo; kk < k_hi; ++kk) {
                        mma_bf16(d, a_hi, b_hi, kIdesc, 1u);
                        if (kLo) {
                            mma_bf16(d, a_lo, b_hi, kIdesc, 1u);
                            mma_bf16(d, a_hi, b_lo, kIdesc, 1u);
                        }
                        a_hi += kAStep;
                        a_lo += kAStep;
                        b_hi += kBStep;
                        b_lo += kBStep;
                    }
                    mma_commit(bar(B_EMPTY + s));
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                }
                if (ok) mma_commit(bar(T_FULL + ab));
                if (++ab == 2) { ab = 0; aph ^= 1u; }
            }
            if (ok) mma_commit(bar(Y_EMPTY + yb));
            if (++yb == YBUF) { yb = 0; yph ^= 1u; }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, kDevTimeout);
        }
        // every MMA issued above has completed once DONE flips
        mma_commit(bar(DONE));
        mbar_wait(bar(DONE), 0, nullptr);
    } else if (warp >= 2) {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;           // TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;    // which half of the BN columns
        const int row = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        float* scratch = (float*)(smem + lay.off_scratch + (warp - 2) * 4096);
        // hand-over area of this row's half-1 warp (warp + 4 for a half-0 warp)
        float* mval = (float*)(smem + lay.off_scratch + (half ? warp - 2 : warp + 2) * 4096);
        int32_t* midx = (int32_t*)(mval + TOPK * 32);
        bool ok = true;
        int it = 0;
        for (int64_t item = blockIdx.x; item < n_tiles; item += gridDim.x, ++it) {
            // seeded with the row's certified upper bound: larger values can never be the minimum
            const float seed = tau0[item * kBM + row];
            float vals[TOPK];
            int32_t idx[TOPK];
#pragma unroll
            for (int t = 0; t < TOPK; ++t) {
                vals[t] = seed;
                idx[t] = INT32_MAX;
            }
            float bv = FLT_MAX;       // kModeMin: running minimum of the row and its index
            int32_t bi = INT32_MAX;
            int32_t nlist = 0;        // kModeList: entries found by this half row
            // list storage of this half row: fixed kListCap slots, or the exact-size compact
            // region of its universe (la.off, counts known from an earlier list round)
            int64_t lbase = ((item * kBM + row) * 2 + half) * (int64_t)kListCap;
            int32_t lcap = kListCap;
            if (MODE == kModeList && la.off) {
                const int32_t u = la.tile_univ[item * kBM + row];
                const int2 nn = (u >= 0) ? la.n[u] : make_int2(0, 0);
                lbase = (u >= 0) ? la.off[u] + (half ? nn.x : 0) : 0;
                lcap = half ? nn.y : nn.x;
            }
            int j = ((tile_j0[item] % n_gt) + n_gt) % n_gt;
            for (int jj = 0; ok && jj < n_gt; ++jj, j = (j + 1 == n_gt) ? 0 : j + 1) {
                const int64_t seq = (int64_t)it * n_gt + jj;
                const int ab = (int)(seq & 1);
                const uint32_t aph = (uint32_t)((seq >> 1) & 1);
                bool w_ok = mbar_wait(bar(T_FULL + ab), aph, abort_flag, wlim);
                if (!__all_sync(0xffffffffu, w_ok)) {
                    ok = false;
                    if (lane == 0) *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem_base + lane_base + (uint32_t)(ab * kBN + half * kHalfCols);
                const int64_t g0 = (int64_t)j * kBN + half * kHalfCols;
                uint32_t r0[32], r1[32], r2[32], r3[32];
                auto chunk = [&](const uint32_t(&r)[32], float m, int64_t gc) {
                    if (MODE == kModeMin)
                        min_chunk(bv, bi, r, m, gc, G);
                    else if (MODE == kModeList)
                        list_chunk(nlist, lcap, cand_val + lbase, cand_idx + lbase, seed, r, m, gc, G);
                    else
                        topk_chunk<TOPK>(vals, idx, r, m, gc, G, scratch, lane);
                };
                // the warp's 128 columns go to registers at once, so the accumulator is
                // handed back to the MMA after one load latency, before any filtering
                tmem_ld32(tb + 0, r0);
                tmem_ld32(tb + 32, r1);
                tmem_ld32(tb + 64, r2);
                tmem_ld32(tb + 96, r3);
                tmem_wait(r0);
                tmem_wait(r1);
                tmem_wait(r2);
                tmem_wait(r3);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(T_EMPTY + ab));
                // the four chunk minima first (independent trees), then the rare slow paths
                const float m0 = min32(r0), m1 = min32(r1), m2 = min32(r2), m3 = min32(r3);
                // top-k: a chunk acts only at or below the row's k-th value, so a warp none of whose
                // 128 values reaches it skips the four chunk steps (the common case once lists fill)
                if (MODE == kModeTopK &&
                    !__any_sync(0xffffffffu, fminf(fminf(m0, m1), fminf(m2, m3)) <= vals[TOPK - 1]))
                    continue;
                chunk(r0, m0, g0 + 0);
                __syncwarp();
                chunk(r1, m1, g0 + 32);
                __syncwarp();
                chunk(r2, m2, g0 + 64);
                __syncwarp();
                chunk(r3, m3, g0 + 96);
                __syncwarp();
            }
            if (MODE == kModeList) {
                cand_count[(item * kBM + row) * 2 + half] = ok ? nlist : -1;
                if (!ok) break;
                continue;
            }
            // both halves of a row reach here once per item even after a timeout, and they leave the
            // item loop together: each posts its ok before the pair barrier and both decide on the
            // two posted values, so neither can wait at that barrier for a partner that has left
            if (lane == 0) pair_ok[quad * 2 + half] = ok ? 1 : 0;
            if (half == 1) {
                if (MODE == kModeMin) {
                    mval[lane] = bv;
                    midx[lane] = bi;
                } else {
#pragma unroll
                    for (int t = 0; t < TOPK; ++t) {
                        mval[t * 32 + lane] = vals[t];
                        midx[t * 32 + lane] = idx[t];
                    }
                }
            }
            named_bar(1 + quad, 64);
            const bool pair_done = pair_ok[quad * 2] && pair_ok[quad * 2 + 1];
            if (half == 0) {
                const int64_t orow = item * kBM + row;
                if (MODE == kModeMin) {
                    const float x = mval[lane];
                    const int32_t xi = midx[lane];
                    if (x < bv || (x == bv && xi < bi)) {
                        bv = x;
                        bi = xi;
                    }
                    // the row's minimum index; k_min_seed turns it into the certified seed after the
                    // launch, so the epilogue never stalls the MMAs on the probe's scattered loads
                    cand_idx[orow] = (pair_done && seed > -FLT_MAX) ? bi : INT32_MAX;
                } else {
#pragma unroll 1
                    for (int t = 0; t < TOPK; ++t) {
                        const float x = mval[t * 32 + lane];
                        const int32_t xi = midx[t * 32 + lane];
                        if (x < vals[TOPK - 1] || (x == vals[TOPK - 1] && xi < idx[TOPK - 1]))
                            topk_insert<TOPK>(vals, idx, x, xi);
                    }
#pragma unroll
                    for (int t = 0; t < TOPK; ++t) {
                        cand_val[orow * TOPK + t] = vals[t];
                        cand_idx[orow * TOPK + t] = (idx[t] == INT32_MAX) ? -1 : idx[t];
                    }
                }
            }
            named_bar(1 + quad, 64);
            if (!pair_done) break;
        }
        if (!ok && lane == 0) {
            *abort_flag = 1;
            atomicOr(status, kDevTimeout);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

template <int TOPK, int MODE, bool KCHUNK>
void run_screen(const ScreenLayout& lay, const uint16_t* Yt, const uint16_t* Bt, const uint16_t* Qb3,
                const int32_t* quad_slot, float* tau0, const int32_t* tile_j0, int64_t n_tiles, int64_t G,
                int64_t G_pad, float* cv, int32_t* ci, int32_t* cc, int* status, const ProbeArgs& pa,
                const ListArgs& la, const WaitTest& wt, int n_sm, cudaStream_t st) {
    auto kern = k_screen<TOPK, MODE, KCHUNK>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes);
    int64_t grid = n_tiles < n_sm ? n_tiles : n_sm;
    if (grid < 1) grid = 1;
    count_launch();
    kern<<<(unsigned)grid, 64 + 32 * kEpiWarps, lay.bytes, st>>>(Yt, Bt, Qb3, quad_slot, tau0, tile_j0, n_tiles, G,
                                                                   G_pad, cv, ci, cc, status, pa, lay, la, wt);
    if (MODE == kModeMin) {
        const int64_t rows = n_tiles * kBM;
        count_launch();
        k_min_seed<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(Yt, quad_slot, ci, tau0, rows, G, G_pad, pa,
                                                                   status);
    }
}

// Shared-memory plan for K with the requested depth / buffering (0 = built-in:
// whole-tile stages at the depths measured on the 100x100, N_fit 45 workload for
// K <= 64; 16-column slices as deep as shared memory allows, up to 8, above).
ScreenLayout choose_layout(int K, int stages, int ybuf) {
    const int kchunk = K > 64 ? 1 : 0;
    if (ybuf <= 0) ybuf = (K <= 32) ? 2 : 1;
    if (stages <= 0) {
        if (!kchunk) {
            stages = K == 16 ? 4 : (K == 64 ? 2 : 3);
        } else {
            const ScreenLayout one = screen_layout(K, 1, ybuf, 1);
            stages = one.bytes > kSmemMax ? 0 : 1 + (int)((kSmemMax - one.bytes) / (one.stage_bytes + 16u));
            stages = stages > 8 ? 8 : stages;
        }
    }
    return screen_layout(K, stages, ybuf, kchunk);
}

}  // namespace

bool screen_config_ok(int K, int stages, int ybuf) {
    if (K < 16 || K % 16 != 0 || K > kMaxScreenK) return false;
    if (stages != 0 && (stages < 2 || stages > 8)) return false;
    if (ybuf < 0 || ybuf > 2) return false;
    const ScreenLayout lay = choose_layout(K, stages, ybuf);
    // a mixed tile's q-step stage puts the four quadrants' slabs in a stage's B part
    return lay.stages >= 2 && lay.bytes <= kSmemMax && lay.bpart_bytes >= kQuads * kQBytes;
}

bool launch_screen(int K, int topk, int mode, int stages, int ybuf, const uint16_t* Yt, const uint16_t* Bt,
                   const uint16_t* Qb3, const int32_t* quad_slot, float* tau0, const int32_t* tile_j0,
                   int64_t n_tiles, int64_t G, int64_t G_pad, float* cv, int32_t* ci, int32_t* cc, int* status,
                   const float* Qc, const float* Qb, const float4* gnorm, const float4* alpha, const GridSpec& gs,
                   int nfit, const ListArgs& la, const WaitTest& wt, int n_sm, cudaStream_t st) {
    if (n_tiles <= 0) return true;
    if (!screen_config_ok(K, stages, ybuf) || (topk != 4 && topk != 8 && topk != 16)) return false;
    const ScreenLayout lay = choose_layout(K, stages, ybuf);
    const ProbeArgs pa{Qc, Qb, gnorm, alpha, gs, nfit};
#define FC_SCREEN_RUN(TT, MM, CC) \
    run_screen<TT, MM, CC>(lay, Yt, Bt, Qb3, quad_slot, tau0, tile_j0, n_tiles, G, G_pad, cv, ci, cc, status, pa, la, \
                           wt, n_sm, st)
#define FC_SCREEN_MODES(TT, CC)                 \
    do {                                        \
        if (mode == kModeMin)                   \
            FC_SCREEN_RUN(TT, kModeMin, CC);    \
        else if (mode == kModeList)             \
            FC_SCREEN_RUN(TT, kModeList, CC);   \
        else                                    \
            FC_SCREEN_RUN(TT, kModeTopK, CC);   \
    } while (0)
    if (topk == 4 && mode == kModeTopK) {
        // top-4 lists; the min and list passes of a top-4 scan use the top-8 instance (they keep no list)
        if (lay.kchunk)
            FC_SCREEN_RUN(4, kModeTopK, true);
        else
            FC_SCREEN_RUN(4, kModeTopK, false);
    } else if (topk <= 8) {
        if (lay.kchunk)
            FC_SCREEN_MODES(8, true);
        else
            FC_SCREEN_MODES(8, false);
    } else {
        if (lay.kchunk)
            FC_SCREEN_MODES(16, true);
        else
            FC_SCREEN_MODES(16, false);
    }
#undef FC_SCREEN_MODES
#undef FC_SCREEN_RUN
    return true;
}

}  // namespace fcdev
