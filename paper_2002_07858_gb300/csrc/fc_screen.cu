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

namespace fcdev {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr uint64_t kWaitNs = 2000000000ull;

// Bounded wait on a phase parity; false on timeout or when another role aborted.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort_flag) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (abort_flag && *abort_flag) return false;
            if (global_ns() - t0 > kWaitNs) return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand without swizzle: 8x8 core matrices of 16-byte rows; LBO steps
// along K between the two core matrices of a K=16 slice, SBO steps 8 rows.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M = BM, N = BN
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Asynchronous 32-column TMEM load (one lane = one row); the registers are only
// valid after tmem_wait() on the same buffer.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// tcgen05.wait::ld; the buffer's registers are in-out operands so no use of
// them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ void named_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// (value, index) insertion into a sorted list, lexicographic order
template <int TOPK>
__device__ __forceinline__ void topk_insert(float (&vals)[TOPK], int32_t (&idx)[TOPK], float x, int32_t g) {
    float cx = x;
    int32_t cg = g;
#pragma unroll
    for (int t = 0; t < TOPK; ++t) {
        const bool sw = cx < vals[t] || (cx == vals[t] && cg < idx[t]);
        const float tv = vals[t];
        const int32_t ti = idx[t];
        vals[t] = sw ? cx : tv;
        idx[t] = sw ? cg : ti;
        cx = sw ? tv : cx;
        cg = sw ? ti : cg;
    }
}

// 32 lower bounds of one row (columns g0..g0+31): running top-k.  Fast path:
// a min over the 32 values and one compare.  If exactly one value is at or
// below the current k-th one it is that minimum and is inserted directly;
// with several, they are parked in this warp's shared scratch ([i][lane]) and
// inserted in a rolled loop (small code for the instruction cache).
template <int TOPK>
__device__ __forceinline__ void topk_chunk(float (&vals)[TOPK], int32_t (&idx)[TOPK], const uint32_t (&r)[32],
                                           int64_t g0, int64_t G, float* scratch, int lane) {
    float m = __uint_as_float(r[0]);
#pragma unroll
    for (int i = 1; i < 32; ++i) m = fminf(m, __uint_as_float(r[i]));
    if (m <= vals[TOPK - 1]) {
        const float tau = vals[TOPK - 1];
        uint32_t mask = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) mask |= (__uint_as_float(r[i]) <= tau ? 1u : 0u) << i;
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

// Screen modes: kModeMin (first pass) uses only the hi*hi products, keeps each
// row's minimum and turns it into a certified upper bound that tightens the
// row's seed tau0 in place; kModeTopK keeps the full top-k; kModeList lists
// every grid point whose lower bound is at or below the seed (kListCap per
// half row, the count says whether the list overflowed).
struct ProbeArgs {
    const float* Qc;
    const float* Qb;
    const float4* gnorm;
    const float4* alpha;
    const float* Sc32;
    int nfit;
};

constexpr int kModeTopK = 0;
constexpr int kModeMin = 1;
constexpr int kModeList = 2;

// List mode: append every value at or below the seed (and its grid index).
__device__ __forceinline__ void list_chunk(int32_t& n, float* __restrict__ lval, int32_t* __restrict__ lidx, float seed,
                                           const uint32_t (&r)[32], int64_t g0, int64_t G) {
    float m = __uint_as_float(r[0]);
#pragma unroll
    for (int i = 1; i < 32; ++i) m = fminf(m, __uint_as_float(r[i]));
    if (m <= seed) {
        uint32_t mask = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) mask |= (__uint_as_float(r[i]) <= seed ? 1u : 0u) << i;
        const int64_t lim = G - g0;
        if (lim < 32) mask &= (lim <= 0) ? 0u : ((1u << lim) - 1u);
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            if (n < kListCap) {
                lidx[n] = (int32_t)(g0 + i);
                lval[n] = m;  // a lower bound of the entry (the chunk minimum); only the index is used
            }
            ++n;
        }
    }
}

// First pass: running minimum of a row.  The index is recovered only when the
// chunk improves the minimum (rare after the first tiles).
__device__ __forceinline__ void min_chunk(float& bv, int32_t& bi, const uint32_t (&r)[32], int64_t g0, int64_t G) {
    float m = __uint_as_float(r[0]);
#pragma unroll
    for (int i = 1; i < 32; ++i) m = fminf(m, __uint_as_float(r[i]));
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
    const float* sg = pa.Sc32 + (int64_t)g * n;
    float dot = 0.0f, adot = 0.0f;
    for (int i = 0; i < n; ++i) {
        const float h = __uint_as_float((uint32_t)Yt[ytile_elem(item, row, i, K)] << 16);
        const float l = __uint_as_float((uint32_t)Yt[ytile_elem(item, row, K + i, K)] << 16);
        const float y = h + l;
        dot = fmaf(y, sg[i], dot);
        adot = fmaf(fabsf(y), fabsf(sg[i]), adot);
    }
    const int64_t qi = (int64_t)slot * G_pad + g;
    const float qc = pa.Qc[qi];
    const float sig = qc + dot;
    const float eps = bound_dot(pa.alpha[item * kBM + row], pa.gnorm[g]) + (qc - pa.Qb[qi]) +
                      (float)(n + 2) * 5.9604645e-08f * (adot + fabsf(qc)) + 1.1920929e-07f * (fabsf(sig) + 1.0f);
    return (sig + 2.0f * eps) * 1.0000005f + 1.0e-6f + 4.7683716e-07f * fabsf(sig);
}

constexpr int kTmemCols = 2 * kBN;  // two accumulator buffers
constexpr int kEpiWarps = 8;
constexpr int kHalfCols = kBN / 2;

template <int K, int STAGES, int YBUF>
struct ScreenSmem {
    static constexpr uint32_t kYBytes = 2u * K * kBM * 2u;   // hi + lo, bf16
    static constexpr uint32_t kBBytes = 2u * K * kBN * 2u;
    static constexpr uint32_t kQBytes = kBN * 16u;           // one 8-column slab of q-step rows
    static constexpr uint32_t kAChunk = kBM * 16u;           // one 8-column slab of the A image
    static constexpr uint32_t kBChunk = kBN * 16u;
    static constexpr uint32_t kOffY = 0;
    static constexpr uint32_t kOffB = YBUF * kYBytes;
    static constexpr uint32_t kOffQ = kOffB + STAGES * kBBytes;
    static constexpr uint32_t kOffOnes = kOffQ + STAGES * kQBytes;   // A slab of the q-step: [1,1,1,0..] per row
    static constexpr uint32_t kOffZero = kOffOnes + kAChunk;         // second slab of the q-step, all zero
    // per epilogue warp 4 KB: slow-path scratch inside a tile, top-k hand-over at the end of a row tile
    static constexpr uint32_t kOffScratch = kOffZero + kBChunk;
    static constexpr uint32_t kOffBar = kOffScratch + kEpiWarps * 4096;
    static constexpr uint32_t kNumBars = 2 + 2 + STAGES + STAGES + 2 + 2 + 1;
    static constexpr uint32_t kBytes = kOffBar + kNumBars * 8 + 16 + 1024;
};

template <int K, int TOPK, int STAGES, int YBUF, int MODE>
__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1)
    k_screen(const uint16_t* __restrict__ Yt, const uint16_t* __restrict__ Bt, const uint16_t* __restrict__ Qb3,
             const int32_t* __restrict__ tile_slot, float* __restrict__ tau0, const int32_t* __restrict__ tile_j0,
             int64_t n_tiles, int64_t G, int64_t G_pad, float* __restrict__ cand_val, int32_t* __restrict__ cand_idx,
             int32_t* __restrict__ cand_count, int* __restrict__ status, ProbeArgs pa) {
    using L = ScreenSmem<K, STAGES, YBUF>;
    static_assert(2 * TOPK * 32 * 4 <= 4096, "top-k hand-over exceeds the warp scratch");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_addr(smem);
    uint64_t* bars = (uint64_t*)(smem + L::kOffBar);
    uint32_t* tmem_holder = (uint32_t*)(smem + L::kOffBar + L::kNumBars * 8);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
    auto bar = [&](int i) { return smem_addr(&bars[i]); };
    const int Y_FULL = 0, Y_EMPTY = 2, B_FULL = 4, B_EMPTY = 4 + STAGES, T_FULL = 4 + 2 * STAGES,
              T_EMPTY = 6 + 2 * STAGES, DONE = 8 + 2 * STAGES;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // constant q-step operand slabs (generic-proxy writes, fenced for the tensor core below)
    {
        uint32_t* ones = (uint32_t*)(smem + L::kOffOnes);
        for (int i = threadIdx.x; i < (int)(L::kAChunk / 4); i += blockDim.x) {
            const int w = i & 3;  // 4 words per 16-byte row: bf16 pairs (1,1), (1,0), (0,0), (0,0)
            ones[i] = (w == 0) ? 0x3F803F80u : (w == 1 ? 0x00003F80u : 0u);
        }
        uint32_t* zero = (uint32_t*)(smem + L::kOffZero);
        for (int i = threadIdx.x; i < (int)(L::kBChunk / 4); i += blockDim.x) zero[i] = 0u;
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

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        int y_par[2] = {-1, -1}, b_par[STAGES];
        for (int s = 0; s < STAGES; ++s) b_par[s] = -1;
        bool ok = true;
        int it = 0;
        for (int64_t item = blockIdx.x; ok && item < n_tiles; item += gridDim.x, ++it) {
            const int yb = it % YBUF;
            const uint32_t yph = (it / YBUF) & 1;
            if (!mbar_wait(bar(Y_EMPTY + yb), yph ^ 1, abort_flag)) { ok = false; break; }
            mbar_expect_tx(bar(Y_FULL + yb), L::kYBytes);
            bulk_g2s(sbase + L::kOffY + yb * L::kYBytes, Yt + item * (int64_t)(L::kYBytes / 2), L::kYBytes,
                     bar(Y_FULL + yb));
            y_par[yb] = (int)yph;
            const uint16_t* qrow = Qb3 + (int64_t)tile_slot[item] * G_pad * 8;
            const int j0 = ((tile_j0[item] % n_gt) + n_gt) % n_gt;
            for (int jj = 0; jj < n_gt; ++jj) {
                const int j = (j0 + jj) % n_gt;
                const int64_t seq = (int64_t)it * n_gt + jj;
                const int s = (int)(seq % STAGES);
                const uint32_t ph = (uint32_t)((seq / STAGES) & 1);
                if (!mbar_wait(bar(B_EMPTY + s), ph ^ 1, abort_flag)) { ok = false; break; }
                mbar_expect_tx(bar(B_FULL + s), L::kBBytes + L::kQBytes);
                bulk_g2s(sbase + L::kOffB + s * L::kBBytes, Bt + (int64_t)j * (L::kBBytes / 2), L::kBBytes,
                         bar(B_FULL + s));
                bulk_g2s(sbase + L::kOffQ + s * L::kQBytes, qrow + (int64_t)j * kBN * 8, L::kQBytes, bar(B_FULL + s));
                b_par[s] = (int)ph;
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, kDevTimeout);
            // let every copy this thread issued land before the CTA can exit
            for (int i = 0; i < YBUF; ++i)
                if (y_par[i] >= 0) mbar_wait(bar(Y_FULL + i), (uint32_t)y_par[i], nullptr);
            for (int s = 0; s < STAGES; ++s)
                if (b_par[s] >= 0) mbar_wait(bar(B_FULL + s), (uint32_t)b_par[s], nullptr);
        }
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------------------- MMA
        bool ok = true;
        int it = 0;
        const uint64_t a_q = smem_desc(sbase + L::kOffOnes, L::kOffZero - L::kOffOnes, 128);
        for (int64_t item = blockIdx.x; ok && item < n_tiles; item += gridDim.x, ++it) {
            const int yb = it % YBUF;
            if (!mbar_wait(bar(Y_FULL + yb), (it / YBUF) & 1, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a0 = sbase + L::kOffY + yb * L::kYBytes;
            for (int jj = 0; jj < n_gt; ++jj) {
                const int64_t seq = (int64_t)it * n_gt + jj;
                const int s = (int)(seq % STAGES);
                const uint32_t ph = (uint32_t)((seq / STAGES) & 1);
                const int ab = (int)(seq & 1);
                const uint32_t aph = (uint32_t)((seq >> 1) & 1);
                if (!mbar_wait(bar(T_EMPTY + ab), aph ^ 1, abort_flag)) { ok = false; break; }
                if (!mbar_wait(bar(B_FULL + s), ph, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t b0 = sbase + L::kOffB + s * L::kBBytes;
                const uint32_t qs = L::kOffQ + s * L::kQBytes;
                const uint32_t d = tmem_base + (uint32_t)(ab * kBN);
                // q-step: accumulator <- qb_g
                mma_bf16(d, a_q, smem_desc(sbase + qs, L::kOffZero - qs, 128), 0u);
#pragma unroll
                for (int kk = 0; kk < K / 16; ++kk) {
                    const uint64_t a_hi = smem_desc(a0 + (2 * kk) * L::kAChunk, L::kAChunk, 128);
                    const uint64_t a_lo = smem_desc(a0 + (K / 8 + 2 * kk) * L::kAChunk, L::kAChunk, 128);
                    const uint64_t b_hi = smem_desc(b0 + (2 * kk) * L::kBChunk, L::kBChunk, 128);
                    const uint64_t b_lo = smem_desc(b0 + (K / 8 + 2 * kk) * L::kBChunk, L::kBChunk, 128);
                    mma_bf16(d, a_hi, b_hi, 1u);
                    if (MODE != kModeMin) {
                        mma_bf16(d, a_lo, b_hi, 1u);
                        mma_bf16(d, a_hi, b_lo, 1u);
                    }
                }
                mma_commit(bar(B_EMPTY + s));
                mma_commit(bar(T_FULL + ab));
            }
            if (ok) mma_commit(bar(Y_EMPTY + yb));
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
        float* scratch = (float*)(smem + L::kOffScratch + (warp - 2) * 4096);
        // hand-over area of this row's half-1 warp (warp + 4 for a half-0 warp)
        float* mval = (float*)(smem + L::kOffScratch + (half ? warp - 2 : warp + 2) * 4096);
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
            const int64_t lbase = ((item * kBM + row) * 2 + half) * (int64_t)kListCap;
            const int j0 = ((tile_j0[item] % n_gt) + n_gt) % n_gt;
            for (int jj = 0; ok && jj < n_gt; ++jj) {
                const int j = (j0 + jj) % n_gt;
                const int64_t seq = (int64_t)it * n_gt + jj;
                const int ab = (int)(seq & 1);
                const uint32_t aph = (uint32_t)((seq >> 1) & 1);
                bool w_ok = mbar_wait(bar(T_FULL + ab), aph, abort_flag);
                if (!__all_sync(0xffffffffu, w_ok)) {
                    ok = false;
                    if (lane == 0) *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem_base + lane_base + (uint32_t)(ab * kBN + half * kHalfCols);
                const int64_t g0 = (int64_t)j * kBN + half * kHalfCols;
                uint32_t r0[32], r1[32], r2[32], r3[32];
                auto chunk = [&](const uint32_t(&r)[32], int64_t gc) {
                    if (MODE == kModeMin)
                        min_chunk(bv, bi, r, gc, G);
                    else if (MODE == kModeList)
                        list_chunk(nlist, cand_val + lbase, cand_idx + lbase, seed, r, gc, G);
                    else
                        topk_chunk<TOPK>(vals, idx, r, gc, G, scratch, lane);
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
                chunk(r0, g0 + 0);
                __syncwarp();
                chunk(r1, g0 + 32);
                __syncwarp();
                chunk(r2, g0 + 64);
                __syncwarp();
                chunk(r3, g0 + 96);
                __syncwarp();
            }
            if (MODE == kModeList) {
                cand_count[(item * kBM + row) * 2 + half] = ok ? nlist : kListCap + 1;
                if (!ok) break;
                continue;
            }
            // both halves of a row reach here even after a timeout, so the pair barrier cannot hang
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
            if (half == 0) {
                const int64_t orow = item * kBM + row;
                if (MODE == kModeMin) {
                    const float x = mval[lane];
                    const int32_t xi = midx[lane];
                    if (x < bv || (x == bv && xi < bi)) {
                        bv = x;
                        bi = xi;
                    }
                    if (ok && bi != INT32_MAX && seed > -FLT_MAX)
                        tau0[orow] = fminf(seed, probe_upper_bound(Yt, item, row, tile_slot[item], bi, G_pad, pa));
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
            if (!ok) break;
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

template <int K, int TOPK, int STAGES, int YBUF, int MODE>
void run_screen(const uint16_t* Yt, const uint16_t* Bt, const uint16_t* Qb3, const int32_t* tile_slot, float* tau0,
                const int32_t* tile_j0, int64_t n_tiles, int64_t G, int64_t G_pad, float* cv, int32_t* ci,
                int32_t* cc, int* status, const ProbeArgs& pa, int n_sm, cudaStream_t st) {
    using L = ScreenSmem<K, STAGES, YBUF>;
    static_assert(L::kBytes <= 232448, "screen tile does not fit in shared memory");
    auto kern = k_screen<K, TOPK, STAGES, YBUF, MODE>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kBytes);
    int64_t grid = n_tiles < n_sm ? n_tiles : n_sm;
    if (grid < 1) grid = 1;
    count_launch();
    kern<<<(unsigned)grid, 64 + 32 * kEpiWarps, L::kBytes, st>>>(Yt, Bt, Qb3, tile_slot, tau0, tile_j0, n_tiles,
                                                                   G, G_pad, cv, ci, cc, status, pa);
}

}  // namespace

bool launch_screen(int K, int topk, int mode, const uint16_t* Yt, const uint16_t* Bt, const uint16_t* Qb3,
                   const int32_t* tile_slot, float* tau0, const int32_t* tile_j0, int64_t n_tiles, int64_t G,
                   int64_t G_pad, float* cv, int32_t* ci, int32_t* cc, int* status, const float* Qc, const float* Qb,
                   const float4* gnorm, const float4* alpha, const float* Sc32, int nfit, int n_sm, cudaStream_t st) {
    if (n_tiles <= 0) return true;
    const ProbeArgs pa{Qc, Qb, gnorm, alpha, Sc32, nfit};
#define FC_SCREEN_RUN(KK, TT, SS, YY, MM) \
    run_screen<KK, TT, SS, YY, MM>(Yt, Bt, Qb3, tile_slot, tau0, tile_j0, n_tiles, G, G_pad, cv, ci, cc, status, pa, n_sm, st)
#define FC_SCREEN_CASE(KK, TT, SS, YY)                                   \
    if (K == KK && topk == TT) {                                         \
        if (mode == kModeMin)                                            \
            FC_SCREEN_RUN(KK, TT, SS, YY, kModeMin);                     \
        else if (mode == kModeList)                                      \
            FC_SCREEN_RUN(KK, TT, SS, YY, kModeList);                    \
        else                                                             \
            FC_SCREEN_RUN(KK, TT, SS, YY, kModeTopK);                    \
        return true;                                                     \
    }
    FC_SCREEN_CASE(16, 8, 4, 2)
    FC_SCREEN_CASE(32, 8, 3, 2)
    FC_SCREEN_CASE(48, 8, 3, 1)
    FC_SCREEN_CASE(64, 8, 2, 1)
    FC_SCREEN_CASE(16, 16, 4, 2)
    FC_SCREEN_CASE(32, 16, 3, 2)
    FC_SCREEN_CASE(48, 16, 3, 1)
    FC_SCREEN_CASE(64, 16, 2, 1)
#undef FC_SCREEN_CASE
#undef FC_SCREEN_RUN
    return false;
}

}  // namespace fcdev
