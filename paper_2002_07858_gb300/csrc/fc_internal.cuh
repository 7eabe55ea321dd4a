// fc_internal.cuh -- declarations shared by the library's translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace fcdev {

// Message returned by fc_last_error() for the calling thread.
void record_error(const char* msg);

// Number of kernels this library has launched (for the launch count of a run).
extern std::atomic<long long> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Screen tile shape: BM universes (TMEM lanes) x BN grid points (TMEM columns).
// A tile's rows come in four quadrants of 32 (the TMEM lane quadrants); each
// quadrant holds universes of one covariance slot, so one tile can serve up to
// four covariances (refit scans leave most covariances with few universes).
constexpr int kBM = 128;
constexpr int kBN = 256;
constexpr int kQuadRows = 32;
constexpr int kQuads = kBM / kQuadRows;
constexpr int kMaxTopK = 16;
constexpr int kMaxBins = 200;
constexpr int kMaxScreenK = 208;  // screen_k(kMaxBins): K of the largest tensor-core screen

// Error flags written by kernels into the context's device status word.
enum : int {
    kDevOk = 0,
    kDevNotSpd = 1,
    kDevTimeout = 2,
    kDevBadIndex = 4,
};

// ---- where a grid's spectra come from (device functions in fc_spec.cuh) ----
constexpr int kMaxOscAxes = 8;
constexpr int kMaxOscTerms = 4;

// The oscillation shape model of a grid on the device; axis_len == nullptr: none.
struct SpecModel {
    int D = 0, n_terms = 0, nf = 0, nfit = 0;
    const int32_t* axis_len = nullptr;  // [D]
    const int32_t* axis_off = nullptr;  // [D] first value of each axis in axis_val
    const int32_t* amp_ax = nullptr;    // [n_terms]
    const int32_t* dm2_ax = nullptr;    // [n_terms]
    const int32_t* sin_off = nullptr;   // [n_terms] first row of each term's sine table
    const double* axis_val = nullptr;
    const double* b = nullptr;          // [nf]
    const double* f = nullptr;          // [n_terms][nf]
    const double* sinT = nullptr;       // [rows][nf] sin(1.27 dm2 L_i / E_i), one row per dm2 value of a term
    const int32_t* mem_off = nullptr;   // [nfit + 1] CSR of the collapse; nullptr: identity
    const int32_t* mem = nullptr;       // [nf] full bins of each fit bin in increasing order
};

// Full-bin spectra rows: stored [G][nf] (S), or the model when S is null.
struct FullSrc {
    const double* S = nullptr;
    SpecModel m;
};

// Fit-space rows of a grid and the copies derived from them.  A null array is
// derived where it is read: from S_fit, or from the model when S_fit is null
// too, with the operation that fills the stored copy.
struct GridSpec {
    const double* S_fit = nullptr;   // [G][nfit]
    const double* Sc = nullptr;      // [G][nfit] S_fit - centre
    const float* Sc32 = nullptr;     // [G][nfit] (float)(S_fit - centre)
    const float2* Sdf = nullptr;     // [G][nfit] double-float S_fit
    const double* centre = nullptr;  // [nfit]
    int nfit = 0;
    SpecModel m;
};

// Padded fit dimension of the tensor-core screen: three spare columns (they
// carry the error-bound terms), rounded up to the MMA K-step of 16.
__host__ __device__ inline int screen_k(int nfit) { return ((nfit + 3 + 15) / 16) * 16; }

// Error-bound coefficients.  Per grid point g (gnorm): |s~_g|, |S_lo,g|, |r_S,g|
// (r_S = s~ - S_hi - S_lo); per universe row (alpha): a_acc (binary32
// accumulation, y^ rounding and |r_Y| with |s~|), |Y_lo|, |Y_hi + Y_lo|.  The
// screen's products are within dot(alpha, gnorm) of -2 y.s~_g.
__device__ __forceinline__ float bound_dot(const float4& a, const float4& n) {
    return 1.0001f * fmaf(a.x, n.x, fmaf(a.y, n.y, a.z * n.z));
}

// Relative slack on q_g: its own binary32 rounding plus its share of the
// screen's binary32 accumulation.  The q-step enters the tensor-core
// accumulator first and 3K products follow; bounding every add as a truncated
// binary32 add of the running sum gives (3K + 3) 2^-23 |q| (K = padded N_fit).
__device__ __forceinline__ float q_rel_slack(int nfit) {
    const int K = screen_k(nfit);
    return (float)(3 * K + 5) * 1.1920929e-07f;
}

// qb as a sum of three bf16 (hi + mid + lo <= qb, residual <= 2^-24 |qb|): the
// B-operand row of the screen's q-step, [hi, mid, lo, 0, 0, 0, 0, 0].
__device__ __forceinline__ void store_qb3(uint16_t* o, float qb) {
    uint16_t h = 0, m = 0, l = 0;
    if (qb < 1.0e38f) {
        const __nv_bfloat16 bh = __float2bfloat16_rn(qb);
        const float r1 = qb - __bfloat162float(bh);
        const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(bm);
        const __nv_bfloat16 bl = __float2bfloat16_rd(r2);
        h = __bfloat16_as_ushort(bh);
        m = __bfloat16_as_ushort(bm);
        l = __bfloat16_as_ushort(bl);
    } else {
        h = __bfloat16_as_ushort(__float2bfloat16_rn(3.0e38f));  // padding rows: never a candidate
    }
    uint4 v;
    v.x = (uint32_t)h | ((uint32_t)m << 16);
    v.y = (uint32_t)l;
    v.z = 0;
    v.w = 0;
    *reinterpret_cast<uint4*>(o) = v;
}

// ---- ingest (a1) ----
void launch_collapse(const double* S_full, int64_t G, int nf, const int32_t* collapse, int nfit, double* S_fit,
                     cudaStream_t st);
// centre <- per-bin approximate median of the fit-space rows of gs
void launch_centre(const GridSpec& gs, int64_t G, double* centre, cudaStream_t st);
// the screen's image and norms from gs (gs.centre set); Sc / Sc32 stored when given
void launch_centred(const GridSpec& gs, int64_t G, int64_t G_pad, int K, double* Sc, float* Sc32, float4* gnorm,
                    uint16_t* Btiles, cudaStream_t st);

// ---- covariances (a2) ----
// L_p (binary64 and binary32 copies) for every true point; gauss adds diag(s).
void launch_chol_sys(const FullSrc& src, int nf, const double* F, const int64_t* ps, int P, int gauss,
                     double* L64, float* L32, float* s32, double* work, int* status, cudaStream_t st);
// A(q) = M(q)^-1 for a list of (slot, q): A64, W64 (A = W^T W), A32, rho (max abs row sum of A).
void launch_build_cov(const FullSrc& src, int nf, int nfit, const int32_t* collapse, const double* F,
                      const int32_t* q_list, const int32_t* slot_list, int n, int cov_mode, double* A64,
                      double* W64, float* A32, float* rho, double* work, int* status, cudaStream_t st);
// q_g = s~_g^T A s~_g for slots: binary64 |W s~_g|^2 (plain) or binary32 central + lower bound (mixed).
void launch_qvec64(const GridSpec& gs, int64_t G, int nfit, const double* W64, const int32_t* slots, int n,
                   int64_t ldq, double* Q64, cudaStream_t st);
void launch_qvec32(const GridSpec& gs, const float4* gnorm, int64_t G, int64_t G_pad, int nfit, const float* A32,
                   const float* rho, const int32_t* slots, int n, float* Qc, float* Qb, uint16_t* Qb3,
                   cudaStream_t st);

// q_g = ||W s~_g||^2 on the tensor cores (A = W^T W), for 16 <= K <= 128:
// W image + norms per slot, then the certified Qc / Qb / Qb3 (see fc_qvec.cu).
bool qvec_tc_supported(int K);
void launch_wimage(const double* W64, const int32_t* slots, int n, int nfit, int K, uint16_t* Wimg, float4* wnorm,
                   cudaStream_t st);
bool launch_qvec_tc(const uint16_t* Bt, const uint16_t* Wimg, const float4* wnorm, const float4* gnorm,
                    const int32_t* slots, int n, int64_t G, int64_t G_pad, int nfit, int K, float* Qc, float* Qb,
                    uint16_t* Qb3, int* status, int n_sm, cudaStream_t st);

// ---- fake data (a3) ----
void launch_fake_data(const float* L32, const float* s32, int nf, const int32_t* collapse, int nfit,
                      const int64_t* ps, int P, int U, uint64_t seed, int gauss, float* d, cudaStream_t st);

// ---- scan bookkeeping ----
void launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t st);
void launch_iota_i32(int32_t* p, int64_t n, cudaStream_t st);
void launch_mark_used(const int32_t* active, int64_t n_active, const int32_t* cur, uint8_t* flag, cudaStream_t st);
void launch_compact_flags(uint8_t* flag, int64_t G, int32_t* list, int32_t* count, cudaStream_t st);
void launch_lookup_slots(const int32_t* active, int64_t n_active, const int32_t* cur, const int32_t* slot_of,
                         int32_t* uslot, cudaStream_t st);
void launch_set_slots(const int32_t* q_list, const int32_t* slot_list, int n, int32_t* slot_of, cudaStream_t st);

// ---- plain binary64 scan ----
void launch_scan64(const int32_t* list, int64_t n, const int32_t* uslot_of_list, const float* d,
                   const GridSpec& gs, int64_t G, int nfit, const double* A64,
                   const double* Q64, int64_t ldq, int32_t* best, cudaStream_t st);

// exact residual-form scan of the mixed path (double-float, split over nsp CTAs per universe)
void launch_scan_resid(const int32_t* list, int64_t n, const int32_t* uslot, const float* d, const GridSpec& gs,
                       int64_t G, int nfit, const float2* Wdf, double* part_v, int32_t* part_g, int nsp,
                       int32_t* best, cudaStream_t st);
// double-float copies: W of a list of slots; any binary64 array
void launch_wdf(const double* W64, const int32_t* slots, int n, int nfit, float2* Wdf, cudaStream_t st);
void launch_to_df(const double* x, int64_t n, float2* y, cudaStream_t st);

// ---- mixed path: grouping, y prep, screen, decision ----
// counting sort of active universes by slot into 32-row quadrants, four per BM-row tile:
// quad_slot [max_tiles * kQuads] (padding quadrants repeat the last slot), tile_univ [max_tiles * BM] (-1 = padding)
// slot_rows: rows per slot granule, 32 (quadrants) or 128 (whole tiles)
void launch_group(const int32_t* active, int64_t n_active, const int32_t* uslot, int n_slots, int32_t* cnt,
                  int32_t* quad_base, int32_t* fill, int32_t* n_tiles_dev, int32_t* quad_slot, int32_t* tile_univ,
                  int64_t max_tiles, int slot_rows, cudaStream_t st);
void launch_yprep(const int32_t* quad_slot, const int32_t* tile_univ, int64_t n_tiles, const float* d,
                  const double* centre, int nfit, int K, const float* A32, const float* rho, const int32_t* cur,
                  const GridSpec& gs, const float4* gnorm, const float* Qc, const float* Qb, int64_t G_pad,
                  uint16_t* Ytiles, float4* alpha, float* tau0, int32_t* tile_j0, cudaStream_t st);
// Tensor-core screen of BM-row tiles (see fc_screen.cu).  mode: kScreenTopK,
// kScreenMin (first pass; tightens tau0 in place) or kScreenList (every point
// with LB <= tau0; cand_count holds the full count per half row, so a count
// above the storage means the list overflowed; -1 = aborted).
// Returns false if the padded K has no compiled instance.
constexpr int kScreenTopK = 0, kScreenMin = 1, kScreenList = 2;
constexpr int kListCap = 64;
// List mode with exact-size storage: universe u's half-row lists start at
// off[u] (half 0, n[u].x entries) and off[u] + n[u].x (half 1, n[u].y).
// off == nullptr: kListCap slots per half row, indexed by tile row.
struct ListArgs {
    const int32_t* tile_univ;
    const int64_t* off;
    const int2* n;
};
// Test hook of the screen's bounded waits: wait_ns = limit of the pipeline waits
// (0 = the built-in 2 s); stop_after >= 0 = the copy producer of every CTA stops
// issuing after that many pipeline stages, so that its consumers' waits run out.
struct WaitTest {
    uint64_t wait_ns;
    int64_t stop_after;
};
// stages / ybuf: pipeline depth and A-image buffers, 0 = built-in choice.
bool screen_config_ok(int K, int stages, int ybuf);
bool launch_screen(int K, int topk, int mode, int stages, int ybuf, const uint16_t* Ytiles, const uint16_t* Btiles,
                   const uint16_t* Qb3,
                   const int32_t* quad_slot, float* tau0, const int32_t* tile_j0, int64_t n_tiles, int64_t G,
                   int64_t G_pad, float* cand_val, int32_t* cand_idx, int32_t* cand_count, int* status,
                   const float* Qc, const float* Qb, const float4* gnorm, const float4* alpha, const GridSpec& gs,
                   int nfit, const ListArgs& la, const WaitTest& wt, int n_sm, cudaStream_t st);
// Resolution of one mixed-path scan per screen tile (see k_resolve).
struct ResolveArgs {
    const int32_t* quad_slot;  // [n_tiles * kQuads] covariance slot of each 32-row quadrant
    const int32_t* tile_univ;
    int topk;
    const float* cval;
    const int32_t* cidx;
    const float4* alpha;
    const float4* gnorm;
    const float* Qc;
    const float* Qb;
    int64_t G_pad;
    const float* d;
    const double* centre;
    GridSpec gs;           // the grid's fit-space rows (stored or recomputed)
    int nfit;
    const double* W64;
    const float2* Wdf;     // [slots][nfit][nfit] double-float W
    const float2* centre_df;  // [nfit] double-float centre
    int32_t* cur;          // [n] covariance grid index, advanced for continuing universes
    const int32_t* pt;     // [n] true point of the universe
    const int8_t* maxit;   // [n] scan limit of the universe
    const int32_t* job_of; // [n] job of the universe
    int32_t* job_left;     // [jobs] universes of the job still running
    int32_t* best;         // [n]
    int8_t* nscan;         // [n] scans done (incremented by every decided scan)
    double* dchi2;         // [n]
    double* chi2min;       // [n] nullable
    int32_t* next;         // next active list
    int32_t* n_next;
    int32_t* fb;           // fallback list
    int32_t* n_fb;
    unsigned long long* counters;  // screened, rescored, handed on
    float* thr;            // [n] nullable: for handed-on universes, an upper bound of min_g (chi2_g - c_u)
    int2* lcount;          // [n] nullable, list rounds: half-row counts of an overflowing universe
    const int64_t* list_off;  // [n] nullable: exact-size list storage (see ListArgs)
    const int2* list_n;
    uint8_t* rmask;        // [n] nullable: bit of the round that decided each universe's scan, OR-ed in
    uint8_t round_bit;     // that bit; 0 = the top-k round (certificate alone or after rescoring)
    // top-k rounds: residual work lists of the flat resolution (launch_resolve), sized by the caller:
    // items/res [n_tiles * BM * (topk + 1)], item_base [n_tiles * BM], items2/res2/cmin2
    // [n_tiles * BM], tile_items / tile_items2 [n_tiles * kQuads], counts [2] (zeroed by launch_resolve)
    int2* items;           // (tile row, grid index; -1 = the centre, for c_u)
    double* res;           // residual chi2 of each item
    int32_t* item_base;    // first item of each tile row
    int2* items2;          // chi2_p of the rescored rows that finish: (tile row, true point)
    double* res2;
    double* cmin2;         // their chi2_min
    int32_t* counts;       // [0] items, [1] items2
    int2* tile_items;      // (first item, item count) of each quadrant's items (a quadrant shares one W)
    int2* tile_items2;     // the same for items2
    unsigned long long* n_resid;  // residual chi2 evaluated (all rounds)
    int n_sm;
};
// Bits of a universe's round record (the FC_DECIDED_* values of fc.h).
constexpr uint8_t kDecidedCert = 1, kDecidedRescored = 2, kDecidedTop16 = 4, kDecidedList = 8,
                  kDecidedExactList = 16, kDecidedScan = 32, kDecidedPlain = 64;
// rmask[list[i]] |= bit for the universes of a list
void launch_or_mask(const int32_t* list, int64_t n, uint8_t bit, uint8_t* rmask, cudaStream_t st);
// tau0[row] = min(tau0[row], thr[u]) for the rows of the tiles
void launch_min_tau(const int32_t* tile_univ, int64_t n_tiles, const float* thr, float* tau0, cudaStream_t st);
// Third round: binary64 residual chi2 of every listed candidate of each row
// (complete lists certify the minimum); overflowing rows go to `fb`.
// list rounds: n_rows = universes in the round's tiles; rows [n_tiles * BM] and n_rows_dev are scratch
// Work split of a list round: chunks of kListChunk listed points of one row.
constexpr int kListChunk = 32;
struct ListPlan {
    int2* chunk;        // [max_chunks] (listed-row index w, chunk k of that row); w < 0: no work
    int32_t* n_chunk;   // device count of chunks
    int32_t* row_base;  // [n_rows] first chunk of row w
    int32_t* row_nc;    // [n_rows] chunks of row w (0: the row has no list work)
    int32_t* row_done;  // [n_rows] chunks of row w finished
    double* pv;         // [max_chunks] chunk minimum
    int32_t* pg;        // [max_chunks] its grid index
    int64_t max_chunks;
};
void launch_resolve_list(const ResolveArgs& a, const int32_t* cand_count, int64_t n_tiles, int64_t n_rows,
                         int32_t* rows, int32_t* n_rows_dev, const ListPlan& lp, cudaStream_t st);
void launch_resolve(const ResolveArgs& a, int64_t n_tiles, cudaStream_t st);

// ---- final residual-form chi2 and dchi2 ----
// Per-universe state of a scan: cur (covariance index), pt (true point),
// nscan (scans done), maxit (limit), job_of / job_left (completion counting).
struct UniverseState {
    int32_t* cur;
    const int32_t* pt;
    int8_t* nscan;
    const int8_t* maxit;
    const int32_t* job_of;
    int32_t* job_left;
};
// Wdf given: the mixed path's double-float residuals; null: binary64 (plain path)
void launch_finish(const int32_t* list, int64_t n, const int32_t* uslot_of_list, const int32_t* best,
                   const UniverseState& us, const float* d, const GridSpec& gs, int nfit, const double* W64,
                   const float2* Wdf, double* dchi2, double* chi2min, cudaStream_t st);
// advance: converged / exhausted universes -> finish list, others stay active
void launch_advance(const int32_t* active, int64_t n_active, const int32_t* best, const UniverseState& us,
                    int32_t* next_active, int32_t* n_next, int32_t* finish_list, int32_t* n_finish, cudaStream_t st);

// ---- peak probes: FP64 / FP32 fma rates of this device (TFLOP/s) ----
bool measure_fma_peaks(int n_sm, double* fp64_tflops, double* fp32_tflops, cudaStream_t st);

// ---- quantiles ----
void launch_quantiles(double* x, int rows, int n, const double* probs, int nq, double* out, cudaStream_t st);
// The shape model's sine table (m.sinT, rows rows of m.nf), from the bins' L and E.
void launch_osc_sin(const SpecModel& m, int rows, const double* L, const double* E, double* sinT, cudaStream_t st);
// Full-bin spectra of the model into S [G][nf] (S null: only checked); bad counts
// entries that are not finite and >= 0.
void launch_osc_spectra(const SpecModel& m, int64_t G, double* S, int* bad, cudaStream_t st);
// counts[r] += #{u : x[r][u] < thr[r]} for rows r < rows of x [rows][n]
void launch_count_below(const double* x, int rows, int n, const double* thr, int64_t* counts, cudaStream_t st);

}  // namespace fcdev
