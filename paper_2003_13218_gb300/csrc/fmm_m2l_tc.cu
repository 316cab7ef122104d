// fmm_m2l_tc.cu -- M2L of Eq. Lcoeffdef on the 5th-generation tensor cores
// (tcgen05) for the mixed-precision path.
//
// For one level and one parity class c, the local coefficients of 128 target
// cells (a brick of parent coordinates) are
//     L[t][j] = sum_{delta in IL(c)} sum_k M[t + delta][k] T_delta[k][j]
// i.e. 189 dense products (128 x K) . (K x N):
//   M dimension = 128 targets, N = (p+1)^2 output coefficients padded to 16,
//   K = (p+1)^2 input coefficients padded to 16 (rows stored padded to a whole copy box).
// The A operand of offset delta is the same brick shifted to class
// (c + delta) & 1 and parent offset (c + delta) >> 1 in {-1, 0, 1}^3; the
// source planes carry a one-cell periodic halo so that every TMA box lies
// inside the array.  Operands are split into bf16 terms, x = x0 + x1 (+ x2),
// and the products x_i y_j with i + j below the split order are summed
// (bf16x3: 6 products, ~2^-24 relative; bf16x2: 3 products, ~2^-16).
//
// fp16x2 split.  fp16 keeps 11 significant bits, so two terms give ~2^-22
// with 3 products, but its range is narrow.  The moments and operators are
// therefore balanced first: with s(n,m) = sqrt((n+m)! (n-m)!),
//     M~ = M^ s(n,m) gM,   T~[k][j] = T[k][j] / (s(k) s(j)) gT,   L^ = L~ s(j) / (gM gT).
// Because |P_n^m| <= sqrt((n+m)!/(n-m)!) and binomial coefficients are at
// most 2^N, |T~| <= 2^N / |delta|^(N+1) <= 1/2 for well-separated cells
// (|delta| >= 2 cells), and |M~| is bounded by the absolute charge of the
// cell.  gT = 2^14 and gM = 2^(14 - E), E the binary exponent of the level's
// largest |M^ s|, put both operands' largest entries at 2^13..2^15, far below
// fp16's 65504 and far above its subnormal range.
//
// The operand rows are stored padded to whole copy boxes (32 K elements = 64
// bytes for the bf16 splits, 64 = 128 bytes for the fp16 split, whose 2-term
// stages still fit twice in shared memory and move in half as many requests),
// but the MMAs stop at K = (p+1)^2 padded to 16.
//
// Degree grading (fp16 split, FMM_OPT_M2L_GRADE = D2 | D1 << 8).  The smaller
// product terms matter less for the higher input degrees: a K chunk whose
// lowest degree is >= D1 takes the one product x0 y0 (two such chunks share a
// pipeline stage), and in a 3-product chunk the K16 steps whose lowest degree
// reaches D2 drop x1 y0 (one compile-time MMA sequence per split point).  The
// defaults D2 = 4, D1 = 8 give 16 K16 MMA steps per offset at p = 12 instead
// of 33.
//
// Accumulation.  The tensor core's FP32 accumulation rounds with a bias, which
// over thousands of MMAs into one accumulator shows up at the 1e-5 level.  So
// the products of a short run of offsets (FMM_OPT_M2L_ACC_GROUP, default 2) go
// into a fresh TMEM accumulator (two, alternating), and the epilogue warps
// drain it and add it to the row held in FP32 registers (round to nearest)
// while the tensor core works on the next run.
//
// Roles (6 warps): warp 0 lane 0 issues TMA loads into a 2..6-stage ring, warp 1
// lane 0 issues tcgen05.mma, warps 2..5 drain TMEM (warp w reads TMEM lanes
// 32 (w mod 4) .. +31, one target row per thread) and write the FP32 level
// array.  Every mbarrier wait is bounded (globaltimer); on a timeout the
// kernel records FMM_ERR_TIMEOUT, waits (bounded) for its copies and MMAs in
// flight, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int TC_THREADS = 192;
constexpr int TC_MAX_STAGES = 6;
constexpr int TC_ROWS = 128;          // MMA M
// Operand rows in shared memory are SW = 64 (bf16 splits) or 128 (fp16 split)
// bytes wide, swizzled with the matching pattern: one copy box carries SW / 2
// K elements of 128 (A) or npad (B) rows.
constexpr int kchunk_of(int sw) { return sw / 2; }
constexpr uint32_t TMEM_COLS = 512;   // two accumulators of up to 256 columns
constexpr int TC_PMAX = 15;           // N = (p+1)^2 rounded to 16 must not exceed 256
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s: the teardown's own limit (and the default budget)
constexpr int GAIN_T_EXP = 14;        // gT = 2^14 (fp16 split)
constexpr int GAIN_M_EXP = 14;        // gM = 2^(14 - E)
constexpr size_t TC_SMEM_BUDGET = 224 * 1024;

// operator slots of the B tables: the noff(ws) M2L offsets, then M2M and L2L per child octant

struct TcState {
    bool f16 = false;               // fp16x2 split with balanced scaling (and tensor-core translations)
    int pa = 0, pb = 0;             // terms of the plan's split
    int parts = 0;                  // terms stored (3 for the bf16 splits: the solute pass uses 3 x 3)
    int npad = 0, kp = 0;
    int noff = 0;                   // M2L operator slots (the slot cube of the plan's ws)
    int sw = 64;                    // bytes per swizzled operand row in shared memory
    uint16_t *planes[9] = {};       // bf16 or fp16 bit patterns
    size_t part_elems[9] = {};
    uint16_t *ops = nullptr;
    size_t ops_part_elems = 0;
    bool ops_borrowed = false;      // ops belongs to another plan's state (tc_share_operators)
    CUtensorMap mapA[9][3];
    CUtensorMap mapB[3];
    CUtensorMap mapB2[2];           // fp16: operator tiles boxed N/2 rows (one half per CTA of a pair)
    CUtensorMap mapL[9][2];         // fp16: parent-level local expansions for the fused L2L of level l
    uint16_t *planesL = nullptr;    // natural order [part][z][y][x][kp], sized for level d - 1
    size_t partL_elems = 0;
    int bx[9], by[9], bz[9];
    int groups[9], per_group[9];    // offset groups per tile (small levels run more CTAs)
    int mgroups[9], mper_group[9];  // the same for the M2M into level l
    float *Lpart = nullptr;         // partial sums of the offset groups
    float *s32 = nullptr;           // [nc] s(n,m) per real coefficient (fp16 split)
    float *s32inv = nullptr;        // [nc] 1 / s(n,m)
    double *s64 = nullptr;
    unsigned *amax = nullptr;       // [9] bits of the largest |M^ s| per level (fp16 split)
    unsigned *amaxL = nullptr;      // [9] bits of the largest |L^ / s| per level
};

struct TcArgs {
    int mode;               // 0: M2L (+ fused L2L), 1: M2M
    int np, bx, by, bz, rows, tiles_x, tiles_y, tiles_per_class;
    int nc, npad, kchunks, ksteps, stages;
    int groups, per_group;  // the offsets split over `groups` CTAs per tile (small levels)
    int n_off;              // offsets: 189 (+1 with the fused L2L) or 8 (M2M)
    int src_np2;            // M2M: halo'd side of the child level's planes
    int ws, n_il, noff;     // well-separatedness, interaction-list length, M2L operator slots
    int out_np;             // M2M: class-layout side of the parent level (0 at level 0)
    uint32_t idesc;
    uint32_t gchunks;       // fp16x2 M2L offsets: products per K chunk, 2 bits per chunk (0 = all 3), FMM_OPT_M2L_GRADE
    uint32_t gsteps;        // in a 3-product chunk, the first K16 step from which x1 y0 is dropped, 3 bits per chunk
                            // (0: none)
    int acc_group;          // offsets summed in one TMEM accumulator before it is drained (>= 1)
    uint64_t wait_ns;       // budget of every pipeline wait (FMM_OPT_WAIT_BUDGET_NS); the teardown keeps its own
    int inject_stall;       // test hook (single-CTA kernel): the MMA issuer first waits on a barrier nothing arrives on
    float *L;               // output level array (L of the level, or M of the parent level)
    float *Lpart;           // [groups][level cells][nc] partial sums when groups > 1
    const float *post;      // fp16 split: s(j) (M2L) or 1 / s(j) (M2M) per output coefficient, else null
    const unsigned *amax;   // fp16 split: largest |M^ s| of the A planes (gM follows from it)
    const unsigned *amaxL;  // fused L2L: largest |L^ / s| of the parent planes (gL), else null
    unsigned *amax_out;     // fp16 split, one offset group: fold max_i |out_i sx(i)| of the written rows in here
    const float *sx;        // with amax_out: s(i) (M2M output, |M^ s|) or 1 / s(i) (M2L output, |L^ / s|)
    int *err;
};

// 2^e as a float for |e| <= 126, built from its bits
__host__ __device__ inline float pow2f(int e)
{
    e = e < -126 ? -126 : (e > 126 ? 126 : e);
    union {
        uint32_t u;
        float f;
    } v;
    v.u = (uint32_t)(e + 127) << 23;
    return v.f;
}

// binary exponent E of a positive float given by its bits (value in [2^E, 2^(E+1)))
__device__ inline int exp_of_bits(unsigned bits) { return (int)((bits >> 23) & 0xFFu) - 127; }

// gM = 2^(GAIN_M_EXP - E), 1 when the level has no moments; kept within 2^+-100
__device__ inline int gain_m_exp(unsigned bits)
{
    if (bits == 0u) return 0;
    const int e = GAIN_M_EXP - exp_of_bits(bits);
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Products of K chunk kc of a graded M2L offset: x0 y0 (+ x0 y1 (+ x1 y0)), 2 bits per chunk (0 = all 3).
__device__ __forceinline__ int chunk_products(uint32_t g, int kc)
{
    const int c = (int)((g >> (2 * kc)) & 3u);
    return c == 0 ? 3 : c;
}

// First K16 step of chunk kc (a 3-product chunk) whose lowest input degree reaches D2: from there on the
// chunk drops x1 y0 (0: no such step).
__device__ __forceinline__ int step_split(uint32_t gs, int kc) { return (int)((gs >> (3 * kc)) & 7u); }

// A graded offset's stages: two consecutive chunks of one product each (x0 y0 only) share one stage, their
// A0 / B0 boxes in the places of the two terms; returns how many chunks the stage starting at kc covers.
__device__ __forceinline__ int stage_chunks(uint32_t g, int kc, int kchunks)
{
    return (chunk_products(g, kc) == 1 && kc + 1 < kchunks && chunk_products(g, kc + 1) == 1) ? 2 : 1;
}

// Accumulation groups of one CTA's offsets: the M2L (or M2M) offsets, local indices 0 .. nm - 1, in runs
// of G that share one TMEM accumulator; the fused L2L offset (when present it is the CTA's last) alone,
// since its drain is scaled by gM / gL.
struct AccGroups {
    int nm, ng, G;
    __device__ AccGroups(int nloc, bool has_l2l, int g) : nm(nloc - (has_l2l ? 1 : 0)), ng(0), G(g < 1 ? 1 : g)
    {
        ng = (nm + G - 1) / G + (has_l2l ? 1 : 0);
    }
    __device__ int begin(int g) const { return g * G < nm ? g * G : nm; }
    __device__ int end(int g) const { return g * G < nm ? min((g + 1) * G, nm) : nm + 1; }
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on phase `parity`; false after limit_ns or when the CTA aborts
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint64_t limit_ns = WAIT_LIMIT_NS)
{
    if (mbar_try(bar, parity)) return true;  // the usual case: no clock read
    uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 63) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, SW-byte swizzle (layout
// code 4 for 64 bytes, 2 for 128 bytes), 8-row groups 8 SW bytes apart
// (stride byte offset), version field 1.
template <int SW>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(((8u * SW) >> 4) & 0x3FFFu) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version
    d |= (uint64_t)(SW == 128 ? 2 : 4) << 61;            // swizzle mode
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Lr[i] += fac * accumulator column i of this warp's 32 TMEM lanes, i < 16 NCH; the loads go out in
// batches of 16-column pieces before one wait, as many as the registers left beside Lr allow
template <int NCH>
__device__ __forceinline__ void drain_accumulator(uint32_t taddr, float fac, float (&Lr)[NCH * 16])
{
    constexpr int DRAIN_BATCH = NCH * 16 + 64 <= 240 ? 4 : (NCH * 16 + 32 <= 240 ? 2 : 1);
#pragma unroll
    for (int c0 = 0; c0 < NCH; c0 += DRAIN_BATCH) {
        uint32_t r[DRAIN_BATCH][16];
#pragma unroll
        for (int c = 0; c < DRAIN_BATCH; ++c)
            if (c0 + c < NCH) tmem_ld16(taddr + (uint32_t)((c0 + c) * 16), r[c]);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < DRAIN_BATCH; ++c)
            if (c0 + c < NCH)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    Lr[(c0 + c) * 16 + j] = fmaf(__uint_as_float(r[c][j]), fac, Lr[(c0 + c) * 16 + j]);
    }
}

// Rows r0 .. r0 + 31 (those below `rows`) of the staged output tile (row stride srow in shared memory) to
// out + idx(r) nc, idx(r) held by lane r - r0: one warp, coalesced stores, four rows in flight
template <int NCH>
__device__ __forceinline__ void store_rows(const float *stage, int srow, int r0, int rows, int64_t my_idx, float *out,
                                           int nc, int lane)
{
#pragma unroll 1
    for (int r = 0; r < 32; r += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t di = __shfl_sync(0xffffffffu, my_idx, r + u);
            if (r0 + r + u < rows) {
                float *dst = out + di * nc;
                const float *src = stage + (r0 + r + u) * srow;
#pragma unroll
                for (int c = 0; c < NCH * 16; c += 32)
                    if (c + lane < nc) dst[c + lane] = src[c + lane];
            }
        }
    }
}

// The warp's rows r0 .. r0 + 31 (those below `rows`), lane r - r0 holding row r in x, to out + idx(r) nc,
// idx(r) held by lane r - r0, without shared memory: each 32 x 32 block of columns is transposed across
// the warp by a 5-step butterfly of shuffles (step m swaps the m-wide off-diagonal blocks between lanes
// l and l ^ m), after which lane l holds column 32 b + l of all 32 rows and every store is coalesced.
template <int NCH>
__device__ __forceinline__ void store_rows_shfl(float (&x)[NCH * 16], int64_t my_idx, int r0, int rows, float *out,
                                                int nc, int lane)
{
    constexpr int C = NCH * 16;
#pragma unroll
    for (int b = 0; b < (C + 31) / 32; ++b) {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 32 * b + k < C ? x[32 * b + k] : 0.f;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            const bool up = (lane & m) != 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j & m) continue;
                const float recv = __shfl_xor_sync(0xffffffffu, up ? v[j] : v[j | m], m);
                if (up) v[j] = recv;
                else v[j | m] = recv;
            }
        }
        const int col = 32 * b + lane;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t di = __shfl_sync(0xffffffffu, my_idx, k);
            if (r0 + k < rows && col < nc) out[di * nc + col] = v[k];
        }
    }
}

// ---- CTA pair (cluster of 2) helpers for the 2-SM MMA
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the object at local shared address `a` in CTA `rank`
__device__ __forceinline__ uint32_t map_shared(uint32_t a, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// bounded wait with cluster-scope acquire (barriers that receive arrivals from the peer CTA)
__device__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                  uint64_t limit_ns = WAIT_LIMIT_NS)
{
    uint32_t ok0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok0)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok0) return true;  // the usual case: no clock read
    uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 63) == 63) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > limit_ns) return false;
        }
    }
}

// arrive on an mbarrier of the peer CTA (shared::cluster address)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// TMA loads into this CTA's shared memory whose completion is counted on the
// pair leader's mbarrier (`bar` a shared::cluster address)
__device__ __forceinline__ void tma_load_4d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                                 int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                                 int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// 2-SM MMA: D (128 lanes in each CTA's TMEM) += A (128 rows per CTA) . B (N/2 rows per CTA)
__device__ __forceinline__ void mma_f16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on the mbarrier at local offset `bar` in both CTAs of the pair once
// every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit_pair(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((uint16_t)3)
        : "memory");
}

// ------------------------------------------------------------------ the kernel
template <int PA, int PB>
struct Products;
template <>
struct Products<3, 3> {  // x_i y_j with i + j <= 2
    static constexpr int n = 6;
    __device__ static constexpr int a(int k) { return k == 0 ? 0 : k == 1 ? 0 : k == 2 ? 1 : k == 3 ? 0 : k == 4 ? 1 : 2; }
    __device__ static constexpr int b(int k) { return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 0 : k == 3 ? 2 : k == 4 ? 1 : 0; }
};
template <>
struct Products<2, 2> {  // i + j <= 1
    static constexpr int n = 3;
    __device__ static constexpr int a(int k) { return k == 2 ? 1 : 0; }
    __device__ static constexpr int b(int k) { return k == 1 ? 1 : 0; }
};
// moments in 2 terms, operator in 3: x0 y0, x0 y1, x1 y0, x0 y2.  The operator
// (the same table for every cell) keeps ~2^-24; the dropped products involve
// the moments' residual, whose error differs from cell to cell.
template <>
struct Products<2, 3> {
    static constexpr int n = 4;
    __device__ static constexpr int a(int k) { return k == 2 ? 1 : 0; }
    __device__ static constexpr int b(int k) { return k == 1 ? 1 : k == 3 ? 2 : 0; }
};

// The MMAs of one K chunk: the first NP products over the chunk's nk valid K16 steps (the third, x1 y0, only
// on steps below S2), straight-line code (operand addresses are compile-time offsets from the stage bases);
// `first` starts a new accumulator.
template <int NP, typename PR, int K16, int SW, bool PAIR, int S2 = K16>
__device__ __forceinline__ void issue_chunk(uint32_t tmem_d, uint32_t a0, uint32_t b0, uint32_t stageA, uint32_t stageB,
                                            int nk, uint32_t idesc, bool first)
{
    // descriptors of the stage bases once; an operand at byte offset o from a base is the base's descriptor
    // plus o / 16 in the address field (14 bits of 16-byte units: shared-memory addresses stay below 2^18,
    // so the sum never carries out of the field)
    const uint64_t ad0 = sdesc<SW>(a0), bd0 = sdesc<SW>(b0);
    const uint64_t sa = stageA >> 4, sb = stageB >> 4;
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
#pragma unroll
        for (int k16 = 0; k16 < K16; ++k16) {
            if (k16 >= nk) continue;         // zero fill beyond K
            if (pr == 2 && k16 >= S2) continue;  // steps of degree >= D2: x0 y0 + x0 y1 only
            const uint64_t ad = ad0 + (uint64_t)PR::a(pr) * sa + (uint64_t)(k16 * 2);
            const uint64_t bd = bd0 + (uint64_t)PR::b(pr) * sb + (uint64_t)(k16 * 2);
            const uint32_t acc = (first && pr == 0 && k16 == 0) ? 0u : 1u;
            if (PAIR) mma_f16_pair(tmem_d, ad, bd, idesc, acc);
            else mma_bf16(tmem_d, ad, bd, idesc, acc);
        }
    }
}

// The MMAs of a merged stage: chunk kc0 + t in term place t (t = 0, 1), product x0 y0 only; nk1 valid
// K16 steps in the second chunk.
template <int K16, int SW, bool PAIR>
__device__ __forceinline__ void issue_merged(uint32_t tmem_d, uint32_t a0, uint32_t b0, uint32_t stageA,
                                             uint32_t stageB, int nk1, uint32_t idesc, bool first)
{
    const uint64_t ad0 = sdesc<SW>(a0), bd0 = sdesc<SW>(b0);  // stepped as in issue_chunk
    const uint64_t sa = stageA >> 4, sb = stageB >> 4;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
#pragma unroll
        for (int k16 = 0; k16 < K16; ++k16) {
            if (t == 1 && k16 >= nk1) continue;
            const uint64_t ad = ad0 + (uint64_t)t * sa + (uint64_t)(k16 * 2);
            const uint64_t bd = bd0 + (uint64_t)t * sb + (uint64_t)(k16 * 2);
            const uint32_t acc = (first && t == 0 && k16 == 0) ? 0u : 1u;
            if (PAIR) mma_f16_pair(tmem_d, ad, bd, idesc, acc);
            else mma_bf16(tmem_d, ad, bd, idesc, acc);
        }
    }
}

// A chunk with all of the split's products, x1 y0 dropped from step s2 on (s2 = 0: on no step): one
// compile-time variant per split point
template <typename PR, int K16, int SW, bool PAIR>
__device__ __forceinline__ void issue_full_chunk(int s2, uint32_t tmem_d, uint32_t a0, uint32_t b0, uint32_t stageA,
                                                 uint32_t stageB, int nk, uint32_t idesc, bool first)
{
    if constexpr (PR::n == 3 && K16 == 4) {
        if (s2 == 1) return issue_chunk<3, PR, K16, SW, PAIR, 1>(tmem_d, a0, b0, stageA, stageB, nk, idesc, first);
        if (s2 == 2) return issue_chunk<3, PR, K16, SW, PAIR, 2>(tmem_d, a0, b0, stageA, stageB, nk, idesc, first);
        if (s2 == 3) return issue_chunk<3, PR, K16, SW, PAIR, 3>(tmem_d, a0, b0, stageA, stageB, nk, idesc, first);
    }
    issue_chunk<PR::n, PR, K16, SW, PAIR>(tmem_d, a0, b0, stageA, stageB, nk, idesc, first);
}

// One CTA sums, for 128 target rows, the products of a list of offsets:
//   mode 0 (M2L): the 189 interaction-list offsets of parity class `cls`, A
//     from the halo'd source planes of the level; with fused L2L (fp16 split)
//     a 190th offset whose A is the parent level's local expansion at the
//     targets' parents (natural-order planes) and whose B is the L2L operator
//     of child octant `cls`; its accumulator is scaled by gM / gL.
//   mode 1 (M2M): the 8 child octants o, A from class plane o of the child
//     level's planes at the targets' own coordinates, B the M2M operator of o;
//     targets are a brick of the parent level in natural order, written to its
//     class layout.
// PA, PB: terms of the A and B operands; NCH: output coefficients / 16 (the
// accumulator width held in registers); SW: bytes per swizzled operand row.
template <int PA, int PB, int NCH, int SW>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
             const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB0,
             const __grid_constant__ CUtensorMap mB1, const __grid_constant__ CUtensorMap mB2,
             const __grid_constant__ CUtensorMap mL0, const __grid_constant__ CUtensorMap mL1, TcArgs a)
{
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[TC_MAX_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[TC_MAX_STAGES];
    __shared__ __align__(8) uint64_t bar_tfull[2];
    __shared__ __align__(8) uint64_t bar_tempty[2];
    __shared__ __align__(8) uint64_t bar_done;
    __shared__ __align__(8) uint64_t bar_never;  // test hook: initialised, never arrived on
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    __shared__ int produced_sh, consumed_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t smem0 = (smem_u32(smem_dyn) + 1023u) & ~1023u;
    constexpr int KCH = kchunk_of(SW);  // K elements per stage
    constexpr int K16 = SW / 32;        // MMAs (K = 16) per stage and product
    const uint32_t stageA = TC_ROWS * SW;
    const uint32_t stageB = (uint32_t)a.npad * SW;
    const uint32_t stage_bytes = PA * stageA + PB * stageB;
    constexpr bool kGradable = PA == 2 && PB == 2;  // the degree grading applies to the 2 x 2-term products

    // M2L: the 8 parity classes of one brick run side by side, so CTAs resident
    // at the same time read overlapping shifted bricks, which stay in L2
    const int grp = blockIdx.x % a.groups;
    const int cls = a.mode == 0 ? (blockIdx.x / a.groups) & 7 : 0;
    const int tile = a.mode == 0 ? (blockIdx.x / a.groups) >> 3 : blockIdx.x / a.groups;
    const int o_begin = grp * a.per_group;
    const int o_end = o_begin + a.per_group < a.n_off ? o_begin + a.per_group : a.n_off;
    const int nloc = o_end > o_begin ? o_end - o_begin : 0;
    const bool has_l2l = a.mode == 0 && a.n_off > a.n_il && a.n_il >= o_begin && a.n_il < o_end;
    const AccGroups groups(nloc, has_l2l, a.acc_group);
    const int x0 = (tile % a.tiles_x) * a.bx;
    const int y0 = ((tile / a.tiles_x) % a.tiles_y) * a.by;
    const int z0 = (tile / (a.tiles_x * a.tiles_y)) * a.bz;
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = (cls >> 2) & 1;
    const int np2 = a.np + 2 * a.ws;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_tfull[b]), 1);
            mbar_init(smem_u32(&bar_tempty[b]), 4);  // one arrival per epilogue warp
        }
        mbar_init(smem_u32(&bar_done), 1);
        mbar_init(smem_u32(&bar_never), 1);
        abort_sh = 0;
        produced_sh = 0;
        consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_sh;
    volatile int *abort_flag = &abort_sh;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: TMA loads of the A brick and the B operator
            const CUtensorMap *mA[3] = {&mA0, &mA1, &mA2};
            const CUtensorMap *mL[3] = {&mL0, &mL1, &mL1};
            const CUtensorMap *mB[3] = {&mB0, &mB1, &mB2};
            int it = 0, s = 0;
            uint32_t round = 0;
            bool ok = true;
            // all K chunks of one offset: A from maps `src` at (c1, c2, c3), B at operator slot `oslot`; a
            // graded (M2L) offset copies only the terms its chunk's products read
            auto load_offset = [&](const CUtensorMap *const *src, int c1, int c2, int c3, int oslot, bool graded) {
                for (int kc = 0; kc < a.kchunks && ok;) {
                    if (it >= a.stages &&
                        !mbar_wait(smem_u32(&bar_empty[s]), (round & 1u) ^ 1u, abort_flag, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_full[s]);
                    const uint32_t base = smem0 + (uint32_t)s * stage_bytes;
                    const int nkc = (kGradable && graded) ? stage_chunks(a.gchunks, kc, a.kchunks) : 1;
                    if (nkc == 2) {  // two x0 y0 chunks: A0 and B0 of chunk kc + t in term place t
                        mbar_expect_tx(full, 2u * ((uint32_t)(a.rows * SW) + stageB));
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            tma_load_4d(base + t * stageA, src[0], full, (kc + t) * KCH, c1, c2, c3);
                            tma_load_3d(base + PA * stageA + t * stageB, mB[0], full, (kc + t) * KCH, 0, oslot);
                        }
                    } else {
                        int na = PA, nb = PB;
                        if (kGradable && graded) {
                            const int np = chunk_products(a.gchunks, kc);
                            na = np == 3 ? 2 : 1;
                            nb = np >= 2 ? 2 : 1;
                        }
                        mbar_expect_tx(full, (uint32_t)(na * a.rows * SW) + (uint32_t)nb * stageB);
#pragma unroll
                        for (int i = 0; i < PA; ++i)
                            if (i < na) tma_load_4d(base + i * stageA, src[i], full, kc * KCH, c1, c2, c3);
#pragma unroll
                        for (int j = 0; j < PB; ++j)
                            if (j < nb) tma_load_3d(base + PA * stageA + j * stageB, mB[j], full, kc * KCH, 0, oslot);
                    }
                    kc += nkc;
                    ++it;
                    if (++s == a.stages) {
                        s = 0;
                        ++round;
                    }
                }
            };
            if (a.mode == 0) {
                int oi = -1;  // position of the offset in the interaction-list order
                // delta per axis in [-2 ws - c, 2 ws + 1 - c], the near (2 ws + 1)^3 block left out;
                // the source brick sits at parent offset (c + delta) >> 1 in [-ws, ws], halo width ws
                const int w = a.ws;
                for (int dz = -2 * w - cz; dz <= 2 * w + 1 - cz && ok; ++dz)
                    for (int dy = -2 * w - cy; dy <= 2 * w + 1 - cy && ok; ++dy)
                        for (int dx = -2 * w - cx; dx <= 2 * w + 1 - cx && ok; ++dx) {
                            if (dx >= -w && dx <= w && dy >= -w && dy <= w && dz >= -w && dz <= w) continue;
                            ++oi;
                            if (oi < o_begin || oi >= o_end) continue;
                            const int sx = cx + dx, sy = cy + dy, sz = cz + dz;
                            const int scls = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
                            load_offset(mA, x0 + (sx >> 1) + w, y0 + (sy >> 1) + w, scls * np2 + z0 + (sz >> 1) + w,
                                        off_slot(dx, dy, dz, w), a.gchunks != 0u);
                        }
                // fused L2L: the parents' local expansions (natural order, no halo)
                if (ok && a.n_off > a.n_il && a.n_il >= o_begin && a.n_il < o_end)
                    load_offset(mL, x0, y0, z0, a.noff + 8 + cls, false);
            } else {
                for (int o = o_begin; o < o_end && ok; ++o)
                    load_offset(mA, x0 + a.ws, y0 + a.ws, o * a.src_np2 + z0 + a.ws, a.noff + o, false);
            }
            produced_sh = it;
            if (!ok) {
                abort_sh = 1;
                atomicOr(a.err, ERRF_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: one fresh accumulator per group of offsets
            using PR = Products<PA, PB>;
            int it = 0, s = 0;
            uint32_t round = 0;
            // the test hook makes this thread's first wait run out (its budget), as a lost copy would
            bool ok = !(a.inject_stall && !mbar_wait(smem_u32(&bar_never), 0, abort_flag, a.wait_ns));
            for (int g = 0; g < groups.ng && ok; ++g) {
                const int acc = g & 1;
                const uint32_t use = (uint32_t)(g >> 1);
                if (g >= 2 && !mbar_wait(smem_u32(&bar_tempty[acc]), (use - 1u) & 1u, abort_flag, a.wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t tmem_d = tmem + (uint32_t)(acc * 256);
                bool first = true;  // the group's first MMA overwrites the accumulator
                for (int o = groups.begin(g); o < groups.end(g) && ok; ++o) {
                    const bool graded =
                        kGradable && (a.gchunks | a.gsteps) != 0u && a.mode == 0 && o_begin + o < a.n_il;
                    for (int kc = 0; kc < a.kchunks;) {
                        if (!mbar_wait(smem_u32(&bar_full[s]), round & 1u, abort_flag, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t base = smem0 + (uint32_t)s * stage_bytes;
                        const int nk = a.ksteps - K16 * kc < K16 ? a.ksteps - K16 * kc : K16;
                        const int np = graded ? chunk_products(a.gchunks, kc) : PR::n;
                        const int nkc = graded ? stage_chunks(a.gchunks, kc, a.kchunks) : 1;
                        if constexpr (kGradable) {
                            if (nkc == 2) {
                                const int nk1 = a.ksteps - K16 * (kc + 1) < K16 ? a.ksteps - K16 * (kc + 1) : K16;
                                issue_merged<K16, SW, false>(tmem_d, base, base + PA * stageA, stageA, stageB, nk1,
                                                             a.idesc, first);
                            } else if (np == 1)
                                issue_chunk<1, PR, K16, SW, false>(tmem_d, base, base + PA * stageA, stageA, stageB, nk,
                                                                   a.idesc, first);
                            else if (np == 2)
                                issue_chunk<2, PR, K16, SW, false>(tmem_d, base, base + PA * stageA, stageA, stageB, nk,
                                                                   a.idesc, first);
                            else
                                issue_full_chunk<PR, K16, SW, false>(graded ? step_split(a.gsteps, kc) : 0, tmem_d, base,
                                                                     base + PA * stageA, stageA, stageB, nk, a.idesc,
                                                                     first);
                        } else {
                            issue_chunk<PR::n, PR, K16, SW, false>(tmem_d, base, base + PA * stageA, stageA, stageB, nk,
                                                                   a.idesc, first);
                        }
                        first = false;
                        kc += nkc;
                        mma_commit(smem_u32(&bar_empty[s]));
                        ++it;
                        if (++s == a.stages) {
                            s = 0;
                            ++round;
                        }
                    }
                }
                if (ok) mma_commit(smem_u32(&bar_tfull[acc]));
            }
            consumed_sh = it;
            if (!ok) {
                abort_sh = 1;
                atomicOr(a.err, ERRF_TIMEOUT);
            }
            mma_commit(smem_u32(&bar_done));  // arrives once every issued MMA has completed
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps: drain each group's accumulator into FP32 registers
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        // fused L2L offset: its A planes carry the gain gL instead of gM
        const float l2l_fac =
            a.amaxL ? pow2f(gain_m_exp(*a.amax) - gain_m_exp(*a.amaxL)) : 1.f;
        float Lr[NCH * 16];
#pragma unroll
        for (int i = 0; i < NCH * 16; ++i) Lr[i] = 0.f;
        bool ok = true;
        for (int g = 0; g < groups.ng; ++g) {
            const int acc = g & 1;
            const uint32_t use = (uint32_t)(g >> 1);
            if (!mbar_wait(smem_u32(&bar_tfull[acc]), use & 1u, abort_flag, a.wait_ns)) {
                ok = false;
                break;
            }
            fence_after();
            const float fac = (has_l2l && g == groups.ng - 1) ? l2l_fac : 1.f;
            drain_accumulator<NCH>(tmem + (uint32_t)(acc * 256) + ((uint32_t)(quad * 32) << 16), fac, Lr);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[acc]));
        }
        float mx = 0.f;  // largest |out_i sx(i)| of this thread's row (a.amax_out)
        if (!__all_sync(0xffffffffu, ok)) {
            abort_sh = 1;
            if (lane == 0) atomicOr(a.err, ERRF_TIMEOUT);
        } else {
            // every MMA has completed, so the stage ring is idle: the rows go through shared memory (stride
            // srow, odd) and leave in coalesced stores, a warp per 32 rows
            float *stage = reinterpret_cast<float *>(smem_dyn + (smem0 - smem_u32(smem_dyn)));
            const int srow = a.nc | 1;
            if (row < a.rows) {
                // with the fp16 split undo the balancing: x^ = x~ post(j) / (gM gT)
                const float g = a.post ? pow2f(-gain_m_exp(__ldcg(a.amax)) - GAIN_T_EXP) : 1.f;
#pragma unroll
                for (int i = 0; i < NCH * 16; ++i)
                    if (i < a.nc) {
                        const float v = a.post ? Lr[i] * (__ldg(a.post + i) * g) : Lr[i];
                        stage[row * srow + i] = v;
                        if (a.amax_out) mx = fmaxf(mx, fabsf(v * __ldg(a.sx + i)));
                    }
            }
            const int64_t np = a.np;
            const int64_t level_cells = a.mode == 0 ? 8 * np * np * np : np * np * np;
            float *out = a.groups == 1 ? a.L : a.Lpart + (int64_t)grp * level_cells * a.nc;
            const int tx = row % a.bx, ty = (row / a.bx) % a.by, tz = row / (a.bx * a.by);
            int64_t my_idx;
            if (a.mode == 0) {
                my_idx = (int64_t)cls * np * np * np + (x0 + tx) + np * ((y0 + ty) + np * (int64_t)(z0 + tz));
            } else {
                // natural coordinates of the parent level -> its class layout
                const int px = x0 + tx, py = y0 + ty, pz = z0 + tz;
                const int64_t on = a.out_np;
                my_idx = on == 0 ? 0
                                 : (int64_t)((px & 1) | ((py & 1) << 1) | ((pz & 1) << 2)) * on * on * on + (px >> 1) +
                                       on * ((py >> 1) + on * (int64_t)(pz >> 1));
            }
            __syncwarp();
            store_rows<NCH>(stage, srow, quad * 32, a.rows, my_idx, out, a.nc, lane);
        }
        if (a.amax_out) {  // the whole warp is here
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0 && mx > 0.f) atomicMax(a.amax_out, __float_as_uint(mx));
        }
    }

    // ---------------- teardown: wait (bounded) for MMAs and copies in flight, free TMEM
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int no_abort = 0;
        if (!mbar_wait(smem_u32(&bar_done), 0, &no_abort)) atomicOr(a.err, ERRF_TIMEOUT);
        if (abort_sh)
            for (int it = consumed_sh; it < produced_sh; ++it)
                mbar_wait(smem_u32(&bar_full[it % a.stages]), (uint32_t)(it / a.stages) & 1u, &no_abort);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Pair variant of mode 0 for the fp16 split (128-byte rows): a cluster of two
// CTAs computes 256 target rows, tiles 2t and 2t + 1 of one class, with 2-SM
// MMAs (M = 256).  Each CTA copies its own 128-row A brick and half of every
// operator tile (N/2 rows); the MMAs, issued by the even CTA, read both CTAs'
// shared memory and leave each CTA's 128 rows in its own TMEM, so each SM
// streams half of the operator bytes of the single-CTA kernel.
//   full[s]   even CTA only: its expect-tx covers both CTAs' copies, which all
//             complete on it
//   empty[s]  both CTAs: the even CTA's MMA commit, multicast to the pair
//   tfull[b]  both CTAs: multicast commit; tempty[b] on the even CTA counts
//             the 4 local and 4 remote epilogue warps
//   done      both CTAs: multicast commit after the last MMA
// Barriers are initialised and TMEM is allocated (collectively) only after a
// cluster barrier, and both CTAs pass a cluster barrier before the collective
// TMEM release, so neither touches the other after it has exited.
struct PairBars {
    uint64_t full[TC_MAX_STAGES];
    uint64_t empty[TC_MAX_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t done;
};

// Pipeline positions of one role thread, carried from tile to tile when a pair runs several tiles (the
// persistent sweep): stages issued, ring stage and pass, accumulator groups used.
struct PairPipe {
    int it = 0, s = 0;
    uint32_t round = 0, g = 0;
};

__device__ __forceinline__ void pair_bars_init(PairBars &b, int stages)
{
    for (int s = 0; s < stages; ++s) {
        mbar_init(smem_u32(&b.full[s]), 1);
        mbar_init(smem_u32(&b.empty[s]), 1);
    }
    for (int i = 0; i < 2; ++i) {
        mbar_init(smem_u32(&b.tfull[i]), 1);
        mbar_init(smem_u32(&b.tempty[i]), 8);  // 4 epilogue warps in each CTA
    }
    mbar_init(smem_u32(&b.done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The roles of both CTAs for pair `pair` of the launch arguments `a` (tiles 2t and 2t + 1 of one class,
// one offset group).  The ring and accumulator phases continue from `pp`; the caller commits `done` after
// its last tile.  A wait that runs out sets *abort_flag and records FMM_ERR_TIMEOUT.  `staged`: the caller
// issues no copies until every thread is done with this tile, so the epilogue may stage the output rows
// in the ring (`stage`, generic address of its start); otherwise each thread writes its row directly.
template <int NCH>
__device__ __forceinline__ void pair_tile(const CUtensorMap *mA0, const CUtensorMap *mA1, const CUtensorMap *mB0,
                                          const CUtensorMap *mB1, const CUtensorMap *mL0, const CUtensorMap *mL1,
                                          const TcArgs &a, int pair, uint32_t rank, uint32_t smem0, float *stage,
                                          bool staged, PairBars &bars, uint32_t tmem, volatile int *abort_flag,
                                          PairPipe &pp)
{
    constexpr int PA = 2, PB = 2, SW = 128;
    constexpr int KCH = kchunk_of(SW), K16 = SW / 32;
    using PR = Products<PA, PB>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool leader = rank == 0;
    const uint32_t halfN = (uint32_t)a.npad / 2;
    const uint32_t stageA = TC_ROWS * SW;
    const uint32_t stageB = halfN * SW;
    const uint32_t stage_bytes = PA * stageA + PB * stageB;

    const int grp = pair % a.groups;
    const int cls = (pair / a.groups) & 7;
    const int tile = 2 * ((pair / a.groups) >> 3) + (int)rank;
    const int o_begin = grp * a.per_group;
    const int o_end = o_begin + a.per_group < a.n_off ? o_begin + a.per_group : a.n_off;
    const int nloc = o_end > o_begin ? o_end - o_begin : 0;
    const bool has_l2l = a.n_off > a.n_il && a.n_il >= o_begin && a.n_il < o_end;
    const AccGroups groups(nloc, has_l2l, a.acc_group);
    const int x0 = (tile % a.tiles_x) * a.bx;
    const int y0 = ((tile / a.tiles_x) % a.tiles_y) * a.by;
    const int z0 = (tile / (a.tiles_x * a.tiles_y)) * a.bz;
    const int cx = cls & 1, cy = (cls >> 1) & 1, cz = (cls >> 2) & 1;
    const int np2 = a.np + 2 * a.ws;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer (both CTAs): own A brick, own half of B, completing on the leader's barrier
            const CUtensorMap *mA[2] = {mA0, mA1};
            const CUtensorMap *mL[2] = {mL0, mL1};
            const CUtensorMap *mB[2] = {mB0, mB1};
            bool ok = true;
            auto load_offset = [&](const CUtensorMap *const *src, int c1, int c2, int c3, int oslot, bool graded) {
                for (int kc = 0; kc < a.kchunks && ok;) {
                    if (pp.it >= a.stages && !mbar_wait_cluster(smem_u32(&bars.empty[pp.s]), (pp.round & 1u) ^ 1u,
                                                                abort_flag, a.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full_local = smem_u32(&bars.full[pp.s]);
                    const uint32_t full = map_shared(full_local, 0);
                    const uint32_t base = smem0 + (uint32_t)pp.s * stage_bytes;
                    const int nkc = graded ? stage_chunks(a.gchunks, kc, a.kchunks) : 1;
                    if (nkc == 2) {  // two x0 y0 chunks: A0 and B0 of chunk kc + t in term place t
                        // the leader's barrier counts both CTAs' copies (the same boxes in each)
                        if (leader) mbar_expect_tx(full_local, 2u * 2u * ((uint32_t)(a.rows * SW) + stageB));
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            tma_load_4d_pair(base + t * stageA, src[0], full, (kc + t) * KCH, c1, c2, c3);
                            tma_load_3d_pair(base + PA * stageA + t * stageB, mB[0], full, (kc + t) * KCH,
                                             (int)(rank * halfN), oslot);
                        }
                    } else {
                        int na = PA, nb = PB;
                        if (graded) {
                            const int np = chunk_products(a.gchunks, kc);
                            na = np == 3 ? 2 : 1;
                            nb = np >= 2 ? 2 : 1;
                        }
                        if (leader)
                            mbar_expect_tx(full_local, 2u * ((uint32_t)(na * a.rows * SW) + (uint32_t)nb * stageB));
#pragma unroll
                        for (int i = 0; i < PA; ++i)
                            if (i < na) tma_load_4d_pair(base + i * stageA, src[i], full, kc * KCH, c1, c2, c3);
#pragma unroll
                        for (int j = 0; j < PB; ++j)
                            if (j < nb)
                                tma_load_3d_pair(base + PA * stageA + j * stageB, mB[j], full, kc * KCH,
                                                 (int)(rank * halfN), oslot);
                    }
                    kc += nkc;
                    ++pp.it;
                    if (++pp.s == a.stages) {
                        pp.s = 0;
                        ++pp.round;
                    }
                }
            };
            int oi = -1;
            const int w = a.ws;
            for (int dz = -2 * w - cz; dz <= 2 * w + 1 - cz && ok; ++dz)
                for (int dy = -2 * w - cy; dy <= 2 * w + 1 - cy && ok; ++dy)
                    for (int dx = -2 * w - cx; dx <= 2 * w + 1 - cx && ok; ++dx) {
                        if (dx >= -w && dx <= w && dy >= -w && dy <= w && dz >= -w && dz <= w) continue;
                        ++oi;
                        if (oi < o_begin || oi >= o_end) continue;
                        const int sx = cx + dx, sy = cy + dy, sz = cz + dz;
                        const int scls = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
                        load_offset(mA, x0 + (sx >> 1) + w, y0 + (sy >> 1) + w, scls * np2 + z0 + (sz >> 1) + w,
                                    off_slot(dx, dy, dz, w), a.gchunks != 0u);
                    }
            if (ok && a.n_off > a.n_il && a.n_il >= o_begin && a.n_il < o_end)
                load_offset(mL, x0, y0, z0, a.noff + 8 + cls, false);
            if (!ok) {
                *abort_flag = 1;
                atomicOr(a.err, ERRF_TIMEOUT);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (even CTA): 256-row MMAs over both CTAs' operands
            bool ok = true;
            for (int g = 0; g < groups.ng && ok; ++g) {
                const uint32_t gg = pp.g + (uint32_t)g;
                const int acc = (int)(gg & 1u);
                const uint32_t use = gg >> 1;
                if (gg >= 2 &&
                    !mbar_wait_cluster(smem_u32(&bars.tempty[acc]), (use - 1u) & 1u, abort_flag, a.wait_ns)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t tmem_d = tmem + (uint32_t)(acc * 256);
                bool first = true;  // the group's first MMA overwrites the accumulator
                for (int o = groups.begin(g); o < groups.end(g) && ok; ++o) {
                    const bool graded = (a.gchunks | a.gsteps) != 0u && o_begin + o < a.n_il;
                    for (int kc = 0; kc < a.kchunks;) {
                        if (!mbar_wait_cluster(smem_u32(&bars.full[pp.s]), pp.round & 1u, abort_flag, a.wait_ns)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t base = smem0 + (uint32_t)pp.s * stage_bytes;
                        const int nk = a.ksteps - K16 * kc < K16 ? a.ksteps - K16 * kc : K16;
                        const int np = graded ? chunk_products(a.gchunks, kc) : PR::n;
                        const int nkc = graded ? stage_chunks(a.gchunks, kc, a.kchunks) : 1;
                        if (nkc == 2) {
                            const int nk1 = a.ksteps - K16 * (kc + 1) < K16 ? a.ksteps - K16 * (kc + 1) : K16;
                            issue_merged<K16, SW, true>(tmem_d, base, base + PA * stageA, stageA, stageB, nk1, a.idesc,
                                                        first);
                        } else if (np == 1)
                            issue_chunk<1, PR, K16, SW, true>(tmem_d, base, base + PA * stageA, stageA, stageB, nk,
                                                              a.idesc, first);
                        else if (np == 2)
                            issue_chunk<2, PR, K16, SW, true>(tmem_d, base, base + PA * stageA, stageA, stageB, nk,
                                                              a.idesc, first);
                        else
                            issue_full_chunk<PR, K16, SW, true>(graded ? step_split(a.gsteps, kc) : 0, tmem_d, base,
                                                                base + PA * stageA, stageA, stageB, nk, a.idesc, first);
                        first = false;
                        kc += nkc;
                        mma_commit_pair(smem_u32(&bars.empty[pp.s]));
                        if (++pp.s == a.stages) {
                            pp.s = 0;
                            ++pp.round;
                        }
                    }
                }
                if (ok) mma_commit_pair(smem_u32(&bars.tfull[acc]));
            }
            pp.g += (uint32_t)groups.ng;
            if (!ok) {
                *abort_flag = 1;
                atomicOr(a.err, ERRF_TIMEOUT);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps (both CTAs): drain this CTA's 128 rows
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const float l2l_fac = a.amaxL ? pow2f(gain_m_exp(__ldcg(a.amax)) - gain_m_exp(__ldcg(a.amaxL))) : 1.f;
        float Lr[NCH * 16];
#pragma unroll
        for (int i = 0; i < NCH * 16; ++i) Lr[i] = 0.f;
        bool ok = true;
        for (int g = 0; g < groups.ng; ++g) {
            const uint32_t gg = pp.g + (uint32_t)g;
            const int acc = (int)(gg & 1u);
            const uint32_t use = gg >> 1;
            if (!mbar_wait_cluster(smem_u32(&bars.tfull[acc]), use & 1u, abort_flag, a.wait_ns)) {
                ok = false;
                break;
            }
            fence_after();
            const float fac = (has_l2l && g == groups.ng - 1) ? l2l_fac : 1.f;
            drain_accumulator<NCH>(tmem + (uint32_t)(acc * 256) + ((uint32_t)(quad * 32) << 16), fac, Lr);
            fence_before();
            __syncwarp();
            if (lane == 0) {
                const uint32_t te = smem_u32(&bars.tempty[acc]);
                if (leader) mbar_arrive(te);
                else mbar_arrive_remote(map_shared(te, 0));
            }
        }
        pp.g += (uint32_t)groups.ng;
        float mx = 0.f;  // largest |out_i sx(i)| of this thread's row (a.amax_out)
        if (!__all_sync(0xffffffffu, ok)) {
            *abort_flag = 1;
            if (lane == 0) atomicOr(a.err, ERRF_TIMEOUT);
        } else if (!staged) {
            // the ring may already hold the next tile's copies: the rows are transposed across each warp in
            // registers for coalesced stores
            const float g = pow2f(-gain_m_exp(__ldcg(a.amax)) - GAIN_T_EXP);
#pragma unroll
            for (int i = 0; i < NCH * 16; ++i) {
                Lr[i] = i < a.nc ? Lr[i] * (__ldg(a.post + i) * g) : 0.f;
                if (a.amax_out && row < a.rows && i < a.nc) mx = fmaxf(mx, fabsf(Lr[i] * __ldg(a.sx + i)));
            }
            const int64_t np = a.np;
            float *out = a.groups == 1 ? a.L : a.Lpart + (int64_t)grp * 8 * np * np * np * a.nc;
            const int tx = row % a.bx, ty = (row / a.bx) % a.by, tz = row / (a.bx * a.by);
            const int64_t my_idx = (int64_t)cls * np * np * np + (x0 + tx) + np * ((y0 + ty) + np * (int64_t)(z0 + tz));
            store_rows_shfl<NCH>(Lr, my_idx, quad * 32, a.rows, out, a.nc, lane);
        } else {
            // every MMA of the tile has completed and no copy is pending, so the stage ring is idle: the rows
            // go through shared memory (stride srow, odd) and leave in coalesced stores, a warp per 32 rows
            const int srow = a.nc | 1;
            const float g = pow2f(-gain_m_exp(__ldcg(a.amax)) - GAIN_T_EXP);
            if (row < a.rows) {
#pragma unroll
                for (int i = 0; i < NCH * 16; ++i)
                    if (i < a.nc) {
                        const float v = Lr[i] * (__ldg(a.post + i) * g);
                        stage[row * srow + i] = v;
                        if (a.amax_out) mx = fmaxf(mx, fabsf(v * __ldg(a.sx + i)));
                    }
            }
            const int64_t np = a.np;
            float *out = a.groups == 1 ? a.L : a.Lpart + (int64_t)grp * 8 * np * np * np * a.nc;
            const int tx = row % a.bx, ty = (row / a.bx) % a.by, tz = row / (a.bx * a.by);
            const int64_t my_idx = (int64_t)cls * np * np * np + (x0 + tx) + np * ((y0 + ty) + np * (int64_t)(z0 + tz));
            __syncwarp();
            store_rows<NCH>(stage, srow, quad * 32, a.rows, my_idx, out, a.nc, lane);
        }
        if (a.amax_out) {  // the whole warp is here
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0 && mx > 0.f) atomicMax(a.amax_out, __float_as_uint(mx));
        }
    }
}

template <int NCH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc_pair(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                  const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
                  const __grid_constant__ CUtensorMap mL0, const __grid_constant__ CUtensorMap mL1, TcArgs a)
{
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) PairBars bars;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;

    const int warp = threadIdx.x >> 5;
    const uint32_t rank = cluster_rank();
    const uint32_t smem0 = (smem_u32(smem_dyn) + 1023u) & ~1023u;
    if (threadIdx.x == 0) {
        pair_bars_init(bars, a.stages);
        abort_sh = 0;
    }
    cluster_sync_all();  // the pair's barriers are initialised and both CTAs are running
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_sh;
    PairPipe pp;
    float *stage = reinterpret_cast<float *>(smem_dyn + (smem0 - smem_u32(smem_dyn)));
    pair_tile<NCH>(&mA0, &mA1, &mB0, &mB1, &mL0, &mL1, a, (int)(blockIdx.x >> 1), rank, smem0, stage, true, bars,
                   tmem, &abort_sh, pp);
    if (warp == 1 && (threadIdx.x & 31) == 0 && rank == 0)
        mma_commit_pair(smem_u32(&bars.done));  // arrives in both CTAs once every MMA has completed

    // ---------------- teardown: every MMA done (bounded wait), pair barrier, collective TMEM release
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int no_abort = 0;
        if (!mbar_wait_cluster(smem_u32(&bars.done), 0, &no_abort)) atomicOr(a.err, ERRF_TIMEOUT);
    }
    fence_before();
    __syncthreads();
    cluster_sync_all();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    cluster_sync_all();
}

// ------------------------------------------------------------------ operand preparation
// x = x0 + x1 (+ x2) in bf16 or fp16 terms, each term the rounding of the
// remaining residual; stored as bit patterns `stride` elements apart
template <bool F16>
__device__ __forceinline__ void split_terms(float v, int parts, uint16_t *o, size_t stride)
{
    float r = v;
    for (int i = 0; i < parts; ++i) {
        if (F16) {
            const __half t = __float2half_rn(r);
            o[i * stride] = __half_as_ushort(t);
            r -= __half2float(t);
        } else {
            const __nv_bfloat16 t = __float2bfloat16_rn(r);
            o[i * stride] = __bfloat16_as_ushort(t);
            r -= __bfloat162float(t);
        }
    }
}

// largest |M^ s(k)| of a level (fp16 split), as float bits into *amax; one
// warp per cell, lanes over the coefficients
__global__ void k_absmax(const float *__restrict__ M, int64_t ncell, int nc, const float *__restrict__ s,
                         unsigned *__restrict__ amax)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    float m = 0.f;
    for (int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell; c += warps) {
        const float *row = M + c * nc;
        for (int k = lane; k < nc; k += 32) m = fmaxf(m, fabsf(row[k] * __ldg(s + k)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > 0.f) atomicMax(amax, __float_as_uint(m));  // positive floats order as integers
}

// FP32 class-layout moments -> split planes [part][class][hz][hy][hx][k] with a
// periodic halo; rows kp wide (zero beyond nc).  fp16: balanced by s(k) gM.
// One warp per halo cell, lanes over the coefficients.
template <bool F16>
__global__ void k_split_halo(const float *__restrict__ M, int np, int hw, int nc, int kp, int parts,
                             const float *__restrict__ s, const unsigned *__restrict__ amax,
                             uint16_t *__restrict__ planes, size_t part_elems)
{
    const int np2 = np + 2 * hw;
    const int64_t ncell = 8 * (int64_t)np2 * np2 * np2;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float g = F16 ? pow2f(gain_m_exp(*amax)) : 1.f;
    for (int64_t cell = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); cell < ncell; cell += warps) {
        const int hx = (int)(cell % np2);
        const int hy = (int)((cell / np2) % np2);
        const int hzc = (int)(cell / ((int64_t)np2 * np2));
        const int c = hzc / np2, hz = hzc % np2;
        const int px = ((hx - hw) % np + np) % np, py = ((hy - hw) % np + np) % np, pz = ((hz - hw) % np + np) % np;
        const float *row = M + ((int64_t)c * np * np * np + px + (int64_t)np * (py + (int64_t)np * pz)) * nc;
        uint16_t *out = planes + cell * kp;
        for (int k = lane; k < kp; k += 32) {
            float v = 0.f;
            if (k < nc) {
                v = row[k];
                if (F16) v *= __ldg(s + k) * g;
            }
            split_terms<F16>(v, parts, out + k, part_elems);
        }
    }
}

// FP32 class-layout local expansion of level `lev` (side n = 2^lev) -> fp16
// split planes in natural order [part][z][y][x][k], balanced L~ = L^ / s(k) gL
// (the A operand of the fused L2L): natural cell `cell`, lanes over the coefficients.
__device__ __forceinline__ void split_L_cell(const float *__restrict__ L, int lev, int nc, int kp,
                                             const float *__restrict__ sinv, float g, uint16_t *__restrict__ planes,
                                             size_t part_elems, int64_t cell, int lane)
{
    const int n = 1 << lev, h = n >> 1;
    const int x = (int)(cell % n), y = (int)((cell / n) % n), z = (int)(cell / ((int64_t)n * n));
    const int64_t src = lev == 0 ? 0
                                 : (int64_t)((x & 1) | ((y & 1) << 1) | ((z & 1) << 2)) * h * h * h + (x >> 1) +
                                       (int64_t)h * ((y >> 1) + (int64_t)h * (z >> 1));
    const float *row = L + src * nc;
    uint16_t *out = planes + cell * kp;
    for (int k = lane; k < kp; k += 32) {
        const float v = k < nc ? __ldcg(row + k) * (__ldg(sinv + k) * g) : 0.f;
        split_terms<true>(v, 2, out + k, part_elems);
    }
}

// all cells of level `lev`, one warp per cell
__global__ void k_split_L(const float *__restrict__ L, int lev, int nc, int kp, const float *__restrict__ sinv,
                          const unsigned *__restrict__ amaxL, uint16_t *__restrict__ planes, size_t part_elems)
{
    const int n = 1 << lev;
    const int64_t ncell = (int64_t)n * n * n;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float g = pow2f(gain_m_exp(*amaxL));
    for (int64_t cell = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); cell < ncell; cell += warps)
        split_L_cell(L, lev, nc, kp, sinv, g, planes, part_elems, cell, lane);
}

// FP64 operators -> split B tables [part][slot][j][k] (K-major, rows kp wide):
// slots < noff the M2L operators T[slot][k][j] (input-major), then per child
// octant o the M2M operator (M2M[j][o nc + k], parent output j) and the L2L
// operator (L2L[o nc + j][k], child output j).  fp16: balanced with gT,
//   M2L  T~ = T / (s(k) s(j)),  M2M  S~ = S s(j) / s(k),  L2L  U~ = U s(k) / s(j);
// bf16: the translation slots stay zero (unused).
template <bool F16>
__global__ void k_split_ops(int noff, const double *__restrict__ T, const double *__restrict__ m2m,
                            const double *__restrict__ l2l, int nc, int npad, int kp, int parts,
                            const double *__restrict__ s, uint16_t *__restrict__ ops, size_t part_elems)
{
    const int64_t total = (int64_t)(noff + 16) * npad * kp;
    const double gT = (double)pow2f(GAIN_T_EXP);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % kp);
        const int j = (int)((e / kp) % npad);
        const int slot = (int)(e / ((int64_t)kp * npad));
        double r = 0.0;
        if (j < nc && k < nc) {
            if (slot < noff) {
                r = T[((int64_t)slot * nc + k) * nc + j];
                if (F16) r = r / (s[k] * s[j]) * gT;
            } else if (F16 && slot < noff + 8) {
                const int o = slot - noff;
                r = m2m[(int64_t)j * 8 * nc + o * nc + k] * s[j] / s[k] * gT;
            } else if (F16) {
                const int o = slot - noff - 8;
                r = l2l[((int64_t)o * nc + j) * nc + k] * s[k] / s[j] * gT;
            }
        }
        for (int i = 0; i < parts; ++i) {
            if (F16) {
                const __half t = __float2half_rn((float)r);
                ops[e + i * part_elems] = __half_as_ushort(t);
                r -= (double)__half2float(t);
            } else {
                const __nv_bfloat16 t = __float2bfloat16_rn((float)r);
                ops[e + i * part_elems] = __bfloat16_as_ushort(t);
                r -= (double)__bfloat162float(t);
            }
        }
    }
}

// L = sum over the offset groups, in group order; with amax (fp16 split) the largest |L_e sx(e mod nc)|
// is folded into *amax.  Elements [e0, e1) by threads t = 0 .. nt - 1, four at a time (16-byte loads and
// stores) when n is a multiple of 4 (the partial arrays then stay 16-byte aligned); each element is the
// same ordered sum either way.  Returns this thread's share of the maximum.
__device__ __forceinline__ float group_sum_range(int64_t n, int groups, const float *__restrict__ part,
                                                 float *__restrict__ L, int nc, const float *__restrict__ sx,
                                                 bool fold, int64_t e0, int64_t e1, int64_t t, int64_t nt)
{
    float mx = 0.f;
    if ((n & 3) == 0 && (e0 & 3) == 0) {
        for (int64_t e = e0 + 4 * t; e < e1; e += 4 * nt) {
            if (e + 4 > e1) {  // a ragged end of the range
                for (int64_t k = e; k < e1; ++k) {
                    float s = 0.f;
                    for (int g = 0; g < groups; ++g) s += __ldcg(part + (int64_t)g * n + k);
                    L[k] = s;
                    if (fold) mx = fmaxf(mx, fabsf(s * __ldg(sx + (int)(k % nc))));
                }
                break;
            }
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int g = 0; g < groups; ++g) {
                const float4 v = __ldcg(reinterpret_cast<const float4 *>(part + (int64_t)g * n + e));
                s.x += v.x;
                s.y += v.y;
                s.z += v.z;
                s.w += v.w;
            }
            *reinterpret_cast<float4 *>(L + e) = s;
            if (fold) {
                const int c = (int)(e % nc);
                mx = fmaxf(mx, fabsf(s.x * __ldg(sx + c)));
                mx = fmaxf(mx, fabsf(s.y * __ldg(sx + (c + 1 < nc ? c + 1 : c + 1 - nc))));
                mx = fmaxf(mx, fabsf(s.z * __ldg(sx + (c + 2 < nc ? c + 2 : c + 2 - nc))));
                mx = fmaxf(mx, fabsf(s.w * __ldg(sx + (c + 3 < nc ? c + 3 : c + 3 - nc))));
            }
        }
    } else {
        for (int64_t e = e0 + t; e < e1; e += nt) {
            float s = 0.f;
            for (int g = 0; g < groups; ++g) s += __ldcg(part + (int64_t)g * n + e);
            L[e] = s;
            if (fold) mx = fmaxf(mx, fabsf(s * __ldg(sx + (int)(e % nc))));
        }
    }
    return mx;
}

__global__ void k_group_sum(int64_t n, int groups, const float *__restrict__ part, float *__restrict__ L, int nc,
                            const float *__restrict__ sx, unsigned *__restrict__ amax)
{
    float mx = group_sum_range(n, groups, part, L, nc, sx, amax != nullptr, 0, n,
                               blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
    if (amax) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(amax, __float_as_uint(mx));
    }
}

// fp16 split: FP32 class-layout moments -> the two balanced fp16 halo planes, 8 coefficients per thread
// (16-byte stores per plane); rows kp wide, zero beyond nc
__global__ void k_split_halo16(const float *__restrict__ M, int np, int hw, int nc, int kp, const float *__restrict__ s,
                               const unsigned *__restrict__ amax, uint16_t *__restrict__ planes, size_t part_elems)
{
    const int np2 = np + 2 * hw;
    const int G = kp / 8;
    const int64_t total = 8 * (int64_t)np2 * np2 * np2 * G;
    const float g = pow2f(gain_m_exp(*amax));
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = t / G;
        const int k0 = (int)(t - cell * G) * 8;
        const int hx = (int)(cell % np2);
        const int hy = (int)((cell / np2) % np2);
        const int hzc = (int)(cell / ((int64_t)np2 * np2));
        const int c = hzc / np2, hz = hzc % np2;
        const int px = ((hx - hw) % np + np) % np, py = ((hy - hw) % np + np) % np, pz = ((hz - hw) % np + np) % np;
        const float *row = M + ((int64_t)c * np * np * np + px + (int64_t)np * (py + (int64_t)np * pz)) * nc;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint16_t h2[2], l2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int k = k0 + 2 * i + u;
                const float v = k < nc ? row[k] * (__ldg(s + k) * g) : 0.f;
                const __half t0 = __float2half_rn(v);
                const __half t1 = __float2half_rn(v - __half2float(t0));
                h2[u] = __half_as_ushort(t0);
                l2[u] = __half_as_ushort(t1);
            }
            hi[i] = (uint32_t)h2[0] | ((uint32_t)h2[1] << 16);
            lo[i] = (uint32_t)l2[0] | ((uint32_t)l2[1] << 16);
        }
        uint16_t *out = planes + cell * kp + k0;
        *reinterpret_cast<uint4 *>(out) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(out + part_elems) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// ------------------------------------------------------------------ persistent sweep of a batch
// The tensor-core levels of many boxes (the lambda windows or frames of a batch) in one launch of
// persistent CTA pairs.  Per (box, level) three stages, each a run of work items:
//   P  the parent level's local expansion split into the fused L2L's fp16 planes (k_split_L), and the
//      reset of the level's largest |L^ / s|;
//   M  the tile pairs of the level's M2L + fused L2L (the k_m2l_tc_pair work, same offset groups): one
//      item per tile pair running its groups in turn, or per offset group where the level is small;
//   G  with offset groups > 1, the group sum into L (k_group_sum), folding the level's maximum.
// The items of all boxes sit in one device queue in level order, and P, M, G within a level, so every
// item depends only on items before it.  A pair claims the next item with an atomic add, waits (bounded,
// globaltimer) until the stage it depends on has counted all its items done, runs it, and adds one to
// its own stage's counter (release after the pair's writes).  Because items are claimed in queue order
// and the oldest unfinished item is always held by a running pair with its inputs complete, the sweep
// makes progress whatever number of pairs is resident.  A wait that runs out sets the queue's abort
// word: every pair stops claiming and the launch ends with FMM_ERR_TIMEOUT recorded.
constexpr int SWEEP_P_CELLS = 512;         // parent cells per P item
constexpr int64_t SWEEP_G_ELEMS = 1 << 16;  // L elements per G item

struct SweepLevel {
    CUtensorMap mA[2], mB[2], mL[2];  // the level's pair-kernel tensor maps
    TcArgs a;                         // the level's pair-kernel arguments
    const float *Lprev;               // P: L of level l - 1 (class layout)
    const float *sinv;                // P: 1 / s(k)
    const unsigned *amaxL_prev;       // P: largest |L^ / s| of level l - 1 (final when P runs)
    uint16_t *planesL;                // P: the fused L2L planes
    size_t partL;                     // P: elements per term of planesL
    unsigned *amaxL;                  // this level's largest |L^ / s|, reset by P, folded by M or G
    int64_t gs_n;                     // G: elements of the level's L
    int lev, nc, kp;
    int gpi;                          // M: offset groups per item (all of a tile pair's, or one)
    int n_items[3];                   // items of stages P, M, G (G: 0 with one offset group)
    int prev;                         // the same box's previous sweep level (-1: done before the launch)
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// counter of stage `st` of level entry `e`: q[2 + 3 e + st]; q[0] is the queue head, q[1] the abort word
__device__ __forceinline__ int *sweep_counter(int *q, int e, int st) { return q + 2 + 3 * e + st; }

// bounded wait for the dependency of item `it` (stage, level entry, index); false after limit_ns or abort
__device__ bool sweep_wait(const SweepLevel *__restrict__ lv, int4 it, int *q, uint64_t limit_ns, int stall)
{
    const int *c;
    int target;
    if (it.x == 0) {
        const int pe = lv[it.y].prev;
        if (pe < 0) return true;
        const int st = lv[pe].n_items[2] > 0 ? 2 : 1;
        c = sweep_counter(q, pe, st);
        target = lv[pe].n_items[st];
    } else {
        c = sweep_counter(q, it.y, it.x - 1);
        target = lv[it.y].n_items[it.x - 1];
    }
    target += stall;  // test hook: a count that is never reached
    if (ld_acquire(c) >= target) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        __nanosleep(100);
        if (ld_acquire(c) >= target) return true;
        if ((i & 15) == 15) {
            if (ld_relaxed(q + 1)) return false;
            if (global_ns() - t0 > limit_ns) return false;
        }
    }
}

template <int NCH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    k_m2l_sweep(const SweepLevel *__restrict__ lv, const int4 *__restrict__ items, int n_items, int stages,
                int *__restrict__ q, uint64_t wait_ns, int stall_item)
{
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) PairBars bars;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;
    __shared__ int item_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const uint32_t smem0 = (smem_u32(smem_dyn) + 1023u) & ~1023u;
    if (threadIdx.x == 0) {
        pair_bars_init(bars, stages);
        abort_sh = 0;
        item_sh = n_items;
    }
    cluster_sync_all();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_sh;
    float *stage = reinterpret_cast<float *>(smem_dyn + (smem0 - smem_u32(smem_dyn)));
    PairPipe pp;
    int done_entry = -1, done_stage = 0;  // the item the pair finished last (leader thread 0)
    for (;;) {
        // ---- the leader's thread 0 publishes the finished item, claims the next and waits for its inputs
        if (leader && threadIdx.x == 0) {
            if (done_entry >= 0) {
                __threadfence();
                atomicAdd(sweep_counter(q, done_entry, done_stage), 1);
            }
            int j = n_items;
            if (!ld_relaxed(q + 1)) {
                j = atomicAdd(q, 1);
                if (j < n_items && !sweep_wait(lv, items[j], q, wait_ns, j == stall_item ? 1 : 0)) {
                    atomicOr(lv[items[j].y].a.err, ERRF_TIMEOUT);
                    atomicExch(q + 1, 1);
                    j = n_items;
                }
                if (j > n_items) j = n_items;
            }
            item_sh = j;
            asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(map_shared(smem_u32(&item_sh), 1)), "r"(j)
                         : "memory");
        }
        __syncwarp();
        cluster_sync_all();
        const int j = item_sh;
        if (j >= n_items) break;
        const int4 it = items[j];
        const SweepLevel &e = lv[it.y];
        if (it.x == 1) {
            // stage M: one tile pair; the maps live in global memory, and the planes it copies were written
            // by other pairs through the generic proxy
            if (warp == 0 && lane == 0) {
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&e.mA[m]) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&e.mB[m]) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&e.mL[m]) : "memory");
                }
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            __syncwarp();
            // the item's offset groups of one tile pair in turn (the ring runs on from group to group); only
            // the last group's epilogue stages its rows in the ring
            for (int g = 0; g < e.gpi; ++g) {
                if (*(volatile int *)&abort_sh) break;  // a wait ran out: the remaining groups are skipped
                pair_tile<NCH>(&e.mA[0], &e.mA[1], &e.mB[0], &e.mB[1], &e.mL[0], &e.mL[1], e.a, it.z * e.gpi + g,
                               rank, smem0, stage, g == e.gpi - 1, bars, tmem, &abort_sh, pp);
            }
        } else if (it.x == 0) {
            // stage P: parent cells [SWEEP_P_CELLS it.z, ...) of level l - 1, one warp per cell over the pair
            const int64_t ncell = (int64_t)1 << (3 * (e.lev - 1));
            const int64_t c0 = (int64_t)it.z * SWEEP_P_CELLS;
            const int64_t c1 = c0 + SWEEP_P_CELLS < ncell ? c0 + SWEEP_P_CELLS : ncell;
            const float g = pow2f(gain_m_exp(__ldcg(e.amaxL_prev)));
            const int gw = (int)rank * (TC_THREADS / 32) + warp;
            for (int64_t cell = c0 + gw; cell < c1; cell += 2 * (TC_THREADS / 32))
                split_L_cell(e.Lprev, e.lev - 1, e.nc, e.kp, e.sinv, g, e.planesL, e.partL, cell, lane);
            if (it.z == 0 && leader && threadIdx.x == 0) atomicExch(e.amaxL, 0u);
            asm volatile("fence.proxy.async.global;" ::: "memory");  // the planes are read by TMA next
        } else {
            // stage G: L elements [SWEEP_G_ELEMS it.z, ...), thread per element over the pair
            const int64_t e0 = (int64_t)it.z * SWEEP_G_ELEMS;
            const int64_t e1 = e0 + SWEEP_G_ELEMS < e.gs_n ? e0 + SWEEP_G_ELEMS : e.gs_n;
            float mx = group_sum_range(e.gs_n, e.a.groups, e.a.Lpart, e.a.L, e.nc, e.sinv, true, e0, e1,
                                       (int64_t)rank * TC_THREADS + threadIdx.x, 2 * TC_THREADS);
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0 && mx > 0.f) atomicMax(e.amaxL, __float_as_uint(mx));
        }
        __syncthreads();
        if (threadIdx.x == 0 && abort_sh) atomicExch(q + 1, 1);
        __syncwarp();
        cluster_sync_all();  // both CTAs are done with the item
        if (leader && threadIdx.x == 0) {
            done_entry = it.y;
            done_stage = it.x;
        }
    }

    // ---------------- teardown: every MMA done (bounded wait), pair barrier, collective TMEM release
    if (warp == 1 && lane == 0 && leader) mma_commit_pair(smem_u32(&bars.done));
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int no_abort = 0;
        if (!mbar_wait_cluster(smem_u32(&bars.done), 0, &no_abort)) atomicExch(q + 1, 1);
    }
    fence_before();
    __syncthreads();
    cluster_sync_all();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    cluster_sync_all();
}

// every box of the sweep reports a launch that stopped early
__global__ void k_sweep_status(const int *__restrict__ q, int *const *__restrict__ errs, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && q[1]) atomicOr(errs[i], ERRF_TIMEOUT);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

int tile_dim(int np, int cap) { return np < cap ? np : cap; }

// stage ring of the split (pa, pb): as many stages as the shared-memory budget allows, 2..6
int tc_stages(int pa, int pb, int npad, int sw)
{
    const size_t stage = (size_t)pa * TC_ROWS * sw + (size_t)pb * npad * sw;
    size_t n = (TC_SMEM_BUDGET - 1024) / stage;
    if (n > (size_t)TC_MAX_STAGES) n = TC_MAX_STAGES;
    return n < 2 ? 2 : (int)n;
}

size_t tc_smem_bytes(int pa, int pb, int npad, int sw)
{
    // at least 120 KB so that a second CTA (and its 512 TMEM columns) never shares the SM
    size_t need = (size_t)tc_stages(pa, pb, npad, sw) * (pa * TC_ROWS * sw + pb * npad * sw) + 1024;
    return need < 120 * 1024 ? 120 * 1024 : need;
}

typedef void (*TcKernel)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap,
                         CUtensorMap, TcArgs);
typedef void (*TcPairKernel)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, TcArgs);

// CTA-pair kernel (fp16, 128-byte rows): stage = 2 A terms of 128 rows + 2 B terms of npad / 2 rows
int tc_pair_stages(int npad)
{
    const size_t stage = (size_t)2 * TC_ROWS * 128 + (size_t)2 * (npad / 2) * 128;
    size_t n = (TC_SMEM_BUDGET - 1024) / stage;
    if (n > (size_t)TC_MAX_STAGES) n = TC_MAX_STAGES;
    return n < 2 ? 2 : (int)n;
}

size_t tc_pair_smem_bytes(int npad)
{
    size_t need = (size_t)tc_pair_stages(npad) * ((size_t)2 * TC_ROWS * 128 + (size_t)2 * (npad / 2) * 128) + 1024;
    return need < 120 * 1024 ? 120 * 1024 : need;
}

TcPairKernel pick_pair_kernel(int nch)
{
    switch (nch) {
#define FMM_TC_CASE(n) \
    case n: return (TcPairKernel)k_m2l_tc_pair<n>;
        FMM_TC_CASE(1) FMM_TC_CASE(2) FMM_TC_CASE(3) FMM_TC_CASE(4) FMM_TC_CASE(6) FMM_TC_CASE(7) FMM_TC_CASE(8)
        FMM_TC_CASE(9) FMM_TC_CASE(11) FMM_TC_CASE(13) FMM_TC_CASE(15) FMM_TC_CASE(16)
#undef FMM_TC_CASE
    default: return nullptr;
    }
}

typedef void (*SweepKernel)(const SweepLevel *, const int4 *, int, int, int *, uint64_t, int);

// the sweep is built for the orders p = 6, 8, 10 and 12 (NCH 4, 6, 8, 11)
SweepKernel pick_sweep_kernel(int nch)
{
    switch (nch) {
    case 4: return k_m2l_sweep<4>;
    case 6: return k_m2l_sweep<6>;
    case 8: return k_m2l_sweep<8>;
    case 11: return k_m2l_sweep<11>;
    default: return nullptr;
    }
}

// NCH = ((p+1)^2 rounded to 16) / 16 takes the values below for p <= 15
template <int PA, int PB, int SW>
TcKernel pick_kernel_n(int nch)
{
    switch (nch) {
#define FMM_TC_CASE(n) \
    case n: return (TcKernel)k_m2l_tc<PA, PB, n, SW>;
        FMM_TC_CASE(1) FMM_TC_CASE(2) FMM_TC_CASE(3) FMM_TC_CASE(4) FMM_TC_CASE(6) FMM_TC_CASE(7) FMM_TC_CASE(8)
        FMM_TC_CASE(9) FMM_TC_CASE(11) FMM_TC_CASE(13) FMM_TC_CASE(15) FMM_TC_CASE(16)
#undef FMM_TC_CASE
    default: return nullptr;
    }
}

TcKernel pick_kernel(int pa, int pb, int nch, int sw)
{
    if (sw == 128) return pa == 2 && pb == 2 ? pick_kernel_n<2, 2, 128>(nch) : nullptr;
    if (pa == 3 && pb == 3) return pick_kernel_n<3, 3, 64>(nch);
    if (pa == 2 && pb == 3) return pick_kernel_n<2, 3, 64>(nch);
    if (pa == 2 && pb == 2) return pick_kernel_n<2, 2, 64>(nch);
    return nullptr;
}

#define TRY_TC(x)                          \
    do {                                   \
        fmm_status st_ = (x);              \
        if (st_ != FMM_OK) return st_;     \
    } while (0)

// Offsets split over `groups` CTAs per tile, per_group offsets each.  With one CTA per SM a launch of
// tiles x g CTAs takes ceil(tiles g / sms) waves of ceil(n_off / g) offsets plus a fixed cost per CTA
// (pipeline fill and the exposed epilogue: about SPLIT_FIXED offsets' worth); g is the smallest that
// minimises that product.
constexpr int SPLIT_FIXED = 10;

void split_offsets(int n_off, int tiles, int max_groups, int sms, int &groups, int &per_group)
{
    long long best = -1;
    int g_best = 1;
    for (int g = 1; g <= max_groups && g <= n_off; ++g) {
        const int per = (n_off + g - 1) / g;
        const int used = (n_off + per - 1) / per;  // groups that actually hold offsets
        if (used != g) continue;
        const long long waves = ((long long)tiles * g + sms - 1) / sms;
        const long long cost = waves * (per + SPLIT_FIXED);
        if (best < 0 || cost < best) {
            best = cost;
            g_best = g;
        }
    }
    per_group = (n_off + g_best - 1) / g_best;
    groups = (n_off + per_group - 1) / per_group;
}

CUtensorMapSwizzle swizzle_of(int sw) { return sw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B; }

fmm_status encode_planes(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *map, CUtensorMapDataType dt, void *base,
                         int kp, int64_t d1, int64_t d2, int64_t d3, int b1, int b2, int b3, int sw)
{
    cuuint64_t dims[4] = {(cuuint64_t)kp, (cuuint64_t)d1, (cuuint64_t)d2, (cuuint64_t)d3};
    cuuint64_t strides[3] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * d1, (cuuint64_t)kp * 2 * d1 * d2};
    cuuint32_t box[4] = {(cuuint32_t)kchunk_of(sw), (cuuint32_t)b1, (cuuint32_t)b2, (cuuint32_t)b3};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(map, dt, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(sw),
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
               ? FMM_OK
               : FMM_ERR_INTERNAL;
}

void fill_common(const Plan &P, const TcState *S, int pa, int pb, TcArgs &a)
{
    a.nc = P.nc;
    a.npad = S->npad;
    a.kchunks = (S->kp + kchunk_of(S->sw) - 1) / kchunk_of(S->sw);
    a.ksteps = (P.nc + 15) / 16;
    a.stages = tc_stages(pa, pb, S->npad, S->sw);
    // instruction descriptor: FP32 accumulator, A and B both bf16 (format 1) or both fp16 (format 0),
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t ab = S->f16 ? 0u : 1u;
    a.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(S->npad >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
    a.Lpart = S->Lpart;
    a.err = P.d_err;
    a.amax_out = nullptr;
    a.sx = nullptr;
    a.acc_group = P.acc_group;
    a.wait_ns = P.wait_ns;
    a.inject_stall = P.inject_stall ? 1 : 0;
    a.src_np2 = 0;
    a.out_np = 0;
    a.amaxL = nullptr;
    a.ws = P.ws;
    a.n_il = n_il(P.ws);
    a.noff = noff(P.ws);
    // degree grading of the fp16x2 M2L (FMM_OPT_M2L_GRADE), per K chunk: chunk kc holds input
    // coefficients KCH kc .. KCH kc + KCH - 1, whose lowest degree is floor(sqrt(KCH kc))
    a.gchunks = 0;
    a.gsteps = 0;
    const int d2 = P.grade & 0xFF, d1 = (P.grade >> 8) & 0xFF;
    auto lowest_degree = [](int k) {  // of input coefficient k: floor(sqrt(k))
        int lam = 0;
        while ((lam + 1) * (lam + 1) <= k) ++lam;
        return lam;
    };
    if (S->f16 && pa == 2 && pb == 2 && (d2 > 0 || d1 > 0)) {
        const int kch = kchunk_of(S->sw);
        for (int kc = 0; kc < a.kchunks && kc < 10; ++kc) {
            const int lam = lowest_degree(kch * kc);
            const int np = (d1 > 0 && lam >= d1) ? 1 : (d2 > 0 && lam >= d2) ? 2 : 3;
            if (np < 3) a.gchunks |= (uint32_t)np << (2 * kc);
            // a 3-product chunk whose later K16 steps reach D2 drops x1 y0 there
            if (np == 3 && d2 > 0)
                for (int st = 1; st * 16 < kch; ++st)
                    if (lowest_degree(kch * kc + 16 * st) >= d2) {
                        a.gsteps |= (uint32_t)st << (3 * kc);
                        break;
                    }
        }
    }
}

}  // namespace

bool tc_available(const Plan &P, int level)
{
    return P.tc != nullptr && level >= 1 && level <= P.d;
}

bool tc_translations(const Plan &P)
{
    return P.tc != nullptr && ((const TcState *)P.tc)->f16;
}

fmm_status tc_prepare(Plan &P)
{
    tc_free(P);
    if (P.precision != FMM_PREC_MIXED || P.p > TC_PMAX) return FMM_OK;  // CUDA-core M2L
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return FMM_OK;
    TcState *S = new (std::nothrow) TcState();
    if (!S) return FMM_ERR_OOM;
    P.tc = S;
    S->f16 = P.split == FMM_SPLIT_FP16X2;
    S->pa = P.split == FMM_SPLIT_BF16X3 ? 3 : 2;
    S->pb = (P.split == FMM_SPLIT_BF16X2 || S->f16) ? 2 : 3;
    S->parts = S->f16 ? 2 : 3;  // bf16: three terms always, the solute-only pass uses the 3 x 3 split
    S->npad = (P.nc + 15) / 16 * 16;
    S->noff = noff(P.ws);
    // 128-byte swizzled rows for the fp16 split (two 2-term stages fit), 64 bytes for the bf16 splits;
    // rows padded to whole copy boxes (aligned pieces); the MMAs stop at (p+1)^2 padded to 16
    S->sw = S->f16 ? 128 : 64;
    S->kp = (P.nc + kchunk_of(S->sw) - 1) / kchunk_of(S->sw) * kchunk_of(S->sw);
    const CUtensorMapDataType dt = S->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (S->f16) {
        // s(n,m) = sqrt((n+m)! (n-m)!) per real coefficient
        double h_s[(TC_PMAX + 1) * (TC_PMAX + 1)];
        float h_s32[(TC_PMAX + 1) * (TC_PMAX + 1)], h_inv[(TC_PMAX + 1) * (TC_PMAX + 1)];
        for (int n = 0; n <= P.p; ++n)
            for (int m = 0; m <= n; ++m) {
                double f = 1.0;
                for (int i = 2; i <= n + m; ++i) f *= i;
                for (int i = 2; i <= n - m; ++i) f *= i;
                const double v = sqrt(f);
                const int re = m == 0 ? n * n : n * n + 2 * m - 1;
                h_s[re] = v;
                if (m > 0) h_s[re + 1] = v;
            }
        for (int k = 0; k < P.nc; ++k) {
            h_s32[k] = (float)h_s[k];
            h_inv[k] = (float)(1.0 / h_s[k]);
        }
        FMM_CUDA_TRY(cudaMalloc(&S->s64, sizeof(double) * P.nc));
        FMM_CUDA_TRY(cudaMalloc(&S->s32, sizeof(float) * P.nc));
        FMM_CUDA_TRY(cudaMalloc(&S->s32inv, sizeof(float) * P.nc));
        FMM_CUDA_TRY(cudaMalloc(&S->amax, sizeof(unsigned) * 9));
        FMM_CUDA_TRY(cudaMalloc(&S->amaxL, sizeof(unsigned) * 9));
        FMM_CUDA_TRY(cudaMemcpyAsync(S->s64, h_s, sizeof(double) * P.nc, cudaMemcpyHostToDevice, P.stream));
        FMM_CUDA_TRY(cudaMemcpyAsync(S->s32, h_s32, sizeof(float) * P.nc, cudaMemcpyHostToDevice, P.stream));
        FMM_CUDA_TRY(cudaMemcpyAsync(S->s32inv, h_inv, sizeof(float) * P.nc, cudaMemcpyHostToDevice, P.stream));
    }
    // operator tables
    S->ops_part_elems = (size_t)(S->noff + 16) * S->npad * S->kp;
    FMM_CUDA_TRY(cudaMalloc(&S->ops, sizeof(uint16_t) * S->ops_part_elems * S->parts));
    if (S->f16)
        k_split_ops<true><<<1216, 256, 0, P.stream>>>(S->noff, P.tab.Top64, P.tab.m2m64, P.tab.l2l64, P.nc, S->npad, S->kp,
                                                      S->parts, S->s64, S->ops, S->ops_part_elems);
    else
        k_split_ops<false><<<1216, 256, 0, P.stream>>>(S->noff, P.tab.Top64, nullptr, nullptr, P.nc, S->npad, S->kp, S->parts,
                                                       nullptr, S->ops, S->ops_part_elems);
    FMM_LAUNCH_CHECK(P);
    for (int j = 0; j < S->parts; ++j) {
        cuuint64_t dims[3] = {(cuuint64_t)S->kp, (cuuint64_t)S->npad, (cuuint64_t)(S->noff + 16)};
        cuuint64_t strides[2] = {(cuuint64_t)S->kp * 2, (cuuint64_t)S->kp * 2 * S->npad};
        cuuint32_t box[3] = {(cuuint32_t)kchunk_of(S->sw), (cuuint32_t)S->npad, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (enc(&S->mapB[j], dt, 3, S->ops + j * S->ops_part_elems, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(S->sw), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return FMM_ERR_INTERNAL;
    }
    for (int j = S->parts; j < 3; ++j) S->mapB[j] = S->mapB[0];  // unused kernel parameters
    if (S->f16) {
        for (int j = 0; j < 2; ++j) {
            cuuint64_t dims[3] = {(cuuint64_t)S->kp, (cuuint64_t)S->npad, (cuuint64_t)(S->noff + 16)};
            cuuint64_t strides[2] = {(cuuint64_t)S->kp * 2, (cuuint64_t)S->kp * 2 * S->npad};
            cuuint32_t box[3] = {(cuuint32_t)kchunk_of(S->sw), (cuuint32_t)(S->npad / 2), 1};
            cuuint32_t es[3] = {1, 1, 1};
            if (enc(&S->mapB2[j], dt, 3, S->ops + j * S->ops_part_elems, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(S->sw), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return FMM_ERR_INTERNAL;
        }
        TcPairKernel kp2 = pick_pair_kernel(S->npad / 16);
        if (!kp2) return FMM_ERR_INTERNAL;
        FMM_CUDA_TRY(cudaFuncSetAttribute((const void *)kp2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc_pair_smem_bytes(S->npad)));
    }
    // natural-order planes of the parent-level local expansions (fused L2L), sized for level d - 1
    if (S->f16) {
        const int64_t n = (int64_t)1 << (P.d - 1);
        S->partL_elems = (size_t)n * n * n * S->kp;
        FMM_CUDA_TRY(cudaMalloc(&S->planesL, sizeof(uint16_t) * S->partL_elems * 2));
    }
    // source planes per level
    size_t lpart_elems = 0;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || sms < 1)
        sms = 152;
    for (int l = 1; l <= P.d; ++l) {
        int np = 1 << (l - 1);
        int64_t np2 = np + 2 * P.ws;  // periodic halo of ws cells
        S->bx[l] = tile_dim(np, TC_ROWS);
        S->by[l] = tile_dim(np, TC_ROWS / S->bx[l]);
        S->bz[l] = tile_dim(np, TC_ROWS / (S->bx[l] * S->by[l]));
        S->part_elems[l] = (size_t)8 * np2 * np2 * np2 * S->kp;
        FMM_CUDA_TRY(cudaMalloc(&S->planes[l], sizeof(uint16_t) * S->part_elems[l] * S->parts));
        for (int i = 0; i < S->parts; ++i)
            TRY_TC(encode_planes(enc, &S->mapA[l][i], dt, S->planes[l] + i * S->part_elems[l], S->kp, np2, np2,
                                 8 * np2, S->bx[l], S->by[l], S->bz[l], S->sw));
        for (int i = S->parts; i < 3; ++i) S->mapA[l][i] = S->mapA[l][0];
        if (S->f16) {
            // L of level l - 1 (side np) in natural order, boxed like the level-l bricks; all levels share
            // one buffer, used one level at a time
            for (int i = 0; i < 2; ++i)
                TRY_TC(encode_planes(enc, &S->mapL[l][i], dt, S->planesL + (size_t)i * np * np * np * S->kp, S->kp,
                                     np, np, np, S->bx[l], S->by[l], S->bz[l], S->sw));
        } else {
            S->mapL[l][0] = S->mapL[l][1] = S->mapA[l][0];  // unused kernel parameters
        }
        const int tiles = 8 * (np / S->bx[l]) * (np / S->by[l]) * (np / S->bz[l]);
        split_offsets(n_il(P.ws) + (S->f16 ? 1 : 0), tiles, 27, sms, S->groups[l], S->per_group[l]);
        if (S->groups[l] > 1) {
            size_t need = (size_t)S->groups[l] * 8 * np * np * np * P.nc;
            if (need > lpart_elems) lpart_elems = need;
        }
        // M2M into level l - 1 (natural side np, bricks of the level-l planes)
        const int mtiles = (np / S->bx[l]) * (np / S->by[l]) * (np / S->bz[l]);
        split_offsets(8, mtiles, 8, sms, S->mgroups[l - 1], S->mper_group[l - 1]);
        if (S->f16 && S->mgroups[l - 1] > 1) {
            size_t need = (size_t)S->mgroups[l - 1] * np * np * np * P.nc;
            if (need > lpart_elems) lpart_elems = need;
        }
    }
    if (lpart_elems) FMM_CUDA_TRY(cudaMalloc(&S->Lpart, sizeof(float) * lpart_elems));
    TcKernel k = pick_kernel(S->pa, S->pb, S->npad / 16, S->sw);
    if (!k) return FMM_ERR_INTERNAL;
    FMM_CUDA_TRY(cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tc_smem_bytes(S->pa, S->pb, S->npad, S->sw)));
    if (!S->f16) {
        TcKernel kp = pick_kernel(3, 3, S->npad / 16, S->sw);  // the solute-only pass
        if (!kp) return FMM_ERR_INTERNAL;
        FMM_CUDA_TRY(cudaFuncSetAttribute((const void *)kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc_smem_bytes(3, 3, S->npad, S->sw)));
    }
    FMM_CUDA_TRY(cudaStreamSynchronize(P.stream));
    return FMM_OK;
}

unsigned *tc_amax(Plan &P, int l)
{
    TcState *S = (TcState *)P.tc;
    return S && S->f16 && l >= 0 && l <= P.d ? S->amax + l : nullptr;
}

fmm_status tc_clear_amax(Plan &P, int l)
{
    unsigned *a = tc_amax(P, l);
    if (!a) return FMM_ERR_INTERNAL;
    FMM_CUDA_TRY(cudaMemsetAsync(a, 0, sizeof(unsigned), P.stream));
    return FMM_OK;
}

const float *tc_scale(const Plan &P)
{
    const TcState *S = (const TcState *)P.tc;
    return S && S->f16 ? S->s32 : nullptr;
}

// fp16 split: the balanced halo planes of M[l]; the level's largest |M^ s| is computed first unless the
// kernel that wrote M[l] folded it in already
fmm_status tc_split_moments(Plan &P, int l, bool amax_ready)
{
    TcState *S = (TcState *)P.tc;
    if (!S || !S->f16 || l < 1 || l > P.d) return FMM_ERR_INTERNAL;
    const int np = 1 << (l - 1);
    const int64_t np2 = np + 2 * P.ws;
    const int64_t ncell = (int64_t)8 * np * np * np;
    if (!amax_ready) {
        FMM_CUDA_TRY(cudaMemsetAsync(S->amax + l, 0, sizeof(unsigned), P.stream));
        k_absmax<<<(unsigned)((ncell + 7) / 8 < 1216 ? (ncell + 7) / 8 : 1216), 256, 0, P.stream>>>(
            (const float *)P.M[l], ncell, P.nc, S->s32, S->amax + l);
        FMM_LAUNCH_CHECK(P);
    }
    const int64_t nthr = 8 * np2 * np2 * np2 * (S->kp / 8);
    k_split_halo16<<<(unsigned)((nthr + 255) / 256 < 8 * 1216 ? (nthr + 255) / 256 : 8 * 1216), 256, 0, P.stream>>>(
        (const float *)P.M[l], np, P.ws, P.nc, S->kp, S->s32, S->amax + l, S->planes[l], S->part_elems[l]);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

// fp16 split: M2M into level l (< d) from the split planes of level l + 1
fmm_status launch_m2m_tc(Plan &P, int l)
{
    TcState *S = (TcState *)P.tc;
    if (!S || !S->f16 || l < 0 || l >= P.d) return FMM_ERR_INTERNAL;
    const int src = l + 1;
    const int n = 1 << l;  // natural side of level l = parent side of the level-(l+1) planes
    TcArgs a;
    fill_common(P, S, S->pa, S->pb, a);
    a.mode = 1;
    a.gchunks = a.gsteps = 0;  // translations keep every product
    a.np = n;
    a.bx = S->bx[src];
    a.by = S->by[src];
    a.bz = S->bz[src];
    a.rows = a.bx * a.by * a.bz;
    a.tiles_x = n / a.bx;
    a.tiles_y = n / a.by;
    a.tiles_per_class = a.tiles_x * a.tiles_y * (n / a.bz);
    a.groups = S->mgroups[l];
    a.per_group = S->mper_group[l];
    a.n_off = 8;
    a.src_np2 = n + 2 * P.ws;
    a.out_np = l == 0 ? 0 : n >> 1;
    a.L = (float *)P.M[l];
    a.post = S->s32inv;
    a.amax = S->amax + src;
    // level l's largest |M^ s| (the gain of its planes) is folded in by whoever writes M[l]
    FMM_CUDA_TRY(cudaMemsetAsync(S->amax + l, 0, sizeof(unsigned), P.stream));
    a.amax_out = a.groups == 1 ? S->amax + l : nullptr;
    a.sx = S->s32;
    TcKernel k = pick_kernel(S->pa, S->pb, S->npad / 16, S->sw);
    if (!k) return FMM_ERR_INTERNAL;
    const unsigned grid = (unsigned)a.tiles_per_class * (unsigned)a.groups;
    k<<<grid, TC_THREADS, tc_smem_bytes(S->pa, S->pb, S->npad, S->sw), P.stream>>>(
        S->mapA[src][0], S->mapA[src][1], S->mapA[src][2], S->mapB[0], S->mapB[1], S->mapB[2], S->mapA[src][0],
        S->mapA[src][0], a);
    FMM_LAUNCH_CHECK(P);
    if (a.groups > 1) {
        const int64_t cnt = (int64_t)n * n * n * P.nc;
        k_group_sum<<<(unsigned)((cnt + 255) / 256 < 2048 ? (cnt + 255) / 256 : 2048), 256, 0, P.stream>>>(
            cnt, a.groups, S->Lpart, a.L, P.nc, S->s32, S->amax + l);
        FMM_LAUNCH_CHECK(P);
    }
    return FMM_OK;
}

// Arguments of the level-l M2L (+ fused L2L with the fp16 split); returns whether the level runs on CTA
// pairs (an even number of full 128-row tiles per class), whose stage ring and M = 256 descriptor it sets
static bool m2l_args(const Plan &P, const TcState *S, int l, bool precise, int pa, int pb, TcArgs &a)
{
    const int np = 1 << (l - 1);
    fill_common(P, S, pa, pb, a);
    if (precise) a.gchunks = a.gsteps = 0;  // the solute-only pass keeps every product
    a.mode = 0;
    a.np = np;
    a.bx = S->bx[l];
    a.by = S->by[l];
    a.bz = S->bz[l];
    a.rows = a.bx * a.by * a.bz;
    a.tiles_x = np / a.bx;
    a.tiles_y = np / a.by;
    a.tiles_per_class = a.tiles_x * a.tiles_y * (np / a.bz);
    a.groups = S->groups[l];
    a.per_group = S->per_group[l];
    a.n_off = a.n_il + (S->f16 ? 1 : 0);
    a.L = (float *)P.L[l];
    a.post = S->f16 ? S->s32 : nullptr;
    a.amax = S->f16 ? S->amax + l : nullptr;
    a.amaxL = S->f16 ? S->amaxL + l - 1 : nullptr;
    if (S->f16) {
        a.amax_out = a.groups == 1 ? S->amaxL + l : nullptr;
        a.sx = S->s32inv;
    }
    const bool pair = S->f16 && P.tc_pair && a.rows == TC_ROWS && a.tiles_per_class % 2 == 0;
    if (pair) {
        a.stages = tc_pair_stages(S->npad);
        a.idesc = (1u << 4) | ((uint32_t)(S->npad >> 3) << 17) | ((uint32_t)((2 * TC_ROWS) >> 4) << 24);  // M = 256
    }
    return pair;
}

fmm_status launch_m2l_tc(Plan &P, int l, bool precise, bool split)
{
    TcState *S = (TcState *)P.tc;
    if (!S) return FMM_ERR_INTERNAL;
    // the fp16 split is already as accurate as the 3 x 3 bf16 one
    const int pa = precise && !S->f16 ? 3 : S->pa;
    const int pb = precise && !S->f16 ? 3 : S->pb;
    int np = 1 << (l - 1);
    int64_t np2 = np + 2 * P.ws;
    if (S->f16) {
        if (split) {
            fmm_status st = tc_split_moments(P, l, false);
            if (st != FMM_OK) return st;
        }
        // parent-level local expansion for the fused L2L; its largest |L^ / s| was folded in by the level
        // l - 1 launch (levels run in order), except at level 0 (the lattice operator's output)
        const int64_t ncl = (int64_t)np * np * np;
        if (l == 1) {
            FMM_CUDA_TRY(cudaMemsetAsync(S->amaxL, 0, sizeof(unsigned), P.stream));
            k_absmax<<<1, 256, 0, P.stream>>>((const float *)P.L[0], 1, P.nc, S->s32inv, S->amaxL);
            FMM_LAUNCH_CHECK(P);
        }
        k_split_L<<<(unsigned)((ncl + 7) / 8 < 1216 ? (ncl + 7) / 8 : 1216), 256, 0, P.stream>>>(
            (const float *)P.L[l - 1], l - 1, P.nc, S->kp, S->s32inv, S->amaxL + l - 1, S->planesL,
            (size_t)ncl * S->kp);
        FMM_LAUNCH_CHECK(P);
    } else {
        const int64_t nhalo = 8 * np2 * np2 * np2;
        k_split_halo<false><<<(unsigned)((nhalo + 7) / 8 < 4864 ? (nhalo + 7) / 8 : 4864), 256, 0, P.stream>>>(
            (const float *)P.M[l], np, P.ws, P.nc, S->kp, pa, nullptr, nullptr, S->planes[l], S->part_elems[l]);
        FMM_LAUNCH_CHECK(P);
    }
    if (S->f16)  // level l's largest |L^ / s|, for the fused L2L of level l + 1
        FMM_CUDA_TRY(cudaMemsetAsync(S->amaxL + l, 0, sizeof(unsigned), P.stream));
    TcArgs a;
    const bool pair = m2l_args(P, S, l, precise, pa, pb, a);
    unsigned grid = 8u * (unsigned)a.tiles_per_class * (unsigned)a.groups;
    const bool time_it = P.timings_on && l == P.d && P.ev_top[0] && !precise;
    if (time_it) cudaEventRecord(P.ev_top[0], P.stream);
    if (pair) {
        TcPairKernel k2 = pick_pair_kernel(S->npad / 16);
        if (!k2) return FMM_ERR_INTERNAL;
        k2<<<grid, TC_THREADS, tc_pair_smem_bytes(S->npad), P.stream>>>(S->mapA[l][0], S->mapA[l][1], S->mapB2[0],
                                                                         S->mapB2[1], S->mapL[l][0], S->mapL[l][1], a);
    } else {
        TcKernel k = pick_kernel(pa, pb, S->npad / 16, S->sw);
        if (!k) return FMM_ERR_INTERNAL;
        k<<<grid, TC_THREADS, tc_smem_bytes(pa, pb, S->npad, S->sw), P.stream>>>(
            S->mapA[l][0], S->mapA[l][1], S->mapA[l][2], S->mapB[0], S->mapB[1], S->mapB[2], S->mapL[l][0],
            S->mapL[l][1], a);
    }
    FMM_LAUNCH_CHECK(P);
    if (time_it) {
        cudaEventRecord(P.ev_top[1], P.stream);
        P.top_recorded = true;
    }
    if (a.groups > 1) {
        int64_t n = (int64_t)8 * np * np * np * P.nc;
        k_group_sum<<<(unsigned)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048), 256, 0, P.stream>>>(
            n, a.groups, S->Lpart, a.L, P.nc, S->f16 ? S->s32inv : nullptr, S->f16 ? S->amaxL + l : nullptr);
        FMM_LAUNCH_CHECK(P);
    }
    return FMM_OK;
}

// ------------------------------------------------------------------ persistent sweep (host)
int tc_sweep_first_level(const Plan &P)
{
    const TcState *S = (const TcState *)P.tc;
    if (!S || !S->f16 || !P.tc_pair || P.precision != FMM_PREC_MIXED) return 0;
    for (int l = 2; l <= P.d; ++l) {  // level 1 reads the lattice's L[0]: it stays on its own launches
        const int np = 1 << (l - 1);
        const int tpc = (np / S->bx[l]) * (np / S->by[l]) * (np / S->bz[l]);
        if (S->bx[l] * S->by[l] * S->bz[l] == TC_ROWS && tpc % 2 == 0) return l;  // and every deeper level
    }
    return 0;
}

struct Sweep {
    std::vector<Plan *> plans;  // the plans taking part
    std::vector<int> first;     // their first sweep level
    int nch = 0, stages = 0, pairs = 0, n_items = 0, n_lv = 0, stall_item = -1;
    size_t smem = 0;
    SweepLevel *d_lv = nullptr;
    int4 *d_items = nullptr;
    int *d_q = nullptr;
    int **d_errs = nullptr;
};

void sweep_destroy(Sweep *sw)
{
    if (!sw) return;
    for (Plan *P : sw->plans) P->sweep_from = 0;
    cudaFree(sw->d_lv);
    cudaFree(sw->d_items);
    cudaFree(sw->d_q);
    cudaFree(sw->d_errs);
    delete sw;
}

void sweep_enable(Sweep *sw, bool on)
{
    if (!sw) return;
    for (size_t k = 0; k < sw->plans.size(); ++k) sw->plans[k]->sweep_from = on ? sw->first[k] : 0;
}

int sweep_plans(const Sweep *sw) { return sw ? (int)sw->plans.size() : 0; }

fmm_status sweep_create(Plan *const *plans, int n, Sweep **out)
{
    *out = nullptr;
    Sweep *sw = new (std::nothrow) Sweep();
    if (!sw) return FMM_ERR_OOM;
    for (int i = 0; i < n; ++i) {
        Plan &P = *plans[i];
        const int l0 = tc_sweep_first_level(P);
        if (l0 <= 0) continue;
        const int c = ((const TcState *)P.tc)->npad / 16;
        if (!pick_sweep_kernel(c) || (sw->nch && c != sw->nch)) continue;  // stays on its per-level launches
        sw->nch = c;
        sw->plans.push_back(&P);
        sw->first.push_back(l0);
    }
    if (sw->plans.empty()) {
        delete sw;
        return FMM_OK;
    }
    // one entry per (plan, level), each pointing at the same plan's previous level
    std::vector<SweepLevel> lv;
    int lmin = 1 << 30, lmax = 0;
    for (size_t k = 0; k < sw->plans.size(); ++k) {
        Plan &P = *sw->plans[k];
        const TcState *S = (const TcState *)P.tc;
        int prev = -1;
        for (int l = sw->first[k]; l <= P.d; ++l) {
            SweepLevel e;
            memset((void *)&e, 0, sizeof(e));
            if (!m2l_args(P, S, l, false, S->pa, S->pb, e.a) || (sw->stages && e.a.stages != sw->stages)) {
                sweep_destroy(sw);
                return FMM_ERR_INTERNAL;
            }
            sw->stages = e.a.stages;
            e.mA[0] = S->mapA[l][0];
            e.mA[1] = S->mapA[l][1];
            e.mB[0] = S->mapB2[0];
            e.mB[1] = S->mapB2[1];
            e.mL[0] = S->mapL[l][0];
            e.mL[1] = S->mapL[l][1];
            const int64_t ncl = (int64_t)1 << (3 * (l - 1));  // cells of level l - 1
            e.Lprev = (const float *)P.L[l - 1];
            e.sinv = S->s32inv;
            e.amaxL_prev = S->amaxL + l - 1;
            e.planesL = S->planesL;
            e.partL = (size_t)ncl * S->kp;
            e.amaxL = S->amaxL + l;
            e.gs_n = 8 * ncl * P.nc;
            e.lev = l;
            e.nc = P.nc;
            e.kp = S->kp;
            e.n_items[0] = (int)((ncl + SWEEP_P_CELLS - 1) / SWEEP_P_CELLS);
            e.gpi = e.a.groups;  // set per level below
            e.n_items[1] = 4 * e.a.tiles_per_class;  // tile pairs: 8 classes x tiles / 2
            e.n_items[2] = e.a.groups > 1 ? (int)((e.gs_n + SWEEP_G_ELEMS - 1) / SWEEP_G_ELEMS) : 0;
            e.prev = prev;
            prev = (int)lv.size();
            lv.push_back(e);
            lmin = l < lmin ? l : lmin;
            lmax = l > lmax ? l : lmax;
        }
    }
    // item grain per level: whole tile pairs (all their offset groups in turn: one ramp and one exposed
    // epilogue per tile pair) when the level's tile pairs over all entries fill the resident pairs twice;
    // otherwise one offset group per item, so that a lone deep box's small levels spread over the GPU
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        for (int l = lmin; l <= lmax; ++l) {
            long long tp = 0;
            for (const SweepLevel &e : lv)
                if (e.lev == l) tp += e.n_items[1];
            for (SweepLevel &e : lv)
                if (e.lev == l && tp < (long long)sms) {  // 2 x (sms / 2) pairs
                    e.gpi = 1;
                    e.n_items[1] *= e.a.groups;
                }
        }
    }
    // the queue: level by level, within a level stage P of every entry, then M, then G
    std::vector<int4> items;
    int m_items = 0;
    for (int l = lmin; l <= lmax; ++l)
        for (int st = 0; st < 3; ++st)
            for (size_t e = 0; e < lv.size(); ++e) {
                if (lv[e].lev != l) continue;
                for (int i = 0; i < lv[e].n_items[st]; ++i) {
                    if (st == 1 && sw->stall_item < 0) sw->stall_item = (int)items.size();
                    if (st == 1) ++m_items;
                    items.push_back(make_int4(st, (int)e, i, 0));
                }
            }
    sw->n_lv = (int)lv.size();
    sw->n_items = (int)items.size();
    std::vector<int *> errs;
    for (Plan *P : sw->plans) errs.push_back(P->d_err);
    fmm_status s = FMM_OK;
    if (cudaMalloc(&sw->d_lv, sizeof(SweepLevel) * lv.size()) != cudaSuccess ||
        cudaMalloc(&sw->d_items, sizeof(int4) * items.size()) != cudaSuccess ||
        cudaMalloc(&sw->d_q, sizeof(int) * (2 + 3 * lv.size())) != cudaSuccess ||
        cudaMalloc(&sw->d_errs, sizeof(int *) * errs.size()) != cudaSuccess)
        s = FMM_ERR_OOM;
    if (s == FMM_OK &&
        (cudaMemcpy(sw->d_lv, lv.data(), sizeof(SweepLevel) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(sw->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(sw->d_errs, errs.data(), sizeof(int *) * errs.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        s = FMM_ERR_CUDA;
    // as many pairs as can be resident (one CTA per SM), at most one per tile pair of the queue
    const int npad = 16 * sw->nch;
    sw->smem = tc_pair_smem_bytes(npad);
    SweepKernel k = pick_sweep_kernel(sw->nch);
    if (s == FMM_OK && cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sw->smem) != cudaSuccess)
        s = FMM_ERR_CUDA;
    if (s == FMM_OK) {
        int dev = 0, sms = 0, clusters = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(sms > 0 ? sms : 2));
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = sw->smem;
        if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)k, &cfg) != cudaSuccess || clusters < 1)
            clusters = sms / 2;
        cudaGetLastError();
        sw->pairs = clusters < m_items ? clusters : m_items;
        if (sw->pairs < 1) sw->pairs = 1;
    }
    if (s != FMM_OK) {
        sweep_destroy(sw);
        return s;
    }
    sweep_enable(sw, true);
    *out = sw;
    return FMM_OK;
}

fmm_status sweep_launch(Sweep *sw, cudaStream_t st, uint64_t wait_ns, bool stall, int max_pairs)
{
    if (!sw) return FMM_OK;
    FMM_CUDA_TRY(cudaMemsetAsync(sw->d_q, 0, sizeof(int) * (2 + 3 * (size_t)sw->n_lv), st));
    SweepKernel k = pick_sweep_kernel(sw->nch);
    const int pairs = max_pairs > 0 && max_pairs < sw->pairs ? max_pairs : sw->pairs;
    k<<<2u * (unsigned)pairs, TC_THREADS, sw->smem, st>>>(sw->d_lv, sw->d_items, sw->n_items, sw->stages, sw->d_q,
                                                              wait_ns, stall ? sw->stall_item : -1);
    FMM_CUDA_TRY(cudaGetLastError());
    const int n = (int)sw->plans.size();
    k_sweep_status<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(sw->d_q, sw->d_errs, n);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// Brick of the level-l tiles: bx x by x bz target cells of one parity class (the MMA's 128 rows), each
// dividing the class side 2^(l-1), an even number of tiles per class (CTA pairs); the level's plane maps
// are encoded for it.  Which targets share a tile changes, no target's arithmetic does.
fmm_status tc_set_brick(Plan &P, int l, int bx, int by, int bz)
{
    TcState *S = (TcState *)P.tc;
    if (!S) return FMM_ERR_UNSUPPORTED;
    if (l < 2 || l > P.d) return FMM_ERR_INVALID_ARG;
    const int np = 1 << (l - 1);
    if (bx < 1 || by < 1 || bz < 1 || bx * by * bz != TC_ROWS || np % bx || np % by || np % bz ||
        ((np / bx) * (np / by) * (np / bz)) % 2)
        return FMM_ERR_INVALID_ARG;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return FMM_ERR_INTERNAL;
    const CUtensorMapDataType dt = S->f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int64_t np2 = np + 2 * P.ws;
    CUtensorMap a[3], lm[2];
    for (int i = 0; i < S->parts; ++i)
        TRY_TC(encode_planes(enc, &a[i], dt, S->planes[l] + i * S->part_elems[l], S->kp, np2, np2, 8 * np2, bx, by,
                             bz, S->sw));
    for (int i = S->parts; i < 3; ++i) a[i] = a[0];
    if (S->f16)
        for (int i = 0; i < 2; ++i)
            TRY_TC(encode_planes(enc, &lm[i], dt, S->planesL + (size_t)i * np * np * np * S->kp, S->kp, np, np, np,
                                 bx, by, bz, S->sw));
    else
        lm[0] = lm[1] = a[0];
    for (int i = 0; i < 3; ++i) S->mapA[l][i] = a[i];
    S->mapL[l][0] = lm[0];
    S->mapL[l][1] = lm[1];
    S->bx[l] = bx;
    S->by[l] = by;
    S->bz[l] = bz;
    return FMM_OK;
}

void tc_get_brick(const Plan &P, int l, int *bx, int *by, int *bz)
{
    const TcState *S = (const TcState *)P.tc;
    *bx = S && l >= 1 && l <= P.d ? S->bx[l] : 0;
    *by = S && l >= 1 && l <= P.d ? S->by[l] : 0;
    *bz = S && l >= 1 && l <= P.d ? S->bz[l] : 0;
}

// The split operator tables depend only on p, ws and the split (the M2L, M2M and L2L operators are
// built for unit cells), so plans that agree on those can read one copy: dst drops its own and reads
// src's, which must outlive it.  A plan with another table is left alone.
fmm_status tc_share_operators(Plan &dst, const Plan &src)
{
    TcState *D = (TcState *)dst.tc;
    const TcState *S = (const TcState *)src.tc;
    if (!D || !S || D == S || D->ops == S->ops) return FMM_OK;
    if (dst.p != src.p || dst.ws != src.ws || D->f16 != S->f16 || D->pa != S->pa || D->pb != S->pb ||
        D->parts != S->parts || D->npad != S->npad || D->kp != S->kp || D->noff != S->noff || D->sw != S->sw ||
        D->ops_part_elems != S->ops_part_elems)
        return FMM_OK;
    FMM_CUDA_TRY(cudaDeviceSynchronize());  // nothing of dst's may still read its own table
    if (!D->ops_borrowed) cudaFree(D->ops);
    D->ops = S->ops;
    D->ops_borrowed = true;
    memcpy((void *)D->mapB, (const void *)S->mapB, sizeof(D->mapB));
    memcpy((void *)D->mapB2, (const void *)S->mapB2, sizeof(D->mapB2));
    return FMM_OK;
}

void tc_free(Plan &P)
{
    TcState *S = (TcState *)P.tc;
    if (!S) return;
    for (int l = 0; l < 9; ++l) cudaFree(S->planes[l]);
    if (!S->ops_borrowed) cudaFree(S->ops);
    cudaFree(S->Lpart);
    cudaFree(S->s32);
    cudaFree(S->s32inv);
    cudaFree(S->s64);
    cudaFree(S->amax);
    cudaFree(S->amaxL);
    cudaFree(S->planesL);
    delete S;
    P.tc = nullptr;
}

}  // namespace fmm
