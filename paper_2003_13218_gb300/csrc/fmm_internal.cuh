// fmm_internal.cuh -- shared declarations of the GB300 periodic FMM library.
//
// Layouts (all device memory owned by the plan):
//  * particles are sorted by leaf (linear leaf index x + n (y + n z), n = 2^d)
//    with a CSR `cell_start[n^3 + 1]`; sorted records hold the coordinates
//    relative to the leaf centre and the charge, in the path's real type;
//  * expansion coefficients are real: for degree n, Re C_n^0 at n^2, and for
//    m >= 1 Re C_n^m at n^2 + 2m - 1 and Im C_n^m at n^2 + 2m (the negative
//    orders follow from C_n^{-m} = (-1)^m conj C_n^m);  (p+1)^2 reals per cell;
//  * coefficients are level-scaled: Mhat_n = M_n / h_l^n and
//    Lhat_n = L_n h_l^(n+1), h_l = b / 2^l, which makes the M2L operator of
//    Eq. Lcoeffdef depend on the cell offset only;
//  * cells of level l >= 1 are stored by parity class: cell (x, y, z) has class
//    c = (x&1) | (y&1)<<1 | (z&1)<<2 and parent coordinates P = (x, y, z) >> 1;
//    index = c * np^3 + P.x + np (P.y + np P.z), np = 2^(l-1).  Level 0 has one
//    cell.  A target of class c and its interaction-list source t + delta then
//    lie in class (c + delta) & 1 at parent offset (c + delta) >> 1, which is
//    -1, 0 or +1 per axis.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmm_gb300.h"

namespace fmm {

constexpr int P_MAX = 20;
constexpr int NC_MAX = (P_MAX + 1) * (P_MAX + 1);
// Offsets delta (in cells of one level) between a target and the sources of
// its interaction list lie in [-(2 ws + 1), 2 ws + 1]^3: operator slots are
// numbered on that cube (7^3 for ws = 1, 11^3 for ws = 2); the (2 ws + 1)^3
// near slots stay zero.  An interaction list holds (4 ws + 2)^3 - (2 ws + 1)^3
// cells: 189 for ws = 1, 875 for ws = 2.
constexpr int WS_MAX = 2;
__host__ __device__ inline int off_side(int ws) { return 4 * ws + 3; }
__host__ __device__ inline int noff(int ws) { return off_side(ws) * off_side(ws) * off_side(ws); }
__host__ __device__ inline int n_il(int ws)
{
    const int a = 4 * ws + 2, b = 2 * ws + 1;
    return a * a * a - b * b * b;
}

enum : int { ERRF_NONFINITE = 1, ERRF_INTERNAL = 2, ERRF_TIMEOUT = 4 };

__host__ __device__ inline int ncoef(int p) { return (p + 1) * (p + 1); }
__host__ __device__ inline int cre(int n, int m) { return m == 0 ? n * n : n * n + 2 * m - 1; }
__host__ __device__ inline int cim(int n, int m) { return n * n + 2 * m; }
__host__ __device__ inline int off_slot(int dx, int dy, int dz, int ws)
{
    const int h = 2 * ws + 1, side = 2 * h + 1;
    return (dx + h) + side * ((dy + h) + side * (dz + h));
}

__host__ __device__ inline int64_t cell_index(int l, int x, int y, int z)
{
    if (l == 0) return 0;
    int64_t np = (int64_t)1 << (l - 1);
    int c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    return c * np * np * np + (x >> 1) + np * ((y >> 1) + np * (int64_t)(z >> 1));
}

template <typename T>
struct Particle {  // sorted record: position relative to the leaf centre, charge
    T x, y, z, q;
};

template <typename T>
struct alignas(2 * sizeof(T)) Cx {
    T re, im;
};
template <typename T>
__host__ __device__ inline Cx<T> cmul(Cx<T> a, Cx<T> b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Level-independent tables built once per plan.
struct Tables {
    double *Rw64 = nullptr;   // [8][NC] real R_n^m(w_c), w_c = child-centre offset / parent side (+-1/4)
    float *Rw32 = nullptr;
    double *S = nullptr;      // [NC2] complex lattice sum S_j^k (j <= 2p, k >= 0), scaled to a unit box
    double *T0 = nullptr;     // [NC][NC] real lattice operator (input-major: T0[k * NC + j])
    double *Top64 = nullptr;  // [noff(ws)][NC][NC] real M2L operators (input-major), FP64 path
    float *Top32 = nullptr;   // same in FP32 for the SIMT FP32 path
    double *l2l64 = nullptr;  // [8 NC][NC] L2L operators of the 8 child octants (row-major)
    float *l2l32 = nullptr;
    double *m2m64 = nullptr;  // [NC][8 NC] M2M operators (row-major)
    float *m2m32 = nullptr;
    float *m2mP32 = nullptr;  // M2M with each octant's K padded to a multiple of 8
    float *l2lP32 = nullptr;  // L2L with K padded likewise
};

struct Plan {
    // problem
    double box = 0;
    int64_t N = 0;
    int d = 0, p = 0, ws = 1;
    int precision = FMM_PREC_FP64;
    int split = FMM_SPLIT_FP16X2;
    double kappa = 0;  // 0 = default 2 / box
    cudaStream_t stream = 0;
    bool timings_on = false;
    bool tc_pair = true;  // CTA-pair (2-SM) tensor-core M2L where the level allows it
    int sweep_from = 0;   // > 0: the full pass's levels >= sweep_from (and its L2P) run in a batch's sweep
    int known_count = -1; // >= 0: the solute count the caller already knows (no host wait; graph capture)
    int boundary = 0;     // FMM_BOUNDARY_CONDUCTING (Eq. Velecfull) or FMM_BOUNDARY_VACUUM (App. D)
    // FMM_OPT_SOFTCORE: soft-core solute-solvent near field (c = 0: off); lambda lives in pinned host memory
    // and is copied to the device at the start of each call (a recorded graph sees the current value)
    int sc_c = 0;
    double sc_A = 0, sc_alpha = 0.2;
    double *sc_out = nullptr;        // device [2N]: per sorted slot q_i sum q_j / reff, and the lambda derivative
    double *sc_lambda = nullptr;     // device [1]
    double *h_sc_lambda = nullptr;   // pinned host [1]
    int acc_group = FMM_ACC_GROUP_DEFAULT;  // FMM_OPT_M2L_ACC_GROUP: offsets per TMEM accumulator drain
    uint64_t wait_ns = 2000000000ull;       // FMM_OPT_WAIT_BUDGET_NS: budget of each tensor-core pipeline wait
    bool inject_stall = false;              // FMM_OPT_INJECT_STALL (test hook)
    int grade = FMM_GRADE_DEFAULT;  // FMM_OPT_M2L_GRADE: D2 | D1 << 8 (input degrees from which the fp16x2 M2L
                                    // drops the moments' / also the operators' second term; 0 = never)
    // FMM_OPT_OVERLAP: evaluate() runs on `exec` (priority above the default), the near field on `near`
    // (lowest priority: it fills what the far field leaves idle), both joined before the reductions
    bool overlap = true;
    cudaStream_t exec = nullptr, near = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_sorted = nullptr, ev_near = nullptr;
    bool near_forked = false;  // work of the current call on `near`, not yet joined
    bool near_p2p = false;     // the current call's near field (P2P) runs on `near`
    int nc = 0;
    int64_t nleaf = 0;  // 8^d
    int64_t launches = 0;

    // particles
    double *in_pos = nullptr, *in_q = nullptr, *out_forces = nullptr;  // staging for host pointers
    double *out_phi = nullptr;
    uint8_t *in_sol = nullptr;
    double *wpos = nullptr;        // [N][3] wrapped input positions (original order)
    int *key = nullptr;            // [N] leaf of each particle
    int *perm = nullptr;           // [N] sorted slot -> original index
    int *sleaf = nullptr;          // [N] leaf of each sorted slot
    int *cell_start = nullptr;     // [nleaf + 1]
    int *cell_fill = nullptr;      // [nleaf]
    int *scan_tmp = nullptr;
    void *sorted = nullptr;        // Particle<T>[N]
    void *sorted_u = nullptr;      // Particle<T>[N] with solvent charges zeroed (solute-only pass)
    uint8_t *sorted_sol = nullptr; // [N]
    void *phi_nf = nullptr, *phi_ff = nullptr;  // T[N] per-particle potentials (sorted order)
    void *phi_u = nullptr;                      // T[N] solute-only far-field potential
    void *f_nf = nullptr, *g_ff = nullptr;      // T[N][3] near-field field, far-field gradient
    // expansions per level (T, class layout)
    void *M[9] = {};
    void *L[9] = {};
    // tensor-core M2L state (bf16 operand planes, operator tables, TMA maps)
    void *tc = nullptr;
    // scratch of the sparse solute-only pass
    void *sol = nullptr;
    // reductions
    double *red_partial = nullptr;  // partial sums
    double *red_out = nullptr;      // [32] final FP64 scalars
    double *h_out = nullptr;        // pinned host mirror
    int *d_err = nullptr;
    Tables tab;
    cudaEvent_t ev[12] = {};
    cudaEvent_t ev_m2l[18] = {};  // around each level's M2L launch (full pass)
    cudaEvent_t ev_top[2] = {};   // around the tensor-core M2L launch of level d
    bool top_recorded = false;
    fmm_timings last{};
};

// ------------------------------------------------------------------ device helpers
// Regular solid harmonics by their Cartesian recurrences:
//   R_0^0 = 1,  R_m^m = -(x + i y) R_{m-1}^{m-1} / (2m),
//   R_n^m = ((2n-1) z R_{n-1}^m - r^2 R_{n-2}^m) / ((n+m)(n-m)).
// out must hold ncoef(p) reals (layout above).
template <typename T>
__host__ __device__ inline void regular_real(int p, T x, T y, T z, T *out)
{
    T r2 = x * x + y * y + z * z;
    T dre = 1, dim = 0;  // R_m^m
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            T s = T(-0.5) / T(m);
            T nre = s * (x * dre - y * dim);
            T nim = s * (x * dim + y * dre);
            dre = nre;
            dim = nim;
        }
        T p2re = 0, p2im = 0, p1re = dre, p1im = dim;
        out[cre(m, m)] = dre;
        if (m > 0) out[cim(m, m)] = dim;
        for (int n = m + 1; n <= p; ++n) {
            T a = T(2 * n - 1) * z, b = r2;
            T inv = T(1) / T((n + m) * (n - m));
            T cr = (a * p1re - b * p2re) * inv;
            T ci = (a * p1im - b * p2im) * inv;
            out[cre(n, m)] = cr;
            if (m > 0) out[cim(n, m)] = ci;
            p2re = p1re;
            p2im = p1im;
            p1re = cr;
            p1im = ci;
        }
    }
}

// Irregular solid harmonics I_n^m (sign (-1)^(n+m) folded in) up to degree pmax,
// complex m >= 0 only: out[n*(n+1)/2 + m].
//   I_0^0 = 1/r,  I_m^m = -(2m-1)(x + i y) I_{m-1}^{m-1} / r^2,
//   I_n^m = (-(2n-1) z I_{n-1}^m - (n+m-1)(n-m-1) I_{n-2}^m) / r^2.
__host__ __device__ inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }

template <typename T>
__host__ __device__ inline void irregular_tri(int pmax, T x, T y, T z, Cx<T> *out)
{
    T r2 = x * x + y * y + z * z;
    T ir2 = T(1) / r2;
    Cx<T> dg = {T(1) / sqrt(r2), T(0)};
    for (int m = 0; m <= pmax; ++m) {
        if (m > 0) {
            T s = -T(2 * m - 1) * ir2;
            Cx<T> nd = {s * (x * dg.re - y * dg.im), s * (x * dg.im + y * dg.re)};
            dg = nd;
        }
        out[tri(m, m)] = dg;
        Cx<T> p2 = {0, 0}, p1 = dg;
        for (int n = m + 1; n <= pmax; ++n) {
            T a = -T(2 * n - 1) * z, b = T((n + m - 1) * (n - m - 1));
            Cx<T> c = {(a * p1.re - b * p2.re) * ir2, (a * p1.im - b * p2.im) * ir2};
            out[tri(n, m)] = c;
            p2 = p1;
            p1 = c;
        }
    }
}

// complex coefficient of order m (any sign) from the real layout
template <typename T>
__host__ __device__ inline Cx<T> coef(const T *a, int n, int m)
{
    if (m == 0) return {a[n * n], T(0)};
    int am = m < 0 ? -m : m;
    Cx<T> v = {a[n * n + 2 * am - 1], a[n * n + 2 * am]};
    if (m < 0) {
        v.im = -v.im;
        if (am & 1) {
            v.re = -v.re;
            v.im = -v.im;
        }
    }
    return v;
}

// ------------------------------------------------------------------ launchers
// sort / reductions (fmm_sort.cu)
fmm_status launch_assign_sort(Plan &P, const double *pos, const double *q, const uint8_t *sol);
fmm_status launch_bc_moments(Plan &P, const double *q, const uint8_t *sol);
fmm_status launch_energy_reduce(Plan &P, bool with_uv);
fmm_status launch_forces_out(Plan &P, const double *q, double *forces);
fmm_status launch_potentials_out(Plan &P, double *potentials);

// expansions (fmm_expand.cu)
fmm_status build_tables(Plan &P);
fmm_status build_lattice(Plan &P);  // the kappa-dependent lattice table only
void free_tables(Plan &P);
fmm_status launch_upward(Plan &P, bool solute_only);
fmm_status launch_lattice(Plan &P);
fmm_status launch_m2l_simt(Plan &P, int level);

// M2M / L2L as dense products (fmm_translate.cu)
fmm_status build_translation_ops(Plan &P);
fmm_status launch_m2m(Plan &P, int level);  // level + 1 -> level
fmm_status launch_l2l(Plan &P, int level);  // level - 1 -> level (accumulates)
fmm_status launch_l2p(Plan &P, bool gradient, bool solute_only);

// near field (fmm_p2p.cu)
fmm_status launch_p2p(Plan &P, bool forces);
fmm_status launch_p2p_uv(Plan &P);

// sparse solute-only pass of Eq. FMMcalc (fmm_solute.cu)
fmm_status solute_prepare(Plan &P);
void solute_free(Plan &P);
// right after the sort: count the solute charges and copy the count to the host asynchronously
fmm_status solute_count(Plan &P);
// the host copy of the last solute count (valid once the plan's stream has passed the copy); -1 when the
// plan has no sparse pass
int solute_count_host(const Plan &P);
// after the full pass's upward sweep: the pass's prologue (active cells, solute moments, FP64 solvent
// expansions at the active cells) on a high-priority side stream, overlapping the full pass's M2L
fmm_status solute_prologue(Plan &P);
// right after the prologue (P.overlap): the rest of the sparse pass on the side stream (it touches none of
// the full pass's expansions) and Phi_u at every charge on the near stream when that is forked; grids
// cover the largest count and the device count decides
fmm_status solute_sparse_fork(Plan &P);
// joins the prologue (or the forked sparse pass) and runs the rest; *done = false when the dense pass must run
fmm_status launch_solute_pass(Plan &P, bool *done);

// tensor-core M2L, and with the fp16 split also M2M and L2L (fmm_m2l_tc.cu)
bool tc_available(const Plan &P, int level);
// fp16 split: M2M on the tensor cores and L2L fused into each level's M2L
bool tc_translations(const Plan &P);
fmm_status tc_prepare(Plan &P);
// fp16 split: balanced halo planes of M[level] (done by the upward pass before the M2M into level - 1);
// amax_ready: the kernel that wrote M[level] has already folded the level's largest |Mhat s| into
// tc_amax(P, level) (else it is computed here)
fmm_status tc_split_moments(Plan &P, int level, bool amax_ready);
// fp16 split: the device word of level l's largest |Mhat s| (float bits), cleared by tc_clear_amax before
// the kernel that produces M[l] folds its maximum in; s(n,m) per real coefficient
unsigned *tc_amax(Plan &P, int level);
fmm_status tc_clear_amax(Plan &P, int level);
const float *tc_scale(const Plan &P);
// fp16 split: M2M into level (< d) from the planes of level + 1
fmm_status launch_m2m_tc(Plan &P, int level);
// precise: at least the accuracy of the 3 x 3 bf16 split whatever the plan's option (solute-only pass);
// split: (re)build the planes of M[level] first (always done for the bf16 splits).  With the fp16
// split the L2L from level - 1 is included: L[level] = M2L + L2L.
fmm_status launch_m2l_tc(Plan &P, int level, bool precise = false, bool split = true);
void tc_free(Plan &P);

// phases of one energy + solute-solvent evaluation on device inputs (fmm_api.cu), for the batch API:
// front (sort .. near field) and back (solute pass, reductions, asynchronous copy of the results into
// P.h_out) only enqueue work, except that back waits for the host copy of the solute count unless
// P.known_count >= 0; results are read after the plan's stream is synchronised
fmm_status eval_enqueue_front(Plan &P, const double *dpos, const double *dq, const uint8_t *dsol);
fmm_status eval_enqueue_far_tail(Plan &P);
fmm_status eval_enqueue_back(Plan &P, const double *dq);

// the level-l tile brick of the tensor-core M2L (and of the M2M from level l); see FMM_OPT_M2L_BRICK
fmm_status tc_set_brick(Plan &P, int l, int bx, int by, int bz);
void tc_get_brick(const Plan &P, int l, int *bx, int *by, int *bz);

// dst reads src's split operator tables when they are the same (p, ws, split); src must outlive dst
fmm_status tc_share_operators(Plan &dst, const Plan &src);

// persistent sweep of the CTA-pair tensor-core levels of many plans in one launch (fmm_m2l_tc.cu)
struct Sweep;
int tc_sweep_first_level(const Plan &P);  // first level a sweep can take (0: none)
// a sweep over the plans that can take part (same expansion order); *out stays null when none can;
// sets their sweep_from
fmm_status sweep_create(Plan *const *plans, int n, Sweep **out);
void sweep_enable(Sweep *sw, bool on);  // sets or clears the plans' sweep_from
int sweep_plans(const Sweep *sw);
// max_pairs > 0 caps the CTA pairs (the rest of the GPU stays free for the boxes' other streams)
fmm_status sweep_launch(Sweep *sw, cudaStream_t st, uint64_t wait_ns, bool stall, int max_pairs);
void sweep_destroy(Sweep *sw);
fmm_status eval_results(Plan &P, fmm_energy_terms *terms, fmm_uv_terms *uv);

#define FMM_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA; \
    } while (0)

#define FMM_LAUNCH_CHECK(P)                                       \
    do {                                                          \
        (P).launches++;                                           \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return FMM_ERR_CUDA;               \
    } while (0)

}  // namespace fmm

struct fmm_plan_s {
    fmm::Plan P;
};

