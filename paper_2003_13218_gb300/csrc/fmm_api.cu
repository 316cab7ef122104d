// fmm_api.cu -- the C ABI declared in include/fmm_gb300.h: plan lifecycle and
// the order of the stages of one evaluation (Appendix B: sort, P2M, M2M,
// level-0 lattice (Eq. 12), M2L + L2L per level, L2P, near field; then the
// background-charge terms of Eq. Velecfull and, on request, the solute-only
// pass of Eq. FMMcalc).
#include <math.h>
#include <string.h>

#include <new>

#include "fmm_internal.cuh"

using namespace fmm;

namespace {

size_t reduction_scratch_bytes() { return sizeof(double) * 304 * 20 * 2; }

void free_buffers(Plan &P)
{
    void *bufs[] = {P.in_pos, P.in_q,   P.out_forces, P.out_phi, P.in_sol, P.wpos,    P.key,    P.perm,   P.sleaf,
                    P.cell_start, P.cell_fill, P.scan_tmp, P.sorted, P.sorted_u, P.sorted_sol, P.phi_nf, P.phi_ff,
                    P.phi_u, P.f_nf, P.g_ff, P.red_partial, P.red_out, P.d_err, P.sc_out, P.sc_lambda};
    for (void *b : bufs) cudaFree(b);
    for (int l = 0; l <= 8; ++l) {
        cudaFree(P.M[l]);
        cudaFree(P.L[l]);
        P.M[l] = P.L[l] = nullptr;
    }
    if (P.h_out) cudaFreeHost(P.h_out);
    if (P.h_sc_lambda) cudaFreeHost(P.h_sc_lambda);
    P.sc_out = P.sc_lambda = P.h_sc_lambda = nullptr;
    P.in_pos = P.in_q = P.out_forces = P.out_phi = nullptr;
    P.in_sol = nullptr;
    P.wpos = nullptr;
    P.key = P.perm = P.sleaf = P.cell_start = P.cell_fill = P.scan_tmp = nullptr;
    P.sorted = P.sorted_u = nullptr;
    P.sorted_sol = nullptr;
    P.phi_nf = P.phi_ff = P.phi_u = P.f_nf = P.g_ff = nullptr;
    P.red_partial = P.red_out = P.h_out = nullptr;
    P.d_err = nullptr;
}

template <typename X>
cudaError_t dalloc(X **p, size_t bytes)
{
    return cudaMalloc((void **)p, bytes < 16 ? 16 : bytes);
}

fmm_status alloc_buffers(Plan &P)
{
    int64_t N = P.N;
    size_t nc = (size_t)P.nc;
    // sized for FP64 so that the precision option can switch without reallocation
    FMM_CUDA_TRY(dalloc(&P.wpos, sizeof(double) * 3 * N));
    FMM_CUDA_TRY(dalloc(&P.key, sizeof(int) * N));
    FMM_CUDA_TRY(dalloc(&P.perm, sizeof(int) * N));
    FMM_CUDA_TRY(dalloc(&P.sleaf, sizeof(int) * N));
    FMM_CUDA_TRY(dalloc(&P.cell_start, sizeof(int) * (P.nleaf + 1)));
    FMM_CUDA_TRY(dalloc(&P.cell_fill, sizeof(int) * P.nleaf));
    FMM_CUDA_TRY(dalloc(&P.scan_tmp, sizeof(int) * (P.nleaf / 4096 + 2)));
    FMM_CUDA_TRY(dalloc(&P.sorted, sizeof(Particle<double>) * N));
    FMM_CUDA_TRY(dalloc(&P.sorted_u, sizeof(Particle<double>) * N));
    FMM_CUDA_TRY(dalloc(&P.sorted_sol, N));
    FMM_CUDA_TRY(dalloc(&P.phi_nf, sizeof(double) * 2 * N));
    FMM_CUDA_TRY(dalloc(&P.phi_ff, sizeof(double) * N));
    FMM_CUDA_TRY(dalloc(&P.phi_u, sizeof(double) * N));
    FMM_CUDA_TRY(dalloc(&P.f_nf, sizeof(double) * 3 * N));
    FMM_CUDA_TRY(dalloc(&P.g_ff, sizeof(double) * 3 * N));
    for (int l = 0; l <= P.d; ++l) {
        size_t cells = (size_t)1 << (3 * l);
        FMM_CUDA_TRY(dalloc(&P.M[l], sizeof(double) * cells * nc));
        FMM_CUDA_TRY(dalloc(&P.L[l], sizeof(double) * cells * nc));
    }
    FMM_CUDA_TRY(dalloc(&P.red_partial, reduction_scratch_bytes()));
    FMM_CUDA_TRY(dalloc(&P.red_out, sizeof(double) * 48));
    FMM_CUDA_TRY(dalloc(&P.d_err, sizeof(int)));
    FMM_CUDA_TRY(cudaMallocHost((void **)&P.h_out, sizeof(double) * 40));
    return FMM_OK;
}

// 0 = device (or managed) memory, 1 = host memory, -1 = null
int pointer_kind(const void *ptr)
{
    if (!ptr) return -1;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 0 : 1;
}

fmm_status ensure_staging(Plan &P)
{
    if (!P.in_pos) FMM_CUDA_TRY(dalloc(&P.in_pos, sizeof(double) * 3 * P.N));
    if (!P.in_q) FMM_CUDA_TRY(dalloc(&P.in_q, sizeof(double) * P.N));
    if (!P.in_sol) FMM_CUDA_TRY(dalloc(&P.in_sol, P.N));
    if (!P.out_forces) FMM_CUDA_TRY(dalloc(&P.out_forces, sizeof(double) * 3 * P.N));
    if (!P.out_phi) FMM_CUDA_TRY(dalloc(&P.out_phi, sizeof(double) * P.N));
    return FMM_OK;
}

struct StageTimer {
    Plan &P;
    int k = 0;
    explicit StageTimer(Plan &p) : P(p) {}
    void mark()
    {
        if (P.timings_on && k < 12) cudaEventRecord(P.ev[k++], P.stream);
    }
};

#define TRY(x)                               \
    do {                                     \
        fmm_status s_ = (x);                 \
        if (s_ != FMM_OK) return s_;         \
    } while (0)

fmm_status far_field_pass(Plan &P, bool gradient, bool solute_only, StageTimer *tm, bool fork_solute = false)
{
    TRY(launch_upward(P, solute_only));
    if (fork_solute) {
        TRY(solute_prologue(P));
        TRY(solute_sparse_fork(P));
    }
    if (tm) tm->mark();
    TRY(launch_lattice(P));
    if (tm) tm->mark();
    bool ev = tm && P.timings_on;
    // a batch's persistent sweep runs the levels >= sweep_from of the full pass, and its L2P after that
    const int last = (!solute_only && P.sweep_from > 0) ? P.sweep_from - 1 : P.d;
    for (int l = 1; l <= last; ++l) {
        if (ev) cudaEventRecord(P.ev_m2l[2 * (l - 1)], P.stream);
        // with the fp16 split the upward pass left the planes split and the L2L is fused
        const bool fused = tc_available(P, l) && tc_translations(P);
        if (tc_available(P, l)) TRY(launch_m2l_tc(P, l, solute_only, !fused));
        else TRY(launch_m2l_simt(P, l));
        if (ev) cudaEventRecord(P.ev_m2l[2 * (l - 1) + 1], P.stream);
        if (!fused) TRY(launch_l2l(P, l));
    }
    if (tm) tm->mark();
    if (last < P.d) return FMM_OK;
    TRY(launch_l2p(P, gradient, solute_only));
    if (tm) tm->mark();
    return FMM_OK;
}

// the work of one call that needs only the sort, on the plan's near stream (P.overlap): the background
// moments, the near field and the solute-solvent near-field sum
fmm_status fork_near_field(Plan &P, const double *dq, const uint8_t *dsol, bool gradient, bool want_uv)
{
    FMM_CUDA_TRY(cudaEventRecord(P.ev_sorted, P.stream));
    FMM_CUDA_TRY(cudaStreamWaitEvent(P.near, P.ev_sorted, 0));
    P.near_forked = P.near_p2p = true;
    cudaStream_t main_stream = P.stream;
    P.stream = P.near;
    fmm_status s = launch_bc_moments(P, dq, dsol);
    if (s == FMM_OK) s = launch_p2p(P, gradient);
    if (s == FMM_OK && want_uv) s = launch_p2p_uv(P);
    P.stream = main_stream;
    return s;
}

// the near stream's work of the call (the forked solute pass may have added to it) into the plan's stream
fmm_status join_near_field(Plan &P)
{
    if (!P.near_forked) return FMM_OK;
    P.near_forked = false;
    FMM_CUDA_TRY(cudaEventRecord(P.ev_near, P.near));
    FMM_CUDA_TRY(cudaStreamWaitEvent(P.stream, P.ev_near, 0));
    return FMM_OK;
}

// front of one evaluation on device inputs: sort, solute count, background
// moments, full far-field pass (with the solute prologue forked), near field
fmm_status eval_front(Plan &P, const double *dpos, const double *dq, const uint8_t *dsol, bool want_uv,
                      bool gradient, StageTimer *tm)
{
    if (tm) tm->mark();
    FMM_CUDA_TRY(cudaMemsetAsync(P.d_err, 0, sizeof(int), P.stream));
    if (want_uv && P.sc_c > 0)  // the soft-core lambda as it is when the call runs
        FMM_CUDA_TRY(cudaMemcpyAsync(P.sc_lambda, P.h_sc_lambda, sizeof(double), cudaMemcpyHostToDevice, P.stream));
    P.near_forked = P.near_p2p = false;
    TRY(launch_assign_sort(P, dpos, dq, dsol));
    if (want_uv) TRY(solute_count(P));
    if (tm) tm->mark();
    if (P.overlap && P.near) TRY(fork_near_field(P, dq, dsol, gradient, want_uv));
    else TRY(launch_bc_moments(P, dq, dsol));
    TRY(far_field_pass(P, gradient, false, tm, want_uv));
    if (!P.near_p2p) TRY(launch_p2p(P, gradient));
    if (tm) tm->mark();
    return FMM_OK;
}

// back of one evaluation: solute pass (its count is read from the host copy,
// or P.known_count), reductions, forces, and the asynchronous copy of the
// totals and the error flags into P.h_out
fmm_status eval_back(Plan &P, const double *dq, bool want_uv, double *dforces, StageTimer *tm,
                     double *dphi = nullptr)
{
    TRY(join_near_field(P));
    if (want_uv) {
        bool sparse_done = false;
        TRY(launch_solute_pass(P, &sparse_done));
        if (!sparse_done) TRY(far_field_pass(P, false, true, nullptr));
        if (!P.near_p2p) TRY(launch_p2p_uv(P));
    }
    if (tm) tm->mark();
    TRY(launch_energy_reduce(P, want_uv));
    if (dforces) TRY(launch_forces_out(P, dq, dforces));
    if (dphi) TRY(launch_potentials_out(P, dphi));
    if (tm) tm->mark();
    FMM_CUDA_TRY(cudaMemcpyAsync(P.h_out, P.red_out, sizeof(double) * 31, cudaMemcpyDeviceToHost, P.stream));
    FMM_CUDA_TRY(cudaMemcpyAsync(P.h_out + 32, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    return FMM_OK;
}

// results of the last evaluation from P.h_out (the plan's stream synchronised)
fmm_status eval_read(Plan &P, fmm_energy_terms *terms, fmm_uv_terms *uv)
{
    int err;
    memcpy(&err, P.h_out + 32, sizeof(int));
    if (terms) {
        terms->near = P.h_out[16];
        terms->far = P.h_out[17];
        terms->charged = P.h_out[18];
        terms->quad_surface = P.h_out[19];
        terms->dipole_surface = P.h_out[20];
        terms->total = P.h_out[21];
    }
    if (uv) {
        uv->e_uv = P.h_out[22];
        uv->W = P.h_out[23];
        uv->A = P.h_out[24];
        uv->B = P.h_out[25];
        uv->C = P.h_out[26];
        uv->nf_uv = P.h_out[27];
        uv->bc_cross = P.h_out[28];
        uv->nf_sc = P.sc_c > 0 ? P.h_out[29] : 0.0;
        uv->dnf_sc = P.sc_c > 0 ? P.h_out[30] : 0.0;
    }
    if (err & ERRF_NONFINITE) return FMM_ERR_NONFINITE;
    if (err & ERRF_TIMEOUT) return FMM_ERR_TIMEOUT;
    if (err) return FMM_ERR_INTERNAL;
    return FMM_OK;
}

// one call on the plan's execution stream (P.overlap): forked from the caller's stream on entry, joined
// back into it on every exit (a failed call's near field included)
struct ExecScope {
    Plan &P;
    cudaStream_t caller = 0;
    bool active = false;
    fmm_status status = FMM_OK;
    explicit ExecScope(Plan &p) : P(p)
    {
        if (!P.overlap || !P.exec) return;
        caller = P.stream;
        if (cudaEventRecord(P.ev_in, caller) != cudaSuccess || cudaStreamWaitEvent(P.exec, P.ev_in, 0) != cudaSuccess) {
            status = FMM_ERR_CUDA;
            return;
        }
        P.stream = P.exec;
        active = true;
    }
    ~ExecScope()
    {
        if (!active) return;
        if (P.near_forked) {  // a failed call
            cudaEventRecord(P.ev_near, P.near);
            cudaStreamWaitEvent(P.exec, P.ev_near, 0);
            P.near_forked = false;
        }
        cudaEventRecord(P.ev_out, P.exec);
        cudaStreamWaitEvent(caller, P.ev_out, 0);
        P.stream = caller;
    }
};

fmm_status evaluate(Plan &P, const double *pos, const double *q, const uint8_t *sol, double *forces,
                    fmm_energy_terms *terms, fmm_uv_terms *uv, double *potentials = nullptr)
{
    if (!pos || !q) return FMM_ERR_INVALID_ARG;
    bool want_uv = sol && uv;
    int kp = pointer_kind(pos), kq = pointer_kind(q);
    int ks = want_uv ? pointer_kind(sol) : -1;
    int kf = pointer_kind(forces);
    int kphi = pointer_kind(potentials);
    bool host_any = kp == 1 || kq == 1 || ks == 1 || kf == 1 || kphi == 1;
    if (host_any) TRY(ensure_staging(P));
    ExecScope xs(P);
    TRY(xs.status);
    P.launches = 0;
    P.top_recorded = false;
    const double *dpos = pos, *dq = q;
    const uint8_t *dsol = want_uv ? sol : nullptr;
    double *dforces = forces;
    if (kp == 1) {
        FMM_CUDA_TRY(cudaMemcpyAsync(P.in_pos, pos, sizeof(double) * 3 * P.N, cudaMemcpyHostToDevice, P.stream));
        dpos = P.in_pos;
    }
    if (kq == 1) {
        FMM_CUDA_TRY(cudaMemcpyAsync(P.in_q, q, sizeof(double) * P.N, cudaMemcpyHostToDevice, P.stream));
        dq = P.in_q;
    }
    if (ks == 1) {
        FMM_CUDA_TRY(cudaMemcpyAsync(P.in_sol, sol, P.N, cudaMemcpyHostToDevice, P.stream));
        dsol = P.in_sol;
    }
    if (kf == 1) dforces = P.out_forces;
    double *dphi = kphi == 1 ? P.out_phi : potentials;

    StageTimer tm(P);
    TRY(eval_front(P, dpos, dq, dsol, want_uv, forces != nullptr, &tm));
    TRY(eval_back(P, dq, want_uv, dforces, &tm, dphi));
    if (kf == 1)
        FMM_CUDA_TRY(cudaMemcpyAsync(forces, P.out_forces, sizeof(double) * 3 * P.N, cudaMemcpyDeviceToHost, P.stream));
    if (kphi == 1)
        FMM_CUDA_TRY(cudaMemcpyAsync(potentials, P.out_phi, sizeof(double) * P.N, cudaMemcpyDeviceToHost, P.stream));
    bool sync = terms || uv || kf == 1 || kphi == 1;
    if (!sync) return FMM_OK;
    FMM_CUDA_TRY(cudaStreamSynchronize(P.stream));
    if (P.timings_on && tm.k >= 9) {
        float t[12];
        for (int i = 0; i + 1 < tm.k; ++i) cudaEventElapsedTime(&t[i], P.ev[i], P.ev[i + 1]);
        P.last.sort = t[0];
        P.last.upward = t[1];
        P.last.lattice = t[2];
        P.last.m2l_l2l = t[3];
        P.last.l2p = t[4];
        P.last.p2p = t[5];
        P.last.solute_pass = t[6];
        P.last.reduce = t[7];
        cudaEventElapsedTime(&P.last.total, P.ev[0], P.ev[tm.k - 1]);
        float m = 0;
        for (int l = 1; l <= P.d; ++l) {
            float x = 0;
            cudaEventElapsedTime(&x, P.ev_m2l[2 * (l - 1)], P.ev_m2l[2 * (l - 1) + 1]);
            m += x;
        }
        P.last.m2l_kernels = m;
        P.last.m2l_top = 0;
        if (P.top_recorded) cudaEventElapsedTime(&P.last.m2l_top, P.ev_top[0], P.ev_top[1]);
    }
    return eval_read(P, terms, uv);
}

// the plan's execution stream (one priority level above the default) and its near-field stream (the
// default, lowest priority): the block scheduler serves the far field first and gives the near field the
// SMs, registers and warp slots the far field leaves free
fmm_status create_streams(Plan &P)
{
    int lo = 0, hi = 0;
    FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    const int mid = hi < lo ? lo - 1 : lo;  // numerically smaller = higher priority
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&P.exec, cudaStreamNonBlocking, mid));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&P.near, cudaStreamNonBlocking, lo));
    for (cudaEvent_t *e : {&P.ev_in, &P.ev_out, &P.ev_sorted, &P.ev_near})
        FMM_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return FMM_OK;
}

// tensor-core operands follow the precision and split options
fmm_status retc(Plan &P)
{
    tc_free(P);
    if (P.precision == FMM_PREC_MIXED && P.split != FMM_SPLIT_FP32) TRY(tc_prepare(P));
    return FMM_OK;
}

fmm_status rebuild(Plan &P)
{
    TRY(build_tables(P));
    return retc(P);
}

}  // namespace

namespace fmm {

// the phases of one energy + solute-solvent evaluation without forces, for the
// batch API (device inputs, no timings, results read after a stream sync)
fmm_status eval_enqueue_front(Plan &P, const double *dpos, const double *dq, const uint8_t *dsol)
{
    P.launches = 0;
    P.top_recorded = false;
    return eval_front(P, dpos, dq, dsol, true, false, nullptr);
}

// the far-field pass's L2P when the deeper levels ran in a batch's sweep (after it, on the plan's stream)
fmm_status eval_enqueue_far_tail(Plan &P) { return P.sweep_from > 0 ? launch_l2p(P, false, false) : FMM_OK; }

fmm_status eval_enqueue_back(Plan &P, const double *dq) { return eval_back(P, dq, true, nullptr, nullptr); }

fmm_status eval_results(Plan &P, fmm_energy_terms *terms, fmm_uv_terms *uv) { return eval_read(P, terms, uv); }

}  // namespace fmm

extern "C" {

fmm_status fmm_plan_create(double box, int64_t N, int depth, int p, fmm_plan *out)
{
    if (!out) return FMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!(box > 0.0) || !isfinite(box) || N < 1 || N > ((int64_t)1 << 31) - 1 || p < 0 || p > P_MAX || depth < 2 ||
        depth > 8)
        return FMM_ERR_INVALID_ARG;
    fmm_plan_s *h = new (std::nothrow) fmm_plan_s();
    if (!h) return FMM_ERR_OOM;
    Plan &P = h->P;
    P.box = box;
    P.N = N;
    P.d = depth;
    P.p = p;
    P.nc = ncoef(p);
    P.nleaf = (int64_t)1 << (3 * depth);
    fmm_status s = alloc_buffers(P);
    if (s == FMM_OK) {
        for (int i = 0; i < 12; ++i) cudaEventCreate(&P.ev[i]);
        for (int i = 0; i < 18; ++i) cudaEventCreate(&P.ev_m2l[i]);
        for (int i = 0; i < 2; ++i) cudaEventCreate(&P.ev_top[i]);
        s = create_streams(P);
        if (s == FMM_OK) s = solute_prepare(P);
        if (s == FMM_OK) s = rebuild(P);
    }
    if (s != FMM_OK) {
        fmm_plan_destroy(h);
        return s;
    }
    *out = h;
    return FMM_OK;
}

fmm_status fmm_plan_set_option(fmm_plan plan, int key, int64_t ival, double dval)
{
    if (!plan) return FMM_ERR_INVALID_ARG;
    Plan &P = plan->P;
    switch (key) {
    case FMM_OPT_WS: {
        if (ival < 1) return FMM_ERR_INVALID_ARG;
        if (ival > WS_MAX) return FMM_ERR_UNSUPPORTED;
        if ((1 << P.d) <= 2 * ival + 1) return FMM_ERR_INVALID_ARG;  // the near field would hold own images
        if (P.ws == (int)ival) return FMM_OK;
        P.ws = (int)ival;
        fmm_status st = solute_prepare(P);  // interaction-list sized buffers
        return st == FMM_OK ? rebuild(P) : st;
    }
    case FMM_OPT_PRECISION:
        if (ival != FMM_PREC_FP64 && ival != FMM_PREC_MIXED) return FMM_ERR_INVALID_ARG;
        if (P.precision == (int)ival) return FMM_OK;
        P.precision = (int)ival;
        return retc(P);
    case FMM_OPT_KAPPA:
        if (!isfinite(dval)) return FMM_ERR_INVALID_ARG;
        P.kappa = dval > 0 ? dval : 0.0;
        return build_lattice(P);
    case FMM_OPT_M2L_SPLIT:
        if (ival != FMM_SPLIT_BF16X3 && ival != FMM_SPLIT_BF16X2 && ival != FMM_SPLIT_FP32 &&
            ival != FMM_SPLIT_BF16_A2B3 && ival != FMM_SPLIT_FP16X2)
            return FMM_ERR_INVALID_ARG;
        if (P.split == (int)ival) return FMM_OK;
        P.split = (int)ival;
        return retc(P);
    case FMM_OPT_STREAM:
        P.stream = (cudaStream_t)(intptr_t)ival;
        return FMM_OK;
    case FMM_OPT_TIMINGS:
        P.timings_on = ival != 0;
        return FMM_OK;
    case FMM_OPT_BOUNDARY:
        if (ival != FMM_BOUNDARY_CONDUCTING && ival != FMM_BOUNDARY_VACUUM) return FMM_ERR_INVALID_ARG;
        P.boundary = (int)ival;
        return FMM_OK;
    case FMM_OPT_M2L_PAIR:
        if (ival != 0 && ival != 1) return FMM_ERR_INVALID_ARG;
        P.tc_pair = ival != 0;
        return FMM_OK;
    case FMM_OPT_M2L_GRADE: {
        const int64_t d2 = ival & 0xFF, d1 = (ival >> 8) & 0xFF;
        if (ival < 0 || (ival >> 16) != 0 || d2 > P_MAX || d1 > P_MAX) return FMM_ERR_INVALID_ARG;
        P.grade = (int)ival;
        return FMM_OK;
    }
    case FMM_OPT_M2L_ACC_GROUP:
        if (ival < 1 || ival > 64) return FMM_ERR_INVALID_ARG;
        P.acc_group = (int)ival;
        return FMM_OK;
    case FMM_OPT_SOFTCORE:
        if (ival < 0 || ival > 12) return FMM_ERR_INVALID_ARG;
        if (ival > 0 && !(dval > 0.0 && isfinite(dval))) return FMM_ERR_INVALID_ARG;
        if (ival > 0 && !P.sc_out) {  // buffers on first use, never inside an evaluation
            FMM_CUDA_TRY(dalloc(&P.sc_out, sizeof(double) * 2 * P.N));
            FMM_CUDA_TRY(dalloc(&P.sc_lambda, sizeof(double)));
            FMM_CUDA_TRY(cudaMallocHost((void **)&P.h_sc_lambda, sizeof(double)));
            *P.h_sc_lambda = 0.0;
        }
        P.sc_c = (int)ival;
        P.sc_A = ival > 0 ? dval : 0.0;
        return FMM_OK;
    case FMM_OPT_SOFTCORE_LAMBDA:
        if (!(dval >= 0.0 && dval <= 1.0)) return FMM_ERR_INVALID_ARG;
        if (!P.h_sc_lambda) return P.sc_c > 0 ? FMM_ERR_INTERNAL : FMM_ERR_INVALID_ARG;  // set FMM_OPT_SOFTCORE first
        *P.h_sc_lambda = dval;
        return FMM_OK;
    case FMM_OPT_SOFTCORE_ALPHA:
        if (!(dval > 0.0 && isfinite(dval))) return FMM_ERR_INVALID_ARG;
        P.sc_alpha = dval;
        return FMM_OK;
    case FMM_OPT_WAIT_BUDGET_NS:
        if (ival < 1000 || ival > 10000000000ll) return FMM_ERR_INVALID_ARG;
        P.wait_ns = (uint64_t)ival;
        return FMM_OK;
    case FMM_OPT_INJECT_STALL:
        if (ival != 0 && ival != 1) return FMM_ERR_INVALID_ARG;
        P.inject_stall = ival != 0;
        return FMM_OK;
    case FMM_OPT_M2L_BRICK:
        if (ival < 0 || ival > 0xFFFFFFFFll) return FMM_ERR_INVALID_ARG;
        return tc_set_brick(P, (int)(ival & 0xFF), (int)((ival >> 8) & 0xFF), (int)((ival >> 16) & 0xFF),
                            (int)((ival >> 24) & 0xFF));
    case FMM_OPT_OVERLAP:
        if (ival != 0 && ival != 1) return FMM_ERR_INVALID_ARG;
        P.overlap = ival != 0;
        return FMM_OK;
    default:
        return FMM_ERR_INVALID_ARG;
    }
}

fmm_status fmm_energy(fmm_plan plan, const double *pos, const double *q, double *energy, fmm_energy_terms *terms)
{
    if (!plan || !energy) return FMM_ERR_INVALID_ARG;
    fmm_energy_terms t;
    fmm_status s = evaluate(plan->P, pos, q, nullptr, nullptr, &t, nullptr);
    if (s != FMM_OK) return s;
    *energy = t.total;
    if (terms) *terms = t;
    return FMM_OK;
}

fmm_status fmm_forces(fmm_plan plan, const double *pos, const double *q, double *forces, double *energy)
{
    if (!plan || !forces) return FMM_ERR_INVALID_ARG;
    fmm_energy_terms t;
    fmm_status s = evaluate(plan->P, pos, q, nullptr, forces, energy ? &t : nullptr, nullptr);
    if (s != FMM_OK) return s;
    if (energy) *energy = t.total;
    return FMM_OK;
}

fmm_status fmm_potentials(fmm_plan plan, const double *pos, const double *q, double *potentials, double *forces,
                          double *energy)
{
    if (!plan || !potentials) return FMM_ERR_INVALID_ARG;
    fmm_energy_terms t;
    fmm_status s = evaluate(plan->P, pos, q, nullptr, forces, energy ? &t : nullptr, nullptr, potentials);
    if (s != FMM_OK) return s;
    if (energy) *energy = t.total;
    return FMM_OK;
}

fmm_status fmm_solute_solvent_energy(fmm_plan plan, const double *pos, const double *q, const uint8_t *is_solute,
                                     double *e_uv, fmm_uv_terms *terms)
{
    if (!plan || !e_uv || !is_solute) return FMM_ERR_INVALID_ARG;
    fmm_uv_terms u;
    fmm_status s = evaluate(plan->P, pos, q, is_solute, nullptr, nullptr, &u);
    if (s != FMM_OK) return s;
    *e_uv = u.e_uv;
    if (terms) *terms = u;
    return FMM_OK;
}

fmm_status fmm_evaluate(fmm_plan plan, const double *pos, const double *q, const uint8_t *is_solute, double *forces,
                        fmm_energy_terms *terms, fmm_uv_terms *uv)
{
    if (!plan) return FMM_ERR_INVALID_ARG;
    return evaluate(plan->P, pos, q, is_solute, forces, terms, uv);
}

fmm_status fmm_plan_get_timings(fmm_plan plan, fmm_timings *out)
{
    if (!plan || !out) return FMM_ERR_INVALID_ARG;
    *out = plan->P.last;
    return FMM_OK;
}

int64_t fmm_plan_last_launch_count(fmm_plan plan) { return plan ? plan->P.launches : -1; }

int fmm_plan_m2l_backend(fmm_plan plan, int level)
{
    if (!plan || level < 1 || level > plan->P.d) return -1;
    if (tc_available(plan->P, level)) return 2;
    return plan->P.precision == FMM_PREC_FP64 ? 0 : 1;
}

void fmm_plan_destroy(fmm_plan plan)
{
    if (!plan) return;
    Plan &P = plan->P;
    cudaStreamSynchronize(P.stream);
    if (P.exec) cudaStreamSynchronize(P.exec);
    if (P.near) cudaStreamSynchronize(P.near);
    tc_free(P);
    solute_free(P);
    free_tables(P);
    free_buffers(P);
    for (int i = 0; i < 12; ++i)
        if (P.ev[i]) cudaEventDestroy(P.ev[i]);
    for (int i = 0; i < 18; ++i)
        if (P.ev_m2l[i]) cudaEventDestroy(P.ev_m2l[i]);
    for (int i = 0; i < 2; ++i)
        if (P.ev_top[i]) cudaEventDestroy(P.ev_top[i]);
    for (cudaEvent_t e : {P.ev_in, P.ev_out, P.ev_sorted, P.ev_near})
        if (e) cudaEventDestroy(e);
    if (P.exec) cudaStreamDestroy(P.exec);
    if (P.near) cudaStreamDestroy(P.near);
    delete plan;
}

const char *fmm_status_string(fmm_status s)
{
    switch (s) {
    case FMM_OK: return "ok";
    case FMM_ERR_INVALID_ARG: return "invalid argument";
    case FMM_ERR_NONFINITE: return "non-finite position or charge";
    case FMM_ERR_CUDA: return "CUDA runtime error";
    case FMM_ERR_OOM: return "out of memory";
    case FMM_ERR_TIMEOUT: return "device wait timed out";
    case FMM_ERR_INTERNAL: return "internal consistency check failed";
    case FMM_ERR_UNSUPPORTED: return "option value not supported by this library";
    default: return "unknown status";
    }
}

}  // extern "C"
