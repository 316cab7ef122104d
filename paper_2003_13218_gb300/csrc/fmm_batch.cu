// fmm_batch.cu -- many independent boxes per call: the lambda windows (or
// trajectory frames) of a free-energy calculation, each box with its own size,
// charges and solute set.  Per box and call: the total energy of Eq.
// Velecfull, the solute-solvent interaction E_uv of Eq. FMMcalc with the
// background cross terms, and with the Coulomb coupling lambda_C of Eq.
// Vswucheme / Eq. FMMVTI, which is linear in lambda_C,
//     V_lambda = E_total - lambda_C E_uv,   dV_lambda / dlambda_C = -E_uv.
//
// GB300 execution: one plan per box, the boxes spread over up to 16 streams
// (longest first, round robin) so that the small, latency-bound boxes fill
// the GPU together.  A call enqueues the front of every box (sort .. near
// field) before any box waits for its solute count, then the back of every
// box, and synchronises once.  The first call also captures the whole batch
// into a CUDA graph with the solute counts it saw; later calls with the same
// input pointers replay the graph and check the counts the graph copied back,
// falling back to the enqueued path (and a new capture) when one changed.
//
// Depth: boxes given depth <= 0 get one chosen by timing: for each distinct
// starting depth d0 = round(log8(N / 3.8)) (about 3.8 charges per leaf, as in
// the paper's water boxes) the box of median size is timed at d0 - 1, d0 and
// d0 + 1 on uniform test charges, and the fastest offset is used for that
// group.
#include <math.h>

#include <algorithm>
#include <utility>
#include <new>
#include <vector>

#include "fmm_internal.cuh"

using namespace fmm;

namespace {

constexpr int BATCH_MAX_STREAMS = 16;

// uniform test charges for the depth tuner: alternating +-0.5 e, one solute
__global__ void k_tune_fill(int64_t N, double box, double *__restrict__ pos, double *__restrict__ q,
                            uint8_t *__restrict__ sol)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
        for (int c = 0; c < 3; ++c) {
            uint64_t x = z + 0xD1B54A32D192ED03ull * (uint64_t)(c + 1);
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            x ^= x >> 31;
            pos[3 * i + c] = box * (double)(x >> 11) * (1.0 / 9007199254740992.0);
        }
        q[i] = (i & 1) ? 0.5 : -0.5;
        sol[i] = i == 0;
    }
}

int depth_guess(int64_t N)
{
    int d = (int)lround(log((double)N / 3.8) / log(8.0));
    return d < 2 ? 2 : (d > 8 ? 8 : d);
}

fmm_status make_plan(double box, int64_t N, int d, int p, int precision, cudaStream_t st, fmm_plan *out)
{
    fmm_status s = fmm_plan_create(box, N, d, p, out);
    if (s == FMM_OK) s = fmm_plan_set_option(*out, FMM_OPT_PRECISION, precision, 0.0);
    if (s == FMM_OK) s = fmm_plan_set_option(*out, FMM_OPT_STREAM, (int64_t)(intptr_t)st, 0.0);
    if (s != FMM_OK && *out) {
        fmm_plan_destroy(*out);
        *out = nullptr;
    }
    return s;
}

// device time of one evaluation of plan h on the tuner's charges
fmm_status time_plan(fmm_plan h, const double *pos, const double *q, const uint8_t *sol, float *ms)
{
    Plan &P = h->P;
    cudaEvent_t e0, e1;
    FMM_CUDA_TRY(cudaEventCreate(&e0));
    FMM_CUDA_TRY(cudaEventCreate(&e1));
    fmm_status s = FMM_OK;
    float best = 1e30f;
    for (int it = 0; it < 3 && s == FMM_OK; ++it) {  // one warm-up, best of two
        cudaEventRecord(e0, P.stream);
        s = eval_enqueue_front(P, pos, q, sol);
        if (s == FMM_OK) s = eval_enqueue_back(P, q);
        cudaEventRecord(e1, P.stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = FMM_ERR_CUDA;
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (it > 0 && t < best) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return s;
}

}  // namespace

struct fmm_batch_s {
    int nbox = 0;
    int precision = FMM_PREC_MIXED;
    std::vector<fmm_plan> plans;
    std::vector<int> depth, order;  // order: boxes by descending N
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_done;
    cudaStream_t origin = nullptr;
    cudaEvent_t ev_start = nullptr;
    bool use_graph = true;
    int sc_c = 0;  // soft-core near field on every plan (fmm_batch_set_softcore)
    Sweep *sweep = nullptr;          // the tensor-core levels of the boxes in one persistent launch
    bool use_sweep = true;
    std::vector<cudaEvent_t> ev_front;
    cudaEvent_t ev_sweep = nullptr;
    uint64_t wait_ns = 2000000000ull;  // budget of the sweep's dependency waits
    bool stall = false;                // test hook: one dependency of the sweep is never met
    int sweep_pairs = 0;               // CTA pairs of the sweep (0: as many as can be resident)
    // what the tuner measured: relative energy error of p = 6, 8, 10, 12 against p = 15 on its water box
    // (-1: not measured), the order it chose (0: none), graph replay times with the sweep off and on (ms)
    double p_err[4] = {-1.0, -1.0, -1.0, -1.0};
    int p_tuned = 0;
    double ms_sweep[2] = {-1.0, -1.0};
    cudaGraphExec_t graph = nullptr;
    std::vector<const void *> gptr;  // input pointers the graph was captured with
    std::vector<int> gcount;         // solute counts it was captured with
    int64_t replays = 0, enqueued = 0;
};

namespace {

void batch_free(fmm_batch b)
{
    if (!b) return;
    for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
    if (b->origin) cudaStreamSynchronize(b->origin);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    sweep_destroy(b->sweep);
    for (cudaEvent_t e : b->ev_front) cudaEventDestroy(e);
    if (b->ev_sweep) cudaEventDestroy(b->ev_sweep);
    for (fmm_plan h : b->plans)
        if (h) fmm_plan_destroy(h);
    for (cudaEvent_t e : b->ev_done) cudaEventDestroy(e);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

// the whole batch once: fronts of all boxes, then (with the sweep) the deeper
// tensor-core levels of every box in one persistent launch on the origin stream
// and each box's L2P after it, then backs (each back waits for its box's
// solute count unless the plan carries a known count)
fmm_status batch_enqueue(fmm_batch b, const double *const *pos, const double *const *q, const uint8_t *const *sol)
{
    for (int i : b->order) {
        fmm_status s = eval_enqueue_front(b->plans[i]->P, pos[i], q[i], sol[i]);
        if (s != FMM_OK) return s;
    }
    if (b->sweep && b->use_sweep) {
        for (size_t k = 0; k < b->streams.size(); ++k) {
            FMM_CUDA_TRY(cudaEventRecord(b->ev_front[k], b->streams[k]));
            FMM_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_front[k], 0));
        }
        fmm_status s = sweep_launch(b->sweep, b->origin, b->wait_ns, b->stall, b->sweep_pairs);
        if (s != FMM_OK) return s;
        FMM_CUDA_TRY(cudaEventRecord(b->ev_sweep, b->origin));
        for (cudaStream_t st : b->streams) FMM_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_sweep, 0));
        for (int i : b->order) {
            s = eval_enqueue_far_tail(b->plans[i]->P);
            if (s != FMM_OK) return s;
        }
    }
    for (int i : b->order) {
        fmm_status s = eval_enqueue_back(b->plans[i]->P, q[i]);
        if (s != FMM_OK) return s;
    }
    return FMM_OK;
}

fmm_status batch_sync(fmm_batch b)
{
    for (cudaStream_t s : b->streams) FMM_CUDA_TRY(cudaStreamSynchronize(s));
    return FMM_OK;
}

// capture the batch with the solute counts of the call just completed
void batch_capture(fmm_batch b, const double *const *pos, const double *const *q, const uint8_t *const *sol)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->gcount.assign(b->nbox, -1);
    for (int i = 0; i < b->nbox; ++i) {
        b->gcount[i] = solute_count_host(b->plans[i]->P);
        b->plans[i]->P.known_count = b->gcount[i];
    }
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        ok = cudaEventRecord(b->ev_start, b->origin) == cudaSuccess;
        for (cudaStream_t s : b->streams) ok = ok && cudaStreamWaitEvent(s, b->ev_start, 0) == cudaSuccess;
        ok = ok && batch_enqueue(b, pos, q, sol) == FMM_OK;
        for (size_t k = 0; k < b->streams.size(); ++k) {
            ok = ok && cudaEventRecord(b->ev_done[k], b->streams[k]) == cudaSuccess;
            ok = ok && cudaStreamWaitEvent(b->origin, b->ev_done[k], 0) == cudaSuccess;
        }
        if (cudaStreamEndCapture(b->origin, &g) != cudaSuccess) ok = false;
    }
    if (ok && g) ok = cudaGraphInstantiate(&b->graph, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->use_graph = false;  // this batch stays on the enqueued path
    }
    cudaGetLastError();
    for (int i = 0; i < b->nbox; ++i) b->plans[i]->P.known_count = -1;
    b->gptr.clear();
    for (int i = 0; i < b->nbox; ++i) {
        b->gptr.push_back(pos[i]);
        b->gptr.push_back(q[i]);
        b->gptr.push_back(sol[i]);
    }
}

bool graph_matches(fmm_batch b, const double *const *pos, const double *const *q, const uint8_t *const *sol)
{
    if (!b->graph || (int)b->gptr.size() != 3 * b->nbox) return false;
    for (int i = 0; i < b->nbox; ++i)
        if (b->gptr[3 * i] != pos[i] || b->gptr[3 * i + 1] != q[i] || b->gptr[3 * i + 2] != sol[i]) return false;
    return true;
}

// SplitMix64 (Steele, Lea and Flood 2014): the tuner's own stream of test coordinates
struct SplitMix {
    uint64_t x;
    uint64_t next()
    {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// A water-like test box for the order tuner: a +2 e ion at the box centre (the corner that cells of every
// level share: the slowest-converging place for a charge) and floor((N - 1) / 3) rigid 3-site waters
// (O -0.834 e, H +0.417 e, O-H 0.9572 A, H-O-H 104.52 deg) with O on the other sites of an n^3 lattice
// of side L, site i at (i + (n mod 2) / 2) L / n (taken in a random order, jittered by U(-0.3, 0.3) A),
// each molecule turned by a uniformly random rotation (a uniform unit quaternion, Shoemake 1992); the
// remaining (N - 1) mod 3 sites carry no charge.  Coordinates wrapped into [0, L).  For even n the
// molecules sit on the faces of the cells of the levels below the lattice spacing and straddle them:
// the harder case for the truncated expansions, so the order found is the safer one.
void water_test_box(int64_t N, double L, uint64_t seed, std::vector<double> &pos, std::vector<double> &q)
{
    SplitMix rng{seed};
    const int64_t nw = (N - 1) / 3, extra = (N - 1) % 3;
    int64_t n = 1;
    while (n * n * n < nw + extra + 1) ++n;
    const double a = L / (double)n;
    std::vector<int64_t> site((size_t)(n * n * n));
    for (int64_t i = 0; i < (int64_t)site.size(); ++i) site[i] = i;
    for (int64_t i = (int64_t)site.size() - 1; i > 0; --i) std::swap(site[i], site[rng.next() % (uint64_t)(i + 1)]);
    const double half = 0.5 * 104.52 * M_PI / 180.0, b = 0.9572;
    const double hx = b * sin(half), hy = b * cos(half);
    pos.assign(3 * (size_t)N, 0.0);
    q.assign((size_t)N, 0.0);
    auto wrap = [&](double x) {
        x = fmod(x, L);
        return x < 0.0 ? x + L : (x >= L ? 0.0 : x);
    };
    // the ion takes the lattice site nearest the centre; the molecules the others
    const int64_t ci = n / 2, centre = ci + n * (ci + n * ci);
    for (int64_t i = 0; i < (int64_t)site.size(); ++i)
        if (site[i] == centre) {
            std::swap(site[i], site.back());
            break;
        }
    int64_t k = 0;
    for (int d = 0; d < 3; ++d) pos[d] = 0.5 * L;
    q[k++] = 2.0;
    for (int64_t m = 0; m < nw + extra; ++m) {
        const int64_t c = site[m];
        const double off = 0.5 * (double)(n % 2);  // site n / 2 at L / 2; for even n the sites lie on cell faces
        double o[3] = {((double)(c % n) + off) * a, ((double)((c / n) % n) + off) * a, ((double)(c / (n * n)) + off) * a};
        for (int d = 0; d < 3; ++d) o[d] += 0.6 * rng.uniform() - 0.3;
        if (m >= nw) {  // an uncharged site
            for (int d = 0; d < 3; ++d) pos[3 * k + d] = wrap(o[d]);
            ++k;
            continue;
        }
        const double u1 = rng.uniform(), u2 = rng.uniform(), u3 = rng.uniform();
        const double qw = sqrt(1.0 - u1) * sin(2.0 * M_PI * u2), qx = sqrt(1.0 - u1) * cos(2.0 * M_PI * u2);
        const double qy = sqrt(u1) * sin(2.0 * M_PI * u3), qz = sqrt(u1) * cos(2.0 * M_PI * u3);
        const double R[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)},
                                {2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)},
                                {2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)}};
        const double h[2][3] = {{hx, hy, 0.0}, {-hx, hy, 0.0}};
        for (int d = 0; d < 3; ++d) pos[3 * k + d] = wrap(o[d]);
        q[k++] = -0.834;
        for (int t = 0; t < 2; ++t) {
            for (int d = 0; d < 3; ++d)
                pos[3 * k + d] = wrap(o[d] + R[d][0] * h[t][0] + R[d][1] * h[t][1] + R[d][2] * h[t][2]);
            q[k++] = 0.417;
        }
    }
}

// Relative energy errors, against an FP64 order-15 evaluation, of mixed-precision evaluations at
// p = 6, 8, 10, 12 on a water test box of N charges in a cell of side L at depth d: err[4].
fmm_status order_errors(int64_t N, double L, int d, cudaStream_t st, double err[4])
{
    std::vector<double> hpos, hq;
    water_test_box(N, L, 0x5EEDull + (uint64_t)N, hpos, hq);
    double *dpos = nullptr, *dq = nullptr;
    fmm_status s = FMM_OK;
    if (cudaMalloc(&dpos, sizeof(double) * hpos.size()) != cudaSuccess ||
        cudaMalloc(&dq, sizeof(double) * hq.size()) != cudaSuccess)
        s = FMM_ERR_OOM;
    if (s == FMM_OK && (cudaMemcpy(dpos, hpos.data(), sizeof(double) * hpos.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(dq, hq.data(), sizeof(double) * hq.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        s = FMM_ERR_CUDA;
    const int cand[5] = {6, 8, 10, 12, 15};
    double e[5] = {0, 0, 0, 0, 0};
    for (int c = 0; c < 5 && s == FMM_OK; ++c) {
        fmm_plan h = nullptr;
        s = make_plan(L, N, d, cand[c], c < 4 ? FMM_PREC_MIXED : FMM_PREC_FP64, st, &h);
        if (s == FMM_OK) s = fmm_energy(h, dpos, dq, &e[c], nullptr);
        if (h) fmm_plan_destroy(h);
    }
    cudaFree(dpos);
    cudaFree(dq);
    if (s != FMM_OK) return s;
    for (int c = 0; c < 4; ++c) err[c] = fabs(e[c] - e[4]) / fmax(fabs(e[4]), 1e-300);
    return FMM_OK;
}

// The deepest level's tile brick per depth group: the group's median box, uniform test charges, each
// power-of-two brick bx >= by >= bz of 128 cells that fits the level (an even number of tiles per class)
// timed on the box's own plan (time_plan: a warm-up and the best of two), the fastest set on every plan
// of the group.
fmm_status tune_bricks(fmm_batch b, const int64_t *N, const double *box)
{
    fmm_status s = FMM_OK;
    std::vector<bool> done(9, false);
    for (int i = 0; i < b->nbox && s == FMM_OK; ++i) {
        Plan &P = b->plans[i]->P;
        const int d = P.d;
        if (done[d] || d < 2 || tc_sweep_first_level(P) == 0) continue;
        done[d] = true;
        std::vector<int> grp;
        for (int j = 0; j < b->nbox; ++j)
            if (b->plans[j]->P.d == d && b->plans[j]->P.p == P.p) grp.push_back(j);
        std::sort(grp.begin(), grp.end(), [&](int x, int y) { return N[x] < N[y]; });
        const int r = grp[grp.size() / 2];
        Plan &R = b->plans[r]->P;
        double *tp = nullptr, *tq = nullptr;
        uint8_t *ts = nullptr;
        if (cudaMalloc(&tp, sizeof(double) * 3 * N[r]) != cudaSuccess ||
            cudaMalloc(&tq, sizeof(double) * N[r]) != cudaSuccess || cudaMalloc(&ts, N[r]) != cudaSuccess) {
            cudaFree(tp);
            cudaFree(tq);
            cudaFree(ts);
            return FMM_ERR_OOM;
        }
        k_tune_fill<<<1216, 256, 0, R.stream>>>(N[r], box[r], tp, tq, ts);
        const int np = 1 << (d - 1);
        int bx0, by0, bz0;
        tc_get_brick(R, d, &bx0, &by0, &bz0);
        float best = 1e30f;
        int bb[3] = {bx0, by0, bz0};
        for (int bx = 128; bx >= 1 && s == FMM_OK; bx >>= 1)
            for (int by = bx; by >= 1 && s == FMM_OK; by >>= 1) {
                const int bz = 128 / (bx * by);
                if (bz < 1 || bz > by || bx * by * bz != 128 || bx > np || by > np || bz > np) continue;
                if (((np / bx) * (np / by) * (np / bz)) % 2) continue;
                if (tc_set_brick(R, d, bx, by, bz) != FMM_OK) continue;
                float ms = 0.f;
                s = time_plan(b->plans[r], tp, tq, ts, &ms);
                if (s == FMM_OK && ms < best) {
                    best = ms;
                    bb[0] = bx;
                    bb[1] = by;
                    bb[2] = bz;
                }
            }
        cudaFree(tp);
        cudaFree(tq);
        cudaFree(ts);
        for (int j : grp)
            if (s == FMM_OK) s = tc_set_brick(b->plans[j]->P, d, bb[0], bb[1], bb[2]);
    }
    return s;
}

// Sweep on or off, whichever replays the recorded graph of the whole batch faster on uniform test charges
// (one solute per box): per mode one run on the streams, a recording, two warm replays and three timed.
fmm_status tune_sweep(fmm_batch b, const int64_t *N, const double *box)
{
    std::vector<double *> tp(b->nbox, nullptr), tq(b->nbox, nullptr);
    std::vector<uint8_t *> ts(b->nbox, nullptr);
    fmm_status s = FMM_OK;
    for (int i = 0; i < b->nbox && s == FMM_OK; ++i) {
        if (cudaMalloc(&tp[i], sizeof(double) * 3 * N[i]) != cudaSuccess ||
            cudaMalloc(&tq[i], sizeof(double) * N[i]) != cudaSuccess || cudaMalloc(&ts[i], N[i]) != cudaSuccess)
            s = FMM_ERR_OOM;
        else k_tune_fill<<<1216, 256, 0, b->origin>>>(N[i], box[i], tp[i], tq[i], ts[i]);
    }
    if (s == FMM_OK && cudaStreamSynchronize(b->origin) != cudaSuccess) s = FMM_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == FMM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) s = FMM_ERR_CUDA;
    const bool graph = b->use_graph;
    for (int mode = 0; mode < 2 && s == FMM_OK; ++mode) {
        b->use_sweep = mode == 1;
        sweep_enable(b->sweep, b->use_sweep);
        s = batch_enqueue(b, tp.data(), tq.data(), (const uint8_t *const *)ts.data());
        if (s == FMM_OK) s = batch_sync(b);
        if (s != FMM_OK) break;
        b->use_graph = true;
        batch_capture(b, tp.data(), tq.data(), (const uint8_t *const *)ts.data());
        if (!b->graph) {  // no graph: time the stream path instead
            for (int it = 0; it < 5 && s == FMM_OK; ++it) {
                if (it == 2) cudaEventRecord(e0, b->origin);
                s = batch_enqueue(b, tp.data(), tq.data(), (const uint8_t *const *)ts.data());
                for (size_t k = 0; k < b->streams.size() && s == FMM_OK; ++k) {
                    cudaEventRecord(b->ev_done[k], b->streams[k]);
                    cudaStreamWaitEvent(b->origin, b->ev_done[k], 0);
                }
            }
        } else {
            for (int it = 0; it < 5; ++it) {
                if (it == 2) cudaEventRecord(e0, b->origin);
                cudaGraphLaunch(b->graph, b->origin);
            }
        }
        cudaEventRecord(e1, b->origin);
        if (s == FMM_OK && cudaEventSynchronize(e1) != cudaSuccess) s = FMM_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->ms_sweep[mode] = ms / 3.0;
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        b->use_graph = graph;
    }
    b->gptr.clear();
    b->gcount.clear();
    b->use_sweep = s == FMM_OK && b->ms_sweep[1] < b->ms_sweep[0];
    sweep_enable(b->sweep, b->use_sweep);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int i = 0; i < b->nbox; ++i) {
        cudaFree(tp[i]);
        cudaFree(tq[i]);
        cudaFree(ts[i]);
    }
    return s;
}

}  // namespace

extern "C" {

fmm_status fmm_batch_create(int nbox, const double *box, const int64_t *N, const int *depth, const int *p,
                            int precision, fmm_batch *out)
{
    fmm_tune_policy pol;
    pol.energy_rel_tol = 0.0;  // p < 0: 12
    pol.sweep = 1;
    pol.tiles = 0;
    return fmm_batch_create_tuned(nbox, box, N, depth, p, precision, &pol, out);
}

fmm_status fmm_batch_create_tuned(int nbox, const double *box, const int64_t *N, const int *depth, const int *p,
                                  int precision, const fmm_tune_policy *policy, fmm_batch *out)
{
    if (!out) return FMM_ERR_INVALID_ARG;
    if (!policy || !(policy->energy_rel_tol >= 0.0) || policy->sweep < -1 || policy->sweep > 1 || policy->tiles < 0 ||
        policy->tiles > 1)
        return FMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (nbox < 1 || !box || !N || (precision != FMM_PREC_MIXED && precision != FMM_PREC_FP64))
        return FMM_ERR_INVALID_ARG;
    for (int i = 0; i < nbox; ++i)
        if (!(box[i] > 0.0) || !isfinite(box[i]) || N[i] < 1 || (p && p[i] > P_MAX) ||
            (depth && depth[i] > 8))
            return FMM_ERR_INVALID_ARG;
    fmm_batch b = new (std::nothrow) fmm_batch_s();
    if (!b) return FMM_ERR_OOM;
    b->nbox = nbox;
    b->precision = precision;
    b->plans.assign(nbox, nullptr);
    b->depth.assign(nbox, 0);
    const int ns = nbox < BATCH_MAX_STREAMS ? nbox : BATCH_MAX_STREAMS;
    fmm_status s = FMM_OK;
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) s = FMM_ERR_CUDA;
    for (int k = 0; k < ns && s == FMM_OK; ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        // one level above the default priority, like a plan's own execution stream: the near fields
        // (default priority) fill the SMs the far fields leave free
        if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi < lo ? lo - 1 : lo) != cudaSuccess)
            s = FMM_ERR_CUDA;
        else b->streams.push_back(st);
        if (s == FMM_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) s = FMM_ERR_CUDA;
        else if (s == FMM_OK) b->ev_done.push_back(ev);
    }
    if (s == FMM_OK && cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) s = FMM_ERR_CUDA;
    if (s == FMM_OK && cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming) != cudaSuccess) s = FMM_ERR_CUDA;
    b->order.resize(nbox);
    for (int i = 0; i < nbox; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return N[x] > N[y]; });

    // order: given, or (p[i] < 0) 12, or tuned after the depths (below)
    std::vector<int> porder(nbox, 12);
    std::vector<int> free_p;
    for (int i = 0; i < nbox; ++i) {
        if (p && p[i] >= 0) porder[i] = p[i];
        else free_p.push_back(i);
    }
    // depth: given, or tuned per group of boxes with the same starting guess
    std::vector<int> offset(9, 0);
    std::vector<bool> tuned(9, false);
    double *tpos = nullptr, *tq = nullptr;
    uint8_t *tsol = nullptr;
    for (int i = 0; i < nbox && s == FMM_OK; ++i) {
        if (depth && depth[i] > 0) {
            b->depth[i] = depth[i];
            continue;
        }
        const int d0 = depth_guess(N[i]);
        if (!tuned[d0]) {
            // the group's box of median size
            std::vector<int> grp;
            for (int j = 0; j < nbox; ++j)
                if (!(depth && depth[j] > 0) && depth_guess(N[j]) == d0) grp.push_back(j);
            std::sort(grp.begin(), grp.end(), [&](int x, int y) { return N[x] < N[y]; });
            const int r = grp[grp.size() / 2];
            const int pr = porder[r];
            cudaFree(tpos);
            cudaFree(tq);
            cudaFree(tsol);
            tpos = tq = nullptr;
            tsol = nullptr;
            if (cudaMalloc(&tpos, sizeof(double) * 3 * N[r]) != cudaSuccess ||
                cudaMalloc(&tq, sizeof(double) * N[r]) != cudaSuccess || cudaMalloc(&tsol, N[r]) != cudaSuccess) {
                s = FMM_ERR_OOM;
                break;
            }
            k_tune_fill<<<1216, 256, 0, b->streams[0]>>>(N[r], box[r], tpos, tq, tsol);
            float best = 1e30f;
            int best_off = 0;
            for (int off = -1; off <= 1 && s == FMM_OK; ++off) {
                const int dc = d0 + off;
                if (dc < 2 || dc > 8) continue;
                fmm_plan h = nullptr;
                if (make_plan(box[r], N[r], dc, pr, precision, b->streams[0], &h) != FMM_OK) continue;
                float ms = 0;
                if (time_plan(h, tpos, tq, tsol, &ms) == FMM_OK && ms < best) {
                    best = ms;
                    best_off = off;
                }
                fmm_plan_destroy(h);
            }
            if (best >= 1e30f) s = FMM_ERR_INTERNAL;
            offset[d0] = best_off;
            tuned[d0] = true;
        }
        b->depth[i] = d0 + offset[d0];
    }
    cudaFree(tpos);
    cudaFree(tq);
    cudaFree(tsol);
    // tuned order: for each group of boxes with the same depth, a water test box of the group's smallest
    // size and its cell at that depth (the fewest charges per leaf: cells cut through more molecules, the
    // largest truncation error of the group); the batch takes the smallest order that keeps every group's
    // error within the budget (one order: one operator table and one sweep), 12 when none does
    if (s == FMM_OK && !free_p.empty() && policy->energy_rel_tol > 0.0) {
        for (int c = 0; c < 4; ++c) b->p_err[c] = 0.0;
        std::vector<bool> done(9, false);
        for (int i : free_p) {
            const int d = b->depth[i];
            if (done[d] || s != FMM_OK) continue;
            done[d] = true;
            std::vector<int> grp;
            for (int j : free_p)
                if (b->depth[j] == d) grp.push_back(j);
            std::sort(grp.begin(), grp.end(), [&](int x, int y) { return N[x] < N[y]; });
            const int r = grp[0];
            double err[4];
            s = order_errors(N[r], box[r], d, b->streams[0], err);
            for (int c = 0; c < 4 && s == FMM_OK; ++c) b->p_err[c] = fmax(b->p_err[c], err[c]);
        }
        const int cand[4] = {6, 8, 10, 12};
        b->p_tuned = 12;
        for (int c = 0; c < 4; ++c)
            if (b->p_err[c] <= policy->energy_rel_tol) {
                b->p_tuned = cand[c];
                break;
            }
        for (int i : free_p) porder[i] = b->p_tuned;
    }
    // the plans, on the streams round robin in size order
    for (int k = 0; k < nbox && s == FMM_OK; ++k) {
        const int i = b->order[k];
        s = make_plan(box[i], N[i], b->depth[i], porder[i], precision, b->streams[k % ns], &b->plans[i]);
    }
    // tile bricks of the deepest level, per depth group, by timing (before anything is recorded)
    if (s == FMM_OK && policy->tiles == 1 && precision == FMM_PREC_MIXED) s = tune_bricks(b, N, box);
    // one copy of the tensor-core operator tables per order: the boxes' tiles then read them from L2
    for (int i = 0; i < nbox && s == FMM_OK; ++i)
        for (int j = 0; j < i && s == FMM_OK; ++j)
            if (b->plans[j]->P.p == b->plans[i]->P.p) {
                s = tc_share_operators(b->plans[i]->P, b->plans[j]->P);
                break;
            }
    // the persistent sweep over the boxes' CTA-pair levels (mixed precision)
    if (s == FMM_OK && precision == FMM_PREC_MIXED) {
        std::vector<Plan *> ps;
        for (fmm_plan h : b->plans) ps.push_back(&h->P);
        s = sweep_create(ps.data(), nbox, &b->sweep);
        for (size_t k = 0; k < b->streams.size() && s == FMM_OK && b->sweep; ++k) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) s = FMM_ERR_CUDA;
            else b->ev_front.push_back(ev);
        }
        if (s == FMM_OK && b->sweep && cudaEventCreateWithFlags(&b->ev_sweep, cudaEventDisableTiming) != cudaSuccess)
            s = FMM_ERR_CUDA;
        if (s == FMM_OK && b->sweep) {
            if (policy->sweep == -1) s = tune_sweep(b, N, box);
            else {
                b->use_sweep = policy->sweep == 1;
                sweep_enable(b->sweep, b->use_sweep);
            }
        }
    }
    if (s != FMM_OK) {
        batch_free(b);
        return s;
    }
    *out = b;
    return FMM_OK;
}

fmm_status fmm_batch_lambda_energies(fmm_batch b, const double *const *pos, const double *const *q,
                                     const uint8_t *const *is_solute, const double *lambda_c, double *e_total,
                                     double *e_uv, double *v_lambda, double *dv_dlambda)
{
    if (!b || !pos || !q || !is_solute) return FMM_ERR_INVALID_ARG;
    for (int i = 0; i < b->nbox; ++i)
        if (!pos[i] || !q[i] || !is_solute[i] || (lambda_c && !(lambda_c[i] >= 0.0 && lambda_c[i] <= 1.0)))
            return FMM_ERR_INVALID_ARG;
    if (b->sc_c > 0)  // each box's soft-core lambda, read by its next (enqueued or replayed) evaluation
        for (int i = 0; i < b->nbox; ++i) *b->plans[i]->P.h_sc_lambda = lambda_c ? lambda_c[i] : 0.0;
    bool fresh = false;  // results come from the enqueued path
    if (b->use_graph && graph_matches(b, pos, q, is_solute)) {
        FMM_CUDA_TRY(cudaGraphLaunch(b->graph, b->origin));
        FMM_CUDA_TRY(cudaStreamSynchronize(b->origin));
        ++b->replays;
        for (int i = 0; i < b->nbox; ++i)
            if (solute_count_host(b->plans[i]->P) != b->gcount[i]) fresh = true;  // a count changed: redo
        if (!fresh) goto results;
    }
    {
        fmm_status s = batch_enqueue(b, pos, q, is_solute);
        if (s != FMM_OK) return s;
        s = batch_sync(b);
        if (s != FMM_OK) return s;
        ++b->enqueued;
        if (b->use_graph) batch_capture(b, pos, q, is_solute);
    }
results:
    fmm_status worst = FMM_OK;
    for (int i = 0; i < b->nbox; ++i) {
        fmm_energy_terms t;
        fmm_uv_terms u;
        fmm_status s = eval_results(b->plans[i]->P, &t, &u);
        if (s != FMM_OK && worst == FMM_OK) worst = s;
        const double lam = lambda_c ? lambda_c[i] : 0.0;
        if (e_total) e_total[i] = t.total;
        if (e_uv) e_uv[i] = u.e_uv;
        if (b->sc_c > 0) {  // the near-field solute-solvent pairs through the soft-core distance
            const double e_sc = u.e_uv - u.nf_uv + u.nf_sc;
            if (v_lambda) v_lambda[i] = t.total - u.e_uv + (1.0 - lam) * e_sc;
            if (dv_dlambda) dv_dlambda[i] = -e_sc + (1.0 - lam) * u.dnf_sc;
        } else {
            if (v_lambda) v_lambda[i] = t.total - lam * u.e_uv;
            if (dv_dlambda) dv_dlambda[i] = -u.e_uv;
        }
    }
    return worst;
}

fmm_status fmm_batch_info(fmm_batch b, int i, int *depth, int *p, int64_t *replays, int64_t *enqueued)
{
    if (!b || i < 0 || i >= b->nbox) return FMM_ERR_INVALID_ARG;
    if (depth) *depth = b->plans[i]->P.d;
    if (p) *p = b->plans[i]->P.p;
    if (replays) *replays = b->replays;
    if (enqueued) *enqueued = b->enqueued;
    return FMM_OK;
}

fmm_status fmm_batch_set_softcore(fmm_batch b, int c, double A, double alpha)
{
    if (!b || c < 0 || c > 12) return FMM_ERR_INVALID_ARG;
    if (c > 0 && !(A > 0.0 && isfinite(A) && alpha > 0.0 && isfinite(alpha))) return FMM_ERR_INVALID_ARG;
    for (fmm_plan h : b->plans) {
        fmm_status s = fmm_plan_set_option(h, FMM_OPT_SOFTCORE, c, c > 0 ? A : 0.0);
        if (s == FMM_OK && c > 0) s = fmm_plan_set_option(h, FMM_OPT_SOFTCORE_ALPHA, 0, alpha);
        if (s != FMM_OK) return s;
    }
    b->sc_c = c;
    if (b->graph) {  // the recorded work changed
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->gptr.clear();
    }
    return FMM_OK;
}

fmm_status fmm_batch_set_option(fmm_batch b, int key, int64_t ival, double dval)
{
    (void)dval;
    if (!b) return FMM_ERR_INVALID_ARG;
    switch (key) {
    case FMM_BATCH_OPT_SWEEP:
        if (ival != 0 && ival != 1) return FMM_ERR_INVALID_ARG;
        b->use_sweep = ival != 0;
        sweep_enable(b->sweep, b->use_sweep);
        break;
    case FMM_BATCH_OPT_WAIT_BUDGET_NS:
        if (ival < 1000 || ival > 10000000000ll) return FMM_ERR_INVALID_ARG;
        b->wait_ns = (uint64_t)ival;
        break;
    case FMM_BATCH_OPT_INJECT_STALL:
        if (ival != 0 && ival != 1) return FMM_ERR_INVALID_ARG;
        b->stall = ival != 0;
        break;
    case FMM_BATCH_OPT_SWEEP_PAIRS:
        if (ival < 0 || ival > 4096) return FMM_ERR_INVALID_ARG;
        b->sweep_pairs = (int)ival;
        break;
    default: return FMM_ERR_INVALID_ARG;
    }
    if (b->graph) {  // the recorded work changed
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->gptr.clear();
    }
    return FMM_OK;
}

fmm_status fmm_batch_sweep_info(fmm_batch b, int *boxes, int *first_level)
{
    if (!b) return FMM_ERR_INVALID_ARG;
    if (boxes) *boxes = (b->use_sweep && b->sweep) ? sweep_plans(b->sweep) : 0;
    if (first_level)
        for (int i = 0; i < b->nbox; ++i) first_level[i] = b->plans[i]->P.sweep_from;
    return FMM_OK;
}

fmm_status fmm_batch_tune_info(fmm_batch b, double *p_err, int *p_chosen, double *ms_sweep_off, double *ms_sweep_on,
                               int *sweep_on)
{
    if (!b) return FMM_ERR_INVALID_ARG;
    if (p_err)
        for (int c = 0; c < 4; ++c) p_err[c] = b->p_err[c];
    if (p_chosen) *p_chosen = b->p_tuned;
    if (ms_sweep_off) *ms_sweep_off = b->ms_sweep[0];
    if (ms_sweep_on) *ms_sweep_on = b->ms_sweep[1];
    if (sweep_on) *sweep_on = (b->sweep && b->use_sweep) ? 1 : 0;
    return FMM_OK;
}

fmm_status fmm_batch_brick_info(fmm_batch b, int i, int *level, int *bx, int *by, int *bz)
{
    if (!b || i < 0 || i >= b->nbox || !level || !bx || !by || !bz) return FMM_ERR_INVALID_ARG;
    *level = b->plans[i]->P.d;
    tc_get_brick(b->plans[i]->P, *level, bx, by, bz);
    return FMM_OK;
}

fmm_status fmm_batch_set_graph(fmm_batch b, int enable)
{
    if (!b || (enable != 0 && enable != 1)) return FMM_ERR_INVALID_ARG;
    b->use_graph = enable != 0;
    if (!b->use_graph && b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return FMM_OK;
}

void fmm_batch_destroy(fmm_batch b) { batch_free(b); }

}  // extern "C"
