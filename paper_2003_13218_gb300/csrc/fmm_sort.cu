// fmm_sort.cu -- leaf assignment and sort (Appendix B, "Division of cells"),
// background-charge moments (Eq. 6, Eq. surfchargedend, Appendix D) and the
// FP64 compensated energy reductions of Eq. Velecfull and Eq. FMMcalc.
#include <math.h>

#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
constexpr int SCAN_ITEMS = 4096; // elements per scan block (256 threads x 16)

// Neumaier compensated accumulator
struct KSum {
    double s, c;
    __device__ void add(double x)
    {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ void merge(const KSum &o)
    {
        add(o.s);
        add(o.c);
    }
    __device__ double val() const { return s + c; }
};

// Wrap each coordinate into [0, b) and assign the leaf:
//   w = x - b floor(x / b)  (w >= b -> w - b),  leaf = floor(w 2^d / b) clamped.
// Explicit round-to-nearest intrinsics keep the arithmetic free of FMA
// contraction, so leaves are assigned exactly as the IEEE expression says.
__global__ void k_assign(int64_t N, const double *__restrict__ pos, const double *__restrict__ q, double box,
                         double scale, int nside, double *__restrict__ wpos, int *__restrict__ key,
                         int *__restrict__ count, int *__restrict__ err)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    bool ok = isfinite(q[i]);
    int c[3];
    for (int a = 0; a < 3; ++a) {
        double x = pos[3 * i + a];
        if (!isfinite(x)) {
            ok = false;
            x = 0.0;
        }
        double f = floor(__ddiv_rn(x, box));
        double w = __dsub_rn(x, __dmul_rn(box, f));
        if (w >= box) w = __dsub_rn(w, box);
        if (w < 0.0) w = 0.0;
        wpos[3 * i + a] = w;
        int k = (int)floor(__dmul_rn(w, scale));
        c[a] = k < 0 ? 0 : (k > nside - 1 ? nside - 1 : k);
    }
    int lin = c[0] + nside * (c[1] + nside * c[2]);
    key[i] = lin;
    atomicAdd(&count[lin], 1);
    if (!ok) atomicOr(err, ERRF_NONFINITE);
}

// three-phase exclusive scan of counts[n] into start[n+1]
__global__ void k_scan_blocks(int64_t n, const int *__restrict__ in, int *__restrict__ out, int *__restrict__ sums)
{
    __shared__ int ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + threadIdx.x * 16;
    int v[16];
    int local = 0;
    for (int k = 0; k < 16; ++k) {
        int64_t idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        local += v[k];
    }
    // inclusive warp scan of per-thread totals
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = local;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int excl = x - local + (wid > 0 ? ws[wid - 1] : 0);
    for (int k = 0; k < 16; ++k) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = excl;
        excl += v[k];
    }
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = excl;
}

__global__ void k_scan_sums(int nb, int *__restrict__ sums)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nb; ++b) {
            int t = sums[b];
            sums[b] = acc;
            acc += t;
        }
        sums[nb] = acc;
    }
}

__global__ void k_scan_add(int64_t n, int *__restrict__ out, const int *__restrict__ sums, int nb)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / SCAN_ITEMS];
    if (i == 0) out[n] = sums[nb];
}

__global__ void k_scatter(int64_t N, const int *__restrict__ key, const int *__restrict__ start, int *__restrict__ fill,
                          int *__restrict__ perm)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = key[i];
    int slot = start[k] + atomicAdd(&fill[k], 1);
    perm[slot] = (int)i;
}

// order each leaf's particles by original index (deterministic results)
__global__ void k_leaf_sort(int64_t nleaf, const int *__restrict__ start, int *__restrict__ perm)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= nleaf) return;
    int b = start[c], e = start[c + 1];
    for (int i = b + 1; i < e; ++i) {
        int v = perm[i];
        int j = i - 1;
        while (j >= b && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
}

template <typename T>
__global__ void k_gather(int64_t N, const int *__restrict__ perm, const int *__restrict__ key,
                         const double *__restrict__ wpos, const double *__restrict__ q, const uint8_t *__restrict__ sol,
                         double h, int nside, Particle<T> *__restrict__ out, Particle<T> *__restrict__ out_u,
                         uint8_t *__restrict__ out_sol, int *__restrict__ sleaf)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int i = perm[s];
    int k = key[i];
    sleaf[s] = k;
    int cx = k % nside, cy = (k / nside) % nside, cz = k / (nside * nside);
    double qi = q[i];
    if (!isfinite(qi)) qi = 0.0;
    Particle<T> r;
    r.x = (T)(wpos[3 * (int64_t)i] - (cx + 0.5) * h);
    r.y = (T)(wpos[3 * (int64_t)i + 1] - (cy + 0.5) * h);
    r.z = (T)(wpos[3 * (int64_t)i + 2] - (cz + 0.5) * h);
    r.q = (T)qi;
    out[s] = r;
    if (sol) {
        uint8_t u = sol[i] ? 1 : 0;
        out_sol[s] = u;
        Particle<T> ru = r;
        if (!u) ru.q = (T)0;
        out_u[s] = ru;
    }
}

// merge (s, c) across the lanes of a warp, fixed xor tree (deterministic); lane 0 holds the total
__device__ inline KSum warp_merge(KSum k)
{
    for (int o = 16; o > 0; o >>= 1) {
        KSum b{__shfl_xor_sync(0xffffffffu, k.s, o), __shfl_xor_sync(0xffffffffu, k.c, o)};
        k.merge(b);
    }
    return k;
}

// block-level reduction of NQ per-thread sums -> partial[block][NQ][2]: the 32 lanes of a warp are added
// plainly in a fixed xor tree (deterministic; GB300's FP64 pipe is slow, and a compensated merge per lane
// and round cost most of the reduction), the block's warp sums compensated (lane q of warp 0, quantity q),
// and the blocks again compensated by final_sum
template <int NQ>
__device__ void block_reduce_store(const double (&acc)[NQ], double *__restrict__ partial)
{
    static_assert(NQ <= 32, "one lane per quantity");
    __shared__ double sh[RED_THREADS / 32][NQ];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[w][q] = v;
    }
    __syncthreads();
    if (w == 0 && lane < NQ) {
        KSum k{0.0, 0.0};
        for (int i = 0; i < RED_THREADS / 32; ++i) k.add(sh[i][lane]);
        partial[(blockIdx.x * NQ + lane) * 2] = k.s;
        partial[(blockIdx.x * NQ + lane) * 2 + 1] = k.c;
    }
}

// Q, mu, S2 = sum q r^2 over all charges and over the solute subset
__global__ void k_bc_partial(int64_t N, const double *__restrict__ wpos, const double *__restrict__ q,
                             const uint8_t *__restrict__ sol, double *__restrict__ partial)
{
    // a thread's own elements (N / 77,824, about 13 at N = 1M) and a warp's lanes are summed
    // plainly; the compensated sums start at the block level
    double acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double qi = q[i];
        if (!isfinite(qi)) qi = 0.0;
        double x = wpos[3 * i], y = wpos[3 * i + 1], z = wpos[3 * i + 2];
        double v[5] = {qi, qi * x, qi * y, qi * z, qi * (x * x + y * y + z * z)};
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += v[k];
        if (sol && sol[i])
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[5 + k] += v[k];
    }
    block_reduce_store<10>(acc, partial);
}

// energies over sorted particles: e_near, e_far, A, B, C, NF_uv and (sc non-null) the soft-core near-field
// pair sum and its lambda derivative
constexpr int NQ_ENERGY = 8;

template <typename T>
__global__ void k_energy_partial(int64_t N, const Particle<T> *__restrict__ sp, const T *__restrict__ phi_nf,
                                 const T *__restrict__ phi_ff, const T *__restrict__ phi_u,
                                 const uint8_t *__restrict__ sol, const T *__restrict__ nfuv,
                                 const double *__restrict__ sc, double *__restrict__ partial)
{
    double acc[NQ_ENERGY];
#pragma unroll
    for (int k = 0; k < NQ_ENERGY; ++k) acc[k] = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        double qs = (double)sp[s].q;
        acc[0] += 0.5 * qs * (double)phi_nf[s];
        acc[1] += 0.5 * qs * (double)phi_ff[s];
        if (sol) {
            if (sol[s]) {
                acc[2] += qs * (double)phi_ff[s];
                acc[3] += qs * (double)phi_u[s];
                acc[5] += (double)nfuv[s];
                if (sc) {
                    acc[6] += sc[s];
                    acc[7] += sc[N + s];
                }
            } else {
                acc[4] += qs * (double)phi_u[s];
            }
        }
    }
    block_reduce_store<NQ_ENERGY>(acc, partial);
}

// block partials -> totals; blockDim.x == RED_THREADS: warp w takes the
// quantities w, w + 8, ...; its lanes stride over the blocks, then a fixed xor tree
template <int NQ>
__device__ void final_sum(const double *__restrict__ partial, int nb, double *out)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = w; q < NQ; q += RED_THREADS / 32) {
        KSum k{0, 0};
        for (int b = lane; b < nb; b += 32) {
            k.add(partial[(b * NQ + q) * 2]);
            k.add(partial[(b * NQ + q) * 2 + 1]);
        }
        k = warp_merge(k);
        if (lane == 0) out[q] = k.val();
    }
}

__global__ void k_bc_final(const double *__restrict__ partial, int nb, double *__restrict__ out)
{
    final_sum<10>(partial, nb, out);
}

// Combine into the terms of Eq. Velecfull and Eq. FMMcalc.
// out layout: [0..9] moments (Q, mu, S2, Qu, mu_u, S2u), [10..15] energy parts,
// [16..21] terms (near, far, charged, quad, dipole, total), [22..28] uv terms,
// [29..30] soft-core near-field sum and its lambda derivative; [40..47] scratch.
// vacuum: the boundary at infinity is vacuum (App. D): the dipole surface term
// -(2 pi / 3V) mu.mu that gives the conducting boundary is left out, and so is
// its solute-solvent cross term -(4 pi / 3V) mu_u.mu_v
__global__ void k_energy_final(const double *__restrict__ partial, int nb, double *__restrict__ out, double box,
                               double kappa, int with_uv, int vacuum)
{
    final_sum<NQ_ENERGY>(partial, nb, out + 40);
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 0; k < 6; ++k) out[10 + k] = out[40 + k];
    out[29] = out[46];
    out[30] = out[47];
    const double PI = 3.14159265358979323846;
    double V = box * box * box;
    double Q = out[0], mx = out[1], my = out[2], mz = out[3], S2 = out[4];
    double e_near = out[10], e_far = out[11];
    double e_cha = -PI / (2.0 * V * kappa * kappa) * Q * Q;
    double e_quad = 2.0 * PI / (3.0 * V) * Q * S2;
    double e_dip = vacuum ? 0.0 : -2.0 * PI / (3.0 * V) * (mx * mx + my * my + mz * mz);
    KSum t{0, 0};
    t.add(e_near);
    t.add(e_far);
    t.add(e_cha);
    t.add(e_quad);
    t.add(e_dip);
    out[16] = e_near;
    out[17] = e_far;
    out[18] = e_cha;
    out[19] = e_quad;
    out[20] = e_dip;
    out[21] = t.val();
    if (with_uv) {
        double Qu = out[5], mux = out[6], muy = out[7], muz = out[8], S2u = out[9];
        double Qv = Q - Qu, mvx = mx - mux, mvy = my - muy, mvz = mz - muz, S2v = S2 - S2u;
        double A = out[12], B = out[13], C = out[14], nf = out[15];
        double bc = -PI * Qu * Qv / (V * kappa * kappa) + 2.0 * PI / (3.0 * V) * (Qu * S2v + Qv * S2u);
        if (!vacuum) bc -= 4.0 * PI / (3.0 * V) * (mux * mvx + muy * mvy + muz * mvz);
        KSum w{0, 0};
        w.add(A);
        w.add(-B);
        w.add(C);
        double W = 0.5 * w.val();
        KSum e{0, 0};
        e.add(nf);
        e.add(W);
        e.add(bc);
        out[22] = e.val();
        out[23] = W;
        out[24] = A;
        out[25] = B;
        out[26] = C;
        out[27] = nf;
        out[28] = bc;
    }
}

// F_i = q_i (E_nf - grad Phi_ff) - (4 pi / 3V) q_i (Q r_i - mu), scattered to
// input order; with the vacuum boundary the mu part (the dipole surface term's
// force) is left out
template <typename T>
__global__ void k_forces_out(int64_t N, const int *__restrict__ perm, const Particle<T> *__restrict__ sp,
                             const T *__restrict__ f_nf, const T *__restrict__ g_ff, const double *__restrict__ wpos,
                             const double *__restrict__ q, const double *__restrict__ mom, double box, int vacuum,
                             double *__restrict__ forces)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double PI = 3.14159265358979323846;
    double c = 4.0 * PI / (3.0 * box * box * box);
    int i = perm[s];
    double qi = q[i];
    if (!isfinite(qi)) qi = 0.0;
    const double Q = mom[0], cq = c * qi;
    for (int a = 0; a < 3; ++a) {
        // the mixed path's field (FP32 near and far parts) is formed in FP32 and converted once
        const double fld = std::is_same<T, float>::value ? (double)(f_nf[3 * s + a] - g_ff[3 * s + a])
                                                         : (double)f_nf[3 * s + a] - (double)g_ff[3 * s + a];
        double f = qi * fld;
        f -= cq * (Q * wpos[3 * (int64_t)i + a] - (vacuum ? 0.0 : mom[1 + a]));
        forces[3 * (int64_t)i + a] = f;
    }
}

// phi_i = dV/dq_i in input order: pair potentials (near + far) plus the
// derivatives of the background terms of Eq. Velecfull,
//   d/dq_i [-pi Q^2/(2 V kappa^2)]      = -pi Q/(V kappa^2),
//   d/dq_i [(2 pi/3V) Q S2]             = (2 pi/3V)(S2 + Q r_i^2),
//   d/dq_i [-(2 pi/3V) mu.mu]           = -(4 pi/3V) mu.r_i   (conducting boundary)
template <typename T>
__global__ void k_potentials_out(int64_t N, const int *__restrict__ perm, const T *__restrict__ phi_nf,
                                 const T *__restrict__ phi_ff, const double *__restrict__ wpos,
                                 const double *__restrict__ mom, double box, double kappa, int vacuum,
                                 double *__restrict__ out)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double PI = 3.14159265358979323846;
    const double V = box * box * box;
    const int i = perm[s];
    const double Q = mom[0], S2 = mom[4];
    const double x = wpos[3 * (int64_t)i], y = wpos[3 * (int64_t)i + 1], z = wpos[3 * (int64_t)i + 2];
    double v = (double)phi_nf[s] + (double)phi_ff[s];
    v += -PI * Q / (V * kappa * kappa);
    v += 2.0 * PI / (3.0 * V) * (S2 + Q * (x * x + y * y + z * z));
    if (!vacuum) v -= 4.0 * PI / (3.0 * V) * (mom[1] * x + mom[2] * y + mom[3] * z);
    out[i] = v;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

fmm_status launch_assign_sort(Plan &P, const double *pos, const double *q, const uint8_t *sol)
{
    int nside = 1 << P.d;
    double scale = (double)nside / P.box;
    FMM_CUDA_TRY(cudaMemsetAsync(P.cell_fill, 0, sizeof(int) * P.nleaf, P.stream));
    k_assign<<<blocks_for(P.N, 256), 256, 0, P.stream>>>(P.N, pos, q, P.box, scale, nside, P.wpos, P.key, P.cell_fill,
                                                          P.d_err);
    FMM_LAUNCH_CHECK(P);
    int nb = (int)((P.nleaf + SCAN_ITEMS - 1) / SCAN_ITEMS);
    k_scan_blocks<<<nb, 256, 0, P.stream>>>(P.nleaf, P.cell_fill, P.cell_start, P.scan_tmp);
    FMM_LAUNCH_CHECK(P);
    k_scan_sums<<<1, 32, 0, P.stream>>>(nb, P.scan_tmp);
    FMM_LAUNCH_CHECK(P);
    k_scan_add<<<blocks_for(P.nleaf, 256), 256, 0, P.stream>>>(P.nleaf, P.cell_start, P.scan_tmp, nb);
    FMM_LAUNCH_CHECK(P);
    FMM_CUDA_TRY(cudaMemsetAsync(P.cell_fill, 0, sizeof(int) * P.nleaf, P.stream));
    k_scatter<<<blocks_for(P.N, 256), 256, 0, P.stream>>>(P.N, P.key, P.cell_start, P.cell_fill, P.perm);
    FMM_LAUNCH_CHECK(P);
    k_leaf_sort<<<blocks_for(P.nleaf, 256), 256, 0, P.stream>>>(P.nleaf, P.cell_start, P.perm);
    FMM_LAUNCH_CHECK(P);
    double h = P.box / nside;
    if (P.precision == FMM_PREC_FP64)
        k_gather<double><<<blocks_for(P.N, 256), 256, 0, P.stream>>>(
            P.N, P.perm, P.key, P.wpos, q, sol, h, nside, (Particle<double> *)P.sorted,
            (Particle<double> *)P.sorted_u, P.sorted_sol, P.sleaf);
    else
        k_gather<float><<<blocks_for(P.N, 256), 256, 0, P.stream>>>(P.N, P.perm, P.key, P.wpos, q, sol, h, nside,
                                                                    (Particle<float> *)P.sorted,
                                                                    (Particle<float> *)P.sorted_u, P.sorted_sol,
                                                                    P.sleaf);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_bc_moments(Plan &P, const double *q, const uint8_t *sol)
{
    k_bc_partial<<<RED_BLOCKS, RED_THREADS, 0, P.stream>>>(P.N, P.wpos, q, sol, P.red_partial);
    FMM_LAUNCH_CHECK(P);
    k_bc_final<<<1, RED_THREADS, 0, P.stream>>>(P.red_partial, RED_BLOCKS, P.red_out);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_energy_reduce(Plan &P, bool with_uv)
{
    double *part = P.red_partial + RED_BLOCKS * 10 * 2;
    const double *sc = with_uv && P.sc_c > 0 ? P.sc_out : nullptr;
    const uint8_t *sol = with_uv ? P.sorted_sol : nullptr;
    if (P.precision == FMM_PREC_FP64) {
        const double *nfuv = (const double *)P.phi_nf + P.N;  // second half of the phi_nf buffer
        k_energy_partial<double><<<RED_BLOCKS, RED_THREADS, 0, P.stream>>>(
            P.N, (const Particle<double> *)P.sorted, (const double *)P.phi_nf, (const double *)P.phi_ff,
            (const double *)P.phi_u, sol, nfuv, sc, part);
    } else {
        const float *nfuv = (const float *)P.phi_nf + P.N;
        k_energy_partial<float><<<RED_BLOCKS, RED_THREADS, 0, P.stream>>>(
            P.N, (const Particle<float> *)P.sorted, (const float *)P.phi_nf, (const float *)P.phi_ff,
            (const float *)P.phi_u, sol, nfuv, sc, part);
    }
    FMM_LAUNCH_CHECK(P);
    double kappa = P.kappa > 0 ? P.kappa : 2.0 / P.box;
    k_energy_final<<<1, RED_THREADS, 0, P.stream>>>(part, RED_BLOCKS, P.red_out, P.box, kappa, with_uv ? 1 : 0,
                                                    P.boundary);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_forces_out(Plan &P, const double *q, double *forces)
{
    if (P.precision == FMM_PREC_FP64)
        k_forces_out<double><<<blocks_for(P.N, 256), 256, 0, P.stream>>>(
            P.N, P.perm, (const Particle<double> *)P.sorted, (const double *)P.f_nf, (const double *)P.g_ff, P.wpos,
            q, P.red_out, P.box, P.boundary, forces);
    else
        k_forces_out<float><<<blocks_for(P.N, 256), 256, 0, P.stream>>>(
            P.N, P.perm, (const Particle<float> *)P.sorted, (const float *)P.f_nf, (const float *)P.g_ff, P.wpos, q,
            P.red_out, P.box, P.boundary, forces);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_potentials_out(Plan &P, double *potentials)
{
    const double kappa = P.kappa > 0 ? P.kappa : 2.0 / P.box;
    if (P.precision == FMM_PREC_FP64)
        k_potentials_out<double><<<blocks_for(P.N, 256), 256, 0, P.stream>>>(
            P.N, P.perm, (const double *)P.phi_nf, (const double *)P.phi_ff, P.wpos, P.red_out, P.box, kappa,
            P.boundary, potentials);
    else
        k_potentials_out<float><<<blocks_for(P.N, 256), 256, 0, P.stream>>>(
            P.N, P.perm, (const float *)P.phi_nf, (const float *)P.phi_ff, P.wpos, P.red_out, P.box, kappa,
            P.boundary, potentials);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

size_t reduction_scratch_doubles() { return (size_t)RED_BLOCKS * 20 * 2; }

}  // namespace fmm
