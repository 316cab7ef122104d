// fmm_p2p.cu -- near field (Eq. EqNF): direct Coulomb sums over the
// (2 ws + 1)^3 leaves around each charge's leaf (27 for ws = 1, 125 for ws = 2),
// periodic, j != i.
//
// Coordinates are relative to each leaf's centre, so the separation of a
// charge in leaf c from one in neighbour leaf c + delta is
// loc_i - loc_j - delta h: the periodic image shift is implicit and the FP32
// path keeps full precision in boxes of any size.
#include <math.h>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
__device__ inline T inv_sqrt(T x);
template <>
__device__ inline float inv_sqrt<float>(float x) { return rsqrtf(x); }
template <>
__device__ inline double inv_sqrt<double>(double x) { return 1.0 / sqrt(x); }

// One thread per sorted charge i: phi_i = sum q_j / r_ij, e_i = sum q_j r_ij / r_ij^3.
template <typename T>
__global__ void k_p2p(int64_t N, int d, int ws, T h, const int *__restrict__ start, const int *__restrict__ sleaf,
                      const Particle<T> *__restrict__ sp, T *__restrict__ phi, T *__restrict__ field)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int nside = 1 << d;
    int leaf = sleaf[s];
    int x = leaf % nside, y = (leaf / nside) % nside, z = leaf / (nside * nside);
    Particle<T> pi = sp[s];
    T acc = 0, ex = 0, ey = 0, ez = 0;
    for (int dz = -ws; dz <= ws; ++dz) {
        int zz = (z + dz + nside) & (nside - 1);
        for (int dy = -ws; dy <= ws; ++dy) {
            int yy = (y + dy + nside) & (nside - 1);
            for (int dx = -ws; dx <= ws; ++dx) {
                int xx = (x + dx + nside) & (nside - 1);
                int c = xx + nside * (yy + nside * zz);
                T ox = pi.x - T(dx) * h, oy = pi.y - T(dy) * h, oz = pi.z - T(dz) * h;
                for (int j = start[c]; j < start[c + 1]; ++j) {
                    if (j == s) continue;
                    Particle<T> pj = sp[j];
                    T rx = ox - pj.x, ry = oy - pj.y, rz = oz - pj.z;
                    T r2 = rx * rx + ry * ry + rz * rz;
                    T ir = inv_sqrt<T>(r2);
                    T qir = pj.q * ir;
                    acc += qir;
                    T qir3 = qir * ir * ir;
                    ex += qir3 * rx;
                    ey += qir3 * ry;
                    ez += qir3 * rz;
                }
            }
        }
    }
    phi[s] = acc;
    if (field) {
        field[3 * s] = ex;
        field[3 * s + 1] = ey;
        field[3 * s + 2] = ez;
    }
}

// near-field solute-solvent pair sum: out_i = q_i sum_{j in NF(i), j solvent} q_j / r_ij
// for solute i, 0 otherwise
template <typename T>
__global__ void k_p2p_uv(int64_t N, int d, int ws, T h, const int *__restrict__ start, const int *__restrict__ sleaf,
                         const Particle<T> *__restrict__ sp, const uint8_t *__restrict__ sol, T *__restrict__ out)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (!sol[s]) {
        out[s] = 0;
        return;
    }
    int nside = 1 << d;
    int leaf = sleaf[s];
    int x = leaf % nside, y = (leaf / nside) % nside, z = leaf / (nside * nside);
    Particle<T> pi = sp[s];
    T acc = 0;
    for (int dz = -ws; dz <= ws; ++dz)
        for (int dy = -ws; dy <= ws; ++dy)
            for (int dx = -ws; dx <= ws; ++dx) {
                int xx = (x + dx + nside) & (nside - 1), yy = (y + dy + nside) & (nside - 1),
                    zz = (z + dz + nside) & (nside - 1);
                int c = xx + nside * (yy + nside * zz);
                T ox = pi.x - T(dx) * h, oy = pi.y - T(dy) * h, oz = pi.z - T(dz) * h;
                for (int j = start[c]; j < start[c + 1]; ++j) {
                    if (sol[j]) continue;
                    Particle<T> pj = sp[j];
                    T rx = ox - pj.x, ry = oy - pj.y, rz = oz - pj.z;
                    acc += pj.q * inv_sqrt<T>(rx * rx + ry * ry + rz * rz);
                }
            }
    out[s] = pi.q * acc;
}

}  // namespace

fmm_status launch_p2p(Plan &P, bool forces)
{
    int nside = 1 << P.d;
    double h = P.box / nside;
    if (P.precision == FMM_PREC_FP64)
        k_p2p<double><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(
            P.N, P.d, P.ws, h, P.cell_start, P.sleaf, (const Particle<double> *)P.sorted, (double *)P.phi_nf,
            forces ? (double *)P.f_nf : nullptr);
    else
        k_p2p<float><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(
            P.N, P.d, P.ws, (float)h, P.cell_start, P.sleaf, (const Particle<float> *)P.sorted, (float *)P.phi_nf,
            forces ? (float *)P.f_nf : nullptr);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_p2p_uv(Plan &P)
{
    int nside = 1 << P.d;
    double h = P.box / nside;
    if (P.precision == FMM_PREC_FP64)
        k_p2p_uv<double><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(
            P.N, P.d, P.ws, h, P.cell_start, P.sleaf, (const Particle<double> *)P.sorted, P.sorted_sol,
            (double *)P.phi_nf + P.N);
    else
        k_p2p_uv<float><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(
            P.N, P.d, P.ws, (float)h, P.cell_start, P.sleaf, (const Particle<float> *)P.sorted, P.sorted_sol,
            (float *)P.phi_nf + P.N);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

}  // namespace fmm
