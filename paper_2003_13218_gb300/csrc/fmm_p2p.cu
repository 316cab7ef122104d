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

// One source of the near field: adds q_j / r and q_j r / r^3 for r = (ox, oy, oz) - x_j.  A source at r = 0
// (the target itself: the same stored coordinates) adds nothing; the near field never holds a charge's own
// periodic image (2^depth > 2 ws + 1).
template <typename T>
__device__ __forceinline__ void p2p_pair(const Particle<T> &pj, T ox, T oy, T oz, T &acc, T &ex, T &ey, T &ez)
{
    const T rx = ox - pj.x, ry = oy - pj.y, rz = oz - pj.z;
    const T r2 = rx * rx + ry * ry + rz * rz;
    const T ir = r2 > T(0) ? inv_sqrt<T>(r2) : T(0);
    const T qir = pj.q * ir;
    acc += qir;
    const T qir3 = qir * ir * ir;
    ex += qir3 * rx;
    ey += qir3 * ry;
    ez += qir3 * rz;
}

// The near field with the neighbour particles staged in shared memory: phi_i = sum q_j / r_ij and
// e_i = sum q_j r_ij / r_ij^3 per sorted charge i.  A block takes a row segment of BX consecutive leaves
// along x at (y, z) -- their charges are contiguous in the sorted order -- and copies the particles of the
// (2 ws + 1)^2 rows around it, each BX + 2 ws leaves long (x wrapped periodically, a leaf may appear twice
// when BX + 2 ws exceeds the side), into shared memory with 16-byte cp.async copies.  Then each thread
// takes one target charge of the segment and sums over its (2 ws + 1)^3 neighbour leaves in a fixed
// order; a block whose rows hold more than `cap` particles reads them from global memory with the same
// arithmetic in the same order, so the staged and unstaged blocks give identical results.
//   shared memory: pre[R W + 1] (staged start of leaf f = r W + i, row r = (dz + ws)(2 ws + 1) + dy + ws,
//   i = x - x0 + ws), gst[R W] (the leaf's first sorted index), then the staged records.
constexpr int P2P_THREADS = 128;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gsrc)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void stage_copy(Particle<T> *dst, const Particle<T> *src)
{
    if (sizeof(Particle<T>) == 16) {
        cp_async16(dst, src);
    } else {
        cp_async16(dst, src);
        cp_async16(reinterpret_cast<char *>(dst) + 16, reinterpret_cast<const char *>(src) + 16);
    }
}

template <typename T>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_tile(int d, int ws, int bx, int cap, T h,
                                                          const int *__restrict__ start,
                                                          const Particle<T> *__restrict__ sp, T *__restrict__ phi,
                                                          T *__restrict__ field)
{
    extern __shared__ __align__(16) unsigned char p2p_smem[];
    const int n = 1 << d, mask = n - 1;
    const int side = 2 * ws + 1, R = side * side, W = bx + 2 * ws, F = R * W;
    const int tiles_x = n / bx;
    const int x0 = (blockIdx.x % tiles_x) * bx;
    const int y = (blockIdx.x / tiles_x) & mask, z = blockIdx.x / (tiles_x * n);
    int *pre = reinterpret_cast<int *>(p2p_smem);
    int *gst = pre + F + 1;
    Particle<T> *stg = reinterpret_cast<Particle<T> *>(p2p_smem + ((sizeof(int) * (2 * F + 1) + 15) / 16) * 16);
    __shared__ int warp_tot[P2P_THREADS / 32];

    auto gleaf = [&](int f) {  // global leaf of staged leaf f
        const int r = f / W, i = f - r * W;
        const int dy = r % side - ws, dz = r / side - ws;
        return ((x0 - ws + i) & mask) + n * (((y + dy) & mask) + n * ((z + dz) & mask));
    };
    // 1. per-leaf counts -> exclusive prefix pre[] (each thread a run of consecutive entries, then a scan of
    //    the run totals across the block)
    const int per = (F + P2P_THREADS - 1) / P2P_THREADS;
    const int f0 = threadIdx.x * per;
    int run = 0;
    for (int f = f0; f < f0 + per && f < F; ++f) {
        const int g = gleaf(f);
        const int b = start[g];
        const int c = start[g + 1] - b;
        gst[f] = b;
        pre[f + 1] = c;
        run += c;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[w] = incl;
    if (threadIdx.x == 0) pre[0] = 0;
    __syncthreads();
    int base = incl - run;
    for (int k = 0; k < w; ++k) base += warp_tot[k];
    for (int f = f0; f < f0 + per && f < F; ++f) {
        const int c = pre[f + 1];
        base += c;
        pre[f + 1] = base;
    }
    __syncthreads();
    const int total = pre[F];
    const bool staged = total <= cap;
    // 2. stage the rows: thread per staged leaf, its records by independent 16-byte copies
    if (staged) {
        for (int f = threadIdx.x; f < F; f += P2P_THREADS) {
            const int b = pre[f], n = pre[f + 1] - b;
            const Particle<T> *src = sp + gst[f];
            for (int k = 0; k < n; ++k) stage_copy<T>(stg + b + k, src + k);
        }
        cp_async_wait_all();
    }
    __syncthreads();
    // 3. targets: the leaves x0 .. x0 + bx - 1 of the centre row
    const int rc = ws * side + ws;
    const int tb = pre[rc * W + ws], te = pre[rc * W + ws + bx];
    for (int st = tb + (int)threadIdx.x; st < te; st += P2P_THREADS) {
        int lo = rc * W + ws, hi = rc * W + ws + bx;  // the target's staged leaf
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= st) lo = mid;
            else hi = mid;
        }
        const int it = lo - rc * W;  // index of the target leaf within its row
        const int s = gst[lo] + (st - pre[lo]);  // sorted index of the target
        const Particle<T> pi = staged ? stg[st] : sp[s];
        // four independent partial sums (sources j, j + 1, j + 2, j + 3 of each leaf), so that the loads and
        // the dependent additions of consecutive pairs overlap; added in a fixed order at the end
        T a[4] = {0, 0, 0, 0}, fx[4] = {0, 0, 0, 0}, fy[4] = {0, 0, 0, 0}, fz[4] = {0, 0, 0, 0};
        for (int dz = -ws; dz <= ws; ++dz)
            for (int dy = -ws; dy <= ws; ++dy)
                for (int dx = -ws; dx <= ws; ++dx) {
                    const int f = ((dz + ws) * side + dy + ws) * W + it + dx;
                    const T ox = pi.x - T(dx) * h, oy = pi.y - T(dy) * h, oz = pi.z - T(dz) * h;
                    int jb, je;
                    const Particle<T> *src;
                    if (staged) {
                        jb = pre[f];
                        je = pre[f + 1];
                        src = stg;
                    } else {  // the leaf's records in the sorted array
                        jb = gst[f];
                        je = jb + (pre[f + 1] - pre[f]);
                        src = sp;
                    }
                    int j = jb;
                    for (; j + 4 <= je; j += 4) {
                        Particle<T> q4[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) q4[u] = src[j + u];
#pragma unroll
                        for (int u = 0; u < 4; ++u) p2p_pair<T>(q4[u], ox, oy, oz, a[u], fx[u], fy[u], fz[u]);
                    }
                    if (j < je) {
                        p2p_pair<T>(src[j], ox, oy, oz, a[0], fx[0], fy[0], fz[0]);
                        if (j + 1 < je) {
                            p2p_pair<T>(src[j + 1], ox, oy, oz, a[1], fx[1], fy[1], fz[1]);
                            if (j + 2 < je) p2p_pair<T>(src[j + 2], ox, oy, oz, a[2], fx[2], fy[2], fz[2]);
                        }
                    }
                }
        phi[s] = (a[0] + a[1]) + (a[2] + a[3]);
        if (field) {
            field[3 * s] = (fx[0] + fx[1]) + (fx[2] + fx[3]);
            field[3 * s + 1] = (fy[0] + fy[1]) + (fy[2] + fy[3]);
            field[3 * s + 2] = (fz[0] + fz[1]) + (fz[2] + fz[3]);
        }
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

namespace {

// staged-tile launch: rows of BX leaves, BX a power of two up to min(32, side) chosen so that a row holds
// about 128 target charges at the mean leaf occupancy (dense leaves: short rows, more blocks); the staging
// capacity is twice the expected particle count of a tile's rows (at least 512 records), within 96 KB of
// shared memory
template <typename T>
fmm_status launch_p2p_tile(Plan &P, T h, T *phi, T *field)
{
    static bool attr = false;
    const size_t smem_max = 96 * 1024;
    if (!attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(k_p2p_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
        attr = true;
    }
    const int n = 1 << P.d;
    const double occ = (double)P.N / (double)P.nleaf;
    int bx = 1;
    while (bx < 32 && bx < n && (double)(2 * bx) * occ <= 128.0) bx *= 2;
    const int side = 2 * P.ws + 1, F = side * side * (bx + 2 * P.ws);
    const size_t head = ((sizeof(int) * (2 * F + 1) + 15) / 16) * 16;
    const double expect = (double)P.N / (double)P.nleaf * F;
    size_t cap = (size_t)(2.0 * expect) + 512;
    const size_t cap_max = (smem_max - head) / sizeof(Particle<T>);
    if (cap > cap_max) cap = cap_max;
    const unsigned blocks = (unsigned)((int64_t)n * n * (n / bx));
    k_p2p_tile<T><<<blocks, P2P_THREADS, head + cap * sizeof(Particle<T>), P.stream>>>(
        P.d, P.ws, bx, (int)cap, h, P.cell_start, (const Particle<T> *)P.sorted, phi, field);
    return FMM_OK;
}

// The same sum together with the soft-core form of the solute-solvent near-field pairs, r -> reff =
// (alpha lambda A^c + r^c)^(1/c) (the paper's soft-core form, which it notes applies to the electrostatic
// NF term), in FP64 from the stored coordinates: sc[s] = q_i sum_j q_j / reff and
// sc[N + s] = -(alpha A^c / c) q_i sum_j q_j / (reff (alpha lambda A^c + r^c)) for solute slot s, 0 elsewhere.
// alpha_Ac = alpha A^c; lambda is read from device memory.
template <typename T>
__global__ void k_p2p_uv_sc(int64_t N, int d, int ws, T h, const int *__restrict__ start, const int *__restrict__ sleaf,
                            const Particle<T> *__restrict__ sp, const uint8_t *__restrict__ sol, T *__restrict__ out,
                            int c, double alpha_Ac, const double *__restrict__ lambda, double *__restrict__ sc)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (!sol[s]) {
        out[s] = 0;
        sc[s] = 0.0;
        sc[N + s] = 0.0;
        return;
    }
    const double b0 = alpha_Ac * *lambda;
    const double ic = 1.0 / (double)c;
    int nside = 1 << d;
    int leaf = sleaf[s];
    int x = leaf % nside, y = (leaf / nside) % nside, z = leaf / (nside * nside);
    Particle<T> pi = sp[s];
    T acc = 0;
    double e = 0.0, de = 0.0;
    for (int dz = -ws; dz <= ws; ++dz)
        for (int dy = -ws; dy <= ws; ++dy)
            for (int dx = -ws; dx <= ws; ++dx) {
                int xx = (x + dx + nside) & (nside - 1), yy = (y + dy + nside) & (nside - 1),
                    zz = (z + dz + nside) & (nside - 1);
                int cidx = xx + nside * (yy + nside * zz);
                T ox = pi.x - T(dx) * h, oy = pi.y - T(dy) * h, oz = pi.z - T(dz) * h;
                const double dox = (double)pi.x - (double)dx * (double)h, doy = (double)pi.y - (double)dy * (double)h,
                             doz = (double)pi.z - (double)dz * (double)h;
                for (int j = start[cidx]; j < start[cidx + 1]; ++j) {
                    if (sol[j]) continue;
                    Particle<T> pj = sp[j];
                    T rx = ox - pj.x, ry = oy - pj.y, rz = oz - pj.z;
                    acc += pj.q * inv_sqrt<T>(rx * rx + ry * ry + rz * rz);
                    const double ux = dox - (double)pj.x, uy = doy - (double)pj.y, uz = doz - (double)pj.z;
                    const double r = sqrt(ux * ux + uy * uy + uz * uz);
                    const double base = b0 + pow(r, (double)c);
                    const double reff = pow(base, ic);
                    e += (double)pj.q / reff;
                    de += (double)pj.q / (reff * base);
                }
            }
    out[s] = pi.q * acc;
    sc[s] = (double)pi.q * e;
    sc[N + s] = -(alpha_Ac * ic) * (double)pi.q * de;
}

}  // namespace

fmm_status launch_p2p(Plan &P, bool forces)
{
    int nside = 1 << P.d;
    double h = P.box / nside;
    fmm_status st;
    if (P.precision == FMM_PREC_FP64)
        st = launch_p2p_tile<double>(P, h, (double *)P.phi_nf, forces ? (double *)P.f_nf : nullptr);
    else
        st = launch_p2p_tile<float>(P, (float)h, (float *)P.phi_nf, forces ? (float *)P.f_nf : nullptr);
    if (st != FMM_OK) return st;
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_p2p_uv(Plan &P)
{
    int nside = 1 << P.d;
    double h = P.box / nside;
    if (P.sc_c > 0) {
        const double alpha_Ac = P.sc_alpha * pow(P.sc_A, (double)P.sc_c);
        if (P.precision == FMM_PREC_FP64)
            k_p2p_uv_sc<double><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(
                P.N, P.d, P.ws, h, P.cell_start, P.sleaf, (const Particle<double> *)P.sorted, P.sorted_sol,
                (double *)P.phi_nf + P.N, P.sc_c, alpha_Ac, P.sc_lambda, P.sc_out);
        else
            k_p2p_uv_sc<float><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(
                P.N, P.d, P.ws, (float)h, P.cell_start, P.sleaf, (const Particle<float> *)P.sorted, P.sorted_sol,
                (float *)P.phi_nf + P.N, P.sc_c, alpha_Ac, P.sc_lambda, P.sc_out);
        FMM_LAUNCH_CHECK(P);
        return FMM_OK;
    }
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
