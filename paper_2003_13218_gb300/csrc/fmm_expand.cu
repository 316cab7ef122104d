// fmm_expand.cu -- the expansion operators of Appendix B on the GPU:
// P2M (Eq. P2M), M2M, the level-0 lattice operator (Eq. 12), M2L over the
// interaction lists (Eq. Lcoeffdef, CUDA-core version), L2L and L2P with its
// gradient (Eq. EqFF); plus the per-plan operator tables.
//
// Solid harmonics (normalisation that makes the printed equations hold with
// no conjugates): R_n^m = r^n P_n^m e^{im phi}/(n+m)!,
// I_n^m = (-1)^(n+m) (n-m)! P_n^m e^{im phi} / r^(n+1); both obey
// C_n^{-m} = (-1)^m conj C_n^m, so only m >= 0 is stored.
#include <math.h>

#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ tables
// R_n^m at the eight child-centre offsets w_c = ((c_x - 1/2)/2, ...) (in
// units of the parent side): the M2M and L2L shift vectors.
__global__ void k_octant_table(int p, double *__restrict__ R64, float *__restrict__ R32)
{
    int c = threadIdx.x;
    if (c >= 8) return;
    int nc = ncoef(p);
    double w[3] = {((c & 1) - 0.5) * 0.5, (((c >> 1) & 1) - 0.5) * 0.5, (((c >> 2) & 1) - 0.5) * 0.5};
    double tmp[NC_MAX];
    regular_real<double>(p, w[0], w[1], w[2], tmp);
    for (int i = 0; i < nc; ++i) {
        R64[c * nc + i] = tmp[i];
        R32[c * nc + i] = (float)tmp[i];
    }
}

// complex I_j^k for any sign of k from the m >= 0 triangle
__device__ inline Cx<double> tri_get(const Cx<double> *t, int j, int k)
{
    int ak = k < 0 ? -k : k;
    Cx<double> v = t[tri(j, ak)];
    if (k < 0) {
        v.im = -v.im;
        if (ak & 1) {
            v.re = -v.re;
            v.im = -v.im;
        }
    }
    return v;
}

// Real form of Eq. Lcoeffdef: L_n^m = sum_{lambda, eta} M_lambda^eta O_{n+lambda}^{-(m+eta)}.
// With M_lambda^{-eta} = (-1)^eta conj M_lambda^eta and M_lambda^eta = x + i y:
//   eta = 0: L += x O(lambda, 0)
//   eta > 0: L += x A + i y B,  A = O(lambda, eta) + (-1)^eta O(lambda, -eta),
//                                B = O(lambda, eta) - (-1)^eta O(lambda, -eta),
// where O(lambda, e) = O_{n+lambda}^{-(m+e)}.  Entry [k][j] maps input real k
// to output real j.
__device__ void build_real_operator(int p, const Cx<double> *O, double *__restrict__ Tout)
{
    int nc = ncoef(p);
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
        int k = e / nc, j = e % nc;
        // output (n, m, part)
        int n = (int)sqrt((double)j);
        while (n * n > j) --n;
        while ((n + 1) * (n + 1) <= j) ++n;
        int r = j - n * n;
        int m = (r + 1) / 2;
        bool out_im = (m > 0) && (r == 2 * m);
        // input (lambda, eta, part)
        int lam = (int)sqrt((double)k);
        while (lam * lam > k) --lam;
        while ((lam + 1) * (lam + 1) <= k) ++lam;
        int ri = k - lam * lam;
        int eta = (ri + 1) / 2;
        bool in_im = (eta > 0) && (ri == 2 * eta);
        double val;
        Cx<double> o1 = tri_get(O, n + lam, -(m + eta));
        if (eta == 0) {
            val = out_im ? o1.im : o1.re;
        } else {
            Cx<double> o2 = tri_get(O, n + lam, eta - m);
            double sg = (eta & 1) ? -1.0 : 1.0;
            if (!in_im) {
                Cx<double> A = {o1.re + sg * o2.re, o1.im + sg * o2.im};
                val = out_im ? A.im : A.re;
            } else {
                Cx<double> B = {o1.re - sg * o2.re, o1.im - sg * o2.im};
                val = out_im ? B.re : -B.im;
            }
        }
        Tout[(size_t)k * nc + j] = val;
    }
}

// one block per offset slot delta in [-(2 ws + 1), 2 ws + 1]^3 (the (2 ws + 1)^3 near slots stay zero)
__global__ void k_m2l_operators(int p, int ws, double *__restrict__ T64, float *__restrict__ T32)
{
    extern __shared__ Cx<double> Ish[];
    int slot = blockIdx.x;
    const int side = off_side(ws), h = 2 * ws + 1;
    int dx = slot % side - h, dy = (slot / side) % side - h, dz = slot / (side * side) - h;
    int nc = ncoef(p);
    double *T = T64 + (size_t)slot * nc * nc;
    if (abs(dx) <= ws && abs(dy) <= ws && abs(dz) <= ws) {
        for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
            T[e] = 0.0;
            T32[(size_t)slot * nc * nc + e] = 0.0f;
        }
        return;
    }
    // I at r_L - r_M = -(delta) in cell units: target t, source t + delta
    if (threadIdx.x == 0) irregular_tri<double>(2 * p, -(double)dx, -(double)dy, -(double)dz, Ish);
    __syncthreads();
    build_real_operator(p, Ish, T);
    __syncthreads();
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) T32[(size_t)slot * nc * nc + e] = (float)T[e];
}

// single irregular harmonic I_j^k (k >= 0) by the column recurrence
__device__ Cx<double> irregular_one(int j, int k, double x, double y, double z)
{
    double r2 = x * x + y * y + z * z, ir2 = 1.0 / r2;
    Cx<double> dg = {1.0 / sqrt(r2), 0.0};
    for (int m = 1; m <= k; ++m) {
        double s = -(2.0 * m - 1.0) * ir2;
        dg = {s * (x * dg.re - y * dg.im), s * (x * dg.im + y * dg.re)};
    }
    Cx<double> p2 = {0, 0}, p1 = dg;
    for (int n = k + 1; n <= j; ++n) {
        double a = -(2.0 * n - 1.0) * z, b = (double)((n + k - 1) * (n - k - 1));
        Cx<double> c = {(a * p1.re - b * p2.re) * ir2, (a * p1.im - b * p2.im) * ir2};
        p2 = p1;
        p1 = c;
    }
    return p1;
}

struct KS {
    double s = 0, c = 0;
    __device__ void add(double x)
    {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ double val() const { return s + c; }
};

// Eq. 12 on a unit box with splitting parameter kb = kappa * b:
//   S_j^k = sum_{nu != 0} I_j^k(nu) Q(j + 1/2, kb^2 nu^2)                         (12a)
//         + pi^{3/2} i^j / (2^{j-2} Gamma(j + 1/2)) sum_{k != 0} I_j^k(k) k^{2j-1} e^{-k^2/4kb^2}  (12b)
//         - 2 kb / sqrt(pi) delta_{j0}                                           (12c)
//         - sum_{nu in {-1,0,1}^3, nu != 0} I_j^k(nu)      (images covered by levels 1..l_max)
// Q(a, x) = Gamma(a, x)/Gamma(a) by Q(1/2, x) = erfc(sqrt x) and
// Q(a + 1, x) = Q(a, x) + x^a e^{-x} / Gamma(a + 1).  One block per (j, k):
// threads stride over the lattice vectors, then a fixed-order reduction.
constexpr int LAT_THREADS = 256;

__device__ void block_merge(KS &v, double (*sh)[2])
{
    sh[threadIdx.x][0] = v.s;
    sh[threadIdx.x][1] = v.c;
    __syncthreads();
    for (int o = LAT_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            KS a;
            a.s = sh[threadIdx.x][0];
            a.c = sh[threadIdx.x][1];
            a.add(sh[threadIdx.x + o][0]);
            a.add(sh[threadIdx.x + o][1]);
            sh[threadIdx.x][0] = a.s;
            sh[threadIdx.x][1] = a.c;
        }
        __syncthreads();
    }
    v.s = sh[0][0];
    v.c = sh[0][1];
    __syncthreads();
}

__global__ void __launch_bounds__(LAT_THREADS) k_lattice_sum(int jmax, double kb, int ws, int nu_max, int nk_max,
                                                              double *__restrict__ S)
{
    __shared__ double sh[LAT_THREADS][2];
    int t = blockIdx.x;
    int j = 0;
    while (tri(j + 1, 0) <= t) ++j;
    int k = t - tri(j, 0);
    const double PI = 3.14159265358979323846;
    KS re, im;
    // real space (12a) and the near block
    const int side = 2 * nu_max + 1;
    const int nvec = side * side * side;
    for (int v = threadIdx.x; v < nvec; v += LAT_THREADS) {
        int nx = v % side - nu_max, ny = (v / side) % side - nu_max, nz = v / (side * side) - nu_max;
        if (nx == 0 && ny == 0 && nz == 0) continue;
        double r2 = (double)(nx * nx + ny * ny + nz * nz);
        double x = kb * kb * r2;
        double Q = erfc(sqrt(x));
        double g = sqrt(PI);  // Gamma(1/2)
        for (int i = 0; i < j; ++i) {
            double a = i + 0.5;
            g *= a;  // Gamma(i + 3/2)
            Q += exp(a * log(x) - x) / g;
        }
        bool near = abs(nx) <= ws && abs(ny) <= ws && abs(nz) <= ws;
        double w = near ? Q - 1.0 : Q;
        Cx<double> I = irregular_one(j, k, nx, ny, nz);
        re.add(w * I.re);
        im.add(w * I.im);
    }
    // reciprocal space (12b), k = 2 pi n
    double gh = sqrt(PI);
    for (int i = 0; i < j; ++i) gh *= (i + 0.5);  // Gamma(j + 1/2)
    double pref = pow(PI, 1.5) / (ldexp(1.0, j - 2) * gh);
    // i^j: j even -> (-1)^(j/2); odd degrees vanish by symmetry (kept exact)
    KS rre, rim;
    const int kside = 2 * nk_max + 1;
    const int nk = kside * kside * kside;
    for (int v = threadIdx.x; v < nk; v += LAT_THREADS) {
        int nx = v % kside - nk_max, ny = (v / kside) % kside - nk_max, nz = v / (kside * kside) - nk_max;
        if (nx == 0 && ny == 0 && nz == 0) continue;
        double kx = 2 * PI * nx, ky = 2 * PI * ny, kz = 2 * PI * nz;
        double k2 = kx * kx + ky * ky + kz * kz;
        double kk = sqrt(k2);
        double w = pow(kk, 2 * j - 1) * exp(-k2 / (4 * kb * kb));
        Cx<double> I = irregular_one(j, k, kx, ky, kz);
        rre.add(w * I.re);
        rim.add(w * I.im);
    }
    block_merge(re, sh);
    block_merge(im, sh);
    block_merge(rre, sh);
    block_merge(rim, sh);
    if (threadIdx.x != 0) return;
    double cr = rre.val() * pref, ci = rim.val() * pref;
    // multiply by i^j
    double ore, oim;
    switch (j & 3) {
    case 0: ore = cr; oim = ci; break;
    case 1: ore = -ci; oim = cr; break;
    case 2: ore = -cr; oim = -ci; break;
    default: ore = ci; oim = -cr; break;
    }
    re.add(ore);
    im.add(oim);
    if (j == 0) re.add(-2.0 * kb / sqrt(PI));
    S[2 * t] = re.val();
    S[2 * t + 1] = im.val();
}

__global__ void k_lattice_operator(int p, const double *__restrict__ S, double *__restrict__ T0)
{
    extern __shared__ Cx<double> Ssh[];
    int ntri = (2 * p + 1) * (2 * p + 2) / 2;
    for (int i = threadIdx.x; i < ntri; i += blockDim.x) Ssh[i] = {S[2 * i], S[2 * i + 1]};
    __syncthreads();
    build_real_operator(p, Ssh, T0);
}

// ------------------------------------------------------------------ P2M
// Eq. P2M in level-scaled form: Mhat_n^m = sum_j q_j R_n^m((r_M - r_j)/h).
// One thread per (leaf, m): the column n = m..p of every particle.  PM >= p is
// a compile-time bound so that the column accumulators stay in registers
// (the loops over n are unrolled and predicated on m <= n <= p).
template <typename T, int PM>
__global__ void k_p2m(int p, int nside, const int *__restrict__ start, const Particle<T> *__restrict__ sp,
                      T inv_h, int d, T *__restrict__ M)
{
    // reciprocals of the recurrences, once per block: -1/(2k) and 1/((n+m)(n-m))
    __shared__ T s_half[PM + 1];
    __shared__ T s_inv[(PM + 1) * (PM + 1)];
    for (int e = threadIdx.x; e < (PM + 1) * (PM + 1); e += blockDim.x) {
        const int n = e / (PM + 1), mm = e % (PM + 1);
        s_inv[e] = n > mm ? T(1) / T((n + mm) * (n - mm)) : T(0);
        if (e <= PM) s_half[e] = e > 0 ? T(-0.5) / T(e) : T(0);
    }
    __syncthreads();
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nleaf = (int64_t)nside * nside * nside;
    if (tid >= nleaf * (p + 1)) return;
    int64_t leaf = tid / (p + 1);
    int m = (int)(tid % (p + 1));
    int x = (int)(leaf % nside), y = (int)((leaf / nside) % nside), z = (int)(leaf / ((int64_t)nside * nside));
    T acc_re[PM + 1], acc_im[PM + 1];
#pragma unroll
    for (int n = 0; n <= PM; ++n) acc_re[n] = acc_im[n] = 0;
    for (int s = start[leaf]; s < start[leaf + 1]; ++s) {
        Particle<T> pt = sp[s];
        T vx = -pt.x * inv_h, vy = -pt.y * inv_h, vz = -pt.z * inv_h;
        T r2 = vx * vx + vy * vy + vz * vz;
        T dre = 1, dim = 0;
        for (int k = 1; k <= m; ++k) {
            T sc = s_half[k];
            T nre = sc * (vx * dre - vy * dim);
            T nim = sc * (vx * dim + vy * dre);
            dre = nre;
            dim = nim;
        }
        T p2re = 0, p2im = 0, p1re = dre, p1im = dim;
#pragma unroll
        for (int n = 0; n <= PM; ++n) {
            if (n == m) {
                acc_re[n] += pt.q * dre;
                acc_im[n] += pt.q * dim;
            } else if (n > m && n <= p) {
                T a = T(2 * n - 1) * vz;
                T inv = s_inv[n * (PM + 1) + m];
                T cr = (a * p1re - r2 * p2re) * inv;
                T ci = (a * p1im - r2 * p2im) * inv;
                acc_re[n] += pt.q * cr;
                acc_im[n] += pt.q * ci;
                p2re = p1re;
                p2im = p1im;
                p1re = cr;
                p1im = ci;
            }
        }
    }
    int nc = ncoef(p);
    T *out = M + cell_index(d, x, y, z) * nc;
#pragma unroll
    for (int n = 0; n <= PM; ++n) {
        if (n < m || n > p) continue;
        out[cre(n, m)] = acc_re[n];
        if (m > 0) out[cim(n, m)] = acc_im[n];
    }
}

// The same P2M at a compile-time order PP in FP32, one lane per leaf: a warp takes 32 leaves of one
// parity class with consecutive parent coordinates (32 consecutive rows of the level's class layout),
// each lane runs the recurrences of Eq. P2M for its leaf's charges with all (PP+1)^2 coefficients in
// registers (indices fold into immediates).  The rows go through shared memory (row stride (PP+1)^2, odd,
// so the 32 lanes hit 32 banks) and leave as 32 contiguous rows.  When `amax` is set (fp16x2 split) the
// warp also folds max_k |Mhat_k s(k)| into *amax (positive floats order as their bit patterns), which
// the tensor-core operand split needs for the level gain.
constexpr int P2M_WARPS = 4;

template <int PP>
__global__ void __launch_bounds__(32 * P2M_WARPS) k_p2m_fixed(int d, const int *__restrict__ start,
                                                              const Particle<float> *__restrict__ sp, float inv_h,
                                                              float *__restrict__ M, const float *__restrict__ s,
                                                              unsigned *__restrict__ amax)
{
    constexpr int NC = (PP + 1) * (PP + 1);
    extern __shared__ float p2m_tile[];  // [P2M_WARPS][32][NC]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *tile = p2m_tile + w * 32 * NC;
    const int np = 1 << (d - 1);
    const int64_t ncls = (int64_t)np * np * np;
    const int64_t row0 = ((int64_t)blockIdx.x * P2M_WARPS + w) * 32;
    if (row0 >= 8 * ncls) return;
    const int64_t row = row0 + lane;
    const bool valid = row < 8 * ncls;
    float acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = 0.f;
    if (valid) {
        const int c = (int)(row / ncls);
        const int64_t P = row - c * ncls;
        const int x = 2 * (int)(P % np) + (c & 1), y = 2 * (int)((P / np) % np) + ((c >> 1) & 1),
                  z = 2 * (int)(P / ((int64_t)np * np)) + ((c >> 2) & 1);
        const int nside = 2 * np;
        const int leaf = x + nside * (y + nside * z);
        const int b = start[leaf], e = start[leaf + 1];
        for (int j = b; j < e; ++j) {
            const Particle<float> pt = sp[j];
            const float vx = -pt.x * inv_h, vy = -pt.y * inv_h, vz = -pt.z * inv_h;
            const float r2 = vx * vx + vy * vy + vz * vz;
            float dre = pt.q, dim = 0.f;  // q R_m^m
#pragma unroll
            for (int m = 0; m <= PP; ++m) {
                if (m > 0) {
                    const float sc = -0.5f / (float)m;
                    const float nre = sc * (vx * dre - vy * dim);
                    const float nim = sc * (vx * dim + vy * dre);
                    dre = nre;
                    dim = nim;
                }
                acc[cre(m, m)] += dre;
                if (m > 0) acc[cim(m, m)] += dim;
                float p2re = 0.f, p2im = 0.f, p1re = dre, p1im = dim;
                // a trip count fixed at compile time (n = m + 1 + i, dead steps folded away) so that both
                // loops unroll completely and acc[] stays in registers
#pragma unroll
                for (int i = 0; i < PP; ++i) {
                    const int n = m + 1 + i;
                    if (n > PP) break;
                    const float a = (float)(2 * n - 1) * vz;
                    const float inv = 1.f / (float)((n + m) * (n - m));
                    const float cr = (a * p1re - r2 * p2re) * inv;
                    const float ci = (a * p1im - r2 * p2im) * inv;
                    acc[cre(n, m)] += cr;
                    if (m > 0) acc[cim(n, m)] += ci;
                    p2re = p1re;
                    p2im = p1im;
                    p1re = cr;
                    p1im = ci;
                }
            }
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        tile[lane * NC + k] = acc[k];
        if (amax) mx = fmaxf(mx, fabsf(acc[k] * __ldg(s + k)));
    }
    __syncwarp();
    const int64_t nrows = 8 * ncls - row0 < 32 ? 8 * ncls - row0 : 32;
    float *dst = M + row0 * NC;
    for (int64_t e = lane; e < nrows * NC; e += 32) dst[e] = tile[e];
    if (amax) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx > 0.f) atomicMax(amax, __float_as_uint(mx));
    }
}

template <int PP>
fmm_status launch_p2m_fixed(Plan &P, const Particle<float> *sp, float inv_h, unsigned *amax, const float *s)
{
    constexpr int NC = (PP + 1) * (PP + 1);
    const size_t sh = sizeof(float) * P2M_WARPS * 32 * NC;
    static bool attr = false;
    if (!attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(k_p2m_fixed<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        attr = true;
    }
    const int64_t rows = P.nleaf;
    const unsigned blocks = (unsigned)((rows + 32 * P2M_WARPS - 1) / (32 * P2M_WARPS));
    k_p2m_fixed<PP><<<blocks, 32 * P2M_WARPS, sh, P.stream>>>(P.d, P.cell_start, sp, inv_h, (float *)P.M[P.d], s, amax);
    return FMM_OK;
}

template <typename T>
void launch_p2m(Plan &P, const Particle<T> *sp, T inv_h)
{
    const int p = P.p, nside = 1 << P.d;
    const int64_t nthr = P.nleaf * (p + 1);
    const unsigned blocks = (unsigned)((nthr + 127) / 128);
    if (p <= 4) k_p2m<T, 4><<<blocks, 128, 0, P.stream>>>(p, nside, P.cell_start, sp, inv_h, P.d, (T *)P.M[P.d]);
    else if (p <= 8) k_p2m<T, 8><<<blocks, 128, 0, P.stream>>>(p, nside, P.cell_start, sp, inv_h, P.d, (T *)P.M[P.d]);
    else if (p <= 12) k_p2m<T, 12><<<blocks, 128, 0, P.stream>>>(p, nside, P.cell_start, sp, inv_h, P.d, (T *)P.M[P.d]);
    else if (p <= 16) k_p2m<T, 16><<<blocks, 128, 0, P.stream>>>(p, nside, P.cell_start, sp, inv_h, P.d, (T *)P.M[P.d]);
    else k_p2m<T, P_MAX><<<blocks, 128, 0, P.stream>>>(p, nside, P.cell_start, sp, inv_h, P.d, (T *)P.M[P.d]);
}

// ------------------------------------------------------------------ lattice apply
// Lbar(0) = T0 . Mhat(0) (Eq. 12 in place of I in Eq. Lcoeffdef), in FP64
template <typename T>
__global__ void k_lattice_apply(int p, const double *__restrict__ T0, const T *__restrict__ M0, T *__restrict__ L0)
{
    int nc = ncoef(p);
    int j = threadIdx.x;
    if (j >= nc) return;
    double acc = 0;
    for (int k = 0; k < nc; ++k) acc += T0[(size_t)k * nc + j] * (double)M0[k];
    L0[j] = (T)acc;
}

// ------------------------------------------------------------------ M2L (CUDA cores)
// Eq. Lcoeffdef over the 189-cell interaction list of each target, as dense
// real operators per offset.  Block: TT targets of one parity class, one
// thread per output coefficient.  Sources are read with periodic wrap.
template <typename T, int TT>
__global__ void k_m2l_simt(int p, int l, int cls, int ws, const T *__restrict__ Top, const T *__restrict__ M,
                           T *__restrict__ L)
{
    extern __shared__ unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);  // [TT][nc]
    int nc = ncoef(p);
    int np = 1 << (l - 1);
    int64_t ncls = (int64_t)np * np * np;
    int64_t t0 = (int64_t)blockIdx.x * TT;
    int cx = cls & 1, cy = (cls >> 1) & 1, cz = (cls >> 2) & 1;
    int j = threadIdx.x;
    T acc[TT];
#pragma unroll
    for (int t = 0; t < TT; ++t) acc[t] = 0;
    // delta per axis in [-2 ws - c, 2 ws + 1 - c]: the children of the parent's
    // (2 ws + 1)^3 neighbours that are not the target's own neighbours
    for (int dz = -2 * ws - cz; dz <= 2 * ws + 1 - cz; ++dz)
        for (int dy = -2 * ws - cy; dy <= 2 * ws + 1 - cy; ++dy)
            for (int dx = -2 * ws - cx; dx <= 2 * ws + 1 - cx; ++dx) {
                if (abs(dx) <= ws && abs(dy) <= ws && abs(dz) <= ws) continue;
                int sx = cx + dx, sy = cy + dy, sz = cz + dz;  // in [-2 ws, 2 ws + 1]
                int scls = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
                int Dx = sx >> 1, Dy = sy >> 1, Dz = sz >> 1;  // floor division
                __syncthreads();
                for (int e = threadIdx.x; e < TT * nc; e += blockDim.x) {
                    int t = e / nc, k = e % nc;
                    int64_t tg = t0 + t;
                    T v = 0;
                    if (tg < ncls) {
                        int Px = (int)(tg % np), Py = (int)((tg / np) % np), Pz = (int)(tg / ((int64_t)np * np));
                        int Qx = ((Px + Dx) % np + np) % np, Qy = ((Py + Dy) % np + np) % np,
                            Qz = ((Pz + Dz) % np + np) % np;
                        int64_t src = scls * ncls + Qx + (int64_t)np * (Qy + (int64_t)np * Qz);
                        v = M[src * nc + k];
                    }
                    S[t * nc + k] = v;
                }
                __syncthreads();
                if (j < nc) {
                    const T *Tp = Top + (size_t)off_slot(dx, dy, dz, ws) * nc * nc + j;
                    for (int k = 0; k < nc; ++k) {
                        T w = Tp[(size_t)k * nc];
#pragma unroll
                        for (int t = 0; t < TT; ++t) acc[t] += w * S[t * nc + k];
                    }
                }
            }
    if (j < nc) {
        for (int t = 0; t < TT; ++t) {
            int64_t tg = t0 + t;
            if (tg < ncls) L[(cls * ncls + tg) * nc + j] = acc[t];
        }
    }
}

// ------------------------------------------------------------------ L2P
// Phi(r) = (1/h) sum L_n^m R_n^m(v), v = (r - r_L')/h, and
// grad Phi = (1/h^2) sum_{n',m'} G_{n'}^{m'} R_{n'}^{m'}(v) with
//   G^z = L_{n'+1}^{m'},  G^x = (L_{n'+1}^{m'-1} - L_{n'+1}^{m'+1})/2,
//   G^y = -i (L_{n'+1}^{m'-1} + L_{n'+1}^{m'+1})/2.
template <typename T>
__global__ void k_l2p(int p, int d, int64_t N, const int *__restrict__ sleaf, const Particle<T> *__restrict__ sp,
                      T inv_h, const T *__restrict__ L, T *__restrict__ phi, T *__restrict__ grad)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int nside = 1 << d;
    int leaf = sleaf[s];
    int x = leaf % nside, y = (leaf / nside) % nside, z = leaf / (nside * nside);
    const T *Lc = L + cell_index(d, x, y, z) * ncoef(p);
    Particle<T> pt = sp[s];
    T vx = pt.x * inv_h, vy = pt.y * inv_h, vz = pt.z * inv_h;
    T r2 = vx * vx + vy * vy + vz * vz;
    T pot = 0, gx = 0, gy = 0, gz = 0;
    T dre = 1, dim = 0;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            T sc = T(-0.5) / T(m);
            T nre = sc * (vx * dre - vy * dim);
            T nim = sc * (vx * dim + vy * dre);
            dre = nre;
            dim = nim;
        }
        T w = m == 0 ? T(1) : T(2);
        T p2re = 0, p2im = 0, rre = dre, rim = dim;
        for (int n = m; n <= p; ++n) {
            if (n > m) {
                T a = T(2 * n - 1) * vz;
                T inv = T(1) / T((n + m) * (n - m));
                T cr = (a * rre - r2 * p2re) * inv;
                T ci = (a * rim - r2 * p2im) * inv;
                p2re = rre;
                p2im = rim;
                rre = cr;
                rim = ci;
            }
            Cx<T> Lnm = coef(Lc, n, m);
            pot += w * (Lnm.re * rre - Lnm.im * rim);
            if (grad && n < p) {
                Cx<T> a = coef(Lc, n + 1, m - 1), b = coef(Lc, n + 1, m + 1), c = coef(Lc, n + 1, m);
                Cx<T> Gx = {T(0.5) * (a.re - b.re), T(0.5) * (a.im - b.im)};
                Cx<T> Gy = {T(0.5) * (a.im + b.im), -T(0.5) * (a.re + b.re)};
                gx += w * (Gx.re * rre - Gx.im * rim);
                gy += w * (Gy.re * rre - Gy.im * rim);
                gz += w * (c.re * rre - c.im * rim);
            }
        }
    }
    phi[s] = pot * inv_h;
    if (grad) {
        T s2 = inv_h * inv_h;
        grad[3 * s] = gx * s2;
        grad[3 * s + 1] = gy * s2;
        grad[3 * s + 2] = gz * s2;
    }
}

// The same L2P at a compile-time order PP: the loops unroll, the recurrences' reciprocals fold into
// constants and the coefficient indices into immediates.  The expansions of the block's leaves
// (consecutive in the sorted order) are staged in shared memory when at most L2P_LEAVES of them span
// the block: a warp's particles sit in several leaves, and each of its coefficient loads would touch
// as many L1 lines.
constexpr int L2P_LEAVES = 48;
constexpr int L2P_THREADS = 128;

template <typename T, int PP>
__global__ void __launch_bounds__(L2P_THREADS) k_l2p_fixed(int d, int64_t N, const int *__restrict__ sleaf,
                                                           const Particle<T> *__restrict__ sp, T inv_h,
                                                           const T *__restrict__ L, T *__restrict__ phi,
                                                           T *__restrict__ grad)
{
    constexpr int NC = (PP + 1) * (PP + 1);
    extern __shared__ __align__(16) unsigned char l2p_smem[];
    T *sL = reinterpret_cast<T *>(l2p_smem);
    const int64_t s0 = (int64_t)blockIdx.x * L2P_THREADS;
    const int64_t slast = (s0 + L2P_THREADS < N ? s0 + L2P_THREADS : N) - 1;
    const int nside = 1 << d, mask = nside - 1;
    const int leaf0 = sleaf[s0];
    const int nl = sleaf[slast] - leaf0 + 1;
    const bool staged = nl <= L2P_LEAVES;
    if (staged) {
        for (int e = threadIdx.x; e < nl * NC; e += L2P_THREADS) {
            const int li = e / NC, c = e - li * NC;
            const int leaf = leaf0 + li;
            sL[e] = L[cell_index(d, leaf & mask, (leaf >> d) & mask, leaf >> (2 * d)) * NC + c];
        }
    }
    __syncthreads();
    const int64_t s = s0 + threadIdx.x;
    if (s >= N) return;
    const int leaf = sleaf[s];
    const T *Lc = staged ? sL + (leaf - leaf0) * NC : L + cell_index(d, leaf & mask, (leaf >> d) & mask, leaf >> (2 * d)) * NC;
    const Particle<T> pt = sp[s];
    const T vx = pt.x * inv_h, vy = pt.y * inv_h, vz = pt.z * inv_h;
    const T r2 = vx * vx + vy * vy + vz * vz;
    T pot = 0, gx = 0, gy = 0, gz = 0;
    T dre = 1, dim = 0;
#pragma unroll
    for (int m = 0; m <= PP; ++m) {
        if (m > 0) {
            const T sc = T(-0.5) / T(m);
            const T nre = sc * (vx * dre - vy * dim);
            const T nim = sc * (vx * dim + vy * dre);
            dre = nre;
            dim = nim;
        }
        const T w = m == 0 ? T(1) : T(2);
        T p2re = 0, p2im = 0, rre = dre, rim = dim;
#pragma unroll
        for (int n = m; n <= PP; ++n) {
            if (n > m) {
                const T a = T(2 * n - 1) * vz;
                const T inv = T(1) / T((n + m) * (n - m));
                const T cr = (a * rre - r2 * p2re) * inv;
                const T ci = (a * rim - r2 * p2im) * inv;
                p2re = rre;
                p2im = rim;
                rre = cr;
                rim = ci;
            }
            const Cx<T> Lnm = coef(Lc, n, m);
            pot += w * (Lnm.re * rre - Lnm.im * rim);
            if (grad && n < PP) {
                const Cx<T> a = coef(Lc, n + 1, m - 1), b = coef(Lc, n + 1, m + 1), c = coef(Lc, n + 1, m);
                const Cx<T> Gx = {T(0.5) * (a.re - b.re), T(0.5) * (a.im - b.im)};
                const Cx<T> Gy = {T(0.5) * (a.im + b.im), -T(0.5) * (a.re + b.re)};
                gx += w * (Gx.re * rre - Gx.im * rim);
                gy += w * (Gy.re * rre - Gy.im * rim);
                gz += w * (c.re * rre - c.im * rim);
            }
        }
    }
    phi[s] = pot * inv_h;
    if (grad) {
        const T s2 = inv_h * inv_h;
        grad[3 * s] = gx * s2;
        grad[3 * s + 1] = gy * s2;
        grad[3 * s + 2] = gz * s2;
    }
}

template <typename T, int PP>
fmm_status launch_l2p_fixed(Plan &P, T inv_h, const T *L, T *phi, T *grad)
{
    const size_t sh = sizeof(T) * L2P_LEAVES * (PP + 1) * (PP + 1);
    static bool attr = false;
    if (!attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(k_l2p_fixed<T, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        attr = true;
    }
    k_l2p_fixed<T, PP><<<blocks_for(P.N, L2P_THREADS), L2P_THREADS, sh, P.stream>>>(
        P.d, P.N, P.sleaf, (const Particle<T> *)(P.sorted), inv_h, L, phi, grad);
    return FMM_OK;
}

// L2P of the plan at its order: the fixed-order kernel for the usual orders, else the generic one
template <typename T>
fmm_status l2p_t(Plan &P, T inv_h, const T *L, T *phi, T *grad)
{
    switch (P.p) {
    case 4: return launch_l2p_fixed<T, 4>(P, inv_h, L, phi, grad);
    case 6: return launch_l2p_fixed<T, 6>(P, inv_h, L, phi, grad);
    case 8: return launch_l2p_fixed<T, 8>(P, inv_h, L, phi, grad);
    case 10: return launch_l2p_fixed<T, 10>(P, inv_h, L, phi, grad);
    case 12: return launch_l2p_fixed<T, 12>(P, inv_h, L, phi, grad);
    default:
        k_l2p<T><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(P.p, P.d, P.N, P.sleaf, (const Particle<T> *)P.sorted,
                                                             inv_h, L, phi, grad);
        return FMM_OK;
    }
}

template <typename T>
fmm_status upward_t(Plan &P, bool solute_only)
{
    const int nside = 1 << P.d;
    const Particle<T> *sp = (const Particle<T> *)(solute_only ? P.sorted_u : P.sorted);
    T inv_h = (T)((double)nside / P.box);
    const bool tc = tc_translations(P);
    // fp16 split: the P2M at a compile-time order folds the level maximum of |Mhat s| in as it writes.  It
    // runs one lane per leaf, so it is used for deep trees of sparse leaves (the benchmark boxes: 262,144
    // leaves of ~4 charges); shallow trees of dense leaves keep the thread-per-(leaf, order) kernel
    bool amax_ready = false;
    const bool lane_per_leaf = P.nleaf >= 32768 && (double)P.N <= 12.0 * (double)P.nleaf;
    if (std::is_same<T, float>::value && lane_per_leaf &&
        (P.p == 4 || P.p == 6 || P.p == 8 || P.p == 10 || P.p == 12)) {
        unsigned *amax = nullptr;
        if (tc) {
            fmm_status st = tc_clear_amax(P, P.d);
            if (st != FMM_OK) return st;
            amax = tc_amax(P, P.d);
        }
        const Particle<float> *spf = (const Particle<float> *)sp;
        const float ih = (float)inv_h;
        const float *sc = tc ? tc_scale(P) : nullptr;
        fmm_status st = P.p == 4    ? launch_p2m_fixed<4>(P, spf, ih, amax, sc)
                        : P.p == 6  ? launch_p2m_fixed<6>(P, spf, ih, amax, sc)
                        : P.p == 8  ? launch_p2m_fixed<8>(P, spf, ih, amax, sc)
                        : P.p == 10 ? launch_p2m_fixed<10>(P, spf, ih, amax, sc)
                                    : launch_p2m_fixed<12>(P, spf, ih, amax, sc);
        if (st != FMM_OK) return st;
        amax_ready = tc;
    } else {
        launch_p2m<T>(P, sp, inv_h);
    }
    FMM_LAUNCH_CHECK(P);
    for (int l = P.d - 1; l >= 0; --l) {
        // the tensor-core M2M into level l folds level l's maximum in (amax of level l + 1 is ready from
        // the P2M or the previous M2M)
        fmm_status st = tc ? tc_split_moments(P, l + 1, amax_ready) : FMM_OK;
        if (st == FMM_OK) st = tc ? launch_m2m_tc(P, l) : launch_m2m(P, l);
        if (st != FMM_OK) return st;
        amax_ready = tc;
    }
    return FMM_OK;
}

}  // namespace

// ------------------------------------------------------------------ host side
fmm_status build_tables(Plan &P)
{
    free_tables(P);
    int p = P.p, nc = P.nc;
    FMM_CUDA_TRY(cudaMalloc(&P.tab.Rw64, sizeof(double) * 8 * nc));
    FMM_CUDA_TRY(cudaMalloc(&P.tab.Rw32, sizeof(float) * 8 * nc));
    int ntri2 = (2 * p + 1) * (2 * p + 2) / 2;
    FMM_CUDA_TRY(cudaMalloc(&P.tab.S, sizeof(double) * 2 * ntri2));
    FMM_CUDA_TRY(cudaMalloc(&P.tab.T0, sizeof(double) * nc * nc));
    FMM_CUDA_TRY(cudaMalloc(&P.tab.Top64, sizeof(double) * (size_t)noff(P.ws) * nc * nc));
    FMM_CUDA_TRY(cudaMalloc(&P.tab.Top32, sizeof(float) * (size_t)noff(P.ws) * nc * nc));
    k_octant_table<<<1, 32, 0, P.stream>>>(p, P.tab.Rw64, P.tab.Rw32);
    FMM_LAUNCH_CHECK(P);
    {
        fmm_status st = build_translation_ops(P);
        if (st != FMM_OK) return st;
    }
    size_t shI = sizeof(Cx<double>) * ntri2;
    k_m2l_operators<<<noff(P.ws), 256, shI, P.stream>>>(p, P.ws, P.tab.Top64, P.tab.Top32);
    FMM_LAUNCH_CHECK(P);
    double kappa = P.kappa > 0 ? P.kappa : 2.0 / P.box;
    double kb = kappa * P.box;
    int nu_max = (int)ceil(8.0 / kb) + 3 + P.ws;
    int nk_max = (int)ceil(2.2 * kb) + 3;
    k_lattice_sum<<<ntri2, LAT_THREADS, 0, P.stream>>>(2 * p, kb, P.ws, nu_max, nk_max, P.tab.S);
    FMM_LAUNCH_CHECK(P);
    k_lattice_operator<<<1, 256, shI, P.stream>>>(p, P.tab.S, P.tab.T0);
    FMM_LAUNCH_CHECK(P);
    FMM_CUDA_TRY(cudaStreamSynchronize(P.stream));
    return FMM_OK;
}

fmm_status build_lattice(Plan &P)
{
    if (!P.tab.S || !P.tab.T0) return build_tables(P);
    int p = P.p;
    int ntri2 = (2 * p + 1) * (2 * p + 2) / 2;
    double kappa = P.kappa > 0 ? P.kappa : 2.0 / P.box;
    double kb = kappa * P.box;
    int nu_max = (int)ceil(8.0 / kb) + 3 + P.ws;
    int nk_max = (int)ceil(2.2 * kb) + 3;
    k_lattice_sum<<<ntri2, LAT_THREADS, 0, P.stream>>>(2 * p, kb, P.ws, nu_max, nk_max, P.tab.S);
    FMM_LAUNCH_CHECK(P);
    k_lattice_operator<<<1, 256, sizeof(Cx<double>) * ntri2, P.stream>>>(p, P.tab.S, P.tab.T0);
    FMM_LAUNCH_CHECK(P);
    FMM_CUDA_TRY(cudaStreamSynchronize(P.stream));
    return FMM_OK;
}

void free_tables(Plan &P)
{
    cudaFree(P.tab.Rw64);
    cudaFree(P.tab.Rw32);
    cudaFree(P.tab.S);
    cudaFree(P.tab.T0);
    cudaFree(P.tab.Top64);
    cudaFree(P.tab.Top32);
    cudaFree(P.tab.l2l64);
    cudaFree(P.tab.l2l32);
    cudaFree(P.tab.m2m64);
    cudaFree(P.tab.m2m32);
    cudaFree(P.tab.m2mP32);
    cudaFree(P.tab.l2lP32);
    P.tab = Tables{};
}

fmm_status launch_upward(Plan &P, bool solute_only)
{
    return P.precision == FMM_PREC_FP64 ? upward_t<double>(P, solute_only) : upward_t<float>(P, solute_only);
}

fmm_status launch_lattice(Plan &P)
{
    if (P.precision == FMM_PREC_FP64)
        k_lattice_apply<double><<<1, ((P.nc + 31) / 32) * 32, 0, P.stream>>>(P.p, P.tab.T0, (const double *)P.M[0],
                                                                            (double *)P.L[0]);
    else
        k_lattice_apply<float><<<1, ((P.nc + 31) / 32) * 32, 0, P.stream>>>(P.p, P.tab.T0, (const float *)P.M[0],
                                                                           (float *)P.L[0]);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

fmm_status launch_m2l_simt(Plan &P, int l)
{
    int nc = P.nc;
    int threads = ((nc + 31) / 32) * 32;
    int64_t np = (int64_t)1 << (l - 1);
    int64_t ncls = np * np * np;
    static bool attr_set = false;
    if (!attr_set) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_simt<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(double) * 16 * NC_MAX)));
        FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_simt<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(float) * 32 * NC_MAX)));
        attr_set = true;
    }
    for (int cls = 0; cls < 8; ++cls) {
        if (P.precision == FMM_PREC_FP64) {
            constexpr int TT = 16;
            size_t sh = sizeof(double) * TT * nc;
            k_m2l_simt<double, TT><<<blocks_for(ncls, TT), threads, sh, P.stream>>>(
                P.p, l, cls, P.ws, P.tab.Top64, (const double *)P.M[l], (double *)P.L[l]);
        } else {
            constexpr int TT = 32;
            size_t sh = sizeof(float) * TT * nc;
            k_m2l_simt<float, TT><<<blocks_for(ncls, TT), threads, sh, P.stream>>>(
                P.p, l, cls, P.ws, P.tab.Top32, (const float *)P.M[l], (float *)P.L[l]);
        }
        FMM_LAUNCH_CHECK(P);
    }
    return FMM_OK;
}

fmm_status launch_l2p(Plan &P, bool gradient, bool solute_only)
{
    int nside = 1 << P.d;
    double inv_h = (double)nside / P.box;
    fmm_status st;
    if (P.precision == FMM_PREC_FP64)
        st = l2p_t<double>(P, inv_h, (const double *)P.L[P.d], (double *)(solute_only ? P.phi_u : P.phi_ff),
                           gradient ? (double *)P.g_ff : nullptr);
    else
        st = l2p_t<float>(P, (float)inv_h, (const float *)P.L[P.d], (float *)(solute_only ? P.phi_u : P.phi_ff),
                          gradient ? (float *)P.g_ff : nullptr);
    if (st != FMM_OK) return st;
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

}  // namespace fmm
